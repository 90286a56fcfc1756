"""Python binding of libpocketvina.so: the same calls as include/pocketvina.h, with PyTorch
supplying device memory (its caching allocator), streams and automatic differentiation.

Every computation runs in the library's CUDA kernels; this module only marshals arguments.
There is no CPU fallback: a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from . import _capi as A

N_XS = 11


class PVError(RuntimeError):
    pass


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a) -> int:
    """Data pointer of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


@dataclasses.dataclass
class DockParams:
    chains: int = 64
    steps: int = 1000
    seed: int = 0
    top_k: int = 9
    rmsd_min: float = 1.0
    mode: str = "batched"          # or "plain" (thread per chain), "plain_warp" (warp per chain), per pair
    bfgs_m: int = 5
    bfgs_max_iter: int = 0
    bfgs_max_trials: int = 10
    bfgs_eps: float = 1e-3
    rho: float = 1e-4
    sigma: float = 0.1
    temperature: float = 1.2
    amplitude: float = 2.0
    steps_per_round: int = 0
    use_graph: bool = True
    warps_per_cta: int = 0
    search_variant: int = -1
    host_copy: bool = True
    timeout_s: float = 0.0
    focc: int = 0                  # first-order consistency check (Eq. 4-5): neighbours kept, 0 = off
    focc_min_delta: float = 1e-4
    rescore: bool = False          # rescore kept poses by direct receptor summation (no grid)
    max_pockets: int = 0           # > 0: each ligand docked into its first max_pockets pockets only
    block_wait_s: float = 30.0     # bound on a step block's wait for its predecessor
    pair_keys: Optional[Sequence[int]] = None   # per pair: its random stream (default: pair index)
    map_layout: int = -1           # 0 plain, 1 cell-packed, -1 autotuned when the set holds both
    resume_state: Optional[bytes] = None   # a checkpoint (DockResult.save_state) of the same job:
                                           # continue its chains from the step it had reached

    def to_c(self) -> A.pv_dock_params:
        p = A.pv_dock_params()
        A.load().pv_dock_params_default(C.byref(p))
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if f.name == "mode":
                v = {"batched": A.PV_MODE_BATCHED, "plain": A.PV_MODE_PLAIN, "plain_warp": A.PV_MODE_PLAIN_WARP}[v]
            elif f.name == "pair_keys":
                if v is None:
                    continue
                v = (C.c_int32 * len(v))(*[int(k) for k in v])   # kept alive by the struct
            elif f.name == "resume_state":
                if v is None:
                    continue
                buf = C.create_string_buffer(bytes(v), len(v))
                p._resume_buf = buf                                  # kept alive with the struct
                p.resume_state = C.addressof(buf)
                p.resume_bytes = len(v)
                continue
            elif isinstance(v, bool):
                v = int(v)
            setattr(p, f.name, v)
        return p


@dataclasses.dataclass
class PocketParams:
    """Parameters of the pocket-side steps (Supplementary Algorithm 1)."""
    probe: float = 1.6             # solvent probe radius added to the atom radii, A
    n_sphere: int = 100            # lattice points per atom sphere
    r_feature: float = 6.0         # Eq. 1 neighbourhood radius, A
    r_protrusion: float = 10.0     # protrusion count radius, A
    threshold: float = 0.5         # points with score >= threshold are clustered
    link: float = 3.0              # single-linkage distance, A

    def to_c(self) -> A.pv_pocket_params:
        p = A.pv_pocket_params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


class Context:
    """A library context on one CUDA device, issuing work on a torch stream and allocating
    device memory through torch's caching allocator."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise PVError("no CUDA device: the docking path runs only on the GPU")
        self.torch = torch
        self.lib = A.load()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.pv_context_create(self.device, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != A.PV_OK:
            raise PVError(f"pv_context_create failed: {A.STATUS_NAMES.get(st, st)}")
        self.h = h
        self._keep = []
        if torch_allocator:
            dev = self.device

            def _alloc(n, stream, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, stream)
                except Exception:   # noqa: BLE001 - out of memory is reported as NULL
                    return None

            def _free(p, _stream, _user):
                torch.cuda.caching_allocator_delete(p)

            fa, ff = A.ALLOC_FN(_alloc), A.FREE_FN(_free)
            self._keep += [fa, ff]
            self._check(self.lib.pv_context_set_allocator(self.h, fa, ff, None), "pv_context_set_allocator")

    # ---------------------------------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != A.PV_OK:
            msg = self.lib.pv_last_error(self.h)
            raise PVError(f"{what}: {A.STATUS_NAMES.get(st, st)}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.pv_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001
            pass

    # ------------------------------------------------------------------------ grid cache --
    def _receptor(self, rec, keep: list) -> A.pv_receptor:
        torch = self.torch
        r = A.pv_receptor()
        if isinstance(rec.xyz, torch.Tensor):
            xyz = rec.xyz.to(torch.float32).contiguous()
            arrs = [xyz] + [t.to(torch.uint8).contiguous() for t in (rec.element, rec.donor, rec.acceptor)]
            r.mem = A.PV_MEM_DEVICE if xyz.is_cuda else A.PV_MEM_HOST
        else:
            arrs = [_np(rec.xyz, np.float32), _np(rec.element, np.uint8), _np(rec.donor, np.uint8),
                    _np(rec.acceptor, np.uint8)]
            r.mem = A.PV_MEM_HOST
        keep += arrs
        r.n_atoms = int(arrs[0].shape[0])
        r.xyz, r.element, r.donor, r.acceptor = (_ptr(a) for a in arrs)
        return r

    @staticmethod
    def _boxes(boxes) -> "C.Array":
        arr = (A.pv_box * len(boxes))()
        for i, b in enumerate(boxes):
            c = b.center if hasattr(b, "center") else b[0]
            s = b.size if hasattr(b, "size") else b[1]
            sp = b.spacing if hasattr(b, "spacing") else (b[2] if len(b) > 2 else 0.375)
            for k in range(3):
                arr[i].center[k] = float(c[k])
                arr[i].size[k] = float(s[k] if np.ndim(s) else s)
            arr[i].spacing = float(sp)
        return arr

    def build_grids(self, receptor, boxes: Sequence, lig_types: Sequence[int] = tuple(range(N_XS))) -> "GridSet":
        keep: list = []
        r = self._receptor(receptor, keep)
        bx = self._boxes(boxes)
        types = (C.c_uint8 * len(lig_types))(*[int(t) for t in lig_types])
        h = C.c_void_p()
        self._check(self.lib.pv_build_grids(self.h, C.byref(r), bx, len(boxes), types, len(lig_types), C.byref(h)),
                    "pv_build_grids")
        return GridSet(self, h)

    # ---------------------------------------------------------------------- pocket side --
    def surface(self, receptor, radius=None, params: Optional[PocketParams] = None) -> "Surface":
        """Step 1 of Supplementary Algorithm 1: the receptor's SAS points (pv_surface_create).
        radius: per-atom vdW radii in the receptor's memory kind, or None for the Bondi radii."""
        torch = self.torch
        keep: list = []
        r = self._receptor(receptor, keep)
        rad = None
        if radius is not None:
            if isinstance(radius, torch.Tensor):
                rad = radius.to(torch.float32).contiguous()
                if rad.is_cuda != (r.mem == A.PV_MEM_DEVICE):
                    raise PVError("radius must live where the receptor does")
            else:
                if r.mem != A.PV_MEM_HOST:
                    raise PVError("radius must live where the receptor does")
                rad = _np(radius, np.float32)
            keep.append(rad)
        p = (params or PocketParams()).to_c()
        h = C.c_void_p()
        self._check(self.lib.pv_surface_create(self.h, C.byref(r), None if rad is None else _ptr(rad), C.byref(p),
                                               C.byref(h)), "pv_surface_create")
        return Surface(self, h)

    def surfaces(self, receptors: Sequence, radii: Optional[Sequence] = None,
                 params: Optional[PocketParams] = None) -> List["Surface"]:
        """Step 1 for several receptors in one call (pv_surface_create_many): the same surfaces as
        one `surface` call each, with one host synchronisation for all of them."""
        torch = self.torch
        k = len(receptors)
        if k == 0:
            return []
        keep: list = []
        recs = (A.pv_receptor * k)()
        rad_ptrs = (C.c_void_p * k)()
        for j, rec in enumerate(receptors):
            recs[j] = self._receptor(rec, keep)
            rad = None if radii is None else radii[j]
            if rad is not None:
                if isinstance(rad, torch.Tensor):
                    rad = rad.to(torch.float32).contiguous()
                    if rad.is_cuda != (recs[j].mem == A.PV_MEM_DEVICE):
                        raise PVError("radius must live where the receptor does")
                else:
                    if recs[j].mem != A.PV_MEM_HOST:
                        raise PVError("radius must live where the receptor does")
                    rad = _np(rad, np.float32)
                keep.append(rad)
                rad_ptrs[j] = _ptr(rad)
        p = (params or PocketParams()).to_c()
        hs = (C.c_void_p * k)()
        self._check(self.lib.pv_surface_create_many(self.h, k, recs, None if radii is None else rad_ptrs, C.byref(p), hs),
                    "pv_surface_create_many")
        return [Surface(self, C.c_void_p(h)) for h in hs]

    def cluster_many(self, sets: Sequence, params: Optional[PocketParams] = None) -> List["Clusters"]:
        """Steps 4-5 for several point sets in one call (pv_cluster_points_many). sets: (points,
        scores) pairs, points a [n, 3] array or tensor, or a Surface (its own points, used in place)."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        k = len(sets)
        if k == 0:
            return []
        keep: list = []
        ns, xs, ss = (C.c_int32 * k)(), (C.c_void_p * k)(), (C.c_void_p * k)()
        for j, (pts, sc) in enumerate(sets):
            if isinstance(pts, Surface):
                ptr = C.c_void_p()
                self._check(self.lib.pv_surface_points(pts.h, C.byref(ptr)), "pv_surface_points")
                n, xp = pts.n_points, ptr.value
                keep.append(pts)
            else:
                t = torch.as_tensor(pts, dtype=torch.float32).to(dev).contiguous().reshape(-1, 3)
                keep.append(t)
                n, xp = int(t.shape[0]), t.data_ptr()
            st = torch.as_tensor(sc, dtype=torch.float32).to(dev).contiguous().reshape(-1)
            if st.shape[0] != n:
                raise PVError("one score per point required")
            keep.append(st)
            ns[j], xs[j], ss[j] = n, xp, st.data_ptr()
        p = (params or PocketParams()).to_c()
        hs = (C.c_void_p * k)()
        self._check(self.lib.pv_cluster_points_many(self.h, k, ns, xs, ss, C.byref(p), hs), "pv_cluster_points_many")
        return [Clusters(self, C.c_void_p(h)) for h in hs]

    def cluster(self, points, scores, params: Optional[PocketParams] = None) -> "Clusters":
        """Steps 4-5: threshold, single-linkage clusters, Eq. 2 scores, centres and ranking of the
        points (pv_cluster_points). points [n, 3] and scores [n] are moved to the device."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        pts = torch.as_tensor(points, dtype=torch.float32).to(dev).contiguous().reshape(-1, 3)
        sc = torch.as_tensor(scores, dtype=torch.float32).to(dev).contiguous().reshape(-1)
        if sc.shape[0] != pts.shape[0]:
            raise PVError("one score per point required")
        p = (params or PocketParams()).to_c()
        h = C.c_void_p()
        self._check(self.lib.pv_cluster_points(self.h, int(pts.shape[0]), pts.data_ptr(), sc.data_ptr(), C.byref(p),
                                               C.byref(h)), "pv_cluster_points")
        return Clusters(self, h)

    # --------------------------------------------------------------------------- ligands --
    def ligand(self, lig) -> "Ligand":
        arrs = [_np(lig.xyz, np.float32), _np(lig.element, np.uint8), _np(lig.donor, np.uint8),
                _np(lig.acceptor, np.uint8), _np(lig.bonds, np.int32).reshape(-1, 2),
                _np(lig.rotatable, np.uint8)]
        d = A.pv_ligand_desc()
        d.n_atoms = int(arrs[0].shape[0])
        d.xyz, d.element, d.donor, d.acceptor = (_ptr(a) for a in arrs[:4])
        d.n_bonds = int(arrs[4].shape[0])
        d.bonds, d.rotatable = _ptr(arrs[4]), _ptr(arrs[5])
        h = C.c_void_p()
        self._check(self.lib.pv_ligand_create(self.h, C.byref(d), C.byref(h)), "pv_ligand_create")
        return Ligand(self, h)

    # --------------------------------------------------------------------------- scoring --
    def score(self, grids: "GridSet", lig: "Ligand", pocket: int, poses, grad: bool = True, parts: bool = False):
        """SF (Eq. 3) of poses [n, 7 + n_rot] (cuda float32). Returns (energy [n], tangent
        gradient [n, 6 + n_rot] or None, (e_inter, e_intra) [n, 2] or None)."""
        torch = self.torch
        poses = poses.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        n = poses.shape[0]
        e = torch.empty(n, device=poses.device, dtype=torch.float32)
        g = torch.empty((n, 6 + lig.n_rot), device=poses.device, dtype=torch.float32) if grad else None
        pr = torch.empty((n, 2), device=poses.device, dtype=torch.float32) if parts else None
        self._check(self.lib.pv_score(self.h, grids.h, lig.h, int(pocket), n, poses.data_ptr(), e.data_ptr(),
                                      g.data_ptr() if g is not None else None,
                                      pr.data_ptr() if pr is not None else None), "pv_score")
        return e, g, pr

    def score_backward(self, grids: "GridSet", lig: "Ligand", pocket: int, poses, grad_energy,
                       want_pose: bool = True, want_xyz: bool = False):
        torch = self.torch
        poses = poses.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        ge = grad_energy.to(device=poses.device, dtype=torch.float32).contiguous()
        n = poses.shape[0]
        gp = torch.empty_like(poses) if want_pose else None
        gx = torch.empty((n, lig.n_atoms, 3), device=poses.device, dtype=torch.float32) if want_xyz else None
        self._check(self.lib.pv_score_backward(self.h, grids.h, lig.h, int(pocket), n, poses.data_ptr(), ge.data_ptr(),
                                               gp.data_ptr() if gp is not None else None,
                                               gx.data_ptr() if gx is not None else None), "pv_score_backward")
        return gp, gx

    def score_xyz(self, grids: "GridSet", lig: "Ligand", pocket: int, xyz, grad: bool = True, grad_energy=None):
        """SF (Eq. 3) of posed atom coordinates xyz [n, n_atoms, 3] (input order, cuda float32).
        Returns (energy [n] or None when grad_energy is given, dSF/dxyz [n, n_atoms, 3] scaled by
        grad_energy [n] if given, or None)."""
        torch = self.torch
        xyz = xyz.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        n = xyz.shape[0]
        ge = grad_energy.to(device=xyz.device, dtype=torch.float32).contiguous() if grad_energy is not None else None
        e = torch.empty(n, device=xyz.device, dtype=torch.float32) if ge is None else None
        g = torch.empty_like(xyz) if grad or ge is not None else None
        self._check(self.lib.pv_score_xyz(self.h, grids.h, lig.h, int(pocket), n, xyz.data_ptr(),
                                          ge.data_ptr() if ge is not None else None,
                                          e.data_ptr() if e is not None else None,
                                          g.data_ptr() if g is not None else None), "pv_score_xyz")
        return e, g

    def pose_coords(self, lig: "Ligand", poses):
        torch = self.torch
        poses = poses.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        out = torch.empty((poses.shape[0], lig.n_atoms, 3), device=poses.device, dtype=torch.float32)
        self._check(self.lib.pv_pose_coords(self.h, lig.h, poses.shape[0], poses.data_ptr(), out.data_ptr()),
                    "pv_pose_coords")
        return out

    def measure_gather(self, grids: "GridSet", pocket: int = 0, n_points: int = 1 << 24, reps: int = 10,
                       layout: int = 0):
        """The trilinear gather alone (value + gradient at hashed positions in the pocket's box;
        pocket -1: over every pocket of the set) in a map layout (0 plain, 1 cell-packed): returns
        (milliseconds per launch, points per second, algorithmic GB/s at 32 B per point)."""
        ms = C.c_float()
        self._check(self.lib.pv_measure_gather_layout(self.h, grids.h, int(pocket), int(n_points), int(reps),
                                                      int(layout), C.byref(ms)), "pv_measure_gather_layout")
        t = ms.value * 1e-3
        return ms.value, n_points / t, 32.0 * n_points / t / 1e9

    # --------------------------------------------------------------------------- docking --
    def dock(self, grids: "GridSet", ligands: Sequence["Ligand"], pocket_ids: Sequence[int],
             params: Optional[DockParams] = None, **kw) -> "DockResult":
        p = dataclasses.replace(params or DockParams(), **kw)
        hs = (C.c_void_p * len(ligands))(*[l.h.value for l in ligands])
        pk = (C.c_int32 * len(pocket_ids))(*[int(x) for x in pocket_ids])
        cp = p.to_c()
        h = C.c_void_p()
        st = self.lib.pv_dock(self.h, grids.h, hs, len(ligands), pk, len(pocket_ids), C.byref(cp), C.byref(h))
        return self._result(st, h, len(ligands), "pv_dock")

    def dock_top_pockets(self, grids: "GridSet", ligands: Sequence["Ligand"], ranked_pocket_ids: Sequence[int],
                         max_pockets: int = 5, params: Optional[DockParams] = None, **kw) -> "DockResult":
        """Docks into the best-ranked pockets only (pocket ids ordered by the pocket predictor's
        score, best first): the first max_pockets of them, as the paper suggests five suffice
        (the library's max_pockets cut)."""
        if max_pockets < 1:
            raise PVError("max_pockets must be >= 1")
        return self.dock(grids, ligands, list(ranked_pocket_ids), params, max_pockets=max_pockets, **kw)

    def dock_pairs(self, grids: "GridSet", ligands: Sequence["Ligand"], pair_ligand: Sequence[int],
                   pair_pocket: Sequence[int], params: Optional[DockParams] = None, **kw) -> "DockResult":
        p = dataclasses.replace(params or DockParams(), **kw)
        hs = (C.c_void_p * len(ligands))(*[l.h.value for l in ligands])
        pl = (C.c_int32 * len(pair_ligand))(*[int(x) for x in pair_ligand])
        pp = (C.c_int32 * len(pair_pocket))(*[int(x) for x in pair_pocket])
        cp = p.to_c()
        h = C.c_void_p()
        st = self.lib.pv_dock_pairs(self.h, grids.h, hs, len(ligands), pl, pp, len(pl), C.byref(cp), C.byref(h))
        return self._result(st, h, len(ligands), "pv_dock_pairs")

    def _result(self, st, h, n_ligs, what):
        # a dock that ran and reports a watchdog timeout, a non-finite energy or a step block that
        # gave up waiting still returns its result handle
        if st not in (A.PV_OK, A.PV_ERR_TIMEOUT, A.PV_ERR_NAN, A.PV_ERR_STATE) or not h.value:
            self._check(st, what)
        res = DockResult(self, h, n_ligs)
        res.status_code = st
        if st != A.PV_OK:
            res.error = self.lib.pv_last_error(self.h).decode()
        return res


class GridSet:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    @property
    def n_pockets(self) -> int:
        n = C.c_int32()
        b = C.c_int64()
        self.ctx.lib.pv_grid_set_info(self.h, C.byref(n), C.byref(b))
        return n.value

    @property
    def bytes(self) -> int:
        n = C.c_int32()
        b = C.c_int64()
        self.ctx.lib.pv_grid_set_info(self.h, C.byref(n), C.byref(b))
        return b.value

    def append(self, receptor, boxes) -> int:
        keep: list = []
        r = self.ctx._receptor(receptor, keep)
        bx = Context._boxes(boxes)
        first = C.c_int32()
        self.ctx._check(self.ctx.lib.pv_grid_set_append(self.ctx.h, self.h, C.byref(r), bx, len(boxes),
                                                        C.byref(first)), "pv_grid_set_append")
        return first.value

    def geometry(self, pocket: int, xs_type: int):
        p = C.c_void_p()
        dims = (C.c_int32 * 3)()
        org = (C.c_float * 3)()
        sp = C.c_float()
        st = self.ctx.lib.pv_grid_set_view(self.h, int(pocket), int(xs_type), C.byref(p), dims, org, C.byref(sp))
        if st != A.PV_OK:
            raise PVError("pv_grid_set_view: no such map")
        return np.array(list(dims)), np.array(list(org), dtype=np.float64), sp.value, p.value

    def pack(self) -> "GridSet":
        """Adds the cell-packed copy of every map (pv_grid_set_pack)."""
        self.ctx._check(self.ctx.lib.pv_grid_set_pack(self.ctx.h, self.h), "pv_grid_set_pack")
        return self

    def build_seconds(self) -> float:
        """Device time of the map-build kernel launches that built this set."""
        t = C.c_double()
        self.ctx._check(self.ctx.lib.pv_grid_set_build_seconds(self.h, C.byref(t)), "pv_grid_set_build_seconds")
        return t.value

    def read_map(self, pocket: int, xs_type: int) -> np.ndarray:
        dims, _, _, _ = self.geometry(pocket, xs_type)
        out = np.zeros((dims[2], dims[1], dims[0]), dtype=np.float32)
        self.ctx._check(self.ctx.lib.pv_grid_set_read_map(self.h, int(pocket), int(xs_type), out.ctypes.data),
                        "pv_grid_set_read_map")
        return out

    def __del__(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.pv_grid_set_destroy(self.h)
            self.h = None


class Ligand:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        na, nr, npair, org = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        ctx.lib.pv_ligand_info(h, C.byref(na), C.byref(nr), C.byref(npair), C.byref(org))
        self.n_atoms, self.n_rot, self.n_pairs, self.origin = na.value, nr.value, npair.value, org.value

    def cost(self):
        """(FP32 operations, gathered grid bytes) of one score + gradient evaluation."""
        f, b = C.c_double(), C.c_double()
        self.ctx._check(self.ctx.lib.pv_ligand_cost(self.h, C.byref(f), C.byref(b)), "pv_ligand_cost")
        return f.value, b.value

    @property
    def xs_types(self) -> np.ndarray:
        out = np.zeros(self.n_atoms, dtype=np.uint8)
        self.ctx.lib.pv_ligand_xs_types(self.h, out.ctypes.data_as(C.POINTER(C.c_uint8)))
        return out

    def __del__(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.pv_ligand_destroy(self.h)
            self.h = None


class DockResult:
    def __init__(self, ctx: Context, h, n_ligs: int):
        self.ctx, self.h, self.n_ligs = ctx, h, n_ligs
        a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        ctx.lib.pv_dock_result_info(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d))
        self.n_pairs, self.top_k, self.pot_stride, self.atom_stride = a.value, b.value, c.value, d.value
        self.status_code = 0
        self.error = ""
        self._host = None

    def fetch(self):
        """Host copies: structured pose records, kept counts, POTs, coordinates."""
        if self._host is None:
            n = self.n_pairs * self.top_k
            poses = (A.pv_pose * n)()
            kept = np.zeros(self.n_pairs, dtype=np.int32)
            pots = np.zeros((self.n_pairs, self.top_k, self.pot_stride), dtype=np.float32)
            xyz = np.zeros((self.n_pairs, self.top_k, self.atom_stride, 3), dtype=np.float32)
            self.ctx._check(self.ctx.lib.pv_dock_result_poses(
                self.h, poses, kept.ctypes.data_as(C.POINTER(C.c_int32)),
                pots.ctypes.data_as(C.POINTER(C.c_float)), xyz.ctypes.data_as(C.POINTER(C.c_float))),
                "pv_dock_result_poses")
            rec = np.array([(p.score, p.e_inter, p.e_intra, p.affinity, p.pair, p.ligand, p.pocket, p.chain,
                             p.score_grid, p.e_inter_grid) for p in poses],
                           dtype=[("score", "f4"), ("e_inter", "f4"), ("e_intra", "f4"), ("affinity", "f4"),
                                  ("pair", "i4"), ("ligand", "i4"), ("pocket", "i4"), ("chain", "i4"),
                                  ("score_grid", "f4"), ("e_inter_grid", "f4")])
            self._host = (rec.reshape(self.n_pairs, self.top_k), kept, pots, xyz)
        return self._host

    @property
    def poses(self):
        return self.fetch()[0]

    @property
    def n_kept(self):
        return self.fetch()[1]

    @property
    def pots(self):
        return self.fetch()[2]

    @property
    def xyz(self):
        return self.fetch()[3]

    def ranking(self, ligand: int) -> np.ndarray:
        cap = self.n_pairs * self.top_k
        out = np.zeros(max(cap, 1), dtype=np.int32)
        n = C.c_int32()
        self.ctx._check(self.ctx.lib.pv_dock_result_ranking(self.h, int(ligand),
                                                            out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)),
                        "pv_dock_result_ranking")
        return out[:n.value]

    def stats(self):
        ev = C.c_uint64()
        sec = C.c_double()
        st = np.zeros(self.n_pairs, dtype=np.int32)
        self.ctx._check(self.ctx.lib.pv_dock_result_stats(self.h, C.byref(ev), C.byref(sec),
                                                          st.ctypes.data_as(C.POINTER(C.c_int32))),
                        "pv_dock_result_stats")
        return ev.value, sec.value, st

    def timing(self):
        """(search kernel seconds, search launches, whole launch sequence seconds)."""
        s, n, t = C.c_double(), C.c_int32(), C.c_double()
        self.ctx._check(self.ctx.lib.pv_dock_result_timing(self.h, C.byref(s), C.byref(n), C.byref(t)),
                        "pv_dock_result_timing")
        return s.value, n.value, t.value

    def map_layout(self) -> int:
        """Map layout the search read: 0 plain, 1 cell-packed."""
        v = C.c_int32()
        self.ctx._check(self.ctx.lib.pv_dock_result_map_layout(self.h, C.byref(v)), "pv_dock_result_map_layout")
        return v.value

    def launch_shape(self):
        """(search kernel variant, warps per CTA) used by the batched search."""
        v, w = C.c_int32(), C.c_int32()
        self.ctx._check(self.ctx.lib.pv_dock_result_launch(self.h, C.byref(v), C.byref(w)), "pv_dock_result_launch")
        return v.value, w.value

    def chain_records(self):
        """Chain states after the search, copied to the host: (best POT [n_pairs, chains,
        pot_stride], best SF [n_pairs, chains])."""
        p = C.c_void_p()
        ch, stride, bo, so = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self.ctx._check(self.ctx.lib.pv_dock_result_chains(self.h, C.byref(p), C.byref(ch), C.byref(stride),
                                                           C.byref(bo), C.byref(so)), "pv_dock_result_chains")
        rec = np.zeros((self.n_pairs, ch.value, stride.value), dtype=np.float32)
        self.ctx._check(self.ctx.lib.pv_dock_result_read_chains(self.h, rec.ctypes.data), "pv_dock_result_read_chains")
        return rec[:, :, bo.value:bo.value + self.pot_stride].copy(), rec[:, :, so.value].copy()

    def save_state(self) -> bytes:
        """Checkpoint of the dock (every chain's state after its last MC step): pass it as
        DockParams.resume_state to a dock of the same job with more steps to continue from there."""
        n = C.c_int64()
        self.ctx._check(self.ctx.lib.pv_dock_result_state_bytes(self.h, C.byref(n)), "pv_dock_result_state_bytes")
        buf = C.create_string_buffer(n.value)
        self.ctx._check(self.ctx.lib.pv_dock_result_save_state(self.h, buf, n.value), "pv_dock_result_save_state")
        return buf.raw

    def __del__(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.pv_dock_result_destroy(self.h)
            self.h = None


class PVScore:
    """torch.autograd.Function over pose parameters: energy = SF(pose) for one ligand in one
    pocket; backward is the library's adjoint kernel (the gradient BFGS consumes), mapped to POT
    coordinates (translation, raw quaternion, torsions)."""

    _fn = None

    @classmethod
    def apply(cls, pose, ctx: Context, grids: GridSet, lig: Ligand, pocket: int):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, pose_t, pv_ctx, grids_, lig_, pocket_):
                    e, _, _ = pv_ctx.score(grids_, lig_, pocket_, pose_t.detach(), grad=False)
                    fctx.save_for_backward(pose_t)
                    fctx.pv = (pv_ctx, grids_, lig_, pocket_)
                    return e

                @staticmethod
                def backward(fctx, ge):
                    (pose_t,) = fctx.saved_tensors
                    pv_ctx, grids_, lig_, pocket_ = fctx.pv
                    gp, _ = pv_ctx.score_backward(grids_, lig_, pocket_, pose_t.detach(), ge.contiguous())
                    return gp.to(pose_t.dtype), None, None, None, None

            cls._fn = _F
        return cls._fn.apply(pose, ctx, grids, lig, pocket)


class PVScoreXYZ:
    """torch.autograd.Function over ligand atom coordinates: energy = SF(xyz) for posed atoms
    [n, n_atoms, 3] of one ligand in one pocket; backward is the library's coordinate gradient
    (dSF/dx_i scaled by the incoming gradient in the kernel)."""

    _fn = None

    @classmethod
    def apply(cls, xyz, ctx: Context, grids: GridSet, lig: Ligand, pocket: int):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, xyz_t, pv_ctx, grids_, lig_, pocket_):
                    e, _ = pv_ctx.score_xyz(grids_, lig_, pocket_, xyz_t.detach(), grad=False)
                    fctx.save_for_backward(xyz_t)
                    fctx.pv = (pv_ctx, grids_, lig_, pocket_)
                    return e

                @staticmethod
                def backward(fctx, ge):
                    (xyz_t,) = fctx.saved_tensors
                    pv_ctx, grids_, lig_, pocket_ = fctx.pv
                    _, gx = pv_ctx.score_xyz(grids_, lig_, pocket_, xyz_t.detach(), grad_energy=ge.contiguous())
                    return gx.to(xyz_t.dtype), None, None, None, None

            cls._fn = _F
        return cls._fn.apply(xyz, ctx, grids, lig, pocket)


class Surface:
    """Solvent-accessible surface points of a receptor (pv_surface_*)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        na, npt = C.c_int32(), C.c_int32()
        ctx.lib.pv_surface_info(h, C.byref(na), C.byref(npt))
        self.n_atoms, self.n_points = na.value, npt.value

    def points(self):
        """float32 [n_points, 3] device tensor (a copy), ordered by atom, then lattice point."""
        torch = self.ctx.torch
        out = torch.empty((self.n_points, 3), dtype=torch.float32, device=torch.device("cuda", self.ctx.device))
        self.ctx._check(self.ctx.lib.pv_surface_read(self.ctx.h, self.h, out.data_ptr(), None, A.PV_MEM_DEVICE),
                        "pv_surface_read")
        return out

    def sources(self) -> np.ndarray:
        """int32 [n_points]: atom * n_sphere + lattice index of every point."""
        out = np.zeros(max(self.n_points, 1), dtype=np.int32)
        self.ctx._check(self.ctx.lib.pv_surface_read(self.ctx.h, self.h, None, out.ctypes.data, A.PV_MEM_HOST),
                        "pv_surface_read")
        return out[:self.n_points]

    def features(self, props, points=None, params: Optional[PocketParams] = None):
        """Step 2 (Eq. 1 and protrusion) at the surface's points, or at given points [n, 3].
        props: [n_atoms, n_props] in receptor atom order. Returns device tensors
        (features float32 [n, n_props], protrusion int32 [n])."""
        torch = self.ctx.torch
        dev = torch.device("cuda", self.ctx.device)
        pr = torch.as_tensor(props, dtype=torch.float32).to(dev).contiguous()
        if pr.ndim != 2 or pr.shape[0] != self.n_atoms:
            raise PVError("props must be [n_atoms, n_props]")
        if points is None:
            n, xp = self.n_points, None
        else:
            pts = torch.as_tensor(points, dtype=torch.float32).to(dev).contiguous().reshape(-1, 3)
            n, xp = int(pts.shape[0]), pts
        feat = torch.empty((n, pr.shape[1]), dtype=torch.float32, device=dev)
        prot = torch.empty(n, dtype=torch.int32, device=dev)
        if n == 0 and xp is not None and pr.shape[1] > 0:
            return feat, prot          # an empty tensor's pointer is NULL, which means "the surface's points"
        p = (params or PocketParams()).to_c()
        self.ctx._check(self.ctx.lib.pv_surface_features(
            self.ctx.h, self.h, n, None if xp is None else xp.data_ptr(), A.PV_MEM_DEVICE, int(pr.shape[1]),
            pr.data_ptr(), A.PV_MEM_DEVICE, C.byref(p), feat.data_ptr(), prot.data_ptr()), "pv_surface_features")
        return feat, prot

    def __del__(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.pv_surface_destroy(self.h)
            self.h = None


class Clusters:
    """Ranked single-linkage clusters of high-scoring points (pv_clusters_*)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        n, k = C.c_int32(), C.c_int32()
        ctx.lib.pv_clusters_info(h, C.byref(n), C.byref(k))
        self.n_points, self.n_clusters = n.value, k.value

    def read(self) -> dict:
        """Host arrays: cluster [n_points] (rank of the point's cluster, -1 below the threshold),
        and per cluster in rank order score [K] (Eq. 2), center [K, 3], size [K], first [K]."""
        n, k = self.n_points, self.n_clusters
        out = {"cluster": np.zeros(max(n, 1), np.int32), "score": np.zeros(max(k, 1), np.float32),
               "center": np.zeros((max(k, 1), 3), np.float32), "size": np.zeros(max(k, 1), np.int32),
               "first": np.zeros(max(k, 1), np.int32)}
        self.ctx._check(self.ctx.lib.pv_clusters_read(self.ctx.h, self.h, *(out[x].ctypes.data for x in
                                                                              ("cluster", "score", "center", "size", "first")),
                                                      A.PV_MEM_HOST), "pv_clusters_read")
        out["cluster"] = out["cluster"][:n]
        for x in ("score", "center", "size", "first"):
            out[x] = out[x][:k]
        return out

    def boxes(self, size: float = 20.0, spacing: float = 0.375, max_pockets: int = 0) -> list:
        """Search boxes centred on the ranked cluster centres (Algorithm 3), best first."""
        c = self.read()["center"]
        if max_pockets > 0:
            c = c[:max_pockets]
        return [(tuple(float(v) for v in x), (size, size, size), spacing) for x in c]

    def __del__(self):
        if getattr(self, "h", None) and self.ctx.h:
            self.ctx.lib.pv_clusters_destroy(self.h)
            self.h = None
