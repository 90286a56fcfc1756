"""FP64 CPU oracle for the PocketVina docking hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. It shares no code with the CUDA path: the arithmetic lives in
``pv_oracle.c`` (docking) and ``pv_oracle_pocket.c`` (pocket side: surface points, Eq. 1 sums,
clusters), plain C in FP64 compiled with gcc here, and this module only marshals numpy arrays
through ctypes and does the final cross-pocket merge with a plain sort.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pv_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "pv_oracle_pocket.c"))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpv_oracle.so")
_lock = threading.Lock()
_lib = None

N_XS = 11
XS_NAMES = ("C_H", "C_P", "N_P", "N_D", "N_A", "N_DA", "O_P", "O_D", "O_A", "O_DA", "S_P")


def build(force: bool = False) -> str:
    """Compile ``pv_oracle.c`` and ``pv_oracle_pocket.c`` into ``oracle/_build/libpv_oracle.so``
    (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-Wall", "-Wno-unused-function", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("spacing", C.c_double), ("dims", C.c_int32 * 3),
                ("map_of_type", C.c_int32 * N_XS), ("maps", C.POINTER(C.c_double))]


class BfgsParams(C.Structure):
    _fields_ = [("m", C.c_int), ("max_iter", C.c_int), ("max_trials", C.c_int),
                ("rho", C.c_double), ("sigma", C.c_double), ("eps", C.c_double)]


class McParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("steps", C.c_int), ("temperature", C.c_double),
                ("amplitude", C.c_double), ("bfgs", BfgsParams), ("focc", C.c_int),
                ("focc_min_delta", C.c_double)]


EVAL_FN = C.CFUNCTYPE(C.c_double, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))
RETRACT_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                         C.POINTER(C.c_double))


class Problem(C.Structure):
    _fields_ = [("n_tan", C.c_int), ("n_state", C.c_int), ("eval", EVAL_FN),
                ("retract", RETRACT_FN), ("ctx", C.c_void_p)]


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, dp, ip, u8p, u32p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), \
                C.POINTER(C.c_uint8), C.POINTER(C.c_uint32)
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_u01.restype = C.c_double
            L.or_u01.argtypes = [C.c_uint32]
            L.or_xs_type_ligand.argtypes = [C.c_int, u8p, u8p, u8p, C.c_int, ip, ip]
            L.or_xs_type_receptor.argtypes = [C.c_int, dp, u8p, u8p, u8p, ip]
            L.or_terms.argtypes = [C.c_double, dp]
            L.or_pair_energy.restype = C.c_double
            L.or_pair_energy.argtypes = [C.c_int, C.c_int, C.c_double, dp]
            L.or_grid_dims.restype = C.c_int
            L.or_grid_dims.argtypes = [C.c_double, C.c_double]
            L.or_grid_node_value.restype = C.c_double
            L.or_grid_node_value.argtypes = [C.c_int, dp, ip, dp, C.c_double, C.c_int, C.c_int,
                                             C.c_int, C.c_int]
            L.or_grid_build.argtypes = [C.c_int, dp, ip, dp, C.c_double, ip, C.c_int, ip, dp, C.c_int]
            L.or_grid_fill_nodes.argtypes = [C.c_int, dp, ip, dp, C.c_double, ip, C.c_int, ip, C.c_long,
                                             C.POINTER(C.c_int64), dp, C.c_int]
            L.or_grid_eval.restype = C.c_double
            L.or_grid_eval.argtypes = [C.POINTER(Grid), C.c_int, dp, dp]
            L.or_ligand_new.restype = vp
            L.or_ligand_new.argtypes = [C.c_int, dp, u8p, u8p, u8p, C.c_int, ip, u8p]
            L.or_ligand_free.argtypes = [vp]
            L.or_ligand_info.argtypes = [vp, ip, dp]
            L.or_ligand_arrays.argtypes = [vp, ip, ip, ip, ip, ip]
            L.or_fk.argtypes = [vp, dp, dp]
            L.or_score.restype = C.c_double
            L.or_score.argtypes = [vp, C.POINTER(Grid), dp, dp, dp]
            L.or_score_atoms.restype = C.c_double
            L.or_score_atoms.argtypes = [vp, C.POINTER(Grid), dp, dp]
            L.or_retract.argtypes = [C.c_int, dp, dp, dp]
            L.or_bfgs.restype = C.c_double
            L.or_bfgs.argtypes = [C.POINTER(Problem), C.POINTER(BfgsParams), dp, dp,
                                  C.POINTER(C.c_long)]
            L.or_bfgs_pose.restype = C.c_double
            L.or_bfgs_pose.argtypes = [vp, C.POINTER(Grid), C.POINTER(BfgsParams), dp, dp,
                                       C.POINTER(C.c_long)]
            L.or_random_conformation.argtypes = [vp, dp, dp, C.c_uint64, C.c_uint32, C.c_uint32, dp]
            L.or_mutate.argtypes = [vp, dp, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, dp]
            L.or_metropolis_uniform.restype = C.c_double
            L.or_metropolis_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int]
            L.or_metropolis_accept.restype = C.c_int
            L.or_metropolis_accept.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.or_mc_chain.argtypes = [vp, C.POINTER(Grid), dp, dp, C.POINTER(McParams), C.c_uint32,
                                      C.c_uint32, dp, dp, C.POINTER(C.c_long)]
            L.or_mc_chains.argtypes = [vp, C.POINTER(Grid), dp, dp, C.POINTER(McParams), C.c_uint32,
                                       C.c_int, dp, dp, C.POINTER(C.c_long), C.c_int]
            L.or_tangent_delta.argtypes = [C.c_int, dp, dp, dp]
            L.or_focc_pass.restype = C.c_int
            L.or_focc_pass.argtypes = [vp, dp, C.c_double, dp, C.c_int, dp, dp, dp, C.c_double]
            L.or_direct_inter.restype = C.c_double
            L.or_direct_inter.argtypes = [vp, C.c_int, dp, ip, dp]
            L.or_topk.restype = C.c_int
            L.or_topk.argtypes = [C.c_int, dp, dp, C.c_int, C.c_int, C.c_double, ip]
            L.or_affinity.restype = C.c_double
            L.or_affinity.argtypes = [C.c_double, C.c_int]
            L.or_sphere_lattice.argtypes = [C.c_int, dp]
            L.or_sas_points.argtypes = [C.c_int, dp, dp, C.c_double, C.c_int, C.c_int, ip, u8p, dp, dp]
            L.or_point_features.argtypes = [C.c_int, dp, C.c_int, dp, C.c_int, dp, C.c_double,
                                            C.c_double, dp, ip]
            L.or_cluster_points.restype = C.c_int
            L.or_cluster_points.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, ip, ip, dp, dp,
                                            ip, ip]
            _lib = L
    return _lib


# ------------------------------------------------------------------------------ primitives --

def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def u01(word: int) -> float:
    return lib().or_u01(int(word))


def terms(d: float) -> np.ndarray:
    o = np.zeros(5)
    lib().or_terms(float(d), _p(o))
    return o


def pair_energy(ti: int, tj: int, r: float):
    de = C.c_double()
    e = lib().or_pair_energy(int(ti), int(tj), float(r), C.byref(de))
    return e, de.value


def xs_type_ligand(lig) -> np.ndarray:
    out = np.zeros(lig.n, dtype=np.int32)
    b = np.ascontiguousarray(lig.bonds, dtype=np.int32)
    lib().or_xs_type_ligand(lig.n, _p(np.ascontiguousarray(lig.element, np.uint8), C.c_uint8),
                            _p(np.ascontiguousarray(lig.donor, np.uint8), C.c_uint8),
                            _p(np.ascontiguousarray(lig.acceptor, np.uint8), C.c_uint8),
                            b.shape[0], _p(b, C.c_int32), _p(out, C.c_int32))
    return out


def xs_type_receptor(rec) -> np.ndarray:
    out = np.zeros(rec.n, dtype=np.int32)
    lib().or_xs_type_receptor(rec.n, _p(np.ascontiguousarray(rec.xyz, np.float64)),
                              _p(np.ascontiguousarray(rec.element, np.uint8), C.c_uint8),
                              _p(np.ascontiguousarray(rec.donor, np.uint8), C.c_uint8),
                              _p(np.ascontiguousarray(rec.acceptor, np.uint8), C.c_uint8),
                              _p(out, C.c_int32))
    return out


def grid_dims(size: float, spacing: float) -> int:
    return lib().or_grid_dims(float(size), float(spacing))


def grid_geometry(box):
    size = np.asarray(box.size, dtype=np.float64)
    dims = np.array([grid_dims(s, box.spacing) for s in size], dtype=np.int32)
    origin = np.asarray(box.center, dtype=np.float64) - size / 2.0
    return origin, dims


class OracleGrid:
    """FP64 maps of one pocket box for a set of ligand XS types (Kernel 1 of the paper)."""

    def __init__(self, rec, box, types: Sequence[int], rec_types: Optional[np.ndarray] = None,
                 threads: int = 0, maps: Optional[np.ndarray] = None):
        self.origin, self.dims = grid_geometry(box)
        self.spacing = float(box.spacing)
        self.types = np.array(sorted(set(int(t) for t in types)), dtype=np.int32)
        nn = int(np.prod(self.dims))
        if maps is None:
            rt = xs_type_receptor(rec) if rec_types is None else np.asarray(rec_types, np.int32)
            maps = np.zeros((len(self.types), nn))
            xyz = np.ascontiguousarray(rec.xyz, np.float64)
            lib().or_grid_build(rec.n, _p(xyz), _p(np.ascontiguousarray(rt), C.c_int32),
                                _p(self.origin), self.spacing, _p(self.dims, C.c_int32),
                                len(self.types), _p(self.types, C.c_int32), _p(maps), int(threads))
        self.maps = np.ascontiguousarray(maps, dtype=np.float64).reshape(len(self.types), nn)
        self.struct = Grid()
        for k in range(3):
            self.struct.origin[k] = self.origin[k]
            self.struct.dims[k] = int(self.dims[k])
        self.struct.spacing = self.spacing
        for t in range(N_XS):
            self.struct.map_of_type[t] = -1
        for m, t in enumerate(self.types):
            self.struct.map_of_type[int(t)] = m
        self.struct.maps = _p(self.maps)

    @classmethod
    def lazy(cls, rec, box, types: Sequence[int], rec_types: np.ndarray, poses_xyz: np.ndarray,
             threads: int = 0) -> "OracleGrid":
        """Maps filled (by direct summation) only at the 8 corner nodes of every cell that the
        given atom positions [..., 3] fall in (clamped like the interpolation); NaN elsewhere."""
        origin, dims = grid_geometry(box)
        sp = float(box.spacing)
        p = np.asarray(poses_xyz, dtype=np.float64).reshape(-1, 3)
        g = np.clip((p - origin) / sp, 0, dims - 1)
        i = np.minimum(np.floor(g).astype(np.int64), dims - 2)
        corners = []
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    c = i + np.array([dx, dy, dz])
                    corners.append((c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0])
        nodes = np.unique(np.concatenate(corners)).astype(np.int64)
        tt = np.array(sorted(set(int(t) for t in types)), dtype=np.int32)
        nn = int(np.prod(dims))
        maps = np.full((len(tt), nn), np.nan)
        lib().or_grid_fill_nodes(rec.n, _p(np.ascontiguousarray(rec.xyz, np.float64)),
                                 _p(np.ascontiguousarray(rec_types, np.int32), C.c_int32), _p(origin), sp,
                                 _p(dims.astype(np.int32), C.c_int32), len(tt), _p(tt, C.c_int32), len(nodes),
                                 nodes.ctypes.data_as(C.POINTER(C.c_int64)), _p(maps), int(threads))
        return cls(None, box, tt, maps=maps)

    def map(self, t: int) -> np.ndarray:
        m = int(np.nonzero(self.types == t)[0][0])
        return self.maps[m].reshape(int(self.dims[2]), int(self.dims[1]), int(self.dims[0]))

    def eval(self, t: int, p) -> tuple:
        p = np.ascontiguousarray(p, dtype=np.float64)
        g = np.zeros(3)
        v = lib().or_grid_eval(C.byref(self.struct), int(t), _p(p), _p(g))
        return v, g


def grid_node_value(rec, rec_types, box, t, ix, iy, iz) -> float:
    origin, _ = grid_geometry(box)
    return lib().or_grid_node_value(rec.n, _p(np.ascontiguousarray(rec.xyz, np.float64)),
                                    _p(np.ascontiguousarray(rec_types, np.int32), C.c_int32),
                                    _p(origin), float(box.spacing), int(t), int(ix), int(iy), int(iz))


class OracleLigand:
    """Torsion tree of one ligand (rigid fragments, torsions in input order, intra pairs)."""

    def __init__(self, lig):
        self.src = lig
        b = np.ascontiguousarray(lig.bonds, dtype=np.int32)
        self._keep = [np.ascontiguousarray(lig.xyz, np.float64),
                      np.ascontiguousarray(lig.element, np.uint8),
                      np.ascontiguousarray(lig.donor, np.uint8),
                      np.ascontiguousarray(lig.acceptor, np.uint8), b,
                      np.ascontiguousarray(lig.rotatable, np.uint8)]
        x, e, d, a, b, r = self._keep
        self.ptr = lib().or_ligand_new(lig.n, _p(x), _p(e, C.c_uint8), _p(d, C.c_uint8),
                                       _p(a, C.c_uint8), b.shape[0], _p(b, C.c_int32),
                                       _p(r, C.c_uint8))
        if not self.ptr:
            raise ValueError("rotatable bond that is not a bridge")
        info = np.zeros(6, dtype=np.int32)
        rg = C.c_double()
        lib().or_ligand_info(self.ptr, _p(info, C.c_int32), C.byref(rg))
        self.n, self.n_rot, self.n_frag, self.root, self.origin, self.n_pairs = (int(v) for v in info)
        self.rgyr = rg.value
        self.xs = np.zeros(self.n, np.int32)
        self.frag_of = np.zeros(self.n, np.int32)
        self.pairs = np.zeros((max(self.n_pairs, 1), 2), np.int32)
        self.tor_p = np.zeros(max(self.n_rot, 1), np.int32)
        self.tor_c = np.zeros(max(self.n_rot, 1), np.int32)
        lib().or_ligand_arrays(self.ptr, _p(self.xs, C.c_int32), _p(self.frag_of, C.c_int32),
                               _p(self.pairs, C.c_int32), _p(self.tor_p, C.c_int32),
                               _p(self.tor_c, C.c_int32))
        self.pairs = self.pairs[:self.n_pairs]
        self.tor_p = self.tor_p[:self.n_rot]
        self.tor_c = self.tor_c[:self.n_rot]

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().or_ligand_free(self.ptr)
            self.ptr = None

    @property
    def n_pot(self) -> int:
        return 7 + self.n_rot

    def fk(self, pot) -> np.ndarray:
        pot = np.ascontiguousarray(pot, dtype=np.float64)
        out = np.zeros((self.n, 3))
        lib().or_fk(self.ptr, _p(pot), _p(out))
        return out

    def score(self, grid: OracleGrid, pot, want_grad: bool = True):
        pot = np.ascontiguousarray(pot, dtype=np.float64)
        g = np.zeros(6 + self.n_rot)
        parts = np.zeros(2)
        e = lib().or_score(self.ptr, C.byref(grid.struct), _p(pot), _p(g) if want_grad else None,
                           _p(parts))
        return e, g, parts

    def score_atoms(self, grid: OracleGrid, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        g = np.zeros_like(xyz)
        e = lib().or_score_atoms(self.ptr, C.byref(grid.struct), _p(xyz), _p(g))
        return e, g

    def direct_inter(self, rec, rec_types, xyz) -> float:
        """e_inter of posed atoms (input order) summed directly over the receptor (no grid)."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        return lib().or_direct_inter(self.ptr, rec.n, _p(np.ascontiguousarray(rec.xyz, np.float64)),
                                     _p(np.ascontiguousarray(rec_types, np.int32), C.c_int32), _p(xyz))

    def retract(self, pot, step) -> np.ndarray:
        pot = np.ascontiguousarray(pot, dtype=np.float64)
        step = np.ascontiguousarray(step, dtype=np.float64)
        out = np.zeros_like(pot)
        lib().or_retract(self.n_rot, _p(pot), _p(step), _p(out))
        return out


@dataclasses.dataclass
class SearchParams:
    """Search constants (paper Eq. 7-8: rho = 1e-4, sigma = 0.1; the rest are readings)."""
    seed: int = 0
    steps: int = 1000
    temperature: float = 1.2
    amplitude: float = 2.0
    m: int = 5
    max_iter: int = 0          # 0: floor((25 + N_atoms) / 3)
    max_trials: int = 10
    rho: float = 1e-4
    sigma: float = 0.1
    eps: float = 1e-3
    top_k: int = 9
    rmsd_min: float = 1.0
    focc: int = 0              # first-order consistency check (Eq. 4-5): neighbours kept, 0 = off
    focc_min_delta: float = 1e-4

    def bfgs(self) -> BfgsParams:
        return BfgsParams(self.m, self.max_iter, self.max_trials, self.rho, self.sigma, self.eps)

    def mc(self) -> McParams:
        return McParams(self.seed, self.steps, self.temperature, self.amplitude, self.bfgs(), self.focc,
                        self.focc_min_delta)


def bfgs_generic(f_and_grad, retract, x0, n_tan: int, params: SearchParams):
    """RILC-BFGS of the oracle on a Python objective (used by the optimiser pins)."""
    n_state = len(x0)

    def _eval(_ctx, xp, gp):
        x = np.ctypeslib.as_array(xp, shape=(n_state,)).copy()
        f, g = f_and_grad(x)
        for i in range(n_tan):
            gp[i] = float(g[i])
        return float(f)

    def _retract(_ctx, xp, sp, op):
        x = np.ctypeslib.as_array(xp, shape=(n_state,)).copy()
        s = np.ctypeslib.as_array(sp, shape=(n_tan,)).copy()
        o = retract(x, s)
        for i in range(n_state):
            op[i] = float(o[i])

    ef, rf = EVAL_FN(_eval), RETRACT_FN(_retract)
    prob = Problem(n_tan, n_state, ef, rf, None)
    x = np.ascontiguousarray(x0, dtype=np.float64).copy()
    g = np.zeros(n_tan)
    ev = C.c_long(0)
    bp = params.bfgs()
    if bp.max_iter <= 0:
        bp.max_iter = 100
    f = lib().or_bfgs(C.byref(prob), C.byref(bp), _p(x), _p(g), C.byref(ev))
    return x, f, g, ev.value


def bfgs_pose(lig: OracleLigand, grid: OracleGrid, pot, params: SearchParams):
    pot = np.ascontiguousarray(pot, dtype=np.float64).copy()
    g = np.zeros(6 + lig.n_rot)
    ev = C.c_long(0)
    bp = params.bfgs()
    f = lib().or_bfgs_pose(lig.ptr, C.byref(grid.struct), C.byref(bp), _p(pot), _p(g), C.byref(ev))
    return pot, f, g, ev.value


def random_conformation(lig: OracleLigand, box, seed: int, unit: int, chain: int) -> np.ndarray:
    pot = np.zeros(lig.n_pot)
    c = np.ascontiguousarray(box.center, np.float64)
    s = np.ascontiguousarray(box.size, np.float64)
    lib().or_random_conformation(lig.ptr, _p(c), _p(s), int(seed), int(unit), int(chain), _p(pot))
    return pot


def mutate(lig: OracleLigand, pot, amplitude: float, seed: int, unit: int, chain: int, step: int):
    pot = np.ascontiguousarray(pot, dtype=np.float64)
    out = np.zeros_like(pot)
    lib().or_mutate(lig.ptr, _p(pot), float(amplitude), int(seed), int(unit), int(chain), int(step),
                    _p(out))
    return out


def metropolis_uniform(seed: int, unit: int, chain: int, step: int) -> float:
    return lib().or_metropolis_uniform(int(seed), int(unit), int(chain), int(step))


def metropolis_accept(e_cur: float, e_new: float, temperature: float, u: float) -> bool:
    return bool(lib().or_metropolis_accept(float(e_cur), float(e_new), float(temperature), float(u)))


def mc_chains(lig: OracleLigand, grid: OracleGrid, box, params: SearchParams, unit: int,
              n_chains: int, chain0: int = 0, threads: int = 0):
    """Runs chains chain0 .. chain0 + n_chains - 1 of one unit. Returns (best_pot, best_e, evals)."""
    np_ = lig.n_pot
    pots = np.zeros((n_chains, np_))
    es = np.zeros(n_chains)
    ev = np.zeros(n_chains, dtype=np.int64)
    mp = params.mc()
    c = np.ascontiguousarray(box.center, np.float64)
    s = np.ascontiguousarray(box.size, np.float64)
    if chain0 == 0:
        lib().or_mc_chains(lig.ptr, C.byref(grid.struct), _p(c), _p(s), C.byref(mp), int(unit),
                           int(n_chains), _p(pots), _p(es), _p(ev, C.c_long), int(threads))
    else:
        for i in range(n_chains):
            e = C.c_double()
            n = C.c_long()
            row = np.zeros(np_)
            lib().or_mc_chain(lig.ptr, C.byref(grid.struct), _p(c), _p(s), C.byref(mp), int(unit),
                              int(chain0 + i), _p(row), C.byref(e), C.byref(n))
            pots[i], es[i], ev[i] = row, e.value, n.value
    return pots, es, ev


def tangent_delta(n_rot: int, a, b) -> np.ndarray:
    """a - b in the optimiser's tangent space (translation, rotation vector, wrapped torsions)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(6 + n_rot)
    lib().or_tangent_delta(int(n_rot), _p(a), _p(b), _p(out))
    return out


def focc_pass(lig: OracleLigand, pot_i, f_i: float, g_i, nb_pots, nb_f, nb_g, min_delta: float = 1e-4) -> bool:
    """First-order consistency check (Eq. 4-5) of a candidate against stored neighbours."""
    pot_i = np.ascontiguousarray(pot_i, dtype=np.float64)
    g_i = np.ascontiguousarray(g_i, dtype=np.float64)
    nb_pots = np.ascontiguousarray(np.reshape(nb_pots, (-1, lig.n_pot)), dtype=np.float64)
    nb_g = np.ascontiguousarray(np.reshape(nb_g, (-1, 6 + lig.n_rot)), dtype=np.float64)
    nb_f = np.ascontiguousarray(nb_f, dtype=np.float64)
    return bool(lib().or_focc_pass(lig.ptr, _p(pot_i), float(f_i), _p(g_i), len(nb_f), _p(nb_pots), _p(nb_f),
                                   _p(nb_g), float(min_delta)))


def topk(scores, xyz, k: int, rmsd_min: float) -> np.ndarray:
    scores = np.ascontiguousarray(scores, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n_cand, n_atoms = xyz.shape[0], xyz.shape[1]
    out = np.zeros(max(k, 1), dtype=np.int32)
    kept = lib().or_topk(n_cand, _p(scores), _p(xyz), n_atoms, int(k), float(rmsd_min),
                         _p(out, C.c_int32))
    return out[:kept]


def affinity(e_inter: float, n_rot: int) -> float:
    return lib().or_affinity(float(e_inter), int(n_rot))


@dataclasses.dataclass
class PairResult:
    ligand: int
    pocket: int
    chain_pots: np.ndarray
    chain_scores: np.ndarray
    evals: int
    kept: np.ndarray        # chain ids in rank order
    scores: np.ndarray      # SF of kept poses
    e_inter: np.ndarray
    e_intra: np.ndarray
    affinity: np.ndarray


def dock_pair(lig: OracleLigand, grid: OracleGrid, box, params: SearchParams, unit: int,
              n_chains: int, ligand_index: int = 0, pocket_index: int = 0,
              threads: int = 0) -> PairResult:
    """All chains of one (ligand, pocket) pair, then sort + RMSD filter + top-k (Algorithm 2)."""
    pots, es, ev = mc_chains(lig, grid, box, params, unit, n_chains, threads=threads)
    xyz = np.stack([lig.fk(p) for p in pots]) if n_chains else np.zeros((0, lig.n, 3))
    kept = topk(es, xyz, params.top_k, params.rmsd_min)
    parts = np.array([lig.score(grid, pots[c], want_grad=False)[2] for c in kept]).reshape(-1, 2)
    aff = np.array([affinity(p[0], lig.n_rot) for p in parts])
    return PairResult(ligand_index, pocket_index, pots, es, int(ev.sum()), kept, es[kept],
                      parts[:, 0], parts[:, 1], aff)


def merge_pockets(results: List[PairResult]):
    """Cross-pocket aggregation of one ligand (Algorithm 3): every kept pose of every pocket,
    ordered by SF, ties by (pocket, chain). Returns a list of (score, pocket, chain)."""
    rows = []
    for r in results:
        for s, c in zip(r.scores, r.kept):
            rows.append((float(s), int(r.pocket), int(c)))
    return sorted(rows)


# ------------------------------------------------- pocket side (Supplementary Algorithm 1) --

def sphere_lattice(n: int) -> np.ndarray:
    """The n directions of the spherical Fibonacci lattice, float64 [n, 3]."""
    out = np.zeros((max(n, 1), 3))
    lib().or_sphere_lattice(int(n), _p(out))
    return out[:n]


def sas_points(xyz, radius, probe: float, n_sphere: int, atoms=None):
    """Step 1 (numerical SAS). Returns (keep uint8, points float64 [., 3], margin float64), rows
    ordered (atom, lattice direction) over ``atoms`` (default: every atom)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    sel = None if atoms is None else np.ascontiguousarray(atoms, dtype=np.int32)
    rows = (xyz.shape[0] if sel is None else sel.shape[0]) * n_sphere
    keep = np.zeros(max(rows, 1), np.uint8)
    pts = np.zeros((max(rows, 1), 3))
    margin = np.zeros(max(rows, 1))
    lib().or_sas_points(xyz.shape[0], _p(xyz), _p(radius), float(probe), int(n_sphere),
                        0 if sel is None else sel.shape[0], None if sel is None else _p(sel, C.c_int32),
                        _p(keep, C.c_uint8), _p(pts), _p(margin))
    return keep[:rows], pts[:rows], margin[:rows]


def point_features(xyz, props, pts, r_feat: float = 6.0, r_prot: float = 10.0):
    """Step 2: Eq. 1 sums [n_pts, n_props] and protrusion counts [n_pts] at the given points."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    props = np.ascontiguousarray(props, dtype=np.float64).reshape(xyz.shape[0], -1)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    feat = np.zeros((max(pts.shape[0], 1), props.shape[1]))
    prot = np.zeros(max(pts.shape[0], 1), np.int32)
    lib().or_point_features(xyz.shape[0], _p(xyz), props.shape[1], _p(props), pts.shape[0], _p(pts),
                            float(r_feat), float(r_prot), _p(feat), _p(prot, C.c_int32))
    return feat[:pts.shape[0]], prot[:pts.shape[0]]


@dataclasses.dataclass
class Clusters:
    root: np.ndarray       # [n] lowest point index of the point's cluster, -1 below threshold
    cluster: np.ndarray    # [n] rank of the point's cluster, -1 below threshold
    score: np.ndarray      # [K] Eq. 2 score, descending
    center: np.ndarray     # [K, 3]
    size: np.ndarray       # [K]
    first: np.ndarray      # [K] lowest point index


def cluster_points(pts, score, theta: float, link: float = 3.0) -> Clusters:
    """Steps 4-5: threshold, single-linkage clusters, Eq. 2 scores, centres, ranking."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    score = np.ascontiguousarray(score, dtype=np.float64)
    n = pts.shape[0]
    m = max(n, 1)
    root, cl = np.zeros(m, np.int32), np.zeros(m, np.int32)
    cs, cc, sz, fi = np.zeros(m), np.zeros((m, 3)), np.zeros(m, np.int32), np.zeros(m, np.int32)
    k = lib().or_cluster_points(n, _p(pts), _p(score), float(theta), float(link), _p(root, C.c_int32),
                                _p(cl, C.c_int32), _p(cs), _p(cc), _p(sz, C.c_int32), _p(fi, C.c_int32))
    return Clusters(root[:n], cl[:n], cs[:k], cc[:k], sz[:k], fi[:k])
