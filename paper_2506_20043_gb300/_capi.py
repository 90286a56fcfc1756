"""ctypes declarations of the C ABI in include/pocketvina.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpocketvina.so")

PV_OK, PV_ERR_ARG, PV_ERR_CUDA, PV_ERR_OOM, PV_ERR_TIMEOUT, PV_ERR_NAN, PV_ERR_STATE = range(7)
PV_MEM_HOST, PV_MEM_DEVICE = 0, 1
PV_MODE_BATCHED, PV_MODE_PLAIN, PV_MODE_PLAIN_WARP = 0, 1, 2
PV_OBJ_QUADRATIC, PV_OBJ_ROSENBROCK = 0, 1
STATUS_NAMES = {0: "PV_OK", 1: "PV_ERR_ARG", 2: "PV_ERR_CUDA", 3: "PV_ERR_OOM", 4: "PV_ERR_TIMEOUT",
                5: "PV_ERR_NAN", 6: "PV_ERR_STATE"}


class pv_receptor(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.c_void_p), ("element", C.c_void_p),
                ("donor", C.c_void_p), ("acceptor", C.c_void_p), ("mem", C.c_int32)]


class pv_box(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("size", C.c_float * 3), ("spacing", C.c_float)]


class pv_ligand_desc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.c_void_p), ("element", C.c_void_p),
                ("donor", C.c_void_p), ("acceptor", C.c_void_p), ("n_bonds", C.c_int32),
                ("bonds", C.c_void_p), ("rotatable", C.c_void_p)]


class pv_dock_params(C.Structure):
    _fields_ = [("chains", C.c_int32), ("steps", C.c_int32), ("seed", C.c_uint64),
                ("top_k", C.c_int32), ("rmsd_min", C.c_float), ("mode", C.c_int32),
                ("bfgs_m", C.c_int32), ("bfgs_max_iter", C.c_int32), ("bfgs_max_trials", C.c_int32),
                ("bfgs_eps", C.c_float), ("rho", C.c_float), ("sigma", C.c_float),
                ("temperature", C.c_float), ("amplitude", C.c_float), ("steps_per_round", C.c_int32),
                ("use_graph", C.c_int32), ("warps_per_cta", C.c_int32), ("search_variant", C.c_int32),
                ("host_copy", C.c_int32),
                ("timeout_s", C.c_double), ("focc", C.c_int32), ("focc_min_delta", C.c_float),
                ("rescore", C.c_int32), ("max_pockets", C.c_int32), ("block_wait_s", C.c_double),
                ("pair_keys", C.POINTER(C.c_int32)), ("map_layout", C.c_int32),
                ("resume_state", C.c_void_p), ("resume_bytes", C.c_int64)]


class pv_pose(C.Structure):
    _fields_ = [("score", C.c_float), ("e_inter", C.c_float), ("e_intra", C.c_float),
                ("affinity", C.c_float), ("pair", C.c_int32), ("ligand", C.c_int32),
                ("pocket", C.c_int32), ("chain", C.c_int32), ("score_grid", C.c_float),
                ("e_inter_grid", C.c_float), ("pad", C.c_int32 * 2)]


class pv_pocket_params(C.Structure):
    _fields_ = [("probe", C.c_float), ("n_sphere", C.c_int32), ("r_feature", C.c_float),
                ("r_protrusion", C.c_float), ("threshold", C.c_float), ("link", C.c_float)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

vp = C.c_void_p
i32, i64, u64 = C.c_int32, C.c_int64, C.c_uint64
pi32 = C.POINTER(C.c_int32)
pf32 = C.POINTER(C.c_float)

SIGNATURES = {
    "pv_context_create": (i32, [C.c_int, vp, C.POINTER(vp)]),
    "pv_context_destroy": (None, [vp]),
    "pv_last_error": (C.c_char_p, [vp]),
    "pv_context_set_stream": (i32, [vp, vp]),
    "pv_context_set_allocator": (i32, [vp, ALLOC_FN, FREE_FN, vp]),
    "pv_build_grids": (i32, [vp, C.POINTER(pv_receptor), C.POINTER(pv_box), i32, C.POINTER(C.c_uint8), i32,
                             C.POINTER(vp)]),
    "pv_grid_set_append": (i32, [vp, vp, C.POINTER(pv_receptor), C.POINTER(pv_box), i32, pi32]),
    "pv_grid_set_destroy": (None, [vp]),
    "pv_grid_set_info": (i32, [vp, pi32, C.POINTER(i64)]),
    "pv_grid_set_build_seconds": (i32, [vp, C.POINTER(C.c_double)]),
    "pv_grid_set_pack": (i32, [vp, vp]),
    "pv_grid_set_view": (i32, [vp, i32, i32, C.POINTER(vp), pi32, pf32, pf32]),
    "pv_grid_set_read_map": (i32, [vp, i32, i32, vp]),
    "pv_ligand_create": (i32, [vp, C.POINTER(pv_ligand_desc), C.POINTER(vp)]),
    "pv_ligand_destroy": (None, [vp]),
    "pv_ligand_info": (i32, [vp, pi32, pi32, pi32, pi32]),
    "pv_ligand_cost": (i32, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pv_ligand_xs_types": (i32, [vp, C.POINTER(C.c_uint8)]),
    "pv_score": (i32, [vp, vp, vp, i32, i32, vp, vp, vp, vp]),
    "pv_score_backward": (i32, [vp, vp, vp, i32, i32, vp, vp, vp, vp]),
    "pv_pose_coords": (i32, [vp, vp, i32, vp, vp]),
    "pv_score_xyz": (i32, [vp, vp, vp, i32, i32, vp, vp, vp, vp]),
    "pv_measure_gather": (i32, [vp, vp, i32, i64, i32, vp]),
    "pv_measure_gather_layout": (i32, [vp, vp, i32, i64, i32, i32, vp]),
    "pv_dock_params_default": (None, [C.POINTER(pv_dock_params)]),
    "pv_check_bfgs": (i32, [vp, i32, i32, i32, i32, vp, vp, C.POINTER(pv_dock_params), vp, vp]),
    "pv_dock": (i32, [vp, vp, C.POINTER(vp), i32, pi32, i32, C.POINTER(pv_dock_params), C.POINTER(vp)]),
    "pv_dock_pairs": (i32, [vp, vp, C.POINTER(vp), i32, pi32, pi32, i32, C.POINTER(pv_dock_params),
                            C.POINTER(vp)]),
    "pv_dock_result_info": (i32, [vp, pi32, pi32, pi32, pi32]),
    "pv_dock_result_poses": (i32, [vp, C.POINTER(pv_pose), pi32, pf32, pf32]),
    "pv_dock_result_ranking": (i32, [vp, i32, pi32, pi32]),
    "pv_dock_result_stats": (i32, [vp, C.POINTER(u64), C.POINTER(C.c_double), pi32]),
    "pv_dock_result_timing": (i32, [vp, C.POINTER(C.c_double), pi32, C.POINTER(C.c_double)]),
    "pv_dock_result_launch": (i32, [vp, pi32, pi32]),
    "pv_dock_result_map_layout": (i32, [vp, pi32]),
    "pv_dock_result_device": (i32, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
    "pv_dock_result_chains": (i32, [vp, C.POINTER(vp), pi32, pi32, pi32, pi32]),
    "pv_dock_result_read_chains": (i32, [vp, vp]),
    "pv_dock_result_state_bytes": (i32, [vp, C.POINTER(C.c_int64)]),
    "pv_dock_result_save_state": (i32, [vp, vp, C.c_int64]),
    "pv_dock_result_destroy": (None, [vp]),
    "pv_build_grid_noalloc": (i32, [vp, C.POINTER(pv_receptor), C.POINTER(pv_box), C.POINTER(C.c_uint8), i32, vp]),
    "pv_pocket_params_default": (i32, [C.POINTER(pv_pocket_params)]),
    "pv_surface_create": (i32, [vp, C.POINTER(pv_receptor), vp, C.POINTER(pv_pocket_params), C.POINTER(vp)]),
    "pv_surface_create_many": (i32, [vp, i32, vp, vp, C.POINTER(pv_pocket_params), C.POINTER(vp)]),
    "pv_surface_info": (i32, [vp, pi32, pi32]),
    "pv_surface_read": (i32, [vp, vp, vp, vp, i32]),
    "pv_surface_points": (i32, [vp, C.POINTER(vp)]),
    "pv_surface_features": (i32, [vp, vp, i32, vp, i32, i32, vp, i32, C.POINTER(pv_pocket_params), vp, vp]),
    "pv_surface_destroy": (None, [vp]),
    "pv_cluster_points": (i32, [vp, i32, vp, vp, C.POINTER(pv_pocket_params), C.POINTER(vp)]),
    "pv_cluster_points_many": (i32, [vp, i32, vp, vp, vp, C.POINTER(pv_pocket_params), C.POINTER(vp)]),
    "pv_clusters_info": (i32, [vp, pi32, pi32]),
    "pv_clusters_read": (i32, [vp, vp, vp, vp, vp, vp, vp, i32]),
    "pv_clusters_destroy": (None, [vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libpocketvina.so and declares every entry point. Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libpocketvina.so not built ({path}); run paper_2506_20043_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
