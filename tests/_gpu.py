"""Shared setup of the GPU parity tests: a library context, synthetic sites and oracle twins."""
import functools
import os

import numpy as np
import pytest

import oracle as O
import pvsynth as S

# Parity tolerance for grid values and per-pose SF (FP32 kernel vs FP64 oracle):
# |gpu - oracle| <= 1e-3 kcal/mol or <= 1e-4 relative.
ABS_TOL, REL_TOL = 1e-3, 1e-4
# Gradient tolerance: |gpu - oracle| <= 1e-3 * max(|oracle|, 1).
GRAD_TOL = 1e-3


def close(gpu, ref, abs_tol=ABS_TOL, rel_tol=REL_TOL):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    return (np.abs(gpu - ref) <= abs_tol) | (np.abs(gpu - ref) <= rel_tol * np.abs(ref))


def threads():
    return len(os.sched_getaffinity(0))


@functools.lru_cache(maxsize=None)
def context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_20043_gb300 as pv
    pv.build()
    from paper_2506_20043_gb300 import api
    return api.Context(0)


def box32(box):
    """The box as the float32 values the library receives (so both sides use the same grid)."""
    return S.Box(np.asarray(box.center, np.float32).astype(np.float64),
                 np.asarray(box.size, np.float32).astype(np.float64), float(np.float32(box.spacing)))


def receptor32(rec):
    return S.Receptor(np.asarray(rec.xyz, np.float32).astype(np.float64), rec.element, rec.donor, rec.acceptor)


def ligand32(lig):
    import dataclasses
    return dataclasses.replace(lig, xyz=np.asarray(lig.xyz, np.float32).astype(np.float64))
