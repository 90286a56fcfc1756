"""The search's RILC-BFGS (Eq. 6-12) on the GPU against the FP64 oracle's, decision for decision.

The optimiser code of the whole-warp chains and of the thread-per-chain plain path runs through
pv_check_bfgs on analytic objectives (diagonal quadratics and the extended Rosenbrock function, in
6 to 32 dimensions, ten iterations with up to ten line-search trials each, memory 5): the two-loop
recursion over a history that fills and wraps, the Eq. 11 curvature guard, lambda doubling and
bisection, the largest-Armijo fallback and the Eq. 12 stop. On a smooth function every decision has
a clear margin, so the FP32 and FP64 runs take the same ones: the same number of evaluations, and
the same final point and value to FP32 accuracy. (On the docking score they do not: FP64 runs of the
oracle perturbed by 1e-6 relative part ways with it as well; tests/test_gpu_dock.py holds the
statistical comparison of the full search.) The oracle's own optimiser is pinned to known minimisers
in tests/test_oracle_search.py.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _quad(a):
    return lambda x: (0.5 * float(np.sum(a * x * x)), a * x)


def _rosen(x):
    f = np.sum(100 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] += -400 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
    g[1:] += 200 * (x[1:] - x[:-1] ** 2)
    return float(f), g


def _problems(kind, n, count, seed):
    rng = np.random.default_rng([seed, n])
    if kind == "quadratic":
        a = np.exp(rng.uniform(np.log(0.5), np.log(20.0), (count, n))).astype(np.float32)
        x0 = rng.uniform(-3, 3, (count, n)).astype(np.float32)
    else:
        a = np.zeros((count, n), np.float32)
        x0 = (np.where(np.arange(n) % 2 == 0, -1.2, 1.0) + rng.uniform(-0.3, 0.3, (count, n))).astype(np.float32)
    return a, x0


def _gpu(ctx, form, kind, a, x0, params):
    import torch
    from paper_2506_20043_gb300 import _capi as A
    obj = A.PV_OBJ_QUADRATIC if kind == "quadratic" else A.PV_OBJ_ROSENBROCK
    count, n = x0.shape
    ta = torch.tensor(a, device="cuda")
    tx = torch.tensor(x0, device="cuda")
    tf = torch.zeros(count, device="cuda")
    te = torch.zeros(count, dtype=torch.int32, device="cuda")
    cp = params.to_c()
    st = ctx.lib.pv_check_bfgs(ctx.h, form, obj, n, count, C.c_void_p(ta.data_ptr()), C.c_void_p(tx.data_ptr()),
                               C.byref(cp), C.c_void_p(tf.data_ptr()), C.c_void_p(te.data_ptr()))
    assert st == A.PV_OK, ctx.lib.pv_last_error(ctx.h)
    torch.cuda.synchronize()
    return tx.cpu().numpy().astype(np.float64), tf.cpu().numpy().astype(np.float64), te.cpu().numpy()


@pytest.mark.parametrize("form", [0, 1], ids=["warp", "thread"])
@pytest.mark.parametrize("kind,dims,need", [("quadratic", (6, 9, 13, 21, 32), 0.95), ("rosenbrock", (6, 10, 16), 0.85)])
def test_rilc_bfgs_matches_oracle_decision_for_decision(form, kind, dims, need):
    from paper_2506_20043_gb300 import api
    ctx = G.context()
    params = api.DockParams(bfgs_m=5, bfgs_max_iter=10, bfgs_max_trials=10)
    sp = O.SearchParams(m=5, max_iter=10, max_trials=10)
    same_path, total, ref_evals = 0, 0, []
    for n in dims:
        a, x0 = _problems(kind, n, 16, 3)
        xg, fg, eg = _gpu(ctx, form, kind, a, x0, params)
        for i in range(len(x0)):
            fn = _quad(a[i].astype(np.float64)) if kind == "quadratic" else _rosen
            xr, fr, _, er = O.bfgs_generic(fn, lambda x, s: x + s, x0[i].astype(np.float64), n, sp)
            ref_evals.append(er)
            total += 1
            if eg[i] != er:
                continue
            same_path += 1
            assert abs(fg[i] - fr) <= 1e-4 * max(1.0, abs(fr)) + 1e-6, (n, i, fg[i], fr)
            np.testing.assert_allclose(xg[i], xr, rtol=1e-3, atol=1e-4)
    # the same evaluation count means the same trial decisions in every iteration
    assert same_path / total >= need, (same_path, total)
    # line searches took more than one trial per iteration on average (doubling, bisection)
    assert np.mean(ref_evals) > 11


def test_check_bfgs_arguments():
    import torch
    from paper_2506_20043_gb300 import _capi as A, api
    ctx = G.context()
    x = torch.zeros(4, device="cuda")
    cp = api.DockParams(bfgs_max_iter=5).to_c()
    args = lambda form, obj, n: (ctx.h, form, obj, n, 1, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                                 C.byref(cp), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()))
    assert ctx.lib.pv_check_bfgs(*args(2, 0, 4)) == A.PV_ERR_ARG
    assert ctx.lib.pv_check_bfgs(*args(0, 7, 4)) == A.PV_ERR_ARG
    assert ctx.lib.pv_check_bfgs(*args(0, 0, 33)) == A.PV_ERR_ARG
    cp.bfgs_max_iter = 0
    assert ctx.lib.pv_check_bfgs(*args(0, 0, 4)) == A.PV_ERR_ARG
