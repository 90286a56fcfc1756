// pv_check.cu -- verification of the search's optimiser: RILC-BFGS (Eq. 6-12) exactly as the
// search kernels run it (the warp_rilc_bfgs and thread_rilc_bfgs templates that the docking chains
// instantiate with the docking score), instantiated here with analytic objectives, so that its
// iterations can be compared with a reference implementation step for step. A docking objective
// cannot serve for that in FP32 against FP64: its trilinear maps and cutoffs make line-search
// decisions that rounding flips, while a smooth analytic function keeps every decision clear.
#include <cstring>
#include <string>

#include "pocketvina.h"
#include "pv_chain.cuh"
#include "pv_thread.cuh"

using namespace pv;

namespace {

constexpr int kCheckWarps = 4;

// Term k of the objective and its partial derivative in coordinate k, from coordinates k - 1, k,
// k + 1 (kind 0: f = sum_k a_k x_k^2 / 2; kind 1, the extended Rosenbrock function:
// f = sum_{k < n-1} 100 (x_{k+1} - x_k^2)^2 + (1 - x_k)^2).
__device__ __forceinline__ float analytic_term(int kind, int n, int k, float xp, float x, float xn, float a,
                                               float& g) {
    if (k >= n) {
        g = 0.f;
        return 0.f;
    }
    if (kind == 0) {
        g = a * x;
        return 0.5f * a * x * x;
    }
    float f = 0.f;
    g = 0.f;
    if (k + 1 < n) {
        const float u = xn - x * x, v = 1.f - x;
        f = 100.f * u * u + v * v;
        g = -400.f * x * u - 2.f * v;
    }
    if (k > 0) g += 200.f * (x - xp * xp);
    return f;
}

// Whole-warp form: lane k holds coordinate k (n <= 32).
struct WarpAnalytic {
    using State = float;
    int kind, n;
    float a;                       // the lane's coefficient (quadratic)
    __device__ __forceinline__ float eval(const float& x, float& g) const {
        const int k = threadIdx.x & 31;
        const float xn = __shfl_down_sync(PV_FULL, x, 1), xp = __shfl_up_sync(PV_FULL, x, 1);
        return Team<32>::sum(analytic_term(kind, n, k, xp, x, xn, a, g));
    }
    __device__ __forceinline__ float retract(const float& x, float step) const { return x + step; }
};

// Thread form: one thread holds all n coordinates.
struct ThreadAnalytic {
    int kind, nt, np;
    const float* a;
    int* evals;
    __device__ __forceinline__ float eval(const float* x, float* g) const {
        float f = 0.f;
        for (int k = 0; k < nt; ++k) {
            float gk;
            f += analytic_term(kind, nt, k, k > 0 ? x[k - 1] : 0.f, x[k], k + 1 < nt ? x[k + 1] : 0.f,
                               kind == 0 ? a[k] : 0.f, gk);
            g[k] = gk;
        }
        ++*evals;
        return f;
    }
    __device__ __forceinline__ void retract(const float* x, const float* s, float* y) const {
        for (int k = 0; k < nt; ++k) y[k] = x[k] + s[k];
    }
};

__global__ void __launch_bounds__(32 * kCheckWarps) bfgs_check_warp_kernel(int kind, int n, int n_problems,
                                                                           const float* coef, float* x,
                                                                           PvSearchConst C, int max_iter,
                                                                           float* f_out, int* evals_out) {
    __shared__ WarpScratch S[kCheckWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int prob = blockIdx.x * kCheckWarps + w;
    if (prob >= n_problems) return;                 // whole warps leave together
    const WarpAnalytic obj{kind, n, (kind == 0 && lane < n) ? coef[(size_t)prob * n + lane] : 0.f};
    float xs = lane < n ? x[(size_t)prob * n + lane] : 0.f;
    uint32_t evals = 0;
    float g = 0.f;
    const float f = warp_rilc_bfgs<false>(obj, S[w], xs, C, max_iter, evals, g, nullptr, 0);
    if (lane < n) x[(size_t)prob * n + lane] = xs;
    if (lane == 0) {
        f_out[prob] = f;
        evals_out[prob] = (int)evals;
    }
}

__global__ void __launch_bounds__(128) bfgs_check_thread_kernel(int kind, int n, int n_problems, const float* coef,
                                                                float* x, PvSearchConst C, int max_iter,
                                                                float* f_out, int* evals_out) {
    const int prob = blockIdx.x * blockDim.x + threadIdx.x;
    if (prob >= n_problems) return;
    float xl[PV_MAX_POT];
    for (int k = 0; k < n; ++k) xl[k] = x[(size_t)prob * n + k];
    int evals = 0;
    const ThreadAnalytic obj{kind, n, n, kind == 0 ? coef + (size_t)prob * n : nullptr, &evals};
    const float f = thread_rilc_bfgs(obj, xl, C, max_iter);
    for (int k = 0; k < n; ++k) x[(size_t)prob * n + k] = xl[k];
    f_out[prob] = f;
    evals_out[prob] = evals;
}

pv_status fail(pv_context* ctx, pv_status s, const std::string& msg) {
    context_set_error(ctx, msg.c_str());
    return s;
}

}  // namespace

extern "C" pv_status pv_check_bfgs(pv_context* ctx, int32_t form, int32_t objective, int32_t n, int32_t n_problems,
                                   const float* dev_coef, float* dev_x, const pv_dock_params* p, float* dev_f,
                                   int32_t* dev_evals) {
    int device = -1;
    cudaStream_t stream = nullptr;
    if (!context_device_stream(ctx, &device, &stream)) return PV_ERR_STATE;
    if (form != 0 && form != 1) return fail(ctx, PV_ERR_ARG, "form must be 0 (whole warp) or 1 (thread)");
    if (objective != PV_OBJ_QUADRATIC && objective != PV_OBJ_ROSENBROCK)
        return fail(ctx, PV_ERR_ARG, "unknown objective");
    if (n < 1 || n > 32) return fail(ctx, PV_ERR_ARG, "n must be in [1, 32]");
    if (n_problems < 0 || !p) return fail(ctx, PV_ERR_ARG, "bad arguments");
    if (n_problems == 0) return PV_OK;
    if (!dev_x || !dev_f || !dev_evals || (objective == PV_OBJ_QUADRATIC && !dev_coef))
        return fail(ctx, PV_ERR_ARG, "device arrays required");
    if (p->bfgs_m < 1 || p->bfgs_m > 5 || p->bfgs_max_iter < 1 || p->bfgs_max_trials < 1)
        return fail(ctx, PV_ERR_ARG, "bfgs_m in [1, 5], bfgs_max_iter >= 1 and bfgs_max_trials >= 1 required");
    PvSearchConst C;
    std::memset(&C, 0, sizeof(C));
    C.bfgs_m = p->bfgs_m;
    C.bfgs_max_iter = p->bfgs_max_iter;
    C.bfgs_max_trials = p->bfgs_max_trials;
    C.eps = p->bfgs_eps;
    C.rho = p->rho;
    C.sigma = p->sigma;
    int prev = -1;
    cudaGetLastError();   // report only this call's launch below
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail(ctx, PV_ERR_CUDA, "cudaSetDevice failed");
    if (form == 0)
        bfgs_check_warp_kernel<<<(n_problems + kCheckWarps - 1) / kCheckWarps, 32 * kCheckWarps, 0, stream>>>(
            objective, n, n_problems, dev_coef, dev_x, C, p->bfgs_max_iter, dev_f, dev_evals);
    else
        bfgs_check_thread_kernel<<<(n_problems + 127) / 128, 128, 0, stream>>>(objective, n, n_problems, dev_coef,
                                                                              dev_x, C, p->bfgs_max_iter, dev_f,
                                                                              dev_evals);
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(ctx, PV_ERR_CUDA, std::string("pv_check_bfgs: ") + cudaGetErrorString(e));
    return PV_OK;
}
