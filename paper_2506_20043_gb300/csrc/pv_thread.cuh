// pv_thread.cuh -- thread-per-chain form of the docking search, the paper's organisation
// ("Kernel 2": n threads per ligand, each one MC + RILC-BFGS chain; Supplementary
// Algorithm 2). It is the plain comparison path: every thread walks the whole ligand serially,
// with its coordinates, forces and optimiser history in per-thread (local) memory. The
// arithmetic follows the same definitions as the warp form in pv_warp.cuh.
#pragma once
#include "pv_device.cuh"
#include "pv_stage.cuh"

namespace pv {

struct ThreadChain {
    const PvLigBlob* L;      // global memory
    const PvPocket* P;
    const float* maps;
    uint64_t slots_lo, slots_hi;
    uint32_t evals;
};

struct ThreadWork {
    float x[64][3];
    float g[64][3];
    Mat3 M[PV_MAX_FRAGS];
    float3 xa[PV_MAX_FRAGS];
};

// SF and its tangent gradient (grad: [6 + n_rot], nullable) of the POT `pot`.
static __device__ __noinline__ float thread_eval(ThreadChain& c, ThreadWork& w, const float* pot, float* grad) {
    const PvLigBlob* L = c.L;
    const int n = L->h.n_atoms, nf = L->h.n_frag, n_rot = L->h.n_rot;
    const float3 T = make_float3(pot[0], pot[1], pot[2]);
    w.M[0] = quat_to_mat(make_float4(pot[3], pot[4], pot[5], pot[6]));
    w.xa[0] = T;
    for (int f = 1; f < nf; ++f) {
        const float4 o = L->frag_off[f], a = L->frag_axis[f];
        const int par = __float_as_int(o.w);
        const Mat3 Rl = axis_angle(f3(a), pot[7 + L->frag_tor[f]]);
        w.M[f] = mat_mul(w.M[par], Rl);
        w.xa[f] = mat_vec(w.M[par], f3(o)) + w.xa[par];
    }
    float e = 0.f;
    const PvPocket& P = *c.P;
    for (int a = 0; a < n; ++a) {
        const float4 loc = L->atom[a];
        const int pw = __float_as_int(loc.w);
        const int fr = pw & 255, xs = (pw >> 8) & 255;
        const float3 p = mat_vec(w.M[fr], f3(loc)) + w.xa[fr];
        w.x[a][0] = p.x; w.x[a][1] = p.y; w.x[a][2] = p.z;
        float3 d;
        const int slot = slot_of(c.slots_lo, c.slots_hi, xs);
        e += grid_eval(c.maps + (long long)slot * P.nxyz, P, p, d);
        w.g[a][0] = d.x; w.g[a][1] = d.y; w.g[a][2] = d.z;
    }
    const int slots = L->h.n_rounds * 32;
    for (int k = 0; k < slots; ++k) {
        const uint32_t pw = (uint32_t)L->pairs[k].meta;
        if (!(pw >> 31)) continue;
        const int i = (k & 31) + 32 * ((pw >> 7) & 1), j = pw & 127;
        const float dx = w.x[i][0] - w.x[j][0], dy = w.x[i][1] - w.x[j][1], dz = w.x[i][2] - w.x[j][2];
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= kCutoff2) continue;
        const float r = sqrtf(r2);
        const int ti = (__float_as_int(L->atom[i].w) >> 8) & 255, tj = (__float_as_int(L->atom[j].w) >> 8) & 255;
        float dedr;
        e += vina_pair(r, xs_radius(ti) + xs_radius(tj), (pw >> 16) & 1, (pw >> 17) & 1, dedr);
        if (r > 1e-6f) {
            const float cf = dedr / r;
            w.g[i][0] += cf * dx; w.g[i][1] += cf * dy; w.g[i][2] += cf * dz;
            w.g[j][0] -= cf * dx; w.g[j][1] -= cf * dy; w.g[j][2] -= cf * dz;
        }
    }
    if (grad) {
        float3 F = make_float3(0.f, 0.f, 0.f), tau = F;
        for (int a = 0; a < n; ++a) {
            const float3 g = make_float3(w.g[a][0], w.g[a][1], w.g[a][2]);
            const float3 p = make_float3(w.x[a][0], w.x[a][1], w.x[a][2]);
            F = F + g;
            tau = tau + cross3(p - T, g);
        }
        grad[0] = F.x; grad[1] = F.y; grad[2] = F.z;
        grad[3] = tau.x; grad[4] = tau.y; grad[5] = tau.z;
        for (int f = 1; f < nf; ++f) {
            float3 t = make_float3(0.f, 0.f, 0.f);
            for (int a = L->frag_a0[f]; a < L->frag_a1[f]; ++a) {
                const float3 g = make_float3(w.g[a][0], w.g[a][1], w.g[a][2]);
                const float3 p = make_float3(w.x[a][0], w.x[a][1], w.x[a][2]);
                t = t + cross3(p - w.xa[f], g);
            }
            grad[6 + L->frag_tor[f]] = dot3(mat_vec(w.M[f], f3(L->frag_axis[f])), t);
        }
        (void)n_rot;
    }
    c.evals++;
    return e;
}

__device__ __forceinline__ void thread_retract(const float* x, const float* s, int n_rot, float* y) {
    y[0] = x[0] + s[0]; y[1] = x[1] + s[1]; y[2] = x[2] + s[2];
    const float4 q = quat_rotate_by(make_float4(x[3], x[4], x[5], x[6]), make_float3(s[3], s[4], s[5]));
    y[3] = q.x; y[4] = q.y; y[5] = q.z; y[6] = q.w;
    for (int k = 0; k < n_rot; ++k) y[7 + k] = x[7 + k] + s[6 + k];
}

// The docking objective of a thread-per-chain chain: SF (Eq. 3) of a POT with its tangent
// gradient, and the retraction of a tangent step. thread_rilc_bfgs is written against this
// interface so that the same optimiser code also runs on analytic objectives (pv_check.cu).
struct ThreadDockObjective {
    ThreadChain& c;
    ThreadWork& w;
    int n_rot, nt, np;             // torsions, tangent and state dimensions
    __device__ __forceinline__ float eval(const float* x, float* g) const { return thread_eval(c, w, x, g); }
    __device__ __forceinline__ void retract(const float* x, const float* s, float* y) const {
        thread_retract(x, s, n_rot, y);
    }
};

// RILC-BFGS on one thread; the same steps as warp_rilc_bfgs (Eq. 6-12).
template <class Obj>
static __device__ float thread_rilc_bfgs(const Obj& obj, float* x, const PvSearchConst& C, int max_iter) {
    const int nt = obj.nt, np = obj.np;
    const int m = C.bfgs_m;
    float g[PV_MAX_TAN], d[PV_MAX_TAN], q[PV_MAX_TAN], gt[PV_MAX_TAN], glo[PV_MAX_TAN];
    float xt[PV_MAX_POT], xlo[PV_MAX_POT], st[PV_MAX_TAN];
    float Sh[PV_MAX_M][PV_MAX_TAN], Yh[PV_MAX_M][PV_MAX_TAN], rh[PV_MAX_M], al[PV_MAX_M];
    int stored = 0;
    float f = obj.eval(x, g);
    for (int it = 0; it < max_iter; ++it) {
        for (int k = 0; k < nt; ++k) q[k] = g[k];
        for (int a = 0; a < stored; ++a) {
            float s = 0.f;
            for (int k = 0; k < nt; ++k) s += Sh[a][k] * q[k];
            al[a] = rh[a] * s;
            for (int k = 0; k < nt; ++k) q[k] -= al[a] * Yh[a][k];
        }
        if (stored > 0) {
            float sy = 0.f, yy = 0.f;
            for (int k = 0; k < nt; ++k) { sy += Sh[0][k] * Yh[0][k]; yy += Yh[0][k] * Yh[0][k]; }
            for (int k = 0; k < nt; ++k) q[k] *= sy / yy;
        }
        for (int a = stored - 1; a >= 0; --a) {
            float b = 0.f;
            for (int k = 0; k < nt; ++k) b += Yh[a][k] * q[k];
            b *= rh[a];
            for (int k = 0; k < nt; ++k) q[k] += Sh[a][k] * (al[a] - b);
        }
        float gd = 0.f;
        for (int k = 0; k < nt; ++k) { d[k] = -q[k]; gd += g[k] * d[k]; }
        if (!(gd < 0.f)) break;
        float lam = 1.f, lo = 0.f, hi = -1.f, ft = 0.f, flo = 0.f;
        bool accepted = false, have_lo = false;
        for (int tr = 0; tr < C.bfgs_max_trials; ++tr) {
            for (int k = 0; k < nt; ++k) st[k] = lam * d[k];
            obj.retract(x, st, xt);
            ft = obj.eval(xt, gt);
            float gtd = 0.f;
            for (int k = 0; k < nt; ++k) gtd += gt[k] * d[k];
            if (!(ft <= f + lam * C.rho * gd)) {
                hi = lam;
            } else if (gtd < C.sigma * gd) {
                lo = lam; have_lo = true; flo = ft;
                for (int k = 0; k < np; ++k) xlo[k] = xt[k];
                for (int k = 0; k < nt; ++k) glo[k] = gt[k];
            } else {
                accepted = true;
                break;
            }
            lam = hi < 0.f ? 2.f * lam : 0.5f * (lo + hi);
        }
        if (!accepted) {
            if (!have_lo) break;
            lam = lo; ft = flo;
            for (int k = 0; k < np; ++k) xt[k] = xlo[k];
            for (int k = 0; k < nt; ++k) gt[k] = glo[k];
        }
        float ys = 0.f, ss = 0.f, gn = 0.f;
        for (int k = 0; k < nt; ++k) {
            const float s = lam * d[k], y = gt[k] - g[k];
            ys += y * s; ss += s * s; gn += g[k] * g[k];
        }
        if (ss > 0.f && ys / ss > C.eps * sqrtf(gn)) {
            for (int a = min(stored, m - 1); a > 0; --a) {
                for (int k = 0; k < nt; ++k) { Sh[a][k] = Sh[a - 1][k]; Yh[a][k] = Yh[a - 1][k]; }
                rh[a] = rh[a - 1];
            }
            for (int k = 0; k < nt; ++k) { Sh[0][k] = lam * d[k]; Yh[0][k] = gt[k] - g[k]; }
            rh[0] = 1.f / ys;
            stored = min(stored + 1, m);
        }
        for (int k = 0; k < np; ++k) x[k] = xt[k];
        float g2 = 0.f;
        for (int k = 0; k < nt; ++k) { g[k] = gt[k]; g2 += g[k] * g[k]; }
        f = ft;
        if (sqrtf(g2) <= C.eps) break;
    }
    return f;
}

static __device__ void thread_run_chain(ThreadChain& c, const PvSearchConst& C, uint32_t chain, uint32_t pair,
                                 int step0, int step1, float* rec, const unsigned long long* t0,
                                 unsigned long long timeout_ns, int* err) {
    ThreadWork w;
    const PvLigBlob* L = c.L;
    const int n_rot = L->h.n_rot, np = 7 + n_rot;
    const int max_iter = C.bfgs_max_iter > 0 ? C.bfgs_max_iter : L->h.bfgs_iters;
    float cur[PV_MAX_POT], cand[PV_MAX_POT], best[PV_MAX_POT];
    float e_cur, e_best;
    uint32_t ev0 = 0;
    if (step0 == 0) {
        uint4 b0 = philox4x32_10(make_uint4(chain, pair, 0u, 0u), C.seed_lo, C.seed_hi);
        uint4 b1 = philox4x32_10(make_uint4(chain, pair, 0u, 1u), C.seed_lo, C.seed_hi);
        const PvPocket& P = *c.P;
        cur[0] = P.center[0] + (u01(b0.x) - 0.5f) * P.size[0];
        cur[1] = P.center[1] + (u01(b0.y) - 0.5f) * P.size[1];
        cur[2] = P.center[2] + (u01(b0.z) - 0.5f) * P.size[2];
        const float u1 = u01(b0.w), u2 = u01(b1.x), u3 = u01(b1.y);
        float s2, c2, s3, c3;
        sincospif(2.f * u2, &s2, &c2);
        sincospif(2.f * u3, &s3, &c3);
        const float a = sqrtf(1.f - u1), b = sqrtf(u1);
        cur[3] = a * s2; cur[4] = a * c2; cur[5] = b * s3; cur[6] = b * c3;
        for (int t = 0; t < n_rot; ++t) {
            const int i = 6 + t;
            const uint32_t wd = pick(philox4x32_10(make_uint4(chain, pair, 0u, (uint32_t)(i >> 2)), C.seed_lo, C.seed_hi), i & 3);
            cur[7 + t] = -PV_PI + 2.f * PV_PI * u01(wd);
        }
        e_cur = thread_eval(c, w, cur, nullptr);
        for (int k = 0; k < np; ++k) best[k] = cur[k];
        e_best = e_cur;
    } else {
        for (int k = 0; k < np; ++k) { cur[k] = rec[PV_CH_CUR + k]; best[k] = rec[PV_CH_BEST + k]; }
        e_cur = rec[PV_CH_ECUR];
        e_best = rec[PV_CH_EBEST];
        ev0 = __float_as_uint(rec[PV_CH_EVALS]);
    }
    int flags = 0;
    for (int s = step0; s < step1; ++s) {
        for (int k = 0; k < np; ++k) cand[k] = cur[k];
        const uint32_t st = (uint32_t)s + 1u;
        const uint4 b0 = philox4x32_10(make_uint4(chain, pair, st, 0u), C.seed_lo, C.seed_hi);
        const uint4 b1 = philox4x32_10(make_uint4(chain, pair, st, 1u), C.seed_lo, C.seed_hi);
        const int entity = (int)__umulhi(b0.x, (uint32_t)(2 + n_rot));
        const float z = 2.f * u01(b0.y) - 1.f, r = cbrtf(u01(b0.w));
        float sp, cp;
        sincospif(2.f * u01(b0.z), &sp, &cp);
        const float sz = sqrtf(fmaxf(0.f, 1.f - z * z));
        const float3 p = make_float3(r * sz * cp, r * sz * sp, r * z);
        if (entity == 0) {
            cand[0] += C.amplitude * p.x; cand[1] += C.amplitude * p.y; cand[2] += C.amplitude * p.z;
        } else if (entity == 1) {
            const float sc = L->h.rgyr > 1e-9f ? C.amplitude / L->h.rgyr : 0.f;
            const float4 q = quat_rotate_by(make_float4(cand[3], cand[4], cand[5], cand[6]), sc * p);
            cand[3] = q.x; cand[4] = q.y; cand[5] = q.z; cand[6] = q.w;
        } else {
            cand[7 + entity - 2] = -PV_PI + 2.f * PV_PI * u01(b1.x);
        }
        const float u = u01(b1.y);
        const ThreadDockObjective obj{c, w, n_rot, 6 + n_rot, 7 + n_rot};
        const float e_new = thread_rilc_bfgs(obj, cand, C, max_iter);
        if (e_new < e_cur || u < expf((e_cur - e_new) / C.temperature)) {
            for (int k = 0; k < np; ++k) cur[k] = cand[k];
            e_cur = e_new;
            if (e_cur < e_best) {
                e_cur = thread_rilc_bfgs(obj, cur, C, max_iter);
                for (int k = 0; k < np; ++k) best[k] = cur[k];
                e_best = e_cur;
            }
        }
        if (timeout_ns && globaltimer() - *t0 > timeout_ns) { flags |= PV_EBIT_TIMEOUT; break; }
    }
    if (!(e_best == e_best)) flags |= PV_EBIT_NAN;
    for (int k = 0; k < np; ++k) { rec[PV_CH_CUR + k] = cur[k]; rec[PV_CH_BEST + k] = best[k]; }
    rec[PV_CH_ECUR] = e_cur;
    rec[PV_CH_EBEST] = e_best;
    rec[PV_CH_EVALS] = __uint_as_float(ev0 + c.evals);
    rec[PV_CH_FLAGS] = __int_as_float((step0 == 0 ? 0 : __float_as_int(rec[PV_CH_FLAGS])) | flags);
    if (flags) atomicOr(err, flags);
}

}  // namespace pv
