// pv_warp.cuh -- one warp evaluates one ligand pose: torsion-tree forward kinematics, trilinear
// e_inter, intra-ligand pair terms, and the reverse-mode gradient over the pose tangent space;
// on top of it the warp runs RILC-BFGS and the Monte-Carlo step of one chain.
//
// Lane roles
//   atoms:      lane l owns device atoms l and l + 32
//   fragments:  lane f owns rigid fragment f (f < n_frag <= 27): its world rotation M_f and
//               anchor position
//   tangent:    lane k owns tangent coordinate k (0-2 translation, 3-5 rotation vector,
//               6 + t torsion t); the torsion angle psi_t itself lives in lane 6 + t
//   pairs:      every intra pair is owned by the lane of one of its atoms (its source), which
//               adds that atom's share of the force in registers; the other atom (its target)
//               receives its share through shared memory. Rounds give each lane one pair and
//               each target one pair, so no atomics are needed and the order of accumulation
//               is fixed (bitwise reproducible).
#pragma once
#include "pv_device.cuh"

namespace pv {

struct WarpScratch {
    float4 x[64];                // posed coordinates; w = XS radius
    float4 g[64];                // dSF/dx
    float hs[PV_MAX_M][32];      // L-BFGS history: s vectors, lane = tangent coordinate
    float hy[PV_MAX_M][32];      //                 y vectors
    float cur[40];               // the chain's current POT (MC state)
};

// A pose held by a warp: translation and quaternion (w, x, y, z) are warp-uniform; psi is the
// lane's torsion in tangent layout (lane 6 + t holds psi_t, other lanes hold 0).
struct Pose {
    float3 T;
    float4 q;
    float psi;
};

struct Site {                      // where a pose is scored
    const float* maps;             // this pocket's maps (slot-major)
    const PvPocket* P;             // pocket geometry (shared or global memory)
};

__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(PV_FULL, v, src); }
__device__ __forceinline__ int shfli(int v, int src) { return __shfl_sync(PV_FULL, v, src); }

// Forward kinematics (Eq. 1: position, orientation, torsions -> atom coordinates). Writes S.x.
// Returns the fragment lane's rotation and anchor (used again by the adjoint).
__device__ __forceinline__ void warp_fk(const PvLigBlob& L, WarpScratch& S, const Pose& x,
                                        float3& axw, float3& xa, float4* own = nullptr) {
    const int lane = threadIdx.x & 31;
    const int nf = L.h.n_frag;
    const bool isf = lane < nf;
    int parent = 0, depth = 0, tor = -1;
    float3 off = make_float3(0.f, 0.f, 0.f), axis = off;
    if (isf) {
        float4 o = L.frag_off[lane], a = L.frag_axis[lane];
        off = f3(o); axis = f3(a);
        parent = __float_as_int(o.w);
        depth = __float_as_int(a.w);
        tor = L.frag_tor[lane];
    }
    float psi = shfl(x.psi, (isf && lane > 0) ? 6 + tor : lane);
    // local rotation of every fragment as a unit quaternion: the root's orientation, or a
    // torsion's half-angle quaternion (cos psi/2, sin psi/2 * axis) about its hinge axis; world
    // rotations compose down the tree level by level (Q_f = Q_parent (x) q_f)
    float s2, c2;
    sincosf(0.5f * (isf ? psi : 0.0f), &s2, &c2);
    float4 Q = lane == 0 ? quat_normalize(x.q) : make_float4(c2, s2 * axis.x, s2 * axis.y, s2 * axis.z);
    const float4 ql = Q;
    xa = (lane == 0) ? x.T : make_float3(0.f, 0.f, 0.f);
    for (int lev = 1; lev <= L.h.max_depth; ++lev) {
        const bool mine = isf && depth == lev;
        const int src = mine ? parent : lane;
        const float4 Qp = make_float4(shfl(Q.x, src), shfl(Q.y, src), shfl(Q.z, src), shfl(Q.w, src));
        const float3 xp = make_float3(shfl(xa.x, src), shfl(xa.y, src), shfl(xa.z, src));
        if (mine) {
            Q = quat_mul(Qp, ql);
            // anchor: parent's anchor + parent rotation applied to the offset, v + 2w(u x v) + 2u x (u x v)
            const float3 u = make_float3(Qp.y, Qp.z, Qp.w);
            const float3 t1 = cross3(u, off);
            const float3 t2 = cross3(u, t1);
            xa = xp + off + (2.f * Qp.x) * t1 + 2.f * t2;
        }
    }
    const Mat3 M = unit_quat_to_mat(Q.x, Q.y, Q.z, Q.w);
    const int n = L.h.n_atoms;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
        float4 loc = a < n ? L.atom[a] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int w = __float_as_int(loc.w);
        const int fa = a < n ? (w & 255) : lane;
        Mat3 Mf;
#pragma unroll
        for (int k = 0; k < 9; ++k) Mf.m[k] = shfl(M.m[k], fa);
        float3 xf = make_float3(shfl(xa.x, fa), shfl(xa.y, fa), shfl(xa.z, fa));
        if (a < n) {
            float3 p = mat_vec(Mf, f3(loc)) + xf;
            const float4 q = make_float4(p.x, p.y, p.z, xs_radius((w >> 8) & 255));
            S.x[a] = q;
            if (own) own[h] = q;
        }
    }
    axw = mat_vec(M, axis);   // the hinge axis in the world frame (rotating about it keeps it)
}

// SF = e_inter + e_intra (Eq. 3) and, if want_grad, its tangent gradient (lane k holds
// component k). parts (optional, lane-uniform): e_inter, e_intra.
static __device__ __forceinline__ float warp_eval(const PvLigBlob& L, WarpScratch& S, const Site& site,
                                               const Pose& x, float& grad, bool want_grad,
                                               float* parts = nullptr) {
    const int lane = threadIdx.x & 31;
    const int n = L.h.n_atoms;
    float3 axw, xa;
    float4 own[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    warp_fk(L, S, x, axw, xa, own);
    const PvPocket& P = *site.P;
    float e_inter = 0.f, e_intra = 0.f;
    float3 acc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
        acc[h] = make_float3(0.f, 0.f, 0.f);
        if (a < n) {
            const int w = __float_as_int(L.atom[a].w);
            const int slot = (w >> 16) & 255;
            e_inter += grid_eval(site.maps + (long long)slot * P.nxyz, P, f3(own[h]), acc[h]);
            S.g[a] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp();
    // Pair rounds. Positions and pair words are read-only here, so the next round's word and
    // partner position are loaded before the current round's force update and its __syncwarp
    // (which orders only the force scatter).
    const int rounds = L.h.n_rounds;
    if (rounds > 0) {
        uint32_t pw = L.pairs[lane];
        float4 xj = S.x[pw & 63];
        if (n <= 32) {                        // every source is the lane's first atom
            for (int r = 0; r < rounds; ++r) {
                const uint32_t pw_n = r + 1 < rounds ? L.pairs[(r + 1) * 32 + lane] : 0u;
                const float4 xj_n = S.x[pw_n & 63];
                const float3 d = make_float3(own[0].x - xj.x, own[0].y - xj.y, own[0].z - xj.z);
                const float r2 = dot3(d, d);
                const bool live = (pw >> 31) && r2 < kCutoff2;
                float c;
                const float e = vina_pair_r2(r2, own[0].w + xj.w, (float)((pw >> 16) & 1), (float)((pw >> 17) & 1), c);
                if (live) {
                    e_intra += e;
                    const float3 f = c * d;
                    acc[0] = acc[0] + f;
                    const int t = pw & 63;
                    const float4 gj = S.g[t];
                    S.g[t] = make_float4(gj.x - f.x, gj.y - f.y, gj.z - f.z, 0.f);
                }
                __syncwarp();
                pw = pw_n;
                xj = xj_n;
            }
        } else {
            for (int r = 0; r < rounds; ++r) {
                const uint32_t pw_n = r + 1 < rounds ? L.pairs[(r + 1) * 32 + lane] : 0u;
                const float4 xj_n = S.x[pw_n & 63];
                const int h = (pw >> 6) & 1;
                const float4 xi = h ? own[1] : own[0];
                const float3 d = make_float3(xi.x - xj.x, xi.y - xj.y, xi.z - xj.z);
                const float r2 = dot3(d, d);
                const bool live = (pw >> 31) && r2 < kCutoff2;
                float c;
                const float e = vina_pair_r2(r2, xi.w + xj.w, (float)((pw >> 16) & 1), (float)((pw >> 17) & 1), c);
                if (live) {
                    e_intra += e;
                    const float3 f = c * d;
                    if (h) acc[1] = acc[1] + f; else acc[0] = acc[0] + f;
                    const int t = pw & 63;
                    const float4 gj = S.g[t];
                    S.g[t] = make_float4(gj.x - f.x, gj.y - f.y, gj.z - f.z, 0.f);
                }
                __syncwarp();
                pw = pw_n;
                xj = xj_n;
            }
        }
    }
    // total dSF/dx of the lane's atoms: own share (registers) + shares received as a target
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
        if (a < n) {
            const float4 gt = S.g[a];
            acc[h] = acc[h] + f3(gt);
            S.g[a] = make_float4(acc[h].x, acc[h].y, acc[h].z, 0.f);
        }
    }
    float ei = warp_sum(e_inter), ej = warp_sum(e_intra);
    if (parts) { parts[0] = ei; parts[1] = ej; }
    if (want_grad) {
        __syncwarp();
        // root: total force and torque about the origin atom (butterfly sums over all atoms)
        float3 F = make_float3(0.f, 0.f, 0.f), tau = F;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int a = lane + 32 * h;
            if (a < n) {
                F = F + acc[h];
                tau = tau + cross3(f3(own[h]) - x.T, acc[h]);
            }
        }
        F = warp_sum3(F);
        tau = warp_sum3(tau);
        // torsions: fragment lane sums torque of its subtree (a contiguous atom range) about
        // its anchor, projected on its world hinge axis
        float gpsi = 0.f;
        const int nf = L.h.n_frag;
        if (lane > 0 && lane < nf) {
            const int a0 = L.frag_a0[lane], a1 = L.frag_a1[lane];
            float3 t = make_float3(0.f, 0.f, 0.f);
            for (int a = a0; a < a1; ++a) t = t + cross3(f3(S.x[a]) - xa, f3(S.g[a]));
            gpsi = dot3(axw, t);
        }
        const int nt = 6 + L.h.n_rot;
        const int src = (lane >= 6 && lane < nt) ? L.tor_frag[lane - 6] : lane;
        float gp = shfl(gpsi, src);
        float c3[6] = {F.x, F.y, F.z, tau.x, tau.y, tau.z};
        grad = lane < 6 ? c3[lane] : (lane < nt ? gp : 0.f);
    }
    __syncwarp();
    return ei + ej;
}

// x (+) step: translation += step[0:3]; q <- exp(step[3:6]/2) (x) q; psi += step[6:].
__device__ __forceinline__ Pose retract(const Pose& x, float step, int n_tan) {
    const int lane = threadIdx.x & 31;
    Pose y;
    y.T = x.T + make_float3(shfl(step, 0), shfl(step, 1), shfl(step, 2));
    y.q = quat_rotate_by(x.q, make_float3(shfl(step, 3), shfl(step, 4), shfl(step, 5)));
    y.psi = x.psi + ((lane >= 6 && lane < n_tan) ? step : 0.f);
    return y;
}

struct ChainCtx {
    const PvLigBlob* L;
    WarpScratch* S;
    Site site;
    uint32_t evals;
};

__device__ __forceinline__ float eval_pose(ChainCtx& c, const Pose& x, float& g) {
    c.evals++;
    return warp_eval(*c.L, *c.S, c.site, x, g, true);
}

// L-BFGS two-loop recursion (Eq. 10-11 history, newest pair first) for the direction d = -H g.
__device__ __forceinline__ float lbfgs_direction(const float* Hs, const float* Hy, float rh, float& al,
                                                 float g, int stored, int head, int m) {
    const int lane = threadIdx.x & 31;
    float q = g;
    for (int a = 0; a < stored; ++a) {
        int k = head - 1 - a;
        if (k < 0) k += m;
        const float alpha = shfl(rh, k) * warp_sum(Hs[k * 32 + lane] * q);
        if (lane == k) al = alpha;
        q -= alpha * Hy[k * 32 + lane];
    }
    if (stored > 0) {
        const int k = head == 0 ? m - 1 : head - 1;
        const float sk = Hs[k * 32 + lane], yk = Hy[k * 32 + lane];
        const float sy = warp_sum(sk * yk), yy = warp_sum(yk * yk);
        q *= sy / yy;
    }
    for (int a = stored - 1; a >= 0; --a) {
        int k = head - 1 - a;
        if (k < 0) k += m;
        const float b = shfl(rh, k) * warp_sum(Hy[k * 32 + lane] * q);
        q += Hs[k * 32 + lane] * (shfl(al, k) - b);
    }
    return -q;
}

// RILC-BFGS (Eq. 6-12): L-BFGS two-loop recursion over the m most recent curvature pairs,
// Lewis-Overton line search (Eq. 7-8 as failure tests of Armijo / weak Wolfe), curvature-
// guarded history update (Eq. 11), stop on ||g|| <= eps (Eq. 12), non-descent, or max_iter.
// Updates x in place and returns SF(x). All control flow is warp-uniform. The history lives in
// the warp's shared scratch (a ring of m slots); rho and alpha of slot k sit in lane k.
// Written as one loop with a single evaluation site (the start point, then every line-search
// trial), so the evaluator's code appears once.
__device__ __forceinline__ float warp_bfgs(ChainCtx& c, Pose& x, const PvSearchConst& C, int max_iter, int m) {
    const int lane = threadIdx.x & 31;
    const int n_tan = 6 + c.L->h.n_rot;
    float* Hs = &c.S->hs[0][0];
    float* Hy = &c.S->hy[0][0];
    float rh = 0.f, al = 0.f;
    int stored = 0, head = 0, it = 0, tr = 0;
    float f = 0.f, g = 0.f, d = 0.f, gd = 0.f;
    float lam = 1.f, lo = 0.f, hi = -1.f, flo = 0.f, glo = 0.f;
    bool have_lo = false, start = true;
    Pose xt = x;
    for (;;) {
        float ge;
        const float fe = eval_pose(c, xt, ge);
        bool next_iter = false, done = false;
        if (start) {                        // the start point: f, g at x
            start = false;
            f = fe;
            g = ge;
            next_iter = true;
        } else {                            // a line-search trial at x + lam d
            const float gtd = warp_sum(ge * d);
            bool take = false;
            float ft = fe, gt = ge;
            if (!(fe <= f + lam * C.rho * gd)) {
                hi = lam;                                   // Eq. 7 holds: Armijo fails
            } else if (gtd < C.sigma * gd) {
                lo = lam; have_lo = true; flo = fe; glo = ge;   // Eq. 8 holds: Wolfe fails
            } else {
                take = true;
            }
            if (!take) {
                ++tr;
                if (tr < C.bfgs_max_trials) {
                    lam = hi < 0.f ? 2.f * lam : 0.5f * (lo + hi);
                    xt = retract(x, lam * d, n_tan);
                    continue;
                }
                if (!have_lo) break;                        // no acceptable step: stop here
                lam = lo; ft = flo; gt = glo;
                xt = retract(x, lam * d, n_tan);            // the same arithmetic as that trial
                take = true;
            }
            // accepted step: curvature-guarded history update, move, convergence test
            const float s = lam * d, y = gt - g;
            const float ys = warp_sum(y * s), ss = warp_sum(s * s), gn = sqrtf(warp_sum(g * g));
            if (ss > 0.f && ys / ss > C.eps * gn) {
                Hs[head * 32 + lane] = s;
                Hy[head * 32 + lane] = y;
                if (lane == head) rh = 1.f / ys;
                head = head + 1 == m ? 0 : head + 1;
                stored = min(stored + 1, m);
            }
            x = xt; g = gt; f = ft;
            ++it;
            if (sqrtf(warp_sum(g * g)) <= C.eps) done = true;
            next_iter = !done;
        }
        if (done) break;
        if (next_iter) {
            if (it >= max_iter) break;
            d = lbfgs_direction(Hs, Hy, rh, al, g, stored, head, m);
            gd = warp_sum(g * d);
            if (!(gd < 0.f)) break;
            lam = 1.f; lo = 0.f; hi = -1.f; have_lo = false; tr = 0;
            xt = retract(x, lam * d, n_tan);
        }
    }
    __syncwarp();
    return f;
}

// Random conformation (Algorithm 2): draws 0-2 translation uniform in the box, 3-5 a uniform
// quaternion (Shoemake), 6 + t torsion t uniform in [-pi, pi).
__device__ __forceinline__ Pose random_pose(const PvLigBlob& L, const PvPocket& P, uint32_t chain,
                                            uint32_t pair, const PvSearchConst& C) {
    const int lane = threadIdx.x & 31;
    uint4 b0 = philox4x32_10(make_uint4(chain, pair, 0u, 0u), C.seed_lo, C.seed_hi);
    uint4 b1 = philox4x32_10(make_uint4(chain, pair, 0u, 1u), C.seed_lo, C.seed_hi);
    Pose x;
    x.T = make_float3(P.center[0] + (u01(b0.x) - 0.5f) * P.size[0],
                      P.center[1] + (u01(b0.y) - 0.5f) * P.size[1],
                      P.center[2] + (u01(b0.z) - 0.5f) * P.size[2]);
    float u1 = u01(b0.w), u2 = u01(b1.x), u3 = u01(b1.y);
    float s2, c2, s3, c3;
    sincospif(2.f * u2, &s2, &c2);
    sincospif(2.f * u3, &s3, &c3);
    float a = sqrtf(1.f - u1), b = sqrtf(u1);
    x.q = make_float4(a * s2, a * c2, b * s3, b * c3);
    x.psi = 0.f;
    if (lane >= 6 && lane < 6 + L.h.n_rot) {
        const int i = lane;   // draw index 6 + t with t = lane - 6
        uint32_t w = pick(philox4x32_10(make_uint4(chain, pair, 0u, (uint32_t)(i >> 2)), C.seed_lo, C.seed_hi), i & 3);
        x.psi = -PV_PI + 2.f * PV_PI * u01(w);
    }
    return x;
}

// Mutation R (Eq. 2) of MC step `step`: word 0 picks one entity among {position, orientation,
// psi_1..psi_Nrot} as floor(w * (2 + N_rot) / 2^32); draws 1-3 give a point p in the unit
// ball (z = 2a - 1, phi = 2 pi b, r = cbrt(c)); position += amplitude p, or orientation
// rotated by (amplitude / R_gyr) p, or the torsion redrawn from draw 4. Returns draw 5
// (the Metropolis uniform).
__device__ __forceinline__ float mutate(const PvLigBlob& L, Pose& x, uint32_t chain, uint32_t pair,
                                        int step, const PvSearchConst& C) {
    const int lane = threadIdx.x & 31;
    const uint32_t st = (uint32_t)step + 1u;
    uint4 b0 = philox4x32_10(make_uint4(chain, pair, st, 0u), C.seed_lo, C.seed_hi);
    uint4 b1 = philox4x32_10(make_uint4(chain, pair, st, 1u), C.seed_lo, C.seed_hi);
    const int n_rot = L.h.n_rot;
    const int entity = (int)__umulhi(b0.x, (uint32_t)(2 + n_rot));
    float z = 2.f * u01(b0.y) - 1.f, r = cbrtf(u01(b0.w));
    float sp, cp;
    sincospif(2.f * u01(b0.z), &sp, &cp);
    float s = sqrtf(fmaxf(0.f, 1.f - z * z));
    float3 p = make_float3(r * s * cp, r * s * sp, r * z);
    if (entity == 0) {
        x.T = x.T + C.amplitude * p;
    } else if (entity == 1) {
        float sc = L.h.rgyr > 1e-9f ? C.amplitude / L.h.rgyr : 0.f;
        x.q = quat_rotate_by(x.q, sc * p);
    } else if (lane == 6 + (entity - 2)) {
        x.psi = -PV_PI + 2.f * PV_PI * u01(b1.x);
    }
    return u01(b1.y);
}

}  // namespace pv
