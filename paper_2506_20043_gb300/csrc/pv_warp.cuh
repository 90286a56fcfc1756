// pv_warp.cuh -- one team of lanes (a whole warp, or half a warp) evaluates one ligand pose:
// torsion-tree forward kinematics, trilinear e_inter, intra-ligand pair terms and the reverse-mode
// gradient over the pose tangent space; it also holds the team's pose arithmetic (retraction,
// L-BFGS direction, random start, mutation) used by the chain runner in pv_search.cu.
//
// Lane roles inside a team of LANES lanes (tl = lane within the team)
//   atoms:      lane tl owns atoms tl and tl + LANES (device order)
//   fragments:  lane tl owns rigid fragment tl (n_frag <= LANES): its world rotation and anchor
//   tangent:    lane k owns tangent coordinate k (0-2 translation, 3-5 rotation vector,
//               6 + t torsion t); the torsion angle psi_t itself lives in lane 6 + t
//   pairs:      every intra pair is computed by the lane of one of its atoms (its source), which
//               adds that atom's share of the force in registers; the other atom's lane (its
//               target's) receives the opposite force by a shuffle. Rounds give each lane at most
//               one pair to send and one to receive, so forces never leave registers and the
//               order of accumulation is fixed (bitwise reproducible).
// Half-warp teams (LANES = 16) serve ligands of at most 32 atoms and 10 torsions: two chains share
// a warp and stay converged at the evaluator (one evaluation per loop iteration).
#pragma once
#include "pv_device.cuh"

namespace pv {

// Team-uniform scalars of a chain's MC step and of its line search, kept in shared memory rather
// than registers: they are used between evaluations only, and every evaluation ends with a team
// barrier, so registers holding them across it would only lower the kernel's occupancy.
struct ChainScalars {
    float e_cur, e_best, u, f, gd, lam, lo, hi, flo;
    int s, stage, flags, nb_n, nb_head, it, tr, stored, head, have_lo;
    uint32_t evals_before;
};

struct WarpScratch {            // one per team
    float4 x[64 + PV_N_DUMMY];  // posed coordinates, w = XS radius; [64 + k] the far dummy atoms
                                // that empty pair slots point to (init_scratch)
    union {                     // one lives after the other within an evaluation (synced between):
        float4 fm[3 * PV_MAX_FRAGS];  // during the kinematics: per fragment, its world rotation rows
                                      // (xyz) with the anchor (w)
        float4 g[64];                 // after the pair rounds: dSF/dx of every atom, until the next
                                      // evaluation's kinematics
    };
    float hs[PV_MAX_M][32];     // L-BFGS history: s vectors, lane = tangent coordinate
    float hy[PV_MAX_M][32];     //                 y vectors
    float cur[40];              // the chain's current POT (MC state)
    float glo[32];              // line search: gradient at the largest Armijo-satisfying trial
    float lg[32];               // line search: the lane's gradient component and search
    float ld[32];               //              direction component (lane-private)
    float lr[32];               // L-BFGS: 1 / (y.s) of history entry `lane` (lane-private)
    float4 xb_tq[2];            // line search: its base point (translation, orientation; torsions
    float xb_psi[32];           //              per lane), kept here across evaluations
    ChainScalars cs;
};

template <int LANES>
struct Team {
    static __device__ __forceinline__ int lane() { return threadIdx.x & (LANES - 1); }
    static __device__ __forceinline__ int index() { return (threadIdx.x & 31) / LANES; }
    static __device__ __forceinline__ unsigned mask() {
        return LANES == 32 ? PV_FULL : (0xffffu << (16 * ((threadIdx.x & 31) >> 4)));
    }
    static __device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(mask(), v, src, LANES); }
    static __device__ __forceinline__ float sum(float v) {
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask(), v, o, LANES);
        return v;
    }
    static __device__ __forceinline__ float3 sum3(float3 v) {
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) {
            v.x += __shfl_xor_sync(mask(), v.x, o, LANES);
            v.y += __shfl_xor_sync(mask(), v.y, o, LANES);
            v.z += __shfl_xor_sync(mask(), v.z, o, LANES);
        }
        return v;
    }
    static __device__ __forceinline__ float3 shfl3(float3 v, int src) {
        return make_float3(shfl(v.x, src), shfl(v.y, src), shfl(v.z, src));
    }
    static __device__ __forceinline__ float3 xor3(float3 v, int o) {
        return make_float3(__shfl_xor_sync(mask(), v.x, o, LANES), __shfl_xor_sync(mask(), v.y, o, LANES),
                           __shfl_xor_sync(mask(), v.z, o, LANES));
    }
    static __device__ __forceinline__ void sync() { __syncwarp(mask()); }
};

// A pose held by a team: translation and quaternion (w, x, y, z) are team-uniform; psi is the
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

// Places the far dummy atoms of a team's scratch (once per kernel, before its first evaluation):
// empty pair slots point to them (each to one in a shared-memory bank group that the other partners
// of its quarter-warp leave free), and their distance to any atom is far beyond the cutoff.
template <int LANES>
__device__ __forceinline__ void init_scratch(WarpScratch& S) {
    const int tl = threadIdx.x & (LANES - 1);
    if (tl < PV_N_DUMMY) S.x[PV_DUMMY_ATOM + tl] = make_float4(1e15f, 1e15f, 1e15f, 0.f);
    __syncwarp();
}

// Pair slots of the team width's schedule.
template <int LANES>
__device__ __forceinline__ const PvPairSlot* pair_rounds(const PvLigBlob& L, int& rounds) {
    if (LANES == 32) {
        rounds = L.h.n_rounds;
        return L.pairs;
    }
    rounds = L.h.n_rounds16;
    return L.pairs + L.h.pairs16_at;
}

// Forward kinematics (Eq. 1: position, orientation, torsions -> atom coordinates). Writes S.x.
// Returns the fragment lane's world hinge axis and anchor (used again by the adjoint) and the
// lane's own atoms' positions.
template <int LANES>
__device__ __forceinline__ void team_fk(const PvLigBlob& L, WarpScratch& S, const Pose& x,
                                        float3& axw, float3& xa, float4* own = nullptr) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    const int nf = L.h.n_frag;
    const bool isf = tl < nf;
    int parent = 0, depth = 0, tor = -1;
    float3 off = make_float3(0.f, 0.f, 0.f), axis = off;
    if (isf) {
        float4 o = L.frag_off[tl], a = L.frag_axis[tl];
        off = f3(o); axis = f3(a);
        parent = __float_as_int(o.w);
        depth = __float_as_int(a.w);
        tor = L.frag_tor[tl];
    }
    float psi = Tm::shfl(x.psi, (isf && tl > 0) ? 6 + tor : tl);
    // local rotation of every fragment as a unit quaternion: the root's orientation, or a
    // torsion's half-angle quaternion (cos psi/2, sin psi/2 * axis) about its hinge axis; world
    // rotations compose down the tree level by level (Q_f = Q_parent (x) q_f)
    float s2, c2;
    sincosf(wrap_pi(0.5f * (isf ? psi : 0.0f)), &s2, &c2);
    float4 Q = tl == 0 ? quat_normalize(x.q) : make_float4(c2, s2 * axis.x, s2 * axis.y, s2 * axis.z);
    const float4 ql = Q;
    xa = (tl == 0) ? x.T : make_float3(0.f, 0.f, 0.f);
    for (int lev = 1; lev <= L.h.max_depth; ++lev) {
        const bool mine = isf && depth == lev;
        const int src = mine ? parent : tl;
        const float4 Qp = make_float4(Tm::shfl(Q.x, src), Tm::shfl(Q.y, src), Tm::shfl(Q.z, src), Tm::shfl(Q.w, src));
        const float3 xp = make_float3(Tm::shfl(xa.x, src), Tm::shfl(xa.y, src), Tm::shfl(xa.z, src));
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
    // each fragment's rotation rows and anchor go through shared memory once; an atom then reads
    // its fragment's three rows as 16-byte words
    if (isf) {
        S.fm[3 * tl + 0] = make_float4(M.m[0], M.m[1], M.m[2], xa.x);
        S.fm[3 * tl + 1] = make_float4(M.m[3], M.m[4], M.m[5], xa.y);
        S.fm[3 * tl + 2] = make_float4(M.m[6], M.m[7], M.m[8], xa.z);
    }
    Tm::sync();
    const int n = L.h.n_atoms;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && n <= LANES) break;
        const int a = tl + LANES * h;
        if (a < n) {
            const float4 loc = L.atom[a];
            const int w = __float_as_int(loc.w);
            const int fa = w & 255;
            const float4 r0 = S.fm[3 * fa], r1 = S.fm[3 * fa + 1], r2 = S.fm[3 * fa + 2];
            const float3 p = make_float3(r0.x * loc.x + r0.y * loc.y + r0.z * loc.z,
                                         r1.x * loc.x + r1.y * loc.y + r1.z * loc.z,
                                         r2.x * loc.x + r2.y * loc.y + r2.z * loc.z) +
                             make_float3(r0.w, r1.w, r2.w);
            const float4 q = make_float4(p.x, p.y, p.z, xs_radius((w >> 8) & 255));
            S.x[a] = q;
            if (own) own[h] = q;
        }
    }
    axw = mat_vec(M, axis);   // the hinge axis in the world frame (rotating about it keeps it)
}

// The lane's pairs of two rounds (slots pa, pb; source atoms xia, xib; partners xa, xb), their
// arithmetic two pairs per instruction (packed FP32x2 adds, multiplies and FMAs; the reciprocal
// square roots and exponentials one pair at a time): adds both energies to e_intra and returns the
// forces on the sources in fa, fb. Per pair the same terms as pair_force.
__device__ __forceinline__ void pair_force2(const PvPairSlot& pa, const PvPairSlot& pb, const float4& xia,
                                            const float4& xib, const float4& xa, const float4& xb, float& e_intra,
                                            float3& fa, float3& fb) {
    const float2 dx = __fadd2_rn(make_float2(xia.x, xib.x), make_float2(-xa.x, -xb.x));
    const float2 dy = __fadd2_rn(make_float2(xia.y, xib.y), make_float2(-xa.y, -xb.y));
    const float2 dz = __fadd2_rn(make_float2(xia.z, xib.z), make_float2(-xa.z, -xb.z));
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const float2 rinv = make_float2(rsqrtf(fmaxf(r2.x, 1e-12f)), rsqrtf(fmaxf(r2.y, 1e-12f)));
    const float2 r = __fmul2_rn(r2, rinv);
    const float2 d = __fadd2_rn(r, make_float2(-(xia.w + xa.w), -(xib.w + xb.w)));   // surface distance
    const float2 a1 = __fmul2_rn(__fmul2_rn(d, d), make_float2(-4.0f * kLog2e, -4.0f * kLog2e));
    const float2 b = __fadd2_rn(d, make_float2(-3.0f, -3.0f));
    const float2 a2 = __fmul2_rn(__fmul2_rn(b, b), make_float2(-0.25f * kLog2e, -0.25f * kLog2e));
    const float2 g1 = make_float2(exp2_approx(a1.x), exp2_approx(a1.y));   // exp(-(d / 0.5)^2)
    const float2 g2 = make_float2(exp2_approx(a2.x), exp2_approx(a2.y));   // exp(-((d - 3) / 2)^2)
    const float2 rep = make_float2(fminf(d.x, 0.f), fminf(d.y, 0.f));
    const float2 c1 = make_float2(pa.c1, pb.c1), w = make_float2(pa.w, pb.w);
    const float2 t = __ffma2_rn(c1, d, make_float2(pa.c0, pb.c0));        // the ramp w sat(c0 + c1 d)
    const float2 v = make_float2(__saturatef(t.x), __saturatef(t.y));
    const float2 dv = make_float2((t.x > 0.0f && t.x <= 1.0f) ? c1.x : 0.0f, (t.y > 0.0f && t.y <= 1.0f) ? c1.y : 0.0f);
    float2 e = __fmul2_rn(make_float2(kWGauss1, kWGauss1), g1);
    e = __ffma2_rn(make_float2(kWGauss2, kWGauss2), g2, e);
    e = __ffma2_rn(__fmul2_rn(make_float2(kWRepulsion, kWRepulsion), rep), rep, e);
    e = __ffma2_rn(w, v, e);
    float2 de = __fmul2_rn(__fmul2_rn(make_float2(-8.0f * kWGauss1, -8.0f * kWGauss1), d), g1);
    de = __ffma2_rn(__fmul2_rn(make_float2(-0.5f * kWGauss2, -0.5f * kWGauss2), b), g2, de);
    de = __ffma2_rn(make_float2(2.0f * kWRepulsion, 2.0f * kWRepulsion), rep, de);
    de = __ffma2_rn(w, dv, de);
    const bool la = r2.x < kCutoff2, lb = r2.y < kCutoff2;
    e_intra += (la ? e.x : 0.f) + (lb ? e.y : 0.f);
    const float2 c = __fmul2_rn(make_float2(la ? de.x : 0.f, lb ? de.y : 0.f), rinv);   // dE/dr / r
    const float2 fx = __fmul2_rn(c, dx), fy = __fmul2_rn(c, dy), fz = __fmul2_rn(c, dz);
    fa = make_float3(fx.x, fy.x, fz.x);
    fb = make_float3(fx.y, fy.y, fz.y);
}

// The lane's pair of one round (source atom xi, partner position xj, the slot's ramp constants):
// its energy and the force on the source, which the target's lane receives with the opposite
// sign. An empty slot's partner is the far dummy atom: beyond the cutoff, it adds nothing.
__device__ __forceinline__ float3 pair_force(const PvPairSlot& ps, const float4& xi, const float4& xj,
                                             float& e_intra) {
    const float3 d = make_float3(xi.x - xj.x, xi.y - xj.y, xi.z - xj.z);
    const float r2 = dot3(d, d);
    const bool live = r2 < kCutoff2;
    float c;
    const float e = vina_pair_ramp(r2, xi.w + xj.w, ps.c0, ps.c1, ps.w, c);
    e_intra += live ? e : 0.f;
    c = live ? c : 0.f;
    return c * d;
}

// SF = e_inter + e_intra (Eq. 3) and, if want_grad, its tangent gradient (lane k holds
// component k). parts (optional, lane-uniform): e_inter, e_intra. On return S.g holds dSF/dx of
// every atom (device order). FK = false: the atoms are already posed in S.x (device order, w = XS
// radius, written and synced by the caller), x is not used and there is no tangent gradient.
template <int LANES, bool FK = true, int LAYOUT = 0>
__device__ __forceinline__ float team_eval(const PvLigBlob& L, WarpScratch& S, const Site& site,
                                           const Pose& x, float& grad, bool want_grad,
                                           float* parts = nullptr) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    const int n = L.h.n_atoms;
    float3 axw = make_float3(0.f, 0.f, 0.f), xa = axw;
    float4 own[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    if constexpr (FK) {
        team_fk<LANES>(L, S, x, axw, xa, own);
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (tl + LANES * h < n) own[h] = S.x[tl + LANES * h];
        want_grad = false;
    }
    const PvPocket& P = *site.P;
    float e_inter = 0.f, e_intra = 0.f;
    float3 acc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = tl + LANES * h;
        acc[h] = make_float3(0.f, 0.f, 0.f);
        if (a < n) {
            const int w = __float_as_int(L.atom[a].w);
            const int slot = (w >> 16) & 255;
            e_inter += grid_eval_slot<LAYOUT>(P, slot, f3(own[h]), acc[h]);
        }
    }
    Tm::sync();
    // Pair rounds, two per step with packed arithmetic. Each lane computes the pair it sends (its
    // atom is the source) and takes the opposite force of the pair it receives from the sending lane
    // by a shuffle, so forces stay in registers and rounds need no barrier.
    int rounds;
    const PvPairSlot* pr = pair_rounds<LANES>(L, rounds);
    if (n <= LANES) {                         // every atom of a pair is its lane's first
        int r = 0;
        for (; r + 1 < rounds; r += 2) {
            const PvPairSlot pa = pr[r * LANES + tl], pb = pr[(r + 1) * LANES + tl];
            const float4 xa = S.x[pa.meta & 127], xb = S.x[pb.meta & 127];
            float3 fa, fb;
            pair_force2(pa, pb, own[0], own[0], xa, xb, e_intra, fa, fb);
            const float3 fia = Tm::shfl3(fa, (pa.meta >> 8) & (LANES - 1));
            const float3 fib = Tm::shfl3(fb, (pb.meta >> 8) & (LANES - 1));
            acc[0] = acc[0] + fa + fb;
            if ((pa.meta >> 13) & 1) acc[0] = acc[0] - fia;
            if ((pb.meta >> 13) & 1) acc[0] = acc[0] - fib;
        }
        if (r < rounds) {
            const PvPairSlot pa = pr[r * LANES + tl];
            const float3 fa = pair_force(pa, own[0], S.x[pa.meta & 127], e_intra);
            const float3 fia = Tm::shfl3(fa, (pa.meta >> 8) & (LANES - 1));
            acc[0] = acc[0] + fa;
            if ((pa.meta >> 13) & 1) acc[0] = acc[0] - fia;
        }
    } else {
        // two atoms per lane: meta bit 7 says the pair's own atom is the lane's second, bit 14 that
        // the received pair's atom is
        int r = 0;
        for (; r + 1 < rounds; r += 2) {
            const PvPairSlot pa = pr[r * LANES + tl], pb = pr[(r + 1) * LANES + tl];
            const float4 xa = S.x[pa.meta & 127], xb = S.x[pb.meta & 127];
            const bool sa = (pa.meta >> 7) & 1, sb = (pb.meta >> 7) & 1;
            float3 fa, fb;
            pair_force2(pa, pb, sa ? own[1] : own[0], sb ? own[1] : own[0], xa, xb, e_intra, fa, fb);
            const float3 fia = Tm::shfl3(fa, (pa.meta >> 8) & (LANES - 1));
            const float3 fib = Tm::shfl3(fb, (pb.meta >> 8) & (LANES - 1));
            if (sa) acc[1] = acc[1] + fa;
            else acc[0] = acc[0] + fa;
            if (sb) acc[1] = acc[1] + fb;
            else acc[0] = acc[0] + fb;
            if ((pa.meta >> 13) & 1) {
                if ((pa.meta >> 14) & 1) acc[1] = acc[1] - fia;
                else acc[0] = acc[0] - fia;
            }
            if ((pb.meta >> 13) & 1) {
                if ((pb.meta >> 14) & 1) acc[1] = acc[1] - fib;
                else acc[0] = acc[0] - fib;
            }
        }
        if (r < rounds) {
            const PvPairSlot pa = pr[r * LANES + tl];
            const bool sa = (pa.meta >> 7) & 1;
            const float3 fa = pair_force(pa, sa ? own[1] : own[0], S.x[pa.meta & 127], e_intra);
            const float3 fia = Tm::shfl3(fa, (pa.meta >> 8) & (LANES - 1));
            if (sa) acc[1] = acc[1] + fa;
            else acc[0] = acc[0] + fa;
            if ((pa.meta >> 13) & 1) {
                if ((pa.meta >> 14) & 1) acc[1] = acc[1] - fia;
                else acc[0] = acc[0] - fia;
            }
        }
    }
    // total dSF/dx of the lane's atoms, kept in shared memory for the torque sums
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = tl + LANES * h;
        if (a < n) S.g[a] = make_float4(acc[h].x, acc[h].y, acc[h].z, 0.f);
    }
    float ei, ej;
    if (parts) {
        ei = Tm::sum(e_inter);
        ej = Tm::sum(e_intra);
        parts[0] = ei;
        parts[1] = ej;
    } else {
        ei = Tm::sum(e_inter + e_intra);
        ej = 0.f;
    }
    if (want_grad) {
        Tm::sync();
        // root: total force and torque about the origin atom (butterfly sums over all atoms)
        float3 F = make_float3(0.f, 0.f, 0.f), tau = F;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int a = tl + LANES * h;
            if (a < n) {
                F = F + acc[h];
                tau = tau + cross3(f3(own[h]) - x.T, acc[h]);
            }
        }
        F = Tm::sum3(F);
        tau = Tm::sum3(tau);
        // torsions: the torque of each fragment's subtree (a contiguous atom range) about its
        // anchor, on its world hinge axis. k lanes share a fragment (k the largest power of two
        // with k * n_frag <= LANES), each summing every k-th atom of the range, then a butterfly
        // within the group; fragment f's anchor and axis come from lane f.
        const int nf = L.h.n_frag;
        int k = LANES;
        while (k * nf > LANES) k >>= 1;
        const int f = tl / k, sub = tl & (k - 1);
        const float3 xa_f = Tm::shfl3(xa, f < nf ? f : 0), ax_f = Tm::shfl3(axw, f < nf ? f : 0);
        float3 t = make_float3(0.f, 0.f, 0.f);
        if (f > 0 && f < nf) {
            const int a0 = L.frag_a0[f], a1 = L.frag_a1[f];
            for (int a = a0 + sub; a < a1; a += k) t = t + cross3(f3(S.x[a]) - xa_f, f3(S.g[a]));
        }
        for (int o = 1; o < k; o <<= 1) t = t + Tm::xor3(t, o);
        const float gpsi = dot3(ax_f, t);
        const int nt = 6 + L.h.n_rot;
        const int src = (tl >= 6 && tl < nt) ? L.tor_frag[tl - 6] * k : tl;
        float gp = Tm::shfl(gpsi, src);
        // lane k takes component k (a select chain: an array indexed by the lane would live in local memory)
        const float rt = tl == 0 ? F.x : (tl == 1 ? F.y : (tl == 2 ? F.z : (tl == 3 ? tau.x : (tl == 4 ? tau.y : tau.z))));
        grad = tl < 6 ? rt : (tl < nt ? gp : 0.f);
    }
    Tm::sync();
    return ei + ej;
}

// x (+) step: translation += step[0:3]; q <- exp(step[3:6]/2) (x) q; psi += step[6:].
template <int LANES>
__device__ __forceinline__ Pose team_retract(const Pose& x, float step, int n_tan) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    Pose y;
    y.T = x.T + make_float3(Tm::shfl(step, 0), Tm::shfl(step, 1), Tm::shfl(step, 2));
    y.q = quat_rotate_by(x.q, make_float3(Tm::shfl(step, 3), Tm::shfl(step, 4), Tm::shfl(step, 5)));
    y.psi = x.psi + ((tl >= 6 && tl < n_tan) ? step : 0.f);
    return y;
}

// L-BFGS two-loop recursion (Eq. 10-11 history, newest pair first) for the direction d = -H g.
template <int LANES>
__device__ __forceinline__ float lbfgs_direction(const float* Hs, const float* Hy, float rh, float& al,
                                                 float g, int stored, int head, int m) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    float q = g;
    for (int a = 0; a < stored; ++a) {
        int k = head - 1 - a;
        if (k < 0) k += m;
        const float alpha = Tm::shfl(rh, k) * Tm::sum(Hs[k * 32 + tl] * q);
        if (tl == k) al = alpha;
        q -= alpha * Hy[k * 32 + tl];
    }
    if (stored > 0) {
        const int k = head == 0 ? m - 1 : head - 1;
        const float sk = Hs[k * 32 + tl], yk = Hy[k * 32 + tl];
        const float sy = Tm::sum(sk * yk), yy = Tm::sum(yk * yk);
        q *= sy / yy;
    }
    for (int a = stored - 1; a >= 0; --a) {
        int k = head - 1 - a;
        if (k < 0) k += m;
        const float b = Tm::shfl(rh, k) * Tm::sum(Hy[k * 32 + tl] * q);
        q += Hs[k * 32 + tl] * (Tm::shfl(al, k) - b);
    }
    return -q;
}

// Random conformation (Algorithm 2): draws 0-2 translation uniform in the box, 3-5 a uniform
// quaternion (Shoemake), 6 + t torsion t uniform in [-pi, pi).
template <int LANES>
__device__ __forceinline__ Pose random_pose(const PvLigBlob& L, const PvPocket& P, uint32_t chain,
                                            uint32_t pair, const PvSearchConst& C) {
    const int tl = Team<LANES>::lane();
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
    if (tl >= 6 && tl < 6 + L.h.n_rot) {
        const int i = tl;   // draw index 6 + t with t = tl - 6
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
template <int LANES>
__device__ __forceinline__ float mutate(const PvLigBlob& L, Pose& x, uint32_t chain, uint32_t pair,
                                        int step, const PvSearchConst& C) {
    const int tl = Team<LANES>::lane();
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
    } else if (tl == 6 + (entity - 2)) {
        x.psi = -PV_PI + 2.f * PV_PI * u01(b1.x);
    }
    return u01(b1.y);
}

// POT record <-> team pose: lanes 0-6 hold (x, y, z, qw, qx, qy, qz), lane 6 + t holds psi_t.
template <int LANES>
__device__ __forceinline__ void store_pose(float* dst, const Pose& x, int n_rot) {
    const int tl = Team<LANES>::lane();
    const float v = tl == 0 ? x.T.x : (tl == 1 ? x.T.y : (tl == 2 ? x.T.z : (tl == 3 ? x.q.x : (tl == 4 ? x.q.y :
                    (tl == 5 ? x.q.z : x.q.w)))));
    if (tl < 7) dst[tl] = v;
    if (tl >= 6 && tl < 6 + n_rot) dst[tl + 1] = x.psi;
}
template <int LANES>
__device__ __forceinline__ Pose load_pose(const float* src, int n_rot) {
    const int tl = Team<LANES>::lane();
    Pose x;
    x.T = make_float3(src[0], src[1], src[2]);
    x.q = make_float4(src[3], src[4], src[5], src[6]);
    x.psi = (tl >= 6 && tl < 6 + n_rot) ? src[tl + 1] : 0.f;
    return x;
}

// ---- first-order consistency check (Eq. 4-5) ----
// The lane's tangent coordinate p of x - nb (nb a POT in memory): translation difference, the
// rotation vector w with q_x = exp(w / 2) (x) q_nb (shortest; both normalised), torsion difference
// wrapped into [-pi, pi); 0 for lanes past the tangent coordinates.
template <int LANES>
__device__ __forceinline__ float tangent_delta(const Pose& x, const float* nb, int n_tan) {
    const int tl = Team<LANES>::lane();
    if (tl < 3) return (tl == 0 ? x.T.x : (tl == 1 ? x.T.y : x.T.z)) - __ldcg(nb + tl);
    if (tl < 6) {
        const float4 a = quat_normalize(x.q);
        const float4 b = quat_normalize(make_float4(__ldcg(nb + 3), -__ldcg(nb + 4), -__ldcg(nb + 5),
                                                    -__ldcg(nb + 6)));                 // conjugate
        float4 r = quat_mul(a, b);
        if (r.x < 0.f) r = make_float4(-r.x, -r.y, -r.z, -r.w);
        const float vn = sqrtf(r.y * r.y + r.z * r.z + r.w * r.w);
        const float scale = vn > 1e-7f ? 2.f * atan2f(vn, r.x) / vn : 2.f;
        return scale * (tl == 3 ? r.y : (tl == 4 ? r.z : r.w));
    }
    if (tl < n_tan) {
        const float d = x.psi - __ldcg(nb + tl + 1);
        return d - 2.f * PV_PI * floorf((d + PV_PI) / (2.f * PV_PI));
    }
    return 0.f;
}

__device__ __forceinline__ int sgnf(float v) { return (v > 0.f) - (v < 0.f); }

// Whether candidate x (SF f, lane gradient g) passes the check against the n neighbours of a
// chain's ring (read past L1: another SM may have written it in the previous step block): every neighbour must show, along some tangent coordinate where the two differ by
// more than min_delta, a derivative sign change (Eq. 4) or a secant slope whose sign disagrees with
// the derivative at x (Eq. 5). Team-uniform result.
template <int LANES>
__device__ __forceinline__ bool focc_pass(const Pose& x, float f, float g, const float* ring, int n, int n_rot,
                                          float min_delta) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane(), n_tan = 6 + n_rot;
    for (int j = 0; j < n; ++j) {
        const float* nb = ring + PV_RING_POT + 40 * j;
        const float dl = tangent_delta<LANES>(x, nb, n_tan);
        bool ev = false;
        if (tl < n_tan && fabsf(dl) > min_delta) {
            const int gi = sgnf(g), gj = sgnf(__ldcg(ring + PV_RING_G + 32 * j + tl));
            ev = gi * gj <= 0 || gi * sgnf((f - __ldcg(ring + PV_RING_F + j)) * dl) <= 0;
        }
        if (!__any_sync(Tm::mask(), ev)) return false;
    }
    return true;
}

// Appends (x, f, g) to the chain's ring of the last `cap` current conformations.
template <int LANES>
__device__ __forceinline__ void focc_push(float* ring, const Pose& x, float f, float g, int n_rot, int cap,
                                          int& n, int& head) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    Tm::sync();
    store_pose<LANES>(ring + PV_RING_POT + 40 * head, x, n_rot);
    if (tl < 6 + n_rot) ring[PV_RING_G + 32 * head + tl] = g;
    if (tl == 0) ring[PV_RING_F + head] = f;
    head = head + 1 == cap ? 0 : head + 1;
    n = min(n + 1, cap);
    Tm::sync();
}

// Whole-warp names used by the selection and scoring kernels (LAYOUT: the maps read, 0 plain, 1
// cell-packed; the same corners and arithmetic either way).
template <int LAYOUT = 0>
static __device__ __forceinline__ float warp_eval(const PvLigBlob& L, WarpScratch& S, const Site& site,
                                                  const Pose& x, float& grad, bool want_grad,
                                                  float* parts = nullptr) {
    return team_eval<32, true, LAYOUT>(L, S, site, x, grad, want_grad, parts);
}
__device__ __forceinline__ void warp_fk(const PvLigBlob& L, WarpScratch& S, const Pose& x, float3& axw, float3& xa) {
    team_fk<32>(L, S, x, axw, xa);
}
__device__ __forceinline__ float shfl(float v, int src) { return __shfl_sync(PV_FULL, v, src); }

}  // namespace pv
