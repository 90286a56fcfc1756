// pv_device.cuh -- device primitives of the docking path: Vina terms, Philox4x32-10, quaternion
// algebra, trilinear grid lookup, warp reductions. Header-only, included by the kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>
#include "pv_layout.h"
#include "pv_terms.h"

#define PV_FULL 0xffffffffu
#define PV_PI 3.14159265358979323846f

namespace pv {

// ------------------------------------------------------------------------------------------
// AutoDock Vina scoring terms (Trott & Olson 2010; the scoring function the paper's engine
// evaluates, Eq. 3). Surface distance d = r - R_i - R_j, cutoff r < 8 A.
// ------------------------------------------------------------------------------------------
// (weights, cutoff and ramp ends in pv_terms.h)
constexpr float kOutSlope = 10.0f;       // kcal/mol/A beyond the grid

// XS type properties, indexed by type id (C_H, C_P, N_P, N_D, N_A, N_DA, O_P, O_D, O_A, O_DA, S_P)
__host__ __device__ inline float xs_radius(int t) {
    return t <= 1 ? 1.9f : (t <= 5 ? 1.8f : (t <= 9 ? 1.7f : 2.0f));
}
__host__ __device__ inline bool xs_hydrophobic(int t) { return t == 0; }
__host__ __device__ inline bool xs_donor(int t) { return t == 3 || t == 5 || t == 7 || t == 9; }
__host__ __device__ inline bool xs_acceptor(int t) { return t == 4 || t == 5 || t == 8 || t == 9; }

// Weighted pair energy at distance r and (dE/dr) / r, from r^2 (< cutoff^2, checked by the caller):
// one reciprocal square root gives both r and the force scale. The hydrophobic and H-bond terms
// never meet in one pair (a hydrophobic carbon is neither donor nor acceptor), so they are one
// clamped ramp sat((p1 - d) p2) with the pair's weight: p1 = 1.5, p2 = 1 for hydrophobic pairs,
// p1 = 0, p2 = 1 / 0.7 for H-bond pairs; its derivative is -p2 on the ramp (the same values and
// one-sided derivatives as vina_pair below).
// 2^x by the PTX approximation (flush-to-zero); the exponentials below use e^y = 2^(y log2 e) with
// log2 e folded into their constants.
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2e = 1.44269504088896341f;

__device__ __forceinline__ float vina_pair_r2(float r2, float rsum, bool hyd, bool hb, float& dedr_over_r) {
    const float rinv = rsqrtf(fmaxf(r2, 1e-12f));
    const float r = r2 * rinv;
    const float d = r - rsum;
    const float g1 = exp2_approx(d * d * (-4.0f * kLog2e));     // exp(-(d / 0.5)^2)
    const float b = d - 3.0f;
    const float g2 = exp2_approx(b * b * (-0.25f * kLog2e));    // exp(-((d - 3) / 2)^2)
    const float rep = fminf(d, 0.0f);
    const float p1 = hyd ? 1.5f : 0.0f, p2 = hyd ? 1.0f : (1.0f / 0.7f);
    const float w = hyd ? kWHydrophobic : (hb ? kWHBond : 0.0f);
    const float t = (p1 - d) * p2;
    const float v = __saturatef(t);
    const float dv = (t > 0.0f && t <= 1.0f) ? -p2 : 0.0f;
    const float e = kWGauss1 * g1 + kWGauss2 * g2 + kWRepulsion * rep * rep + w * v;
    const float de = (-8.0f * kWGauss1) * d * g1 + (-0.5f * kWGauss2) * b * g2 + (2.0f * kWRepulsion) * rep + w * dv;
    dedr_over_r = r2 > 1e-12f ? de * rinv : 0.0f;
    return e;
}

// The same pair energy with the ramp of the hydrophobic or H-bond term given by its constants,
// w sat(c0 + c1 d) (c0 = c1 = w = 0 for neither; the values of the ramps above), as the intra-pair
// records of a ligand carry them: no per-pair flag decoding. r2 > 0 (a pair of distinct atoms).
__device__ __forceinline__ float vina_pair_ramp(float r2, float rsum, float c0, float c1, float w,
                                                float& dedr_over_r) {
    const float rinv = rsqrtf(fmaxf(r2, 1e-12f));
    const float r = r2 * rinv;
    const float d = r - rsum;
    const float g1 = exp2_approx(d * d * (-4.0f * kLog2e));     // exp(-(d / 0.5)^2)
    const float b = d - 3.0f;
    const float g2 = exp2_approx(b * b * (-0.25f * kLog2e));    // exp(-((d - 3) / 2)^2)
    const float rep = fminf(d, 0.0f);
    const float t = fmaf(c1, d, c0);
    const float v = __saturatef(t);
    const float dv = (t > 0.0f && t <= 1.0f) ? c1 : 0.0f;
    const float e = kWGauss1 * g1 + kWGauss2 * g2 + kWRepulsion * rep * rep + w * v;
    const float de = (-8.0f * kWGauss1) * d * g1 + (-0.5f * kWGauss2) * b * g2 + (2.0f * kWRepulsion) * rep + w * dv;
    dedr_over_r = de * rinv;
    return e;
}

// Weighted pair energy at distance r (< cutoff, checked by the caller) and dE/dr.
__device__ __forceinline__ float vina_pair(float r, float rsum, bool hyd, bool hb, float& dedr) {
    float d = r - rsum;
    float a = 2.0f * d;                    // d / 0.5
    float g1 = __expf(-a * a);
    float b = 0.5f * (d - 3.0f);           // (d - 3) / 2
    float g2 = __expf(-b * b);
    float e = kWGauss1 * g1 + kWGauss2 * g2;
    float de = kWGauss1 * g1 * (-4.0f * a) + kWGauss2 * g2 * (-b);
    if (d < 0.0f) { e += kWRepulsion * d * d; de += 2.0f * kWRepulsion * d; }
    if (hyd) {
        if (d < 0.5f) e += kWHydrophobic;
        else if (d < 1.5f) { e += kWHydrophobic * (1.5f - d); de -= kWHydrophobic; }
    }
    if (hb) {
        if (d < -0.7f) e += kWHBond;
        else if (d < 0.0f) { e += kWHBond * (-d * (1.0f / 0.7f)); de -= kWHBond * (1.0f / 0.7f); }
    }
    dedr = de;
    return e;
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57,
// key schedule increments 0x9E3779B9 / 0xBB67AE85.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
__device__ __forceinline__ uint32_t pick(uint4 v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
// Word i of the draw stream of (chain, pair, step): word i % 4 of philox(ctr = {chain, pair,
// step, i / 4}, key = seed).
__device__ __forceinline__ uint32_t draw_word(uint32_t chain, uint32_t pair, uint32_t step, int i,
                                              uint32_t k0, uint32_t k1) {
    return pick(philox4x32_10(make_uint4(chain, pair, step, (uint32_t)(i >> 2)), k0, k1), i & 3);
}
// Uniform in [0, 1) from the top 24 bits (exact in binary32).
__device__ __forceinline__ float u01(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------------------------------------
// Quaternions (w, x, y, z), Hamilton product; rotation matrices row-major.
// ------------------------------------------------------------------------------------------
struct Mat3 { float m[9]; };

__device__ __forceinline__ float4 quat_normalize(float4 q) {
    float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    return make_float4(q.x * n, q.y * n, q.z * n, q.w * n);
}
// q stored as float4(w, x, y, z)
__device__ __forceinline__ Mat3 quat_to_mat(float4 qi) {
    float4 q = quat_normalize(qi);
    float w = q.x, x = q.y, y = q.z, z = q.w;
    Mat3 R;
    R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - w * z); R.m[2] = 2.f * (x * z + w * y);
    R.m[3] = 2.f * (x * y + w * z); R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - w * x);
    R.m[6] = 2.f * (x * z - w * y); R.m[7] = 2.f * (y * z + w * x); R.m[8] = 1.f - 2.f * (x * x + y * y);
    return R;
}
__device__ __forceinline__ float4 quat_mul(float4 a, float4 b) {
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                       a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                       a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}
// x reduced to [-pi, pi] by the two-constant reduction of Cody & Waite ("Software Manual for the
// Elementary Functions", 1980): x - k 2pi with k = rint(x / 2pi) and 2pi split into its nearest float
// and the remainder; the fast sine and cosine (the build uses them) are accurate on [-pi, pi], and
// angles here (torsions that a search moves freely) can lie anywhere.
__device__ __forceinline__ float wrap_pi(float x) {
    const float k = rintf(x * (1.0f / (2.0f * PV_PI)));
    const float r = fmaf(k, -6.28318548e+00f, x);     // 2pi rounded to float
    return fmaf(k, 1.74845560e-07f, r);               // minus (2pi - that float)
}

// q <- normalize(exp(omega / 2) (x) q): world-frame rotation by the rotation vector omega.
__device__ __forceinline__ float4 quat_rotate_by(float4 q, float3 om) {
    float th2 = om.x * om.x + om.y * om.y + om.z * om.z;
    float4 e;
    if (th2 < 1e-16f) {
        e = make_float4(1.0f, 0.5f * om.x, 0.5f * om.y, 0.5f * om.z);
    } else {
        float th = sqrtf(th2), s, c;
        sincosf(wrap_pi(0.5f * th), &s, &c);
        s /= th;
        e = make_float4(c, s * om.x, s * om.y, s * om.z);
    }
    return quat_normalize(quat_mul(e, q));
}
// Rotation matrix of the unit quaternion (w, x, y, z) given already normalised.
__device__ __forceinline__ Mat3 unit_quat_to_mat(float w, float x, float y, float z) {
    Mat3 R;
    R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - w * z); R.m[2] = 2.f * (x * z + w * y);
    R.m[3] = 2.f * (x * y + w * z); R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - w * x);
    R.m[6] = 2.f * (x * z - w * y); R.m[7] = 2.f * (y * z + w * x); R.m[8] = 1.f - 2.f * (x * x + y * y);
    return R;
}

// Rotation by angle t about the unit axis a (Rodrigues).
__device__ __forceinline__ Mat3 axis_angle(float3 a, float t) {
    float s, c;
    sincosf(wrap_pi(t), &s, &c);
    float C = 1.0f - c;
    Mat3 R;
    R.m[0] = c + a.x * a.x * C;        R.m[1] = a.x * a.y * C - a.z * s; R.m[2] = a.x * a.z * C + a.y * s;
    R.m[3] = a.y * a.x * C + a.z * s;  R.m[4] = c + a.y * a.y * C;       R.m[5] = a.y * a.z * C - a.x * s;
    R.m[6] = a.z * a.x * C - a.y * s;  R.m[7] = a.z * a.y * C + a.x * s; R.m[8] = c + a.z * a.z * C;
    return R;
}
__device__ __forceinline__ Mat3 mat_mul(const Mat3& A, const Mat3& B) {
    Mat3 C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C.m[3 * i + j] = A.m[3 * i] * B.m[j] + A.m[3 * i + 1] * B.m[3 + j] + A.m[3 * i + 2] * B.m[6 + j];
    return C;
}
__device__ __forceinline__ float3 mat_vec(const Mat3& A, float3 v) {
    return make_float3(A.m[0] * v.x + A.m[1] * v.y + A.m[2] * v.z,
                       A.m[3] * v.x + A.m[4] * v.y + A.m[5] * v.z,
                       A.m[6] * v.x + A.m[7] * v.y + A.m[8] * v.z);
}
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ------------------------------------------------------------------------------------------
// Trilinear interpolation of one map (Eq. 3: e_inter from the grid cache) with its gradient.
// Outside the grid the point is clamped to it and kOutSlope * distance is added. Two layouts hold
// the same node values: plain maps [z][y][x], whose eight corners take eight scalar loads from at
// least four 32-byte sectors, and cell-packed maps (each cell's eight corners contiguous, 32 bytes:
// two 16-byte loads from one sector). Both interpolate the same eight values with the same
// arithmetic, so they give the same bits.
// ------------------------------------------------------------------------------------------
struct GridCell {
    int i[3];          // the cell's lowest node
    float f[3];        // position inside the cell, [0, 1]
    float out[3];      // distance outside the grid per axis (A), 0 inside
    bool cl[3];        // clamped per axis
};

__device__ __forceinline__ GridCell grid_locate(const PvPocket& P, float3 p) {
    const float g[3] = {(p.x - P.origin[0]) * P.inv_spacing, (p.y - P.origin[1]) * P.inv_spacing,
                        (p.z - P.origin[2]) * P.inv_spacing};
    GridCell c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float hi = (float)(P.dims[k] - 1);
        c.cl[k] = (g[k] < 0.0f) || (g[k] > hi);
        const float gc = fminf(fmaxf(g[k], 0.0f), hi);
        int ii = (int)floorf(gc);
        ii = min(ii, P.dims[k] - 2);
        c.i[k] = ii;
        c.f[k] = gc - (float)ii;
        c.out[k] = c.cl[k] ? (g[k] - gc) * P.spacing : 0.0f;
    }
    return c;
}

// v = the corners (x fastest): v000, v100, v010, v110, v001, v101, v011, v111
__device__ __forceinline__ float grid_interpolate(const PvPocket& P, const GridCell& c, const float4 lo,
                                                  const float4 hi, float3& dEdx) {
    const float v000 = lo.x, v100 = lo.y, v010 = lo.z, v110 = lo.w;
    const float v001 = hi.x, v101 = hi.y, v011 = hi.z, v111 = hi.w;
    const float fx = c.f[0], fy = c.f[1], fz = c.f[2];
    const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
    // along x
    const float a00 = gx * v000 + fx * v100, a10 = gx * v010 + fx * v110;
    const float a01 = gx * v001 + fx * v101, a11 = gx * v011 + fx * v111;
    const float b0 = gy * a00 + fy * a10, b1 = gy * a01 + fy * a11;
    float val = gz * b0 + fz * b1;
    const float dx = gz * (gy * (v100 - v000) + fy * (v110 - v010)) + fz * (gy * (v101 - v001) + fy * (v111 - v011));
    const float dy = gz * (a10 - a00) + fz * (a11 - a01);
    const float dz = b1 - b0;
    dEdx = make_float3(c.cl[0] ? 0.f : dx * P.inv_spacing, c.cl[1] ? 0.f : dy * P.inv_spacing,
                       c.cl[2] ? 0.f : dz * P.inv_spacing);
    const float d2 = c.out[0] * c.out[0] + c.out[1] * c.out[1] + c.out[2] * c.out[2];
    if (d2 > 0.0f) {
        const float dist = sqrtf(d2);
        val += kOutSlope * dist;
        const float sl = kOutSlope / dist;
        dEdx.x += sl * c.out[0]; dEdx.y += sl * c.out[1]; dEdx.z += sl * c.out[2];
    }
    return val;
}

// Plain layout: `map` is one map [z][y][x].
__device__ __forceinline__ float grid_eval(const float* __restrict__ map, const PvPocket& P,
                                           float3 p, float3& dEdx) {
    const GridCell c = grid_locate(P, p);
    const float* base = map + ((long long)c.i[2] * P.nxy + (long long)c.i[1] * P.dims[0] + c.i[0]);
    const float4 lo = make_float4(__ldg(base), __ldg(base + 1), __ldg(base + P.dims[0]), __ldg(base + P.dims[0] + 1));
    const float4 hi = make_float4(__ldg(base + P.nxy), __ldg(base + P.nxy + 1), __ldg(base + P.nxy + P.dims[0]),
                                  __ldg(base + P.nxy + P.dims[0] + 1));
    return grid_interpolate(P, c, lo, hi, dEdx);
}

// Cell-packed layout: `cells` holds one map's cells [z][y][x] over (dims - 1) per axis, two float4
// per cell (the corners in grid_interpolate's order).
__device__ __forceinline__ float grid_eval_cells(const float4* __restrict__ cells, const PvPocket& P,
                                                 float3 p, float3& dEdx) {
    const GridCell c = grid_locate(P, p);
    const float4* cp = cells + 2 * (((long long)c.i[2] * (P.dims[1] - 1) + c.i[1]) * (P.dims[0] - 1) + c.i[0]);
    return grid_interpolate(P, c, __ldg(cp), __ldg(cp + 1), dEdx);
}

// The lookup of map slot `slot` of a pocket in the layout LAYOUT (0 plain, 1 cell-packed).
template <int LAYOUT>
__device__ __forceinline__ float grid_eval_slot(const PvPocket& P, int slot, float3 p, float3& dEdx) {
    if constexpr (LAYOUT == 0) return grid_eval(P.maps + (long long)slot * P.nxyz, P, p, dEdx);
    else return grid_eval_cells(P.cells + 2LL * slot * P.ncells, P, p, dEdx);
}

// ------------------------------------------------------------------------------------------
// Warp helpers (butterfly reductions: every lane gets the same, order-fixed result)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(PV_FULL, v, o);
    return v;
}
__device__ __forceinline__ float3 warp_sum3(float3 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(PV_FULL, v.x, o);
        v.y += __shfl_xor_sync(PV_FULL, v.y, o);
        v.z += __shfl_xor_sync(PV_FULL, v.z, o);
    }
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace pv
