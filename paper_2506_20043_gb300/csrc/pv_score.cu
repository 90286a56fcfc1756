// pv_score.cu -- batched scoring of given poses (Eq. 3) with the adjoint gradient, one warp per
// pose; the vector-Jacobian product used by automatic differentiation; forward kinematics only.
#include <algorithm>

#include "pv_internal.h"
#include "pv_stage.cuh"
#include "pv_warp.cuh"

namespace pv {

constexpr int kScoreWarps = 8;

struct ScoreArgs {
    const PvLigBlob* lig;
    int lig_bytes;
    const PvPocket* pocket;
    uint64_t slots_lo, slots_hi;
    int n_poses, pot_stride;
    const float* pose;
    float* energy;        // forward outputs (nullable)
    float* grad;
    float* parts;
    const float* grad_energy;   // backward (nullable)
    float* grad_pose;
    float* grad_xyz;
    int fk_only;
    float* xyz;
};

__device__ __forceinline__ Pose read_pose(const float* p, int n_rot) {
    const int lane = threadIdx.x & 31;
    Pose x;
    x.T = make_float3(p[0], p[1], p[2]);
    x.q = make_float4(p[3], p[4], p[5], p[6]);
    x.psi = (lane >= 6 && lane < 6 + n_rot) ? p[lane + 1] : 0.f;
    return x;
}

template <int LAYOUT>
__global__ void __launch_bounds__(kScoreWarps * 32) score_kernel(ScoreArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    PvLigBlob& L = *reinterpret_cast<PvLigBlob*>(smem);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + ((A.lig_bytes + 127) & ~127));
    __shared__ PvPocket s_pocket;
    if (!A.fk_only && threadIdx.x < (int)(sizeof(PvPocket) / 4))
        reinterpret_cast<int*>(&s_pocket)[threadIdx.x] = reinterpret_cast<const int*>(A.pocket)[threadIdx.x];
    stage_ligand(&L, A.lig, A.slots_lo, A.slots_hi);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_rot = L.h.n_rot, n = L.h.n_atoms, nt = 6 + n_rot;
    WarpScratch& S = scratch[warp];
    init_scratch<32>(S);
    Site site;
    site.maps = s_pocket.maps;
    site.P = &s_pocket;
    for (int i = blockIdx.x * kScoreWarps + warp; i < A.n_poses; i += gridDim.x * kScoreWarps) {
        const float* p = A.pose + (size_t)i * A.pot_stride;
        const Pose x = read_pose(p, n_rot);
        if (A.fk_only) {
            float3 axw, xa;
            warp_fk(L, S, x, axw, xa);
            __syncwarp();
            for (int a = lane; a < n; a += 32) {
                float* dst = A.xyz + ((size_t)i * n + L.atom_src[a]) * 3;
                dst[0] = S.x[a].x; dst[1] = S.x[a].y; dst[2] = S.x[a].z;
            }
            __syncwarp();
            continue;
        }
        const bool want_grad = A.grad || A.grad_pose || A.grad_xyz;
        float g = 0.f, parts[2];
        const float e = warp_eval<LAYOUT>(L, S, site, x, g, want_grad, parts);
        if (A.energy && lane == 0) A.energy[i] = e;
        if (A.parts && lane == 0) { A.parts[2 * i] = parts[0]; A.parts[2 * i + 1] = parts[1]; }
        if (A.grad && lane < nt) A.grad[(size_t)i * nt + lane] = g;
        if (A.grad_energy) {
            const float dE = A.grad_energy[i];
            if (A.grad_pose) {
                float* out = A.grad_pose + (size_t)i * A.pot_stride;
                // translation
                if (lane < 3) out[lane] = dE * g;
                // raw quaternion through the normalisation: with unit (w, v) = q / |q| and the
                // world rotation gradient G, dSF/dq_w = -2 v.G / |q|, dSF/dv = 2 (w G + G x v) / |q|
                const float3 G = make_float3(shfl(g, 3), shfl(g, 4), shfl(g, 5));
                const float qn = sqrtf(x.q.x * x.q.x + x.q.y * x.q.y + x.q.z * x.q.z + x.q.w * x.q.w);
                const float w = x.q.x / qn;
                const float3 v = make_float3(x.q.y / qn, x.q.z / qn, x.q.w / qn);
                const float3 gv = (2.f / qn) * (w * G + cross3(G, v));
                const float gw = -2.f / qn * dot3(v, G);
                if (lane == 3) out[3] = dE * gw;
                if (lane == 4) out[4] = dE * gv.x;
                if (lane == 5) out[5] = dE * gv.y;
                if (lane == 6) out[6] = dE * gv.z;
                if (lane >= 6 && lane < nt) out[lane + 1] = dE * g;
            }
            if (A.grad_xyz) {
                for (int a = lane; a < n; a += 32) {
                    float* dst = A.grad_xyz + ((size_t)i * n + L.atom_src[a]) * 3;
                    const float4 gg = S.g[a];
                    dst[0] = dE * gg.x; dst[1] = dE * gg.y; dst[2] = dE * gg.z;
                }
            }
        }
        __syncwarp();
    }
}

static cudaError_t launch(const ScoreArgs& a, int layout, cudaStream_t s) {
    const int smem = ((a.lig_bytes + 127) & ~127) + kScoreWarps * (int)sizeof(WarpScratch);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int configured[2][64];
    if (dev < 0 || dev >= 64 || layout < 0 || layout > 1) return cudaErrorInvalidValue;
    const void* fn = layout == 1 ? (const void*)score_kernel<1> : (const void*)score_kernel<0>;
    if (smem > configured[layout][dev]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[layout][dev] = smem;
    }
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kScoreWarps * 32, smem);
    if (e != cudaSuccess) return e;
    int need = (a.n_poses + kScoreWarps - 1) / kScoreWarps;
    int grid = sms * (occ > 0 ? occ : 1);
    if (need < grid) grid = need;
    if (grid < 1) return cudaSuccess;
    if (layout == 1) score_kernel<1><<<grid, kScoreWarps * 32, smem, s>>>(a);
    else score_kernel<0><<<grid, kScoreWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_score(const PvLigBlob* lig, int lig_bytes, const PvPocket* pocket,
                         PvSlots slots, int n_poses, int pot_stride,
                         const float* pose, float* energy, float* grad, float* parts,
                         const float* grad_energy, float* grad_pose, float* grad_xyz,
                         int layout, cudaStream_t s) {
    ScoreArgs a{};
    a.lig = lig; a.lig_bytes = lig_bytes; a.pocket = pocket;
    uint64_t lo = 0, hi = 0;
    for (int t = 0; t < 16; ++t) {
        uint64_t b = (uint64_t)(uint8_t)slots.slot[t];
        if (t < 8) lo |= b << (8 * t); else hi |= b << (8 * (t - 8));
    }
    a.slots_lo = lo; a.slots_hi = hi;
    a.n_poses = n_poses; a.pot_stride = pot_stride; a.pose = pose;
    a.energy = energy; a.grad = grad; a.parts = parts;
    a.grad_energy = grad_energy; a.grad_pose = grad_pose; a.grad_xyz = grad_xyz;
    return launch(a, layout, s);
}

// SF of posed ligands given by their atom coordinates (input order), one warp per ligand: the atoms
// go to S.x in device order, then the same interpolation and pair rounds as for a pose; the
// coordinate gradient, scaled by grad_energy when given, comes from S.g.
struct ScoreXyzArgs {
    const PvLigBlob* lig;
    int lig_bytes;
    const PvPocket* pocket;
    uint64_t slots_lo, slots_hi;
    int n_poses;
    const float* xyz;
    const float* grad_energy;   // nullable: scale 1
    float* energy;              // nullable
    float* grad_xyz;            // nullable
};

template <int LAYOUT>
__global__ void __launch_bounds__(kScoreWarps * 32) score_xyz_kernel(ScoreXyzArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    PvLigBlob& L = *reinterpret_cast<PvLigBlob*>(smem);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + ((A.lig_bytes + 127) & ~127));
    __shared__ PvPocket s_pocket;
    if (threadIdx.x < (int)(sizeof(PvPocket) / 4))
        reinterpret_cast<int*>(&s_pocket)[threadIdx.x] = reinterpret_cast<const int*>(A.pocket)[threadIdx.x];
    stage_ligand(&L, A.lig, A.slots_lo, A.slots_hi);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = L.h.n_atoms;
    WarpScratch& S = scratch[warp];
    init_scratch<32>(S);
    Site site;
    site.maps = s_pocket.maps;
    site.P = &s_pocket;
    const Pose none{};
    for (int i = blockIdx.x * kScoreWarps + warp; i < A.n_poses; i += gridDim.x * kScoreWarps) {
        for (int a = lane; a < n; a += 32) {
            const float* src = A.xyz + ((size_t)i * n + L.atom_src[a]) * 3;
            const int t = (__float_as_int(L.atom[a].w) >> 8) & 255;
            S.x[a] = make_float4(src[0], src[1], src[2], xs_radius(t));
        }
        __syncwarp();
        float g = 0.f;
        const float e = team_eval<32, false, LAYOUT>(L, S, site, none, g, false);
        if (A.energy && lane == 0) A.energy[i] = e;
        if (A.grad_xyz) {
            const float s = A.grad_energy ? A.grad_energy[i] : 1.f;
            for (int a = lane; a < n; a += 32) {
                float* dst = A.grad_xyz + ((size_t)i * n + L.atom_src[a]) * 3;
                const float4 gg = S.g[a];
                dst[0] = s * gg.x; dst[1] = s * gg.y; dst[2] = s * gg.z;
            }
        }
        __syncwarp();
    }
}

cudaError_t launch_score_xyz(const PvLigBlob* lig, int lig_bytes, const PvPocket* pocket, PvSlots slots,
                             int n_poses, const float* xyz, const float* grad_energy, float* energy,
                             float* grad_xyz, int layout, cudaStream_t s) {
    ScoreXyzArgs a{};
    a.lig = lig; a.lig_bytes = lig_bytes; a.pocket = pocket;
    uint64_t lo = 0, hi = 0;
    for (int t = 0; t < 16; ++t) {
        uint64_t b = (uint64_t)(uint8_t)slots.slot[t];
        if (t < 8) lo |= b << (8 * t); else hi |= b << (8 * (t - 8));
    }
    a.slots_lo = lo; a.slots_hi = hi;
    a.n_poses = n_poses; a.xyz = xyz; a.grad_energy = grad_energy; a.energy = energy; a.grad_xyz = grad_xyz;
    const int smem = ((lig_bytes + 127) & ~127) + kScoreWarps * (int)sizeof(WarpScratch);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int configured[2][64];
    if (dev < 0 || dev >= 64 || layout < 0 || layout > 1) return cudaErrorInvalidValue;
    const void* fn = layout == 1 ? (const void*)score_xyz_kernel<1> : (const void*)score_xyz_kernel<0>;
    if (smem > configured[layout][dev]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[layout][dev] = smem;
    }
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kScoreWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const int need = (n_poses + kScoreWarps - 1) / kScoreWarps;
    const int grid = std::min(need, sms * (occ > 0 ? occ : 1));
    if (grid < 1) return cudaSuccess;
    if (layout == 1) score_xyz_kernel<1><<<grid, kScoreWarps * 32, smem, s>>>(a);
    else score_xyz_kernel<0><<<grid, kScoreWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pose_coords(const PvLigBlob* lig, int lig_bytes, int n_poses, int pot_stride,
                               const float* pose, float* xyz, cudaStream_t s) {
    ScoreArgs a{};
    a.lig = lig; a.lig_bytes = lig_bytes; a.n_poses = n_poses; a.pot_stride = pot_stride;
    a.pose = pose; a.fk_only = 1; a.xyz = xyz;
    return launch(a, 0, s);
}

}  // namespace pv
