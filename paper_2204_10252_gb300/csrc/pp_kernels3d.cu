// 3-D Cartesian normal operator (Sec. 5.1) in one kernel on 16-CTA thread
// block clusters:
//   out[:, :, x] = scale * sum_c conj(S_c) F_yz^H M F_yz (S_c x)[:, :, x] + alpha * operand
// The readout axis x is never transformed (the mask is constant along it),
// so every x column is an independent (z, y) problem.  A cluster owns four
// adjacent x columns (a 32-byte run of every row) and keeps their (z, y)
// planes on chip for one coil at a time: CTA q holds z rows 8q .. 8q + 7 for
// the y transforms and the ky set {q + 16 k2} for the z transforms, and the
// two distributions exchange data through distributed shared memory.  Per
// coil: y FFT of S_c x -> local P; cluster barrier; z FFT, mask, z IFFT of
// the CTA's ky set, reading every CTA's P -> local Q; cluster barrier; y IFFT
// reading every CTA's Q, times conj(S_c), accumulated in registers.  The
// coil maps are read from HBM once per coil and once more from L2.
// nz = 128 (16 x 8); ny = 16 * N2Y with N2Y in {8, 12, 16}.  XB = 4 x columns
// per task needs one CTA per SM (160 KB of shared memory); XB = 2 halves the
// footprint so two CTAs share an SM and a 16-CTA cluster spans 8 SMs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "pp_fft4.cuh"
#include "pp_internal.h"

namespace cg = cooperative_groups;

namespace pp {
namespace {

constexpr int N1 = 16;
constexpr int NCL = 16;   // CTAs per cluster
constexpr int NZ2 = 8;    // nz = 16 * NZ2

template <int N2> __host__ __device__ constexpr int tpr() { return N2 > N1 ? N2 : N1; }

// Element (block, zl, xi) of a [block][8 z][XB x] array, the 8 XB entries of
// a block rotated by XB k2 (k2 = the block's ky / 16): the stores and the
// remote reads of both exchanges then never meet twice in a bank.
template <int XB>
__device__ __forceinline__ int swz(int blk, int zl, int xi, int k2) {
    return blk * (8 * XB) + ((zl * XB + xi + XB * k2) & (8 * XB - 1));
}

// Distributed shared memory: the address of `a` (a shared-memory address of
// this CTA) in CTA `rank` of the cluster, and an 8-byte load from it.
__device__ __forceinline__ uint32_t dsmem_map(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 dsmem_ld(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

template <int N2Y, int XB> struct C3Cl {
    // LT: y transforms per CTA (8 z rows x XB columns) = lanes of one transform row
    static constexpr int NY = 16 * N2Y, NZ = 16 * NZ2, LT = NZ2 * XB, THREADS = LT * tpr<N2Y>();
    // P and Q: 16 * N2Y blocks of LT; Yz: one round of LT z transforms
    static constexpr size_t SMEM = sizeof(float2) * (2 * LT * NY + LT * NZ + NY + NZ);
};

template <int N2Y, int XB>
__global__ void __launch_bounds__(C3Cl<N2Y, XB>::THREADS, XB == 2 ? 2 : 1)
c3_cluster_kernel(const float2* __restrict__ tw_y, const float2* __restrict__ tw_z,
                  const float2* __restrict__ x, const float2* __restrict__ S, int C, int nx,
                  const float* __restrict__ mask_fo, float2* out, float scale,
                  const float2* operand, float alpha) {
    constexpr int NY = C3Cl<N2Y, XB>::NY, NZ = C3Cl<N2Y, XB>::NZ, LT = C3Cl<N2Y, XB>::LT;
    constexpr int NZT = XB * N2Y;                // z transforms per CTA: (k2, xi)
    constexpr int ROUNDS = (NZT + LT - 1) / LT;
    extern __shared__ float4 sm4[];
    float2* P = reinterpret_cast<float2*>(sm4);  // y-FFT results (and the y transpose)
    float2* Q = P + LT * NY;                     // z-FFT results
    float2* Yz = Q + LT * NY;                    // z transpose, one round
    float2* twy = Yz + LT * NZ;
    float2* twz = twy + NY;
    cg::cluster_group cluster = cg::this_cluster();
    const int self = (int)cluster.block_rank();
    const uint32_t sP = (uint32_t)__cvta_generic_to_shared(P), sQ = (uint32_t)__cvta_generic_to_shared(Q);
    const int cid = blockIdx.x / NCL, ncid = gridDim.x / NCL;
    for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = tw_y[i];
    for (int i = threadIdx.x; i < NZ; i += blockDim.x) twz[i] = tw_z[i];
    __syncthreads();
    const int64_t plane = (int64_t)NY * nx, vol = (int64_t)NZ * plane;
    const int t = threadIdx.x % LT, r = threadIdx.x / LT;   // t = (zl, xi) or z transform
    const int zl = t / XB, xi = t % XB;
    const int ntasks = nx / XB;
    for (int task = cid; task < ntasks; task += ncid) {
        const int64_t base = (int64_t)(NZ2 * self + zl) * plane + task * XB + xi;
        float2 acc[N2Y];
#pragma unroll
        for (int k2 = 0; k2 < N2Y; ++k2) acc[k2] = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float2* Sc = S + c * vol;
            // ---- y FFT of S_c x on rows z = 8 self + zl; ky = k1 + 16 k2 -> P
            if (r < N2Y) {
                float2 v[N1];
#pragma unroll
                for (int m1 = 0; m1 < N1; ++m1) {
                    const int64_t o = base + (int64_t)(N2Y * m1 + r) * nx;
                    v[m1] = cmul(Sc[o], x[o]);
                }
                fft4_phase1<N1, N2Y, false>(v, r, twy);
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) P[(k1 * N2Y + r) * LT + t] = v[k1];
            }
            __syncthreads();
            float2 u[N2Y];
            if (r < N1) {
#pragma unroll
                for (int m2 = 0; m2 < N2Y; ++m2) u[m2] = P[(r * N2Y + m2) * LT + t];
                fft4_phase2<N1, N2Y, false>(u, twy);
            }
            __syncthreads();
            if (r < N1) {
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) P[swz<XB>(r * N2Y + k2, zl, xi, k2)] = u[k2];
            }
            cluster.sync();
            // ---- z FFT, mask, z IFFT for ky = self + 16 k2 (all z: one value per CTA) -> Q
            for (int rd = 0; rd < ROUNDS; ++rd) {
                const int T = rd * LT + t, k2 = T / XB, xz = T % XB;
                const bool live = T < NZT;
                if (r < NZ2 && live) {
                    float2 v[N1];
#pragma unroll
                    for (int m1 = 0; m1 < N1; ++m1)
                        v[m1] = dsmem_ld(dsmem_map(sP, m1) + 8u * swz<XB>(self * N2Y + k2, r, xz, k2));
                    fft4_phase1<N1, NZ2, false>(v, r, twz);
#pragma unroll
                    for (int k1 = 0; k1 < N1; ++k1) Yz[(k1 * NZ2 + r) * LT + t] = v[k1];
                }
                __syncthreads();
                float2 w[NZ2];
                if (r < N1 && live) {
#pragma unroll
                    for (int m2 = 0; m2 < NZ2; ++m2) w[m2] = Yz[(r * NZ2 + m2) * LT + t];
                    fft4_phase2<N1, NZ2, false>(w, twz);
                    const int ky = self + N1 * k2;
#pragma unroll
                    for (int kb = 0; kb < NZ2; ++kb) w[kb] = cscale(w[kb], mask_fo[(r + N1 * kb) * NY + ky]);
                    // inverse with the mirrored decomposition: length-8 DFT over kb,
                    // twiddle W_nz^(-m2 k1), then the length-16 DFT over k1 below
                    RegFft<NZ2, true>::run(w, twz, N1);
#pragma unroll
                    for (int m2 = 1; m2 < NZ2; ++m2) {
                        float2 tw = twz[m2 * r];
                        tw.y = -tw.y;
                        w[m2] = cmul(w[m2], tw);
                    }
                }
                __syncthreads();   // every phase-2 read of Yz is done
                if (r < N1 && live) {
#pragma unroll
                    for (int m2 = 0; m2 < NZ2; ++m2) Yz[(r * NZ2 + m2) * LT + t] = w[m2];
                }
                __syncthreads();
                if (r < NZ2 && live) {
                    float2 v[N1];
#pragma unroll
                    for (int k1 = 0; k1 < N1; ++k1) v[k1] = Yz[(k1 * NZ2 + r) * LT + t];
                    RegFft<N1, true>::run(v, twz, NZ2);
                    // z = 8 m1 + r belongs to CTA m1
#pragma unroll
                    for (int m1 = 0; m1 < N1; ++m1) Q[swz<XB>(m1 * N2Y + k2, r, xz, k2)] = v[m1];
                }
                __syncthreads();   // Yz is reused by the next round
            }
            cluster.sync();
            // ---- y IFFT on rows z = 8 self + zl, reading ky = N2Y m1 + r from CTA ky % 16
            if (r < N2Y) {
                float2 v[N1];
#pragma unroll
                for (int m1 = 0; m1 < N1; ++m1) {
                    const int ky = N2Y * m1 + r, k2 = ky >> 4;
                    v[m1] = dsmem_ld(dsmem_map(sQ, ky & 15) + 8u * swz<XB>(self * N2Y + k2, zl, xi, k2));
                }
                fft4_phase1<N1, N2Y, true>(v, r, twy);
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) P[(k1 * N2Y + r) * LT + t] = v[k1];
            }
            __syncthreads();
            if (r < N1) {
#pragma unroll
                for (int m2 = 0; m2 < N2Y; ++m2) u[m2] = P[(r * N2Y + m2) * LT + t];
                fft4_phase2<N1, N2Y, true>(u, twy);
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) {
                    const int64_t o = base + (int64_t)(r + N1 * k2) * nx;
                    acc[k2] = cadd(acc[k2], cmulc(Sc[o], u[k2]));
                }
            }
            __syncthreads();   // P is rewritten by the next coil
        }
        if (r < N1) {
#pragma unroll
            for (int k2 = 0; k2 < N2Y; ++k2) {
                const int64_t o = base + (int64_t)(r + N1 * k2) * nx;
                float2 v = cscale(acc[k2], scale);
                if (operand) v = cadd(v, cscale(operand[o], alpha));
                out[o] = v;
            }
        }
    }
    cluster.sync();   // no CTA leaves while another may still read its Q
}

}  // namespace

extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

template <int N2Y, int XB>
static int c3cl_clusters_for() {
    auto fn = c3_cluster_kernel<N2Y, XB>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C3Cl<N2Y, XB>::SMEM) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(NCL * 64);
    cfg.blockDim = dim3(C3Cl<N2Y, XB>::THREADS);
    cfg.dynamicSmemBytes = C3Cl<N2Y, XB>::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Clusters that can be resident at once for this plan's sizes with XB x
// columns per task (0: the cluster kernel does not apply: nz != 128, ny not
// in {128, 192, 256}, nx not a multiple of XB, or no 16-CTA cluster fits).
int c3cl_prepare(const Plan& p, int xb) {
    if (p.kind != PP_CARTESIAN || p.ndim != 3 || p.nz != 16 * NZ2 || p.nx % xb) return 0;
    if (xb == 2) {
        switch (p.ny) {
            case 128: return c3cl_clusters_for<8, 2>();
            case 192: return c3cl_clusters_for<12, 2>();
            case 256: return c3cl_clusters_for<16, 2>();
            default: return 0;
        }
    }
    switch (p.ny) {
        case 128: return c3cl_clusters_for<8, 4>();
        case 192: return c3cl_clusters_for<12, 4>();
        case 256: return c3cl_clusters_for<16, 4>();
        default: return 0;
    }
}

pp_status c3cl_normal(const Plan& p, int xb, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st) {
    const int ntasks = p.nx / xb;
    const int avail = xb == 2 ? p.c3cl2_clusters : p.c3cl_clusters;
    const int ncl = std::max(1, std::min(avail, ntasks));
    cudaError_t e = cudaErrorInvalidValue;
#define PP_C3L(N2Y_, XB_)                                                                         \
    if (p.ny == 16 * N2Y_ && xb == XB_)                                                           \
        e = launch_ex(c3_cluster_kernel<N2Y_, XB_>, dim3(NCL * ncl), dim3(C3Cl<N2Y_, XB_>::THREADS), \
                      C3Cl<N2Y_, XB_>::SMEM, st, false, NCL, (const float2*)p.fy.tw,              \
                      (const float2*)p.fz.tw, x, p.sens, p.C, p.nx, (const float*)p.mask_fo, out, \
                      scale, operand, alpha);
    PP_C3L(8, 4) PP_C3L(12, 4) PP_C3L(16, 4) PP_C3L(8, 2) PP_C3L(12, 2) PP_C3L(16, 2)
#undef PP_C3L
    if (e != cudaSuccess) return cuda_status(e, "c3_cluster_kernel launch");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "c3_cluster_kernel");
    ++g_launches;
    if (g_profiler) g_profiler->mark("c3_cluster_kernel");
    return PP_OK;
}

}  // namespace pp
