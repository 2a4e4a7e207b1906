// Row and column FFT stages on the register four-step FFT (pp_fft4.cuh) for
// the lengths n = 16 * N2, N2 in {8, 12, 16, 20, 24}.  Same contracts as the
// Stockham kernels in pp_kernels.cu (RowArgs / ColArgs index maps), one
// shared-memory transpose per transform instead of one pass per radix stage.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "pp_fft4.cuh"
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int N1 = 16;
constexpr int TXF = 8;      // columns per CTA (column stage)
constexpr int LGTXF = 3;
constexpr int RBF = 8;      // rows / coils per CTA (row stages)


template <int N2> __host__ __device__ constexpr int tpr() { return N2 > N1 ? N2 : N1; }
// Minimum resident CTAs of the row stages: for N2 = 20 this caps them at 56
// registers, so that 7 CTAs of 160 threads fit an SM and the 1024 CTAs of a
// 256-row, 32-coil stage run in one wave on 152 SMs.
template <int N2> __host__ __device__ constexpr int row_min_ctas() { return N2 == 20 ? 7 : 1; }
// Minimum resident CTAs of the 3-D z pass (TX columns per CTA): at most 80
// registers per thread.
template <int N2, int TX> __host__ __device__ constexpr int c3_min_ctas() {
    return 65536 / (TX * tpr<N2>() * 80);
}

// Column stage: TXF adjacent columns of one batch, transform along rows.
template <int N2, bool INV>
__global__ void __launch_bounds__(TXF * tpr<N2>())
cols4_kernel(const float2* __restrict__ tw, ColArgs a, const float2* src, float2* dst) {
    constexpr int n = N1 * N2;
    __shared__ float2 tws[n];
    __shared__ float2 Y[N1 * N2 * TXF];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    const int col0 = blockIdx.x * TXF;
    const float2* sb = src + (int64_t)blockIdx.y * a.in_batch_stride;
    float2* db = dst + (int64_t)blockIdx.y * a.out_batch_stride;
    const int lane = threadIdx.x & (TXF - 1);
    const int r = threadIdx.x >> LGTXF;
    const int col = col0 + lane;
    __syncthreads();
    if (r < N2) {
        const int m2 = r;
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + m2;
            int row = p + a.off_in;
            if (row >= n) row -= n;
            float2 x = make_float2(0.f, 0.f);
            if (row < a.Hin && col < a.ncols) {
                x = sb[(int64_t)row * a.ncols + col];
                if (a.mul_in) x = cscale(x, a.mul_in[row * a.mi_q + (col / a.mi_cdiv) * a.mi_c]);
            }
            v[m1] = x;
        }
        fft4_phase1<N1, N2, INV>(v, m2, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[((k1 * N2) + m2) * TXF + lane] = v[k1];
    }
    __syncthreads();
    if (r < N1 && col < a.ncols) {
        const int k1 = r;
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[((k1 * N2) + m2) * TXF + lane];
        fft4_phase2<N1, N2, INV>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int k = k1 + N1 * k2;
            int q = k + a.off_out;
            if (q >= n) q -= n;
            if (q < a.Hout) {
                float s = a.scale;
                if (a.mul_out) s *= a.mul_out[q * a.mo_q + (col / a.mo_cdiv) * a.mo_c];
                db[(int64_t)q * a.ncols + col] = cscale(u[k2], s);
            }
        }
    }
}

// Row stage image -> k rows (coil expansion, weights, circular placement).
template <int N2>
__global__ void __launch_bounds__(RBF * tpr<N2>(), row_min_ctas<N2>())
rows4_fwd_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ x,
                 int64_t x_batch_stride, const float2* __restrict__ sens,
                 const float* __restrict__ wrow, const float* __restrict__ wcol,
                 float2* __restrict__ out) {
    constexpr int n = N1 * N2, T = tpr<N2>(), YS = N2 + 1;
    __shared__ float2 tws[n];
    __shared__ float2 Y[RBF * N1 * YS];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    const int b = threadIdx.x / T, r = threadIdx.x - (threadIdx.x / T) * T;
    const int c = blockIdx.y;
    const int row = blockIdx.x * RBF + b;
    const bool live = row < a.nrows;
    const float2* xc = x + (int64_t)c * x_batch_stride;
    const float2* sc = sens ? sens + (int64_t)c * a.coil_img_stride : nullptr;
    if (r < N2) {
        const int m2 = r;
        const float wr = (wrow && live) ? wrow[row] : 1.f;
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + m2;
            int i = p + a.off_in;
            if (i >= n) i -= n;
            float2 val = make_float2(0.f, 0.f);
            if (live && i < a.n) {
                const int64_t o = (int64_t)row * a.n + i;
                val = xc[o];
                if (sc) val = cmul(val, sc[o]);
                float w = a.scale * wr;
                if (wcol) w *= wcol[i];
                val = cscale(val, w);
            }
            v[m1] = val;
        }
        fft4_phase1<N1, N2, false>(v, m2, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[(b * N1 + k1) * YS + m2] = v[k1];
    }
    __syncthreads();
    if (r < N1 && live) {
        const int k1 = r;
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(b * N1 + k1) * YS + m2];
        fft4_phase2<N1, N2, false>(u, tws);
        float2* oc = out + ((int64_t)c * a.nrows + row) * n;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            int q = k1 + N1 * k2 + a.off_out;
            if (q >= n) q -= n;
            oc[q] = u[k2];
        }
    }
}

// Row stage k rows -> image for many coils: one image row per CTA, the
// transform batch runs over RBF coils at a time; conjugate-coil reduction
// and axpy epilogue as rows_adj_cb_kernel.
template <int N2>
__global__ void __launch_bounds__(RBF * tpr<N2>())
rows4_adj_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ src,
                 const float2* __restrict__ sens, const float* __restrict__ wrow,
                 const float* __restrict__ wcol, float2* out, const float2* operand, float alpha,
                 int ncoils) {
    constexpr int n = N1 * N2, T = tpr<N2>(), YS = N2 + 1, RS = n + 1;
    static_assert(RBF * RS <= RBF * N1 * YS, "R must fit in Y's space");
    __shared__ float2 tws[n];
    __shared__ float2 Y[RBF * N1 * YS];
    float2* R = Y;   // the transposed rows overwrite Y once it has been read
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    const int b = threadIdx.x / T, r = threadIdx.x - (threadIdx.x / T) * T;
    const int row = blockIdx.x;
    const float wr = wrow ? wrow[row] : 1.f;
    constexpr int KO = (512 + RBF * T - 1) / (RBF * T);   // outputs per thread, a.n <= 512
    float2 acc[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) acc[k] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int c0 = 0; c0 < ncoils; c0 += RBF) {
        const int c = c0 + b;
        if (r < N2) {
            const int m2 = r;
            float2 v[N1];
#pragma unroll
            for (int m1 = 0; m1 < N1; ++m1) {
                int s = N2 * m1 + m2 + a.off_in;
                if (s >= n) s -= n;
                v[m1] = (c < ncoils) ? src[((int64_t)c * a.nrows + row) * n + s] : make_float2(0.f, 0.f);
            }
            fft4_phase1<N1, N2, true>(v, m2, tws);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) Y[(b * N1 + k1) * YS + m2] = v[k1];
        }
        __syncthreads();
        float2 u[N2];
        if (r < N1) {
#pragma unroll
            for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(b * N1 + r) * YS + m2];
        }
        __syncthreads();
        if (r < N1) {
            const int k1 = r;
            fft4_phase2<N1, N2, true>(u, tws);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) R[b * RS + k1 + N1 * k2] = u[k2];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int i = threadIdx.x + k * (RBF * T);
            if (i < a.n) {
                int p = i - a.off_out;
                if (p < 0) p += n;
                const float w = wcol ? wr * wcol[i] : wr;
                for (int bb = 0; bb < RBF; ++bb) {
                    const int cc = c0 + bb;
                    if (cc >= ncoils) break;
                    float2 v = cscale(R[bb * RS + p], w);
                    if (sens) v = cmulc(sens[(int64_t)cc * a.coil_img_stride + (int64_t)row * a.n + i], v);
                    acc[k] = cadd(acc[k], v);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        const int i = threadIdx.x + k * (RBF * T);
        if (i < a.n) {
            const int64_t o = (int64_t)row * a.n + i;
            float2 v = cscale(acc[k], a.scale);
            if (operand) v = cadd(v, cscale(operand[o], alpha));
            out[o] = v;
        }
    }
}

// rows4_adj_kernel with the coil loop split over a cluster of up to 4 CTAs
// (one image row per cluster): CTA q of the cluster takes coil groups
// q, q + CL, ... (RBF coils each), then the partial sums are reduced through
// distributed shared memory by rank 0, which applies the epilogue.
template <int N2>
__global__ void __launch_bounds__(RBF * tpr<N2>())
rows4_adj_cl_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ src,
                    const float2* __restrict__ sens, const float* __restrict__ wrow,
                    const float* __restrict__ wcol, float2* out, const float2* operand, float alpha,
                    int ncoils) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    constexpr int n = N1 * N2, T = tpr<N2>(), YS = N2 + 1, RS = n + 1;
    static_assert(RBF * RS <= RBF * N1 * YS, "R must fit in Y's space");
    __shared__ float2 tws[n];
    __shared__ float2 Y[RBF * N1 * YS];
    __shared__ float2 part[512];
    float2* R = Y;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    const int b = threadIdx.x / T, r = threadIdx.x - (threadIdx.x / T) * T;
    const int row = blockIdx.x / CL;
    const float wr = wrow ? wrow[row] : 1.f;
    constexpr int KO = (512 + RBF * T - 1) / (RBF * T);
    float2 acc[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) acc[k] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int c0 = q * RBF; c0 < ncoils; c0 += CL * RBF) {
        const int c = c0 + b;
        if (r < N2) {
            const int m2 = r;
            float2 v[N1];
#pragma unroll
            for (int m1 = 0; m1 < N1; ++m1) {
                int s = N2 * m1 + m2 + a.off_in;
                if (s >= n) s -= n;
                v[m1] = (c < ncoils) ? src[((int64_t)c * a.nrows + row) * n + s] : make_float2(0.f, 0.f);
            }
            fft4_phase1<N1, N2, true>(v, m2, tws);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) Y[(b * N1 + k1) * YS + m2] = v[k1];
        }
        __syncthreads();
        float2 u[N2];
        if (r < N1) {
#pragma unroll
            for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(b * N1 + r) * YS + m2];
        }
        __syncthreads();
        if (r < N1) {
            fft4_phase2<N1, N2, true>(u, tws);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) R[b * RS + r + N1 * k2] = u[k2];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int i = threadIdx.x + k * (RBF * T);
            if (i < a.n) {
                int p = i - a.off_out;
                if (p < 0) p += n;
                const float w = wcol ? wr * wcol[i] : wr;
                for (int bb = 0; bb < RBF; ++bb) {
                    const int cc = c0 + bb;
                    if (cc >= ncoils) break;
                    float2 v = cscale(R[bb * RS + p], w);
                    if (sens) v = cmulc(sens[(int64_t)cc * a.coil_img_stride + (int64_t)row * a.n + i], v);
                    acc[k] = cadd(acc[k], v);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        const int i = threadIdx.x + k * (RBF * T);
        if (i < a.n) part[i] = acc[k];
    }
    cluster.sync();
    if (q == 0) {
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int i = threadIdx.x + k * (RBF * T);
            if (i < a.n) {
                float2 v = acc[k];
                for (int j = 1; j < CL; ++j) v = cadd(v, cluster.map_shared_rank(part, j)[i]);
                const int64_t o = (int64_t)row * a.n + i;
                v = cscale(v, a.scale);
                if (operand) v = cadd(v, cscale(operand[o], alpha));
                out[o] = v;
            }
        }
    }
    // keep every CTA's partial sums alive until rank 0 has read them (rank 0's
    // remote loads have fed its stores: the arrive needs no release)
    cluster_arrive_relaxed();
    cluster_wait_acquire();
}

// Row IFFT per (coil, row) with the crop, deapodisation and conj(S_c)
// product fused into the store: contrib[c][row][i] = w conj(S_c) IFFT(src_c[row])
// at image index i.  The coil sum follows in coil_sum_kernel.
template <int N2>
__global__ void __launch_bounds__(RBF * tpr<N2>(), row_min_ctas<N2>())
rows4_inv_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ src,
                 const float2* __restrict__ sens, const float* __restrict__ wrow,
                 const float* __restrict__ wcol, float2* __restrict__ contrib) {
    constexpr int n = N1 * N2, T = tpr<N2>(), YS = N2 + 1;
    __shared__ float2 tws[n];
    __shared__ float2 Y[RBF * N1 * YS];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    const int b = threadIdx.x / T, r = threadIdx.x - (threadIdx.x / T) * T;
    const int c = blockIdx.y;
    const int row = blockIdx.x * RBF + b;
    const bool live = row < a.nrows;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int sidx = N2 * m1 + r + a.off_in;
            if (sidx >= n) sidx -= n;
            v[m1] = live ? src[((int64_t)c * a.nrows + row) * n + sidx] : make_float2(0.f, 0.f);
        }
        fft4_phase1<N1, N2, true>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[(b * N1 + k1) * YS + r] = v[k1];
    }
    __syncthreads();
    if (r < N1 && live) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(b * N1 + r) * YS + m2];
        fft4_phase2<N1, N2, true>(u, tws);
        const float wr = wrow ? wrow[row] : 1.f;
        const float2* sc = sens + (int64_t)c * a.coil_img_stride + (int64_t)row * a.n;
        float2* oc = contrib + ((int64_t)c * a.nrows + row) * a.n;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            int i = r + N1 * k2 + a.off_out;
            if (i >= n) i -= n;
            if (i < a.n) {
                const float w = wcol ? wr * wcol[i] : wr;
                oc[i] = cmulc(sc[i], cscale(u[k2], w));
            }
        }
    }
}

// out[o] = scale * sum_c contrib[c][o] + alpha * operand[o].  A block of
// 64 x 4 threads covers 64 outputs; thread row g sums coils g, g + 4, ...,
// and the four partial sums meet in shared memory (fixed order).
__global__ void __launch_bounds__(256)
coil_sum_kernel(const float2* __restrict__ contrib, int C, int64_t n, float scale,
                const float2* operand, float alpha, float2* out) {
    __shared__ float2 part[4][64];
    const int lx = threadIdx.x & 63, g = threadIdx.x >> 6;
    for (int64_t base = (int64_t)blockIdx.x * 64; base < n; base += (int64_t)gridDim.x * 64) {
        const int64_t o = base + lx;
        float2 acc = make_float2(0.f, 0.f);
        if (o < n)
            for (int c = g; c < C; c += 4) acc = cadd(acc, contrib[(int64_t)c * n + o]);
        part[g][lx] = acc;
        __syncthreads();
        if (g == 0 && o < n) {
            float2 v = cadd(cadd(part[0][lx], part[1][lx]), cadd(part[2][lx], part[3][lx]));
            v = cscale(v, scale);
            if (operand) v = cadd(v, cscale(operand[o], alpha));
            out[o] = v;
        }
        __syncthreads();
    }
}

// Fused 2-D Cartesian normal operator (one CTA per 8 columns, all coils);
// dynamic shared memory: the double-buffered coil-map tiles, 2 * n * 8 float2.
template <int N2>
__global__ void __launch_bounds__(8 * tpr<N2>(), 2)
cart2d4_normal_kernel(const float2* __restrict__ tw, const float2* __restrict__ x,
                      const float2* __restrict__ sens, int C, int nx,
                      const float* __restrict__ mask_fo, float2* out, float scale,
                      const float2* operand, float alpha) {
    constexpr int n = N1 * N2;
    __shared__ float2 tws[n];
    __shared__ float pm[n];
    __shared__ float2 Y[N1 * N2 * 8];
    extern __shared__ float4 sb4[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        pm[i] = mask_fo[i];
    }
    __syncthreads();
    cart_item4<N2>(tws, pm, Y, reinterpret_cast<float2*>(sb4), x, sens, C, nx, blockIdx.x * 8, out,
                   scale, operand, alpha);
}

// The same with the coils split over a cluster of CL CTAs per 8-column
// group (for images too narrow to fill the GPU with column groups alone):
// CTA q takes coils q, q + CL, ...; the CL partial sums meet in distributed
// shared memory, CTA q summing rows [q n / CL, (q + 1) n / CL) in rank order.
// grid (CL * ceil(nx / 8)), cluster (CL, 1, 1).
template <int N2>
__global__ void __launch_bounds__(8 * tpr<N2>(), 2)
cart2d4_cluster_kernel(const float2* __restrict__ tw, const float2* __restrict__ x,
                       const float2* __restrict__ sens, int C, int nx,
                       const float* __restrict__ mask_fo, float2* out, float scale,
                       const float2* operand, float alpha) {
    constexpr int n = N1 * N2;
    __shared__ float2 tws[n];
    __shared__ float pm[n];
    __shared__ float2 Y[N1 * N2 * 8];
    extern __shared__ float4 sb4[];
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int col0 = (int)(blockIdx.x / CL) * 8;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        pm[i] = mask_fo[i];
    }
    __syncthreads();
    float2 acc[N1];
    cart_item4_acc<N2>(tws, pm, Y, reinterpret_cast<float2*>(sb4), x, sens, C, nx, col0, q, CL, acc);
    const int lane = threadIdx.x & 7, r = threadIdx.x >> 3;
    if (r < N2) {
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) Y[(N2 * m1 + r) * 8 + lane] = acc[m1];   // Y[row][lane]
    }
    // split barrier: publish the partials, load the first operand value of
    // this CTA's rows (independent of the cluster) while the others arrive
    cluster_arrive_release();
    const int rpr = n / CL;
    float2 op0 = make_float2(0.f, 0.f);
    {
        const int row = q * rpr + ((int)threadIdx.x >> 3), col = col0 + ((int)threadIdx.x & 7);
        if (operand && (int)threadIdx.x < rpr * 8 && col < nx) op0 = operand[(int64_t)row * nx + col];
    }
    cluster_wait_acquire();
    for (int idx = threadIdx.x; idx < rpr * 8; idx += blockDim.x) {
        const int row = q * rpr + (idx >> 3), l = idx & 7, col = col0 + l;
        float2 v = cluster.map_shared_rank(Y, 0)[row * 8 + l];
        for (int b = 1; b < CL; ++b) v = cadd(v, cluster.map_shared_rank(Y, b)[row * 8 + l]);
        if (col < nx) {
            const int64_t o = (int64_t)row * nx + col;
            v = cscale(v, scale);
            if (operand) v = cadd(v, cscale(idx == (int)threadIdx.x ? op0 : operand[o], alpha));
            out[o] = v;
        }
    }
    // keep every CTA's partials alive until the others have read them (their
    // remote loads have fed their stores: the arrive needs no release)
    cluster_arrive_relaxed();
    cluster_wait_acquire();
}

template <int N2> constexpr size_t cart4_dyn_smem() { return sizeof(float2) * 2 * 16 * N2 * 8; }

// ---------------------------------------------------------------------------
// 3-D Cartesian normal operator, x-block by x-block and coil by coil, with
// every pass on the register FFT.  Arrays are [nz][ny][nx]; a CTA owns 8
// columns x0 .. x0+7 of one z plane (y passes) or of one y row (z pass).
//   ypass_fwd:  W[z][:, x] = F_y (S_c x)[z][:, x]              (FFT order ky)
//   zpass:      W[:, ky, x] = F_z^H (M_fo[kz][ky] F_z W[:, ky, x])
//   ypass_inv:  out[z][:, x] (+)= conj(S_c) F_y^H W[z][:, x]; on the last
//               coil out = scale * out + alpha * operand
// ---------------------------------------------------------------------------
template <int N2, int TX>
__global__ void __launch_bounds__(TX * tpr<N2>())
c3_ypass_fwd_kernel(const float2* __restrict__ tw, const float2* __restrict__ x,
                    const float2* __restrict__ S, float2* __restrict__ W, int nx, int x0) {
    constexpr int n = N1 * N2;
    __shared__ float2 tws[n];
    __shared__ float2 Y[N1 * N2 * TX];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    const int lane = threadIdx.x % TX, r = threadIdx.x / TX;
    const int col = x0 + blockIdx.x * TX + lane;
    const bool ok = col < nx;
    const int64_t plane = (int64_t)blockIdx.y * n * nx;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int64_t o = plane + (int64_t)(N2 * m1 + r) * nx + col;
            v[m1] = ok ? cmul(S[o], x[o]) : make_float2(0.f, 0.f);
        }
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[(k1 * N2 + r) * TX + lane] = v[k1];
    }
    __syncthreads();
    if (r < N1 && ok) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(r * N2 + m2) * TX + lane];
        fft4_phase2<N1, N2, false>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) W[plane + (int64_t)(r + N1 * k2) * nx + col] = u[k2];
    }
}

template <int N2, int TX>
__global__ void __launch_bounds__(TX * tpr<N2>(), c3_min_ctas<N2, TX>())
c3_zpass_kernel(const float2* __restrict__ tw, float2* W, const float* __restrict__ mask_fo,
                int ny, int nx, int x0) {
    constexpr int n = N1 * N2;   // nz
    __shared__ float2 tws[n];
    __shared__ float2 Y[N1 * N2 * TX];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    const int lane = threadIdx.x % TX, r = threadIdx.x / TX;
    const int col = x0 + blockIdx.x * TX + lane;
    const int ky = blockIdx.y;
    const bool ok = col < nx;
    const int64_t zs = (int64_t)ny * nx, base = (int64_t)ky * nx + col;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) v[m1] = ok ? W[(N2 * m1 + r) * zs + base] : make_float2(0.f, 0.f);
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[(k1 * N2 + r) * TX + lane] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(r * N2 + m2) * TX + lane];
        fft4_phase2<N1, N2, false>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) u[k2] = cscale(u[k2], mask_fo[(r + N1 * k2) * ny + ky]);
        RegFft<N2, true>::run(u, tws, N1);
#pragma unroll
        for (int m2 = 1; m2 < N2; ++m2) {
            float2 w = tws[m2 * r];
            w.y = -w.y;
            u[m2] = cmul(u[m2], w);
        }
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) Y[(r * N2 + m2) * TX + lane] = u[m2];
    }
    __syncthreads();
    if (r < N2 && ok) {
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = Y[(k1 * N2 + r) * TX + lane];
        RegFft<N1, true>::run(v, tws, N2);
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) W[(N2 * m1 + r) * zs + base] = v[m1];
    }
}

template <int N2, int TX>
__global__ void __launch_bounds__(TX * tpr<N2>())
c3_ypass_inv_kernel(const float2* __restrict__ tw, const float2* __restrict__ W,
                    const float2* __restrict__ S, float2* out, int nx, int x0, int first, int last,
                    float scale, const float2* operand, float alpha) {
    constexpr int n = N1 * N2;
    __shared__ float2 tws[n];
    __shared__ float2 Y[N1 * N2 * TX];
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    const int lane = threadIdx.x % TX, r = threadIdx.x / TX;
    const int col = x0 + blockIdx.x * TX + lane;
    const bool ok = col < nx;
    const int64_t plane = (int64_t)blockIdx.y * n * nx;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1)
            v[m1] = ok ? W[plane + (int64_t)(N2 * m1 + r) * nx + col] : make_float2(0.f, 0.f);
        fft4_phase1<N1, N2, true>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[(k1 * N2 + r) * TX + lane] = v[k1];
    }
    __syncthreads();
    if (r < N1 && ok) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(r * N2 + m2) * TX + lane];
        fft4_phase2<N1, N2, true>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int64_t o = plane + (int64_t)(r + N1 * k2) * nx + col;
            float2 v = cmulc(S[o], u[k2]);
            if (!first) v = cadd(v, out[o]);
            if (last) {
                v = cscale(v, scale);
                if (operand) v = cadd(v, cscale(operand[o], alpha));
            }
            out[o] = v;
        }
    }
}

}  // namespace

extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

static pp_status check4(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    if (g_profiler) g_profiler->mark(what);
    return PP_OK;
}

// Returns PP_UNSUPPORTED-free status; *done = false when n has no fast kernel.
pp_status launch_cols4(const DevFft& f, const ColArgs& a, const float2* src, float2* dst, bool inv,
                       cudaStream_t st, bool* done) {
    *done = false;
    const int n2 = fft4_n2(a.G);
    if (!n2) return PP_OK;
    dim3 grid((a.ncols + TXF - 1) / TXF, a.nbatch);
#define PP_C4(N2_)                                                                                 \
    if (n2 == N2_) {                                                                               \
        const int thr = TXF * tpr<N2_>();                                                          \
        if (inv) cols4_kernel<N2_, true><<<grid, thr, 0, st>>>(f.tw, a, src, dst);                 \
        else cols4_kernel<N2_, false><<<grid, thr, 0, st>>>(f.tw, a, src, dst);                    \
    }
    PP_C4(8) PP_C4(12) PP_C4(16) PP_C4(20) PP_C4(24)
#undef PP_C4
    *done = true;
    return check4("cols4_kernel");
}

pp_status launch_rows4_fwd(const DevFft& f, const RowArgs& a, const float2* x, const float2* sens,
                           const float* wrow, const float* wcol, float2* out, int ncoils,
                           int64_t img_batch_stride, cudaStream_t st, bool* done) {
    *done = false;
    const int n2 = fft4_n2(a.G);
    if (!n2) return PP_OK;
    dim3 grid((a.nrows + RBF - 1) / RBF, ncoils);
#define PP_R4(N2_)                                                                                  \
    if (n2 == N2_)                                                                                  \
        rows4_fwd_kernel<N2_><<<grid, RBF * tpr<N2_>(), 0, st>>>(f.tw, a, x, img_batch_stride, sens, \
                                                                 wrow, wcol, out);
    PP_R4(8) PP_R4(12) PP_R4(16) PP_R4(20) PP_R4(24)
#undef PP_R4
    *done = true;
    return check4("rows4_fwd_kernel");
}

pp_status launch_rows4_adj(const DevFft& f, const RowArgs& a, const float2* src, const float2* sens,
                           const float* wrow, const float* wcol, float2* out, const float2* operand,
                           float alpha, int ncoils, cudaStream_t st, bool* done, int cluster) {
    *done = false;
    const int n2 = fft4_n2(a.G);
    if (!n2 || a.n > 512 || ncoils < 4) return PP_OK;
    const int ngroups = (ncoils + RBF - 1) / RBF;
    int CL = cluster > 0 ? cluster : 1;
    while (CL > 1 && CL > ngroups) CL >>= 1;
    if (CL > 1) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(a.nrows * CL);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaSuccess;
#define PP_CL4(N2_)                                                                              \
        if (n2 == N2_) {                                                                         \
            cfg.blockDim = dim3(RBF * tpr<N2_>());                                               \
            e = cudaLaunchKernelEx(&cfg, rows4_adj_cl_kernel<N2_>, f.tw, a, src, sens, wrow, wcol, \
                                   out, operand, alpha, ncoils);                                  \
        }
        PP_CL4(8) PP_CL4(12) PP_CL4(16) PP_CL4(20) PP_CL4(24)
#undef PP_CL4
        if (e != cudaSuccess) return cuda_status(e, "rows4_adj_cl_kernel launch");
        *done = true;
        return check4("rows4_adj_cl_kernel");
    }
#define PP_A4(N2_)                                                                                 \
    if (n2 == N2_)                                                                                 \
        rows4_adj_kernel<N2_><<<a.nrows, RBF * tpr<N2_>(), 0, st>>>(f.tw, a, src, sens, wrow, wcol, \
                                                                    out, operand, alpha, ncoils);
    PP_A4(8) PP_A4(12) PP_A4(16) PP_A4(20) PP_A4(24)
#undef PP_A4
    *done = true;
    return check4("rows4_adj_kernel");
}

pp_status prepare_cart4() {
#define PP_P4(N2_)                                                                                \
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d4_normal_kernel<N2_>,                                  \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                                     (int)cart4_dyn_smem<N2_>()));
    PP_P4(8) PP_P4(12) PP_P4(16) PP_P4(20) PP_P4(24)
#undef PP_P4
#define PP_P4C(N2_)                                                                               \
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d4_cluster_kernel<N2_>,                                 \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                                     (int)cart4_dyn_smem<N2_>()));
    PP_P4C(8) PP_P4C(12) PP_P4C(16) PP_P4C(20) PP_P4C(24)
#undef PP_P4C
    return PP_OK;
}

pp_status launch_cart2d4_normal(const Plan& p, const float2* x, float2* out, float scale,
                                const float2* operand, float alpha, cudaStream_t st, bool* done) {
    *done = false;
    const int n2 = fft4_n2(p.ny);
    if (!n2) return PP_OK;
    const int grid = (p.nx + 7) / 8;
    const int CL = p.tune_c2;
    if (CL == 2 || CL == 4 || CL == 8) {
        cudaError_t e = cudaSuccess;
#define PP_K4C(N2_)                                                                              \
        if (n2 == N2_)                                                                           \
            e = launch_ex(cart2d4_cluster_kernel<N2_>, dim3(grid * CL), dim3(8 * tpr<N2_>()),    \
                          cart4_dyn_smem<N2_>(), st, false, CL, (const float2*)p.fy.tw, x,       \
                          (const float2*)p.sens, p.C, p.nx, (const float*)p.mask_fo, out, scale, \
                          operand, alpha);
        PP_K4C(8) PP_K4C(12) PP_K4C(16) PP_K4C(20) PP_K4C(24)
#undef PP_K4C
        if (e != cudaSuccess) return cuda_status(e, "cart2d4_cluster_kernel launch");
        *done = true;
        return check4("cart2d4_cluster_kernel");
    }
#define PP_K4(N2_)                                                                                 \
    if (n2 == N2_)                                                                                 \
        cart2d4_normal_kernel<N2_><<<grid, 8 * tpr<N2_>(), cart4_dyn_smem<N2_>(), st>>>(           \
            p.fy.tw, x, p.sens, p.C, p.nx, p.mask_fo, out, scale, operand, alpha);
    PP_K4(8) PP_K4(12) PP_K4(16) PP_K4(20) PP_K4(24)
#undef PP_K4
    *done = true;
    return check4("cart2d4_normal_kernel");
}

template <int N2>
static void c3_yf(int tx, dim3 g, cudaStream_t st, const float2* tw, const float2* x, const float2* S,
                  float2* W, int nx, int x0) {
    if constexpr (N2 <= 16) {
        if (tx == 16) {
            c3_ypass_fwd_kernel<N2, 16><<<g, 16 * tpr<N2>(), 0, st>>>(tw, x, S, W, nx, x0);
            return;
        }
    }
    c3_ypass_fwd_kernel<N2, 8><<<g, 8 * tpr<N2>(), 0, st>>>(tw, x, S, W, nx, x0);
}
template <int N2>
static void c3_z(int tx, dim3 g, cudaStream_t st, const float2* tw, float2* W, const float* m, int ny,
                 int nx, int x0) {
    if constexpr (N2 <= 16) {
        if (tx == 16) {
            c3_zpass_kernel<N2, 16><<<g, 16 * tpr<N2>(), 0, st>>>(tw, W, m, ny, nx, x0);
            return;
        }
    }
    c3_zpass_kernel<N2, 8><<<g, 8 * tpr<N2>(), 0, st>>>(tw, W, m, ny, nx, x0);
}
template <int N2>
static void c3_yi(int tx, dim3 g, cudaStream_t st, const float2* tw, const float2* W, const float2* S,
                  float2* out, int nx, int x0, int first, int last, float scale, const float2* op,
                  float alpha) {
    if constexpr (N2 <= 16) {
        if (tx == 16) {
            c3_ypass_inv_kernel<N2, 16><<<g, 16 * tpr<N2>(), 0, st>>>(tw, W, S, out, nx, x0, first, last,
                                                                      scale, op, alpha);
            return;
        }
    }
    c3_ypass_inv_kernel<N2, 8><<<g, 8 * tpr<N2>(), 0, st>>>(tw, W, S, out, nx, x0, first, last, scale,
                                                            op, alpha);
}

// 3-D normal operator on L2-sized x-blocks (see the kernels above); false
// in *done when ny or nz has no register FFT.
pp_status cart3d4_normal(const Plan& p, const float2* x, float2* out, float scale,
                         const float2* operand, float alpha, float2* W, cudaStream_t st, bool* done) {
    *done = false;
    const int ny2 = fft4_n2(p.ny), nz2 = fft4_n2(p.nz);
    if (!ny2 || !nz2) return PP_OK;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    // x-block width: x, W, out and one coil map of the block within ~64 MB
    int wb = (int)((64ll << 20) / (4ll * 8 * ny * nz));
    wb = std::max(8, std::min(nx, (wb / 8) * 8));
    const int64_t n = p.nimg;
    for (int x0 = 0; x0 < nx; x0 += wb) {
        const int w = std::min(wb, nx - x0);
        // 16 columns per CTA (whole 128-byte lines of the maps) when the
        // shared tile fits the static limit, else 8
        const int tyx = ny2 <= 16 ? 16 : 8, tzx = nz2 <= 16 ? 16 : 8;
        const dim3 gy((w + tyx - 1) / tyx, nz), gz((w + tzx - 1) / tzx, ny);
        for (int c = 0; c < p.C; ++c) {
            const float2* S = p.sens + (int64_t)c * n;
#define PP_Y(N2_) if (ny2 == N2_) c3_yf<N2_>(tyx, gy, st, p.fy.tw, x, S, W, nx, x0);
            PP_Y(8) PP_Y(12) PP_Y(16) PP_Y(20) PP_Y(24)
#undef PP_Y
            PP_TRY(check4("c3_ypass_fwd_kernel"));
#define PP_Z(N2_) if (nz2 == N2_) c3_z<N2_>(tzx, gz, st, p.fz.tw, W, p.mask_fo, ny, nx, x0);
            PP_Z(8) PP_Z(12) PP_Z(16) PP_Z(20) PP_Z(24)
#undef PP_Z
            PP_TRY(check4("c3_zpass_kernel"));
            const int first = c == 0, last = c == p.C - 1;
#define PP_I(N2_) if (ny2 == N2_) c3_yi<N2_>(tyx, gy, st, p.fy.tw, W, S, out, nx, x0, first, last, scale, operand, alpha);
            PP_I(8) PP_I(12) PP_I(16) PP_I(20) PP_I(24)
#undef PP_I
            PP_TRY(check4("c3_ypass_inv_kernel"));
        }
    }
    *done = true;
    return PP_OK;
}

pp_status launch_rows4_adj_split(const DevFft& f, const RowArgs& a, const float2* src,
                                 const float2* sens, const float* wrow, const float* wcol,
                                 float2* contrib, float2* out, const float2* operand, float alpha,
                                 int ncoils, cudaStream_t st, bool* done) {
    *done = false;
    const int n2 = fft4_n2(a.G);
    if (!n2 || !sens || !contrib) return PP_OK;
    dim3 grid((a.nrows + RBF - 1) / RBF, ncoils);
#define PP_S4(N2_)                                                                              \
    if (n2 == N2_)                                                                              \
        rows4_inv_kernel<N2_><<<grid, RBF * tpr<N2_>(), 0, st>>>(f.tw, a, src, sens, wrow, wcol, \
                                                                 contrib);
    PP_S4(8) PP_S4(12) PP_S4(16) PP_S4(20) PP_S4(24)
#undef PP_S4
    PP_TRY(check4("rows4_inv_kernel"));
    const int64_t n = (int64_t)a.nrows * a.n;
    int64_t blocks = (n + 63) / 64;
    if (blocks > 152 * 16) blocks = 152 * 16;
    coil_sum_kernel<<<(int)blocks, 256, 0, st>>>(contrib, ncoils, n, a.scale, operand, alpha, out);
    PP_TRY(check4("coil_sum_kernel"));
    *done = true;
    return PP_OK;
}

}  // namespace pp
