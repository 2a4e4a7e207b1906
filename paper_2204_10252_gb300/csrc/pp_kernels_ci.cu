// Coil-innermost pipeline of the non-Cartesian normal operator (Sec. 5.2):
//   out = scale * sum_c conj(S_c) D F^H G^T G F D (S_c x) + alpha * operand
// with every per-coil array stored as [row][col][coil] and the coil count
// padded to CP = 32.  The row and column FFT stages run one transform per
// (line, coil) with the 8 coils of a CTA in adjacent lanes, so every global
// access is a 64-byte coil run; the G^T G stencil puts the 32 coils of one
// grid point in the 32 lanes of a warp, so each stencil weight is a single
// shared-memory broadcast and each halo row a contiguous copy; the row IFFT
// reduces its 8 coils in shared memory and leaves one partial sum per CTA.
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
constexpr int CB = 8;    // coils per CTA in the FFT stages
constexpr int CP = 32;   // coil pitch of the coil-innermost arrays
constexpr int NCB = CP / CB;

template <int N2> __host__ __device__ constexpr int tpr() { return N2 > N1 ? N2 : N1; }
// k1 pitch of the transpose buffer Y[k1][m2][coil]: an odd multiple of 8
// float2 apart, so the two k1 rows of a half-warp fall on disjoint banks
template <int N2> __host__ __device__ constexpr int ypitch() { return N2 * CB + 8; }
template <int N2> __host__ __device__ constexpr int min_ctas() { return N2 == 20 ? 7 : 1; }

__device__ __forceinline__ int wrap1(int a, int G) { return a < 0 ? a + G : (a >= G ? a - G : a); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// S_ci[(y nx + x) CP + c] = S[c][y][x] (zero for c >= C)
__global__ void ci_pack_sens_kernel(const float2* __restrict__ S, int C, int64_t n,
                                    float2* __restrict__ Sci) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * CP;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % CP);
        const int64_t o = e / CP;
        Sci[e] = c < C ? S[c * n + o] : make_float2(0.f, 0.f);
    }
}

// Row stage image -> k rows: A[row][q][c] = F_G(place(w S_c x[row]))[q].
// grid (nrows, NCB), block CB * tpr(N2); lane j = threadIdx % 8 is the coil.
template <int N2>
__global__ void __launch_bounds__(CB * tpr<N2>(), min_ctas<N2>())
ci_rows_fwd_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ x,
                   const float2* __restrict__ S, const float* __restrict__ wrow,
                   const float* __restrict__ wcol, float2* __restrict__ out) {
    constexpr int n = N1 * N2, YP = ypitch<N2>();
    static_assert(N1 * YP >= n * CB, "the coil-map row must fit the transpose buffer");
    __shared__ float2 tws[n];
    __shared__ __align__(16) float2 Y[N1 * YP];
    pdl_trigger();
    const int row = blockIdx.x;
    // The CTA's 8-coil run of the map row (a plan constant) streams into Y
    // while the previous kernel finishes: Ss[i * 8 + j] = S_ci[row][i][cb * 8 + j].
    float2* Ss = Y;
    {
        const float2* Srow = S + (int64_t)row * a.n * CP + blockIdx.y * CB;
        for (int e = threadIdx.x; e < a.n * 4; e += blockDim.x) {
            const int i = e >> 2, q = e & 3;
            cp_async16(Ss + i * CB + 2 * q, Srow + (int64_t)i * CP + 2 * q, true);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    pdl_wait();
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int j = threadIdx.x & (CB - 1), r = threadIdx.x / CB;
    const int c = blockIdx.y * CB + j;
    float2 v[N1];
    if (r < N2) {
        const float wr = a.scale * (wrow ? wrow[row] : 1.f);
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int i = N2 * m1 + r + a.off_in;
            if (i >= n) i -= n;
            float2 val = make_float2(0.f, 0.f);
            if (i < a.n) {
                const int64_t o = (int64_t)row * a.n + i;
                val = cscale(cmul(x[o], Ss[i * CB + j]), wcol ? wr * wcol[i] : wr);
            }
            v[m1] = val;
        }
    }
    __syncthreads();   // Ss (aliasing Y) is consumed
    if (r < N2) {
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, false>(u, tws);
        float2* orow = out + (int64_t)row * n * CP + c;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            int q = r + N1 * k2 + a.off_out;
            if (q >= n) q -= n;
            orow[(int64_t)q * CP] = u[k2];
        }
    }
}

// Column stage along rows of [H][Gx][CP]: input row (p + off_in) mod n of
// transform position p (zero at or past Hin), output position k at row
// (k + off_out) mod n when below Hout.  grid (Gx, NCB), block CB * tpr(N2).
template <int N2, bool INV>
__global__ void __launch_bounds__(CB * tpr<N2>(), min_ctas<N2>())
ci_cols_kernel(const float2* __restrict__ tw, int Hin, int Hout, int off_in, int off_out, int Gx,
               const float2* __restrict__ src, float2* __restrict__ dst) {
    constexpr int n = N1 * N2, YP = ypitch<N2>();
    __shared__ float2 tws[n];
    __shared__ float2 Y[N1 * YP];
    pdl_trigger();
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    pdl_wait();
    const int j = threadIdx.x & (CB - 1), r = threadIdx.x / CB;
    const int64_t rs = (int64_t)Gx * CP;
    const int64_t cofs = (int64_t)blockIdx.x * CP + blockIdx.y * CB + j;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int row = N2 * m1 + r + off_in;
            if (row >= n) row -= n;
            v[m1] = row < Hin ? src[row * rs + cofs] : make_float2(0.f, 0.f);
        }
        fft4_phase1<N1, N2, INV>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, INV>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            int q = r + N1 * k2 + off_out;
            if (q >= n) q -= n;
            if (q < Hout) dst[q * rs + cofs] = u[k2];
        }
    }
}

// G^T G stencil on [Gy][Gx][CP] grids: out_j = sum_d T[d][j] in_{j + delta_d}
// (periodic).  A CTA owns a 16 x (4 RY) output tile; warp w covers the 8
// columns 8 (w & 1) .. and the RY rows (w >> 1) RY .. of it, lane = coil.
// cp.async stages the halo rows (contiguous [col][coil] runs) and the tile's
// weights from the [row][col/8][tap][8] copy.
template <int RY> struct CiStencil {
    static constexpr int TX = 16, TY = 4 * RY, HX = TX + 6, HY = TY + 6;
    static constexpr size_t HALO = sizeof(float2) * HY * HX * CP;
    static constexpr size_t SMEM = HALO + sizeof(float) * TY * TX * 49;
};

template <int RY>
__global__ void __launch_bounds__(256)
ci_stencil_kernel(const float* __restrict__ T8, int Gx, int Gy, int nxb,
                  const float2* __restrict__ in, float2* __restrict__ out) {
    using S = CiStencil<RY>;
    constexpr int TX = S::TX, TY = S::TY, HX = S::HX, HY = S::HY, D = 7, H = 3;
    extern __shared__ float4 sm4[];
    float2* halo = reinterpret_cast<float2*>(sm4);
    float4* wts = sm4 + S::HALO / sizeof(float4);
    const int ntx = (Gx + TX - 1) / TX;
    const int tx0 = (blockIdx.x % ntx) * TX, ty0 = (blockIdx.x / ntx) * TY;
    pdl_trigger();
    // weights: per tile row, blocks xb0 and xb0 + 1 are 2 x 49 x 8 contiguous floats
    const int xb0 = tx0 / 8;
    for (int e = threadIdx.x; e < TY * 196; e += blockDim.x) {
        const int yy = e / 196, rem = e - yy * 196, s = rem / 98;
        const int y = ty0 + yy;
        const bool ok = y < Gy && xb0 + s < nxb;
        cp_async16(wts + e, T8 + (ok ? ((int64_t)y * nxb + xb0) * 392 + rem * 4 : 0), ok);
    }
    pdl_wait();
    // halo: HY rows of HX points x 32 coils = 16 sixteen-byte chunks per point
    for (int e = threadIdx.x; e < HY * HX * 16; e += blockDim.x) {
        const int hp = e >> 4, q = e & 15;
        const int hy = hp / HX, hx = hp - hy * HX;
        const int gy = wrap1(ty0 - H + hy, Gy), gx = wrap1(tx0 - H + hx, Gx);
        cp_async16(halo + (size_t)hp * CP + 2 * q, in + ((int64_t)gy * Gx + gx) * CP + 2 * q, true);
    }
    cp_async_commit_wait_all();
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, s = w & 1, yb = (w >> 1) * RY;
    float2 acc[RY][8];
#pragma unroll
    for (int ry = 0; ry < RY; ++ry)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[ry][r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < RY + D - 1; ++i) {
        const float2* hrow = halo + ((yb + i) * HX + 8 * s) * CP + lane;
        float2 xv[14];
#pragma unroll
        for (int jx = 0; jx < 14; ++jx) xv[jx] = hrow[jx * CP];
#pragma unroll
        for (int ry = 0; ry < RY; ++ry) {
            const int dy = i - ry;
            if (dy < 0 || dy >= D) continue;
            const float4* wq = wts + ((yb + ry) * 2 + s) * 98 + dy * 14;
#pragma unroll
            for (int dx = 0; dx < D; ++dx) {
                const float4 wa = wq[2 * dx], wb = wq[2 * dx + 1];
                const float wr[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)   // packed two-lane FP32 FMA (re, im)
                    acc[ry][r] = __ffma2_rn(make_float2(wr[r], wr[r]), xv[r + dx], acc[ry][r]);
            }
        }
    }
#pragma unroll
    for (int ry = 0; ry < RY; ++ry) {
        const int gy = ty0 + yb + ry;
        if (gy >= Gy) continue;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int gx = tx0 + 8 * s + r;
            if (gx < Gx) out[((int64_t)gy * Gx + gx) * CP + lane] = acc[ry][r];
        }
    }
}

// Tail of the cluster row-IFFT kernels: every CTA of the row's 4-CTA cluster
// holds its coil block's partial row in Y[i * 9 + 8]; CTA q sums the four
// partials of its quarter [q n/4, (q + 1) n/4) through distributed shared
// memory and writes scale * sum + alpha * operand.  The cluster barrier is
// split: the release-arrive publishes this CTA's partials, and the operand
// of the quarter (written by earlier kernels, independent of the cluster) is
// loaded before the acquire-wait.  The closing barrier only keeps the
// partials alive until every CTA has read them; its arrive is relaxed (the
// remote loads have fed the stores before it).
__device__ __forceinline__ void cluster_row_sum(const float2* Y, int n, int row, int q, float scale,
                                                const float2* operand, float alpha, float2* out) {
    namespace cgx = cooperative_groups;
    cgx::cluster_group cluster = cgx::this_cluster();
    cluster_arrive_release();
    const int chunk = (n + NCB - 1) / NCB;
    const int i0 = q * chunk, i1 = min(n, i0 + chunk);
    const int ifirst = i0 + (int)threadIdx.x;
    float2 op0 = make_float2(0.f, 0.f);
    if (operand && ifirst < i1) op0 = operand[(int64_t)row * n + ifirst];
    cluster_wait_acquire();
    for (int i = ifirst; i < i1; i += blockDim.x) {
        float2 v = cluster.map_shared_rank(Y, 0)[i * 9 + 8];
#pragma unroll
        for (int b = 1; b < NCB; ++b) v = cadd(v, cluster.map_shared_rank(Y, b)[i * 9 + 8]);
        v = cscale(v, scale);
        const int64_t o = (int64_t)row * n + i;
        if (operand) v = cadd(v, cscale(i == ifirst ? op0 : operand[o], alpha));
        out[o] = v;
    }
    cluster_arrive_relaxed();
    cluster_wait_acquire();
}

// Row stage k rows -> image with the coil reduction of one coil block:
// P[cb][row][i] = sum_{c in block cb} w conj(S_c) IFFT(src_c[row])[place(i)].
template <int N2> __host__ __device__ constexpr int inv_buf() {
    return N1 * ypitch<N2>() > N1 * N2 * 9 ? N1 * ypitch<N2>() : N1 * N2 * 9;
}

// Coil-pair variant of the coil-innermost stencil: lane = (segment h =
// lane / 16, coil pair cp = lane % 16), so a warp covers 16 adjacent outputs
// of one row for all 32 coils and each lane two coils of 8 outputs.  One
// 16-byte halo read serves both coils and each weight is duplicated once for
// two packed FMAs.  CTA: 16 x 8 output tile, one warp per row.
constexpr int CPS_TX = 16, CPS_TY = 8, CPS_HX = CPS_TX + 6, CPS_HY = CPS_TY + 6;
constexpr size_t CPS_HALO = sizeof(float2) * CPS_HY * CPS_HX * CP;
constexpr size_t CPS_SMEM = CPS_HALO + sizeof(float) * CPS_TY * CPS_TX * 49;

// Tiles whose 16 x 8 points carry no G^T G weight (grid points that no
// sample's kernel reaches: the corners outside the trajectory's disc) have an
// exactly zero output; tile_nz marks the others (null: every tile is live).
__global__ void __launch_bounds__(256)
ci_tile_flags_kernel(const float* __restrict__ T8, int Gx, int Gy, int nxb, int* __restrict__ tile_nz) {
    const int ntx = (Gx + CPS_TX - 1) / CPS_TX;
    const int tx0 = (blockIdx.x % ntx) * CPS_TX, ty0 = (blockIdx.x / ntx) * CPS_TY;
    const int xb0 = tx0 / 8;
    int any = 0;
    for (int e = threadIdx.x; e < CPS_TY * 784; e += blockDim.x) {
        const int yy = e / 784, rem = e - yy * 784, s = rem / 392;
        const int y = ty0 + yy;
        if (y < Gy && xb0 + s < nxb && T8[((int64_t)y * nxb + xb0) * 392 + rem] != 0.f) any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) tile_nz[blockIdx.x] = any;
}

__global__ void __launch_bounds__(256, 2)
ci_stencil_cp_kernel(const float* __restrict__ T8, int Gx, int Gy, int nxb, const int* __restrict__ tile_nz,
                     const float2* __restrict__ in, float2* __restrict__ out) {
    constexpr int D = 7, H = 3;
    extern __shared__ float4 sm4[];
    float4* halo4 = sm4;                                  // [hy][hx][16 coil pairs]
    float4* wts = sm4 + CPS_HALO / sizeof(float4);        // [row][2][49][2]
    const int ntx = (Gx + CPS_TX - 1) / CPS_TX;
    const int tx0 = (blockIdx.x % ntx) * CPS_TX, ty0 = (blockIdx.x / ntx) * CPS_TY;
    pdl_trigger();
    if (tile_nz && !tile_nz[blockIdx.x]) {
        // no weight in the tile: its output is zero (written once the
        // predecessor is done, like every other store of this kernel)
        pdl_wait();
        for (int e = threadIdx.x; e < CPS_TY * CPS_TX * 16; e += blockDim.x) {
            const int pt = e >> 4, q = e & 15;
            const int gy = ty0 + pt / CPS_TX, gx = tx0 + pt % CPS_TX;
            if (gy < Gy && gx < Gx)
                reinterpret_cast<float4*>(out)[((int64_t)gy * Gx + gx) * 16 + q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    const int xb0 = tx0 / 8;
    for (int e = threadIdx.x; e < CPS_TY * 196; e += blockDim.x) {
        const int yy = e / 196, rem = e - yy * 196, s = rem / 98;
        const int y = ty0 + yy;
        const bool ok = y < Gy && xb0 + s < nxb;
        cp_async16(wts + e, T8 + (ok ? ((int64_t)y * nxb + xb0) * 392 + rem * 4 : 0), ok);
    }
    pdl_wait();
    {
        // thread = (column group g, coil pair q): columns g and g + 16 of every halo row
        const int q = threadIdx.x & 15, g = threadIdx.x >> 4;
        const int gx0 = wrap1(tx0 - H + g, Gx);
        const int gx1 = g + 16 < CPS_HX ? wrap1(tx0 - H + g + 16, Gx) : 0;
        for (int hy = 0; hy < CPS_HY; ++hy) {
            const float2* row = in + (int64_t)wrap1(ty0 - H + hy, Gy) * Gx * CP + 2 * q;
            cp_async16(halo4 + (hy * CPS_HX + g) * 16 + q, row + (int64_t)gx0 * CP, true);
            if (g + 16 < CPS_HX)
                cp_async16(halo4 + (hy * CPS_HX + g + 16) * 16 + q, row + (int64_t)gx1 * CP, true);
        }
    }
    cp_async_commit_wait_all();
    __syncthreads();
    const int yy = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, cp = lane & 15;
    const float4* wq = wts + (yy * 2 + h) * 98;
    float2 a0[8], a1[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a0[r] = a1[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int dy = 0; dy < D; ++dy) {
        const float4* hrow = halo4 + ((yy + dy) * CPS_HX + 8 * h) * 16 + cp;
        float4 xv[14];
#pragma unroll
        for (int j = 0; j < 14; ++j) xv[j] = hrow[j * 16];
#pragma unroll
        for (int dx = 0; dx < D; ++dx) {
            const float4 wa = wq[(dy * D + dx) * 2], wb = wq[(dy * D + dx) * 2 + 1];
            const float wr[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2 wd = make_float2(wr[r], wr[r]);
                const float4 v = xv[r + dx];
                a0[r] = __ffma2_rn(wd, make_float2(v.x, v.y), a0[r]);
                a1[r] = __ffma2_rn(wd, make_float2(v.z, v.w), a1[r]);
            }
        }
    }
    const int gy = ty0 + yy;
    if (gy < Gy) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int gx = tx0 + 8 * h + r;
            if (gx < Gx)
                reinterpret_cast<float4*>(out)[((int64_t)gy * Gx + gx) * 16 + cp] =
                    make_float4(a0[r].x, a0[r].y, a1[r].x, a1[r].y);
        }
    }
}

// Body shared by both row-IFFT kernels: leaves R[i * 9 + j] = w conj(S_c)
// IFFT(src_c[row])[place(i)] for the CTA's 8 coils c = cb * 8 + j, and
// R[i * 9 + 8] = their sum (i < a.n); ends with a barrier.
template <int N2>
__device__ __forceinline__ void ci_rows_inv_body(const float2* __restrict__ tw, const RowArgs& a,
                                                 const float2* __restrict__ src,
                                                 const float2* __restrict__ S,
                                                 const float* __restrict__ wrow,
                                                 const float* __restrict__ wcol, int row, int cb,
                                                 float2* tws, float2* Y) {
    constexpr int n = N1 * N2, YP = ypitch<N2>();
    pdl_trigger();
    {
        // pull the CTA's 8-coil runs of the map row (a plan constant, read in
        // the epilogue) into L2 while the previous kernel finishes: one
        // 64-byte run, inside one 128-byte line, per image column
        const float2* Srow = S + (int64_t)row * a.n * CP + cb * CB;
        for (int i = threadIdx.x; i < a.n; i += blockDim.x)
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(Srow + (int64_t)i * CP));
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    __syncthreads();
    pdl_wait();
    const int j = threadIdx.x & (CB - 1), r = threadIdx.x / CB;
    const int c = cb * CB + j;
    if (r < N2) {
        float2 v[N1];
        const float2* srow = src + (int64_t)row * n * CP + c;
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int sidx = N2 * m1 + r + a.off_in;
            if (sidx >= n) sidx -= n;
            v[m1] = srow[(int64_t)sidx * CP];
        }
        fft4_phase1<N1, N2, true>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    float2 u[N2];
    if (r < N1) {
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, true>(u, tws);
    }
    __syncthreads();   // Y is reused below as R[i][9]
    float2* R = Y;
    if (r < N1) {
        const float wr = a.scale * (wrow ? wrow[row] : 1.f);
        const float2* srow = S + (int64_t)row * a.n * CP + c;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            int i = r + N1 * k2 + a.off_out;
            if (i >= n) i -= n;
            if (i < a.n)
                R[i * 9 + j] = cmulc(srow[(int64_t)i * CP], cscale(u[k2], wcol ? wr * wcol[i] : wr));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
        float2 acc = R[i * 9];
#pragma unroll
        for (int jj = 1; jj < CB; ++jj) acc = cadd(acc, R[i * 9 + jj]);
        R[i * 9 + 8] = acc;
    }
    __syncthreads();
}

// Row stage k rows -> image, one coil block per CTA:
// P[cb][row][i] = sum_{c in block cb} w conj(S_c) IFFT(src_c[row])[place(i)].
// grid (nrows, NCB).
template <int N2>
__global__ void __launch_bounds__(CB * tpr<N2>(), min_ctas<N2>())
ci_rows_inv_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ src,
                   const float2* __restrict__ S, const float* __restrict__ wrow,
                   const float* __restrict__ wcol, float2* __restrict__ P) {
    __shared__ float2 tws[N1 * N2];
    __shared__ float2 Y[inv_buf<N2>()];
    const int row = blockIdx.x, cb = blockIdx.y;
    ci_rows_inv_body<N2>(tw, a, src, S, wrow, wcol, row, cb, tws, Y);
    float2* prow = P + ((int64_t)cb * a.nrows + row) * a.n;
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) prow[i] = Y[i * 9 + 8];
}

// The same with the NCB coil blocks of a row in one thread-block cluster:
// CTA q of the cluster sums the four blocks' partials for its quarter of the
// row through distributed shared memory (fixed order) and writes
// out = scale * sum + alpha * operand.  grid (NCB, nrows), cluster (NCB, 1, 1).
template <int N2>
__global__ void __launch_bounds__(CB * tpr<N2>(), min_ctas<N2>())
ci_rows_inv_cl_kernel(const float2* __restrict__ tw, RowArgs a, const float2* __restrict__ src,
                      const float2* __restrict__ S, const float* __restrict__ wrow,
                      const float* __restrict__ wcol, float2* out, float scale,
                      const float2* operand, float alpha) {
    __shared__ float2 tws[N1 * N2];
    __shared__ float2 Y[inv_buf<N2>()];
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int row = blockIdx.y;
    ci_rows_inv_body<N2>(tw, a, src, S, wrow, wcol, row, q, tws, Y);
    cluster_row_sum(Y, a.n, row, q, scale, operand, alpha, out);
}

// out[o] = scale * sum_b P[b][o] + alpha * operand[o]
__global__ void ci_sum_kernel(const float2* __restrict__ P, int64_t n, float scale,
                              const float2* operand, float alpha, float2* out) {
    pdl_trigger();
    pdl_wait();
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        float2 acc = P[o];
#pragma unroll
        for (int b = 1; b < NCB; ++b) acc = cadd(acc, P[b * n + o]);
        acc = cscale(acc, scale);
        if (operand) acc = cadd(acc, cscale(operand[o], alpha));
        out[o] = acc;
    }
}

// Column stage of the Toeplitz-embedded normal operator: for column q of
// the [H][M][CP] row-transformed array, the length-n (= 2H) column transform,
// the product with the embedded kernel's spectrum Tc[q][k] (real, the
// 1/(n_img M) normalisation folded in), and the inverse transform, in
// registers: forward phase 1 by (m2, coil) threads, phase 2 by (k1, coil)
// threads, then the mirrored inverse (input k = k1 + 16 k2, output
// m = N2 m1 + m2): inverse length-N2 DFT over k2 and W_n^(-m2 k1) by the
// same (k1) threads, inverse length-16 DFT over k1 by the (m2) threads.
// Rows: transform position p <-> row (p + off) mod n, stored when below H.
// grid (M, coil blocks), block CB * tpr(N2).
template <int N2>
__global__ void __launch_bounds__(CB * tpr<N2>(), 1)
toep_cols_kernel(const float2* __restrict__ tw, const float* __restrict__ Tc, int H, int off, int M,
                 const float2* __restrict__ src, float2* __restrict__ dst) {
    constexpr int n = N1 * N2, YP = ypitch<N2>();
    __shared__ float2 tws[n];
    __shared__ float Ts[n];
    __shared__ float2 Y[N1 * YP];
    pdl_trigger();
    // twiddles and this column's kernel spectrum are plan constants
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        Ts[i] = Tc[(int64_t)blockIdx.x * n + i];
    }
    __syncthreads();
    pdl_wait();
    const int j = threadIdx.x & (CB - 1), r = threadIdx.x / CB;
    const int64_t rs = (int64_t)M * CP;
    const int64_t cofs = (int64_t)blockIdx.x * CP + blockIdx.y * CB + j;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int row = N2 * m1 + r + off;
            if (row >= n) row -= n;
            v[m1] = row < H ? src[row * rs + cofs] : make_float2(0.f, 0.f);
        }
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Y[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, false>(u, tws);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) u[k2] = cscale(u[k2], Ts[r + N1 * k2]);
        RegFft<N2, true>::run(u, tws, N1);
#pragma unroll
        for (int m2 = 1; m2 < N2; ++m2) {
            float2 w = tws[m2 * r];
            w.y = -w.y;
            u[m2] = cmul(u[m2], w);
        }
        // the same (k1, coil) slots this thread read: no other thread touches them
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) Y[r * YP + m2 * CB + j] = u[m2];
    }
    __syncthreads();
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = Y[k1 * YP + r * CB + j];
        RegFft<N1, true>::run(v, tws, N2);
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            int q = N2 * m1 + r + off;
            if (q >= n) q -= n;
            if (q < H) dst[q * rs + cofs] = v[m1];
        }
    }
}

// Toeplitz row stages on length-n halves.  The row of the M = 2n embedding
// holds the n image samples at positions [-n/2, n/2) mod M and zeros
// elsewhere, so its length-M DFT splits into two length-n DFTs of the folded
// row y[p] = x[(p + n/2) mod n] (p < n):
//   X[2k]     = FFT_n(y)[k],
//   X[2k + 1] = FFT_n(s W_M^p y)[k],   s = +1 for p < n/2, -1 above,
// and, mirrored, the cropped inverse is
//   v[p] = IFFT_n(X[2k])[p] + s(p) W_M^(-p) IFFT_n(X[2k + 1])[p],
// with image sample (p + n/2) mod n.  Each CTA runs both halves for its 8
// coils at once (thread group par = 0 even, 1 odd), on the balanced
// register four-step of length n = 16 N2.
template <int N2> __host__ __device__ constexpr int half_threads() { return 2 * CB * tpr<N2>(); }

// A[row][k][c] = FFT_M(place(S_c x[row]))[k] for the CTA's 8 coils.
// grid (ny, coil blocks), block half_threads.
template <int N2>
__global__ void __launch_bounds__(half_threads<N2>())
toep_rows_fwd_half_kernel(const float2* __restrict__ tw, const float2* __restrict__ twM,
                          const float2* __restrict__ x, const float2* __restrict__ S,
                          float2* __restrict__ out) {
    constexpr int n = N1 * N2, YP = ypitch<N2>(), T = CB * tpr<N2>(), M = 2 * n;
    static_assert(2 * N1 * YP >= n * CB, "the coil-map row must fit the transpose buffers");
    __shared__ float2 tws[n], twm[n];
    __shared__ __align__(16) float2 Y[2 * N1 * YP];
    pdl_trigger();
    const int row = blockIdx.x;
    float2* Ss = Y;   // Ss[i * 8 + j] = S_ci[row][i][cb * 8 + j], streamed in before the wait
    {
        const float2* Srow = S + (int64_t)row * n * CP + blockIdx.y * CB;
        for (int e = threadIdx.x; e < n * 4; e += blockDim.x) {
            const int i = e >> 2, q = e & 3;
            cp_async16(Ss + i * CB + 2 * q, Srow + (int64_t)i * CP + 2 * q, true);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        twm[i] = twM[i];
    }
    pdl_wait();
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int par = threadIdx.x / T, t = threadIdx.x - par * T, j = t & (CB - 1), r = t / CB;
    const int c = blockIdx.y * CB + j;
    float2 v[N1];
    if (r < N2) {
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + r;
            int i = p + n / 2;
            if (i >= n) i -= n;
            float2 val = cmul(x[(int64_t)row * n + i], Ss[i * CB + j]);
            if (par) {
                float2 w = twm[p];
                if (p >= n / 2) w = make_float2(-w.x, -w.y);
                val = cmul(val, w);
            }
            v[m1] = val;
        }
    }
    __syncthreads();   // Ss (aliasing Y) is consumed
    float2* Yp = Y + par * N1 * YP;
    if (r < N2) {
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Yp[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Yp[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, false>(u, tws);
        float2* orow = out + (int64_t)row * M * CP + c;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) orow[(int64_t)(2 * (r + N1 * k2) + par) * CP] = u[k2];
    }
}

// out[row][i] = scale * sum_c conj(S_c) v_c[(i + n/2) mod n ...] + alpha * operand,
// v_c the cropped inverse of src_c[row] (length M = 2n), the four coil blocks
// of a row summed in a 4-CTA cluster through distributed shared memory.
// grid (NCB, ny), cluster (NCB, 1, 1), block half_threads.
template <int N2>
__global__ void __launch_bounds__(half_threads<N2>())
toep_rows_inv_half_cl_kernel(const float2* __restrict__ tw, const float2* __restrict__ twM,
                             const float2* __restrict__ src, const float2* __restrict__ S,
                             float2* out, float scale, const float2* operand, float alpha) {
    constexpr int n = N1 * N2, YP = ypitch<N2>(), T = CB * tpr<N2>(), M = 2 * n;
    constexpr int RZ = n * 9;   // R[i * 9 + j] (j < 8 coils, 8 = their sum), then Z[p * 8 + j]
    static_assert(2 * N1 * YP >= RZ + n * CB, "R and Z must fit the transpose buffers");
    __shared__ float2 tws[n], twm[n];
    __shared__ __align__(16) float2 Y[2 * N1 * YP];
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank(), row = blockIdx.y;
    pdl_trigger();
    {
        const float2* Srow = S + (int64_t)row * n * CP + q * CB;
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(Srow + (int64_t)i * CP));
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        twm[i] = twM[i];
    }
    __syncthreads();
    pdl_wait();
    const int par = threadIdx.x / T, t = threadIdx.x - par * T, j = t & (CB - 1), r = t / CB;
    const int c = q * CB + j;
    float2* Yp = Y + par * N1 * YP;
    if (r < N2) {
        float2 v[N1];
        const float2* srow = src + (int64_t)row * M * CP + c;
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) v[m1] = srow[(int64_t)(2 * (N2 * m1 + r) + par) * CP];
        fft4_phase1<N1, N2, true>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Yp[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    float2 u[N2];
    if (r < N1) {
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Yp[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, true>(u, tws);   // u[k2] = IFFT_n(X_par)[r + 16 k2]
    }
    __syncthreads();   // Y is reused below as R and Z
    float2* R = Y;
    float2* Z = Y + RZ;
    if (par == 1 && r < N1) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int p = r + N1 * k2;
            float2 w = twm[p];                       // W_M^(-p) = conj(twm[p]), sign s(p)
            w = p >= n / 2 ? make_float2(-w.x, w.y) : make_float2(w.x, -w.y);
            Z[p * CB + j] = cmul(u[k2], w);
        }
    }
    __syncthreads();
    if (par == 0 && r < N1) {
        const float2* srow = S + (int64_t)row * n * CP + c;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int p = r + N1 * k2;
            int i = p + n / 2;
            if (i >= n) i -= n;
            R[i * 9 + j] = cmulc(srow[(int64_t)i * CP], cadd(u[k2], Z[p * CB + j]));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float2 acc = R[i * 9];
#pragma unroll
        for (int jj = 1; jj < CB; ++jj) acc = cadd(acc, R[i * 9 + jj]);
        R[i * 9 + 8] = acc;
    }
    cluster_row_sum(Y, n, row, q, scale, operand, alpha, out);
}

// Column stage of the Toeplitz operator on length-n halves (n = ny = 16 N2,
// M = 2n): the column's n image rows sit at positions [-n/2, n/2) mod M, so
// X[2k + par] = FFT_n(f_par)[k] as in the row stage; the product with the
// kernel spectrum Tc[q][2k + par]; the mirrored inverse of each half
// (length-N2 DFT over k2 and W_n^(-m2 k1) by the (k1) threads, length-16
// DFT over k1 by the (m2) threads); and the cropped combination
// v[p] = F_0[p] + s(p) W_M^(-p) F_1[p] stored at row (p + n/2) mod n.
// grid (Mx, coil blocks), block half_threads; rows of src/dst: [ny][Mx][CP].
template <int N2>
__global__ void __launch_bounds__(half_threads<N2>(), 3)
toep_cols_half_kernel(const float2* __restrict__ tw, const float2* __restrict__ twM,
                      const float* __restrict__ Tc, int Mx, const float2* __restrict__ src,
                      float2* __restrict__ dst) {
    constexpr int n = N1 * N2, YP = ypitch<N2>(), T = CB * tpr<N2>(), M = 2 * n;
    static_assert(2 * N1 * YP >= n * CB, "Z must fit the transpose buffers");
    __shared__ float2 tws[n], twm[n];
    __shared__ float Ts[M];
    __shared__ float2 Y[2 * N1 * YP];
    pdl_trigger();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tws[i] = tw[i];
        twm[i] = twM[i];
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) Ts[i] = Tc[(int64_t)blockIdx.x * M + i];
    __syncthreads();
    pdl_wait();
    const int par = threadIdx.x / T, t = threadIdx.x - par * T, j = t & (CB - 1), r = t / CB;
    const int64_t rs = (int64_t)Mx * CP;
    const int64_t cofs = (int64_t)blockIdx.x * CP + blockIdx.y * CB + j;
    float2* Yp = Y + par * N1 * YP;
    if (r < N2) {
        float2 v[N1];
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + r;
            int i = p + n / 2;
            if (i >= n) i -= n;
            float2 val = src[i * rs + cofs];
            if (par) {
                float2 w = twm[p];
                if (p >= n / 2) w = make_float2(-w.x, -w.y);
                val = cmul(val, w);
            }
            v[m1] = val;
        }
        fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Yp[k1 * YP + r * CB + j] = v[k1];
    }
    __syncthreads();
    if (r < N1) {
        float2 u[N2];
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) u[m2] = Yp[r * YP + m2 * CB + j];
        fft4_phase2<N1, N2, false>(u, tws);          // u[k2] = X[2 (r + 16 k2) + par]
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) u[k2] = cscale(u[k2], Ts[2 * (r + N1 * k2) + par]);
        RegFft<N2, true>::run(u, tws, N1);
#pragma unroll
        for (int m2 = 1; m2 < N2; ++m2) {
            float2 w = tws[m2 * r];
            w.y = -w.y;
            u[m2] = cmul(u[m2], w);
        }
        // the same (k1, coil) slots this thread read: no other thread touches them
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) Yp[r * YP + m2 * CB + j] = u[m2];
    }
    __syncthreads();
    float2 f[N1];
    if (r < N2) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) f[k1] = Yp[k1 * YP + r * CB + j];
        RegFft<N1, true>::run(f, tws, N2);           // f[m1] = F_par[N2 m1 + r]
    }
    __syncthreads();   // Y is reused as Z
    float2* Z = Y;
    if (par == 1 && r < N2) {
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + r;
            float2 w = twm[p];
            w = p >= n / 2 ? make_float2(-w.x, w.y) : make_float2(w.x, -w.y);
            Z[p * CB + j] = cmul(f[m1], w);
        }
    }
    __syncthreads();
    if (par == 0 && r < N2) {
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int p = N2 * m1 + r;
            int i = p + n / 2;
            if (i >= n) i -= n;
            dst[i * rs + cofs] = cadd(f[m1], Z[p * CB + j]);
        }
    }
}

static pp_status check_ci(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    if (g_profiler) g_profiler->mark(what);
    return PP_OK;
}

}  // namespace

bool ci_supported(const Plan& p) {
    return p.kind == PP_NONCARTESIAN && p.ndim == 2 && p.C <= CP && fft4_n2(p.G_x) &&
           fft4_n2(p.G_y) && p.gtg8 != nullptr;
}

size_t ci_grid_elems(const Plan& p) { return (size_t)p.G_y * p.G_x * CP; }
size_t ci_stencil_tiles(const Plan& p) {
    return (size_t)((p.G_x + CPS_TX - 1) / CPS_TX) * ((p.G_y + CPS_TY - 1) / CPS_TY);
}
size_t ci_rows_elems(const Plan& p) { return (size_t)p.ny * p.G_x * CP; }
size_t ci_sens_elems(const Plan& p) { return (size_t)p.ny * p.nx * CP; }
size_t ci_partial_elems(const Plan& p) { return (size_t)NCB * p.ny * p.nx; }

pp_status ci_prepare(Plan& p, cudaStream_t st) {
    PP_TRY_CUDA(cudaFuncSetAttribute(ci_stencil_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CiStencil<1>::SMEM));
    PP_TRY_CUDA(cudaFuncSetAttribute(ci_stencil_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CiStencil<2>::SMEM));
    PP_TRY_CUDA(cudaFuncSetAttribute(ci_stencil_cp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)CPS_SMEM));
    const int64_t n = (int64_t)p.ny * p.nx;
    ci_pack_sens_kernel<<<152 * 4, 256, 0, st>>>(p.sens, p.C, n, p.ci_sens);
    PP_TRY(check_ci("ci_pack_sens_kernel"));
    if (p.ci_tile_nz && p.gtg8) {
        ci_tile_flags_kernel<<<(unsigned)ci_stencil_tiles(p), 256, 0, st>>>(p.gtg8, p.G_x, p.G_y,
                                                                           (p.G_x + 7) / 8, p.ci_tile_nz);
        PP_TRY(check_ci("ci_tile_flags_kernel"));
    }
    return PP_OK;
}

// out = scale * A^H A x + alpha * operand on the coil-innermost buffers
pp_status ci_normal(const Plan& p, const float2* x, float2* out, float scale, const float2* operand,
                    float alpha, int ry, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, Gx = p.G_x, Gy = p.G_y;
    const int n2x = fft4_n2(Gx), n2y = fft4_n2(Gy);
    const bool pdl = p.pdl != 0;
    RowArgs rf{};
    rf.n = nx; rf.G = Gx; rf.off_in = nx / 2; rf.off_out = 0; rf.nrows = ny; rf.scale = 1.f;
#define PP_CIR(N2_)                                                                                \
    if (n2x == N2_)                                                                                \
        PP_TRY_CUDA(launch_ex(ci_rows_fwd_kernel<N2_>, dim3(ny, NCB), dim3(CB * tpr<N2_>()), 0, st, \
                              pdl, 0, (const float2*)p.gx.tw, rf, x, (const float2*)p.ci_sens,    \
                              (const float*)p.deapod_y, (const float*)p.deapod_x, p.ci_a));
    PP_CIR(8) PP_CIR(12) PP_CIR(16) PP_CIR(20) PP_CIR(24)
#undef PP_CIR
    PP_TRY(check_ci("ci_rows_fwd_kernel"));
#define PP_CIC(N2_, INV_, HIN, HOUT, OIN, OOUT, SRC, DST)                                          \
    if (n2y == N2_)                                                                                \
        PP_TRY_CUDA(launch_ex(ci_cols_kernel<N2_, INV_>, dim3(Gx, NCB), dim3(CB * tpr<N2_>()), 0,   \
                              st, pdl, 0, (const float2*)p.gy.tw, (int)(HIN), (int)(HOUT),        \
                              (int)(OIN), (int)(OOUT), Gx, (const float2*)(SRC), (float2*)(DST)));
    PP_CIC(8, false, ny, Gy, ny / 2, 0, p.ci_a, p.ci_b)
    PP_CIC(12, false, ny, Gy, ny / 2, 0, p.ci_a, p.ci_b)
    PP_CIC(16, false, ny, Gy, ny / 2, 0, p.ci_a, p.ci_b)
    PP_CIC(20, false, ny, Gy, ny / 2, 0, p.ci_a, p.ci_b)
    PP_CIC(24, false, ny, Gy, ny / 2, 0, p.ci_a, p.ci_b)
    PP_TRY(check_ci("ci_cols_kernel"));
    const int ntiles = ry ? ((Gx + 15) / 16) * ((Gy + 4 * ry - 1) / (4 * ry)) : 0;
    if (ry == 0)
        PP_TRY_CUDA(launch_ex(ci_stencil_cp_kernel,
                              dim3(((Gx + CPS_TX - 1) / CPS_TX) * ((Gy + CPS_TY - 1) / CPS_TY)), dim3(256),
                              CPS_SMEM, st, pdl, 0, (const float*)p.gtg8, Gx, Gy, (Gx + 7) / 8,
                              (const int*)p.ci_tile_nz, (const float2*)p.ci_b, p.ci_c));
    else if (ry == 2)
        PP_TRY_CUDA(launch_ex(ci_stencil_kernel<2>, dim3(ntiles), dim3(256), CiStencil<2>::SMEM, st,
                              pdl, 0, (const float*)p.gtg8, Gx, Gy, (Gx + 7) / 8,
                              (const float2*)p.ci_b, p.ci_c));
    else
        PP_TRY_CUDA(launch_ex(ci_stencil_kernel<1>, dim3(ntiles), dim3(256), CiStencil<1>::SMEM, st,
                              pdl, 0, (const float*)p.gtg8, Gx, Gy, (Gx + 7) / 8,
                              (const float2*)p.ci_b, p.ci_c));
    PP_TRY(check_ci("ci_stencil_kernel"));
    PP_CIC(8, true, Gy, ny, 0, ny / 2, p.ci_c, p.ci_a)
    PP_CIC(12, true, Gy, ny, 0, ny / 2, p.ci_c, p.ci_a)
    PP_CIC(16, true, Gy, ny, 0, ny / 2, p.ci_c, p.ci_a)
    PP_CIC(20, true, Gy, ny, 0, ny / 2, p.ci_c, p.ci_a)
    PP_CIC(24, true, Gy, ny, 0, ny / 2, p.ci_c, p.ci_a)
#undef PP_CIC
    PP_TRY(check_ci("ci_cols_kernel"));
    RowArgs ra = rf;
    ra.off_in = 0; ra.off_out = nx / 2;
    if (p.tune_rows_adj_cl == 4) {
        cudaError_t e = cudaSuccess;
#define PP_CIL(N2_)                                                                          \
        if (n2x == N2_)                                                                      \
            e = launch_ex(ci_rows_inv_cl_kernel<N2_>, dim3(NCB, ny), dim3(CB * tpr<N2_>()), 0, \
                          st, pdl, NCB, (const float2*)p.gx.tw, ra, (const float2*)p.ci_a,   \
                          (const float2*)p.ci_sens, (const float*)p.deapod_y,                \
                          (const float*)p.deapod_x, out, scale, operand, alpha);
        PP_CIL(8) PP_CIL(12) PP_CIL(16) PP_CIL(20) PP_CIL(24)
#undef PP_CIL
        if (e != cudaSuccess) return cuda_status(e, "ci_rows_inv_cl_kernel launch");
        return check_ci("ci_rows_inv_cl_kernel");
    }
#define PP_CII(N2_)                                                                                \
    if (n2x == N2_)                                                                                \
        PP_TRY_CUDA(launch_ex(ci_rows_inv_kernel<N2_>, dim3(ny, NCB), dim3(CB * tpr<N2_>()), 0, st,  \
                              pdl, 0, (const float2*)p.gx.tw, ra, (const float2*)p.ci_a,          \
                              (const float2*)p.ci_sens, (const float*)p.deapod_y,                 \
                              (const float*)p.deapod_x, p.ci_part));
    PP_CII(8) PP_CII(12) PP_CII(16) PP_CII(20) PP_CII(24)
#undef PP_CII
    PP_TRY(check_ci("ci_rows_inv_kernel"));
    const int64_t n = (int64_t)ny * nx;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    PP_TRY_CUDA(launch_ex(ci_sum_kernel, dim3(blocks), dim3(256), 0, st, pdl, 0,
                          (const float2*)p.ci_part, n, scale, operand, alpha, out));
    return check_ci("ci_sum_kernel");
}

bool toep_supported(int nx, int ny, int C) {
    // each axis: n itself a register length (two length-n halves) or 2n
    return C >= 1 && C <= CP && (fft4_n2(nx) || fft4_n2(2 * nx)) && (fft4_n2(ny) || fft4_n2(2 * ny));
}

size_t toep_rows_elems(const Plan& p) { return (size_t)p.ny * 2 * p.nx * CP; }

// out = scale * A^H A x + alpha * operand with F^H F evaluated through its
// Toeplitz structure: embed in the 2ny x 2nx circulant, so that
//   F^H F v = crop(IFFT(Tk . FFT(zero-pad(v))))
// with Tk the spectrum of the embedded kernel.  Three kernels: coil expand +
// row FFT, column FFT * Tk * column IFFT, row IFFT + conj(S) coil reduction
// (4-CTA cluster) + Horner axpy.
pp_status toep_normal(const Plan& p, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, Mx = 2 * nx, My = 2 * ny;
    const int n2x = fft4_n2(Mx), n2y = fft4_n2(My);
    const int ncb = (p.C + CB - 1) / CB;
    const bool pdl = p.pdl != 0;
    RowArgs rf{};
    rf.n = nx; rf.G = Mx; rf.off_in = nx / 2; rf.off_out = 0; rf.nrows = ny; rf.scale = 1.f;
    cudaError_t e = cudaErrorInvalidValue;
    const int n2h = fft4_n2(nx);   // rows of a register length: two length-nx halves
#define PP_TH(N2_)                                                                              \
    if (n2h == N2_)                                                                             \
        e = launch_ex(toep_rows_fwd_half_kernel<N2_>, dim3(ny, ncb), dim3(half_threads<N2_>()), 0, \
                      st, pdl, 0, (const float2*)p.toep_hx.tw, (const float2*)p.tx.tw, x,        \
                      (const float2*)p.ci_sens, p.toep_a);
    PP_TH(8) PP_TH(12) PP_TH(16)
#undef PP_TH
#define PP_TR(N2_)                                                                              \
    if (n2x == N2_)                                                                             \
        e = launch_ex(ci_rows_fwd_kernel<N2_>, dim3(ny, ncb), dim3(CB * tpr<N2_>()), 0, st, pdl, 0, \
                      (const float2*)p.tx.tw, rf, x, (const float2*)p.ci_sens, (const float*)nullptr, \
                      (const float*)nullptr, p.toep_a);
    if (!n2h) { PP_TR(8) PP_TR(12) PP_TR(16) PP_TR(20) PP_TR(24) }
#undef PP_TR
    if (e != cudaSuccess) return cuda_status(e, "Toeplitz row FFT launch");
    PP_TRY(check_ci(n2h ? "toep_rows_fwd_half_kernel" : "ci_rows_fwd_kernel"));
    e = cudaErrorInvalidValue;
    const int n2hy = fft4_n2(ny);   // columns of a register length: two length-ny halves
#define PP_TD(N2_)                                                                              \
    if (n2hy == N2_)                                                                            \
        e = launch_ex(toep_cols_half_kernel<N2_>, dim3(Mx, ncb), dim3(half_threads<N2_>()), 0, st,  \
                      pdl, 0, (const float2*)p.toep_hy.tw, (const float2*)p.ty.tw,              \
                      (const float*)p.toep_T, Mx, (const float2*)p.toep_a, p.toep_b);
    PP_TD(8) PP_TD(12) PP_TD(16)
#undef PP_TD
#define PP_TC(N2_)                                                                              \
    if (n2y == N2_)                                                                             \
        e = launch_ex(toep_cols_kernel<N2_>, dim3(Mx, ncb), dim3(CB * tpr<N2_>()), 0, st, pdl, 0,   \
                      (const float2*)p.ty.tw, (const float*)p.toep_T, ny, ny / 2, Mx,            \
                      (const float2*)p.toep_a, p.toep_b);
    if (!n2hy) { PP_TC(8) PP_TC(12) PP_TC(16) PP_TC(20) PP_TC(24) }
#undef PP_TC
    if (e != cudaSuccess) return cuda_status(e, "Toeplitz column stage launch");
    PP_TRY(check_ci(n2hy ? "toep_cols_half_kernel" : "toep_cols_kernel"));
    RowArgs ra = rf;
    ra.off_in = 0; ra.off_out = nx / 2;
    e = cudaErrorInvalidValue;
#define PP_TJ(N2_)                                                                              \
    if (n2h == N2_)                                                                             \
        e = launch_ex(toep_rows_inv_half_cl_kernel<N2_>, dim3(NCB, ny), dim3(half_threads<N2_>()),  \
                      0, st, pdl, NCB, (const float2*)p.toep_hx.tw, (const float2*)p.tx.tw,      \
                      (const float2*)p.toep_b, (const float2*)p.ci_sens, out, scale, operand,   \
                      alpha);
    PP_TJ(8) PP_TJ(12) PP_TJ(16)
#undef PP_TJ
#define PP_TI(N2_)                                                                              \
    if (n2x == N2_)                                                                             \
        e = launch_ex(ci_rows_inv_cl_kernel<N2_>, dim3(NCB, ny), dim3(CB * tpr<N2_>()), 0, st, pdl, \
                      NCB, (const float2*)p.tx.tw, ra, (const float2*)p.toep_b,                  \
                      (const float2*)p.ci_sens, (const float*)nullptr, (const float*)nullptr, out,  \
                      scale, operand, alpha);
    if (!n2h) { PP_TI(8) PP_TI(12) PP_TI(16) PP_TI(20) PP_TI(24) }
#undef PP_TI
    if (e != cudaSuccess) return cuda_status(e, "Toeplitz row IFFT launch");
    return check_ci(n2h ? "toep_rows_inv_half_cl_kernel" : "ci_rows_inv_cl_kernel");
}

}  // namespace pp
