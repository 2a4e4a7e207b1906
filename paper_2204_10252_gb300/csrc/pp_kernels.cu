// CUDA kernels of the SENSE operators (Sec. 5.1 Cartesian, Sec. 5.2
// non-Cartesian with Kaiser-Bessel gridding) and of the solver's elementwise
// and reduction steps (Algorithm "pfista", Sec. 3.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp_internal.h"

namespace pp {

namespace {

constexpr int RB = 8;        // rows per CTA in the row stages
constexpr int LGRB = 3;
constexpr int TX = 8;        // columns per CTA in the column stages
constexpr int LGTX = 3;
constexpr int KMAX = 16;     // owned elements per thread (rows: RB*n/256, n <= 512)

__device__ __forceinline__ int wrapG(int a, int G) {
    a %= G;
    return a < 0 ? a + G : a;
}

__device__ __forceinline__ void load_table(float2* dst, const float2* __restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__host__ __device__ __forceinline__ int row_stride(int G) { return G + 2; }

// ---------------------------------------------------------------------------
// Row stage, image -> k rows.  CTA (bx, by): rows bx*RB .. +RB of batch by.
//   v(i) = scale * wrow[r] * wcol[i] * x_by[r][i] * S_by[r][i]
//   transform position (i - off_in) mod G, FFT of length G,
//   out_by[r][q] = V((q - off_out) mod G).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
rows_fwd_kernel(FftDesc fd, const float2* __restrict__ tw, RowArgs a,
                const float2* __restrict__ x, int64_t x_batch_stride,
                const float2* __restrict__ sens, const float* __restrict__ wrow,
                const float* __restrict__ wcol, float2* __restrict__ out) {
    extern __shared__ float2 sm[];
    const int G = a.G, n = a.n, bs = row_stride(G);
    float2* tws = sm;
    float2* b0 = sm + G;
    float2* b1 = b0 + RB * bs;
    load_table(tws, tw, G);
    const int c = blockIdx.y;
    const int row0 = blockIdx.x * RB;
    const float2* xc = x + (int64_t)c * x_batch_stride;
    const float2* sc = sens ? sens + (int64_t)c * a.coil_img_stride : nullptr;
    for (int idx = threadIdx.x; idx < RB * G; idx += blockDim.x) {
        const int b = idx / G;
        const int p = idx - b * G;
        const int r = row0 + b;
        int i = p + a.off_in;
        if (i >= G) i -= G;
        float2 v = make_float2(0.f, 0.f);
        if (r < a.nrows && i < n) {
            const int64_t o = (int64_t)r * n + i;
            v = xc[o];
            if (sc) v = cmul(v, sc[o]);
            float w = a.scale;
            if (wrow) w *= wrow[r];
            if (wcol) w *= wcol[i];
            v = cscale(v, w);
        }
        b0[p + b * bs] = v;
    }
    __syncthreads();
    float2* res = fft_batch<false>(b0, b1, fd, 1, bs, LGRB, tws, nullptr);
    float2* oc = out + (int64_t)c * a.nrows * G;
    for (int idx = threadIdx.x; idx < RB * G; idx += blockDim.x) {
        const int b = idx / G;
        const int q = idx - b * G;
        const int r = row0 + b;
        if (r < a.nrows) {
            int p = q - a.off_out;
            if (p < 0) p += G;
            oc[(int64_t)r * G + q] = res[p + b * bs];
        }
    }
}

// ---------------------------------------------------------------------------
// Row stage, k rows -> image, with the conjugate-coil reduction and an axpy
// epilogue:  out[r][i] = scale * sum_c conj(S_c[r][i]) wrow[r] wcol[i]
//                        * IFFT(src_c[r])((i - off_out) mod G)
//                        + alpha * operand[r][i].
// src_c[r][s] sits at transform position (s - off_in) mod G.
// ---------------------------------------------------------------------------
template <int KM>
__global__ void __launch_bounds__(kThreads)
rows_adj_kernel(FftDesc fd, const float2* __restrict__ tw, RowArgs a,
                const float2* __restrict__ src, const float2* __restrict__ sens,
                const float* __restrict__ wrow, const float* __restrict__ wcol,
                float2* out, const float2* operand, float alpha, int ncoils) {
    extern __shared__ float2 sm[];
    const int G = a.G, n = a.n, bs = row_stride(G);
    float2* tws = sm;
    float2* b0 = sm + G;
    float2* b1 = b0 + RB * bs;
    load_table(tws, tw, G);
    const int row0 = blockIdx.x * RB;
    float2 acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int c = 0; c < ncoils; ++c) {
        const float2* scn = src + (int64_t)c * a.nrows * G;
        for (int idx = threadIdx.x; idx < RB * G; idx += blockDim.x) {
            const int b = idx / G;
            const int p = idx - b * G;
            const int r = row0 + b;
            int s = p + a.off_in;
            if (s >= G) s -= G;
            b0[p + b * bs] = (r < a.nrows) ? scn[(int64_t)r * G + s] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2* res = fft_batch<true>(b0, b1, fd, 1, bs, LGRB, tws, nullptr);
        const float2* sc = sens ? sens + (int64_t)c * a.coil_img_stride : nullptr;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int e = threadIdx.x + k * kThreads;
            if (e < RB * n) {
                const int b = e / n;
                const int i = e - b * n;
                const int r = row0 + b;
                if (r < a.nrows) {
                    int p = i - a.off_out;
                    if (p < 0) p += G;
                    float2 v = res[p + b * bs];
                    float w = 1.f;
                    if (wrow) w *= wrow[r];
                    if (wcol) w *= wcol[i];
                    v = cscale(v, w);
                    if (sc) v = cmulc(sc[(int64_t)r * n + i], v);
                    acc[k] = cadd(acc[k], v);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int e = threadIdx.x + k * kThreads;
        if (e < RB * n) {
            const int b = e / n;
            const int i = e - b * n;
            const int r = row0 + b;
            if (r < a.nrows) {
                const int64_t o = (int64_t)r * n + i;
                float2 v = cscale(acc[k], a.scale);
                if (operand) v = cadd(v, cscale(operand[o], alpha));
                out[o] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Column stage: FFT along the strided axis for TX adjacent columns of one
// batch.  Input row r -> position (r - off_in) mod G (rows >= Hin are zero);
// output row q <- position (q - off_out) mod G, q < Hout.
// ---------------------------------------------------------------------------
template <bool INV>
__global__ void __launch_bounds__(kThreads)
cols_kernel(FftDesc fd, const float2* __restrict__ tw, ColArgs a, const float2* src, float2* dst) {
    // src == dst is allowed: a CTA reads all of its columns before writing them.
    extern __shared__ float2 sm[];
    const int G = a.G;
    float2* tws = sm;
    float2* b0 = sm + G;
    float2* b1 = b0 + G * TX;
    load_table(tws, tw, G);
    const int col0 = blockIdx.x * TX;
    const float2* sb = src + (int64_t)blockIdx.y * a.in_batch_stride;
    float2* db = dst + (int64_t)blockIdx.y * a.out_batch_stride;
    for (int idx = threadIdx.x; idx < G * TX; idx += blockDim.x) {
        const int p = idx >> LGTX;
        const int b = idx & (TX - 1);
        int r = p + a.off_in;
        if (r >= G) r -= G;
        const int col = col0 + b;
        float2 v = make_float2(0.f, 0.f);
        if (r < a.Hin && col < a.ncols) {
            v = sb[(int64_t)r * a.ncols + col];
            if (a.mul_in) v = cscale(v, a.mul_in[r * a.mi_q + (col / a.mi_cdiv) * a.mi_c]);
        }
        b0[idx] = v;
    }
    __syncthreads();
    float2* res = fft_batch<INV>(b0, b1, fd, TX, 1, LGTX, tws, nullptr);
    for (int idx = threadIdx.x; idx < a.Hout * TX; idx += blockDim.x) {
        const int q = idx >> LGTX;
        const int b = idx & (TX - 1);
        const int col = col0 + b;
        if (col < a.ncols) {
            int p = q - a.off_out;
            p = wrapG(p, G);
            float s = a.scale;
            if (a.mul_out) s *= a.mul_out[q * a.mo_q + (col / a.mo_cdiv) * a.mo_c];
            db[(int64_t)q * a.ncols + col] = cscale(res[(p << LGTX) + b], s);
        }
    }
}

// Column round trip in FFT order: IFFT(mask . FFT(col)), mask value of
// transform position p for column col: mask_fo[p * mo_q + (col / mo_cdiv) * mo_c]
// (normalisation folded into the mask).  Used along z by the 3-D operator.
__global__ void __launch_bounds__(kThreads)
cols_roundtrip_kernel(FftDesc fd, const float2* __restrict__ tw, ColArgs a,
                      const float* __restrict__ mask_fo, const float2* __restrict__ src,
                      float2* __restrict__ dst) {
    extern __shared__ float2 sm[];
    const int G = a.G;
    float2* tws = sm;
    float2* b0 = sm + G;
    float2* b1 = b0 + G * TX;
    load_table(tws, tw, G);
    const int col0 = blockIdx.x * TX;
    const float2* sb = src + (int64_t)blockIdx.y * a.in_batch_stride;
    float2* db = dst + (int64_t)blockIdx.y * a.out_batch_stride;
    for (int idx = threadIdx.x; idx < G * TX; idx += blockDim.x) {
        const int p = idx >> LGTX;
        const int col = col0 + (idx & (TX - 1));
        b0[idx] = (col < a.ncols) ? sb[(int64_t)p * a.ncols + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* r1 = fft_batch<false>(b0, b1, fd, TX, 1, LGTX, tws, nullptr);
    for (int idx = threadIdx.x; idx < G * TX; idx += blockDim.x) {
        const int p = idx >> LGTX;
        const int col = col0 + (idx & (TX - 1));
        const float m = (col < a.ncols) ? mask_fo[p * a.mo_q + (col / a.mo_cdiv) * a.mo_c] : 0.f;
        r1[idx] = cscale(r1[idx], m);
    }
    __syncthreads();
    float2* other = (r1 == b0) ? b1 : b0;
    float2* r2 = fft_batch<true>(r1, other, fd, TX, 1, LGTX, tws, nullptr);
    for (int idx = threadIdx.x; idx < G * TX; idx += blockDim.x) {
        const int p = idx >> LGTX;
        const int col = col0 + (idx & (TX - 1));
        if (col < a.ncols) db[(int64_t)p * a.ncols + col] = r2[idx];
    }
}

// ---------------------------------------------------------------------------
// Fused 2-D Cartesian normal operator for a mask constant along x:
//   out = scale * sum_c conj(S_c) F_y^H (M_fo/ny) F_y (S_c x) + alpha * operand
// One CTA owns TX columns and loops over every coil; S_c is read once and
// kept in registers between the coil expansion and the conjugate product.
// ---------------------------------------------------------------------------
template <int KM>
__global__ void __launch_bounds__(kThreads)
cart2d_normal_kernel(FftDesc fd, const float2* __restrict__ tw, const float2* __restrict__ x,
                     const float2* __restrict__ sens, int C, int ny, int nx,
                     const float* __restrict__ mask_fo, float2* __restrict__ out, float scale,
                     const float2* __restrict__ operand, float alpha) {
    extern __shared__ float2 sm[];
    float2* tws = sm;
    float2* b0 = sm + ny;
    float2* b1 = b0 + ny * TX;
    float* pm = reinterpret_cast<float*>(b1 + ny * TX);
    load_table(tws, tw, ny);
    for (int i = threadIdx.x; i < ny; i += blockDim.x) pm[i] = mask_fo[i];
    const int col0 = blockIdx.x * TX;
    const int nel = ny * TX;
    float2 xr[KM], sr[KM], acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int e = threadIdx.x + k * kThreads;
        const int yy = e >> LGTX;
        const int col = col0 + (e & (TX - 1));
        xr[k] = (e < nel && col < nx) ? x[(int64_t)yy * nx + col] : make_float2(0.f, 0.f);
        acc[k] = make_float2(0.f, 0.f);
    }
    const int64_t cs = (int64_t)ny * nx;
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int e = threadIdx.x + k * kThreads;
            if (e < nel) {
                const int yy = e >> LGTX;
                const int col = col0 + (e & (TX - 1));
                sr[k] = (col < nx) ? sens[c * cs + (int64_t)yy * nx + col] : make_float2(0.f, 0.f);
                b0[e] = cmul(sr[k], xr[k]);
            }
        }
        __syncthreads();
        float2* r1 = fft_batch<false>(b0, b1, fd, TX, 1, LGTX, tws, nullptr);
        float2* other = (r1 == b0) ? b1 : b0;
        float2* r2 = fft_batch<true>(r1, other, fd, TX, 1, LGTX, tws, pm);
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int e = threadIdx.x + k * kThreads;
            if (e < nel) acc[k] = cadd(acc[k], cmulc(sr[k], r2[e]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int e = threadIdx.x + k * kThreads;
        const int yy = e >> LGTX;
        const int col = col0 + (e & (TX - 1));
        if (e < nel && col < nx) {
            const int64_t o = (int64_t)yy * nx + col;
            float2 v = cscale(acc[k], scale);
            if (operand) v = cadd(v, cscale(operand[o], alpha));
            out[o] = v;
        }
    }
}

__global__ void expand_kernel(const float2* __restrict__ x, const float2* __restrict__ s,
                              float2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cmul(s[i], x[i]);
}

// out (+)= conj(s) * w; on the last coil out = scale * out + alpha * operand.
__global__ void conj_accum_kernel(const float2* __restrict__ s, const float2* __restrict__ wv,
                                  float2* __restrict__ out, int64_t n, int first, float scale,
                                  const float2* __restrict__ operand, float alpha, int last) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = cmulc(s[i], wv[i]);
        if (!first) v = cadd(v, out[i]);
        if (last) {
            v = cscale(v, scale);
            if (operand) v = cadd(v, cscale(operand[i], alpha));
        }
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Kaiser-Bessel spreading (the adjoint's gridding, G^T) on tiles of the
// oversampled grid (FFT order).  A CTA owns one T x T output tile and a chunk
// of coils; every sample whose W x W footprint meets the tile is listed for
// it (plan time), and the CTA adds the sample's value times the tap weights
// that fall inside the tile into a shared-memory accumulator (shared-memory
// atomics), then writes the tile once.  No global atomics.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
nufft_spread_tile_kernel(const TileEntry* __restrict__ entries, const int* __restrict__ tile_start,
                         int T, int ntx, int Gx, int Gy, int C, int coils_per_cta,
                         const float2* __restrict__ ksp, int K, float2* __restrict__ grid_out) {
    extern __shared__ float2 sm[];
    constexpr int H = W - 1;
    float* acc = reinterpret_cast<float*>(sm);
    const int tile = blockIdx.x;
    const int tyi = tile / ntx, txi = tile - tyi * ntx;
    const int ty0 = tyi * T, tx0 = txi * T;
    const int th = min(T, Gy - ty0), tw_ = min(T, Gx - tx0);
    const int e0 = tile_start[tile], e1 = tile_start[tile + 1];
    const int64_t gsz = (int64_t)Gx * Gy;
    const int c0 = blockIdx.y * coils_per_cta;
    const int c1 = min(C, c0 + coils_per_cta);
    for (int c = c0; c < c1; ++c) {
        for (int idx = threadIdx.x; idx < 2 * T * T; idx += blockDim.x) acc[idx] = 0.f;
        __syncthreads();
        // lane l of a warp takes entries l*S, l*S + 1, ... of the tile's list
        // (trajectory order), so the 32 samples spread at one time lie far
        // apart along the trajectory and their shared-memory atomics rarely
        // hit the same grid point
        const int ne = e1 - e0, S = (ne + 31) / 32;
        for (int i = threadIdx.x; i < 32 * S; i += blockDim.x) {
            const int e = e0 + (i & 31) * S + (i >> 5);
            if (e >= e1) continue;
            const TileEntry te = entries[e];
            const float wx[4] = {te.wx.x, te.wx.y, te.wx.z, te.wx.w};
            const float wy[4] = {te.wy.x, te.wy.y, te.wy.z, te.wy.w};
            const int ly0 = te.lyx & 0xffff, lx0 = te.lyx >> 16;
            const float2 v = ksp[(int64_t)c * K + te.k];
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const int yy = ly0 + b - H;
                if (yy < 0 || yy >= th) continue;
                const float vyx = wy[b] * v.x, vyy = wy[b] * v.y;
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const int xx = lx0 + a - H;
                    if (xx < 0 || xx >= tw_) continue;
                    atomicAdd(&acc[2 * (yy * T + xx)], wx[a] * vyx);
                    atomicAdd(&acc[2 * (yy * T + xx) + 1], wx[a] * vyy);
                }
            }
        }
        __syncthreads();
        float2* gout = grid_out + c * gsz;
        for (int idx = threadIdx.x; idx < th * T; idx += blockDim.x) {
            const int yy = idx / T, xx = idx - yy * T;
            if (xx < tw_)
                gout[(int64_t)(ty0 + yy) * Gx + tx0 + xx] = make_float2(acc[2 * idx], acc[2 * idx + 1]);
        }
        __syncthreads();
    }
}

// Degridding in trajectory order: ksp[c][k] = sum_ab wy_b wx_a grid_c[iy0+b][ix0+a].
template <int W>
__global__ void nufft_degrid_kernel(const SampleTaps* __restrict__ st, int K, int Gx, int Gy,
                                    const float2* __restrict__ grid, float2* __restrict__ ksp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (k >= K) return;
    const SampleTaps s = st[k];
    const float wx[4] = {s.wx.x, s.wx.y, s.wx.z, s.wx.w};
    const float wy[4] = {s.wy.x, s.wy.y, s.wy.z, s.wy.w};
    const float2* gc = grid + (int64_t)c * Gx * Gy;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < W; ++b) {
        const int gy = wrapG(s.iy0 + b, Gy);
        float2 rs = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            const int gx = wrapG(s.ix0 + a, Gx);
            const float2 g = gc[(int64_t)gy * Gx + gx];
            rs.x += wx[a] * g.x;
            rs.y += wx[a] * g.y;
        }
        v.x += wy[b] * rs.x;
        v.y += wy[b] * rs.y;
    }
    ksp[(int64_t)c * K + k] = v;
}


// ---------------------------------------------------------------------------
// Gridding pair of the normal operator as a stencil.  With interpolation
// G (samples <- grid) and spreading G^T, the normal operator needs G^T G on
// the oversampled grid, a real symmetric matrix that couples grid points at
// most W-1 apart per axis.  The plan stores it as (2W-1)^2 weight planes
// T[d][gy][gx] (d = (dy+W-1)(2W-1) + dx+W-1), so
//   out_j = sum_d T[d][j] in_{j + delta_d}   (indices periodic on the grid).
// A CTA owns a 16 x 16 output tile, keeps each point's weights in registers
// and loops over its coils, staging the input halo in shared memory.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
gtg_stencil_kernel(const float* __restrict__ T, int Gx, int Gy, int C, int coils_per_cta,
                   const float2* __restrict__ grid_in, float2* __restrict__ grid_out) {
    constexpr int H = W - 1, D = 2 * W - 1, TS = 16, HW = TS + 2 * H;
    constexpr int HE = (HW * HW + kThreads - 1) / kThreads;   // halo elements per thread
    __shared__ float2 halo[2][HW * HW];
    const int tx0 = blockIdx.x * TS, ty0 = blockIdx.y * TS;
    const int lx = threadIdx.x & (TS - 1), ly = threadIdx.x >> 4;
    const int gx = tx0 + lx, gy = ty0 + ly;
    const bool live = gx < Gx && gy < Gy;
    const int64_t plane = (int64_t)Gx * Gy;
    // halo source offsets of this thread's elements (fixed for every coil)
    int64_t hsrc[HE];
#pragma unroll
    for (int e = 0; e < HE; ++e) {
        const int idx = threadIdx.x + e * kThreads;
        const int hy = idx / HW, hx = idx - hy * HW;
        hsrc[e] = (idx < HW * HW)
                      ? (int64_t)wrapG(ty0 - H + hy, Gy) * Gx + wrapG(tx0 - H + hx, Gx)
                      : -1;
    }
    float w[D * D];
#pragma unroll
    for (int d = 0; d < D * D; ++d) w[d] = live ? T[d * plane + (int64_t)gy * Gx + gx] : 0.f;
    const int c0 = blockIdx.z * coils_per_cta, c1 = min(C, c0 + coils_per_cta);
    if (c0 >= c1) return;
    float2 pre[HE];
#pragma unroll
    for (int e = 0; e < HE; ++e)
        pre[e] = hsrc[e] >= 0 ? grid_in[c0 * plane + hsrc[e]] : make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) {
        float2* hb = halo[(c - c0) & 1];
#pragma unroll
        for (int e = 0; e < HE; ++e) {
            const int idx = threadIdx.x + e * kThreads;
            if (idx < HW * HW) hb[idx] = pre[e];
        }
        __syncthreads();
        // prefetch the next coil's halo while this one is computed
        if (c + 1 < c1) {
#pragma unroll
            for (int e = 0; e < HE; ++e)
                pre[e] = hsrc[e] >= 0 ? grid_in[(c + 1) * plane + hsrc[e]] : make_float2(0.f, 0.f);
        }
        float ax = 0.f, ay = 0.f;
#pragma unroll
        for (int dy = 0; dy < D; ++dy)
#pragma unroll
            for (int dx = 0; dx < D; ++dx) {
                const float2 v = hb[(ly + dy) * HW + lx + dx];
                const float t = w[dy * D + dx];
                ax += t * v.x;
                ay += t * v.y;
            }
        if (live) grid_out[c * plane + (int64_t)gy * Gx + gx] = make_float2(ax, ay);
        // the next iteration writes the other buffer; the one after that
        // rewrites this one only after the next __syncthreads
    }
}

// Variant of gtg_stencil_kernel with two vertically adjacent outputs per
// thread (16 x 16 tile, 128 threads): their 7 x 7 windows share 6 rows, so a
// thread reads 8 x 7 halo values for 2 outputs instead of 2 x 49.
template <int W>
__global__ void __launch_bounds__(128)
gtg_stencil2_kernel(const float* __restrict__ T, int Gx, int Gy, int C, int coils_per_cta,
                    const float2* __restrict__ grid_in, float2* __restrict__ grid_out) {
    constexpr int H = W - 1, D = 2 * W - 1, TS = 16, HW = TS + 2 * H;
    constexpr int HE = (HW * HW + 127) / 128;
    __shared__ float2 halo[2][HW * HW];
    const int tx0 = blockIdx.x * TS, ty0 = blockIdx.y * TS;
    const int lx = threadIdx.x & (TS - 1), ly = (threadIdx.x >> 4) * 2;   // rows ly, ly + 1
    const int gx = tx0 + lx, gy = ty0 + ly;
    const bool live0 = gx < Gx && gy < Gy, live1 = gx < Gx && gy + 1 < Gy;
    const int64_t plane = (int64_t)Gx * Gy;
    int64_t hsrc[HE];
#pragma unroll
    for (int e = 0; e < HE; ++e) {
        const int idx = threadIdx.x + e * 128;
        const int hy = idx / HW, hx = idx - hy * HW;
        hsrc[e] = (idx < HW * HW)
                      ? (int64_t)wrapG(ty0 - H + hy, Gy) * Gx + wrapG(tx0 - H + hx, Gx)
                      : -1;
    }
    float w0[D * D], w1[D * D];
#pragma unroll
    for (int d = 0; d < D * D; ++d) {
        w0[d] = live0 ? T[d * plane + (int64_t)gy * Gx + gx] : 0.f;
        w1[d] = live1 ? T[d * plane + (int64_t)(gy + 1) * Gx + gx] : 0.f;
    }
    const int c0 = blockIdx.z * coils_per_cta, c1 = min(C, c0 + coils_per_cta);
    if (c0 >= c1) return;
    float2 pre[HE];
#pragma unroll
    for (int e = 0; e < HE; ++e)
        pre[e] = hsrc[e] >= 0 ? grid_in[c0 * plane + hsrc[e]] : make_float2(0.f, 0.f);
    for (int c = c0; c < c1; ++c) {
        float2* hb = halo[(c - c0) & 1];
#pragma unroll
        for (int e = 0; e < HE; ++e) {
            const int idx = threadIdx.x + e * 128;
            if (idx < HW * HW) hb[idx] = pre[e];
        }
        __syncthreads();
        if (c + 1 < c1) {
#pragma unroll
            for (int e = 0; e < HE; ++e)
                pre[e] = hsrc[e] >= 0 ? grid_in[(c + 1) * plane + hsrc[e]] : make_float2(0.f, 0.f);
        }
        float a0x = 0.f, a0y = 0.f, a1x = 0.f, a1y = 0.f;
#pragma unroll
        for (int hy = 0; hy < D + 1; ++hy)
#pragma unroll
            for (int dx = 0; dx < D; ++dx) {
                const float2 v = hb[(ly + hy) * HW + lx + dx];
                if (hy < D) {
                    a0x += w0[hy * D + dx] * v.x;
                    a0y += w0[hy * D + dx] * v.y;
                }
                if (hy > 0) {
                    a1x += w1[(hy - 1) * D + dx] * v.x;
                    a1y += w1[(hy - 1) * D + dx] * v.y;
                }
            }
        if (live0) grid_out[c * plane + (int64_t)gy * Gx + gx] = make_float2(a0x, a0y);
        if (live1) grid_out[c * plane + (int64_t)(gy + 1) * Gx + gx] = make_float2(a1x, a1y);
    }
}

// Periodic wrap for a in [-G, 2G) (halo coordinates of a grid at least as
// large as the halo; plans guarantee G >= 40).
__device__ __forceinline__ int wrap1(int a, int G) { return a < 0 ? a + G : (a >= G ? a - G : a); }

// Asynchronous 8-byte global -> shared copy (zero-filled when !valid).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Register-blocked variant of the G^T G stencil.  Work item = (32 x TY
// output tile, group of CG coils); a persistent CTA takes a contiguous run
// of items (tile-major, so consecutive items reuse the tile's weights) and
// stages the next item's halo with cp.async while it computes the current
// one.  A warp covers 32 adjacent columns; a thread holds R vertically
// adjacent outputs of CG coils, so each halo word (two coils, 16 bytes) is
// read once for every output whose window contains it, and each weight once
// for CG coils.
template <int R, int CG, int NWY>
__global__ void __launch_bounds__(32 * NWY)
gtg_stencil_rb_kernel(const float* __restrict__ T, int Gx, int Gy, int C,
                      const float2* __restrict__ grid_in, float2* __restrict__ grid_out) {
    constexpr int W = 4, H = W - 1, D = 2 * W - 1;
    constexpr int TX = 32, TY = R * NWY, HX = TX + 2 * H, HY = TY + 2 * H, NP = CG / 2;
    constexpr int BUF = NP * HY * HX;   // float4 words per halo buffer
    extern __shared__ float4 hs[];
    const int ntx = (Gx + TX - 1) / TX, nty = (Gy + TY - 1) / TY, ngrp = (C + CG - 1) / CG;
    const int nitems = ntx * nty * ngrp;
    const int it0 = (int)((int64_t)blockIdx.x * nitems / gridDim.x);
    const int it1 = (int)((int64_t)(blockIdx.x + 1) * nitems / gridDim.x);
    if (it0 >= it1) return;
    const int plane = Gx * Gy;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    // halo rows are spread over the warps, halo columns over the lanes
    auto stage = [&](int it, float4* buf) {
        const int g = it % ngrp, tile = it / ngrp;
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY, c0 = g * CG;
        const int gx0 = wrap1(tx0 - H + lane, Gx);
        const int gx1 = wrap1(tx0 - H + 32 + lane, Gx);
        float2* b2 = reinterpret_cast<float2*>(buf);
        for (int rr = wy; rr < CG * HY; rr += NWY) {
            const int j = rr / HY, hy = rr - j * HY;
            const bool ok = c0 + j < C;
            const float2* src = grid_in + (int64_t)min(c0 + j, C - 1) * plane +
                                (int64_t)wrap1(ty0 - H + hy, Gy) * Gx;
            float2* dst = b2 + (size_t)(((j >> 1) * HY + hy) * HX) * 2 + (j & 1);
            cp_async8(dst + 2 * lane, src + gx0, ok);
            if (lane < HX - 32) cp_async8(dst + 2 * (32 + lane), src + gx1, ok);
        }
    };
    stage(it0, hs);
    cp_async_commit();
    for (int it = it0; it < it1; ++it) {
        const float4* cur = hs + ((it - it0) & 1) * BUF;
        if (it + 1 < it1) stage(it + 1, hs + ((it + 1 - it0) & 1) * BUF);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int g = it % ngrp, tile = it / ngrp;
        const int tx0 = (tile % ntx) * TX, ty0 = (tile / ntx) * TY, c0 = g * CG;
        const int x = tx0 + lane, y0 = ty0 + wy * R;
        // weight offsets, clamped into the grid for outputs that are not stored
        int off[R];
#pragma unroll
        for (int r = 0; r < R; ++r) off[r] = min(y0 + r, Gy - 1) * Gx + min(x, Gx - 1);
        float2 acc[R][CG];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < CG; ++j) acc[r][j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int iy = 0; iy < R + D - 1; ++iy)
#pragma unroll
            for (int dx = 0; dx < D; ++dx) {
                float4 v[NP];
#pragma unroll
                for (int q = 0; q < NP; ++q) v[q] = cur[(q * HY + wy * R + iy) * HX + lane + dx];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int dy = iy - r;
                    if (dy < 0 || dy >= D) continue;
                    const float w = __ldg(T + (dy * D + dx) * plane + off[r]);
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        acc[r][2 * q].x += w * v[q].x;
                        acc[r][2 * q].y += w * v[q].y;
                        acc[r][2 * q + 1].x += w * v[q].z;
                        acc[r][2 * q + 1].y += w * v[q].w;
                    }
                }
            }
        if (x < Gx) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (y0 + r < Gy) {
#pragma unroll
                    for (int j = 0; j < CG; ++j)
                        if (c0 + j < C)
                            grid_out[(int64_t)(c0 + j) * plane + (y0 + r) * Gx + x] = acc[r][j];
                }
        }
        __syncthreads();   // the next iteration restages the buffer read here
    }
}

// Coil-lane G^T G stencil: lanes are coils, so every weight is one
// shared-memory broadcast serving 32 coils.  A CTA owns a 16 x 4 output
// tile for a chunk of 32 coils.  cp.async stages the input halo as
// [row][col][coil] (coil stride 33 float2: conflict-free both for the
// transposing copy and for the per-position coil reads) and the tile's
// weights from the plan's [row][col/8][tap][8] copy of the planes.  A warp
// computes 8 adjacent outputs of one row; the results return through
// shared memory so that they leave coalesced along x.
constexpr int CL_TX = 16, CL_TY = 4, CL_CS = 33;
constexpr int CL_HX = CL_TX + 6, CL_HY = CL_TY + 6;
constexpr size_t CL_HALO_BYTES = sizeof(float2) * CL_HY * CL_HX * CL_CS;       // 58080
constexpr size_t CL_SMEM = CL_HALO_BYTES + sizeof(float) * CL_TY * CL_TX * 49;  // + 12544

__global__ void __launch_bounds__(256, 3)
gtg_stencil_cl_kernel(const float* __restrict__ T8, int Gx, int Gy, int C, int nxb,
                      const float2* __restrict__ grid_in, float2* __restrict__ grid_out) {
    constexpr int H = 3, D = 7;
    extern __shared__ float4 sm4[];
    float2* halo = reinterpret_cast<float2*>(sm4);
    const float4* wts = sm4 + CL_HALO_BYTES / sizeof(float4);
    const int ntx = (Gx + CL_TX - 1) / CL_TX, nch = (C + 31) / 32;
    const int ch = blockIdx.x % nch, tile = blockIdx.x / nch;
    const int tx0 = (tile % ntx) * CL_TX, ty0 = (tile / ntx) * CL_TY, c0 = ch * 32;
    const int plane = Gx * Gy;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // halo: warp w copies coils w, w + 8, w + 16, w + 24 of every halo row,
    // lane = column
    if (lane < CL_HX) {
        const int gx = wrap1(tx0 - H + lane, Gx);
        const float2* src[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ok[k] = c0 + w + 8 * k < C;
            src[k] = grid_in + (int64_t)min(c0 + w + 8 * k, C - 1) * plane + gx;
        }
        float2* dst = halo + lane * CL_CS + w;
#pragma unroll 2
        for (int hy = 0; hy < CL_HY; ++hy) {
            const int roff = wrap1(ty0 - H + hy, Gy) * Gx;
#pragma unroll
            for (int k = 0; k < 4; ++k) cp_async8(dst + hy * CL_HX * CL_CS + 8 * k, src[k] + roff, ok[k]);
        }
    }
    // weights: per tile row, the two 8-column blocks are 2 x 49 x 8 contiguous floats
    {
        const int xb0 = tx0 / 8;
        for (int e = threadIdx.x; e < CL_TY * 2 * 49 * 2; e += blockDim.x) {
            const int yy = e / 196, rem = e - yy * 196;   // rem = (s * 49 + d) * 2 + half
            const int s = rem / 98;
            const int y = ty0 + yy, xb = xb0 + s;
            const bool ok = y < Gy && xb < nxb;
            const float* src = T8 + (ok ? ((int64_t)y * nxb + xb0) * 392 + rem * 4 : 0);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(wts + e);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                         "r"(ok ? 16 : 0)
                         : "memory");
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int yy = w >> 1, s = w & 1;
    const float4* wq = wts + (yy * 2 + s) * 49 * 2;
    float2 acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int dy = 0; dy < D; ++dy) {
        const float2* hrow = halo + ((yy + dy) * CL_HX + 8 * s) * CL_CS + lane;
        float2 xv[14];
#pragma unroll
        for (int j = 0; j < 14; ++j) xv[j] = hrow[j * CL_CS];
#pragma unroll
        for (int dx = 0; dx < D; ++dx) {
            const float4 wa = wq[(dy * D + dx) * 2], wb = wq[(dy * D + dx) * 2 + 1];
            const float wr[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                acc[r].x += wr[r] * xv[r + dx].x;
                acc[r].y += wr[r] * xv[r + dx].y;
            }
        }
    }
    __syncthreads();   // every warp is done with the halo: reuse it for the transpose
#pragma unroll
    for (int r = 0; r < 8; ++r) halo[(yy * CL_TX + 8 * s + r) * CL_CS + lane] = acc[r];
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * CL_TY * CL_TX; e += blockDim.x) {
        const int x = e & (CL_TX - 1), y2 = (e / CL_TX) & (CL_TY - 1), c = e / (CL_TX * CL_TY);
        const int gx = tx0 + x, gy = ty0 + y2;
        if (c0 + c < C && gx < Gx && gy < Gy)
            grid_out[(int64_t)(c0 + c) * plane + gy * Gx + gx] = halo[(y2 * CL_TX + x) * CL_CS + c];
    }
}

template <int R, int CG, int NWY>
constexpr size_t rb_smem() {
    return sizeof(float4) * 2 * (CG / 2) * (R * NWY + 6) * (32 + 6);
}

// Row stage k rows -> image for many coils: the FFT batch runs over 8 coils
// of one image row, so a CTA per row covers every coil in ceil(C/8) rounds.
// Same result as rows_adj_kernel (conj-coil reduction + axpy epilogue).
template <int KO>
__global__ void __launch_bounds__(kThreads)
rows_adj_cb_kernel(FftDesc fd, const float2* __restrict__ tw, RowArgs a,
                   const float2* __restrict__ src, const float2* __restrict__ sens,
                   const float* __restrict__ wrow, const float* __restrict__ wcol, float2* out,
                   const float2* operand, float alpha, int ncoils) {
    extern __shared__ float2 sm[];
    const int G = a.G, n = a.n, bs = row_stride(G);
    float2* tws = sm;
    float2* b0 = sm + G;
    float2* b1 = b0 + RB * bs;
    load_table(tws, tw, G);
    const int r = blockIdx.x;
    const float wr = wrow ? wrow[r] : 1.f;
    float2 acc[KO];
#pragma unroll
    for (int k = 0; k < KO; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int c0 = 0; c0 < ncoils; c0 += RB) {
        for (int idx = threadIdx.x; idx < RB * G; idx += blockDim.x) {
            const int b = idx / G;
            const int p = idx - b * G;
            const int c = c0 + b;
            int s = p + a.off_in;
            if (s >= G) s -= G;
            b0[p + b * bs] = (c < ncoils) ? src[((int64_t)c * a.nrows + r) * G + s] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2* res = fft_batch<true>(b0, b1, fd, 1, bs, LGRB, tws, nullptr);
#pragma unroll
        for (int k = 0; k < KO; ++k) {
            const int i = threadIdx.x + k * kThreads;
            if (i < n) {
                int p = i - a.off_out;
                if (p < 0) p += G;
                const float w = wcol ? wr * wcol[i] : wr;
                for (int b = 0; b < RB; ++b) {
                    const int c = c0 + b;
                    if (c >= ncoils) break;
                    float2 v = cscale(res[p + b * bs], w);
                    if (sens) v = cmulc(sens[(int64_t)c * a.coil_img_stride + (int64_t)r * n + i], v);
                    acc[k] = cadd(acc[k], v);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KO; ++k) {
        const int i = threadIdx.x + k * kThreads;
        if (i < n) {
            const int64_t o = (int64_t)r * n + i;
            float2 v = cscale(acc[k], a.scale);
            if (operand) v = cadd(v, cscale(operand[o], alpha));
            out[o] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Orthonormal Haar prox on 2^L-tiles.  The one-level 2-D (3-D) Haar of a 2x2
// (2x2x2) block is H (x) H ((x) H) with H = [[1,1],[1,-1]]/sqrt(2): symmetric
// and orthogonal, so it is its own inverse.  Level 2 applies the same block
// transform to the level-1 approximation coefficients of a 4x4 (4x4x4) tile;
// the inverse runs the levels in reverse order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void haar2x2(float2& a, float2& b, float2& c, float2& d) {
    // [a b; c d] (rows y, columns x) -> [LL HL; LH HH]
    const float2 s0 = cadd(a, b), d0 = csub(a, b), s1 = cadd(c, d), d1 = csub(c, d);
    a = cscale(cadd(s0, s1), 0.5f);
    b = cscale(cadd(d0, d1), 0.5f);
    c = cscale(csub(s0, s1), 0.5f);
    d = cscale(csub(d0, d1), 0.5f);
}

__device__ __forceinline__ void haar2x2x2(float2* t /*[z][y][x], 8*/) {
    haar2x2(t[0], t[1], t[2], t[3]);
    haar2x2(t[4], t[5], t[6], t[7]);
    const float r = 0.70710678118654752f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 a = t[i], b = t[4 + i];
        t[i] = cscale(cadd(a, b), r);
        t[4 + i] = cscale(csub(a, b), r);
    }
}

// Block transform on the 2x2(x2) blocks with corner (sz, sy, sx) step `st`
// inside a TS-tile held in registers, index (z*TS + y)*TS + x.
template <int NDIM, int TS>
__device__ __forceinline__ void haar_blocks(float2* v, int st) {
    if (NDIM == 2) {
#pragma unroll
        for (int by = 0; by < TS; by += 2 * st)
#pragma unroll
            for (int bx = 0; bx < TS; bx += 2 * st)
                haar2x2(v[by * TS + bx], v[by * TS + bx + st], v[(by + st) * TS + bx],
                        v[(by + st) * TS + bx + st]);
    } else {
#pragma unroll
        for (int bz = 0; bz < TS; bz += 2 * st)
#pragma unroll
            for (int by = 0; by < TS; by += 2 * st)
#pragma unroll
                for (int bx = 0; bx < TS; bx += 2 * st) {
                    float2 t[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        t[q] = v[((bz + (q >> 2) * st) * TS + by + ((q >> 1) & 1) * st) * TS + bx +
                                 (q & 1) * st];
                    haar2x2x2(t);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        v[((bz + (q >> 2) * st) * TS + by + ((q >> 1) & 1) * st) * TS + bx +
                          (q & 1) * st] = t[q];
                }
    }
}

__device__ __forceinline__ float2 soft(float2 v, float lam) {
    const float m2 = v.x * v.x + v.y * v.y;
    // |v| <= lambda -> 0 (also v = 0, so no 0 * inf); a NaN fails the test and
    // stays NaN instead of being thresholded to 0
    if (m2 <= lam * lam) return make_float2(0.f, 0.f);
    return cscale(v, 1.f - lam * rsqrtf(m2));
}

template <int NDIM, int LEVELS>
__device__ __forceinline__ void prox_tile(float2* v, float lam) {
    constexpr int TS = 1 << LEVELS;
    haar_blocks<NDIM, TS>(v, 1);
    if (LEVELS == 2) haar_blocks<NDIM, TS>(v, 2);
    constexpr int NV = (NDIM == 2) ? TS * TS : TS * TS * TS;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = soft(v[i], lam);
    if (LEVELS == 2) haar_blocks<NDIM, TS>(v, 2);
    haar_blocks<NDIM, TS>(v, 1);
}

// Tile (thread) t covers x in [tx*TS, +TS), y in [ty*TS, +TS), z in [tz*TS, +TS).
template <int NDIM, int LEVELS>
__device__ __forceinline__ int64_t tile_origin(int64_t t, int nx, int ny, int nz, bool& ok) {
    constexpr int TS = 1 << LEVELS;
    const int64_t ntx = nx / TS, nty = ny / TS, ntz = (NDIM == 3) ? nz / TS : 1;
    ok = t < ntx * nty * ntz;
    const int64_t tx = t % ntx;
    const int64_t r = t / ntx;
    const int64_t ty = r % nty;
    const int64_t tz = r / nty;
    return ((tz * TS) * ny + ty * TS) * (int64_t)nx + tx * TS;
}

template <int NDIM, int LEVELS>
__global__ void __launch_bounds__(kThreads)
prox_kernel(int nx, int ny, int nz, float lam, const float2* __restrict__ in,
            float2* __restrict__ out) {
    constexpr int TS = 1 << LEVELS;
    constexpr int ZS = (NDIM == 3) ? TS : 1;
    bool ok;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t o = tile_origin<NDIM, LEVELS>(t, nx, ny, nz, ok);
    if (!ok) return;
    float2 v[ZS * TS * TS];
#pragma unroll
    for (int z = 0; z < ZS; ++z)
#pragma unroll
        for (int y = 0; y < TS; ++y)
#pragma unroll
            for (int x = 0; x < TS; ++x)
                v[(z * TS + y) * TS + x] = in[o + ((int64_t)z * ny + y) * nx + x];
    prox_tile<NDIM, LEVELS>(v, lam);
#pragma unroll
    for (int z = 0; z < ZS; ++z)
#pragma unroll
        for (int y = 0; y < TS; ++y)
#pragma unroll
            for (int x = 0; x < TS; ++x)
                out[o + ((int64_t)z * ny + y) * nx + x] = v[(z * TS + y) * TS + x];
}

// Fused prox + momentum of Algorithm "pfista":
//   y_new = prox(z - gamma*u);  z <- y_new + beta (y_new - y);  y <- y_new.
// Optional FP64 statistics ||y_new - y||^2, ||y_new||^2 into hist[0..1].
template <int NDIM, int LEVELS>
__global__ void __launch_bounds__(kThreads)
prox_fista_kernel(int nx, int ny, int nz, float lam, float gamma, float beta,
                  float2* __restrict__ z, const float2* __restrict__ u, float2* __restrict__ y,
                  const float2* __restrict__ ref, double* __restrict__ hist) {
    constexpr int TS = 1 << LEVELS;
    constexpr int ZS = (NDIM == 3) ? TS : 1;
    pdl_trigger();
    pdl_wait();
    bool ok;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t o = tile_origin<NDIM, LEVELS>(t, nx, ny, nz, ok);
    double dd = 0.0, yy = 0.0, rr = 0.0;
    if (ok) {
        float2 v[ZS * TS * TS];
#pragma unroll
        for (int zz = 0; zz < ZS; ++zz)
#pragma unroll
            for (int r = 0; r < TS; ++r)
#pragma unroll
                for (int x = 0; x < TS; ++x) {
                    const int64_t a = o + ((int64_t)zz * ny + r) * nx + x;
                    const float2 zv = z[a], uv = u[a];
                    v[(zz * TS + r) * TS + x] = make_float2(zv.x - gamma * uv.x, zv.y - gamma * uv.y);
                }
        prox_tile<NDIM, LEVELS>(v, lam);
#pragma unroll
        for (int zz = 0; zz < ZS; ++zz)
#pragma unroll
            for (int r = 0; r < TS; ++r)
#pragma unroll
                for (int x = 0; x < TS; ++x) {
                    const int64_t a = o + ((int64_t)zz * ny + r) * nx + x;
                    const float2 yn = v[(zz * TS + r) * TS + x];
                    const float2 yo = y[a];
                    const float2 df = csub(yn, yo);
                    z[a] = make_float2(yn.x + beta * df.x, yn.y + beta * df.y);
                    y[a] = yn;
                    if (hist) {
                        dd += (double)df.x * df.x + (double)df.y * df.y;
                        yy += (double)yn.x * yn.x + (double)yn.y * yn.y;
                    }
                    if (ref) {
                        const float2 rv = ref[a];
                        const double ex = (double)yn.x - rv.x, ey = (double)yn.y - rv.y;
                        rr += ex * ex + ey * ey;
                    }
                }
    }
    if (hist) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dd += __shfl_down_sync(0xffffffffu, dd, off);
            yy += __shfl_down_sync(0xffffffffu, yy, off);
            rr += __shfl_down_sync(0xffffffffu, rr, off);
        }
        __shared__ double sd[kThreads / 32], sy[kThreads / 32], sr[kThreads / 32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            sd[wid] = dd;
            sy[wid] = yy;
            sr[wid] = rr;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                a += sd[i];
                b += sy[i];
                c += sr[i];
            }
            atomicAdd(&hist[0], a);
            atomicAdd(&hist[1], b);
            atomicAdd(&hist[2], c);
        }
    }
}

// 2-D, 2-level variant of prox_fista_kernel with four threads per 4x4 tile:
// a thread owns one 2x2 block (level 1 in registers); the level-2 transform
// of the tile's four approximation coefficients runs across the four
// threads with shuffles (x partner lane ^ 1, y partner lane ^ 16), in the
// same operation order as haar2x2.  A warp covers 2 block rows x 16 block
// columns (one tile row of 8 tiles).  Needs nx % 32 == 0 and ny % 4 == 0.
__device__ __forceinline__ float2 haar_l2_shfl(float2 a, int qx, int qy) {
    float2 p;
    p.x = __shfl_xor_sync(0xffffffffu, a.x, 1);
    p.y = __shfl_xor_sync(0xffffffffu, a.y, 1);
    const float2 t = qx ? csub(p, a) : cadd(a, p);      // row sum (qx 0) or difference (qx 1)
    float2 u;
    u.x = __shfl_xor_sync(0xffffffffu, t.x, 16);
    u.y = __shfl_xor_sync(0xffffffffu, t.y, 16);
    return cscale(qy ? csub(u, t) : cadd(t, u), 0.5f);
}

__global__ void __launch_bounds__(kThreads)
prox_fista2q_kernel(int nx, int ny, float lam, float gamma, float beta, float2* __restrict__ z,
                    const float2* __restrict__ u, float2* __restrict__ y,
                    const float2* __restrict__ ref, double* __restrict__ hist) {
    pdl_trigger();
    pdl_wait();
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, qx = lane & 1, qy = (lane >> 4) & 1;
    const int nwc = nx / 32;
    const int64_t W = g >> 5;
    const bool ok = W < (int64_t)(ny / 4) * nwc;   // warp-uniform
    double dd = 0.0, yy = 0.0, rr = 0.0;
    if (ok) {
        const int wr = (int)(W / nwc), wc = (int)(W - (int64_t)wr * nwc);
        const int by = 2 * wr + (lane >> 4), bx = 16 * wc + (lane & 15);
        const int64_t o0 = (int64_t)(2 * by) * nx + 2 * bx, o1 = o0 + nx;
        const float4 z0 = *reinterpret_cast<const float4*>(z + o0);
        const float4 z1 = *reinterpret_cast<const float4*>(z + o1);
        const float4 u0 = *reinterpret_cast<const float4*>(u + o0);
        const float4 u1 = *reinterpret_cast<const float4*>(u + o1);
        float2 a = make_float2(z0.x - gamma * u0.x, z0.y - gamma * u0.y);
        float2 b = make_float2(z0.z - gamma * u0.z, z0.w - gamma * u0.w);
        float2 c = make_float2(z1.x - gamma * u1.x, z1.y - gamma * u1.y);
        float2 d = make_float2(z1.z - gamma * u1.z, z1.w - gamma * u1.w);
        haar2x2(a, b, c, d);
        a = haar_l2_shfl(a, qx, qy);
        a = soft(a, lam);
        b = soft(b, lam);
        c = soft(c, lam);
        d = soft(d, lam);
        a = haar_l2_shfl(a, qx, qy);
        haar2x2(a, b, c, d);
        const float4 y0 = *reinterpret_cast<const float4*>(y + o0);
        const float4 y1 = *reinterpret_cast<const float4*>(y + o1);
        const float2 yo[4] = {make_float2(y0.x, y0.y), make_float2(y0.z, y0.w),
                              make_float2(y1.x, y1.y), make_float2(y1.z, y1.w)};
        const float2 yn[4] = {a, b, c, d};
        float2 zn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 df = csub(yn[k], yo[k]);
            zn[k] = make_float2(yn[k].x + beta * df.x, yn[k].y + beta * df.y);
            if (hist) {   // FP64 arithmetic is slow on this part: only when asked for
                dd += (double)df.x * df.x + (double)df.y * df.y;
                yy += (double)yn[k].x * yn[k].x + (double)yn[k].y * yn[k].y;
            }
        }
        *reinterpret_cast<float4*>(z + o0) = make_float4(zn[0].x, zn[0].y, zn[1].x, zn[1].y);
        *reinterpret_cast<float4*>(z + o1) = make_float4(zn[2].x, zn[2].y, zn[3].x, zn[3].y);
        *reinterpret_cast<float4*>(y + o0) = make_float4(a.x, a.y, b.x, b.y);
        *reinterpret_cast<float4*>(y + o1) = make_float4(c.x, c.y, d.x, d.y);
        if (ref) {
            const float4 r0 = *reinterpret_cast<const float4*>(ref + o0);
            const float4 r1 = *reinterpret_cast<const float4*>(ref + o1);
            const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double ex = (double)yn[k].x - rv[2 * k], ey = (double)yn[k].y - rv[2 * k + 1];
                rr += ex * ex + ey * ey;
            }
        }
    }
    if (hist) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dd += __shfl_down_sync(0xffffffffu, dd, off);
            yy += __shfl_down_sync(0xffffffffu, yy, off);
            rr += __shfl_down_sync(0xffffffffu, rr, off);
        }
        __shared__ double sd[kThreads / 32], sy[kThreads / 32], sr[kThreads / 32];
        const int wid = threadIdx.x >> 5;
        if (lane == 0) {
            sd[wid] = dd;
            sy[wid] = yy;
            sr[wid] = rr;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                s0 += sd[i];
                s1 += sy[i];
                s2 += sr[i];
            }
            atomicAdd(&hist[0], s0);
            atomicAdd(&hist[1], s1);
            atomicAdd(&hist[2], s2);
        }
    }
}

// 3-D, 2-level Haar prox with eight threads per 4x4x4 tile: a thread owns one
// 2x2x2 block (level 1 in registers); the level-2 transform of the tile's
// eight approximation coefficients runs across the eight threads with
// shuffles (x partner lane ^ 1, y partner lane ^ 8, z partner lane ^ 16), in
// haar2x2x2's operation order.  A warp covers 8 block columns x 2 block rows
// x 2 block planes.  Needs nx % 16 == 0 and ny, nz % 4 == 0.
__device__ __forceinline__ float2 haar3_l2_shfl(float2 a, int qx, int qy, int qz) {
    float2 p;
    p.x = __shfl_xor_sync(0xffffffffu, a.x, 1);
    p.y = __shfl_xor_sync(0xffffffffu, a.y, 1);
    const float2 t = qx ? csub(p, a) : cadd(a, p);
    float2 u;
    u.x = __shfl_xor_sync(0xffffffffu, t.x, 8);
    u.y = __shfl_xor_sync(0xffffffffu, t.y, 8);
    const float2 v = cscale(qy ? csub(u, t) : cadd(t, u), 0.5f);
    float2 w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, 16);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, 16);
    return cscale(qz ? csub(w, v) : cadd(v, w), 0.70710678118654752f);
}

// FISTA = false: out = prox(in).  FISTA = true: the fused step of
// prox_fista_kernel with z read from `in` and written to `out` (same array).
template <bool FISTA>
__global__ void __launch_bounds__(kThreads)
prox3q_kernel(int nx, int ny, int nz, float lam, float gamma, float beta, const float2* in,
              const float2* __restrict__ u, float2* out, float2* __restrict__ y,
              const float2* __restrict__ ref, double* __restrict__ hist) {
    pdl_trigger();
    pdl_wait();
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, qx = lane & 1, qy = (lane >> 3) & 1, qz = lane >> 4;
    const int nwx = nx / 16, nwy = ny / 4;
    const int64_t W = g >> 5;
    const bool ok = W < (int64_t)nwx * nwy * (nz / 4);   // warp-uniform
    double dd = 0.0, yy = 0.0, rr = 0.0;
    if (ok) {
        const int wx = (int)(W % nwx);
        const int64_t rest = W / nwx;
        const int wy = (int)(rest % nwy), wz = (int)(rest / nwy);
        const int bx = 8 * wx + (lane & 7), by = 2 * wy + qy, bz = 2 * wz + qz;
        int64_t o[4];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                o[k * 2 + j] = ((int64_t)(2 * bz + k) * ny + (2 * by + j)) * nx + 2 * bx;
        float2 t[8];   // [z][y][x]
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(in + o[q]);
            float2 e0 = make_float2(a.x, a.y), e1 = make_float2(a.z, a.w);
            if (FISTA) {
                const float4 b = *reinterpret_cast<const float4*>(u + o[q]);
                e0 = make_float2(a.x - gamma * b.x, a.y - gamma * b.y);
                e1 = make_float2(a.z - gamma * b.z, a.w - gamma * b.w);
            }
            t[2 * q] = e0;
            t[2 * q + 1] = e1;
        }
        haar2x2x2(t);
        t[0] = haar3_l2_shfl(t[0], qx, qy, qz);
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = soft(t[q], lam);
        t[0] = haar3_l2_shfl(t[0], qx, qy, qz);
        haar2x2x2(t);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (FISTA) {
                const float4 yo4 = *reinterpret_cast<const float4*>(y + o[q]);
                const float2 yo[2] = {make_float2(yo4.x, yo4.y), make_float2(yo4.z, yo4.w)};
                float2 zn[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 yn = t[2 * q + h];
                    const float2 df = csub(yn, yo[h]);
                    zn[h] = make_float2(yn.x + beta * df.x, yn.y + beta * df.y);
                    if (hist) {
                        dd += (double)df.x * df.x + (double)df.y * df.y;
                        yy += (double)yn.x * yn.x + (double)yn.y * yn.y;
                    }
                }
                if (ref) {
                    const float4 rv = *reinterpret_cast<const float4*>(ref + o[q]);
                    const double e0 = (double)t[2 * q].x - rv.x, e1 = (double)t[2 * q].y - rv.y;
                    const double e2 = (double)t[2 * q + 1].x - rv.z, e3 = (double)t[2 * q + 1].y - rv.w;
                    rr += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
                }
                *reinterpret_cast<float4*>(out + o[q]) = make_float4(zn[0].x, zn[0].y, zn[1].x, zn[1].y);
                *reinterpret_cast<float4*>(y + o[q]) =
                    make_float4(t[2 * q].x, t[2 * q].y, t[2 * q + 1].x, t[2 * q + 1].y);
            } else {
                *reinterpret_cast<float4*>(out + o[q]) =
                    make_float4(t[2 * q].x, t[2 * q].y, t[2 * q + 1].x, t[2 * q + 1].y);
            }
        }
    }
    if (FISTA && hist) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dd += __shfl_down_sync(0xffffffffu, dd, off);
            yy += __shfl_down_sync(0xffffffffu, yy, off);
            rr += __shfl_down_sync(0xffffffffu, rr, off);
        }
        __shared__ double sd[kThreads / 32], sy[kThreads / 32], sr[kThreads / 32];
        const int wid = threadIdx.x >> 5;
        if (lane == 0) {
            sd[wid] = dd;
            sy[wid] = yy;
            sr[wid] = rr;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                s0 += sd[i];
                s1 += sy[i];
                s2 += sr[i];
            }
            atomicAdd(&hist[0], s0);
            atomicAdd(&hist[1], s1);
            atomicAdd(&hist[2], s2);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions (deterministic: fixed grid, per-block partials, one
// finishing block).  partial layout [nblocks][3] = Re<a,b>, Im<a,b>, |b|^2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
dot_partial_kernel(const float2* __restrict__ a, const float2* __restrict__ b, int64_t n,
                   double* __restrict__ partials) {
    double re = 0.0, im = 0.0, nb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 bv = b[i];
        if (a) {
            const float2 av = a[i];
            re += (double)av.x * bv.x + (double)av.y * bv.y;
            im += (double)av.x * bv.y - (double)av.y * bv.x;
        }
        nb += (double)bv.x * bv.x + (double)bv.y * bv.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, off);
        im += __shfl_down_sync(0xffffffffu, im, off);
        nb += __shfl_down_sync(0xffffffffu, nb, off);
    }
    __shared__ double s[3][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][wid] = re;
        s[1][wid] = im;
        s[2][wid] = nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0, r2 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            r0 += s[0][i];
            r1 += s[1][i];
            r2 += s[2][i];
        }
        partials[3 * blockIdx.x + 0] = r0;
        partials[3 * blockIdx.x + 1] = r1;
        partials[3 * blockIdx.x + 2] = r2;
    }
}

__global__ void dot_final_kernel(const double* __restrict__ partials, int nblocks,
                                 double* __restrict__ out_re, double* __restrict__ out_nb) {
    __shared__ double s[2][kThreads];
    double re = 0.0, nb = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        re += partials[3 * i];
        nb += partials[3 * i + 2];
    }
    s[0][threadIdx.x] = re;
    s[1][threadIdx.x] = nb;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (out_re) *out_re = s[0][0];
        if (out_nb) *out_nb = s[1][0];
    }
}

// out = in * factor / sqrt(norm2) (invert) or in * factor * sqrt(norm2)
__global__ void scale_by_norm_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                     int64_t n, const double* __restrict__ norm2, double factor,
                                     int invert) {
    const double nv = sqrt(*norm2);
    // a zero norm scales by 0 (b = 0 has the solution 0); a NaN or infinite
    // norm scales by NaN, so a non-finite input is not turned into zeros
    const double fi = isfinite(nv) ? (nv > 0.0 ? factor / nv : 0.0) : __longlong_as_double(0x7ff8000000000000ll);
    const float f = (float)(invert ? fi : factor * nv);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cscale(in[i], f);
}

__global__ void axpby_kernel(const float2* __restrict__ x, float a, const float2* __restrict__ y,
                             float b, float2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = cscale(x[i], a);
        if (y) v = cadd(v, cscale(y[i], b));
        out[i] = v;
    }
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
// output j mixes seed + (j+1) * 0x9E3779B97F4A7C15.  Entry i of the start
// vector is (2u_{2i} - 1) + i (2u_{2i+1} - 1), u_j = (out_j >> 11) 2^-53.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j) {
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void start_vector_kernel(float2* __restrict__ v, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double u0 = (double)(splitmix64_at(seed, 2 * i) >> 11) * 0x1.0p-53;
        const double u1 = (double)(splitmix64_at(seed, 2 * i + 1) >> 11) * 0x1.0p-53;
        v[i] = make_float2((float)(2.0 * u0 - 1.0), (float)(2.0 * u1 - 1.0));
    }
}

inline int ew_blocks(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ===========================================================================
// Launchers
// ===========================================================================
thread_local int64_t g_launches = 0;
thread_local Profiler* g_profiler = nullptr;

static pp_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    if (g_profiler) g_profiler->mark(what);
    return PP_OK;
}

static size_t rows_smem(int G) { return sizeof(float2) * (size_t)(G + 2 * RB * row_stride(G)); }
static size_t cols_smem(int G) { return sizeof(float2) * (size_t)(G + 2 * G * TX); }

pp_status configure_kernels() {
    const int big = 200 * 1024;
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cols_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cols_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cols_roundtrip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d_normal_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d_normal_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d_normal_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(cart2d_normal_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_cb_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(rows_adj_cb_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    PP_TRY_CUDA(cudaFuncSetAttribute(nufft_spread_tile_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    return PP_OK;
}

pp_status launch_rows_fwd(const Plan& p, const DevFft& f, const RowArgs& a, const float2* x,
                          const float2* sens, const float* wrow, const float* wcol, float2* out,
                          int ncoils, int64_t img_batch_stride, cudaStream_t st) {
    (void)p;
    bool done = false;
    PP_TRY(launch_rows4_fwd(f, a, x, sens, wrow, wcol, out, ncoils, img_batch_stride, st, &done));
    if (done) return PP_OK;
    dim3 grid((a.nrows + RB - 1) / RB, ncoils);
    rows_fwd_kernel<<<grid, kThreads, rows_smem(a.G), st>>>(f.d, f.tw, a, x, img_batch_stride, sens,
                                                            wrow, wcol, out);
    return check_launch("rows_fwd_kernel");
}

pp_status launch_rows_adj(const Plan& p, const DevFft& f, const RowArgs& a, const float2* src,
                          const float2* sens, const float* wrow, const float* wcol, float2* out,
                          const float2* operand, float alpha, int ncoils, cudaStream_t st) {
    (void)p;
    bool done = false;
    PP_TRY(launch_rows4_adj(f, a, src, sens, wrow, wcol, out, operand, alpha, ncoils, st, &done,
                            p.tune_rows_adj_cl));
    if (done) return PP_OK;
    if (RB * a.n > KMAX * kThreads) {
        set_error("row length %d exceeds the row stage limit", a.n);
        return PP_ERR_UNSUPPORTED;
    }
    if (ncoils >= 4 && a.n <= 2 * kThreads) {
        const size_t smc = rows_smem(a.G);
        if (a.n <= kThreads)
            rows_adj_cb_kernel<1><<<a.nrows, kThreads, smc, st>>>(f.d, f.tw, a, src, sens, wrow, wcol,
                                                                   out, operand, alpha, ncoils);
        else
            rows_adj_cb_kernel<2><<<a.nrows, kThreads, smc, st>>>(f.d, f.tw, a, src, sens, wrow, wcol,
                                                                   out, operand, alpha, ncoils);
        return check_launch("rows_adj_cb_kernel");
    }
    dim3 grid((a.nrows + RB - 1) / RB);
    const int need = (RB * a.n + kThreads - 1) / kThreads;
    const size_t sm = rows_smem(a.G);
#define PP_ROWS_ADJ(KM_) rows_adj_kernel<KM_><<<grid, kThreads, sm, st>>>(f.d, f.tw, a, src, sens, wrow, wcol, out, operand, alpha, ncoils)
    if (need <= 4) PP_ROWS_ADJ(4);
    else if (need <= 8) PP_ROWS_ADJ(8);
    else if (need <= 12) PP_ROWS_ADJ(12);
    else PP_ROWS_ADJ(16);
#undef PP_ROWS_ADJ
    return check_launch("rows_adj_kernel");
}

pp_status launch_cols(const DevFft& f, const ColArgs& a, const float2* src, float2* dst, bool inv,
                      cudaStream_t st) {
    bool done = false;
    PP_TRY(launch_cols4(f, a, src, dst, inv, st, &done));
    if (done) return PP_OK;
    dim3 grid((a.ncols + TX - 1) / TX, a.nbatch);
    if (inv)
        cols_kernel<true><<<grid, kThreads, cols_smem(a.G), st>>>(f.d, f.tw, a, src, dst);
    else
        cols_kernel<false><<<grid, kThreads, cols_smem(a.G), st>>>(f.d, f.tw, a, src, dst);
    return check_launch("cols_kernel");
}

pp_status launch_cols_roundtrip(const DevFft& f, const ColArgs& a, const float* mask_fo,
                                const float2* src, float2* dst, cudaStream_t st) {
    dim3 grid((a.ncols + TX - 1) / TX, a.nbatch);
    cols_roundtrip_kernel<<<grid, kThreads, cols_smem(a.G), st>>>(f.d, f.tw, a, mask_fo, src, dst);
    return check_launch("cols_roundtrip_kernel");
}

pp_status launch_cart2d_normal(const Plan& p, const float2* x, float2* out, float scale,
                               const float2* operand, float alpha, cudaStream_t st) {
    bool done = false;
    PP_TRY(launch_cart2d4_normal(p, x, out, scale, operand, alpha, st, &done));
    if (done) return PP_OK;
    if (p.ny * TX > KMAX * kThreads) {
        set_error("ny = %d exceeds the fused Cartesian kernel limit", p.ny);
        return PP_ERR_UNSUPPORTED;
    }
    dim3 grid((p.nx + TX - 1) / TX);
    const size_t smem = sizeof(float2) * (size_t)(p.ny + 2 * p.ny * TX) + sizeof(float) * p.ny;
    const int need = (p.ny * TX + kThreads - 1) / kThreads;
#define PP_CART(KM_) cart2d_normal_kernel<KM_><<<grid, kThreads, smem, st>>>(p.fy.d, p.fy.tw, x, p.sens, p.C, p.ny, p.nx, p.mask_fo, out, scale, operand, alpha)
    if (need <= 4) PP_CART(4);
    else if (need <= 8) PP_CART(8);
    else if (need <= 12) PP_CART(12);
    else PP_CART(16);
#undef PP_CART
    return check_launch("cart2d_normal_kernel");
}

pp_status launch_expand(const float2* x, const float2* s, float2* out, int64_t n, cudaStream_t st) {
    expand_kernel<<<ew_blocks(n), kThreads, 0, st>>>(x, s, out, n);
    return check_launch("expand_kernel");
}

pp_status launch_conj_accum(const float2* s, const float2* wv, float2* out, int64_t n, int first,
                            float scale, const float2* operand, float alpha, int last,
                            cudaStream_t st) {
    conj_accum_kernel<<<ew_blocks(n), kThreads, 0, st>>>(s, wv, out, n, first, scale, operand, alpha,
                                                          last);
    return check_launch("conj_accum_kernel");
}

static size_t tile_smem(const Plan& p) { return sizeof(float2) * (size_t)p.T * p.T; }

template <int R, int CG, int NWY>
static pp_status rb_prepare(const Plan& p, int* grid) {
    auto fn = gtg_stencil_rb_kernel<R, CG, NWY>;
    constexpr size_t sm = rb_smem<R, CG, NWY>();
    PP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int occ = 0, nsm = 0, dev = 0;
    PP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * NWY, sm));
    PP_TRY_CUDA(cudaGetDevice(&dev));
    PP_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nitems = (int64_t)((p.G_x + 31) / 32) * ((p.G_y + R * NWY - 1) / (R * NWY)) *
                           ((p.C + CG - 1) / CG);
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)std::max(occ, 1) * nsm));
    return PP_OK;
}

template <int R, int CG, int NWY>
static pp_status rb_launch(const Plan& p, int grid, const float2* in, float2* out, cudaStream_t st) {
    gtg_stencil_rb_kernel<R, CG, NWY><<<grid, 32 * NWY, rb_smem<R, CG, NWY>(), st>>>(
        p.gtg, p.G_x, p.G_y, p.C, in, out);
    return check_launch("gtg_stencil_rb_kernel");
}

// G^T G of the gridding pair as (2W-1)^2 weight planes, built on the device:
// for every sample and every pair of its taps j, j' (offset d = j' - j),
// T[d][j] += phi_j phi_j' with the products and sums in FP64 (atomic adds:
// only the order of the additions differs from a sequential build).
__global__ void gtg_accumulate_kernel(const SampleTaps* __restrict__ samp, int K, int Gx, int Gy,
                                      double* __restrict__ T) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const SampleTaps s = samp[k];
    const double wx[4] = {s.wx.x, s.wx.y, s.wx.z, s.wx.w};
    const double wy[4] = {s.wy.x, s.wy.y, s.wy.z, s.wy.w};
    const int64_t plane = (int64_t)Gx * Gy;
    int gy[4], gx[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int yv = (s.iy0 + b) % Gy, xv = (s.ix0 + b) % Gx;
        gy[b] = yv < 0 ? yv + Gy : yv;
        gx[b] = xv < 0 ? xv + Gx : xv;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double pj = wy[b] * wx[a];
            double* Tj = T + (int64_t)gy[b] * Gx + gx[a];
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
                for (int a2 = 0; a2 < 4; ++a2)
                    atomicAdd(Tj + (int64_t)((b2 - b + 3) * 7 + (a2 - a + 3)) * plane, pj * (wy[b2] * wx[a2]));
        }
}

// FP32 copies of the planes: Tf[d][y][x], and T8[y][x/8][d][x%8] (zero past Gx).
__global__ void gtg_convert_kernel(const double* __restrict__ T, int Gx, int Gy, int nxb,
                                   float* __restrict__ Tf, float* __restrict__ T8) {
    const int64_t plane = (int64_t)Gx * Gy, n8 = (int64_t)Gy * nxb * 49 * 8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n8;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int xl = (int)(e & 7);
        int64_t r = e >> 3;
        const int d = (int)(r % 49);
        r /= 49;
        const int xb = (int)(r % nxb), y = (int)(r / nxb), x = xb * 8 + xl;
        float v = 0.f;
        if (x < Gx) {
            const int64_t i = (int64_t)d * plane + (int64_t)y * Gx + x;
            v = (float)T[i];
            Tf[i] = v;
        }
        T8[e] = v;
    }
}

pp_status build_gtg_device(Plan& p, cudaStream_t st) {
    const int Gx = p.G_x, Gy = p.G_y, nxb = (Gx + 7) / 8;
    const size_t planes = (size_t)49 * Gx * Gy;
    double* T = nullptr;
    PP_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&T), planes * sizeof(double), st));
    pp_status rc = PP_OK;
    cudaError_t e = cudaMemsetAsync(T, 0, planes * sizeof(double), st);
    if (e == cudaSuccess) {
        gtg_accumulate_kernel<<<(p.K + 127) / 128, 128, 0, st>>>(p.samp, p.K, Gx, Gy, T);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        gtg_convert_kernel<<<152 * 8, kThreads, 0, st>>>(T, Gx, Gy, nxb, p.gtg, p.gtg8);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_status(e, "gtg build");
    cudaFreeAsync(T, st);
    return rc;
}

pp_status prepare_gtg_stencil(Plan& p) {
    // the register-blocked kernels index the weight planes with 32-bit offsets
    if ((int64_t)49 * p.G_x * p.G_y >= ((int64_t)1 << 31)) return PP_OK;
    if (p.gtg8)
        PP_TRY_CUDA(cudaFuncSetAttribute(gtg_stencil_cl_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM));
    PP_TRY((rb_prepare<4, 4, 4>(p, &p.stencil_rb_grid[0])));
    PP_TRY((rb_prepare<8, 4, 2>(p, &p.stencil_rb_grid[1])));
    PP_TRY((rb_prepare<4, 8, 4>(p, &p.stencil_rb_grid[2])));
    PP_TRY((rb_prepare<2, 8, 4>(p, &p.stencil_rb_grid[3])));
    return PP_OK;
}

pp_status launch_gtg_stencil(const Plan& p, const float2* grid_in, float2* grid_out, cudaStream_t st) {
    const int cpc = p.tune_stencil_cpc > 0 ? p.tune_stencil_cpc : 8;
    const int kind = p.tune_stencil_kind;
    if (kind == 6 && p.gtg8 && p.stencil_rb_grid[0] > 0) {
        const int64_t nitems = (int64_t)((p.G_x + CL_TX - 1) / CL_TX) * ((p.G_y + CL_TY - 1) / CL_TY) *
                               ((p.C + 31) / 32);
        gtg_stencil_cl_kernel<<<(unsigned)nitems, 256, CL_SMEM, st>>>(p.gtg8, p.G_x, p.G_y, p.C,
                                                                     (p.G_x + 7) / 8, grid_in, grid_out);
        return check_launch("gtg_stencil_cl_kernel");
    }
    if (kind >= 2 && kind <= 5 && p.stencil_rb_grid[kind - 2] > 0) {
        const int g = p.stencil_rb_grid[kind - 2];
        switch (kind) {
            case 2: return rb_launch<4, 4, 4>(p, g, grid_in, grid_out, st);
            case 3: return rb_launch<8, 4, 2>(p, g, grid_in, grid_out, st);
            case 4: return rb_launch<4, 8, 4>(p, g, grid_in, grid_out, st);
            default: return rb_launch<2, 8, 4>(p, g, grid_in, grid_out, st);
        }
    }
    if (kind == 1) {
        dim3 grid((p.G_x + 15) / 16, (p.G_y + 15) / 16, (p.C + cpc - 1) / cpc);
        gtg_stencil2_kernel<4><<<grid, 128, 0, st>>>(p.gtg, p.G_x, p.G_y, p.C, cpc, grid_in, grid_out);
        return check_launch("gtg_stencil2_kernel");
    }
    dim3 grid((p.G_x + 15) / 16, (p.G_y + 15) / 16, (p.C + cpc - 1) / cpc);
    gtg_stencil_kernel<4><<<grid, kThreads, 0, st>>>(p.gtg, p.G_x, p.G_y, p.C, cpc, grid_in, grid_out);
    return check_launch("gtg_stencil_kernel");
}

pp_status launch_nufft_spread(const Plan& p, const float2* ksp, float2* grid_out, cudaStream_t st) {
    const int cpc = 4;
    dim3 grid(p.ntx * p.nty, (p.C + cpc - 1) / cpc);
    nufft_spread_tile_kernel<4><<<grid, kThreads, tile_smem(p), st>>>(
        p.tiles, p.tile_start, p.T, p.ntx, p.G_x, p.G_y, p.C, cpc, ksp, p.K, grid_out);
    return check_launch("nufft_spread_tile_kernel");
}

pp_status launch_nufft_degrid(const Plan& p, const float2* grid_in, float2* ksp, cudaStream_t st) {
    dim3 grid((p.K + kThreads - 1) / kThreads, p.C);
    nufft_degrid_kernel<4><<<grid, kThreads, 0, st>>>(p.samp, p.K, p.G_x, p.G_y, grid_in, ksp);
    return check_launch("nufft_degrid_kernel");
}

pp_status launch_prox(int ndim, int nx, int ny, int nz, int levels, float lambda,
                      const float2* in, float2* out, cudaStream_t st) {
    const int ts = 1 << levels;
    const int64_t ntiles = (int64_t)(nx / ts) * (ny / ts) * (ndim == 3 ? nz / ts : 1);
    const int blocks = (int)((ntiles + kThreads - 1) / kThreads);
    if (blocks == 0) return PP_OK;
    if (ndim == 3 && levels == 2 && nx % 16 == 0 && ny % 4 == 0 && nz % 4 == 0 &&
        ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        const int64_t nthr = (int64_t)nx * ny * nz / 8;
        PP_TRY_CUDA(launch_ex(prox3q_kernel<false>, dim3((unsigned)((nthr + kThreads - 1) / kThreads)),
                              dim3(kThreads), 0, st, false, 0, nx, ny, nz, lambda, 0.f, 0.f, in,
                              (const float2*)nullptr, out, (float2*)nullptr, (const float2*)nullptr,
                              (double*)nullptr));
        return check_launch("prox3q_kernel");
    }
    if (ndim == 2 && levels == 1) prox_kernel<2, 1><<<blocks, kThreads, 0, st>>>(nx, ny, nz, lambda, in, out);
    else if (ndim == 2) prox_kernel<2, 2><<<blocks, kThreads, 0, st>>>(nx, ny, nz, lambda, in, out);
    else if (levels == 1) prox_kernel<3, 1><<<blocks, kThreads, 0, st>>>(nx, ny, nz, lambda, in, out);
    else prox_kernel<3, 2><<<blocks, kThreads, 0, st>>>(nx, ny, nz, lambda, in, out);
    return check_launch("prox_kernel");
}

pp_status launch_prox_fista(const Plan& p, int levels, float lambda, float gamma, float beta,
                            const float2* u, const float2* ref, double* hist_slot, cudaStream_t st) {
    const int ts = 1 << levels;
    const int64_t ntiles = (int64_t)(p.nx / ts) * (p.ny / ts) * (p.ndim == 3 ? p.nz / ts : 1);
    const int blocks = (int)((ntiles + kThreads - 1) / kThreads);
    const bool pdl = p.pdl != 0;
    if (p.ndim == 3 && levels == 2 && p.nx % 16 == 0 && p.ny % 4 == 0 && p.nz % 4 == 0 &&
        ((uintptr_t)ref & 15) == 0 && ((uintptr_t)u & 15) == 0) {
        const int64_t nthr = (int64_t)p.nx * p.ny * p.nz / 8;
        PP_TRY_CUDA(launch_ex(prox3q_kernel<true>, dim3((unsigned)((nthr + kThreads - 1) / kThreads)),
                              dim3(kThreads), 0, st, pdl, 0, p.nx, p.ny, p.nz, lambda, gamma, beta,
                              (const float2*)p.z, u, p.z, p.y, ref, hist_slot));
        return check_launch("prox_fista3q_kernel");
    }
    if (p.ndim == 2 && levels == 2 && p.nx % 32 == 0 && p.ny % 4 == 0 &&
        ((uintptr_t)ref & 15) == 0 && ((uintptr_t)u & 15) == 0) {
        const int64_t nthr = (int64_t)p.nx * p.ny / 4;
        PP_TRY_CUDA(launch_ex(prox_fista2q_kernel, dim3((unsigned)((nthr + kThreads - 1) / kThreads)),
                              dim3(kThreads), 0, st, pdl, 0, p.nx, p.ny, lambda, gamma, beta, p.z, u,
                              p.y, ref, hist_slot));
        return check_launch("prox_fista2q_kernel");
    }
#define PP_PF(ND_, LV_)                                                                         \
    PP_TRY_CUDA(launch_ex(prox_fista_kernel<ND_, LV_>, dim3(blocks), dim3(kThreads), 0, st, pdl, 0, \
                          p.nx, p.ny, p.nz, lambda, gamma, beta, p.z, u, p.y, ref, hist_slot))
    if (p.ndim == 2 && levels == 1)
        PP_PF(2, 1);
    else if (p.ndim == 2)
        PP_PF(2, 2);
    else if (levels == 1)
        PP_PF(3, 1);
    else
        PP_PF(3, 2);
#undef PP_PF
    return check_launch("prox_fista_kernel");
}

pp_status launch_dot(const float2* a, const float2* b, int64_t n, double* partials, int nblocks,
                     double* out_re, double* out_norm_b, cudaStream_t st) {
    dot_partial_kernel<<<nblocks, kThreads, 0, st>>>(a, b, n, partials);
    PP_TRY(check_launch("dot_partial_kernel"));
    dot_final_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, out_re, out_norm_b);
    return check_launch("dot_final_kernel");
}

pp_status launch_norm2(const float2* a, int64_t n, double* partials, int nblocks, double* out,
                       cudaStream_t st) {
    return launch_dot(nullptr, a, n, partials, nblocks, nullptr, out, st);
}

pp_status launch_scale_by_rnorm(const float2* in, float2* out, int64_t n, const double* norm2,
                                double factor, int invert, cudaStream_t st) {
    scale_by_norm_kernel<<<ew_blocks(n), kThreads, 0, st>>>(in, out, n, norm2, factor, invert);
    return check_launch("scale_by_norm_kernel");
}

pp_status launch_axpby(const float2* x, float a, const float2* y, float b, float2* out, int64_t n,
                       cudaStream_t st) {
    axpby_kernel<<<ew_blocks(n), kThreads, 0, st>>>(x, a, y, b, out, n);
    return check_launch("axpby_kernel");
}

pp_status launch_start_vector(float2* v, int64_t n, uint64_t seed, cudaStream_t st) {
    start_vector_kernel<<<ew_blocks(n), kThreads, 0, st>>>(v, n, seed);
    return check_launch("start_vector_kernel");
}

}  // namespace pp
