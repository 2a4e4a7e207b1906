// Batched kernels for many independent 2-D Cartesian problems of uneven size
// (one persistent launch per stage over a work list).  Each slice s is its
// own SENSE problem (Sec. 5.1 operator) with its own L_s; the batch shares
// the iteration index k of Algorithm "pfista" (Sec. 3.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "pp_batch.h"
#include "pp_fft4.cuh"

namespace pp {

namespace {

__device__ __forceinline__ void load_table_b(float2* dst, const float2* __restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Work item (s, col0): columns col0 .. col0 + 2^LGT - 1 of slice s, all coils.
//   out_s = coef * invL_s * sum_c conj(S_c) F_y^H M_fo F_y (S_c x_s) + alpha * operand_s
template <int KM, int LGT>
__global__ void __launch_bounds__(kThreads)
cart2d_batch_normal_kernel(const SliceDesc* __restrict__ descs, const int2* __restrict__ items,
                           int nitems, int ny_max, const float2* __restrict__ x,
                           float2* __restrict__ out, float coef, const float2* __restrict__ operand,
                           float alpha) {
    constexpr int T = 1 << LGT;
    extern __shared__ float2 sm[];
    float2* tws = sm;
    float2* b0 = sm + ny_max;
    float2* b1 = b0 + ny_max * T;
    float* pm = reinterpret_cast<float*>(b1 + ny_max * T);
    int cur = -1;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = items[it];
        const int s = item.x, col0 = item.y;
        const SliceDesc D = descs[s];
        const int ny = D.ny, nx = D.nx;
        if (s != cur) {
            load_table_b(tws, D.tw, ny);
            for (int i = threadIdx.x; i < ny; i += blockDim.x) pm[i] = D.mask_fo[i];
            cur = s;
        }
        const float2* xs = x + D.img_off;
        const int nel = ny * T;
        float2 xr[KM], sr[KM], acc[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int e = threadIdx.x + k * kThreads;
            const int yy = e >> LGT;
            const int col = col0 + (e & (T - 1));
            xr[k] = (e < nel && col < nx) ? xs[(int64_t)yy * nx + col] : make_float2(0.f, 0.f);
            acc[k] = make_float2(0.f, 0.f);
        }
        const int64_t cs = (int64_t)ny * nx;
        for (int c = 0; c < D.C; ++c) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int e = threadIdx.x + k * kThreads;
                if (e < nel) {
                    const int yy = e >> LGT;
                    const int col = col0 + (e & (T - 1));
                    sr[k] = (col < nx) ? D.sens[c * cs + (int64_t)yy * nx + col] : make_float2(0.f, 0.f);
                    b0[e] = cmul(sr[k], xr[k]);
                }
            }
            __syncthreads();
            float2* r1 = fft_batch<false>(b0, b1, D.fd, T, 1, LGT, tws, nullptr);
            float2* other = (r1 == b0) ? b1 : b0;
            float2* r2 = fft_batch<true>(r1, other, D.fd, T, 1, LGT, tws, pm);
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int e = threadIdx.x + k * kThreads;
                if (e < nel) acc[k] = cadd(acc[k], cmulc(sr[k], r2[e]));
            }
            __syncthreads();
        }
        const float sc = coef * D.invL;
        float2* os = out + D.img_off;
        const float2* ops = operand ? operand + D.img_off : nullptr;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int e = threadIdx.x + k * kThreads;
            const int yy = e >> LGT;
            const int col = col0 + (e & (T - 1));
            if (e < nel && col < nx) {
                const int64_t o = (int64_t)yy * nx + col;
                float2 v = cscale(acc[k], sc);
                if (ops) v = cadd(v, cscale(ops[o], alpha));
                os[o] = v;
            }
        }
    }
}

// Segmented FP64 reduction: block b works on segment seg = blk_seg[b], as
// block j = b - seg_first_blk[seg] of that segment's nb blocks.
// partials[b] = (Re<a,b>, Im<a,b>, |b|^2) over the block's share.
__global__ void __launch_bounds__(kThreads)
seg_dot_partial_kernel(const float2* __restrict__ a, const float2* __restrict__ bv,
                       const int64_t* __restrict__ seg_off, const int* __restrict__ blk_seg,
                       const int* __restrict__ seg_first_blk, double* __restrict__ partials) {
    const int seg = blk_seg[blockIdx.x];
    const int j = blockIdx.x - seg_first_blk[seg];
    const int nb = seg_first_blk[seg + 1] - seg_first_blk[seg];
    const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
    double re = 0.0, im = 0.0, nn = 0.0;
    for (int64_t i = lo + (int64_t)j * blockDim.x + threadIdx.x; i < hi; i += (int64_t)nb * blockDim.x) {
        const float2 y = bv[i];
        if (a) {
            const float2 x = a[i];
            re += (double)x.x * y.x + (double)x.y * y.y;
            im += (double)x.x * y.y - (double)x.y * y.x;
        }
        nn += (double)y.x * y.x + (double)y.y * y.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, off);
        im += __shfl_down_sync(0xffffffffu, im, off);
        nn += __shfl_down_sync(0xffffffffu, nn, off);
    }
    __shared__ double s[3][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][wid] = re;
        s[1][wid] = im;
        s[2][wid] = nn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0, r2 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            r0 += s[0][i];
            r1 += s[1][i];
            r2 += s[2][i];
        }
        partials[3 * blockIdx.x] = r0;
        partials[3 * blockIdx.x + 1] = r1;
        partials[3 * blockIdx.x + 2] = r2;
    }
}

// One block per segment: out_re[seg*stride], out_nb[seg*stride].
__global__ void seg_dot_final_kernel(const double* __restrict__ partials,
                                     const int* __restrict__ seg_first_blk, double* out_re,
                                     double* out_nb, int stride) {
    __shared__ double s[2][kThreads];
    const int seg = blockIdx.x;
    const int b0 = seg_first_blk[seg], b1 = seg_first_blk[seg + 1];
    double re = 0.0, nn = 0.0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        re += partials[3 * i];
        nn += partials[3 * i + 2];
    }
    s[0][threadIdx.x] = re;
    s[1][threadIdx.x] = nn;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (out_re) out_re[seg * stride] = s[0][0];
        if (out_nb) out_nb[seg * stride] = s[1][0];
    }
}

// out = in * factor_seg / sqrt(norm2[seg*stride]) (invert) or * sqrt(...) (not)
__global__ void seg_scale_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                 const int64_t* __restrict__ seg_off, const int* __restrict__ blk_seg,
                                 const int* __restrict__ seg_first_blk,
                                 const double* __restrict__ norm2, int stride,
                                 const double* __restrict__ factor, int invert) {
    const int seg = blk_seg[blockIdx.x];
    const int j = blockIdx.x - seg_first_blk[seg];
    const int nb = seg_first_blk[seg + 1] - seg_first_blk[seg];
    const int64_t lo = seg_off[seg], hi = seg_off[seg + 1];
    const double nv = norm2 ? sqrt(norm2[seg * stride]) : 1.0;
    const double fs = factor ? factor[seg] : 1.0;
    const double fi = isfinite(nv) ? (nv > 0.0 ? fs / nv : 0.0) : __longlong_as_double(0x7ff8000000000000ll);
    const float f = (float)(invert ? fi : fs * nv);
    for (int64_t i = lo + (int64_t)j * blockDim.x + threadIdx.x; i < hi; i += (int64_t)nb * blockDim.x)
        out[i] = cscale(in[i], f);
}

__device__ __forceinline__ void haar2x2_b(float2& a, float2& b, float2& c, float2& d) {
    const float2 s0 = cadd(a, b), d0 = csub(a, b), s1 = cadd(c, d), d1 = csub(c, d);
    a = cscale(cadd(s0, s1), 0.5f);
    b = cscale(cadd(d0, d1), 0.5f);
    c = cscale(csub(s0, s1), 0.5f);
    d = cscale(csub(d0, d1), 0.5f);
}

__device__ __forceinline__ float2 soft_b(float2 v, float lam) {
    const float m2 = v.x * v.x + v.y * v.y;
    // |v| <= lambda -> 0 (also v = 0, so no 0 * inf); a NaN fails the test and
    // stays NaN instead of being thresholded to 0
    if (m2 <= lam * lam) return make_float2(0.f, 0.f);
    return cscale(v, 1.f - lam * rsqrtf(m2));
}

// 2-level 2-D Haar prox of a 4x4 tile (same transform as the single-plan
// prox kernel: block transform on 2x2 blocks, then on the four level-1
// approximation coefficients; each block transform is its own inverse).
__device__ __forceinline__ void prox44(float2* v, float lam) {
#pragma unroll
    for (int by = 0; by < 4; by += 2)
#pragma unroll
        for (int bx = 0; bx < 4; bx += 2)
            haar2x2_b(v[by * 4 + bx], v[by * 4 + bx + 1], v[(by + 1) * 4 + bx], v[(by + 1) * 4 + bx + 1]);
    haar2x2_b(v[0], v[2], v[8], v[10]);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = soft_b(v[i], lam);
    haar2x2_b(v[0], v[2], v[8], v[10]);
#pragma unroll
    for (int by = 0; by < 4; by += 2)
#pragma unroll
        for (int bx = 0; bx < 4; bx += 2)
            haar2x2_b(v[by * 4 + bx], v[by * 4 + bx + 1], v[(by + 1) * 4 + bx], v[(by + 1) * 4 + bx + 1]);
}

// Batched fused prox + momentum over 4x4 tiles; block -> slice map as above
// (segments count tiles).  Statistics are summed over the whole batch.
__global__ void __launch_bounds__(kThreads)
batch_prox_fista_kernel(const SliceDesc* __restrict__ descs, const int64_t* __restrict__ tile_off,
                        const int* __restrict__ blk_seg, const int* __restrict__ seg_first_blk,
                        float lam, float gamma, float beta, float2* __restrict__ z,
                        const float2* __restrict__ u, float2* __restrict__ y,
                        const float2* __restrict__ ref, double* __restrict__ hist) {
    const int s = blk_seg[blockIdx.x];
    const int j = blockIdx.x - seg_first_blk[s];
    const SliceDesc D = descs[s];
    const int64_t t = (int64_t)j * blockDim.x + threadIdx.x;
    const int64_t ntl = tile_off[s + 1] - tile_off[s];
    double dd = 0.0, yy = 0.0, rr = 0.0;
    if (t < ntl) {
        const int ntx = D.nx / 4;
        const int64_t ty = t / ntx, tx = t - ty * ntx;
        const int64_t o = D.img_off + ty * 4 * D.nx + tx * 4;
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int64_t a = o + (int64_t)r * D.nx + x;
                const float2 zv = z[a], uv = u[a];
                v[r * 4 + x] = make_float2(zv.x - gamma * uv.x, zv.y - gamma * uv.y);
            }
        prox44(v, lam);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int64_t a = o + (int64_t)r * D.nx + x;
                const float2 yn = v[r * 4 + x];
                const float2 yo = y[a];
                const float2 df = csub(yn, yo);
                z[a] = make_float2(yn.x + beta * df.x, yn.y + beta * df.y);
                y[a] = yn;
                if (hist) {   // FP64 arithmetic is slow on this part: only when asked for
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

// Reverse pass of one unrolled iteration at the prox (per 4x4 tile):
//   ybar_{k+1} = Ybar + (1 + beta) Zbar          (adjoint of y_{k+1})
//   Ybar      <- -beta Zbar                      (partial adjoint of y_k)
//   wbar       = W^T J_s^T W ybar_{k+1},  J_s the soft threshold's Jacobian
//                at the coefficients W w_k
//   lam_bar   += sum Re(conj(W ybar_{k+1}) . (-v/|v|)) over |v| > lambda
__global__ void __launch_bounds__(kThreads)
batch_prox_vjp_kernel(const SliceDesc* __restrict__ descs, const int64_t* __restrict__ tile_off,
                      const int* __restrict__ blk_seg, const int* __restrict__ seg_first_blk,
                      float lam, float beta, const float2* __restrict__ w, float2* __restrict__ Ybar,
                      const float2* __restrict__ Zbar, float2* __restrict__ wbar,
                      double* __restrict__ lam_bar) {
    const int s = blk_seg[blockIdx.x];
    const int j = blockIdx.x - seg_first_blk[s];
    const SliceDesc D = descs[s];
    const int64_t t = (int64_t)j * blockDim.x + threadIdx.x;
    const int64_t ntl = tile_off[s + 1] - tile_off[s];
    double lb = 0.0;
    if (t < ntl) {
        const int ntx = D.nx / 4;
        const int64_t ty = t / ntx, tx = t - ty * ntx;
        const int64_t o = D.img_off + ty * 4 * D.nx + tx * 4;
        float2 cw[16], cy[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int64_t a = o + (int64_t)r * D.nx + x;
                const float2 zb = Zbar[a], yb = Ybar[a];
                cy[r * 4 + x] = make_float2(yb.x + (1.f + beta) * zb.x, yb.y + (1.f + beta) * zb.y);
                Ybar[a] = make_float2(-beta * zb.x, -beta * zb.y);
                cw[r * 4 + x] = w[a];
            }
        // forward Haar of both tiles
#pragma unroll
        for (int by = 0; by < 4; by += 2)
#pragma unroll
            for (int bx = 0; bx < 4; bx += 2) {
                haar2x2_b(cw[by * 4 + bx], cw[by * 4 + bx + 1], cw[(by + 1) * 4 + bx], cw[(by + 1) * 4 + bx + 1]);
                haar2x2_b(cy[by * 4 + bx], cy[by * 4 + bx + 1], cy[(by + 1) * 4 + bx], cy[(by + 1) * 4 + bx + 1]);
            }
        haar2x2_b(cw[0], cw[2], cw[8], cw[10]);
        haar2x2_b(cy[0], cy[2], cy[8], cy[10]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 v = cw[i], g = cy[i];
            const float m2 = v.x * v.x + v.y * v.y;
            if (m2 > lam * lam) {
                const float rm = rsqrtf(m2);
                const float hx = v.x * rm, hy = v.y * rm;          // v / |v|
                const float q = lam * rm;                            // lambda / |v|
                const float proj = hx * g.x + hy * g.y;              // Re(conj(vhat) g)
                cy[i] = make_float2((1.f - q) * g.x + q * hx * proj, (1.f - q) * g.y + q * hy * proj);
                lb -= (double)proj;
            } else {
                cy[i] = make_float2(0.f, 0.f);
            }
        }
        haar2x2_b(cy[0], cy[2], cy[8], cy[10]);
#pragma unroll
        for (int by = 0; by < 4; by += 2)
#pragma unroll
            for (int bx = 0; bx < 4; bx += 2)
                haar2x2_b(cy[by * 4 + bx], cy[by * 4 + bx + 1], cy[(by + 1) * 4 + bx], cy[(by + 1) * 4 + bx + 1]);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int x = 0; x < 4; ++x) wbar[o + (int64_t)r * D.nx + x] = cy[r * 4 + x];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lb += __shfl_down_sync(0xffffffffu, lb, off);
    __shared__ double sl[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = lb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += sl[i];
        atomicAdd(lam_bar, a);
    }
}

// out = (accumulate ? out : 0) + sum_i coef_i * v_i
__global__ void lincomb_kernel(LinComb lc, float2* __restrict__ out, int64_t n, int accumulate) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 a = accumulate ? out[i] : make_float2(0.f, 0.f);
        for (int k = 0; k < lc.count; ++k) {
            const float2 v = lc.v[k][i];
            a.x += lc.coef[k] * v.x;
            a.y += lc.coef[k] * v.y;
        }
        out[i] = a;
    }
}

// Four-step register-FFT version of cart2d_batch_normal_kernel: every slice
// must have ny = 16 * n2 with n2 in {8, 12, 16, 20, 24}; items are 8 columns.
__global__ void __launch_bounds__(192, 2)
cart2d_batch4_kernel(const SliceDesc* __restrict__ descs, const int2* __restrict__ items, int nitems,
                     const float2* __restrict__ x, float2* out, float coef, const float2* operand,
                     float alpha) {
    __shared__ float2 tws[384];
    __shared__ float pm[384];
    __shared__ float2 Y[16 * 24 * 8];
    extern __shared__ float4 sb4[];   // double-buffered coil-map tiles, 2 * 384 * 8 float2
    float2* Sb = reinterpret_cast<float2*>(sb4);
    int cur = -1;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = items[it];
        const int s = item.x;
        const SliceDesc D = descs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < D.ny; i += blockDim.x) {
                tws[i] = D.tw[i];
                pm[i] = D.mask_fo[i];
            }
            __syncthreads();
            cur = s;
        }
        const float2* xs = x + D.img_off;
        float2* os = out + D.img_off;
        const float2* ops = operand ? operand + D.img_off : nullptr;
        const float sc = coef * D.invL;
        switch (D.n2) {
            case 8: cart_item4<8>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, item.y, os, sc, ops, alpha); break;
            case 12: cart_item4<12>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, item.y, os, sc, ops, alpha); break;
            case 16: cart_item4<16>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, item.y, os, sc, ops, alpha); break;
            case 20: cart_item4<20>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, item.y, os, sc, ops, alpha); break;
            default: cart_item4<24>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, item.y, os, sc, ops, alpha); break;
        }
    }
}

// One item of cart2d_batch4_cl_kernel: CTA q of the cluster runs coils q,
// q + CL, ... of the slice; the partial sums meet in distributed shared
// memory and CTA q writes rows [q n / CL, (q + 1) n / CL) (sum in rank order).
template <int N2>
__device__ __forceinline__ void batch_item_cl(const float2* tws, const float* pm, float2* Y, float2* Sb,
                                              const SliceDesc& D, int col0, const float2* xs,
                                              float2* os, float sc, const float2* ops, float alpha,
                                              int q, int CL) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int n = 16 * N2;
    float2 acc[16];
    cart_item4_acc<N2>(tws, pm, Y, Sb, xs, D.sens, D.C, D.nx, col0, q, CL, acc);
    const int lane = threadIdx.x & 7, r = threadIdx.x >> 3;
    if (r < N2) {
#pragma unroll
        for (int m1 = 0; m1 < 16; ++m1) Y[(N2 * m1 + r) * 8 + lane] = acc[m1];
    }
    cluster.sync();
    const int rpr = n / CL;
    for (int idx = threadIdx.x; idx < rpr * 8; idx += blockDim.x) {
        const int row = q * rpr + (idx >> 3), l = idx & 7, col = col0 + l;
        float2 v = cluster.map_shared_rank(Y, 0)[row * 8 + l];
        for (int b = 1; b < CL; ++b) v = cadd(v, cluster.map_shared_rank(Y, b)[row * 8 + l]);
        if (col < D.nx) {
            const int64_t o = (int64_t)row * D.nx + col;
            v = cscale(v, sc);
            if (ops) v = cadd(v, cscale(ops[o], alpha));
            os[o] = v;
        }
    }
    // Y is rewritten by the next item only after every CTA has read it (the
    // remote loads have fed the stores above: the arrive needs no release)
    cluster_arrive_relaxed();
    cluster_wait_acquire();
}

// cart2d_batch4_kernel with the coils of every item split over a cluster of
// CL CTAs (batches with fewer column items than resident CTAs).
// grid CL * clusters, cluster (CL, 1, 1); the clusters walk the item list.
__global__ void __launch_bounds__(192, 2)
cart2d_batch4_cl_kernel(const SliceDesc* __restrict__ descs, const int2* __restrict__ items,
                        int nitems, const float2* __restrict__ x, float2* out, float coef,
                        const float2* operand, float alpha) {
    __shared__ float2 tws[384];
    __shared__ float pm[384];
    __shared__ float2 Y[16 * 24 * 8];
    extern __shared__ float4 sb4[];
    float2* Sb = reinterpret_cast<float2*>(sb4);
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int cid = blockIdx.x / CL, ncid = gridDim.x / CL;
    int cur = -1;
    for (int it = cid; it < nitems; it += ncid) {
        const int2 item = items[it];
        const int s = item.x;
        const SliceDesc D = descs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < D.ny; i += blockDim.x) {
                tws[i] = D.tw[i];
                pm[i] = D.mask_fo[i];
            }
            __syncthreads();
            cur = s;
        }
        const float2* xs = x + D.img_off;
        float2* os = out + D.img_off;
        const float2* ops = operand ? operand + D.img_off : nullptr;
        const float sc = coef * D.invL;
        switch (D.n2) {
            case 8: batch_item_cl<8>(tws, pm, Y, Sb, D, item.y, xs, os, sc, ops, alpha, q, CL); break;
            case 12: batch_item_cl<12>(tws, pm, Y, Sb, D, item.y, xs, os, sc, ops, alpha, q, CL); break;
            case 16: batch_item_cl<16>(tws, pm, Y, Sb, D, item.y, xs, os, sc, ops, alpha, q, CL); break;
            case 20: batch_item_cl<20>(tws, pm, Y, Sb, D, item.y, xs, os, sc, ops, alpha, q, CL); break;
            default: batch_item_cl<24>(tws, pm, Y, Sb, D, item.y, xs, os, sc, ops, alpha, q, CL); break;
        }
    }
}

// cart2d_batch4_kernel for a batch whose slices all share one length
// ny = 16 N2: a block of 8 * max(16, N2) threads (no idle threads for the
// shorter lengths) and shared memory sized for that length, so more CTAs
// fit an SM.
template <int N2>
__global__ void __launch_bounds__(8 * (N2 > 16 ? N2 : 16), N2 <= 16 ? 4 : 2)
cart2d_batch4u_kernel(const SliceDesc* __restrict__ descs, const int2* __restrict__ items,
                      int nitems, const float2* __restrict__ x, float2* out, float coef,
                      const float2* operand, float alpha) {
    constexpr int n = 16 * N2;
    __shared__ float2 tws[n];
    __shared__ float pm[n];
    __shared__ float2 Y[16 * N2 * 8];
    extern __shared__ float4 sb4[];   // 2 * n * 8 float2
    float2* Sb = reinterpret_cast<float2*>(sb4);
    int cur = -1;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = items[it];
        const int s = item.x;
        const SliceDesc D = descs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                tws[i] = D.tw[i];
                pm[i] = D.mask_fo[i];
            }
            __syncthreads();
            cur = s;
        }
        cart_item4<N2>(tws, pm, Y, Sb, x + D.img_off, D.sens, D.C, D.nx, item.y, out + D.img_off,
                       coef * D.invL, operand ? operand + D.img_off : nullptr, alpha);
    }
}

// The uniform-length kernel with each item's coils split over a cluster of
// CL CTAs (batches with fewer items than resident CTAs: one pass over the
// items instead of several coil-serial rounds).  grid CL * clusters.
template <int N2>
__global__ void __launch_bounds__(8 * (N2 > 16 ? N2 : 16), N2 <= 16 ? 4 : 2)
cart2d_batch4u_cl_kernel(const SliceDesc* __restrict__ descs, const int2* __restrict__ items,
                         int nitems, const float2* __restrict__ x, float2* out, float coef,
                         const float2* operand, float alpha) {
    constexpr int n = 16 * N2;
    __shared__ float2 tws[n];
    __shared__ float pm[n];
    __shared__ float2 Y[16 * N2 * 8];
    extern __shared__ float4 sb4[];
    float2* Sb = reinterpret_cast<float2*>(sb4);
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int cid = blockIdx.x / CL, ncid = gridDim.x / CL;
    int cur = -1;
    for (int it = cid; it < nitems; it += ncid) {
        const int2 item = items[it];
        const int s = item.x;
        const SliceDesc D = descs[s];
        if (s != cur) {
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                tws[i] = D.tw[i];
                pm[i] = D.mask_fo[i];
            }
            __syncthreads();
            cur = s;
        }
        batch_item_cl<N2>(tws, pm, Y, Sb, D, item.y, x + D.img_off, out + D.img_off, coef * D.invL,
                          operand ? operand + D.img_off : nullptr, alpha, q, CL);
    }
}

}  // namespace

extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

static pp_status check_launch_b(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    if (g_profiler) g_profiler->mark(what);
    return PP_OK;
}

size_t batch_normal_smem(int ny_max, int lgt) {
    return sizeof(float2) * (size_t)(ny_max + 2 * ny_max * (1 << lgt)) + sizeof(float) * ny_max;
}

template <int KM, int LGT>
static void* batch_kernel_ptr() {
    return reinterpret_cast<void*>(cart2d_batch_normal_kernel<KM, LGT>);
}

// kernel pointer for (km, lgt); nullptr when not instantiated
void* batch_normal_fn(int km, int lgt) {
#define PP_B(KM_, L_) if (km == KM_ && lgt == L_) return batch_kernel_ptr<KM_, L_>();
    PP_B(4, 2) PP_B(8, 2)
    PP_B(4, 3) PP_B(8, 3) PP_B(12, 3)
    PP_B(4, 4) PP_B(8, 4) PP_B(12, 4) PP_B(16, 4)
#undef PP_B
    return nullptr;
}

pp_status configure_batch_kernels() {
    const int big = 200 * 1024;
    const int kms[] = {4, 8, 12, 16};
    for (int lgt = 2; lgt <= 4; ++lgt)
        for (int km : kms) {
            void* f = batch_normal_fn(km, lgt);
            if (f) PP_TRY_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        }
    return PP_OK;
}

constexpr size_t kBatch4Dyn = sizeof(float2) * 2 * 384 * 8;

// Persistent grid of the uniform-length kernel (0 when n2 has none).
int batch4u_grid(int n2) {
    int occ = 0, nsm = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define PP_G4U(N2_)                                                                                \
    if (n2 == N2_) {                                                                               \
        const size_t dyn = sizeof(float2) * 2 * 16 * N2_ * 8;                                      \
        cudaFuncSetAttribute(cart2d_batch4u_kernel<N2_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)dyn);                                                            \
        cudaFuncSetAttribute(cart2d_batch4u_cl_kernel<N2_>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);               \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cart2d_batch4u_kernel<N2_>,        \
                                                          8 * (N2_ > 16 ? N2_ : 16), dyn);         \
    }
    PP_G4U(8) PP_G4U(12) PP_G4U(16) PP_G4U(20) PP_G4U(24)
#undef PP_G4U
    if (e != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return 0;
    }
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) nsm = 152;
    return occ * nsm;
}

int batch4_grid() {
    int occ = 0, nsm = 0;
    cudaFuncSetAttribute(cart2d_batch4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBatch4Dyn);
    cudaFuncSetAttribute(cart2d_batch4_cl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBatch4Dyn);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cart2d_batch4_kernel, 192, kBatch4Dyn) !=
        cudaSuccess)
        occ = 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) nsm = 152;
    return std::max(1, occ) * nsm;
}

pp_status launch_batch_normal(const BatchDev& b, const float2* x, float2* out, float coef,
                              const float2* operand, float alpha, cudaStream_t st) {
    if (b.fast4 && b.cl == 1 && b.un2) {
        cudaError_t e = cudaErrorInvalidValue;
#define PP_B4U(N2_)                                                                                \
        if (b.un2 == N2_)                                                                          \
            e = launch_ex(cart2d_batch4u_kernel<N2_>, dim3(std::min(b.ugrid, b.nitems)),           \
                          dim3(8 * (N2_ > 16 ? N2_ : 16)), sizeof(float2) * 2 * 16 * N2_ * 8, st,  \
                          false, 0, (const SliceDesc*)b.descs, (const int2*)b.items, b.nitems, x, \
                          out, coef, operand, alpha);
        PP_B4U(8) PP_B4U(12) PP_B4U(16) PP_B4U(20) PP_B4U(24)
#undef PP_B4U
        if (e != cudaSuccess) return cuda_status(e, "cart2d_batch4u_kernel launch");
        return check_launch_b("cart2d_batch4u_kernel");
    }
    if (b.fast4 && b.cl > 1 && b.un2) {
        const int ncl = std::max(1, std::min(b.ugrid / b.cl, b.nitems));
        cudaError_t e = cudaErrorInvalidValue;
#define PP_B4UC(N2_)                                                                               \
        if (b.un2 == N2_)                                                                          \
            e = launch_ex(cart2d_batch4u_cl_kernel<N2_>, dim3(ncl * b.cl),                          \
                          dim3(8 * (N2_ > 16 ? N2_ : 16)), sizeof(float2) * 2 * 16 * N2_ * 8, st,  \
                          false, b.cl, (const SliceDesc*)b.descs, (const int2*)b.items, b.nitems, \
                          x, out, coef, operand, alpha);
        PP_B4UC(8) PP_B4UC(12) PP_B4UC(16) PP_B4UC(20) PP_B4UC(24)
#undef PP_B4UC
        if (e != cudaSuccess) return cuda_status(e, "cart2d_batch4u_cl_kernel launch");
        return check_launch_b("cart2d_batch4u_cl_kernel");
    }
    if (b.fast4 && b.cl > 1) {
        const int ncl = std::max(1, std::min(b.grid / b.cl, b.nitems));
        PP_TRY_CUDA(launch_ex(cart2d_batch4_cl_kernel, dim3(ncl * b.cl), dim3(192), kBatch4Dyn, st,
                              false, b.cl, (const SliceDesc*)b.descs, (const int2*)b.items, b.nitems,
                              x, out, coef, operand, alpha));
        return check_launch_b("cart2d_batch4_cl_kernel");
    }
    if (b.fast4) {
        cart2d_batch4_kernel<<<std::min(b.grid, b.nitems), 192, kBatch4Dyn, st>>>(
            b.descs, b.items, b.nitems, x, out, coef, operand, alpha);
        return check_launch_b("cart2d_batch4_kernel");
    }
    void* fn = batch_normal_fn(b.km, b.lgt);
    if (!fn) {
        set_error("no batched kernel for km=%d lgt=%d", b.km, b.lgt);
        return PP_ERR_UNSUPPORTED;
    }
    void* args[] = {(void*)&b.descs, (void*)&b.items, (void*)&b.nitems, (void*)&b.ny_max,
                    (void*)&x, (void*)&out, (void*)&coef, (void*)&operand, (void*)&alpha};
    PP_TRY_CUDA(cudaLaunchKernel(fn, dim3(b.grid), dim3(kThreads), args,
                                 batch_normal_smem(b.ny_max, b.lgt), st));
    return check_launch_b("cart2d_batch_normal_kernel");
}

pp_status launch_seg_dot(const float2* a, const float2* bv, const Segments& sg, double* partials,
                         double* out_re, double* out_nb, int stride, cudaStream_t st) {
    seg_dot_partial_kernel<<<sg.nblocks, kThreads, 0, st>>>(a, bv, sg.off, sg.blk_seg,
                                                             sg.seg_first_blk, partials);
    PP_TRY(check_launch_b("seg_dot_partial_kernel"));
    seg_dot_final_kernel<<<sg.nseg, kThreads, 0, st>>>(partials, sg.seg_first_blk, out_re, out_nb,
                                                        stride);
    return check_launch_b("seg_dot_final_kernel");
}

pp_status launch_seg_scale(const float2* in, float2* out, const Segments& sg, const double* norm2,
                           int stride, const double* factor, int invert, cudaStream_t st) {
    seg_scale_kernel<<<sg.nblocks, kThreads, 0, st>>>(in, out, sg.off, sg.blk_seg, sg.seg_first_blk,
                                                       norm2, stride, factor, invert);
    return check_launch_b("seg_scale_kernel");
}

pp_status launch_batch_prox_fista(const BatchDev& b, float lam, float gamma, float beta,
                                  float2* z, const float2* u, float2* y, const float2* ref,
                                  double* hist, cudaStream_t st) {
    batch_prox_fista_kernel<<<b.tiles.nblocks, kThreads, 0, st>>>(
        b.descs, b.tiles.off, b.tiles.blk_seg, b.tiles.seg_first_blk, lam, gamma, beta, z, u, y, ref,
        hist);
    return check_launch_b("batch_prox_fista_kernel");
}

pp_status launch_batch_prox_vjp(const BatchDev& b, float lam, float beta, const float2* w,
                                float2* Ybar, const float2* Zbar, float2* wbar, double* lam_bar,
                                cudaStream_t st) {
    batch_prox_vjp_kernel<<<b.tiles.nblocks, kThreads, 0, st>>>(
        b.descs, b.tiles.off, b.tiles.blk_seg, b.tiles.seg_first_blk, lam, beta, w, Ybar, Zbar, wbar,
        lam_bar);
    return check_launch_b("batch_prox_vjp_kernel");
}

pp_status launch_lincomb(const LinComb& lc, float2* out, int64_t n, int accumulate, cudaStream_t st) {
    int64_t blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    lincomb_kernel<<<(int)std::max<int64_t>(blocks, 1), kThreads, 0, st>>>(lc, out, n, accumulate);
    return check_launch_b("lincomb_kernel");
}

}  // namespace pp
