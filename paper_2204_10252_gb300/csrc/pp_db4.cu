// Daubechies-4 l1 prox (Eq. "proxdef" with W the Daubechies-4 wavelet, the
// transform of the paper's experiments, Sec. 5.1 and Sec. 5.2), 2-D.
//
// W: the four-coefficient orthonormal Daubechies filter
//   h = ((1 + s3), (3 + s3), (3 - s3), (1 - s3)) / (4 sqrt 2),  s3 = sqrt 3,
//   g[k] = (-1)^k h[3 - k],
// periodic boundary, separable, Mallat layout: at level l the band of
// ny >> (l-1) rows and nx >> (l-1) columns is transformed along x (rows),
// then along y (columns), approximation first:
//   a[i] = sum_k h[k] v[(2i + k) mod n],  d[i] = sum_k g[k] v[(2i + k) mod n].
// The inverse is the transpose: v[2m] = h0 a[m] + h2 a[m-1] + g0 d[m] + g2 d[m-1],
// v[2m+1] = h1 a[m] + h3 a[m-1] + g1 d[m] + g3 d[m-1] (indices mod n/2).
//
// Unlike the 2-level Haar (tile-local), every level couples neighbouring
// tiles, so the prox runs as one pass per level and direction: a CTA owns
// whole rows (or 8 whole columns) of the band, stages them in shared memory
// and writes its outputs back in place.  The soft threshold is applied when
// a coefficient becomes final (column passes); the FISTA step w = z - gamma u
// is fused into the first pass, the momentum update and the FP64 statistics
// into the last.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pp_fft.cuh"
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int MAXN = 512;   // longest row / column
constexpr int CW = 8;       // columns per CTA in the column passes

struct Db4 {
    float h[4], g[4];
};

Db4 db4_filter() {
    const double s3 = sqrt(3.0), r = 1.0 / (4.0 * sqrt(2.0));
    const double h[4] = {(1 + s3) * r, (3 + s3) * r, (3 - s3) * r, (1 - s3) * r};
    Db4 f;
    for (int k = 0; k < 4; ++k) {
        f.h[k] = (float)h[k];
        f.g[k] = (float)((k & 1) ? -h[3 - k] : h[3 - k]);
    }
    return f;
}

__device__ __forceinline__ float2 soft4(float2 v, float lam) {
    const float m2 = v.x * v.x + v.y * v.y;
    // |v| <= lambda -> 0 (also v = 0, so no 0 * inf); a NaN fails the test and
    // stays NaN instead of being thresholded to 0
    if (m2 <= lam * lam) return make_float2(0.f, 0.f);
    return cscale(v, 1.f - lam * rsqrtf(m2));
}

__device__ __forceinline__ float2 fma2(float c, float2 v, float2 acc) {
    return make_float2(fmaf(c, v.x, acc.x), fmaf(c, v.y, acc.y));
}

// FISTA epilogue arguments of the last inverse pass (z, y updated in place).
struct Epi {
    float2* z;
    float2* y;
    const float2* ref;
    double* hist;
    float beta;
};

// Block-level FP64 sums of (dd, yy, rr) added to hist[0..2].
__device__ __forceinline__ void hist_add(double dd, double yy, double rr, double* hist) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dd += __shfl_down_sync(0xffffffffu, dd, off);
        yy += __shfl_down_sync(0xffffffffu, yy, off);
        rr += __shfl_down_sync(0xffffffffu, rr, off);
    }
    __shared__ double s[3][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][wid] = dd;
        s[1][wid] = yy;
        s[2][wid] = rr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += s[0][i];
            b += s[1][i];
            c += s[2][i];
        }
        atomicAdd(&hist[0], a);
        atomicAdd(&hist[1], b);
        atomicAdd(&hist[2], c);
    }
}

// Row pass over the band [0, h) x [0, w) of an image with row pitch nx.
// Forward: reads src (or z - gamma u when u != NULL), writes [a | d] to dst.
// Inverse: reads [a | d] from src, writes v to dst, or, with EPI, runs the
// FISTA epilogue on v.  grid (h), block kThreads; src may equal dst.
template <bool INV, bool EPI>
__global__ void __launch_bounds__(kThreads)
db4_rows_kernel(Db4 f, int w, int nx, const float2* src, const float2* __restrict__ u, float gamma,
                float2* dst, Epi e) {
    __shared__ float2 s[MAXN];
    pdl_trigger();
    pdl_wait();
    const int64_t row = (int64_t)blockIdx.x * nx;
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
        float2 v = src[row + i];
        if (u) {
            const float2 q = u[row + i];
            v = make_float2(v.x - gamma * q.x, v.y - gamma * q.y);
        }
        s[i] = v;
    }
    __syncthreads();
    const int hw = w >> 1;
    if (!INV) {
        for (int i = threadIdx.x; i < hw; i += blockDim.x) {
            float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int j = 2 * i + k;
                if (j >= w) j -= w;
                a = fma2(f.h[k], s[j], a);
                d = fma2(f.g[k], s[j], d);
            }
            dst[row + i] = a;
            dst[row + hw + i] = d;
        }
        return;
    }
    double dd = 0.0, yy = 0.0, rr = 0.0;
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const int m = j >> 1, par = j & 1, m1 = m == 0 ? hw - 1 : m - 1;
        float2 v = make_float2(0.f, 0.f);
        v = fma2(f.h[par], s[m], v);
        v = fma2(f.h[par + 2], s[m1], v);
        v = fma2(f.g[par], s[hw + m], v);
        v = fma2(f.g[par + 2], s[hw + m1], v);
        if (!EPI) {
            dst[row + j] = v;
        } else {
            const float2 yo = e.y[row + j];
            const float2 df = csub(v, yo);
            e.z[row + j] = make_float2(v.x + e.beta * df.x, v.y + e.beta * df.y);
            e.y[row + j] = v;
            if (e.hist) {
                dd += (double)df.x * df.x + (double)df.y * df.y;
                yy += (double)v.x * v.x + (double)v.y * v.y;
                if (e.ref) {
                    const float2 r = e.ref[row + j];
                    const double ex = (double)v.x - r.x, ey = (double)v.y - r.y;
                    rr += ex * ex + ey * ey;
                }
            }
        }
    }
    if (EPI && e.hist) hist_add(dd, yy, rr, e.hist);
}

// Column pass over the band [0, h) x [0, w): CTA b owns columns
// 8b .. 8b+7 (those below w).  Forward writes [a ; d] down each column and
// soft-thresholds the coefficients that are final: every d, and a when the
// level is the last or the column holds row details (col >= w/2).
// grid (ceil(w / 8)), block kThreads; in place.
template <bool INV>
__global__ void __launch_bounds__(kThreads)
db4_cols_kernel(Db4 f, int h, int w, int nx, float lam, int last, float2* v) {
    __shared__ float2 s[MAXN * CW];
    pdl_trigger();
    pdl_wait();
    const int col0 = blockIdx.x * CW;
    for (int e = threadIdx.x; e < h * CW; e += blockDim.x) {
        const int r = e / CW, c = e % CW;
        if (col0 + c < w) s[e] = v[(int64_t)r * nx + col0 + c];
    }
    __syncthreads();
    const int hh = h >> 1;
    if (!INV) {
        for (int e = threadIdx.x; e < hh * CW; e += blockDim.x) {
            const int i = e / CW, c = e % CW, col = col0 + c;
            if (col >= w) continue;
            float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int j = 2 * i + k;
                if (j >= h) j -= h;
                a = fma2(f.h[k], s[j * CW + c], a);
                d = fma2(f.g[k], s[j * CW + c], d);
            }
            if (last || col >= (w >> 1)) a = soft4(a, lam);
            v[(int64_t)i * nx + col] = a;
            v[(int64_t)(hh + i) * nx + col] = soft4(d, lam);
        }
        return;
    }
    for (int e = threadIdx.x; e < h * CW; e += blockDim.x) {
        const int j = e / CW, c = e % CW, col = col0 + c;
        if (col >= w) continue;
        const int m = j >> 1, par = j & 1, m1 = m == 0 ? hh - 1 : m - 1;
        float2 x = make_float2(0.f, 0.f);
        x = fma2(f.h[par], s[m * CW + c], x);
        x = fma2(f.h[par + 2], s[m1 * CW + c], x);
        x = fma2(f.g[par], s[(hh + m) * CW + c], x);
        x = fma2(f.g[par + 2], s[(hh + m1) * CW + c], x);
        v[(int64_t)j * nx + col] = x;
    }
}

pp_status check_db4(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    if (g_profiler) g_profiler->mark(what);
    return PP_OK;
}

// The whole prox: forward levels 1..L, thresholds, inverse levels L..1.
// First pass reads `in` (minus gamma u when u != NULL) and writes `coef`;
// the rest runs in place on `coef`; the last pass writes `out` or, with
// `epi`, the FISTA epilogue.
pp_status db4_prox(int nx, int ny, int levels, float lambda, const float2* in, const float2* u,
                   float gamma, float2* coef, float2* out, const Epi* epi, bool pdl,
                   cudaStream_t st) {
    const Db4 f = db4_filter();
    const Epi none{nullptr, nullptr, nullptr, nullptr, 0.f};
    for (int l = 0; l < levels; ++l) {
        const int h = ny >> l, w = nx >> l;
        PP_TRY_CUDA(launch_ex(db4_rows_kernel<false, false>, dim3(h), dim3(kThreads), 0, st, pdl, 0, f,
                              w, nx, l == 0 ? in : (const float2*)coef, l == 0 ? u : nullptr, gamma,
                              coef, none));
        PP_TRY(check_db4("db4_rows_kernel"));
        PP_TRY_CUDA(launch_ex(db4_cols_kernel<false>, dim3((w + CW - 1) / CW), dim3(kThreads), 0, st,
                              pdl, 0, f, h, w, nx, lambda, (int)(l == levels - 1), coef));
        PP_TRY(check_db4("db4_cols_kernel"));
    }
    for (int l = levels - 1; l >= 0; --l) {
        const int h = ny >> l, w = nx >> l;
        PP_TRY_CUDA(launch_ex(db4_cols_kernel<true>, dim3((w + CW - 1) / CW), dim3(kThreads), 0, st,
                              pdl, 0, f, h, w, nx, lambda, 0, coef));
        PP_TRY(check_db4("db4_cols_kernel"));
        if (l == 0 && epi) {
            PP_TRY_CUDA(launch_ex(db4_rows_kernel<true, true>, dim3(h), dim3(kThreads), 0, st, pdl, 0,
                                  f, w, nx, (const float2*)coef, (const float2*)nullptr, 0.f,
                                  (float2*)nullptr, *epi));
        } else {
            PP_TRY_CUDA(launch_ex(db4_rows_kernel<true, false>, dim3(h), dim3(kThreads), 0, st, pdl, 0,
                                  f, w, nx, (const float2*)coef, (const float2*)nullptr, 0.f,
                                  l == 0 ? out : coef, none));
        }
        PP_TRY(check_db4("db4_rows_kernel"));
    }
    return PP_OK;
}

}  // namespace

bool db4_supported(int ndim, int nx, int ny, int levels) {
    return ndim == 2 && levels >= 1 && levels <= 4 && nx <= MAXN && ny <= MAXN && nx > 0 && ny > 0 &&
           nx % (1 << levels) == 0 && ny % (1 << levels) == 0;
}

pp_status launch_prox_db4(int nx, int ny, int levels, float lambda, const float2* in, float2* out,
                          cudaStream_t st) {
    return db4_prox(nx, ny, levels, lambda, in, nullptr, 0.f, out, out, nullptr, false, st);
}

pp_status launch_prox_fista_db4(const Plan& p, int levels, float lambda, float gamma, float beta,
                                const float2* u, float2* scratch, const float2* ref, double* hist_slot,
                                cudaStream_t st) {
    const Epi e{p.z, p.y, ref, hist_slot, beta};
    return db4_prox(p.nx, p.ny, levels, lambda, p.z, u, gamma, scratch, nullptr, &e, p.pdl != 0, st);
}

}  // namespace pp
