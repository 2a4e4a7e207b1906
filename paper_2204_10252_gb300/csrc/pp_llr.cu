// Locally-low-rank prox (the LLR regulariser of the MRF experiment, Sec. 5.3):
// for every block of block^ndim voxels (non-overlapping, after a circular
// shift of the volume), the Casorati matrix M (one row per voxel, one column
// per coefficient image) is replaced by U max(S - lambda, 0) V^H, its
// singular values soft-thresholded.
//
// One CTA per block.  The SVD is a one-sided Jacobi iteration in FP32:
// columns i, j of M are rotated until every pair is orthogonal; the rotated
// matrix is U S and the accumulated rotations are V, so the output is
// (M V) diag(max(0, 1 - lambda / s_i)) V^H.  One-sided Jacobi works on M
// itself, so small singular values keep their relative accuracy (no Gram
// matrix whose rounding is relative to the largest one).  A sweep visits all
// T(T-1)/2 pairs in T'-1 rounds of disjoint pairs (round-robin schedule,
// T' = T rounded up to even); the column norms and inner products of one
// round's pairs are summed over the block's voxels in one block reduction.
// The sweeps stop when every pair's |a_i^H a_j| <= tol sqrt(|a_i|^2 |a_j|^2)
// (the same decision in every thread: it is taken from the reduced sums),
// tol = sqrt(R) * 2^-24 for R voxels per block: the rounding level of an
// R-term FP32 inner product (the threshold LAPACK's one-sided Jacobi uses
// with its own precision), below which a rotation only moves noise.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp_fft.cuh"
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int kLlrSweeps = 12;

struct LlrArgs {
    const float2* in;
    float2* out;
    int64_t nimg;          // voxels per coefficient image
    int nx, ny, nz, ndim;
    int block, lb;         // block edge and log2
    int sx, sy, sz;        // circular shift of the block grid
    int nbx, nby;          // blocks per axis (x, y)
    int R;                 // voxels per block
    float lam;
};

// Round-robin (circle method) schedule of T' players: in round r the pairs
// are (r, T'-1) and ((r + k) mod (T'-1), (r - k) mod (T'-1)), k = 1 .. T'/2-1.
template <int TP>
__host__ __device__ constexpr int rr_i(int r, int k) {
    return k == 0 ? r : ((r + k) % (TP - 1) < (r - k + (TP - 1)) % (TP - 1) ? (r + k) % (TP - 1)
                                                                              : (r - k + (TP - 1)) % (TP - 1));
}
template <int TP>
__host__ __device__ constexpr int rr_j(int r, int k) {
    return k == 0 ? TP - 1 : ((r + k) % (TP - 1) < (r - k + (TP - 1)) % (TP - 1) ? (r - k + (TP - 1)) % (TP - 1)
                                                                                  : (r + k) % (TP - 1));
}

// Sum N <= 16 floats per thread over the block (NT threads, NT/32 warps):
// the result in every thread.  Within a warp a butterfly reduce-scatter
// halves the values each step (16 shuffles for 16 values instead of 5 per
// value): after the step with offset o a lane keeps the half its bit o
// selects, so lanes 2i and 2i+1 end with the warp sum of value i.  One lane
// per value writes it to `buf` ([NT/32][16] floats), and after the barrier
// every thread adds the warps' rows with 16-byte reads.
template <int NT, int N>
__device__ __forceinline__ void block_sum(float* v, float* buf) {
    static_assert(N <= 16, "block_sum handles up to 16 values");
    float t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = i < N ? v[i] : 0.f;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? t[i] : t[i + h];
            const float keep = up ? t[i + h] : t[i];
            t[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    t[0] += __shfl_xor_sync(0xffffffffu, t[0], 1);
    const int w = threadIdx.x >> 5;
    if ((lane & 1) == 0) buf[w * 16 + (lane >> 1)] = t[0];
    __syncthreads();
    const float4* b4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
    for (int q = 0; q < (N + 3) / 4; ++q) {
        float4 acc = b4[q];
#pragma unroll
        for (int ww = 1; ww < NT / 32; ++ww) {
            const float4 u = b4[ww * 4 + q];
            acc.x += u.x; acc.y += u.y; acc.z += u.z; acc.w += u.w;
        }
        if (4 * q + 0 < N) v[4 * q + 0] = acc.x;
        if (4 * q + 1 < N) v[4 * q + 1] = acc.y;
        if (4 * q + 2 < N) v[4 * q + 2] = acc.z;
        if (4 * q + 3 < N) v[4 * q + 3] = acc.w;
    }
}

// Offset of voxel `row` of block `b` in one coefficient image.
__device__ __forceinline__ int64_t llr_voxel(const LlrArgs& a, int b, int row) {
    const int m = a.block - 1;
    const int bx = b % a.nbx, byz = b / a.nbx, by = byz % a.nby, bz = byz / a.nby;
    const int dx = row & m, dy = (row >> a.lb) & m, dz = row >> (2 * a.lb);
    int x = bx * a.block + dx + a.sx, y = by * a.block + dy + a.sy;
    x -= x >= a.nx ? a.nx : 0;
    y -= y >= a.ny ? a.ny : 0;
    if (a.ndim == 2) return (int64_t)y * a.nx + x;
    int z = bz * a.block + dz + a.sz;
    z -= z >= a.nz ? a.nz : 0;
    return ((int64_t)z * a.ny + y) * a.nx + x;
}

template <int T, int RPT, int NT>
__global__ void __launch_bounds__(NT) llr_prox_kernel(LlrArgs a) {
    constexpr int TP = T + (T & 1);
    constexpr int NPR = TP / 2;                       // pairs per round
    __shared__ float2 Vs[T][T];                       // Vs[k][i] = V(k, i)
    __shared__ __align__(16) float red[2][NT / 32][16];
    const int b = blockIdx.x;
    float2 m[RPT][T];
    int64_t off[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int row = threadIdx.x + q * NT;
        const bool live = row < a.R;
        off[q] = live ? llr_voxel(a, b, row) : -1;
#pragma unroll
        for (int t = 0; t < T; ++t)
            m[q][t] = live ? a.in[t * a.nimg + off[q]] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < T)
#pragma unroll
        for (int i = 0; i < T; ++i) Vs[threadIdx.x][i] = make_float2(i == (int)threadIdx.x ? 1.f : 0.f, 0.f);
    const float tol = sqrtf((float)a.R) * 5.9604645e-8f;
    int par = 0;
    if (T > 1) {
        for (int sweep = 0; sweep < kLlrSweeps; ++sweep) {
            float offmax = 0.f;
#pragma unroll
            for (int r = 0; r < TP - 1; ++r) {
                float s[4 * NPR];
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                    const int i = rr_i<TP>(r, p), j = rr_j<TP>(r, p);
                    float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
                    if (j < T) {
#pragma unroll
                        for (int q = 0; q < RPT; ++q) {
                            const float2 u = m[q][i], v = m[q][j];
                            al = fmaf(u.x, u.x, fmaf(u.y, u.y, al));
                            be = fmaf(v.x, v.x, fmaf(v.y, v.y, be));
                            gr = fmaf(u.x, v.x, fmaf(u.y, v.y, gr));   // Re conj(u) v
                            gi = fmaf(u.x, v.y, fmaf(-u.y, v.x, gi));  // Im conj(u) v
                        }
                    }
                    s[4 * p] = al; s[4 * p + 1] = be; s[4 * p + 2] = gr; s[4 * p + 3] = gi;
                }
                block_sum<NT, 4 * NPR>(s, &red[par][0][0]);
                par ^= 1;   // the next reduction writes the other buffer: no second barrier
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                    const int i = rr_i<TP>(r, p), j = rr_j<TP>(r, p);
                    if (j >= T) continue;
                    const float al = s[4 * p], be = s[4 * p + 1], gr = s[4 * p + 2], gi = s[4 * p + 3];
                    const float g = sqrtf(gr * gr + gi * gi), nab = sqrtf(al * be);
                    if (!(g > tol * nab)) continue;
                    offmax = fmaxf(offmax, g / nab);
                    // real symmetric Schur rotation of [[al, g], [g, be]], after the
                    // phase e^{-i phi} = conj(gamma)/|gamma| that makes gamma real
                    const float zeta = (be - al) / (2.f * g);
                    const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                    const float c = rsqrtf(fmaf(t, t, 1.f)), sn = c * t;
                    const float2 ph = make_float2(gr / g, -gi / g);
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        const float2 u = m[q][i], w = cmul(ph, m[q][j]);
                        m[q][i] = make_float2(c * u.x - sn * w.x, c * u.y - sn * w.y);
                        m[q][j] = make_float2(sn * u.x + c * w.x, sn * u.y + c * w.y);
                    }
                    if (threadIdx.x < T) {
                        const int k = threadIdx.x;
                        const float2 u = Vs[k][i], w = cmul(ph, Vs[k][j]);
                        Vs[k][i] = make_float2(c * u.x - sn * w.x, c * u.y - sn * w.y);
                        Vs[k][j] = make_float2(sn * u.x + c * w.x, sn * u.y + c * w.y);
                    }
                }
            }
            if (offmax <= tol) break;
        }
    }
    // singular values = final column norms; shrink factors
    float nr[T];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc = fmaf(m[q][i].x, m[q][i].x, fmaf(m[q][i].y, m[q][i].y, acc));
        nr[i] = acc;
    }
    block_sum<NT, T>(nr, &red[par][0][0]);
    float f[T];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const float sg = sqrtf(nr[i]);
        // s <= lambda (also s = 0) -> 0; a NaN fails the test and stays NaN
        f[i] = sg <= a.lam ? 0.f : 1.f - a.lam / sg;
    }
    // every thread's Vs updates are visible after block_sum's barrier
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        if (off[q] < 0) continue;
#pragma unroll
        for (int k = 0; k < T; ++k) {
            float2 y = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < T; ++i) y = cadd(y, cscale(cmulc(Vs[k][i], m[q][i]), f[i]));
            a.out[k * a.nimg + off[q]] = y;
        }
    }
}

template <int T>
cudaError_t llr_launch_t(const LlrArgs& a, int nblocks, cudaStream_t st) {
    if (a.R > 256) {
        llr_prox_kernel<T, 4, 128><<<nblocks, 128, 0, st>>>(a);
    } else if (a.R > 128) {
        llr_prox_kernel<T, 2, 128><<<nblocks, 128, 0, st>>>(a);
    } else if (a.R > 64) {
        llr_prox_kernel<T, 1, 128><<<nblocks, 128, 0, st>>>(a);
    } else if (a.R > 32) {
        llr_prox_kernel<T, 1, 64><<<nblocks, 64, 0, st>>>(a);
    } else {
        llr_prox_kernel<T, 1, 32><<<nblocks, 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

pp_status launch_prox_llr(int ndim, int nx, int ny, int nz, int T, int block, const int* shift,
                          float lambda, const float2* in, float2* out, cudaStream_t st) {
    LlrArgs a;
    a.in = in; a.out = out;
    a.ndim = ndim; a.nx = nx; a.ny = ny; a.nz = ndim == 3 ? nz : 1;
    a.nimg = (int64_t)nx * ny * a.nz;
    a.block = block;
    a.lb = block == 4 ? 2 : (block == 8 ? 3 : 4);
    auto wrap = [](int s, int n) { s %= n; return s < 0 ? s + n : s; };
    a.sx = shift ? wrap(shift[0], nx) : 0;
    a.sy = shift ? wrap(shift[1], ny) : 0;
    a.sz = (shift && ndim == 3) ? wrap(shift[2], a.nz) : 0;
    a.nbx = nx / block;
    a.nby = ny / block;
    a.R = ndim == 3 ? block * block * block : block * block;
    a.lam = lambda;
    const int64_t nblocks = (int64_t)a.nbx * a.nby * (ndim == 3 ? a.nz / block : 1);
    if (nblocks <= 0) return PP_OK;
    if (nblocks > 0x7fffffff) {
        set_error("pp_prox_llr: too many blocks");
        return PP_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaErrorInvalidValue;
    switch (T) {
        case 1: e = llr_launch_t<1>(a, (int)nblocks, st); break;
        case 2: e = llr_launch_t<2>(a, (int)nblocks, st); break;
        case 3: e = llr_launch_t<3>(a, (int)nblocks, st); break;
        case 4: e = llr_launch_t<4>(a, (int)nblocks, st); break;
        case 5: e = llr_launch_t<5>(a, (int)nblocks, st); break;
        case 6: e = llr_launch_t<6>(a, (int)nblocks, st); break;
        case 7: e = llr_launch_t<7>(a, (int)nblocks, st); break;
        case 8: e = llr_launch_t<8>(a, (int)nblocks, st); break;
        default: break;
    }
    if (e != cudaSuccess) return cuda_status(e, "llr_prox_kernel");
    ++g_launches;
    if (g_profiler) g_profiler->mark("llr_prox_kernel");
    return PP_OK;
}

}  // namespace pp
