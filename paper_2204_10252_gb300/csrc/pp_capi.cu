// C ABI of libpp: plan set-up on the host, operator orchestration, the
// Horner recursion of Listing "pcode" and Algorithm "pfista" (Sec. 3.1, 3.6).
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "pp_batch.h"
#include "pp_fft4.cuh"
#include "pp_internal.h"

namespace pp {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

pp_status cuda_status(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
// Stage radices for length n: as many 8s as the power of two allows (a
// remainder of 2^1 becomes 4*4 in place of one 8, or a single 2), then 5s and
// 3s.  Returns false when n has a prime factor above 5.
static bool factorize(int n, FftDesc& d) {
    if (n < 2) return false;
    int e2 = 0, m = n;
    while (m % 2 == 0) { m /= 2; ++e2; }
    int n5 = 0, n3 = 0;
    while (m % 5 == 0) { m /= 5; ++n5; }
    while (m % 3 == 0) { m /= 3; ++n3; }
    if (m != 1) return false;
    std::vector<int> r;
    int q = e2 / 3, rem = e2 % 3;
    if (rem == 1 && q >= 1) { for (int i = 0; i < q - 1; ++i) r.push_back(8); r.push_back(4); r.push_back(4); }
    else { for (int i = 0; i < q; ++i) r.push_back(8); if (rem == 2) r.push_back(4); if (rem == 1) r.push_back(2); }
    for (int i = 0; i < n5; ++i) r.push_back(5);
    for (int i = 0; i < n3; ++i) r.push_back(3);
    if ((int)r.size() > 8) return false;
    d.n = n;
    d.nst = (int)r.size();
    for (int i = 0; i < 8; ++i) d.rad[i] = i < d.nst ? r[i] : 0;
    return true;
}

static pp_status dev_alloc(Plan& p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return PP_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return cuda_status(e, "cudaMalloc");
    }
    p.allocs.push_back(*ptr);
    return PP_OK;
}

template <class T>
static pp_status alloc_n(Plan& p, T** ptr, size_t n) {
    return dev_alloc(p, reinterpret_cast<void**>(ptr), n * sizeof(T));
}

static pp_status make_fft(Plan& p, int n, DevFft& f) {
    if (!factorize(n, f.d)) {
        set_error("FFT length %d has a prime factor above 5", n);
        return PP_ERR_UNSUPPORTED;
    }
    std::vector<float2> tw(n);
    for (int t = 0; t < n; ++t) {
        const double a = -2.0 * M_PI * (double)t / (double)n;
        tw[t] = make_float2((float)cos(a), (float)sin(a));
    }
    PP_TRY(alloc_n(p, &f.tw, n));
    PP_TRY_CUDA(cudaMemcpy(f.tw, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    return PP_OK;
}

template <class T>
static pp_status upload(Plan& p, T** dst, const std::vector<T>& src) {
    PP_TRY(alloc_n(p, dst, src.size()));
    PP_TRY_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return PP_OK;
}

// Kaiser-Bessel pieces (width W, shape beta):
//   kernel  phi(u) = I0(beta sqrt(1 - (2u/W)^2)), |u| <= W/2
//   its Fourier transform psi(nu) = W sinh(sqrt(a))/sqrt(a), a = beta^2 - (pi W nu)^2
// Kaiser-Bessel kernel phi(u) = I0(beta sqrt(1 - (2u/W)^2)) for |u| <= W/2,
// 0 outside, by the power series I0(x) = sum_k q^k / (k!)^2, q = x^2 / 4.
// Every argument of a plan is at most beta, so one term count serves all:
// the first k at which q_max^k / (k!)^2 < 1e-17 (the sum is >= 1, and past
// the largest term each term shrinks by q / (k + 1)^2 < 1).
static int kb_series_terms(double beta) {
    const double q = 0.25 * beta * beta;
    double t = 1.0;
    int k = 1;
    for (; k < 200; ++k) {
        t *= q / ((double)k * k);
        if (t < 1e-17) break;
    }
    return k;
}
// phi at the 8 offsets u[0..7] (a sample's 4 x-taps and 4 y-taps), the 8
// series summed side by side; inv_k2[k - 1] = 1 / k^2
static void kb_phi8(const double* u, double W, double beta, int nterms, const double* inv_k2,
                    float* out) {
    double q[8], term[8], sum[8];
    for (int i = 0; i < 8; ++i) {
        const double r = 2.0 * u[i] / W, t = 1.0 - r * r;
        q[i] = t < 0.0 ? 0.0 : 0.25 * beta * beta * t;
        term[i] = 1.0;
        sum[i] = 1.0;
    }
    for (int k = 0; k < nterms; ++k)
        for (int i = 0; i < 8; ++i) {
            term[i] *= q[i] * inv_k2[k];
            sum[i] += term[i];
        }
    for (int i = 0; i < 8; ++i) {
        const double r = 2.0 * u[i] / W;
        out[i] = 1.0 - r * r < 0.0 ? 0.f : (float)sum[i];
    }
}
static double kb_psi(double nu, double W, double beta) {
    const double a = beta * beta - (M_PI * W * nu) * (M_PI * W * nu);
    if (a > 0) return W * sinh(sqrt(a)) / sqrt(a);
    if (a < 0) return W * sin(sqrt(-a)) / sqrt(-a);
    return W;
}

static inline int wrap_host(int a, int G) {
    a %= G;
    return a < 0 ? a + G : a;
}

// ---------------------------------------------------------------------------
// operator orchestration
// ---------------------------------------------------------------------------
static ColArgs col_args(int Hin, int Hout, int G, int off_in, int off_out, int ncols,
                        int64_t ibs, int64_t obs, int nbatch, float scale) {
    ColArgs a;
    a.Hin = Hin; a.Hout = Hout; a.G = G; a.off_in = off_in; a.off_out = off_out;
    a.ncols = ncols; a.in_batch_stride = ibs; a.out_batch_stride = obs; a.nbatch = nbatch;
    a.scale = scale; a.mul_in = nullptr; a.mul_out = nullptr; a.mo_q = 0; a.mo_c = 0; a.mo_cdiv = 1;
    a.mi_q = 1; a.mi_c = 0; a.mi_cdiv = 1;
    return a;
}

static RowArgs row_args(int n, int G, int off_in, int off_out, int nrows, int64_t cis, float scale) {
    RowArgs a;
    a.n = n; a.G = G; a.off_in = off_in; a.off_out = off_out; a.nrows = nrows;
    a.coil_img_stride = cis; a.scale = scale;
    return a;
}

// out = scale * (A^H A x) + alpha * operand   (operand may be NULL)
static pp_status normal_into(const Plan& p, const float2* x, float2* out, float scale,
                             const float2* operand, float alpha, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t n = p.nimg;
    if (p.kind == PP_CARTESIAN && p.ndim == 2)
        return launch_cart2d_normal(p, x, out, scale, operand, alpha, st);
    if (p.kind == PP_CARTESIAN) {
        if (p.tune_c3 == 1 && p.c3cl_clusters > 0)
            return c3cl_normal(p, 4, x, out, scale, operand, alpha, st);
        if (p.tune_c3 == 2 && p.c3cl2_clusters > 0)
            return c3cl_normal(p, 2, x, out, scale, operand, alpha, st);
        if (p.tune_c3 == 3 && p.c3df_ctas > 0)
            return c3df_normal(p, x, out, scale, operand, alpha, st);
        bool done = false;
        PP_TRY(cart3d4_normal(p, x, out, scale, operand, alpha, p.wk_a, st, &done));
        if (done) return PP_OK;
        // 3-D: per coil, y FFT -> (z FFT, mask, z IFFT) -> y IFFT -> conj accumulate
        for (int c = 0; c < p.C; ++c) {
            const float2* sc = p.sens + (int64_t)c * n;
            PP_TRY(launch_expand(x, sc, p.wk_a, n, st));
            ColArgs ay = col_args(ny, ny, ny, 0, 0, nx, (int64_t)ny * nx, (int64_t)ny * nx, nz, 1.f);
            PP_TRY(launch_cols(p.fy, ay, p.wk_a, p.wk_b, false, st));
            ColArgs az = col_args(nz, nz, nz, 0, 0, ny * nx, 0, 0, 1, 1.f);
            az.mo_q = ny; az.mo_c = 1; az.mo_cdiv = nx;
            PP_TRY(launch_cols_roundtrip(p.fz, az, p.mask_fo, p.wk_b, p.wk_a, st));
            PP_TRY(launch_cols(p.fy, ay, p.wk_a, p.wk_b, true, st));
            PP_TRY(launch_conj_accum(sc, p.wk_b, out, n, c == 0, scale, operand, alpha, c == p.C - 1, st));
        }
        return PP_OK;
    }
    if (p.toep) return toep_normal(p, x, out, scale, operand, alpha, st);
    // non-Cartesian: rows -> cols -> G^T G stencil -> cols^H -> rows^H
    if (p.tune_stencil_kind >= 7 && p.ci_sens)
        return ci_normal(p, x, out, scale, operand, alpha,
                         p.tune_stencil_kind == 9 ? 0 : (p.tune_stencil_kind == 8 ? 2 : 1), st);
    const int Gx = p.G_x, Gy = p.G_y;
    RowArgs rf = row_args(nx, Gx, nx / 2, 0, ny, (int64_t)ny * nx, 1.f);
    PP_TRY(launch_rows_fwd(p, p.gx, rf, x, p.sens, p.deapod_y, p.deapod_x, p.wk_a, p.C, 0, st));
    ColArgs cf = col_args(ny, Gy, Gy, ny / 2, 0, Gx, (int64_t)ny * Gx, (int64_t)Gy * Gx, p.C, 1.f);
    PP_TRY(launch_cols(p.gy, cf, p.wk_a, p.wk_b, false, st));
    PP_TRY(launch_gtg_stencil(p, p.wk_b, p.wk_c, st));
    ColArgs ci = col_args(Gy, ny, Gy, 0, ny / 2, Gx, (int64_t)Gy * Gx, (int64_t)ny * Gx, p.C, 1.f);
    PP_TRY(launch_cols(p.gy, ci, p.wk_c, p.wk_a, true, st));
    RowArgs ra = row_args(nx, Gx, 0, nx / 2, ny, (int64_t)ny * nx, scale);
    if (p.tune_rows_adj_cl == -1) {
        bool done = false;
        PP_TRY(launch_rows4_adj_split(p.gx, ra, p.wk_a, p.sens, p.deapod_y, p.deapod_x, p.wk_c, out,
                                      operand, alpha, p.C, st, &done));
        if (done) return PP_OK;
    }
    return launch_rows_adj(p, p.gx, ra, p.wk_a, p.sens, p.deapod_y, p.deapod_x, out, operand, alpha,
                           p.C, st);
}

// y = A x (unscaled)
static pp_status forward_into(const Plan& p, const float2* x, float2* y, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t n = p.nimg;
    if (p.kind == PP_CARTESIAN) {
        // centred orthonormal FFT along x, then y (then z), mask on the last axis pass
        RowArgs rf = row_args(nx, nx, nx / 2, nx / 2, ny * nz, n, (float)(1.0 / sqrt((double)nx)));
        PP_TRY(launch_rows_fwd(p, p.fx, rf, x, p.sens, nullptr, nullptr, y, p.C, 0, st));
        ColArgs ay = col_args(ny, ny, ny, ny / 2, ny / 2, nx, (int64_t)ny * nx, (int64_t)ny * nx,
                              p.C * nz, (float)(1.0 / sqrt((double)ny)));
        if (p.ndim == 2) {
            ay.mul_out = p.mask_c; ay.mo_q = 1; ay.mo_c = 0; ay.mo_cdiv = 1;
            return launch_cols(p.fy, ay, y, y, false, st);
        }
        PP_TRY(launch_cols(p.fy, ay, y, y, false, st));
        ColArgs az = col_args(nz, nz, nz, nz / 2, nz / 2, ny * nx, n, n, p.C,
                              (float)(1.0 / sqrt((double)nz)));
        az.mul_out = p.mask_c; az.mo_q = ny; az.mo_c = 1; az.mo_cdiv = nx;
        return launch_cols(p.fz, az, y, y, false, st);
    }
    const int Gx = p.G_x, Gy = p.G_y;
    RowArgs rf = row_args(nx, Gx, nx / 2, 0, ny, (int64_t)ny * nx, 1.f);
    PP_TRY(launch_rows_fwd(p, p.gx, rf, x, p.sens, p.deapod_y, p.deapod_x, p.wk_a, p.C, 0, st));
    ColArgs cf = col_args(ny, Gy, Gy, ny / 2, 0, Gx, (int64_t)ny * Gx, (int64_t)Gy * Gx, p.C, 1.f);
    PP_TRY(launch_cols(p.gy, cf, p.wk_a, p.wk_b, false, st));
    return launch_nufft_degrid(p, p.wk_b, y, st);
}

// x = A^H y (unscaled) with the intermediates in wa and wb (plan workspace, or the
// library's fixed scratch array for pp_adjoint_apply_static): Cartesian 2-D
// needs C*n elements in wa; 3-D n in wa and n in wb; non-Cartesian C*ny*G_x
// in wa and C*G_y*G_x in wb.
pp_status adjoint_ws(const Plan& p, const float2* y, float2* x, float2* wa, float2* wb,
                     cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t n = p.nimg;
    if (p.kind == PP_CARTESIAN && p.ndim == 2) {
        ColArgs ay = col_args(ny, ny, ny, ny / 2, ny / 2, nx, (int64_t)ny * nx, (int64_t)ny * nx, p.C,
                              (float)(1.0 / sqrt((double)ny)));
        ay.mul_in = p.mask_c;   // centred mask indexed by the input row ky
        PP_TRY(launch_cols(p.fy, ay, y, wa, true, st));
        RowArgs ra = row_args(nx, nx, nx / 2, nx / 2, ny, n, (float)(1.0 / sqrt((double)nx)));
        return launch_rows_adj(p, p.fx, ra, wa, p.sens, nullptr, nullptr, x, nullptr, 0.f, p.C, st);
    }
    if (p.kind == PP_CARTESIAN) {
        // 3-D, per coil: mask and inverse centred FFT along z, then y, then
        // the x rows with the conjugate sensitivity, accumulated into x.
        for (int c = 0; c < p.C; ++c) {
            const float2* yc = y + (int64_t)c * n;
            ColArgs az = col_args(nz, nz, nz, nz / 2, nz / 2, ny * nx, 0, 0, 1,
                                  (float)(1.0 / sqrt((double)nz)));
            az.mul_in = p.mask_c; az.mi_q = ny; az.mi_c = 1; az.mi_cdiv = nx;
            PP_TRY(launch_cols(p.fz, az, yc, wa, true, st));
            ColArgs ay = col_args(ny, ny, ny, ny / 2, ny / 2, nx, (int64_t)ny * nx, (int64_t)ny * nx,
                                  nz, (float)(1.0 / sqrt((double)ny)));
            PP_TRY(launch_cols(p.fy, ay, wa, wb, true, st));
            RowArgs ra = row_args(nx, nx, nx / 2, nx / 2, ny * nz, 0, (float)(1.0 / sqrt((double)nx)));
            PP_TRY(launch_rows_adj(p, p.fx, ra, wb, p.sens + (int64_t)c * n, nullptr, nullptr, x,
                                   c == 0 ? nullptr : x, 1.f, 1, st));
        }
        return PP_OK;
    }
    const int Gx = p.G_x, Gy = p.G_y;
    PP_TRY(launch_nufft_spread(p, y, wb, st));
    ColArgs ci = col_args(Gy, ny, Gy, 0, ny / 2, Gx, (int64_t)Gy * Gx, (int64_t)ny * Gx, p.C, 1.f);
    PP_TRY(launch_cols(p.gy, ci, wb, wa, true, st));
    RowArgs ra = row_args(nx, Gx, 0, nx / 2, ny, (int64_t)ny * nx, 1.f);
    return launch_rows_adj(p, p.gx, ra, wa, p.sens, p.deapod_y, p.deapod_x, x, nullptr, 0.f,
                           p.C, st);
}

static pp_status adjoint_into(const Plan& p, const float2* y, float2* x, cudaStream_t st) {
    return adjoint_ws(p, y, x, p.wk_a, p.wk_b, st);
}

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------
static pp_status build_cartesian(Plan& p, const uint8_t* mask) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    // readout invariance: mask[z][y][x] == mask[z][y][0]
    std::vector<float> mc((size_t)nz * ny), mfo((size_t)nz * ny);
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy) {
            const uint8_t* row = mask + ((size_t)z * ny + yy) * nx;
            const uint8_t m0 = row[0] ? 1 : 0;
            for (int x = 1; x < nx; ++x)
                if ((row[x] ? 1 : 0) != m0) {
                    set_error("Cartesian mask varies along the readout axis x (z=%d, y=%d)", z, yy);
                    return PP_ERR_UNSUPPORTED;
                }
            mc[(size_t)z * ny + yy] = (float)m0;
        }
    // FFT order: centred index q holds frequency q - n/2, stored at (q - n/2) mod n
    const double norm = 1.0 / ((double)ny * (double)nz);
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy) {
            const int zf = wrap_host(z - nz / 2, nz), yf = wrap_host(yy - ny / 2, ny);
            mfo[(size_t)zf * ny + yf] = (float)(mc[(size_t)z * ny + yy] * norm);
        }
    PP_TRY(upload(p, &p.mask_c, mc));
    PP_TRY(upload(p, &p.mask_fo, mfo));
    PP_TRY(make_fft(p, nx, p.fx));
    PP_TRY(make_fft(p, ny, p.fy));
    if (p.ndim == 3) PP_TRY(make_fft(p, nz, p.fz));
    if (p.external_wk) {
        // workspace set by the owner
    } else if (p.ndim == 2) {
        PP_TRY(alloc_n(p, &p.wk_a, (size_t)p.C * p.nimg));
    } else {
        PP_TRY(alloc_n(p, &p.wk_a, (size_t)p.nimg));
        PP_TRY(alloc_n(p, &p.wk_b, (size_t)p.nimg));
    }
    p.nksp = (int64_t)p.C * p.nimg;
    return PP_OK;
}

static pp_status build_noncartesian(Plan& p, const pp_sampling* s) {
    const int nx = p.nx, ny = p.ny;
    const int W = s->kb_width;
    const double sigma = s->oversamp;
    if (W != 4) {
        set_error("kb_width must be 4");
        return PP_ERR_UNSUPPORTED;
    }
    if (!(sigma >= 1.125 && sigma <= 2.0)) {
        set_error("oversamp must lie in [1.125, 2]");
        return PP_ERR_INVALID_ARG;
    }
    if (s->K < 1 || s->K > (1 << 26)) {
        set_error("K out of range");
        return PP_ERR_INVALID_ARG;
    }
    const int Gx = (int)ceil(sigma * nx - 1e-9), Gy = (int)ceil(sigma * ny - 1e-9);
    if ((Gx & 1) || (Gy & 1)) {
        set_error("oversampled grid %dx%d must be even", Gy, Gx);
        return PP_ERR_UNSUPPORTED;
    }
    p.G_x = Gx; p.G_y = Gy; p.W = W; p.K = (int)s->K;
    if (Gx < p.T + 2 * W || Gy < p.T + 2 * W) {
        set_error("oversampled grid too small for gridding tiles");
        return PP_ERR_UNSUPPORTED;
    }
    PP_TRY(make_fft(p, Gx, p.gx));
    PP_TRY(make_fft(p, Gy, p.gy));
    // Beatty et al. (2005) shape parameter
    const double beta = M_PI * sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
    std::vector<float> dx(nx), dy(ny);
    for (int i = 0; i < nx; ++i)
        dx[i] = (float)(1.0 / (sqrt((double)nx) * kb_psi((double)(i - nx / 2) / Gx, W, beta)));
    for (int i = 0; i < ny; ++i)
        dy[i] = (float)(1.0 / (sqrt((double)ny) * kb_psi((double)(i - ny / 2) / Gy, W, beta)));
    PP_TRY(upload(p, &p.deapod_x, dx));
    PP_TRY(upload(p, &p.deapod_y, dy));
    // per-sample taps: m in (s - W/2, s + W/2], s = kappa * G / n.  The Bessel
    // series of 8 taps per sample dominates plan set-up at tens of thousands
    // of samples, so contiguous sample ranges run on the host's cores (each
    // sample's taps depend on that sample alone: the result is the same for
    // any thread count)
    const int nterms = kb_series_terms(beta);
    double inv_k2[200];
    for (int k = 1; k <= nterms; ++k) inv_k2[k - 1] = 1.0 / ((double)k * k);
    const int K = p.K;
    std::vector<SampleTaps> st(K);
    std::atomic<int> bad(K);   // the first sample outside the grid, if any
    auto taps = [&](int k0, int k1) {
        for (int k = k0; k < k1; ++k) {
            const double kx = s->traj[2 * k], ky = s->traj[2 * k + 1];
            if (!(kx >= -nx / 2.0 && kx < nx / 2.0 && ky >= -ny / 2.0 && ky < ny / 2.0)) {
                int cur = bad.load();
                while (k < cur && !bad.compare_exchange_weak(cur, k)) {
                }
                continue;
            }
            const double sx = kx * Gx / nx, sy = ky * Gy / ny;
            const int ix0 = (int)floor(sx - W / 2.0) + 1, iy0 = (int)floor(sy - W / 2.0) + 1;
            double u[8];
            for (int a = 0; a < 4; ++a) {
                u[a] = sx - (ix0 + a);
                u[4 + a] = sy - (iy0 + a);
            }
            float w[8];
            kb_phi8(u, W, beta, nterms, inv_k2, w);
            st[k].wx = make_float4(w[0], w[1], w[2], w[3]);
            st[k].wy = make_float4(w[4], w[5], w[6], w[7]);
            st[k].ix0 = ix0;
            st[k].iy0 = iy0;
        }
    };
    // runs body(k0, k1) over nth contiguous ranges of [0, K) on host threads
    const int nth = std::max(1, std::min({16, (int)std::thread::hardware_concurrency(), K / 4096 + 1}));
    auto on_threads = [&](auto&& body) {
        std::vector<std::thread> pool;
        size_t handed = 1;
        try {
            for (int t = 1; t < nth; ++t, ++handed)
                pool.emplace_back(body, t, (int)((int64_t)K * t / nth), (int)((int64_t)K * (t + 1) / nth));
        } catch (const std::exception&) {
            // no more threads: the calling thread takes the ranges not handed out
            for (int t = (int)handed; t < nth; ++t)
                body(t, (int)((int64_t)K * t / nth), (int)((int64_t)K * (t + 1) / nth));
        }
        body(0, 0, (int)((int64_t)K / nth));
        for (auto& th : pool) th.join();
    };
    on_threads([&](int, int k0, int k1) { taps(k0, k1); });
    if (bad.load() < K) {
        const int k = bad.load();
        set_error("trajectory sample %d (%g, %g) outside [-n/2, n/2)", k, s->traj[2 * k], s->traj[2 * k + 1]);
        return PP_ERR_INVALID_ARG;
    }
    PP_TRY(upload(p, &p.samp, st));
    // tile lists (with halo): every tile whose rows and columns meet the footprint
    const int T = p.T, H = W - 1;
    p.ntx = (Gx + T - 1) / T;
    p.nty = (Gy + T - 1) / T;
    const int ntiles = p.ntx * p.nty;
    // per-tile lists in ascending sample order: each thread fills the lists of
    // its sample range, and the ranges are concatenated in order
    std::vector<std::vector<std::vector<TileEntry>>> lists(nth, std::vector<std::vector<TileEntry>>(ntiles));
    on_threads([&](int t, int k0, int k1) {
        for (int k = k0; k < k1; ++k) {
            int trow[4], tcol[4], nr = 0, nc = 0;
            for (int b = 0; b < W; ++b) {
                const int ty = wrap_host(st[k].iy0 + b, Gy) / T;
                if (std::find(trow, trow + nr, ty) == trow + nr) trow[nr++] = ty;
                const int tx = wrap_host(st[k].ix0 + b, Gx) / T;
                if (std::find(tcol, tcol + nc, tx) == tcol + nc) tcol[nc++] = tx;
            }
            for (int i = 0; i < nr; ++i)
                for (int j = 0; j < nc; ++j) {
                    const int ty0 = trow[i] * T, tx0 = tcol[j] * T;
                    const int ly0 = wrap_host(st[k].iy0 - ty0 + H, Gy);
                    const int lx0 = wrap_host(st[k].ix0 - tx0 + H, Gx);
                    TileEntry e;
                    e.wx = st[k].wx;
                    e.wy = st[k].wy;
                    e.lyx = ly0 | (lx0 << 16);
                    e.k = k;
                    lists[t][trow[i] * p.ntx + tcol[j]].push_back(e);
                }
        }
    });
    std::vector<int> start(ntiles + 1, 0);
    std::vector<TileEntry> flat;
    for (int t = 0; t < ntiles; ++t) {
        start[t] = (int)flat.size();
        for (int r = 0; r < nth; ++r) flat.insert(flat.end(), lists[r][t].begin(), lists[r][t].end());
        p.max_tile_len = std::max(p.max_tile_len, (int)flat.size() - start[t]);
    }
    start[ntiles] = (int)flat.size();
    if (flat.empty()) flat.push_back(TileEntry());
    PP_TRY(upload(p, &p.tiles, flat));
    PP_TRY(upload(p, &p.tile_start, start));
    // G^T G as (2W-1)^2 weight planes (FP64 sums of the taps' pairwise
    // products, stored FP32), in both layouts, built on the device
    if (!p.toep) {   // (a Toeplitz plan's normal operator needs no stencil)
        const int D = 2 * W - 1, nxb = (Gx + 7) / 8;
        PP_TRY(alloc_n(p, &p.gtg, (size_t)D * D * Gx * Gy));
        PP_TRY(alloc_n(p, &p.gtg8, (size_t)Gy * nxb * D * D * 8));
        PP_TRY(build_gtg_device(p, 0));
        PP_TRY_CUDA(cudaStreamSynchronize(0));   // weights complete before any use on another stream
        PP_TRY(prepare_gtg_stencil(p));
    }
    PP_TRY(alloc_n(p, &p.wk_a, (size_t)p.C * ny * Gx));
    PP_TRY(alloc_n(p, &p.wk_b, (size_t)p.C * Gy * Gx));
    PP_TRY(alloc_n(p, &p.wk_c, (size_t)p.C * Gy * Gx));
    p.nksp = (int64_t)p.C * K;
    return PP_OK;
}

// Plan-time candidates that launch on thread-block clusters may not fit
// another device: a candidate whose first launch fails (a launch-time error,
// which does not poison the context) is skipped instead of failing the plan.
template <typename F>
static bool launches_ok(F&& fn) {
    if (fn() == PP_OK) return true;
    cudaGetLastError();
    return false;
}

// Plan-time autotuning of the non-Cartesian operator's launch shapes: the
// row-IFFT variant and the stencil kernel are each timed on the plan's own
// buffers (10 launches after two warm-ups, three rounds over all candidates,
// best round kept per candidate) and the fastest is kept.
static pp_status tune_noncartesian(Plan& p, cudaStream_t st) {
    cudaEvent_t e0, e1;
    PP_TRY_CUDA(cudaEventCreate(&e0));
    PP_TRY_CUDA(cudaEventCreate(&e1));
    // warm-up launches, then `reps` timed ones (the whole-operator candidates
    // below, 60-100 us each, are timed 5 at a time: plan set-up is part of a
    // solve's time to target)
    auto timeit = [&](auto&& fn, float* ms, int warm = 2, int reps = 10) -> pp_status {
        for (int r = 0; r < warm; ++r) PP_TRY(fn());
        PP_TRY_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < reps; ++r) PP_TRY(fn());
        PP_TRY_CUDA(cudaEventRecord(e1, st));
        PP_TRY_CUDA(cudaEventSynchronize(e1));
        PP_TRY_CUDA(cudaEventElapsedTime(ms, e0, e1));
        *ms /= (float)reps;
        return PP_OK;
    };
    PP_TRY_CUDA(cudaMemsetAsync(p.wk_a, 0, sizeof(float2) * (size_t)p.C * p.ny * p.G_x, st));
    PP_TRY_CUDA(cudaMemsetAsync(p.wk_b, 0, sizeof(float2) * (size_t)p.C * p.G_y * p.G_x, st));
    const int nx = p.nx, ny = p.ny, Gx = p.G_x;
    RowArgs ra = row_args(nx, Gx, 0, nx / 2, ny, (int64_t)ny * nx, 1.f);
    // With the coil-innermost pipeline available the choice is made on the
    // whole operator below, where the [coil][row][col] pipeline enters with one
    // default launch shape per stage (it lost to the coil-innermost one on
    // every measured shape): the per-stage sweeps, which dominate plan time,
    // run only for plans without that pipeline.
    const bool sweep = !p.ci_sens;
    const int kRounds = sweep ? 3 : 0;
    std::vector<int> rows;
    for (int cl : {1, 2, 4, -1})
        if (cl != -1 || fft4_n2(Gx)) rows.push_back(cl);
    std::vector<float> rbest(rows.size(), 1e30f);
    for (int round = 0; round < kRounds; ++round)
        for (size_t i = 0; i < rows.size(); ++i) {
            const int cl = rows[i];
            p.tune_rows_adj_cl = cl;
            float ms = 0.f;
            if (cl == -1) {
                PP_TRY(timeit([&]() {
                    bool done = false;
                    return launch_rows4_adj_split(p.gx, ra, p.wk_a, p.sens, p.deapod_y, p.deapod_x,
                                                  p.wk_c, p.t, nullptr, 0.f, p.C, st, &done);
                }, &ms));
            } else {
                PP_TRY(timeit([&]() { return launch_rows_adj(p, p.gx, ra, p.wk_a, p.sens, p.deapod_y,
                                                             p.deapod_x, p.t, nullptr, 0.f, p.C, st); },
                              &ms));
            }
            rbest[i] = std::min(rbest[i], ms);
        }
    p.tune_rows_adj_cl = sweep ? rows[std::min_element(rbest.begin(), rbest.end()) - rbest.begin()] : 1;
    std::vector<std::pair<int, int>> sten;   // (kind, coils per CTA)
    for (int kind = 0; kind <= 6; ++kind)
        for (int cpc : {2, 4, 8, 16, 32}) {
            if (kind >= 2 && cpc != 8) continue;
            if (kind >= 2 && kind <= 5 && p.stencil_rb_grid[kind - 2] == 0) continue;
            if (kind == 6 && (!p.gtg8 || p.stencil_rb_grid[0] == 0)) continue;
            if (cpc > p.C && cpc != 2) continue;
            sten.push_back({kind, cpc});
        }
    std::vector<float> sbest(sten.size(), 1e30f);
    for (int round = 0; round < kRounds; ++round)
        for (size_t i = 0; i < sten.size(); ++i) {
            p.tune_stencil_kind = sten[i].first;
            p.tune_stencil_cpc = sten[i].second;
            float ms = 0.f;
            PP_TRY(timeit([&]() { return launch_gtg_stencil(p, p.wk_b, p.wk_c, st); }, &ms));
            sbest[i] = std::min(sbest[i], ms);
        }
    const size_t bi = std::min_element(sbest.begin(), sbest.end()) - sbest.begin();
    p.tune_stencil_kind = sweep ? sten[bi].first : 1;
    p.tune_stencil_cpc = sweep ? sten[bi].second : 8;
    // whole operator: the tuned [coil][row][col] pipeline against the
    // coil-innermost one (kinds 7, 8)
    if (p.ci_sens) {
        // (stencil kind, row variant): for kinds 7 and 8 the row variant 4
        // reduces the four 8-coil blocks of a row in a thread-block cluster
        std::vector<std::pair<int, int>> whole = {{p.tune_stencil_kind, p.tune_rows_adj_cl},
                                                  {7, 1}, {7, 4}, {8, 1}, {8, 4}, {9, 1}, {9, 4}};
        PP_TRY_CUDA(cudaMemsetAsync(p.v, 0, sizeof(float2) * (size_t)p.nimg, st));
        std::vector<float> wbest(whole.size(), 1e30f);
        for (int round = 0; round < 2; ++round) {
            // the second round re-times only the candidates within 10 % of
            // the first round's best
            const float cut = round == 0 ? 1.5e30f
                                         : 1.1f * *std::min_element(wbest.begin(), wbest.end());
            for (size_t i = 0; i < whole.size(); ++i) {
                p.tune_stencil_kind = whole[i].first;
                p.tune_rows_adj_cl = whole[i].second;
                if (round == 0 && i > 0 && !launches_ok([&]() {
                        return normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st); }))
                    wbest[i] = 2e30f;   // a cluster shape this device cannot place
                if (wbest[i] > cut) continue;
                float ms = 0.f;
                PP_TRY(timeit([&]() { return normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st); }, &ms, 1, 5));
                wbest[i] = std::min(wbest[i], ms);
            }
        }
        const size_t wi = std::min_element(wbest.begin(), wbest.end()) - wbest.begin();
        p.tune_stencil_kind = whole[wi].first;
        p.tune_rows_adj_cl = whole[wi].second;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return PP_OK;
}

// Launch shapes chosen by the plan-time tuners are kept per geometry for the
// life of the process: a later plan with the same geometry and sampling on
// the same device takes them instead of timing the candidates again (the
// choice depends on the shapes and, through tile lists and empty stencil
// tiles, on the trajectory; not on the coil maps or the image).
struct TuneKey {
    int dev, kind, ndim, nx, ny, nz, C, K, kb, toep;
    uint64_t data;   // FNV-1a of the trajectory (non-Cartesian) or the mask (Cartesian)
    double oversamp;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, kind, ndim, nx, ny, nz, C, K, kb, toep, data, oversamp) <
               std::tie(o.dev, o.kind, o.ndim, o.nx, o.ny, o.nz, o.C, o.K, o.kb, o.toep, o.data, o.oversamp);
    }
};
struct TuneVal {
    int rows_adj_cl, stencil_kind, stencil_cpc, c3, c3df_cg, c3df_hi, c2;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune_cache;

static uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}
static TuneKey tune_key(const Plan& p, const pp_sampling* s, int dev) {
    TuneKey k{};
    k.dev = dev; k.kind = (int)s->kind; k.ndim = p.ndim; k.nx = p.nx; k.ny = p.ny; k.nz = p.nz;
    k.C = p.C; k.K = s->kind == PP_CARTESIAN ? 0 : (int)s->K; k.kb = s->kb_width;
    k.toep = p.toep ? 1 : 0; k.oversamp = s->kind == PP_CARTESIAN ? 0.0 : s->oversamp;
    k.data = s->kind == PP_CARTESIAN ? fnv1a(s->mask, (size_t)p.nimg)
                                     : fnv1a(s->traj, sizeof(float) * 2 * (size_t)s->K);
    return k;
}
static bool tune_lookup(const TuneKey& k, Plan& p) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(k);
    if (it == g_tune_cache.end()) return false;
    const TuneVal& v = it->second;
    p.tune_rows_adj_cl = v.rows_adj_cl; p.tune_stencil_kind = v.stencil_kind;
    p.tune_stencil_cpc = v.stencil_cpc; p.tune_c3 = v.c3; p.c3df_cg = v.c3df_cg;
    p.c3df_hi = v.c3df_hi; p.tune_c2 = v.c2;
    return true;
}
static void tune_store(const TuneKey& k, const Plan& p) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[k] = TuneVal{p.tune_rows_adj_cl, p.tune_stencil_kind, p.tune_stencil_cpc, p.tune_c3,
                              p.c3df_cg, p.c3df_hi, p.tune_c2};
}

// 3-D Cartesian: the three passes per coil, the one-kernel cluster operator
// and the dataflow operator with 2, 4 or 8 coils per group, timed on the
// plan's buffers (two rounds of 3 applies after one warm-up); the fastest is
// kept.
static pp_status tune_cart3d(Plan& p, cudaStream_t st) {
    struct Cand { int kind, cg, hi; };
    std::vector<Cand> cand = {{0, 0, 0}};
    if (p.c3cl_clusters > 0) cand.push_back({1, 0, 0});
    if (p.c3cl2_clusters > 0) cand.push_back({2, 0, 0});
    for (int hi = 0; hi < 6; ++hi)
        if ((hi == 3 ? p.c3df_ctas_tma1 : hi == 2 ? p.c3df_ctas_tma
             : (hi == 1 || hi == 5) ? p.c3df_ctas_hi : p.c3df_ctas) > 0)
            for (int cgc : {2, 4, 8})
                if (cgc <= std::max(2, p.C) && (cgc == 2 || cgc <= p.C) &&
                    2 * c3df_slot_elems(p, cgc) <= p.c3df_w_elems)
                    cand.push_back({3, cgc, hi});
    if (cand.size() == 1) return PP_OK;
    cudaEvent_t e0, e1;
    PP_TRY_CUDA(cudaEventCreate(&e0));
    PP_TRY_CUDA(cudaEventCreate(&e1));
    PP_TRY_CUDA(cudaMemsetAsync(p.v, 0, sizeof(float2) * (size_t)p.nimg, st));
    std::vector<float> best(cand.size(), 1e30f);
    for (int round = 0; round < 2; ++round)
        for (size_t i = 0; i < cand.size(); ++i) {
            p.tune_c3 = cand[i].kind;
            if (cand[i].cg) {
                p.c3df_cg = cand[i].cg;
                p.c3df_hi = cand[i].hi;
            }
            if (best[i] > 1.5e30f) continue;
            if (!launches_ok([&]() { return normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st); }) ||
                (p.tune_c3 == 3 && c3df_check(p, st) != PP_OK)) {
                best[i] = 2e30f;
                continue;
            }
            PP_TRY_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < 3; ++r) PP_TRY(normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st));
            PP_TRY_CUDA(cudaEventRecord(e1, st));
            PP_TRY_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            PP_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (p.tune_c3 == 3 && c3df_check(p, st) != PP_OK) ms = 2e30f;
            best[i] = std::min(best[i], ms);
        }
    const size_t bi = std::min_element(best.begin(), best.end()) - best.begin();
    p.tune_c3 = cand[bi].kind;
    if (cand[bi].cg) {
        p.c3df_cg = cand[bi].cg;
        p.c3df_hi = cand[bi].hi;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return PP_OK;
}

// 2-D Cartesian: one CTA per 8-column group against the coils split over a
// cluster of 2, 4 or 8 CTAs per group (narrow images leave most SMs idle
// otherwise), timed on the plan's buffers; the fastest is kept.
static pp_status tune_cart2d(Plan& p, cudaStream_t st) {
    if (!fft4_n2(p.ny)) return PP_OK;
    cudaEvent_t e0, e1;
    PP_TRY_CUDA(cudaEventCreate(&e0));
    PP_TRY_CUDA(cudaEventCreate(&e1));
    PP_TRY_CUDA(cudaMemsetAsync(p.v, 0, sizeof(float2) * (size_t)p.nimg, st));
    std::vector<int> cand = {1};
    for (int cl : {2, 4, 8})
        if (cl <= p.C) cand.push_back(cl);
    std::vector<float> best(cand.size(), 1e30f);
    for (int round = 0; round < 3; ++round)
        for (size_t i = 0; i < cand.size(); ++i) {
            p.tune_c2 = cand[i];
            if (best[i] > 1.5e30f) continue;
            if (!launches_ok([&]() { return normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st); })) {
                best[i] = 2e30f;
                continue;
            }
            PP_TRY(normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st));
            PP_TRY_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < 10; ++r) PP_TRY(normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st));
            PP_TRY_CUDA(cudaEventRecord(e1, st));
            PP_TRY_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            PP_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best[i] = std::min(best[i], ms);
        }
    p.tune_c2 = cand[std::min_element(best.begin(), best.end()) - best.begin()];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return PP_OK;
}

// Toeplitz-embedded normal operator: twiddles of the 2n transforms, the
// coil-innermost maps, the two [ny][2nx][32] arrays (zeroed once, so that
// coil blocks past C read zeros) and the kernel spectrum.
static pp_status setup_toeplitz(Plan& p, const pp_sampling* s, cudaStream_t st) {
    PP_TRY(make_fft(p, 2 * p.nx, p.tx));
    PP_TRY(make_fft(p, 2 * p.ny, p.ty));
    PP_TRY(make_fft(p, p.nx, p.toep_hx));
    PP_TRY(make_fft(p, p.ny, p.toep_hy));
    if (!p.ci_sens) {
        PP_TRY(alloc_n(p, &p.ci_sens, ci_sens_elems(p)));
        PP_TRY(ci_prepare(p, st));
    }
    const size_t nr = toep_rows_elems(p);
    PP_TRY(alloc_n(p, &p.toep_a, nr));
    PP_TRY(alloc_n(p, &p.toep_b, nr));
    PP_TRY_CUDA(cudaMemsetAsync(p.toep_a, 0, sizeof(float2) * nr, st));
    PP_TRY_CUDA(cudaMemsetAsync(p.toep_b, 0, sizeof(float2) * nr, st));
    PP_TRY(alloc_n(p, &p.toep_T, (size_t)4 * p.nx * p.ny));
    return toep_build_kernel(p, s->traj, s->K, st);
}

// Buffers of the coil-innermost pipeline (when the plan supports it).
static pp_status setup_ci(Plan& p, cudaStream_t st) {
    if (!ci_supported(p)) return PP_OK;
    PP_TRY(alloc_n(p, &p.ci_sens, ci_sens_elems(p)));
    PP_TRY(alloc_n(p, &p.ci_part, ci_partial_elems(p)));
    if (p.C == 32) {
        p.ci_a = p.wk_a;
        p.ci_b = p.wk_b;
        p.ci_c = p.wk_c;
    } else {
        PP_TRY(alloc_n(p, &p.ci_a, ci_rows_elems(p)));
        PP_TRY(alloc_n(p, &p.ci_b, ci_grid_elems(p)));
        PP_TRY(alloc_n(p, &p.ci_c, ci_grid_elems(p)));
    }
    PP_TRY(alloc_n(p, &p.ci_tile_nz, ci_stencil_tiles(p)));
    return ci_prepare(p, st);
}

static pp_status power_iteration(Plan& p, uint64_t seed, int iters, cudaStream_t st) {
    const int64_t n = p.nimg;
    PP_TRY(launch_start_vector(p.v, n, seed, st));
    PP_TRY(launch_norm2(p.v, n, p.red, p.red_blocks, p.scal + 2, st));
    PP_TRY(launch_scale_by_rnorm(p.v, p.v, n, p.scal + 2, 1.0, 1, st));
    for (int it = 0; it < iters; ++it) {
        PP_TRY(normal_into(p, p.v, p.t, 1.f, nullptr, 0.f, st));
        PP_TRY(launch_dot(p.v, p.t, n, p.red, p.red_blocks, p.scal + 1, p.scal + 2, st));
        PP_TRY(launch_scale_by_rnorm(p.t, p.v, n, p.scal + 2, 1.0, 1, st));
    }
    double L = 0.0;
    PP_TRY_CUDA(cudaMemcpyAsync(&L, p.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    PP_TRY(c3df_check(p, st));
    if (!(L > 0.0) || !isfinite(L)) {
        set_error("power iteration gave a non-positive or non-finite norm estimate (%g)", L);
        return PP_ERR_NONFINITE;
    }
    p.L = L;
    return PP_OK;
}

// Power iteration on I - N_hat (the remark closing the Chebyshev design of
// Sec. 3.4): converges to 1 - mu, mu the smallest eigenvalue of N_hat when
// A^H A is injective.  Same start vector and FP64 reductions as
// power_iteration; returns mu = 1 - (last Rayleigh quotient).
static pp_status mu_iteration(Plan& p, uint64_t seed, int iters, double* mu, cudaStream_t st) {
    const int64_t n = p.nimg;
    PP_TRY(launch_start_vector(p.v, n, seed, st));
    PP_TRY(launch_norm2(p.v, n, p.red, p.red_blocks, p.scal + 2, st));
    PP_TRY(launch_scale_by_rnorm(p.v, p.v, n, p.scal + 2, 1.0, 1, st));
    const float s = (float)(-1.0 / p.L);
    for (int it = 0; it < iters; ++it) {
        PP_TRY(normal_into(p, p.v, p.t, s, p.v, 1.f, st));   // t = v - N_hat v
        PP_TRY(launch_dot(p.v, p.t, n, p.red, p.red_blocks, p.scal + 1, p.scal + 2, st));
        PP_TRY(launch_scale_by_rnorm(p.t, p.v, n, p.scal + 2, 1.0, 1, st));
    }
    double rho = 0.0;
    PP_TRY_CUDA(cudaMemcpyAsync(&rho, p.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    PP_TRY(c3df_check(p, st));
    if (!isfinite(rho)) {
        set_error("pp_plan_mu: non-finite Rayleigh quotient");
        return PP_ERR_NONFINITE;
    }
    *mu = 1.0 - rho;
    return PP_OK;
}

static bool fft_len_ok(int n) {
    FftDesc d;
    return factorize(n, d);
}

// ---------------------------------------------------------------------------
// Horner recursion (Listing "pcode"): u = c_d v; u = c_i v + N_hat u.
// The first step folds c_d into the apply: u = c_{d-1} v + (c_d/L) N v.
// Writes the result into `out`; bufA/bufB are scratch images.
// ---------------------------------------------------------------------------
static pp_status horner_into(const Plan& p, const double* c, int d, const float2* v, float2* out,
                             float2* bufA, float2* bufB, cudaStream_t st) {
    const float invL = (float)(1.0 / p.L);
    if (d == 0) return launch_axpby(v, (float)c[0], nullptr, 0.f, out, p.nimg, st);
    const float2* cur = v;
    float scale = (float)(c[d] / p.L);
    for (int i = d - 1; i >= 0; --i) {
        float2* dst = (i == 0) ? out : ((cur == bufA) ? bufB : bufA);
        PP_TRY(normal_into(p, cur, dst, scale, v, (float)c[i], st));
        cur = dst;
        scale = invL;
    }
    return PP_OK;
}

// `shift` (sh_a, sh_b): the iteration runs on a N_hat + sh_b I instead of
// N_hat (the proximal subproblem of pp_fista_solve_prox); the caller then
// passes the preconditioner already rewritten as a polynomial in N_hat.
struct Shift {
    bool on = false;
    float a = 1.f, b = 0.f;
};

static pp_status fista_iterations(Plan& p, float lambda, int iters, const double* c, int d,
                                  int levels, bool hist, const float2* ref, bool momentum,
                                  int wavelet, cudaStream_t st, Shift sh = Shift()) {
    const float invL = (float)(1.0 / p.L);
    for (int k = 0; k < iters; ++k) {
        if (sh.on) {
            // g = (a N_hat + b I) z - rhs: u = b z - rhs, then g = a N_hat z + u
            PP_TRY(launch_axpby(p.z, sh.b, p.ahb, -1.f, p.u, p.nimg, st));
            PP_TRY(normal_into(p, p.z, p.g, sh.a * invL, p.u, 1.f, st));
        } else {
            // g = N_hat z - A_hat^H b_hat
            PP_TRY(normal_into(p, p.z, p.g, invL, p.ahb, -1.f, st));
        }
        const float2* u = p.g;
        float gamma = 1.f;
        if (c && d >= 1) {
            PP_TRY(horner_into(p, c, d, p.g, p.u, p.t, p.w3, st));
            u = p.u;
        } else if (c) {
            gamma = (float)c[0];
        }
        const float beta = momentum ? (float)((double)k / (k + 3.0)) : 0.f;
        if (wavelet == 1)   // Daubechies-4: multi-pass, p.t (free after Horner) holds the coefficients
            PP_TRY(launch_prox_fista_db4(p, levels, lambda, gamma, beta, u, p.t, hist ? ref : nullptr,
                                         hist ? p.hist + 3 * k : nullptr, st));
        else
            PP_TRY(launch_prox_fista(p, levels, lambda, gamma, beta, u, hist ? ref : nullptr,
                                     hist ? p.hist + 3 * k : nullptr, st));
    }
    return PP_OK;
}


// ---------------------------------------------------------------------------
// Batched uneven 2-D Cartesian problems
// ---------------------------------------------------------------------------
struct Batch {
    int n = 0;
    std::vector<Plan*> sub;
    std::vector<int64_t> img_off, ksp_off, tile_off;
    int64_t nimg = 0, nksp = 0;
    std::vector<double> L;
    std::vector<SliceDesc> hdesc;
    BatchDev dev;
    std::vector<void*> allocs;
    float2 *z = nullptr, *y = nullptr, *g = nullptr, *u = nullptr, *t = nullptr, *ahb = nullptr,
           *v = nullptr, *w3 = nullptr, *wk = nullptr;
    double *partials = nullptr, *scal = nullptr, *dfac = nullptr, *hist = nullptr;
    int hist_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<double> gkey;
    int64_t graph_kernels = 0;
    int uni_n2 = 0;   // common N2 of all slices when the uniform-length kernel applies, else 0
    // differentiable unrolled solve: arena of image vectors and FP64 slots
    float2* arena = nullptr;
    size_t arena_vecs = 0;
    double* dslots = nullptr;
    size_t dslots_n = 0;
    std::vector<double> tape_key;
};

template <class T>
static pp_status balloc(Batch& b, T** ptr, size_t n) {
    *ptr = nullptr;
    if (n == 0) return PP_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), n * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return cuda_status(e, "cudaMalloc");
    }
    b.allocs.push_back(*ptr);
    return PP_OK;
}

template <class T>
static pp_status bupload(Batch& b, T** dst, const std::vector<T>& src) {
    PP_TRY(balloc(b, dst, src.size()));
    PP_TRY_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return PP_OK;
}

// blocks per segment: ceil(len / per_block) clamped to [1, max_blocks]
static pp_status make_segments(Batch& b, Segments& sg, const std::vector<int64_t>& off,
                               int64_t per_block, int max_blocks) {
    const int nseg = (int)off.size() - 1;
    std::vector<int> blk_seg, first(nseg + 1, 0);
    for (int s = 0; s < nseg; ++s) {
        const int64_t len = off[s + 1] - off[s];
        int64_t nb = (len + per_block - 1) / per_block;
        nb = std::max<int64_t>(1, std::min<int64_t>(nb, max_blocks));
        first[s] = (int)blk_seg.size();
        for (int64_t j = 0; j < nb; ++j) blk_seg.push_back(s);
    }
    first[nseg] = (int)blk_seg.size();
    sg.nseg = nseg;
    sg.nblocks = (int)blk_seg.size();
    PP_TRY(bupload(b, &sg.off, off));
    PP_TRY(bupload(b, &sg.blk_seg, blk_seg));
    PP_TRY(bupload(b, &sg.seg_first_blk, first));
    return PP_OK;
}

static int km_for(int ny_max, int lgt) {
    const int need = (ny_max * (1 << lgt) + kThreads - 1) / kThreads;
    const int kms[] = {4, 8, 12, 16};
    for (int km : kms)
        if (need <= km && batch_normal_fn(km, lgt)) return km;
    return 0;
}

// Work items (slice, first column) for column tiles of 2^lgt, most expensive
// first so that the persistent grid's round-robin balances the load.
static pp_status set_items(Batch& b, int lgt, std::vector<int2>* scratch) {
    const int T = 1 << lgt;
    std::vector<std::pair<double, int2>> it;
    for (int s = 0; s < b.n; ++s) {
        const SliceDesc& d = b.hdesc[s];
        const double cost = (double)d.C * d.ny * log2((double)d.ny);
        for (int c0 = 0; c0 < d.nx; c0 += T) it.push_back({cost, make_int2(s, c0)});
    }
    std::stable_sort(it.begin(), it.end(),
                     [](const std::pair<double, int2>& a, const std::pair<double, int2>& c) {
                         return a.first > c.first;
                     });
    scratch->clear();
    for (auto& e : it) scratch->push_back(e.second);
    if (b.dev.items) {
        cudaFree(b.dev.items);
        b.allocs.erase(std::remove(b.allocs.begin(), b.allocs.end(), (void*)b.dev.items), b.allocs.end());
        b.dev.items = nullptr;
    }
    PP_TRY(bupload(b, &b.dev.items, *scratch));
    b.dev.nitems = (int)scratch->size();
    b.dev.lgt = lgt;
    b.dev.km = km_for(b.dev.ny_max, lgt);
    int occ = 0;
    PP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, batch_normal_fn(b.dev.km, lgt), kThreads, batch_normal_smem(b.dev.ny_max, lgt)));
    int nsm = 0;
    PP_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
    b.dev.grid = std::max(1, std::min(b.dev.nitems, nsm * std::max(occ, 1)));
    return PP_OK;
}

static pp_status upload_descs(Batch& b) {
    for (int s = 0; s < b.n; ++s) b.hdesc[s].invL = (float)(1.0 / b.L[s]);
    PP_TRY_CUDA(cudaMemcpy(b.dev.descs, b.hdesc.data(), b.n * sizeof(SliceDesc), cudaMemcpyHostToDevice));
    std::vector<double> f(b.n);
    for (int s = 0; s < b.n; ++s) f[s] = 1.0 / sqrt(b.L[s]);
    PP_TRY_CUDA(cudaMemcpy(b.dfac, f.data(), b.n * sizeof(double), cudaMemcpyHostToDevice));
    b.gkey.clear();
    return PP_OK;
}

// Column-tile autotuner: time each feasible tile width on the batch itself
// and keep the fastest.
static pp_status autotune(Batch& b, cudaStream_t st) {
    std::vector<int2> items;
    int best = -1, best_cl = 1;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    PP_TRY_CUDA(cudaEventCreate(&e0));
    PP_TRY_CUDA(cudaEventCreate(&e1));
    bool all_fast = true;
    for (const SliceDesc& d : b.hdesc) all_fast = all_fast && d.n2 != 0;
    // candidates: Stockham kernels with 4, 8 or 16 columns per item (lgt 2..4)
    // and, when every slice length has one, the register four-step kernel (5)
    // with 1, 2 or 4 CTAs per item (coils split over a cluster)
    for (int lgt = 2; lgt <= 5; ++lgt)
        for (int cl : {1, 2, 4}) {
            if (lgt < 5 && cl > 1) continue;
            if (lgt == 5) {
                if (!all_fast) continue;
                PP_TRY(set_items(b, 3, &items));
                b.dev.fast4 = 1;
                b.dev.cl = cl;
                b.dev.un2 = b.uni_n2;
                b.dev.grid = batch4_grid();
            } else {
                if (!km_for(b.dev.ny_max, lgt)) continue;
                b.dev.fast4 = 0;
                b.dev.cl = 1;
                b.dev.un2 = 0;
                PP_TRY(set_items(b, lgt, &items));
            }
            if (!launches_ok([&]() { return launch_batch_normal(b.dev, b.v, b.t, 1.f, nullptr, 0.f, st); }))
                continue;   // a cluster shape this device cannot place
            PP_TRY_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < 3; ++r) PP_TRY(launch_batch_normal(b.dev, b.v, b.t, 1.f, nullptr, 0.f, st));
            PP_TRY_CUDA(cudaEventRecord(e1, st));
            PP_TRY_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = lgt;
                best_cl = cl;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        set_error("no batched kernel fits ny_max = %d", b.dev.ny_max);
        return PP_ERR_UNSUPPORTED;
    }
    if (best == 5) {
        PP_TRY(set_items(b, 3, &items));
        b.dev.fast4 = 1;
        b.dev.cl = best_cl;
        b.dev.un2 = b.uni_n2;
        b.dev.grid = batch4_grid();
        return PP_OK;
    }
    b.dev.fast4 = 0;
    b.dev.cl = 1;
    b.dev.un2 = 0;
    return set_items(b, best, &items);
}

static pp_status batch_power_iteration(Batch& b, uint64_t seed, int iters, cudaStream_t st) {
    for (int s = 0; s < b.n; ++s)
        PP_TRY(launch_start_vector(b.v + b.img_off[s], b.img_off[s + 1] - b.img_off[s], seed + s, st));
    PP_TRY(launch_seg_dot(nullptr, b.v, b.dev.img, b.partials, nullptr, b.scal + 2, 4, st));
    PP_TRY(launch_seg_scale(b.v, b.v, b.dev.img, b.scal + 2, 4, nullptr, 1, st));
    for (int it = 0; it < iters; ++it) {
        PP_TRY(launch_batch_normal(b.dev, b.v, b.t, 1.f, nullptr, 0.f, st));
        PP_TRY(launch_seg_dot(b.v, b.t, b.dev.img, b.partials, b.scal + 1, b.scal + 2, 4, st));
        PP_TRY(launch_seg_scale(b.t, b.v, b.dev.img, b.scal + 2, 4, nullptr, 1, st));
    }
    std::vector<double> h(4 * b.n);
    PP_TRY_CUDA(cudaMemcpyAsync(h.data(), b.scal, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < b.n; ++s) {
        if (!(h[4 * s + 1] > 0.0) || !isfinite(h[4 * s + 1])) {
            set_error("power iteration: non-positive estimate for slice %d", s);
            return PP_ERR_NONFINITE;
        }
        b.L[s] = h[4 * s + 1];
    }
    return upload_descs(b);
}

static pp_status batch_horner(Batch& b, const double* c, int d, const float2* v, float2* out,
                              cudaStream_t st) {
    if (d == 0) return launch_axpby(v, (float)c[0], nullptr, 0.f, out, b.nimg, st);
    const float2* cur = v;
    float coef = (float)c[d];
    for (int i = d - 1; i >= 0; --i) {
        float2* dst = (i == 0) ? out : ((cur == b.t) ? b.w3 : b.t);
        PP_TRY(launch_batch_normal(b.dev, cur, dst, coef, v, (float)c[i], st));
        cur = dst;
        coef = 1.f;
    }
    return PP_OK;
}

static pp_status batch_iterations(Batch& b, float lambda, int iters, const double* c, int d,
                                  bool hist, const float2* ref, bool momentum, cudaStream_t st) {
    for (int k = 0; k < iters; ++k) {
        PP_TRY(launch_batch_normal(b.dev, b.z, b.g, 1.f, b.ahb, -1.f, st));
        const float2* u = b.g;
        float gamma = 1.f;
        if (c && d >= 1) {
            PP_TRY(batch_horner(b, c, d, b.g, b.u, st));
            u = b.u;
        } else if (c) {
            gamma = (float)c[0];
        }
        const float beta = momentum ? (float)((double)k / (k + 3.0)) : 0.f;
        PP_TRY(launch_batch_prox_fista(b.dev, lambda, gamma, beta, b.z, u, b.y, hist ? ref : nullptr,
                                       hist ? b.hist + 3 * k : nullptr, st));
    }
    return PP_OK;
}


// ---------------------------------------------------------------------------
// Differentiable unrolled solve on a batch: raw b (no normalisation, L_s
// fixed), Algorithm "pfista" for a fixed iteration count, checkpoints
// (y_k, z_k) every `ce` iterations, and the reverse pass.
// Arena layout (image-sized vectors): [0] ahb, [1 .. 2*ncp] checkpoints,
// then 3*ce segment vectors (z_k, g_k, w_k), d+2 Horner-adjoint vectors and
// Ybar, Zbar, wbar, ahb_bar, yw, zw.
// ---------------------------------------------------------------------------
static pp_status ensure_arena(Batch& b, size_t vecs, size_t slots) {
    if (vecs > b.arena_vecs) {
        if (b.arena) {
            cudaFree(b.arena);
            b.allocs.erase(std::remove(b.allocs.begin(), b.allocs.end(), (void*)b.arena), b.allocs.end());
            b.arena = nullptr;
            b.arena_vecs = 0;
        }
        PP_TRY(balloc(b, &b.arena, vecs * (size_t)b.nimg));
        b.arena_vecs = vecs;
        b.tape_key.clear();
    }
    if (slots > b.dslots_n) {
        if (b.dslots) {
            cudaFree(b.dslots);
            b.allocs.erase(std::remove(b.allocs.begin(), b.allocs.end(), (void*)b.dslots), b.allocs.end());
            b.dslots = nullptr;
            b.dslots_n = 0;
        }
        PP_TRY(balloc(b, &b.dslots, slots));
        b.dslots_n = slots;
    }
    return PP_OK;
}

static inline float2* avec(Batch& b, size_t i) { return b.arena + i * (size_t)b.nimg; }

static size_t unrolled_vecs(int iters, int ce, int d) {
    const size_t ncp = (size_t)((iters + ce - 1) / ce);
    return 1 + 2 * ncp + 3 * (size_t)ce + (size_t)(d + 2) + 6;
}

static pp_status unrolled_step(Batch& b, const double* c, int d, float lambda, int k, float2* z,
                               float2* y, float2* g_out, float2* w_out, cudaStream_t st) {
    const float2* ahb = avec(b, 0);
    PP_TRY(launch_batch_normal(b.dev, z, g_out, 1.f, ahb, -1.f, st));
    PP_TRY(batch_horner(b, c, d, g_out, b.u, st));
    if (w_out) {
        LinComb lc;
        lc.count = 2;
        lc.v[0] = z; lc.coef[0] = 1.f;
        lc.v[1] = b.u; lc.coef[1] = -1.f;
        PP_TRY(launch_lincomb(lc, w_out, b.nimg, 0, st));
    }
    const float beta = (float)((double)k / (k + 3.0));
    return launch_batch_prox_fista(b.dev, lambda, 1.f, beta, z, b.u, y, nullptr, nullptr, st);
}

static pp_status unrolled_forward(Batch& b, const float2* bk, float lambda, int iters,
                                  const double* c, int d, int ce, float2* x_out, cudaStream_t st) {
    PP_TRY(ensure_arena(b, unrolled_vecs(iters, ce, d), (size_t)iters * (d + 1) + 1));
    float2* ahb = avec(b, 0);
    for (int s = 0; s < b.n; ++s)
        PP_TRY(adjoint_into(*b.sub[s], bk + b.ksp_off[s], ahb + b.img_off[s], st));
    PP_TRY(launch_seg_scale(ahb, ahb, b.dev.img, nullptr, 0, b.dfac, 0, st));
    PP_TRY_CUDA(cudaMemsetAsync(b.y, 0, b.nimg * sizeof(float2), st));
    PP_TRY_CUDA(cudaMemsetAsync(b.z, 0, b.nimg * sizeof(float2), st));
    const size_t bytes = (size_t)b.nimg * sizeof(float2);
    for (int k = 0; k < iters; ++k) {
        if (k % ce == 0) {
            const int cp = k / ce;
            PP_TRY_CUDA(cudaMemcpyAsync(avec(b, 1 + 2 * cp), b.y, bytes, cudaMemcpyDeviceToDevice, st));
            PP_TRY_CUDA(cudaMemcpyAsync(avec(b, 2 + 2 * cp), b.z, bytes, cudaMemcpyDeviceToDevice, st));
        }
        PP_TRY(unrolled_step(b, c, d, lambda, k, b.z, b.y, b.g, nullptr, st));
    }
    PP_TRY_CUDA(cudaMemcpyAsync(x_out, b.y, bytes, cudaMemcpyDeviceToDevice, st));
    return PP_OK;
}

static pp_status unrolled_backward(Batch& b, float lambda, int iters, const double* c, int d,
                                   int ce, const float2* gout, float2* grad_b, double* grad_lam,
                                   double* grad_c, cudaStream_t st) {
    const size_t ncp = (size_t)((iters + ce - 1) / ce);
    const size_t seg0 = 1 + 2 * ncp, v0 = seg0 + 3 * (size_t)ce, r0 = v0 + (size_t)(d + 2);
    float2 *Ybar = avec(b, r0), *Zbar = avec(b, r0 + 1), *wbar = avec(b, r0 + 2),
           *ahb_bar = avec(b, r0 + 3), *yw = avec(b, r0 + 4), *zw = avec(b, r0 + 5);
    const size_t bytes = (size_t)b.nimg * sizeof(float2);
    double* lam_bar = b.dslots;
    double* dots = b.dslots + 1;   // [iters][d+1]
    PP_TRY_CUDA(cudaMemcpyAsync(Ybar, gout, bytes, cudaMemcpyDeviceToDevice, st));
    PP_TRY_CUDA(cudaMemsetAsync(Zbar, 0, bytes, st));
    PP_TRY_CUDA(cudaMemsetAsync(ahb_bar, 0, bytes, st));
    PP_TRY_CUDA(cudaMemsetAsync(b.dslots, 0, sizeof(double) * (1 + (size_t)iters * (d + 1)), st));
    for (int sg = (int)ncp - 1; sg >= 0; --sg) {
        const int k0 = sg * ce, k1 = std::min(iters, k0 + ce);
        // recompute the segment forward from its checkpoint, keeping z_k, g_k, w_k
        PP_TRY_CUDA(cudaMemcpyAsync(yw, avec(b, 1 + 2 * sg), bytes, cudaMemcpyDeviceToDevice, st));
        PP_TRY_CUDA(cudaMemcpyAsync(zw, avec(b, 2 + 2 * sg), bytes, cudaMemcpyDeviceToDevice, st));
        for (int k = k0; k < k1; ++k) {
            const int j = k - k0;
            PP_TRY_CUDA(cudaMemcpyAsync(avec(b, seg0 + 3 * j), zw, bytes, cudaMemcpyDeviceToDevice, st));
            PP_TRY(unrolled_step(b, c, d, lambda, k, zw, yw, avec(b, seg0 + 3 * j + 1),
                                 avec(b, seg0 + 3 * j + 2), st));
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const int j = k - k0;
            const float beta = (float)((double)k / (k + 3.0));
            PP_TRY(launch_batch_prox_vjp(b.dev, lambda, beta, avec(b, seg0 + 3 * j + 2), Ybar, Zbar,
                                         wbar, lam_bar, st));
            // v_0 = wbar, v_i = N_hat v_{i-1}, i = 1..d+1
            const float2* prev = wbar;
            for (int i = 1; i <= d + 1; ++i) {
                PP_TRY(launch_batch_normal(b.dev, prev, avec(b, v0 + i), 1.f, nullptr, 0.f, st));
                prev = avec(b, v0 + i);
            }
            const float2* gk = avec(b, seg0 + 3 * j + 1);
            for (int i = 0; i <= d; ++i)
                PP_TRY(launch_dot(i == 0 ? wbar : avec(b, v0 + i), gk, b.nimg, b.partials,
                                  b.dev.img.nblocks, dots + (size_t)k * (d + 1) + i, nullptr, st));
            // Zbar = wbar - sum_i c_i v_{i+1};  ahb_bar += sum_i c_i v_i
            LinComb za, ab;
            za.count = d + 2;
            za.v[0] = wbar; za.coef[0] = 1.f;
            ab.count = d + 1;
            for (int i = 0; i <= d; ++i) {
                za.v[i + 1] = avec(b, v0 + i + 1);
                za.coef[i + 1] = -(float)c[i];
                ab.v[i] = (i == 0) ? wbar : avec(b, v0 + i);
                ab.coef[i] = (float)c[i];
            }
            PP_TRY(launch_lincomb(za, Zbar, b.nimg, 0, st));
            PP_TRY(launch_lincomb(ab, ahb_bar, b.nimg, 1, st));
        }
    }
    // b_bar = A_s ahb_bar_s / sqrt(L_s)
    for (int s = 0; s < b.n; ++s)
        PP_TRY(forward_into(*b.sub[s], ahb_bar + b.img_off[s], grad_b + b.ksp_off[s], st));
    PP_TRY(launch_seg_scale(grad_b, grad_b, b.dev.ksp, nullptr, 0, b.dfac, 0, st));
    std::vector<double> h(1 + (size_t)iters * (d + 1));
    PP_TRY_CUDA(cudaMemcpyAsync(h.data(), b.dslots, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    *grad_lam = h[0];
    for (int i = 0; i <= d; ++i) {
        double acc = 0.0;
        for (int k = 0; k < iters; ++k) acc += h[1 + (size_t)k * (d + 1) + i];
        grad_c[i] = -acc;
    }
    return PP_OK;
}

}  // namespace pp

// ===========================================================================
// extern "C" entry points
// ===========================================================================
using namespace pp;

extern "C" {

const char* pp_last_error(void) { return g_last_error.c_str(); }

pp_status pp_poly_max_zp(const double* c, int d, double* m) {
    if (!c || !m || d < 0 || d > 16) {
        set_error("pp_poly_max_zp: need c != NULL, m != NULL, 0 <= d <= 16");
        return PP_ERR_INVALID_ARG;
    }
    // z p(z) on 4096 equal steps of [0, 1], then golden-section refinement
    // of the best bracket (z p(z) is a polynomial: one smooth maximum there)
    auto f = [&](double z) {
        double acc = 0.0;
        for (int i = d; i >= 0; --i) acc = acc * z + c[i];
        return z * acc;
    };
    const int n = 4096;
    int best = 0;
    double fb = f(0.0);
    for (int i = 1; i <= n; ++i) {
        const double v = f((double)i / n);
        if (v > fb) {
            fb = v;
            best = i;
        }
    }
    double a = std::max(0.0, (best - 1.0) / n), b = std::min(1.0, (best + 1.0) / n);
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    for (int it = 0; it < 80; ++it) {
        const double x1 = b - g * (b - a), x2 = a + g * (b - a);
        if (f(x1) < f(x2)) a = x1;
        else b = x2;
    }
    *m = std::max(fb, f(0.5 * (a + b)));
    if (!std::isfinite(*m)) {
        set_error("pp_poly_max_zp: non-finite value");
        return PP_ERR_NONFINITE;
    }
    return PP_OK;
}

pp_status pp_poly_coeffs_l2(int d, double* c) {
    if (!c || d < 0 || d > 8) {
        set_error("pp_poly_coeffs_l2: need 0 <= d <= 8 and c != NULL");
        return PP_ERR_INVALID_ARG;
    }
    // r(z) = 1 - z p(z) is the degree-(d+1) polynomial with r(0) = 1 of least
    // L2([0,1]) norm.  With the orthonormal shifted Legendre polynomials
    // Q_j(z) = sqrt(2j+1) P_j(2z-1) this is the normalised Christoffel-Darboux
    // kernel r(z) = sum_j Q_j(0) Q_j(z) / sum_j Q_j(0)^2, j = 0..m, m = d+1.
    // Since P_j(2z-1) = sum_k (-1)^(j+k) C(j,k) C(j+k,k) z^k and Q_j(0)^2 = 2j+1,
    //   [z^k] r = (-1)^k sum_{j=k..m} (2j+1) C(j,k) C(j+k,k) / (m+1)^2,
    // an exact integer ratio; c_i = -[z^(i+1)] r.
    const int m = d + 1;
    auto binom = [](int a, int b) {
        long long r = 1;
        for (int t = 1; t <= b; ++t) r = r * (a - b + t) / t;
        return r;
    };
    const double den = (double)((m + 1) * (m + 1));
    for (int i = 0; i <= d; ++i) {
        const int k = i + 1;
        long long S = 0;
        for (int j = k; j <= m; ++j) S += (long long)(2 * j + 1) * binom(j, k) * binom(j + k, k);
        c[i] = ((k + 1) % 2 == 0 ? 1.0 : -1.0) * (double)S / den;
    }
    return PP_OK;
}

// r_i = h_i - sum_j G_ij c_j with the products' rounding errors (fma) and the
// sum's (two-sum) carried in a second word: the residual of a Hankel system
// whose condition grows like that of the Hilbert matrix.
static double residual_dd(const double* G, const double* h, const double* c, int n, int i) {
    double hi = h[i], lo = 0.0;
    for (int j = 0; j < n; ++j) {
        const double p = G[i * n + j] * c[j];
        const double pe = std::fma(G[i * n + j], c[j], -p);
        const double s = hi - p;
        const double bb = s - hi;
        lo += ((hi - (s - bb)) + (-p - bb)) - pe;
        hi = s;
    }
    return hi + lo;
}

pp_status pp_poly_coeffs_wl2(int d, const double* moments, double* c) {
    if (!c || !moments || d < 0 || d > 8) {
        set_error("pp_poly_coeffs_wl2: need 0 <= d <= 8 and non-NULL moments, c");
        return PP_ERR_INVALID_ARG;
    }
    for (int k = 0; k <= 2 * d + 2; ++k)
        if (!std::isfinite(moments[k])) {
            set_error("pp_poly_coeffs_wl2: moment %d is not finite", k);
            return PP_ERR_INVALID_ARG;
        }
    // normal equations of int_0^1 w (1 - z p)^2: sum_j m_{i+j+2} c_j = m_{i+1}
    const int n = d + 1;
    double G[81], h[9], LU[81];
    int piv[9];
    for (int i = 0; i < n; ++i) {
        h[i] = moments[i + 1];
        for (int j = 0; j < n; ++j) G[i * n + j] = LU[i * n + j] = moments[i + j + 2];
    }
    double gmax = 0.0;
    for (int i = 0; i < n * n; ++i) gmax = std::max(gmax, std::fabs(G[i]));
    // LU with partial pivoting
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (std::fabs(LU[r * n + k]) > std::fabs(LU[p * n + k])) p = r;
        piv[k] = p;
        if (!(std::fabs(LU[p * n + k]) > 1e-15 * gmax)) {
            set_error("pp_poly_coeffs_wl2: the moments do not define a positive weight "
                      "(singular normal equations)");
            return PP_ERR_INVALID_ARG;
        }
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(LU[k * n + j], LU[p * n + j]);
        for (int r = k + 1; r < n; ++r) {
            LU[r * n + k] /= LU[k * n + k];
            for (int j = k + 1; j < n; ++j) LU[r * n + j] -= LU[r * n + k] * LU[k * n + j];
        }
    }
    auto lu_solve = [&](double* x) {
        for (int k = 0; k < n; ++k) std::swap(x[k], x[piv[k]]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) x[i] -= LU[i * n + j] * x[j];
        for (int i = n - 1; i >= 0; --i) {
            for (int j = i + 1; j < n; ++j) x[i] -= LU[i * n + j] * x[j];
            x[i] /= LU[i * n + i];
        }
    };
    for (int i = 0; i < n; ++i) c[i] = h[i];
    lu_solve(c);
    // iterative refinement with compensated residuals: each step multiplies
    // the error by about cond(G) * 2^-53, which stays below 1 up to d = 8 for
    // weights that are not extremely concentrated; stop once the correction
    // no longer changes c
    for (int it = 0; it < 60; ++it) {
        double r[9], dmax = 0.0, cmax = 0.0;
        for (int i = 0; i < n; ++i) r[i] = residual_dd(G, h, c, n, i);
        lu_solve(r);
        for (int i = 0; i < n; ++i) {
            c[i] += r[i];
            dmax = std::max(dmax, std::fabs(r[i]));
            cmax = std::max(cmax, std::fabs(c[i]));
        }
        if (!(dmax > 1e-17 * cmax)) break;
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(c[i])) {
            set_error("pp_poly_coeffs_wl2: non-finite coefficients");
            return PP_ERR_NONFINITE;
        }
    return PP_OK;
}

pp_status pp_poly_coeffs_cheb(int d, double mu, double* c) {
    if (!c || d < 0 || d > 8 || !(mu > 0.0 && mu < 1.0)) {
        set_error("pp_poly_coeffs_cheb: need 0 <= d <= 8, 0 < mu < 1, c != NULL");
        return PP_ERR_INVALID_ARG;
    }
    // T_k(a + b z) as monomial coefficients in z by T_{k+1} = 2 (a + b z) T_k - T_{k-1}
    const double a = (1.0 + mu) / (1.0 - mu), bz = -2.0 / (1.0 - mu);
    const int m = d + 1;
    double Tm1[10] = {0}, T0[10] = {0}, T1[10] = {0};
    T0[0] = 1.0;                         // T_0
    T1[0] = a; T1[1] = bz;               // T_1
    if (m == 1) {
        for (int i = 0; i < 10; ++i) Tm1[i] = T1[i];
    } else {
        double prev[10], cur[10];
        for (int i = 0; i < 10; ++i) { prev[i] = T0[i]; cur[i] = T1[i]; }
        for (int k = 1; k < m; ++k) {
            double next[10] = {0};
            for (int i = 0; i <= k; ++i) {
                next[i] += 2.0 * a * cur[i];
                next[i + 1] += 2.0 * bz * cur[i];
            }
            for (int i = 0; i < 10; ++i) next[i] -= prev[i];
            for (int i = 0; i < 10; ++i) { prev[i] = cur[i]; cur[i] = next[i]; }
        }
        for (int i = 0; i < 10; ++i) Tm1[i] = cur[i];
    }
    // r = T_m(a + b z) / T_m(a); T_m(a) is the constant term
    const double t0 = Tm1[0];
    for (int i = 0; i <= d; ++i) c[i] = -Tm1[i + 1] / t0;
    return PP_OK;
}

pp_status pp_plan_create(pp_plan** out, pp_dims dims, int coils, const pp_c64* sens,
                         const pp_sampling* s, uint64_t seed, int power_iters, pp_stream stream) {
    if (!out) {
        set_error("pp_plan_create: out is NULL");
        return PP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!sens || !s) {
        set_error("pp_plan_create: sens and sampling must be non-NULL");
        return PP_ERR_INVALID_ARG;
    }
    if ((uintptr_t)sens & 15) {
        set_error("pp_plan_create: sens must be 16-byte aligned");
        return PP_ERR_INVALID_ARG;
    }
    if (dims.ndim != 2 && dims.ndim != 3) {
        set_error("pp_plan_create: ndim must be 2 or 3");
        return PP_ERR_UNSUPPORTED;
    }
    const int nx = dims.n[0], ny = dims.n[1], nz = dims.ndim == 3 ? dims.n[2] : 1;
    if (nx < 4 || ny < 4 || nz < 1 || (dims.ndim == 3 && nz < 4) || nx > 512 || ny > 512 ||
        nz > 512) {
        set_error("pp_plan_create: image size out of range (4..512 per axis)");
        return PP_ERR_INVALID_ARG;
    }
    if ((nx % 4) || (ny % 4) || (dims.ndim == 3 && (nz % 4))) {
        set_error("pp_plan_create: every image axis must be a multiple of 4");
        return PP_ERR_UNSUPPORTED;
    }
    if (coils < 1 || coils > 64) {
        set_error("pp_plan_create: coils must be in 1..64");
        return PP_ERR_INVALID_ARG;
    }
    if (power_iters < 0 || power_iters > 100000) {
        set_error("pp_plan_create: power_iters out of range");
        return PP_ERR_INVALID_ARG;
    }
    if (s->kind == PP_CARTESIAN) {
        if (!s->mask) {
            set_error("pp_plan_create: Cartesian sampling needs a mask");
            return PP_ERR_INVALID_ARG;
        }
        if (!fft_len_ok(nx) || !fft_len_ok(ny) || (dims.ndim == 3 && !fft_len_ok(nz))) {
            set_error("pp_plan_create: FFT lengths need prime factors <= 5");
            return PP_ERR_UNSUPPORTED;
        }
    } else if (s->kind == PP_NONCARTESIAN || s->kind == PP_NONCARTESIAN_TOEPLITZ) {
        if (!s->traj) {
            set_error("pp_plan_create: non-Cartesian sampling needs a trajectory");
            return PP_ERR_INVALID_ARG;
        }
        if (dims.ndim != 2) {
            set_error("pp_plan_create: non-Cartesian plans are 2-D only");
            return PP_ERR_UNSUPPORTED;
        }
        if (s->kind == PP_NONCARTESIAN_TOEPLITZ && !toep_supported(nx, ny, coils)) {
            set_error("pp_plan_create: the Toeplitz normal operator needs coils <= 32 and "
                      "nx, ny in {64, 96, 128, 160, 192, 256}");
            return PP_ERR_UNSUPPORTED;
        }
    } else {
        set_error("pp_plan_create: unknown sampling kind %d", s->kind);
        return PP_ERR_INVALID_ARG;
    }
    static std::once_flag once;
    static pp_status cfg = PP_OK;
    std::call_once(once, [] { cfg = configure_kernels(); });
    if (cfg != PP_OK) return cfg;

    pp_plan* h = new pp_plan();
    Plan& p = h->impl;
    p.ndim = dims.ndim; p.nx = nx; p.ny = ny; p.nz = nz; p.C = coils;
    p.kind = s->kind == PP_NONCARTESIAN_TOEPLITZ ? PP_NONCARTESIAN : s->kind;
    p.toep = s->kind == PP_NONCARTESIAN_TOEPLITZ;
    p.nimg = (int64_t)nx * ny * nz;
    p.sens = reinterpret_cast<const float2*>(sens);
    cudaGetDevice(&p.dev);
    cudaStream_t st = (cudaStream_t)stream;
    pp_status rc = (s->kind == PP_CARTESIAN) ? build_cartesian(p, s->mask) : build_noncartesian(p, s);
    if (rc == PP_OK && s->kind == PP_CARTESIAN && p.ndim == 2) rc = prepare_cart4();
    if (rc == PP_OK) {
        const size_t n = (size_t)p.nimg;
        p.red_blocks = 2 * 152;
        if ((rc = alloc_n(p, &p.z, n)) == PP_OK && (rc = alloc_n(p, &p.y, n)) == PP_OK &&
            (rc = alloc_n(p, &p.g, n)) == PP_OK && (rc = alloc_n(p, &p.u, n)) == PP_OK &&
            (rc = alloc_n(p, &p.t, n)) == PP_OK && (rc = alloc_n(p, &p.ahb, n)) == PP_OK &&
            (rc = alloc_n(p, &p.v, n)) == PP_OK && (rc = alloc_n(p, &p.w3, n)) == PP_OK &&
            (rc = alloc_n(p, &p.red, (size_t)3 * p.red_blocks)) == PP_OK &&
            (rc = alloc_n(p, &p.scal, 8)) == PP_OK) {
            cudaError_t e = cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) rc = cuda_status(e, "cudaStreamCreate");
        }
    }
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    const TuneKey tkey = tune_key(p, s, dev_now);
    bool tuned = false;   // launch shapes taken from an earlier plan of the same geometry
    if (rc == PP_OK && p.kind == PP_CARTESIAN && p.ndim == 2 && !(tuned = tune_lookup(tkey, p)))
        rc = tune_cart2d(p, st);
    if (rc == PP_OK && p.kind == PP_CARTESIAN && p.ndim == 3) {
        p.c3cl_clusters = c3cl_prepare(p, 4);
        p.c3cl2_clusters = c3cl_prepare(p, 2);
        p.c3df_ctas = c3df_prepare(p, 0);
        p.c3df_ctas_hi = c3df_prepare(p, 1);
        p.c3df_ctas_tma = (p.c3df_ctas > 0 && c3df_make_tensor_map(p)) ? c3df_prepare(p, 2) : 0;
        p.c3df_ctas_tma1 = p.c3df_ctas_tma > 0 ? c3df_prepare(p, 3) : 0;
        if (p.c3df_ctas > 0) {
            // two phase slots for up to 8 coils per group; counters for 1
            p.c3df_w_elems = 2 * c3df_slot_elems(p, std::min(8, std::max(2, p.C)));
            p.c3df_cnt_ints = 0;
            for (int cgc = 1; cgc <= 8; ++cgc)
                p.c3df_cnt_ints = std::max(p.c3df_cnt_ints, c3df_counter_ints(p, cgc));
            if ((rc = alloc_n(p, &p.c3df_w, p.c3df_w_elems)) == PP_OK &&
                (rc = alloc_n(p, &p.c3df_cnt, p.c3df_cnt_ints)) == PP_OK)
                rc = cudaMemsetAsync(p.c3df_cnt, 0, sizeof(int) * p.c3df_cnt_ints, st) == cudaSuccess
                         ? PP_OK : cuda_status(cudaGetLastError(), "cudaMemsetAsync");
            p.c3df_cg = std::min(4, p.C);
        }
        if (rc == PP_OK && !(tuned = tune_lookup(tkey, p))) rc = tune_cart3d(p, st);
    }
    if (rc == PP_OK && p.kind == PP_NONCARTESIAN) rc = setup_ci(p, st);
    if (rc == PP_OK && p.toep) rc = setup_toeplitz(p, s, st);
    if (rc == PP_OK && p.kind == PP_NONCARTESIAN && !p.toep && !(tuned = tune_lookup(tkey, p)))
        rc = tune_noncartesian(p, st);
    if (rc == PP_OK && !tuned) tune_store(tkey, p);
    if (rc == PP_OK && power_iters > 0) rc = power_iteration(p, seed, power_iters, st);
    if (rc != PP_OK) {
        cudaStreamSynchronize(st);
        for (void* a : p.allocs) cudaFree(a);
        if (p.cap_stream) cudaStreamDestroy(p.cap_stream);
        delete h;
        return rc;
    }
    *out = h;
    return PP_OK;
}

pp_status pp_plan_destroy(pp_plan* plan) {
    if (!plan) return PP_OK;
    Plan& p = plan->impl;
    if (p.gexec) cudaGraphExecDestroy(p.gexec);
    if (p.cap_stream) cudaStreamDestroy(p.cap_stream);
    for (void* a : p.allocs) cudaFree(a);
    delete plan;
    return PP_OK;
}

pp_status pp_plan_scale(const pp_plan* plan, double* L) {
    if (!plan || !L) {
        set_error("pp_plan_scale: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    *L = plan->impl.L;
    return PP_OK;
}

pp_status pp_plan_set_scale(pp_plan* plan, double L) {
    if (!plan || !(L > 0.0) || !isfinite(L)) {
        set_error("pp_plan_set_scale: need a plan and a finite L > 0");
        return PP_ERR_INVALID_ARG;
    }
    if (plan->impl.L != L) {
        plan->impl.L = L;
        plan->impl.gkey.clear();   // captured graphs bake 1/L into their kernels
    }
    return PP_OK;
}

pp_status pp_plan_tuning(const pp_plan* plan, int* row_ifft_variant, int* stencil_kind,
                         int* stencil_coils) {
    if (!plan) {
        set_error("pp_plan_tuning: NULL plan");
        return PP_ERR_INVALID_ARG;
    }
    if (row_ifft_variant) {
        const Plan& p = plan->impl;
        if (p.kind == PP_CARTESIAN && p.ndim == 3)
            *row_ifft_variant = p.tune_c3 == 1 ? 16 : (p.tune_c3 == 2 ? -16 : (p.tune_c3 == 3 ? 3 : 1));
        else if (p.kind == PP_CARTESIAN)
            *row_ifft_variant = p.tune_c2;
        else
            *row_ifft_variant = p.tune_rows_adj_cl ? p.tune_rows_adj_cl : 1;
    }
    if (stencil_kind) {
        const Plan& p = plan->impl;
        *stencil_kind = (p.kind == PP_CARTESIAN && p.ndim == 3 && p.tune_c3 == 3) ? p.c3df_hi
                                                                                  : p.tune_stencil_kind;
    }
    if (stencil_coils) {
        const Plan& p = plan->impl;
        *stencil_coils = (p.kind == PP_CARTESIAN && p.ndim == 3 && p.tune_c3 == 3)
                             ? p.c3df_cg : (p.tune_stencil_cpc ? p.tune_stencil_cpc : 8);
    }
    return PP_OK;
}

pp_status pp_plan_set_tuning(pp_plan* plan, int row_ifft_variant, int stencil_kind, int stencil_coils) {
    if (!plan || !(row_ifft_variant == 1 || row_ifft_variant == 2 || row_ifft_variant == 4 ||
                   row_ifft_variant == -1 || row_ifft_variant == 8 || row_ifft_variant == 16 ||
                   row_ifft_variant == -16 || row_ifft_variant == 3) ||
        stencil_kind < 0 || stencil_kind > 9 || stencil_coils < 1 || stencil_coils > 64) {
        set_error("pp_plan_set_tuning: row variant must be 1, 2, 3, 4, 8, -1, 16 or -16; stencil "
                  "kind 0..9; stencil coils 1..64");
        return PP_ERR_INVALID_ARG;
    }
    Plan& p = plan->impl;
    if (row_ifft_variant == 3) {
        const int cgv = std::min(stencil_coils, std::max(1, p.C));   // the kernel's group size
        if (!(p.kind == PP_CARTESIAN && p.ndim == 3) || p.c3df_ctas <= 0 ||
            2 * c3df_slot_elems(p, cgv) > p.c3df_w_elems ||
            c3df_counter_ints(p, cgv) > p.c3df_cnt_ints) {
            set_error("pp_plan_set_tuning: row variant 3 (the 3-D dataflow operator) needs a 3-D "
                      "Cartesian plan with register-FFT lengths ny, nz and at most 8 coils per group");
            return PP_ERR_UNSUPPORTED;
        }
        if (stencil_kind < 0 || stencil_kind > 5 || ((stencil_kind == 1 || stencil_kind == 5) && p.c3df_ctas_hi <= 0) ||
            (stencil_kind == 2 && p.c3df_ctas_tma <= 0) || (stencil_kind == 3 && p.c3df_ctas_tma1 <= 0)) {
            set_error("pp_plan_set_tuning: the 3-D dataflow operator takes stencil kind 0 (two "
                      "blocks per SM), 1 (three), 2 (map tiles staged by TMA), 3 (staged by TMA "
                      "into one buffer, three blocks per SM), 4 or 5 (0 or 1 with two z planes "
                      "per y-FFT item and two line units per z item)");
            return PP_ERR_UNSUPPORTED;
        }
        p.tune_c3 = 3;
        p.c3df_cg = stencil_coils;
        p.c3df_hi = stencil_kind;
        p.gkey.clear();
        return PP_OK;
    }
    if ((row_ifft_variant == 16 && p.c3cl_clusters <= 0) ||
        (row_ifft_variant == -16 && p.c3cl2_clusters <= 0)) {
        set_error("pp_plan_set_tuning: the one-kernel cluster operator needs a 3-D Cartesian plan "
                  "with nz = 128, ny in {128, 192, 256} and a device that fits 16-CTA clusters");
        return PP_ERR_UNSUPPORTED;
    }
    if (row_ifft_variant == 8 && !(p.kind == PP_CARTESIAN && p.ndim == 2)) {
        set_error("pp_plan_set_tuning: row variant 8 (coils split over 8-CTA clusters) applies to "
                  "2-D Cartesian plans");
        return PP_ERR_UNSUPPORTED;
    }
    if (p.kind == PP_CARTESIAN && p.ndim == 3)
        p.tune_c3 = row_ifft_variant == 16 ? 1 : (row_ifft_variant == -16 ? 2 : 0);
    if (p.kind == PP_CARTESIAN && p.ndim == 2) {
        if (row_ifft_variant == -1 || row_ifft_variant == 16 || row_ifft_variant == -16) {
            set_error("pp_plan_set_tuning: 2-D Cartesian plans take row variant 1, 2, 4 or 8");
            return PP_ERR_UNSUPPORTED;
        }
        p.tune_c2 = row_ifft_variant;
        p.gkey.clear();
        return PP_OK;
    }
    if (row_ifft_variant == -1 && (p.kind != PP_NONCARTESIAN || !fft4_n2(p.G_x))) {
        set_error("pp_plan_set_tuning: the split row IFFT needs a non-Cartesian plan with a "
                  "register-FFT grid length");
        return PP_ERR_UNSUPPORTED;
    }
    if (stencil_kind >= 2 && (p.kind != PP_NONCARTESIAN || p.stencil_rb_grid[0] == 0 ||
                              (stencil_kind <= 5 && p.stencil_rb_grid[stencil_kind - 2] == 0))) {
        set_error("pp_plan_set_tuning: register-blocked stencil kinds need a non-Cartesian plan "
                  "whose 49 weight planes hold fewer than 2^31 values");
        return PP_ERR_UNSUPPORTED;
    }
    if (stencil_kind >= 7 && !p.ci_sens) {
        set_error("pp_plan_set_tuning: the coil-innermost pipeline needs at most 32 coils and "
                  "register-FFT grid lengths");
        return PP_ERR_UNSUPPORTED;
    }
    p.tune_rows_adj_cl = row_ifft_variant;
    p.tune_stencil_kind = stencil_kind;
    p.tune_stencil_cpc = stencil_coils;
    p.gkey.clear();
    return PP_OK;
}

pp_status pp_plan_mu(pp_plan* plan, int iters, uint64_t seed, double* mu, pp_stream stream) {
    if (!plan || !mu || iters < 1 || iters > 1000000) {
        set_error("pp_plan_mu: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    return mu_iteration(plan->impl, seed, iters, mu, (cudaStream_t)stream);
}

pp_status pp_prox_llr(pp_dims dims, int T, int block, const int* shift, float lambda,
                      const pp_c64* in, pp_c64* out, pp_stream stream) {
    if (!in || !out || !(lambda >= 0.f) || !isfinite(lambda) || (dims.ndim != 2 && dims.ndim != 3)) {
        set_error("pp_prox_llr: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    const int nz = dims.ndim == 3 ? dims.n[2] : 1;
    if (T < 1 || T > 8 || !(block == 4 || block == 8 || (block == 16 && dims.ndim == 2)) ||
        dims.n[0] < 1 || dims.n[1] < 1 || nz < 1 || dims.n[0] % block || dims.n[1] % block ||
        (dims.ndim == 3 && nz % block)) {
        set_error("pp_prox_llr: need 1 <= T <= 8, block 4 or 8 (16 in 2-D) dividing every axis");
        return PP_ERR_UNSUPPORTED;
    }
    return launch_prox_llr(dims.ndim, dims.n[0], dims.n[1], nz, T, block, shift, lambda,
                           reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                           (cudaStream_t)stream);
}

pp_status pp_selftest_wait(int64_t limit_ns, pp_stream stream) {
    if (limit_ns < 1000000 || limit_ns > 1000000000) {
        set_error("pp_selftest_wait: limit must be 1 ms .. 1 s");
        return PP_ERR_INVALID_ARG;
    }
    return selftest_wait((long long)limit_ns, (cudaStream_t)stream);
}

pp_status pp_plan_sizes(const pp_plan* plan, int64_t* image_elems, int64_t* kspace_elems) {
    if (!plan) {
        set_error("pp_plan_sizes: NULL plan");
        return PP_ERR_INVALID_ARG;
    }
    if (image_elems) *image_elems = plan->impl.nimg;
    if (kspace_elems) *kspace_elems = plan->impl.nksp;
    return PP_OK;
}

pp_status pp_forward_apply(const pp_plan* plan, const pp_c64* x, pp_c64* y, pp_stream stream) {
    if (!plan || !x || !y) {
        set_error("pp_forward_apply: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    return forward_into(plan->impl, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                        (cudaStream_t)stream);
}

pp_status pp_adjoint_apply(const pp_plan* plan, const pp_c64* y, pp_c64* x, pp_stream stream) {
    if (!plan || !x || !y) {
        set_error("pp_adjoint_apply: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    return adjoint_into(plan->impl, reinterpret_cast<const float2*>(y), reinterpret_cast<float2*>(x),
                        (cudaStream_t)stream);
}

pp_status pp_normal_apply(const pp_plan* plan, const pp_c64* x, pp_c64* y, pp_stream stream) {
    if (!plan || !x || !y || (const void*)x == (const void*)y) {
        set_error("pp_normal_apply: NULL or aliased argument");
        return PP_ERR_INVALID_ARG;
    }
    const Plan& p = plan->impl;
    return normal_into(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                       (float)(1.0 / p.L), nullptr, 0.f, (cudaStream_t)stream);
}

pp_status pp_poly_apply(const pp_plan* plan, const double* c, int d, const pp_c64* v, pp_c64* out,
                        pp_stream stream) {
    if (!plan || !c || !v || !out || d < 0 || d > 16 || (const void*)v == (const void*)out) {
        set_error("pp_poly_apply: bad argument (NULL, aliased, or d outside 0..16)");
        return PP_ERR_INVALID_ARG;
    }
    Plan& p = const_cast<Plan&>(plan->impl);
    return horner_into(p, c, d, reinterpret_cast<const float2*>(v), reinterpret_cast<float2*>(out),
                       p.t, p.w3, (cudaStream_t)stream);
}

pp_status pp_prox_l1_haar(pp_dims dims, int levels, float lambda, const pp_c64* in, pp_c64* out,
                          pp_stream stream) {
    if (!in || !out || (dims.ndim != 2 && dims.ndim != 3) || !(lambda >= 0.f) || !isfinite(lambda)) {
        set_error("pp_prox_l1_haar: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    if (levels < 1 || levels > 2) {
        set_error("pp_prox_l1_haar: levels must be 1 or 2");
        return PP_ERR_UNSUPPORTED;
    }
    const int ts = 1 << levels;
    const int nx = dims.n[0], ny = dims.n[1], nz = dims.ndim == 3 ? dims.n[2] : 1;
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx % ts || ny % ts || (dims.ndim == 3 && nz % ts)) {
        set_error("pp_prox_l1_haar: every axis must be a positive multiple of 2^levels");
        return PP_ERR_UNSUPPORTED;
    }
    return launch_prox(dims.ndim, nx, ny, nz, levels, lambda, reinterpret_cast<const float2*>(in),
                       reinterpret_cast<float2*>(out), (cudaStream_t)stream);
}

pp_status pp_prox_l1_db4(pp_dims dims, int levels, float lambda, const pp_c64* in, pp_c64* out,
                         pp_stream stream) {
    if (!in || !out || (dims.ndim != 2 && dims.ndim != 3) || !(lambda >= 0.f) || !isfinite(lambda)) {
        set_error("pp_prox_l1_db4: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    if (!db4_supported(dims.ndim, dims.n[0], dims.n[1], levels)) {
        set_error("pp_prox_l1_db4: 2-D only, levels 1..4, axes <= 512 and multiples of 2^levels");
        return PP_ERR_UNSUPPORTED;
    }
    return launch_prox_db4(dims.n[0], dims.n[1], levels, lambda, reinterpret_cast<const float2*>(in),
                           reinterpret_cast<float2*>(out), (cudaStream_t)stream);
}

// After a synchronising solve: a NaN or infinite ||b||^2 (first slice's for
// a batch) or history entry means the input held a non-finite value.
static pp_status check_history(const char* who, double bn2, const double* h, int iters) {
    bool ok = std::isfinite(bn2);
    for (int i = 0; ok && i < 3 * iters; ++i) ok = std::isfinite(h[i]);
    if (!ok) {
        set_error("%s: non-finite value in b (||b||^2 = %g) or in the iterates", who, bn2);
        return PP_ERR_NONFINITE;
    }
    return PP_OK;
}

// info->safe_scale: c divided by max_{z in [0, 1]} z p(z), in buf
static pp_status safe_coeffs(const pp_solve_info* info, const double*& c, int d, std::vector<double>& buf) {
    if (!info || !info->safe_scale || !c) return PP_OK;
    double m = 0.0;
    PP_TRY(pp_poly_max_zp(c, d, &m));
    if (!(m > 0.0)) {
        set_error("safe_scale: max of z p(z) on [0, 1] is not positive");
        return PP_ERR_INVALID_ARG;
    }
    buf.assign(c, c + d + 1);
    for (double& v : buf) v /= m;
    c = buf.data();
    return PP_OK;
}

pp_status pp_fista_solve(pp_plan* plan, const pp_c64* b, float lambda, int iters, const double* c,
                         int d, pp_c64* x_out, pp_solve_info* info, pp_stream stream) {
    if (!plan || !b || !x_out || iters < 0 || iters > 1000000 || !(lambda >= 0.f) ||
        !isfinite(lambda) || d < 0 || d > 16 || (!c && d != 0)) {
        set_error("pp_fista_solve: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    Plan& p = plan->impl;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> c_safe;
    PP_TRY(safe_coeffs(info, c, d, c_safe));
    const int levels = (info && info->levels) ? info->levels : 2;
    const int wavelet = info ? info->wavelet : 0;
    if (wavelet != 0 && wavelet != 1) {
        set_error("pp_fista_solve: wavelet must be 0 (Haar) or 1 (Daubechies-4)");
        return PP_ERR_INVALID_ARG;
    }
    if (wavelet == 1 && !db4_supported(p.ndim, p.nx, p.ny, levels)) {
        set_error("pp_fista_solve: the Daubechies-4 prox is 2-D with levels 1..4 and axes "
                  "multiples of 2^levels");
        return PP_ERR_UNSUPPORTED;
    }
    if (wavelet == 0 && (levels < 1 || levels > 2 || p.nx % (1 << levels) || p.ny % (1 << levels) ||
                         (p.ndim == 3 && p.nz % (1 << levels)))) {
        set_error("pp_fista_solve: unsupported Haar levels");
        return PP_ERR_UNSUPPORTED;
    }
    const bool hist = info && info->history;
    const bool momentum = !(info && info->no_momentum);
    const float2* ref = info ? reinterpret_cast<const float2*>(info->ref) : nullptr;
    const int64_t n = p.nimg;
    const int64_t launches0 = g_launches;
    // A_hat^H b_hat = A^H b / (sqrt(L) ||b||)
    PP_TRY(launch_norm2(reinterpret_cast<const float2*>(b), p.nksp, p.red, p.red_blocks, p.scal + 0, st));
    PP_TRY(adjoint_into(p, reinterpret_cast<const float2*>(b), p.ahb, st));
    PP_TRY(launch_scale_by_rnorm(p.ahb, p.ahb, n, p.scal + 0, 1.0 / sqrt(p.L), 1, st));
    PP_TRY_CUDA(cudaMemsetAsync(p.y, 0, n * sizeof(float2), st));
    PP_TRY_CUDA(cudaMemsetAsync(p.z, 0, n * sizeof(float2), st));
    if (hist) {
        if (p.hist_cap < iters) {
            if (p.hist) {
                cudaStreamSynchronize(st);
                cudaFree(p.hist);
                p.allocs.erase(std::remove(p.allocs.begin(), p.allocs.end(), (void*)p.hist), p.allocs.end());
                p.hist = nullptr;
            }
            PP_TRY(alloc_n(p, &p.hist, (size_t)3 * std::max(iters, 1)));
            p.hist_cap = iters;
            p.gkey.clear();
        }
        PP_TRY_CUDA(cudaMemsetAsync(p.hist, 0, sizeof(double) * 3 * std::max(iters, 1), st));
    }
    if (iters > 0) {
        std::vector<double> key = {0.0 /* normalised solve */, (double)iters, (double)d,
                                   (double)lambda, (double)levels, hist ? 1.0 : 0.0, c ? 1.0 : 0.0, p.L,
                                   (double)(uintptr_t)p.hist, (double)(uintptr_t)ref,
                                   momentum ? 1.0 : 0.0, (double)wavelet};
        if (c)
            for (int i = 0; i <= d; ++i) key.push_back(c[i]);
        if (!p.gexec || key != p.gkey) {
            if (p.gexec) {
                cudaGraphExecDestroy(p.gexec);
                p.gexec = nullptr;
            }
            p.gkey.clear();
            cudaGraph_t graph = nullptr;
            PP_TRY_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = g_launches;
            pp_status rc = fista_iterations(p, lambda, iters, c, d, levels, hist, ref, momentum,
                                            wavelet, p.cap_stream);
            cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
            p.graph_kernels = g_launches - before;
            g_launches = before;
            if (rc != PP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&p.gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                p.gexec = nullptr;
                return cuda_status(e, "cudaGraphInstantiate");
            }
            p.gkey = key;
        }
        PP_TRY_CUDA(cudaGraphLaunch(p.gexec, st));
    }
    float2* xo = reinterpret_cast<float2*>(x_out);
    if (info && info->rescale)
        PP_TRY(launch_scale_by_rnorm(p.y, xo, n, p.scal + 0, 1.0 / sqrt(p.L), 0, st));
    else
        PP_TRY_CUDA(cudaMemcpyAsync(xo, p.y, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (info) {
        info->L = p.L;
        info->launches = (g_launches - launches0) + (iters > 0 ? p.graph_kernels : 0);
        if (hist) {
            double bn2 = 0.0;
            PP_TRY_CUDA(cudaMemcpyAsync(&bn2, p.scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaMemcpyAsync(info->history, p.hist, sizeof(double) * 3 * iters,
                                        cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaStreamSynchronize(st));
            info->bnorm = sqrt(bn2);
            PP_TRY(c3df_check(p, st));
            PP_TRY(check_history("pp_fista_solve", bn2, info->history, iters));
        }
    }
    return PP_OK;
}

pp_status pp_fista_solve_prox(pp_plan* plan, const pp_c64* b, const pp_c64* v, double sigma,
                              float lambda, int iters, const double* c, int d, pp_c64* x_out,
                              pp_solve_info* info, pp_stream stream) {
    if (!plan || !x_out || iters < 0 || iters > 1000000 || !(lambda >= 0.f) || !isfinite(lambda) ||
        !(sigma >= 0.0) || !isfinite(sigma) || d < 0 || d > 16 || (!c && d != 0)) {
        set_error("pp_fista_solve_prox: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    Plan& p = plan->impl;
    cudaStream_t st = (cudaStream_t)stream;
    const int levels = (info && info->levels) ? info->levels : 2;
    const int wavelet = info ? info->wavelet : 0;
    if (wavelet != 0 && wavelet != 1) {
        set_error("pp_fista_solve_prox: wavelet must be 0 (Haar) or 1 (Daubechies-4)");
        return PP_ERR_INVALID_ARG;
    }
    if ((wavelet == 1 && !db4_supported(p.ndim, p.nx, p.ny, levels)) ||
        (wavelet == 0 && (levels < 1 || levels > 2 || p.nx % (1 << levels) || p.ny % (1 << levels) ||
                          (p.ndim == 3 && p.nz % (1 << levels))))) {
        set_error("pp_fista_solve_prox: unsupported wavelet levels for this image");
        return PP_ERR_UNSUPPORTED;
    }
    const bool hist = info && info->history;
    const bool momentum = !(info && info->no_momentum);
    const float2* ref = info ? reinterpret_cast<const float2*>(info->ref) : nullptr;
    const int64_t n = p.nimg;
    const int64_t launches0 = g_launches;
    // L' = L + sigma; the iteration runs on N_hat' = a N_hat + b I with
    // a = L/L', b = sigma/L', gradient constant rhs = (A^H b + sigma v)/L'
    // and threshold lambda/L'; p(N_hat') = q(N_hat) with
    // q_j = sum_{i >= j} c_i C(i, j) a^j b^(i-j) (binomial expansion, FP64)
    const double Lp = p.L + sigma, sa = p.L / Lp, sb = sigma / Lp;
    std::vector<double> q;
    if (c) {
        q.assign(d + 1, 0.0);
        std::vector<double> binom(d + 1, 0.0);
        for (int i = 0; i <= d; ++i) {
            // binom[j] = C(i, j), row i of Pascal's triangle
            for (int j = i; j >= 1; --j) binom[j] += binom[j - 1];
            binom[0] = 1.0;
            for (int j = 0; j <= i; ++j) q[j] += c[i] * binom[j] * std::pow(sa, j) * std::pow(sb, i - j);
        }
    }
    if (b) {
        PP_TRY(launch_norm2(reinterpret_cast<const float2*>(b), p.nksp, p.red, p.red_blocks, p.scal + 0, st));
        PP_TRY(adjoint_into(p, reinterpret_cast<const float2*>(b), p.ahb, st));
        PP_TRY(launch_axpby(p.ahb, (float)(1.0 / Lp), reinterpret_cast<const float2*>(v),
                            (float)(sigma / Lp), p.ahb, n, st));
    } else if (v) {
        PP_TRY(launch_axpby(reinterpret_cast<const float2*>(v), (float)(sigma / Lp), nullptr, 0.f, p.ahb,
                            n, st));
    } else {
        PP_TRY_CUDA(cudaMemsetAsync(p.ahb, 0, n * sizeof(float2), st));
    }
    if (!b) PP_TRY_CUDA(cudaMemsetAsync(p.scal, 0, sizeof(double), st));
    PP_TRY_CUDA(cudaMemsetAsync(p.y, 0, n * sizeof(float2), st));
    PP_TRY_CUDA(cudaMemsetAsync(p.z, 0, n * sizeof(float2), st));
    if (hist) {
        if (p.hist_cap < iters) {
            if (p.hist) {
                cudaStreamSynchronize(st);
                cudaFree(p.hist);
                p.allocs.erase(std::remove(p.allocs.begin(), p.allocs.end(), (void*)p.hist), p.allocs.end());
                p.hist = nullptr;
            }
            PP_TRY(alloc_n(p, &p.hist, (size_t)3 * std::max(iters, 1)));
            p.hist_cap = iters;
            p.gkey.clear();
        }
        PP_TRY_CUDA(cudaMemsetAsync(p.hist, 0, sizeof(double) * 3 * std::max(iters, 1), st));
    }
    Shift sh;
    sh.on = true;
    sh.a = (float)sa;
    sh.b = (float)sb;
    const float lam_hat = (float)(lambda / Lp);
    if (iters > 0) {
        // the graph cache is shared with pp_fista_solve: the key tells the two apart
        std::vector<double> key = {1.0 /* proximal subproblem */, (double)iters, (double)d,
                                   (double)lam_hat, (double)levels, hist ? 1.0 : 0.0, c ? 1.0 : 0.0,
                                   p.L, (double)(uintptr_t)p.hist, (double)(uintptr_t)ref,
                                   momentum ? 1.0 : 0.0, (double)wavelet, sa, sb};
        for (double qj : q) key.push_back(qj);
        if (!p.gexec || key != p.gkey) {
            if (p.gexec) {
                cudaGraphExecDestroy(p.gexec);
                p.gexec = nullptr;
            }
            p.gkey.clear();
            cudaGraph_t graph = nullptr;
            PP_TRY_CUDA(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = g_launches;
            pp_status rc = fista_iterations(p, lam_hat, iters, c ? q.data() : nullptr, d, levels, hist,
                                            ref, momentum, wavelet, p.cap_stream, sh);
            cudaError_t e = cudaStreamEndCapture(p.cap_stream, &graph);
            p.graph_kernels = g_launches - before;
            g_launches = before;
            if (rc != PP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&p.gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                p.gexec = nullptr;
                return cuda_status(e, "cudaGraphInstantiate");
            }
            p.gkey = key;
        }
        PP_TRY_CUDA(cudaGraphLaunch(p.gexec, st));
    }
    PP_TRY_CUDA(cudaMemcpyAsync(x_out, p.y, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (info) {
        info->L = p.L;
        info->launches = (g_launches - launches0) + (iters > 0 ? p.graph_kernels : 0);
        if (hist) {
            double bn2 = 0.0;
            PP_TRY_CUDA(cudaMemcpyAsync(&bn2, p.scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaMemcpyAsync(info->history, p.hist, sizeof(double) * 3 * iters,
                                        cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaStreamSynchronize(st));
            info->bnorm = sqrt(bn2);
            PP_TRY(c3df_check(p, st));
            PP_TRY(check_history("pp_fista_solve_prox", bn2, info->history, iters));
        }
    }
    return PP_OK;
}

pp_status pp_profile_normal(const pp_plan* plan, const pp_c64* x, pp_c64* y, int reps,
                            int max_stages, char* names, double* ms, int* nstages,
                            pp_stream stream) {
    if (!plan || !x || !y || reps < 1 || max_stages < 1 || !names || !ms || !nstages ||
        (const void*)x == (const void*)y) {
        set_error("pp_profile_normal: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    const Plan& p = plan->impl;
    cudaStream_t st = (cudaStream_t)stream;
    Profiler prof;
    prof.st = st;
    cudaEvent_t start;
    PP_TRY_CUDA(cudaEventCreate(&start));
    PP_TRY_CUDA(cudaEventRecord(start, st));
    g_profiler = &prof;
    pp_status rc = PP_OK;
    for (int r = 0; r < reps && rc == PP_OK; ++r)
        rc = normal_into(p, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                         (float)(1.0 / p.L), nullptr, 0.f, st);
    g_profiler = nullptr;
    cudaError_t e = cudaStreamSynchronize(st);
    std::vector<std::string> uniq;
    std::vector<double> tot;
    if (rc == PP_OK && e == cudaSuccess) {
        cudaEvent_t prev = start;
        for (size_t i = 0; i < prof.events.size(); ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, prev, prof.events[i]);
            prev = prof.events[i];
            size_t j = std::find(uniq.begin(), uniq.end(), prof.names[i]) - uniq.begin();
            if (j == uniq.size()) {
                uniq.push_back(prof.names[i]);
                tot.push_back(0.0);
            }
            tot[j] += t;
        }
    }
    for (cudaEvent_t ev : prof.events) cudaEventDestroy(ev);
    cudaEventDestroy(start);
    if (rc != PP_OK) return rc;
    if (e != cudaSuccess) return cuda_status(e, "pp_profile_normal sync");
    const int ns = std::min((int)uniq.size(), max_stages);
    for (int i = 0; i < ns; ++i) {
        strncpy(names + 48 * i, uniq[i].c_str(), 47);
        names[48 * i + 47] = 0;
        ms[i] = tot[i] / reps;
    }
    *nstages = ns;
    return PP_OK;
}

struct pp_batch {
    Batch impl;
};

pp_status pp_batch_create(pp_batch** out, int nslices, const pp_dims* dims, const int* coils,
                          const pp_c64* const* sens, const uint8_t* const* masks, uint64_t seed,
                          int power_iters, pp_stream stream) {
    if (!out) {
        set_error("pp_batch_create: out is NULL");
        return PP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (nslices < 1 || nslices > 4096 || !dims || !coils || !sens || !masks || power_iters < 0) {
        set_error("pp_batch_create: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    for (int s = 0; s < nslices; ++s) {
        const pp_dims& d = dims[s];
        if (d.ndim != 2) {
            set_error("pp_batch_create: slice %d is not 2-D", s);
            return PP_ERR_UNSUPPORTED;
        }
        const int nx = d.n[0], ny = d.n[1];
        if (nx < 4 || ny < 4 || nx > 512 || ny > 512 || (nx % 4) || (ny % 4) || coils[s] < 1 ||
            coils[s] > 64 || !sens[s] || ((uintptr_t)sens[s] & 15) || !masks[s]) {
            set_error("pp_batch_create: slice %d has a bad size, coil count or pointer", s);
            return PP_ERR_INVALID_ARG;
        }
        if (!fft_len_ok(nx) || !fft_len_ok(ny)) {
            set_error("pp_batch_create: slice %d FFT length has a prime factor above 5", s);
            return PP_ERR_UNSUPPORTED;
        }
    }
    static std::once_flag once;
    static pp_status cfg = PP_OK;
    std::call_once(once, [] {
        cfg = configure_kernels();
        if (cfg == PP_OK) cfg = configure_batch_kernels();
    });
    if (cfg != PP_OK) return cfg;
    cudaStream_t st = (cudaStream_t)stream;
    pp_batch* h = new pp_batch();
    Batch& b = h->impl;
    b.n = nslices;
    b.img_off.assign(nslices + 1, 0);
    b.ksp_off.assign(nslices + 1, 0);
    b.tile_off.assign(nslices + 1, 0);
    b.L.assign(nslices, 1.0);
    b.hdesc.resize(nslices);
    pp_status rc = PP_OK;
    size_t wk_max = 0;
    for (int s = 0; s < nslices && rc == PP_OK; ++s) {
        Plan* p = new Plan();
        b.sub.push_back(p);
        p->ndim = 2; p->nx = dims[s].n[0]; p->ny = dims[s].n[1]; p->nz = 1; p->C = coils[s];
        p->kind = PP_CARTESIAN;
        p->nimg = (int64_t)p->nx * p->ny;
        p->sens = reinterpret_cast<const float2*>(sens[s]);
        p->external_wk = true;
        rc = build_cartesian(*p, masks[s]);
        if (rc != PP_OK) break;
        wk_max = std::max(wk_max, (size_t)p->C * p->nimg);
        b.img_off[s + 1] = b.img_off[s] + p->nimg;
        b.ksp_off[s + 1] = b.ksp_off[s] + p->nksp;
        b.tile_off[s + 1] = b.tile_off[s] + p->nimg / 16;
        SliceDesc& d = b.hdesc[s];
        d.fd = p->fy.d; d.tw = p->fy.tw; d.sens = p->sens; d.mask_fo = p->mask_fo;
        d.ny = p->ny; d.nx = p->nx; d.C = p->C; d.n2 = fft4_n2(p->ny); d.img_off = b.img_off[s];
        d.invL = 1.f; d.pad1 = 0.f;
        b.dev.ny_max = std::max(b.dev.ny_max, p->ny);
    }
    b.nimg = b.img_off[nslices];
    b.nksp = b.ksp_off[nslices];
    if (rc == PP_OK) rc = balloc(b, &b.wk, wk_max);
    if (rc == PP_OK)
        for (Plan* p : b.sub) p->wk_a = b.wk;
    const size_t n = (size_t)b.nimg;
    if (rc == PP_OK && (rc = balloc(b, &b.z, n)) == PP_OK && (rc = balloc(b, &b.y, n)) == PP_OK &&
        (rc = balloc(b, &b.g, n)) == PP_OK && (rc = balloc(b, &b.u, n)) == PP_OK &&
        (rc = balloc(b, &b.t, n)) == PP_OK && (rc = balloc(b, &b.ahb, n)) == PP_OK &&
        (rc = balloc(b, &b.v, n)) == PP_OK && (rc = balloc(b, &b.w3, n)) == PP_OK &&
        (rc = balloc(b, &b.scal, (size_t)4 * nslices)) == PP_OK &&
        (rc = balloc(b, &b.dfac, (size_t)nslices)) == PP_OK &&
        (rc = balloc(b, &b.dev.descs, (size_t)nslices)) == PP_OK &&
        (rc = make_segments(b, b.dev.img, b.img_off, (int64_t)kThreads * 8, 64)) == PP_OK &&
        (rc = make_segments(b, b.dev.ksp, b.ksp_off, (int64_t)kThreads * 8, 64)) == PP_OK &&
        (rc = make_segments(b, b.dev.tiles, b.tile_off, (int64_t)kThreads, 1 << 30)) == PP_OK) {
        const int nb = std::max(b.dev.img.nblocks, b.dev.ksp.nblocks);
        rc = balloc(b, &b.partials, (size_t)3 * nb);
    }
    if (rc == PP_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_status(e, "cudaStreamCreate");
    }
    if (rc == PP_OK) rc = upload_descs(b);
    if (rc == PP_OK) {
        cudaError_t e = cudaMemsetAsync(b.v, 0, n * sizeof(float2), st);
        if (e != cudaSuccess) rc = cuda_status(e, "cudaMemsetAsync");
    }
    if (rc == PP_OK) {
        // a batch of one slice length can run the uniform-length kernel
        int un2 = b.hdesc.empty() ? 0 : b.hdesc[0].n2;
        for (const SliceDesc& d : b.hdesc)
            if (d.n2 != un2) un2 = 0;
        b.dev.ugrid = un2 ? batch4u_grid(un2) : 0;
        b.uni_n2 = b.dev.ugrid > 0 ? un2 : 0;
    }
    if (rc == PP_OK) rc = autotune(b, st);
    if (rc == PP_OK && power_iters > 0) rc = batch_power_iteration(b, seed, power_iters, st);
    if (rc != PP_OK) {
        cudaStreamSynchronize(st);
        if (b.gexec) cudaGraphExecDestroy(b.gexec);
        if (b.cap_stream) cudaStreamDestroy(b.cap_stream);
        for (Plan* p : b.sub) {
            for (void* a : p->allocs) cudaFree(a);
            delete p;
        }
        for (void* a : b.allocs) cudaFree(a);
        delete h;
        return rc;
    }
    *out = h;
    return PP_OK;
}

pp_status pp_batch_destroy(pp_batch* batch) {
    if (!batch) return PP_OK;
    Batch& b = batch->impl;
    if (b.gexec) cudaGraphExecDestroy(b.gexec);
    if (b.cap_stream) cudaStreamDestroy(b.cap_stream);
    for (Plan* p : b.sub) {
        for (void* a : p->allocs) cudaFree(a);
        delete p;
    }
    for (void* a : b.allocs) cudaFree(a);
    delete batch;
    return PP_OK;
}

pp_status pp_batch_offsets(const pp_batch* batch, int64_t* image_off, int64_t* kspace_off) {
    if (!batch) {
        set_error("pp_batch_offsets: NULL batch");
        return PP_ERR_INVALID_ARG;
    }
    const Batch& b = batch->impl;
    for (int s = 0; s <= b.n; ++s) {
        if (image_off) image_off[s] = b.img_off[s];
        if (kspace_off) kspace_off[s] = b.ksp_off[s];
    }
    return PP_OK;
}

pp_status pp_batch_scales(const pp_batch* batch, double* L) {
    if (!batch || !L) {
        set_error("pp_batch_scales: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    for (int s = 0; s < batch->impl.n; ++s) L[s] = batch->impl.L[s];
    return PP_OK;
}

pp_status pp_batch_set_scales(pp_batch* batch, const double* L) {
    if (!batch || !L) {
        set_error("pp_batch_set_scales: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    Batch& b = batch->impl;
    for (int s = 0; s < b.n; ++s)
        if (!(L[s] > 0.0) || !isfinite(L[s])) {
            set_error("pp_batch_set_scales: L[%d] must be finite and > 0", s);
            return PP_ERR_INVALID_ARG;
        }
    for (int s = 0; s < b.n; ++s) {
        b.L[s] = L[s];
        b.sub[s]->L = L[s];
    }
    b.tape_key.clear();   // checkpoints taken under the old L_s are stale
    return upload_descs(b);
}

pp_status pp_batch_tile(const pp_batch* batch, int* cols_per_cta, int* persistent_ctas) {
    if (!batch) {
        set_error("pp_batch_tile: NULL batch");
        return PP_ERR_INVALID_ARG;
    }
    if (cols_per_cta)
        *cols_per_cta = batch->impl.dev.fast4 ? -8 * batch->impl.dev.cl : 1 << batch->impl.dev.lgt;
    if (persistent_ctas) *persistent_ctas = batch->impl.dev.grid;
    return PP_OK;
}

pp_status pp_batch_set_tile(pp_batch* batch, int cols_per_cta) {
    if (!batch) {
        set_error("pp_batch_set_tile: NULL batch");
        return PP_ERR_INVALID_ARG;
    }
    Batch& b = batch->impl;
    std::vector<int2> items;
    if (cols_per_cta == -8 || cols_per_cta == -16 || cols_per_cta == -32) {
        for (const SliceDesc& d : b.hdesc)
            if (!d.n2) {
                set_error("pp_batch_set_tile: slice length %d has no register FFT kernel", d.ny);
                return PP_ERR_UNSUPPORTED;
            }
        PP_TRY(set_items(b, 3, &items));
        b.dev.fast4 = 1;
        b.dev.cl = -cols_per_cta / 8;
        b.dev.un2 = b.uni_n2;
        b.dev.grid = batch4_grid();
    } else {
        b.dev.cl = 1;
        b.dev.un2 = 0;
        const int lgt = cols_per_cta == 4 ? 2 : cols_per_cta == 8 ? 3 : cols_per_cta == 16 ? 4 : -1;
        if (lgt < 0 || !km_for(b.dev.ny_max, lgt)) {
            set_error("pp_batch_set_tile: unsupported tile width %d", cols_per_cta);
            return PP_ERR_UNSUPPORTED;
        }
        b.dev.fast4 = 0;
        PP_TRY(set_items(b, lgt, &items));
    }
    b.gkey.clear();
    b.tape_key.clear();
    return PP_OK;
}

pp_status pp_batch_forward_apply(const pp_batch* batch, const pp_c64* x, pp_c64* y, pp_stream stream) {
    if (!batch || !x || !y) {
        set_error("pp_batch_forward_apply: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    const Batch& b = batch->impl;
    for (int s = 0; s < b.n; ++s)
        PP_TRY(forward_into(*b.sub[s], reinterpret_cast<const float2*>(x) + b.img_off[s],
                            reinterpret_cast<float2*>(y) + b.ksp_off[s], (cudaStream_t)stream));
    return PP_OK;
}

pp_status pp_batch_adjoint_apply(const pp_batch* batch, const pp_c64* y, pp_c64* x, pp_stream stream) {
    if (!batch || !x || !y) {
        set_error("pp_batch_adjoint_apply: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    const Batch& b = batch->impl;
    for (int s = 0; s < b.n; ++s)
        PP_TRY(adjoint_into(*b.sub[s], reinterpret_cast<const float2*>(y) + b.ksp_off[s],
                            reinterpret_cast<float2*>(x) + b.img_off[s], (cudaStream_t)stream));
    return PP_OK;
}

pp_status pp_batch_normal_apply(const pp_batch* batch, const pp_c64* x, pp_c64* y, pp_stream stream) {
    if (!batch || !x || !y || (const void*)x == (const void*)y) {
        set_error("pp_batch_normal_apply: NULL or aliased argument");
        return PP_ERR_INVALID_ARG;
    }
    return launch_batch_normal(batch->impl.dev, reinterpret_cast<const float2*>(x),
                               reinterpret_cast<float2*>(y), 1.f, nullptr, 0.f, (cudaStream_t)stream);
}

pp_status pp_batch_fista_solve(pp_batch* batch, const pp_c64* bk, float lambda, int iters,
                               const double* c, int d, pp_c64* x_out, pp_solve_info* info,
                               pp_stream stream) {
    if (!batch || !bk || !x_out || iters < 0 || iters > 1000000 || !(lambda >= 0.f) ||
        !isfinite(lambda) || d < 0 || d > 16 || (!c && d != 0)) {
        set_error("pp_batch_fista_solve: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    if (info && info->levels && info->levels != 2) {
        set_error("pp_batch_fista_solve: batched prox supports 2 Haar levels only");
        return PP_ERR_UNSUPPORTED;
    }
    if (info && info->wavelet) {
        set_error("pp_batch_fista_solve: the batched prox is the 2-level Haar");
        return PP_ERR_UNSUPPORTED;
    }
    std::vector<double> c_safe;
    PP_TRY(safe_coeffs(info, c, d, c_safe));
    Batch& b = batch->impl;
    cudaStream_t st = (cudaStream_t)stream;
    const bool hist = info && info->history;
    const bool momentum = !(info && info->no_momentum);
    const float2* ref = info ? reinterpret_cast<const float2*>(info->ref) : nullptr;
    const int64_t launches0 = g_launches;
    const float2* bd = reinterpret_cast<const float2*>(bk);
    PP_TRY(launch_seg_dot(nullptr, bd, b.dev.ksp, b.partials, nullptr, b.scal + 0, 4, st));
    for (int s = 0; s < b.n; ++s)
        PP_TRY(adjoint_into(*b.sub[s], bd + b.ksp_off[s], b.ahb + b.img_off[s], st));
    PP_TRY(launch_seg_scale(b.ahb, b.ahb, b.dev.img, b.scal + 0, 4, b.dfac, 1, st));
    PP_TRY_CUDA(cudaMemsetAsync(b.y, 0, b.nimg * sizeof(float2), st));
    PP_TRY_CUDA(cudaMemsetAsync(b.z, 0, b.nimg * sizeof(float2), st));
    if (hist) {
        if (b.hist_cap < iters) {
            if (b.hist) {
                cudaStreamSynchronize(st);
                cudaFree(b.hist);
                b.allocs.erase(std::remove(b.allocs.begin(), b.allocs.end(), (void*)b.hist), b.allocs.end());
                b.hist = nullptr;
            }
            PP_TRY(balloc(b, &b.hist, (size_t)3 * std::max(iters, 1)));
            b.hist_cap = iters;
            b.gkey.clear();
        }
        PP_TRY_CUDA(cudaMemsetAsync(b.hist, 0, sizeof(double) * 3 * std::max(iters, 1), st));
    }
    if (iters > 0) {
        std::vector<double> key = {(double)iters, (double)d, (double)lambda, hist ? 1.0 : 0.0,
                                   c ? 1.0 : 0.0, (double)(uintptr_t)b.hist, (double)(uintptr_t)ref,
                                   (double)b.dev.lgt, (double)b.dev.fast4, momentum ? 1.0 : 0.0};
        if (c)
            for (int i = 0; i <= d; ++i) key.push_back(c[i]);
        if (!b.gexec || key != b.gkey) {
            if (b.gexec) {
                cudaGraphExecDestroy(b.gexec);
                b.gexec = nullptr;
            }
            b.gkey.clear();
            cudaGraph_t graph = nullptr;
            PP_TRY_CUDA(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = g_launches;
            pp_status rc = batch_iterations(b, lambda, iters, c, d, hist, ref, momentum, b.cap_stream);
            cudaError_t e = cudaStreamEndCapture(b.cap_stream, &graph);
            b.graph_kernels = g_launches - before;
            g_launches = before;
            if (rc != PP_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b.gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b.gexec = nullptr;
                return cuda_status(e, "cudaGraphInstantiate");
            }
            b.gkey = key;
        }
        PP_TRY_CUDA(cudaGraphLaunch(b.gexec, st));
    }
    float2* xo = reinterpret_cast<float2*>(x_out);
    if (info && info->rescale)
        PP_TRY(launch_seg_scale(b.y, xo, b.dev.img, b.scal + 0, 4, b.dfac, 0, st));
    else
        PP_TRY_CUDA(cudaMemcpyAsync(xo, b.y, b.nimg * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (info) {
        info->L = b.L[0];
        info->launches = (g_launches - launches0) + (iters > 0 ? b.graph_kernels : 0);
        if (hist) {
            double bn2 = 0.0;
            PP_TRY_CUDA(cudaMemcpyAsync(&bn2, b.scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaMemcpyAsync(info->history, b.hist, sizeof(double) * 3 * iters,
                                        cudaMemcpyDeviceToHost, st));
            PP_TRY_CUDA(cudaStreamSynchronize(st));
            PP_TRY(check_history("pp_batch_fista_solve", bn2, info->history, iters));
        }
    }
    return PP_OK;
}

static bool unrolled_args_ok(const pp_batch* batch, const void* bk, int iters, const double* c,
                             int d, int ce, float lambda) {
    return batch && bk && c && iters >= 1 && iters <= 100000 && d >= 0 && d <= 10 && ce >= 1 &&
           ce <= iters && lambda >= 0.f && isfinite(lambda);
}

// What the checkpoints of an unrolled forward depend on besides the contents
// of b: b's address, lambda, the iteration count, the polynomial, the
// checkpoint spacing and every slice's L_s.
static std::vector<double> tape_key_of(const Batch& B, const void* bk, float lambda, int iters,
                                       const double* c, int d, int ce) {
    std::vector<double> key = {(double)(uintptr_t)bk, (double)lambda, (double)iters, (double)d,
                               (double)ce};
    for (int i = 0; i <= d; ++i) key.push_back(c[i]);
    key.insert(key.end(), B.L.begin(), B.L.end());
    return key;
}

pp_status pp_batch_unrolled_forward(pp_batch* batch, const pp_c64* b, float lambda, int iters,
                                    const double* c, int d, int checkpoint_every, pp_c64* x_out,
                                    pp_stream stream) {
    if (!unrolled_args_ok(batch, b, iters, c, d, checkpoint_every, lambda) || !x_out) {
        set_error("pp_batch_unrolled_forward: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    Batch& B = batch->impl;
    pp_status rc = unrolled_forward(B, reinterpret_cast<const float2*>(b), lambda, iters, c, d,
                                    checkpoint_every, reinterpret_cast<float2*>(x_out),
                                    (cudaStream_t)stream);
    if (rc != PP_OK) return rc;
    B.tape_key = tape_key_of(B, b, lambda, iters, c, d, checkpoint_every);
    return PP_OK;
}

pp_status pp_batch_unrolled_backward(pp_batch* batch, const pp_c64* b, float lambda, int iters,
                                     const double* c, int d, int checkpoint_every,
                                     const pp_c64* grad_out, pp_c64* grad_b, double* grad_lambda,
                                     double* grad_c, pp_stream stream) {
    if (!unrolled_args_ok(batch, b, iters, c, d, checkpoint_every, lambda) || !grad_out ||
        !grad_b || !grad_lambda || !grad_c) {
        set_error("pp_batch_unrolled_backward: bad argument");
        return PP_ERR_INVALID_ARG;
    }
    Batch& B = batch->impl;
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<double> key = tape_key_of(B, b, lambda, iters, c, d, checkpoint_every);
    if (key != B.tape_key) {
        // no matching forward on the tape: run it (its output goes to the solve buffer)
        PP_TRY(unrolled_forward(B, reinterpret_cast<const float2*>(b), lambda, iters, c, d,
                                checkpoint_every, B.w3, st));
        B.tape_key = key;
    }
    return unrolled_backward(B, lambda, iters, c, d, checkpoint_every,
                             reinterpret_cast<const float2*>(grad_out), reinterpret_cast<float2*>(grad_b),
                             grad_lambda, grad_c, st);
}

}  // extern "C"
