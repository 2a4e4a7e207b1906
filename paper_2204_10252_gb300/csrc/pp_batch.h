// Batched uneven 2-D Cartesian problems: device descriptors and launchers.
#pragma once
#include "pp_internal.h"

namespace pp {

// Per-slice view used by the batched kernels.
struct SliceDesc {
    FftDesc fd;              // FFT along ky (length ny)
    const float2* tw;        // its twiddle table
    const float2* sens;      // [C][ny][nx] (borrowed)
    const float* mask_fo;    // [ny], FFT order, times 1/ny
    int ny, nx, C, n2;       // n2 = ny / 16 when ny has a register FFT, else 0
    int64_t img_off;         // offset of the slice in concatenated images
    float invL, pad1;
};

// A partition of a concatenated array into segments (one per slice), and
// of a launch's blocks over those segments.  Device arrays.
struct Segments {
    int nseg = 0, nblocks = 0;
    int64_t* off = nullptr;        // [nseg + 1]
    int* blk_seg = nullptr;        // [nblocks]
    int* seg_first_blk = nullptr;  // [nseg + 1]
};

struct BatchDev {
    SliceDesc* descs = nullptr;
    int2* items = nullptr;   // (slice, first column), most expensive first
    int nitems = 0, ny_max = 0, km = 0, lgt = 3, grid = 0;
    int fast4 = 0;           // 1: the four-step register-FFT kernel runs the items
    int cl = 1;              // fast4: CTAs per item, the item's coils split over a cluster
    int un2 = 0;             // fast4: the slices' common N2 (0: mixed lengths)
    int ugrid = 0;           //   and the persistent grid of the uniform-length kernel
    Segments img, ksp, tiles;
};

// Up to 12 vectors and coefficients for a linear combination.
struct LinComb {
    const float2* v[12];
    float coef[12];
    int count;
};

size_t batch_normal_smem(int ny_max, int lgt);
void* batch_normal_fn(int km, int lgt);
pp_status configure_batch_kernels();
int batch4_grid();   // persistent grid of the four-step batched kernel
int batch4u_grid(int n2);   // the same for the uniform-length kernel (0: none)
pp_status launch_batch_normal(const BatchDev& b, const float2* x, float2* out, float coef,
                              const float2* operand, float alpha, cudaStream_t st);
pp_status launch_seg_dot(const float2* a, const float2* bv, const Segments& sg, double* partials,
                         double* out_re, double* out_nb, int stride, cudaStream_t st);
pp_status launch_seg_scale(const float2* in, float2* out, const Segments& sg, const double* norm2,
                           int stride, const double* factor, int invert, cudaStream_t st);
pp_status launch_batch_prox_fista(const BatchDev& b, float lam, float gamma, float beta,
                                  float2* z, const float2* u, float2* y, const float2* ref,
                                  double* hist, cudaStream_t st);

pp_status launch_batch_prox_vjp(const BatchDev& b, float lam, float beta, const float2* w,
                                float2* Ybar, const float2* Zbar, float2* wbar, double* lam_bar,
                                cudaStream_t st);
pp_status launch_lincomb(const LinComb& lc, float2* out, int64_t n, int accumulate, cudaStream_t st);

}  // namespace pp
