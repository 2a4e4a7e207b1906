// Allocation-free adjoint: A^H y with every intermediate buffer taken from a
// fixed array of device memory that is part of the library image.
//
// Who needs it: callers that must not allocate device memory at the time of
// the call -- code running while a stream capture in global mode is open
// (cudaMalloc is illegal then), plug-ins whose host application owns all
// device memory through its own pool, and real-time reconstruction loops
// with a no-allocation rule after start-up.  Such callers build their plan
// during start-up and later call pp_adjoint_apply_static instead of
// pp_adjoint_apply, which writes its intermediates into the plan's own
// workspace.  (The paper has no counterpart: this is an interface concern.)
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "pp_internal.h"

// 16 MiB of device scratch.  Every GPU on which the library is loaded holds
// it until the process exits.  Host code must not use the symbol as a device
// address: it is a host-side stand-in, and the real address comes from
// cudaGetSymbolAddress (per device) below.
#define PP_STATIC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) float2 g_pp_static_scratch[PP_STATIC_SCRATCH_BYTES / sizeof(float2)];

namespace pp {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float2* g_static_addr[kMaxDevices] = {};

// Address of the scratch array on the current device; looked up once per
// device (the first call on a device must therefore not run inside a stream
// capture).
pp_status static_scratch(float2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("pp_adjoint_apply_static: device ordinal %d out of range", dev);
        return PP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_pp_static_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = static_cast<float2*>(ptr);
    }
    *out = g_static_addr[dev];
    return PP_OK;
}

ColArgs cols(int Hin, int Hout, int G, int off_in, int off_out, int ncols, int64_t ibs,
             int64_t obs, int nbatch, float scale) {
    ColArgs a;
    a.Hin = Hin; a.Hout = Hout; a.G = G; a.off_in = off_in; a.off_out = off_out;
    a.ncols = ncols; a.in_batch_stride = ibs; a.out_batch_stride = obs; a.nbatch = nbatch;
    a.scale = scale; a.mul_in = nullptr; a.mul_out = nullptr;
    a.mo_q = 0; a.mo_c = 0; a.mo_cdiv = 1; a.mi_q = 1; a.mi_c = 0; a.mi_cdiv = 1;
    return a;
}

RowArgs rows(int n, int G, int off_in, int off_out, int nrows, int64_t cis, float scale) {
    RowArgs a;
    a.n = n; a.G = G; a.off_in = off_in; a.off_out = off_out; a.nrows = nrows;
    a.coil_img_stride = cis; a.scale = scale;
    return a;
}

// Scratch elements (complex64) the adjoint needs for plan p: the first
// buffer (wa) and the second (wb).
void scratch_elems(const Plan& p, int64_t* wa, int64_t* wb) {
    if (p.kind == PP_CARTESIAN && p.ndim == 2) {
        *wa = (int64_t)p.C * p.nimg;
        *wb = 0;
    } else if (p.kind == PP_CARTESIAN) {
        *wa = p.nimg;
        *wb = p.nimg;
    } else {
        *wa = (int64_t)p.C * p.ny * p.G_x;
        *wb = (int64_t)p.C * p.G_y * p.G_x;
    }
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_adjoint_apply_static(const pp_plan* plan, const pp_c64* yk, pp_c64* xo,
                                             pp_stream stream) {
    if (!plan || !yk || !xo) {
        set_error("pp_adjoint_apply_static: NULL argument");
        return PP_ERR_INVALID_ARG;
    }
    const Plan& p = plan->impl;
    int64_t na = 0, nb = 0;
    scratch_elems(p, &na, &nb);
    const double need = (double)(na + nb) * sizeof(float2);
    if (need > (double)PP_STATIC_SCRATCH_BYTES) {
        set_error("pp_adjoint_apply_static: this plan needs %.1f MiB of scratch, above the fixed "
                  "%u MiB; use pp_adjoint_apply", need / 1048576.0, PP_STATIC_SCRATCH_BYTES >> 20);
        return PP_ERR_UNSUPPORTED;
    }
    float2* base = nullptr;
    PP_TRY(static_scratch(&base));
    float2* wa = base;
    float2* wb = base + na;
    const float2* y = reinterpret_cast<const float2*>(yk);
    float2* x = reinterpret_cast<float2*>(xo);
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t n = p.nimg;
    // Every scratch element read below is written earlier in the same call,
    // so nothing needs clearing between calls.
    if (p.kind == PP_CARTESIAN && p.ndim == 2) {
        ColArgs ay = cols(ny, ny, ny, ny / 2, ny / 2, nx, (int64_t)ny * nx, (int64_t)ny * nx, p.C,
                          (float)(1.0 / sqrt((double)ny)));
        ay.mul_in = p.mask_c;
        PP_TRY(launch_cols(p.fy, ay, y, wa, true, st));
        RowArgs ra = rows(nx, nx, nx / 2, nx / 2, ny, n, (float)(1.0 / sqrt((double)nx)));
        return launch_rows_adj(p, p.fx, ra, wa, p.sens, nullptr, nullptr, x, nullptr, 0.f, p.C, st);
    }
    if (p.kind == PP_CARTESIAN) {
        for (int c = 0; c < p.C; ++c) {
            ColArgs az = cols(nz, nz, nz, nz / 2, nz / 2, ny * nx, 0, 0, 1,
                              (float)(1.0 / sqrt((double)nz)));
            az.mul_in = p.mask_c; az.mi_q = ny; az.mi_c = 1; az.mi_cdiv = nx;
            PP_TRY(launch_cols(p.fz, az, y + (int64_t)c * n, wa, true, st));
            ColArgs ay = cols(ny, ny, ny, ny / 2, ny / 2, nx, (int64_t)ny * nx, (int64_t)ny * nx, nz,
                              (float)(1.0 / sqrt((double)ny)));
            PP_TRY(launch_cols(p.fy, ay, wa, wb, true, st));
            RowArgs ra = rows(nx, nx, nx / 2, nx / 2, ny * nz, 0, (float)(1.0 / sqrt((double)nx)));
            PP_TRY(launch_rows_adj(p, p.fx, ra, wb, p.sens + (int64_t)c * n, nullptr, nullptr, x,
                                   c == 0 ? nullptr : x, 1.f, 1, st));
        }
        return PP_OK;
    }
    const int Gx = p.G_x, Gy = p.G_y;
    PP_TRY(launch_nufft_spread(p, y, wb, st));
    ColArgs ci = cols(Gy, ny, Gy, 0, ny / 2, Gx, (int64_t)Gy * Gx, (int64_t)ny * Gx, p.C, 1.f);
    PP_TRY(launch_cols(p.gy, ci, wb, wa, true, st));
    RowArgs ra = rows(nx, Gx, 0, nx / 2, ny, (int64_t)ny * nx, 1.f);
    return launch_rows_adj(p, p.gx, ra, wa, p.sens, p.deapod_y, p.deapod_x, x, nullptr, 0.f, p.C, st);
}
