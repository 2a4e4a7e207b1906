// Allocation-free adjoint: A^H y with every intermediate buffer taken from a
// fixed array of device memory that is part of the library image.
//
// Who needs it: callers that must not allocate device memory at the time of
// the call -- plug-ins whose host application owns all device memory
// through its own pool (a cudaMalloc behind its back can fail or break the
// host's accounting), and real-time reconstruction loops with a
// no-allocation rule after start-up (an allocation can stall or fail when
// memory is fragmented).  Such callers build their plan during start-up and
// later call pp_adjoint_apply_static instead of pp_adjoint_apply, which
// writes its intermediates into the plan's own workspace.  Both run the same
// kernel sequence (adjoint_ws).  The paper has no counterpart: this is an
// interface concern.
#include <cuda_runtime.h>

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

// Address of the scratch array on the current device, looked up on the first
// call on each device and kept for the life of the process (a
// cudaDeviceReset of that device, which also frees every plan, ends the
// library's use of it).
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

// Scratch elements (complex64) the adjoint needs for plan p: the first
// buffer (wa) and the second (wb) of adjoint_ws.
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
    // Every scratch element read by the adjoint is written earlier in the
    // same call, so nothing needs clearing between calls.
    return adjoint_ws(p, reinterpret_cast<const float2*>(yk), reinterpret_cast<float2*>(xo), base,
                      base + na, (cudaStream_t)stream);
}
