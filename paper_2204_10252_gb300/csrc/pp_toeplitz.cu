// Spectrum of the embedded kernel of the Toeplitz-structured F^H F (the
// remark on Toeplitz normal operators in Sec. 2, used by the spiral
// experiment of Sec. 5.2).
//
// With F the exact non-uniform DFT, (F^H F)[r, r'] = h(r - r') where
//   h(d) = 1/n sum_k exp(2 pi i (kx dx / nx + ky dy / ny)),  |dy| < ny, |dx| < nx.
// Embedded in the 2ny x 2nx circulant (h at offset d mod 2n, zero at n), F^H F v
// is the crop of a circular convolution, i.e. IFFT(Tk . FFT(zero-pad(v))) with
//   Tk(q) = sum_d h(d) exp(-2 pi i (qy dy / My + qx dx / Mx)) / (My Mx)
//         = 1/(n My Mx) sum_k Dy(ky / ny - qy / My) Dx(kx / nx - qx / Mx),
//   D(theta) = sum_{d = -(n-1)}^{n-1} exp(2 pi i d theta) = sin((2n-1) pi theta) / sin(pi theta),
// which is real (h(-d) = conj(h(d))).  The sum over samples is a real matrix
// product of the per-axis Dirichlet kernels, computed here in chunks of
// samples with FP32 products and FP64 accumulation across chunks.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pp_internal.h"

namespace pp {
namespace {

constexpr int KC = 4096;     // samples per chunk
constexpr int KSLICE = 256;  // samples per CTA of the product (FP32 partial sums)
constexpr int TG = 64;       // product tile (TG x TG outputs per CTA)
constexpr int KSTEP = 16;    // samples per shared-memory step

// D[k][q] = D(traj[k0 + k][axis] / n - q / M) for k < kc (zero for samples
// at or past K), q < M.  theta and (2n-1) theta are reduced in FP64, so the
// FP32 sines take exact phases: theta to [-1/2, 1/2] (D has period 1), the
// numerator's argument to [-1, 1] (sin(pi a) has period 2).
__global__ void toep_dirichlet_kernel(const float* __restrict__ traj, int axis, int64_t k0,
                                      int64_t K, int kc, int n, int M, float* __restrict__ D) {
    const int64_t total = (int64_t)kc * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / M), q = (int)(e - (int64_t)k * M);
        float v = 0.f;
        if (k0 + k < K) {
            const double th = (double)traj[(k0 + k) * 2 + axis] / n - (double)q / M;
            const double tr = th - rint(th);
            if (tr == 0.0) {
                v = (float)(2 * n - 1);
            } else {
                const double a = (double)(2 * n - 1) * tr;
                const double ar = a - 2.0 * rint(0.5 * a);
                v = sinpif((float)ar) / sinpif((float)tr);
            }
        }
        D[e] = v;
    }
}

// P[s][qy][qx] = sum over samples k of slice s of Dy[k][qy] Dx[k][qx].
// grid (Mx / TG, My / TG, slices), 256 threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256)
toep_gemm_kernel(const float* __restrict__ Dy, const float* __restrict__ Dx, int My, int Mx, int kc,
                 float* __restrict__ P) {
    __shared__ __align__(16) float As[KSTEP][TG];
    __shared__ __align__(16) float Bs[KSTEP][TG];
    const int qx0 = blockIdx.x * TG, qy0 = blockIdx.y * TG, s = blockIdx.z;
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int kb = s * KSLICE, ke = min(kc, kb + KSLICE);
    for (int k = kb; k < ke; k += KSTEP) {
        for (int e = threadIdx.x; e < KSTEP * TG; e += blockDim.x) {
            const int kk = e / TG, q = e % TG;
            const bool ok = k + kk < ke;
            As[kk][q] = ok ? Dy[(int64_t)(k + kk) * My + qy0 + q] : 0.f;
            Bs[kk][q] = ok ? Dx[(int64_t)(k + kk) * Mx + qx0 + q] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KSTEP; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            P[((int64_t)s * My + qy0 + ty * 4 + i) * Mx + qx0 + tx * 4 + j] = acc[i][j];
}

// acc[q] += sum_s P[s][q], slices in order (FP64).
__global__ void toep_accumulate_kernel(const float* __restrict__ P, int slices, int64_t m,
                                       double* __restrict__ acc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m;
         q += (int64_t)gridDim.x * blockDim.x) {
        double a = acc[q];
        for (int s = 0; s < slices; ++s) a += (double)P[s * m + q];
        acc[q] = a;
    }
}

// T[qx][qy] = acc[qy][qx] * inv  (column-major for the column stage)
__global__ void toep_finalize_kernel(const double* __restrict__ acc, int My, int Mx, double inv,
                                     float* __restrict__ T) {
    const int64_t m = (int64_t)My * Mx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int qx = (int)(e / My), qy = (int)(e - (int64_t)qx * My);
        T[e] = (float)(acc[(int64_t)qy * Mx + qx] * inv);
    }
}

struct TempBuffers {
    void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    ~TempBuffers() {
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

pp_status check_toep(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    ++g_launches;
    return PP_OK;
}

}  // namespace

// Fills p.toep_T (allocated by the caller, [2nx][2ny]) from the host
// trajectory traj[K][2] = (kx, ky) in cycles per field of view.  Synchronises
// the stream before its temporaries are freed.
pp_status toep_build_kernel(Plan& p, const float* traj, int64_t K, cudaStream_t st) {
    const int nx = p.nx, ny = p.ny, Mx = 2 * nx, My = 2 * ny;
    if (Mx % TG || My % TG) {
        set_error("Toeplitz kernel: 2 nx and 2 ny must be multiples of %d", TG);
        return PP_ERR_UNSUPPORTED;
    }
    const int64_t m = (int64_t)My * Mx;
    const int slices_max = KC / KSLICE;
    TempBuffers t;
    float *dtraj, *Dy, *Dx, *P;
    double* acc;
    PP_TRY_CUDA(cudaMalloc(&t.p[0], sizeof(float) * 2 * std::max<int64_t>(K, 1)));
    PP_TRY_CUDA(cudaMalloc(&t.p[1], sizeof(float) * (size_t)KC * My));
    PP_TRY_CUDA(cudaMalloc(&t.p[2], sizeof(float) * (size_t)KC * Mx));
    PP_TRY_CUDA(cudaMalloc(&t.p[3], sizeof(float) * (size_t)slices_max * m));
    PP_TRY_CUDA(cudaMalloc(&t.p[4], sizeof(double) * (size_t)m));
    dtraj = (float*)t.p[0]; Dy = (float*)t.p[1]; Dx = (float*)t.p[2]; P = (float*)t.p[3];
    acc = (double*)t.p[4];
    PP_TRY_CUDA(cudaMemcpyAsync(dtraj, traj, sizeof(float) * 2 * K, cudaMemcpyHostToDevice, st));
    PP_TRY_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)m, st));
    for (int64_t k0 = 0; k0 < K; k0 += KC) {
        const int kc = (int)std::min<int64_t>(KC, K - k0);
        const int slices = (kc + KSLICE - 1) / KSLICE;
        toep_dirichlet_kernel<<<152 * 4, 256, 0, st>>>(dtraj, 1, k0, K, kc, ny, My, Dy);
        PP_TRY(check_toep("toep_dirichlet_kernel"));
        toep_dirichlet_kernel<<<152 * 4, 256, 0, st>>>(dtraj, 0, k0, K, kc, nx, Mx, Dx);
        PP_TRY(check_toep("toep_dirichlet_kernel"));
        toep_gemm_kernel<<<dim3(Mx / TG, My / TG, slices), 256, 0, st>>>(Dy, Dx, My, Mx, kc, P);
        PP_TRY(check_toep("toep_gemm_kernel"));
        toep_accumulate_kernel<<<152 * 4, 256, 0, st>>>(P, slices, m, acc);
        PP_TRY(check_toep("toep_accumulate_kernel"));
    }
    const double inv = 1.0 / ((double)nx * ny * (double)My * Mx);
    toep_finalize_kernel<<<152 * 4, 256, 0, st>>>(acc, My, Mx, inv, p.toep_T);
    PP_TRY(check_toep("toep_finalize_kernel"));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    return PP_OK;
}

}  // namespace pp
