// Register-resident FFTs for the transform lengths of the workloads
// (n = N1 * N2 with N1 = 16 and N2 in {8, 12, 16, 20, 24}: 128 ... 384).
//
// Four-step decomposition, input index m = N2*m1 + m2, output k = k1 + N1*k2:
//   X[k] = sum_m2 W_N2^(m2 k2) [ W_n^(m2 k1) sum_m1 x[N2 m1 + m2] W_N1^(m1 k1) ]
// Phase 1: one thread per (transform, m2) loads N1 inputs into registers,
//          runs the length-N1 DFT, applies W_n^(m2 k1), writes Y[k1][m2] to
//          shared memory.
// Phase 2: one thread per (transform, k1) reads Y[k1][0..N2), runs the
//          length-N2 DFT and holds X[k1 + N1 k2] in registers.
// Each register DFT of composite length A*B is itself a four-step over the
// radix-2/3/4/5/8 kernels of pp_fft.cuh, fully unrolled.  Twiddles come from
// the shared table w[t] = exp(-2 pi i t / n): W_L^m = w[m * n / L].
#pragma once
#include "pp_fft.cuh"

namespace pp {

// W_N^m = exp(-2 pi i m / N) for the register DFT lengths (mathematical
// constants, rounded to float); indexed with compile-time m after unrolling,
// so they become constant-bank operands.
static __constant__ float2 c_w12[12] = {{1.000000000e+00f, -0.000000000e+00f}, {8.660254038e-01f, -5.000000000e-01f}, {5.000000000e-01f, -8.660254038e-01f}, {6.123233996e-17f, -1.000000000e+00f}, {-5.000000000e-01f, -8.660254038e-01f}, {-8.660254038e-01f, -5.000000000e-01f}, {-1.000000000e+00f, -1.224646799e-16f}, {-8.660254038e-01f, 5.000000000e-01f}, {-5.000000000e-01f, 8.660254038e-01f}, {-1.836970199e-16f, 1.000000000e+00f}, {5.000000000e-01f, 8.660254038e-01f}, {8.660254038e-01f, 5.000000000e-01f}};
static __constant__ float2 c_w16[16] = {{1.000000000e+00f, -0.000000000e+00f}, {9.238795325e-01f, -3.826834324e-01f}, {7.071067812e-01f, -7.071067812e-01f}, {3.826834324e-01f, -9.238795325e-01f}, {6.123233996e-17f, -1.000000000e+00f}, {-3.826834324e-01f, -9.238795325e-01f}, {-7.071067812e-01f, -7.071067812e-01f}, {-9.238795325e-01f, -3.826834324e-01f}, {-1.000000000e+00f, -1.224646799e-16f}, {-9.238795325e-01f, 3.826834324e-01f}, {-7.071067812e-01f, 7.071067812e-01f}, {-3.826834324e-01f, 9.238795325e-01f}, {-1.836970199e-16f, 1.000000000e+00f}, {3.826834324e-01f, 9.238795325e-01f}, {7.071067812e-01f, 7.071067812e-01f}, {9.238795325e-01f, 3.826834324e-01f}};
static __constant__ float2 c_w20[20] = {{1.000000000e+00f, -0.000000000e+00f}, {9.510565163e-01f, -3.090169944e-01f}, {8.090169944e-01f, -5.877852523e-01f}, {5.877852523e-01f, -8.090169944e-01f}, {3.090169944e-01f, -9.510565163e-01f}, {6.123233996e-17f, -1.000000000e+00f}, {-3.090169944e-01f, -9.510565163e-01f}, {-5.877852523e-01f, -8.090169944e-01f}, {-8.090169944e-01f, -5.877852523e-01f}, {-9.510565163e-01f, -3.090169944e-01f}, {-1.000000000e+00f, -1.224646799e-16f}, {-9.510565163e-01f, 3.090169944e-01f}, {-8.090169944e-01f, 5.877852523e-01f}, {-5.877852523e-01f, 8.090169944e-01f}, {-3.090169944e-01f, 9.510565163e-01f}, {-1.836970199e-16f, 1.000000000e+00f}, {3.090169944e-01f, 9.510565163e-01f}, {5.877852523e-01f, 8.090169944e-01f}, {8.090169944e-01f, 5.877852523e-01f}, {9.510565163e-01f, 3.090169944e-01f}};
static __constant__ float2 c_w24[24] = {{1.000000000e+00f, -0.000000000e+00f}, {9.659258263e-01f, -2.588190451e-01f}, {8.660254038e-01f, -5.000000000e-01f}, {7.071067812e-01f, -7.071067812e-01f}, {5.000000000e-01f, -8.660254038e-01f}, {2.588190451e-01f, -9.659258263e-01f}, {6.123233996e-17f, -1.000000000e+00f}, {-2.588190451e-01f, -9.659258263e-01f}, {-5.000000000e-01f, -8.660254038e-01f}, {-7.071067812e-01f, -7.071067812e-01f}, {-8.660254038e-01f, -5.000000000e-01f}, {-9.659258263e-01f, -2.588190451e-01f}, {-1.000000000e+00f, -1.224646799e-16f}, {-9.659258263e-01f, 2.588190451e-01f}, {-8.660254038e-01f, 5.000000000e-01f}, {-7.071067812e-01f, 7.071067812e-01f}, {-5.000000000e-01f, 8.660254038e-01f}, {-2.588190451e-01f, 9.659258263e-01f}, {-1.836970199e-16f, 1.000000000e+00f}, {2.588190451e-01f, 9.659258263e-01f}, {5.000000000e-01f, 8.660254038e-01f}, {7.071067812e-01f, 7.071067812e-01f}, {8.660254038e-01f, 5.000000000e-01f}, {9.659258263e-01f, 2.588190451e-01f}};

template <int L> __device__ __forceinline__ float2 cw(int m);
template <> __device__ __forceinline__ float2 cw<12>(int m) { return c_w12[m]; }
template <> __device__ __forceinline__ float2 cw<16>(int m) { return c_w16[m]; }
template <> __device__ __forceinline__ float2 cw<20>(int m) { return c_w20[m]; }
template <> __device__ __forceinline__ float2 cw<24>(int m) { return c_w24[m]; }

template <int N, bool INV> struct RegFft;

template <bool INV> struct RegFft<2, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2*, int) { Dft<2, INV>::run(v); }
};
template <bool INV> struct RegFft<3, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2*, int) { Dft<3, INV>::run(v); }
};
template <bool INV> struct RegFft<4, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2*, int) { Dft<4, INV>::run(v); }
};
template <bool INV> struct RegFft<5, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2*, int) { Dft<5, INV>::run(v); }
};
template <bool INV> struct RegFft<8, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2*, int) { Dft<8, INV>::run(v); }
};

// Length A*B in registers; `step` = n / (A*B) indexes the shared twiddle table.
template <int A, int B, bool INV>
__device__ __forceinline__ void reg_fft_ab(float2* v, const float2* __restrict__ tw, int step) {
    float2 t[A * B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        float2 u[A];
#pragma unroll
        for (int a = 0; a < A; ++a) u[a] = v[B * a + b];
        RegFft<A, INV>::run(u, tw, step * B);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) t[b * A + k1] = u[k1];
    }
#pragma unroll
    for (int b = 1; b < B; ++b)
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1) {
            float2 w = cw<A * B>(b * k1);
            if (INV) w.y = -w.y;
            t[b * A + k1] = cmul(t[b * A + k1], w);
        }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        float2 u[B];
#pragma unroll
        for (int b = 0; b < B; ++b) u[b] = t[b * A + k1];
        RegFft<B, INV>::run(u, tw, step * A);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = u[k2];
    }
}

template <bool INV> struct RegFft<12, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2* tw, int s) { reg_fft_ab<4, 3, INV>(v, tw, s); }
};
template <bool INV> struct RegFft<16, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2* tw, int s) { reg_fft_ab<4, 4, INV>(v, tw, s); }
};
template <bool INV> struct RegFft<20, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2* tw, int s) { reg_fft_ab<4, 5, INV>(v, tw, s); }
};
template <bool INV> struct RegFft<24, INV> {
    static __device__ __forceinline__ void run(float2* v, const float2* tw, int s) { reg_fft_ab<8, 3, INV>(v, tw, s); }
};

// Fast lengths: returns N2 for n = 16 * N2 with a register kernel, else 0.
__host__ __device__ __forceinline__ int fft4_n2(int n) {
    if (n % 16) return 0;
    const int n2 = n / 16;
    return (n2 == 8 || n2 == 12 || n2 == 16 || n2 == 20 || n2 == 24) ? n2 : 0;
}

// Phase 1 for one (transform, m2): v holds x[N2*m1 + m2], m1 < N1, on entry;
// on exit v[k1] = W_n^(m2 k1) * sum_m1 x[N2 m1 + m2] W_N1^(m1 k1).
template <int N1, int N2, bool INV>
__device__ __forceinline__ void fft4_phase1(float2* v, int m2, const float2* __restrict__ tw) {
    RegFft<N1, INV>::run(v, tw, N2);
    // W_n^(m2 k1): four table loads (k1 = 1..4), the rest by w_k = w_(k-4) w_4
    float2 w[N1];
    w[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int k1 = 1; k1 <= 4 && k1 < N1; ++k1) w[k1] = tw[m2 * k1];
#pragma unroll
    for (int k1 = 5; k1 < N1; ++k1) w[k1] = cmul(w[k1 - 4], w[4]);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
        float2 ww = w[k1];
        if (INV) ww.y = -ww.y;
        v[k1] = cmul(v[k1], ww);
    }
}

// Phase 2 for one (transform, k1): u holds Y[k1][m2], m2 < N2; on exit
// u[k2] = X[k1 + N1 k2].
template <int N1, int N2, bool INV>
__device__ __forceinline__ void fft4_phase2(float2* u, const float2* __restrict__ tw) {
    RegFft<N2, INV>::run(u, tw, N1);
}

}  // namespace pp

namespace pp {

// Split thread-block-cluster barrier.  arrive_release publishes this CTA's
// earlier shared-memory writes to the cluster, wait_acquire makes the other
// CTAs' visible; arrive_relaxed orders nothing (for a barrier that only
// says "done reading").  All threads of the CTA execute each of them.
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// 16-byte asynchronous global -> shared copy, zero-filled when !valid.
__device__ __forceinline__ void cpa16(void* smem, const void* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// Stage the n x 8 tile S[0..n)[col0 .. col0+8) of one coil map (row pitch
// nx, nx even) into dst[row * 8 + j] with cp.async and commit it as one group;
// columns at or past nx read as zero.
template <int N2>
__device__ __forceinline__ void stage_s_tile(float2* dst, const float2* __restrict__ S, int nx,
                                             int col0) {
    constexpr int n = 16 * N2;
    for (int e = threadIdx.x; e < n * 4; e += blockDim.x) {
        const int row = e >> 2, q = e & 3, c = col0 + 2 * q;
        const bool ok = c < nx;
        cpa16(dst + row * 8 + 2 * q, S + (ok ? (int64_t)row * nx + c : 0), ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Coil loop of the fused Cartesian item for coils c_first, c_first + c_step,
// ... < C: acc[m1] (rows N2 m1 + r of column col0 + lane, threads r < N2)
// accumulates conj(S_c) F^H (mask_fo . F (S_c x)).  Ends with a barrier.
template <int N2>
__device__ __forceinline__ void cart_item4_acc(const float2* __restrict__ tws,
                                               const float* __restrict__ pm, float2* Y, float2* Sb,
                                               const float2* __restrict__ x,
                                               const float2* __restrict__ sens, int C, int nx,
                                               int col0, int c_first, int c_step, float2* acc) {
    constexpr int N1 = 16, n = N1 * N2;
    const int lane = threadIdx.x & 7, r = threadIdx.x >> 3, col = col0 + lane;
    const bool colok = col < nx;
    const bool p1 = r < N2, p2 = r < N1;
    const int64_t cs = (int64_t)n * nx;
    float2 xr[N1];
#pragma unroll
    for (int m1 = 0; m1 < N1; ++m1) acc[m1] = make_float2(0.f, 0.f);
    if (c_first >= C) {
        __syncthreads();
        return;
    }
    stage_s_tile<N2>(Sb, sens + c_first * cs, nx, col0);
#pragma unroll
    for (int m1 = 0; m1 < N1; ++m1)
        xr[m1] = (p1 && colok) ? x[(int64_t)(N2 * m1 + r) * nx + col] : make_float2(0.f, 0.f);
    int it = 0;
    for (int c = c_first; c < C; c += c_step, ++it) {
        const float2* St = Sb + (it & 1) * n * 8;
        // the other buffer was last read in the previous coil, before its final barrier
        if (c + c_step < C)
            stage_s_tile<N2>(Sb + ((it + 1) & 1) * n * 8, sens + (c + c_step) * cs, nx, col0);
        else
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        if (p1) {
            float2 v[N1];
#pragma unroll
            for (int m1 = 0; m1 < N1; ++m1) v[m1] = cmul(St[(N2 * m1 + r) * 8 + lane], xr[m1]);
            fft4_phase1<N1, N2, false>(v, r, tws);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) Y[(k1 * N2 + r) * 8 + lane] = v[k1];
        }
        __syncthreads();
        if (p2) {
            float2 u[N2];
#pragma unroll
            for (int m2 = 0; m2 < N2; ++m2) u[m2] = Y[(r * N2 + m2) * 8 + lane];
            fft4_phase2<N1, N2, false>(u, tws);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) u[k2] = cscale(u[k2], pm[r + N1 * k2]);
            RegFft<N2, true>::run(u, tws, N1);
#pragma unroll
            for (int m2 = 1; m2 < N2; ++m2) {
                float2 w = tws[m2 * r];
                w.y = -w.y;
                u[m2] = cmul(u[m2], w);
            }
#pragma unroll
            for (int m2 = 0; m2 < N2; ++m2) Y[(r * N2 + m2) * 8 + lane] = u[m2];
        }
        __syncthreads();
        if (p1) {
            float2 v[N1];
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = Y[(k1 * N2 + r) * 8 + lane];
            RegFft<N1, true>::run(v, tws, N2);
#pragma unroll
            for (int m1 = 0; m1 < N1; ++m1)
                acc[m1] = cadd(acc[m1], cmulc(St[(N2 * m1 + r) * 8 + lane], v[m1]));
        }
        __syncthreads();
    }
}

// Fused Cartesian normal-operator work item on the four-step FFT:
//   out[:, col] = sc * sum_c conj(S_c) F^H (mask_fo . F (S_c x)) + alpha * operand
// for TXF = 8 columns col0.. of an ny x nx image, ny = 16 * N2, transform
// along y.  Forward: phase 1 by (m2, col) threads, phase 2 by (k1, col)
// threads, which then hold X[k1 + 16 k2].  Inverse, with the mirrored
// decomposition (input k = k1 + 16 k2, output m = N2 m1 + m2):
//   I1 (same (k1, col) threads): inverse length-N2 DFT over k2, times
//      W_n^(-m2 k1);   I2 ((m2, col) threads): inverse length-16 DFT over k1,
// which leaves x'[N2 m1 + m2] with the thread that loaded S_c at those rows.
// The coil maps' n x 8 tiles are double-buffered in shared memory: coil
// c + 1's tile streams in by cp.async while coil c is transformed.
// Shared memory: tws[n] twiddles, pm[n] mask (FFT order, 1/ny folded in),
// Y[16 * N2 * 8], Sb[2 * n * 8].  Threads: 8 * max(16, N2); all threads
// must call it.
template <int N2>
__device__ __forceinline__ void cart_item4(const float2* __restrict__ tws,
                                           const float* __restrict__ pm, float2* Y, float2* Sb,
                                           const float2* __restrict__ x,
                                           const float2* __restrict__ sens, int C, int nx,
                                           int col0, float2* out, float sc,
                                           const float2* operand, float alpha) {
    constexpr int N1 = 16;
    const int lane = threadIdx.x & 7, r = threadIdx.x >> 3, col = col0 + lane;
    float2 acc[N1];
    cart_item4_acc<N2>(tws, pm, Y, Sb, x, sens, C, nx, col0, 0, 1, acc);
    if (r < N2 && col < nx) {
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int64_t o = (int64_t)(N2 * m1 + r) * nx + col;
            float2 v = cscale(acc[m1], sc);
            if (operand) v = cadd(v, cscale(operand[o], alpha));
            out[o] = v;
        }
    }
}

}  // namespace pp
