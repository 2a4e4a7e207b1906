// Shared-memory Stockham FFT for batches of short transforms (lengths whose
// prime factors are 2, 3 and 5), used by every k-space stage of the SENSE
// operators (Sec. 5.1 F, Sec. 5.2 oversampled-grid F).
//
// A batch of B transforms lives in shared memory with element i of transform
// b at offset i*es + b*bs.  Each radix-R stage reads from one buffer and
// writes the other (autosort: natural order in, natural order out), so the
// caller supplies two buffers and gets back the one holding the result.
// Stage s with sub-transform length Ns (product of the previous radices):
// butterfly j takes inputs j + r*n/R (r < R), multiplies input r by
// w^(r*k*n/(Ns*R)) with k = j mod Ns and w = exp(-2 pi i / n), applies the
// R-point DFT, and writes output q to (j - k)*R + k + q*Ns.
#pragma once
#include <cuda_runtime.h>

namespace pp {

struct FftDesc {
    int n;        // transform length
    int nst;      // number of stages
    int rad[8];   // radix of each stage (2, 3, 4, 5 or 8)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// Complex add and subtract as single packed two-lane FP32 instructions
// (per-component IEEE round-to-nearest, so bitwise the same as two scalar
// operations; b * (-1) + a rounds once to a - b).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// R-point DFTs, X_q = sum_r v_r exp(-+2 pi i r q / R) (sign + for INV).
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV> struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <bool INV> struct Dft<8, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        // split into even / odd 4-point DFTs, combine with w8^k
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        const float h = 0.70710678118654752f;   // 1/sqrt(2)
        // w8 = exp(-i pi/4) (forward); conjugate for the inverse
        float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                        : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        float2 o2 = mul_mi<INV>(o[2]);
        float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                        : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = cadd(e[0], o[0]);  v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);    v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);    v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);    v[7] = csub(e[3], o3);
    }
};

template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        const float s3 = 0.86602540378443865f;  // sqrt(3)/2
        float2 t = cadd(v[1], v[2]);
        float2 d = cscale(csub(v[1], v[2]), s3);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 id = mul_mi<INV>(d);
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, id);
        v[2] = csub(m, id);
    }
};

template <bool INV> struct Dft<5, INV> {
    static __device__ __forceinline__ void run(float2* v) {
        // cos and sin of 2 pi/5 and 4 pi/5
        const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
        const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        float2 a = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 b = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float2 p = mul_mi<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
        float2 q = mul_mi<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
        v[0] = make_float2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
        v[1] = cadd(a, p);
        v[4] = csub(a, p);
        v[2] = cadd(b, q);
        v[3] = csub(b, q);
    }
};

// One radix-R stage over a batch.  Thread t handles butterfly j = t >> lgB of
// transform b = t & (B-1) (B a power of two), striding by blockDim.x.
// `pm`, if set, scales input element i by pm[i] (first stage only).
template <int R, bool INV>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                          int n, int Ns, int es, int bs, int lgB,
                                          const float2* __restrict__ tw,
                                          const float* __restrict__ pm) {
    const int nb = n / R;
    const int total = nb << lgB;
    const int tstep = n / (Ns * R);
    const int bmask = (1 << lgB) - 1;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int b = t & bmask;
        const int j = t >> lgB;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int idx = j + r * nb;
            float2 x = src[idx * es + b * bs];
            if (pm) {
                const float m = pm[idx];
                x.x *= m;
                x.y *= m;
            }
            v[r] = x;
        }
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * k * tstep];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        Dft<R, INV>::run(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * es + b * bs] = v[r];
    }
}

// Full transform; the caller has synchronised after filling `a`.  Returns the
// buffer (a or b) that holds the result; ends with a __syncthreads().
template <bool INV>
__device__ float2* fft_batch(float2* a, float2* b, const FftDesc& f, int es, int bs, int lgB,
                             const float2* __restrict__ tw, const float* __restrict__ premul) {
    int Ns = 1;
    for (int s = 0; s < f.nst; ++s) {
        const int R = f.rad[s];
        const float* pm = (s == 0) ? premul : nullptr;
        switch (R) {
            case 8: fft_stage<8, INV>(a, b, f.n, Ns, es, bs, lgB, tw, pm); break;
            case 4: fft_stage<4, INV>(a, b, f.n, Ns, es, bs, lgB, tw, pm); break;
            case 5: fft_stage<5, INV>(a, b, f.n, Ns, es, bs, lgB, tw, pm); break;
            case 3: fft_stage<3, INV>(a, b, f.n, Ns, es, bs, lgB, tw, pm); break;
            default: fft_stage<2, INV>(a, b, f.n, Ns, es, bs, lgB, tw, pm); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace pp
