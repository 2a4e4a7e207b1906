// 3-D Cartesian normal operator (Sec. 5.1) as ONE persistent kernel whose
// CTAs claim work items in dependency order:
//   out[:, :, x] = scale * sum_c conj(S_c) F_yz^H M F_yz (S_c x)[:, :, x] + alpha * operand
// The readout axis x is never transformed (M is constant along it), so every
// x column is its own (z, y) problem.  The volume is cut into x-blocks of 16
// columns (128-byte rows of every map) and the coils into groups of CG; a
// phase k = (x-block b, coil group g) runs three kinds of item:
//   A (c, z):  y FFT of S_c x on z-plane z            -> W[c][z][ky][16]
//   B (c, ky): z FFT, mask M[kz][ky], z IFFT in place  on W[c][:, ky][16]
//   C (z):     y IFFT of W[c][z] for c in the group, times conj(S_c),
//              summed over the group in registers; added to the partial sum
//              of the earlier groups in `out` (the last group applies scale
//              and the Horner axpy epilogue)
// W holds two phases (slots k mod 2) and stays in L2 with the group's maps,
// which the C items re-read.  Items are numbered phase by phase (A, then B,
// then C, coil-major), and a CTA takes the next number from a global counter
// once it has finished its current item, so every item waits only on items
// with smaller numbers that running CTAs hold:
//   A(k, c, z) after C(k-2, z)  (slot reuse: plane z of the slot is free once
//                                that item, which itself waited for every
//                                B item of phase k-2, is done)
//   B(k, c)    after all A(k, c)
//   C(k, z)    after all B(k, c) of each coil c, and after C(k-1, z) (the
//              partial sum of plane z in `out`) when g > 0
// The cross-phase waits are per z plane, so consecutive coil groups of an
// x-block overlap instead of running their C items one group after another.
// The smallest unfinished number is therefore always runnable, and the HBM
// stream of phase k+1's maps (A items) overlaps phase k's transforms.
// Completion is counted per (phase, coil) with release atomics; a wait is an
// acquire poll bounded in time: past the limit the CTA records a timeout in
// the error word and every CTA leaves (the host reports PP_ERR_TIMEOUT).
// Data made by other items (W, the partial sums) is read with ld.global.cg
// (L2, never a stale L1 line).
// TMA variant: a block claims its next item while it starts the current one;
// when that next item is an A item, one thread issues a tensor-map bulk copy
// (cp.async.bulk.tensor, completion on an mbarrier) of its ny x 16 coil-map
// tile into the spare of two shared buffers, so the map's HBM stream overlaps
// the current item's transforms; the A item then reads the map from shared
// memory.  The mbarrier wait is bounded in time like the dependency waits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pp_fft4.cuh"
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int DN1 = 16;   // first factor of every register FFT
constexpr int DTX = 16;   // x columns per item
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s bound on one wait
constexpr int kClaimT = 32;   // the thread (warp 1) that claims items and issues tile copies

template <int N2Y, int N2Z> struct Df {
    static constexpr int NY = 16 * N2Y, NZ = 16 * N2Z;
    static constexpr int RMAX = (N2Y > N2Z ? (N2Y > DN1 ? N2Y : DN1) : (N2Z > DN1 ? N2Z : DN1));
    static constexpr int THREADS = DTX * RMAX;
    // ky lines per B item: as many as the thread rows hold in the z
    // transforms' first phase (N2Z rows each), so no row idles there
    static constexpr int LPB = (RMAX % N2Z == 0 && NY % (RMAX / N2Z) == 0) ? RMAX / N2Z : 1;
    static constexpr int YE = DN1 * RMAX * DTX;   // transpose buffer elements
    static constexpr size_t SMEM = sizeof(float2) * (YE + NY + NZ);
    // TMA variant: two ny x 16 map tiles after the above, 1024-byte aligned
    static constexpr size_t TILE = sizeof(float2) * NY * DTX;
    static constexpr size_t SOFF = (SMEM + 1023) / 1024 * 1024;
    static constexpr size_t SMEM_TMA = SOFF + 2 * TILE + 1024;   // + slack to align the base
    static constexpr size_t SMEM_TMA1 = SOFF + TILE + 1024;      // one tile buffer (three blocks per SM)
    static constexpr int BOXR = NY <= 256 ? NY : NY / 2;        // tensor-map box rows (<= 256)
};

struct DfArgs {
    const float2* x;
    const float2* S;
    float2* out;
    const float2* operand;
    float scale, alpha;
    const float* mask_fo;   // [nz][ny], FFT order, 1/(ny nz) folded in
    const float2* twy;
    const float2* twz;
    float2* W;              // 2 slots of CG * nz * ny * 16
    int* cnt;               // cntA[P*CG], cntB[P*CG], cntCz[P*NZ], next, err
    int nx, C, CG, ng, nb;
    int ma, mb;             // z planes per A item, LPB-line units per B item (1 or 2)
    int64_t slot;           // elements per slot
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// 2-D tensor-map tile load into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1),
                   "r"(smem_u32(bar))
                 : "memory");
}

// L2 residency.  W (two slots) is written and re-read four times per element
// within about one phase, while the maps stream through: W's accesses carry
// an evict_last policy, the C items' map reads (the maps' last use) an
// evict_first one.  kDfL2: 0 no hints, 1 W evict_last, 2 C maps evict_first,
// 3 both.
constexpr int kDfL2 = 2;
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
// W element store / load (L2 only, never L1: other blocks produce and consume W)
__device__ __forceinline__ void w_store(float2* p, float2 v, uint64_t pol) {
    if (kDfL2 & 1)
        asm volatile("st.global.cg.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;\n"
                     ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
    else
        __stcg(p, v);
}
__device__ __forceinline__ float2 w_load(const float2* p, uint64_t pol) {
    float2 v;
    if (kDfL2 & 1)
        asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;\n"
                     : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol) : "memory");
    else
        v = __ldcg(p);
    return v;
}
// read-only map element at its last use in the apply
__device__ __forceinline__ float2 s_load_last(const float2* p, uint64_t pol) {
    float2 v;
    if (kDfL2 & 2)
        asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;\n"
            : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    else
        v = __ldg(p);
    return v;
}

// the same with an L2 eviction policy (createpolicy) for the loaded lines
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar,
                                                 uint64_t pol) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1, {%2, %3}], [%4], %5;\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1),
                   "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}

// Block-wide: wait until *cnt >= target (thread 0 polls).  Returns false when
// the error word is set (by this wait's time limit or by another CTA).
__device__ __forceinline__ bool df_wait(const int* cnt, int target, int* err,
                                        unsigned long long limit_ns = kWaitNs) {
    int good = 1;
    if (threadIdx.x == 0) {
        if (ld_acquire(cnt) < target) {
            const unsigned long long t0 = gtimer();
            while (ld_acquire(cnt) < target) {
                if (*(volatile int*)err) {
                    good = 0;
                    break;
                }
                if (gtimer() - t0 > limit_ns) {
                    atomicExch(err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(200);
            }
        }
        if (good && *(volatile int*)err) good = 0;
    }
    return __syncthreads_and(good) != 0;
}

// Block-wide: the item's stores are done; count its v units (release).
__device__ __forceinline__ void df_signal(int* cnt, int v = 1) {
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(cnt, v);
}

template <int N2Y, int N2Z, int MB, bool TMA>
__global__ void __launch_bounds__(Df<N2Y, N2Z>::THREADS, MB)
c3_dataflow_kernel(DfArgs a, const __grid_constant__ CUtensorMap tmS) {
    constexpr int NY = Df<N2Y, N2Z>::NY, NZ = Df<N2Y, N2Z>::NZ, LPB = Df<N2Y, N2Z>::LPB;
    constexpr int NBI = NY / LPB;   // B items per coil
    // TMA tile buffers: two, or one when three blocks share an SM (the next
    // tile is then issued once the current one has been read)
    constexpr int NBUF = (TMA && MB >= 3) ? 1 : 2;
    extern __shared__ float4 df_sm4[];
    float2* Y = reinterpret_cast<float2*>(df_sm4);
    float2* twy = Y + Df<N2Y, N2Z>::YE;
    float2* twz = twy + NY;
    __shared__ int s_item;
    __shared__ unsigned s_bdone;   // C item: coils of the group whose B items were all done at its start
    // TMA variant: two map-tile buffers (1024-byte aligned), their mbarriers,
    // the item each holds (-1: none) and each barrier's phase
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_pref[2], s_pending[2];
    float2* Sb = nullptr;
    if (TMA) {
        const uint32_t base = smem_u32(df_sm4) + (uint32_t)Df<N2Y, N2Z>::SOFF;
        Sb = reinterpret_cast<float2*>(reinterpret_cast<char*>(df_sm4) + Df<N2Y, N2Z>::SOFF +
                                       ((1024u - (base & 1023u)) & 1023u));
        if (threadIdx.x == 0) {
            mbar_init(&s_bar[0]);
            mbar_init(&s_bar[1]);
            s_pref[0] = s_pref[1] = -1;
            s_pending[0] = s_pending[1] = 0;
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    uint32_t phase[2] = {0u, 0u};
    int iter = 0;
    const uint64_t pol_w = l2_policy_last(), pol_s = l2_policy_first();
    for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = a.twy[i];
    for (int i = threadIdx.x; i < NZ; i += blockDim.x) twz[i] = a.twz[i];
    const int lane = threadIdx.x % DTX, r = threadIdx.x / DTX;
    const int P = a.nb * a.ng;
    int* cntA = a.cnt;
    int* cntB = cntA + (int64_t)P * a.CG;
    int* cntCz = cntB + (int64_t)P * a.CG;   // [phase][z]: C item done
    int* next = cntCz + (int64_t)P * NZ;
    int* err = next + 1;
    const int cg_last = a.C - (a.ng - 1) * a.CG;
    // items per coil: NA A items of ma planes, NBm B items of mb line units
    // (the counters count planes and units, so their targets do not change)
    const int NA = NZ / a.ma, NBm = NBI / a.mb;
    const int per_full = a.CG * (NA + NBm) + NZ;
    const int per_last = cg_last * (NA + NBm) + NZ;
    const int per_blk = (a.ng - 1) * per_full + per_last;
    const int total = a.nb * per_blk;
    const int64_t plane = (int64_t)NY * a.nx, vol = (int64_t)NZ * plane;
    if (threadIdx.x == kClaimT) s_item = atomicAdd(next, 1);
    __syncthreads();
    // TMA: the A item `it` (if it is one) -> its map tile's coordinates
    auto a_tile = [&](int it, int* cx, int* cy) -> bool {
        if (it >= total) return false;
        const int bb = it / per_blk;
        int q = it - bb * per_blk;
        const int gg = min(q / per_full, a.ng - 1);
        q -= gg * per_full;
        const int cgg = (gg == a.ng - 1) ? cg_last : a.CG;
        if (q >= cgg * NA) return false;
        const int cc = q / NA, zz = (q - cc * NA) * a.ma;
        *cx = bb * DTX;
        *cy = ((gg * a.CG + cc) * NZ + zz) * NY;
        return true;
    };
    // one thread: load the map tile at (cx, cy) into buffer buf; `tag` is
    // the A item it serves (-2: a coil of a C item, the maps' last use)
    auto issue_at = [&](int buf, int cx, int cy, int tag) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier reads of the buffer
        mbar_expect_tx(&s_bar[buf], (uint32_t)Df<N2Y, N2Z>::TILE);
        for (int h = 0; h < NY / Df<N2Y, N2Z>::BOXR; ++h) {
            float2* dst = Sb + buf * NY * DTX + h * Df<N2Y, N2Z>::BOXR * DTX;
            if (tag == -2 && (kDfL2 & 2))
                tma_load_2d_hint(dst, &tmS, cx, cy + h * Df<N2Y, N2Z>::BOXR, &s_bar[buf], pol_s);
            else
                tma_load_2d(dst, &tmS, cx, cy + h * Df<N2Y, N2Z>::BOXR, &s_bar[buf]);
        }
        s_pref[buf] = tag;
        s_pending[buf] = 1;
    };
    auto issue = [&](int it, int buf) {   // one thread
        int cx, cy;
        if (a_tile(it, &cx, &cy)) issue_at(buf, cx, cy, it);
    };
    // block-wide: the tile in buffer buf has landed (bounded wait); false on
    // a timeout (error word set)
    auto tile_wait = [&](int buf) -> bool {
        int good = 1;
        if (threadIdx.x == 0) {
            if (!mbar_try_wait(&s_bar[buf], phase[buf])) {
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(&s_bar[buf], phase[buf])) {
                    if (gtimer() - t0 > kWaitNs) {
                        atomicExch(err, 1);
                        good = 0;
                        break;
                    }
                }
            }
        }
        if (!__syncthreads_and(good)) return false;
        mbar_try_wait(&s_bar[buf], phase[buf]);   // this thread's acquire of the tile
        phase[buf] ^= 1u;
        if (threadIdx.x == 0) s_pending[buf] = 0;
        return true;
    };
    for (;;) {
        const int item = s_item;
        // block-uniform stop test; the barrier also ends every read of s_item
        if (__syncthreads_or(item >= total || (threadIdx.x == 0 && *(volatile int*)err))) break;
        // ---- decode (x-block b, group g, kind, index)
        const int b = item / per_blk;
        int rr = item - b * per_blk;
        const int g = min(rr / per_full, a.ng - 1);
        rr -= g * per_full;
        const int k = b * a.ng + g;
        const int cg = (g == a.ng - 1) ? cg_last : a.CG;
        const bool a_item = rr < cg * NA, c_item = rr >= cg * (NA + NBm);
        const int cur_buf = NBUF == 2 ? (iter & 1) : 0;
        // the claim and the tile copies are issued by warp 1, so that their
        // round trips overlap thread 0's dependency polls
        if (threadIdx.x == kClaimT) {
            if (TMA && s_pref[cur_buf] != item) issue(item, cur_buf);   // not prefetched: load it now
            // claim the next item early (its map tile streams in meanwhile),
            // except under a C item: that one runs for the whole coil group,
            // and an item claimed that early would hold up its dependants
            if (!c_item) {
                const int nxt = atomicAdd(next, 1);
                s_item = nxt;
                // the next item's map tile, if it is an A item: into the spare
                // buffer, or with one buffer only when this item holds none
                if (TMA && (NBUF == 2 || !a_item)) issue(nxt, cur_buf ^ (NBUF - 1));
            }
        }
        ++iter;
        const int c0 = g * a.CG;
        const int x0 = b * DTX, col = x0 + lane;
        const bool ok = col < a.nx;
        float2* Wk = a.W + (k & 1) * a.slot;
        if (rr < cg * NA) {
            // ---- A (c, z .. z + ma - 1): y FFT of S_c x on each plane -> W[c][z][ky]
            const int c = rr / NA, z0 = (rr - c * NA) * a.ma;
            bool fail = false;
            for (int j = 0; j < a.ma; ++j) {
                const int z = z0 + j;
                const float2* Sc = a.S + (int64_t)(c0 + c) * vol + (int64_t)z * plane;
                const float2* xz = a.x + (int64_t)z * plane;
                // the image is read-only in the apply: its loads go out before the
                // slot-reuse wait, which only orders this item's W stores
                float2 xv[DN1];
#pragma unroll
                for (int m1 = 0; m1 < DN1; ++m1)
                    xv[m1] = (r < N2Y && ok) ? __ldg(xz + (int64_t)(N2Y * m1 + r) * a.nx + col) : make_float2(0.f, 0.f);
                if (k >= 2 && !df_wait(cntCz + (int64_t)(k - 2) * NZ + z, 1, err)) {
                    fail = true;
                    break;
                }
                const float2* St = nullptr;
                if (TMA) {
                    // the tile is in Sb[cur_buf] (issued now or one item ago; TMA
                    // launches take one plane per A item)
                    if (!tile_wait(cur_buf)) {
                        fail = true;
                        break;
                    }
                    St = Sb + cur_buf * NY * DTX;
                }
                if (r < N2Y) {
                    float2 v[DN1];
#pragma unroll
                    for (int m1 = 0; m1 < DN1; ++m1) {
                        const int64_t o = (int64_t)(N2Y * m1 + r) * a.nx + col;
                        const float2 sv = TMA ? St[(N2Y * m1 + r) * DTX + lane] : (ok ? __ldg(Sc + o) : make_float2(0.f, 0.f));
                        v[m1] = ok ? cmul(sv, xv[m1]) : make_float2(0.f, 0.f);
                    }
                    fft4_phase1<DN1, N2Y, false>(v, r, twy);
#pragma unroll
                    for (int k1 = 0; k1 < DN1; ++k1) Y[(k1 * N2Y + r) * DTX + lane] = v[k1];
                }
                __syncthreads();
                // one buffer: the tile has been read, so the next item's may land
                if (TMA && NBUF == 1 && threadIdx.x == kClaimT) issue(s_item, 0);
                if (r < DN1) {
                    float2 u[N2Y];
#pragma unroll
                    for (int m2 = 0; m2 < N2Y; ++m2) u[m2] = Y[(r * N2Y + m2) * DTX + lane];
                    fft4_phase2<DN1, N2Y, false>(u, twy);
                    float2* Wz = Wk + ((int64_t)(c * NZ + z) * NY) * DTX + lane;
#pragma unroll
                    for (int k2 = 0; k2 < N2Y; ++k2) w_store(Wz + (r + DN1 * k2) * DTX, u[k2], pol_w);
                }
                if (j + 1 < a.ma) __syncthreads();   // Y is rewritten by the next plane
            }
            if (fail) break;
            df_signal(cntA + (int64_t)k * a.CG + c, a.ma);
        } else if (rr < cg * (NA + NBm)) {
            // ---- B (c, mb units of LPB ky lines): z FFT, mask, z IFFT of
            // W[c][:, ky] in place; thread row r < LPB N2Z takes line r / N2Z in
            // the first and last phase, rows r < 16 loop over the lines in the
            // middle one
            const int q = rr - cg * NA;
            const int c = q / NBm, u0 = (q - c * NBm) * a.mb;
            if (!df_wait(cntA + (int64_t)k * a.CG + c, NZ, err)) break;
            for (int j = 0; j < a.mb; ++j) {
                const int ky0 = (u0 + j) * LPB;
                constexpr int ZS = NY * DTX;
                constexpr int YL = DN1 * N2Z * DTX;   // one line's transpose block
                const int l1 = r / N2Z, m2r = r - l1 * N2Z;
                float2* Wc = Wk + (int64_t)c * NZ * NY * DTX + lane;
                if (r < LPB * N2Z) {
                    const float2* Wl = Wc + (ky0 + l1) * DTX;
                    float2 v[DN1];
#pragma unroll
                    for (int m1 = 0; m1 < DN1; ++m1) v[m1] = w_load(Wl + (int64_t)(N2Z * m1 + m2r) * ZS, pol_w);
                    fft4_phase1<DN1, N2Z, false>(v, m2r, twz);
#pragma unroll
                    for (int k1 = 0; k1 < DN1; ++k1) Y[l1 * YL + (k1 * N2Z + m2r) * DTX + lane] = v[k1];
                }
                __syncthreads();
                if (r < DN1) {
#pragma unroll 1
                    for (int l = 0; l < LPB; ++l) {
                        float2 u[N2Z];
#pragma unroll
                        for (int m2 = 0; m2 < N2Z; ++m2) u[m2] = Y[l * YL + (r * N2Z + m2) * DTX + lane];
                        fft4_phase2<DN1, N2Z, false>(u, twz);
                        const int ky = ky0 + l;
#pragma unroll
                        for (int k2 = 0; k2 < N2Z; ++k2)
                            u[k2] = cscale(u[k2], __ldg(a.mask_fo + (r + DN1 * k2) * NY + ky));
                        // inverse with the mirrored decomposition: length-N2Z DFT over
                        // k2, twiddle W_nz^(-m2 k1), then the length-16 DFT over k1;
                        // this thread reads and writes only its own row r of the block
                        RegFft<N2Z, true>::run(u, twz, DN1);
#pragma unroll
                        for (int m2 = 1; m2 < N2Z; ++m2) {
                            float2 w = twz[m2 * r];
                            w.y = -w.y;
                            u[m2] = cmul(u[m2], w);
                        }
#pragma unroll
                        for (int m2 = 0; m2 < N2Z; ++m2) Y[l * YL + (r * N2Z + m2) * DTX + lane] = u[m2];
                    }
                }
                __syncthreads();
                if (r < LPB * N2Z) {
                    float2* Wl = Wc + (ky0 + l1) * DTX;
                    float2 v[DN1];
#pragma unroll
                    for (int k1 = 0; k1 < DN1; ++k1) v[k1] = Y[l1 * YL + (k1 * N2Z + m2r) * DTX + lane];
                    RegFft<DN1, true>::run(v, twz, N2Z);
#pragma unroll
                    for (int m1 = 0; m1 < DN1; ++m1) w_store(Wl + (int64_t)(N2Z * m1 + m2r) * ZS, v[m1], pol_w);
                }
                if (j + 1 < a.mb) __syncthreads();   // Y is rewritten by the next unit
            }
            df_signal(cntB + (int64_t)k * a.CG + c, a.mb);
        } else {
            // ---- C (z): y IFFT, conj(S_c), sum over the group, partial sum
            const int z = rr - cg * (NA + NBm);
            float2 acc[N2Y];
#pragma unroll
            for (int k2 = 0; k2 < N2Y; ++k2) acc[k2] = make_float2(0.f, 0.f);
            bool alive = true;
            // TMA: coil c's map tile goes to buffer cur_buf ^ (c & 1), coil
            // c + 1's is issued before coil c is transformed (no item was
            // claimed ahead, so both buffers are free)
            if (TMA && threadIdx.x == 0) issue_at(cur_buf, x0, (c0 * NZ + z) * NY, -2);
            // the group's B counters are read once, in parallel (one acquire per
            // coil by warp 0, published by the barrier); only coils still
            // running their B items are waited for one by one
            if (threadIdx.x < 32) {
                const bool done =
                    (int)threadIdx.x < cg && ld_acquire(cntB + (int64_t)k * a.CG + threadIdx.x) >= NBI;
                const unsigned m = __ballot_sync(0xffffffffu, done);
                if (threadIdx.x == 0) s_bdone = m;
            }
            __syncthreads();
            for (int c = 0; c < cg; ++c) {
                if (!((s_bdone >> c) & 1u) && !df_wait(cntB + (int64_t)k * a.CG + c, NBI, err)) {
                    alive = false;
                    break;
                }
                const int cb = NBUF == 2 ? (cur_buf ^ (c & 1)) : 0;
                if (TMA && NBUF == 2 && threadIdx.x == 0 && c + 1 < cg)
                    issue_at(cb ^ 1, x0, ((c0 + c + 1) * NZ + z) * NY, -2);
                const float2* Wz = Wk + ((int64_t)(c * NZ + z) * NY) * DTX + lane;
                if (r < N2Y) {
                    float2 v[DN1];
#pragma unroll
                    for (int m1 = 0; m1 < DN1; ++m1) v[m1] = w_load(Wz + (N2Y * m1 + r) * DTX, pol_w);
                    fft4_phase1<DN1, N2Y, true>(v, r, twy);
#pragma unroll
                    for (int k1 = 0; k1 < DN1; ++k1) Y[(k1 * N2Y + r) * DTX + lane] = v[k1];
                }
                if (TMA) {
                    if (!tile_wait(cb)) {   // also the barrier before Y is read
                        alive = false;
                        break;
                    }
                } else {
                    __syncthreads();
                }
                if (r < DN1 && ok) {
                    float2 u[N2Y];
#pragma unroll
                    for (int m2 = 0; m2 < N2Y; ++m2) u[m2] = Y[(r * N2Y + m2) * DTX + lane];
                    fft4_phase2<DN1, N2Y, true>(u, twy);
                    if (TMA) {
                        const float2* St = Sb + cb * NY * DTX + lane;
#pragma unroll
                        for (int k2 = 0; k2 < N2Y; ++k2)
                            acc[k2] = cadd(acc[k2], cmulc(St[(r + DN1 * k2) * DTX], u[k2]));
                    } else {
                        const float2* Sc = a.S + (int64_t)(c0 + c) * vol + (int64_t)z * plane + col;
#pragma unroll
                        for (int k2 = 0; k2 < N2Y; ++k2)
                            acc[k2] = cadd(acc[k2], cmulc(s_load_last(Sc + (int64_t)(r + DN1 * k2) * a.nx, pol_s), u[k2]));
                    }
                }
                __syncthreads();   // Y and the tile buffer are rewritten by the next coil
                if (TMA && NBUF == 1 && threadIdx.x == 0 && c + 1 < cg)
                    issue_at(0, x0, ((c0 + c + 1) * NZ + z) * NY, -2);
            }
            if (!alive) break;
            if (g > 0 && !df_wait(cntCz + (int64_t)(k - 1) * NZ + z, 1, err)) break;
            if (r < DN1 && ok) {
                float2* oz = a.out + (int64_t)z * plane + col;
                const bool last = g == a.ng - 1;
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) {
                    const int64_t o = (int64_t)(r + DN1 * k2) * a.nx;
                    float2 v = acc[k2];
                    if (g > 0) v = cadd(v, __ldcg(oz + o));
                    if (last) {
                        v = cscale(v, a.scale);
                        if (a.operand) v = cadd(v, cscale(__ldg(a.operand + (int64_t)z * plane + col + o), a.alpha));
                    }
                    __stcg(oz + o, v);
                }
            }
            df_signal(cntCz + (int64_t)k * NZ + z);
            if (threadIdx.x == kClaimT) s_item = atomicAdd(next, 1);   // the claim, made late
        }
        __syncthreads();   // s_item (the claim made at the top, or after a C item) is visible
    }
    if (TMA && threadIdx.x == 0) {
        // after an early exit, wait (bounded) for this block's copies still in flight
        for (int b2 = 0; b2 < NBUF; ++b2) {
            if (!s_pending[b2]) continue;
            const unsigned long long t0 = gtimer();
            while (!mbar_try_wait(&s_bar[b2], phase[b2]) && gtimer() - t0 < kWaitNs) {
            }
        }
    }
}

template <int N2Y, int N2Z, int MB, bool TMA> constexpr size_t df_smem() {
    return TMA ? (MB >= 3 ? Df<N2Y, N2Z>::SMEM_TMA1 : Df<N2Y, N2Z>::SMEM_TMA) : Df<N2Y, N2Z>::SMEM;
}

template <int N2Y, int N2Z, int MB, bool TMA>
int df_resident() {
    auto fn = c3_dataflow_kernel<N2Y, N2Z, MB, TMA>;
    const size_t smem = df_smem<N2Y, N2Z, MB, TMA>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, Df<N2Y, N2Z>::THREADS, smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

// One block waits for a counter that nothing increments: the bounded wait
// must give up after limit_ns and leave the error word set.
__global__ void selftest_wait_kernel(int* words, unsigned long long limit_ns) {
    df_wait(words, 1, words + 1, limit_ns);
}

}  // namespace

extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

#define PP_DF_CASES(X) X(8, 8) X(12, 8) X(16, 8) X(20, 8) X(24, 8) \
    X(8, 12) X(12, 12) X(16, 12) X(8, 16) X(12, 16) X(16, 16)

// Blocks per SM the kernel is compiled for: variant 0 leaves the registers
// of two 256-thread blocks per SM, variant 1 of three (fewer registers, a
// few spilled, more warps to cover latency); larger blocks get one.
template <int N2Y, int N2Z> constexpr int df_mb(int v) {
    return Df<N2Y, N2Z>::THREADS <= 256 ? (v ? 3 : 2) : 1;
}

template <int N2Y, int N2Z, int MB, bool TMA>
cudaError_t df_launch(int grid, cudaStream_t st, const DfArgs& a, const CUtensorMap& tm) {
    return launch_ex(c3_dataflow_kernel<N2Y, N2Z, MB, TMA>, dim3(grid), dim3(Df<N2Y, N2Z>::THREADS),
                     df_smem<N2Y, N2Z, MB, TMA>(), st, false, 0, a, tm);
}
// variant v of the kernel for (N2Y, N2Z): the numbering of c3df_prepare
template <int N2Y, int N2Z>
cudaError_t df_launch_v(int v, int grid, cudaStream_t st, const DfArgs& a, const CUtensorMap& tm) {
    constexpr int m0 = df_mb<N2Y, N2Z>(0), m1 = df_mb<N2Y, N2Z>(1);
    switch (v) {
        case 3: return df_launch<N2Y, N2Z, m1, true>(grid, st, a, tm);
        case 2: return df_launch<N2Y, N2Z, m0, true>(grid, st, a, tm);
        case 1: return df_launch<N2Y, N2Z, m1, false>(grid, st, a, tm);
        default: return df_launch<N2Y, N2Z, m0, false>(grid, st, a, tm);
    }
}

// Resident CTAs of the dataflow kernel (variant v: 0 two blocks per SM, 1
// three, 2 TMA-staged map tiles in two buffers, 3 TMA-staged tiles in one
// buffer with three blocks per SM) for this plan's (ny, nz), 0 when the
// kernel does not apply (a length without a register FFT).
int c3df_prepare(const Plan& p, int v) {
    if (p.kind != PP_CARTESIAN || p.ndim != 3) return 0;
    const int n2y = fft4_n2(p.ny), n2z = fft4_n2(p.nz);
#define PP_DF_PREP(Y_, Z_)                                                           \
    if (n2y == Y_ && n2z == Z_)                                                      \
        return v == 3   ? df_resident<Y_, Z_, df_mb<Y_, Z_>(1), true>()              \
               : v == 2 ? df_resident<Y_, Z_, df_mb<Y_, Z_>(0), true>()              \
               : v      ? df_resident<Y_, Z_, df_mb<Y_, Z_>(1), false>()             \
                        : df_resident<Y_, Z_, df_mb<Y_, Z_>(0), false>();
    PP_DF_CASES(PP_DF_PREP)
#undef PP_DF_PREP
    return 0;
}

// The coil maps as a 2-D tensor map for the TMA variant: [C nz ny] rows of nx
// 8-byte elements, boxes of 16 columns x BOXR rows (BOXR = ny, or ny/2 when
// ny > 256); columns past nx read as zero.  false when the driver entry
// point or the encoding is unavailable (the variant is then not offered).
bool c3df_make_tensor_map(Plan& p) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    if ((p.nx * 8) % 16 || ((uintptr_t)p.sens & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)p.nx, (cuuint64_t)p.C * p.nz * p.ny};
    const cuuint64_t strides[1] = {(cuuint64_t)p.nx * 8};
    const cuuint32_t box[2] = {(cuuint32_t)DTX, (cuuint32_t)(p.ny <= 256 ? p.ny : p.ny / 2)};
    const cuuint32_t estr[2] = {1, 1};
    if (box[1] > 256 || p.ny % box[1]) return false;
    const CUresult r = reinterpret_cast<Encode>(fn)(
        &p.c3df_tmS, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2*>(p.sens), dims, strides, box,
        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t c3df_slot_elems(const Plan& p, int cg) { return (size_t)cg * p.nz * p.ny * DTX; }
size_t c3df_counter_ints(const Plan& p, int cg) {
    const int nb = (p.nx + DTX - 1) / DTX, ng = (p.C + cg - 1) / cg;
    return (size_t)nb * ng * (2 * (size_t)cg + p.nz) + 2;
}

pp_status c3df_normal(const Plan& p, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st) {
    const int cg = std::max(1, std::min(p.c3df_cg, p.C));
    DfArgs a;
    a.x = x; a.S = p.sens; a.out = out; a.operand = operand; a.scale = scale; a.alpha = alpha;
    a.mask_fo = p.mask_fo; a.twy = p.fy.tw; a.twz = p.fz.tw;
    a.W = p.c3df_w; a.cnt = p.c3df_cnt;
    a.nx = p.nx; a.C = p.C; a.CG = cg; a.ng = (p.C + cg - 1) / cg; a.nb = (p.nx + DTX - 1) / DTX;
    a.slot = (int64_t)c3df_slot_elems(p, cg);
    // variants 4 and 5: variants 0 and 1 with two planes per A item and two
    // line units per B item (half the items, each twice the work)
    const int v = p.c3df_hi >= 4 ? p.c3df_hi - 4 : p.c3df_hi;
    a.ma = a.mb = p.c3df_hi >= 4 ? 2 : 1;
    if ((size_t)2 * a.slot > p.c3df_w_elems || c3df_counter_ints(p, cg) > p.c3df_cnt_ints) {
        set_error("c3df_normal: coil group %d exceeds the plan's dataflow buffers", cg);
        return PP_ERR_INVALID_ARG;
    }
    PP_TRY_CUDA(cudaMemsetAsync(p.c3df_cnt, 0, sizeof(int) * c3df_counter_ints(p, cg), st));
    const int n2y = fft4_n2(p.ny), n2z = fft4_n2(p.nz);
    const int per_full = cg * (p.nz + p.ny) + p.nz;   // an upper bound on the items of a phase
    const int64_t total = (int64_t)a.nb * a.ng * per_full;
    const int ctas = v == 3 ? p.c3df_ctas_tma1 : v == 2 ? p.c3df_ctas_tma : (v ? p.c3df_ctas_hi : p.c3df_ctas);
    if (ctas <= 0) {
        set_error("c3df_normal: this dataflow variant cannot be resident on the device");
        return PP_ERR_UNSUPPORTED;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, total));
    cudaError_t e = cudaErrorInvalidValue;
#define PP_DF_LAUNCH(Y_, Z_) \
    if (n2y == Y_ && n2z == Z_) e = df_launch_v<Y_, Z_>(v, grid, st, a, p.c3df_tmS);
    PP_DF_CASES(PP_DF_LAUNCH)
#undef PP_DF_LAUNCH
    if (e != cudaSuccess) return cuda_status(e, "c3_dataflow_kernel launch");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "c3_dataflow_kernel");
    ++g_launches;
    if (g_profiler) g_profiler->mark("c3_dataflow_kernel");
    return PP_OK;
}

// The error word of the last dataflow launch (host, after a synchronisation):
// nonzero when a wait ran out of time.
pp_status c3df_check(const Plan& p, cudaStream_t st) {
    if (!p.c3df_cnt) return PP_OK;
    int errw = 0;
    const int cg = std::max(1, std::min(p.c3df_cg, p.C));
    const size_t off = c3df_counter_ints(p, cg) - 1;
    PP_TRY_CUDA(cudaMemcpyAsync(&errw, p.c3df_cnt + off, sizeof(int), cudaMemcpyDeviceToHost, st));
    PP_TRY_CUDA(cudaStreamSynchronize(st));
    if (errw) {
        set_error("3-D normal operator: a dependency wait ran past its time limit");
        return PP_ERR_TIMEOUT;
    }
    return PP_OK;
}

}  // namespace pp

namespace pp {

pp_status selftest_wait(long long limit_ns, cudaStream_t st) {
    int* words = nullptr;
    PP_TRY_CUDA(cudaMalloc(&words, 2 * sizeof(int)));
    pp_status rc = PP_OK;
    int h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(words, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        selftest_wait_kernel<<<1, 32, 0, st>>>(words, (unsigned long long)limit_ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, words, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e, "selftest_wait_kernel");
    cudaFree(words);
    if (rc != PP_OK) return rc;
    ++g_launches;
    if (h[1]) {
        set_error("pp_selftest_wait: the wait gave up after its limit (counter %d, expected 1)", h[0]);
        return PP_ERR_TIMEOUT;
    }
    return PP_OK;
}

}  // namespace pp
