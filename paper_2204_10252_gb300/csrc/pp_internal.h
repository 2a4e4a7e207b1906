// Internal declarations shared by the libpp translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pp.h"
#include "pp_fft.cuh"

namespace pp {

void set_error(const char* fmt, ...);
pp_status cuda_status(cudaError_t e, const char* what);

#define PP_TRY_CUDA(call)                                         \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return ::pp::cuda_status(_e, #call); \
    } while (0)
#define PP_TRY(call)                          \
    do {                                      \
        pp_status _s = (call);                \
        if (_s != PP_OK) return _s;           \
    } while (0)

constexpr int kThreads = 256;

// Programmatic dependent launch.  A kernel launched with
// launch_ex(..., pdl = true) may be scheduled while its predecessor in the
// stream is still running; it runs its independent prologue (plan constants
// only), then pdl_wait() blocks until the predecessor has completed and its
// writes are visible, before any access to data that other kernels write.
// pdl_trigger() lets this grid's own successor be scheduled.  Both are no-ops
// for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// cudaLaunchKernelEx with optional programmatic stream serialization and an
// optional 1-D cluster of `cluster_x` CTAs (0: none).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t st, bool pdl, int cluster_x, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (cluster_x > 0) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = cluster_x;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Device FFT: stage plan plus the table w^t = exp(-2 pi i t / n), t < n.
struct DevFft {
    FftDesc d;
    float2* tw = nullptr;
};

// One (tile, sample) pair of the gridding tile lists.  Taps of the sample are
// at halo rows ly0 .. ly0+W-1 and columns lx0 .. lx0+W-1, where halo row 0
// is grid row ty0 - H (H = W-1 the halo width) of the tile starting at ty0.
struct TileEntry {
    float4 wx;   // x-tap weights a = 0..3 (unused taps are 0)
    float4 wy;   // y-tap weights
    int lyx;     // ly0 | (lx0 << 16)
    int k;       // sample index (trajectory order)
};

// Per-sample gridding metadata in trajectory order.
struct SampleTaps {
    float4 wx;
    float4 wy;
    int iy0, ix0;   // first tap's grid index (unwrapped; wrap mod G)
};

// Row stage: per row, FFT along the contiguous axis between an image row of
// length n and a k-space row of length G, with circular placement
// pos = (i - off) mod G.
struct RowArgs {
    int n;          // image row length
    int G;          // transform length (>= n)
    int off_in;     // input index i -> transform position (i - off_in) mod G
    int off_out;    // output index q <- transform position (q - off_out) mod G
    int nrows;      // rows per coil
    int64_t coil_img_stride;   // elements between coils in the sensitivity array (0 = none)
    float scale;
};

struct ColArgs {
    int Hin, Hout, G;
    int off_in, off_out;
    int ncols;                  // columns (contiguous axis length)
    int64_t in_batch_stride;    // elements between batches (coils) in src
    int64_t out_batch_stride;
    int nbatch;
    float scale;
    const float* mul_in;        // input multiplier: mul_in[r * mi_q + (col / mi_cdiv) * mi_c]
    int mi_q, mi_c, mi_cdiv;
    const float* mul_out;       // mask value for output row q and column col:
                                // mul_out[q * mo_q + (col / mo_cdiv) * mo_c]
    int mo_q, mo_c, mo_cdiv;
};

struct Plan {
    int ndim = 2, nx = 0, ny = 0, nz = 1, C = 0, kind = PP_CARTESIAN;
    int64_t nimg = 0, nksp = 0;
    const float2* sens = nullptr;
    double L = 1.0;
    int dev = 0;

    // FFTs
    DevFft fx, fy, fz, gx, gy;

    // Cartesian masks: centred order (forward/adjoint) and FFT order with the
    // 1/n normalisation folded in (normal operator round trip).
    float* mask_c = nullptr;    // 2-D: [ny]; 3-D: [nz][ny]
    float* mask_fo = nullptr;   // same shape, FFT order, times 1/(ny nz)

    // Non-Cartesian
    int G_x = 0, G_y = 0, W = 0, K = 0, T = 32, ntx = 0, nty = 0;
    float* deapod_x = nullptr;   // [nx] 1/(sqrt(nx) psi_x)
    float* deapod_y = nullptr;   // [ny]
    TileEntry* tiles = nullptr;
    int* tile_start = nullptr;   // [ntiles + 1]
    int max_tile_len = 0;
    SampleTaps* samp = nullptr;  // [K]
    float* gtg = nullptr;        // [(2W-1)^2][G_y][G_x] stencil of G^T G
    float* gtg8 = nullptr;       // the same weights as [G_y][ceil(G_x/8)][(2W-1)^2][8]
    // coil-innermost pipeline ([row][col][32 coils]; ci_a/b/c alias wk_a/b/c when C = 32)
    float2* ci_sens = nullptr;   // [ny][nx][32]
    float2 *ci_a = nullptr, *ci_b = nullptr, *ci_c = nullptr;
    int* ci_tile_nz = nullptr;   // per 16 x 8 stencil tile: any G^T G weight nonzero
    float2* ci_part = nullptr;   // [4][ny][nx] coil-block partial sums
    // Toeplitz-embedded normal operator (exact F^H F on the 2ny x 2nx circulant)
    int toep = 0;                // 1: the normal operator takes the Toeplitz path
    DevFft tx, ty;               // length-2nx / 2ny twiddle tables
    DevFft toep_hx, toep_hy;     // length-nx / ny tables (two half-length transforms)
    float* toep_T = nullptr;     // [2nx][2ny] kernel spectrum, column-major, 1/(n M) folded in
    float2 *toep_a = nullptr, *toep_b = nullptr;   // [ny][2nx][32] row-transformed arrays

    // Workspace
    float2* wk_a = nullptr;   // C * ny * G_x (rows) or C * n (Cartesian)
    float2* wk_b = nullptr;   // C * G_y * G_x (grid)
    float2* wk_c = nullptr;   // C * G_y * G_x (grid)
    float2 *z = nullptr, *y = nullptr, *g = nullptr, *u = nullptr, *t = nullptr, *ahb = nullptr,
           *v = nullptr, *w3 = nullptr;
    double* red = nullptr;    // reduction partials
    double* scal = nullptr;   // device scalars: [0] |b|^2, [1] rayleigh, [2] |w|^2, [3..] history
    int red_blocks = 0;
    int hist_cap = 0;
    double* hist = nullptr;   // [hist_cap][3]
    int64_t graph_kernels = 0;

    // Graph cache for the solve loop
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<double> gkey;

    bool external_wk = false;   // workspace supplied by an owner (batched plans)
    // plan-time autotuned launch shapes (0 = default)
    int tune_rows_adj_cl = 0;   // row-IFFT variant: cluster size 1, 2 or 4, or -1 = split
                                // into per-coil IFFTs plus a coil sum (normal operator only)
    int tune_stencil_kind = 0;  // G^T G stencil kernel: 0 one output per thread, 1 two,
                                // 2..5 register-blocked (R x CG = 4x4, 8x4, 4x8, 2x8),
                                // 6 coil-lane, 7 / 8 / 9 coil-innermost pipeline with
                                // a 1- / 2-row coil-lane or a coil-pair stencil
    int tune_stencil_cpc = 0;   // coils per CTA of kinds 0 and 1
    int stencil_rb_grid[4] = {0, 0, 0, 0};   // persistent grid of kinds 2..5 (0: unavailable)
    int c3cl_clusters = 0;      // 3-D: resident 16-CTA clusters of the one-kernel operator, 4 columns
    int c3cl2_clusters = 0;     //      the same with 2 columns per task (0: n/a)
    // 3-D dataflow operator (one persistent kernel per apply, pp_cart3d_df.cu)
    int c3df_ctas = 0;          // resident CTAs (0: not available for this plan)
    int c3df_ctas_hi = 0;       //   the same for the variant with three blocks per SM
    int c3df_ctas_tma = 0;      //   the same for the variant that stages map tiles by TMA
    int c3df_ctas_tma1 = 0;     //   ... by TMA into one buffer, three blocks per SM
    int c3df_hi = 0;            // variant: 0 two blocks per SM, 1 three, 2 TMA-staged map tiles,
                                // 3 TMA-staged tiles in one buffer with three blocks per SM
    CUtensorMap c3df_tmS;       // the coil maps as a 2-D tensor [C nz ny][nx] of 8-byte elements
    int c3df_cg = 4;            // coils per group
    float2* c3df_w = nullptr;   // two phase slots
    size_t c3df_w_elems = 0;
    int* c3df_cnt = nullptr;    // completion counters, claim counter, error word
    size_t c3df_cnt_ints = 0;
    int tune_c3 = 0;            // 3-D: 0 = three passes per coil, 1 / 2 = one-kernel cluster operator
                                //      with 4 / 2 columns per task
    int pdl = 1;                // programmatic dependent launch in the solve's kernel chain
    int tune_c2 = 1;            // 2-D Cartesian: CTAs per 8-column group (coils split over a cluster)
    std::vector<void*> allocs;
};

// Records a CUDA event after every kernel launch (see check_launch) so that
// consecutive events bracket one kernel each.
struct Profiler {
    cudaStream_t st = nullptr;
    std::vector<std::string> names;
    std::vector<cudaEvent_t> events;
    void mark(const char* what) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, st);
        names.push_back(what);
        events.push_back(e);
    }
};
extern thread_local int64_t g_launches;
extern thread_local Profiler* g_profiler;

// ---- launchers (pp_kernels.cu) -------------------------------------------
pp_status configure_kernels();
// register four-step FFT stages (pp_kernels4.cu); *done = false when the
// transform length has no register kernel
pp_status launch_cols4(const DevFft& f, const ColArgs& a, const float2* src, float2* dst, bool inv,
                       cudaStream_t st, bool* done);
pp_status launch_rows4_fwd(const DevFft& f, const RowArgs& a, const float2* x, const float2* sens,
                           const float* wrow, const float* wcol, float2* out, int ncoils,
                           int64_t img_batch_stride, cudaStream_t st, bool* done);
pp_status launch_rows4_adj_split(const DevFft& f, const RowArgs& a, const float2* src,
                                 const float2* sens, const float* wrow, const float* wcol,
                                 float2* contrib, float2* out, const float2* operand, float alpha,
                                 int ncoils, cudaStream_t st, bool* done);
pp_status cart3d4_normal(const Plan& p, const float2* x, float2* out, float scale,
                         const float2* operand, float alpha, float2* W, cudaStream_t st, bool* done);
pp_status launch_cart2d4_normal(const Plan& p, const float2* x, float2* out, float scale,
                                const float2* operand, float alpha, cudaStream_t st, bool* done);
pp_status launch_rows4_adj(const DevFft& f, const RowArgs& a, const float2* src, const float2* sens,
                           const float* wrow, const float* wcol, float2* out, const float2* operand,
                           float alpha, int ncoils, cudaStream_t st, bool* done, int cluster = 0);
pp_status launch_rows_fwd(const Plan& p, const DevFft& f, const RowArgs& a, const float2* x,
                          const float2* sens, const float* wrow, const float* wcol, float2* out,
                          int ncoils, int64_t img_batch_stride, cudaStream_t st);
pp_status launch_rows_adj(const Plan& p, const DevFft& f, const RowArgs& a, const float2* src,
                          const float2* sens, const float* wrow, const float* wcol, float2* out,
                          const float2* operand, float alpha, int ncoils, cudaStream_t st);
pp_status launch_cols(const DevFft& f, const ColArgs& a, const float2* src, float2* dst, bool inv,
                      cudaStream_t st);
pp_status launch_cols_roundtrip(const DevFft& f, const ColArgs& a, const float* mask_fo,
                                const float2* src, float2* dst, cudaStream_t st);
pp_status launch_cart2d_normal(const Plan& p, const float2* x, float2* out, float scale,
                               const float2* operand, float alpha, cudaStream_t st);
pp_status launch_expand(const float2* x, const float2* s, float2* out, int64_t n, cudaStream_t st);
pp_status launch_conj_accum(const float2* s, const float2* wv, float2* out, int64_t n, int first,
                            float scale, const float2* operand, float alpha, int last,
                            cudaStream_t st);
pp_status launch_nufft_spread(const Plan& p, const float2* ksp, float2* grid_out, cudaStream_t st);
pp_status launch_gtg_stencil(const Plan& p, const float2* grid_in, float2* grid_out, cudaStream_t st);
pp_status prepare_gtg_stencil(Plan& p);
pp_status build_gtg_device(Plan& p, cudaStream_t st);
pp_status prepare_cart4();
int c3cl_prepare(const Plan& p, int xb);
int c3df_prepare(const Plan& p, int variant);
bool c3df_make_tensor_map(Plan& p);
size_t c3df_slot_elems(const Plan& p, int cg);
size_t c3df_counter_ints(const Plan& p, int cg);
pp_status c3df_normal(const Plan& p, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st);
pp_status c3df_check(const Plan& p, cudaStream_t st);
pp_status selftest_wait(long long limit_ns, cudaStream_t st);
pp_status launch_prox_llr(int ndim, int nx, int ny, int nz, int T, int block, const int* shift,
                          float lambda, const float2* in, float2* out, cudaStream_t st);
pp_status c3cl_normal(const Plan& p, int xb, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st);
bool ci_supported(const Plan& p);
size_t ci_grid_elems(const Plan& p);
size_t ci_stencil_tiles(const Plan& p);
size_t ci_rows_elems(const Plan& p);
size_t ci_sens_elems(const Plan& p);
size_t ci_partial_elems(const Plan& p);
pp_status ci_prepare(Plan& p, cudaStream_t st);
bool toep_supported(int nx, int ny, int C);
size_t toep_rows_elems(const Plan& p);
pp_status toep_normal(const Plan& p, const float2* x, float2* out, float scale,
                      const float2* operand, float alpha, cudaStream_t st);
pp_status toep_build_kernel(Plan& p, const float* traj, int64_t K, cudaStream_t st);
bool db4_supported(int ndim, int nx, int ny, int levels);
pp_status launch_prox_db4(int nx, int ny, int levels, float lambda, const float2* in, float2* out,
                          cudaStream_t st);
pp_status launch_prox_fista_db4(const Plan& p, int levels, float lambda, float gamma, float beta,
                                const float2* u, float2* scratch, const float2* ref, double* hist_slot,
                                cudaStream_t st);
pp_status ci_normal(const Plan& p, const float2* x, float2* out, float scale, const float2* operand,
                    float alpha, int ry, cudaStream_t st);   // ry 0: coil-pair stencil
pp_status launch_nufft_degrid(const Plan& p, const float2* grid_in, float2* ksp, cudaStream_t st);
pp_status launch_prox(int ndim, int nx, int ny, int nz, int levels, float lambda,
                      const float2* in, float2* out, cudaStream_t st);
pp_status launch_prox_fista(const Plan& p, int levels, float lambda, float gamma, float beta,
                            const float2* u, const float2* ref, double* hist_slot, cudaStream_t st);
pp_status launch_dot(const float2* a, const float2* b, int64_t n, double* partials, int nblocks,
                     double* out_re, double* out_norm_b, cudaStream_t st);
pp_status launch_norm2(const float2* a, int64_t n, double* partials, int nblocks, double* out,
                       cudaStream_t st);
pp_status launch_scale_by_rnorm(const float2* in, float2* out, int64_t n, const double* norm2,
                                double factor, int invert, cudaStream_t st);
pp_status launch_axpby(const float2* x, float a, const float2* y, float b, float2* out, int64_t n,
                       cudaStream_t st);
pp_status launch_start_vector(float2* v, int64_t n, uint64_t seed, cudaStream_t st);
// x = A^H y with caller-chosen intermediate buffers (pp_capi.cu)
pp_status adjoint_ws(const Plan& p, const float2* y, float2* x, float2* wa, float2* wb,
                     cudaStream_t st);

}  // namespace pp

// Opaque handle of the C ABI (include/pp.h).
struct pp_plan {
    pp::Plan impl;
};
