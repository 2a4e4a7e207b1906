/*
 * pp.h - C ABI of the polynomial-preconditioned FISTA library (libpp).
 *
 * Iyer et al., "Polynomial Preconditioners for Regularized Linear Inverse
 * Problems": solve  min_x 1/2 ||A x - b||_2^2 + lambda ||W x||_1  (Eq. "ucopt",
 * Sec. 1) with Algorithm "pfista" (Sec. 3.1), where A is a multi-coil SENSE
 * operator (Sec. 5.1 Cartesian, Sec. 5.2 non-Cartesian), W an orthonormal
 * Haar wavelet and p(A^H A) the preconditioner of Eq. "l2cost", applied by the
 * recursion of Listing "pcode" (Sec. 3.6).
 *
 * Conventions shared by every call
 *  - Complex data are interleaved complex64 (pp_c64: re, im), C order with
 *    the readout axis x fastest:
 *      image           [nz][ny][nx]          (nz = 1 in 2-D)
 *      sensitivities   [C][nz][ny][nx]
 *      Cartesian k     [C][nz][ny][nx]       centred order, zero off-mask
 *      non-Cartesian k [C][K]                sample order of the trajectory
 *  - "device" pointers are CUDA global memory on the current device; "host"
 *    pointers are ordinary CPU memory.  The library never takes ownership of
 *    caller memory.  A plan owns the device workspace it allocates.
 *  - pp_stream is a cudaStream_t (NULL = legacy default stream).  Device
 *    work is enqueued on that stream; calls return without synchronising
 *    except where they return a value computed on the device (plan creation,
 *    pp_fista_solve when info->history is set).
 *  - Every call returns a pp_status.  On failure pp_last_error() gives a
 *    thread-local message.  No call throws, aborts or traps.
 *  - Input and output arrays of one call must not overlap unless the call
 *    says otherwise.
 *  - Calls on different plans or batches may run at the same time from
 *    different host threads (the library's shared state, the launch-shape
 *    cache and the one-time kernel set-up, is locked); calls on one plan or
 *    batch share its workspaces and must be serialised by the caller.
 *    The first solve of a plan or batch with given parameters captures its
 *    iterations into a CUDA graph, and CUDA forbids, in every thread, a
 *    synchronisation of the whole device while a capture is open
 *    (cudaDeviceSynchronize, and the implicit one of cudaFree, which
 *    pp_plan_destroy and pp_batch_destroy call): such a call made during
 *    that capture fails, and so does the capturing solve (PP_ERR_CUDA).
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad enum          */
    PP_ERR_UNSUPPORTED = 2,  /* valid but not implemented (see each call) */
    PP_ERR_OOM = 3,          /* device allocation failed                  */
    PP_ERR_CUDA = 4,         /* a CUDA runtime call failed                */
    PP_ERR_NONFINITE = 5,    /* NaN/Inf met in a reduction                */
    PP_ERR_TIMEOUT = 6       /* a bounded device wait expired (see the
                                3-D dataflow operator, pp_selftest_wait) */
} pp_status;

typedef struct { float re, im; } pp_c64;
typedef void* pp_stream;

/* Image size: n[0] = nx (fastest), n[1] = ny, n[2] = nz (used when ndim == 3). */
typedef struct { int ndim; int n[3]; } pp_dims;

enum { PP_CARTESIAN = 0, PP_NONCARTESIAN = 1, PP_NONCARTESIAN_TOEPLITZ = 2 };

/* Sampling pattern (the M of Sec. 5.1, or the trajectory of Sec. 5.2).
 *  kind == PP_CARTESIAN:    mask = host uint8 [nz][ny][nx], centred order,
 *                           nonzero = sampled.  It must be constant along x
 *                           (readout); otherwise PP_ERR_UNSUPPORTED.
 *  kind == PP_NONCARTESIAN: traj = host float [K][2] = (kx, ky) in cycles per
 *                           field of view, each in [-n/2, n/2); 2-D only.
 *                           Gridding uses a Kaiser-Bessel kernel of width
 *                           kb_width (must be 4) on a grid of
 *                           ceil(oversamp * n) points per axis (oversamp in
 *                           [1.125, 2]); the grid size must be even, have no
 *                           prime factor above 5 and be at least 40.
 *  kind == PP_NONCARTESIAN_TOEPLITZ: the same trajectory and gridding
 *                           parameters (used by the forward and adjoint
 *                           applies), but the normal operator is the exact
 *                           F^H F of the non-uniform DFT, evaluated through
 *                           its Toeplitz structure (the remark on Toeplitz
 *                           normal operators in Sec. 2; the spiral experiment
 *                           of Sec. 5.2): an FFT convolution on the 2ny x 2nx
 *                           circulant embedding, with no gridding in the
 *                           loop.  The embedded kernel's spectrum is computed
 *                           at plan time from the trajectory.  Needs coils
 *                           <= 32 and nx, ny in {64, 96, 128, 160, 192, 256};
 *                           else PP_ERR_UNSUPPORTED.  pp_plan_set_tuning does
 *                           not affect it.
 *  The plan copies what it needs; the host arrays may be freed on return. */
typedef struct {
    int kind;
    const uint8_t* mask;
    const float* traj;
    int64_t K;
    int kb_width;
    float oversamp;
} pp_sampling;

typedef struct pp_plan pp_plan;

/* Build a plan for the operator A = [P S_1; ...; P S_C] (Sec. 5.1/5.2) and
 * estimate L = lambda_max(A^H A) by power_iters steps of power iteration
 * from a SplitMix64 start vector drawn from `seed` (Sec. 5 normalises A to
 * unit induced norm; the solver divides by L).  power_iters = 0 leaves L = 1
 * (set it with pp_plan_set_scale).
 *   dims   2-D (ndim 2) or 3-D (ndim 3, Cartesian only).  Every FFT length
 *          (ny, nz; and nx plus the grid size for non-Cartesian) must have no
 *          prime factor above 5 and be even; nx and ny (and nz) must be
 *          multiples of 4 (the 2-level Haar tile).  Else PP_ERR_UNSUPPORTED.
 *   coils  1..64.
 *   sens   device [C][nz][ny][nx] complex64, 16-byte aligned (else
 *          PP_ERR_INVALID_ARG), BORROWED: it must stay valid and unchanged
 *          until pp_plan_destroy.
 *   s      sampling pattern, see pp_sampling.
 * Set-up times the plan's candidate launch shapes on its own buffers and
 * keeps the fastest (see pp_plan_tuning); the choice is remembered for the
 * life of the process per device, shape, coil count and sampling (the
 * trajectory's or the mask's bytes), so a later plan of the same geometry
 * takes it without timing again.  Non-Cartesian set-up computes the
 * per-sample gridding taps and tile lists on up to 16 host threads.
 * Synchronises `stream` (the set-up work is complete on return).  On
 * failure *out is NULL. */
pp_status pp_plan_create(pp_plan** out, pp_dims dims, int coils, const pp_c64* sens,
                         const pp_sampling* s, uint64_t seed, int power_iters, pp_stream stream);

/* Free the plan and its device workspace.  Call after the plan's last
 * enqueued work has finished.  NULL is accepted. */
pp_status pp_plan_destroy(pp_plan* plan);

/* L used for A_hat = A / sqrt(L) (host double out). */
pp_status pp_plan_scale(const pp_plan* plan, double* L);

/* Replace L (L > 0, finite); used to share one estimate between runs. */
pp_status pp_plan_set_scale(pp_plan* plan, double L);

/* Estimate mu, the smallest eigenvalue of N_hat = A^H A / L, for the
 * Chebyshev preconditioner (pp_poly_coeffs_cheb): `iters` steps of power
 * iteration on I - N_hat from a SplitMix64 start vector drawn from `seed`
 * (the remark closing the Chebyshev design of Sec. 3.4: when A^H A is
 * injective, the largest eigenvalue of I - N_hat is 1 - mu), FP64
 * reductions; *mu (host) = 1 - the last Rayleigh quotient.  The estimate
 * approaches mu from above.  A value at or below 0 (up to rounding) means
 * A^H A has a null space or near-null directions: no Chebyshev interval
 * [mu, 1] with mu > 0 exists, and the l2 design of Eq. "l2cost" applies.
 * Uses the plan's L and workspace; synchronises `stream`. */
pp_status pp_plan_mu(pp_plan* plan, int iters, uint64_t seed, double* mu, pp_stream stream);

/* Element counts of the image ([nz][ny][nx]) and of the k-space array
 * ([C][...] as above); either pointer may be NULL. */
pp_status pp_plan_sizes(const pp_plan* plan, int64_t* image_elems, int64_t* kspace_elems);

/* Launch shapes the plan chose by timing at creation:
 *  - row_ifft_variant: for non-Cartesian plans the row-IFFT stage of the
 *    normal operator (1, 2 or 4 = CTAs per image row, coil groups reduced
 *    through distributed shared memory; -1 = one IFFT per coil and row
 *    followed by a coil sum); for 3-D Cartesian plans 16 = the whole normal
 *    operator as one kernel on 16-CTA clusters, 4 x columns per cluster task
 *    (nz = 128, ny in {128, 192, 256}), -16 = the same with 2 columns per
 *    task and two CTAs per SM, 1 = three passes per coil, 3 = one persistent
 *    kernel whose blocks claim y-FFT, z round-trip and y-IFFT work items of
 *    16-column x-blocks and stencil_coils-coil groups in dependency order
 *    (ny, nz register-FFT lengths; up to 8 coils per group; stencil_kind 0
 *    or 1 = compiled for two or three resident blocks per SM, 2 = two blocks
 *    per SM with the coil-map tiles of the y-FFT and y-IFFT items streamed
 *    into two shared buffers by tensor-map bulk copies (TMA), 3 = the same
 *    with one buffer and three blocks per SM, 4 or 5 = 0 or 1 with two z
 *    planes per y-FFT item and two line units per z item); for 2-D
 *    Cartesian plans 1, 2, 4 or 8
 *    = CTAs per 8-column group, the coils split over a cluster of that size;
 *  - stencil_kind: the G^T G stencil kernel (0 = one output per thread,
 *    1 = two outputs per thread, both staging one coil at a time with
 *    stencil_coils coils per CTA; 2..5 = register-blocked, a thread holding
 *    R outputs of CG coils with (R, CG) = (4, 4), (8, 4), (4, 8), (2, 8), on
 *    a persistent grid; 6 = coil-lane, the 32 lanes of a warp being 32
 *    coils of 8 adjacent outputs; 7, 8 = the whole normal operator on
 *    coil-innermost ([row][col][coil], 32-coil pitch) copies with a
 *    coil-lane stencil of 1 or 2 rows per warp, 9 = the same with a
 *    coil-pair stencil (two coils per lane) (plans with at most 32
 *    coils and register-FFT grid lengths); there row_ifft_variant 4 sums
 *    the four 8-coil blocks of a row in a thread-block cluster, any other
 *    value through a partial-sum buffer;
 *    stencil_coils is ignored for kinds 2..8);
 *  - stencil_coils: 1..64.
 * pp_plan_set_tuning overrides them (results are identical up to rounding
 * order; PP_ERR_UNSUPPORTED for a variant the plan cannot run).  Any output
 * pointer may be NULL.  No counterpart in the paper. */
pp_status pp_plan_tuning(const pp_plan* plan, int* row_ifft_variant, int* stencil_kind,
                         int* stencil_coils);
pp_status pp_plan_set_tuning(pp_plan* plan, int row_ifft_variant, int stencil_kind,
                             int stencil_coils);

/* y = A x (unscaled forward model; Sec. 5.1: M F S_c x with the centred
 * orthonormal FFT; Sec. 5.2: gridding NUFFT of S_c x).
 * x device image, y device k-space. */
pp_status pp_forward_apply(const pp_plan* plan, const pp_c64* x, pp_c64* y, pp_stream stream);

/* x = A^H y (unscaled adjoint).  y device k-space, x device image. */
pp_status pp_adjoint_apply(const pp_plan* plan, const pp_c64* y, pp_c64* x, pp_stream stream);

/* x = A^H y like pp_adjoint_apply, but allocating nothing: every
 * intermediate buffer lives in a fixed 16 MiB array of device memory that
 * is part of the library (each GPU that loads the library holds it until the
 * process exits).  For callers that must not allocate device memory when
 * they call: a plug-in whose host application owns all device memory through
 * its own pool (an allocation behind its back can fail or upset the host's
 * accounting), or a real-time loop that forbids allocation after start-up
 * (an allocation can stall or fail on fragmented memory).  The plan is built
 * beforehand with pp_plan_create.  Runs the same kernels as
 * pp_adjoint_apply.  The paper has no counterpart.
 *  - Plans whose adjoint needs more than 16 MiB of scratch (Cartesian 2-D:
 *    8*C*ny*nx bytes; 3-D: 16*nz*ny*nx; non-Cartesian: 8*C*G*(ny+G))
 *    return PP_ERR_UNSUPPORTED.
 *  - The first call on a device looks up the array's device address (and,
 *    with lazy module loading, is when the runtime commits the array's
 *    memory); make that first call before any stream capture.  The address
 *    is kept for the life of the process: after a cudaDeviceReset of that
 *    device (which also frees every plan) the library is not usable there.
 *  - All calls share the one array and it keeps the last call's contents
 *    (nothing in it needs clearing: every element read is written first in
 *    the same call).  Calls that overlap on the GPU (other streams, other
 *    host threads) race on it and must be serialised by the caller. */
pp_status pp_adjoint_apply_static(const pp_plan* plan, const pp_c64* y, pp_c64* x, pp_stream stream);

/* y = (A^H A / L) x, the normalised normal operator N_hat of Algorithm
 * "pfista".  x, y device images.  Cartesian plans use the readout
 * shortcut F_x^H (F_yz^H M F_yz) F_x = F_yz^H M F_yz, exact because M is
 * constant along x. */
pp_status pp_normal_apply(const pp_plan* plan, const pp_c64* x, pp_c64* y, pp_stream stream);

/* c[0..d] (host double) minimising int_0^1 (1 - z p(z))^2 dz, Eq. "l2cost"
 * (Sec. 3.1), p(z) = sum_i c[i] z^i (order of Sec. 3.6).  0 <= d <= 8.
 * Computed in closed form as exact integer ratios (shifted-Legendre
 * Christoffel-Darboux kernel), each rounded once to double.  Host only; no
 * device work. */
pp_status pp_poly_coeffs_l2(int d, double* c);

/* c[0..d] (host double) of the Chebyshev minimax preconditioner of Sec. 3.4:
 * with a = (1 + mu)/(1 - mu), r(z) = T_{d+1}(a - 2z/(1 - mu)) / T_{d+1}(a)
 * (T the Chebyshev polynomial of the first kind) and p(z) = (1 - r(z))/z,
 * which minimises max |1 - z p(z)| over [mu, 1].  0 < mu < 1, 0 <= d <= 8.
 * Host only. */
pp_status pp_poly_coeffs_cheb(int d, double mu, double* c);

/* c[0..d] (host double) minimising the weighted cost of Eq. "wl2cost",
 * int_0^1 w(z) (1 - z p(z))^2 dz, for a weight given by its moments
 * moments[k] = int_0^1 w(z) z^k dz, k = 0..2d+2 (host double; moments[0] is
 * not used).  The paper leaves the choice of w open (a prior on the spectrum
 * of A^H A); w = 1 (moments 1/(k+1)) gives pp_poly_coeffs_l2.  Solves the
 * normal equations sum_j m_{i+j+2} c_j = m_{i+1} by LU with partial
 * pivoting and compensated iterative refinement.  0 <= d <= 8; moments that
 * give singular equations (no positive weight) -> PP_ERR_INVALID_ARG.  Host
 * only; no device work. */
pp_status pp_poly_coeffs_wl2(int d, const double* moments, double* c);

/* *m (host) = max over z in [0, 1] of z p(z), p(z) = sum_i c[i] z^i: the
 * Lipschitz constant of the preconditioned gradient step on the normalised
 * problem (spectrum of N_hat in (0, 1]).  FISTA's step rule wants it <= 1;
 * the l2 polynomials exceed it mildly (1.2, 1.15, 1.14 for d = 1, 3, 5) and
 * the Chebyshev ones reach 1 + 1/T_{d+1}((1 + mu)/(1 - mu)) on [mu, 1]
 * (near 2 for small mu), which diverges under momentum; dividing c by m
 * gives a step within the rule (the paper applies p unscaled).  Dense
 * sampling of [0, 1] refined by golden-section search.  Host only.
 * 0 <= d <= 16. */
pp_status pp_poly_max_zp(const double* c, int d, double* m);

/* out = p(N_hat) v by the recursion of Listing "pcode": u = c_d v, then
 * u = c_i v + N_hat u for i = d-1..0 (d applies of N_hat).  c host double
 * [d+1], 0 <= d <= 16.  v, out device images. */
pp_status pp_poly_apply(const pp_plan* plan, const double* c, int d, const pp_c64* v,
                        pp_c64* out, pp_stream stream);

/* out = prox_{lambda ||W.||_1}(in) = W^T soft_lambda(W in) (Eq. "proxdef",
 * Sec. 2.1) with W the orthonormal separable Haar wavelet of `levels` levels
 * (1 or 2) over every image axis; soft_lambda(v) = v max(0, 1 - lambda/|v|)
 * on every coefficient.  Each image axis must be a multiple of 2^levels.
 * in, out device images; in == out is allowed. */
pp_status pp_prox_l1_haar(pp_dims dims, int levels, float lambda, const pp_c64* in, pp_c64* out,
                          pp_stream stream);

/* prox_{lambda ||W.||_1}(in) = W^T soft_lambda(W in) (Eq. "proxdef") with W the
 * orthonormal Daubechies-4 wavelet, the transform of the paper's experiments
 * (Sec. 5.1, Sec. 5.2): the four-coefficient Daubechies filter
 * h = ((1+sqrt3), (3+sqrt3), (3-sqrt3), (1-sqrt3)) / (4 sqrt2), high-pass
 * g[k] = (-1)^k h[3-k], periodic boundary, separable, `levels` levels in
 * Mallat layout; every coefficient is soft-thresholded.
 *   dims    2-D only; nx, ny <= 512 and multiples of 2^levels; levels 1..4
 *           (else PP_ERR_UNSUPPORTED).
 *   in/out  device [ny][nx] complex64; out may equal in.
 * Runs as 4 * levels kernels on `stream` (each level couples neighbouring
 * rows and columns, so the transform is not tile-local like the Haar). */
pp_status pp_prox_l1_db4(pp_dims dims, int levels, float lambda, const pp_c64* in, pp_c64* out,
                         pp_stream stream);

/* prox_{lambda LLR}(in) for the locally-low-rank regulariser of the MRF
 * experiment (Sec. 5.3; Tamir et al.): LLR(x) = the sum over blocks of the
 * nuclear norm of the block's Casorati matrix, one row per voxel of the
 * block and one column per coefficient image.  The prox replaces each
 * block's matrix M = U S V^H by U max(S - lambda, 0) V^H.
 *   dims    2-D or 3-D image size of ONE coefficient image; every axis a
 *           multiple of `block`.
 *   T       coefficient images, 1..8.
 *   block   block edge: 4 or 8 (3-D: 64 or 512 voxels), or 16 in 2-D.
 *   shift   host int[3] (x, y, z) or NULL: the block grid starts at voxel
 *           shift (circularly), so a caller can move it between iterations.
 *   in/out  device [T][nz][ny][nx] complex64; out may equal in.
 * FP32 one-sided Jacobi SVD per block (one thread block each); else
 * PP_ERR_UNSUPPORTED. */
pp_status pp_prox_llr(pp_dims dims, int T, int block, const int* shift, float lambda,
                      const pp_c64* in, pp_c64* out, pp_stream stream);

/* Optional solve inputs/outputs.
 *  history  host double [iters][3] or NULL.  Row k receives, as FP64
 *           reductions on the device, ||y_{k+1} - y_k||^2, ||y_{k+1}||^2 and
 *           ||y_{k+1} - ref||^2 (0 when ref is NULL).  Setting it makes the
 *           call synchronise.
 *  ref      device image or NULL: reference for the third history column
 *           (e.g. a converged solution, for NRMSE against it as in Sec. 5).
 *  launches out: kernels this call enqueued (graph nodes included). */
typedef struct {
    int rescale;         /* in: 1 = multiply x_out by ||b|| / sqrt(L)        */
    int levels;          /* in: Haar levels (0 means 2)                      */
    int no_momentum;     /* in: 1 = beta_k = 0, i.e. Algorithms "pgd"/"ppgd" */
    double* history;     /* in: optional host buffer, see above              */
    const pp_c64* ref;   /* in: optional device reference image              */
    double bnorm;        /* out: ||b||_2 (valid when history != NULL)        */
    double L;            /* out: the L used                                  */
    int64_t launches;    /* out: kernels enqueued by this call               */
    int wavelet;         /* in: W of the prox: 0 = orthonormal Haar (levels
                            1..2), 1 = Daubechies-4 (2-D, levels 1..4), see
                            pp_prox_l1_db4; else PP_ERR_INVALID_ARG         */
    int safe_scale;      /* in: 1 = divide c by max over [0, 1] of z p(z)
                            (pp_poly_max_zp) before the solve, so that the
                            preconditioned step keeps FISTA's step rule; 0 =
                            apply c as given, as the paper does.  Used by
                            pp_fista_solve and pp_batch_fista_solve         */
} pp_solve_info;

/* Algorithm "pfista" on the normalised problem (Sec. 5): A_hat = A/sqrt(L),
 * b_hat = b/||b||_2, y_{-1} = y_0 = z_0 = 0, for k = 0..iters-1:
 *   g = N_hat z_k - A_hat^H b_hat;  u = p(N_hat) g;
 *   y_{k+1} = prox_{lambda ||W.||_1}(z_k - u);
 *   z_{k+1} = y_{k+1} + (k/(k+3)) (y_{k+1} - y_k).
 * c host double [d+1] (Eq. "l2cost" coefficients or any other); c == NULL
 * with d == 0 is plain FISTA (Algorithm "fista", p = 1).  b device k-space,
 * x_out device image (y_iters).  info may be NULL.  The iteration loop runs
 * as one CUDA graph, captured on first use and reused while iters, c, d,
 * lambda and levels are unchanged.
 * b = 0 gives x_out = 0 (the solution for b = 0).  A NaN or infinite value
 * in b makes every iterate NaN; with info->history set the call (which then
 * synchronises) returns PP_ERR_NONFINITE, x_out still written.  Without a
 * history the call does not synchronise and cannot report it. */
pp_status pp_fista_solve(pp_plan* plan, const pp_c64* b, float lambda, int iters, const double* c,
                         int d, pp_c64* x_out, pp_solve_info* info, pp_stream stream);

/* Algorithm "pfista" for the proximal subproblem of consensus ADMM
 * (Algorithm "cadmm", Sec. 5.3):
 *   x_out = argmin_x 1/2 ||A x - b||^2 + (sigma/2) ||x - v||^2 + lambda ||W x||_1,
 * i.e. prox_{rho f}(v) with rho = 1/sigma for f = 1/2 ||A x - b||^2 +
 * lambda ||W x||_1, in the problem's own units (b is NOT normalised; lambda
 * is in the units of the objective above).  With N' = A^H A + sigma I and
 * L' = L + sigma the iteration runs with step 1 on N'/L', the gradient's
 * constant term (A^H b + sigma v)/L' and the threshold lambda/L'; the
 * preconditioner p(N'/L') (coefficients c[0..d] designed on (0, 1], as for
 * pp_fista_solve) is applied as the same-degree polynomial in N/L with
 * coefficients expanded on the host, so every apply is the plan's normal
 * operator.  y_0 = z_0 = 0.
 *   b  device k-space or NULL (no data term); v device image or NULL (0);
 *   sigma >= 0 (0: the plain problem in its own units).
 * info as for pp_fista_solve (rescale is ignored).  The iteration loop runs
 * as a cached CUDA graph like pp_fista_solve's. */
pp_status pp_fista_solve_prox(pp_plan* plan, const pp_c64* b, const pp_c64* v, double sigma,
                              float lambda, int iters, const double* c, int d, pp_c64* x_out,
                              pp_solve_info* info, pp_stream stream);

/* ---- Batches of independent 2-D Cartesian problems of uneven size ----
 * Slice s is its own problem (Sec. 5.1 operator, its own L_s, its own ||b_s||)
 * of size dims[s] (2-D, axes multiples of 4, FFT lengths with prime factors
 * <= 5, at most 512), coils[s] coils (1..64), borrowed 16-byte aligned device maps
 * sens[s] [C_s][ny_s][nx_s] and a host line mask masks[s] [ny_s][nx_s] constant along
 * x.  Images, k-space and solutions are concatenated in slice order; the
 * offsets come from pp_batch_offsets.  Every stage of an iteration is one
 * persistent kernel launch over a work list of (slice, column tile) items,
 * and the tile width is chosen at creation by timing the candidates. */
typedef struct pp_batch pp_batch;

/* Build a batch; power_iters > 0 estimates every L_s (one seed per slice:
 * seed + s).  Synchronises `stream`. */
pp_status pp_batch_create(pp_batch** out, int nslices, const pp_dims* dims, const int* coils,
                          const pp_c64* const* sens, const uint8_t* const* masks, uint64_t seed,
                          int power_iters, pp_stream stream);
pp_status pp_batch_destroy(pp_batch* batch);
/* host int64 [nslices + 1] each (either may be NULL) */
pp_status pp_batch_offsets(const pp_batch* batch, int64_t* image_off, int64_t* kspace_off);
/* host double [nslices] */
pp_status pp_batch_scales(const pp_batch* batch, double* L);
pp_status pp_batch_set_scales(pp_batch* batch, const double* L);
/* autotuned column tile width and persistent grid size (either may be NULL);
 * a positive width is the shared-memory Stockham kernel's columns per item;
 * -8, -16, -32 mean the register four-step FFT kernel on 8-column items
 * with 1, 2 or 4 CTAs per item (the item's coils split over a thread-block
 * cluster) */
pp_status pp_batch_tile(const pp_batch* batch, int* cols_per_cta, int* persistent_ctas);
/* override the autotuner: 4, 8 or 16 (Stockham) or -8, -16, -32 (register
 * four-step, every slice length must be 16 * {8, 12, 16, 20, 24}) */
pp_status pp_batch_set_tile(pp_batch* batch, int cols_per_cta);
/* per-slice A x and A^H y (one launch sequence per slice; set-up work) */
pp_status pp_batch_forward_apply(const pp_batch* batch, const pp_c64* x, pp_c64* y, pp_stream stream);
pp_status pp_batch_adjoint_apply(const pp_batch* batch, const pp_c64* y, pp_c64* x, pp_stream stream);
/* y_s = (A_s^H A_s / L_s) x_s for every slice in one launch */
pp_status pp_batch_normal_apply(const pp_batch* batch, const pp_c64* x, pp_c64* y, pp_stream stream);
/* Algorithm "pfista" on every slice's normalised problem, one shared lambda,
 * iteration count and polynomial; as pp_fista_solve otherwise (history sums
 * over the batch, so a non-finite value in any slice's b gives
 * PP_ERR_NONFINITE when history is set; levels must be 0 or 2). */
pp_status pp_batch_fista_solve(pp_batch* batch, const pp_c64* b, float lambda, int iters,
                               const double* c, int d, pp_c64* x_out, pp_solve_info* info,
                               pp_stream stream);

/* Differentiable unrolled solve on a batch (the training pattern): Algorithm
 * "pfista" for exactly `iters` iterations on each slice with RAW b (no
 * normalisation of b; A_hat_s = A_s / sqrt(L_s) with L_s fixed), checkpoints
 * (y_k, z_k) every checkpoint_every iterations.  x_out is the concatenated
 * y_iters.  c host double [d+1], 0 <= d <= 10. */
pp_status pp_batch_unrolled_forward(pp_batch* batch, const pp_c64* b, float lambda, int iters,
                                    const double* c, int d, int checkpoint_every, pp_c64* x_out,
                                    pp_stream stream);

/* Reverse pass: for the real loss Re<grad_out, y_iters>, writes grad_b (device
 * k-space, dLoss/dRe b + i dLoss/dIm b), *grad_lambda and grad_c[0..d] (host).
 * Uses the checkpoints of the last pp_batch_unrolled_forward with the same
 * b pointer, lambda, iters, c, d, checkpoint_every and per-slice L_s, else
 * reruns that forward first (pp_batch_set_scales and pp_batch_set_tile
 * discard the checkpoints).  The checkpoints are keyed by b's ADDRESS, not
 * its contents: a caller that rewrites b in place between the forward and
 * this call must run the forward again.  Each segment is recomputed from its checkpoint; the
 * Horner adjoint uses v_j = N_hat^j wbar (N_hat is self-adjoint), d+1
 * applies per iteration.  Synchronises `stream`. */
pp_status pp_batch_unrolled_backward(pp_batch* batch, const pp_c64* b, float lambda, int iters,
                                     const double* c, int d, int checkpoint_every,
                                     const pp_c64* grad_out, pp_c64* grad_b, double* grad_lambda,
                                     double* grad_c, pp_stream stream);

/* Stage timing of the normal operator N_hat (no counterpart in the paper:
 * instrumentation).  Runs `reps` applies of N_hat x -> y on `stream`,
 * recording a CUDA event after every kernel launch, synchronises, and
 * returns per kernel name the average milliseconds per apply: names is host
 * char [max_stages][48], ms host double [max_stages], *nstages the count. */
pp_status pp_profile_normal(const pp_plan* plan, const pp_c64* x, pp_c64* y, int reps,
                            int max_stages, char* names, double* ms, int* nstages,
                            pp_stream stream);

/* Self-test of the bounded device wait (no counterpart in the paper).  Kernels
 * that wait on work of other thread blocks (the 3-D dataflow normal operator)
 * poll with a time limit and, past it, record the failure and return instead
 * of hanging; the next synchronising call on the plan reports
 * PP_ERR_TIMEOUT.  This call runs one block that waits on a counter nothing
 * increments, with a limit of limit_ns (1e6 .. 1e9 ns), and returns
 * PP_ERR_TIMEOUT when the wait gave up as it must; the device stays usable.
 * Allocates 8 bytes of device memory; synchronises `stream`. */
pp_status pp_selftest_wait(int64_t limit_ns, pp_stream stream);

/* Message for the last failing call on this thread ("" if none). */
const char* pp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PP_H */
