/*
 * bpdn.h -- C ABI of libbpdn: batched complex basis pursuit denoising on GB300 (sm_103a).
 *
 * Each pixel of a SAR stack solves (Eq. 1 / Eq. 6, Sec. I and III-A)
 *
 *     x* = argmin_x  ||A x - g||_2^2 + lambda * sum_l |x_l|,    x in C^L, g in C^N,
 *
 * with the steering matrix of the discrete tomographic model (Eq. 5, Sec. II)
 *
 *     A_nl = exp(-j 2 pi xi_n s_l),   xi_n = 2 b_n / (wavelength * range),
 *     s_l  = s_min + l (s_max - s_min)/(L - 1),  l = 0..L-1.
 *
 * The solver is Algorithm 1 (randomized blockwise proximal gradient with Nesterov
 * extrapolation, Eqs. 11-13, backtracking, Eq. 15, and the monotone accept step),
 * one block per pixel, followed by an optional FP64 refit on the detected support.
 *
 * Conventions for every entry point
 *   - Device buffers are owned by the caller (e.g. torch tensors passed by data
 *     pointer).  The library never allocates or frees device memory and never
 *     synchronises the stream in bpdn_solve / bpdn_refit / bpdn_backward.
 *   - Complex arrays are interleaved (re, im) float32 pairs ("c64") or float64
 *     pairs ("c128"), row-major, pixel-major (row p holds pixel p).
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).
 *   - A negative return value means nothing was launched; bpdn_last_error() then
 *     returns a message (thread-local).  Per-pixel numerical outcomes are never
 *     errors: they are reported as status bits.
 */
#ifndef BPDN_H
#define BPDN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bpdn_op *bpdn_op_t; /* opaque host handle of one stack's operator */

enum bpdn_status {
    BPDN_OK = 0,
    BPDN_EINVAL = -1, /* bad argument (null pointer, non-finite or out-of-range value)  */
    BPDN_ECUDA = -2,  /* a CUDA call failed; message in bpdn_last_error()             */
    BPDN_ESIZE = -3,  /* N, L, P or a workspace size outside the supported range      */
    BPDN_EALIGN = -4, /* a device pointer is not aligned as documented                */
    BPDN_ESTATE = -5  /* wrong device current, destroyed handle, ...                  */
};

/* per-pixel status bits (int32 written to d_status) */
#define BPDN_PX_NOT_CONVERGED 1     /* max_iter reached before the stopping test held  */
#define BPDN_PX_BT_LIMIT 2          /* an iteration needed more than max_bt step cuts   */
#define BPDN_PX_NONFINITE 4         /* g held NaN/Inf; x = 0, iters = 0                 */
#define BPDN_PX_SUPPORT_OVERFLOW 8  /* refit skipped: |supp x| > s_max                  */
#define BPDN_PX_KKT_FAIL 16         /* refit ran but could not certify optimality       */
#define BPDN_PX_ZERO_SOLUTION 32    /* returned x is exactly 0                          */
#define BPDN_PX_CERTIFIED 64        /* refit certified x as the minimiser of Eq. 6      */
#define BPDN_PX_DEVICE_TIMEOUT 128  /* precision 1: a bounded wait for the tensor cores  */
                                    /* ran out; x is the last accepted iterate (or 0)    */

/* limits */
#define BPDN_MAX_N 80
#define BPDN_MAX_L 65536 /* grids of more than 1024 points: see bpdn_solve */
#define BPDN_MAX_SMAX 32
#define BPDN_MAX_KSEL 4  /* scatterers per pixel bpdn_select considers */
#define BPDN_MAX_MOTION 2 /* motion dimensions of bpdn_make_operator_md */

typedef struct {
    int32_t max_iter;     /* N_K of Algorithm 1 (default 500)                                  */
    float tol;            /* stop when ||xbar - x^k|| <= tol ||xbar|| (default 1e-6)            */
    float c_alpha;        /* step reduction factor C_alpha of Eq. 15, in (0,1) (default 0.5)    */
    float alpha0_scale;   /* alpha_0 = alpha0_scale / (2N)  (default 1)                         */
    int32_t precision;    /* 0: FP32 contraction (CUDA cores); 1: BF16 operands, FP32 accumulate */
                          /* (tensor cores: the grid-point kernel for 2N <= 128 and L <= 512, */
                          /* the split-grid kernel for 2N <= 160 at any L)                    */
    int32_t refit;        /* 0: none; 1: FP64 restricted solve on the support + certificate     */
    int32_t s_max;        /* largest support the refit handles (<= BPDN_MAX_SMAX, default 32)   */
    int32_t max_bt;       /* step cuts allowed per iteration before BT_LIMIT (default 64)        */
    int32_t tile_pixels;  /* pixels in flight per SM: 8 or 16; 0 = library choice: groups of 8 */
                          /* pixels, as many as fit (16 at L = 400, up to 64 on small grids)   */
    int32_t refit_rounds; /* working-set rounds of the refit (default 4)                         */
    int32_t blocks;       /* 0 or 1: Algorithm 1 on each pixel's whole grid (default); 2..8:     */
                          /* the grid split into that many contiguous blocks, one drawn per    */
                          /* iteration with probability L_j / sum L_j (Eqs. 13-14); FP32 only */
    uint32_t seed;        /* stream of the block draws: pixel p uses SplitMix64 from state     */
                          /* seed + p * 2^40 (default 0)                                       */
    int32_t kernel;       /* iteration kernel: 0 = library choice (the split-grid kernel for    */
                          /* grids of more than 1024 points, and for FP32 grids of more than  */
                          /* 512 with tile_pixels 0; else the grid-point kernel); 1 = the      */
                          /* grid-point kernel (L <= 1024); 2 = the split-grid kernel (FP32,   */
                          /* tile_pixels 0, blocks <= 1) (default 0)                           */
    int32_t reserved[3];
} bpdn_options;

/* Fill *opt with the defaults above. */
void bpdn_default_options(bpdn_options *opt);

/* ---------------------------------------------------------------- operator */

/* Bytes of device workspace an operator with N acquisitions and L grid points
 * needs (A in the layouts the kernels read, A in FP64, the Toeplitz generator of
 * A^H A, A A^H and scalars).  0 if N or L is out of range. */
size_t bpdn_op_workspace_bytes(int32_t N, int32_t L);

/*
 * Build the operator of one stack on the device (Eq. 5 and the definitions after
 * Eq. 2): A_nl = exp(-j 2 pi xi_n s_l) with xi_n = 2 b_n/(wavelength range), the
 * Toeplitz generator h(d) = sum_n exp(j 2 pi xi_n d ds) of A^H A, A A^H, and the
 * Lipschitz constant L_f = 2 lambda_max(A^H A) that the remark after Eq. 14 names
 * (computed in FP64 on the device).
 *
 * baselines_m   host pointer, N finite values (metres)
 * N             1..BPDN_MAX_N;  L  1..BPDN_MAX_L (L = 1 needs s_min == s_max)
 * wavelength_m, range_m  > 0;   s_min_m <= s_max_m (metres)
 * d_workspace   device, >= bpdn_op_workspace_bytes(N, L) bytes, 256-byte aligned;
 *               owned by the caller and must outlive the handle
 * cuda_stream   stream for the set-up kernels.  The call synchronises this
 *               stream once (to read lambda_max back); do not capture it.
 * out           receives a host handle; free it with bpdn_destroy_operator().
 */
int bpdn_make_operator(const double *baselines_m, int32_t N, double wavelength_m, double range_m,
                       double s_min_m, double s_max_m, int32_t L, void *d_workspace,
                       size_t workspace_bytes, void *cuda_stream, bpdn_op_t *out);

/*
 * The multi-component operator of Eq. 4 (differential tomography): the grid is the
 * product of the elevation grid (L_s points on [s_min, s_max]) and M <= BPDN_MAX_MOTION
 * motion-coefficient grids (L_p[m] points on [p_min[m], p_max[m]]), flattened with the
 * elevation index fastest, l = l_s + L_s (l_1 + L_p[0] l_2), and
 *     A_nl = exp(-j 2 pi (xi_n s_{l_s} + sum_m eta_{m,n} p_{m,l_m})),
 * where eta_{m,n} is the temporal frequency of motion base function m at acquisition n
 * (for linear motion 2 t_n / wavelength).  Everything else is as bpdn_make_operator,
 * with L = L_s * prod L_p[m] <= BPDN_MAX_L.  A^H A is not Toeplitz in one index here, so
 * the refit and the adjoint form its entries from the FP64 operator; bpdn_select (an
 * elevation-only reading) refuses such operators, and so does the export of h.
 *
 * eta      host, M x N values (row m holds eta_{m,n}), finite
 * p_min, p_max, L_p   host, M values each: p_min <= p_max, L_p >= 1 (L_p = 1 needs p_min == p_max)
 * Returns BPDN_EINVAL / BPDN_ESIZE / BPDN_EALIGN as bpdn_make_operator, before any launch.
 */
int bpdn_make_operator_md(const double *baselines_m, int32_t N, double wavelength_m, double range_m,
                          double s_min_m, double s_max_m, int32_t L_s, int32_t M, const double *eta,
                          const double *p_min, const double *p_max, const int32_t *L_p, void *d_workspace,
                          size_t workspace_bytes, void *cuda_stream, bpdn_op_t *out);

/* Free the host handle (the caller's workspace is not touched). NULL is ignored. */
void bpdn_destroy_operator(bpdn_op_t op);

/* N, L and grid spacing of an operator; L_f = 2 lambda_max(A^H A) (FP64) and
 * alpha_0 = 1/(2N).  Return BPDN_EINVAL on a NULL handle. */
int bpdn_op_info(bpdn_op_t op, int32_t *N, int32_t *L, double *ds_m, double *lipschitz);
double bpdn_op_lipschitz(bpdn_op_t op);

/* Copy one of the operator's device tables into a caller buffer (for inspection):
 *   what = 0: A as c64, N x L           (dst_bytes >= 8 N L)
 *          1: A as c128, N x L          (16 N L)
 *          2: h(d), c128, d = -(L-1)..L-1 stored at [d + L - 1]   (16 (2L-1))
 *          3: A A^H as c128, N x N      (16 N N)
 * Asynchronous on cuda_stream. */
int bpdn_op_export(bpdn_op_t op, int32_t what, void *d_dst, size_t dst_bytes, void *cuda_stream);

/* ------------------------------------------------------------------- solve */

/* Bytes of device workspace for bpdn_solve on P pixels (256-byte aligned buffer;
 * independent of the data): a work counter, an error word and the block draw table
 * (256 bytes), A_j A_j^H per block when opt->blocks >= 2, and, with the refit, 460 bytes
 * per pixel of scratch for the refit in three launches (the FP32 support search of every
 * pixel, the FP64 finish and certificate, further rounds for the pixels that need them).  A workspace smaller than this, down to the first two parts,
 * is accepted too: the refit then runs in a single launch, with the same results.
 * Solves that run the split-grid kernel (see bpdn_solve) add its scratch, which they cannot
 * do without: two FP32 copies of the operator (16 N L bytes) and three rows of L complex
 * values per pixel in flight (at most 8 per CTA, as many CTAs as the device holds at once
 * and P needs). */
size_t bpdn_solve_workspace_bytes(bpdn_op_t op, int64_t P, const bpdn_options *opt);

/*
 * Solve P pixels that share the operator (Algorithm 1 per pixel, then the refit
 * when opt->refit != 0).  Asynchronous on cuda_stream; no host synchronisation.
 *
 * d_g        device c64 [P, N]   pixel vectors g (8-byte aligned)
 * d_lambda   device float32 [1] (lambda_per_pixel = 0) or [P] (= 1); lambda > 0
 * d_x        device c64 [P, L]   out: x (8-byte aligned)
 * d_support  device int32 [P, s_max] out (may be NULL): ascending support indices,
 *            -1 padded (written only when opt->refit != 0)
 * d_nsupp    device int32 [P] out (may be NULL): number of nonzeros of x
 * d_status   device int32 [P] out: BPDN_PX_* bits
 * d_iters    device int32 [P] out: iterations of Algorithm 1 run
 * d_nbt      device int32 [P] out (may be NULL): total step cuts (Eq. 15 failures)
 * d_workspace  >= bpdn_solve_workspace_bytes(op, P, opt) bytes, 256-byte aligned
 * The operator's workspace must be resident on the current device.
 * Algorithm 1 runs in a split-grid kernel (a CTA's warps walk the grid in 32-point chunks,
 * the iterate in the workspace; FP32 CUDA cores, or BF16 tensor cores with precision 1)
 * for grids of more than 1024 points (L up to BPDN_MAX_L, e.g. the multi-component grids
 * of Eq. 4), which need tile_pixels 0 and blocks <= 1, for FP32 solves of 513..1024 points
 * and for BF16 solves beyond the grid-point kernel's sizes (2N > 128 or L > 512), both with
 * tile_pixels 0 and blocks <= 1; opt->kernel overrides that choice (1: the grid-point
 * kernel, 2: the split-grid kernel at any L).  The choice depends on the operator and the
 * options only.  Such a solve needs a workspace of at least
 * bpdn_solve_workspace_bytes(op, P, opt) bytes; otherwise BPDN_ESIZE before any launch.
 */
int bpdn_solve(bpdn_op_t op, const void *d_g, int64_t P, const float *d_lambda,
               int32_t lambda_per_pixel, const bpdn_options *opt, void *d_x, int32_t *d_support,
               int32_t *d_nsupp, int32_t *d_status, int32_t *d_iters, int32_t *d_nbt,
               void *d_workspace, size_t workspace_bytes, void *cuda_stream);

/*
 * Support extraction and FP64 refit on its own (the refinement that follows
 * Algorithm 1; SL1MMER step (3) "parameter estimation", Sec. III-A):
 * W = {l : x_in[l] != 0}; minimise ||A_W z - g||^2 + lambda sum |z_i| exactly in
 * FP64 over z in C^W, then certify Eq. 6's optimality conditions over the whole
 * grid; grid points that violate them are added to W and the solve repeated
 * (at most opt->refit_rounds rounds).  Certified pixels get BPDN_PX_CERTIFIED
 * and x = the minimiser; the others keep x_in and get KKT_FAIL or
 * SUPPORT_OVERFLOW.  Status bits already in d_status are kept (OR-ed).
 * d_x_in and d_x_out may alias.  d_workspace (may be NULL) with
 * workspace_bytes >= bpdn_refit_workspace_bytes(op, P), 256-byte aligned, lets the refit
 * run as three launches (the FP32 support search of every pixel, the FP64 finish and
 * certificate, then further rounds for the pixels that need them);
 * without it the refit runs in one launch, with the same results.  Other arguments as in
 * bpdn_solve.
 */
int bpdn_refit(bpdn_op_t op, const void *d_g, int64_t P, const float *d_lambda,
               int32_t lambda_per_pixel, const bpdn_options *opt, const void *d_x_in,
               void *d_x_out, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               void *d_workspace, size_t workspace_bytes, void *cuda_stream);

/* Bytes of scratch that let bpdn_refit run as three launches for P pixels (460 per pixel). */
size_t bpdn_refit_workspace_bytes(bpdn_op_t op, int64_t P);

/* ------------------------------------------------------------ ragged batch */

/* One stack of a ragged batch: its operator and the buffers bpdn_solve would take. */
typedef struct {
    bpdn_op_t op;
    const void *d_g;           /* device c64 [P, N] */
    int64_t P;
    const float *d_lambda;     /* device float32 [1] or [P] */
    int32_t lambda_per_pixel;
    void *d_x;                 /* device c64 [P, L] out */
    int32_t *d_support;        /* device int32 [P, s_max] out, or NULL */
    int32_t *d_nsupp;          /* device int32 [P] out, or NULL */
    int32_t *d_status;         /* device int32 [P] out */
    int32_t *d_iters;          /* device int32 [P] out */
    int32_t *d_nbt;            /* device int32 [P] out, or NULL */
    int32_t tile_pixels;       /* this stack's tile_pixels (0 = the options' value) */
    int32_t kernel;            /* this stack's kernel option (0 = the options' value) */
} bpdn_stack;

/* Least workspace of bpdn_solve_ragged: 256 bytes per stack (the refits then run as single
 * launches).  A batch with stacks that run the split-grid kernel (see bpdn_solve) needs
 * bpdn_solve_ragged_workspace_bytes_for. */
size_t bpdn_solve_ragged_workspace_bytes(int32_t n_stacks);

/* Workspace with which bpdn_solve_ragged runs each stack's refit in three launches (as
 * bpdn_solve does): 256 bytes per stack, the split-grid kernel's scratch of the stacks that
 * run it (bpdn_solve_workspace_bytes's part for it), then, when opt->refit, 460 bytes per
 * pixel of every stack.  Same results with or without the last part.  0 if stacks is NULL
 * with n_stacks > 0. */
size_t bpdn_solve_ragged_workspace_bytes_for(const bpdn_stack *stacks, int32_t n_stacks,
                                             const bpdn_options *opt);

/*
 * Solve many stacks, each with its own operator (N, L, grid) and pixel count, in one
 * call: every stack gets exactly the results bpdn_solve would give it.  Every
 * stack's arguments are checked first; on any error nothing is launched and the
 * message names the stack.  Algorithm 1 runs for all stacks in one persistent launch
 * per kernel variant present (BF16 or FP32, A in shared or global memory; 64 stacks
 * per launch): every CTA works through the stacks while they have pixels left.  Stacks
 * that bpdn_solve would give the split-grid kernel run it in their own launches after
 * that one, on the library's streams.  The
 * refits follow, one launch per stack, on a few library-owned streams that fork from
 * and join back into cuda_stream through events, so the whole call can be captured
 * into one CUDA graph.  The streams and events are created by the first call on a
 * device that needs a refit: make that call before any stream capture.  Calls on the
 * same device are serialised on the host.  Allocates no device memory.
 * The paper solves one stack at a time; this is the batched form of the same solve.
 */
int bpdn_solve_ragged(const bpdn_stack *stacks, int32_t n_stacks, const bpdn_options *opt,
                      void *d_workspace, size_t workspace_bytes, void *cuda_stream);

/* ---------------------------------------------------------------- adjoint */

/* Bytes of device workspace bpdn_backward needs for P pixels: 8 P (the per-pixel
 * dL/dlambda terms summed when lambda is shared), rounded up to 256.  Nothing is
 * needed when lambda_per_pixel != 0. */
size_t bpdn_backward_workspace_bytes(bpdn_op_t op, int64_t P);

/*
 * Derivatives of the BPDN minimiser (Eq. 6) with respect to g and lambda for a loss
 * L(x) whose gradient dL/dx is given.  On the support S the optimality condition of
 * Eq. 6, 2 A_S^H (A_S x_S - g) + lambda x_S/|x_S| = 0, is smooth; with J its real
 * symmetric Jacobian in x_S (each complex unknown as (Re, Im)) and v = J^{-1} (dL/dx)_S,
 *     dL/dg = 2 A_S v,    dL/dlambda = -sum_{l in S} (x_l/|x_l|) . v_l,
 * solved in FP64 per pixel.  Meaningful where x is the certified minimiser (the
 * refit's output) and its support is strict (every dual constraint off S slack):
 * then S does not move under small changes of g and lambda.
 *
 * Complex gradients follow PyTorch's convention for real losses:
 * grad = dL/dRe + j dL/dIm.
 *
 * d_lambda    device float32 [1] (lambda_per_pixel = 0) or [P] (= 1)
 * d_x         device c64 [P, L]   the solution (bpdn_solve / bpdn_refit output)
 * d_support   device int32 [P, s_max]  its ascending support (-1 padded), as written
 *             by bpdn_solve / bpdn_refit with the same s_max
 * d_nsupp     device int32 [P]    number of nonzeros; entries beyond s_max are ignored,
 *             as are support entries outside [0, L) or where x is 0
 * d_status    device int32 [P] (may be NULL): BPDN_PX_* bits of the solve; pixels
 *             without BPDN_PX_CERTIFIED (x is then not the minimiser) get zero derivatives
 * s_max       1..BPDN_MAX_SMAX
 * d_dL_dx     device c64 [P, L]   upstream gradient (entries off the support are unused)
 * d_dL_dg     device c64 [P, N]   out
 * d_dL_dlambda device float32 [P] (lambda_per_pixel = 1) or [1] (= 0; the sum over
 *             pixels, accumulated in FP64 in a fixed order) out
 * d_workspace >= bpdn_backward_workspace_bytes(op, P) bytes, 256-byte aligned, when
 *             lambda_per_pixel = 0 (may be NULL otherwise)
 * A pixel whose system is not positive definite (a degenerate support) gets zero
 * derivatives.  Asynchronous on cuda_stream; allocates nothing.  The paper
 * differentiates nothing: this is the adjoint of its solution map for learning lambda.
 */
int bpdn_backward(bpdn_op_t op, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
                  const void *d_x, const int32_t *d_support, const int32_t *d_nsupp,
                  const int32_t *d_status, int32_t s_max,
                  const void *d_dL_dx, void *d_dL_dg, float *d_dL_dlambda, void *d_workspace,
                  size_t workspace_bytes, void *cuda_stream);

/*
 * SL1MMER model selection and parameter estimation (Sec. III-A, steps (2) and (3))
 * on the output of a solve with refit: the number of scatterers in each pixel, their
 * elevations and amplitudes.  The paper defines these steps only by reference; the
 * library's reading:
 *   candidates   maximal runs of adjacent grid points of supp(x); elevation = the
 *                modulus-weighted centroid of the run, energy = sum |x_l|^2; ranked by
 *                energy (ties: lower grid index first), the first kmax kept
 *   model order  K_hat = the first minimiser over K = 0..K_c of
 *                C(K) = 2 N ln RSS_K + K * penalty, where RSS_K is the residual of the
 *                least-squares fit of g by the steering vectors (Eq. 5) of the first K
 *                candidates at their off-grid elevations (a BIC; penalty <= 0 selects
 *                3 ln(2N))
 *   estimates    the K_hat elevations, ascending, and the amplitudes of that fit
 * All arithmetic in FP64, one warp per pixel.
 *
 * d_g         device c64 [P, N]  the pixels' measurements (as given to bpdn_solve)
 * d_x         device c64 [P, L]  the solution (bpdn_solve / bpdn_refit output)
 * d_support   device int32 [P, s_max]  its ascending support (-1 padded), as written by
 *             bpdn_solve / bpdn_refit with the same s_max
 * d_nsupp     device int32 [P]  number of nonzeros (entries beyond s_max are ignored,
 *             as are support entries outside [0, L) or where x is 0)
 * d_status    device int32 [P] (may be NULL): pixels with BPDN_PX_NONFINITE or
 *             BPDN_PX_SUPPORT_OVERFLOW get K_hat = -1
 * s_max       1..BPDN_MAX_SMAX;  kmax  1..BPDN_MAX_KSEL
 * d_khat      device int32 [P] out: K_hat (or -1)
 * d_s_hat     device float64 [P, kmax] out: elevations in metres, ascending; NaN past K_hat
 * d_gamma_hat device c128 [P, kmax] out: amplitudes matching d_s_hat; 0 past K_hat
 * Asynchronous on cuda_stream; allocates nothing.  Returns BPDN_EINVAL (NULL pointer,
 * bad s_max / kmax, P < 0) or BPDN_EALIGN before launching anything.
 */
int bpdn_select(bpdn_op_t op, const void *d_g, int64_t P, const void *d_x, const int32_t *d_support,
                const int32_t *d_nsupp, const int32_t *d_status, int32_t s_max, int32_t kmax,
                double penalty, int32_t *d_khat, double *d_s_hat, void *d_gamma_hat, void *cuda_stream);

/*
 * Pre-classification before the L1 solve: the hybrid processing the paper recommends
 * (Sec. I: a fast linear estimator for the pixels that need no super-resolution and the
 * L1 solve only for the others; Sec. V expects a further speed-up of about 50 from it).
 * The paper leaves the classifier to its reference; the library's reading, per pixel:
 *   u = A^H g  (beamforming on the grid, the classic linear estimator)
 *   class 0  2 max_l |u_l| <= lambda: x* = 0 exactly (the zero vector satisfies Eq. 6's
 *            optimality conditions), K_hat = 0
 *   class 1  otherwise the single-scatterer linear estimate -- s^ = the elevation in
 *            [s_{l^-1}, s_{l^+1}] (l^ = argmax |u_l|) where |a(s)^H g| peaks,
 *            gamma^ = a(s^)^H g / N -- when its residual r = g - gamma^ a(s^) satisfies
 *            2 max_l |a_l^H r| <= lambda: K_hat = 1 with (s^, gamma^).  This is the linear
 *            estimator's answer, not the minimiser of Eq. 6.
 *   class 2  every other pixel (and any pixel with non-finite g): left to the L1 path
 *            (bpdn_solve with the refit, then bpdn_select); K_hat = -1 here.
 * The class decisions are taken in FP64 (FP32 beam sums, grid points within 1e-4 of a
 * decision boundary recomputed in FP64); s^ by a safeguarded Newton iteration in FP64.
 * Elevation-only operators (bpdn_make_operator); others are refused.
 *
 * d_g, P, d_lambda, lambda_per_pixel   as in bpdn_solve
 * kmax            1..BPDN_MAX_KSEL: row length of d_s_hat / d_gamma_hat (as bpdn_select)
 * d_class         device int32 [P] out: 0, 1 or 2
 * d_khat          device int32 [P] out: 0, 1, or -1 for class 2
 * d_s_hat         device float64 [P, kmax] out: s^ in column 0 for class 1, NaN elsewhere
 * d_gamma_hat     device c128 [P, kmax] out (16-byte aligned): gamma^ for class 1, 0 elsewhere
 * d_idx           device int64 [P] out: the class-2 pixels, in the order found (not sorted)
 * d_count         device uint64 [1] out: how many (cleared by the call on cuda_stream)
 * d_g_compact     device c64 [P, N] out, or NULL: row i = g of pixel d_idx[i], ready for
 *                 bpdn_solve on the first *d_count rows
 * Asynchronous on cuda_stream; allocates nothing.  Returns BPDN_EINVAL / BPDN_EALIGN /
 * BPDN_ESTATE before launching anything.
 */
int bpdn_classify(bpdn_op_t op, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
                  int32_t kmax, int32_t *d_class, int32_t *d_khat, double *d_s_hat, void *d_gamma_hat,
                  int64_t *d_idx, uint64_t *d_count, void *d_g_compact, void *cuda_stream);

/*
 * Write the selection of the class-2 pixels (bpdn_select run on the compacted rows of
 * bpdn_classify) into the full outputs: row i of d_khat_c / d_s_hat_c / d_gamma_hat_c goes
 * to pixel d_idx[i], for i < P_c.  Shapes and alignment as in bpdn_select with the same
 * kmax.  Asynchronous on cuda_stream; BPDN_EINVAL / BPDN_EALIGN before any launch.
 */
int bpdn_classify_merge(int64_t P_c, const int64_t *d_idx, int32_t kmax, const int32_t *d_khat_c,
                        const double *d_s_hat_c, const void *d_gamma_hat_c, int32_t *d_khat, double *d_s_hat,
                        void *d_gamma_hat, void *cuda_stream);

/*
 * bpdn_solve without a workspace, for callers that cannot allocate device memory
 * (for example a processing chain whose host application owns every GPU buffer
 * and forbids its modules to call cudaMalloc).  The paper has no counterpart: it
 * is a deployment variant of bpdn_solve, with the same arguments minus the
 * workspace and the same results.
 *
 * The iteration kernel's scratch (a work counter) lives in a file-scope device
 * array of 256 bytes that every GPU loading the library keeps until the process
 * exits.  The first call on a device looks up its address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is kept for the life
 * of the process, so after a cudaDeviceReset of a device do not call this entry point
 * on that device again (the kept address would be stale).  All calls share the array and
 * each clears what it uses, so calls whose work overlaps on the GPU race and must
 * be serialised by the caller.  A solve whose scratch would exceed 256 bytes is
 * rejected with BPDN_ESIZE: randomized blocks, the pixel-per-thread kernel and every solve
 * that runs the split-grid kernel (see bpdn_solve; kernel 1 keeps FP32 solves of up to
 * 1024 points on the grid-point kernel, which needs none).  No device memory is allocated
 * or freed.
 */
int bpdn_solve_noalloc(bpdn_op_t op, const void *d_g, int64_t P, const float *d_lambda,
                       int32_t lambda_per_pixel, const bpdn_options *opt, void *d_x,
                       int32_t *d_support, int32_t *d_nsupp, int32_t *d_status, int32_t *d_iters,
                       int32_t *d_nbt, void *cuda_stream);

/* Thread-local message of the last failed call ("" if none). */
const char *bpdn_last_error(void);

/* Library version string. */
const char *bpdn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BPDN_H */
