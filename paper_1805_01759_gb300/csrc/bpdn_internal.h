// Internal declarations shared by the libbpdn translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bpdn.h"

namespace bpdn {

constexpr uint32_t kOpMagic = 0xB9D4A11Cu;
constexpr int kTilePixels = 16;   // pixel slots per CTA of the iteration kernel
constexpr int kRefitMax = BPDN_MAX_SMAX;

// Host handle of one stack's operator.  All device pointers point into the
// caller's workspace.
struct OpHandle {
    uint32_t magic;
    int device;
    int N, L;
    int Lpad;     // L rounded up to a multiple of 32 (= threads of the iteration CTA)
    int lda;      // row stride (floats) of the planar FP32 tables: Lpad + 1 (odd, bank spread)
    double wavelength, range, s_min, s_max, ds;
    double lambda_max, lipschitz;
    // device tables
    float *A_re, *A_im;  // [N][lda], zero for l >= L
    double2 *A64;        // [N][L]
    double2 *h;          // [2L-1], h[d + L - 1]
    double2 *aah;        // [N][N]
    double *xi;          // [N]
    double *scal;        // [8] device scalars (lambda_max, ...)
    size_t ws_bytes;
    // multi-component grid (Eq. 4): elevation x motion coefficients; A^H A is then not
    // Toeplitz, h is unused and kernels build Gram entries from A64
    int md;
    int Ls;  // elevation points (= L when md == 0)
};

// The motion part of a multi-component grid: grid index l = l_s + Ls (l_1 + Lp[0] l_2),
// A_nl = exp(-j 2 pi (xi_n s_{l_s} + eta[0][n] p_{0,l_1} + eta[1][n] p_{1,l_2})).
struct MdGrid {
    int M;  // motion dimensions, 1 or BPDN_MAX_MOTION
    int Lp[BPDN_MAX_MOTION];
    double pmin[BPDN_MAX_MOTION], pmax[BPDN_MAX_MOTION];
    double eta[BPDN_MAX_MOTION][BPDN_MAX_N];
};

// Workspace layout of an operator (offsets in bytes, 256-aligned sections).
struct OpLayout {
    size_t A_re, A_im, A64, h, aah, xi, scal, total;
};
OpLayout op_layout(int N, int L);

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Set the thread-local error message; returns code.
int set_error(int code, const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);

// ---- launches (each returns a cudaError_t from the launch) ----
cudaError_t launch_make_operator(const OpHandle &op, const double *d_b, cudaStream_t s);
cudaError_t launch_make_operator_md(const OpHandle &op, const double *d_b, const MdGrid &md, cudaStream_t s);

struct SolvePlan;
// bpdn_solve's argument checks and launch records (sp->a.P == 0: nothing to launch)
// (split_at: the split-grid kernel's scratch outside the workspace, for bpdn_solve_ragged)
int solve_plan(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
               const bpdn_options *opt, void *d_x, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               int32_t *d_iters, int32_t *d_nbt, void *d_workspace, size_t workspace_bytes, SolvePlan *sp,
               unsigned char *split_at = nullptr);
// whether a solve with these options runs the split-grid FP32 kernel (it then needs that
// kernel's scratch: rbpg_split_scratch_bytes)
bool solve_uses_split(const OpHandle *op, const bpdn_options *opt);
int device_sms(int dev);
// bpdn_solve's argument checks, followed by its launches when `launch` is true
int solve_impl(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
               const bpdn_options *opt, void *d_x, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               int32_t *d_iters, int32_t *d_nbt, void *d_workspace, size_t workspace_bytes, void *cuda_stream,
               bool launch);
cudaError_t launch_export(const OpHandle &op, int what, void *dst, cudaStream_t s);

struct SolveLaunch {
    const float2 *g;
    int64_t P;
    const float *lam;
    int lam_pp;
    float2 *x;
    int32_t *nsupp, *status, *iters, *nbt;
    unsigned long long *counter;
    int max_iter;
    float tol;
    float c_alpha;
    float alpha0;
    int max_bt;
    int precision;
    int groups;  // slot groups of 8 pixels per CTA: 0 = the kernel's choice, 1 or 2
    int *err;    // set to 1 if a bounded wait ran out (may be NULL)
    // randomized blocks of the grid (blocks >= 2; Eqs. 13-14)
    int blocks;
    unsigned seed;
    double2 *bscratch;  // [blocks][N][N]: A_j A_j^H
    double *blip;       // [blocks]: lambda_max(A_j A_j^H)
    double *cum;        // [blocks]: cumulative draw probabilities, last = 1
    // pixel-per-thread BF16 kernel (k_rbpg_px): per-slot iterate lists and residual state,
    // or NULL when the solve runs the grid-point-per-thread kernel
    unsigned char *px_scratch;
    // split-grid FP32 kernel (k_rbpg_split, grids of more than 1024 points): the transposed
    // operator and the per-CTA row buffers, or NULL
    unsigned char *split_scratch;
};
// iteration kernel (a.precision 0: FP32 CUDA cores, 1: BF16 tensor cores)
cudaError_t launch_rbpg(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s);
// the pixel-per-thread BF16 iteration kernel: bytes of its per-slot scratch on this device
// (0 when the operator's sizes do not suit it), and its launch
size_t rbpg_px_scratch_bytes(const OpHandle &op, int64_t P, int num_sms, int max_smem);
cudaError_t launch_rbpg_px(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s);
// the split-grid iteration kernel (FP32 CUDA cores, or BF16 tensor cores with precision 1):
// "" when it takes the operator, else the reason; bytes of its scratch for P pixels on this
// device (0: it cannot launch); its launch (the variant follows a.precision)
const char *rbpg_split_check(const OpHandle &op, int precision, int blocks, int max_smem);
size_t rbpg_split_scratch_bytes(const OpHandle &op, int precision, int64_t P, int num_sms);
cudaError_t launch_rbpg_split(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s);
// many stacks in persistent launches, one per kernel variant present (at most 64 stacks each)
cudaError_t launch_rbpg_batch(const OpHandle *const *ops, const SolveLaunch *as, int n, int num_sms,
                              cudaStream_t s);
// "" when the operator's sizes suit the kernel at this precision, else the reason
const char *rbpg_check(const OpHandle &op, int precision, int groups, int max_smem);
// Algorithm 1 with randomized blocks (a.blocks >= 2), FP32, one warp per pixel
cudaError_t launch_rbpg_block(const OpHandle &op, const SolveLaunch &a, cudaStream_t s);
const char *rbpg_block_check(const OpHandle &op, int blocks, int max_smem);
// Eq. 14's draw table: lambda_max(A_j A_j^H) per block and cumulative probabilities
cudaError_t launch_block_probs(const OpHandle &op, int J, double2 *M, double *lmax, double *cum, cudaStream_t s);
// scratch bytes of a solve with `blocks` (0 when blocks < 2)
size_t block_scratch_bytes(int blocks);

struct RefitLaunch {
    const float2 *g;
    int64_t P;
    const float *lam;
    int lam_pp;
    const float2 *x_in;
    float2 *x_out;
    int32_t *support, *nsupp, *status;
    int s_max;
    int rounds;
    // scratch of the split refit (refit_scratch_bytes(P)), or NULL: one launch
    unsigned char *split;
};
cudaError_t launch_refit(const OpHandle &op, const RefitLaunch &a, cudaStream_t s);
// bytes of scratch the split refit needs for P pixels (256-byte multiple)
size_t refit_scratch_bytes(int64_t P);
// the least solve workspace (work counter, error word, block draw table and matrices);
// bpdn_solve_workspace_bytes adds the split refit's scratch to it
size_t solve_min_workspace_bytes(const bpdn_options *opt);

struct SolvePlan {
    OpHandle *op;
    SolveLaunch a;
    RefitLaunch r;
    bool refit;
};

struct BackwardLaunch {
    int64_t P;
    const float *lam;
    int lam_pp;
    const float2 *x;
    const int32_t *support, *nsupp;
    const int32_t *status;  // may be NULL
    int s_max;
    const float2 *dLdx;
    float2 *dLdg;
    float *dLdlam;  // [P] (lam_pp) or [1]
    double *part;   // [P] per-pixel dL/dlambda terms when lambda is shared
};
cudaError_t launch_backward(const OpHandle &op, const BackwardLaunch &a, cudaStream_t s);

struct SelectLaunch {
    int64_t P;
    const float2 *g, *x;
    const int32_t *support, *nsupp;
    const int32_t *status;  // may be NULL
    int s_max, kmax;
    double penalty;         // <= 0: 3 ln(2N)
    int32_t *khat;
    double *s_hat;
    double2 *gamma_hat;
};
cudaError_t launch_select(const OpHandle &op, const SelectLaunch &a, cudaStream_t s);

}  // namespace bpdn
