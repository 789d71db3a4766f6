// C ABI of libbpdn (declared in include/bpdn.h): argument checks, workspace
// layout, and kernel launches on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "bpdn_internal.h"

namespace bpdn {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess)
        return BPDN_OK;
    return set_error(BPDN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

OpLayout op_layout(int N, int L)
{
    OpLayout o;
    const int Lpad = round_up(L, 32);
    const int lda = Lpad + 1;
    size_t off = 0;
    o.A_re = off; off = a256(off + sizeof(float) * (size_t)N * lda);
    o.A_im = off; off = a256(off + sizeof(float) * (size_t)N * lda);
    o.A64 = off;  off = a256(off + sizeof(double2) * (size_t)N * L);
    o.h = off;    off = a256(off + sizeof(double2) * (size_t)(2 * L - 1));
    o.aah = off;  off = a256(off + sizeof(double2) * (size_t)N * N);
    o.xi = off;   off = a256(off + sizeof(double) * (size_t)N);
    o.scal = off; off = a256(off + sizeof(double) * 8);
    o.total = off;
    return o;
}

static int current_device(int *dev)
{
    cudaError_t e = cudaGetDevice(dev);
    return check_cuda(e, "cudaGetDevice");
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_op(bpdn_op_t h, OpHandle **out)
{
    OpHandle *op = reinterpret_cast<OpHandle *>(h);
    if (!op || op->magic != kOpMagic)
        return set_error(BPDN_EINVAL, "invalid operator handle");
    int dev = -1;
    int rc = current_device(&dev);
    if (rc)
        return rc;
    if (dev != op->device)
        return set_error(BPDN_ESTATE, "operator lives on device %d but device %d is current",
                         op->device, dev);
    *out = op;
    return BPDN_OK;
}

static int num_sms(int dev)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
        v = 1;
    return v;
}

static int max_smem_optin(int dev)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        v = 48 * 1024;
    return v;
}

static int check_options(const bpdn_options *o)
{
    if (!o)
        return set_error(BPDN_EINVAL, "options pointer is NULL");
    if (o->max_iter < 0)
        return set_error(BPDN_EINVAL, "max_iter must be >= 0");
    if (!(o->tol >= 0.f) || !isfinite(o->tol))
        return set_error(BPDN_EINVAL, "tol must be finite and >= 0");
    if (!(o->c_alpha > 0.f && o->c_alpha < 1.f))
        return set_error(BPDN_EINVAL, "c_alpha must lie in (0, 1)");
    if (!(o->alpha0_scale > 0.f) || !isfinite(o->alpha0_scale))
        return set_error(BPDN_EINVAL, "alpha0_scale must be finite and > 0");
    if (o->precision != 0 && o->precision != 1)
        return set_error(BPDN_EINVAL, "precision must be 0 (FP32) or 1 (BF16)");
    if (o->refit != 0 && o->refit != 1)
        return set_error(BPDN_EINVAL, "refit must be 0 or 1");
    if (o->s_max < 1 || o->s_max > BPDN_MAX_SMAX)
        return set_error(BPDN_EINVAL, "s_max must lie in [1, %d]", BPDN_MAX_SMAX);
    if (o->max_bt < 0)
        return set_error(BPDN_EINVAL, "max_bt must be >= 0");
    if (o->refit_rounds < 0 || o->refit_rounds > 64)
        return set_error(BPDN_EINVAL, "refit_rounds must lie in [0, 64]");
    if (o->tile_pixels != 0 && o->tile_pixels != 8 && o->tile_pixels != 16 && o->tile_pixels != 128)
        return set_error(BPDN_EINVAL, "tile_pixels must be 0 (library choice), 8, 16 or 128");
    if (o->tile_pixels == 128 && o->precision != 1)
        return set_error(BPDN_EINVAL, "tile_pixels 128 (one pixel per thread) is the BF16 kernel: precision 1");
    if (o->kernel < 0 || o->kernel > 2)
        return set_error(BPDN_EINVAL, "kernel must be 0 (library choice), 1 (grid-point) or 2 (split-grid)");
    if (o->kernel == 2 && (o->tile_pixels != 0 || o->blocks >= 2))
        return set_error(BPDN_EINVAL, "kernel 2 (split-grid) runs with tile_pixels 0 and blocks <= 1");
    if (o->blocks < 0 || o->blocks > 8)
        return set_error(BPDN_EINVAL, "blocks must lie in [0, 8]");
    if (o->blocks >= 2 && o->precision != 0)
        return set_error(BPDN_EINVAL, "randomized blocks (blocks >= 2) run in FP32 only (precision 0)");
    if (o->blocks >= 2 && o->max_iter > (1 << 27))
        return set_error(BPDN_EINVAL, "max_iter must be <= 2^27 with randomized blocks");
    return BPDN_OK;
}

}  // namespace bpdn

using namespace bpdn;

namespace bpdn {
size_t solve_min_workspace_bytes(const bpdn_options *opt)
{
    // a 64-bit work counter, an error word and the block draw table, padded; with
    // randomized blocks, A_j A_j^H of every block after that
    return 256 + block_scratch_bytes(opt ? opt->blocks : 0);
}

// scratch of the pixel-per-thread BF16 iteration kernel for this solve (0: the solve runs the
// grid-point-per-thread kernel): precision 1, one block per pixel, tile_pixels 0 or 128, and
// sizes the kernel takes
static size_t px_scratch_for(const OpHandle *op, int64_t P, const bpdn_options *opt)
{
    if (!op || !opt || opt->precision != 1 || opt->blocks >= 2 || opt->tile_pixels != 128)
        return 0;
    return rbpg_px_scratch_bytes(*op, P, num_sms(op->device), max_smem_optin(op->device));
}

// The split-grid FP32 kernel runs grids of more than 1024 points, and FP32 solves of
// 513..1024 points with the library's choice of tile (tile_pixels 0, no randomized
// blocks): there the grid-point kernel fits only one group of slots per CTA, and the
// split kernel is faster (1.2-1.7x on such stacks).  The choice depends on the operator and
// the options only, never on the workspace, so that results do not depend on it.
bool solve_uses_split(const OpHandle *op, const bpdn_options *opt)
{
    if (!op)
        return false;
    if (opt && opt->kernel == 2)
        return true;
    if (op->L > 1024)
        return true;  // (kernel 1 is then refused by the plan)
    if (!opt || opt->kernel == 1 || opt->tile_pixels != 0 || opt->blocks >= 2)
        return false;
    if (opt->precision == 1)  // the grid-point BF16 kernel takes 2N <= 128 and L <= 512
        return op->L > 512 || 2 * op->N > 128;
    return op->L > 512;
}

static bool split_grid(const OpHandle *op, const bpdn_options *opt) { return solve_uses_split(op, opt); }

// scratch of the split-grid kernel for this solve (0 when the grid does not need it or the
// options or sizes rule it out: solve_plan then names the reason)
static size_t split_scratch_for(const OpHandle *op, int64_t P, const bpdn_options *opt)
{
    if (!split_grid(op, opt) || !opt || opt->tile_pixels != 0 ||
        rbpg_split_check(*op, opt->precision, opt->blocks, max_smem_optin(op->device))[0] != '\0')
        return 0;
    return rbpg_split_scratch_bytes(*op, opt->precision, P, num_sms(op->device));
}

static int check_solve_buffers(const OpHandle *op, const void *d_g, int64_t P, const float *d_lambda,
                               const void *d_x, const int32_t *d_status)
{
    if (P < 0)
        return set_error(BPDN_EINVAL, "P must be >= 0");
    if (P > ((int64_t)1 << 40))
        return set_error(BPDN_ESIZE, "P = %lld too large", (long long)P);
    if (P == 0)
        return BPDN_OK;
    if (!d_g || !d_lambda || !d_x || !d_status)
        return set_error(BPDN_EINVAL, "g, lambda, x and status pointers must be non-NULL");
    if (!aligned(d_g, 8) || !aligned(d_x, 8) || !aligned(d_lambda, 4) || !aligned(d_status, 4))
        return set_error(BPDN_EALIGN, "g and x must be 8-byte aligned, lambda and status 4-byte");
    (void)op;
    return BPDN_OK;
}

// Checks every argument of a solve; launches it when `launch` is true.
int solve_plan(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
               const bpdn_options *opt, void *d_x, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               int32_t *d_iters, int32_t *d_nbt, void *d_workspace, size_t workspace_bytes, SolvePlan *sp,
               unsigned char *split_at)
{
    OpHandle *op = nullptr;
    int rc = check_op(h, &op);
    if (rc)
        return rc;
    rc = check_options(opt);
    if (rc)
        return rc;
    rc = check_solve_buffers(op, d_g, P, d_lambda, d_x, d_status);
    if (rc)
        return rc;
    sp->op = op;
    sp->refit = false;
    sp->a.P = 0;
    if (P == 0)
        return BPDN_OK;
    if (!d_iters)
        return set_error(BPDN_EINVAL, "iters pointer must be non-NULL");
    if (!d_workspace || workspace_bytes < solve_min_workspace_bytes(opt))
        return set_error(BPDN_ESIZE, "solve workspace too small");
    if (!aligned(d_workspace, 256))
        return set_error(BPDN_EALIGN, "solve workspace must be 256-byte aligned");
    if (opt->refit && d_support && !aligned(d_support, 4))
        return set_error(BPDN_EALIGN, "support must be 4-byte aligned");
    // the pixel-per-thread BF16 kernel when it suits the sizes and the workspace holds its scratch
    const size_t base = solve_min_workspace_bytes(opt);
    const bool split = split_grid(op, opt);
    const size_t pxb = split ? 0 : px_scratch_for(op, P, opt);
    const bool use_px = pxb > 0 && workspace_bytes >= base + pxb;
    const size_t spb = split_scratch_for(op, P, opt);
    if (opt->tile_pixels == 128 && !use_px && !split)
        return set_error(BPDN_ESIZE, pxb ? "tile_pixels 128: the workspace does not hold the kernel's scratch"
                                         : "tile_pixels 128 needs 2N <= 64 and the operator within shared memory");
    const char *why = (opt->kernel == 1 && op->L > 1024) ? "the grid-point kernel (kernel 1) handles L <= 1024"
                      : split ? (opt->tile_pixels != 0 ? "grids of more than 1024 points take tile_pixels 0"
                                                     : rbpg_split_check(*op, opt->precision, opt->blocks,
                                                                        max_smem_optin(op->device)))
                      : (opt->blocks >= 2) ? rbpg_block_check(*op, opt->blocks, max_smem_optin(op->device))
                      : use_px             ? ""
                                           : rbpg_check(*op, opt->precision, opt->tile_pixels / 8,
                                                        max_smem_optin(op->device));
    if (why[0] != '\0')
        return set_error(BPDN_ESIZE, "N = %d, L = %d, precision %d: %s", op->N, op->L, opt->precision, why);
    if (split && (spb == 0 || (!split_at && workspace_bytes < base + spb)))
        return set_error(BPDN_ESIZE, "L = %d: the workspace does not hold the split-grid kernel's scratch "
                                     "(bpdn_solve_workspace_bytes gives the size)", op->L);
    SolveLaunch &a = sp->a;
    a.g = (const float2 *)d_g;
    a.P = P;
    a.lam = d_lambda;
    a.lam_pp = lambda_per_pixel ? 1 : 0;
    a.x = (float2 *)d_x;
    a.nsupp = d_nsupp;
    a.status = d_status;
    a.iters = d_iters;
    a.nbt = d_nbt;
    // work counter (8 bytes) and the kernel's error word (4 bytes) at the workspace start
    a.counter = (unsigned long long *)d_workspace;
    a.max_iter = opt->max_iter;
    a.tol = opt->tol;
    a.c_alpha = opt->c_alpha;
    a.alpha0 = (float)(opt->alpha0_scale / (2.0 * op->N));
    a.max_bt = opt->max_bt;
    a.precision = opt->precision;
    a.groups = opt->tile_pixels / 8;
    a.err = (int *)((char *)d_workspace + 8);
    // randomized blocks: draw table at bytes 16.., A_j A_j^H after the first 256 bytes
    a.blocks = opt->blocks >= 2 ? opt->blocks : 0;
    a.seed = opt->seed;
    a.blip = (double *)((char *)d_workspace + 16);
    a.cum = (double *)((char *)d_workspace + 16 + 8 * 8);
    a.bscratch = a.blocks ? (double2 *)((char *)d_workspace + 256) : nullptr;
    a.px_scratch = use_px ? (unsigned char *)d_workspace + base : nullptr;
    a.split_scratch = !split ? nullptr : split_at ? split_at : (unsigned char *)d_workspace + base;
    sp->refit = opt->refit != 0;
    RefitLaunch &r = sp->r;
    r.g = a.g;
    r.P = P;
    r.lam = d_lambda;
    r.lam_pp = a.lam_pp;
    r.x_in = a.x;
    r.x_out = a.x;
    r.support = d_support;
    r.nsupp = d_nsupp;
    r.status = d_status;
    r.s_max = opt->s_max;
    r.rounds = opt->refit_rounds;
    // the split refit when the workspace holds its scratch (after the iteration kernel's), else
    // the fused refit
    const size_t rbase = base + (use_px ? pxb : 0) + (split && !split_at ? spb : 0);
    r.split = (workspace_bytes >= rbase + refit_scratch_bytes(P)) ? (unsigned char *)d_workspace + rbase : nullptr;
    return BPDN_OK;
}

int solve_impl(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
               const bpdn_options *opt, void *d_x, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               int32_t *d_iters, int32_t *d_nbt, void *d_workspace, size_t workspace_bytes, void *cuda_stream,
               bool launch)
{
    SolvePlan sp;
    int rc = solve_plan(h, d_g, P, d_lambda, lambda_per_pixel, opt, d_x, d_support, d_nsupp, d_status, d_iters,
                        d_nbt, d_workspace, workspace_bytes, &sp);
    if (rc || !launch || sp.a.P == 0)
        return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rc = check_cuda(cudaMemsetAsync(sp.a.counter, 0, 16, s), "reset work counter");
    if (rc)
        return rc;
    if (sp.a.blocks) {
        rc = check_cuda(launch_block_probs(*sp.op, sp.a.blocks, sp.a.bscratch, sp.a.blip, sp.a.cum, s),
                        "block draw table");
        if (rc)
            return rc;
        rc = check_cuda(launch_rbpg_block(*sp.op, sp.a, s), "block iteration kernel");
    } else if (sp.a.split_scratch) {
        rc = check_cuda(launch_rbpg_split(*sp.op, sp.a, num_sms(sp.op->device), s), "iteration kernel (split grid)");
    } else if (sp.a.px_scratch) {
        rc = check_cuda(launch_rbpg_px(*sp.op, sp.a, num_sms(sp.op->device), s), "iteration kernel (pixel per thread)");
    } else {
        rc = check_cuda(launch_rbpg(*sp.op, sp.a, num_sms(sp.op->device), s), "iteration kernel");
    }
    if (rc || !sp.refit)
        return rc;
    return check_cuda(launch_refit(*sp.op, sp.r, s), "refit kernel");
}

int device_sms(int dev) { return num_sms(dev); }
}  // namespace bpdn

extern "C" {

const char *bpdn_last_error(void) { return g_err; }

const char *bpdn_version(void) { return "bpdn-gb300 0.1 (sm_103a)"; }

void bpdn_default_options(bpdn_options *opt)
{
    if (!opt)
        return;
    memset(opt, 0, sizeof(*opt));
    opt->max_iter = 500;
    opt->tol = 1e-6f;
    opt->c_alpha = 0.5f;
    opt->alpha0_scale = 1.0f;
    opt->precision = 0;
    opt->refit = 1;
    opt->s_max = BPDN_MAX_SMAX;
    opt->max_bt = 64;
    opt->tile_pixels = 0;
    opt->refit_rounds = 4;
}

size_t bpdn_op_workspace_bytes(int32_t N, int32_t L)
{
    if (N < 1 || N > BPDN_MAX_N || L < 1 || L > BPDN_MAX_L)
        return 0;
    return op_layout(N, L).total;
}

}  // extern "C"

namespace bpdn {
static int make_operator_impl(const double *baselines_m, int32_t N, double wavelength_m, double range_m,
                              double s_min_m, double s_max_m, int32_t L, int32_t Ls, const MdGrid *md,
                              void *d_workspace, size_t workspace_bytes, void *cuda_stream, bpdn_op_t *out)
{
    if (!out)
        return set_error(BPDN_EINVAL, "out is NULL");
    *out = nullptr;
    if (!baselines_m || !d_workspace)
        return set_error(BPDN_EINVAL, "baselines or workspace pointer is NULL");
    if (N < 1 || N > BPDN_MAX_N)
        return set_error(BPDN_ESIZE, "N = %d outside [1, %d]", N, BPDN_MAX_N);
    if (L < 1 || L > BPDN_MAX_L)
        return set_error(BPDN_ESIZE, "L = %d outside [1, %d]", L, BPDN_MAX_L);
    for (int n = 0; n < N; ++n)
        if (!isfinite(baselines_m[n]))
            return set_error(BPDN_EINVAL, "baseline %d is not finite", n);
    if (!(wavelength_m > 0.0) || !isfinite(wavelength_m) || !(range_m > 0.0) || !isfinite(range_m))
        return set_error(BPDN_EINVAL, "wavelength and range must be finite and > 0");
    if (!isfinite(s_min_m) || !isfinite(s_max_m) || s_max_m < s_min_m)
        return set_error(BPDN_EINVAL, "elevation extent must be finite with s_min <= s_max");
    if (Ls > 1 && !(s_max_m > s_min_m))
        return set_error(BPDN_EINVAL, "more than one elevation point needs s_max > s_min");
    const OpLayout lay = op_layout(N, L);
    if (workspace_bytes < lay.total)
        return set_error(BPDN_ESIZE, "operator workspace %zu bytes < %zu needed", workspace_bytes,
                         lay.total);
    if (!aligned(d_workspace, 256))
        return set_error(BPDN_EALIGN, "operator workspace must be 256-byte aligned");
    int dev = 0;
    int rc = current_device(&dev);
    if (rc)
        return rc;

    OpHandle *op = (OpHandle *)calloc(1, sizeof(OpHandle));
    if (!op)
        return set_error(BPDN_EINVAL, "out of host memory");
    op->magic = kOpMagic;
    op->device = dev;
    op->N = N;
    op->L = L;
    op->Lpad = round_up(L, 32);
    op->lda = op->Lpad + 1;
    op->wavelength = wavelength_m;
    op->range = range_m;
    op->s_min = s_min_m;
    op->s_max = s_max_m;
    op->ds = (Ls > 1) ? (s_max_m - s_min_m) / (double)(Ls - 1) : 0.0;
    op->md = md ? 1 : 0;
    op->Ls = Ls;
    char *base = (char *)d_workspace;
    op->A_re = (float *)(base + lay.A_re);
    op->A_im = (float *)(base + lay.A_im);
    op->A64 = (double2 *)(base + lay.A64);
    op->h = (double2 *)(base + lay.h);
    op->aah = (double2 *)(base + lay.aah);
    op->xi = (double *)(base + lay.xi);
    op->scal = (double *)(base + lay.scal);
    op->ws_bytes = workspace_bytes;

    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the baselines are staged in the xi table; k_xi turns each b_n into xi_n in place
    double *d_b = op->xi;
    rc = check_cuda(cudaMemcpyAsync(d_b, baselines_m, sizeof(double) * N, cudaMemcpyHostToDevice, s),
                    "copy baselines");
    if (!rc)
        rc = check_cuda(md ? launch_make_operator_md(*op, d_b, *md, s) : launch_make_operator(*op, d_b, s),
                        "operator kernels");
    double lmax = 0.0;
    if (!rc)
        rc = check_cuda(cudaMemcpyAsync(&lmax, op->scal, sizeof(double), cudaMemcpyDeviceToHost, s),
                        "read lambda_max");
    if (!rc)
        rc = check_cuda(cudaStreamSynchronize(s), "synchronise operator stream");
    if (rc) {
        free(op);
        return rc;
    }
    op->lambda_max = lmax;
    op->lipschitz = 2.0 * lmax;
    *out = reinterpret_cast<bpdn_op_t>(op);
    return BPDN_OK;
}

}  // namespace bpdn

extern "C" {

int bpdn_make_operator(const double *baselines_m, int32_t N, double wavelength_m, double range_m,
                       double s_min_m, double s_max_m, int32_t L, void *d_workspace,
                       size_t workspace_bytes, void *cuda_stream, bpdn_op_t *out)
{
    return make_operator_impl(baselines_m, N, wavelength_m, range_m, s_min_m, s_max_m, L, L, nullptr,
                              d_workspace, workspace_bytes, cuda_stream, out);
}

int bpdn_make_operator_md(const double *baselines_m, int32_t N, double wavelength_m, double range_m,
                          double s_min_m, double s_max_m, int32_t L_s, int32_t M, const double *eta,
                          const double *p_min, const double *p_max, const int32_t *L_p, void *d_workspace,
                          size_t workspace_bytes, void *cuda_stream, bpdn_op_t *out)
{
    if (!out)
        return set_error(BPDN_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 1 || M > BPDN_MAX_MOTION)
        return set_error(BPDN_EINVAL, "M must lie in 1..%d", BPDN_MAX_MOTION);
    if (!eta || !p_min || !p_max || !L_p)
        return set_error(BPDN_EINVAL, "eta, p_min, p_max and L_p must be non-NULL");
    if (N < 1 || N > BPDN_MAX_N)
        return set_error(BPDN_ESIZE, "N = %d outside [1, %d]", N, BPDN_MAX_N);
    if (L_s < 1 || L_s > BPDN_MAX_L)
        return set_error(BPDN_ESIZE, "L_s = %d outside [1, %d]", L_s, BPDN_MAX_L);
    MdGrid md;
    memset(&md, 0, sizeof(md));
    md.M = M;
    long long L = L_s;
    for (int m = 0; m < M; ++m) {
        if (L_p[m] < 1 || L_p[m] > BPDN_MAX_L)
            return set_error(BPDN_ESIZE, "L_p[%d] = %d outside [1, %d]", m, L_p[m], BPDN_MAX_L);
        if (!isfinite(p_min[m]) || !isfinite(p_max[m]) || p_max[m] < p_min[m])
            return set_error(BPDN_EINVAL, "motion grid %d must be finite with p_min <= p_max", m);
        if (L_p[m] > 1 && !(p_max[m] > p_min[m]))
            return set_error(BPDN_EINVAL, "motion grid %d: more than one point needs p_max > p_min", m);
        for (int n = 0; n < N; ++n) {
            if (!isfinite(eta[(size_t)m * N + n]))
                return set_error(BPDN_EINVAL, "eta[%d][%d] is not finite", m, n);
            md.eta[m][n] = eta[(size_t)m * N + n];
        }
        md.Lp[m] = L_p[m];
        md.pmin[m] = p_min[m];
        md.pmax[m] = p_max[m];
        L *= L_p[m];
        if (L > BPDN_MAX_L)
            return set_error(BPDN_ESIZE, "grid of %lld points exceeds %d", L, BPDN_MAX_L);
    }
    return make_operator_impl(baselines_m, N, wavelength_m, range_m, s_min_m, s_max_m, (int32_t)L, L_s, &md,
                              d_workspace, workspace_bytes, cuda_stream, out);
}

void bpdn_destroy_operator(bpdn_op_t h)
{
    OpHandle *op = reinterpret_cast<OpHandle *>(h);
    if (!op || op->magic != kOpMagic)
        return;
    op->magic = 0;
    free(op);
}

int bpdn_op_info(bpdn_op_t h, int32_t *N, int32_t *L, double *ds_m, double *lipschitz)
{
    OpHandle *op = reinterpret_cast<OpHandle *>(h);
    if (!op || op->magic != kOpMagic)
        return set_error(BPDN_EINVAL, "invalid operator handle");
    if (N)
        *N = op->N;
    if (L)
        *L = op->L;
    if (ds_m)
        *ds_m = op->ds;
    if (lipschitz)
        *lipschitz = op->lipschitz;
    return BPDN_OK;
}

double bpdn_op_lipschitz(bpdn_op_t h)
{
    OpHandle *op = reinterpret_cast<OpHandle *>(h);
    if (!op || op->magic != kOpMagic)
        return NAN;
    return op->lipschitz;
}

int bpdn_op_export(bpdn_op_t h, int32_t what, void *d_dst, size_t dst_bytes, void *cuda_stream)
{
    OpHandle *op = nullptr;
    int rc = check_op(h, &op);
    if (rc)
        return rc;
    if (!d_dst)
        return set_error(BPDN_EINVAL, "destination is NULL");
    size_t need = 0;
    switch (what) {
    case 0: need = 8 * (size_t)op->N * op->L; break;
    case 1: need = 16 * (size_t)op->N * op->L; break;
    case 2:
        if (op->md)
            return set_error(BPDN_EINVAL, "a multi-component operator has no Toeplitz generator");
        need = 16 * (size_t)(2 * op->L - 1);
        break;
    case 3: need = 16 * (size_t)op->N * op->N; break;
    default: return set_error(BPDN_EINVAL, "unknown table %d", what);
    }
    if (dst_bytes < need)
        return set_error(BPDN_ESIZE, "destination %zu bytes < %zu needed", dst_bytes, need);
    if (!aligned(d_dst, what == 0 ? 8 : 16))
        return set_error(BPDN_EALIGN, "destination misaligned");
    return check_cuda(launch_export(*op, what, d_dst, (cudaStream_t)cuda_stream), "export");
}

size_t bpdn_solve_workspace_bytes(bpdn_op_t h, int64_t P, const bpdn_options *opt)
{
    // the least workspace, the pixel-per-thread kernel's scratch when the solve would run it,
    // then the scratch of the split refit (a smaller workspace, down to the least one, runs
    // the other iteration kernel and the fused refit)
    const OpHandle *op = reinterpret_cast<const OpHandle *>(h);
    const bool ok = op && op->magic == kOpMagic && P > 0;
    const size_t pxb = ok ? (split_grid(op, opt) ? split_scratch_for(op, P, opt) : px_scratch_for(op, P, opt)) : 0;
    return solve_min_workspace_bytes(opt) + pxb + ((opt && opt->refit) ? refit_scratch_bytes(P) : 0);
}


int bpdn_solve(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda,
               int32_t lambda_per_pixel, const bpdn_options *opt, void *d_x, int32_t *d_support,
               int32_t *d_nsupp, int32_t *d_status, int32_t *d_iters, int32_t *d_nbt,
               void *d_workspace, size_t workspace_bytes, void *cuda_stream)
{
    return bpdn::solve_impl(h, d_g, P, d_lambda, lambda_per_pixel, opt, d_x, d_support, d_nsupp, d_status,
                            d_iters, d_nbt, d_workspace, workspace_bytes, cuda_stream, true);
}

size_t bpdn_refit_workspace_bytes(bpdn_op_t h, int64_t P)
{
    (void)h;
    return refit_scratch_bytes(P);
}

int bpdn_refit(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda,
               int32_t lambda_per_pixel, const bpdn_options *opt, const void *d_x_in,
               void *d_x_out, int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
               void *d_workspace, size_t workspace_bytes, void *cuda_stream)
{
    OpHandle *op = nullptr;
    int rc = check_op(h, &op);
    if (rc)
        return rc;
    rc = check_options(opt);
    if (rc)
        return rc;
    rc = check_solve_buffers(op, d_g, P, d_lambda, d_x_out, d_status);
    if (rc)
        return rc;
    if (P == 0)
        return BPDN_OK;
    if (!d_x_in || !aligned(d_x_in, 8))
        return set_error(d_x_in ? BPDN_EALIGN : BPDN_EINVAL, "x_in must be non-NULL and 8-byte aligned");
    RefitLaunch r;
    r.g = (const float2 *)d_g;
    r.P = P;
    r.lam = d_lambda;
    r.lam_pp = lambda_per_pixel ? 1 : 0;
    r.x_in = (const float2 *)d_x_in;
    r.x_out = (float2 *)d_x_out;
    r.support = d_support;
    r.nsupp = d_nsupp;
    r.status = d_status;
    r.s_max = opt->s_max;
    r.rounds = opt->refit_rounds;
    // the split refit when the caller's workspace holds its scratch
    r.split = (d_workspace && aligned(d_workspace, 256) && workspace_bytes >= refit_scratch_bytes(P))
                  ? (unsigned char *)d_workspace
                  : nullptr;
    return check_cuda(launch_refit(*op, r, (cudaStream_t)cuda_stream), "refit kernel");
}

size_t bpdn_backward_workspace_bytes(bpdn_op_t h, int64_t P)
{
    (void)h;
    return P > 0 ? a256(sizeof(double) * (size_t)P) : 0;
}

int bpdn_backward(bpdn_op_t h, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
                  const void *d_x, const int32_t *d_support, const int32_t *d_nsupp,
                  const int32_t *d_status, int32_t s_max,
                  const void *d_dL_dx, void *d_dL_dg, float *d_dL_dlambda, void *d_workspace,
                  size_t workspace_bytes, void *cuda_stream)
{
    OpHandle *op = nullptr;
    int rc = check_op(h, &op);
    if (rc)
        return rc;
    if (P < 0)
        return set_error(BPDN_EINVAL, "P must be >= 0");
    if (s_max < 1 || s_max > BPDN_MAX_SMAX)
        return set_error(BPDN_EINVAL, "s_max must lie in 1..%d", BPDN_MAX_SMAX);
    if (!d_lambda || !d_dL_dlambda)
        return set_error(BPDN_EINVAL, "lambda and dL/dlambda must be non-NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (P == 0) {
        if (!lambda_per_pixel)
            return check_cuda(cudaMemsetAsync(d_dL_dlambda, 0, sizeof(float), s), "clear dL/dlambda");
        return BPDN_OK;
    }
    if (!d_x || !d_support || !d_nsupp || !d_dL_dx || !d_dL_dg)
        return set_error(BPDN_EINVAL, "x, support, nsupp, dL/dx and dL/dg must be non-NULL");
    if (!aligned(d_x, 8) || !aligned(d_dL_dx, 8) || !aligned(d_dL_dg, 8))
        return set_error(BPDN_EALIGN, "x, dL/dx and dL/dg must be 8-byte aligned");
    if (!aligned(d_support, 4) || !aligned(d_nsupp, 4) || !aligned(d_lambda, 4) || !aligned(d_dL_dlambda, 4) ||
        (d_status && !aligned(d_status, 4)))
        return set_error(BPDN_EALIGN, "int32 / float32 arrays must be 4-byte aligned");
    if (!lambda_per_pixel) {
        if (!d_workspace || workspace_bytes < bpdn_backward_workspace_bytes(h, P))
            return set_error(BPDN_ESIZE, "backward workspace too small");
        if (!aligned(d_workspace, 256))
            return set_error(BPDN_EALIGN, "backward workspace must be 256-byte aligned");
    }
    BackwardLaunch a;
    a.P = P;
    a.lam = d_lambda;
    a.lam_pp = lambda_per_pixel ? 1 : 0;
    a.x = (const float2 *)d_x;
    a.support = d_support;
    a.nsupp = d_nsupp;
    a.status = d_status;
    a.s_max = s_max;
    a.dLdx = (const float2 *)d_dL_dx;
    a.dLdg = (float2 *)d_dL_dg;
    a.dLdlam = d_dL_dlambda;
    a.part = (double *)d_workspace;
    return check_cuda(launch_backward(*op, a, s), "backward kernel");
}

int bpdn_select(bpdn_op_t h, const void *d_g, int64_t P, const void *d_x, const int32_t *d_support,
                const int32_t *d_nsupp, const int32_t *d_status, int32_t s_max, int32_t kmax,
                double penalty, int32_t *d_khat, double *d_s_hat, void *d_gamma_hat, void *cuda_stream)
{
    OpHandle *op = nullptr;
    int rc = check_op(h, &op);
    if (rc)
        return rc;
    if (P < 0)
        return set_error(BPDN_EINVAL, "P must be >= 0");
    if (s_max < 1 || s_max > BPDN_MAX_SMAX)
        return set_error(BPDN_EINVAL, "s_max must lie in 1..%d", BPDN_MAX_SMAX);
    if (kmax < 1 || kmax > BPDN_MAX_KSEL)
        return set_error(BPDN_EINVAL, "kmax must lie in 1..%d", BPDN_MAX_KSEL);
    if (op->md)
        return set_error(BPDN_EINVAL, "model selection reads an elevation-only grid; this operator has motion dimensions");
    if (!(penalty == penalty))
        return set_error(BPDN_EINVAL, "penalty must not be NaN");
    if (P == 0)
        return BPDN_OK;
    if (!d_g || !d_x || !d_support || !d_nsupp || !d_khat || !d_s_hat || !d_gamma_hat)
        return set_error(BPDN_EINVAL, "g, x, support, nsupp, khat, s_hat and gamma_hat must be non-NULL");
    if (!aligned(d_g, 8) || !aligned(d_x, 8) || !aligned(d_s_hat, 8) || !aligned(d_gamma_hat, 16))
        return set_error(BPDN_EALIGN, "g and x must be 8-byte aligned, s_hat 8-byte, gamma_hat 16-byte");
    if (!aligned(d_support, 4) || !aligned(d_nsupp, 4) || !aligned(d_khat, 4) || (d_status && !aligned(d_status, 4)))
        return set_error(BPDN_EALIGN, "int32 arrays must be 4-byte aligned");
    SelectLaunch a;
    a.P = P;
    a.g = (const float2 *)d_g;
    a.x = (const float2 *)d_x;
    a.support = d_support;
    a.nsupp = d_nsupp;
    a.status = d_status;
    a.s_max = s_max;
    a.kmax = kmax;
    a.penalty = penalty;
    a.khat = d_khat;
    a.s_hat = d_s_hat;
    a.gamma_hat = (double2 *)d_gamma_hat;
    return check_cuda(launch_select(*op, a, (cudaStream_t)cuda_stream), "select kernel");
}

}  // extern "C"
