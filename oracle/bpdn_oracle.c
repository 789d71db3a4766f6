/*
 * FP64 CPU oracle for batched complex basis pursuit denoising (BPDN).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code with the CUDA implementation.
 *
 * Problem (Eq. 1 / Eq. 6):  min_x F(x) = ||A x - g||_2^2 + lambda * sum_l |x_l|
 * with x in C^L and |.| the complex modulus (the SOCP remark of Sec. III-A makes the
 * L1 norm of a complex vector the sum of moduli).
 *
 * Operator (Eq. 5 and the definitions after Eq. 2): A_nl = exp(-j 2 pi xi_n s_l),
 * xi_n = 2 b_n / (wavelength * range), s_l uniform on [s_min, s_max] with both
 * end points included.
 *
 * Everything is plain double-precision loops in the order the definitions are
 * written; no blocking, no fusion.  Complex numbers use C99 `double complex`.
 *
 * Contents
 *   orc_grid / orc_operator / orc_gram_toeplitz / orc_aah   : the operator (Eq. 5)
 *   orc_soft                                                 : complex soft threshold (Eq. 10)
 *   orc_rbpg                                                 : Algorithm 1 (RBPG with backtracking)
 *   orc_rbpg_block                                           : Algorithm 1 with randomized blocks of
 *                                                              one pixel's grid (Eqs. 13-14), drawn
 *                                                              by SplitMix64 (orc_splitmix64)
 *   orc_cd                                                   : cyclic coordinate descent (exact minimiser)
 *   orc_newton_polish                                        : Newton on the smooth optimality
 *                                                              system restricted to a support
 *   orc_kkt                                                  : optimality certificate (Eq. 6)
 *   orc_adjoint                                              : derivatives of the minimiser in
 *                                                              (g, lambda) by implicit
 *                                                              differentiation on the support
 *   orc_*_batch                                              : OpenMP loops over pixels
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_NOT_CONVERGED 1
#define ORC_BT_LIMIT 2
#define ORC_NONFINITE 4
#define ORC_ZERO_SOLUTION 32

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------- operator */

/* s_l = s_min + l * (s_max - s_min) / (L - 1), l = 0..L-1 (Eq. 5: "uniformly sampled"). */
void orc_grid(double s_min, double s_max, int L, double *s)
{
    for (int l = 0; l < L; ++l)
        s[l] = (L > 1) ? s_min + (double)l * (s_max - s_min) / (double)(L - 1) : s_min;
}

/* xi_n = 2 b_n / (wavelength * range)   (Sec. II, after Eq. 2) */
void orc_xi(const double *b, int N, double wavelength, double range, double *xi)
{
    for (int n = 0; n < N; ++n)
        xi[n] = 2.0 * b[n] / (wavelength * range);
}

/* A (row-major N x L): A_nl = exp(-j 2 pi xi_n s_l)   (Eq. 5) */
void orc_operator(const double *b, int N, double wavelength, double range,
                  double s_min, double s_max, int L, cplx *A)
{
    double *s = (double *)malloc(sizeof(double) * (size_t)L);
    double *xi = (double *)malloc(sizeof(double) * (size_t)N);
    orc_grid(s_min, s_max, L, s);
    orc_xi(b, N, wavelength, range, xi);
    for (int n = 0; n < N; ++n)
        for (int l = 0; l < L; ++l)
            A[(size_t)n * L + l] = cexp(-2.0 * ORC_PI * I * xi[n] * s[l]);
    free(s);
    free(xi);
}

/* Toeplitz generator of the Gram matrix on a uniform grid:
 * (A^H A)_{lm} = sum_n exp(j 2 pi xi_n (s_l - s_m)) = h(l - m),
 * h(d) = sum_n exp(j 2 pi xi_n d ds), stored as h[d + L - 1], d = -(L-1)..(L-1). */
void orc_gram_toeplitz(const double *xi, int N, double ds, int L, cplx *h)
{
    for (int d = -(L - 1); d <= L - 1; ++d) {
        cplx acc = 0.0;
        for (int n = 0; n < N; ++n)
            acc += cexp(2.0 * ORC_PI * I * xi[n] * (double)d * ds);
        h[d + L - 1] = acc;
    }
}

/* A A^H (N x N), by the plain sum over the grid. */
void orc_aah(const cplx *A, int N, int L, cplx *M)
{
    for (int n = 0; n < N; ++n)
        for (int m = 0; m < N; ++m) {
            cplx acc = 0.0;
            for (int l = 0; l < L; ++l)
                acc += A[(size_t)n * L + l] * conj(A[(size_t)m * L + l]);
            M[(size_t)n * N + m] = acc;
        }
}

/* ------------------------------------------------------------- primitives */

/* Complex soft threshold, the proximal map of tau*|.| (Eq. 10 read for complex v):
 * S_tau(v) = v * max(0, 1 - tau/|v|);  |v| <= tau -> 0 (closed middle case). */
cplx orc_soft(cplx v, double tau)
{
    double a = cabs(v);
    if (!(a > tau))
        return 0.0;
    return v * (1.0 - tau / a);
}

void orc_soft_vec(const cplx *v, int n, double tau, cplx *out)
{
    for (int i = 0; i < n; ++i)
        out[i] = orc_soft(v[i], tau);
}

static void matvec(const cplx *A, int N, int L, const cplx *x, cplx *out) /* out = A x */
{
    for (int n = 0; n < N; ++n) {
        cplx acc = 0.0;
        for (int l = 0; l < L; ++l)
            acc += A[(size_t)n * L + l] * x[l];
        out[n] = acc;
    }
}

static void matvec_h(const cplx *A, int N, int L, const cplx *r, cplx *out) /* out = A^H r */
{
    for (int l = 0; l < L; ++l) {
        cplx acc = 0.0;
        for (int n = 0; n < N; ++n)
            acc += conj(A[(size_t)n * L + l]) * r[n];
        out[l] = acc;
    }
}

static double norm2sq(const cplx *v, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return s;
}

static double l1(const cplx *v, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += cabs(v[i]);
    return s;
}

/* F(x) = ||A x - g||^2 + lambda ||x||_1   (Eq. 6) */
double orc_objective(const cplx *A, int N, int L, const cplx *g, double lam, const cplx *x)
{
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    matvec(A, N, L, x, r);
    for (int n = 0; n < N; ++n)
        r[n] -= g[n];
    double F = norm2sq(r, N) + lam * l1(x, L);
    free(r);
    return F;
}

static int all_finite(const cplx *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(creal(v[i])) || !isfinite(cimag(v[i])))
            return 0;
    return 1;
}

/*
 * Round v to bfloat16 (the upper 16 bits of IEEE binary32), the operand format of the
 * tensor-core contraction: v is first rounded to binary32, then to the nearest
 * bfloat16, ties to even (add 0x7FFF plus the lowest kept bit, drop the low 16 bits).
 * *dist (may be NULL) receives the distance of the binary32 value from the nearest
 * bfloat16 rounding boundary, in units of one bfloat16 step (0: on a boundary, 0.5: on
 * a bfloat16 value).  Finite inputs only.
 */
double orc_bf16_round(double v, double *dist)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    const uint32_t rem = b & 0xFFFFu;
    if (dist)
        *dist = fabs((double)rem - 32768.0) / 65536.0;
    b += 0x7FFFu + ((b >> 16) & 1u);
    b &= 0xFFFF0000u;
    memcpy(&f, &b, sizeof f);
    return (double)f;
}

static cplx bf16_c(cplx v, double *dist)
{
    double d1, d2;
    cplx r = orc_bf16_round(creal(v), &d1) + I * orc_bf16_round(cimag(v), &d2);
    if (dist)
        *dist = fmin(d1, d2);
    return r;
}

/* --------------------------------------------------------- Algorithm 1 */

/*
 * RBPG with backtracking (Algorithm 1, Eqs. 11-15) for one pixel, FP64.
 *
 * Block = the pixel's whole x (the patch objective is separable over pixels;
 * with equal block Lipschitz constants the sampling of Eq. 14 is uniform, so
 * each pixel's iterate sequence is the one written here).
 *
 * Readings of the points the paper leaves open:
 *   - Nesterov weight theta_k = 2/(k+1) (after Eq. 12), so the extrapolation
 *     factor theta_k (1/theta_{k-1} - 1) = (k-2)/(k+1); with x^{0} = x^{-1} = 0
 *     the k = 1 term vanishes.  The counter k never resets.
 *   - f(x) = ||A x - g||^2, grad f(y) = 2 A^H (A y - g) (Wirtinger gradient).
 *   - Eq. 10 read as the complex soft threshold with tau = alpha_k * lambda.
 *   - Backtracking (Eq. 15) loops while the condition does NOT hold; for the
 *     quadratic f, Eq. 15 at base point y is ||A (x' - y)||^2 <= ||x' - y||^2 / (2 alpha).
 *     alpha starts at alpha0 and is carried from iteration to iteration
 *     (non-increasing), shrunk by C_alpha on each failure.
 *   - Monotone step: x^{k+1} = xbar if F(xbar) <= F(x^k), else x^k (ties accept).
 *   - Stop when the candidate step is small, ||xbar - x^k|| <= tol * max(||xbar||, 1e-30)
 *     (accepted or not: on acceptance this is ||x^{k+1} - x^k||; a rejected candidate
 *     that close to x^k means x^k is a fixed point up to rounding), or after
 *     max_iter iterations (status NOT_CONVERGED).  x = xbar = 0 at k = 1 stops at once.
 *
 * trace arrays (length >= max_iter, may be NULL): alpha after backtracking,
 * accept flag, number of step reductions, F(xbar), the smallest relative
 * margin of any discrete decision taken in the iteration (prox thresholds,
 * line-search test, accept test) and the relative candidate step
 * ||xbar - x^k|| / max(||xbar||, 1e-30) that the stopping test compares with tol.
 * bf16_operands != 0: the gradient's two operands, A and r = A y - g, are rounded to
 * bfloat16 (orc_bf16_round) before the products, which are summed in FP64 -- the
 * arithmetic of a BF16 tensor-core contraction up to its FP32 accumulation; the distance of
 * every rounded r_n from its rounding boundary then enters the trace's margin.
 */
int orc_rbpg(const cplx *A, int N, int L, const cplx *g, double lam, double alpha0,
             double c_alpha, double tol, int max_iter, int max_bt, int bf16_operands, cplx *x_out,
             int *iters_out, double *tr_alpha, int *tr_acc, int *tr_nbt, double *tr_F,
             double *tr_margin, double *tr_step)
{
    int status = 0;
    size_t Lz = (size_t)L, Nz = (size_t)N;
    cplx *x = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *xp = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *y = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *grad = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *v = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *xb = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *Ay = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *r = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *Axb = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *tmp = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *Ab = NULL; /* A rounded to bfloat16 (bf16_operands) */
    int k = 0;

    if (!all_finite(g, N)) {
        status = ORC_NONFINITE;
        goto done;
    }

    double alpha = alpha0;
    double Fx = norm2sq(g, N); /* F(0) */
    int stopped = 0;
    if (bf16_operands) {
        Ab = (cplx *)malloc(sizeof(cplx) * Nz * Lz);
        for (size_t i = 0; i < Nz * Lz; ++i)
            Ab[i] = bf16_c(A[i], NULL);
    }
    for (k = 1; k <= max_iter; ++k) {
        double beta = (double)(k - 2) / (double)(k + 1);
        for (int l = 0; l < L; ++l)
            y[l] = x[l] + beta * (x[l] - xp[l]);
        matvec(A, N, L, y, Ay);
        for (int n = 0; n < N; ++n)
            r[n] = Ay[n] - g[n];
        double rmargin = INFINITY;
        if (bf16_operands) {
            for (int n = 0; n < N; ++n) {
                double dn;
                r[n] = bf16_c(r[n], &dn);
                rmargin = fmin(rmargin, dn);
            }
            matvec_h(Ab, N, L, r, grad);
        } else {
            matvec_h(A, N, L, r, grad);
        }
        for (int l = 0; l < L; ++l)
            grad[l] *= 2.0;

        int nbt = 0;
        double margin = INFINITY;
        for (;;) {
            double tau = alpha * lam;
            double pm = INFINITY;
            for (int l = 0; l < L; ++l) {
                v[l] = y[l] - alpha * grad[l];
                xb[l] = orc_soft(v[l], tau);
                double mm = fabs(cabs(v[l]) - tau) / tau;
                if (mm < pm)
                    pm = mm;
            }
            matvec(A, N, L, xb, Axb);
            for (int n = 0; n < N; ++n)
                tmp[n] = Axb[n] - Ay[n];
            double lhs = norm2sq(tmp, N);
            double dd = 0.0;
            for (int l = 0; l < L; ++l) {
                cplx d = xb[l] - y[l];
                dd += creal(d) * creal(d) + cimag(d) * cimag(d);
            }
            double rhs = dd / (2.0 * alpha);
            double bm = (lhs + rhs > 0.0) ? fabs(rhs - lhs) / fmax(lhs, rhs) : INFINITY;
            margin = fmin(fmin(pm, bm), rmargin);
            if (lhs <= rhs)
                break;
            if (nbt >= max_bt) {
                status |= ORC_BT_LIMIT;
                break;
            }
            alpha *= c_alpha;
            ++nbt;
        }
        for (int n = 0; n < N; ++n)
            tmp[n] = Axb[n] - g[n];
        double Fb = norm2sq(tmp, N) + lam * l1(xb, L);
        double am = fabs(Fb - Fx) / fmax(fabs(Fx), 1e-300);
        margin = fmin(margin, am);

        int accepted = (Fb <= Fx);
        /* x^{k} becomes x_prev; x^{k+1} is xbar (accept) or x^{k} (reject).
         * The stopping test measures the candidate step ||xbar - x^k|| against ||xbar||. */
        double dnorm = 0.0, xnorm = 0.0;
        for (int l = 0; l < L; ++l) {
            cplx xk = x[l];
            cplx d = xb[l] - xk;
            dnorm += creal(d) * creal(d) + cimag(d) * cimag(d);
            xnorm += creal(xb[l]) * creal(xb[l]) + cimag(xb[l]) * cimag(xb[l]);
            xp[l] = xk;
            if (accepted)
                x[l] = xb[l];
        }
        if (accepted)
            Fx = Fb;
        if (tr_alpha)
            tr_alpha[k - 1] = alpha;
        if (tr_acc)
            tr_acc[k - 1] = accepted;
        if (tr_nbt)
            tr_nbt[k - 1] = nbt;
        if (tr_F)
            tr_F[k - 1] = Fb;
        if (tr_margin)
            tr_margin[k - 1] = margin;
        if (tr_step)
            tr_step[k - 1] = sqrt(dnorm) / fmax(sqrt(xnorm), 1e-30);
        if (sqrt(dnorm) <= tol * fmax(sqrt(xnorm), 1e-30)) {
            stopped = 1;
            break;
        }
    }
    if (!stopped) {
        status |= ORC_NOT_CONVERGED;
        k = max_iter;
    }
    {
        int nz = 0;
        for (int l = 0; l < L; ++l)
            nz |= (x[l] != 0.0);
        if (!nz)
            status |= ORC_ZERO_SOLUTION;
    }
done:
    for (int l = 0; l < L; ++l)
        x_out[l] = x[l];
    if (iters_out)
        *iters_out = k;
    free(Ab);
    free(x); free(xp); free(y); free(grad); free(v); free(xb);
    free(Ay); free(r); free(Axb); free(tmp);
    return status;
}

/* ------------------------------------------- randomized blocks (Eqs. 13-14) */

/*
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", 2014): the state advances by the golden-ratio increment and each
 * output is the state passed through the generator's mixing function.  n outputs
 * from the given state.
 */
static uint64_t orc_sm64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_splitmix64(uint64_t state, int n, uint64_t *out)
{
    for (int i = 0; i < n; ++i)
        out[i] = orc_sm64_next(&state);
}

/* Block i_k of Eq. 14 for one uniform draw: the first j with u < cum[j]. */
static int orc_draw_block(uint64_t *state, int J, const double *cum)
{
    double u = (double)(orc_sm64_next(state) >> 11) * 0x1.0p-53;
    for (int j = 0; j < J - 1; ++j)
        if (u < cum[j])
            return j;
    return J - 1;
}

/*
 * Algorithm 1 with the elevation grid of one pixel split into J contiguous blocks
 * (block j = [floor(jL/J), floor((j+1)L/J))), the reading of Eqs. 13-14 in which the
 * blocks are coordinates of one pixel.  Per iteration k:
 *   i = block drawn with P_i = L_i / sum_j L_j (cum = cumulative P, last entry 1),
 *       from SplitMix64 started at state seed + pixel * 2^40;
 *   y = x, and on block i  y_i = x_i + beta_k (x_i - x_i^{k-1}),  beta_k = (k-2)/(k+1)
 *       (x^{k-1} is the previous iterate, as Algorithm 1 writes it);
 *   xbar = y, and on block i  xbar_i = S_{alpha_i lambda}(y_i - alpha_i grad_i f(y)),
 *       grad_i f(y) = 2 A_i^H (A y - g), with Eq. 15 on block i:
 *       ||A (xbar - y)||^2 <= ||xbar - y||^2 / (2 alpha_i), else alpha_i *= c_alpha;
 *       each block carries its own alpha_i (Eq. 13's alpha_{i_k}), all starting at alpha0;
 *   accept xbar when F(xbar) <= F(x^k) (x^{k+1} = xbar), else x^{k+1} = x^k;
 *   a step is small when ||xbar - x^k|| <= tol ||xbar||; stop once every block has taken a
 *       small step since the last step that was not small (each block's proximal-gradient
 *       step is then small: a block that stays zero takes a zero step, so counting small
 *       steps without regard to the block would stop on the empty blocks of a sparse
 *       iterate), or after max_iter * J iterations (NOT_CONVERGED).
 * trace (may be NULL, max_iter*J entries) receives the drawn blocks.
 */
int orc_rbpg_block(const cplx *A, int N, int L, const cplx *g, double lam, double alpha0,
                   double c_alpha, double tol, int max_iter, int max_bt, int J, const double *cum,
                   uint64_t seed, int64_t pixel, cplx *x_out, int *iters_out, int *trace)
{
    int status = 0;
    size_t Lz = (size_t)L, Nz = (size_t)N;
    cplx *x = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *xp = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *y = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *grad = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *xb = (cplx *)calloc(Lz, sizeof(cplx));
    cplx *Ay = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *r = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *Axb = (cplx *)calloc(Nz, sizeof(cplx));
    cplx *tmp = (cplx *)calloc(Nz, sizeof(cplx));
    double *alpha = (double *)malloc(sizeof(double) * (size_t)J);
    uint64_t state = seed + ((uint64_t)pixel << 40);
    int kmax = max_iter * J, k = 0, stopped = 0;
    unsigned done_mask = 0, all_mask = (J >= 32) ? 0xFFFFFFFFu : ((1u << J) - 1u);

    if (!all_finite(g, N)) {
        status = ORC_NONFINITE;
        goto done;
    }
    for (int j = 0; j < J; ++j)
        alpha[j] = alpha0;
    double Fx = norm2sq(g, N); /* F(0) */
    for (k = 1; k <= kmax; ++k) {
        const int i = orc_draw_block(&state, J, cum);
        const int lo = (int)(((int64_t)i * L) / J), hi = (int)(((int64_t)(i + 1) * L) / J);
        if (trace)
            trace[k - 1] = i;
        double beta = (double)(k - 2) / (double)(k + 1);
        for (int l = 0; l < L; ++l)
            y[l] = (l >= lo && l < hi) ? x[l] + beta * (x[l] - xp[l]) : x[l];
        matvec(A, N, L, y, Ay);
        for (int n = 0; n < N; ++n)
            r[n] = Ay[n] - g[n];
        matvec_h(A, N, L, r, grad);
        int nbt = 0;
        for (;;) {
            double tau = alpha[i] * lam;
            for (int l = 0; l < L; ++l)
                xb[l] = (l >= lo && l < hi) ? orc_soft(y[l] - alpha[i] * 2.0 * grad[l], tau) : y[l];
            matvec(A, N, L, xb, Axb);
            for (int n = 0; n < N; ++n)
                tmp[n] = Axb[n] - Ay[n];
            double lhs = norm2sq(tmp, N), dd = 0.0;
            for (int l = 0; l < L; ++l) {
                cplx d = xb[l] - y[l];
                dd += creal(d) * creal(d) + cimag(d) * cimag(d);
            }
            if (lhs <= dd / (2.0 * alpha[i]))
                break;
            if (nbt >= max_bt) {
                status |= ORC_BT_LIMIT;
                break;
            }
            alpha[i] *= c_alpha;
            ++nbt;
        }
        for (int n = 0; n < N; ++n)
            tmp[n] = Axb[n] - g[n];
        double Fb = norm2sq(tmp, N) + lam * l1(xb, L);
        int accepted = (Fb <= Fx);
        double dnorm = 0.0, xnorm = 0.0;
        for (int l = 0; l < L; ++l) {
            cplx xk = x[l];
            cplx d = xb[l] - xk;
            dnorm += creal(d) * creal(d) + cimag(d) * cimag(d);
            xnorm += creal(xb[l]) * creal(xb[l]) + cimag(xb[l]) * cimag(xb[l]);
            xp[l] = xk;
            if (accepted)
                x[l] = xb[l];
        }
        if (accepted)
            Fx = Fb;
        done_mask = (sqrt(dnorm) <= tol * fmax(sqrt(xnorm), 1e-30)) ? (done_mask | (1u << i)) : 0u;
        if (done_mask == all_mask) {
            stopped = 1;
            break;
        }
    }
    if (!stopped) {
        status |= ORC_NOT_CONVERGED;
        k = kmax;
    }
    {
        int nz = 0;
        for (int l = 0; l < L; ++l)
            nz |= (x[l] != 0.0);
        if (!nz)
            status |= ORC_ZERO_SOLUTION;
    }
done:
    for (int l = 0; l < L; ++l)
        x_out[l] = x[l];
    if (iters_out)
        *iters_out = k;
    free(x); free(xp); free(y); free(grad); free(xb);
    free(Ay); free(r); free(Axb); free(tmp); free(alpha);
    return status;
}

/* ------------------------------------------------------ exact minimiser */

/*
 * Cyclic coordinate descent for Eq. 6 (an algorithm unrelated to RBPG; used
 * only to find the minimiser).  Minimising F over x_l alone with the others
 * fixed gives x_l = S_{lambda/2}(a_l^H (g - A x + a_l x_l)) / ||a_l||^2.
 * q = A^H (g - A x) is kept up to date and recomputed from scratch every 64
 * sweeps.  Stops when max_l |dx_l| <= tol * max(1, max_l |x_l|).
 * Returns 0 on convergence, 1 if max_sweeps was reached.
 */
int orc_cd(const cplx *A, int N, int L, const cplx *g, double lam, double tol,
           long max_sweeps, cplx *x, long *sweeps_out)
{
    size_t Lz = (size_t)L;
    cplx *G = (cplx *)malloc(sizeof(cplx) * Lz * Lz);
    cplx *c = (cplx *)malloc(sizeof(cplx) * Lz);
    cplx *q = (cplx *)malloc(sizeof(cplx) * Lz);
    /* G = A^H A, c = A^H g */
    for (int l = 0; l < L; ++l)
        for (int m = 0; m < L; ++m) {
            cplx acc = 0.0;
            for (int n = 0; n < N; ++n)
                acc += conj(A[(size_t)n * L + l]) * A[(size_t)n * L + m];
            G[(size_t)l * L + m] = acc;
        }
    matvec_h(A, N, L, g, c);
    for (int l = 0; l < L; ++l)
        x[l] = 0.0;
    long sw;
    int rc = 1;
    for (sw = 0; sw < max_sweeps; ++sw) {
        if (sw % 64 == 0) {
            for (int l = 0; l < L; ++l) {
                cplx acc = c[l];
                for (int m = 0; m < L; ++m)
                    acc -= G[(size_t)l * L + m] * x[m];
                q[l] = acc;
            }
        }
        double maxd = 0.0, maxx = 0.0;
        for (int l = 0; l < L; ++l) {
            double Gll = creal(G[(size_t)l * L + l]);
            cplx old = x[l];
            cplx vv = q[l] + Gll * old;
            cplx nw = orc_soft(vv, 0.5 * lam) / Gll;
            cplx dlt = nw - old;
            if (dlt != 0.0) {
                for (int m = 0; m < L; ++m)
                    q[m] -= G[(size_t)m * L + l] * dlt;
                x[l] = nw;
                double ad = cabs(dlt);
                if (ad > maxd)
                    maxd = ad;
            }
            double ax = cabs(x[l]);
            if (ax > maxx)
                maxx = ax;
        }
        if (maxd <= tol * fmax(1.0, maxx)) {
            rc = 0;
            ++sw;
            break;
        }
    }
    if (sweeps_out)
        *sweeps_out = sw;
    free(G); free(c); free(q);
    return rc;
}

/* Solve the real n x n system M z = rhs by Gaussian elimination with partial
 * pivoting (M and rhs are overwritten).  Returns 0 on success. */
static int solve_real(double *M, double *rhs, int n)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(M[(size_t)i * n + k]) > best) {
                best = fabs(M[(size_t)i * n + k]);
                p = i;
            }
        if (!(best > 0.0))
            return 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = M[(size_t)k * n + j];
                M[(size_t)k * n + j] = M[(size_t)p * n + j];
                M[(size_t)p * n + j] = t;
            }
            double t = rhs[k];
            rhs[k] = rhs[p];
            rhs[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
            for (int j = k; j < n; ++j)
                M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
            rhs[i] -= f * rhs[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = rhs[k];
        for (int j = k + 1; j < n; ++j)
            s -= M[(size_t)k * n + j] * rhs[j];
        rhs[k] = s / M[(size_t)k * n + k];
    }
    return 0;
}

/* restricted objective F_S(z) = ||A_S z - g||^2 + lambda sum |z_i| */
static double restricted_F(const cplx *AS, int N, int m, const cplx *g, double lam, const cplx *z)
{
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
        cplx acc = -g[n];
        for (int i = 0; i < m; ++i)
            acc += AS[(size_t)n * m + i] * z[i];
        s += creal(acc) * creal(acc) + cimag(acc) * cimag(acc);
    }
    for (int i = 0; i < m; ++i)
        s += lam * cabs(z[i]);
    return s;
}

/* Phi(z) = 2 (G z - c) + lambda z/|z|: the gradient of F_S where no z_i is 0. */
static void restricted_phi(const cplx *G, const cplx *c, int m, double lam, const cplx *z, cplx *phi)
{
    for (int i = 0; i < m; ++i) {
        cplx acc = -c[i];
        for (int j = 0; j < m; ++j)
            acc += G[(size_t)i * m + j] * z[j];
        phi[i] = 2.0 * acc + lam * z[i] / cabs(z[i]);
    }
}

/*
 * Newton's method for the optimality system of Eq. 6 restricted to the index
 * set S (all |z_i| > 0):  Phi(z) = 2 A_S^H (A_S z - g) + lambda z/|z| = 0.
 * In real coordinates (Re z_i, Im z_i) the Jacobian is
 *     J = 2 [[Re G, -Im G], [Im G, Re G]] (per 2x2 block) + lambda/|z_i| (I - u u^T),
 * u = (Re z_i, Im z_i)/|z_i|, G = A_S^H A_S; it is the Hessian of F_S.  Steps are
 * halved until F_S or ||Phi|| decreases and no component reaches zero.
 * z: in = starting point (all nonzero), out = solution.  Returns 0 when
 * max_i |Phi_i| <= ftol * lambda, 1 otherwise.  *res_out = final max |Phi_i| / lambda.
 */
int orc_newton_polish(const cplx *A, int N, int L, const cplx *g, double lam, int m,
                      const int *S, cplx *z, int max_it, double ftol, double *res_out)
{
    (void)L;
    int rc = 1;
    size_t mz = (size_t)m;
    cplx *AS = (cplx *)malloc(sizeof(cplx) * (size_t)N * mz);
    cplx *G = (cplx *)malloc(sizeof(cplx) * mz * mz);
    cplx *c = (cplx *)malloc(sizeof(cplx) * mz);
    cplx *phi = (cplx *)malloc(sizeof(cplx) * mz);
    cplx *zt = (cplx *)malloc(sizeof(cplx) * mz);
    cplx *pt = (cplx *)malloc(sizeof(cplx) * mz);
    double *J = (double *)malloc(sizeof(double) * 4 * mz * mz);
    double *rhs = (double *)malloc(sizeof(double) * 2 * mz);
    double res = INFINITY;
    for (int n = 0; n < N; ++n)
        for (int i = 0; i < m; ++i)
            AS[(size_t)n * m + i] = A[(size_t)n * L + S[i]];
    for (int i = 0; i < m; ++i) {
        cplx acc = 0.0;
        for (int n = 0; n < N; ++n)
            acc += conj(AS[(size_t)n * m + i]) * g[n];
        c[i] = acc;
        for (int j = 0; j < m; ++j) {
            cplx a2 = 0.0;
            for (int n = 0; n < N; ++n)
                a2 += conj(AS[(size_t)n * m + i]) * AS[(size_t)n * m + j];
            G[(size_t)i * m + j] = a2;
        }
    }
    for (int i = 0; i < m; ++i)
        if (z[i] == 0.0)
            goto out;
    for (int it = 0; it <= max_it; ++it) {
        restricted_phi(G, c, m, lam, z, phi);
        res = 0.0;
        double nphi = 0.0;
        for (int i = 0; i < m; ++i) {
            double a = cabs(phi[i]);
            res = fmax(res, a);
            nphi += a * a;
        }
        if (res <= ftol * lam) {
            rc = 0;
            break;
        }
        if (it == max_it)
            break;
        int n2 = 2 * m;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double gr = creal(G[(size_t)i * m + j]), gi = cimag(G[(size_t)i * m + j]);
                J[(size_t)(2 * i) * n2 + 2 * j] = 2.0 * gr;
                J[(size_t)(2 * i) * n2 + 2 * j + 1] = -2.0 * gi;
                J[(size_t)(2 * i + 1) * n2 + 2 * j] = 2.0 * gi;
                J[(size_t)(2 * i + 1) * n2 + 2 * j + 1] = 2.0 * gr;
            }
        for (int i = 0; i < m; ++i) {
            double a = cabs(z[i]);
            double ur = creal(z[i]) / a, ui = cimag(z[i]) / a;
            double w = lam / a;
            J[(size_t)(2 * i) * n2 + 2 * i] += w * (1.0 - ur * ur);
            J[(size_t)(2 * i) * n2 + 2 * i + 1] += w * (-ur * ui);
            J[(size_t)(2 * i + 1) * n2 + 2 * i] += w * (-ui * ur);
            J[(size_t)(2 * i + 1) * n2 + 2 * i + 1] += w * (1.0 - ui * ui);
            rhs[2 * i] = -creal(phi[i]);
            rhs[2 * i + 1] = -cimag(phi[i]);
        }
        if (solve_real(J, rhs, n2))
            break;
        double F0 = restricted_F(AS, N, m, g, lam, z);
        double t = 1.0;
        int ok = 0;
        for (int h = 0; h < 60; ++h, t *= 0.5) {
            int zero = 0;
            for (int i = 0; i < m; ++i) {
                zt[i] = z[i] + t * (rhs[2 * i] + I * rhs[2 * i + 1]);
                if (zt[i] == 0.0)
                    zero = 1;
            }
            if (zero)
                continue;
            double F1 = restricted_F(AS, N, m, g, lam, zt);
            restricted_phi(G, c, m, lam, zt, pt);
            double np = 0.0;
            for (int i = 0; i < m; ++i)
                np += creal(pt[i]) * creal(pt[i]) + cimag(pt[i]) * cimag(pt[i]);
            if (F1 < F0 || np < nphi) {
                ok = 1;
                break;
            }
        }
        if (!ok)
            break;
        for (int i = 0; i < m; ++i)
            z[i] = zt[i];
    }
out:
    if (res_out)
        *res_out = res / lam;
    free(AS); free(G); free(c); free(phi); free(zt); free(pt); free(J); free(rhs);
    return rc;
}

/*
 * Optimality certificate for Eq. 6.  With r = A x - g and z_l = 2 a_l^H r:
 *   on S = supp(x):   z_l = -lambda x_l/|x_l|       -> on_res = max_S |z_l + lambda x_l/|x_l|| / lambda
 *   off S:            |z_l| <= lambda               -> off_max = max_{l not in S} |z_l| / lambda
 * (off_max = 0 when S is everything; on_res = 0 when S is empty.)
 */
void orc_kkt(const cplx *A, int N, int L, const cplx *g, double lam, const cplx *x,
             double *on_res, double *off_max, double *min_abs_on, int *nS)
{
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *z = (cplx *)malloc(sizeof(cplx) * (size_t)L);
    matvec(A, N, L, x, r);
    for (int n = 0; n < N; ++n)
        r[n] -= g[n];
    matvec_h(A, N, L, r, z);
    double on = 0.0, off = 0.0, mn = INFINITY;
    int cnt = 0;
    for (int l = 0; l < L; ++l) {
        cplx zl = 2.0 * z[l];
        if (x[l] != 0.0) {
            double a = cabs(x[l]);
            on = fmax(on, cabs(zl + lam * x[l] / a) / lam);
            mn = fmin(mn, a);
            ++cnt;
        } else {
            off = fmax(off, cabs(zl) / lam);
        }
    }
    *on_res = on;
    *off_max = off;
    *min_abs_on = cnt ? mn : 0.0;
    *nS = cnt;
    free(r);
    free(z);
}

/*
 * Coordinate descent on Eq. 6 restricted to the index set S (x_l = 0 for l not in S):
 * the same one-coordinate minimisations as orc_cd, over the m columns of A_S only,
 * starting from z.  Stops when max |dz_i| <= tol * max(1, max |z_i|).  Returns 0 on
 * convergence, 1 if max_sweeps was reached.
 */
static int cd_restricted(const cplx *A, int N, int L, const cplx *g, double lam, int m, const int *S,
                         cplx *z, double tol, long max_sweeps)
{
    size_t mz = (size_t)m;
    cplx *G = (cplx *)malloc(sizeof(cplx) * mz * mz);
    cplx *q = (cplx *)malloc(sizeof(cplx) * mz);
    for (int i = 0; i < m; ++i) {
        cplx c = 0.0;
        for (int n = 0; n < N; ++n)
            c += conj(A[(size_t)n * L + S[i]]) * g[n];
        q[i] = c;
        for (int j = 0; j < m; ++j) {
            cplx acc = 0.0;
            for (int n = 0; n < N; ++n)
                acc += conj(A[(size_t)n * L + S[i]]) * A[(size_t)n * L + S[j]];
            G[(size_t)i * m + j] = acc;
        }
    }
    /* q = c - G z */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            q[i] -= G[(size_t)i * m + j] * z[j];
    int rc = 1;
    for (long sw = 0; sw < max_sweeps; ++sw) {
        double maxd = 0.0, maxz = 0.0;
        for (int i = 0; i < m; ++i) {
            double Gii = creal(G[(size_t)i * m + i]);
            cplx old = z[i];
            cplx nw = orc_soft(q[i] + Gii * old, 0.5 * lam) / Gii;
            cplx dlt = nw - old;
            if (dlt != 0.0) {
                for (int j = 0; j < m; ++j)
                    q[j] -= G[(size_t)j * m + i] * dlt;
                z[i] = nw;
                if (cabs(dlt) > maxd)
                    maxd = cabs(dlt);
            }
            if (cabs(z[i]) > maxz)
                maxz = cabs(z[i]);
        }
        if (maxd <= tol * fmax(1.0, maxz)) {
            rc = 0;
            break;
        }
    }
    free(G);
    free(q);
    return rc;
}

/*
 * Working-set repair of a minimiser whose certificate failed: S = supp(x) plus the
 * grid points whose dual constraint |2 a_l^H (A x - g)| <= lambda is violated (the
 * eight largest violations per round); the restricted problem on S is solved by
 * coordinate descent and polished by Newton on its nonzeros; repeated until the
 * certificate holds or the rounds run out.  x is replaced by the last restricted
 * solution.  Returns 0 when the certificate holds.
 */
static int repair_working_set(const cplx *A, int N, int L, const cplx *g, double lam, cplx *x, int rounds)
{
    int *S = (int *)malloc(sizeof(int) * (size_t)L);
    int *inS = (int *)malloc(sizeof(int) * (size_t)L);
    cplx *z = (cplx *)malloc(sizeof(cplx) * (size_t)L);
    cplx *r = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *u = (cplx *)malloc(sizeof(cplx) * (size_t)L);
    int ok = 1;
    for (int round = 0; round < rounds; ++round) {
        double on, off, mn;
        int nS;
        orc_kkt(A, N, L, g, lam, x, &on, &off, &mn, &nS);
        if (on <= 1e-9 && off <= 1.0 + 1e-9) {
            ok = 0;
            break;
        }
        /* S = supp(x) and the largest violators off it */
        int m = 0;
        for (int l = 0; l < L; ++l) {
            inS[l] = (x[l] != 0.0);
            if (inS[l])
                S[m++] = l;
        }
        matvec(A, N, L, x, r);
        for (int n = 0; n < N; ++n)
            r[n] -= g[n];
        matvec_h(A, N, L, r, u);
        for (int add = 0; add < 8; ++add) {
            int best = -1;
            double bv = lam * (1.0 + 1e-12);
            for (int l = 0; l < L; ++l)
                if (!inS[l] && 2.0 * cabs(u[l]) > bv) {
                    bv = 2.0 * cabs(u[l]);
                    best = l;
                }
            if (best < 0)
                break;
            inS[best] = 1;
            S[m++] = best;
        }
        /* ascending order of S */
        for (int i = 1; i < m; ++i) {
            int v = S[i], j = i - 1;
            while (j >= 0 && S[j] > v) {
                S[j + 1] = S[j];
                --j;
            }
            S[j + 1] = v;
        }
        for (int i = 0; i < m; ++i)
            z[i] = x[S[i]];
        cd_restricted(A, N, L, g, lam, m, S, z, 1e-13, 200000);
        /* Newton on the nonzero coordinates of the restricted solution */
        int k = 0;
        for (int i = 0; i < m; ++i)
            if (z[i] != 0.0) {
                S[k] = S[i];
                z[k] = z[i];
                ++k;
            }
        double res;
        if (k > 0)
            orc_newton_polish(A, N, L, g, lam, k, S, z, 50, 1e-13, &res);
        for (int l = 0; l < L; ++l)
            x[l] = 0.0;
        for (int i = 0; i < k; ++i)
            x[S[i]] = z[i];
    }
    if (ok) {
        double on, off, mn;
        int nS;
        orc_kkt(A, N, L, g, lam, x, &on, &off, &mn, &nS);
        ok = !(on <= 1e-9 && off <= 1.0 + 1e-9);
    }
    free(S); free(inS); free(z); free(r); free(u);
    return ok;
}

/*
 * Exact minimiser of Eq. 6 from x = 0 by the working-set loop above alone (restricted
 * coordinate descent on the support and the largest dual violators, Newton on the
 * nonzeros, until the certificate holds): for grids whose full L x L Gram matrix, which
 * coordinate descent over the whole grid keeps, is too large.  Flags as orc_min (bit2 when
 * the certificate fails, bit3 for non-finite input).
 */
int orc_min_ws(const cplx *A, int N, int L, const cplx *g, double lam, cplx *x, double *on_res,
               double *off_max, double *min_abs_on, int *nS)
{
    for (int l = 0; l < L; ++l)
        x[l] = 0.0;
    if (!all_finite(g, N)) {
        *on_res = *off_max = *min_abs_on = 0.0;
        *nS = 0;
        return 8;
    }
    const int rc = repair_working_set(A, N, L, g, lam, x, 400);
    orc_kkt(A, N, L, g, lam, x, on_res, off_max, min_abs_on, nS);
    return rc ? 4 : 0;
}

/* grids beyond this many points skip the full-grid coordinate descent of orc_min */
#define ORC_CD_MAX_L 4096

/*
 * Exact minimiser of Eq. 6 for one pixel: coordinate descent, then Newton on
 * the support CD found (when CD stops, its support is the minimiser's unless
 * a component sits at a tie), then the certificate.  When the certificate fails
 * (CD stopped early at a wrong support), the working-set repair above continues
 * from that point.
 * flags (0 whenever the final certificate holds): bit0 CD hit max_sweeps, bit1 Newton
 * did not converge (CD result kept), bit2 certificate failed (on_res > 1e-9 or
 * off_max > 1 + 1e-9) even after the repair, bit3 non-finite input.
 */
int orc_min(const cplx *A, int N, int L, const cplx *g, double lam, double cd_tol,
            long max_sweeps, cplx *x, double *on_res, double *off_max, double *min_abs_on,
            int *nS, long *sweeps)
{
    int flags = 0;
    if (!all_finite(g, N)) {
        for (int l = 0; l < L; ++l)
            x[l] = 0.0;
        *on_res = *off_max = *min_abs_on = 0.0;
        *nS = 0;
        if (sweeps)
            *sweeps = 0;
        return 8;
    }
    if (L > ORC_CD_MAX_L) {
        if (sweeps)
            *sweeps = 0;
        return orc_min_ws(A, N, L, g, lam, x, on_res, off_max, min_abs_on, nS);
    }
    if (orc_cd(A, N, L, g, lam, cd_tol, max_sweeps, x, sweeps))
        flags |= 1;
    int m = 0;
    int *S = (int *)malloc(sizeof(int) * (size_t)L);
    for (int l = 0; l < L; ++l)
        if (x[l] != 0.0)
            S[m++] = l;
    if (m > 0) {
        cplx *z = (cplx *)malloc(sizeof(cplx) * (size_t)m);
        for (int i = 0; i < m; ++i)
            z[i] = x[S[i]];
        double res;
        if (orc_newton_polish(A, N, L, g, lam, m, S, z, 50, 1e-13, &res) == 0) {
            for (int i = 0; i < m; ++i)
                x[S[i]] = z[i];
        } else {
            flags |= 2;
        }
        free(z);
    }
    free(S);
    orc_kkt(A, N, L, g, lam, x, on_res, off_max, min_abs_on, nS);
    if (*on_res > 1e-9 || *off_max > 1.0 + 1e-9) {
        if (repair_working_set(A, N, L, g, lam, x, 50) == 0) {
            orc_kkt(A, N, L, g, lam, x, on_res, off_max, min_abs_on, nS);
            return 0;
        }
        orc_kkt(A, N, L, g, lam, x, on_res, off_max, min_abs_on, nS);
        flags |= 4;
    } else if (flags) {
        flags = 0;  /* certified: how CD and Newton got there does not matter */
    }
    return flags;
}

/* ----------------------------------------------------------------- adjoint */

/*
 * Derivatives of the minimiser x of Eq. 6 with respect to g and lambda, for a loss
 * L(x) whose gradient dL/dx is given as dL/dRe x + j dL/dIm x.
 *
 * On the support S = {l : x_l != 0} the optimality condition of Eq. 6 is the smooth
 * system  Phi(x_S, g, lambda) = 2 A_S^H (A_S x_S - g) + lambda x_S / |x_S| = 0
 * (componentwise modulus).  With each complex unknown written as (Re, Im), the
 * Jacobian of Phi in x_S is the real symmetric matrix
 *     J = 2 realify(A_S^H A_S) + lambda * blockdiag((I - u_l u_l^T) / |x_l|),
 * u_l = (Re x_l, Im x_l) / |x_l|, realify(M) = [[Re M, -Im M], [Im M, Re M]] per entry.
 * The support of a strict minimiser does not move under small changes of (g, lambda),
 * so implicit differentiation gives
 *     dx_S = J^{-1} (realify(2 A_S^H) dg - u dlambda),   dx = 0 off S,
 * and with v = J^{-1} c, c = dL/dx on S (J is symmetric):
 *     dL/dg = 2 A_S v  (v read as a complex vector),   dL/dlambda = -sum_l u_l . v_l.
 * Returns 1 when J could not be solved, 0 otherwise (x = 0 gives zero derivatives).
 */
int orc_adjoint(const cplx *A, int N, int L, double lam, const cplx *x, const cplx *dLdx,
                cplx *dLdg, double *dLdlam)
{
    int m = 0;
    for (int l = 0; l < L; ++l)
        if (x[l] != 0.0)
            ++m;
    for (int n = 0; n < N; ++n)
        dLdg[n] = 0.0;
    *dLdlam = 0.0;
    if (m == 0)
        return 0;
    int *S = (int *)malloc(sizeof(int) * (size_t)m);
    double *Jm = (double *)malloc(sizeof(double) * 4 * (size_t)m * (size_t)m);
    double *v = (double *)malloc(sizeof(double) * 2 * (size_t)m);
    int k = 0;
    for (int l = 0; l < L; ++l)
        if (x[l] != 0.0)
            S[k++] = l;
    const int n2 = 2 * m;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            cplx Gij = 0.0;  /* (A_S^H A_S)_ij */
            for (int n = 0; n < N; ++n)
                Gij += conj(A[(size_t)n * L + S[i]]) * A[(size_t)n * L + S[j]];
            Jm[(size_t)(2 * i) * n2 + 2 * j] = 2.0 * creal(Gij);
            Jm[(size_t)(2 * i) * n2 + 2 * j + 1] = -2.0 * cimag(Gij);
            Jm[(size_t)(2 * i + 1) * n2 + 2 * j] = 2.0 * cimag(Gij);
            Jm[(size_t)(2 * i + 1) * n2 + 2 * j + 1] = 2.0 * creal(Gij);
        }
    for (int i = 0; i < m; ++i) {
        const double mod = cabs(x[S[i]]);
        const double u0 = creal(x[S[i]]) / mod, u1 = cimag(x[S[i]]) / mod;
        const double curv = lam / mod;  /* curvature of lambda |x_l| across the phase */
        Jm[(size_t)(2 * i) * n2 + 2 * i] += curv * (1.0 - u0 * u0);
        Jm[(size_t)(2 * i) * n2 + 2 * i + 1] -= curv * u0 * u1;
        Jm[(size_t)(2 * i + 1) * n2 + 2 * i] -= curv * u1 * u0;
        Jm[(size_t)(2 * i + 1) * n2 + 2 * i + 1] += curv * (1.0 - u1 * u1);
        v[2 * i] = creal(dLdx[S[i]]);
        v[2 * i + 1] = cimag(dLdx[S[i]]);
    }
    int rc = solve_real(Jm, v, n2);
    if (rc == 0) {
        for (int n = 0; n < N; ++n) {
            cplx acc = 0.0;
            for (int i = 0; i < m; ++i)
                acc += A[(size_t)n * L + S[i]] * (v[2 * i] + I * v[2 * i + 1]);
            dLdg[n] = 2.0 * acc;
        }
        double dl = 0.0;
        for (int i = 0; i < m; ++i) {
            const double mod = cabs(x[S[i]]);
            dl += (creal(x[S[i]]) * v[2 * i] + cimag(x[S[i]]) * v[2 * i + 1]) / mod;
        }
        *dLdlam = -dl;
    }
    free(S);
    free(Jm);
    free(v);
    return rc;
}

/* ------------------------------------------------------------- batches */

void orc_rbpg_batch(const cplx *A, int N, int L, const cplx *g, int64_t P, const double *lam,
                    double alpha0, double c_alpha, double tol, int max_iter, int max_bt,
                    cplx *x, int *iters, int *status)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p)
        status[p] = orc_rbpg(A, N, L, g + (size_t)p * N, lam[p], alpha0, c_alpha, tol, max_iter,
                             max_bt, 0, x + (size_t)p * L, iters + p, NULL, NULL, NULL, NULL, NULL, NULL);
}

void orc_rbpg_block_batch(const cplx *A, int N, int L, const cplx *g, int64_t P, const double *lam,
                          double alpha0, double c_alpha, double tol, int max_iter, int max_bt, int J,
                          const double *cum, uint64_t seed, cplx *x, int *iters, int *status)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p)
        status[p] = orc_rbpg_block(A, N, L, g + (size_t)p * N, lam[p], alpha0, c_alpha, tol, max_iter,
                                   max_bt, J, cum, seed, p, x + (size_t)p * L, iters + p, NULL);
}

void orc_min_batch(const cplx *A, int N, int L, const cplx *g, int64_t P, const double *lam,
                   double cd_tol, long max_sweeps, cplx *x, double *on_res, double *off_max,
                   double *min_abs_on, int *nS, long *sweeps, int *flags)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < P; ++p)
        flags[p] = orc_min(A, N, L, g + (size_t)p * N, lam[p], cd_tol, max_sweeps,
                           x + (size_t)p * L, on_res + p, off_max + p, min_abs_on + p, nS + p,
                           sweeps + p);
}

int orc_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}

void orc_adjoint_batch(const cplx *A, int N, int L, const double *lam, int64_t P, const cplx *x,
                       const cplx *dLdx, cplx *dLdg, double *dLdlam, int *flags)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p)
        flags[p] = orc_adjoint(A, N, L, lam[p], x + (size_t)p * L, dLdx + (size_t)p * L,
                               dLdg + (size_t)p * N, dLdlam + p);
}
