// Operator set-up kernels: the steering matrix of Eq. 5, the Toeplitz generator
// of its Gram matrix, A A^H and the Lipschitz constant of the remark after Eq. 14.
#include <cuda_runtime.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

// exp(j 2 pi t) with the argument reduced to [-1/2, 1/2] in FP64 first.
__device__ __forceinline__ double2 cis2pi(double t)
{
    double f = t - rint(t);
    double sn, cs;
    sincospi(2.0 * f, &sn, &cs);
    return make_double2(cs, sn);
}

__device__ __forceinline__ double grid_point(double s_min, double s_max, int L, int l)
{
    return (L > 1) ? s_min + (double)l * (s_max - s_min) / (double)(L - 1) : s_min;
}

// xi_n = 2 b_n / (wavelength * range)   (Sec. II, after Eq. 2)
__global__ void k_xi(const double *b, int N, double wavelength, double range, double *xi)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N)
        xi[n] = 2.0 * b[n] / (wavelength * range);
}

// A_nl = exp(-j 2 pi xi_n s_l) (Eq. 5): FP64 table plus the planar FP32 tables
// (row stride lda, zero padded) the iteration kernels read.
__global__ void k_operator(const double *xi, int N, int L, int lda, double s_min, double s_max,
                           double2 *A64, float *A_re, float *A_im)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * lda)
        return;
    int n = idx / lda, l = idx % lda;
    if (l >= L) {
        A_re[idx] = 0.f;
        A_im[idx] = 0.f;
        return;
    }
    double2 a = cis2pi(-xi[n] * grid_point(s_min, s_max, L, l));
    A64[(size_t)n * L + l] = a;
    A_re[idx] = (float)a.x;
    A_im[idx] = (float)a.y;
}

// h(d) = sum_n exp(j 2 pi xi_n d ds), d = -(L-1)..L-1:  (A^H A)_{lm} = h(l - m).
__global__ void k_gram_h(const double *xi, int N, int L, double ds, double2 *h)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * L - 1)
        return;
    double d = (double)(i - (L - 1));
    double2 acc = make_double2(0.0, 0.0);
    for (int n = 0; n < N; ++n) {
        double2 e = cis2pi(xi[n] * d * ds);
        acc.x += e.x;
        acc.y += e.y;
    }
    h[i] = acc;
}

// (A A^H)_{nm} = sum_l A_nl conj(A_ml)
__global__ void k_aah(const double2 *A64, int N, int L, double2 *M)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N)
        return;
    int n = idx / N, m = idx % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < L; ++l) {
        double2 a = A64[(size_t)n * L + l], b = A64[(size_t)m * L + l];
        acc.x += a.x * b.x + a.y * b.y;
        acc.y += a.y * b.x - a.x * b.y;
    }
    M[idx] = acc;
}

// lambda_max of the Hermitian PSD matrix M (N x N) in FP64.  Repeated squaring
// with trace normalisation drives B = M^(2^k)/tr(.) to the projector on the top
// eigenspace (40 squarings separate eigenvalues down to a relative gap of ~1e-11);
// the Rayleigh quotient of M at the strongest column of B is lambda_max.
// One block; dynamic shared memory 2 N^2 double2.
__global__ void k_lambda_max(const double2 *M, int N, double *out)
{
    extern __shared__ double2 sm[];
    double2 *B = sm, *T = sm + N * N;
    __shared__ double s_tr;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < N * N; i += nt)
        B[i] = M[i];
    __syncthreads();
    for (int it = 0; it < 40; ++it) {
        for (int i = tid; i < N * N; i += nt) {
            int r = i / N, c = i % N;
            double2 acc = make_double2(0.0, 0.0);
            for (int k = 0; k < N; ++k) {
                double2 a = B[r * N + k], b = B[k * N + c];
                acc.x += a.x * b.x - a.y * b.y;
                acc.y += a.x * b.y + a.y * b.x;
            }
            T[i] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            double tr = 0.0;
            for (int k = 0; k < N; ++k)
                tr += T[k * N + k].x;
            s_tr = tr;
        }
        __syncthreads();
        double inv = (s_tr > 0.0) ? 1.0 / s_tr : 0.0;
        for (int i = tid; i < N * N; i += nt)
            B[i] = make_double2(T[i].x * inv, T[i].y * inv);
        __syncthreads();
    }
    // strongest column c of B, then lambda = c^H M c / c^H c
    if (tid == 0) {
        int best = 0;
        double bd = -1.0;
        for (int k = 0; k < N; ++k)
            if (B[k * N + k].x > bd) {
                bd = B[k * N + k].x;
                best = k;
            }
        double num = 0.0, den = 0.0;
        for (int r = 0; r < N; ++r) {
            double2 Mc = make_double2(0.0, 0.0);
            for (int k = 0; k < N; ++k) {
                double2 m = M[r * N + k], v = B[k * N + best];
                Mc.x += m.x * v.x - m.y * v.y;
                Mc.y += m.x * v.y + m.y * v.x;
            }
            double2 v = B[r * N + best];
            num += v.x * Mc.x + v.y * Mc.y;
            den += v.x * v.x + v.y * v.y;
        }
        out[0] = (den > 0.0) ? num / den : 0.0;
    }
}

// Eq. 4 on a multi-component grid (elevation fastest, then the motion coefficients):
// A_nl = exp(-j 2 pi (xi_n s + sum_m eta_{m,n} p_m)), FP64 table plus the planar FP32 tables.
__global__ void k_operator_md(const double *xi, int N, int L, int Ls, int lda, double s_min, double s_max,
                              MdGrid md, double2 *A64, float *A_re, float *A_im)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * lda)
        return;
    int n = idx / lda, l = idx % lda;
    if (l >= L) {
        A_re[idx] = 0.f;
        A_im[idx] = 0.f;
        return;
    }
    const int ls = l % Ls;
    int rest = l / Ls;
    double t = xi[n] * grid_point(s_min, s_max, Ls, ls);
    for (int m = 0; m < md.M; ++m) {
        const int lm = rest % md.Lp[m];
        rest /= md.Lp[m];
        t += md.eta[m][n] * grid_point(md.pmin[m], md.pmax[m], md.Lp[m], lm);
    }
    double2 a = cis2pi(-t);
    A64[(size_t)n * L + l] = a;
    A_re[idx] = (float)a.x;
    A_im[idx] = (float)a.y;
}

// (A_j A_j^H)_{nm} over the grid columns [lo, hi) of one block
__global__ void k_aah_cols(const double2 *A64, int N, int L, int lo, int hi, double2 *M)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N)
        return;
    int n = idx / N, m = idx % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = lo; l < hi; ++l) {
        double2 a = A64[(size_t)n * L + l], b = A64[(size_t)m * L + l];
        acc.x += a.x * b.x + a.y * b.y;
        acc.y += a.y * b.x - a.x * b.y;
    }
    M[idx] = acc;
}

// cumulative draw probabilities P_j = lmax_j / sum lmax (Eq. 14; the factor 2 of
// L_j = 2 lambda_max cancels), the last entry exactly 1
__global__ void k_block_cum(const double *lmax, int J, double *cum)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    double tot = 0.0;
    for (int j = 0; j < J; ++j)
        tot += lmax[j];
    double run = 0.0;
    for (int j = 0; j < J; ++j) {
        run += lmax[j];
        cum[j] = (tot > 0.0) ? run / tot : (double)(j + 1) / J;
    }
    cum[J - 1] = 1.0;
}

__global__ void k_export_c64(const double2 *src, size_t n, float2 *dst)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

}  // namespace

cudaError_t launch_make_operator(const OpHandle &op, const double *d_b, cudaStream_t s)
{
    const int N = op.N, L = op.L;
    k_xi<<<(N + 63) / 64, 64, 0, s>>>(d_b, N, op.wavelength, op.range, op.xi);
    int tot = N * op.lda;
    k_operator<<<(tot + 255) / 256, 256, 0, s>>>(op.xi, N, L, op.lda, op.s_min, op.s_max, op.A64,
                                                 op.A_re, op.A_im);
    k_gram_h<<<(2 * L - 1 + 127) / 128, 128, 0, s>>>(op.xi, N, L, op.ds, op.h);
    k_aah<<<(N * N + 127) / 128, 128, 0, s>>>(op.A64, N, L, op.aah);
    size_t smem = 2 * (size_t)N * N * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_lambda_max, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    k_lambda_max<<<1, 1024, smem, s>>>(op.aah, N, op.scal);
    return cudaGetLastError();
}

cudaError_t launch_make_operator_md(const OpHandle &op, const double *d_b, const MdGrid &md, cudaStream_t s)
{
    const int N = op.N, L = op.L;
    k_xi<<<(N + 63) / 64, 64, 0, s>>>(d_b, N, op.wavelength, op.range, op.xi);
    int tot = N * op.lda;
    k_operator_md<<<(tot + 255) / 256, 256, 0, s>>>(op.xi, N, L, op.Ls, op.lda, op.s_min, op.s_max, md, op.A64,
                                                    op.A_re, op.A_im);
    cudaError_t e = cudaMemsetAsync(op.h, 0, (2 * (size_t)L - 1) * sizeof(double2), s);
    if (e != cudaSuccess)
        return e;
    k_aah<<<(N * N + 127) / 128, 128, 0, s>>>(op.A64, N, L, op.aah);
    size_t smem = 2 * (size_t)N * N * sizeof(double2);
    e = cudaFuncSetAttribute(k_lambda_max, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_lambda_max<<<1, 1024, smem, s>>>(op.aah, N, op.scal);
    return cudaGetLastError();
}

size_t block_scratch_bytes(int blocks)
{
    if (blocks < 2)
        return 0;
    return (size_t)round_up(blocks * BPDN_MAX_N * BPDN_MAX_N * (int)sizeof(double2), 256);
}

cudaError_t launch_block_probs(const OpHandle &op, int J, double2 *M, double *lmax, double *cum, cudaStream_t s)
{
    const int N = op.N, L = op.L;
    size_t smem = 2 * (size_t)N * N * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_lambda_max, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    for (int j = 0; j < J; ++j) {
        const int lo = (int)(((long long)j * L) / J), hi = (int)(((long long)(j + 1) * L) / J);
        double2 *Mj = M + (size_t)j * N * N;
        k_aah_cols<<<(N * N + 127) / 128, 128, 0, s>>>(op.A64, N, L, lo, hi, Mj);
        k_lambda_max<<<1, 1024, smem, s>>>(Mj, N, lmax + j);
    }
    k_block_cum<<<1, 32, 0, s>>>(lmax, J, cum);
    return cudaGetLastError();
}

cudaError_t launch_export(const OpHandle &op, int what, void *dst, cudaStream_t s)
{
    size_t nA = (size_t)op.N * op.L;
    switch (what) {
    case 0:
        k_export_c64<<<(unsigned)((nA + 255) / 256), 256, 0, s>>>(op.A64, nA, (float2 *)dst);
        return cudaGetLastError();
    case 1:
        return cudaMemcpyAsync(dst, op.A64, nA * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    case 2:
        return cudaMemcpyAsync(dst, op.h, (2 * (size_t)op.L - 1) * sizeof(double2),
                               cudaMemcpyDeviceToDevice, s);
    case 3:
        return cudaMemcpyAsync(dst, op.aah, (size_t)op.N * op.N * sizeof(double2),
                               cudaMemcpyDeviceToDevice, s);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace bpdn
