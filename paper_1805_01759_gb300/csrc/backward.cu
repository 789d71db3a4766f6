// Adjoint of the BPDN minimiser (Eq. 6) with respect to the data g and the
// regularisation weight lambda, for a loss whose gradient dL/dx is given.
//
// On the support S the optimality condition of Eq. 6 is the smooth system
//     Phi(x_S, g, lambda) = 2 A_S^H (A_S x_S - g) + lambda x_S / |x_S| = 0,
// whose Jacobian in x_S (each complex unknown as (Re, Im)) is the real symmetric
//     J = 2 realify(G_S) + lambda blockdiag((I - u_l u_l^T) / |x_l|),
// G_S = A_S^H A_S (from the Toeplitz generator h of the uniform grid, Eq. 5),
// u_l = (Re x_l, Im x_l) / |x_l|.  The support of a strict minimiser is locally
// constant, so implicit differentiation gives, with v = J^{-1} (dL/dx)_S,
//     dL/dg = 2 A_S v,     dL/dlambda = -sum_l u_l . v_l,     (dx = 0 off S).
// Pixels the solve did not certify get zero derivatives.  One warp per pixel in
// FP64: lanes over the columns of J for the elimination (two per lane for the few
// supports of 17 to 32 entries, in a second launch), lanes over the rows of A for dL/dg.  With one lambda for all pixels the per-pixel terms are summed by a
// second kernel in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kWarps = 4;        // pixels per block of the fast kernel
constexpr int kSF = 16;          // fast kernel: support <= 16 (2|S| <= 32, one unknown per lane)
constexpr int kSW = kRefitMax;   // wide kernel: support <= 32 (two unknowns per lane)
constexpr int kSumThreads = 1024;

template <int KS>
struct BwdSmem {
    double J[2 * KS][2 * KS + 1];  // the system, right-hand side in column n2
    double inv[2 * KS];            // reciprocal pivots
    double2 xs[KS];                // x on the support (FP64)
    int W[KS];                     // support indices
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Solve J[0..n2) v = J[.][n2] (symmetric positive definite) by elimination without
// pivoting, lanes over columns; lane i returns v_i.  ok = false on a non-positive pivot.
__device__ double spd_solve(BwdSmem<kSF> &S, int n2, int lane, bool &ok)
{
    // lanes k+1..n2-1 own the columns still being eliminated; the right-hand side
    // (column n2) belongs to lane n2, or to lane 0 (never a column owner) when n2 = 32
    const int rc = (n2 < 32) ? n2 : 0;
    ok = true;
    for (int k = 0; k < n2; ++k) {
        __syncwarp();
        const double piv = S.J[k][k];
        if (!(piv > 0.0)) {
            ok = false;
            return 0.0;
        }
        const double ip = 1.0 / piv;
        const double pk = (lane > k && lane < n2) ? S.J[k][lane] : 0.0;
        const double pr = (lane == rc) ? S.J[k][n2] : 0.0;
        __syncwarp();
        if (lane == 0)
            S.inv[k] = ip;
        for (int i = k + 1; i < n2; ++i) {
            const double f = S.J[i][k] * ip;
            if (lane > k && lane < n2)
                S.J[i][lane] -= f * pk;
            if (lane == rc)
                S.J[i][n2] -= f * pr;
        }
    }
    __syncwarp();
    double b = (lane < n2) ? S.J[lane][n2] : 0.0;
    for (int k = n2 - 1; k >= 0; --k) {
        const double vk = __shfl_sync(0xffffffffu, b, k) * S.inv[k];
        if (lane < k)
            b -= S.J[lane][k] * vk;
        else if (lane == k)
            b = vk;
    }
    return b;
}

// The same for up to 64 unknowns: lane i owns columns i, i + 32 and i + 64 (the
// right-hand side sits in column n2 and is owned like any column), and rows i and
// i + 32 in the back substitution.  v0 = v_i, v1 = v_{i+32}.
__device__ void spd_solve_wide(BwdSmem<kSW> &S, int n2, int lane, bool &ok, double &v0, double &v1)
{
    ok = true;
    v0 = v1 = 0.0;
    for (int k = 0; k < n2; ++k) {
        __syncwarp();
        const double piv = S.J[k][k];
        if (!(piv > 0.0)) {
            ok = false;
            return;
        }
        const double ip = 1.0 / piv;
        int col[3];
        double pc[3];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const int c = lane + 32 * h;
            col[h] = (c > k && c <= n2) ? c : -1;
            pc[h] = (col[h] >= 0) ? S.J[k][c] : 0.0;
        }
        __syncwarp();
        if (lane == 0)
            S.inv[k] = ip;
        for (int i = k + 1; i < n2; ++i) {
            const double f = S.J[i][k] * ip;
#pragma unroll
            for (int h = 0; h < 3; ++h)
                if (col[h] >= 0)
                    S.J[i][col[h]] -= f * pc[h];
        }
    }
    __syncwarp();
    double b0 = (lane < n2) ? S.J[lane][n2] : 0.0;
    double b1 = (lane + 32 < n2) ? S.J[lane + 32][n2] : 0.0;
    for (int k = n2 - 1; k >= 0; --k) {
        const double src = (k >= 32) ? b1 : b0;  // k is the same in every lane
        const double vk = __shfl_sync(0xffffffffu, src, k & 31) * S.inv[k];
        if (lane < k)
            b0 -= S.J[lane][k] * vk;
        else if (lane == k)
            b0 = vk;
        if (lane + 32 < k)
            b1 -= S.J[lane + 32][k] * vk;
        else if (lane + 32 == k)
            b1 = vk;
    }
    v0 = b0;
    v1 = b1;
}

// valid support entries of pixel p (a grid index with x != 0), at most s_max of them
__device__ __forceinline__ int support_entry(const BackwardLaunch &a, int64_t p, int L, int lane, int &l,
                                             double2 &xv)
{
    int m0 = a.nsupp[p];
    m0 = m0 < 0 ? 0 : (m0 > a.s_max ? a.s_max : m0);
    if (a.status && !(a.status[p] & BPDN_PX_CERTIFIED))
        m0 = 0;  // x is not the minimiser: no derivative
    l = -1;
    xv = make_double2(0.0, 0.0);
    if (lane < m0) {
        const int li = a.support[p * a.s_max + lane];
        if (li >= 0 && li < L) {
            const float2 xf = a.x[p * L + li];
            if (xf.x != 0.f || xf.y != 0.f) {
                l = li;
                xv = make_double2((double)xf.x, (double)xf.y);
            }
        }
    }
    return __popc(__ballot_sync(0xffffffffu, l >= 0));
}

// The adjoint of one pixel whose support holds m <= KS valid entries (one warp).
template <int KS>
__device__ void backward_pixel(BwdSmem<KS> &S, int64_t p, const BackwardLaunch &a, const double2 *__restrict__ A64,
                               const double2 *__restrict__ h, int N, int L, int lane, int l, double2 xv)
{
    constexpr int NC = (2 * KS + 31) / 32;  // unknowns (rows / columns) per lane
    const double lam = a.lam_pp ? (double)a.lam[p] : (double)a.lam[0];
    const unsigned bal = __ballot_sync(0xffffffffu, l >= 0);
    const int m = __popc(bal), n2 = 2 * m;
    if (l >= 0) {
        const int i = __popc(bal & ((1u << lane) - 1u));
        S.W[i] = l;
        S.xs[i] = xv;
    }
    __syncwarp();
    bool ok = (m > 0);
    double v[NC];
#pragma unroll
    for (int hh = 0; hh < NC; ++hh)
        v[hh] = 0.0;
    if (m > 0) {
        // J: row r = 2a + ra, column c = 2b + cb (columns lane + 32 hh)
        for (int r = 0; r < n2; ++r) {
#pragma unroll
            for (int hh = 0; hh < NC; ++hh) {
                const int c = lane + 32 * hh;
                if (c < n2) {
                    const int ia = r >> 1, ra = r & 1, ib = c >> 1, cb = c & 1;
                    // (A^H A)_{W_a W_b}: the Toeplitz generator, or the FP64 operator on a
                    // multi-component grid
                    double2 gv;
                    if (h) {
                        gv = h[S.W[ia] - S.W[ib] + L - 1];
                    } else {
                        gv = make_double2(0.0, 0.0);
                        for (int n = 0; n < N; ++n) {
                            const double2 ca = A64[(size_t)n * L + S.W[ia]], cb2 = A64[(size_t)n * L + S.W[ib]];
                            gv.x += ca.x * cb2.x + ca.y * cb2.y;
                            gv.y += ca.x * cb2.y - ca.y * cb2.x;
                        }
                    }
                    double val = (ra == 0) ? (cb == 0 ? gv.x : -gv.y) : (cb == 0 ? gv.y : gv.x);
                    val *= 2.0;
                    if (ia == ib) {
                        const double2 xa = S.xs[ia];
                        const double mod = hypot(xa.x, xa.y);
                        const double wr = (ra ? xa.y : xa.x) / mod, wc = (cb ? xa.y : xa.x) / mod;
                        val += lam / mod * ((ra == cb ? 1.0 : 0.0) - wr * wc);
                    }
                    S.J[r][c] = val;
                }
            }
        }
#pragma unroll
        for (int hh = 0; hh < NC; ++hh) {
            const int c = lane + 32 * hh;
            if (c < n2) {
                const float2 cg = a.dLdx[p * L + S.W[c >> 1]];
                S.J[c][n2] = (c & 1) ? (double)cg.y : (double)cg.x;
            }
        }
        if constexpr (NC == 1)
            v[0] = spd_solve(S, n2, lane, ok);
        else
            spd_solve_wide(S, n2, lane, ok, v[0], v[NC - 1]);
    }
    double dl = 0.0;
    if (ok) {
        double t = 0.0;
#pragma unroll
        for (int hh = 0; hh < NC; ++hh) {
            const int c = lane + 32 * hh;
            if (c < n2) {
                const double2 xa = S.xs[c >> 1];
                t += ((c & 1) ? xa.y : xa.x) / hypot(xa.x, xa.y) * v[hh];
            }
        }
        dl = -warp_sum(t);
    }
    // dL/dg_n = 2 sum_a A_{n, W_a} (v_{2a} + j v_{2a+1})
    for (int n0 = 0; n0 < N; n0 += 32) {
        const int n = n0 + lane;
        double ar = 0.0, ai = 0.0;
        if (ok) {
            for (int ia = 0; ia < m; ++ia) {
                // rows 2 ia and 2 ia + 1 sit in register (2 ia) / 32 of lanes (2 ia) mod 32, + 1
                const int hs = (2 * ia) >> 5;  // the same in every lane
                const double src = (NC == 1 || hs == 0) ? v[0] : v[NC - 1];
                const double vr = __shfl_sync(0xffffffffu, src, (2 * ia) & 31);
                const double vi = __shfl_sync(0xffffffffu, src, (2 * ia + 1) & 31);
                if (n < N) {
                    const double2 av = A64[(size_t)n * L + S.W[ia]];
                    ar += av.x * vr - av.y * vi;
                    ai += av.x * vi + av.y * vr;
                }
            }
        }
        if (n < N)
            a.dLdg[p * N + n] = make_float2((float)(2.0 * ar), (float)(2.0 * ai));
    }
    if (lane == 0) {
        if (a.lam_pp)
            a.dLdlam[p] = (float)dl;
        else
            a.part[p] = dl;
    }
}

// one warp per pixel; pixels with more than 16 support entries are left to the wide kernel
__global__ void __launch_bounds__(kWarps * 32) k_backward(BackwardLaunch a, const double2 *__restrict__ A64,
                                                         const double2 *__restrict__ h, int N, int L)
{
    __shared__ BwdSmem<kSF> smem[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
    if (p >= a.P)
        return;
    int l;
    double2 xv;
    if (support_entry(a, p, L, lane, l, xv) > kSF)
        return;
    backward_pixel<kSF>(smem[warp], p, a, A64, h, N, L, lane, l, xv);
}

// the pixels with 17..32 support entries: a persistent launch, one warp per block, each
// warp reading the support counts of 32 pixels at a time
__global__ void __launch_bounds__(32) k_backward_wide(BackwardLaunch a, const double2 *__restrict__ A64,
                                                      const double2 *__restrict__ h, int N, int L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<kSW> &S = *(BwdSmem<kSW> *)smem_raw;
    const int lane = threadIdx.x & 31;
    for (int64_t p0 = 32LL * blockIdx.x; p0 < a.P; p0 += 32LL * gridDim.x) {
        const int64_t q = p0 + lane;
        const bool maybe = (q < a.P) && a.nsupp[q] > kSF;
        unsigned bal = __ballot_sync(0xffffffffu, maybe);
        while (bal) {
            const int j = __ffs(bal) - 1;
            bal &= bal - 1;
            int l;
            double2 xv;
            if (support_entry(a, p0 + j, L, lane, l, xv) > kSF)
                backward_pixel<kSW>(S, p0 + j, a, A64, h, N, L, lane, l, xv);
            __syncwarp();
        }
    }
}

// sum of the per-pixel terms in a fixed order: strided partial sums, then a tree
__global__ void __launch_bounds__(kSumThreads) k_sum_fixed(const double *__restrict__ part, int64_t P, float *out)
{
    __shared__ double red[kSumThreads];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < P; i += kSumThreads)
        s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = kSumThreads / 2; off >= 1; off >>= 1) {
        if ((int)threadIdx.x < off)
            red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[0] = (float)red[0];
}

}  // namespace

cudaError_t launch_backward(const OpHandle &op, const BackwardLaunch &a, cudaStream_t s)
{
    const long long blocks = (a.P + kWarps - 1) / kWarps;
    const double2 *h = op.md ? nullptr : op.h;
    k_backward<<<(unsigned)blocks, kWarps * 32, 0, s>>>(a, op.A64, h, op.N, op.L);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && a.s_max > kSF) {
        const size_t smem = sizeof(BwdSmem<kSW>);
        e = cudaFuncSetAttribute(k_backward_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0, per_sm = 0;
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward_wide, 32, smem);
        if (e != cudaSuccess)
            return e;
        long long wb = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        const long long groups = (a.P + 31) / 32;
        if (wb > groups)
            wb = groups;
        k_backward_wide<<<(unsigned)wb, 32, smem, s>>>(a, op.A64, h, op.N, op.L);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || a.lam_pp)
        return e;
    k_sum_fixed<<<1, kSumThreads, 0, s>>>(a.part, a.P, a.dLdlam);
    return cudaGetLastError();
}

}  // namespace bpdn
