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
// FP64: lanes over the columns of J for the elimination, lanes over the rows of A
// for dL/dg.  With one lambda for all pixels the per-pixel terms are summed by a
// second kernel in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kWarps = 4;        // pixels per block
constexpr int kS = kRefitMax;    // support capacity (2|S| <= 32 lanes)
constexpr int kSumThreads = 1024;

struct BwdSmem {
    double J[2 * kS][2 * kS + 1];  // the system, right-hand side in column n2
    double inv[2 * kS];            // reciprocal pivots
    double2 xs[kS];                // x on the support (FP64)
    int W[kS];                     // support indices
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
__device__ double spd_solve(BwdSmem &S, int n2, int lane, bool &ok)
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

__global__ void __launch_bounds__(kWarps * 32) k_backward(BackwardLaunch a, const double2 *__restrict__ A64,
                                                         const double2 *__restrict__ h, int N, int L)
{
    __shared__ BwdSmem smem[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
    if (p >= a.P)
        return;
    BwdSmem &S = smem[warp];
    const double lam = a.lam_pp ? (double)a.lam[p] : (double)a.lam[0];
    int m0 = a.nsupp[p];
    m0 = m0 < 0 ? 0 : (m0 > a.s_max ? a.s_max : m0);
    if (a.status && !(a.status[p] & BPDN_PX_CERTIFIED))
        m0 = 0;  // x is not the minimiser: no derivative
    // the support entries that name a grid index with x != 0
    int l = -1;
    double2 xv = make_double2(0.0, 0.0);
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
    const unsigned bal = __ballot_sync(0xffffffffu, l >= 0);
    const int m = __popc(bal), n2 = 2 * m;
    if (l >= 0) {
        const int i = __popc(bal & ((1u << lane) - 1u));
        S.W[i] = l;
        S.xs[i] = xv;
    }
    __syncwarp();
    bool ok = (m > 0);
    double v = 0.0;
    if (m > 0) {
        // J: row r = 2a + ra, column lane = 2b + cb
        for (int r = 0; r < n2; ++r) {
            if (lane < n2) {
                const int ia = r >> 1, ra = r & 1, ib = lane >> 1, cb = lane & 1;
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
                S.J[r][lane] = val;
            }
        }
        if (lane < n2) {
            const float2 c = a.dLdx[p * L + S.W[lane >> 1]];
            S.J[lane][n2] = (lane & 1) ? (double)c.y : (double)c.x;
        }
        v = spd_solve(S, n2, lane, ok);
    }
    double dl = 0.0;
    if (ok) {
        double t = 0.0;
        if (lane < n2) {
            const double2 xa = S.xs[lane >> 1];
            t = ((lane & 1) ? xa.y : xa.x) / hypot(xa.x, xa.y) * v;
        }
        dl = -warp_sum(t);
    }
    // dL/dg_n = 2 sum_a A_{n, W_a} (v_{2a} + j v_{2a+1})
    for (int n0 = 0; n0 < N; n0 += 32) {
        const int n = n0 + lane;
        double ar = 0.0, ai = 0.0;
        if (ok) {
            for (int ia = 0; ia < m; ++ia) {
                const double vr = __shfl_sync(0xffffffffu, v, 2 * ia);
                const double vi = __shfl_sync(0xffffffffu, v, 2 * ia + 1);
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
    k_backward<<<(unsigned)blocks, kWarps * 32, 0, s>>>(a, op.A64, op.md ? nullptr : op.h, op.N, op.L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.lam_pp)
        return e;
    k_sum_fixed<<<1, kSumThreads, 0, s>>>(a.part, a.P, a.dLdlam);
    return cudaGetLastError();
}

}  // namespace bpdn
