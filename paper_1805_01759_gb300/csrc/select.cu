// SL1MMER model selection and parameter estimation (Sec. III-A, steps (2) and (3)),
// one warp per pixel, FP64.  The paper names the steps and defers their definition
// to the original SL1MMER publication; this kernel implements the following reading.
//
//   Candidates: maximal runs of adjacent grid points in the support of the minimiser
//   x.  A run's elevation is the modulus-weighted centroid sum |x_l| s_l / sum |x_l|,
//   its energy sum |x_l|^2 (both summed in ascending grid order).  Runs are ranked by
//   energy, largest first (ties: lower first grid point first); at most kmax are kept.
//   Model order: for K = 0 .. K_c the first K candidates are fitted by least squares
//   with the steering vectors of Eq. 5 at their (off-grid) elevations,
//       gamma_K = argmin ||g - A_K gamma||^2,   RSS_K = ||g - A_K gamma_K||^2,
//   and K_hat is the first minimiser of the information criterion
//       C(K) = 2 N ln RSS_K + K * penalty,   penalty = 3 ln(2N) by default
//   (circular Gaussian likelihood with unknown noise power; three real parameters per
//   scatterer, 2N real observations).  Estimates: the K_hat elevations in ascending
//   order with the amplitudes of that fit.
//
// The normal equations (K <= 4) are solved by a complex Cholesky factorisation; the
// residual is formed explicitly, not from ||g||^2 - b^H gamma.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int KS = BPDN_MAX_KSEL;
constexpr int NRW = (BPDN_MAX_N + 31) / 32;  // rows n = lane + 32 c, c < NRW, per lane
constexpr int WARPS = 4;  // pixels per block

struct SelSmem {
    double2 a[KS][BPDN_MAX_N];  // steering vectors of the ranked candidates
    double2 gram[KS][KS];       // A^H A of the candidates
    double2 b[KS];              // A^H g
    double2 fit[KS + 1][KS];    // gamma_K for each K
    double crit[KS + 1];
    double w[BPDN_MAX_SMAX];    // |x_l| of the support entries (ascending l)
    int l[BPDN_MAX_SMAX];
    double cen[BPDN_MAX_SMAX], en[BPDN_MAX_SMAX];
    int first[BPDN_MAX_SMAX], rank[BPDN_MAX_SMAX];
    int kc;                     // candidates kept (<= kmax)
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ double2 cmulc(double2 a, double2 b)  // conj(a) * b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Solve G[0..K) z = b by G = R R^H (R lower, real diagonal); false if G is not
// numerically positive definite.  One thread.
__device__ bool chol_solve(const double2 (&G)[KS][KS], const double2 *b, int K, double2 *z)
{
    double2 R[KS][KS];
    for (int j = 0; j < K; ++j) {
        double d = G[j][j].x;
        for (int k = 0; k < j; ++k)
            d -= R[j][k].x * R[j][k].x + R[j][k].y * R[j][k].y;
        if (!(d > 0.0))
            return false;
        const double rj = sqrt(d);
        R[j][j] = make_double2(rj, 0.0);
        for (int i = j + 1; i < K; ++i) {
            // G_ij for i > j is conj(G_ji)
            double2 v = make_double2(G[j][i].x, -G[j][i].y);
            for (int k = 0; k < j; ++k) {
                const double2 t = cmul(R[i][k], make_double2(R[j][k].x, -R[j][k].y));
                v.x -= t.x;
                v.y -= t.y;
            }
            R[i][j] = make_double2(v.x / rj, v.y / rj);
        }
    }
    double2 y[KS];
    for (int i = 0; i < K; ++i) {
        double2 v = b[i];
        for (int k = 0; k < i; ++k) {
            const double2 t = cmul(R[i][k], y[k]);
            v.x -= t.x;
            v.y -= t.y;
        }
        y[i] = make_double2(v.x / R[i][i].x, v.y / R[i][i].x);
    }
    for (int i = K - 1; i >= 0; --i) {
        double2 v = y[i];
        for (int k = i + 1; k < K; ++k) {
            const double2 t = cmulc(R[k][i], z[k]);
            v.x -= t.x;
            v.y -= t.y;
        }
        z[i] = make_double2(v.x / R[i][i].x, v.y / R[i][i].x);
    }
    return true;
}

__global__ void __launch_bounds__(WARPS * 32) k_select(const double *__restrict__ xi, int N, int L, double s_min,
                                                       double s_max, SelectLaunch a)
{
    __shared__ SelSmem smem[WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SelSmem &S = smem[warp];
    const long long p = (long long)blockIdx.x * WARPS + warp;
    if (p >= a.P)
        return;
    const int kmax = a.kmax;
    double *sh = a.s_hat + (size_t)p * kmax;
    double2 *gh = a.gamma_hat + (size_t)p * kmax;
    if (lane < kmax) {
        sh[lane] = __longlong_as_double(0x7ff8000000000000LL);  // NaN: no estimate
        gh[lane] = make_double2(0.0, 0.0);
    }
    const int st = a.status ? a.status[p] : 0;
    if (st & (BPDN_PX_NONFINITE | BPDN_PX_SUPPORT_OVERFLOW)) {
        if (lane == 0)
            a.khat[p] = -1;
        return;
    }

    // support entries with nonzero x, ascending (the support array is ascending)
    const int ns = min(max(a.nsupp[p], 0), a.s_max);
    int l = -1;
    double w = 0.0;
    bool valid = false;
    if (lane < ns) {
        l = a.support[(size_t)p * a.s_max + lane];
        if (l >= 0 && l < L) {
            const float2 v = a.x[(size_t)p * L + l];
            const double vx = (double)v.x, vy = (double)v.y;
            valid = (vx != 0.0 || vy != 0.0);
            w = sqrt(vx * vx + vy * vy);
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    if (valid) {
        const int pos = __popc(bal & ((1u << lane) - 1u));
        S.l[pos] = l;
        S.w[pos] = w;
    }
    __syncwarp();
    if (lane == 0) {
        const int nv = __popc(bal);
        int nc = 0;
        double sw = 0.0, sws = 0.0, e = 0.0;
        for (int i = 0; i < nv; ++i) {
            if (i == 0 || S.l[i] != S.l[i - 1] + 1) {
                if (nc > 0) {
                    S.cen[nc - 1] = sws / sw;
                    S.en[nc - 1] = e;
                }
                S.first[nc] = S.l[i];
                ++nc;
                sw = sws = e = 0.0;
            }
            const double sl = (L > 1) ? s_min + (double)S.l[i] * (s_max - s_min) / (double)(L - 1) : s_min;
            sw += S.w[i];
            sws += S.w[i] * sl;
            e += S.w[i] * S.w[i];
        }
        if (nc > 0) {
            S.cen[nc - 1] = sws / sw;
            S.en[nc - 1] = e;
        }
        // rank by energy, largest first; ties: lower first grid point first
        for (int i = 0; i < nc; ++i)
            S.rank[i] = i;
        for (int i = 1; i < nc; ++i) {
            const int c = S.rank[i];
            int j = i - 1;
            while (j >= 0 && (S.en[S.rank[j]] < S.en[c] ||
                              (S.en[S.rank[j]] == S.en[c] && S.first[S.rank[j]] > S.first[c]))) {
                S.rank[j + 1] = S.rank[j];
                --j;
            }
            S.rank[j + 1] = c;
        }
        S.kc = min(nc, kmax);
    }
    __syncwarp();
    const int kc = S.kc;

    // steering vectors and g: lane owns rows n = lane + 32 c
    double2 gv[NRW];
#pragma unroll
    for (int c = 0; c < NRW; ++c) {
        const int n = lane + 32 * c;
        gv[c] = make_double2(0.0, 0.0);
        if (n < N) {
            const float2 gg = a.g[(size_t)p * N + n];
            gv[c] = make_double2((double)gg.x, (double)gg.y);
            for (int k = 0; k < kc; ++k) {
                double sn, cs;
                sincospi(2.0 * xi[n] * S.cen[S.rank[k]], &sn, &cs);
                S.a[k][n] = make_double2(cs, -sn);  // exp(-j 2 pi xi_n s)
            }
        }
    }
    __syncwarp();
    // Gram matrix, A^H g and ||g||^2 by warp sums
    for (int i = 0; i < kc; ++i) {
        for (int j = i; j < kc; ++j) {
            double2 t = make_double2(0.0, 0.0);
#pragma unroll
            for (int c = 0; c < NRW; ++c) {
                const int n = lane + 32 * c;
                if (n < N) {
                    const double2 v = cmulc(S.a[i][n], S.a[j][n]);
                    t.x += v.x;
                    t.y += v.y;
                }
            }
            t.x = warp_sum_d(t.x);
            t.y = warp_sum_d(t.y);
            if (lane == 0)
                S.gram[i][j] = t;
        }
        double2 t = make_double2(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < NRW; ++c) {
            const int n = lane + 32 * c;
            if (n < N) {
                const double2 v = cmulc(S.a[i][n], gv[c]);
                t.x += v.x;
                t.y += v.y;
            }
        }
        t.x = warp_sum_d(t.x);
        t.y = warp_sum_d(t.y);
        if (lane == 0)
            S.b[i] = t;
    }
    double g2 = 0.0;
#pragma unroll
    for (int c = 0; c < NRW; ++c)
        g2 += gv[c].x * gv[c].x + gv[c].y * gv[c].y;
    g2 = warp_sum_d(g2);
    const double pen = (a.penalty > 0.0) ? a.penalty : 3.0 * log(2.0 * (double)N);
    if (lane == 0)
        S.crit[0] = 2.0 * (double)N * log(g2);
    __syncwarp();

    // nested least-squares fits K = 1 .. kc
    int kok = kc;  // fits beyond a singular Gram block are not considered
    for (int K = 1; K <= kc; ++K) {
        int ok = 1;
        if (lane == 0)
            ok = chol_solve(S.gram, S.b, K, S.fit[K]) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
        if (!ok) {
            kok = K - 1;
            break;
        }
        double r2 = 0.0;
#pragma unroll
        for (int c = 0; c < NRW; ++c) {
            const int n = lane + 32 * c;
            if (n < N) {
                double2 r = gv[c];
                for (int k = 0; k < K; ++k) {
                    const double2 t = cmul(S.a[k][n], S.fit[K][k]);
                    r.x -= t.x;
                    r.y -= t.y;
                }
                r2 += r.x * r.x + r.y * r.y;
            }
        }
        r2 = warp_sum_d(r2);
        if (lane == 0)
            S.crit[K] = 2.0 * (double)N * log(r2) + pen * (double)K;
        __syncwarp();
    }
    if (lane == 0) {
        int kh = 0;
        for (int K = 1; K <= kok; ++K)
            if (S.crit[K] < S.crit[kh])
                kh = K;
        // the kh estimates in ascending elevation
        int ord[KS];
        for (int k = 0; k < kh; ++k)
            ord[k] = k;
        for (int i = 1; i < kh; ++i) {
            const int c = ord[i];
            int j = i - 1;
            while (j >= 0 && S.cen[S.rank[ord[j]]] > S.cen[S.rank[c]]) {
                ord[j + 1] = ord[j];
                --j;
            }
            ord[j + 1] = c;
        }
        for (int k = 0; k < kh; ++k) {
            sh[k] = S.cen[S.rank[ord[k]]];
            gh[k] = S.fit[kh][ord[k]];
        }
        a.khat[p] = kh;
    }
}

}  // namespace

cudaError_t launch_select(const OpHandle &op, const SelectLaunch &a, cudaStream_t s)
{
    if (a.P <= 0)
        return cudaSuccess;
    const long long blocks = (a.P + WARPS - 1) / WARPS;
    k_select<<<(unsigned)blocks, WARPS * 32, 0, s>>>(op.xi, op.N, op.L, op.s_min, op.s_max, a);
    return cudaGetLastError();
}

}  // namespace bpdn
