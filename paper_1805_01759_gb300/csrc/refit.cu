// Support extraction and FP64 refit (the refinement after Algorithm 1; SL1MMER
// step (3), Sec. III-A), one warp per pixel.
//
//   1. W = {l : x_in[l] != 0}, ascending (warp ballots over the grid).
//   2. Exact minimiser of the problem of Eq. 6 restricted to W,
//          min_z  z^H G z - 2 Re(c^H z) + lambda sum_i |z_i|,   G = A_W^H A_W, c = A_W^H g,
//      in FP64 (G from the Toeplitz generator h, c from the FP64 operator).
//      Each round alternates one sweep of exact one-coordinate minimisations
//      (which can switch a coordinate on or off) with one damped Newton step on
//      the coordinates that are nonzero.  The Newton system is the Hessian in real
//      coordinates, 2 [[Re G, -Im G],[Im G, Re G]] + lambda/|z_i| (I - u_i u_i^T);
//      the step is kept where the objective is smooth (no modulus falls below a
//      tenth of its value along the step) and must lower the objective or the
//      gradient norm.  Done when 2 (G z - c)_i + lambda z_i/|z_i| = 0 on the nonzeros
//      and |2 (G z - c)_i| <= lambda on the zeros of W.
//   3. Certificate over the whole grid: |2 a_l^H (A z - g)| <= lambda for l not in W
//      (FP32 products against an FP64 residual, relative slack 1e-5).  Violating grid
//      points join W (largest first) and step 2 repeats, for at most `rounds` rounds.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int KW = kRefitMax;       // working-set capacity (<= 16, so 2|W| <= 32 lanes)
constexpr int WARPS = 4;            // pixels per block
constexpr int kFastRounds = 15;
constexpr double kOptTol = 1e-12;  // optimality residual relative to lambda

struct WarpSmem {
    double2 G[KW][KW];
    double J[2 * KW][2 * KW + 1];
    double rhs[2 * KW];
    double2 z[KW], c[KW], zt[KW], dz[KW], gam[KW];
    double2 r[BPDN_MAX_N];   // g (FP64)
    double2 rr[BPDN_MAX_N];  // A_W z - g (FP64)
    float2 rf[BPDN_MAX_N];   // A_W z - g (FP32 copy)
    int W[KW];
    int T[KW];
    int m, nt;
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// (G z)_i for lane i < m
__device__ __forceinline__ double2 gz_row(const WarpSmem &S, int i, int m, const double2 *z)
{
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < m; ++j)
        acc = cadd(acc, cmul(S.G[i][j], z[j]));
    return acc;
}

// gam_i = 2 (G z - c)_i for i < m (into S.gam); returns the optimality residual
// max( max_{z_i != 0} |gam_i + lam u_i| / lam,  max_{z_i == 0} (|gam_i|/lam - 1) )
__device__ double optimality(WarpSmem &S, int m, double lam, int lane)
{
    double res = 0.0;
    if (lane < m) {
        double2 gz = gz_row(S, lane, m, S.z);
        double2 gm = make_double2(2.0 * (gz.x - S.c[lane].x), 2.0 * (gz.y - S.c[lane].y));
        S.gam[lane] = gm;
        double2 zi = S.z[lane];
        double a = sqrt(cabs2(zi));
        if (a > 0.0) {
            double ex = gm.x + lam * zi.x / a, ey = gm.y + lam * zi.y / a;
            res = sqrt(ex * ex + ey * ey) / lam;
        } else {
            res = sqrt(cabs2(gm)) / lam - 1.0;
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        res = fmax(res, __shfl_xor_sync(0xffffffffu, res, off));
    __syncwarp();
    return res;
}

// Solve S.J[0..n2) x = S.rhs in place (symmetric positive definite: Gaussian
// elimination without pivoting, lanes over columns).  Returns false on a
// non-positive pivot.  The solution is left in S.rhs.
__device__ bool solve_spd(WarpSmem &S, int n2, int lane)
{
    for (int k = 0; k < n2; ++k) {
        const double piv = S.J[k][k];
        if (!(piv > 0.0))
            return false;
        for (int i = k + 1; i < n2; ++i) {
            const double f = S.J[i][k] / piv;
            __syncwarp();
            if (lane >= k && lane < n2)
                S.J[i][lane] -= f * S.J[k][lane];
            if (lane == 0)
                S.rhs[i] -= f * S.rhs[k];
            __syncwarp();
        }
    }
    if (lane == 0) {
        for (int k = n2 - 1; k >= 0; --k) {
            double sacc = S.rhs[k];
            for (int j = k + 1; j < n2; ++j)
                sacc -= S.J[k][j] * S.rhs[j];
            S.rhs[k] = sacc / S.J[k][k];
        }
    }
    __syncwarp();
    return true;
}

// One exact coordinate-minimisation sweep over W:
//   z_i <- S_{lam/2}(c_i - sum_{j != i} G_ij z_j) / G_ii
__device__ void cd_sweep(WarpSmem &S, int m, double lam, int lane)
{
    for (int i = 0; i < m; ++i) {
        double2 t = make_double2(0.0, 0.0);
        if (lane < m && lane != i)
            t = cmul(S.G[i][lane], S.z[lane]);
        double qx = warp_sum(t.x), qy = warp_sum(t.y);
        if (lane == 0) {
            qx = S.c[i].x - qx;
            qy = S.c[i].y - qy;
            const double a = sqrt(qx * qx + qy * qy);
            const double th = 0.5 * lam;
            const double gii = S.G[i][i].x;
            if (a > th) {
                const double sc = (1.0 - th / a) / gii;
                S.z[i] = make_double2(qx * sc, qy * sc);
            } else {
                S.z[i] = make_double2(0.0, 0.0);
            }
        }
        __syncwarp();
    }
}

// Newton direction for the objective restricted to the nonzero coordinates of
// `z` (exact modulus, eps = 0) or for the smoothed objective over all of W
// (|z_i| replaced by sqrt(|z_i|^2 + eps^2), eps > 0).  Writes S.dz (zero off
// the variable set) and returns the directional derivative (negative for a
// descent direction), or +1 when the system could not be solved.
__device__ double newton_dir(WarpSmem &S, int m, const double2 *z, double lam, double eps, int lane)
{
    if (lane == 0) {
        int nt = 0;
        for (int i = 0; i < m; ++i)
            if (eps > 0.0 || z[i].x != 0.0 || z[i].y != 0.0)
                S.T[nt++] = i;
        S.nt = nt;
    }
    __syncwarp();
    const int nt = S.nt, n2 = 2 * nt;
    if (nt == 0)
        return 1.0;
    // gradient of the (smoothed) objective: 2 (G z - c)_i + lam z_i / q_i
    if (lane < m) {
        double2 gz = gz_row(S, lane, m, z);
        S.gam[lane] = make_double2(2.0 * (gz.x - S.c[lane].x), 2.0 * (gz.y - S.c[lane].y));
    }
    __syncwarp();
    for (int rI = 0; rI < n2; ++rI) {
        const int a = rI >> 1, ra = rI & 1;
        const int ia = S.T[a];
        if (lane < n2) {
            const int b = lane >> 1, cb = lane & 1;
            const int ib = S.T[b];
            const double2 g = S.G[ia][ib];
            double v = (ra == 0) ? (cb == 0 ? g.x : -g.y) : (cb == 0 ? g.y : g.x);
            v *= 2.0;
            if (a == b) {
                const double2 zi = z[ia];
                const double q = sqrt(cabs2(zi) + eps * eps);
                const double w0 = zi.x / q, w1 = zi.y / q;
                const double wr = ra ? w1 : w0, wc = cb ? w1 : w0;
                v += lam / q * ((ra == cb ? 1.0 : 0.0) - wr * wc);
            }
            S.J[rI][lane] = v;
        }
    }
    double slope_part = 0.0;
    if (lane < n2) {
        const int ia = S.T[lane >> 1];
        const double2 zi = z[ia];
        const double q = sqrt(cabs2(zi) + eps * eps);
        const double gcomp = (lane & 1) ? (S.gam[ia].y + lam * zi.y / q) : (S.gam[ia].x + lam * zi.x / q);
        S.rhs[lane] = -gcomp;
        slope_part = gcomp;  // times d below
    }
    __syncwarp();
    if (!solve_spd(S, n2, lane))
        return 1.0;
    if (lane < m)
        S.dz[lane] = make_double2(0.0, 0.0);
    __syncwarp();
    double sl = 0.0;
    if (lane < n2)
        sl = slope_part * S.rhs[lane];
    if (lane < nt)
        S.dz[S.T[lane]] = make_double2(S.rhs[2 * lane], S.rhs[2 * lane + 1]);
    __syncwarp();
    return warp_sum(sl);
}

// objective over W with |z| smoothed by eps (eps = 0: exact)
__device__ double objective_W(const WarpSmem &S, int m, const double2 *z, double lam, double eps, int lane)
{
    double v = 0.0;
    if (lane < m) {
        const double2 gz = gz_row(S, lane, m, z);
        const double2 zi = z[lane];
        v = (zi.x * gz.x + zi.y * gz.y) - 2.0 * (S.c[lane].x * zi.x + S.c[lane].y * zi.y) +
            lam * sqrt(cabs2(zi) + eps * eps);
    }
    return warp_sum(v);
}

// does the segment z_i + s dz_i, s in [0, t], come within a tenth of |z_i| of zero?
__device__ __forceinline__ bool passes_zero(double2 zi, double2 d, double t)
{
    const double dd = cabs2(d);
    if (!(dd > 0.0) || (zi.x == 0.0 && zi.y == 0.0))
        return false;
    double s = -(zi.x * d.x + zi.y * d.y) / dd;
    s = fmin(fmax(s, 0.0), t);
    const double2 p = make_double2(zi.x + s * d.x, zi.y + s * d.y);
    return cabs2(p) < 0.01 * cabs2(zi);
}

// Fast path of step 2: coordinate sweeps alternating with Newton steps on the
// nonzero coordinates.  A coordinate that a full Newton step would carry through
// zero is set to zero and the step recomputed; the swap is kept when the
// objective falls.  Returns true on convergence.
__device__ bool solve_fast(WarpSmem &S, double lam, int lane, int max_outer)
{
    const int m = S.m;
    for (int outer = 0; outer < max_outer; ++outer) {
        cd_sweep(S, m, lam, lane);
        double res = optimality(S, m, lam, lane);
        if (res <= kOptTol)
            return true;
        const double F0 = objective_W(S, m, S.z, lam, 0.0, lane);
        double slope = newton_dir(S, m, S.z, lam, 0.0, lane);
        if (slope > 0.0)
            continue;
        // coordinates the full step carries through zero
        bool blk = (lane < m) && passes_zero(S.z[lane], S.dz[lane], 1.0);
        const unsigned bmask = __ballot_sync(0xffffffffu, blk);
        if (bmask) {
            double2 zkeep = (lane < m) ? S.z[lane] : make_double2(0.0, 0.0);
            if (lane < m)
                S.zt[lane] = blk ? make_double2(0.0, 0.0) : zkeep;
            __syncwarp();
            const double sl2 = newton_dir(S, m, S.zt, lam, 0.0, lane);
            bool ok2 = sl2 < 0.0;
            if (ok2) {
                bool blk2 = (lane < m) && passes_zero(S.zt[lane], S.dz[lane], 1.0);
                ok2 = !__any_sync(0xffffffffu, blk2);
            }
            if (ok2) {
                if (lane < m)
                    S.zt[lane] = make_double2(S.zt[lane].x + S.dz[lane].x, S.zt[lane].y + S.dz[lane].y);
                __syncwarp();
                const double F2 = objective_W(S, m, S.zt, lam, 0.0, lane);
                if (F2 < F0) {
                    if (lane < m)
                        S.z[lane] = S.zt[lane];
                    __syncwarp();
                    if (optimality(S, m, lam, lane) <= kOptTol)
                        return true;
                    continue;
                }
            }
            // recompute the plain direction for the damped step below
            slope = newton_dir(S, m, S.z, lam, 0.0, lane);
            if (slope > 0.0)
                continue;
        }
        // damped step kept inside the smooth region
        double t = 1.0;
        for (int h = 0; h < 60; ++h) {
            const bool bad = (lane < m) && passes_zero(S.z[lane], S.dz[lane], t);
            if (!__any_sync(0xffffffffu, bad))
                break;
            t *= 0.5;
        }
        const double2 keep = (lane < m) ? S.z[lane] : make_double2(0.0, 0.0);
        bool accepted = false;
        for (int h = 0; h < 50 && t > 1e-14; ++h, t *= 0.5) {
            if (lane < m)
                S.zt[lane] = make_double2(keep.x + t * S.dz[lane].x, keep.y + t * S.dz[lane].y);
            __syncwarp();
            const double F1 = objective_W(S, m, S.zt, lam, 0.0, lane);
            if (F1 <= F0 + 1e-4 * t * slope) {
                accepted = true;
                break;
            }
            if (h == 0) {
                // near the minimiser the objective no longer resolves the decrease
                if (lane < m)
                    S.z[lane] = S.zt[lane];
                __syncwarp();
                const double r1 = optimality(S, m, lam, lane);
                if (lane < m)
                    S.z[lane] = keep;
                __syncwarp();
                if (r1 < 0.5 * res) {
                    accepted = true;
                    break;
                }
            }
        }
        if (accepted && lane < m)
            S.z[lane] = S.zt[lane];
        __syncwarp();
        if (optimality(S, m, lam, lane) <= kOptTol)
            return true;
    }
    return false;
}

// Fallback of step 2: damped Newton on the smoothed objective (|z| replaced by
// sqrt(|z|^2 + eps^2): smooth and strictly convex, so damped Newton converges
// from any start) for eps = 1e-1, 1e-2, ..., 1e-13 times the scale of z, each
// level warm-started from the last; then coordinates below 1e-6 of the scale are
// set to zero and exact Newton steps on the rest finish.  Returns true on convergence.
__device__ bool solve_continuation(WarpSmem &S, double lam, int lane)
{
    const int m = S.m;
    double sc = (lane < m) ? sqrt(cabs2(S.z[lane])) : 0.0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, off));
    sc = fmax(sc, 1e-3);
    for (double eps = 1e-1 * sc; eps >= 1e-13 * sc; eps *= 0.1) {
        for (int it = 0; it < 40; ++it) {
            const double slope = newton_dir(S, m, S.z, lam, eps, lane);
            if (!(slope < 0.0) || -slope <= 1e-28 * fmax(1.0, sc * sc))
                break;
            const double F0 = objective_W(S, m, S.z, lam, eps, lane);
            const double2 keep = (lane < m) ? S.z[lane] : make_double2(0.0, 0.0);
            double t = 1.0;
            for (int h = 0; h < 45; ++h, t *= 0.5) {
                if (lane < m)
                    S.zt[lane] = make_double2(keep.x + t * S.dz[lane].x, keep.y + t * S.dz[lane].y);
                __syncwarp();
                if (objective_W(S, m, S.zt, lam, eps, lane) <= F0 + 1e-4 * t * slope)
                    break;
            }
            if (lane < m)
                S.z[lane] = S.zt[lane];
            __syncwarp();
            if (-slope < 1e-20 * fmax(1.0, fabs(F0)))
                break;
        }
    }
    if (lane < m && sqrt(cabs2(S.z[lane])) <= 1e-6 * sc)
        S.z[lane] = make_double2(0.0, 0.0);
    __syncwarp();
    for (int it = 0; it < 20; ++it) {
        if (optimality(S, m, lam, lane) <= kOptTol)
            return true;
        const double slope = newton_dir(S, m, S.z, lam, 0.0, lane);
        if (slope > 0.0)
            break;
        if (lane < m)
            S.z[lane] = make_double2(S.z[lane].x + S.dz[lane].x, S.z[lane].y + S.dz[lane].y);
        __syncwarp();
    }
    return optimality(S, m, lam, lane) <= kOptTol;
}

__global__ void __launch_bounds__(WARPS * 32) k_refit(const double2 *__restrict__ A64,
                                                      const double2 *__restrict__ h,
                                                      const float *__restrict__ A_re,
                                                      const float *__restrict__ A_im, int N,
                                                      int L, int lda, RefitLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem &S = ((WarpSmem *)smem_raw)[warp];
    const long long p = (long long)blockIdx.x * WARPS + warp;
    if (p >= a.P)
        return;
    const int smax = a.s_max;
    const float2 *xin = a.x_in + (size_t)p * L;
    const float2 *gp = a.g + (size_t)p * N;
    const double lam = (double)(a.lam_pp ? a.lam[p] : a.lam[0]);

    // 1. working set W: the nonzeros of x_in (ascending), or the s_max largest of them
    int nnz = 0;
    for (int l0 = 0; l0 < L; l0 += 32) {
        const int l = l0 + lane;
        const float2 v = (l < L) ? xin[l] : make_float2(0.f, 0.f);
        nnz += __popc(__ballot_sync(0xffffffffu, v.x != 0.f || v.y != 0.f));
    }
    const bool truncated = nnz > smax;
    if (!truncated) {
        int m = 0;
        for (int l0 = 0; l0 < L; l0 += 32) {
            const int l = l0 + lane;
            const float2 v = (l < L) ? xin[l] : make_float2(0.f, 0.f);
            const bool nz = (v.x != 0.f || v.y != 0.f);
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            if (nz) {
                S.W[pos] = l;
                S.z[pos] = make_double2((double)v.x, (double)v.y);
            }
            m += __popc(bal);
        }
        if (lane == 0)
            S.m = m;
    } else {
        // s_max rounds of a warp arg-max over |x_l|^2, excluding grid points taken
        uint32_t taken = 0;  // bit j: l = lane + 32 j already in W (L <= 1024)
        for (int k = 0; k < smax; ++k) {
            float best = -1.f;
            int bl = -1;
            for (int j = 0; lane + 32 * j < L; ++j) {
                if (taken & (1u << j))
                    continue;
                const float2 v = xin[lane + 32 * j];
                const float a2 = v.x * v.x + v.y * v.y;
                if (a2 > best) {
                    best = a2;
                    bl = lane + 32 * j;
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
                if (ob > best || (ob == best && ol >= 0 && (bl < 0 || ol < bl))) {
                    best = ob;
                    bl = ol;
                }
            }
            if (bl < 0)
                break;  // cannot happen: more than s_max grid points are nonzero
            if ((bl & 31) == lane)
                taken |= 1u << (bl >> 5);
            if (lane == 0) {
                const float2 v = xin[bl];
                S.W[k] = bl;
                S.z[k] = make_double2((double)v.x, (double)v.y);
            }
        }
        __syncwarp();
        if (lane == 0) {
            S.m = smax;
            for (int i = 1; i < smax; ++i) {
                const int w = S.W[i];
                const double2 zz = S.z[i];
                int j = i - 1;
                while (j >= 0 && S.W[j] > w) {
                    S.W[j + 1] = S.W[j];
                    S.z[j + 1] = S.z[j];
                    --j;
                }
                S.W[j + 1] = w;
                S.z[j + 1] = zz;
            }
        }
    }
    const int status = a.status[p];
    for (int n = lane; n < N; n += 32) {
        const float2 gg = gp[n];
        S.r[n] = make_double2((double)gg.x, (double)gg.y);
    }
    __syncwarp();

    bool certified = false, noroom = false;
    for (int round = 0; round <= a.rounds; ++round) {
        const int m = S.m;
        // G_ij = h(l_i - l_j), c_i = a_{l_i}^H g
        for (int e = lane; e < m * m; e += 32) {
            const int i = e / m, j = e % m;
            S.G[i][j] = h[S.W[i] - S.W[j] + L - 1];
        }
        if (lane < m) {
            const int l = S.W[lane];
            double2 acc = make_double2(0.0, 0.0);
            for (int n = 0; n < N; ++n) {
                const double2 av = A64[(size_t)n * L + l], gv = S.r[n];
                acc.x += av.x * gv.x + av.y * gv.y;
                acc.y += av.x * gv.y - av.y * gv.x;
            }
            S.c[lane] = acc;
        }
        __syncwarp();
        // 2. exact minimiser over W
        bool conv = solve_fast(S, lam, lane, kFastRounds);
        if (!conv)
            conv = solve_continuation(S, lam, lane);
        if (!conv)
            break;
        // residual A_W z - g in FP64 and its FP32 copy
        for (int n = lane; n < N; n += 32) {
            double2 acc = make_double2(-S.r[n].x, -S.r[n].y);
            for (int i = 0; i < m; ++i)
                acc = cadd(acc, cmul(A64[(size_t)n * L + S.W[i]], S.z[i]));
            S.rr[n] = acc;
            S.rf[n] = make_float2((float)acc.x, (float)acc.y);
        }
        __syncwarp();
        // 3. certificate off W: |2 a_l^H r| <= lambda.  FP32 products first; grid
        // points within 1e-4 of the bound are recomputed in FP64 and must satisfy
        // it to 1e-9.
        const float near = (float)lam * (1.0f - 1e-4f);
        double worst = 0.0;
        int worst_l = -1;
        for (int l = lane; l < L; l += 32) {
            bool inW = false;
            for (int i = 0; i < m; ++i)
                inW |= (S.W[i] == l);
            if (inW)
                continue;
            float ux = 0.f, uy = 0.f;
            for (int n = 0; n < N; ++n) {
                const float ar = A_re[n * lda + l], ai = A_im[n * lda + l];
                const float2 rv = S.rf[n];
                ux = fmaf(ar, rv.x, fmaf(ai, rv.y, ux));
                uy = fmaf(ar, rv.y, fmaf(-ai, rv.x, uy));
            }
            if (2.f * sqrtf(ux * ux + uy * uy) <= near)
                continue;
            double vx = 0.0, vy = 0.0;
            for (int n = 0; n < N; ++n) {
                const double2 av = A64[(size_t)n * L + l], rv = S.rr[n];
                vx += av.x * rv.x + av.y * rv.y;
                vy += av.x * rv.y - av.y * rv.x;
            }
            const double u = 2.0 * sqrt(vx * vx + vy * vy);
            if (u > lam * (1.0 + 1e-9) && u > worst) {
                worst = u;
                worst_l = l;
            }
        }
        // violators join W, largest first, at most 4 per round
        int added = 0;
        for (;;) {
            double bw = worst;
            int bl = worst_l;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const double ow = __shfl_xor_sync(0xffffffffu, bw, off);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
                if (ow > bw || (ow == bw && ol >= 0 && (bl < 0 || ol < bl))) {
                    bw = ow;
                    bl = ol;
                }
            }
            if (bl < 0)
                break;
            if (m + added >= smax) {
                noroom = true;
                break;
            }
            if (lane == 0) {
                S.W[m + added] = bl;
                S.z[m + added] = make_double2(0.0, 0.0);
            }
            ++added;
            if (worst_l == bl) {
                worst = 0.0;
                worst_l = -1;
            }
            __syncwarp();
            if (added >= 4)
                break;
        }
        if (added == 0) {
            certified = !noroom;
            break;
        }
        // keep W ascending (insertion sort, lane 0)
        if (lane == 0) {
            S.m = m + added;
            for (int i = 1; i < S.m; ++i) {
                const int w = S.W[i];
                const double2 zz = S.z[i];
                int j = i - 1;
                while (j >= 0 && S.W[j] > w) {
                    S.W[j + 1] = S.W[j];
                    S.z[j + 1] = S.z[j];
                    --j;
                }
                S.W[j + 1] = w;
                S.z[j + 1] = zz;
            }
        }
        __syncwarp();
        if (noroom)
            break;
    }

    float2 *xo = a.x_out + (size_t)p * L;
    if (certified) {
        const int m = S.m;
        // x = z on W (zeros of z stay zero), 0 elsewhere
        for (int l = lane; l < L; l += 32) {
            float2 v = make_float2(0.f, 0.f);
            for (int i = 0; i < m; ++i)
                if (S.W[i] == l)
                    v = make_float2((float)S.z[i].x, (float)S.z[i].y);
            xo[l] = v;
        }
        int ns = 0;
        for (int i = 0; i < m; ++i) {
            const bool nz = (S.z[i].x != 0.0 || S.z[i].y != 0.0);
            if (a.support && lane == 0 && nz)
                a.support[(size_t)p * smax + ns] = S.W[i];
            ns += nz;
        }
        if (a.support)
            for (int i = ns + lane; i < smax; i += 32)
                a.support[(size_t)p * smax + i] = -1;
        if (lane == 0) {
            int st = (status & ~BPDN_PX_ZERO_SOLUTION) | BPDN_PX_CERTIFIED;
            if (ns == 0)
                st |= BPDN_PX_ZERO_SOLUTION;
            a.status[p] = st;
            if (a.nsupp)
                a.nsupp[p] = ns;
        }
    } else {
        if (xo != xin)
            for (int l = lane; l < L; l += 32)
                xo[l] = xin[l];
        if (a.support) {
            // the support of x_in (ascending, first s_max entries), -1 padded
            int cnt = 0;
            for (int l0 = 0; l0 < L; l0 += 32) {
                const int l = l0 + lane;
                const float2 v = (l < L) ? xin[l] : make_float2(0.f, 0.f);
                const bool nz = (v.x != 0.f || v.y != 0.f);
                const unsigned bal = __ballot_sync(0xffffffffu, nz);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (nz && pos < smax)
                    a.support[(size_t)p * smax + pos] = l;
                cnt += __popc(bal);
            }
            for (int i = cnt + lane; i < smax; i += 32)
                a.support[(size_t)p * smax + i] = -1;
        }
        if (lane == 0) {
            a.status[p] = status | ((truncated || noroom) ? BPDN_PX_SUPPORT_OVERFLOW : BPDN_PX_KKT_FAIL);
            if (a.nsupp)
                a.nsupp[p] = nnz;
        }
    }
}

}  // namespace

cudaError_t launch_refit(const OpHandle &op, const RefitLaunch &a, cudaStream_t s)
{
    if (a.P <= 0)
        return cudaSuccess;
    const size_t smem = WARPS * sizeof(WarpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_refit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long blocks = (a.P + WARPS - 1) / WARPS;
    k_refit<<<(unsigned)blocks, WARPS * 32, smem, s>>>(op.A64, op.h, op.A_re, op.A_im, op.N, op.L,
                                                       op.lda, a);
    return cudaGetLastError();
}

}  // namespace bpdn
