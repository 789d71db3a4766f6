// Support extraction and FP64 refit (the refinement after Algorithm 1; SL1MMER
// step (3), Sec. III-A), one warp per pixel.
//
//   1. W = {l : x_in[l] != 0}, ascending (warp ballots over the grid); the s_max
//      largest moduli when x_in has more nonzeros.
//   2. The exact minimiser of Eq. 6 restricted to W,
//          min_z  z^H G z - 2 Re(c^H z) + lambda sum_i |z_i|,   G = A_W^H A_W, c = A_W^H g
//      (G from the Toeplitz generator h, c from the FP64 operator).  A solve is
//      coordinate sweeps (exact one-coordinate minimisations, which switch
//      coordinates on and off) alternating with Newton steps on the nonzero
//      coordinates; the Newton system is the Hessian in real coordinates,
//      2 [[Re G, -Im G],[Im G, Re G]] + lambda/|z_i| (I - u_i u_i^T).  A step is kept
//      where the objective is smooth (no modulus falls below a tenth of its value
//      along it); a coordinate that a full step carries through zero is set to zero
//      and the step recomputed.  If that does not converge, damped Newton on the
//      smoothed objective (|z| -> sqrt(|z|^2 + eps^2), strictly convex) for a
//      decreasing eps finds the support first.
//      Precision: the support is found in FP32 (residual <= 3e-6 lambda); the
//      answer is then finished and checked in FP64 (residual <= 1e-12 lambda) by plain
//      Newton steps, then by the sweep/Newton solve if those stall, falling back to an
//      all-FP64 solve when the FP32 support was wrong.  The
//      Newton systems are factored in FP32 in both phases: each step is then an
//      inexact Newton step (relative error about cond * 6e-8), while the objective,
//      the residual that decides convergence and the line search stay in the
//      phase's precision, so the FP64 answer is still checked in FP64.
//   The helpers stay out of line: inlined into every call site of both precisions
//   the kernel's code no longer fits the instruction cache.  This file is compiled
//   with approximate FP32 division and square root (and FP32 denormals flushed):
//   that touches only the FP32 support search and the FP32 screen of the
//   certificate, whose answers the FP64 phase and the FP64 recheck decide.
//   3. Coordinates of W that came out zero leave W.  Certificate over the grid:
//      |2 a_l^H (A_W z - g)| <= lambda for l not in W (FP32 products; grid points
//      within 1e-4 of the bound recomputed in FP64 against 1e-9).  Violators join W,
//      largest first, and step 2 repeats (at most `rounds` rounds).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

// working-set capacities: the fast path holds 16 grid points (2|W| <= 32 real unknowns, one
// per lane); the wide pass, for the pixels the fast path leaves uncertified, holds 32
// (2|W| <= 64, two unknowns per lane)
constexpr int KWF = 16;
constexpr int KWW = 32;
static_assert(KWW == kRefitMax, "the wide pass covers the library's largest s_max");
constexpr int kFastRounds32 = 15;
// FP32 phase tolerance, near FP32 resolution: every FP32 step saved here costs ~5x in FP64
constexpr float kTol32 = 3e-6f;
constexpr int kFastRounds64 = 8;
constexpr int kFallbackRounds = 20;

template <typename T>
struct C2 {
    T x, y;
};
template <typename T>
__device__ __forceinline__ C2<T> mk(T x, T y)
{
    C2<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b)
{
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ T cabs2(C2<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T>
__device__ __forceinline__ bool cnz(C2<T> a) { return a.x != T(0) || a.y != T(0); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Working storage of one restricted solve in precision T.
template <typename T, int KW>
struct Solve {
    C2<T> G[KW][KW];
    float J[2 * KW][2 * KW + 1];  // Newton system in FP32, right-hand side in column n2
    float inv[2 * KW];            // reciprocal pivots
    C2<T> z[KW], c[KW], zt[KW], dz[KW], gam[KW];
    T q[KW], u0[KW], u1[KW];  // per variable: lambda / (smoothed) modulus and unit vector
    int T_[KW];
};

// Everything one pixel (one warp) keeps in shared memory.  The FP32 and FP64
// solves never run at the same time and share storage.
template <int KW>
struct PixelSmem {
    union {
        Solve<double, KW> s64;
        Solve<float, KW> s32;
    };
    double2 *g;   // [N] g in FP64       (these three follow the struct, sized by N)
    double2 *rr;  // [N] A_W z - g (FP64)
    float2 *rf;   // [N] its FP32 copy
    double2 zkeep[KW];  // z between the precisions (FP64)
    double2 c64[KW];    // c = A_W^H g (FP64) of the current W
    int W[KW];
    int m;
};

// shared memory of one pixel: the struct, then g, rr (FP64) and rf (FP32) of length N
template <int KW>
__host__ __device__ inline size_t pixel_smem_bytes(int N)
{
    const size_t b = sizeof(PixelSmem<KW>) + (size_t)N * (sizeof(double2) * 2 + sizeof(float2));
    return (b + 15) & ~(size_t)15;
}

constexpr int WARPS = 1;  // pixels (warps) per block

// G_ij = h(l_i - l_j), c_i = a_{l_i}^H g in precision T
// c_i = a_{l_i}^H g in FP64 for the current W (lane i), into P.c64
template <int KW>
__device__ __noinline__ void load_c(PixelSmem<KW> &P, const double2 *__restrict__ A64, int N, int L, int lane)
{
    if (lane < P.m) {
        const int l = P.W[lane];
        double ax = 0.0, ay = 0.0;
        for (int n = 0; n < N; ++n) {
            const double2 av = A64[(size_t)n * L + l], gv = P.g[n];
            ax += av.x * gv.x + av.y * gv.y;
            ay += av.x * gv.y - av.y * gv.x;
        }
        P.c64[lane] = make_double2(ax, ay);
    }
    __syncwarp();
}

// G_ij = h(l_i - l_j) from the Toeplitz generator, or (no generator: a multi-component
// grid) sum_n conj(A_{n l_i}) A_{n l_j} from the FP64 operator
template <typename T, int KW>
__device__ __noinline__ void load_Gc(Solve<T, KW> &S, const PixelSmem<KW> &P, const double2 *__restrict__ A64,
                                     const double2 *__restrict__ h, int N, int L, int lane)
{
    const int m = P.m;
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - (e / m) * m;
        double2 v;
        if (h) {
            v = h[P.W[i] - P.W[j] + L - 1];
        } else {
            v = make_double2(0.0, 0.0);
            for (int n = 0; n < N; ++n) {
                const double2 a = A64[(size_t)n * L + P.W[i]], b = A64[(size_t)n * L + P.W[j]];
                v.x += a.x * b.x + a.y * b.y;
                v.y += a.x * b.y - a.y * b.x;
            }
        }
        S.G[i][j] = mk<T>((T)v.x, (T)v.y);
    }
    if (lane < m)
        S.c[lane] = mk<T>((T)P.c64[lane].x, (T)P.c64[lane].y);
    __syncwarp();
}

// (G z)_i
template <typename T, int KW>
__device__ __forceinline__ C2<T> gz_row(const Solve<T, KW> &S, int i, int m, const C2<T> *z)
{
    C2<T> acc = mk<T>(T(0), T(0));
    for (int j = 0; j < m; ++j)
        acc = cadd(acc, cmul(S.G[i][j], z[j]));
    return acc;
}

// objective over W (|z| smoothed by eps; eps = 0 is exact), without the constant ||g||^2
template <typename T, int KW>
__device__ __noinline__ T objective(const Solve<T, KW> &S, int m, const C2<T> *z, T lam, T eps, int lane)
{
    T v = T(0);
    if (lane < m) {
        const C2<T> gz = gz_row(S, lane, m, z);
        const C2<T> zi = z[lane];
        v = (zi.x * gz.x + zi.y * gz.y) - T(2) * (S.c[lane].x * zi.x + S.c[lane].y * zi.y) +
            lam * sqrt(cabs2(zi) + eps * eps);
    }
    return warp_sum(v);
}

// gam = 2 (G z - c); returns the optimality residual
//   max( max_{z_i != 0} |gam_i + lam u_i| / lam,  max_{z_i = 0} (|gam_i| / lam - 1) )
template <typename T, int KW>
__device__ __noinline__ T optimality(Solve<T, KW> &S, int m, T lam, int lane)
{
    T res = T(0);
    if (lane < m) {
        const C2<T> gz = gz_row(S, lane, m, S.z);
        const C2<T> gm = mk<T>(T(2) * (gz.x - S.c[lane].x), T(2) * (gz.y - S.c[lane].y));
        S.gam[lane] = gm;
        const C2<T> zi = S.z[lane];
        const T a = sqrt(cabs2(zi));
        if (a > T(0)) {
            const T la = lam / a;
            const T ex = fma(la, zi.x, gm.x), ey = fma(la, zi.y, gm.y);
            res = sqrt(ex * ex + ey * ey) / lam;
        } else {
            res = sqrt(cabs2(gm)) / lam - T(1);
        }
    }
    res = warp_max(res);
    __syncwarp();
    return res;
}

// One sweep of exact coordinate minimisations:
//   z_i <- S_{lam/2}(c_i - sum_{j != i} G_ij z_j) / G_ii
template <typename T, int KW>
__device__ __noinline__ void cd_sweep(Solve<T, KW> &S, int m, T lam, int lane)
{
    for (int i = 0; i < m; ++i) {
        C2<T> t = mk<T>(T(0), T(0));
        if (lane < m && lane != i)
            t = cmul(S.G[i][lane], S.z[lane]);
        const T qx = S.c[i].x - warp_sum(t.x), qy = S.c[i].y - warp_sum(t.y);
        if (lane == 0) {
            const T a = sqrt(qx * qx + qy * qy);
            const T th = T(0.5) * lam;
            if (a > th) {
                const T sc = (T(1) - th / a) / S.G[i][i].x;
                S.z[i] = mk<T>(qx * sc, qy * sc);
            } else {
                S.z[i] = mk<T>(T(0), T(0));
            }
        }
        __syncwarp();
    }
}

// Solve J[0..n2) x = J[.][n2] (symmetric positive definite): elimination without
// pivoting with lanes over columns (one reciprocal per pivot), then column-wise
// back substitution with lanes over rows.  Lane i returns x_i.  `ok` is false on
// a non-positive pivot.
template <typename T, int KW>
__device__ __noinline__ T solve_spd(Solve<T, KW> &S, int n2, int lane, bool &ok)
{
    const int rc = (n2 < 32) ? n2 : 0;  // lane that owns the right-hand-side column
    ok = true;
    for (int k = 0; k < n2; ++k) {
        __syncwarp();
        const float piv = S.J[k][k];
        if (!(piv > 0.f)) {
            ok = false;
            return T(0);
        }
        const float ip = 1.f / piv;
        const float pk = (lane > k && lane < n2) ? S.J[k][lane] : 0.f;
        const float pr = (lane == rc) ? S.J[k][n2] : 0.f;
        if (lane == 0)
            S.inv[k] = ip;
        // four rows at a time, every load of a block before its stores
        const int col = (lane > k && lane < n2) ? lane : ((lane == rc) ? n2 : -1);
        const float pc = (lane == rc) ? pr : pk;
        for (int i = k + 1; i < n2; i += 4) {
            float f[4], v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = (i + u < n2);
                f[u] = in ? S.J[i + u][k] * ip : 0.f;
                v[u] = (in && col >= 0) ? S.J[i + u][col] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u < n2 && col >= 0)
                    S.J[i + u][col] = v[u] - f[u] * pc;
        }
    }
    __syncwarp();
    float b = (lane < n2) ? S.J[lane][n2] : 0.f;
    for (int k = n2 - 1; k >= 0; --k) {
        const float xk = __shfl_sync(0xffffffffu, b, k) * S.inv[k];
        if (lane < k)
            b -= S.J[lane][k] * xk;
        else if (lane == k)
            b = xk;
    }
    return (T)b;
}

// The same solve for systems of up to 64 unknowns (the wide pass): lane i owns
// columns i and i + 32 during the elimination, and the right-hand side, stored in
// column n2, is owned like any other column (by lane n2 mod 32); the back substitution
// keeps rows i and i + 32 in lane i.  Returns x_i in x0 and x_{i+32} in x1.
template <typename T, int KW>
__device__ __noinline__ void solve_spd_wide(Solve<T, KW> &S, int n2, int lane, bool &ok, T &x0, T &x1)
{
    static_assert(2 * KW <= 64, "two rows per lane");
    ok = true;
    x0 = x1 = T(0);
    for (int k = 0; k < n2; ++k) {
        __syncwarp();
        const float piv = S.J[k][k];
        if (!(piv > 0.f)) {
            ok = false;
            return;
        }
        const float ip = 1.f / piv;
        // this lane's columns still being eliminated (the right-hand side, column n2, included)
        int col[3];
        float pc[3];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
            const int c = lane + 32 * h;
            col[h] = (c > k && c <= n2) ? c : -1;
            pc[h] = (col[h] >= 0) ? S.J[k][c] : 0.f;
        }
        if (lane == 0)
            S.inv[k] = ip;
        for (int i = k + 1; i < n2; i += 4) {
            float f[4], v[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = (i + u < n2);
                f[u] = in ? S.J[i + u][k] * ip : 0.f;
#pragma unroll
                for (int h = 0; h < 3; ++h)
                    v[u][h] = (in && col[h] >= 0) ? S.J[i + u][col[h]] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int h = 0; h < 3; ++h)
                    if (i + u < n2 && col[h] >= 0)
                        S.J[i + u][col[h]] = v[u][h] - f[u] * pc[h];
        }
    }
    __syncwarp();
    float b0 = (lane < n2) ? S.J[lane][n2] : 0.f;
    float b1 = (lane + 32 < n2) ? S.J[lane + 32][n2] : 0.f;
    for (int k = n2 - 1; k >= 0; --k) {
        const float src = (k >= 32) ? b1 : b0;  // k is the same in every lane
        const float xk = __shfl_sync(0xffffffffu, src, k & 31) * S.inv[k];
        if (lane < k)
            b0 -= S.J[lane][k] * xk;
        else if (lane == k)
            b0 = xk;
        if (lane + 32 < k)
            b1 -= S.J[lane + 32][k] * xk;
        else if (lane + 32 == k)
            b1 = xk;
    }
    x0 = (T)b0;
    x1 = (T)b1;
}

// Newton direction for the objective restricted to the nonzero coordinates of z
// (eps = 0) or for the smoothed objective over all of W (eps > 0).  Writes S.dz
// (zero off the variables) and returns the directional derivative (negative for
// a descent direction), or +1 when the system could not be solved.
template <typename T, int KW>
__device__ __noinline__ T newton_dir(Solve<T, KW> &S, int m, const C2<T> *z, T lam, T eps, int lane,
                                     bool have_gam = false)
{
    const bool use = (lane < m) && (eps > T(0) || cnz(z[lane]));
    const unsigned bal = __ballot_sync(0xffffffffu, use);
    const int nt = __popc(bal), n2 = 2 * nt;
    if (use)
        S.T_[__popc(bal & ((1u << lane) - 1u))] = lane;
    if (lane < m && !have_gam) {
        const C2<T> gz = gz_row(S, lane, m, z);
        S.gam[lane] = mk<T>(T(2) * (gz.x - S.c[lane].x), T(2) * (gz.y - S.c[lane].y));
    }
    __syncwarp();
    if (nt == 0)
        return T(1);
    if (lane < nt) {
        const C2<T> zi = z[S.T_[lane]];
        const T q = sqrt(cabs2(zi) + eps * eps);
        const T iq = T(1) / q;
        S.q[lane] = lam * iq;
        S.u0[lane] = zi.x * iq;
        S.u1[lane] = zi.y * iq;
    }
    __syncwarp();
    if constexpr (KW <= 16) {
    // lane 2b + cb fills column 2b + cb, two rows (re, im of variable a) per step
    if (lane < n2) {
        const int b = lane >> 1, cb = lane & 1;
        const int tb = S.T_[b];
        const T wc = cb ? S.u1[b] : S.u0[b];
#pragma unroll 4
        for (int a = 0; a < nt; ++a) {
            const C2<T> g = S.G[S.T_[a]][tb];
            T v0 = T(2) * (cb == 0 ? g.x : -g.y);
            T v1 = T(2) * (cb == 0 ? g.y : g.x);
            if (a == b) {
                const T sc = S.q[a];
                v0 += sc * ((cb == 0 ? T(1) : T(0)) - S.u0[a] * wc);
                v1 += sc * ((cb == 1 ? T(1) : T(0)) - S.u1[a] * wc);
            }
            S.J[2 * a][lane] = (float)v0;
            S.J[2 * a + 1][lane] = (float)v1;
        }
    }
    if (sizeof(T) == 4) {
        // FP32 phase: a Levenberg-Marquardt shift of 1e-7 of the largest diagonal entry
        // keeps the FP32 elimination positive definite when the support holds nearly
        // collinear columns (adjacent grid points); without it about a fifth of the
        // FP32 Newton directions failed.  The FP64 phase keeps the plain system for its
        // fast final convergence.
        const float dg = (lane < n2) ? S.J[lane][lane] : 0.f;
        const float mx = warp_max(dg);
        if (lane < n2)
            S.J[lane][lane] = dg + 1e-7f * mx;
        __syncwarp();
    }
    T gcomp = T(0);
    if (lane < n2) {
        const int a = lane >> 1;
        const int ia = S.T_[a];
        const T w = (lane & 1) ? S.u1[a] : S.u0[a];
        gcomp = ((lane & 1) ? S.gam[ia].y : S.gam[ia].x) + lam * w;
        S.J[lane][n2] = (float)(-gcomp);
    }
    bool ok;
    const T d = solve_spd(S, n2, lane, ok);
    if (!ok)
        return T(1);
    if (lane < m)
        S.dz[lane] = mk<T>(T(0), T(0));
    __syncwarp();
    // gather (re, im) pairs: lane a takes rows 2a and 2a+1
    const T dre = __shfl_sync(0xffffffffu, d, (2 * lane) & 31);
    const T dim = __shfl_sync(0xffffffffu, d, (2 * lane + 1) & 31);
    if (lane < nt)
        S.dz[S.T_[lane]] = mk<T>(dre, dim);
    __syncwarp();
    return warp_sum((lane < n2) ? gcomp * d : T(0));
    } else {
    // lane i fills columns i and i + 32 (2b + cb: re/im part cb of variable b)
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < n2) {
            const int b = c >> 1, cb = c & 1;
            const int tb = S.T_[b];
            const T wc = cb ? S.u1[b] : S.u0[b];
            for (int a = 0; a < nt; ++a) {
                const C2<T> g = S.G[S.T_[a]][tb];
                T v0 = T(2) * (cb == 0 ? g.x : -g.y);
                T v1 = T(2) * (cb == 0 ? g.y : g.x);
                if (a == b) {
                    const T sc = S.q[a];
                    v0 += sc * ((cb == 0 ? T(1) : T(0)) - S.u0[a] * wc);
                    v1 += sc * ((cb == 1 ? T(1) : T(0)) - S.u1[a] * wc);
                }
                S.J[2 * a][c] = (float)v0;
                S.J[2 * a + 1][c] = (float)v1;
            }
        }
    }
    __syncwarp();
    if (sizeof(T) == 4) {
        // the Levenberg-Marquardt shift of the FP32 phase, as in the fast path
        const float dg0 = (lane < n2) ? S.J[lane][lane] : 0.f;
        const float dg1 = (lane + 32 < n2) ? S.J[lane + 32][lane + 32] : 0.f;
        const float mx = warp_max(fmaxf(dg0, dg1));
        if (lane < n2)
            S.J[lane][lane] = dg0 + 1e-7f * mx;
        if (lane + 32 < n2)
            S.J[lane + 32][lane + 32] = dg1 + 1e-7f * mx;
    }
    T gc[2] = {T(0), T(0)};
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < n2) {
            const int a = c >> 1;
            const int ia = S.T_[a];
            const T w = (c & 1) ? S.u1[a] : S.u0[a];
            gc[h] = ((c & 1) ? S.gam[ia].y : S.gam[ia].x) + lam * w;
            S.J[c][n2] = (float)(-gc[h]);
        }
    }
    bool ok;
    T d0, d1;
    solve_spd_wide(S, n2, lane, ok, d0, d1);
    if (!ok)
        return T(1);
    if (lane < m)
        S.dz[lane] = mk<T>(T(0), T(0));
    __syncwarp();
    // variable a takes rows 2a and 2a + 1, held by lane 2a mod 32 in register (2a) / 32
    const int r0 = (2 * lane) & 31, r1 = (2 * lane + 1) & 31;
    const T e0 = __shfl_sync(0xffffffffu, d0, r0), f0 = __shfl_sync(0xffffffffu, d1, r0);
    const T e1 = __shfl_sync(0xffffffffu, d0, r1), f1 = __shfl_sync(0xffffffffu, d1, r1);
    const bool hi = (2 * lane) >= 32;
    if (lane < nt)
        S.dz[S.T_[lane]] = mk<T>(hi ? f0 : e0, hi ? f1 : e1);
    __syncwarp();
    T sl = T(0);
    if (lane < n2)
        sl += gc[0] * d0;
    if (lane + 32 < n2)
        sl += gc[1] * d1;
    return warp_sum(sl);
    }
}

// does the segment z_i + s dz_i, s in [0, t], come within a tenth of |z_i| of zero?
template <typename T>
__device__ __forceinline__ bool passes_zero(C2<T> zi, C2<T> d, T t)
{
    const T dd = cabs2(d);
    if (!(dd > T(0)) || !cnz(zi))
        return false;
    // the closest point to zero along the line is at s* = zd / dd
    const T zz = cabs2(zi), zd = -(zi.x * d.x + zi.y * d.y);
    if (!(zd > T(0)))
        return false;  // |z_i + s dz_i| grows for s > 0
    if (zd <= t * dd)  // s* in (0, t]: the minimum modulus^2 is zz - zd^2 / dd
        return T(0.99) * zz * dd < zd * zd;
    const C2<T> p = mk<T>(zi.x + t * d.x, zi.y + t * d.y);
    return cabs2(p) < T(0.01) * zz;
}

// coordinate sweeps alternating with Newton steps (see the file header)
template <typename T, int KW>
__device__ __noinline__ bool fast_path(Solve<T, KW> &S, int m, T lam, int lane, int max_outer, T tol)
{
    for (int outer = 0; outer < max_outer; ++outer) {
        // the FP64 phase starts from the FP32 answer, whose support is settled: Newton first.
        // The FP32 phase opens with three sweeps: they zero most of the small spurious
        // coordinates of the iterate, which would otherwise block the Newton steps.
        if (sizeof(T) == 4 || outer > 0)
            for (int e = (sizeof(T) == 4 && outer == 0) ? 3 : 1; e > 0; --e)
                cd_sweep(S, m, lam, lane);
        const T res = optimality(S, m, lam, lane);
        if (res <= tol)
            return true;
        const T F0 = objective(S, m, S.z, lam, T(0), lane);
        T slope = newton_dir(S, m, S.z, lam, T(0), lane, true);  // optimality() left gam for z
        if (slope > T(0))
            continue;
        const bool blk = (lane < m) && passes_zero(S.z[lane], S.dz[lane], T(1));
        if (__any_sync(0xffffffffu, blk)) {
            // the direction from z, kept for the line search if the step with the
            // blocked coordinates set to zero does not pay
            const C2<T> dz0 = (lane < m) ? S.dz[lane] : mk<T>(T(0), T(0));
            const T slope0 = slope;
            const C2<T> zk = (lane < m) ? S.z[lane] : mk<T>(T(0), T(0));
            if (lane < m)
                S.zt[lane] = blk ? mk<T>(T(0), T(0)) : zk;
            __syncwarp();
            const T sl2 = newton_dir(S, m, S.zt, lam, T(0), lane);
            bool ok2 = sl2 < T(0);
            if (ok2) {
                const bool blk2 = (lane < m) && passes_zero(S.zt[lane], S.dz[lane], T(1));
                ok2 = !__any_sync(0xffffffffu, blk2);
            }
            if (ok2) {
                if (lane < m)
                    S.zt[lane] = cadd(S.zt[lane], S.dz[lane]);
                __syncwarp();
                if (objective(S, m, S.zt, lam, T(0), lane) < F0) {
                    if (lane < m)
                        S.z[lane] = S.zt[lane];
                    __syncwarp();
                    if (optimality(S, m, lam, lane) <= tol)
                        return true;
                    continue;
                }
            }
            if (lane < m)
                S.dz[lane] = dz0;
            __syncwarp();
            slope = slope0;
        }
        T t = T(1);
        for (int hh = 0; hh < 60; ++hh) {
            const bool bad = (lane < m) && passes_zero(S.z[lane], S.dz[lane], t);
            if (!__any_sync(0xffffffffu, bad))
                break;
            t *= T(0.5);
        }
        const C2<T> keep = (lane < m) ? S.z[lane] : mk<T>(T(0), T(0));
        bool accepted = false;
        for (int hh = 0; hh < 50 && t > T(1e-14); ++hh, t *= T(0.5)) {
            if (lane < m)
                S.zt[lane] = mk<T>(keep.x + t * S.dz[lane].x, keep.y + t * S.dz[lane].y);
            __syncwarp();
            if (objective(S, m, S.zt, lam, T(0), lane) <= F0 + T(1e-4) * t * slope) {
                accepted = true;
                break;
            }
            if (hh == 0) {
                // near the minimiser the objective no longer resolves the decrease:
                // take the step if it halves the optimality residual instead
                if (lane < m)
                    S.z[lane] = S.zt[lane];
                __syncwarp();
                const T r1 = optimality(S, m, lam, lane);
                if (lane < m)
                    S.z[lane] = keep;
                __syncwarp();
                if (r1 < T(0.5) * res) {
                    accepted = true;
                    break;
                }
            }
        }
        if (accepted && lane < m)
            S.z[lane] = S.zt[lane];
        __syncwarp();
        if (optimality(S, m, lam, lane) <= tol)
            return true;
    }
    return false;
}

// damped Newton on the smoothed objective for eps = e0, e0/10, ..., e1 (times the
// scale of z), at most maxit steps per level; then coordinates below 1e-6 of the
// scale are set to zero
template <typename T, int KW>
__device__ __noinline__ void continuation(Solve<T, KW> &S, int m, T lam, int lane, T e0, T e1, int maxit)
{
    T sc = warp_max((lane < m) ? sqrt(cabs2(S.z[lane])) : T(0));
    sc = fmax(sc, T(1e-3));
    for (T eps = e0 * sc; eps >= T(0.999) * e1 * sc; eps *= T(0.1)) {
        for (int it = 0; it < maxit; ++it) {
            const T slope = newton_dir(S, m, S.z, lam, eps, lane);
            if (!(slope < T(0)) || -slope <= T(1e-28) * fmax(T(1), sc * sc))
                break;
            const T F0 = objective(S, m, S.z, lam, eps, lane);
            const C2<T> keep = (lane < m) ? S.z[lane] : mk<T>(T(0), T(0));
            T t = T(1);
            for (int hh = 0; hh < 40; ++hh, t *= T(0.5)) {
                if (lane < m)
                    S.zt[lane] = mk<T>(keep.x + t * S.dz[lane].x, keep.y + t * S.dz[lane].y);
                __syncwarp();
                if (objective(S, m, S.zt, lam, eps, lane) <= F0 + T(1e-4) * t * slope)
                    break;
            }
            if (lane < m)
                S.z[lane] = S.zt[lane];
            __syncwarp();
            if (-slope < T(1e-12) * fmax(T(1), fabs(F0)))
                break;
        }
    }
    if (lane < m && sqrt(cabs2(S.z[lane])) <= T(1e-6) * sc)
        S.z[lane] = mk<T>(T(0), T(0));
    __syncwarp();
}

// Newton refinement from a start whose support is settled (the FP32 answer): full
// Newton steps on the nonzero coordinates while no modulus passes near zero and the
// residual at least halves.  true when the residual reaches tol; false hands over to
// fast_path.  Far less code and FP64 work than fast_path's sweeps and line searches.
template <typename T, int KW>
__device__ __noinline__ bool newton_refine(Solve<T, KW> &S, int m, T lam, int lane, int maxit, T tol)
{
    T prev = T(1e300);
    for (int it = 0; it < maxit; ++it) {
        const T res = optimality(S, m, lam, lane);
        if (res <= tol)
            return true;
        if (!(res < T(0.5) * prev))
            return false;
        prev = res;
        const T slope = newton_dir(S, m, S.z, lam, T(0), lane, true);  // gam from optimality()
        if (slope > T(0))
            return false;
        const bool bad = (lane < m) && passes_zero(S.z[lane], S.dz[lane], T(1));
        if (__any_sync(0xffffffffu, bad))
            return false;
        if (lane < m)
            S.z[lane] = cadd(S.z[lane], S.dz[lane]);
        __syncwarp();
    }
    return optimality(S, m, lam, lane) <= tol;
}

// Step 2 on the current W from the start values in P.zkeep: FP32 support search,
// FP64 finish.  The FP64 answer is left in P.zkeep.  Returns true on convergence.
template <int KW>
__device__ __noinline__ void fp32_phase(PixelSmem<KW> &P, const double2 *A64, const double2 *h, int N, int L,
                                        double lam, int lane)
{
    const int m = P.m;
    const double2 start = (lane < m) ? P.zkeep[lane] : make_double2(0.0, 0.0);
    {
        Solve<float, KW> &S = P.s32;
        load_Gc(S, P, A64, h, N, L, lane);
        if (lane < m)
            S.z[lane] = mk<float>((float)start.x, (float)start.y);
        __syncwarp();
        const float lf = (float)lam;
        if (!fast_path(S, m, lf, lane, kFastRounds32, kTol32)) {
            // four damped steps per smoothing level: the FP32 phase only has to land in
            // the support's basin, and the FP64 phase finishes
            continuation(S, m, lf, lane, 1e-2f, 1e-6f, 4);
            fast_path(S, m, lf, lane, kFastRounds32, kTol32);
        }
        if (lane < m)
            P.zkeep[lane] = make_double2((double)S.z[lane].x, (double)S.z[lane].y);
        __syncwarp();
    }
}

template <int KW>
__device__ __noinline__ bool fp64_phase(PixelSmem<KW> &P, const double2 *A64, const double2 *h, int N, int L,
                                        double lam, int lane, double2 start)
{
    const int m = P.m;
    Solve<double, KW> &S = P.s64;
    load_Gc(S, P, A64, h, N, L, lane);
    if (lane < m)
        S.z[lane] = mk<double>(P.zkeep[lane].x, P.zkeep[lane].y);
    __syncwarp();
    bool ok = newton_refine(S, m, lam, lane, 6, 1e-12);
    if (!ok) {
        if (lane < m)
            S.z[lane] = mk<double>(P.zkeep[lane].x, P.zkeep[lane].y);
        __syncwarp();
        ok = fast_path(S, m, lam, lane, kFastRounds64, 1e-12);
    }
    if (!ok) {
        // the FP32 support was wrong: solve in FP64 from the start values
        if (lane < m)
            S.z[lane] = mk<double>(start.x, start.y);
        __syncwarp();
        continuation(S, m, lam, lane, 1e-2, 1e-8, 8);
        ok = fast_path(S, m, lam, lane, kFallbackRounds, 1e-12);
    }
    if (lane < m)
        P.zkeep[lane] = make_double2(S.z[lane].x, S.z[lane].y);
    __syncwarp();
    return ok;
}

template <int KW>
__device__ __noinline__ bool restricted_minimiser(PixelSmem<KW> &P, const double2 *A64, const double2 *h, int N,
                                     int L, double lam, int lane)
{
    const int m = P.m;
    if (m == 0)
        return true;
    const double2 start = (lane < m) ? P.zkeep[lane] : make_double2(0.0, 0.0);
    load_c(P, A64, N, L, lane);
    fp32_phase(P, A64, h, N, L, lam, lane);
    return fp64_phase(P, A64, h, N, L, lam, lane, start);
}

template <int KW>
__device__ void sort_W(PixelSmem<KW> &P)
{
    for (int i = 1; i < P.m; ++i) {
        const int w = P.W[i];
        const double2 zz = P.zkeep[i];
        int j = i - 1;
        while (j >= 0 && P.W[j] > w) {
            P.W[j + 1] = P.W[j];
            P.zkeep[j + 1] = P.zkeep[j];
            --j;
        }
        P.W[j + 1] = w;
        P.zkeep[j + 1] = zz;
    }
}

// Between the launches of the split refit, per pixel: the working set, its FP32 answer of
// round 0 and the support count of x_in (launch 1 -> 2); whether the pixel needs further
// rounds, with its working set and FP64 state (launch 2 -> 3).
struct SplitScratch {
    int *m;       // [P]
    int *meta;    // [P]: nnz | truncated << 30
    int *W;       // [P][16]
    float2 *z;    // [P][16]
    int *pend;    // [P]: 1 when launch 3 continues the pixel
    double2 *zs;  // [P][16]
    unsigned long long *queue;  // [2]: work counters of the scan launches (phases 3 and 4)
};

// Phases of the refit of one pixel (one warp):
//   PH 0  the whole refit (fast path, working set <= 16);
//   PH 1  working set and the FP32 support search of round 0, into the scratch;
//   PH 2  from the scratch, the FP64 finish and the certificate of round 0; a pixel the
//         certificate sends to another round is handed on, the others get their outputs;
//   PH 3  the further rounds (both precisions) of the handed-on pixels;
//   PH 4  the wide pass: the whole refit again with a working set of up to 32 grid points,
//         for a pixel the fast path left with SUPPORT_OVERFLOW or KKT_FAIL (its output x,
//         which the fast path left equal to the iterate, is the input).
// Splitting keeps each launch's executed code small: one fused launch stalled on
// instruction fetch while the warps of an SM ran different phases.
template <int PH, int KW>
__device__ __forceinline__ void refit_pixel(PixelSmem<KW> &P, const long long p, const SplitScratch &sc,
                                            const double2 *__restrict__ A64, const double2 *__restrict__ h,
                                            const float *__restrict__ A_re, const float *__restrict__ A_im,
                                            const int N, const int L, const int lda, const RefitLaunch &a,
                                            const int lane)
{
    const int smax = a.s_max;                       // row length of the support output
    const int cap = smax < KW ? smax : KW;          // working-set capacity of this pass
    const float2 *xin = (PH == 4 ? a.x_out : a.x_in) + (size_t)p * L;
    const float2 *gp = a.g + (size_t)p * N;
    const double lam = (double)(a.lam_pp ? a.lam[p] : a.lam[0]);

    int nnz = 0;
    bool truncated = false;
    if constexpr (PH == 2 || PH == 3) {
        const int mm = sc.m[p];
        const int meta = sc.meta[p];
        nnz = meta & ((1 << 30) - 1);
        truncated = (meta >> 30) & 1;
        if (lane < mm) {
            P.W[lane] = sc.W[(size_t)p * 16 + lane];
            if constexpr (PH == 2) {
                const float2 zz = sc.z[(size_t)p * 16 + lane];
                P.zkeep[lane] = make_double2((double)zz.x, (double)zz.y);
            } else {
                P.zkeep[lane] = sc.zs[(size_t)p * 16 + lane];
            }
        }
        if (lane == 0)
            P.m = mm;
    } else {
    // 1. working set W
    for (int l0 = 0; l0 < L; l0 += 32) {
        const int l = l0 + lane;
        const float2 v = (l < L) ? xin[l] : make_float2(0.f, 0.f);
        nnz += __popc(__ballot_sync(0xffffffffu, v.x != 0.f || v.y != 0.f));
    }
    truncated = nnz > cap;
    if (!truncated) {
        int m = 0;
        for (int l0 = 0; l0 < L; l0 += 32) {
            const int l = l0 + lane;
            const float2 v = (l < L) ? xin[l] : make_float2(0.f, 0.f);
            const bool nz = (v.x != 0.f || v.y != 0.f);
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            if (nz)
                P.W[m + __popc(bal & ((1u << lane) - 1u))] = l;
            m += __popc(bal);
        }
        if (lane == 0)
            P.m = m;
    } else {
        // cap rounds of a warp arg-max over |x_l|^2 in the order (|x_l|^2 descending, l
        // ascending): round k takes the largest point after the one round k-1 took
        float prev_a2 = INFINITY;
        int prev_l = -1;
        for (int k = 0; k < cap; ++k) {
            float best = -1.f;
            int bl = -1;
            for (int l = lane; l < L; l += 32) {
                const float2 v = xin[l];
                const float a2 = v.x * v.x + v.y * v.y;
                if (a2 > prev_a2 || (a2 == prev_a2 && l <= prev_l))
                    continue;  // taken in an earlier round
                if (a2 > best) {
                    best = a2;
                    bl = l;
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
                break;  // cannot happen: more than cap grid points are nonzero
            prev_a2 = best;
            prev_l = bl;
            if (lane == 0)
                P.W[k] = bl;
        }
        __syncwarp();
        if (lane == 0) {
            P.m = cap;
            for (int i = 1; i < cap; ++i) {  // ascending
                const int w = P.W[i];
                int j = i - 1;
                while (j >= 0 && P.W[j] > w) {
                    P.W[j + 1] = P.W[j];
                    --j;
                }
                P.W[j + 1] = w;
            }
        }
    }
    }  // working set
    int status = a.status[p];
    if constexpr (PH == 4)
        status &= ~(BPDN_PX_SUPPORT_OVERFLOW | BPDN_PX_KKT_FAIL);  // this pass decides them anew
    for (int n = lane; n < N; n += 32) {
        const float2 gg = gp[n];
        P.g[n] = make_double2((double)gg.x, (double)gg.y);
    }
    __syncwarp();
    if constexpr (PH == 0 || PH == 1 || PH == 4) {
        if (lane < P.m) {
            const float2 v = xin[P.W[lane]];
            P.zkeep[lane] = make_double2((double)v.x, (double)v.y);
        }
        __syncwarp();
    }
    if constexpr (PH == 1) {
        // FP32 support search of round 0, stored for the second launch
        const int mm = P.m;
        if (mm > 0) {
            load_c(P, A64, N, L, lane);
            fp32_phase(P, A64, h, N, L, lam, lane);
        }
        if (lane < mm) {
            sc.W[(size_t)p * 16 + lane] = P.W[lane];
            sc.z[(size_t)p * 16 + lane] = make_float2((float)P.zkeep[lane].x, (float)P.zkeep[lane].y);
        }
        if (lane == 0) {
            sc.m[p] = mm;
            sc.meta[p] = nnz | (truncated ? (1 << 30) : 0);
        }
        return;
    }

    bool certified = false, noroom = false, more = false;
    bool have_z = false;  // P.zkeep holds a converged restricted minimiser over W
    // the wide pass gets four times the rounds: it only runs on the few pixels whose
    // working set the fast path could not settle
    const int round_first = (PH == 3) ? 1 : 0;
    const int round_last = (PH == 2) ? 0 : ((PH == 4) ? 4 * a.rounds : a.rounds);
    for (int round = round_first; round <= round_last; ++round) {
        more = false;
        // 2. exact minimiser over W
        bool okr;
        if (PH == 2 && round == 0) {
            // the FP32 phase ran in the first launch: finish in FP64 from its answer
            const int mm = P.m;
            okr = true;
            if (mm > 0) {
                const float2 v = (lane < mm) ? xin[P.W[lane]] : make_float2(0.f, 0.f);
                load_c(P, A64, N, L, lane);
                okr = fp64_phase(P, A64, h, N, L, lam, lane, make_double2((double)v.x, (double)v.y));
            }
        } else {
            okr = restricted_minimiser(P, A64, h, N, L, lam, lane);
        }
        have_z = okr;
        if (!okr)
            break;
        // drop the coordinates the restricted minimiser set to zero: their dual
        // constraint holds (|2 (G z - c)_i| <= lambda), and the room they free lets the
        // certificate add violators when x_in had more than cap nonzeros
        if (lane == 0) {
            int k = 0;
            for (int i = 0; i < P.m; ++i)
                if (P.zkeep[i].x != 0.0 || P.zkeep[i].y != 0.0) {
                    P.W[k] = P.W[i];
                    P.zkeep[k] = P.zkeep[i];
                    ++k;
                }
            P.m = k;
        }
        __syncwarp();
        const int m = P.m;
        // residual A_W z - g in FP64 and its FP32 copy
        for (int n = lane; n < N; n += 32) {
            double2 acc = make_double2(-P.g[n].x, -P.g[n].y);
            for (int i = 0; i < m; ++i) {
                const double2 av = A64[(size_t)n * L + P.W[i]], zi = P.zkeep[i];
                acc.x += av.x * zi.x - av.y * zi.y;
                acc.y += av.x * zi.y + av.y * zi.x;
            }
            P.rr[n] = acc;
            P.rf[n] = make_float2((float)acc.x, (float)acc.y);
        }
        __syncwarp();
        // 3. certificate off W
        const float near = (float)lam * (1.0f - 1e-4f);
        double worst = 0.0;
        int worst_l = -1;
        for (int l = lane; l < L; l += 32) {
            float ux = 0.f, uy = 0.f;
            for (int n = 0; n < N; ++n) {
                const float ar = A_re[n * lda + l], ai = A_im[n * lda + l];
                const float2 rv = P.rf[n];
                ux = fmaf(ar, rv.x, fmaf(ai, rv.y, ux));
                uy = fmaf(ar, rv.y, fmaf(-ai, rv.x, uy));
            }
            if (2.f * sqrtf(ux * ux + uy * uy) <= near)
                continue;
            // the points of W sit at the threshold: they pass the screen, and skip the FP64
            // recheck here (only points past the screen pay for the scan over W)
            bool inW = false;
            for (int i = 0; i < m; ++i)
                inW = inW || (P.W[i] == l);
            if (inW)
                continue;
            double vx = 0.0, vy = 0.0;
            for (int n = 0; n < N; ++n) {
                const double2 av = A64[(size_t)n * L + l], rv = P.rr[n];
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
            if (m + added >= cap) {
                noroom = true;
                break;
            }
            if (lane == 0) {
                P.W[m + added] = bl;
                P.zkeep[m + added] = make_double2(0.0, 0.0);
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
        if (lane == 0) {
            P.m = m + added;
            sort_W(P);
        }
        __syncwarp();
        if (noroom)
            break;
        more = true;  // violators joined W: another round follows, if the limit allows one
    }
    if constexpr (PH == 2) {
        // hand the pixel on to the third launch when it needs a further round
        const int hand = (more && a.rounds >= 1) ? 1 : 0;
        if (hand) {
            const int mm = P.m;
            if (lane < mm) {
                sc.W[(size_t)p * 16 + lane] = P.W[lane];
                sc.zs[(size_t)p * 16 + lane] = P.zkeep[lane];
            }
            if (lane == 0)
                sc.m[p] = mm;
        }
        if (lane == 0)
            sc.pend[p] = hand;
        if (hand)
            return;
    }

    float2 *xo = a.x_out + (size_t)p * L;
    // A pixel that is not certified but whose last restricted solve converged returns that
    // restricted minimiser (at most cap nonzeros, the working set's violators at zero): a
    // sparse point that minimises Eq. 6 over its own support, from which a pass with a
    // larger working set (or another caller) continues; otherwise it keeps x_in.
    if (certified || have_z) {
        const int m = P.m;
        for (int l = lane; l < L; l += 32) {
            float2 v = make_float2(0.f, 0.f);
            for (int i = 0; i < m; ++i)
                if (P.W[i] == l)
                    v = make_float2((float)P.zkeep[i].x, (float)P.zkeep[i].y);
            xo[l] = v;
        }
        int ns = 0;
        for (int i = 0; i < m; ++i) {
            const bool nz = (P.zkeep[i].x != 0.0 || P.zkeep[i].y != 0.0);
            if (a.support && lane == 0 && nz)
                a.support[(size_t)p * smax + ns] = P.W[i];
            ns += nz;
        }
        if (a.support)
            for (int i = ns + lane; i < smax; i += 32)
                a.support[(size_t)p * smax + i] = -1;
        if (lane == 0) {
            int st = status & ~BPDN_PX_ZERO_SOLUTION;
            if (certified)
                st |= BPDN_PX_CERTIFIED;
            else
                st |= (truncated || noroom) ? BPDN_PX_SUPPORT_OVERFLOW : BPDN_PX_KKT_FAIL;
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

// set up one warp's shared memory: the struct, then g, rr and rf of length N
template <int KW>
__device__ __forceinline__ PixelSmem<KW> &pixel_smem(unsigned char *base, int N, int lane)
{
    PixelSmem<KW> &P = *(PixelSmem<KW> *)base;
    if (lane == 0) {
        P.g = (double2 *)(base + sizeof(PixelSmem<KW>));
        P.rr = P.g + N;
        P.rf = (float2 *)(P.rr + N);
    }
    __syncwarp();
    return P;
}

// one warp per block, one pixel per warp (phases 0, 1, 2: every pixel takes them)
template <int PH>
__global__ void __launch_bounds__(WARPS * 32) k_refit_t(SplitScratch sc, const double2 *__restrict__ A64,
                                                      const double2 *__restrict__ h,
                                                      const float *__restrict__ A_re,
                                                      const float *__restrict__ A_im, int N,
                                                      int L, int lda, RefitLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long p = (long long)blockIdx.x * WARPS + warp;
    if (p >= a.P)
        return;
    PixelSmem<KWF> &P = pixel_smem<KWF>(smem_raw + (size_t)warp * pixel_smem_bytes<KWF>(N), N, lane);
    refit_pixel<PH, KWF>(P, p, sc, A64, h, A_re, A_im, N, L, lda, a, lane);
}

// Persistent launches over the pixels that need them: each warp reads the flags of 32
// pixels at a time (a coalesced load) and works through those that are set, so that the
// few pixels of these passes cost no launch of a block per pixel.
//   PH 3: sc.pend set by launch 2;
//   PH 4 (wide pass): status with SUPPORT_OVERFLOW or KKT_FAIL and without CERTIFIED.
template <int PH, int KW>
__global__ void __launch_bounds__(32) k_refit_scan(SplitScratch sc, const double2 *__restrict__ A64,
                                                   const double2 *__restrict__ h,
                                                   const float *__restrict__ A_re,
                                                   const float *__restrict__ A_im, int N, int L, int lda,
                                                   RefitLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    PixelSmem<KW> &P = pixel_smem<KW>(smem_raw, N, lane);
    // groups of 32 pixels from the work counter when there is one (the few long pixels
    // then spread over the warps as they finish), else a fixed stride over the groups
    unsigned long long *queue = sc.queue ? sc.queue + (PH == 3 ? 0 : 1) : nullptr;
    for (long long it = 0;; ++it) {
        long long grp;
        if (queue) {
            unsigned long long t = 0;
            if (lane == 0)
                t = atomicAdd(queue, 1ULL);
            grp = (long long)__shfl_sync(0xffffffffu, t, 0);
        } else {
            grp = (long long)blockIdx.x + it * (long long)gridDim.x;
        }
        const long long p0 = 32LL * grp;
        if (p0 >= a.P)
            break;
        const long long q = p0 + lane;
        bool want = false;
        if (q < a.P) {
            if constexpr (PH == 3) {
                want = sc.pend[q] != 0;
            } else {
                const int st = a.status[q];
                want = (st & (BPDN_PX_SUPPORT_OVERFLOW | BPDN_PX_KKT_FAIL)) && !(st & BPDN_PX_CERTIFIED);
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, want);
        while (bal) {
            const int j = __ffs(bal) - 1;
            bal &= bal - 1;
            refit_pixel<PH, KW>(P, p0 + j, sc, A64, h, A_re, A_im, N, L, lda, a, lane);
            __syncwarp();
        }
    }
}

}  // namespace

size_t refit_scratch_bytes(int64_t P)
{
    if (P <= 0)
        return 0;
    return (size_t)((12 * P + 64 * P + 128 * P + 256 * P + 7 * 256 + 255) / 256 * 256);
}

namespace {
// blocks of a persistent scan launch: every SM as full as the shared memory allows
template <int PH, int KW>
cudaError_t launch_scan(const OpHandle &op, const SplitScratch &sc, const RefitLaunch &a, cudaStream_t s)
{
    const size_t smem = pixel_smem_bytes<KW>(op.N);
    cudaError_t e = cudaFuncSetAttribute(k_refit_scan<PH, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refit_scan<PH, KW>, 32, smem);
    if (e != cudaSuccess)
        return e;
    long long blocks = (long long)std::max(per_sm, 1) * std::max(sms, 1);
    const long long groups = (a.P + 31) / 32;  // no more warps than groups of 32 pixels
    if (blocks > groups)
        blocks = groups;
    const double2 *h = op.md ? nullptr : op.h;
    k_refit_scan<PH, KW><<<(unsigned)blocks, 32, smem, s>>>(sc, op.A64, h, op.A_re, op.A_im, op.N, op.L, op.lda, a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_refit(const OpHandle &op, const RefitLaunch &a, cudaStream_t s)
{
    if (a.P <= 0)
        return cudaSuccess;
    const size_t smem = WARPS * pixel_smem_bytes<KWF>(op.N);
    const long long blocks = (a.P + WARPS - 1) / WARPS;
    const double2 *h = op.md ? nullptr : op.h;
    SplitScratch sc = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e;
    if (a.split) {
        // three launches: the FP32 support search of every pixel, the FP64 finish and
        // certificate, then further rounds for the pixels that need them
        unsigned char *b = a.split;
        auto take = [&](size_t bytes) {
            unsigned char *r = b;
            b += (bytes + 255) / 256 * 256;
            return r;
        };
        sc.m = (int *)take(4 * (size_t)a.P);
        sc.meta = (int *)take(4 * (size_t)a.P);
        sc.W = (int *)take(64 * (size_t)a.P);
        sc.z = (float2 *)take(128 * (size_t)a.P);
        sc.pend = (int *)take(4 * (size_t)a.P);
        sc.zs = (double2 *)take(256 * (size_t)a.P);
        sc.queue = (unsigned long long *)take(2 * sizeof(unsigned long long));
        e = cudaMemsetAsync(sc.queue, 0, 2 * sizeof(unsigned long long), s);
        if (e != cudaSuccess)
            return e;
        e = cudaFuncSetAttribute(k_refit_t<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_refit_t<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_refit_t<1><<<(unsigned)blocks, WARPS * 32, smem, s>>>(sc, op.A64, h, op.A_re, op.A_im, op.N, op.L, op.lda, a);
        k_refit_t<2><<<(unsigned)blocks, WARPS * 32, smem, s>>>(sc, op.A64, h, op.A_re, op.A_im, op.N, op.L, op.lda, a);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = launch_scan<3, KWF>(op, sc, a, s);
    } else {
        e = cudaFuncSetAttribute(k_refit_t<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_refit_t<0><<<(unsigned)blocks, WARPS * 32, smem, s>>>(sc, op.A64, h, op.A_re, op.A_im, op.N, op.L, op.lda, a);
        e = cudaGetLastError();
    }
    // the wide pass over the pixels whose support the fast path could not hold or settle
    if (e == cudaSuccess && a.s_max > KWF)
        e = launch_scan<4, KWW>(op, sc, a, s);
    return e;
}

}  // namespace bpdn
