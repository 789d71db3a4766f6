// Split-grid iteration kernel: Algorithm 1 (RBPG with backtracking, Eqs. 11-15) in FP32 for
// grids too large for one thread per grid point in a CTA (the multi-component grids of Eq. 4,
// L up to BPDN_MAX_L).  A CTA holds KS pixels (slots); its eight warps walk the grid in
// 32-point chunks (warp w takes chunks w, w + 8, ...), and every operator load of the
// gradient serves all KS slots.  x^k, x^{k-1} and xbar of a slot are rows of the CTA's
// scratch in global memory, gated by per-chunk nonzero masks in shared memory: only nonzeros
// are read or written, so the rows cost traffic in proportion to the support, not to L.
//
// One sweep:
//   1. per chunk and lane (one grid point l): the gradient sum_n conj(A_nl) r_n of every
//      slot from an interleaved copy of the FP32 operator (one 8-byte load per lane and
//      row, coalesced over l; r in shared memory), then per slot the
//      extrapolation y = x + beta (x - x^{k-1}) and the complex soft threshold of
//      v = y - 2 alpha grad.  Only chunks where xbar, x^k or x^{k-1} has a nonzero go on to
//      the sums of Eq. 15, F and the stopping test (a warp sum per chunk, added to the
//      warp's running sums in chunk order) and to A xbar over the chunk's nonzeros
//      (ascending l, from the transposed table, coalesced over n);
//   2. warp p decides slot p: the warps' sums and A xbar added in warp order, Eq. 15, the
//      monotone accept, the stopping test, the N-space update (A x^k, A x^{k-1}, A y and the
//      next residual); a finished pixel's x goes to its output row and the slot is refilled.
// Every sum has a fixed order, so results do not depend on timing.  There are no waits on
// other CTAs or on asynchronous units: only CTA barriers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kWarps = 8;  // warps per CTA
constexpr int kThreads = 32 * kWarps;

struct SplitParams {
    const unsigned char *Abf;  // BF16 operator tiles of 128 grid points, K-major core-matrix layout (tensor-core variant)
    const float2 *AT;          // transposed FP32 table [L][N]
    const float2 *A2;          // interleaved FP32 table [N][L]: (Re A_nl, Im A_nl)
    int N, L, NC;
    int Kp, NCT;               // tensor-core variant: K = 2N padded to 16; 128-point tiles
    float2 *rows;              // [ctas][KS][3][L]
    SolveLaunch a;
};

// per-slot state (shared memory)
struct SlotSt {
    long long pix;  // -1: the slot is empty
    int k, nbt, nbt_it, status, nnz;
    float alpha, Fx, lam;
    int bx, bxp, bb;  // row buffers of x^k, x^{k-1} and xbar (bx == bxp after a rejected step)
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// packed FP32 pair FMA: d = a * b + c on both halves (each half rounded as fmaf)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)),
          "l"(*reinterpret_cast<unsigned long long *>(&c)));
    return *reinterpret_cast<float2 *>(&d);
}

// sweep parameters of a slot: beta, 2 alpha, tau = alpha lambda, and the three row buffers
// (x^k | x^{k-1} << 2 | xbar << 4) as an int
__device__ __forceinline__ float4 slot_par(float beta, float alpha, float lam, int bx, int bxp, int bb)
{
    return make_float4(beta, 2.f * alpha, alpha * lam, __int_as_float(bx | (bxp << 2) | (bb << 4)));
}

// shared memory carve-up (16-byte aligned sections)
struct SplitSmem {
    float2 *G, *Ax, *Axp, *Ay;  // [KS][N]
    float *R;                   // [N][2][KS]: Re r_n of every slot, then Im r_n (slot-minor)
    float2 *Wacc;               // [KS][kWarps][N]
    float4 *Wsum;               // [KS][kWarps]: dd, l1, dx, xn
    float4 *Par;                // [KS]: slot_par
    int *Wnnz;                  // [KS][kWarps]
    uint32_t *M;                // [KS][3][NC] nonzero masks of the row buffers
    SlotSt *S;                  // [KS]
    unsigned char *Bop;         // tensor-core variant: the residual rows as the MMA's B operand (BF16)
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) / 16 * 16; }

__host__ __device__ inline size_t split_smem_bytes(int KS, int N, int NC, int nw = kWarps)
{
    size_t b = 0;
    b += align16((size_t)4 * KS * N * sizeof(float2));
    b += align16((size_t)N * KS * sizeof(float2));
    b += align16((size_t)KS * nw * N * sizeof(float2));
    b += (size_t)KS * nw * sizeof(float4);
    b += (size_t)KS * sizeof(float4);
    b += align16((size_t)KS * nw * sizeof(int));
    b += align16((size_t)KS * 3 * NC * sizeof(uint32_t));
    b += (size_t)KS * sizeof(SlotSt);
    return b;
}

template <int KS>
__device__ __forceinline__ SplitSmem carve(unsigned char *base, int N, int NC, int nw = kWarps)
{
    SplitSmem s;
    s.Bop = nullptr;
    unsigned char *p = base;
    s.G = (float2 *)p;
    s.Ax = s.G + KS * N;
    s.Axp = s.Ax + KS * N;
    s.Ay = s.Axp + KS * N;
    p += align16((size_t)4 * KS * N * sizeof(float2));
    s.R = (float *)p;
    p += align16((size_t)N * KS * sizeof(float2));
    s.Wacc = (float2 *)p;
    p += align16((size_t)KS * nw * N * sizeof(float2));
    s.Wsum = (float4 *)p;
    p += (size_t)KS * nw * sizeof(float4);
    s.Par = (float4 *)p;
    p += (size_t)KS * sizeof(float4);
    s.Wnnz = (int *)p;
    p += align16((size_t)KS * nw * sizeof(int));
    s.M = (uint32_t *)p;
    p += align16((size_t)KS * 3 * NC * sizeof(uint32_t));
    s.S = (SlotSt *)p;
    return s;
}

// The launch's two copies of the FP32 operator: AT[l][n] = A_nl for the gather of A xbar
// (lanes over n), and A2[n][l] = A_nl for the gradient (one 8-byte load per lane and row,
// lanes over l)
__global__ void k_operator_copies(const float *__restrict__ A_re, const float *__restrict__ A_im, int N, int L,
                                  int lda, float2 *__restrict__ AT, float2 *__restrict__ A2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * L)
        return;
    const int l = (int)(i / N), n = (int)(i % N);
    const float2 v = make_float2(A_re[(size_t)n * lda + l], A_im[(size_t)n * lda + l]);
    AT[i] = v;
    if (A2)
        A2[(size_t)n * L + l] = v;
}

// byte offset of element (row, k) of a K-major BF16 MMA operand with Kp columns (no swizzle):
// core matrices of 8 rows x 16 bytes, the K-adjacent one 128 bytes on, the next 8-row group
// Kp/8 x 128 bytes on
__host__ __device__ inline int kmaj(int row, int k, int Kp)
{
    return (row >> 3) * (Kp / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// residual r_n of slot p for the next gradient: FP32 rows (CUDA-core variant), or the B
// operand of the tensor-core variant, B[p] = (Re r, Im r), B[KS + p] = (Im r, -Re r) in BF16
// (so that D[l, p] = Re sum_n conj(A_nl) r_n and D[l, KS + p] its imaginary part)
template <int KS, bool TC>
__device__ __forceinline__ void put_r(const SplitParams &prm, const SplitSmem &sm, int p, int n, float re, float im)
{
    if constexpr (TC) {
        const int N = prm.N, Kp = prm.Kp;
        const __nv_bfloat16 bre = __float2bfloat16_rn(re), bim = __float2bfloat16_rn(im);
        const __nv_bfloat16 nre = __float2bfloat16_rn(-re);
        *(__nv_bfloat16 *)(sm.Bop + kmaj(p, n, Kp)) = bre;
        *(__nv_bfloat16 *)(sm.Bop + kmaj(p, N + n, Kp)) = bim;
        *(__nv_bfloat16 *)(sm.Bop + kmaj(KS + p, n, Kp)) = bim;
        *(__nv_bfloat16 *)(sm.Bop + kmaj(KS + p, N + n, Kp)) = nre;
    } else {
        sm.R[n * 2 * KS + p] = re;
        sm.R[n * 2 * KS + KS + p] = im;
    }
}

// Refill slot p (warp p) from the work counter: x^0 = x^{-1} = 0, so A y = 0 and r = -g.
// Pixels with a non-finite g (or a solve with max_iter <= 0) get x = 0 at once.  With no
// pixel left the slot is marked empty and its residual column zeroed, so that the shared
// gradient loop adds nothing for it.
template <int KS, bool TC>
__device__ void refill_slot(const SplitParams &prm, const SplitSmem &sm, int p, int lane)
{
    const SolveLaunch &a = prm.a;
    const int N = prm.N, L = prm.L, NC = prm.NC;
    SlotSt &S = sm.S[p];
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0)
            q = atomicAdd(a.counter, 1ULL);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= (unsigned long long)a.P) {
            for (int n = lane; n < N; n += 32)
                put_r<KS, TC>(prm, sm, p, n, 0.f, 0.f);
            if (lane == 0)
                S.pix = -1;
            __syncwarp();
            return;
        }
        const float2 *gq = a.g + (size_t)q * N;
        bool fin = true;
        for (int n = lane; n < N; n += 32) {
            const float2 v = gq[n];
            fin = fin && isfinite(v.x) && isfinite(v.y);
        }
        const bool allfin = __all_sync(0xffffffffu, fin);
        if (!allfin || a.max_iter <= 0) {
            float2 *xq = a.x + (size_t)q * L;
            for (int l = lane; l < L; l += 32)
                xq[l] = make_float2(0.f, 0.f);
            if (lane == 0) {
                a.status[q] = allfin ? (BPDN_PX_NOT_CONVERGED | BPDN_PX_ZERO_SOLUTION) : BPDN_PX_NONFINITE;
                a.iters[q] = 0;
                if (a.nbt)
                    a.nbt[q] = 0;
                if (a.nsupp)
                    a.nsupp[q] = 0;
            }
            continue;
        }
        float gg2 = 0.f;
        for (int n = lane; n < N; n += 32) {
            const float2 v = gq[n];
            sm.G[p * N + n] = v;
            sm.Ax[p * N + n] = make_float2(0.f, 0.f);
            sm.Axp[p * N + n] = make_float2(0.f, 0.f);
            sm.Ay[p * N + n] = make_float2(0.f, 0.f);
            put_r<KS, TC>(prm, sm, p, n, -v.x, -v.y);
            gg2 = fmaf(v.x, v.x, fmaf(v.y, v.y, gg2));
        }
        gg2 = warp_sum(gg2);
        // x^k (buffer 0) and x^{k-1} (buffer 1) are zero; buffer 2 takes xbar
        for (int c = lane; c < NC; c += 32) {
            sm.M[(p * 3 + 0) * NC + c] = 0u;
            sm.M[(p * 3 + 1) * NC + c] = 0u;
        }
        if (lane == 0) {
            const float lam = a.lam_pp ? a.lam[q] : a.lam[0];
            S.pix = (long long)q;
            S.k = 1;
            S.nbt = 0;
            S.nbt_it = 0;
            S.status = 0;
            S.nnz = 0;
            S.alpha = a.alpha0;
            S.Fx = gg2;  // F(0) = ||g||^2
            S.lam = lam;
            S.bx = 0;
            S.bxp = 1;
            S.bb = 2;
            sm.Par[p] = slot_par(0.f, a.alpha0, lam, 0, 1, 2);  // x^0 - x^{-1} = 0: beta unused
        }
        __syncwarp();
        return;
    }
}

// Warp p: the end of slot p's sweep (Eq. 15, accept, stopping test, N-space update).
template <int KS, int NCH, bool TC>
__device__ void decide_slot(const SplitParams &prm, const SplitSmem &sm, float2 *rows, int p, int lane, int nw)
{
    const SolveLaunch &a = prm.a;
    const int N = prm.N, L = prm.L, NC = prm.NC;
    SlotSt &S = sm.S[p];
    // the warps' sums, in warp order
    float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
    int nnz = 0;
    for (int v = 0; v < nw; ++v) {
        const float4 t = sm.Wsum[p * nw + v];
        dd += t.x;
        l1 += t.y;
        dx += t.z;
        xn += t.w;
        nnz += sm.Wnnz[p * nw + v];
    }
    float2 axb[NCH], gg[NCH];
    float lhs = 0.f, res = 0.f;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        axb[c] = make_float2(0.f, 0.f);
        gg[c] = make_float2(0.f, 0.f);
        const int n = lane + 32 * c;
        if (n < N) {
            for (int v = 0; v < nw; ++v) {
                const float2 t = sm.Wacc[(p * nw + v) * N + n];
                axb[c].x += t.x;
                axb[c].y += t.y;
            }
            const float2 ay = sm.Ay[p * N + n];
            gg[c] = sm.G[p * N + n];
            const float d0 = axb[c].x - ay.x, d1 = axb[c].y - ay.y;
            lhs = fmaf(d0, d0, fmaf(d1, d1, lhs));
            const float e0 = axb[c].x - gg[c].x, e1 = axb[c].y - gg[c].y;
            res = fmaf(e0, e0, fmaf(e1, e1, res));
        }
    }
    lhs = warp_sum(lhs);
    res = warp_sum(res);
    const float al = S.alpha, lam = S.lam, Fx = S.Fx;
    const int nbt_it = S.nbt_it, k = S.k, obx = S.bx, obxp = S.bxp, obb = S.bb;
    const long long q = S.pix;
    const float beta_o = sm.Par[p].x;
    const bool bt_ok = lhs <= dd / (2.f * al);
    __syncwarp();  // every lane has read the slot state lane 0 updates below
    if (!bt_ok && nbt_it < a.max_bt) {
        // Eq. 15 failed: the next sweep redoes the prox with the smaller step
        if (lane == 0) {
            const float an = al * a.c_alpha;
            S.alpha = an;
            S.nbt += 1;
            S.nbt_it = nbt_it + 1;
            sm.Par[p] = slot_par(beta_o, an, lam, obx, obxp, obb);
        }
        __syncwarp();
        return;
    }
    const float Fb = fmaf(lam, l1, res);
    const bool accepted = Fb <= Fx;
    const float tol2 = a.tol * a.tol;
    const bool conv = (dx <= tol2 * xn) || (dx == 0.f);
    const bool fin = conv || (k >= a.max_iter);
    // rows after this iteration: x^{k-1} <- x^k; x^k <- xbar when accepted
    const int nbx = accepted ? obb : obx;
    const int nbb = accepted ? 3 - obb - obx : obb;
    const float beta_n = (float)(k - 1) / (float)(k + 2);
    if (!fin) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int n = lane + 32 * c;
            if (n < N) {
                const float2 axo = sm.Ax[p * N + n];
                const float2 axn = accepted ? axb[c] : axo;
                sm.Axp[p * N + n] = axo;
                sm.Ax[p * N + n] = axn;
                const float2 ayn =
                    make_float2(fmaf(beta_n, axn.x - axo.x, axn.x), fmaf(beta_n, axn.y - axo.y, axn.y));
                sm.Ay[p * N + n] = ayn;
                put_r<KS, TC>(prm, sm, p, n, ayn.x - gg[c].x, ayn.y - gg[c].y);
            }
        }
    }
    int st = S.status;
    if (!bt_ok)
        st |= BPDN_PX_BT_LIMIT;
    if (fin && !conv)
        st |= BPDN_PX_NOT_CONVERGED;
    const int nz = accepted ? nnz : S.nnz;
    __syncwarp();
    if (!fin) {
        if (lane == 0) {
            S.status = st;
            S.nnz = nz;
            if (accepted)
                S.Fx = Fb;
            S.k = k + 1;
            S.nbt_it = 0;
            S.bx = nbx;
            S.bxp = obx;
            S.bb = nbb;
            sm.Par[p] = slot_par(beta_n, al, lam, nbx, obx, nbb);
        }
        __syncwarp();
        return;
    }
    // finished: x^k to the output row (zeros off the mask), the counters, then a new pixel
    const float2 *xr = rows + ((size_t)p * 3 + nbx) * L;
    const uint32_t *mr = sm.M + ((size_t)p * 3 + nbx) * NC;
    float2 *xq = a.x + (size_t)q * L;
    for (int c = 0; c < NC; ++c) {
        const int l = 32 * c + lane;
        if (l < L)
            xq[l] = ((mr[c] >> lane) & 1u) ? xr[l] : make_float2(0.f, 0.f);
    }
    if (lane == 0) {
        a.status[q] = (nz == 0) ? (st | BPDN_PX_ZERO_SOLUTION) : st;
        a.iters[q] = k;
        if (a.nbt)
            a.nbt[q] = S.nbt;
        if (a.nsupp)
            a.nsupp[q] = nz;
    }
    __syncwarp();
    refill_slot<KS, TC>(prm, sm, p, lane);
}

// Extrapolation, complex soft threshold, the sums of Eq. 15, F and the stopping test, and A xbar
// for every active slot on the 32-point block c (lane: grid point l = 32 c + lane; gx, gy: its
// gradient per slot).  Blocks where xbar, x^k or x^{k-1} has a nonzero add their warp sums to
// warp w's running sums (sm.Wsum[p * nw + w], in block order) and their share of A xbar to acc.
template <int KS, int NCH>
__device__ __forceinline__ void prox_block(const SplitParams &prm, const SplitSmem &sm, float2 *rows, int c,
                                           int lane, int w, int nw, unsigned actm, const float (&gx)[KS],
                                           const float (&gy)[KS], float2 (&acc)[KS][NCH])
{
    const int N = prm.N, L = prm.L, NC = prm.NC;
    const int l = 32 * c + lane;
    const bool inl = l < L;
#pragma unroll
    for (int p = 0; p < KS; ++p) {
        if (!((actm >> p) & 1u))
            continue;  // the same for the whole CTA
        const float4 par = sm.Par[p];
        const int bits = __float_as_int(par.w);
        const int bx = bits & 3, bxp = (bits >> 2) & 3, bb = (bits >> 4) & 3;
        const uint32_t mx = sm.M[(p * 3 + bx) * NC + c];
        const uint32_t mxp = sm.M[(p * 3 + bxp) * NC + c];
        float2 xv = make_float2(0.f, 0.f), xpv = make_float2(0.f, 0.f);
        if ((mx >> lane) & 1u)
            xv = rows[((size_t)p * 3 + bx) * L + l];
        if ((mxp >> lane) & 1u)
            xpv = rows[((size_t)p * 3 + bxp) * L + l];
        const float yx = fmaf(par.x, xv.x - xpv.x, xv.x), yy = fmaf(par.x, xv.y - xpv.y, xv.y);
        const float vx = fmaf(-par.y, gx[p], yx), vy = fmaf(-par.y, gy[p], yy);
        const float m2 = fmaf(vx, vx, vy * vy);
        // soft threshold (Eq. 12): scale 1 - tau / |v| where that is positive
        const float rs = rsqrtf(m2);
        const float sc = fmaf(-par.z, rs, 1.f);
        const bool nz = inl && sc > 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0)
            sm.M[(p * 3 + bb) * NC + c] = bal;
        if ((bal | mx | mxp) == 0u)
            continue;  // xbar = y = 0 on the whole chunk: nothing to add
        float xbx = 0.f, xby = 0.f, l1 = 0.f;
        if (nz) {
            xbx = vx * sc;
            xby = vy * sc;
            l1 = fmaf(m2, rs, -par.z);
            rows[((size_t)p * 3 + bb) * L + l] = make_float2(xbx, xby);
        }
        const float ex = xbx - yx, ey = xby - yy;
        const float fx = xbx - xv.x, fy = xby - xv.y;
        const float dd = warp_sum(fmaf(ex, ex, ey * ey));
        const float s1 = warp_sum(l1);
        const float dx = warp_sum(fmaf(fx, fx, fy * fy));
        const float xn = warp_sum(fmaf(xbx, xbx, xby * xby));
        if (lane == 0) {
            float4 t = sm.Wsum[p * nw + w];
            t.x += dd;
            t.y += s1;
            t.z += dx;
            t.w += xn;
            sm.Wsum[p * nw + w] = t;
            sm.Wnnz[p * nw + w] += __popc(bal);
        }
        // this chunk's share of A xbar, ascending l; lane n owns rows n + 32 c
        unsigned m = bal;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1u;
            const float xr = __shfl_sync(0xffffffffu, xbx, j), xi = __shfl_sync(0xffffffffu, xby, j);
            const float2 *at = prm.AT + (size_t)(32 * c + j) * N;
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc) {
                const int n = lane + 32 * cc;
                if (n < N) {
                    const float2 av = __ldg(at + n);
                    acc[p][cc].x = fmaf(av.x, xr, fmaf(-av.y, xi, acc[p][cc].x));
                    acc[p][cc].y = fmaf(av.x, xi, fmaf(av.y, xr, acc[p][cc].y));
                }
            }
        }
    }
}

template <int KS, int NCH>
__global__ void __launch_bounds__(kThreads, 3) k_rbpg_split(const __grid_constant__ SplitParams prm)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = prm.N, L = prm.L, NC = prm.NC;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SplitSmem sm = carve<KS>(smem_raw, N, NC);
    float2 *rows = prm.rows + (size_t)blockIdx.x * KS * 3 * L;
    for (int p = w; p < KS; p += kWarps)
        refill_slot<KS, false>(prm, sm, p, lane);
    __syncthreads();
    for (;;) {
        // this sweep's slots; each warp's running sums start at zero
        unsigned actm = 0;
#pragma unroll
        for (int p = 0; p < KS; ++p)
            actm |= (sm.S[p].pix >= 0) ? (1u << p) : 0u;
        if (!actm)
            break;
        if (lane < KS) {
            sm.Wsum[lane * kWarps + w] = make_float4(0.f, 0.f, 0.f, 0.f);
            sm.Wnnz[lane * kWarps + w] = 0;
        }
        __syncwarp();  // lane 0 adds to these below
        float2 acc[KS][NCH];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                acc[p][c] = make_float2(0.f, 0.f);
        for (int c = w; c < NC; c += kWarps) {
            const int l = 32 * c + lane;
            const bool inl = l < L;
            // gradient of every slot: one pair of operator loads feeds all of them; slot
            // pairs (2q, 2q+1) in packed FP32 FMAs
            float2 gx2[KS / 2], gy2[KS / 2];
#pragma unroll
            for (int q = 0; q < KS / 2; ++q)
                gx2[q] = gy2[q] = make_float2(0.f, 0.f);
            if (inl) {
                const float2 *pa = prm.A2 + l;
#pragma unroll 4
                for (int n = 0; n < N; ++n) {
                    const float2 av = __ldg(pa + (size_t)n * L);
                    const float2 ar2 = make_float2(av.x, av.x), ai2 = make_float2(av.y, av.y);
                    const float2 nai2 = make_float2(-av.y, -av.y);
                    const float4 *rre = (const float4 *)(sm.R + n * 2 * KS);
                    const float4 *rim = (const float4 *)(sm.R + n * 2 * KS + KS);
#pragma unroll
                    for (int h = 0; h < KS / 4; ++h) {
                        const float4 rx = rre[h], ry = rim[h];  // slots 4h .. 4h+3
                        const float2 rx0 = make_float2(rx.x, rx.y), rx1 = make_float2(rx.z, rx.w);
                        const float2 ry0 = make_float2(ry.x, ry.y), ry1 = make_float2(ry.z, ry.w);
                        // conj(a) r = (ar r.x + ai r.y) + j (ar r.y - ai r.x)
                        gx2[2 * h] = ffma2(ar2, rx0, ffma2(ai2, ry0, gx2[2 * h]));
                        gy2[2 * h] = ffma2(ar2, ry0, ffma2(nai2, rx0, gy2[2 * h]));
                        gx2[2 * h + 1] = ffma2(ar2, rx1, ffma2(ai2, ry1, gx2[2 * h + 1]));
                        gy2[2 * h + 1] = ffma2(ar2, ry1, ffma2(nai2, rx1, gy2[2 * h + 1]));
                    }
                }
            }
            float gx[KS], gy[KS];
#pragma unroll
            for (int q = 0; q < KS / 2; ++q) {
                gx[2 * q] = gx2[q].x;
                gx[2 * q + 1] = gx2[q].y;
                gy[2 * q] = gy2[q].x;
                gy[2 * q + 1] = gy2[q].y;
            }
            prox_block<KS, NCH>(prm, sm, rows, c, lane, w, kWarps, actm, gx, gy, acc);
        }
#pragma unroll
        for (int p = 0; p < KS; ++p) {
            if (!((actm >> p) & 1u))
                continue;
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc) {
                const int n = lane + 32 * cc;
                if (n < N)
                    sm.Wacc[(p * kWarps + w) * N + n] = acc[p][cc];
            }
        }
        __syncthreads();
        for (int p = w; p < KS; p += kWarps)
            if ((actm >> p) & 1u)
                decide_slot<KS, NCH, false>(prm, sm, rows, p, lane, kWarps);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ tensor-core variant
// The same sweep with the gradient from tcgen05 MMAs (BF16 operands, FP32 accumulators): per
// 128-point tile of the grid D[l, j] = sum_k Aop[l, k] B[j, k], Aop[l, :] = (Re A_.l, Im A_.l)
// (K = 2N padded to 16) from the launch's BF16 tiled copy of the operator, staged in shared
// memory by cp.async into three buffers (the copy of tile c+2 and the MMA of tile c+1 run
// while the warps work on tile c), and B = the residual rows (put_r).  Four warps: warp w holds tensor-memory lanes 32w ..
// 32w+31 = grid points 128c + 32w + lane = 32-point block 4c + w.  Every wait for the tensor
// cores is bounded; after one runs out the CTA ends its pixels with DEVICE_TIMEOUT.

constexpr int kTcWarps = 4;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTcKS = 8;          // slots: B has 2 KS = 16 rows, the MMA's N
constexpr uint32_t kTcCols = 32;  // tensor-memory columns: two accumulator buffers of 16
// instruction descriptor: D FP32, A and B BF16, both K-major, N = 16, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// shared-memory matrix descriptor of tcgen05 (no swizzle)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) [+]= A (shared memory) x B (shared memory)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t accum)
{
    asm volatile(
        "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accum)
        : "memory");
}

// bounded wait for an mbarrier phase; false when the bound ran out
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    for (int it = 0; it < (1 << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p;}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done)
            return true;
    }
    return false;
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i)
        v[i] = __uint_as_float(r[i]);
}

// all threads: copy 128-point tile `tile` of the BF16 operator (128 x Kp, 256 Kp bytes, laid
// out as the MMA reads it) into buf, 16 bytes per cp.async
__device__ __forceinline__ void stage_tile(const SplitParams &prm, unsigned char *buf, int tile, int tid)
{
    const uint32_t tb = 256u * (uint32_t)prm.Kp;
    const unsigned char *src = prm.Abf + (size_t)tile * tb;
    const uint32_t dst = smem_addr(buf);
    for (uint32_t o = 16u * tid; o < tb; o += 16u * kTcThreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + o), "l"(src + o) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// thread 0: the MMAs of one tile into accumulator columns d, committed to mbar
__device__ __forceinline__ void issue_tile_mma(uint32_t d, const unsigned char *abuf, const unsigned char *bop,
                                               int Kp, uint32_t mbar)
{
    const uint32_t a0 = smem_addr(abuf), b0 = smem_addr(bop);
    const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
    for (int j = 0; j < Kp / 16; ++j)
        tc_mma(d, tc_desc(a0 + 256u * j, 128u, sbo), tc_desc(b0 + 256u * j, 128u, sbo), j > 0 ? 1u : 0u);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bytes of the tensor-core variant's dynamic shared memory
__host__ __device__ inline size_t split_tc_smem_bytes(int N, int NC, int Kp)
{
    return (size_t)3 * 256 * Kp + align16((size_t)2 * kTcKS * Kp * 2) + split_smem_bytes(kTcKS, N, NC, kTcWarps);
}

template <int NCH>
__global__ void __launch_bounds__(kTcThreads, 1) k_rbpg_split_tc(const __grid_constant__ SplitParams prm)
{
    constexpr int KS = kTcKS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) unsigned long long s_mbar[2];
    const SolveLaunch &a = prm.a;
    const int N = prm.N, L = prm.L, NC = prm.NC, Kp = prm.Kp, NCT = prm.NCT;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const size_t tb = (size_t)256 * Kp;
    // three operator buffers: tile t sits in abuf(t % 3); its copy is issued two tiles ahead
    auto abuf = [&](long long tt) -> unsigned char * { return smem_raw + (size_t)(tt % 3) * tb; };
    unsigned char *bop = smem_raw + 3 * tb;
    SplitSmem sm = carve<KS>(bop + align16((size_t)2 * KS * Kp * 2), N, NC, kTcWarps);
    sm.Bop = bop;
    float2 *rows = prm.rows + (size_t)blockIdx.x * KS * 3 * L;
    const uint32_t mb0 = smem_addr(&s_mbar[0]), mb1 = smem_addr(&s_mbar[1]);
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = tid; i < 2 * KS * Kp * 2 / 4; i += kTcThreads)
        ((uint32_t *)bop)[i] = 0u;  // the K padding of B stays zero
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tlane = tmem + ((uint32_t)(32 * w) << 16);
    for (int p = w; p < KS; p += kTcWarps)
        refill_slot<KS, true>(prm, sm, p, lane);
    stage_tile(prm, abuf(0), 0, tid);
    stage_tile(prm, abuf(1), NCT > 1 ? 1 : 0, tid);
    asm volatile("cp.async.wait_all;" ::: "memory");
    proxy_fence();  // the operator tile and the B rows, for the first MMA
    tc_before();
    __syncthreads();
    tc_after();
    uint32_t ph0 = 0u, ph1 = 0u;
    long long t = 0;  // tiles of all sweeps so far: tile t sits in buffer t & 1
    bool abort = false;
    int pend = -1;  // after a wait ran out: the accumulator buffer not seen complete
    uint32_t pend_ph = 0u;
    for (;;) {
        unsigned actm = 0;
#pragma unroll
        for (int p = 0; p < KS; ++p)
            actm |= (sm.S[p].pix >= 0) ? (1u << p) : 0u;
        if (!actm)
            break;
        if (lane < KS) {
            sm.Wsum[lane * kTcWarps + w] = make_float4(0.f, 0.f, 0.f, 0.f);
            sm.Wnnz[lane * kTcWarps + w] = 0;
        }
        __syncwarp();
        float2 acc[KS][NCH];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc)
                acc[p][cc] = make_float2(0.f, 0.f);
        if (tid == 0)
            issue_tile_mma(tmem + 16u * (uint32_t)(t & 1), abuf(t), bop, Kp, (t & 1) ? mb1 : mb0);
        for (int c = 0; c < NCT; ++c, ++t) {
            const int b = (int)(t & 1);
            const uint32_t ph = b ? ph1 : ph0;
            // every lane polls the barrier on its own: vote, which also reconverges the warp
            // before the warp-wide (.sync.aligned) tensor-memory loads below
            const bool ok = __all_sync(0xffffffffu, tc_wait(b ? mb1 : mb0, ph));
            if (b)
                ph1 ^= 1u;
            else
                ph0 ^= 1u;
            tc_after();
            float d[16];
            if (ok) {
                tc_ld8(tlane + 16u * b, d);
                tc_ld8(tlane + 16u * b + 8u, d + 8);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
                pend = b;
                pend_ph = ph;
            }
            // the copy of tile t + 1, issued a step ago, is in place for its MMA
            asm volatile("cp.async.wait_all;" ::: "memory");
            proxy_fence();
            tc_before();
            const int bad = __syncthreads_or(ok ? 0 : 1);
            tc_after();
            if (bad) {
                if (!ok && a.err)
                    atomicExch(a.err, 1);
                abort = true;
                break;
            }
            if (c + 1 < NCT && tid == 0)
                issue_tile_mma(tmem + 16u * (uint32_t)(b ^ 1), abuf(t + 1), bop, Kp, b ? mb0 : mb1);
            // tile t + 2 (of this sweep or the next) into the buffer of tile t - 1, whose MMA
            // was waited for a step ago; the copy runs while the warps work on tile t
            stage_tile(prm, abuf(t + 2), (int)((c + 2) % NCT), tid);
            float gx[KS], gy[KS];
#pragma unroll
            for (int p = 0; p < KS; ++p) {
                gx[p] = d[p];
                gy[p] = d[KS + p];
            }
            prox_block<KS, NCH>(prm, sm, rows, 4 * c + w, lane, w, kTcWarps, actm, gx, gy, acc);
        }
        if (abort)
            break;
#pragma unroll
        for (int p = 0; p < KS; ++p) {
            if (!((actm >> p) & 1u))
                continue;
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc) {
                const int n = lane + 32 * cc;
                if (n < N)
                    sm.Wacc[(p * kTcWarps + w) * N + n] = acc[p][cc];
            }
        }
        __syncthreads();
        for (int p = w; p < KS; p += kTcWarps)
            if ((actm >> p) & 1u)
                decide_slot<KS, NCH, true>(prm, sm, rows, p, lane, kTcWarps);
        proxy_fence();  // the B rows the decisions wrote, for the next MMAs
        tc_before();
        __syncthreads();
        tc_after();
    }
    if (abort) {
        // a tensor-core wait ran out: every pixel in a slot keeps its last accepted iterate
        // and every pixel not yet taken gets x = 0, both with DEVICE_TIMEOUT
        for (int p = w; p < KS; p += kTcWarps) {
            const SlotSt &S = sm.S[p];
            const long long q = S.pix;
            if (q < 0)
                continue;
            const float2 *xr = rows + ((size_t)p * 3 + S.bx) * L;
            const uint32_t *mr = sm.M + ((size_t)p * 3 + S.bx) * NC;
            float2 *xq = a.x + (size_t)q * L;
            for (int c = 0; c < NC; ++c) {
                const int l = 32 * c + lane;
                if (l < L)
                    xq[l] = ((mr[c] >> lane) & 1u) ? xr[l] : make_float2(0.f, 0.f);
            }
            if (lane == 0) {
                a.status[q] = S.status | BPDN_PX_DEVICE_TIMEOUT | (S.nnz == 0 ? BPDN_PX_ZERO_SOLUTION : 0);
                a.iters[q] = S.k;
                if (a.nbt)
                    a.nbt[q] = S.nbt;
                if (a.nsupp)
                    a.nsupp[q] = S.nnz;
            }
        }
        if (w == 0) {
            for (;;) {
                unsigned long long q = 0;
                if (lane == 0)
                    q = atomicAdd(a.counter, 1ULL);
                q = __shfl_sync(0xffffffffu, q, 0);
                if (q >= (unsigned long long)a.P)
                    break;
                float2 *xq = a.x + (size_t)q * L;
                for (int l = lane; l < L; l += 32)
                    xq[l] = make_float2(0.f, 0.f);
                if (lane == 0) {
                    a.status[q] = BPDN_PX_DEVICE_TIMEOUT | BPDN_PX_ZERO_SOLUTION;
                    a.iters[q] = 0;
                    if (a.nbt)
                        a.nbt[q] = 0;
                    if (a.nsupp)
                        a.nsupp[q] = 0;
                }
            }
        }
    }
    // retire the barriers and the tensor memory: no MMA is in flight, except the one a wait
    // gave up on, which gets one more bounded wait first; the last operator copies land
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc_before();
    __syncthreads();
    tc_after();
    if (tid == 0) {
        if (pend >= 0)
            (void)tc_wait(pend ? mb1 : mb0, pend_ph);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb1) : "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// the BF16 operator in 128-point tiles as the MMA reads them: Aop[l, k] = Re A_kl (k < N),
// Im A_{k-N},l (N <= k < 2N), 0 beyond 2N and beyond L
__global__ void k_operator_tiles(const float *__restrict__ A_re, const float *__restrict__ A_im, int N, int L,
                                 int lda, int Kp, int NCT, unsigned char *__restrict__ Abf)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)NCT * 128 * Kp)
        return;
    const int l = (int)(i / Kp), k = (int)(i % Kp);
    float v = 0.f;
    if (l < L) {
        if (k < N)
            v = A_re[(size_t)k * lda + l];
        else if (k < 2 * N)
            v = A_im[(size_t)(k - N) * lda + l];
    }
    *(__nv_bfloat16 *)(Abf + (size_t)(l >> 7) * 256 * Kp + kmaj(l & 127, k, Kp)) = __float2bfloat16_rn(v);
}

template <int KS, int NCH>
void *split_fn()
{
    return (void *)k_rbpg_split<KS, NCH>;
}

template <int NCH>
void *split_tc_fn()
{
    return (void *)k_rbpg_split_tc<NCH>;
}

// the variant for these sizes: in FP32 8 slots when their shared memory fits the device, else
// 4; with BF16 the tensor-core kernel (8 slots, K = 2N padded to 16, at most 160); NCH =
// rows of A per lane in the gather (N <= 32 NCH)
struct SplitVariant {
    void *fn;
    int ks, threads;
    int nc;       // 32-point blocks the masks cover
    int kp, nct;  // tensor-core variant: K and the 128-point tiles
    size_t smem;
};

SplitVariant split_variant(const OpHandle &op, int precision, int max_smem)
{
    const int nch = (op.N + 31) / 32;
    SplitVariant v{nullptr, 0, 0, 0, 0, 0, 0};
    if (nch > 3)
        return v;
    if (precision == 1) {
        const int kp = (2 * op.N + 15) / 16 * 16;
        const int nct = (op.L + 127) / 128;
        const size_t smem = split_tc_smem_bytes(op.N, 4 * nct, kp);
        if (kp > 160 || smem > (size_t)max_smem)
            return v;
        v.fn = nch == 1 ? split_tc_fn<1>() : nch == 2 ? split_tc_fn<2>() : split_tc_fn<3>();
        v.ks = kTcKS;
        v.threads = kTcThreads;
        v.nc = 4 * nct;
        v.kp = kp;
        v.nct = nct;
        v.smem = smem;
        return v;
    }
    const int NC = (op.L + 31) / 32;
    for (int ks : {8, 4}) {
        const size_t smem = split_smem_bytes(ks, op.N, NC);
        if (smem > (size_t)max_smem)
            continue;
        v.ks = ks;
        v.threads = kThreads;
        v.nc = NC;
        v.smem = smem;
        if (ks == 8)
            v.fn = nch == 1 ? split_fn<8, 1>() : nch == 2 ? split_fn<8, 2>() : split_fn<8, 3>();
        else
            v.fn = nch == 1 ? split_fn<4, 1>() : nch == 2 ? split_fn<4, 2>() : split_fn<4, 3>();
        return v;
    }
    return v;
}

int max_smem_dev(int dev)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 48 * 1024;
    }
    return v;
}

// CTAs of a split launch on this device: as many as fit (at most one per KS pixels)
int split_ctas(const SplitVariant &v, int64_t P, int num_sms)
{
    int per_sm = 0;
    if (!v.fn ||
        cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, v.threads, v.smem) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    const int64_t want = (P + v.ks - 1) / v.ks;
    return (int)std::min<int64_t>((int64_t)per_sm * num_sms, want);
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// bytes of the FP32 operator copy AT (and, for the FP32 kernel, A2) at the start of the scratch
size_t at_bytes(const OpHandle &op) { return round256((size_t)op.L * op.N * sizeof(float2)); }

// scratch layout: AT, then A2 (FP32 kernel) or the BF16 tiles (tensor-core kernel), then rows
size_t operator_copies_bytes(const OpHandle &op, const SplitVariant &v)
{
    return at_bytes(op) + (v.kp ? round256((size_t)v.nct * 256 * v.kp) : at_bytes(op));
}

}  // namespace

const char *rbpg_split_check(const OpHandle &op, int precision, int blocks, int max_smem)
{
    if (blocks >= 2)
        return "randomized blocks handle grids of at most 1024 points";
    if (op.N > 96)
        return "the split kernel handles N <= 96";
    if (precision == 1 && 2 * op.N > 160)
        return "the tensor-core split kernel handles 2N <= 160";
    if (!split_variant(op, precision, max_smem).fn)
        return "the split kernel's shared memory exceeds the device limit";
    return "";
}

size_t rbpg_split_scratch_bytes(const OpHandle &op, int precision, int64_t P, int num_sms)
{
    if (P <= 0)
        return 0;
    const SplitVariant v = split_variant(op, precision, max_smem_dev(op.device));
    const int ctas = split_ctas(v, P, num_sms);
    if (ctas < 1)
        return 0;
    return operator_copies_bytes(op, v) + (size_t)ctas * v.ks * 3 * op.L * sizeof(float2);
}

cudaError_t launch_rbpg_split(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
{
    const SplitVariant v = split_variant(op, a.precision, max_smem_dev(op.device));
    const int ctas = split_ctas(v, a.P, num_sms);
    if (ctas < 1)
        return cudaErrorInvalidConfiguration;
    SplitParams prm;
    prm.AT = (const float2 *)a.split_scratch;
    prm.A2 = v.kp ? nullptr : (const float2 *)(a.split_scratch + at_bytes(op));
    prm.Abf = v.kp ? a.split_scratch + at_bytes(op) : nullptr;
    prm.N = op.N;
    prm.L = op.L;
    prm.NC = v.nc;
    prm.Kp = v.kp;
    prm.NCT = v.nct;
    prm.rows = (float2 *)(a.split_scratch + operator_copies_bytes(op, v));
    prm.a = a;
    const long long tot = (long long)op.N * op.L;
    k_operator_copies<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        op.A_re, op.A_im, op.N, op.L, op.lda, (float2 *)a.split_scratch,
        v.kp ? nullptr : (float2 *)(a.split_scratch + at_bytes(op)));
    if (v.kp) {
        const long long tt = (long long)v.nct * 128 * v.kp;
        k_operator_tiles<<<(unsigned)((tt + 255) / 256), 256, 0, s>>>(op.A_re, op.A_im, op.N, op.L, op.lda, v.kp,
                                                                      v.nct, a.split_scratch + at_bytes(op));
    }
    void *args[] = {(void *)&prm};
    cudaError_t e = cudaLaunchKernel(v.fn, dim3((unsigned)ctas), dim3(v.threads), args, v.smem, s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace bpdn
