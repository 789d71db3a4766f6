// Split-grid iteration kernel: Algorithm 1 (RBPG with backtracking, Eqs. 11-15) in FP32 for
// grids too large for one thread per grid point in a CTA (the multi-component grids of Eq. 4,
// L up to BPDN_MAX_L).  A CTA holds kSlots pixels; its eight warps walk the grid in 32-point
// chunks (warp w takes chunks w, w + 8, ...), and every operator load of the gradient
// serves all slots.  x^k, x^{k-1} and xbar of a slot are rows of the CTA's scratch in
// global memory, gated by per-chunk nonzero masks in shared memory: only nonzeros are read
// or written, so the rows cost traffic in proportion to the support, not to L.
//
// One sweep:
//   1. per chunk and lane (one grid point l): the gradient sum_n conj(A_nl) r_n of every
//      slot from the FP32 tables (coalesced over l; r in shared memory), then per slot the
//      extrapolation y = x + beta (x - x^{k-1}), the complex soft threshold of
//      v = y - 2 alpha grad, the sums of Eq. 15, F and the stopping test, and A xbar over
//      the chunk's nonzeros (ascending l) from the transposed table (coalesced over n);
//   2. warp p decides slot p: the warps' sums and A xbar added in warp order, Eq. 15, the
//      monotone accept, the stopping test, the N-space update (A x^k, A x^{k-1}, A y and the
//      next residual); a finished pixel's x goes to its output row and the slot is refilled.
// Every sum has a fixed order, so results do not depend on timing.  There are no waits on
// other CTAs or on asynchronous units: only CTA barriers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kWarps = 8;   // warps per CTA
constexpr int kSlots = 4;   // pixels per CTA
constexpr int kNCH = 3;     // rows n = lane + 32 c per lane (N <= 96)
constexpr int kThreads = 32 * kWarps;

struct SplitParams {
    const float *A_re, *A_im;  // planar FP32 tables [N][lda]
    const float2 *AT;          // transposed FP32 table [L][N]
    int N, L, lda, NC;
    float2 *rows;              // [ctas][kSlots][3][L]
    SolveLaunch a;
};

// per-slot state (shared memory)
struct SlotSt {
    long long pix;  // -1: the slot is empty
    int k, nbt, nbt_it, status, nnz;
    float alpha, Fx, lam, beta;
    int bx, bxp, bb;  // row buffers of x^k, x^{k-1} and xbar (bx == bxp after a rejected step)
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// shared memory carve-up (float2 / float4 / uint32 sections, 16-byte aligned)
struct SplitSmem {
    float2 *G, *Ax, *Axp, *Ay;  // [kSlots][N]
    float2 *R;                  // [N][kSlots]: r_n of every slot, slot-minor
    float2 *Wacc;               // [kSlots][kWarps][N]
    float4 *Wsum;               // [kSlots][kWarps]: dd, l1, dx, xn
    int *Wnnz;                  // [kSlots][kWarps]
    uint32_t *M;                // [kSlots][3][NC] nonzero masks of the row buffers
    SlotSt *S;                  // [kSlots]
};

__host__ __device__ inline size_t split_smem_bytes(int N, int NC)
{
    size_t b = 0;
    b += (size_t)4 * kSlots * N * sizeof(float2);
    b += (size_t)N * kSlots * sizeof(float2);
    b += (size_t)kSlots * kWarps * N * sizeof(float2);
    b += (size_t)kSlots * kWarps * sizeof(float4);
    b += (size_t)kSlots * kWarps * sizeof(int);
    b += (size_t)kSlots * 3 * NC * sizeof(uint32_t);
    b = (b + 15) / 16 * 16;
    b += (size_t)kSlots * sizeof(SlotSt);
    return b;
}

__device__ __forceinline__ SplitSmem carve(unsigned char *base, int N, int NC)
{
    SplitSmem s;
    unsigned char *p = base;
    s.G = (float2 *)p;
    p += (size_t)kSlots * N * sizeof(float2);
    s.Ax = (float2 *)p;
    p += (size_t)kSlots * N * sizeof(float2);
    s.Axp = (float2 *)p;
    p += (size_t)kSlots * N * sizeof(float2);
    s.Ay = (float2 *)p;
    p += (size_t)kSlots * N * sizeof(float2);
    s.R = (float2 *)p;
    p += (size_t)N * kSlots * sizeof(float2);
    s.Wacc = (float2 *)p;
    p += (size_t)kSlots * kWarps * N * sizeof(float2);
    s.Wsum = (float4 *)p;
    p += (size_t)kSlots * kWarps * sizeof(float4);
    s.Wnnz = (int *)p;
    p += (size_t)kSlots * kWarps * sizeof(int);
    s.M = (uint32_t *)p;
    p += (size_t)kSlots * 3 * NC * sizeof(uint32_t);
    p = base + ((size_t)(p - base) + 15) / 16 * 16;
    s.S = (SlotSt *)p;
    return s;
}

// A^T in FP32: AT[l][n] = A_nl, for the gather of A xbar (lanes over n)
__global__ void k_transpose_a(const float *__restrict__ A_re, const float *__restrict__ A_im, int N, int L, int lda,
                              float2 *__restrict__ AT)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * L)
        return;
    const int l = (int)(i / N), n = (int)(i % N);
    AT[i] = make_float2(A_re[(size_t)n * lda + l], A_im[(size_t)n * lda + l]);
}

// Refill slot p (warp p) from the work counter: x^0 = x^{-1} = 0, so A y = 0 and r = -g.
// Pixels with a non-finite g (or a solve with max_iter <= 0) get x = 0 at once.  With no
// pixel left the slot is marked empty and its residual column zeroed, so that the shared
// gradient loop adds nothing for it.
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
                sm.R[n * kSlots + p] = make_float2(0.f, 0.f);
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
            sm.R[n * kSlots + p] = make_float2(-v.x, -v.y);
            gg2 = fmaf(v.x, v.x, fmaf(v.y, v.y, gg2));
        }
        gg2 = warp_sum(gg2);
        // x^k (buffer 0) and x^{k-1} (buffer 1) are zero; buffer 2 takes xbar
        for (int c = lane; c < NC; c += 32) {
            sm.M[(p * 3 + 0) * NC + c] = 0u;
            sm.M[(p * 3 + 1) * NC + c] = 0u;
        }
        if (lane == 0) {
            S.pix = (long long)q;
            S.k = 1;
            S.nbt = 0;
            S.nbt_it = 0;
            S.status = 0;
            S.nnz = 0;
            S.alpha = a.alpha0;
            S.Fx = gg2;  // F(0) = ||g||^2
            S.lam = a.lam_pp ? a.lam[q] : a.lam[0];
            S.beta = 0.f;  // x^0 - x^{-1} = 0
            S.bx = 0;
            S.bxp = 1;
            S.bb = 2;
        }
        __syncwarp();
        return;
    }
}

// Warp p: the end of slot p's sweep (Eq. 15, accept, stopping test, N-space update).
__device__ void decide_slot(const SplitParams &prm, const SplitSmem &sm, float2 *rows, int p, int lane)
{
    const SolveLaunch &a = prm.a;
    const int N = prm.N, L = prm.L, NC = prm.NC;
    SlotSt &S = sm.S[p];
    // the warps' sums, in warp order
    float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
    int nnz = 0;
    for (int v = 0; v < kWarps; ++v) {
        const float4 t = sm.Wsum[p * kWarps + v];
        dd += t.x;
        l1 += t.y;
        dx += t.z;
        xn += t.w;
        nnz += sm.Wnnz[p * kWarps + v];
    }
    float2 axb[kNCH], gg[kNCH];
    float lhs = 0.f, res = 0.f;
#pragma unroll
    for (int c = 0; c < kNCH; ++c) {
        axb[c] = make_float2(0.f, 0.f);
        gg[c] = make_float2(0.f, 0.f);
        const int n = lane + 32 * c;
        if (n < N) {
            for (int v = 0; v < kWarps; ++v) {
                const float2 t = sm.Wacc[(p * kWarps + v) * N + n];
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
    const int nbt_it = S.nbt_it, k = S.k, obx = S.bx, obb = S.bb;
    const long long q = S.pix;
    const bool bt_ok = lhs <= dd / (2.f * al);
    __syncwarp();  // every lane has read the slot state lane 0 updates below
    if (!bt_ok && nbt_it < a.max_bt) {
        // Eq. 15 failed: the next sweep redoes the prox with the smaller step
        if (lane == 0) {
            S.alpha = al * a.c_alpha;
            S.nbt += 1;
            S.nbt_it = nbt_it + 1;
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
        for (int c = 0; c < kNCH; ++c) {
            const int n = lane + 32 * c;
            if (n < N) {
                const float2 axo = sm.Ax[p * N + n];
                const float2 axn = accepted ? axb[c] : axo;
                sm.Axp[p * N + n] = axo;
                sm.Ax[p * N + n] = axn;
                const float2 ayn =
                    make_float2(fmaf(beta_n, axn.x - axo.x, axn.x), fmaf(beta_n, axn.y - axo.y, axn.y));
                sm.Ay[p * N + n] = ayn;
                sm.R[n * kSlots + p] = make_float2(ayn.x - gg[c].x, ayn.y - gg[c].y);
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
            S.beta = beta_n;
            S.bx = nbx;
            S.bxp = obx;
            S.bb = nbb;
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
    refill_slot(prm, sm, p, lane);
}

__global__ void __launch_bounds__(kThreads, 2) k_rbpg_split(const __grid_constant__ SplitParams prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = prm.N, L = prm.L, lda = prm.lda, NC = prm.NC;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SplitSmem sm = carve(smem_raw, N, NC);
    float2 *rows = prm.rows + (size_t)blockIdx.x * kSlots * 3 * L;
    const float *__restrict__ A_re = prm.A_re;
    const float *__restrict__ A_im = prm.A_im;
    if (w < kSlots)
        refill_slot(prm, sm, w, lane);
    __syncthreads();
    for (;;) {
        // this sweep's slot parameters
        bool act[kSlots];
        float beta[kSlots], a2[kSlots], tau[kSlots];
        int bx[kSlots], bxp[kSlots], bb[kSlots];
        bool any = false;
#pragma unroll
        for (int p = 0; p < kSlots; ++p) {
            const SlotSt &S = sm.S[p];
            act[p] = S.pix >= 0;
            any = any || act[p];
            beta[p] = S.beta;
            a2[p] = 2.f * S.alpha;
            tau[p] = S.alpha * S.lam;
            bx[p] = S.bx;
            bxp[p] = S.bxp;
            bb[p] = S.bb;
        }
        if (!any)
            break;
        float sdd[kSlots], sl1[kSlots], sdx[kSlots], sxn[kSlots];
        int snz[kSlots];
        float2 acc[kSlots][kNCH];
#pragma unroll
        for (int p = 0; p < kSlots; ++p) {
            sdd[p] = sl1[p] = sdx[p] = sxn[p] = 0.f;
            snz[p] = 0;
#pragma unroll
            for (int c = 0; c < kNCH; ++c)
                acc[p][c] = make_float2(0.f, 0.f);
        }
        for (int c = w; c < NC; c += kWarps) {
            const int l = 32 * c + lane;
            const bool inl = l < L;
            // gradient of every slot: one pair of operator loads feeds all of them
            float gx[kSlots], gy[kSlots];
#pragma unroll
            for (int p = 0; p < kSlots; ++p)
                gx[p] = gy[p] = 0.f;
            if (inl) {
#pragma unroll 4
                for (int n = 0; n < N; ++n) {
                    const float ar = __ldg(A_re + (size_t)n * lda + l), ai = __ldg(A_im + (size_t)n * lda + l);
#pragma unroll
                    for (int p = 0; p < kSlots; p += 2) {
                        const float4 r2 = *(const float4 *)(sm.R + n * kSlots + p);  // r_n of slots p, p+1
                        // conj(a) r = (ar r.x + ai r.y) + j (ar r.y - ai r.x)
                        gx[p] = fmaf(ar, r2.x, fmaf(ai, r2.y, gx[p]));
                        gy[p] = fmaf(ar, r2.y, fmaf(-ai, r2.x, gy[p]));
                        gx[p + 1] = fmaf(ar, r2.z, fmaf(ai, r2.w, gx[p + 1]));
                        gy[p + 1] = fmaf(ar, r2.w, fmaf(-ai, r2.z, gy[p + 1]));
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < kSlots; ++p) {
                if (!act[p])
                    continue;  // the same for the whole CTA
                const uint32_t mx = sm.M[(p * 3 + bx[p]) * NC + c];
                const uint32_t mxp = sm.M[(p * 3 + bxp[p]) * NC + c];
                float xbx = 0.f, xby = 0.f;
                bool nz = false;
                if (inl) {
                    const float2 xv =
                        ((mx >> lane) & 1u) ? rows[((size_t)p * 3 + bx[p]) * L + l] : make_float2(0.f, 0.f);
                    const float2 xpv =
                        ((mxp >> lane) & 1u) ? rows[((size_t)p * 3 + bxp[p]) * L + l] : make_float2(0.f, 0.f);
                    const float yx = fmaf(beta[p], xv.x - xpv.x, xv.x), yy = fmaf(beta[p], xv.y - xpv.y, xv.y);
                    const float vx = fmaf(-a2[p], gx[p], yx), vy = fmaf(-a2[p], gy[p], yy);
                    const float m2 = fmaf(vx, vx, vy * vy);
                    // soft threshold (Eq. 12): scale 1 - tau / |v| where that is positive
                    const float rs = rsqrtf(m2);
                    const float sc = fmaf(-tau[p], rs, 1.f);
                    nz = sc > 0.f;
                    if (nz) {
                        xbx = vx * sc;
                        xby = vy * sc;
                        sl1[p] += fmaf(m2, rs, -tau[p]);
                        rows[((size_t)p * 3 + bb[p]) * L + l] = make_float2(xbx, xby);
                    }
                    const float ex = xbx - yx, ey = xby - yy;
                    sdd[p] = fmaf(ex, ex, fmaf(ey, ey, sdd[p]));
                    const float fx = xbx - xv.x, fy = xby - xv.y;
                    sdx[p] = fmaf(fx, fx, fmaf(fy, fy, sdx[p]));
                    sxn[p] = fmaf(xbx, xbx, fmaf(xby, xby, sxn[p]));
                }
                const unsigned bal = __ballot_sync(0xffffffffu, nz);
                if (lane == 0)
                    sm.M[(p * 3 + bb[p]) * NC + c] = bal;
                snz[p] += __popc(bal);
                // this chunk's share of A xbar, ascending l; lane n owns rows n + 32 c
                unsigned m = bal;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    const float xr = __shfl_sync(0xffffffffu, xbx, j), xi = __shfl_sync(0xffffffffu, xby, j);
                    const float2 *at = prm.AT + (size_t)(32 * c + j) * N;
#pragma unroll
                    for (int cc = 0; cc < kNCH; ++cc) {
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
#pragma unroll
        for (int p = 0; p < kSlots; ++p) {
            if (!act[p])
                continue;
            const float dd = warp_sum(sdd[p]), l1 = warp_sum(sl1[p]);
            const float dx = warp_sum(sdx[p]), xn = warp_sum(sxn[p]);
            if (lane == 0) {
                sm.Wsum[p * kWarps + w] = make_float4(dd, l1, dx, xn);
                sm.Wnnz[p * kWarps + w] = snz[p];
            }
#pragma unroll
            for (int cc = 0; cc < kNCH; ++cc) {
                const int n = lane + 32 * cc;
                if (n < N)
                    sm.Wacc[(p * kWarps + w) * N + n] = acc[p][cc];
            }
        }
        __syncthreads();
        if (w < kSlots && sm.S[w].pix >= 0)  // the slots of this sweep: unchanged since its start
            decide_slot(prm, sm, rows, w, lane);
        __syncthreads();
    }
}

}  // namespace

// CTAs of a split launch on this device: as many as fit (at most one per kSlots pixels)
static int split_ctas(const OpHandle &op, int64_t P, int num_sms, size_t smem)
{
    int per_sm = 0;
    if (cudaFuncSetAttribute(k_rbpg_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbpg_split, kThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    (void)op;
    const int64_t want = (P + kSlots - 1) / kSlots;
    return (int)std::min<int64_t>((int64_t)per_sm * num_sms, want);
}

const char *rbpg_split_check(const OpHandle &op, int precision, int blocks, int max_smem)
{
    if (precision != 0)
        return "grids of more than 1024 points run in FP32 only (precision 0)";
    if (blocks >= 2)
        return "randomized blocks handle grids of at most 1024 points";
    if (op.N > 32 * kNCH)
        return "the split kernel handles N <= 96";
    const int NC = (op.L + 31) / 32;
    if (split_smem_bytes(op.N, NC) > (size_t)max_smem)
        return "the split kernel's shared memory exceeds the device limit";
    return "";
}

size_t rbpg_split_scratch_bytes(const OpHandle &op, int64_t P, int num_sms)
{
    if (P <= 0)
        return 0;
    const int NC = (op.L + 31) / 32;
    const int ctas = split_ctas(op, P, num_sms, split_smem_bytes(op.N, NC));
    if (ctas < 1)
        return 0;
    const size_t at = ((size_t)op.L * op.N * sizeof(float2) + 255) / 256 * 256;
    return at + (size_t)ctas * kSlots * 3 * op.L * sizeof(float2);
}

cudaError_t launch_rbpg_split(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
{
    const int NC = (op.L + 31) / 32;
    const size_t smem = split_smem_bytes(op.N, NC);
    const int ctas = split_ctas(op, a.P, num_sms, smem);
    if (ctas < 1)
        return cudaErrorInvalidConfiguration;
    SplitParams prm;
    prm.A_re = op.A_re;
    prm.A_im = op.A_im;
    prm.AT = (const float2 *)a.split_scratch;
    prm.N = op.N;
    prm.L = op.L;
    prm.lda = op.lda;
    prm.NC = NC;
    prm.rows = (float2 *)(a.split_scratch + ((size_t)op.L * op.N * sizeof(float2) + 255) / 256 * 256);
    prm.a = a;
    const long long tot = (long long)op.N * op.L;
    k_transpose_a<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(op.A_re, op.A_im, op.N, op.L, op.lda,
                                                                (float2 *)a.split_scratch);
    k_rbpg_split<<<(unsigned)ctas, kThreads, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bpdn
