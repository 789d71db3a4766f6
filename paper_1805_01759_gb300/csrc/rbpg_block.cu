// Algorithm 1 with randomized blocks of one pixel's elevation grid (Eqs. 13-14), FP32,
// one warp per pixel.  The library's default reading makes a block one pixel (every
// pixel takes a full step each sweep, k_rbpg); this kernel is the other reading, in which
// the blocks are J contiguous pieces of the grid, block j = [floor(jL/J), floor((j+1)L/J)):
//
//   i_k      drawn with P_i = L_i / sum_j L_j (Eq. 14; L_i = 2 lambda_max(A_i^H A_i) from
//            the draw table), by SplitMix64 (Steele, Lea and Flood 2014) started at state
//            seed + p * 2^40 for pixel p: u = (next >> 11) 2^-53, i = first j with u < cum_j
//   y        = x, and on block i  y_i = x_i + beta_k (x_i - x_i^{k-1}), beta_k = (k-2)/(k+1)
//            (x^{k-1} is the previous iterate; since x^k - x^{k-1} lives on the block
//            updated at k-1, A y = A x + beta_k (A x^k - A x^{k-1}) when i_k = i_{k-1} and
//            A y = A x otherwise)
//   xbar     = y, and on block i  xbar_i = S_{alpha_i lambda}(y_i - alpha_i 2 A_i^H (A y - g))
//            with Eq. 15 on block i, ||A (xbar - y)||^2 <= ||xbar - y||^2 / (2 alpha_i), else
//            alpha_i *= C_alpha; each block carries its own alpha_i (Eq. 13's alpha_{i_k})
//   accept   xbar when F(xbar) <= F(x^k)
//   stop     once every block has taken a small step (||xbar - x^k|| <= tol ||xbar||)
//            since the last step that was not small, or after max_iter * J iterations
//
// Per warp in shared memory: x and x^{k-1} over the grid, y, the block gradient and the
// candidate over the drawn block, the list of grid points where the candidate moved,
// and the N-vectors g and r = A y - g.  A x, A x^{k-1} stay in registers (lane n holds
// rows n and n + 32).  A is read in FP32 from the operator's planar tables.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int WPB = 4;  // warps (pixels) per block

struct BlkLayout {
    int x, xp, yb, gb, xbb, dl, g, r, alpha, bytes;
};

__host__ __device__ inline int align16(int v) { return (v + 15) & ~15; }

__host__ __device__ inline BlkLayout blk_layout(int N, int L, int J)
{
    const int B = (L + J - 1) / J;  // largest block
    BlkLayout s;
    int o = 0;
    s.x = o;     o = align16(o + 8 * L);
    s.xp = o;    o = align16(o + 8 * L);
    s.yb = o;    o = align16(o + 8 * B);
    s.gb = o;    o = align16(o + 8 * B);
    s.xbb = o;   o = align16(o + 8 * B);
    s.dl = o;    o = align16(o + 4 * B);
    s.g = o;     o = align16(o + 8 * N);
    s.r = o;     o = align16(o + 8 * N);
    s.alpha = o; o = align16(o + 4 * 8);
    s.bytes = o;
    return s;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ uint64_t sm64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(WPB * 32) k_rbpg_block(const float *__restrict__ A_re,
                                                         const float *__restrict__ A_im, int lda, int N,
                                                         int L, SolveLaunch a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int J = a.blocks;
    const BlkLayout lay = blk_layout(N, L, J);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)warp * lay.bytes;
    float2 *sx = (float2 *)(base + lay.x), *sxp = (float2 *)(base + lay.xp);
    float2 *syb = (float2 *)(base + lay.yb), *sgb = (float2 *)(base + lay.gb), *sxbb = (float2 *)(base + lay.xbb);
    int *sdl = (int *)(base + lay.dl);
    float2 *sg = (float2 *)(base + lay.g), *sr = (float2 *)(base + lay.r);
    float *salpha = (float *)(base + lay.alpha);
    const long long p = (long long)blockIdx.x * WPB + warp;
    if (p >= a.P)
        return;

    // g, finiteness
    float2 gv[2];
    bool fin = true;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int n = lane + 32 * c;
        gv[c] = make_float2(0.f, 0.f);
        if (n < N) {
            gv[c] = a.g[(size_t)p * N + n];
            sg[n] = gv[c];
            fin = fin && isfinite(gv[c].x) && isfinite(gv[c].y);
        }
    }
    const bool allfin = __all_sync(0xffffffffu, fin);
    float2 *xo = a.x + (size_t)p * L;
    if (!allfin || a.max_iter <= 0) {
        for (int l = lane; l < L; l += 32)
            xo[l] = make_float2(0.f, 0.f);
        if (lane == 0) {
            a.status[p] = allfin ? (BPDN_PX_NOT_CONVERGED | BPDN_PX_ZERO_SOLUTION) : BPDN_PX_NONFINITE;
            a.iters[p] = 0;
            if (a.nbt)
                a.nbt[p] = 0;
            if (a.nsupp)
                a.nsupp[p] = 0;
        }
        return;
    }
    for (int l = lane; l < L; l += 32) {
        sx[l] = make_float2(0.f, 0.f);
        sxp[l] = make_float2(0.f, 0.f);
    }
    if (lane < J)
        salpha[lane] = a.alpha0;
    double cum[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        cum[j] = (j < J) ? a.cum[j] : 2.0;
    const float lam = a.lam_pp ? a.lam[p] : a.lam[0];
    const float tol2 = a.tol * a.tol;
    float Fx = warp_sum_f(gv[0].x * gv[0].x + gv[0].y * gv[0].y + gv[1].x * gv[1].x + gv[1].y * gv[1].y);
    float2 Ax[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float2 Axp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    uint64_t state = (uint64_t)a.seed + ((uint64_t)p << 40);
    const unsigned all_mask = (1u << J) - 1u;
    unsigned done_mask = 0;
    int prev = -1, status = 0, nbt_total = 0, k = 0;
    bool stopped = false;
    __syncwarp();

    const int kmax = a.max_iter * J;
    for (k = 1; k <= kmax; ++k) {
        const double u = (double)(sm64_next(state) >> 11) * 0x1.0p-53;
        int i = J - 1;
        for (int j = J - 2; j >= 0; --j)
            if (u < cum[j])
                i = j;
        const int lo = (int)(((long long)i * L) / J), hi = (int)(((long long)(i + 1) * L) / J);
        const int nb = hi - lo;
        const float beta = (float)(k - 2) / (float)(k + 1);
        const bool same = (i == prev);

        // A y and r = A y - g
        float2 Ay[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int n = lane + 32 * c;
            Ay[c] = same ? make_float2(fmaf(beta, Ax[c].x - Axp[c].x, Ax[c].x), fmaf(beta, Ax[c].y - Axp[c].y, Ax[c].y))
                         : Ax[c];
            if (n < N)
                sr[n] = make_float2(Ay[c].x - gv[c].x, Ay[c].y - gv[c].y);
        }
        __syncwarp();
        // y and 2 A_i^H (A y - g) on the block (x - x^{k-1} is zero on it unless same)
        for (int e = lane; e < nb; e += 32) {
            const int l = lo + e;
            const float2 xv = sx[l], xpv = sxp[l];
            syb[e] = make_float2(fmaf(beta, xv.x - xpv.x, xv.x), fmaf(beta, xv.y - xpv.y, xv.y));
            float gx = 0.f, gy = 0.f;
            for (int n = 0; n < N; ++n) {
                const float ar = __ldg(A_re + (size_t)n * lda + l), ai = __ldg(A_im + (size_t)n * lda + l);
                const float2 rv = sr[n];
                gx = fmaf(ar, rv.x, fmaf(ai, rv.y, gx));
                gy = fmaf(ar, rv.y, fmaf(-ai, rv.x, gy));
            }
            sgb[e] = make_float2(2.f * gx, 2.f * gy);
        }
        __syncwarp();

        // prox on the block with backtracking (Eq. 15)
        int nbt = 0;
        float2 Ad[2];
        for (;;) {
            const float al = salpha[i];
            const float tau = al * lam;
            float dd = 0.f;
            int cnt = 0;
            for (int e0 = 0; e0 < nb; e0 += 32) {
                const int e = e0 + lane;
                bool moved = false;
                if (e < nb) {
                    const float2 y = syb[e], g2 = sgb[e];
                    const float vx = fmaf(-al, g2.x, y.x), vy = fmaf(-al, g2.y, y.y);
                    const float m2 = fmaf(vx, vx, vy * vy);
                    const float sc = fmaf(-tau, rsqrtf(m2), 1.f);
                    const float2 xb = (sc > 0.f) ? make_float2(vx * sc, vy * sc) : make_float2(0.f, 0.f);
                    sxbb[e] = xb;
                    const float ex = xb.x - y.x, ey = xb.y - y.y;
                    dd = fmaf(ex, ex, fmaf(ey, ey, dd));
                    moved = (ex != 0.f || ey != 0.f);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, moved);
                if (moved)
                    sdl[cnt + __popc(bal & ((1u << lane) - 1u))] = e;
                cnt += __popc(bal);
            }
            dd = warp_sum_f(dd);
            __syncwarp();
            // A (xbar - y) over the grid points that moved
#pragma unroll
            for (int c = 0; c < 2; ++c)
                Ad[c] = make_float2(0.f, 0.f);
            for (int j = 0; j < cnt; ++j) {
                const int e = sdl[j];
                const int l = lo + e;
                const float2 xb = sxbb[e], y = syb[e];
                const float dx = xb.x - y.x, dy = xb.y - y.y;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int n = lane + 32 * c;
                    if (n < N) {
                        const float ar = __ldg(A_re + (size_t)n * lda + l), ai = __ldg(A_im + (size_t)n * lda + l);
                        Ad[c].x = fmaf(ar, dx, fmaf(-ai, dy, Ad[c].x));
                        Ad[c].y = fmaf(ar, dy, fmaf(ai, dx, Ad[c].y));
                    }
                }
            }
            const float lhs = warp_sum_f(Ad[0].x * Ad[0].x + Ad[0].y * Ad[0].y + Ad[1].x * Ad[1].x + Ad[1].y * Ad[1].y);
            if (lhs <= dd / (2.f * al))
                break;
            if (nbt >= a.max_bt) {
                status |= BPDN_PX_BT_LIMIT;
                break;
            }
            __syncwarp();
            if (lane == 0)
                salpha[i] = al * a.c_alpha;
            __syncwarp();
            ++nbt;
        }
        nbt_total += nbt;

        // F(xbar), the step and ||xbar||
        float2 Axb[2];
        float res = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int n = lane + 32 * c;
            Axb[c] = make_float2(Ay[c].x + Ad[c].x, Ay[c].y + Ad[c].y);
            if (n < N) {
                const float ex = Axb[c].x - gv[c].x, ey = Axb[c].y - gv[c].y;
                res = fmaf(ex, ex, fmaf(ey, ey, res));
            }
        }
        res = warp_sum_f(res);
        float l1 = 0.f, xn = 0.f, dxs = 0.f;
        for (int l = lane; l < L; l += 32) {
            const float2 xv = sx[l];
            float2 v = xv;
            if (l >= lo && l < hi) {
                v = sxbb[l - lo];
                const float fx = v.x - xv.x, fy = v.y - xv.y;
                dxs = fmaf(fx, fx, fmaf(fy, fy, dxs));
            }
            const float m2 = fmaf(v.x, v.x, v.y * v.y);
            xn += m2;
            l1 += sqrtf(m2);
        }
        l1 = warp_sum_f(l1);
        xn = warp_sum_f(xn);
        dxs = warp_sum_f(dxs);
        const float Fb = fmaf(lam, l1, res);
        const bool accepted = (Fb <= Fx);
        const bool small = (dxs <= tol2 * xn) || (dxs == 0.f);

        // x^{k-1} <- x^k, then x^{k+1}
        for (int l = lane; l < L; l += 32)
            sxp[l] = sx[l];
        __syncwarp();
        if (accepted) {
            for (int e = lane; e < nb; e += 32)
                sx[lo + e] = sxbb[e];
            Fx = Fb;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            Axp[c] = Ax[c];
            if (accepted)
                Ax[c] = Axb[c];
        }
        done_mask = small ? (done_mask | (1u << i)) : 0u;
        prev = i;
        __syncwarp();
        if (done_mask == all_mask) {
            stopped = true;
            break;
        }
    }
    if (!stopped) {
        status |= BPDN_PX_NOT_CONVERGED;
        k = kmax;
    }
    int nz = 0;
    for (int l = lane; l < L; l += 32) {
        const float2 v = sx[l];
        xo[l] = v;
        nz += (v.x != 0.f || v.y != 0.f);
    }
    nz = (int)__reduce_add_sync(0xffffffffu, (unsigned)nz);
    if (lane == 0) {
        a.status[p] = (nz == 0) ? (status | BPDN_PX_ZERO_SOLUTION) : status;
        a.iters[p] = k;
        if (a.nbt)
            a.nbt[p] = nbt_total;
        if (a.nsupp)
            a.nsupp[p] = nz;
    }
}

}  // namespace

const char *rbpg_block_check(const OpHandle &op, int blocks, int max_smem)
{
    if (blocks < 2 || blocks > 8)
        return "blocks must lie in 2..8";
    if (op.N > 64)
        return "the randomized-block kernel keeps two rows of N per lane: N <= 64";
    if (op.L < blocks)
        return "fewer grid points than blocks";
    if ((size_t)WPB * blk_layout(op.N, op.L, blocks).bytes > (size_t)max_smem)
        return "the per-pixel iterates of four pixels do not fit in shared memory";
    return "";
}

cudaError_t launch_rbpg_block(const OpHandle &op, const SolveLaunch &a, cudaStream_t s)
{
    if (a.P <= 0)
        return cudaSuccess;
    const size_t smem = (size_t)WPB * blk_layout(op.N, op.L, a.blocks).bytes;
    cudaError_t e = cudaFuncSetAttribute(k_rbpg_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long blocks = (a.P + WPB - 1) / WPB;
    k_rbpg_block<<<(unsigned)blocks, WPB * 32, smem, s>>>(op.A_re, op.A_im, op.lda, op.N, op.L, a);
    return cudaGetLastError();
}

}  // namespace bpdn
