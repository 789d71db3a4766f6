// Persistent iteration kernel: Algorithm 1 (RBPG with backtracking) for many
// pixels that share one operator.
//
// Block = one pixel's whole x (the patch objective separates over pixels; with
// equal block Lipschitz constants the sampling of Eq. 14 is uniform, and each
// pixel's iterate sequence does not depend on the visiting order), so every
// resident pixel takes one step of Eqs. 11-13 per sweep.
//
// Work decomposition (one CTA per SM, persistent):
//   * the CTA holds kTilePixels pixel "slots"; a slot whose pixel has stopped is
//     refilled from a global work counter (converged-slot refill);
//   * thread t owns grid index l = t for every slot: its x^k and gradient values
//     stay in registers, x^{k-1} and xbar in shared memory;
//   * A (planar FP32) stays in shared memory for the whole launch.
//
// One iteration for all slots (readings of the paper in the oracle's header):
//   A  N-space:  beta = (k-2)/(k+1); A y = A x^k + beta (A x^k - A x^{k-1});  r = A y - g
//   B  gradient: grad_l = 2 sum_n conj(A_nl) r_n                      (dense, FP32 FMA)
//   C  prox:     xbar = S_{alpha lambda}(y - alpha grad),  y = x + beta (x - x_prev)
//                (Eq. 10 read as the complex soft threshold), plus per-pixel partial
//                sums ||xbar - y||^2, ||xbar||_1, ||xbar - x||^2, ||xbar||^2
//   D  A xbar:   sum over the nonzeros of xbar only (found by warp ballots)
//   E  Eq. 15:   ||A xbar - A y||^2 <= ||xbar - y||^2 / (2 alpha)?  else alpha *= C_alpha
//                and redo C-E for that pixel; then the monotone accept test
//                F(xbar) <= F(x^k) and the stopping test ||xbar - x^k|| <= tol ||xbar||
//   G  registers: x_prev <- x, x <- xbar (accepted); finished pixels write x out
//   H  slots:    finished slots record status and take the next pixel
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int TP = kTilePixels;

struct Smem {
    size_t A_re, A_im, R, Xb, Xp, mask, G, Ax, Axp, Ay, Axb, red, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Smem smem_layout(int N, int Lpad, int lda)
{
    Smem s;
    const int NW = Lpad / 32;
    size_t o = 0;
    s.A_re = o; o = align16(o + sizeof(float) * (size_t)N * lda);
    s.A_im = o; o = align16(o + sizeof(float) * (size_t)N * lda);
    s.R = o;    o = align16(o + sizeof(float2) * (size_t)N * TP);
    s.Xb = o;   o = align16(o + sizeof(float2) * (size_t)TP * Lpad);
    s.Xp = o;   o = align16(o + sizeof(float2) * (size_t)TP * Lpad);
    s.mask = o; o = align16(o + sizeof(uint32_t) * (size_t)TP * NW);
    s.G = o;    o = align16(o + sizeof(float2) * (size_t)TP * N);
    s.Ax = o;   o = align16(o + sizeof(float2) * (size_t)TP * N);
    s.Axp = o;  o = align16(o + sizeof(float2) * (size_t)TP * N);
    s.Ay = o;   o = align16(o + sizeof(float2) * (size_t)TP * N);
    s.Axb = o;  o = align16(o + sizeof(float2) * (size_t)TP * N);
    s.red = o;  o = align16(o + sizeof(float) * (size_t)NW * TP * 4);
    s.total = o;
    return s;
}

struct Params {
    const float *A_re, *A_im;  // global planar tables [N][lda]
    int N, L, Lpad, lda;
    SolveLaunch a;
};

// Reduce v[0..K-1] (K = 32) over the 32 lanes of a warp with a fixed butterfly:
// at each step a lane keeps one half of its values, sends the other half to its
// partner and adds what it receives.  Afterwards lane `lane` holds the total of
// value number `lane` in v[0].  The summation order never depends on timing.
__device__ __forceinline__ void warp_transpose_reduce32(float (&v)[32], int lane)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
            const float keep = up ? v[off + j] : v[j];
            const float send = up ? v[j] : v[off + j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

__global__ void __launch_bounds__(512, 1) k_rbpg_fp32(Params prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = prm.N, L = prm.L, Lpad = prm.Lpad, lda = prm.lda;
    const int NW = Lpad / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SolveLaunch &a = prm.a;
    const Smem lay = smem_layout(N, Lpad, lda);
    float *sA_re = (float *)(smem_raw + lay.A_re);
    float *sA_im = (float *)(smem_raw + lay.A_im);
    float2 *sR = (float2 *)(smem_raw + lay.R);      // [N][TP]
    float2 *sXb = (float2 *)(smem_raw + lay.Xb);    // [TP][Lpad]
    float2 *sXp = (float2 *)(smem_raw + lay.Xp);    // [TP][Lpad]
    uint32_t *sMask = (uint32_t *)(smem_raw + lay.mask);  // [TP][NW]
    float2 *sG = (float2 *)(smem_raw + lay.G);      // [TP][N]
    float2 *sAx = (float2 *)(smem_raw + lay.Ax);
    float2 *sAxp = (float2 *)(smem_raw + lay.Axp);
    float2 *sAy = (float2 *)(smem_raw + lay.Ay);
    float2 *sAxb = (float2 *)(smem_raw + lay.Axb);
    float *sRed = (float *)(smem_raw + lay.red);    // [NW][TP][4]

    __shared__ long long s_pix[TP];
    __shared__ int s_k[TP], s_nbt[TP], s_nbt_it[TP], s_status[TP], s_nnz[TP];
    __shared__ int s_need[TP], s_acc[TP], s_fin[TP];
    __shared__ float s_alpha[TP], s_Fx[TP], s_lam[TP], s_beta[TP];
    __shared__ int s_nactive;
    __shared__ int s_retry[2];

    // operator tables into shared memory
    for (int i = tid; i < N * lda; i += blockDim.x) {
        sA_re[i] = prm.A_re[i];
        sA_im[i] = prm.A_im[i];
    }
    for (int i = tid; i < TP * Lpad; i += blockDim.x)
        sXp[i] = make_float2(0.f, 0.f);

    float2 x[TP];
#pragma unroll
    for (int p = 0; p < TP; ++p)
        x[p] = make_float2(0.f, 0.f);

    if (tid < TP) {
        s_fin[tid] = 1;  // every slot starts empty and asks for a pixel
        s_pix[tid] = -1;
    }
    if (tid == 0) {
        s_retry[0] = s_retry[1] = 0;
    }
    __syncthreads();

    const float alpha0 = a.alpha0;
    const float tol2 = a.tol * a.tol;

    for (;;) {
        // ---------------- H: record finished pixels, refill their slots --------------
        for (int p = warp; p < TP; p += NW) {
            if (!s_fin[p])
                continue;
            long long q;
            for (;;) {
                if (lane == 0)
                    q = (long long)atomicAdd(a.counter, 1ULL);
                q = __shfl_sync(0xffffffffu, q, 0);
                if (q >= a.P) {
                    q = -1;
                    break;
                }
                const float2 *gq = a.g + (size_t)q * N;
                float2 g0 = (lane < N) ? gq[lane] : make_float2(0.f, 0.f);
                float2 g1 = (lane + 32 < N) ? gq[lane + 32] : make_float2(0.f, 0.f);
                const bool fin = isfinite(g0.x) && isfinite(g0.y) && isfinite(g1.x) && isfinite(g1.y);
                const bool allfin = __all_sync(0xffffffffu, fin);
                if (!allfin || a.max_iter <= 0) {
                    // non-finite g (or no iteration allowed): x = 0 at once
                    float2 *xq = a.x + (size_t)q * L;
                    for (int l = lane; l < L; l += 32)
                        xq[l] = make_float2(0.f, 0.f);
                    if (lane == 0) {
                        a.status[q] = allfin ? (BPDN_PX_NOT_CONVERGED | BPDN_PX_ZERO_SOLUTION)
                                             : BPDN_PX_NONFINITE;
                        a.iters[q] = 0;
                        if (a.nbt)
                            a.nbt[q] = 0;
                        if (a.nsupp)
                            a.nsupp[q] = 0;
                    }
                    continue;
                }
                if (lane < N) {
                    sG[p * N + lane] = g0;
                    sAx[p * N + lane] = make_float2(0.f, 0.f);
                    sAxp[p * N + lane] = make_float2(0.f, 0.f);
                }
                if (lane + 32 < N) {
                    sG[p * N + lane + 32] = g1;
                    sAx[p * N + lane + 32] = make_float2(0.f, 0.f);
                    sAxp[p * N + lane + 32] = make_float2(0.f, 0.f);
                }
                float gg = g0.x * g0.x + g0.y * g0.y + g1.x * g1.x + g1.y * g1.y;
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1)
                    gg += __shfl_xor_sync(0xffffffffu, gg, off);
                if (lane == 0) {
                    s_k[p] = 1;
                    s_beta[p] = -0.5f;  // (k-2)/(k+1) at k = 1 (multiplies x - x_prev = 0)
                    s_alpha[p] = alpha0;
                    s_Fx[p] = gg;       // F(0) = ||g||^2
                    s_lam[p] = a.lam_pp ? a.lam[q] : a.lam[0];
                    s_nbt[p] = 0;
                    s_status[p] = 0;
                    s_nnz[p] = 0;
                }
                break;
            }
            if (lane == 0) {
                s_pix[p] = q;
                s_fin[p] = 0;
                s_need[p] = (q >= 0);
                s_nbt_it[p] = 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int c = 0;
            for (int p = 0; p < TP; ++p)
                c += (s_pix[p] >= 0);
            s_nactive = c;
        }
        __syncthreads();
        if (s_nactive == 0)
            break;

        // ---------------- A: N-space extrapolation and residual -------------------------
        for (int it = tid; it < TP * N; it += blockDim.x) {
            const int p = it / N, n = it - (it / N) * N;
            float2 r = make_float2(0.f, 0.f);
            if (s_pix[p] >= 0) {
                const float b = s_beta[p];
                const float2 ax = sAx[p * N + n], axp = sAxp[p * N + n];
                float2 ay = make_float2(fmaf(b, ax.x - axp.x, ax.x), fmaf(b, ax.y - axp.y, ax.y));
                sAy[p * N + n] = ay;
                const float2 gg = sG[p * N + n];
                r = make_float2(ay.x - gg.x, ay.y - gg.y);
            }
            sR[n * TP + p] = r;
        }
        __syncthreads();

        // ---------------- B: gradient 2 A^H (A y - g) for grid index l = tid -------------
        float2 gr[TP];
#pragma unroll
        for (int p = 0; p < TP; ++p)
            gr[p] = make_float2(0.f, 0.f);
        {
            const float *pre = sA_re + tid, *pim = sA_im + tid;
            const float4 *rr = (const float4 *)sR;
#pragma unroll 2
            for (int n = 0; n < N; ++n) {
                const float ar = pre[n * lda], ai = pim[n * lda];
#pragma unroll
                for (int q = 0; q < TP / 2; ++q) {
                    const float4 r2 = rr[n * (TP / 2) + q];
                    // conj(a) r = (ar rr + ai ri) + j (ar ri - ai rr)
                    gr[2 * q].x = fmaf(ar, r2.x, fmaf(ai, r2.y, gr[2 * q].x));
                    gr[2 * q].y = fmaf(ar, r2.y, fmaf(-ai, r2.x, gr[2 * q].y));
                    gr[2 * q + 1].x = fmaf(ar, r2.z, fmaf(ai, r2.w, gr[2 * q + 1].x));
                    gr[2 * q + 1].y = fmaf(ar, r2.w, fmaf(-ai, r2.z, gr[2 * q + 1].y));
                }
            }
        }
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            gr[p].x *= 2.f;
            gr[p].y *= 2.f;
        }

        // ---------------- C-E with backtracking --------------------------------------------
        for (int round = 0;; ++round) {
            // C: prox, ballots, partial sums (two halves of 8 slots keep register use low)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float part[32];
#pragma unroll
                for (int pp = 0; pp < TP / 2; ++pp) {
                    const int p = half * (TP / 2) + pp;
                    float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
                    if (s_need[p]) {
                        const float b = s_beta[p], al = s_alpha[p];
                        const float tau = al * s_lam[p];
                        const float2 xp = sXp[p * Lpad + tid];
                        const float2 y = make_float2(fmaf(b, x[p].x - xp.x, x[p].x),
                                                     fmaf(b, x[p].y - xp.y, x[p].y));
                        const float2 v = make_float2(fmaf(-al, gr[p].x, y.x),
                                                     fmaf(-al, gr[p].y, y.y));
                        const float m2 = fmaf(v.x, v.x, v.y * v.y);
                        float2 xb = make_float2(0.f, 0.f);
                        if (m2 > tau * tau) {
                            const float mag = sqrtf(m2);
                            if (mag > tau) {
                                const float sc = 1.f - tau / mag;
                                xb = make_float2(v.x * sc, v.y * sc);
                                l1 = mag - tau;
                            }
                        }
                        sXb[p * Lpad + tid] = xb;
                        const unsigned bal = __ballot_sync(0xffffffffu, xb.x != 0.f || xb.y != 0.f);
                        if (lane == 0)
                            sMask[p * NW + warp] = bal;
                        const float ex = xb.x - y.x, ey = xb.y - y.y;
                        dd = fmaf(ex, ex, ey * ey);
                        const float fx = xb.x - x[p].x, fy = xb.y - x[p].y;
                        dx = fmaf(fx, fx, fy * fy);
                        xn = fmaf(xb.x, xb.x, xb.y * xb.y);
                    }
                    part[4 * pp + 0] = dd;
                    part[4 * pp + 1] = l1;
                    part[4 * pp + 2] = dx;
                    part[4 * pp + 3] = xn;
                }
                warp_transpose_reduce32(part, lane);
                // lane holds value number `lane`: slot half*8 + lane/4, quantity lane%4
                sRed[(warp * TP + half * (TP / 2) + (lane >> 2)) * 4 + (lane & 3)] = part[0];
            }
            if (tid == 0)
                s_retry[(round + 1) & 1] = 0;
            __syncthreads();

            // D: A xbar over the nonzeros of xbar
            for (int it = tid; it < TP * N; it += blockDim.x) {
                const int p = it / N, n = it - (it / N) * N;
                if (!s_need[p])
                    continue;
                float2 acc = make_float2(0.f, 0.f);
                const float *pre = sA_re + n * lda, *pim = sA_im + n * lda;
                for (int w = 0; w < NW; ++w) {
                    uint32_t m = sMask[p * NW + w];
                    while (m) {
                        const int bit = __ffs(m) - 1;
                        m &= m - 1;
                        const int l = w * 32 + bit;
                        const float ar = pre[l], ai = pim[l];
                        const float2 xb = sXb[p * Lpad + l];
                        acc.x = fmaf(ar, xb.x, fmaf(-ai, xb.y, acc.x));
                        acc.y = fmaf(ar, xb.y, fmaf(ai, xb.x, acc.y));
                    }
                }
                sAxb[p * N + n] = acc;
            }
            __syncthreads();

            // E: line-search test, accept test, stopping test (one warp per pixel)
            for (int p = warp; p < TP; p += NW) {
                if (!s_need[p])
                    continue;
                float lhs = 0.f, res = 0.f, dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
                for (int n = lane; n < N; n += 32) {
                    const float2 xb = sAxb[p * N + n], ay = sAy[p * N + n], gg = sG[p * N + n];
                    const float d0 = xb.x - ay.x, d1 = xb.y - ay.y;
                    lhs = fmaf(d0, d0, fmaf(d1, d1, lhs));
                    const float e0 = xb.x - gg.x, e1 = xb.y - gg.y;
                    res = fmaf(e0, e0, fmaf(e1, e1, res));
                }
                if (lane < NW) {
                    const float *rd = sRed + (lane * TP + p) * 4;
                    dd = rd[0];
                    l1 = rd[1];
                    dx = rd[2];
                    xn = rd[3];
                }
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    lhs += __shfl_xor_sync(0xffffffffu, lhs, off);
                    res += __shfl_xor_sync(0xffffffffu, res, off);
                    dd += __shfl_xor_sync(0xffffffffu, dd, off);
                    l1 += __shfl_xor_sync(0xffffffffu, l1, off);
                    dx += __shfl_xor_sync(0xffffffffu, dx, off);
                    xn += __shfl_xor_sync(0xffffffffu, xn, off);
                }
                const float al = s_alpha[p];
                int decided = 0, accepted = 0;
                if (lhs <= dd / (2.f * al)) {
                    decided = 1;
                } else if (s_nbt_it[p] < a.max_bt) {
                    decided = 0;
                } else {
                    decided = 1;
                }
                if (decided) {
                    const float Fb = fmaf(s_lam[p], l1, res);
                    accepted = (Fb <= s_Fx[p]);
                    const bool conv = (dx <= tol2 * xn) || (dx == 0.f);
                    const bool last = s_k[p] >= a.max_iter;
                    // N-space state: A x^{k-1} <- A x^k, A x^{k+1} <- A xbar (accepted)
                    for (int n = lane; n < N; n += 32) {
                        const float2 ax = sAx[p * N + n];
                        sAxp[p * N + n] = ax;
                        if (accepted)
                            sAx[p * N + n] = sAxb[p * N + n];
                    }
                    if (lane == 0) {
                        if (!(lhs <= dd / (2.f * al)))
                            s_status[p] |= BPDN_PX_BT_LIMIT;
                        s_acc[p] = accepted;
                        if (accepted) {
                            s_Fx[p] = Fb;
                            int c = 0;
                            for (int w = 0; w < NW; ++w)
                                c += __popc(sMask[p * NW + w]);
                            s_nnz[p] = c;
                        }
                        if (conv) {
                            s_fin[p] = 1;
                        } else if (last) {
                            s_fin[p] = 1;
                            s_status[p] |= BPDN_PX_NOT_CONVERGED;
                        }
                        s_need[p] = 0;
                    }
                } else if (lane == 0) {
                    s_alpha[p] = al * a.c_alpha;
                    s_nbt[p] += 1;
                    s_nbt_it[p] += 1;
                    atomicAdd(&s_retry[round & 1], 1);
                }
            }
            __syncthreads();
            if (s_retry[round & 1] == 0)
                break;
        }

        // ---------------- G: registers and outputs -----------------------------------------
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            if (s_pix[p] < 0)
                continue;
            const float2 xo = x[p];
            if (s_acc[p])
                x[p] = sXb[p * Lpad + tid];
            if (s_fin[p]) {
                if (tid < L)
                    a.x[(size_t)s_pix[p] * L + tid] = x[p];
                x[p] = make_float2(0.f, 0.f);
                sXp[p * Lpad + tid] = make_float2(0.f, 0.f);
            } else {
                sXp[p * Lpad + tid] = xo;
            }
        }
        __syncthreads();
        if (tid < TP) {
            const int p = tid;
            if (s_pix[p] >= 0) {
                if (s_fin[p]) {
                    const long long q = s_pix[p];
                    int st = s_status[p];
                    if (s_nnz[p] == 0)
                        st |= BPDN_PX_ZERO_SOLUTION;
                    a.status[q] = st;
                    a.iters[q] = s_k[p];
                    if (a.nbt)
                        a.nbt[q] = s_nbt[p];
                    if (a.nsupp)
                        a.nsupp[q] = s_nnz[p];
                } else {
                    const int k = s_k[p] + 1;
                    s_k[p] = k;
                    s_beta[p] = (float)(k - 2) / (float)(k + 1);
                    s_need[p] = 1;
                    s_nbt_it[p] = 0;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t rbpg_smem_bytes(const OpHandle &op)
{
    return smem_layout(op.N, op.Lpad, op.lda).total;
}

cudaError_t launch_rbpg(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
{
    Params prm;
    prm.A_re = op.A_re;
    prm.A_im = op.A_im;
    prm.N = op.N;
    prm.L = op.L;
    prm.Lpad = op.Lpad;
    prm.lda = op.lda;
    prm.a = a;
    const size_t smem = rbpg_smem_bytes(op);
    cudaError_t e = cudaFuncSetAttribute(k_rbpg_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    long long tiles = (a.P + TP - 1) / TP;
    int grid = (int)((tiles < num_sms) ? tiles : num_sms);
    if (grid < 1)
        grid = 1;
    k_rbpg_fp32<<<grid, op.Lpad, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bpdn
