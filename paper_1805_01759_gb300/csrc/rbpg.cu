// Persistent iteration kernel: Algorithm 1 (RBPG with backtracking) for many
// pixels that share one operator.
//
// Block = one pixel's whole x (the patch objective separates over pixels; with
// equal block Lipschitz constants the sampling of Eq. 14 is uniform, and each
// pixel's iterate sequence does not depend on the visiting order), so every
// resident pixel takes one step of Eqs. 11-13 per sweep.
//
// Work decomposition (one CTA per SM, persistent):
//   * A (FP32, complex interleaved) stays in shared memory for the whole launch and
//     is shared by G independent slot groups; each group has its own Lpad threads,
//     TPG pixel slots, slot state and named barrier, so the latency-bound phases
//     of one group overlap the arithmetic of another;
//   * a slot whose pixel has stopped is refilled from a global work counter
//     (converged-slot refill);
//   * thread l of a group owns grid index l of its group's slots: x^k and the
//     gradient stay in registers, x^{k-1} and xbar in shared memory.
//
// One iteration of a group (readings of the paper in the oracle's header):
//   B  gradient: sum_n conj(A_nl) r_n, r = A y - g   (dense; packed f32x2 FMA; the
//                factor 2 of grad f = 2 A^H (A y - g) is folded into the step)
//   C  prox:     xbar = S_{alpha lambda}(y - alpha grad),  y = x + beta (x - x_prev),
//                beta = (k-2)/(k+1) (Eq. 10 read as the complex soft threshold), plus
//                per-slot partial sums ||xbar - y||^2, ||xbar||_1, ||xbar - x||^2, ||xbar||^2
//   ---- group barrier
//   A xbar: slots with few nonzeros sum over them in the next phase; slots with
//                many get a dense pass of the whole group (partial sums over
//                ranges of l, added in a fixed order) ---- group barrier
//   DE one half-warp per slot: Eq. 15 ||A xbar - A y||^2 <= ||xbar - y||^2 / (2 alpha),
//                else alpha *= C_alpha and the slot redoes C-DE; then the monotone
//                accept test F(xbar) <= F(x^k), the stopping test
//                ||xbar - x^k|| <= tol ||xbar||, and the next iteration's
//                r: A y = A x^k + beta (A x^k - A x^{k-1}) (linearity)
//   ---- group barrier
//   G  registers: x_prev <- x, x <- xbar (accepted); finished slots write x out
//   H  (only when a slot finished) record status and take the next pixel
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int TPG = 8;          // pixel slots per group
constexpr int kMaxGroups = 4;   // groups per CTA (named barriers 1..kMaxGroups)
constexpr int kMaxThreads = 832;  // threads per CTA: the register budget is 65536 / 832
constexpr int kSparseMax = 24;  // A xbar by gathering when xbar has at most this many nonzeros
constexpr int kChunks = 4;      // ranges of l per slot in the dense A xbar pass (fixed, so the
                                // summation order depends on nothing but the pixel)

// slot flags
constexpr int F_ACTIVE = 1, F_ACC = 2, F_FIN = 4;

struct SlotState {
    long long pix[TPG];
    int k[TPG], nbt[TPG], nbt_it[TPG], status[TPG], nnz[TPG], flags[TPG];
    int need[2][TPG];  // [iteration parity][slot]: evaluate the slot in this sweep / retry round
    int cnt[2][TPG];   // [sweep parity][slot]: nonzeros of xbar
    int dense[TPG];    // slots whose A xbar comes from the dense pass this sweep
    float alpha[TPG], Fx[TPG], lam[TPG];
    float4 par[TPG];   // (beta, 2 alpha, alpha lambda, unused)
    int retry[3];      // by retry round mod 3: reset two barriers after its last read
    int ndense, nfin, nactive;
};

// shared-memory layout: A once, then one block of arrays per group
struct GroupLayout {
    size_t Rre, Rim, Xb, Xp, mask, G, Ax, Axp, Ay, red, part, st, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GroupLayout group_layout(int N, int Lpad)
{
    GroupLayout s;
    const int NW = Lpad / 32;
    size_t o = 0;
    s.Rre = o;  o = align16(o + sizeof(float) * (size_t)N * TPG);
    s.Rim = o;  o = align16(o + sizeof(float) * (size_t)N * TPG);
    s.Xb = o;   o = align16(o + sizeof(float2) * (size_t)TPG * Lpad);
    s.Xp = o;   o = align16(o + sizeof(float2) * (size_t)TPG * Lpad);
    s.mask = o; o = align16(o + sizeof(uint32_t) * (size_t)TPG * NW);
    s.G = o;    o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Ax = o;   o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Axp = o;  o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Ay = o;   o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.red = o;  o = align16(o + sizeof(float) * (size_t)NW * TPG * 4);
    s.part = o; o = align16(o + sizeof(float2) * (size_t)TPG * kChunks * N);
    s.st = o;   o = align16(o + sizeof(SlotState));
    s.bytes = o;
    return s;
}

__host__ __device__ inline size_t a_bytes(int N, int lda) { return align16(sizeof(float2) * (size_t)N * lda); }

struct Params {
    const float *A_re, *A_im;  // global planar tables [N][lda]
    int N, L, Lpad, lda;
    SolveLaunch a;
};

// packed FP32 pair FMA: d = a * b + c on both halves (Blackwell f32x2)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)),
          "l"(*reinterpret_cast<unsigned long long *>(&b)),
          "l"(*reinterpret_cast<unsigned long long *>(&c)));
    return *reinterpret_cast<float2 *>(&d);
}

// barrier of one group (ids 1..kMaxGroups; id 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int grp, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(nthreads) : "memory");
}

// Reduce v[0..15] over the 32 lanes of a warp with a fixed butterfly: at each step a
// lane keeps one half of its values, sends the other half to its partner and adds
// what it receives; a last exchange adds the two copies.  Afterwards lanes 2i and
// 2i+1 hold the total of value number i in v[0].  The summation order never
// depends on timing.
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane)
{
#pragma unroll
    for (int off = 16, h = 8; off >= 2; off >>= 1, h >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float keep = up ? v[h + j] : v[j];
            const float send = up ? v[j] : v[h + j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__global__ void __launch_bounds__(kMaxThreads, 1) k_rbpg_fp32(Params prm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = prm.N, L = prm.L, Lpad = prm.Lpad, lda = prm.lda;
    const int NW = Lpad / 32;  // warps per group
    const int grp = threadIdx.x / Lpad;
    const int tid = threadIdx.x - grp * Lpad;  // grid index l owned by this thread
    const int lane = tid & 31, warp = tid >> 5;  // warp within the group
    const SolveLaunch &a = prm.a;
    float2 *sA = (float2 *)smem_raw;  // [N][lda] (re, im)
    const GroupLayout lay = group_layout(N, Lpad);
    unsigned char *gbase = smem_raw + a_bytes(N, lda) + (size_t)grp * lay.bytes;
    float *sRre = (float *)(gbase + lay.Rre);        // [N][TPG]
    float *sRim = (float *)(gbase + lay.Rim);        // [N][TPG]
    float2 *sXb = (float2 *)(gbase + lay.Xb);        // [TPG][Lpad]
    float2 *sXp = (float2 *)(gbase + lay.Xp);        // [TPG][Lpad]
    uint32_t *sMask = (uint32_t *)(gbase + lay.mask);  // [TPG][NW]
    float2 *sG = (float2 *)(gbase + lay.G);          // [TPG][N]
    float2 *sAx = (float2 *)(gbase + lay.Ax);
    float2 *sAxp = (float2 *)(gbase + lay.Axp);
    float2 *sAy = (float2 *)(gbase + lay.Ay);
    float *sRed = (float *)(gbase + lay.red);        // [NW][TPG][4]
    float2 *sPart = (float2 *)(gbase + lay.part);    // [TPG][kChunks][N]
    SlotState &S = *(SlotState *)(gbase + lay.st);

    for (int i = threadIdx.x; i < N * lda; i += blockDim.x)
        sA[i] = make_float2(prm.A_re[i], prm.A_im[i]);
    for (int i = tid; i < TPG * Lpad; i += Lpad)
        sXp[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < N * TPG; i += Lpad) {
        sRre[i] = 0.f;
        sRim[i] = 0.f;
    }
    float2 x[TPG];
#pragma unroll
    for (int p = 0; p < TPG; ++p)
        x[p] = make_float2(0.f, 0.f);
    if (tid < TPG) {
        S.flags[tid] = F_FIN;  // every slot starts empty and asks for a pixel
        S.need[0][tid] = 0;
        S.need[1][tid] = 0;
        S.cnt[0][tid] = 0;
        S.cnt[1][tid] = 0;
        S.pix[tid] = -1;
    }
    if (tid == 0) {
        S.retry[0] = S.retry[1] = S.retry[2] = 0;
        S.nfin = TPG;
        S.nactive = 0;
        S.ndense = 0;
    }
    __syncthreads();  // A is complete for every group

    const float alpha0 = a.alpha0;
    const float tol2 = a.tol * a.tol;
    int sweep = 0;  // C-DE sweeps so far (iterations and step-size retries)

    for (int iter = 0;; ++iter) {
        const int cur = iter & 1, nxt = cur ^ 1;
        // ---------------- H: record finished pixels and refill their slots -----------
        if (S.nfin) {
            for (int p = warp; p < TPG; p += NW) {
                if (!(S.flags[p] & F_FIN))
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
                    const float2 g0 = (lane < N) ? gq[lane] : make_float2(0.f, 0.f);
                    const float2 g1 = (lane + 32 < N) ? gq[lane + 32] : make_float2(0.f, 0.f);
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
                    // x^0 = x^{-1} = 0: A y = 0 and r = -g for the first iteration
                    for (int n = lane; n < N; n += 32) {
                        const float2 gg = (n < 32) ? g0 : g1;
                        sG[p * N + n] = gg;
                        sAx[p * N + n] = make_float2(0.f, 0.f);
                        sAxp[p * N + n] = make_float2(0.f, 0.f);
                        sAy[p * N + n] = make_float2(0.f, 0.f);
                        sRre[n * TPG + p] = -gg.x;
                        sRim[n * TPG + p] = -gg.y;
                    }
                    float gg2 = g0.x * g0.x + g0.y * g0.y + g1.x * g1.x + g1.y * g1.y;
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1)
                        gg2 += __shfl_xor_sync(0xffffffffu, gg2, off);
                    if (lane == 0) {
                        const float lam = a.lam_pp ? a.lam[q] : a.lam[0];
                        S.k[p] = 1;
                        S.alpha[p] = alpha0;
                        S.Fx[p] = gg2;  // F(0) = ||g||^2
                        S.lam[p] = lam;
                        // (k-2)/(k+1) at k = 1 multiplies x - x_prev = 0
                        S.par[p] = make_float4(-0.5f, 2.f * alpha0, alpha0 * lam, 0.f);
                        S.nbt[p] = 0;
                        S.status[p] = 0;
                        S.nnz[p] = 0;
                    }
                    break;
                }
                if (lane == 0) {
                    S.pix[p] = q;
                    S.flags[p] = (q >= 0) ? F_ACTIVE : 0;
                    S.need[cur][p] = (q >= 0);
                    S.nbt_it[p] = 0;
                }
            }
            group_sync(grp, Lpad);
            if (tid == 0) {
                int c = 0;
                for (int p = 0; p < TPG; ++p)
                    c += (S.flags[p] & F_ACTIVE) ? 1 : 0;
                S.nactive = c;
                S.nfin = 0;
            }
            group_sync(grp, Lpad);
            if (S.nactive == 0)
                break;
        }

        // ---------------- B: gradient sum_n conj(A_nl) r_n for l = tid -------------------
        float2 gx[TPG / 2], gy[TPG / 2];  // slot pairs (2q, 2q+1): real and imaginary parts
#pragma unroll
        for (int q = 0; q < TPG / 2; ++q) {
            gx[q] = make_float2(0.f, 0.f);
            gy[q] = make_float2(0.f, 0.f);
        }
        {
            const float2 *pa = sA + tid;
            const float4 *rre = (const float4 *)sRre;
            const float4 *rim = (const float4 *)sRim;
#pragma unroll 2
            for (int n = 0; n < N; ++n) {
                const float2 av = pa[n * lda];
                const float2 ar2 = make_float2(av.x, av.x);
                const float2 ai2 = make_float2(av.y, av.y);
                const float2 nai2 = make_float2(-av.y, -av.y);
#pragma unroll
                for (int q4 = 0; q4 < TPG / 4; ++q4) {
                    const float4 rx = rre[n * (TPG / 4) + q4];
                    const float4 ry = rim[n * (TPG / 4) + q4];
                    const float2 rx0 = make_float2(rx.x, rx.y), rx1 = make_float2(rx.z, rx.w);
                    const float2 ry0 = make_float2(ry.x, ry.y), ry1 = make_float2(ry.z, ry.w);
                    // Re conj(a) r = ar rx + ai ry ;  Im conj(a) r = ar ry - ai rx
                    gx[2 * q4] = ffma2(ai2, ry0, ffma2(ar2, rx0, gx[2 * q4]));
                    gy[2 * q4] = ffma2(nai2, rx0, ffma2(ar2, ry0, gy[2 * q4]));
                    gx[2 * q4 + 1] = ffma2(ai2, ry1, ffma2(ar2, rx1, gx[2 * q4 + 1]));
                    gy[2 * q4 + 1] = ffma2(nai2, rx1, ffma2(ar2, ry1, gy[2 * q4 + 1]));
                }
            }
        }

        // ---------------- C, A xbar, DE with backtracking ----------------------------------------
        for (int round = 0;; ++round) {
            // C: prox, ballots, partial sums (two passes of 4 slots keep register use low)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float part[16];
#pragma unroll
                for (int pp = 0; pp < TPG / 2; ++pp) {
                    const int p = half * (TPG / 2) + pp;
                    float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
                    if (S.need[cur][p]) {
                        const float4 par = S.par[p];  // beta, 2 alpha, tau = alpha lambda
                        const float gre = (p & 1) ? gx[p >> 1].y : gx[p >> 1].x;
                        const float gim = (p & 1) ? gy[p >> 1].y : gy[p >> 1].x;
                        const float2 xp = sXp[p * Lpad + tid];
                        const float yx = fmaf(par.x, x[p].x - xp.x, x[p].x);
                        const float yy = fmaf(par.x, x[p].y - xp.y, x[p].y);
                        const float vx = fmaf(-par.y, gre, yx), vy = fmaf(-par.y, gim, yy);
                        const float m2 = fmaf(vx, vx, vy * vy);
                        const float tau = par.z;
                        float bx = 0.f, by = 0.f;
                        bool nz = false;
                        if (m2 > tau * tau) {
                            const float mag = sqrtf(m2);
                            if (mag > tau) {
                                const float sc = 1.f - tau / mag;
                                bx = vx * sc;
                                by = vy * sc;
                                l1 = mag - tau;
                                nz = true;
                            }
                        }
                        sXb[p * Lpad + tid] = make_float2(bx, by);
                        const unsigned bal = __ballot_sync(0xffffffffu, nz);
                        if (lane == 0) {
                            sMask[p * NW + warp] = bal;
                            if (bal)
                                atomicAdd(&S.cnt[sweep & 1][p], __popc(bal));
                        }
                        const float ex = bx - yx, ey = by - yy;
                        dd = fmaf(ex, ex, ey * ey);
                        const float fx = bx - x[p].x, fy = by - x[p].y;
                        dx = fmaf(fx, fx, fy * fy);
                        xn = fmaf(bx, bx, by * by);
                    }
                    part[4 * pp + 0] = dd;
                    part[4 * pp + 1] = l1;
                    part[4 * pp + 2] = dx;
                    part[4 * pp + 3] = xn;
                }
                warp_transpose_reduce16(part, lane);
                // lanes 2i, 2i+1 hold value i: slot half*4 + i/4, quantity i%4
                if ((lane & 1) == 0) {
                    const int v = lane >> 1;
                    sRed[(warp * TPG + half * (TPG / 2) + (v >> 2)) * 4 + (v & 3)] = part[0];
                }
            }
            if (tid == 0)
                S.retry[(round + 1) % 3] = 0;
            group_sync(grp, Lpad);

            // which slots need the dense A xbar pass
            if (tid == 0) {
                int nd = 0;
                for (int p = 0; p < TPG; ++p)
                    if (S.need[cur][p] && S.cnt[sweep & 1][p] > kSparseMax)
                        S.dense[nd++] = p;
                S.ndense = nd;
            }
            if (tid < TPG)
                S.cnt[(sweep + 1) & 1][tid] = 0;  // counts of the next sweep
            group_sync(grp, Lpad);
            const int ndense = S.ndense;
            if (ndense) {
                const int CH = Lpad / kChunks;  // Lpad is a multiple of 32
                for (int it = tid; it < ndense * kChunks * N; it += Lpad) {
                    const int jc = it / N, n = it - (it / N) * N;  // jc = j * kChunks + c
                    const int j = jc / kChunks, c = jc - (jc / kChunks) * kChunks;
                    const int p = S.dense[j];
                    const float2 *xr = sXb + p * Lpad + c * CH;
                    const float2 *ar = sA + n * lda + c * CH;
                    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
                    for (int l = 0; l < CH; l += 2) {
                        const float2 x0 = xr[l], a0 = ar[l], x1 = xr[l + 1], a1 = ar[l + 1];
                        s0.x = fmaf(a0.x, x0.x, fmaf(-a0.y, x0.y, s0.x));
                        s0.y = fmaf(a0.x, x0.y, fmaf(a0.y, x0.x, s0.y));
                        s1.x = fmaf(a1.x, x1.x, fmaf(-a1.y, x1.y, s1.x));
                        s1.y = fmaf(a1.x, x1.y, fmaf(a1.y, x1.x, s1.y));
                    }
                    sPart[(p * kChunks + c) * N + n] = make_float2(s0.x + s1.x, s0.y + s1.y);
                }
                group_sync(grp, Lpad);
            }

            // DE: one half-warp per slot (slots 2 pw, 2 pw + 1 on warp pw mod #warps)
            for (int pw = warp; pw < TPG / 2; pw += NW) {
                const int p = 2 * pw + (lane >> 4);
                const int h = lane & 15;
                const unsigned hmask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
                if (!S.need[cur][p])
                    continue;
                // A xbar; lane h owns n = h + 16 j
                float2 axb[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    axb[j] = make_float2(0.f, 0.f);
                const bool dense = S.cnt[sweep & 1][p] > kSparseMax;
                if (dense) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = h + 16 * j;
                        if (n < N)
#pragma unroll
                            for (int c = 0; c < kChunks; ++c) {
                                const float2 v = sPart[(p * kChunks + c) * N + n];
                                axb[j].x += v.x;
                                axb[j].y += v.y;
                            }
                    }
                } else {
                    // over the nonzeros of xbar in ascending l, four per trip
                    for (int w = 0; w < NW; ++w) {
                        uint32_t msk = sMask[p * NW + w];
                        while (msk) {
                            int lq[4];
                            float2 xq[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                lq[u] = msk ? (w * 32 + __ffs(msk) - 1) : -1;
                                msk &= msk - 1;
                                xq[u] = (lq[u] >= 0) ? sXb[p * Lpad + lq[u]] : make_float2(0.f, 0.f);
                            }
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int n = h + 16 * j;
                                if (n < N) {
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        if (lq[u] >= 0) {
                                            const float2 av = sA[n * lda + lq[u]];
                                            axb[j].x = fmaf(av.x, xq[u].x, fmaf(-av.y, xq[u].y, axb[j].x));
                                            axb[j].y = fmaf(av.x, xq[u].y, fmaf(av.y, xq[u].x, axb[j].y));
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                float lhs = 0.f, res = 0.f, dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int n = h + 16 * j;
                    if (n < N) {
                        const float2 ay = sAy[p * N + n], gg = sG[p * N + n];
                        const float d0 = axb[j].x - ay.x, d1 = axb[j].y - ay.y;
                        lhs = fmaf(d0, d0, fmaf(d1, d1, lhs));
                        const float e0 = axb[j].x - gg.x, e1 = axb[j].y - gg.y;
                        res = fmaf(e0, e0, fmaf(e1, e1, res));
                    }
                }
                if (h < NW) {
                    const float4 rd = *(const float4 *)(sRed + (h * TPG + p) * 4);
                    dd = rd.x;
                    l1 = rd.y;
                    dx = rd.z;
                    xn = rd.w;
                }
#pragma unroll
                for (int off = 8; off >= 1; off >>= 1) {
                    lhs += __shfl_xor_sync(hmask, lhs, off);
                    res += __shfl_xor_sync(hmask, res, off);
                    dd += __shfl_xor_sync(hmask, dd, off);
                    l1 += __shfl_xor_sync(hmask, l1, off);
                    dx += __shfl_xor_sync(hmask, dx, off);
                    xn += __shfl_xor_sync(hmask, xn, off);
                }
                const float al = S.alpha[p];
                const bool bt_ok = lhs <= dd / (2.f * al);
                if (!bt_ok && S.nbt_it[p] < a.max_bt) {
                    // Eq. 15 failed: shrink the step and redo the prox for this slot
                    __syncwarp(hmask);
                    if (h == 0) {
                        const float an = al * a.c_alpha;
                        S.alpha[p] = an;
                        S.par[p].y = 2.f * an;
                        S.par[p].z = an * S.lam[p];
                        S.nbt[p] += 1;
                        S.nbt_it[p] += 1;
                        atomicAdd(&S.retry[round % 3], 1);
                    }
                    continue;
                }
                const float Fb = fmaf(S.lam[p], l1, res);
                const bool accepted = (Fb <= S.Fx[p]);
                const bool conv = (dx <= tol2 * xn) || (dx == 0.f);
                const int k = S.k[p];
                const bool fin = conv || (k >= a.max_iter);
                // N-space state: A x^{k-1} <- A x^k, A x^{k+1} <- A xbar (accepted); for the
                // next iteration A y = A x + beta (A x - A x_prev), r = A y - g
                const float beta_n = (float)(k - 1) / (float)(k + 2);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int n = h + 16 * j;
                    if (n < N) {
                        const float2 axo = sAx[p * N + n];
                        const float2 axn = accepted ? axb[j] : axo;
                        sAxp[p * N + n] = axo;
                        sAx[p * N + n] = axn;
                        if (!fin) {
                            const float2 ay = make_float2(fmaf(beta_n, axn.x - axo.x, axn.x),
                                                          fmaf(beta_n, axn.y - axo.y, axn.y));
                            const float2 gg = sG[p * N + n];
                            sAy[p * N + n] = ay;
                            sRre[n * TPG + p] = ay.x - gg.x;
                            sRim[n * TPG + p] = ay.y - gg.y;
                        }
                    }
                }
                __syncwarp(hmask);
                if (h == 0) {
                    int st = S.status[p];
                    if (!bt_ok)
                        st |= BPDN_PX_BT_LIMIT;
                    int nnz = S.nnz[p];
                    if (accepted) {
                        S.Fx[p] = Fb;
                        nnz = 0;
                        for (int w = 0; w < NW; ++w)
                            nnz += __popc(sMask[p * NW + w]);
                        S.nnz[p] = nnz;
                    }
                    if (fin && !conv)
                        st |= BPDN_PX_NOT_CONVERGED;
                    S.status[p] = st;
                    S.flags[p] = F_ACTIVE | (accepted ? F_ACC : 0) | (fin ? F_FIN : 0);
                    S.need[cur][p] = 0;
                    S.need[nxt][p] = fin ? 0 : 1;
                    if (fin) {
                        atomicAdd(&S.nfin, 1);
                        const long long q = S.pix[p];
                        a.status[q] = (nnz == 0) ? (st | BPDN_PX_ZERO_SOLUTION) : st;
                        a.iters[q] = k;
                        if (a.nbt)
                            a.nbt[q] = S.nbt[p];
                        if (a.nsupp)
                            a.nsupp[q] = nnz;
                    } else {
                        S.k[p] = k + 1;
                        S.par[p].x = beta_n;
                        S.nbt_it[p] = 0;
                    }
                }
            }
            group_sync(grp, Lpad);
            ++sweep;
            if (S.retry[round % 3] == 0)
                break;
        }

        // ---------------- G: registers and outputs -------------------------------------------
#pragma unroll
        for (int p = 0; p < TPG; ++p) {
            const int fl = S.flags[p];
            if (!(fl & F_ACTIVE))
                continue;
            const float2 xo = x[p];
            if (fl & F_ACC)
                x[p] = sXb[p * Lpad + tid];
            if (fl & F_FIN) {
                if (tid < L)
                    a.x[(size_t)S.pix[p] * L + tid] = x[p];
                x[p] = make_float2(0.f, 0.f);
                sXp[p * Lpad + tid] = make_float2(0.f, 0.f);
            } else {
                sXp[p * Lpad + tid] = xo;
            }
        }
        if (S.nfin)
            group_sync(grp, Lpad);
    }
}

int choose_groups(const OpHandle &op, int max_smem, size_t *smem_out)
{
    const GroupLayout lay = group_layout(op.N, op.Lpad);
    const size_t base = a_bytes(op.N, op.lda);
    int g = kMaxThreads / op.Lpad;
    if (g > kMaxGroups)
        g = kMaxGroups;
    while (g > 1 && base + (size_t)g * lay.bytes > (size_t)max_smem)
        --g;
    *smem_out = base + (size_t)g * lay.bytes;
    return g;
}

}  // namespace

size_t rbpg_smem_bytes(const OpHandle &op)
{
    // the smallest configuration (one group)
    return a_bytes(op.N, op.lda) + group_layout(op.N, op.Lpad).bytes;
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
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    size_t smem = 0;
    const int groups = choose_groups(op, max_smem, &smem);
    e = cudaFuncSetAttribute(k_rbpg_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long tiles = (a.P + (long long)groups * TPG - 1) / ((long long)groups * TPG);
    int grid = (int)((tiles < num_sms) ? tiles : num_sms);
    if (grid < 1)
        grid = 1;
    k_rbpg_fp32<<<grid, groups * op.Lpad, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bpdn
