// Persistent iteration kernel: Algorithm 1 (RBPG with backtracking) for many pixels
// that share one operator, one pixel per slot, eight slots per group of warps.
//
// Two variants share everything but the gradient contraction sum_n conj(A_nl) r_n:
//   FP32  CUDA cores, packed f32x2 FMAs against the FP32 residuals in shared memory;
//   BF16  tcgen05 MMAs from BF16 operands into FP32 accumulators in tensor memory,
//         D[l, j] = sum_k Aop[l, k] B[j, k] per 128-row tile of the grid, K = 64
//         (2N <= 64) or 128 (2N <= 128), zero padded, N = 16, with the constant operator rows
//         Aop[l, :] = (Re A[:, l], Im A[:, l]) in tensor memory for the whole launch and
//         B[p, :] = (Re r_p, Im r_p), B[8 + p, :] = (Im r_p, -Re r_p) in shared memory,
//         so that D[l, p] = Re sum_n conj(A_nl) r_n and D[l, 8 + p] its imaginary part.
// The iterate, prox, line search (Eq. 15), accept and stopping tests and A xbar run in
// FP32 in both.  A sits in shared memory when it fits, else it is read from global
// memory (it stays in L2).
//
// Per-pixel state: thread l (one grid point) keeps x^k of its slots in registers and
// x^{k-1}, xbar in its own tensor-memory lane.  One sweep of a group:
//   transition  apply the previous decisions (x^{k-1} <- x^k, x^k <- xbar, write out
//               finished pixels, zero refilled slots), overlapping the MMAs (BF16);
//   C           gradient, prox (Eq. 12) per slot, partial sums over the warp's 32 grid
//               points and the warp's share of A xbar (ascending l over the nonzeros
//               its ballot finds);
//   DE          one warp per slot: A xbar and the sums over warps in a fixed order,
//               Eq. 15, monotone accept, stopping test, next residual r = A y - g in
//               N space, and the refill of finished slots from the work counter.
// A slot whose step fails Eq. 15 runs the next sweep with the smaller step and the
// same residual (the gradient is recomputed bit for bit).  Two group barriers per
// sweep; every sum has a fixed order, so results do not depend on timing.
//
// Warps are assigned to (group, tile, lane quadrant) so that a warp only touches the
// tensor-memory lanes 32 (w mod 4) .. 32 (w mod 4) + 31 it may access; the partial last
// tile of group g sits at quadrants s_g .. (the BF16 operator rows are duplicated there),
// so two groups of L = 416 take 26 warps.
//
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int TPG = 8;          // pixel slots per group
constexpr int kMaxGroups = 8;   // groups per CTA (named barriers 1..kMaxGroups)
// BF16 contraction length 2N zero padded: 64 with one row per lane (N <= 32), 128 with two
constexpr int kK1 = 64, kK2 = 128;
__host__ __device__ constexpr int tc_k(int nch) { return nch == 1 ? kK1 : kK2; }
constexpr int kTmemCols = 512;
constexpr int kMaxNW = 32;      // 32-point blocks of the grid per group: Lpad <= 1024

// transition bits, applied at the start of a sweep
constexpr int T_ACTIVE = 1;  // the slot holds a pixel during this sweep
constexpr int T_ACC = 2;     // x^k <- xbar (the last evaluation was accepted)
constexpr int T_SHIFT = 4;   // x^{k-1} <- x^k (an iteration ended)
constexpr int T_OUT = 8;     // write x^k (after T_ACC) to the output row of pix_out
constexpr int T_RESET = 16;  // x^k = x^{k-1} = 0: a new pixel starts in this sweep

struct SlotState {
    long long pix[TPG];      // pixel in the slot, -1 when none
    long long pix_out[TPG];  // pixel whose x the next transition writes out
    float4 par[TPG];         // (beta, 2 alpha, alpha lambda, transition bits)
    float alpha[TPG], Fx[TPG], lam[TPG];
    int k[TPG], nbt[TPG], nbt_it[TPG], status[TPG], nnz[TPG];
    int abort;          // BF16: a bounded wait for the tensor cores ran out in this group
    uint32_t abort_ph;  // the mbarrier phase that was not seen complete
};

// shared-memory layout: A (when it fits) once, then one block per group
struct GroupLayout {
    size_t Bop, Rre, Rim, mbar, G, Ax, Axp, Ay, mask, red, part, st, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GroupLayout group_layout(int N, int Lpad, bool tc, int kk)
{
    GroupLayout s;
    const int NW = Lpad / 32;
    size_t o = 0;
    s.Bop = s.Rre = s.Rim = s.mbar = 0;
    if (tc) {
        s.Bop = o;  o = align16(o + 16 * kk * 2);  // B: 16 rows x K bf16, core-matrix layout
        s.mbar = o; o = align16(o + 8);
    } else {
        s.Rre = o;  o = align16(o + sizeof(float) * (size_t)N * TPG);  // [N][TPG]
        s.Rim = o;  o = align16(o + sizeof(float) * (size_t)N * TPG);
    }
    s.G = o;    o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Ax = o;   o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Axp = o;  o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.Ay = o;   o = align16(o + sizeof(float2) * (size_t)TPG * N);
    s.mask = o; o = align16(o + sizeof(uint32_t) * (size_t)TPG * NW);
    s.red = o;  o = align16(o + sizeof(float4) * (size_t)NW * TPG);
    s.part = o; o = align16(o + sizeof(float2) * (size_t)TPG * NW * N);
    s.st = o;   o = align16(o + sizeof(SlotState));
    s.bytes = o;
    return s;
}

// A as float2 [N][lda] (lda = Lpad + 1, odd): lanes over l and lanes over n both
// read without bank conflicts
__host__ __device__ inline size_t a_bytes(int N, int lda) { return align16(sizeof(float2) * (size_t)N * lda); }

// ---- warp roles ----
// Tiles T = ceil(Lpad / 128); the last one holds qlast blocks of 32 grid points.  Group g
// places the blocks of a partial last tile at quadrants s_g .. s_g + qlast - 1.
struct TileShape {
    int T, F, qlast, partial;  // tiles, full tiles, blocks in the last tile, has a partial tile
};

__host__ __device__ inline TileShape tile_shape(int Lpad)
{
    TileShape s;
    s.T = (Lpad + 127) / 128;
    s.qlast = (Lpad - 128 * (s.T - 1)) / 32;
    s.partial = s.qlast < 4;
    s.F = s.partial ? s.T - 1 : s.T;
    return s;
}

__host__ __device__ inline int partial_start(const TileShape &s, int G, int g)
{
    return (G * s.qlast <= 4) ? g * s.qlast : 0;
}

// role of warp w: group, block of 32 grid points (l = 32 blk + lane) and tile; false = idle
__host__ __device__ inline bool warp_role(int w, int G, int Lpad, int *grp, int *blk, int *tile)
{
    const TileShape s = tile_shape(Lpad);
    const int q = w & 3, i = w >> 2;
    if (i < G * s.F) {
        *grp = i / s.F;
        *tile = i % s.F;
        *blk = 4 * (*tile) + q;
        return true;
    }
    if (!s.partial)
        return false;
    int j = i - G * s.F;
    for (int g = 0; g < G; ++g) {
        const int s0 = partial_start(s, G, g);
        if (q >= s0 && q < s0 + s.qlast) {
            if (j == 0) {
                *grp = g;
                *tile = s.T - 1;
                *blk = 4 * (s.T - 1) + (q - s0);
                return true;
            }
            --j;
        }
    }
    return false;
}

int warps_for(int Lpad, int G)
{
    const TileShape s = tile_shape(Lpad);
    int W = 0;
    for (int q = 0; q < 4; ++q) {
        int n = G * s.F;
        if (s.partial)
            for (int g = 0; g < G; ++g) {
                const int s0 = partial_start(s, G, g);
                n += (q >= s0 && q < s0 + s.qlast) ? 1 : 0;
            }
        if (n > 0 && 4 * (n - 1) + q + 1 > W)
            W = 4 * (n - 1) + q + 1;
    }
    return W;
}

// tensor-memory columns: [BF16 operator rows, K/2 per tile][BF16 accumulators per group]
// [x^{k-1} per group][xbar per group], 16 columns per tile for each per-group table
__host__ __device__ inline int tmem_cols_used(int T, int G, bool tc, int kk)
{
    return (tc ? kk / 2 * T + 16 * T * G : 0) + 32 * T * G;
}

// one stack of a launch: its operator, sizes and solve
struct StackDesc {
    const float *A_re, *A_im;  // global planar tables [N][lda]
    int N, L, Lpad, lda;
    int groups;  // slot groups of 8 pixels per CTA for this stack
    int ctas;    // CTAs 0 .. ctas-1 take this stack's pixels
    SolveLaunch a;
};

constexpr int kMaxStacks = 64;  // stacks per launch (kernel parameters stay below 32 KB)

struct Params {
    int nstacks;
    StackDesc st[kMaxStacks];
};

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

// packed FP32 pair FMA: d = a * b + c on both halves
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

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

// two FP32 values -> packed BF16 pair (element 2c in the low half, as tensor memory
// holds a K-major operand row: element k in column k/2)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

// byte offset of element (row, k) of a K-major operand with kk columns, no swizzle:
// core matrices of 8 rows x 16 bytes; the K-adjacent core matrix 128 bytes on (LBO),
// the next 8-row group kk/8 * 128 bytes on (SBO)
__host__ __device__ inline int kmaj_off(int row, int k, int kk)
{
    return (row >> 3) * (kk / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor of tcgen05 (no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (tmem) [+]= A (tmem) x B (smem descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t accum)
{
    asm volatile(
        "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait for an mbarrier phase; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
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

// tensor-memory loads and stores of this warp's 32 lanes, consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
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

__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8])
{
    uint32_t u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        u[i] = __float_as_uint(v[i]);
    tmem_st8u(taddr, u);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Algorithm 1 for one stack, by the whole CTA, until the stack's pixels run out and every
// slot has drained; tensor memory is allocated by the caller
template <bool TC, bool SA, int NCH>
__device__ __forceinline__ void run_stack(const StackDesc &prm, uint32_t tmem, unsigned char *smem_raw)
{
    const int G = prm.groups;
    const int N = prm.N, L = prm.L, Lpad = prm.Lpad, lda = prm.lda;
    const int NW = Lpad / 32;  // warps (blocks of 32 grid points) per group
    // rows n = lane + 32 c, c < NCH, per lane (BF16: N <= 32 or 64; FP32: N <= 64, or N <= 96 for three)
    static_assert(!TC || NCH <= 2, "the BF16 contraction holds 2N <= 128 terms");
    constexpr int KK = TC ? tc_k(NCH) : 0;  // BF16 contraction length
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q4 = w & 3;
    int grp = 0, blk = 0, tile = 0;
    const bool live = warp_role(w, G, Lpad, &grp, &blk, &tile);
    const int l = 32 * blk + lane;  // grid index owned by this thread
    const SolveLaunch &a = prm.a;
    float2 *sA = (float2 *)smem_raw;  // [N][lda] when SA
    const GroupLayout lay = group_layout(N, Lpad, TC, KK);
    unsigned char *gbase = smem_raw + (SA ? a_bytes(N, lda) : 0) + (size_t)grp * lay.bytes;
    unsigned char *sBop = gbase + lay.Bop;  // BF16
    float *sRre = (float *)(gbase + lay.Rre), *sRim = (float *)(gbase + lay.Rim);  // FP32: [N][TPG]
    const uint32_t mbar = smem_u32(gbase + lay.mbar);
    float2 *sG = (float2 *)(gbase + lay.G);  // [TPG][N]
    float2 *sAx = (float2 *)(gbase + lay.Ax);
    float2 *sAxp = (float2 *)(gbase + lay.Axp);
    float2 *sAy = (float2 *)(gbase + lay.Ay);
    uint32_t *sMask = (uint32_t *)(gbase + lay.mask);  // [TPG][NW] ballots of xbar != 0
    float4 *sRed = (float4 *)(gbase + lay.red);        // [NW][TPG] (dd, l1, dx, xn)
    float2 *sPart = (float2 *)(gbase + lay.part);      // [TPG][NW][N] A xbar over one block
    SlotState &S = *(SlotState *)(gbase + lay.st);

    // A_{n, ll}
    auto Aat = [&](int n, int ll) -> float2 {
        if constexpr (SA)
            return sA[n * lda + ll];
        else
            return make_float2(__ldg(prm.A_re + n * lda + ll), __ldg(prm.A_im + n * lda + ll));
    };
    // residual of slot p at row n for the next gradient
    auto put_r = [&](int p, int n, float re, float im) {
        if constexpr (TC) {
            const __nv_bfloat16 bre = __float2bfloat16_rn(re), bim = __float2bfloat16_rn(im);
            const __nv_bfloat16 nre = __float2bfloat16_rn(-re);
            *(__nv_bfloat16 *)(sBop + kmaj_off(p, n, KK)) = bre;
            *(__nv_bfloat16 *)(sBop + kmaj_off(p, N + n, KK)) = bim;
            *(__nv_bfloat16 *)(sBop + kmaj_off(TPG + p, n, KK)) = bim;
            *(__nv_bfloat16 *)(sBop + kmaj_off(TPG + p, N + n, KK)) = nre;
        } else {
            sRre[n * TPG + p] = re;
            sRim[n * TPG + p] = im;
        }
    };

    if constexpr (SA) {
        for (int i = threadIdx.x; i < N * lda; i += blockDim.x)
            sA[i] = make_float2(prm.A_re[i], prm.A_im[i]);
    }
    if (live && blk == 0) {
        if (lane == 0)
            S.abort = 0;
        if constexpr (TC) {
            for (int i = lane; i < 16 * KK * 2 / 4; i += 32)
                ((uint32_t *)sBop)[i] = 0u;  // K padding of B stays zero
            if (lane == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
                asm volatile("fence.mbarrier_init.release.cluster;");
            }
        } else {
            for (int i = lane; i < N * TPG; i += 32) {
                sRre[i] = 0.f;
                sRim[i] = 0.f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
    const int T = (Lpad + 127) / 128;
    const int colD = TC ? KK / 2 * T : 0;
    const int colXp = colD + (TC ? 16 * T * G : 0);
    const int colXb = colXp + 16 * T * G;
    const uint32_t taD = lane_base + colD + 16 * T * grp + 16 * tile;
    const uint32_t taXp = lane_base + colXp + 16 * T * grp + 16 * tile;
    const uint32_t taXb = lane_base + colXb + 16 * T * grp + 16 * tile;
    if (live) {
        if constexpr (TC) {
            // operator rows of this thread's grid index into its tensor-memory lane: full
            // tiles by group 0, the partial tile by every group at its own quadrants
            if (grp == 0 || tile == T - 1) {
                const uint32_t ta = lane_base + KK / 2 * tile;
#pragma unroll
                for (int part = 0; part < KK / 16; ++part) {
                    uint32_t v[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float e2[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int k = 2 * (8 * part + c) + e;
                            float val = 0.f;
                            if (k < N)
                                val = Aat(k, l).x;
                            else if (k < 2 * N)
                                val = Aat(k - N, l).y;
                            e2[e] = val;
                        }
                        v[c] = pack_bf16(e2[0], e2[1]);
                    }
                    tmem_st8u(ta + 8 * part, v);
                }
            }
        }
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        tmem_st8(taXp, z);
        tmem_st8(taXp + 8, z);
        tmem_st8(taXb, z);
        tmem_st8(taXb + 8, z);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();  // A, operator rows of every tile in place before any group's MMA
    if (!live)
        return;  // idle warp of this stack: the caller's barrier waits for the groups

    const float alpha0 = a.alpha0;
    const float tol2 = a.tol * a.tol;

    // refill slot p from the work counter (one warp, lane n owns rows n and n + 32);
    // returns the transition bits
    auto refill = [&](int p) -> int {
        long long q;
        for (;;) {
            if (lane == 0)
                q = (long long)atomicAdd(a.counter, 1ULL);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= a.P) {
                q = -1;
                break;
            }
            if (TC && S.abort) {
                // the group's tensor-core wait ran out: it no longer iterates, but every
                // pixel it takes still gets x = 0 and a status that says so
                float2 *xq = a.x + (size_t)q * L;
                for (int ll = lane; ll < L; ll += 32)
                    xq[ll] = make_float2(0.f, 0.f);
                if (lane == 0) {
                    a.status[q] = BPDN_PX_DEVICE_TIMEOUT | BPDN_PX_ZERO_SOLUTION;
                    a.iters[q] = 0;
                    if (a.nbt)
                        a.nbt[q] = 0;
                    if (a.nsupp)
                        a.nsupp[q] = 0;
                }
                continue;
            }
            const float2 *gq = a.g + (size_t)q * N;
            float2 gr[NCH];
            bool fin = true;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                gr[c] = (lane + 32 * c < N) ? gq[lane + 32 * c] : make_float2(0.f, 0.f);
                fin = fin && isfinite(gr[c].x) && isfinite(gr[c].y);
            }
            const bool allfin = __all_sync(0xffffffffu, fin);
            if (!allfin || a.max_iter <= 0) {
                // non-finite g (or no iteration allowed): x = 0 at once
                float2 *xq = a.x + (size_t)q * L;
                for (int ll = lane; ll < L; ll += 32)
                    xq[ll] = make_float2(0.f, 0.f);
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
            // x^0 = x^{-1} = 0: A y = 0 and r = -g for the first iteration
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int n = lane + 32 * c;
                if (n < N) {
                    const float2 gg = gr[c];
                    sG[p * N + n] = gg;
                    sAx[p * N + n] = make_float2(0.f, 0.f);
                    sAxp[p * N + n] = make_float2(0.f, 0.f);
                    sAy[p * N + n] = make_float2(0.f, 0.f);
                    put_r(p, n, -gg.x, -gg.y);
                }
            }
            float gg2 = 0.f;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                gg2 += gr[c].x * gr[c].x + gr[c].y * gr[c].y;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
                gg2 += __shfl_xor_sync(0xffffffffu, gg2, off);
            if (lane == 0) {
                const float lam = a.lam_pp ? a.lam[q] : a.lam[0];
                S.k[p] = 1;
                S.alpha[p] = alpha0;
                S.Fx[p] = gg2;  // F(0) = ||g||^2
                S.lam[p] = lam;
                S.nbt[p] = 0;
                S.nbt_it[p] = 0;
                S.status[p] = 0;
                S.nnz[p] = 0;
                // (k-2)/(k+1) at k = 1 multiplies x - x_prev = 0
                S.par[p] = make_float4(-0.5f, 2.f * alpha0, alpha0 * lam, 0.f);
            }
            break;
        }
        if (lane == 0)
            S.pix[p] = q;
        return (q >= 0) ? (T_ACTIVE | T_RESET) : 0;
    };

    // prologue: fill every slot
    for (int p = blk; p < TPG; p += NW) {
        const int bits = refill(p);
        __syncwarp();
        if (lane == 0)
            S.par[p].w = __int_as_float(bits);
    }
    float2 x[TPG];
#pragma unroll
    for (int p = 0; p < TPG; ++p)
        x[p] = make_float2(0.f, 0.f);
    uint32_t mma_phase = 0;
    if constexpr (TC)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(grp, 32 * NW);

    for (;;) {
        tc_fence_after();
        // ---------------- issue the gradient MMAs (BF16); transition --------------------------
        int any = 0;
#pragma unroll
        for (int p = 0; p < TPG; ++p)
            any |= __float_as_int(S.par[p].w);
        const bool running = (any & T_ACTIVE) != 0;
        const bool aborted = TC && S.abort != 0;  // read after the group barrier: one view
        if constexpr (TC) {
            if (running && !aborted && blk == 0 && lane == 0) {
                const uint32_t b0 = smem_u32(sBop);
                for (int t = 0; t < T; ++t) {
                    const uint32_t d = tmem + colD + 16 * T * grp + 16 * t;
                    const uint32_t arow = tmem + KK / 2 * t;
#pragma unroll
                    for (int j = 0; j < KK / 16; ++j)
                        tc_mma_ts(d, arow + 8 * j, smem_desc(b0 + 256 * j, 128, (KK / 8) * 128), j > 0);
                }
                tc_commit(mbar);
            }
        }
        if (any & (T_ACC | T_SHIFT | T_OUT | T_RESET)) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float xb[8], xp[8];
                tmem_ld8(taXb + 8 * h, xb);
                tmem_ld8(taXp + 8 * h, xp);
                tmem_wait_ld();
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int p = 4 * h + pp;
                    const int b = __float_as_int(S.par[p].w);
                    if (b & T_SHIFT) {
                        xp[2 * pp] = x[p].x;
                        xp[2 * pp + 1] = x[p].y;
                    }
                    if (b & T_ACC)
                        x[p] = make_float2(xb[2 * pp], xb[2 * pp + 1]);
                    if ((b & T_OUT) && l < L)
                        a.x[(size_t)S.pix_out[p] * L + l] = x[p];
                    if (b & T_RESET) {
                        x[p] = make_float2(0.f, 0.f);
                        xp[2 * pp] = 0.f;
                        xp[2 * pp + 1] = 0.f;
                    }
                }
                tmem_st8(taXp + 8 * h, xp);
            }
            tmem_wait_st();
        }
        if (!running)
            break;

        // ---------------- gradient sum_n conj(A_nl) r_n -----------------------------------------
        float2 gx[TPG / 2], gy[TPG / 2];  // FP32 variant: slot pairs (2q, 2q+1), re and im
        if constexpr (TC) {
            if (!aborted) {
                if (!mbar_wait(mbar, mma_phase)) {
                    // no further MMAs or waits in this group; DE below ends its pixels
                    S.abort = 1;
                    S.abort_ph = mma_phase;
                    if (a.err)
                        atomicExch(a.err, 1);
                }
                mma_phase ^= 1u;
            }
            __syncwarp();  // lanes leave the polling loop apart: reconverge before tcgen05.ld
            tc_fence_after();
        } else {
#pragma unroll
            for (int q = 0; q < TPG / 2; ++q) {
                gx[q] = make_float2(0.f, 0.f);
                gy[q] = make_float2(0.f, 0.f);
            }
            const float4 *rre = (const float4 *)sRre;
            const float4 *rim = (const float4 *)sRim;
#pragma unroll 2
            for (int n = 0; n < N; ++n) {
                const float2 av = Aat(n, l);
                const float2 ar2 = make_float2(av.x, av.x);
                const float2 ai2 = make_float2(av.y, av.y);
                const float2 nai2 = make_float2(-av.y, -av.y);
#pragma unroll
                for (int h4 = 0; h4 < TPG / 4; ++h4) {
                    const float4 rx = rre[n * (TPG / 4) + h4];
                    const float4 ry = rim[n * (TPG / 4) + h4];
                    const float2 rx0 = make_float2(rx.x, rx.y), rx1 = make_float2(rx.z, rx.w);
                    const float2 ry0 = make_float2(ry.x, ry.y), ry1 = make_float2(ry.z, ry.w);
                    // Re conj(a) r = ar rx + ai ry ;  Im conj(a) r = ar ry - ai rx
                    gx[2 * h4] = ffma2(ai2, ry0, ffma2(ar2, rx0, gx[2 * h4]));
                    gy[2 * h4] = ffma2(nai2, rx0, ffma2(ar2, ry0, gy[2 * h4]));
                    gx[2 * h4 + 1] = ffma2(ai2, ry1, ffma2(ar2, rx1, gx[2 * h4 + 1]));
                    gy[2 * h4 + 1] = ffma2(nai2, rx1, ffma2(ar2, ry1, gy[2 * h4 + 1]));
                }
            }
        }

        // ---------------- C: prox, partial sums, A xbar over this block ---------------------------
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float gre[4], gim[4], xp[8], xbv[8];
            if constexpr (TC) {
                tmem_ld4(taD + 4 * h, gre);
                tmem_ld4(taD + 8 + 4 * h, gim);
            } else {
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int p = 4 * h + pp;
                    gre[pp] = (p & 1) ? gx[p >> 1].y : gx[p >> 1].x;
                    gim[pp] = (p & 1) ? gy[p >> 1].y : gy[p >> 1].x;
                }
            }
            tmem_ld8(taXp + 8 * h, xp);
            tmem_wait_ld();
            float part[16];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int p = 4 * h + pp;
                float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
                float bx = 0.f, by = 0.f;
                const float4 par = S.par[p];  // beta, 2 alpha, tau = alpha lambda, bits
                if (__float_as_int(par.w) & T_ACTIVE) {
                    const float yx = fmaf(par.x, x[p].x - xp[2 * pp], x[p].x);
                    const float yy = fmaf(par.x, x[p].y - xp[2 * pp + 1], x[p].y);
                    const float vx = fmaf(-par.y, gre[pp], yx), vy = fmaf(-par.y, gim[pp], yy);
                    const float m2 = fmaf(vx, vx, vy * vy);
                    const float tau = par.z;
                    // soft threshold (Eq. 12): scale 1 - tau / |v| where that is positive
                    const float rs = rsqrtf(m2);
                    const float sc = fmaf(-tau, rs, 1.f);
                    const bool nz = sc > 0.f;
                    if (nz) {
                        bx = vx * sc;
                        by = vy * sc;
                        l1 = fmaf(m2, rs, -tau);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, nz);
                    if (lane == 0)
                        sMask[p * NW + blk] = bal;
                    if (bal) {
                        // this block's share of A xbar, ascending l; lane n owns rows n + 32 c
                        float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
                        float2 acc2 = make_float2(0.f, 0.f);
                        // two nonzeros per trip (two loads in flight), still ascending l
                        unsigned m = bal;
                        while (m) {
                            const int j0 = __ffs(m) - 1;
                            m &= m - 1;
                            const bool two = (m != 0);
                            const int j1 = two ? (__ffs(m) - 1) : j0;
                            if (two)
                                m &= m - 1;
                            const float xr0 = __shfl_sync(0xffffffffu, bx, j0);
                            const float xi0 = __shfl_sync(0xffffffffu, by, j0);
                            const float xr1 = __shfl_sync(0xffffffffu, bx, j1);
                            const float xi1 = __shfl_sync(0xffffffffu, by, j1);
                            if (lane < N) {
                                const float2 a0 = Aat(lane, 32 * blk + j0);
                                const float2 a1 = Aat(lane, 32 * blk + j1);
                                acc0.x = fmaf(a0.x, xr0, fmaf(-a0.y, xi0, acc0.x));
                                acc0.y = fmaf(a0.x, xi0, fmaf(a0.y, xr0, acc0.y));
                                if (two) {
                                    acc0.x = fmaf(a1.x, xr1, fmaf(-a1.y, xi1, acc0.x));
                                    acc0.y = fmaf(a1.x, xi1, fmaf(a1.y, xr1, acc0.y));
                                }
                            }
                            if (NCH > 1 && lane + 32 < N) {
                                const float2 a0 = Aat(lane + 32, 32 * blk + j0);
                                acc1.x = fmaf(a0.x, xr0, fmaf(-a0.y, xi0, acc1.x));
                                acc1.y = fmaf(a0.x, xi0, fmaf(a0.y, xr0, acc1.y));
                                if (two) {
                                    const float2 a1 = Aat(lane + 32, 32 * blk + j1);
                                    acc1.x = fmaf(a1.x, xr1, fmaf(-a1.y, xi1, acc1.x));
                                    acc1.y = fmaf(a1.x, xi1, fmaf(a1.y, xr1, acc1.y));
                                }
                            }
                            if (NCH > 2 && lane + 64 < N) {
                                const float2 a0 = Aat(lane + 64, 32 * blk + j0);
                                acc2.x = fmaf(a0.x, xr0, fmaf(-a0.y, xi0, acc2.x));
                                acc2.y = fmaf(a0.x, xi0, fmaf(a0.y, xr0, acc2.y));
                                if (two) {
                                    const float2 a1 = Aat(lane + 64, 32 * blk + j1);
                                    acc2.x = fmaf(a1.x, xr1, fmaf(-a1.y, xi1, acc2.x));
                                    acc2.y = fmaf(a1.x, xi1, fmaf(a1.y, xr1, acc2.y));
                                }
                            }
                        }
                        if (lane < N)
                            sPart[(p * NW + blk) * N + lane] = acc0;
                        if (NCH > 1 && lane + 32 < N)
                            sPart[(p * NW + blk) * N + lane + 32] = acc1;
                        if (NCH > 2 && lane + 64 < N)
                            sPart[(p * NW + blk) * N + lane + 64] = acc2;
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
                xbv[2 * pp] = bx;
                xbv[2 * pp + 1] = by;
            }
            tmem_st8(taXb + 8 * h, xbv);
            warp_transpose_reduce16(part, lane);
            // lanes 2i, 2i+1 hold value i: slot 4h + i/4, quantity i%4
            if ((lane & 1) == 0) {
                const int v = lane >> 1;
                ((float *)sRed)[(blk * TPG + 4 * h + (v >> 2)) * 4 + (v & 3)] = part[0];
            }
        }
        tmem_wait_st();
        tc_fence_before();
        group_sync(grp, 32 * NW);

        // ---------------- DE: one warp per slot ------------------------------------------------
        for (int p = blk; p < TPG; p += NW) {
            const int bits = __float_as_int(S.par[p].w);
            if (!(bits & T_ACTIVE)) {
                __syncwarp();
                if (lane == 0)
                    S.par[p].w = __int_as_float(0);
                continue;
            }
            // A xbar and nnz over the blocks in ascending order; lane n owns rows n + 32 c
            const uint32_t mw = (lane < NW) ? sMask[p * NW + lane] : 0u;
            const int nnz = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(mw));
            unsigned wm = __ballot_sync(0xffffffffu, mw != 0u);
            float2 axb[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                axb[c] = make_float2(0.f, 0.f);
            while (wm) {
                const int b = __ffs(wm) - 1;
                wm &= wm - 1;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int n = lane + 32 * c;
                    if (n < N) {
                        const float2 v = sPart[(p * NW + b) * N + n];
                        axb[c].x += v.x;
                        axb[c].y += v.y;
                    }
                }
            }
            // sums over the grid: lane b < NW holds block b's partial sums
            float4 rd = (lane < NW) ? sRed[lane * TPG + p] : make_float4(0.f, 0.f, 0.f, 0.f);
            float lhs = 0.f, res = 0.f;
            float2 gg[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                gg[c] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int n = lane + 32 * c;
                if (n < N) {
                    const float2 ay = sAy[p * N + n];
                    gg[c] = sG[p * N + n];
                    const float d0 = axb[c].x - ay.x, d1 = axb[c].y - ay.y;
                    lhs = fmaf(d0, d0, fmaf(d1, d1, lhs));
                    const float e0 = axb[c].x - gg[c].x, e1 = axb[c].y - gg[c].y;
                    res = fmaf(e0, e0, fmaf(e1, e1, res));
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                lhs += __shfl_xor_sync(0xffffffffu, lhs, off);
                res += __shfl_xor_sync(0xffffffffu, res, off);
                rd.x += __shfl_xor_sync(0xffffffffu, rd.x, off);
                rd.y += __shfl_xor_sync(0xffffffffu, rd.y, off);
                rd.z += __shfl_xor_sync(0xffffffffu, rd.z, off);
                rd.w += __shfl_xor_sync(0xffffffffu, rd.w, off);
            }
            const float dd = rd.x, l1 = rd.y, dx = rd.z, xn = rd.w;
            const float al = S.alpha[p];
            const bool dead = TC && S.abort != 0;  // the gradient of this sweep is stale
            const bool bt_ok = dead || lhs <= dd / (2.f * al);
            const int nbt_it = S.nbt_it[p];
            __syncwarp();
            if (!bt_ok && nbt_it < a.max_bt) {
                // Eq. 15 failed: the next sweep redoes the prox with the smaller step
                if (lane == 0) {
                    const float an = al * a.c_alpha;
                    S.alpha[p] = an;
                    S.nbt[p] += 1;
                    S.nbt_it[p] = nbt_it + 1;
                    S.par[p] = make_float4(S.par[p].x, 2.f * an, an * S.lam[p], __int_as_float(T_ACTIVE));
                }
                continue;
            }
            const float Fb = fmaf(S.lam[p], l1, res);
            const bool accepted = !dead && (Fb <= S.Fx[p]);
            const bool conv = !dead && ((dx <= tol2 * xn) || (dx == 0.f));
            const int k = S.k[p];
            const bool fin = dead || conv || (k >= a.max_iter);
            // N-space state: A x^{k-1} <- A x^k, A x^k <- A xbar (accepted); for the next
            // iteration A y = A x + beta (A x - A x_prev), r = A y - g
            const float beta_n = (float)(k - 1) / (float)(k + 2);
            __syncwarp();  // every lane has read the slot state lane 0 updates below
            if (!fin) {
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int n = lane + 32 * c;
                    if (n < N) {
                        const float2 axo = sAx[p * N + n];
                        const float2 axn = accepted ? axb[c] : axo;
                        sAxp[p * N + n] = axo;
                        sAx[p * N + n] = axn;
                        const float2 ayn = make_float2(fmaf(beta_n, axn.x - axo.x, axn.x),
                                                       fmaf(beta_n, axn.y - axo.y, axn.y));
                        sAy[p * N + n] = ayn;
                        put_r(p, n, ayn.x - gg[c].x, ayn.y - gg[c].y);
                    }
                }
            }
            int nbits = T_SHIFT | (accepted ? T_ACC : 0);
            if (lane == 0) {
                int st = S.status[p];
                if (!bt_ok)
                    st |= BPDN_PX_BT_LIMIT;
                if (fin && !conv)
                    st |= BPDN_PX_NOT_CONVERGED;
                if (dead)
                    st |= BPDN_PX_DEVICE_TIMEOUT;
                int nz = S.nnz[p];
                if (accepted) {
                    S.Fx[p] = Fb;
                    nz = nnz;
                    S.nnz[p] = nz;
                }
                S.status[p] = st;
                if (fin) {
                    const long long q = S.pix[p];
                    a.status[q] = (nz == 0) ? (st | BPDN_PX_ZERO_SOLUTION) : st;
                    a.iters[q] = k;
                    if (a.nbt)
                        a.nbt[q] = S.nbt[p];
                    if (a.nsupp)
                        a.nsupp[q] = nz;
                    S.pix_out[p] = q;
                } else {
                    S.k[p] = k + 1;
                    S.nbt_it[p] = 0;
                    S.par[p] = make_float4(beta_n, S.par[p].y, S.par[p].z, __int_as_float(nbits | T_ACTIVE));
                }
            }
            if (fin) {
                __syncwarp();
                nbits |= T_OUT | refill(p);
                __syncwarp();
                if (lane == 0)
                    S.par[p].w = __int_as_float(nbits);
            }
        }
        if constexpr (TC)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B rows for the MMA
        tc_fence_before();
        group_sync(grp, 32 * NW);
    }
    // this group has drained and its last MMA was waited for: retire its mbarrier.  After
    // a wait that ran out, give the MMA that was not seen complete one more bounded wait,
    // so that it no longer writes tensor memory or arrives on the barrier afterwards.
    if constexpr (TC) {
        if (blk == 0 && lane == 0) {
            if (S.abort)
                (void)mbar_wait(mbar, S.abort_ph);
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
        }
    }
}

// The persistent kernel: every CTA walks the launch's stacks in order and works on
// each one it may take (blockIdx.x < ctas) while that stack has pixels left.
template <bool TC, bool SA, int MAXT, int NCH>
__global__ void __launch_bounds__(MAXT, 1) k_rbpg(const __grid_constant__ Params prm)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_go;
    const int w = threadIdx.x >> 5;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    for (int si = 0; si < prm.nstacks; ++si) {
        const StackDesc &sd = prm.st[si];
        if ((int)blockIdx.x >= sd.ctas)
            continue;
        if (threadIdx.x == 0)
            s_go = (*(volatile unsigned long long *)sd.a.counter < (unsigned long long)sd.a.P) ? 1 : 0;
        __syncthreads();
        const int go = s_go;
        __syncthreads();  // everyone has read s_go before it is written again
        if (!go)
            continue;  // the other CTAs took every pixel of this stack
        run_stack<TC, SA, NCH>(sd, tmem, smem_raw);
        tc_fence_before();
        __syncthreads();  // every group of this stack has drained; no MMA in flight
        tc_fence_after();
    }
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// launch shape of one solve
struct Plan {
    int groups, threads;
    bool smem_a;
    int nch;  // BF16: rows per lane (contraction length 64 or 128)
    size_t smem;
};

// Pick groups per CTA and where A lives.  FP32: A in shared memory before A in global
// memory (its contraction reads A every sweep), then more groups before fewer.  BF16 (A only
// feeds A xbar): two or more groups with A in shared memory, then two or more with A in
// global memory (more before fewer), then one group.
// Threads (832 BF16, 1024 FP32), tensor-memory columns and shared memory bound the groups:
// two at L = 400, up to eight on grids of at most 128 points.  A fixed groups count is taken
// when asked for.  BF16 solves with N <= 32 use K = 64 where A
// fits in shared memory, else K = 128 (the zero padding adds exact zeros: same results).
// Returns an empty string on success, else the reason.
const char *make_plan(const OpHandle &op, bool tc, int groups, int max_smem, Plan *pl)
{
    if (op.Lpad > 32 * kMaxNW)
        return "the iteration kernel handles L <= 1024";
    if (tc && (2 * op.N > kK2 || op.Lpad > 512))
        return "precision 1 (BF16 tensor cores) needs 2N <= 128 and L <= 512";
    const int T = (op.Lpad + 127) / 128;
    const size_t abytes = a_bytes(op.N, op.lda);
    // candidates (groups, A in shared memory) in order of preference
    int cg[2 * kMaxGroups];
    bool csa[2 * kMaxGroups];
    int nc = 0;
    for (int i = 0; i < 2 * kMaxGroups; ++i) {
        if (tc) {
            // two or more groups with A in shared memory, then with A in global memory,
            // then one group
            const int j = i < 2 * (kMaxGroups - 1) ? i % (kMaxGroups - 1) : 0;
            cg[nc] = i < 2 * (kMaxGroups - 1) ? kMaxGroups - j : 1;
            csa[nc] = i < 2 * (kMaxGroups - 1) ? (i < kMaxGroups - 1) : (i == 2 * (kMaxGroups - 1));
        } else {
            cg[nc] = kMaxGroups - i % kMaxGroups;
            csa[nc] = i < kMaxGroups;
        }
        ++nc;
    }
    for (int c = 0; c < nc; ++c) {
        {
            const int g = cg[c];
            const bool smem_a = csa[c];
            if (groups && g != groups)
                continue;
            const int nch = tc ? ((2 * op.N <= kK1 && smem_a) ? 1 : 2) : 0;
            const int kk = tc ? tc_k(nch) : 0;
            const GroupLayout lay = group_layout(op.N, op.Lpad, tc, kk);
            const int W = warps_for(op.Lpad, g);
            // the BF16 variant is built for at most 832 threads, the FP32 ones for 1024
            if (32 * W > (tc ? 832 : 1024) || tmem_cols_used(T, g, tc, kk) > kTmemCols)
                continue;
            const size_t smem = (smem_a ? abytes : 0) + (size_t)g * lay.bytes;
            if (smem > (size_t)max_smem)
                continue;
            pl->groups = g;
            pl->threads = 32 * W;
            pl->smem_a = smem_a;
            pl->nch = nch;
            pl->smem = smem;
            return "";
        }
    }
    return groups ? "this tile_pixels does not fit the iteration kernel at these N and L"
                  : "the iteration kernel's shared memory does not fit (N and L too large)";
}

template <bool TC, bool SA, int MAXT, int NCH>
cudaError_t launch_variant(const Params &prm, int threads, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_rbpg<TC, SA, MAXT, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_rbpg<TC, SA, MAXT, NCH><<<grid, threads, smem, s>>>(prm);
    return cudaGetLastError();
}

static_assert(sizeof(Params) <= 32000, "kernel parameters must stay below 32 KB");

}  // namespace

const char *rbpg_check(const OpHandle &op, int precision, int groups, int max_smem)
{
    Plan pl;
    return make_plan(op, precision == 1, groups, max_smem, &pl);
}

cudaError_t launch_rbpg_batch(const OpHandle *const *ops, const SolveLaunch *as, int n, int num_sms, cudaStream_t s)
{
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    struct Item {
        int i;
        Plan pl;
    };
    // kernel variant: precision, rows per lane, where A lives, launch bound
    std::vector<Item> byvar[16];
    for (int i = 0; i < n; ++i) {
        if (as[i].P <= 0)
            continue;
        Item it;
        it.i = i;
        const bool tc = (as[i].precision == 1);
        if (make_plan(*ops[i], tc, as[i].groups, max_smem, &it.pl)[0] != '\0')
            return cudaErrorInvalidValue;
        // FP32: three rows per lane beyond N = 64; BF16: two rows per lane (K = 128)
        const bool wide = tc ? it.pl.nch == 2 : ops[i]->N > 64;
        byvar[(tc ? 8 : 0) + (wide ? 4 : 0) + (it.pl.smem_a ? 2 : 0) + (it.pl.threads > 832 ? 1 : 0)].push_back(it);
    }
    std::unique_ptr<Params> prm(new Params);
    for (int v = 0; v < 16; ++v) {
        std::vector<Item> &list = byvar[v];
        // small stacks first: the large pools at the end absorb the CTAs' uneven progress
        std::stable_sort(list.begin(), list.end(), [&](const Item &x, const Item &y) { return as[x.i].P < as[y.i].P; });
        for (size_t c0 = 0; c0 < list.size(); c0 += kMaxStacks) {
            const size_t c1 = std::min(list.size(), c0 + (size_t)kMaxStacks);
            prm->nstacks = (int)(c1 - c0);
            int threads = 32, grid = 1;
            size_t smem = 0;
            for (size_t k = c0; k < c1; ++k) {
                const Item &it = list[k];
                const OpHandle &op = *ops[it.i];
                StackDesc &sd = prm->st[k - c0];
                sd.A_re = op.A_re;
                sd.A_im = op.A_im;
                sd.N = op.N;
                sd.L = op.L;
                sd.Lpad = op.Lpad;
                sd.lda = op.lda;
                sd.groups = it.pl.groups;
                sd.a = as[it.i];
                // one stack alone: up to one pixel per slot; a batch: at least four pixels per
                // slot per CTA, so that the drain at each stack switch stays small
                const long long per = (n == 1 ? 1LL : 4LL) * TPG * it.pl.groups;
                const long long want = (as[it.i].P + per - 1) / per;
                sd.ctas = (int)std::max(1LL, std::min((long long)num_sms, want));
                threads = std::max(threads, it.pl.threads);
                grid = std::max(grid, sd.ctas);
                smem = std::max(smem, it.pl.smem);
            }
            // one CTA per SM: each CTA allocates all 512 tensor-memory columns
            if (smem < (size_t)max_smem / 2 + 1024)
                smem = (size_t)max_smem / 2 + 1024;
            const bool tc = (v & 8) != 0, wide = (v & 4) != 0, sa = (v & 2) != 0, big = (v & 1) != 0;
            if (tc && !wide)
                e = launch_variant<true, true, 832, 1>(*prm, threads, grid, smem, s);
            else if (tc)
                e = sa ? launch_variant<true, true, 832, 2>(*prm, threads, grid, smem, s)
                       : launch_variant<true, false, 832, 2>(*prm, threads, grid, smem, s);
            else if (!wide && sa)
                e = big ? launch_variant<false, true, 1024, 2>(*prm, threads, grid, smem, s)
                        : launch_variant<false, true, 832, 2>(*prm, threads, grid, smem, s);
            else if (!wide)
                e = big ? launch_variant<false, false, 1024, 2>(*prm, threads, grid, smem, s)
                        : launch_variant<false, false, 832, 2>(*prm, threads, grid, smem, s);
            else if (sa)
                e = big ? launch_variant<false, true, 1024, 3>(*prm, threads, grid, smem, s)
                        : launch_variant<false, true, 832, 3>(*prm, threads, grid, smem, s);
            else
                e = big ? launch_variant<false, false, 1024, 3>(*prm, threads, grid, smem, s)
                        : launch_variant<false, false, 832, 3>(*prm, threads, grid, smem, s);
            if (e != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_rbpg(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
{
    const OpHandle *ops[1] = {&op};
    return launch_rbpg_batch(ops, &a, 1, num_sms, s);
}

}  // namespace bpdn
