// Persistent iteration kernel with the gradient contraction on the tensor cores:
// Algorithm 1 (RBPG with backtracking) for many pixels that share one operator,
// with sum_n conj(A_nl) r_n computed by tcgen05 MMAs from BF16 operands into FP32
// accumulators in tensor memory; everything else (iterate, prox, line search,
// accept and stopping tests, A xbar) stays in FP32 exactly as in the CUDA-core
// kernel (rbpg.cu).
//
// The contraction, per group of 8 pixel slots and per 128-row tile of the grid:
//   D_re[l, p] = sum_k Aop_re[l, k] R[p, k],   D_im[l, p] = sum_k Aop_im[l, k] R[p, k]
// with K = 64 (2N <= 64, zero padded), R[p, :] = (Re r_p, Im r_p) in BF16 written by the
// decision phase into shared memory (canonical K-major layout, no swizzle), and the
// constant operator rows
//   Aop_re[l, :] = ( Re A[:, l],  Im A[:, l]),   Aop_im[l, :] = (-Im A[:, l], Re A[:, l])
// in BF16 held in tensor memory for the whole launch.  M = 128, N = 16 (rows 8..15 of
// R are zero).  One thread per group issues the MMAs and commits them to the group's
// mbarrier; every thread then reads its own row (TMEM lane = l mod 128) with
// tcgen05.ld.  Warps are interleaved between groups four at a time so that the warp
// holding rows 32q..32q+31 of a tile has index = q mod 4, as tensor-memory access needs.
//
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int TPG = 8;          // pixel slots per group
constexpr int kMaxGroups = 2;   // groups per CTA (named barriers 1..kMaxGroups)
constexpr int kMaxThreads = 928;  // 29 warps: two groups of L = 416 interleaved by 4 warps
constexpr int kK = 64;          // contraction length 2N padded to a multiple of 16
constexpr int kTmemCols = 512;  // D: 128 columns per group; operator rows: 256 columns
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
    size_t Bop, mbar, Xb, Xp, mask, G, Ax, Axp, Ay, red, part, st, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline GroupLayout group_layout(int N, int Lpad)
{
    GroupLayout s;
    const int NW = Lpad / 32;
    size_t o = 0;
    s.Bop = o;  o = align16(o + 16 * kK * 2);   // R: 16 rows x K bf16, core-matrix layout
    s.mbar = o; o = align16(o + 8);
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

// byte offset of element (row, k) of a K-major operand with kK columns, no swizzle:
// core matrices of 8 rows x 16 bytes; the K-adjacent core matrix 128 bytes on (LBO),
// the next 8-row group kK/8 * 128 bytes on (SBO)
__host__ __device__ inline int kmaj_off(int row, int k)
{
    return (row >> 3) * (kK / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
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

// 8 consecutive FP32 columns of this warp's 32 tensor-memory lanes
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

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}

// R row p (BF16): (Re r, Im r) at k = n and k = N + n
__device__ __forceinline__ void put_r(unsigned char *bop, int p, int n, int N, float re, float im)
{
    *(__nv_bfloat16 *)(bop + kmaj_off(p, n)) = __float2bfloat16_rn(re);
    *(__nv_bfloat16 *)(bop + kmaj_off(p, N + n)) = __float2bfloat16_rn(im);
}

__global__ void __launch_bounds__(kMaxThreads, 1) k_rbpg_bf16(Params prm, int G)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    const int N = prm.N, L = prm.L, Lpad = prm.Lpad, lda = prm.lda;
    const int NW = Lpad / 32;  // warps per group
    // warp w = 4 (t G + g) + q: tile t of group g, lane quadrant q
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q4 = w & 3, tg = w >> 2;
    const int tile = tg / G, grp = tg - tile * G;
    const int tid = 128 * tile + 32 * q4 + lane;  // grid index l owned by this thread
    const bool live = tid < Lpad;                 // warps of the last tile beyond Lpad idle
    const int warp = tid >> 5;                    // warp within the group (l / 32)
    const SolveLaunch &a = prm.a;
    float2 *sA = (float2 *)smem_raw;  // [N][lda] (re, im)
    const GroupLayout lay = group_layout(N, Lpad);
    unsigned char *gbase = smem_raw + a_bytes(N, lda) + (size_t)grp * lay.bytes;
    unsigned char *sBop = gbase + lay.Bop;           // R of this group (BF16 operand)
    const uint32_t mbar = smem_u32(gbase + lay.mbar);
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
    if (live) {
        for (int i = tid; i < TPG * Lpad; i += Lpad)
            sXp[i] = make_float2(0.f, 0.f);
        for (int i = tid; i < 16 * kK * 2 / 4; i += Lpad)
            ((uint32_t *)sBop)[i] = 0u;  // rows 8..15 of R stay zero
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
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    // operator rows of this thread's grid index into tensor memory (group 0 writes them
    // for both groups): columns 256 + 64 tile (+32 for the imaginary-output rows)
    if (live && grp == 0) {
        const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + 256 + 64 * tile;
        // Aop_re row at column 0, Aop_im row at column 32; 16 columns (32 elements) at a time
        for (int part = 0; part < 4; ++part) {
            const int im_row = part >> 1, c0 = 16 * (part & 1);
            uint32_t v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float e2[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int k = 2 * (c0 + c) + e;
                    float val = 0.f;
                    if (k < N)
                        val = im_row ? -sA[k * lda + tid].y : sA[k * lda + tid].x;
                    else if (k < 2 * N)
                        val = im_row ? sA[(k - N) * lda + tid].x : sA[(k - N) * lda + tid].y;
                    e2[e] = val;
                }
                v[c] = pack_bf16(e2[0], e2[1]);
            }
            tmem_st16(ta + 32 * im_row + c0, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();  // A, operator rows and R padding complete for every group
    tc_fence_after();
    if (!live) {
        // idle warp of the last tile: wait for the groups to finish, then leave
        __syncthreads();
        return;
    }
    float2 x[TPG];
#pragma unroll
    for (int p = 0; p < TPG; ++p)
        x[p] = make_float2(0.f, 0.f);
    uint32_t mma_phase = 0;
    // issue this group's gradient MMAs (one thread per group)
    auto issue_mma = [&]() {
        if (tid == 0) {
            tc_fence_after();
            const uint32_t b0 = smem_u32(sBop);
            const int tiles = (Lpad + 127) / 128;
            for (int t = 0; t < tiles; ++t)
                for (int half = 0; half < 2; ++half) {
                    const uint32_t d = tmem + 128 * grp + 32 * t + 16 * half;
                    const uint32_t arow = tmem + 256 + 64 * t + 32 * half;
#pragma unroll
                    for (int j = 0; j < kK / 16; ++j)
                        tc_mma_ts(d, arow + 8 * j, smem_desc(b0 + 256 * j, 128, (kK / 8) * 128), j > 0);
                }
            tc_commit(mbar);
        }
    };

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
                        put_r(sBop, p, n, N, -gg.x, -gg.y);
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
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
            issue_mma();  // R of every slot is in place
        }

        // ---------------- B: gradient sum_n conj(A_nl) r_n for l = tid, from the MMAs -----------
        float2 gx[TPG / 2], gy[TPG / 2];  // slot pairs (2q, 2q+1): real and imaginary parts
        {
            if (!mbar_wait(mbar, mma_phase) && a.err)
                atomicExch(a.err, 1);
            mma_phase ^= 1u;
            tc_fence_after();
            float vre[8], vim[8];
            const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + 128 * grp + 32 * tile;
            tmem_ld8(ta, vre);
            tmem_ld8(ta + 16, vim);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            tc_fence_before();
#pragma unroll
            for (int q = 0; q < TPG / 2; ++q) {
                gx[q] = make_float2(vre[2 * q], vre[2 * q + 1]);
                gy[q] = make_float2(vim[2 * q], vim[2 * q + 1]);
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
                            put_r(sBop, p, n, N, ay.x - gg.x, ay.y - gg.y);
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
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // R rows for the MMA
            group_sync(grp, Lpad);
            ++sweep;
            if (S.retry[round % 3] == 0)
                break;
        }
        if (S.nfin == 0)
            issue_mma();  // no slot to refill: the next gradient overlaps the register update

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
    // every group has finished and no MMA is in flight: release tensor memory
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// warps of a CTA with G groups: 4 per tile and group, the last tile only as many as it needs
int warps_for(int Lpad, int G)
{
    const int T = (Lpad + 127) / 128;
    const int qlast = (Lpad - 128 * (T - 1)) / 32;
    return 4 * (T * G - 1) + qlast;
}

int choose_groups(const OpHandle &op, int max_smem, size_t *smem_out)
{
    const GroupLayout lay = group_layout(op.N, op.Lpad);
    const size_t base = a_bytes(op.N, op.lda);
    int g = kMaxGroups;
    while (g > 1 && (32 * warps_for(op.Lpad, g) > kMaxThreads ||
                     base + (size_t)g * lay.bytes > (size_t)max_smem))
        --g;
    *smem_out = base + (size_t)g * lay.bytes;
    return g;
}

}  // namespace

bool rbpg_tc_supported(const OpHandle &op, int max_smem)
{
    if (2 * op.N > kK || op.Lpad > 512)
        return false;
    size_t smem = 0;
    choose_groups(op, max_smem, &smem);
    return smem <= (size_t)max_smem && 32 * warps_for(op.Lpad, 1) <= kMaxThreads;
}

cudaError_t launch_rbpg_tc(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
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
    e = cudaFuncSetAttribute(k_rbpg_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const long long tiles = (a.P + (long long)groups * TPG - 1) / ((long long)groups * TPG);
    int grid = (int)((tiles < num_sms) ? tiles : num_sms);
    if (grid < 1)
        grid = 1;
    k_rbpg_bf16<<<grid, 32 * warps_for(op.Lpad, groups), smem, s>>>(prm, groups);
    return cudaGetLastError();
}

}  // namespace bpdn
