// Pixel-per-thread iteration kernel: Algorithm 1 (RBPG with backtracking, Eqs. 11-15)
// with the gradient contraction on the tensor cores (BF16 operands, FP32 accumulation)
// and one pixel per thread for everything else.
//
// A CTA holds kTiles tiles of 128 pixel slots; thread i of tile t owns slot (t, i) and is
// tensor-memory lane i of that tile's accumulators.  One sweep of a tile:
//   1. every thread forms its pixel's residual r = A y - g in N space (FP32, from the
//      kept A x^k - g and A x^{k-1} - g: A y - g = (1 + beta)(A x^k - g) - beta (A x^{k-1} - g))
//      and stores it, rounded to BF16, as its row of the MMA's A operand in tensor memory:
//      R[i, :] = (Re r, Im r, 0 ...), K = 64;
//   2. the gradient sum_n conj(A_nl) r_n of all 128 pixels comes out in chunks of 32 grid
//      points: D[i, 2l] + j D[i, 2l + 1] = (R B^T)[i, .] with the operator rows
//      B[2l] = (Re A[:, l], Im A[:, l]), B[2l + 1] = (-Im A[:, l], Re A[:, l]) (BF16, in
//      shared memory for the whole launch), M = 128, N = 64 per chunk, two accumulator
//      buffers so that the MMA of chunk c + 2 overlaps the processing of chunk c;
//   3. each thread walks its pixel's grid points in ascending order: the extrapolation
//      y = x + beta (x - x^{k-1}) (Eqs. 11-12), the complex soft threshold (Eq. 10 read
//      for complex values) of v = y - 2 alpha grad, and the sums that Eq. 15, F and the
//      stopping test need, all in FP32 registers;
//   4. A xbar over the nonzeros of xbar (FP32 A in shared memory), Eq. 15, the monotone
//      accept, the stopping test, and the slot's refill when its pixel is done.
// The iterates are sparse: x^k, x^{k-1} and xbar are lists of (grid index, value) in
// ascending order, three buffers per slot in global memory (the touched part stays in
// L2), merged with the dense gradient as the thread walks the grid.  Every sum runs in
// one thread in a fixed order, so the results do not depend on timing.
//
// Scope: precision 1, 2N <= 64, and A (FP32) plus the BF16 operator rows within shared
// memory; other solves run the grid-point-per-thread kernel (rbpg.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kTiles = 2;         // tiles of 128 pixel slots per CTA
constexpr int kSlots = 128;       // MMA M: pixel slots per tile
constexpr int kK = 64;            // contraction length 2N, zero padded
constexpr int kChunkPts = 32;     // grid points per gradient chunk
constexpr int kChunkCols = 64;    // accumulator columns per chunk (re, im per grid point)
constexpr int kColR = 0;          // tensor-memory columns of a tile: R (32), then two chunks
constexpr int kColD = 32;
constexpr int kTileCols = 32 + 2 * kChunkCols;  // 160
constexpr int kTmemCols = 512;
static_assert(kTiles * kTileCols <= kTmemCols, "tensor memory of the tiles");

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// byte offset of element (row, k) of a K-major BF16 operand with kK columns, no swizzle:
// core matrices of 8 rows x 16 bytes; the K-adjacent core matrix 128 bytes on (LBO), the
// next 8-row group kK/8 * 128 bytes on (SBO)
__host__ __device__ inline size_t kmaj_off(int row, int k)
{
    return (size_t)(row >> 3) * (kK / 8) * 128 + (size_t)(k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kChunkCols >> 3) << 17) |
                            ((128u >> 4) << 24);

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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st32u(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

// barrier of the 128 threads of tile t (named barriers 1..kTiles; 0 is __syncthreads)
__device__ __forceinline__ void tile_sync(int t) { asm volatile("bar.sync %0, %1;" ::"r"(t + 1), "r"(kSlots) : "memory"); }

// shared memory: the BF16 operator rows (K-major, 2L rows padded to whole chunks), A in
// FP32 [L][N] (row l contiguous for the thread that gathers A xbar), then small per-tile state
struct SmemLayout {
    size_t B, A, bar, flag, bytes;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline int chunks_of(int L) { return (L + kChunkPts - 1) / kChunkPts; }

__host__ __device__ inline SmemLayout smem_layout(int N, int L)
{
    SmemLayout s;
    size_t o = 0;
    s.B = o;    o = al16(o + (size_t)chunks_of(L) * kChunkCols * kK * 2);
    s.A = o;    o = al16(o + sizeof(float2) * (size_t)L * N);
    s.bar = o;  o = al16(o + sizeof(uint64_t) * 2 * kTiles);
    s.flag = o; o = al16(o + sizeof(int) * 8 * kTiles);  // per tile: 4 warp flags, the timeout flag, 3 spare
    s.bytes = o;
    return s;
}

// per-slot scratch in global memory: A x - g for the two kept iterates (2 x 2N floats),
// then three iterate lists (indices uint16 [L], values float2 [L] each)
struct SlotLayout {
    size_t U, LM, LV, bytes;
};

// per-slot scratch in global memory: A x - g of the two kept iterates ([2][N] complex), then
// three sparse iterates, each a 32-bit mask per 32-point chunk of the grid (bit j: grid point
// 32 c + j is nonzero) and its nonzero values packed in ascending order
__host__ __device__ inline SlotLayout slot_layout(int N, int L)
{
    SlotLayout s;
    size_t o = 0;
    s.U = o;  o = al16(o + sizeof(float2) * 2 * (size_t)N);
    s.LM = o; o = al16(o + sizeof(uint32_t) * 3 * (size_t)chunks_of(L));
    s.LV = o; o = al16(o + sizeof(float2) * 3 * (size_t)L);
    s.bytes = (o + 255) & ~(size_t)255;
    return s;
}

struct PxParams {
    const float *A_re, *A_im;  // planar FP32 tables [N][lda]
    int N, L, lda;
    size_t slot_bytes;
    SolveLaunch a;
};

// the MMAs of gradient chunk c into accumulator buffer buf of tile t, committed to its mbarrier
__device__ __forceinline__ void issue_chunk(uint32_t tbase, uint32_t bbase, uint32_t mbar, int c, int buf)
{
    const uint32_t d = tbase + kColD + kChunkCols * buf;
    const uint32_t brow = bbase + (uint32_t)kmaj_off(kChunkCols * c, 0);
#pragma unroll
    for (int j = 0; j < kK / 16; ++j)
        tc_mma_ts(d, tbase + kColR + 8 * j, smem_desc(brow + 256 * j, 128, (kK / 8) * 128), j > 0);
    tc_commit(mbar);
}

__global__ void __launch_bounds__(kTiles * kSlots, 1) k_rbpg_px(const __grid_constant__ PxParams prm)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    const int N = prm.N, L = prm.L, lda = prm.lda;
    const SolveLaunch &a = prm.a;
    const SmemLayout lay = smem_layout(N, L);
    unsigned char *sB = smem_raw + lay.B;
    float2 *sA = (float2 *)(smem_raw + lay.A);
    uint64_t *sbar = (uint64_t *)(smem_raw + lay.bar);
    int *sflag = (int *)(smem_raw + lay.flag);  // per tile: [0..3] warps with a pixel, [4] wait ran out
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int tile = tid / kSlots, slot_i = tid % kSlots;  // slot_i = tensor-memory lane of the tile
    const int NC = chunks_of(L);

    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // operator rows, two BF16 K elements per 32-bit word: row 2l = (Re A[:, l], Im A[:, l]),
    // row 2l + 1 = (-Im A[:, l], Re A[:, l]); zero for l >= L and for K >= 2N
    for (int e = tid; e < NC * kChunkCols * (kK / 2); e += blockDim.x) {
        const int row = e / (kK / 2), kp = e % (kK / 2);
        const int l = row >> 1, im = row & 1;
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * kp + h;
            float val = 0.f;
            if (l < L) {
                if (k < N)
                    val = im ? -prm.A_im[k * lda + l] : prm.A_re[k * lda + l];
                else if (k < 2 * N)
                    val = im ? prm.A_re[(k - N) * lda + l] : prm.A_im[(k - N) * lda + l];
            }
            v[h] = val;
        }
        *(uint32_t *)(sB + kmaj_off(row, 2 * kp)) = pack_bf16(v[0], v[1]);
    }
    for (int e = tid; e < L * N; e += blockDim.x) {
        const int l = e / N, n = e - (e / N) * N;
        sA[e] = make_float2(prm.A_re[n * lda + l], prm.A_im[n * lda + l]);
    }
    if (tid < 2 * kTiles)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(sbar + tid)));
    if (tid < 8 * kTiles)
        sflag[tid] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B rows for the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tbase = tmem + tile * kTileCols;                       // lane 0 of this tile
    const uint32_t lbase = tbase + ((uint32_t)(32 * (w & 3)) << 16);       // this warp's lanes
    const uint32_t bbase = smem_u32(sB);
    const uint32_t mbar0 = smem_u32(sbar + 2 * tile), mbar1 = smem_u32(sbar + 2 * tile + 1);
    int *tflag = sflag + 8 * tile;

    // the slot's scratch (this thread's, and any slot of the warp for the cooperative parts)
    const SlotLayout SL = slot_layout(N, L);
    unsigned char *const slot0 = a.px_scratch + (size_t)(blockIdx.x * (kTiles * kSlots) + tid - lane) * prm.slot_bytes;
    auto slot_of = [&](int t) -> unsigned char * { return slot0 + (size_t)t * prm.slot_bytes; };
    unsigned char *slot = slot_of(lane);
    float2 *U = (float2 *)(slot + SL.U);        // [2][N]
    uint32_t *LM = (uint32_t *)(slot + SL.LM);  // [3][NC]
    float2 *LV = (float2 *)(slot + SL.LV);      // [3][L]

    long long pix = -1;
    int k = 0, nbt = 0, nbt_it = 0, st = 0, nnz = 0;
    float alpha = 0.f, Fx = 0.f, lam = 0.f, beta = 0.f;
    int bx = 0, bxp = 0, nx = 0, nxp = 0;  // buffers and nonzero counts of x^k and x^{k-1}
    int ub = 0, upb = 0;                   // U buffers of A x^k - g and A x^{k-1} - g
    bool aborted = false;                  // this tile's tensor-core wait ran out

    // take the next pixel from the work counter (x^0 = x^{-1} = 0: A x - g = -g)
    auto refill = [&]() {
        for (;;) {
            const unsigned long long q = atomicAdd(a.counter, 1ULL);
            if (q >= (unsigned long long)a.P) {
                pix = -1;
                return;
            }
            const float2 *gq = a.g + (size_t)q * N;
            bool fin = true;
            float gg2 = 0.f;
            for (int n = 0; n < N; ++n) {
                const float2 gv = gq[n];
                fin = fin && isfinite(gv.x) && isfinite(gv.y);
                gg2 = fmaf(gv.x, gv.x, fmaf(gv.y, gv.y, gg2));
                U[n] = make_float2(-gv.x, -gv.y);
            }
            if (!fin || a.max_iter <= 0 || aborted) {
                float2 *xq = a.x + (size_t)q * L;
                for (int l = 0; l < L; ++l)
                    xq[l] = make_float2(0.f, 0.f);
                a.status[q] = aborted ? (BPDN_PX_DEVICE_TIMEOUT | BPDN_PX_ZERO_SOLUTION)
                              : fin   ? (BPDN_PX_NOT_CONVERGED | BPDN_PX_ZERO_SOLUTION)
                                      : BPDN_PX_NONFINITE;
                a.iters[q] = 0;
                if (a.nbt)
                    a.nbt[q] = 0;
                if (a.nsupp)
                    a.nsupp[q] = 0;
                continue;
            }
            pix = (long long)q;
            ub = upb = 0;
            bx = bxp = 0;
            nx = nxp = 0;
            k = 1;
            alpha = a.alpha0;
            Fx = gg2;  // F(0) = ||g||^2
            lam = a.lam_pp ? a.lam[q] : a.lam[0];
            beta = 0.f;  // multiplies x - x_prev = 0 at k = 1
            nbt = nbt_it = st = nnz = 0;
            return;
        }
    };
    refill();
    uint32_t ph0 = 0, ph1 = 0;

    for (;;) {
        // does any slot of this tile hold a pixel?  (a tile-uniform decision)
        const unsigned bal = __ballot_sync(0xffffffffu, pix >= 0);
        if (lane == 0)
            tflag[w & 3] = (bal != 0u) ? 1 : 0;
        tile_sync(tile);
        const int any = tflag[0] | tflag[1] | tflag[2] | tflag[3];
        aborted = tflag[4] != 0;
        tile_sync(tile);  // every thread has read the flags before they are written again
        if (!any)
            break;
        const bool act = pix >= 0;

        // ---- 1. residual r = (1 + beta)(A x^k - g) - beta (A x^{k-1} - g) as this thread's BF16 row:
        // element kk = Re r_kk (kk < N), Im r_{kk-N} (N <= kk < 2N), 0 beyond
        {
            uint32_t rw[32];
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                float e[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kk = 2 * p + h;
                    float v = 0.f;
                    if (act && kk < 2 * N) {
                        const int n = (kk < N) ? kk : kk - N;
                        const float2 u = U[ub * N + n], up = U[upb * N + n];
                        v = (kk < N) ? fmaf(beta, u.x - up.x, u.x) : fmaf(beta, u.y - up.y, u.y);
                    }
                    e[h] = v;
                }
                rw[p] = pack_bf16(e[0], e[1]);
            }
            tmem_st32u(lbase + kColR, rw);
            tmem_wait_st();
        }
        tc_fence_before();
        tile_sync(tile);
        tc_fence_after();
        if (slot_i == 0 && !aborted) {
            issue_chunk(tbase, bbase, mbar0, 0, 0);
            if (NC > 1)
                issue_chunk(tbase, bbase, mbar1, 1, 1);
        }

        // ---- 2. gradient chunks: prox and sums, grid points in ascending order
        const float a2 = 2.f * alpha, tau = alpha * lam;
        const uint32_t *mkx = LM + bx * NC, *mkp = LM + bxp * NC;
        const float2 *vlx = LV + bx * L, *vlp = LV + bxp * L;
        const int bb = (bx == bxp) ? (bx + 1) % 3 : 3 - bx - bxp;  // the free buffer: xbar
        uint32_t *mkb = LM + bb * NC;
        float2 *vlb = LV + bb * L;
        int ox = 0, op = 0, nb = 0;  // values consumed / written so far
        float dd = 0.f, l1 = 0.f, dx = 0.f, xn = 0.f;
        for (int c = 0; c < NC; ++c) {
            const int buf = c & 1;
            const uint32_t mb = buf ? mbar1 : mbar0;
            // this chunk's nonzero masks of x^k and x^{k-1} (loaded before the wait)
            const uint32_t mx = (act && nx > 0) ? mkx[c] : 0u;
            const uint32_t mp = (act && nxp > 0) ? mkp[c] : 0u;
            if (!aborted && tflag[4] == 0) {  // no wait for MMAs that a timed-out tile never issued
                if (!mbar_wait(mb, buf ? ph1 : ph0)) {
                    atomicExch(tflag + 4, 1);
                    if (a.err)
                        atomicExch(a.err, 1);
                }
                if (buf)
                    ph1 ^= 1u;
                else
                    ph0 ^= 1u;
            }
            __syncwarp();  // lanes leave the polling loop apart: reconverge before tcgen05.ld
            tc_fence_after();
            float d0[32], d1[32];
            tmem_ld32(lbase + kColD + kChunkCols * buf, d0);
            tmem_ld32(lbase + kColD + kChunkCols * buf + 32, d1);
            tmem_wait_ld();
            tc_fence_before();
            tile_sync(tile);  // every thread has read this buffer: the MMA of chunk c + 2 may overwrite it
            tc_fence_after();
            const bool ab_now = tflag[4] != 0;
            if (slot_i == 0 && !ab_now && c + 2 < NC)
                issue_chunk(tbase, bbase, mb, c + 2, buf);
            if (!act)
                continue;
            uint32_t mnew = 0;
            // every point of the chunk: past L the operator rows are zero, so the gradient and
            // the iterates are zero there and v = 0 gives xbar = 0 and no contribution
#pragma unroll
            for (int j = 0; j < kChunkPts; ++j) {
                const float gre = (j < 16) ? d0[2 * j] : d1[2 * (j - 16)];
                const float gim = (j < 16) ? d0[2 * j + 1] : d1[2 * (j - 16) + 1];
                // x^k_l and x^{k-1}_l from the packed values (addresses from the masks alone)
                const bool hx = (mx >> j) & 1u, hp = (mp >> j) & 1u;
                float2 xv = make_float2(0.f, 0.f), xpv = make_float2(0.f, 0.f);
                if (hx)
                    xv = vlx[ox];
                if (hp)
                    xpv = vlp[op];
                ox += hx;
                op += hp;
                // y = x + beta (x - x^{k-1}); v = y - 2 alpha grad; xbar = soft threshold of v at tau
                const float yx = fmaf(beta, xv.x - xpv.x, xv.x), yy = fmaf(beta, xv.y - xpv.y, xv.y);
                const float vre = fmaf(-a2, gre, yx), vim = fmaf(-a2, gim, yy);
                const float m2 = fmaf(vre, vre, vim * vim);
                const float rs = rsqrtf(m2);
                const float sc = fmaf(-tau, rs, 1.f);
                const bool nz = sc > 0.f;
                const float bre = nz ? vre * sc : 0.f, bim = nz ? vim * sc : 0.f;
                if (nz)
                    vlb[nb] = make_float2(bre, bim);
                nb += nz;
                mnew |= (uint32_t)nz << j;
                l1 += nz ? fmaf(m2, rs, -tau) : 0.f;
                const float ex = bre - yx, ey = bim - yy;
                dd = fmaf(ex, ex, fmaf(ey, ey, dd));
                const float fx = bre - xv.x, fy = bim - xv.y;
                dx = fmaf(fx, fx, fmaf(fy, fy, dx));
                xn = fmaf(bre, bre, fmaf(bim, bim, xn));
            }
            mkb[c] = mnew;
        }

        // ---- 3. A xbar over the nonzeros of xbar (ascending l, FP32 A in shared memory), then
        // ||A xbar - A y||^2 = ||(A xbar - g) - r|| ^2 and F's ||A xbar - g||^2 with r = A y - g
        const bool dead = aborted || (tflag[4] != 0);  // the gradient of this sweep is stale
        float my_lhs = 0.f, my_res = 0.f;
        float2 acc[32];
        if (act) {
#pragma unroll
            for (int n = 0; n < 32; ++n)
                acc[n] = make_float2(0.f, 0.f);
            int q = 0;
            for (int c = 0; c < NC; ++c) {
                uint32_t m = mkb[c];
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1u;
                    const float2 v = vlb[q++];
                    const float2 *Al = sA + (kChunkPts * c + j) * N;
#pragma unroll
                    for (int n = 0; n < 32; ++n) {
                        if (n < N) {
                            const float2 av = Al[n];
                            acc[n].x = fmaf(av.x, v.x, fmaf(-av.y, v.y, acc[n].x));
                            acc[n].y = fmaf(av.x, v.y, fmaf(av.y, v.x, acc[n].y));
                        }
                    }
                }
            }
            const float2 *gp = a.g + (size_t)pix * N;
#pragma unroll
            for (int n = 0; n < 32; ++n) {
                if (n < N) {
                    const float2 gv = gp[n], u = U[ub * N + n], up = U[upb * N + n];
                    const float rx = fmaf(beta, u.x - up.x, u.x), ry = fmaf(beta, u.y - up.y, u.y);
                    acc[n].x -= gv.x;  // A xbar - g
                    acc[n].y -= gv.y;
                    const float e0 = acc[n].x - rx, e1 = acc[n].y - ry;
                    my_lhs = fmaf(e0, e0, fmaf(e1, e1, my_lhs));
                    my_res = fmaf(acc[n].x, acc[n].x, fmaf(acc[n].y, acc[n].y, my_res));
                }
            }
        }

        // ---- 4. this thread's pixel: the same decision, the state update, output and refill
        if (act) {
            const bool bt_ok = dead || my_lhs <= dd / (2.f * alpha);
            if (!bt_ok && nbt_it < a.max_bt) {
                // Eq. 15 failed: the next sweep redoes the prox with the smaller step and the
                // same residual (the same rows give the same gradient)
                alpha *= a.c_alpha;
                ++nbt;
                ++nbt_it;
            } else {
                const float Fb = fmaf(lam, l1, my_res);
                const bool accepted = !dead && (Fb <= Fx);
                const bool conv = !dead && ((dx <= a.tol * a.tol * xn) || (dx == 0.f));
                const bool fin = dead || conv || (k >= a.max_iter);
                if (!bt_ok)
                    st |= BPDN_PX_BT_LIMIT;
                if (fin && !conv)
                    st |= BPDN_PX_NOT_CONVERGED;
                if (dead)
                    st |= BPDN_PX_DEVICE_TIMEOUT;
                if (accepted) {
                    Fx = Fb;
                    nnz = nb;
                }
                // x^{k-1} <- x^k; x^k <- xbar when accepted (buffers of the lists and of A x - g)
                if (accepted && !fin) {
                    const int nu = 1 - ub;
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        if (n < N)
                            U[nu * N + n] = acc[n];
                    upb = ub;
                    ub = nu;
                } else {
                    upb = ub;
                }
                bxp = bx;
                nxp = nx;
                if (accepted) {
                    bx = bb;
                    nx = nb;
                }
                if (fin) {
                    // write x^k into the output row
                    float2 *xq = a.x + (size_t)pix * L;
                    const uint32_t *mk = LM + bx * NC;
                    const float2 *vl = LV + bx * L;
                    int q = 0;
                    for (int c = 0; c < NC; ++c) {
                        const uint32_t m = (nx > 0) ? mk[c] : 0u;
                        for (int j = 0; j < kChunkPts; ++j) {
                            const int l = kChunkPts * c + j;
                            if (l >= L)
                                break;
                            float2 v = make_float2(0.f, 0.f);
                            if ((m >> j) & 1u)
                                v = vl[q++];
                            xq[l] = v;
                        }
                    }
                    a.status[pix] = (nnz == 0) ? (st | BPDN_PX_ZERO_SOLUTION) : st;
                    a.iters[pix] = k;
                    if (a.nbt)
                        a.nbt[pix] = nbt;
                    if (a.nsupp)
                        a.nsupp[pix] = nnz;
                    aborted = dead;
                    refill();
                } else {
                    beta = (float)(k - 1) / (float)(k + 2);
                    ++k;
                    nbt_it = 0;
                }
            }
        }
    }

    // every slot of this tile has drained.  After a wait that ran out, give the MMAs that
    // may still be in flight one more bounded wait before the tensor memory is released.
    if (slot_i == 0 && tflag[4]) {
        (void)mbar_wait(mbar0, ph0);
        (void)mbar_wait(mbar1, ph1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 2 * kTiles)
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(sbar + tid)) : "memory");
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

// CTAs of a launch: one per SM at most, no more than tiles of pixels
static int px_grid(int64_t P, int num_sms)
{
    const long long per = (long long)kTiles * kSlots;
    return (int)std::max(1LL, std::min((long long)num_sms, ((long long)P + per - 1) / per));
}

size_t rbpg_px_scratch_bytes(const OpHandle &op, int64_t P, int num_sms, int max_smem)
{
    if (2 * op.N > kK || op.L > 1024 || op.L < 1 || P <= 0)
        return 0;
    if (smem_layout(op.N, op.L).bytes > (size_t)max_smem)
        return 0;
    return (size_t)px_grid(P, num_sms) * kTiles * kSlots * slot_layout(op.N, op.L).bytes;
}

cudaError_t launch_rbpg_px(const OpHandle &op, const SolveLaunch &a, int num_sms, cudaStream_t s)
{
    if (a.P <= 0)
        return cudaSuccess;
    PxParams prm;
    prm.A_re = op.A_re;
    prm.A_im = op.A_im;
    prm.N = op.N;
    prm.L = op.L;
    prm.lda = op.lda;
    prm.slot_bytes = slot_layout(op.N, op.L).bytes;
    prm.a = a;
    const size_t smem = smem_layout(op.N, op.L).bytes;
    cudaError_t e = cudaFuncSetAttribute(k_rbpg_px, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // one CTA per SM (each allocates all 512 tensor-memory columns); no more CTAs than tiles of pixels
    const int grid = px_grid(a.P, num_sms);
    k_rbpg_px<<<grid, kTiles * kSlots, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace bpdn
