// Pre-classification of pixels before the L1 solve: the hybrid strategy the paper
// recommends (Sec. I: a fast linear estimator for the pixels that need no
// super-resolution, L1 only for the others; Sec. V: a further speed-up of about 50
// expected from it).  The paper does not define the classifier; the library's reading:
//
//   u = A^H g (beamforming, the classic linear estimator, on the grid)
//   class 0  2 max_l |u_l| <= lambda: x* = 0 exactly (0 satisfies Eq. 6's optimality
//            conditions), so the pixel holds no scatterer: K = 0
//   else     the single-scatterer linear estimate: l^ = argmax |u_l| (first on ties),
//            s^ = the elevation in [s_{l^-1}, s_{l^+1}] where |a(s)^H g| peaks,
//            gamma^ = a(s^)^H g / N, r = g - gamma^ a(s^)
//   class 1  2 max_l |a_l^H r| <= lambda (the residual would itself be screened out):
//            K = 1 with (s^, gamma^)
//   class 2  everything else, left to the L1 solve (bpdn_solve with the refit, then
//            bpdn_select): these pixels' indices and measurements are compacted.
//
// One warp per pixel.  The beam sums run in FP32 from the operator's FP32 tables (in
// shared memory when they fit); grid points within 1e-4 of a decision boundary are
// recomputed in FP64, so every class decision is the FP64 one.  The peak search is a
// safeguarded Newton iteration on d|F|^2/ds = 0, F(s) = sum_n g_n exp(j 2 pi xi_n s),
// in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bpdn_internal.h"

namespace bpdn {

namespace {

constexpr int kWarps = 8;  // pixels in flight per block

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t classify_smem(int N, int L, bool sa)
{
    return (sa ? a16(sizeof(float2) * (size_t)N * L) : 0) + a16(sizeof(double) * (size_t)N) +
           (size_t)kWarps * a16((size_t)N * (2 * sizeof(double2) + sizeof(float2)));
}

struct PreLaunch {
    int64_t P;
    const float2 *g;
    const float *lam;
    int lam_pp;
    int kmax;
    int32_t *cls;     // [P]
    int32_t *khat;    // [P]
    double *s_hat;    // [P][kmax]
    double2 *gamma;   // [P][kmax]
    int64_t *idx;     // [P]: pixels of class 2, in the order they were found
    unsigned long long *count;
    float2 *g_c;      // [P][N] or NULL: their measurements, in the same order
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// max over the warp of (value, index): the larger value, the lower index on ties
__device__ __forceinline__ void warp_argmax(float &v, int &i)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        if (ov > v || (ov == v && oi >= 0 && (i < 0 || oi < i))) {
            v = ov;
            i = oi;
        }
    }
}

// 2 |a_l^H r| in FP64 for one grid point (r in shared memory, FP64)
__device__ __forceinline__ double beam64(const double2 *__restrict__ A64, int N, int L, int l, const double2 *r)
{
    double vx = 0.0, vy = 0.0;
    for (int n = 0; n < N; ++n) {
        const double2 a = A64[(size_t)n * L + l], v = r[n];
        vx += a.x * v.x + a.y * v.y;
        vy += a.x * v.y - a.y * v.x;
    }
    return 2.0 * sqrt(vx * vx + vy * vy);
}

// The beam over the grid for the vector in rf (FP32) / rd (FP64): returns the largest
// 2 |a_l^H r| as the FP64 value where it matters (exact when it lies within 1e-4 of lam)
// and its grid index (first on ties of the FP32 values).  Lanes over l.
template <bool SA>
__device__ double beam_max(const float2 *sA, const float *__restrict__ A_re, const float *__restrict__ A_im,
                           const double2 *__restrict__ A64, int N, int L, int lda, const float2 *rf,
                           const double2 *rd, double lam, int lane, int &l_best)
{
    float best = -1.f;
    int bl = -1;
    double near_max = 0.0;  // the FP64 value of grid points in the band around lam
    const float lo = (float)(lam * (1.0 - 1e-4)), hi = (float)(lam * (1.0 + 1e-4));
    for (int l = lane; l < L; l += 32) {
        float ux = 0.f, uy = 0.f;
        for (int n = 0; n < N; ++n) {
            float ar, ai;
            if constexpr (SA) {
                const float2 a = sA[n * L + l];
                ar = a.x;
                ai = a.y;
            } else {
                ar = __ldg(A_re + n * lda + l);
                ai = __ldg(A_im + n * lda + l);
            }
            const float2 v = rf[n];
            ux = fmaf(ar, v.x, fmaf(ai, v.y, ux));
            uy = fmaf(ar, v.y, fmaf(-ai, v.x, uy));
        }
        const float b = 2.f * sqrtf(ux * ux + uy * uy);
        if (b > best) {
            best = b;
            bl = l;
        }
        if (b >= lo && b <= hi)
            near_max = fmax(near_max, beam64(A64, N, L, l, rd));
    }
    float bv = best;
    warp_argmax(bv, bl);
    l_best = bl;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        near_max = fmax(near_max, __shfl_xor_sync(0xffffffffu, near_max, off));
    // a beam value clear of the band decides in FP32; inside it the FP64 values decide
    if (bv > hi)
        return (double)bv;
    return near_max > 0.0 ? near_max : (double)bv;
}

// F(s) = sum_n g_n exp(j w_n s), w_n = 2 pi xi_n, and its first two derivatives
// (lanes over n, two rows each; every lane gets the sums)
struct Beam {
    double fr, fi, dr, di, er, ei;  // F, F', F''
};

__device__ __forceinline__ Beam beam_at(const double *xi, const double2 *g, int N, double s, int lane)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int n = lane; n < N; n += 32) {
        const double w = 2.0 * M_PI * xi[n];
        double sn, cs;
        sincospi(2.0 * xi[n] * s, &sn, &cs);
        const double2 gg = g[n];
        const double tr = gg.x * cs - gg.y * sn, ti = gg.x * sn + gg.y * cs;  // g_n e^{j w s}
        v[0] += tr;
        v[1] += ti;
        v[2] += -w * ti;  // j w (tr + j ti)
        v[3] += w * tr;
        v[4] += -w * w * tr;
        v[5] += -w * w * ti;
    }
    Beam b;
    b.fr = warp_sum(v[0]);
    b.fi = warp_sum(v[1]);
    b.dr = warp_sum(v[2]);
    b.di = warp_sum(v[3]);
    b.er = warp_sum(v[4]);
    b.ei = warp_sum(v[5]);
    return b;
}

// the elevation in [lo, hi] where |F|^2 peaks, from s0: Newton steps on the derivative of
// |F|^2 kept inside a bracket that the derivative's sign shrinks (bisection when a step
// leaves it or the curvature is not negative); the end points win if |F| is larger there
__device__ double peak_search(const double *xi, const double2 *g, int N, double lo, double hi, double s0, int lane)
{
    double a = lo, b = hi, s = s0;
    for (int it = 0; it < 60 && b - a > 1e-13 * fmax(1.0, fabs(a) + fabs(b)); ++it) {
        const Beam f = beam_at(xi, g, N, s, lane);
        const double d1 = f.fr * f.dr + f.fi * f.di;                             // (|F|^2)' / 2
        const double d2 = f.dr * f.dr + f.di * f.di + f.fr * f.er + f.fi * f.ei;  // (|F|^2)'' / 2
        if (d1 > 0.0)
            a = s;
        else if (d1 < 0.0)
            b = s;
        else
            break;
        double sn = (d2 < 0.0) ? s - d1 / d2 : 0.5 * (a + b);
        if (!(sn > a && sn < b))
            sn = 0.5 * (a + b);
        if (fabs(sn - s) <= 1e-13 * fmax(1.0, fabs(s))) {
            s = sn;
            break;
        }
        s = sn;
    }
    const Beam fs = beam_at(xi, g, N, s, lane), fl = beam_at(xi, g, N, lo, lane), fh = beam_at(xi, g, N, hi, lane);
    const double ps = fs.fr * fs.fr + fs.fi * fs.fi, pl = fl.fr * fl.fr + fl.fi * fl.fi,
                 ph = fh.fr * fh.fr + fh.fi * fh.fi;
    if (pl > ps && pl >= ph)
        return lo;
    if (ph > ps && ph > pl)
        return hi;
    return s;
}

template <bool SA>
__global__ void __launch_bounds__(kWarps * 32) k_classify(PreLaunch a, const float *__restrict__ A_re,
                                                         const float *__restrict__ A_im,
                                                         const double2 *__restrict__ A64,
                                                         const double *__restrict__ xi_g, int N, int L, int lda,
                                                         double s_min, double ds)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [A as float2 N x L when SA] [xi N] then per warp: g (FP64), r (FP64), rf (FP32);
    // every section starts on a 16-byte boundary
    float2 *sA = (float2 *)smem_raw;
    double *sxi = (double *)(smem_raw + (SA ? a16(sizeof(float2) * (size_t)N * L) : 0));
    unsigned char *wbase = (unsigned char *)sxi + a16(sizeof(double) * (size_t)N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2 *sg = (double2 *)(wbase + (size_t)warp * a16((size_t)N * (2 * sizeof(double2) + sizeof(float2))));
    double2 *sr = sg + N;
    float2 *srf = (float2 *)(sr + N);
    if constexpr (SA)
        for (int i = threadIdx.x; i < N * L; i += blockDim.x)
            sA[i] = make_float2(A_re[(i / L) * lda + i % L], A_im[(i / L) * lda + i % L]);
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        sxi[i] = xi_g[i];
    __syncthreads();
    const int kmax = a.kmax;
    for (int64_t p = (int64_t)blockIdx.x * kWarps + warp; p < a.P; p += (int64_t)gridDim.x * kWarps) {
        const double lam = (double)(a.lam_pp ? a.lam[p] : a.lam[0]);
        const float2 *gp = a.g + (size_t)p * N;
        bool fin = true;
        for (int n = lane; n < N; n += 32) {
            const float2 v = gp[n];
            fin = fin && isfinite(v.x) && isfinite(v.y);
            sg[n] = make_double2((double)v.x, (double)v.y);
            srf[n] = v;
        }
        fin = __all_sync(0xffffffffu, fin);
        __syncwarp();
        double *sh = a.s_hat + (size_t)p * kmax;
        double2 *gh = a.gamma + (size_t)p * kmax;
        if (lane < kmax) {
            sh[lane] = __longlong_as_double(0x7ff8000000000000LL);  // NaN: no estimate
            gh[lane] = make_double2(0.0, 0.0);
        }
        int cls = 2;
        double s_est = 0.0;
        double2 gam = make_double2(0.0, 0.0);
        if (fin) {
            int lhat;
            const double umax = beam_max<SA>(sA, A_re, A_im, A64, N, L, lda, srf, sg, lam, lane, lhat);
            if (umax <= lam) {
                cls = 0;
            } else {
                const double lo = s_min + ds * (double)max(lhat - 1, 0);
                const double hi = s_min + ds * (double)min(lhat + 1, L - 1);
                const double s0 = s_min + ds * (double)lhat;
                s_est = (hi > lo) ? peak_search(sxi, sg, N, lo, hi, s0, lane) : s0;
                const Beam f = beam_at(sxi, sg, N, s_est, lane);
                gam = make_double2(f.fr / N, f.fi / N);
                // r = g - gamma^ a(s^), a(s)_n = exp(-j 2 pi xi_n s)
                for (int n = lane; n < N; n += 32) {
                    double sn, cs;
                    sincospi(2.0 * sxi[n] * s_est, &sn, &cs);
                    const double ar = cs, ai = -sn;
                    const double2 v = make_double2(sg[n].x - (gam.x * ar - gam.y * ai),
                                                   sg[n].y - (gam.x * ai + gam.y * ar));
                    sr[n] = v;
                    srf[n] = make_float2((float)v.x, (float)v.y);
                }
                __syncwarp();
                int dummy;
                const double rmax = beam_max<SA>(sA, A_re, A_im, A64, N, L, lda, srf, sr, lam, lane, dummy);
                if (rmax <= lam)
                    cls = 1;
            }
        }
        if (lane == 0) {
            a.cls[p] = cls;
            a.khat[p] = (cls == 2) ? -1 : cls;
            if (cls == 1) {
                sh[0] = s_est;
                gh[0] = gam;
            }
        }
        if (cls == 2) {
            unsigned long long slot = 0;
            if (lane == 0) {
                slot = atomicAdd(a.count, 1ULL);
                a.idx[slot] = p;
            }
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (a.g_c)
                for (int n = lane; n < N; n += 32)
                    a.g_c[(size_t)slot * N + n] = gp[n];
        }
        __syncwarp();
    }
}

// rows of the L1 pixels' selection (compact, in idx order) into the full outputs
__global__ void k_merge(int64_t Pc, const int64_t *__restrict__ idx, int kmax, const int32_t *__restrict__ khat_c,
                        const double *__restrict__ s_c, const double2 *__restrict__ g_c, int32_t *khat, double *s_hat,
                        double2 *gamma)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Pc)
        return;
    const int64_t p = idx[i];
    khat[p] = khat_c[i];
    for (int k = 0; k < kmax; ++k) {
        s_hat[(size_t)p * kmax + k] = s_c[(size_t)i * kmax + k];
        gamma[(size_t)p * kmax + k] = g_c[(size_t)i * kmax + k];
    }
}

}  // namespace
}  // namespace bpdn

using namespace bpdn;

extern "C" int bpdn_classify(bpdn_op_t h, const void *d_g, int64_t P, const float *d_lambda, int32_t lambda_per_pixel,
                             int32_t kmax, int32_t *d_class, int32_t *d_khat, double *d_s_hat, void *d_gamma_hat,
                             int64_t *d_idx, uint64_t *d_count, void *d_g_compact, void *cuda_stream)
{
    OpHandle *op = reinterpret_cast<OpHandle *>(h);
    if (!op || op->magic != kOpMagic)
        return set_error(BPDN_EINVAL, "invalid operator handle");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != op->device)
        return set_error(BPDN_ESTATE, "the operator's device is not current");
    if (op->md)
        return set_error(BPDN_EINVAL, "pre-classification reads an elevation-only grid; this operator has motion dimensions");
    if (P < 0)
        return set_error(BPDN_EINVAL, "P must be >= 0");
    if (kmax < 1 || kmax > BPDN_MAX_KSEL)
        return set_error(BPDN_EINVAL, "kmax must lie in 1..%d", BPDN_MAX_KSEL);
    if (!d_count)
        return set_error(BPDN_EINVAL, "count pointer must be non-NULL");
    if (((uintptr_t)d_count % 8) != 0)
        return set_error(BPDN_EALIGN, "count must be 8-byte aligned");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int rc = check_cuda(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s), "clear the count");
    if (rc || P == 0)
        return rc;
    if (!d_g || !d_lambda || !d_class || !d_khat || !d_s_hat || !d_gamma_hat || !d_idx)
        return set_error(BPDN_EINVAL, "g, lambda, class, khat, s_hat, gamma_hat and idx must be non-NULL");
    if (((uintptr_t)d_g % 8) || ((uintptr_t)d_s_hat % 8) || ((uintptr_t)d_gamma_hat % 16) || ((uintptr_t)d_idx % 8) ||
        (d_g_compact && ((uintptr_t)d_g_compact % 8)) || ((uintptr_t)d_class % 4) || ((uintptr_t)d_khat % 4) ||
        ((uintptr_t)d_lambda % 4))
        return set_error(BPDN_EALIGN, "g, g_compact, s_hat, idx 8-byte, gamma_hat 16-byte, the int32/float arrays 4-byte aligned");
    PreLaunch a;
    a.P = P;
    a.g = (const float2 *)d_g;
    a.lam = d_lambda;
    a.lam_pp = lambda_per_pixel ? 1 : 0;
    a.kmax = kmax;
    a.cls = d_class;
    a.khat = d_khat;
    a.s_hat = d_s_hat;
    a.gamma = (double2 *)d_gamma_hat;
    a.idx = d_idx;
    a.count = (unsigned long long *)d_count;
    a.g_c = (float2 *)d_g_compact;
    int max_smem = 0, sms = 1;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool sa = classify_smem(op->N, op->L, true) <= (size_t)max_smem;
    const size_t smem = classify_smem(op->N, op->L, sa);
    cudaError_t e;
    int per_sm = 1;
    if (sa) {
        e = cudaFuncSetAttribute(k_classify<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_classify<true>, kWarps * 32, smem);
    } else {
        e = cudaFuncSetAttribute(k_classify<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_classify<false>, kWarps * 32, smem);
    }
    if (e != cudaSuccess)
        return check_cuda(e, "classify launch set-up");
    long long blocks = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    const long long need = (P + kWarps - 1) / kWarps;
    if (blocks > need)
        blocks = need;
    if (sa)
        k_classify<true><<<(unsigned)blocks, kWarps * 32, smem, s>>>(a, op->A_re, op->A_im, op->A64, op->xi, op->N,
                                                                      op->L, op->lda, op->s_min, op->ds);
    else
        k_classify<false><<<(unsigned)blocks, kWarps * 32, smem, s>>>(a, op->A_re, op->A_im, op->A64, op->xi, op->N,
                                                                       op->L, op->lda, op->s_min, op->ds);
    return check_cuda(cudaGetLastError(), "classify kernel");
}

extern "C" int bpdn_classify_merge(int64_t P_c, const int64_t *d_idx, int32_t kmax, const int32_t *d_khat_c,
                                   const double *d_s_hat_c, const void *d_gamma_hat_c, int32_t *d_khat,
                                   double *d_s_hat, void *d_gamma_hat, void *cuda_stream)
{
    if (P_c < 0)
        return set_error(BPDN_EINVAL, "P_c must be >= 0");
    if (kmax < 1 || kmax > BPDN_MAX_KSEL)
        return set_error(BPDN_EINVAL, "kmax must lie in 1..%d", BPDN_MAX_KSEL);
    if (P_c == 0)
        return BPDN_OK;
    if (!d_idx || !d_khat_c || !d_s_hat_c || !d_gamma_hat_c || !d_khat || !d_s_hat || !d_gamma_hat)
        return set_error(BPDN_EINVAL, "every array must be non-NULL");
    if (((uintptr_t)d_gamma_hat_c % 16) || ((uintptr_t)d_gamma_hat % 16) || ((uintptr_t)d_s_hat_c % 8) ||
        ((uintptr_t)d_s_hat % 8) || ((uintptr_t)d_idx % 8))
        return set_error(BPDN_EALIGN, "gamma_hat arrays 16-byte, s_hat and idx 8-byte aligned");
    const int threads = 256;
    const long long blocks = (P_c + threads - 1) / threads;
    k_merge<<<(unsigned)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(
        P_c, d_idx, kmax, d_khat_c, d_s_hat_c, (const double2 *)d_gamma_hat_c, d_khat, d_s_hat, (double2 *)d_gamma_hat);
    return check_cuda(cudaGetLastError(), "merge kernel");
}
