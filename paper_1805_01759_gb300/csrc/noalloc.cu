// bpdn_solve_noalloc: bpdn_solve for callers that cannot allocate device memory.
//
// Some programs that embed this library are not allowed to call cudaMalloc: a
// SAR processor that reserves the whole GPU memory for its own pool at start-up
// and hands modules only its own buffers, or a real-time chain that must not risk
// an allocation failing in the middle of a run.  They can still pass the inputs
// and outputs they already own, but not a workspace.  For them the iteration
// kernel's scratch (its 64-bit work counter) lives in the fixed-size device array
// below instead of in a caller-provided workspace.
//
// Facts a caller needs:
//   * the array occupies kNoAllocScratchBytes of device memory on every GPU that
//     loads the library, until the process exits;
//   * its device address is looked up once per device (cudaGetSymbolAddress) by
//     the first call made with that device current -- make that first call before
//     any stream capture.  The address is kept for the life of the process: after a
//     cudaDeviceReset of that device it would be stale, so a process that resets a
//     device must not call bpdn_solve_noalloc on it again;
//   * every call shares the array, and each call clears the counter it needs on
//     its own stream before the launch: calls whose work overlaps on the GPU (two
//     streams, or two host threads) race on the counter and must be serialised by
//     the caller;
//   * nothing here calls cudaMalloc, cudaFree or any allocating library routine.
#include <cuda_runtime.h>
#include <mutex>

#include "bpdn_internal.h"

namespace bpdn {
namespace {

constexpr size_t kNoAllocScratchBytes = 256;  // holds the work counter of one launch
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (resolved once).
int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(BPDN_ESTATE, "device %d outside the %d devices the static scratch supports",
                         dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return check_cuda(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BPDN_OK;
}

}  // namespace
}  // namespace bpdn

using namespace bpdn;

extern "C" int bpdn_solve_noalloc(bpdn_op_t op, const void *d_g, int64_t P, const float *d_lambda,
                                  int32_t lambda_per_pixel, const bpdn_options *opt, void *d_x,
                                  int32_t *d_support, int32_t *d_nsupp, int32_t *d_status,
                                  int32_t *d_iters, int32_t *d_nbt, void *cuda_stream)
{
    (void)P;
    const size_t need = solve_min_workspace_bytes(opt);
    if (need > kNoAllocScratchBytes)
        return set_error(BPDN_ESIZE,
                         "this solve needs %zu bytes of scratch; the static scratch holds %zu",
                         need, kNoAllocScratchBytes);
    int dev = -1;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc)
        return rc;
    void *scratch = nullptr;
    rc = scratch_address(dev, &scratch);
    if (rc)
        return rc;
    return bpdn_solve(op, d_g, P, d_lambda, lambda_per_pixel, opt, d_x, d_support, d_nsupp, d_status,
                      d_iters, d_nbt, scratch, kNoAllocScratchBytes, cuda_stream);
}
