// bpdn_solve_ragged: many stacks with their own operators in one call.
//
// Each stack is an independent bpdn_solve.  The call checks every stack, then runs
// Algorithm 1 for all of them in one persistent launch of the iteration kernel per
// kernel variant present (BF16 or FP32; A in shared or in global memory; at most 64
// stacks each): every CTA walks the stacks, smallest first, and works on each one
// while it has pixels left.  Stacks that bpdn_solve would give the split-grid kernel
// (grids of more than 512 points in FP32 with the library's tile, more than 1024 in any
// case) run it in their own launches, with their scratch in the call's workspace.  The
// refits follow, one launch per stack, spread over a small pool of library-owned streams
// that fork from and join back into the caller's stream through events, so the call can
// be captured into one CUDA graph.  A stack may carry its own tile_pixels (pixels in
// flight per SM) and kernel option, as the autotuner of the Python binding picks them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "bpdn_internal.h"

namespace bpdn {
namespace {

constexpr int kWorkers = 4;
constexpr int kMaxDevices = 64;
constexpr size_t kStackScratch = 256;

struct Pool {
    bool ready = false;
    cudaStream_t stream[kWorkers];
    cudaEvent_t fork;
    cudaEvent_t join[kWorkers];
};

std::mutex g_mu;
Pool g_pool[kMaxDevices];

int pool_for(int dev, Pool **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(BPDN_ESTATE, "device %d outside the %d devices the stream pool supports", dev, kMaxDevices);
    Pool &p = g_pool[dev];
    if (!p.ready) {
        int rc = check_cuda(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming), "create fork event");
        for (int i = 0; i < kWorkers && !rc; ++i) {
            rc = check_cuda(cudaStreamCreateWithFlags(&p.stream[i], cudaStreamNonBlocking), "create worker stream");
            if (!rc)
                rc = check_cuda(cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming), "create join event");
        }
        if (rc)
            return rc;
        p.ready = true;
    }
    *out = &p;
    return BPDN_OK;
}

// the split-grid kernel's scratch of a stack (0 when the stack runs in the batch launch)
size_t stack_split_bytes(const bpdn_stack &st, const bpdn_options &o)
{
    const OpHandle *op = reinterpret_cast<const OpHandle *>(st.op);
    if (!op || op->magic != kOpMagic || st.P <= 0 || !solve_uses_split(op, &o))
        return 0;
    return (rbpg_split_scratch_bytes(*op, o.precision, st.P, device_sms(op->device)) + 255) / 256 * 256;
}

// each stack's options: the call's, with the stack's tile_pixels and kernel when it names them
std::vector<bpdn_options> stack_options(const bpdn_stack *stacks, int n, const bpdn_options &opt)
{
    std::vector<bpdn_options> sopt(n, opt);
    for (int i = 0; i < n; ++i) {
        if (stacks[i].tile_pixels)
            sopt[i].tile_pixels = stacks[i].tile_pixels;
        if (stacks[i].kernel)
            sopt[i].kernel = stacks[i].kernel;
    }
    return sopt;
}

double stack_cost(const bpdn_stack &st)
{
    int32_t N = 0, L = 0;
    double ds = 0.0, lip = 0.0;
    if (bpdn_op_info(st.op, &N, &L, &ds, &lip) != BPDN_OK)
        return 0.0;
    return (double)st.P * (double)N * (double)L;
}

}  // namespace
}  // namespace bpdn

using namespace bpdn;

extern "C" {

size_t bpdn_solve_ragged_workspace_bytes_for(const bpdn_stack *stacks, int32_t n_stacks, const bpdn_options *opt)
{
    if (n_stacks <= 0)
        return 0;
    if (!stacks)
        return 0;
    // per-stack headers, then the split-grid kernel's scratch of the stacks that run it, then
    // the refits' scratch
    size_t b = kStackScratch * (size_t)n_stacks;
    if (opt) {
        const std::vector<bpdn_options> sopt = stack_options(stacks, n_stacks, *opt);
        for (int i = 0; i < n_stacks; ++i)
            b += stack_split_bytes(stacks[i], sopt[i]);
    }
    if (opt && opt->refit)
        for (int i = 0; i < n_stacks; ++i)
            b += refit_scratch_bytes(stacks[i].P);
    return b;
}

size_t bpdn_solve_ragged_workspace_bytes(int32_t n_stacks)
{
    return n_stacks > 0 ? kStackScratch * (size_t)n_stacks : 0;
}

int bpdn_solve_ragged(const bpdn_stack *stacks, int32_t n_stacks, const bpdn_options *opt,
                      void *d_workspace, size_t workspace_bytes, void *cuda_stream)
{
    if (n_stacks < 0)
        return set_error(BPDN_EINVAL, "n_stacks must be >= 0");
    if (n_stacks == 0)
        return BPDN_OK;
    if (!stacks)
        return set_error(BPDN_EINVAL, "stacks must be non-NULL");
    if (!d_workspace || workspace_bytes < bpdn_solve_ragged_workspace_bytes(n_stacks))
        return set_error(BPDN_ESIZE, "ragged workspace too small (%zu bytes for %d stacks)",
                         bpdn_solve_ragged_workspace_bytes(n_stacks), n_stacks);
    if (((uintptr_t)d_workspace % 256) != 0)
        return set_error(BPDN_EALIGN, "ragged workspace must be 256-byte aligned");
    int dev = -1;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc)
        return rc;
    if (!opt)
        return set_error(BPDN_EINVAL, "options pointer is NULL");
    if (opt->blocks >= 2)
        return set_error(BPDN_EINVAL, "randomized blocks (blocks >= 2) are not available in bpdn_solve_ragged");
    const std::vector<bpdn_options> sopt = stack_options(stacks, n_stacks, *opt);
    // the split-grid kernel's scratch follows the headers, in stack order
    std::vector<unsigned char *> split_at(n_stacks, nullptr);
    size_t off = kStackScratch * (size_t)n_stacks;
    for (int i = 0; i < n_stacks; ++i) {
        const size_t sb = stack_split_bytes(stacks[i], sopt[i]);
        if (sb == 0)
            continue;
        if (workspace_bytes < off + sb)
            return set_error(BPDN_ESIZE, "stack %d runs the split-grid kernel: the workspace must hold its scratch "
                                         "(bpdn_solve_ragged_workspace_bytes_for gives the size)", i);
        split_at[i] = (unsigned char *)d_workspace + off;
        off += sb;
    }
    // every stack is checked before anything is launched
    std::vector<SolvePlan> plans(n_stacks);
    for (int i = 0; i < n_stacks; ++i) {
        const bpdn_stack &st = stacks[i];
        unsigned char *ws = (unsigned char *)d_workspace + kStackScratch * (size_t)i;
        rc = solve_plan(st.op, st.d_g, st.P, st.d_lambda, st.lambda_per_pixel, &sopt[i], st.d_x, st.d_support,
                        st.d_nsupp, st.d_status, st.d_iters, st.d_nbt, ws, kStackScratch, &plans[i], split_at[i]);
        if (rc) {
            char msg[512];
            snprintf(msg, sizeof(msg), "%s", bpdn_last_error());
            return set_error(rc, "stack %d: %s", i, msg);
        }
    }
    // with room for it, each stack's refit runs in three launches: its scratch follows the
    // split-grid region, in stack order
    if (opt->refit && workspace_bytes >= bpdn_solve_ragged_workspace_bytes_for(stacks, n_stacks, opt)) {
        unsigned char *b = (unsigned char *)d_workspace + off;
        for (int i = 0; i < n_stacks; ++i) {
            if (plans[i].refit)
                plans[i].r.split = b;
            b += refit_scratch_bytes(stacks[i].P);
        }
    }
    std::vector<const OpHandle *> ops;
    std::vector<SolveLaunch> as;
    std::vector<int> refit_order, split_order;
    for (int i = 0; i < n_stacks; ++i) {
        if (plans[i].a.P == 0)
            continue;
        if (plans[i].a.split_scratch) {
            split_order.push_back(i);
        } else {
            ops.push_back(plans[i].op);
            as.push_back(plans[i].a);
        }
        if (plans[i].refit)
            refit_order.push_back(i);
    }
    cudaStream_t origin = (cudaStream_t)cuda_stream;
    // every stack's work counter and error word in one clear
    rc = check_cuda(cudaMemsetAsync(d_workspace, 0, kStackScratch * (size_t)n_stacks, origin), "clear work counters");
    if (rc)
        return rc;
    if (!as.empty())
        rc = check_cuda(launch_rbpg_batch(ops.data(), as.data(), (int)as.size(), device_sms(dev), origin),
                        "iteration kernel");
    if (rc || (refit_order.empty() && split_order.empty()))
        return rc;
    std::stable_sort(refit_order.begin(), refit_order.end(),
                     [&](int x, int y) { return stack_cost(stacks[x]) > stack_cost(stacks[y]); });
    std::lock_guard<std::mutex> lk(g_mu);
    Pool *pool = nullptr;
    rc = pool_for(dev, &pool);
    if (rc)
        return rc;
    const int want = (int)std::max(refit_order.size(), split_order.size());
    const int used = want < kWorkers ? want : kWorkers;
    rc = check_cuda(cudaEventRecord(pool->fork, origin), "record fork event");
    for (int k = 0; k < used && !rc; ++k)
        rc = check_cuda(cudaStreamWaitEvent(pool->stream[k], pool->fork, 0), "fork worker stream");
    // the split-grid stacks, each in its own launch on a worker stream (after the batch
    // launch); a stack's refit follows on the same stream
    std::vector<int> worker(n_stacks, -1);
    for (size_t j = 0; j < split_order.size() && !rc; ++j) {
        const int i = split_order[j];
        worker[i] = (int)(j % used);
        rc = check_cuda(launch_rbpg_split(*plans[i].op, plans[i].a, device_sms(dev), pool->stream[worker[i]]),
                        "iteration kernel (split grid)");
    }
    // the refits, largest stacks first, on the worker streams
    int next = 0;
    for (size_t j = 0; j < refit_order.size() && !rc; ++j) {
        const int i = refit_order[j];
        const int k = worker[i] >= 0 ? worker[i] : (next++ % used);
        rc = check_cuda(launch_refit(*plans[i].op, plans[i].r, pool->stream[k]), "refit kernel");
    }
    // join every forked stream back into the caller's stream, also after an error
    for (int k = 0; k < used; ++k) {
        const int r1 = check_cuda(cudaEventRecord(pool->join[k], pool->stream[k]), "record join event");
        const int r2 = r1 ? r1 : check_cuda(cudaStreamWaitEvent(origin, pool->join[k], 0), "join worker stream");
        if (!rc)
            rc = r2;
    }
    return rc;
}

}  // extern "C"
