// stage_noalloc.cu -- rsi_propagate_stage_noalloc: the stage sum for callers
// that cannot hand the library any device memory of their own for scratch.
//
// rsi_propagate_stage needs a caller-provided workspace (staged source tiles
// and split partial sums).  Some callers cannot obtain one: a real-time
// acquisition or imaging loop whose latency budget rules out cudaMalloc (it
// can synchronise the device and its cost is unpredictable), a plug-in
// living inside a host application whose allocator owns all device memory
// and must not be bypassed, or a thin foreign-language host that only ever
// receives finished device pointers for its inputs and outputs.  For them
// this file keeps one fixed scratch area in device memory, declared at file
// scope, and passes it to the ordinary entry point.
//
// Costs and rules of the static area:
//   * its size is fixed (RSI_NOALLOC_SCRATCH_BYTES) and every GPU that loads
//     the library holds it until the process exits;
//   * all calls on a device share it, so calls whose work overlaps on the GPU
//     (different streams, or different host threads) race on it -- order
//     them on one stream;
//   * it keeps the previous call's bytes; nothing in it has to start at zero,
//     because every call writes each tile header, record and partial sum it
//     later reads.
#include <stdint.h>

#include <mutex>

#include "rsi_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[RSI_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
// per device: the area's device address and the context it was looked up in
void* g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the static area in the current device's context.  In
// host code the name g_noalloc_scratch is only a host-side stand-in, so the
// address is looked up with the device current.  The lookup is kept per
// device and redone whenever the device's context is not the one it was made
// in (after cudaDeviceReset the old address would be dangling).
int scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rsi_cuda_fail(e, "rsi_propagate_stage_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return rsi_fail(RSI_E_UNSUPPORTED, "rsi_propagate_stage_noalloc: device %d out of range", dev);
    const unsigned long long ctx = rsi_context_id();
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return rsi_cuda_fail(e, "rsi_propagate_stage_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = rsi_context_id();
    }
    *out = g_scratch_addr[dev];
    return RSI_OK;
}

}  // namespace

extern "C" int rsi_propagate_stage_noalloc(const rsi_stage* st, const void* src_points, int64_t n_src,
                                           const double* src_sigma, const void* tgt_points, int64_t n_tgt,
                                           double* tgt_field, void* stream) {
    if (!st) return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_noalloc: null stage");
    constexpr size_t kArea = RSI_NOALLOC_SCRATCH_BYTES;
    rsi_stage s = *st;
    size_t need = rsi_stage_workspace_bytes(&s, n_src, n_tgt);
    if (need == 0) return RSI_E_INVAL;  // the stage description was rejected; message already set
    if (need > kArea && s.splits == 0) {
        // The automatic split count wants more room for partial sums than the
        // static area has.  Each split holds n_tgt complex partial sums next to
        // the staged tiles (the split-free plan's workspace), so bound the
        // split count by what is left and let the planner choose below that
        // bound as it always does (fewest waves x tiles per CTA).  The sums are
        // the same, grouped differently.
        rsi_stage one = s;
        one.splits = 1;
        const size_t tiles = rsi_stage_workspace_bytes(&one, n_src, n_tgt);
        if (tiles != 0 && tiles <= kArea) {
            const size_t per_split = size_t(n_tgt) * 2 * sizeof(double);
            const size_t cap = (kArea - tiles) / per_split;
            int chosen = 1;
            if (cap >= 2) {
                need = rsi_stage_workspace_bytes_capped(&s, n_src, n_tgt, int(cap < 128 ? cap : 128), &chosen);
            } else {
                need = tiles;
            }
            s.splits = chosen;
        }
    }
    if (need == 0 || need > RSI_NOALLOC_SCRATCH_BYTES)
        return rsi_fail(RSI_E_NOMEM,
                        "rsi_propagate_stage_noalloc: %lld sources x %lld targets need %zu bytes of scratch, "
                        "more than the %zu-byte static area; use rsi_propagate_stage with a workspace",
                        (long long)n_src, (long long)n_tgt, need, (size_t)RSI_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != RSI_OK) return rc;
    return rsi_propagate_stage(&s, src_points, n_src, src_sigma, tgt_points, n_tgt, tgt_field, scratch,
                               RSI_NOALLOC_SCRATCH_BYTES, stream);
}
