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
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the static area for the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
int scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rsi_cuda_fail(e, "rsi_propagate_stage_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return rsi_fail(RSI_E_UNSUPPORTED, "rsi_propagate_stage_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return rsi_cuda_fail(e, "rsi_propagate_stage_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RSI_OK;
}

}  // namespace

extern "C" int rsi_propagate_stage_noalloc(const rsi_stage* st, const void* src_points, int64_t n_src,
                                           const double* src_sigma, const void* tgt_points, int64_t n_tgt,
                                           double* tgt_field, void* stream) {
    if (!st) return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_noalloc: null stage");
    rsi_stage s = *st;
    size_t need = rsi_stage_workspace_bytes(&s, n_src, n_tgt);
    if (need == 0) return RSI_E_INVAL;  // the stage description was rejected; message already set
    if (need > RSI_NOALLOC_SCRATCH_BYTES && s.splits == 0) {
        // the automatic split count wants more room for partial sums than the
        // static area has: use fewer splits (the same sums, grouped differently)
        for (int sp = 64; sp >= 1; sp /= 2) {
            s.splits = sp;
            need = rsi_stage_workspace_bytes(&s, n_src, n_tgt);
            if (need != 0 && need <= RSI_NOALLOC_SCRATCH_BYTES) break;
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
