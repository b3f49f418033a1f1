// rsi_internal.cuh -- shared internals of the sm_103a RSI library: error
// reporting, point-set views, double-float arithmetic, and the mbarrier /
// bulk-copy (TMA) primitives with bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rsi.h"

#define RSI_ABI_VERSION 1

// ---------------------------------------------------------------------------
// host-side error reporting (thread-local message, see rsi_last_error)
// ---------------------------------------------------------------------------
int rsi_fail(int code, const char* fmt, ...);
int rsi_cuda_fail(cudaError_t e, const char* what);
#define RSI_CUDA_TRY(call, what)                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return rsi_cuda_fail(e_, what); \
    } while (0)
void rsi_note_launch();
#define RSI_CHECK_LAUNCH(what)                            \
    do {                                                  \
        cudaError_t e_ = cudaGetLastError();              \
        if (e_ != cudaSuccess) return rsi_cuda_fail(e_, what); \
        rsi_note_launch();                                \
    } while (0)

// device status word of the current device (device pointer); nullptr + error
// message on failure
int* rsi_status_ptr();

// Identity of the calling thread's current CUDA context (cuCtxGetId); 0 when
// no context is current yet or the driver does not offer the query.  State
// that belongs to a context -- kernel attributes, device addresses of module
// variables -- is cached under this id, so that a context that is torn down
// and created again (cudaDeviceReset, another primary context) is set up
// afresh instead of reusing stale attributes or addresses.
unsigned long long rsi_context_id();

// One-time set-up per context: needed() is true until done() has been called
// with the same context current.  Several devices used in turn simply repeat
// the (cheap) set-up.
struct RsiCtxOnce {
    unsigned long long ctx = 0;
    bool needed() const {
        const unsigned long long id = rsi_context_id();
        return id == 0 || id != __atomic_load_n(&ctx, __ATOMIC_ACQUIRE);
    }
    void done() { __atomic_store_n(&ctx, rsi_context_id(), __ATOMIC_RELEASE); }
};

// Workspace of rsi_propagate_stage with the automatic split count (st->splits
// == 0) limited to max_splits >= 1, chosen as rsi_propagate_stage chooses it
// below that limit; the split count of that plan goes to *splits.  0 on
// invalid input.
size_t rsi_stage_workspace_bytes_capped(const rsi_stage* st, int64_t n_src, int64_t n_tgt, int max_splits,
                                        int* splits);

// status codes written by kernels
#define RSI_DEV_TIMEOUT 1
#define RSI_DEV_NONFINITE 2

// ---------------------------------------------------------------------------
// point-set views
// ---------------------------------------------------------------------------
struct PointsView {
    uint32_t *idx, *su, *sv;
    double *x, *y, *z, *nx, *ny, *nz, *w;
    float *xh, *xl, *yh, *yl, *zh, *zl;
};

size_t rsi_field_bytes_(int32_t field, int64_t n);
PointsView rsi_points_view(void* base, int64_t n);

// ---------------------------------------------------------------------------
// double-float (pairs of FP32) arithmetic: error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based TwoProduct
// (Ogita, Rump & Oishi 2005).  The _rn intrinsics keep the compiler from
// contracting or reassociating these sequences.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (ah + al) - (bh + bl) as a normalised double-float (h, l)
__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    two_sum(s, e, h, l);
}
// sum of two non-negative double-floats
__device__ __forceinline__ void df_add_pos(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, h, l);
}
// (h + l)^2 as a double-float
__device__ __forceinline__ void df_sqr(float h, float l, float& ph, float& pl) {
    two_prod(h, h, ph, pl);
    pl = __fmaf_rn(__fmul_rn(2.0f, h), l, pl);
}

// ---------------------------------------------------------------------------
// mbarrier and bulk copy (cp.async.bulk, the non-tensor TMA path)
// ---------------------------------------------------------------------------
// Upper bound of a wait on one mbarrier phase, in SM clock cycles (~1 s).
#define RSI_WAIT_CYCLES (2000000000LL)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait: false if the phase did not complete within `limit` cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long limit = RSI_WAIT_CYCLES) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
// global -> shared bulk copy completing on `bar`; dst, src 16-byte aligned,
// bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
int rsi_num_sms();
