// api.cu -- ABI version, error reporting, the device status word and the
// point-set buffer layout of include/rsi.h.
#include <stdarg.h>
#include <stdio.h>

#include <cuda.h>

#include <atomic>
#include <mutex>

#include "rsi_internal.cuh"

static thread_local char g_last_error[512] = "";

int rsi_fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return code;
}

int rsi_cuda_fail(cudaError_t e, const char* what) {
    return rsi_fail(RSI_E_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" int rsi_version(void) { return RSI_ABI_VERSION; }

static std::atomic<uint64_t> g_launches{0};
void rsi_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t rsi_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char* rsi_last_error(void) { return g_last_error; }

// ---------------------------------------------------------------------------
// context identity: cuCtxGetCurrent and cuCtxGetId, taken through the
// runtime's driver entry points (no link against libcuda)
// ---------------------------------------------------------------------------
namespace {
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<Fn>(p);
}
}  // namespace

unsigned long long rsi_context_id() {
    static CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// one status word per device (a module-scope __device__ variable exists once
// per device context)
static __device__ int g_rsi_status;

#define RSI_MAX_DEVICES 64
// per device: the status word's device address and the context it belongs to
static int* g_status_ptr[RSI_MAX_DEVICES];
static unsigned long long g_status_ctx[RSI_MAX_DEVICES];
static std::mutex g_status_mu;

int* rsi_status_ptr() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RSI_MAX_DEVICES) {
        rsi_fail(RSI_E_CUDA, "rsi_status_ptr: no current CUDA device");
        return nullptr;
    }
    const unsigned long long ctx = rsi_context_id();
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status_ptr[dev] || ctx == 0 || ctx != g_status_ctx[dev]) {
        // first use on this device, or its context was created anew: the
        // address of the previous context's word is no longer valid
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rsi_status);
        if (e != cudaSuccess) {
            rsi_cuda_fail(e, "cudaGetSymbolAddress(status)");
            return nullptr;
        }
        g_status_ptr[dev] = static_cast<int*>(p);
        g_status_ctx[dev] = rsi_context_id();
    }
    return g_status_ptr[dev];
}

extern "C" int rsi_sync_status(void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* st = rsi_status_ptr();
    if (!st) return RSI_E_CUDA;
    int host = 0;
    RSI_CUDA_TRY(cudaMemcpyAsync(&host, st, sizeof(int), cudaMemcpyDeviceToHost, s), "read status");
    RSI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (host != 0) {
        RSI_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int), s), "clear status");
        RSI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    if (host == RSI_DEV_TIMEOUT) return rsi_fail(RSI_E_TIMEOUT, "a device-side wait expired");
    if (host == RSI_DEV_NONFINITE) return rsi_fail(RSI_E_NONFINITE, "non-finite result");
    if (host != 0) return rsi_fail(RSI_E_CUDA, "unknown device status %d", host);
    return RSI_OK;
}

// ---------------------------------------------------------------------------
// point-set layout: fields in enum order, each 256-byte aligned
// ---------------------------------------------------------------------------
static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

size_t rsi_field_bytes_(int32_t field, int64_t n) {
    if (field <= RSI_PF_SV) return sizeof(uint32_t) * size_t(n);
    if (field <= RSI_PF_W) return sizeof(double) * size_t(n);
    return sizeof(float) * size_t(n);
}

extern "C" int64_t rsi_points_offset(int32_t field, int64_t n) {
    if (field < 0 || field >= RSI_PF_COUNT || n < 0) return -1;
    size_t off = 0;
    for (int32_t f = 0; f < field; ++f) off += align256(rsi_field_bytes_(f, n));
    return int64_t(off);
}

extern "C" size_t rsi_points_bytes(int64_t n) {
    if (n < 0) return 0;
    return size_t(rsi_points_offset(RSI_PF_COUNT - 1, n)) + align256(rsi_field_bytes_(RSI_PF_COUNT - 1, n));
}

PointsView rsi_points_view(void* base, int64_t n) {
    char* b = static_cast<char*>(base);
    auto at = [&](int32_t f) { return b + rsi_points_offset(f, n); };
    PointsView v;
    v.idx = reinterpret_cast<uint32_t*>(at(RSI_PF_IDX));
    v.su = reinterpret_cast<uint32_t*>(at(RSI_PF_SU));
    v.sv = reinterpret_cast<uint32_t*>(at(RSI_PF_SV));
    v.x = reinterpret_cast<double*>(at(RSI_PF_X));
    v.y = reinterpret_cast<double*>(at(RSI_PF_Y));
    v.z = reinterpret_cast<double*>(at(RSI_PF_Z));
    v.nx = reinterpret_cast<double*>(at(RSI_PF_NX));
    v.ny = reinterpret_cast<double*>(at(RSI_PF_NY));
    v.nz = reinterpret_cast<double*>(at(RSI_PF_NZ));
    v.w = reinterpret_cast<double*>(at(RSI_PF_W));
    v.xh = reinterpret_cast<float*>(at(RSI_PF_XH));
    v.xl = reinterpret_cast<float*>(at(RSI_PF_XL));
    v.yh = reinterpret_cast<float*>(at(RSI_PF_YH));
    v.yl = reinterpret_cast<float*>(at(RSI_PF_YL));
    v.zh = reinterpret_cast<float*>(at(RSI_PF_ZH));
    v.zl = reinterpret_cast<float*>(at(RSI_PF_ZL));
    return v;
}

int rsi_num_sms() {
    static int cached[RSI_MAX_DEVICES];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RSI_MAX_DEVICES) return 1;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// self-test of the device-side failure path: every thread of one CTA waits on
// an mbarrier that nothing completes, with a limit of `cycles`; the expired
// wait records RSI_DEV_TIMEOUT in the status word (as the stage kernels do)
// and the kernel returns.  Nothing faults or hangs.
// ---------------------------------------------------------------------------
static __global__ void wait_timeout_kernel(long long cycles, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool ok = mbar_wait_bounded(smem_u32(&bar), 0, cycles);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, RSI_DEV_TIMEOUT);
}

extern "C" int rsi_selftest_wait_timeout(int64_t cycles, void* stream) {
    if (cycles < 1 || cycles > (int64_t(1) << 32))
        return rsi_fail(RSI_E_INVAL, "rsi_selftest_wait_timeout: cycles out of range");
    int* st = rsi_status_ptr();
    if (!st) return RSI_E_CUDA;
    wait_timeout_kernel<<<1, 64, 0, static_cast<cudaStream_t>(stream)>>>(cycles, st);
    RSI_CHECK_LAUNCH("wait_timeout_kernel");
    return RSI_OK;
}
