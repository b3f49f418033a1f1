// qmc.cu -- steps a1-a2: integer Sobol points (dimensions 1-2) with a nested
// bit scramble, mapped onto the piston disk (Eq. circle_sampling), a flat
// patch (Eq. square_sampling) or a cylinder, written in cell order; and the
// cell-centred field-image grid as a target point set.  Per-point code is in
// qmc_body.cuh.
#include "qmc_body.cuh"

namespace {

using namespace rsi_qmc;

__global__ void qmc_points_kernel(SurfaceDev s, SobolDirs dirs, uint64_t k0, uint64_t k1, int scramble,
                                  int64_t n, PointsView out) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) make_point(s, dirs, k0, k1, scramble, i, n, out);
}

// slots [first, first + count) of a point set, every field, into a set of
// `count` points (one thread per slot)
__global__ void points_slice_kernel(PointsView in, int64_t first, int64_t count, PointsView out) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t j = first + i;
    out.idx[i] = in.idx[j];
    out.su[i] = in.su[j];
    out.sv[i] = in.sv[j];
    out.x[i] = in.x[j];
    out.y[i] = in.y[j];
    out.z[i] = in.z[j];
    out.nx[i] = in.nx[j];
    out.ny[i] = in.ny[j];
    out.nz[i] = in.nz[j];
    out.w[i] = in.w[j];
    out.xh[i] = in.xh[j];
    out.xl[i] = in.xl[j];
    out.yh[i] = in.yh[j];
    out.yl[i] = in.yl[j];
    out.zh[i] = in.zh[j];
    out.zl[i] = in.zl[j];
}

__global__ void grid_points_kernel(rsi_grid g, PointsView out) {
    int64_t n = int64_t(g.nx) * g.nz;
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < n) make_grid_point(g, q, out);
}

}  // namespace

extern "C" int rsi_make_qmc_points(const rsi_surface* surf, uint64_t seed, uint32_t set_id, int64_t n,
                                   void* points, size_t points_bytes, void* stream) {
    if (!surf || !points) return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: null argument");
    if (n < 1 || n > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: n = %lld outside [1, 2^31]", (long long)n);
    if (points_bytes < rsi_points_bytes(n))
        return rsi_fail(RSI_E_NOMEM, "rsi_make_qmc_points: buffer of %zu bytes < %zu", points_bytes,
                        rsi_points_bytes(n));
    if (reinterpret_cast<uintptr_t>(points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: buffer not 256-byte aligned");
    int rc = check_surface(*surf);
    if (rc != RSI_OK) return rc;
    static const SobolDirs dirs = make_dirs();
    PointsView v = rsi_points_view(points, n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    qmc_points_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        surface_dev(*surf), dirs, dim_key(seed, set_id, 0), dim_key(seed, set_id, 1), surf->scramble ? 1 : 0, n, v);
    RSI_CHECK_LAUNCH("qmc_points_kernel");
    return RSI_OK;
}

extern "C" int rsi_grid_points(const rsi_grid* g, void* points, size_t points_bytes, void* stream) {
    if (!g || !points) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: null argument");
    if (g->nx < 1 || g->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: empty grid");
    int64_t n = int64_t(g->nx) * g->nz;
    if (n > (int64_t(1) << 31)) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: grid too large");
    if (points_bytes < rsi_points_bytes(n)) return rsi_fail(RSI_E_NOMEM, "rsi_grid_points: buffer too small");
    if (reinterpret_cast<uintptr_t>(points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_grid_points: buffer not 256-byte aligned");
    PointsView v = rsi_points_view(points, n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    grid_points_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(*g, v);
    RSI_CHECK_LAUNCH("grid_points_kernel");
    return RSI_OK;
}

extern "C" int rsi_points_slice(const void* points, int64_t n, int64_t first, int64_t count, void* out_points,
                                size_t out_bytes, void* stream) {
    if (!points || !out_points) return rsi_fail(RSI_E_INVAL, "rsi_points_slice: null argument");
    if (n < 1 || n > (int64_t(1) << 31) || first < 0 || count < 1 || first > n - count)
        return rsi_fail(RSI_E_INVAL, "rsi_points_slice: slots [%lld, %lld) outside a set of %lld points",
                        (long long)first, (long long)(first + count), (long long)n);
    if (out_bytes < rsi_points_bytes(count))
        return rsi_fail(RSI_E_NOMEM, "rsi_points_slice: buffer of %zu bytes < %zu", out_bytes,
                        rsi_points_bytes(count));
    if (reinterpret_cast<uintptr_t>(points) % 256 || reinterpret_cast<uintptr_t>(out_points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_points_slice: buffers must be 256-byte aligned");
    const char* a = static_cast<const char*>(points);
    const char* b = static_cast<const char*>(out_points);
    if (a < b + rsi_points_bytes(count) && b < a + rsi_points_bytes(n))
        return rsi_fail(RSI_E_INVAL, "rsi_points_slice: input and output overlap");
    PointsView in = rsi_points_view(const_cast<void*>(points), n);
    PointsView out = rsi_points_view(out_points, count);
    int threads = 256;
    unsigned blocks = unsigned((count + threads - 1) / threads);
    points_slice_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(in, first, count, out);
    RSI_CHECK_LAUNCH("points_slice_kernel");
    return RSI_OK;
}
