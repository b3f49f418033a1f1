// interface.cu -- step a4 (transmission coefficient and source density on an
// interface, Eqs. transmission_coefficient / reflection_coefficient /
// root_searching; per-point code in interface_body.cuh) and step a7
// (normalised field image k phi / v0).
#include "interface_body.cuh"

namespace {

using namespace rsi_iface;

__global__ void transmit_kernel(rsi_interface it, int64_t n, const double* __restrict__ nxp,
                                const double* __restrict__ nzp, const double2* __restrict__ phi,
                                double2* __restrict__ sigma) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) sigma[i] = transmit_point(it, nxp[i], nzp[i], phi[i]);
}

__global__ void reflect_kernel(rsi_interface it, int64_t n, const double* __restrict__ nxp,
                               const double* __restrict__ nzp, const double2* __restrict__ phi,
                               double2* __restrict__ sigma) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) sigma[i] = reflect_point(it, nxp[i], nzp[i], phi[i]);
}

// field2 may be null
__global__ void image_kernel(int64_t n, const double2* __restrict__ field, const double2* __restrict__ field2,
                             double scale, int format, void* out) {
    int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 f = field[j];
    if (field2) {
        const double2 g = field2[j];
        f.x += g.x;
        f.y += g.y;
    }
    double re = scale * f.x, im = scale * f.y;
    if (format == RSI_IMG_C128) {
        static_cast<double2*>(out)[j] = make_double2(re, im);
    } else if (format == RSI_IMG_C64) {
        static_cast<float2*>(out)[j] = make_float2(float(re), float(im));
    } else {
        static_cast<float*>(out)[j] = float(hypot(re, im));
    }
}

}  // namespace

extern "C" int rsi_interface_transmit(const rsi_interface* it, const void* points, int64_t n,
                                      const double* phi, double* sigma, void* stream) {
    if (!it || !points || !phi || !sigma) return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: null argument");
    if (n < 1) return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: n < 1");
    int rc = check_interface(*it);
    if (rc != RSI_OK) return rc;
    if (reinterpret_cast<uintptr_t>(phi) % 16 || reinterpret_cast<uintptr_t>(sigma) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: complex arrays must be 16-byte aligned");
    PointsView v = rsi_points_view(const_cast<void*>(points), n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    transmit_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        *it, n, v.nx, v.nz, reinterpret_cast<const double2*>(phi), reinterpret_cast<double2*>(sigma));
    RSI_CHECK_LAUNCH("transmit_kernel");
    return RSI_OK;
}

extern "C" int rsi_interface_reflect(const rsi_interface* it, const void* points, int64_t n, const double* phi,
                                     double* sigma, void* stream) {
    if (!it || !points || !phi || !sigma) return rsi_fail(RSI_E_INVAL, "rsi_interface_reflect: null argument");
    if (n < 1) return rsi_fail(RSI_E_INVAL, "rsi_interface_reflect: n < 1");
    int rc = check_interface(*it);
    if (rc != RSI_OK) return rc;
    if (reinterpret_cast<uintptr_t>(phi) % 16 || reinterpret_cast<uintptr_t>(sigma) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_interface_reflect: complex arrays must be 16-byte aligned");
    PointsView v = rsi_points_view(const_cast<void*>(points), n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    reflect_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        *it, n, v.nx, v.nz, reinterpret_cast<const double2*>(phi), reinterpret_cast<double2*>(sigma));
    RSI_CHECK_LAUNCH("reflect_kernel");
    return RSI_OK;
}

extern "C" int rsi_field_image_sum(const rsi_grid* g, const double* field, const double* field_b, double k, double v0,
                                   int32_t format, void* out, void* stream) {
    if (!g || !field || !out) return rsi_fail(RSI_E_INVAL, "rsi_field_image: null argument");
    if (g->nx < 1 || g->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_field_image: empty grid");
    if (format < RSI_IMG_C128 || format > RSI_IMG_ABS32)
        return rsi_fail(RSI_E_INVAL, "rsi_field_image: unknown format %d", format);
    if (!(v0 != 0.0)) return rsi_fail(RSI_E_INVAL, "rsi_field_image: v0 must be non-zero");
    if (reinterpret_cast<uintptr_t>(field) % 16 || reinterpret_cast<uintptr_t>(field_b) % 16 ||
        reinterpret_cast<uintptr_t>(out) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_field_image: arrays must be 16-byte aligned");
    int64_t n = int64_t(g->nx) * g->nz;
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    image_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n, reinterpret_cast<const double2*>(field), reinterpret_cast<const double2*>(field_b), k / v0, format, out);
    RSI_CHECK_LAUNCH("image_kernel");
    return RSI_OK;
}

extern "C" int rsi_field_image(const rsi_grid* g, const double* field, double k, double v0, int32_t format,
                               void* out, void* stream) {
    return rsi_field_image_sum(g, field, nullptr, k, v0, format, out, stream);
}
