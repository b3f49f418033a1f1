// interface.cu -- step a4 (transmission coefficient and source density on an
// interface, Eqs. transmission_coefficient / reflection_coefficient /
// root_searching) and step a7 (normalised field image k phi / v0).
#include <math.h>

#include "rsi_internal.cuh"

namespace {

struct Cplx {
    double re, im;
};
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cplx cdiv(Cplx a, Cplx b) {
    // Smith's algorithm (1962) for complex division
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    double r = b.re / b.im, d = b.im + b.re * r;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
// cosine of an angle with real sine s: sqrt(1 - s^2), or i sqrt(s^2 - 1)
// past the critical angle (Im >= 0, evanescent for e^{-i w t})
__device__ __forceinline__ Cplx cos_of_sin(double s) {
    double q = 1.0 - s * s;
    if (q >= 0.0) return {sqrt(q), 0.0};
    return {0.0, sqrt(-q)};
}

__global__ void transmit_kernel(rsi_interface it, int64_t n, const double* __restrict__ nxp,
                                const double* __restrict__ nyp, const double* __restrict__ nzp,
                                const double2* __restrict__ phi, double2* __restrict__ sigma) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Cplx cos1, cos2;
    if (it.mode == RSI_T_GLOBAL) {
        cos1 = cos_of_sin(it.c1 * it.snell_C);
        cos2 = cos_of_sin(it.c2 * it.snell_C);
    } else {
        // beam direction in medium 1 from Snell's invariant, against the local normal
        double s1 = it.c1 * it.snell_C;
        double dz = sqrt(fmax(0.0, 1.0 - s1 * s1));
        double c = s1 * nxp[i] + dz * nzp[i];
        c = fmin(fmax(c, 0.0), 1.0);
        cos1 = {c, 0.0};
        cos2 = cos_of_sin(it.c2 / it.c1 * sqrt(1.0 - c * c));
    }
    // T12 = 2 rho1 c2 cos a1 / (rho2 c2 cos a1 + rho1 c1 cos a2)
    Cplx num = {2.0 * it.rho1 * it.c2 * cos1.re, 2.0 * it.rho1 * it.c2 * cos1.im};
    Cplx den = {it.rho2 * it.c2 * cos1.re + it.rho1 * it.c1 * cos2.re,
                it.rho2 * it.c2 * cos1.im + it.rho1 * it.c1 * cos2.im};
    Cplx T = cdiv(num, den);
    double2 p = phi[i];
    Cplx s = cmul(T, {p.x, p.y});
    sigma[i] = make_double2(s.re, s.im);
}

__global__ void image_kernel(int64_t n, const double2* __restrict__ field, double scale, int format, void* out) {
    int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 f = field[j];
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
    if (it->mode != RSI_T_GLOBAL && it->mode != RSI_T_LOCAL)
        return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: unknown mode %d", it->mode);
    if (!(it->rho1 > 0 && it->c1 > 0 && it->rho2 > 0 && it->c2 > 0))
        return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: densities and speeds must be > 0");
    if (it->mode == RSI_T_LOCAL && fabs(it->c1 * it->snell_C) > 1.0)
        return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: local mode needs a real beam direction");
    if (reinterpret_cast<uintptr_t>(phi) % 16 || reinterpret_cast<uintptr_t>(sigma) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_interface_transmit: complex arrays must be 16-byte aligned");
    PointsView v = rsi_points_view(const_cast<void*>(points), n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    transmit_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        *it, n, v.nx, v.ny, v.nz, reinterpret_cast<const double2*>(phi), reinterpret_cast<double2*>(sigma));
    RSI_CHECK_LAUNCH("transmit_kernel");
    return RSI_OK;
}

extern "C" int rsi_field_image(const rsi_grid* g, const double* field, double k, double v0, int32_t format,
                               void* out, void* stream) {
    if (!g || !field || !out) return rsi_fail(RSI_E_INVAL, "rsi_field_image: null argument");
    if (g->nx < 1 || g->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_field_image: empty grid");
    if (format < RSI_IMG_C128 || format > RSI_IMG_ABS32)
        return rsi_fail(RSI_E_INVAL, "rsi_field_image: unknown format %d", format);
    if (!(v0 != 0.0)) return rsi_fail(RSI_E_INVAL, "rsi_field_image: v0 must be non-zero");
    if (reinterpret_cast<uintptr_t>(field) % 16 || reinterpret_cast<uintptr_t>(out) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_field_image: arrays must be 16-byte aligned");
    int64_t n = int64_t(g->nx) * g->nz;
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    image_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        n, reinterpret_cast<const double2*>(field), k / v0, format, out);
    RSI_CHECK_LAUNCH("image_kernel");
    return RSI_OK;
}
