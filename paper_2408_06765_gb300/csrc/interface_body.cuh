// interface_body.cuh -- step a4 per point: the plane-wave transmission
// coefficient T12 (Eq. transmission_coefficient) at the incidence angle of
// the point and the source density sigma = T12 phi; shared by the
// single-interface kernel (interface.cu) and the batched kernels (batch.cu).
#pragma once

#include <math.h>

#include "rsi_internal.cuh"

namespace rsi_iface {

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

// cosines of the incidence and refraction angles at a point with unit
// normal (nx, ny, nz): one angle per interface (global) or against the local
// normal (local)
__device__ __forceinline__ void incidence_cosines(const rsi_interface& it, double nx, double nz, Cplx& cos1,
                                                  Cplx& cos2) {
    if (it.mode == RSI_T_GLOBAL) {
        cos1 = cos_of_sin(it.c1 * it.snell_C);
        cos2 = cos_of_sin(it.c2 * it.snell_C);
    } else {
        // beam direction in medium 1 from Snell's invariant, against the local normal
        double s1 = it.c1 * it.snell_C;
        double dz = sqrt(fmax(0.0, 1.0 - s1 * s1));
        double c = s1 * nx + dz * nz;
        c = fmin(fmax(c, 0.0), 1.0);
        cos1 = {c, 0.0};
        cos2 = cos_of_sin(it.c2 / it.c1 * sqrt(1.0 - c * c));
    }
}

// sigma = T12 phi at a point with unit normal (nx, ny, nz)
__device__ __forceinline__ double2 transmit_point(const rsi_interface& it, double nx, double nz, double2 phi) {
    Cplx cos1, cos2;
    incidence_cosines(it, nx, nz, cos1, cos2);
    // T12 = 2 rho1 c2 cos a1 / (rho2 c2 cos a1 + rho1 c1 cos a2)
    Cplx num = {2.0 * it.rho1 * it.c2 * cos1.re, 2.0 * it.rho1 * it.c2 * cos1.im};
    Cplx den = {it.rho2 * it.c2 * cos1.re + it.rho1 * it.c1 * cos2.re,
                it.rho2 * it.c2 * cos1.im + it.rho1 * it.c1 * cos2.im};
    Cplx T = cdiv(num, den);
    Cplx s = cmul(T, {phi.x, phi.y});
    return make_double2(s.re, s.im);
}

// sigma = R12 phi at a point (Eq. reflection_coefficient), the reflected
// field's value on the interface
__device__ __forceinline__ double2 reflect_point(const rsi_interface& it, double nx, double nz, double2 phi) {
    Cplx cos1, cos2;
    incidence_cosines(it, nx, nz, cos1, cos2);
    // R12 = (rho2 c2 cos a1 - rho1 c1 cos a2) / (rho2 c2 cos a1 + rho1 c1 cos a2)
    const Cplx a = {it.rho2 * it.c2 * cos1.re, it.rho2 * it.c2 * cos1.im};
    const Cplx b = {it.rho1 * it.c1 * cos2.re, it.rho1 * it.c1 * cos2.im};
    const Cplx R = cdiv({a.re - b.re, a.im - b.im}, {a.re + b.re, a.im + b.im});
    Cplx s = cmul(R, {phi.x, phi.y});
    return make_double2(s.re, s.im);
}

// host-side check of an interface description
inline int check_interface(const rsi_interface& it) {
    if (it.mode != RSI_T_GLOBAL && it.mode != RSI_T_LOCAL)
        return rsi_fail(RSI_E_INVAL, "unknown transmission mode %d", it.mode);
    if (!(it.rho1 > 0 && it.c1 > 0 && it.rho2 > 0 && it.c2 > 0))
        return rsi_fail(RSI_E_INVAL, "densities and speeds must be > 0");
    if (it.mode == RSI_T_LOCAL && fabs(it.c1 * it.snell_C) > 1.0)
        return rsi_fail(RSI_E_INVAL, "local mode needs a real beam direction");
    return RSI_OK;
}

}  // namespace rsi_iface
