// raytrace.cu -- the ray-tracing model of Sec. 2.2 (Eq. transmitted_ray_tracing)
// on the GPU: for every field point Q in medium 2, below the plane interface
// z = z_I, the sum over transducer points P of
//   A_P T12 e^{i (k1 D1 + k2 D2)} / sqrt((D1 + c2 cos^2 a1 / (c1 cos^2 a2) D2) (D1 + (c2 / c1) D2)),
// A_P = -v0 w_P / (2 pi), along the refracted ray from P to Q (Snell's law,
// Eq. root_searching; Fermat's principle, Eq. fermat_principle).
//
// Sources are the piston stage's FP32C tiles (offsets p = P - c from the
// tile centre c, amplitudes A).  Per (target, tile) a reference ray through
// the tile centre is solved once: its crossing point X_c (safeguarded Newton
// on Snell's residual, FP32: the travel time is stationary in the crossing
// point, so an FP32 crossing costs no phase accuracy), the path lengths D1c,
// D2c and tau = k1 D1c + k2 D2c mod 2 pi in double-float.  Per pair only the
// offset of the pair's crossing from X_c is solved (Newton from the first-
// order guess), and D1 - D1c, D2 - D2c follow from differences of squares of
// small offsets, so the phase carries about 2^-23 k (tile size) of error, as
// in the RSI stage kernel.
#include <math.h>

#include "stage.cuh"

namespace {

constexpr int kRtThreads = 256;
// Crossing-point convergence: the phase is second order in the crossing
// error (Fermat), the amplitude first order; 1 nm keeps both below 1e-6 for
// path legs down to 0.1 mm at 10 MHz in water.
//
// The test is on the error left after the last Newton step, not on the step
// itself: for Snell's residual G(t) = s1 t / D1 - s2 b / D2 (b = rho - t),
//   G'  = s1 h1^2 / D1^3 + s2 h2^2 / D2^3,
//   |G''| <= 3 s1 h1^2 t / D1^5 + 3 s2 h2^2 b / D2^5 <= 3 G' max(1/D1, 1/D2),
// so a Newton step of length q from t leaves |t' - t*| <~ |G''| q^2 / (2 G')
// <= 1.5 max(1/D1, 1/D2) q^2.  In FP32 the step itself never settles below
// the rounding of G (a few nm on 50 mm legs), so a test on |q| would send
// most rays into the safeguarded loop for nothing.
constexpr float kCrossTol = 1e-9f;
constexpr float kCrossCurv = 1.5f;
constexpr int kCrossExtra = 12;

struct RtArgs {
    const uint8_t* tiles;
    size_t tile_bytes;
    int S, n_tiles, tiles_per_split, splits;
    TgtView tgt;
    int64_t n_tgt;
    float zIh, zIl;          // interface plane, double-float
    float k1h, k1l, k2h, k2l;
    float s1, s2;            // slownesses 1/c1, 1/c2
    float c21;               // c2 / c1
    float Tn, Td1, Td2;      // T12 = Tn cos a1 / (Td1 cos a1 + Td2 cos a2), scaled by 1/(rho1 c1)
    int newton;              // Newton steps per pair
    TwoPiSplit tp;
    double2* out;            // [splits][n_tgt] partials, or the field
    int* status;
};

// reference ray of one target through one tile centre
struct RayRef {
    float dx, dy;      // horizontal offset target - centre
    float ux, uy;      // its direction
    float rho, irho;   // its length and 1/length (0 when the target is straight below)
    float H1, H2;      // heights of the centre above and of the target below the interface
    float tc, bc;      // horizontal legs of the reference ray in media 1 and 2 (tc + bc = rho)
    float D1, D2;      // path lengths of the reference ray
    float tau;         // k1 D1 + k2 D2 mod 2 pi
    float a_r, a_h;    // linear response of the crossing to the foot distance and the source height
    float s2h22;       // s2 H2^2 (Snell residual slope, medium-2 term)
    float ih22;        // 1 / H2^2
};

__device__ __forceinline__ float rsqrt_ap(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// square root of a positive double-float (one Newton step from rsqrt)
__device__ __forceinline__ void df_sqrt(float sh, float sl, float& rh, float& rl) {
    rh = 0.0f;
    rl = 0.0f;
    if (sh > 0.0f) {
        float y = rsqrtf(sh);
        float r0 = __fmul_rn(sh, y);
        float p, pe;
        two_prod(r0, r0, p, pe);
        float e = __fadd_rn(__fsub_rn(__fsub_rn(sh, p), pe), sl);
        fast_two_sum(r0, __fmul_rn(e, __fmul_rn(0.5f, y)), rh, rl);
    }
}

// Snell's residual of a crossing at horizontal distance t from the source
// foot (b = rho - t beyond it): G = s1 sin a1 - s2 sin a2, its slope
// dG = s1 h1^2 / D1^3 + s2 h2^2 / D2^3 (h1q = h1^2, s1h = s1 h1^2, s2h = s2 h2^2)
// and m = max(1/D1, 1/D2), the curvature bound of the convergence test
__device__ __forceinline__ void snell_residual(float t, float b, float h1q, float h2q, float s1, float s2, float s1h,
                                               float s2h, float& G, float& dG, float& m) {
    const float r1 = rsqrt_ap(fmaf(t, t, h1q));
    const float r2 = rsqrt_ap(fmaf(b, b, h2q));
    G = fmaf(s1 * t, r1, -(s2 * b) * r2);
    dG = fmaf(s1h, r1 * r1 * r1, s2h * (r2 * r2 * r2));
    m = fmaxf(r1, r2);
}

__device__ __forceinline__ RayRef ray_reference(float qxh, float qxl, float qyh, float qyl, float qzh, float qzl,
                                                const float* c, const RtArgs& a) {
    RayRef R;
    float dxh, dxl, dyh, dyl, h1h, h1l, h2h, h2l;
    df_diff(qxh, qxl, c[0], c[1], dxh, dxl);
    df_diff(qyh, qyl, c[2], c[3], dyh, dyl);
    df_diff(a.zIh, a.zIl, c[4], c[5], h1h, h1l);  // z_I - c_z
    df_diff(qzh, qzl, a.zIh, a.zIl, h2h, h2l);    // q_z - z_I
    float ax, axl, ay, ayl, sh, sl, rh, rl;
    df_sqr(dxh, dxl, ax, axl);
    df_sqr(dyh, dyl, ay, ayl);
    df_add_pos(ax, axl, ay, ayl, sh, sl);
    df_sqrt(sh, sl, rh, rl);  // rho_c
    R.dx = dxh;
    R.dy = dyh;
    R.rho = rh;
    R.irho = rh > 1e-9f ? 1.0f / rh : 0.0f;
    R.ux = rh > 1e-9f ? dxh * R.irho : 1.0f;
    R.uy = rh > 1e-9f ? dyh * R.irho : 0.0f;
    R.H1 = h1h;
    R.H2 = h2h;
    // crossing: safeguarded Newton on the monotone residual over [0, rho],
    // from the small-angle guess t = rho h1 / (h1 + (c2/c1) h2)
    float lo = 0.0f, hi = rh;
    float t = rh * __fdividef(h1h, fmaf(a.c21, h2h, h1h));
    const float h1q = h1h * h1h, h2q = h2h * h2h;
#pragma unroll 1
    for (int it = 0; it < 24; ++it) {
        float G, dG, m;
        snell_residual(t, rh - t, h1q, h2q, a.s1, a.s2, a.s1 * h1q, a.s2 * h2q, G, dG, m);
        if (G > 0.0f)
            hi = t;
        else
            lo = t;
        float tn = t - __fdividef(G, dG);
        t = (tn >= lo && tn <= hi) ? tn : 0.5f * (lo + hi);
    }
    R.tc = t;
    // b = rho_c - t_c and the path lengths, as double-floats
    float bh, bl;
    two_sum(rh, -t, bh, bl);
    bl = __fadd_rn(bl, rl);
    fast_two_sum(bh, bl, bh, bl);
    R.bc = bh;
    float p1h, p1l, p2h, p2l, qh, ql, D1h, D1l, D2h, D2l;
    two_prod(t, t, p1h, p1l);
    df_sqr(h1h, h1l, qh, ql);
    df_add_pos(p1h, p1l, qh, ql, p1h, p1l);
    df_sqrt(p1h, p1l, D1h, D1l);
    df_sqr(bh, bl, p2h, p2l);
    df_sqr(h2h, h2l, qh, ql);
    df_add_pos(p2h, p2l, qh, ql, p2h, p2l);
    df_sqrt(p2h, p2l, D2h, D2l);
    R.D1 = D1h;
    R.D2 = D2h;
    // implicit differentiation of Snell's residual at the reference ray:
    // a pair whose source sits pz higher and whose feet are drho closer
    // crosses about -(a_r drho + a_h pz) further along its own line
    {
        const float i1 = 1.0f / D1h, i2 = 1.0f / D2h;
        const float i13 = i1 * i1 * i1, i23 = i2 * i2 * i2;
        const float gr = a.s2 * h2h * h2h * i23;
        const float gp = fmaf(a.s1 * h1h * h1h, i13, gr);
        const float ig = 1.0f / gp;
        R.a_r = gr * ig;
        R.a_h = a.s1 * t * h1h * i13 * ig;
    }
    R.s2h22 = a.s2 * h2q;
    R.ih22 = 1.0f / h2q;
    // k1 D1 + k2 D2 as a double-float, reduced modulo 2 pi (Cody & Waite)
    float ph, pl, eh, el;
    two_prod(a.k1h, D1h, ph, pl);
    pl = __fmaf_rn(a.k1h, D1l, __fmaf_rn(a.k1l, D1h, pl));
    two_prod(a.k2h, D2h, eh, el);
    el = __fmaf_rn(a.k2h, D2l, __fmaf_rn(a.k2l, D2h, el));
    float sh2, sl2;
    two_sum(ph, eh, sh2, sl2);
    sl2 = __fadd_rn(sl2, __fadd_rn(pl, el));
    fast_two_sum(sh2, sl2, ph, pl);
    float n = rintf(__fmul_rn(ph, a.tp.inv));
    float x = __fmaf_rn(-n, a.tp.p1, ph);
    x = __fmaf_rn(-n, a.tp.p2, x);
    x = __fmaf_rn(-n, a.tp.p3, x);
    R.tau = __fadd_rn(x, pl);
    return R;
}

// safeguarded steps for the crossing offset dt of one pair whose Newton
// steps may still leave more than kCrossTol (est, the bound above): Newton
// inside a bracket of the monotone residual, bisection otherwise, until a
// Newton step's bound falls below kCrossTol
__device__ __forceinline__ float cross_safeguarded(const RayRef& R, const RtArgs& a, float h1q, float h2q, float s1h,
                                                float bfix, float lo0, float hi0, float dt, float est) {
    float lo = lo0, hi = hi0;
#pragma unroll 1
    for (int it = 0; it < kCrossExtra && est > kCrossTol; ++it) {
        float G, dG, m;
        snell_residual(R.tc + dt, bfix - dt, h1q, h2q, a.s1, a.s2, s1h, R.s2h22, G, dG, m);
        if (G > 0.0f)
            hi = dt;
        else
            lo = dt;
        const float q = __fdividef(G, dG);
        const float dn = dt - q;
        const bool in = dn >= lo && dn <= hi;
        est = in ? kCrossCurv * m * (q * q) : INFINITY;
        dt = in ? dn : 0.5f * (lo + hi);
    }
    return dt;
}

// one transducer point (offset p, amplitude A) onto one reference ray; NW
// Newton steps for the crossing (0: a.newton at run time)
template <int NW>
__device__ __forceinline__ void ray_pair(const RayRef& R, const float4& rec, float A, const RtArgs& a, float k1,
                                         float k2, float& acc_r, float& acc_i) {
    const float px = rec.x, py = rec.y, pz = rec.z;
    // horizontal foot-to-foot vector v = d - p_h, its length and direction
    const float vx = R.dx - px, vy = R.dy - py;
    const float v2 = fmaf(vx, vx, vy * vy);
    const float iv = v2 > 1e-24f ? rsqrt_ap(v2) : 0.0f;
    const float rho = v2 * iv;
    const float ux = v2 > 1e-24f ? vx * iv : R.ux, uy = v2 > 1e-24f ? vy * iv : R.uy;
    // rho_c - rho from rho_c^2 - rho^2 = 2 d.p_h - |p_h|^2, and u - u_c
    const float dpp = fmaf(2.0f * R.dx, px, fmaf(2.0f * R.dy, py, -fmaf(px, px, py * py)));
    const float drho = __fdividef(dpp, R.rho + rho + 1e-30f);
    float wx, wy;  // u - u_c
    if (R.irho > 0.0f && iv > 0.0f) {
        const float s = R.irho * iv;  // 1 / (rho rho_c)
        wx = fmaf(R.dx, drho, -px * R.rho) * s;
        wy = fmaf(R.dy, drho, -py * R.rho) * s;
    } else {
        wx = ux - R.ux;
        wy = uy - R.uy;
    }
    const float h1 = R.H1 - pz, h2 = R.H2;
    const float h1q = h1 * h1, h2q = h2 * h2, s1h = a.s1 * h1q;
    // crossing offset dt = t - t_c along u; the legs are t_c + dt and b_c - drho - dt
    const float bfix = R.bc - drho;
    const float lo0 = -R.tc, hi0 = bfix;
    float dt = -fmaf(R.a_r, drho, R.a_h * pz);  // linear prediction from the reference ray
    dt = fminf(fmaxf(dt, lo0), hi0);
    float est = INFINITY;
    // plain Newton steps (kept inside the segment) from the prediction; the
    // bound uses the unclamped step, which also bounds a clamped one (the
    // root lies inside the segment)
    const int nw = NW ? NW : a.newton;
#pragma unroll
    for (int it = 0; it < (NW ? NW : 16); ++it) {
        if (!NW && it >= nw) break;
        float G, dG, m;
        snell_residual(R.tc + dt, bfix - dt, h1q, h2q, a.s1, a.s2, s1h, R.s2h22, G, dG, m);
        const float q = __fdividef(G, dG);
        est = kCrossCurv * m * (q * q);
        dt = fminf(fmaxf(dt - q, lo0), hi0);
    }
    // then, for the rays that may still be off by more than kCrossTol (those
    // that graze the interface near the target converge more slowly),
    // safeguarded steps
    if (est > kCrossTol) dt = cross_safeguarded(R, a, h1q, h2q, s1h, bfix, lo0, hi0, dt, est);
    // e1 = (X - P) - (X_c - c) = (dt u + t_c (u - u_c), -p_z); e2 = -(p_h + e1_h, 0)
    const float e1x = fmaf(dt, ux, R.tc * wx), e1y = fmaf(dt, uy, R.tc * wy), e1z = -pz;
    const float e2x = -(px + e1x), e2y = -(py + e1y);
    // D^2 - Dc^2 = 2 b.e + |e|^2 with b1 = (t_c u_c, H1), b2 = (b_c u_c, H2)
    const float t1 = fmaf(2.0f * R.tc, fmaf(R.ux, e1x, R.uy * e1y), fmaf(2.0f * R.H1, e1z, fmaf(e1x, e1x, fmaf(e1y, e1y, e1z * e1z))));
    const float t2 = fmaf(2.0f * R.bc, fmaf(R.ux, e2x, R.uy * e2y), fmaf(e2x, e2x, e2y * e2y));
    const float q1 = fmaf(R.D1, R.D1, t1), q2 = fmaf(R.D2, R.D2, t2);
    const float ir1 = rsqrt_ap(q1), ir2 = rsqrt_ap(q2);
    const float D1 = q1 * ir1, D2 = q2 * ir2;
    // D - Dc without a division: (D0 - Dc) + (q - D0^2) / (2 D0), D0 = q / sqrt(q) from the
    // approximate reciprocal square root, q - D0^2 = t - (D0 - Dc)(D0 + Dc) (one Newton step)
    const float am1 = D1 - R.D1, am2 = D2 - R.D2;
    const float dD1 = fmaf(fmaf(-am1, D1 + R.D1, t1), 0.5f * ir1, am1);
    const float dD2 = fmaf(fmaf(-am2, D2 + R.D2, t2), 0.5f * ir2, am2);
    const float u = fmaf(k1, dD1, fmaf(k2, dD2, R.tau));
    // angles of the ray, T12 (Eq. transmission_coefficient) and the spreading
    const float cos1 = h1 * ir1, cos2 = h2 * ir2;
    // T12 = Tn cos1 / td folded into the spreading's reciprocal square root:
    // A T / sqrt(den) = A Tn cos1 / sqrt(den td^2)
    const float td = fmaf(a.Td1, cos1, a.Td2 * cos2);
    // cos^2 a1 / cos^2 a2 D2 = cos^2 a1 D2^3 / h2^2
    const float den = fmaf(a.c21 * cos1 * cos1 * R.ih22, D2 * q2, D1) * fmaf(a.c21, D2, D1);
    const float amp = A * (a.Tn * cos1) * rsqrt_ap(den * (td * td));
    float s, c;
    __sincosf(u, &s, &c);
    acc_r = fmaf(amp, c, acc_r);
    acc_i = fmaf(amp, s, acc_i);
}

#ifndef RSI_RT_PACKED
#define RSI_RT_PACKED 1  // two transducer points per f32x2 instruction
#endif

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
// x - y as one packed FMA, y (-1) + x: rounded once, so equal to the
// subtraction; a packed negation would be an instruction of its own
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2(-1.0f), x); }

// ray_pair for two transducer points at once: the same quantities, the
// additions, products and FMAs two at a time (f32x2), every sign folded into
// a negated per-tile constant or an FMA by -1 (no packed negations), the
// reciprocal square roots, divisions, clamps and sincos per point, and the
// safeguarded steps only for a point whose ray has not converged
template <int NW>
__device__ __forceinline__ void ray_pair2(const RayRef& R, float2 px, float2 py, float2 pzn, float2 A,
                                          const RtArgs& a, float k1, float k2, float2& acc_r, float2& acc_i) {
    const float2 vx = sub2(f2(R.dx), px), vy = sub2(f2(R.dy), py);
    const float2 v2 = __ffma2_rn(vx, vx, __fmul2_rn(vy, vy));
    const bool okx = v2.x > 1e-24f, oky = v2.y > 1e-24f;
    const float2 iv = make_float2(okx ? rsqrt_ap(v2.x) : 0.0f, oky ? rsqrt_ap(v2.y) : 0.0f);
    const float2 rho = __fmul2_rn(v2, iv);
    float2 ux = __fmul2_rn(vx, iv), uy = __fmul2_rn(vy, iv);
    if (!okx) ux.x = R.ux, uy.x = R.uy;
    if (!oky) ux.y = R.ux, uy.y = R.uy;
    // rho_c^2 - rho^2 = 2 d.p_h - |p_h|^2 = px (2 dx - px) + py (2 dy - py)
    const float2 dpp = __ffma2_rn(px, sub2(f2(2.0f * R.dx), px), __fmul2_rn(py, sub2(f2(2.0f * R.dy), py)));
    const float2 dd = __fadd2_rn(f2(R.rho + 1e-30f), rho);
    const float2 drho = make_float2(__fdividef(dpp.x, dd.x), __fdividef(dpp.y, dd.y));
    const float2 sw = __fmul2_rn(f2(R.irho), iv);
    float2 wx = __fmul2_rn(__ffma2_rn(f2(R.dx), drho, __fmul2_rn(px, f2(-R.rho))), sw);
    float2 wy = __fmul2_rn(__ffma2_rn(f2(R.dy), drho, __fmul2_rn(py, f2(-R.rho))), sw);
    if (!(R.irho > 0.0f && iv.x > 0.0f)) wx.x = ux.x - R.ux, wy.x = uy.x - R.uy;
    if (!(R.irho > 0.0f && iv.y > 0.0f)) wx.y = ux.y - R.ux, wy.y = uy.y - R.uy;
    const float2 h1 = __fadd2_rn(f2(R.H1), pzn);  // pzn = -p_z
    const float h2 = R.H2;
    const float2 h1q = __fmul2_rn(h1, h1);
    const float h2q = h2 * h2;
    const float2 s1h = __fmul2_rn(f2(a.s1), h1q);
    const float2 bfix = sub2(f2(R.bc), drho);
    const float lo0 = -R.tc;
    float2 dt = __ffma2_rn(f2(-R.a_r), drho, __fmul2_rn(f2(R.a_h), pzn));
    dt.x = fminf(fmaxf(dt.x, lo0), bfix.x);
    dt.y = fminf(fmaxf(dt.y, lo0), bfix.y);
    float2 est = f2(INFINITY);
    const int nw = NW ? NW : a.newton;
#pragma unroll
    for (int it = 0; it < (NW ? NW : 16); ++it) {
        if (!NW && it >= nw) break;
        const float2 t = __fadd2_rn(f2(R.tc), dt), b = sub2(bfix, dt);
        const float2 q1 = __ffma2_rn(t, t, h1q), q2 = __ffma2_rn(b, b, f2(h2q));
        const float2 e1 = make_float2(rsqrt_ap(q1.x), rsqrt_ap(q1.y));
        const float2 e2 = make_float2(rsqrt_ap(q2.x), rsqrt_ap(q2.y));
        const float2 G = __ffma2_rn(__fmul2_rn(f2(a.s1), t), e1, __fmul2_rn(__fmul2_rn(f2(-a.s2), b), e2));
        const float2 dG = __ffma2_rn(s1h, __fmul2_rn(__fmul2_rn(e1, e1), e1),
                                     __fmul2_rn(f2(R.s2h22), __fmul2_rn(__fmul2_rn(e2, e2), e2)));
        const float2 q = make_float2(__fdividef(G.x, dG.x), __fdividef(G.y, dG.y));
        const float2 m = make_float2(fmaxf(e1.x, e2.x), fmaxf(e1.y, e2.y));
        est = __fmul2_rn(__fmul2_rn(f2(kCrossCurv), m), __fmul2_rn(q, q));
        const float2 dn = sub2(dt, q);
        dt = make_float2(fminf(fmaxf(dn.x, lo0), bfix.x), fminf(fmaxf(dn.y, lo0), bfix.y));
    }
    if (est.x > kCrossTol) dt.x = cross_safeguarded(R, a, h1q.x, h2q, s1h.x, bfix.x, lo0, bfix.x, dt.x, est.x);
    if (est.y > kCrossTol) dt.y = cross_safeguarded(R, a, h1q.y, h2q, s1h.y, bfix.y, lo0, bfix.y, dt.y, est.y);
    // e1 = (dt u + t_c w, -p_z) and g = -e2_h = p_h + e1_h; the squares of
    // -p_z and -g equal those of p_z and g, and the signs of the cross terms
    // go into the per-tile constants -2 H1 and -2 b_c
    const float2 e1x = __ffma2_rn(dt, ux, __fmul2_rn(f2(R.tc), wx));
    const float2 e1y = __ffma2_rn(dt, uy, __fmul2_rn(f2(R.tc), wy));
    const float2 gx = __fadd2_rn(px, e1x), gy = __fadd2_rn(py, e1y);
    const float2 t1 = __ffma2_rn(f2(2.0f * R.tc), __ffma2_rn(f2(R.ux), e1x, __fmul2_rn(f2(R.uy), e1y)),
                                 __ffma2_rn(f2(2.0f * R.H1), pzn,
                                            __ffma2_rn(e1x, e1x, __ffma2_rn(e1y, e1y, __fmul2_rn(pzn, pzn)))));
    const float2 t2 = __ffma2_rn(f2(-2.0f * R.bc), __ffma2_rn(f2(R.ux), gx, __fmul2_rn(f2(R.uy), gy)),
                                 __ffma2_rn(gx, gx, __fmul2_rn(gy, gy)));
    const float2 q1 = __ffma2_rn(f2(R.D1), f2(R.D1), t1), q2 = __ffma2_rn(f2(R.D2), f2(R.D2), t2);
    const float2 ir1 = make_float2(rsqrt_ap(q1.x), rsqrt_ap(q1.y)), ir2 = make_float2(rsqrt_ap(q2.x), rsqrt_ap(q2.y));
    const float2 D1 = __fmul2_rn(q1, ir1), D2 = __fmul2_rn(q2, ir2);
    // D - Dc by one Newton step, as in ray_pair: am = D - Dc, and
    // t - am (D + Dc) = am (-(D + Dc)) + t with -(D + Dc) = D (-1) - Dc
    const float2 am1 = __fadd2_rn(D1, f2(-R.D1)), am2 = __fadd2_rn(D2, f2(-R.D2));
    const float2 ns1 = __ffma2_rn(D1, f2(-1.0f), f2(-R.D1)), ns2 = __ffma2_rn(D2, f2(-1.0f), f2(-R.D2));
    const float2 dD1 = __ffma2_rn(__ffma2_rn(am1, ns1, t1), __fmul2_rn(f2(0.5f), ir1), am1);
    const float2 dD2 = __ffma2_rn(__ffma2_rn(am2, ns2, t2), __fmul2_rn(f2(0.5f), ir2), am2);
    const float2 u = __ffma2_rn(f2(k1), dD1, __ffma2_rn(f2(k2), dD2, f2(R.tau)));
    const float2 cos1 = __fmul2_rn(h1, ir1), cos2 = __fmul2_rn(f2(h2), ir2);
    const float2 tn = __fmul2_rn(f2(a.Tn), cos1), td = __ffma2_rn(f2(a.Td1), cos1, __fmul2_rn(f2(a.Td2), cos2));
    // T12 = tn / td folded into the spreading's reciprocal square root, as in ray_pair
    const float2 cc = __fmul2_rn(__fmul2_rn(__fmul2_rn(f2(a.c21), cos1), cos1), f2(R.ih22));
    const float2 den = __fmul2_rn(__ffma2_rn(cc, __fmul2_rn(D2, q2), D1), __ffma2_rn(f2(a.c21), D2, D1));
    const float2 dt2 = __fmul2_rn(den, __fmul2_rn(td, td));
    const float2 amp = __fmul2_rn(__fmul2_rn(A, tn), make_float2(rsqrt_ap(dt2.x), rsqrt_ap(dt2.y)));
    float2 sn, cs;
    __sincosf(u.x, &sn.x, &cs.x);
    __sincosf(u.y, &sn.y, &cs.y);
    acc_r = __ffma2_rn(amp, cs, acc_r);
    acc_i = __ffma2_rn(amp, sn, acc_i);
}

// resident CTAs per SM asked of the compiler: 4 (64 registers) measured best
// for the packed form on the f2 workload (171.6 Gpair/s; 3 CTAs 160.6, no
// bound 143.7), although ptxas then keeps 20 bytes per thread in local memory
#ifndef RSI_RT_MIN_BLOCKS
#define RSI_RT_MIN_BLOCKS 4
#endif

template <int TPT, int NW>
__global__ void __launch_bounds__(kRtThreads, RSI_RT_MIN_BLOCKS) raytrace_kernel(RtArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * a.tile_bytes);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < RSI_PIPE_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int split = blockIdx.y;
    const int t_begin = split * a.tiles_per_split;
    const int ntile = max(0, min(a.n_tiles, t_begin + a.tiles_per_split) - t_begin);
    const uint32_t tb = uint32_t(a.tile_bytes);
    int64_t jt[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int64_t j = int64_t(blockIdx.x) * TPT * kRtThreads + int64_t(q) * kRtThreads + tid;
        jt[q] = j < a.n_tgt ? j : a.n_tgt - 1;
    }
    if (tid == 0)
        for (int s = 0; s < RSI_PIPE_STAGES && s < ntile; ++s) {
            const uint32_t bar = smem_u32(&bars[s]);
            mbar_expect_tx(bar, tb);
            bulk_g2s(smem_u32(smem + s * tb), a.tiles + size_t(t_begin + s) * tb, tb, bar);
        }
    float hr[TPT], lr[TPT], hi[TPT], li[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) hr[q] = lr[q] = hi[q] = li[q] = 0.0f;
    const float k1 = a.k1h, k2 = a.k2h;
    int failed_at = -1;
    for (int it = 0; it < ntile; ++it) {
        const int buf = it % RSI_PIPE_STAGES;
        const bool ok = mbar_wait_bounded(smem_u32(&bars[buf]), uint32_t(it / RSI_PIPE_STAGES) & 1u);
        if (__syncthreads_or(!ok)) {
            failed_at = it;
            break;
        }
        const uint8_t* tile = smem + buf * tb;
        const float* hdr = reinterpret_cast<const float*>(tile);
        const float4* rec = reinterpret_cast<const float4*>(tile + RSI_TILE_HDR_BYTES);
        RayRef ref[TPT];
        float ar[TPT], ai[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t j = jt[q];
            ref[q] = ray_reference(__ldg(a.tgt.xh + j), __ldg(a.tgt.xl + j), __ldg(a.tgt.yh + j), __ldg(a.tgt.yl + j),
                                   __ldg(a.tgt.zh + j), __ldg(a.tgt.zl + j), hdr, a);
            ar[q] = ai[q] = 0.0f;
        }
#if RSI_RT_PACKED
        {  // tiles hold an even number of points (32 .. 256), pair-interleaved:
           // per point pair (px, px', py, py'), (-pz, -pz', ...), (A, A', 0, 0), 0
            float2 pr[TPT], pi[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) pr[q] = pi[q] = f2(0.0f);
#pragma unroll 1
            for (int i = 0; i < a.S; i += 2) {
                const float4 v0 = rec[2 * i], v1 = rec[2 * i + 1], v2 = rec[2 * i + 2];
                const float2 px = make_float2(v0.x, v0.y), py = make_float2(v0.z, v0.w);
                const float2 pzn = make_float2(v1.x, v1.y), A = make_float2(v2.x, v2.y);
#pragma unroll
                for (int q = 0; q < TPT; ++q) ray_pair2<NW>(ref[q], px, py, pzn, A, a, k1, k2, pr[q], pi[q]);
            }
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                ar[q] = pr[q].x + pr[q].y;
                ai[q] = pi[q].x + pi[q].y;
            }
        }
#else
#pragma unroll 1
        for (int i = 0; i < a.S; ++i) {
            const float4 ra = rec[2 * i];
            const float A = rec[2 * i + 1].x;
#pragma unroll
            for (int q = 0; q < TPT; ++q) ray_pair<NW>(ref[q], ra, A, a, k1, k2, ar[q], ai[q]);
        }
#endif
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            float s, e;
            two_sum(hr[q], ar[q], s, e);
            hr[q] = s;
            lr[q] = __fadd_rn(lr[q], e);
            two_sum(hi[q], ai[q], s, e);
            hi[q] = s;
            li[q] = __fadd_rn(li[q], e);
        }
        __syncthreads();  // every thread is done with this buffer
        if (tid == 0 && it + RSI_PIPE_STAGES < ntile) {
            const uint32_t bar = smem_u32(&bars[buf]);
            mbar_expect_tx(bar, tb);
            bulk_g2s(smem_u32(smem + buf * tb), a.tiles + size_t(t_begin + it + RSI_PIPE_STAGES) * tb, tb, bar);
        }
    }
    if (failed_at >= 0) {
        if (tid == 0) {
            atomicExch(a.status, RSI_DEV_TIMEOUT);
            for (int it = failed_at; it < ntile && it < failed_at + RSI_PIPE_STAGES; ++it)
                mbar_wait_bounded(smem_u32(&bars[it % RSI_PIPE_STAGES]), uint32_t(it / RSI_PIPE_STAGES) & 1u);
        }
        return;
    }
    double2* out = a.out + (a.splits > 1 ? size_t(split) * size_t(a.n_tgt) : 0);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int64_t j = int64_t(blockIdx.x) * TPT * kRtThreads + int64_t(q) * kRtThreads + tid;
        if (j < a.n_tgt) {
            const double re = double(hr[q]) + double(lr[q]), im = double(hi[q]) + double(li[q]);
            if (!isfinite(re) || !isfinite(im)) atomicExch(a.status, RSI_DEV_NONFINITE);
            out[j] = make_double2(re, im);
        }
    }
}

constexpr int kTpt = 1;

size_t rt_smem(size_t tile_bytes) { return RSI_PIPE_STAGES * tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t); }

struct RtPlan {
    int S, n_tiles, tiles_per_split, splits;
    size_t tile_bytes, tiles_bytes, partial_bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int rt_plan(const rsi_raytrace& rt, int64_t n_src, int64_t n_tgt, RtPlan& p) {
    if (n_src < 1 || n_tgt < 1) return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: empty source or target set");
    if (n_src > (int64_t(1) << 31) || n_tgt > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: more than 2^31 sources or targets");
    if (!(rt.k1 > 0 && rt.k2 > 0 && rt.c1 > 0 && rt.c2 > 0 && rt.rho1 > 0 && rt.rho2 > 0) || !isfinite(rt.k1) ||
        !isfinite(rt.k2) || !isfinite(rt.z_interface) || !isfinite(rt.v0))
        return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: wavenumbers, speeds and densities must be finite and > 0");
    if (rt.newton < 0 || rt.newton > 16) return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: newton must be in [0, 16]");
    if (rt.tile) {
        p.S = rt.tile;
        if (p.S != 32 && p.S != 64 && p.S != 128 && p.S != 256)
            return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: tile must be 32, 64, 128 or 256");
    } else {  // tiles of at most 1/64 of the transducer, 32 .. 256 points
        const int64_t cap = n_src / 64;
        p.S = 256;
        while (p.S > 32 && p.S > cap) p.S >>= 1;
    }
    p.n_tiles = int((n_src + p.S - 1) / p.S);
    p.tile_bytes = RSI_TILE_HDR_BYTES + size_t(p.S) * fp32_record_bytes(RSI_STAGE_PISTON, RSI_NORMALS_Z);
    p.tiles_bytes = align256(size_t(p.n_tiles) * p.tile_bytes);
    const int64_t blocks = (n_tgt + int64_t(kRtThreads) * kTpt - 1) / (int64_t(kRtThreads) * kTpt);
    int splits = rt.splits;
    if (splits < 0) return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: splits must be >= 0");
    if (splits == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, raytrace_kernel<kTpt, 1>, kRtThreads,
                                                          rt_smem(p.tile_bytes)) != cudaSuccess ||
            occ < 1)
            occ = 1;
        const int64_t slots = int64_t(rsi_num_sms()) * occ;
        int64_t best = INT64_MAX;
        splits = 1;
        for (int s = 1; s <= 128 && s <= p.n_tiles; ++s) {
            const int64_t tps = (p.n_tiles + s - 1) / s, s_act = (p.n_tiles + tps - 1) / tps;
            const int64_t cost = ((blocks * s_act + slots - 1) / slots) * tps;
            if (cost < best) {
                best = cost;
                splits = int(s_act);
            }
        }
    }
    if (splits > p.n_tiles) splits = p.n_tiles;
    if (splits > 65535) return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: too many splits");
    p.tiles_per_split = (p.n_tiles + splits - 1) / splits;
    p.splits = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    p.partial_bytes = p.splits > 1 ? align256(size_t(p.splits) * size_t(n_tgt) * sizeof(double2)) : 0;
    return RSI_OK;
}

template <int NW>
int launch_rt(dim3 grid, size_t smem, const RtArgs& a, cudaStream_t s) {
    static RsiCtxOnce attr;
    if (attr.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(raytrace_kernel<kTpt, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          64 * 1024),
                     "cudaFuncSetAttribute(raytrace)");
        attr.done();
    }
    raytrace_kernel<kTpt, NW><<<grid, kRtThreads, smem, s>>>(a);
    RSI_CHECK_LAUNCH("raytrace_kernel");
    return RSI_OK;
}

void split_df(double v, float& h, float& l) {
    h = float(v);
    l = float(v - double(h));
}

}  // namespace

extern "C" size_t rsi_raytrace_workspace_bytes(const rsi_raytrace* rt, int64_t n_src, int64_t n_tgt) {
    if (!rt) return 0;
    RtPlan p;
    if (rt_plan(*rt, n_src, n_tgt, p) != RSI_OK) return 0;
    return p.tiles_bytes + p.partial_bytes;
}

extern "C" int rsi_raytrace_field(const rsi_raytrace* rt, const void* src_points, int64_t n_src,
                                  const void* tgt_points, int64_t n_tgt, double* tgt_field, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    if (!rt || !src_points || !tgt_points || !tgt_field || !workspace)
        return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: null argument");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 || reinterpret_cast<uintptr_t>(src_points) % 256 ||
        reinterpret_cast<uintptr_t>(tgt_points) % 256 || reinterpret_cast<uintptr_t>(tgt_field) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_raytrace_field: misaligned pointer");
    RtPlan p;
    int rc = rt_plan(*rt, n_src, n_tgt, p);
    if (rc != RSI_OK) return rc;
    if (workspace_bytes < p.tiles_bytes + p.partial_bytes)
        return rsi_fail(RSI_E_NOMEM, "rsi_raytrace_field: workspace %zu < %zu bytes", workspace_bytes,
                        p.tiles_bytes + p.partial_bytes);
    int* status = rsi_status_ptr();
    if (!status) return RSI_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PointsView src = rsi_points_view(const_cast<void*>(src_points), n_src);
    PointsView tgt = rsi_points_view(const_cast<void*>(tgt_points), n_tgt);
    uint8_t* tiles = static_cast<uint8_t*>(workspace);
    rsi_stage st = {};
    st.kind = RSI_STAGE_PISTON;
    st.precision = RSI_PREC_FP32C;
    st.k = rt->k1;
    st.v0 = rt->v0;
    rc = launch_prep_fp32(st, src, n_src, nullptr, p.S, tiles, p.tile_bytes, p.n_tiles, s, RSI_RT_PACKED != 0);
    if (rc != RSI_OK) return rc;

    RtArgs a = {};
    a.tiles = tiles;
    a.tile_bytes = p.tile_bytes;
    a.S = p.S;
    a.n_tiles = p.n_tiles;
    a.tiles_per_split = p.tiles_per_split;
    a.splits = p.splits;
    a.tgt = {tgt.xh, tgt.xl, tgt.yh, tgt.yl, tgt.zh, tgt.zl, tgt.x, tgt.y, tgt.z};
    a.n_tgt = n_tgt;
    split_df(rt->z_interface, a.zIh, a.zIl);
    split_df(rt->k1, a.k1h, a.k1l);
    split_df(rt->k2, a.k2h, a.k2l);
    a.s1 = float(1.0 / rt->c1);
    a.s2 = float(1.0 / rt->c2);
    a.c21 = float(rt->c2 / rt->c1);
    const double z1 = rt->rho1 * rt->c1;  // T12 scaled by 1 / (rho1 c1)
    a.Tn = float(2.0 * rt->rho1 * rt->c2 / z1);
    a.Td1 = float(rt->rho2 * rt->c2 / z1);
    a.Td2 = 1.0f;
    a.newton = rt->newton ? rt->newton : 1;
    a.tp = two_pi_split();
    double2* field = reinterpret_cast<double2*>(tgt_field);
    a.out = p.splits > 1 ? reinterpret_cast<double2*>(tiles + p.tiles_bytes) : field;
    a.status = status;

    TimingScope tsc = timing_begin(s);
    const int64_t per_block = int64_t(kRtThreads) * kTpt;
    dim3 grid(unsigned((n_tgt + per_block - 1) / per_block), unsigned(p.splits));
    switch (a.newton) {  // the common step counts unrolled
        case 1: rc = launch_rt<1>(grid, rt_smem(p.tile_bytes), a, s); break;
        case 2: rc = launch_rt<2>(grid, rt_smem(p.tile_bytes), a, s); break;
        case 3: rc = launch_rt<3>(grid, rt_smem(p.tile_bytes), a, s); break;
        default: rc = launch_rt<0>(grid, rt_smem(p.tile_bytes), a, s); break;
    }
    if (rc != RSI_OK) return rc;
    timing_end(tsc, RSI_TIMING_RAYTRACE, double(n_src) * double(n_tgt), s);
    if (p.splits > 1) return launch_reduce_partials(a.out, p.splits, n_tgt, field, status, s);
    return RSI_OK;
}
