// stage_fp32_body.cuh -- device code of the FP32C source x target sum (steps
// a3, a5), shared by the single-stage kernel (stage_fp32.cu) and the
// persistent multi-instance kernel (batch.cu).
//
// Every target keeps, per source tile, a reference built in double-float
// arithmetic: D = Q - c (c = tile centre), R = |D| and the phase
// tau = k R mod 2 pi.  A pair then needs only FP32 work on small offsets
// p = P - c: t = |p|^2 - 2 D.p = r^2 - R^2, and r - R follows without
// cancellation from a Newton step on r^2 = R^2 + t (or from t / (R + r)), so
// the phase tau + k (r - R) is accurate to about 2^-23 k |r - R| <= 2^-23 k
// (tile radius) instead of 2^-24 k r.
//
// Two pair paths, chosen per (warp, tile):
//   far   every target of the warp is more than two tile radii from the tile
//         centre, so r > R/2 > 0: r^2 = R^2 + t is accurate to a few ulps and
//         r - R is exact to form; no coincidence test is needed.
//   near  r^2 = |D - p|^2 from the FP32 offsets (accurate for r << R), and
//         pairs closer than 1e-12 m are dropped.
// Tiles arrive in shared memory by bulk copy (cp.async.bulk) on mbarriers,
// RSI_PIPE_STAGES deep; each thread owns TPT targets and loops over the
// tile; tile sums are FP32 and are added into a double-float accumulator.
#pragma once

#include <math.h>

#include "stage.cuh"

// Build-time tuning knobs (the defaults are the measured best).
#ifndef RSI_FP32_MIN_BLOCKS
#define RSI_FP32_MIN_BLOCKS 3  // resident CTAs per SM asked of the compiler at 2 targets/thread
#endif
#ifndef RSI_FP32_UNROLL
#define RSI_FP32_UNROLL 2  // unrolling of the loop over a tile's sources
#endif
// the packed RSI kernel (variant 3) measured best with its own settings: 3
// resident CTAs (80 registers, no spills; 1453 Gpair/s on the 2^18 x 256^2
// stage against 1400 at 2 CTAs)
#ifndef RSI_FP32_PACKED_RSI_MIN_BLOCKS
#define RSI_FP32_PACKED_RSI_MIN_BLOCKS 3
#endif
#ifndef RSI_FP32_PACKED_RSI_UNROLL
#define RSI_FP32_PACKED_RSI_UNROLL 2
#endif

namespace rsi_fp32 {

constexpr int kThreads = 256;
constexpr int kUnroll = RSI_FP32_UNROLL;
// resident CTAs asked of the compiler, and the unrolling of the packed loop
// one target per thread: 4 resident CTAs (64 registers)
#ifndef RSI_FP32_TPT1_MIN_BLOCKS
#define RSI_FP32_TPT1_MIN_BLOCKS 4
#endif
template <int KIND, int TPT, int VAR>
constexpr int min_blocks() {
    return TPT == 1   ? RSI_FP32_TPT1_MIN_BLOCKS
           : TPT != 2 ? 2
           : (KIND == RSI_STAGE_RSI && VAR == 3) ? RSI_FP32_PACKED_RSI_MIN_BLOCKS
                                                  : RSI_FP32_MIN_BLOCKS;
}
template <int KIND>
constexpr int packed_unroll() {
    return KIND == RSI_STAGE_RSI ? RSI_FP32_PACKED_RSI_UNROLL : RSI_FP32_UNROLL;
}

struct TgtRef {
    float Dx, Dy, Dz, mx, my, mz, R, R2, tau;
};

// double-float reference of one target against one tile centre
__device__ __forceinline__ TgtRef target_reference(float qxh, float qxl, float qyh, float qyl, float qzh,
                                                   float qzl, const float* c, float kh, float kl,
                                                   const TwoPiSplit& tp) {
    float dxh, dxl, dyh, dyl, dzh, dzl;
    df_diff(qxh, qxl, c[0], c[1], dxh, dxl);
    df_diff(qyh, qyl, c[2], c[3], dyh, dyl);
    df_diff(qzh, qzl, c[4], c[5], dzh, dzl);
    float ax, axl, ay, ayl, az, azl, sh, sl;
    df_sqr(dxh, dxl, ax, axl);
    df_sqr(dyh, dyl, ay, ayl);
    df_sqr(dzh, dzl, az, azl);
    df_add_pos(ax, axl, ay, ayl, sh, sl);
    df_add_pos(sh, sl, az, azl, sh, sl);
    float Rh = 0.0f, Rl = 0.0f;
    if (sh > 0.0f) {
        // one Newton step from the FP32 reciprocal square root: ~2^-44 relative
        float y = rsqrtf(sh);
        float r0 = __fmul_rn(sh, y);
        float p, pe;
        two_prod(r0, r0, p, pe);
        float e = __fadd_rn(__fsub_rn(__fsub_rn(sh, p), pe), sl);
        fast_two_sum(r0, __fmul_rn(e, __fmul_rn(0.5f, y)), Rh, Rl);
    }
    // k R as a double-float, reduced modulo 2 pi (Cody & Waite)
    float ph, pl;
    two_prod(kh, Rh, ph, pl);
    pl = __fmaf_rn(kh, Rl, __fmaf_rn(kl, Rh, pl));
    float n = rintf(__fmul_rn(ph, tp.inv));
    float x = __fmaf_rn(-n, tp.p1, ph);
    x = __fmaf_rn(-n, tp.p2, x);
    x = __fmaf_rn(-n, tp.p3, x);
    x = __fadd_rn(x, pl);
    TgtRef t;
    t.Dx = dxh;
    t.Dy = dyh;
    t.Dz = dzh;
    t.mx = -2.0f * dxh;
    t.my = -2.0f * dyh;
    t.mz = -2.0f * dzh;
    t.R = Rh;
    t.R2 = Rh * Rh;
    t.tau = x;
    return t;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// the source term once the phase u and 1/r are known
template <int KIND, int NORM>
__device__ __forceinline__ void accumulate(float u, float ir, float nd, const float4& b, float& acc_r,
                                           float& acc_i) {
    float s, c;
    __sincosf(u, &s, &c);
    if (KIND == RSI_STAGE_PISTON) {
        float amp = b.x * ir;
        acc_r = fmaf(amp, c, acc_r);
        acc_i = fmaf(amp, s, acc_i);
    } else {
        float h = nd * (ir * ir);        // cos(theta) / r
        float vr = fmaf(-ir, b.x, b.z);  // B (ik - 1/r)
        float vi = fmaf(-ir, b.y, b.w);
        float wr = fmaf(vr, c, -vi * s);
        float wi = fmaf(vr, s, vi * c);
        acc_r = fmaf(h, wr, acc_r);
        acc_i = fmaf(h, wi, acc_i);
    }
}

// near path: one source (records a, b[, n]) onto one target reference
template <int KIND, int NORM, int VAR>
__device__ __forceinline__ void pair_near(const TgtRef& t, const float4& a, const float4& b, const float4& nr,
                                          float k, float& acc_r, float& acc_i) {
    float dx = t.Dx - a.x, dy = t.Dy - a.y, dz = t.Dz - a.z;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float tt = fmaf(t.mx, a.x, fmaf(t.my, a.y, fmaf(t.mz, a.z, a.w)));  // r^2 - R^2
    float ir = rsqrt_approx(r2);
    ir = r2 > 1e-24f ? ir : 0.0f;  // pairs closer than 1e-12 m contribute nothing
    float dr;
    if (VAR == 1) {
        float r = r2 * ir;
        dr = __fdividef(tt, fmaxf(t.R + r, 1e-30f));
    } else {
        float r0 = r2 * ir;
        float am = t.R - r0;
        float e = fmaf(am, t.R + r0, tt);  // r^2 - r0^2
        dr = fmaf(e, 0.5f * ir, -am);
    }
    float nd = (NORM == RSI_NORMALS_Z) ? dz : fmaf(nr.x, dx, fmaf(nr.y, dy, nr.z * dz));
    accumulate<KIND, NORM>(fmaf(k, dr, t.tau), ir, nd, b, acc_r, acc_i);
}

// far path: R > 2 (tile radius), so r / R lies in (1/2, 3/2)
template <int KIND, int NORM, int VAR>
__device__ __forceinline__ void pair_far(const TgtRef& t, const float4& a, const float4& b, const float4& nr,
                                         float k, float& acc_r, float& acc_i) {
    float tt = fmaf(t.mx, a.x, fmaf(t.my, a.y, fmaf(t.mz, a.z, a.w)));  // r^2 - R^2
    float r2 = t.R2 + tt;
    float ir = rsqrt_approx(r2);
    float r0 = r2 * ir;
    float dr;
    if (VAR == 1) {
        dr = __fdividef(tt, t.R + r0);
    } else {
        float am = r0 - t.R;                // exact: r0 and R within a factor 2
        float e = fmaf(-am, t.R + r0, tt);  // r^2 - r0^2, accurate to 2^-24 |t|
        dr = fmaf(e, 0.5f * ir, am);
    }
    float nd;
    if (NORM == RSI_NORMALS_Z)
        nd = t.Dz - a.z;
    else
        nd = fmaf(nr.x, t.Dx, fmaf(nr.y, t.Dy, fmaf(nr.z, t.Dz, -nr.w)));  // n.D - n.p
    accumulate<KIND, NORM>(fmaf(k, dr, t.tau), ir, nd, b, acc_r, acc_i);
}

// ---------------------------------------------------------------------------
// Packed variant (3): two sources per instruction with the f32x2 arithmetic of
// sm_100-family GPUs.  Tiles are written pair-interleaved (field f of source
// 2i+L at float (2i)*rec_f + 2f + L) with signs and scales chosen so that no
// per-pair negation is needed:
//   f0 px, f1 py, f2 -pz, f3 |p|^2 / 2, then
//   PISTON f4 A, f5..f7 0
//   RSI    f4 beta, f5 m (B = m e^{i beta}, beta = arg sigma), f6 -m pz, f7 0
//          [f8..f10 m n, f11 -m n.p  for per-point normals]
// The distance update is the Newton variant with the factor 1/2 folded in
// exactly: th = t/2 = |p|^2/2 - D.p, r^2 = R^2 + 2 th, and
// r - R = (r0 - R) + (th - (r0 - R)(r0 + R)/2) / r0, the last product and sum
// one fused multiply-add.  The RSI term B (ik - 1/r) (n.(Q-P)/r^2) e^{i u}
// is taken in polar form: with g = m n.(Q-P) / r^2 (the normal carries m),
//   B (ik - 1/r) e^{iu} n.(Q-P)/r^2 = g (-1/r + ik) e^{i (k (r - R) + beta)} e^{i tau},
// so each pair adds to four accumulators (g/r cos, g sin, g/r sin, g cos) and
// the factor k and the target's reference phase e^{i tau} are applied once
// per tile.
// ---------------------------------------------------------------------------
struct TgtRef2 {
    float2 mx, my, mz, R2, nR, nRh, tau, Dx, Dy, Dz;
};
__device__ __forceinline__ TgtRef2 packed_reference(const TgtRef& t) {
    TgtRef2 r;
    r.mx = make_float2(-t.Dx, -t.Dx);  // -D.p (half of -2 D.p)
    r.my = make_float2(-t.Dy, -t.Dy);
    r.mz = make_float2(t.Dz, t.Dz);    // pz is stored negated
    r.R2 = make_float2(t.R2, t.R2);
    r.nR = make_float2(-t.R, -t.R);
    r.nRh = make_float2(-0.5f * t.R, -0.5f * t.R);
    r.tau = make_float2(t.tau, t.tau);
    r.Dx = make_float2(t.Dx, t.Dx);
    r.Dy = make_float2(t.Dy, t.Dy);
    r.Dz = make_float2(t.Dz, t.Dz);
    return r;
}

// two sources (v0 = px, py; v1 = -pz, |p|^2/2; v2, v3 amplitudes; n0, n1
// scaled normals) onto one target reference, once th = (r^2 - R^2)/2, r^2 and
// 1/r are known.  PISTON: ar1 += A/r cos, ai1 += A/r sin of k (r - R) + tau.
// RSI: the four polar accumulators of k (r - R) + beta (the caller applies k
// and e^{i tau}).
template <int KIND, int NORM>
__device__ __forceinline__ void pair_terms2(const TgtRef2& t, float2 th, float2 r2, float2 ir, const float4& v1,
                                            const float4& v2, const float4& v3, const float4& n0, const float4& n1,
                                            float2 k, float2& ar1, float2& ar2, float2& ai1, float2& ai2) {
    const float2 r0 = __fmul2_rn(r2, ir);
    const float2 am = __fadd2_rn(r0, t.nR);                              // r0 - R (exact on the far path)
    const float2 hs = __ffma2_rn(r0, make_float2(-0.5f, -0.5f), t.nRh);  // -(r0 + R)/2
    const float2 eh = __ffma2_rn(am, hs, th);                            // (r^2 - r0^2)/2
    const float2 dr = __ffma2_rn(eh, ir, am);                            // r - R
    float2 sn, cs;
    if (KIND == RSI_STAGE_PISTON) {
        const float2 u = __ffma2_rn(k, dr, t.tau);
        __sincosf(u.x, &sn.x, &cs.x);
        __sincosf(u.y, &sn.y, &cs.y);
        const float2 amp = __fmul2_rn(make_float2(v2.x, v2.y), ir);
        ar1 = __ffma2_rn(amp, cs, ar1);
        ai1 = __ffma2_rn(amp, sn, ai1);
    } else {
        const float2 u = __ffma2_rn(k, dr, make_float2(v2.x, v2.y));  // k (r - R) + beta
        __sincosf(u.x, &sn.x, &cs.x);
        __sincosf(u.y, &sn.y, &cs.y);
        float2 nd;  // m n . (Q - P)
        if (NORM == RSI_NORMALS_Z)
            nd = __ffma2_rn(make_float2(v2.z, v2.w), t.Dz, make_float2(v3.x, v3.y));
        else
            nd = __ffma2_rn(make_float2(n0.x, n0.y), t.Dx,
                            __ffma2_rn(make_float2(n0.z, n0.w), t.Dy,
                                       __ffma2_rn(make_float2(n1.x, n1.y), t.Dz, make_float2(n1.z, n1.w))));
        const float2 g = __fmul2_rn(nd, __fmul2_rn(ir, ir));  // m cos(theta) / r
        const float2 gr = __fmul2_rn(g, ir);
        ar1 = __ffma2_rn(gr, cs, ar1);
        ar2 = __ffma2_rn(g, sn, ar2);
        ai1 = __ffma2_rn(gr, sn, ai1);
        ai2 = __ffma2_rn(g, cs, ai2);
    }
}

// two sources onto one target reference.  Far path (R > 2 tile radii, so
// r / R lies in (1/2, 3/2)): r^2 = R^2 + 2 th.  Near path: r^2 from the
// offsets Q - P, and pairs closer than 1e-12 m contribute nothing.
template <int KIND, int NORM, bool NEAR>
__device__ __forceinline__ void pair2(const TgtRef2& t, const float4& v0, const float4& v1, const float4& v2,
                                      const float4& v3, const float4& n0, const float4& n1, float2 k, float2& ar1,
                                      float2& ar2, float2& ai1, float2& ai2) {
    const float2 px = make_float2(v0.x, v0.y), py = make_float2(v0.z, v0.w);
    const float2 pzn = make_float2(v1.x, v1.y), pwh = make_float2(v1.z, v1.w);
    const float2 th = __ffma2_rn(t.mx, px, __ffma2_rn(t.my, py, __ffma2_rn(t.mz, pzn, pwh)));  // (r^2 - R^2)/2
    float2 r2, ir;
    if (NEAR) {
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 dx = __ffma2_rn(px, m1, t.Dx), dy = __ffma2_rn(py, m1, t.Dy), dz = __fadd2_rn(t.Dz, pzn);
        r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        ir.x = r2.x > 1e-24f ? rsqrt_approx(r2.x) : 0.0f;
        ir.y = r2.y > 1e-24f ? rsqrt_approx(r2.y) : 0.0f;
    } else {
        r2 = __ffma2_rn(th, make_float2(2.0f, 2.0f), t.R2);
        ir.x = rsqrt_approx(r2.x);
        ir.y = rsqrt_approx(r2.y);
    }
    pair_terms2<KIND, NORM>(t, th, r2, ir, v1, v2, v3, n0, n1, k, ar1, ar2, ai1, ai2);
}

// every source pair of a staged packed tile onto the thread's TPT targets
template <int KIND, int NORM, int TPT, bool NEAR>
__device__ __forceinline__ void packed_tile(const float4* rec, int S, const TgtRef2 (&r2)[TPT], float2 k2,
                                            float2 (&a1)[TPT], float2 (&a2)[TPT], float2 (&b1)[TPT],
                                            float2 (&b2)[TPT]) {
    constexpr int rec_f4 = (KIND == RSI_STAGE_RSI && NORM == RSI_NORMALS_POINTS) ? 3 : 2;
#pragma unroll packed_unroll<KIND>()
    for (int i = 0; i < S / 2; ++i) {
        const float4* pr = rec + i * 2 * rec_f4;
        const float4 v0 = pr[0], v1 = pr[1], v2 = pr[2], v3 = pr[3];
        const float4 n0 = (rec_f4 == 3) ? pr[4] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 n1 = (rec_f4 == 3) ? pr[5] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < TPT; ++q)
            pair2<KIND, NORM, NEAR>(r2[q], v0, v1, v2, v3, n0, n1, k2, a1[q], a2[q], b1[q], b2[q]);
    }
}

// One CTA's share of a stage: targets j0 .. j0 + TPT*kThreads - 1 against
// the `ntile` staged tiles starting at `t_begin`.
struct BlockWork {
    const uint8_t* tiles;
    uint32_t tile_bytes;
    int S;
    int t_begin, ntile;
    TgtView tgt;
    int64_t n_tgt, j0;
    float kh, kl;
    TwoPiSplit tp;
    double2* out;  // out[j] for the targets of this block
    int* status;
};

// Shared memory: RSI_PIPE_STAGES tile buffers, then one mbarrier per buffer
// (initialised once per CTA).  `uses` counts buffer fills of this CTA so far
// and keeps the mbarrier phases consistent across successive calls.
// Returns false (after recording RSI_DEV_TIMEOUT) if a bounded wait expired.
template <int KIND, int NORM, int TPT, int VAR>
__device__ __forceinline__ bool run_block(const BlockWork& w, uint8_t* smem, uint64_t* bars, uint32_t& uses) {
    const int tid = threadIdx.x;
    const int rec_f4 = (KIND == RSI_STAGE_RSI && NORM == RSI_NORMALS_POINTS) ? 3 : 2;
    int64_t jt[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int64_t j = w.j0 + int64_t(q) * kThreads + tid;
        jt[q] = j < w.n_tgt ? j : w.n_tgt - 1;
    }
    if (tid == 0) {
        for (int s = 0; s < RSI_PIPE_STAGES && s < w.ntile; ++s) {
            const uint32_t b = (uses + s) % RSI_PIPE_STAGES;
            uint32_t bar = smem_u32(&bars[b]);
            mbar_expect_tx(bar, w.tile_bytes);
            bulk_g2s(smem_u32(smem + b * w.tile_bytes), w.tiles + size_t(w.t_begin + s) * w.tile_bytes,
                     w.tile_bytes, bar);
        }
    }
    float hr[TPT], lr[TPT], hi[TPT], li[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) hr[q] = lr[q] = hi[q] = li[q] = 0.0f;
    const float k = w.kh;
    int failed_at = -1;

    for (int it = 0; it < w.ntile; ++it) {
        const uint32_t u = uses + it;
        const uint32_t buf = u % RSI_PIPE_STAGES;
        bool ok = mbar_wait_bounded(smem_u32(&bars[buf]), (u / RSI_PIPE_STAGES) & 1u);
        if (__syncthreads_or(!ok)) {
            failed_at = it;
            break;
        }
        const uint8_t* tile = smem + buf * w.tile_bytes;
        const float* hdr = reinterpret_cast<const float*>(tile);
        const float4* rec = reinterpret_cast<const float4*>(tile + RSI_TILE_HDR_BYTES);
        TgtRef ref[TPT];
        float ar[TPT], ai[TPT];
        const float far_min = 2.0f * hdr[6];  // twice the tile radius
        bool far_lane = true;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t j = jt[q];
            ref[q] = target_reference(__ldg(w.tgt.xh + j), __ldg(w.tgt.xl + j), __ldg(w.tgt.yh + j),
                                      __ldg(w.tgt.yl + j), __ldg(w.tgt.zh + j), __ldg(w.tgt.zl + j), hdr, w.kh,
                                      w.kl, w.tp);
            far_lane = far_lane && ref[q].R > far_min && ref[q].R > 0.0f;
            ar[q] = 0.0f;
            ai[q] = 0.0f;
        }
        if (VAR == 3) {
            TgtRef2 r2[TPT];
            float2 a1[TPT], a2[TPT], b1[TPT], b2[TPT];
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                r2[q] = packed_reference(ref[q]);
                a1[q] = a2[q] = b1[q] = b2[q] = make_float2(0.f, 0.f);
            }
            const float2 k2 = make_float2(k, k);
            if (__all_sync(0xffffffffu, far_lane))
                packed_tile<KIND, NORM, TPT, false>(rec, w.S, r2, k2, a1, a2, b1, b2);
            else
                packed_tile<KIND, NORM, TPT, true>(rec, w.S, r2, k2, a1, a2, b1, b2);
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                if (KIND == RSI_STAGE_PISTON) {
                    ar[q] = a1[q].x + a1[q].y;
                    ai[q] = b1[q].x + b1[q].y;
                } else {
                    // (-sum g/r cos - k sum g sin) + i (-sum g/r sin + k sum g cos), times e^{i tau}
                    const float sr = fmaf(-k, a2[q].x + a2[q].y, -(a1[q].x + a1[q].y));
                    const float si = fmaf(k, b2[q].x + b2[q].y, -(b1[q].x + b1[q].y));
                    float st, ct;
                    __sincosf(ref[q].tau, &st, &ct);
                    ar[q] = fmaf(ct, sr, -st * si);
                    ai[q] = fmaf(st, sr, ct * si);
                }
            }
        } else if (__all_sync(0xffffffffu, far_lane)) {
#pragma unroll kUnroll
            for (int i = 0; i < w.S; ++i) {
                const float4 ra = rec[i * rec_f4];
                const float4 rb = rec[i * rec_f4 + 1];
                const float4 rn = (rec_f4 == 3) ? rec[i * rec_f4 + 2] : make_float4(0.f, 0.f, 1.f, 0.f);
#pragma unroll
                for (int q = 0; q < TPT; ++q) pair_far<KIND, NORM, VAR>(ref[q], ra, rb, rn, k, ar[q], ai[q]);
            }
        } else {
#pragma unroll kUnroll
            for (int i = 0; i < w.S; ++i) {
                const float4 ra = rec[i * rec_f4];
                const float4 rb = rec[i * rec_f4 + 1];
                const float4 rn = (rec_f4 == 3) ? rec[i * rec_f4 + 2] : make_float4(0.f, 0.f, 1.f, 0.f);
#pragma unroll
                for (int q = 0; q < TPT; ++q) pair_near<KIND, NORM, VAR>(ref[q], ra, rb, rn, k, ar[q], ai[q]);
            }
        }
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
        if (tid == 0 && it + RSI_PIPE_STAGES < w.ntile) {
            uint32_t bar = smem_u32(&bars[buf]);
            mbar_expect_tx(bar, w.tile_bytes);
            bulk_g2s(smem_u32(smem + buf * w.tile_bytes),
                     w.tiles + size_t(w.t_begin + it + RSI_PIPE_STAGES) * w.tile_bytes, w.tile_bytes, bar);
        }
    }

    if (failed_at >= 0) {
        if (tid == 0) {
            atomicExch(w.status, RSI_DEV_TIMEOUT);
            // let the copies still in flight land (bounded) before returning
            for (int it = failed_at; it < w.ntile && it < failed_at + RSI_PIPE_STAGES; ++it) {
                const uint32_t u = uses + it;
                mbar_wait_bounded(smem_u32(&bars[u % RSI_PIPE_STAGES]), (u / RSI_PIPE_STAGES) & 1u);
            }
        }
        return false;
    }
    uses += uint32_t(w.ntile);

#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int64_t j = w.j0 + int64_t(q) * kThreads + tid;
        if (j < w.n_tgt) {
            double re = double(hr[q]) + double(lr[q]);
            double im = double(hi[q]) + double(li[q]);
            if (!isfinite(re) || !isfinite(im)) atomicExch(w.status, RSI_DEV_NONFINITE);
            w.out[j] = make_double2(re, im);
        }
    }
    return true;
}

__device__ __forceinline__ void init_barriers(uint64_t* bars) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < RSI_PIPE_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// tile preparation: one CTA per tile, one thread per record
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_reduce(double v, bool is_max, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, w) : fmin(v, w);
    }
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = sh[0];
    for (int q = 1; q < nw; ++q) v = is_max ? fmax(v, sh[q]) : fmin(v, sh[q]);
    return v;
}

// Writes tile `tile` (header + S records) of a source set; called by every
// thread of a CTA of blockDim.x >= S threads (threads past S only take part
// in the block reductions).
__device__ __forceinline__ void prep_tile(int kind, int normals, int S, int64_t n_src, const PointsView& src,
                                          const double2* __restrict__ sigma, double amp_scale, double k,
                                          uint8_t* tiles, size_t tile_bytes, int64_t tile, double* red,
                                          bool packed = false) {
    const bool in_tile = int(threadIdx.x) < S;
    const int64_t i = tile * S + threadIdx.x;
    const bool valid = in_tile && i < n_src;
    double c[3];
    const double* coord[3] = {src.x, src.y, src.z};
    for (int d = 0; d < 3; ++d) {
        double v = valid ? coord[d][i] : 0.0;
        double lo = block_reduce(valid ? v : INFINITY, false, red);
        double hi = block_reduce(valid ? v : -INFINITY, true, red);
        c[d] = 0.5 * (lo + hi);
    }
    float ch[3], cl[3];
    for (int d = 0; d < 3; ++d) {
        ch[d] = __double2float_rn(c[d]);
        cl[d] = __double2float_rn(c[d] - double(ch[d]));
    }
    const int rec_f = (kind == RSI_STAGE_RSI && normals == RSI_NORMALS_POINTS) ? 12 : 8;
    float* rec = reinterpret_cast<float*>(tiles + size_t(tile) * tile_bytes + RSI_TILE_HDR_BYTES) +
                 (packed ? size_t(threadIdx.x >> 1) * 2 * rec_f + (threadIdx.x & 1) : size_t(threadIdx.x) * rec_f);
    const int fs = packed ? 2 : 1;  // stride between the fields of one source
    // padding records (past the last source of the last tile) carry a zero
    // amplitude and sit metres from the tile centre, so that no target comes
    // near them; they sit behind the transducer (-z), so that the ray-tracing
    // kernel, which reads the piston's tiles, solves a proper crossing for
    // them too and every padding term is a finite value times zero
    float px = 4.0f, py = 4.0f, pz = -4.0f, radius2 = 0.0f;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
    float nx = 0.f, ny = 0.f, nz = 1.f;
    float beta = 0.f, mag = 0.f;  // packed RSI records: B = mag e^{i beta}
    if (valid) {
        float h, l;
        df_diff(src.xh[i], src.xl[i], ch[0], cl[0], h, l);
        px = h;
        df_diff(src.yh[i], src.yl[i], ch[1], cl[1], h, l);
        py = h;
        df_diff(src.zh[i], src.zl[i], ch[2], cl[2], h, l);
        pz = h;
        radius2 = px * px + py * py + pz * pz;
        if (kind == RSI_STAGE_PISTON) {
            r0 = float(amp_scale * src.w[i]);
        } else {
            double2 sg = sigma[i];
            double br = amp_scale * src.w[i] * sg.x, bi = amp_scale * src.w[i] * sg.y;
            r0 = float(br);
            r1 = float(bi);
            r2 = float(-k * bi);
            r3 = float(k * br);
            // B = mag e^{i beta} with beta = arg sigma and the signs of the
            // amplitude scale and the weight in mag, so that reversed normals
            // (a negated scale) negate every term exactly
            beta = float(atan2(sg.y, sg.x));
            mag = float(amp_scale * src.w[i] * hypot(sg.x, sg.y));
            nx = float(src.nx[i]);
            ny = float(src.ny[i]);
            nz = float(src.nz[i]);
        }
    }
    if (in_tile && !packed) {
        rec[0] = px;
        rec[1] = py;
        rec[2] = pz;
        rec[3] = fmaf(px, px, fmaf(py, py, pz * pz));
        rec[4] = r0;
        rec[5] = r1;
        rec[6] = r2;
        rec[7] = r3;
        if (rec_f == 12) {
            rec[8] = nx;
            rec[9] = ny;
            rec[10] = nz;
            rec[11] = fmaf(nx, px, fmaf(ny, py, nz * pz));  // n . p
        }
    } else if (in_tile) {  // packed: signs and the 1/2 of the packed far path
        const bool rsi = kind == RSI_STAGE_RSI;
        rec[0 * fs] = px;
        rec[1 * fs] = py;
        rec[2 * fs] = -pz;
        rec[3 * fs] = 0.5f * fmaf(px, px, fmaf(py, py, pz * pz));
        rec[4 * fs] = rsi ? beta : r0;
        rec[5 * fs] = rsi ? mag : 0.0f;
        rec[6 * fs] = rsi ? -mag * pz : 0.0f;
        rec[7 * fs] = 0.0f;
        if (rec_f == 12) {
            rec[8 * fs] = mag * nx;
            rec[9 * fs] = mag * ny;
            rec[10 * fs] = mag * nz;
            rec[11 * fs] = -mag * fmaf(nx, px, fmaf(ny, py, nz * pz));  // -m n . p
        }
    }
    double rad = block_reduce(double(radius2), true, red);
    if (threadIdx.x == 0) {
        float* hdr = reinterpret_cast<float*>(tiles + size_t(tile) * tile_bytes);
        hdr[0] = ch[0];
        hdr[1] = cl[0];
        hdr[2] = ch[1];
        hdr[3] = cl[1];
        hdr[4] = ch[2];
        hdr[5] = cl[2];
        hdr[6] = sqrtf(float(rad));
        hdr[7] = 0.0f;
    }
}

}  // namespace rsi_fp32
