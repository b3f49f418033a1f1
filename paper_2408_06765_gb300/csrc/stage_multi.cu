// stage_multi.cu -- rsi_propagate_stage_multi: the FP32C stage sum (steps a3,
// a5, a6) for nf frequencies at once on the same point sets.  A broadband
// field is the superposition of single-frequency fields (Sec. 4), and the
// frequencies of one transducer and one interface share every point, so per
// pair the geometry -- r - R (Newton update), 1/r and the obliquity -- is
// formed once; each frequency adds only its phase k_f (r - R) + tau_f, its
// sincos and its source amplitude.  MUFU work per pair-term falls from 3 to
// 2 + 1/nf.  Each frequency's arithmetic is that of the single-frequency
// kernel (stage_fp32_body.cuh), so the results agree with nf separate stages
// to rounding.
#include <math.h>

#include "stage_fp32_body.cuh"

namespace {

using namespace rsi_fp32;

constexpr int kMaxNF = 4;
constexpr int kMTpt = 2;
// resident CTAs per SM asked of the compiler for the packed form (one target
// per thread): 4 measured best on the 3-frequency RSI stage (1910 Gpair-terms/s
// at 64 registers; 3 CTAs 1890, 2 CTAs 1782); four frequencies keep 3 CTAs
// (at the 64-register cap of 4 CTAs their accumulators spill)
#ifndef RSI_MULTI_PACKED_MIN_BLOCKS
#define RSI_MULTI_PACKED_MIN_BLOCKS 4
#endif

struct MultiArgs {
    int kind, normals, nf, packed, S, n_tiles, tiles_per_split, splits;
    int64_t n_tgt;
    size_t tile_bytes;
    const uint8_t* tiles;
    TgtView tgt;
    float kh[kMaxNF], kl[kMaxNF];
    TwoPiSplit tp;
    double2* out;    // [splits][nf][n_tgt] partial sums, or the fields [nf][n_tgt]
    double2* field;  // the fields [nf][n_tgt] (the last split of a target block sums into it)
    unsigned* done;  // per target block: splits finished (zeroed before the launch)
    int* status;
    // frequency f of the kernel is the caller's frequency perm[f]; with harm,
    // k_{nf-1} = 2 k_0 and the far path takes frequency nf-1 from frequency 0
    // (double angle) instead of its own sincos
    int perm[kMaxNF];
    int harm;
};

// Tile records (float4 units): [p.x, p.y, p.z, |p|^2], then
//   PISTON  [A, 0, 0, 0]                   (A = -v0 w / 2 pi, frequency independent)
//   RSI     nf x [B.re, B.im, C.re, C.im]  (B = -w sigma_f / 2 pi, C = i k_f B)
//           [+ (nx, ny, nz, n.p)]
// The packed form keeps each RSI amplitude in polar form, nf x [beta_f, m_f]
// padded to whole float4s (see MRef2).
template <int KIND, int NORM, int NF, int PK>
constexpr int mrec_f4() {
    return KIND == RSI_STAGE_PISTON ? 2 : 1 + (PK ? (NF + 1) / 2 : NF) + (NORM == RSI_NORMALS_POINTS ? 1 : 0);
}
__host__ __device__ inline int mrec_f4_rt(int kind, int normals, int nf, bool packed) {
    return kind == RSI_STAGE_PISTON ? 2 : 1 + (packed ? (nf + 1) / 2 : nf) + (normals == RSI_NORMALS_POINTS ? 1 : 0);
}

struct MRef {
    float Dx, Dy, Dz, mx, my, mz, R, R2;
    float tau[kMaxNF];
};

// double-float reference of one target against one tile centre: D, R and the
// phase k_f R mod 2 pi of every frequency
template <int NF>
__device__ __forceinline__ MRef multi_reference(float qxh, float qxl, float qyh, float qyl, float qzh, float qzl,
                                                const float* c, const MultiArgs& a) {
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
        float y = rsqrtf(sh);
        float r0 = __fmul_rn(sh, y);
        float p, pe;
        two_prod(r0, r0, p, pe);
        float e = __fadd_rn(__fsub_rn(__fsub_rn(sh, p), pe), sl);
        fast_two_sum(r0, __fmul_rn(e, __fmul_rn(0.5f, y)), Rh, Rl);
    }
    MRef t;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        float ph, pl;
        two_prod(a.kh[f], Rh, ph, pl);
        pl = __fmaf_rn(a.kh[f], Rl, __fmaf_rn(a.kl[f], Rh, pl));
        float n = rintf(__fmul_rn(ph, a.tp.inv));
        float x = __fmaf_rn(-n, a.tp.p1, ph);
        x = __fmaf_rn(-n, a.tp.p2, x);
        x = __fmaf_rn(-n, a.tp.p3, x);
        t.tau[f] = __fadd_rn(x, pl);
    }
    t.Dx = dxh;
    t.Dy = dyh;
    t.Dz = dzh;
    t.mx = -2.0f * dxh;
    t.my = -2.0f * dyh;
    t.mz = -2.0f * dzh;
    t.R = Rh;
    t.R2 = Rh * Rh;
    return t;
}

// the terms of one pair for every frequency once r - R, 1/r and the obliquity are known
template <int KIND, int NORM, int NF>
__device__ __forceinline__ void mterms(const MRef& t, const float4* r, float dr, float ir, float nd, const float* kv,
                                       float (&ar)[NF], float (&ai)[NF]) {
    if (KIND == RSI_STAGE_PISTON) {
        const float amp = r[1].x * ir;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float s, c;
            __sincosf(fmaf(kv[f], dr, t.tau[f]), &s, &c);
            ar[f] = fmaf(amp, c, ar[f]);
            ai[f] = fmaf(amp, s, ai[f]);
        }
    } else {
        const float h = nd * (ir * ir);  // cos(theta) / r
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float4 b = r[1 + f];
            float s, c;
            __sincosf(fmaf(kv[f], dr, t.tau[f]), &s, &c);
            const float vr = fmaf(-ir, b.x, b.z), vi = fmaf(-ir, b.y, b.w);  // B (ik - 1/r)
            ar[f] = fmaf(h, fmaf(vr, c, -vi * s), ar[f]);
            ai[f] = fmaf(h, fmaf(vr, s, vi * c), ai[f]);
        }
    }
}

// the same with the packed form's polar amplitudes r[1 + f] = (beta_f, m_f, 0, 0)
template <int KIND, int NORM, int NF>
__device__ __forceinline__ void mterms_polar(const MRef& t, const float4* r, float dr, float ir, float nd,
                                             const float* kv, float (&ar)[NF], float (&ai)[NF]) {
    if (KIND == RSI_STAGE_PISTON) {
        mterms<KIND, NORM, NF>(t, r, dr, ir, nd, kv, ar, ai);
    } else {
        const float h = nd * (ir * ir);  // cos(theta) / r
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float4 b = r[1 + f];
            float s, c;
            __sincosf(fmaf(kv[f], dr, t.tau[f] + b.x), &s, &c);  // tau + beta first: |tau + beta| <= 2 pi
            const float g = h * b.y;
            ar[f] = fmaf(-g, fmaf(ir, c, kv[f] * s), ar[f]);  // g (-c/r - k s)
            ai[f] = fmaf(g, fmaf(-ir, s, kv[f] * c), ai[f]);  // g (-s/r + k c)
        }
    }
}

// far path: R > 2 (tile radius)
template <int KIND, int NORM, int NF>
__device__ __forceinline__ void mpair_far(const MRef& t, const float4* r, const float* kv, float (&ar)[NF],
                                          float (&ai)[NF]) {
    const float4 a = r[0];
    const float tt = fmaf(t.mx, a.x, fmaf(t.my, a.y, fmaf(t.mz, a.z, a.w)));  // r^2 - R^2
    const float r2 = t.R2 + tt;
    const float ir = rsqrt_approx(r2);
    const float r0 = r2 * ir;
    const float am = r0 - t.R;
    const float e = fmaf(-am, t.R + r0, tt);
    const float dr = fmaf(e, 0.5f * ir, am);
    float nd = 0.0f;
    if (KIND == RSI_STAGE_RSI) {
        if (NORM == RSI_NORMALS_Z) {
            nd = t.Dz - a.z;
        } else {
            const float4 n = r[1 + NF];
            nd = fmaf(n.x, t.Dx, fmaf(n.y, t.Dy, fmaf(n.z, t.Dz, -n.w)));
        }
    }
    mterms<KIND, NORM, NF>(t, r, dr, ir, nd, kv, ar, ai);
}

// near path: r^2 from the FP32 offsets; pairs closer than 1e-12 m contribute
// nothing.  PK: records unpacked from the packed form (polar amplitudes).
template <int KIND, int NORM, int NF, int PK>
__device__ __forceinline__ void mpair_near(const MRef& t, const float4* r, const float* kv, float (&ar)[NF],
                                           float (&ai)[NF]) {
    const float4 a = r[0];
    const float dx = t.Dx - a.x, dy = t.Dy - a.y, dz = t.Dz - a.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float tt = fmaf(t.mx, a.x, fmaf(t.my, a.y, fmaf(t.mz, a.z, a.w)));
    float ir = rsqrt_approx(r2);
    ir = r2 > 1e-24f ? ir : 0.0f;
    const float r0 = r2 * ir;
    const float am = t.R - r0;
    const float e = fmaf(am, t.R + r0, tt);
    const float dr = fmaf(e, 0.5f * ir, -am);
    float nd = 0.0f;
    if (KIND == RSI_STAGE_RSI) {
        if (NORM == RSI_NORMALS_Z) {
            nd = dz;
        } else {
            const float4 n = r[1 + NF];
            nd = fmaf(n.x, dx, fmaf(n.y, dy, n.z * dz));
        }
    }
    if (PK)
        mterms_polar<KIND, NORM, NF>(t, r, dr, ir, nd, kv, ar, ai);
    else
        mterms<KIND, NORM, NF>(t, r, dr, ir, nd, kv, ar, ai);
}

// ---------------------------------------------------------------------------
// Packed form: two sources per f32x2 instruction, records pair-interleaved
// with the signs and the factor 1/2 of the single-frequency packed kernel
// (field f of source 2i+L at float (2i) rf + 2f + L):
//   [px, py, -pz, |p|^2/2], then RSI nf x [beta_f, m_f] (B_f = m_f e^{i beta_f})
//   (padded to a whole float4) or PISTON [A, 0, 0, 0], then [nx, ny, nz,
//   -n.p] for per-point normals.
// With h = n.(Q-P)/r^2 formed once per pair, frequency f adds
//   B_f (ik_f - 1/r) h e^{i u_f} = m_f h (-1/r + ik_f) e^{i (k_f (r - R) + beta_f)} e^{i tau_f}
// to four accumulators (m_f h/r cos, m_f h sin, m_f h/r sin, m_f h cos); the
// factor k_f and e^{i tau_f} are applied once per tile.
// ---------------------------------------------------------------------------
struct MRef2 {
    float2 mx, my, mz, R2, nR, nRh, Dx, Dy, Dz;
    float2 tau[kMaxNF];
};
template <int NF>
__device__ __forceinline__ MRef2 packed_mref(const MRef& t) {
    MRef2 r;
    r.mx = make_float2(-t.Dx, -t.Dx);
    r.my = make_float2(-t.Dy, -t.Dy);
    r.mz = make_float2(t.Dz, t.Dz);
    r.R2 = make_float2(t.R2, t.R2);
    r.nR = make_float2(-t.R, -t.R);
    r.nRh = make_float2(-0.5f * t.R, -0.5f * t.R);
    r.Dx = make_float2(t.Dx, t.Dx);
    r.Dy = make_float2(t.Dy, t.Dy);
    r.Dz = make_float2(t.Dz, t.Dz);
#pragma unroll
    for (int f = 0; f < NF; ++f) r.tau[f] = make_float2(t.tau[f], t.tau[f]);
    return r;
}

// Harmonic sharing (HM, three frequencies with k_2 = 2 k_0): with
// E_0 = e^{i u_0} from frequency 0's sincos, e^{2 i u_0} = (c - s)(c + s) + i 2 s c
// by the double angle (that form keeps the modulus |E_0|^2 at every angle;
// 2 c^2 - 1 would turn the sincos's modulus error into an angle-dependent one,
// 1.4e-5 on the coherent piston sum of the 5 and 10 MHz workload), and
//   piston  u_2 = k_2 (r - R) + tau_2 = 2 u_0 + (tau_2 - 2 tau_0): the sums of
//           A e^{2 i u_0} / r are turned by e^{i (tau_2 - 2 tau_0)} once per tile;
//   RSI     m_2 e^{i u_2} = c_2 e^{2 i u_0} with the per-source constant
//           c_2 = m_2 e^{i (beta_2 - 2 beta_0)}, kept in the record's padding
//           float4 (the near path still reads beta_2, m_2).
// That replaces two MUFU operations per pair by a few FP32 ones.  The doubled
// angle carries twice the sincos's angle error of u_0: on the 2.25, 5 and
// 10 MHz workload the 10 MHz image is 1.0e-6 from the FP64 oracle (5.5e-7
// with its own sincos).
//
// two sources (records pr[0..RF4*2-1], packed) onto one target, far path;
// acc[f] = (sum m h/r c, sum m h s, sum m h/r s, sum m h c) of k_f (r - R) +
// beta_f for RSI, or (sum A c / r, -, sum A s / r, -) of k_f (r - R) + tau_f
// for the piston (2 u_0 for the shared frequency)
template <int KIND, int NORM, int NF, int HM>
__device__ __forceinline__ void mpair_far2(const MRef2& t, const float4* pr, const float2* kv,
                                           float2 (&acc)[NF][4]) {
    const float4 v0 = pr[0], v1 = pr[1];
    const float2 px = make_float2(v0.x, v0.y), py = make_float2(v0.z, v0.w);
    const float2 pzn = make_float2(v1.x, v1.y), pwh = make_float2(v1.z, v1.w);
    const float2 th = __ffma2_rn(t.mx, px, __ffma2_rn(t.my, py, __ffma2_rn(t.mz, pzn, pwh)));
    const float2 r2 = __ffma2_rn(th, make_float2(2.0f, 2.0f), t.R2);
    float2 ir;
    ir.x = rsqrt_approx(r2.x);
    ir.y = rsqrt_approx(r2.y);
    const float2 r0 = __fmul2_rn(r2, ir);
    const float2 am = __fadd2_rn(r0, t.nR);                              // r0 - R, exact
    const float2 hs = __ffma2_rn(r0, make_float2(-0.5f, -0.5f), t.nRh);  // -(r0 + R)/2
    const float2 eh = __ffma2_rn(am, hs, th);                            // (r^2 - r0^2)/2
    const float2 dr = __ffma2_rn(eh, ir, am);
    float2 sn0, cs0;  // e^{i u_0}, kept for the shared frequency
    if (KIND == RSI_STAGE_PISTON) {
        const float4 va = pr[2];
        const float2 amp = __fmul2_rn(make_float2(va.x, va.y), ir);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float2 sn, cs;
            if (HM && f == NF - 1) {
                // e^{2 i u_0} = (c - s)(c + s) + i 2 s c
                const float2 c2 = __fadd2_rn(cs0, cs0);
                cs = __fmul2_rn(__ffma2_rn(sn0, make_float2(-1.0f, -1.0f), cs0), __fadd2_rn(cs0, sn0));
                sn = __fmul2_rn(sn0, c2);
            } else {
                const float2 u = __ffma2_rn(kv[f], dr, t.tau[f]);
                __sincosf(u.x, &sn.x, &cs.x);
                __sincosf(u.y, &sn.y, &cs.y);
                if (f == 0) sn0 = sn, cs0 = cs;
            }
            acc[f][0] = __ffma2_rn(amp, cs, acc[f][0]);
            acc[f][2] = __ffma2_rn(amp, sn, acc[f][2]);
        }
    } else {
        float2 nd;
        if (NORM == RSI_NORMALS_Z) {
            nd = __fadd2_rn(t.Dz, pzn);
        } else {
            constexpr int nb = 2 + 2 * ((NF + 1) / 2);  // first normal float4 of the pair
            const float4 n0 = pr[nb], n1 = pr[nb + 1];
            nd = __ffma2_rn(make_float2(n0.x, n0.y), t.Dx,
                            __ffma2_rn(make_float2(n0.z, n0.w), t.Dy,
                                       __ffma2_rn(make_float2(n1.x, n1.y), t.Dz, make_float2(n1.z, n1.w))));
        }
        const float2 h = __fmul2_rn(nd, __fmul2_rn(ir, ir));  // cos(theta) / r
        const float2 hr = __fmul2_rn(h, ir);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (HM && f == NF - 1) {
                // (er, ei) = c_2 e^{2 i u_0}, c_2 = (cr, ci) from the padding float4
                const float4 cc = pr[2 + NF];
                const float2 cr = make_float2(cc.x, cc.y), ci = make_float2(cc.z, cc.w);
                const float2 c2 = __fadd2_rn(cs0, cs0);
                // cos 2 u_0 = (c - s)(c + s): modulus |E_0|^2 whatever the angle
                const float2 cq = __fmul2_rn(__ffma2_rn(sn0, make_float2(-1.0f, -1.0f), cs0), __fadd2_rn(cs0, sn0));
                const float2 sq = __fmul2_rn(sn0, c2);                                      // sin 2 u_0
                const float2 nsq = __fmul2_rn(sq, make_float2(-1.0f, -1.0f));  // -sin 2 u_0, exact
                const float2 er = __ffma2_rn(cr, cq, __fmul2_rn(ci, nsq));
                const float2 ei = __ffma2_rn(cr, sq, __fmul2_rn(ci, cq));
                acc[f][0] = __ffma2_rn(hr, er, acc[f][0]);
                acc[f][1] = __ffma2_rn(h, ei, acc[f][1]);
                acc[f][2] = __ffma2_rn(hr, ei, acc[f][2]);
                acc[f][3] = __ffma2_rn(h, er, acc[f][3]);
                continue;
            }
            const float4 b = pr[2 + f];  // (beta_f, m_f) of both sources
            const float2 u = __ffma2_rn(kv[f], dr, make_float2(b.x, b.y));
            float2 sn, cs;
            __sincosf(u.x, &sn.x, &cs.x);
            __sincosf(u.y, &sn.y, &cs.y);
            if (f == 0) sn0 = sn, cs0 = cs;
            const float2 m = make_float2(b.z, b.w);
            const float2 g = __fmul2_rn(h, m), gr = __fmul2_rn(hr, m);
            acc[f][0] = __ffma2_rn(gr, cs, acc[f][0]);
            acc[f][1] = __ffma2_rn(g, sn, acc[f][1]);
            acc[f][2] = __ffma2_rn(gr, sn, acc[f][2]);
            acc[f][3] = __ffma2_rn(g, cs, acc[f][3]);
        }
    }
}

// one source of a packed tile, unpacked into the scalar record format
// (r[0 .. mrec_f4<KIND, NORM, NF, 0>() - 1], amplitudes in polar form)
template <int KIND, int NORM, int NF>
__device__ __forceinline__ void munpack(const float* tile_rec, int i, float4* r) {
    constexpr int rf = 4 * mrec_f4<KIND, NORM, NF, 1>();
    const float* q = tile_rec + (i >> 1) * 2 * rf + (i & 1);
    r[0] = make_float4(q[0], q[2], -q[4], 2.0f * q[6]);
    if (KIND == RSI_STAGE_PISTON) {
        r[1] = make_float4(q[8], 0.f, 0.f, 0.f);
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float* b = q + 8 + 4 * f;  // fields 4 + 2f (beta_f), 5 + 2f (m_f)
            r[1 + f] = make_float4(b[0], b[2], 0.f, 0.f);
        }
        if (NORM == RSI_NORMALS_POINTS) {
            const float* n = q + 2 * (4 + 4 * ((NF + 1) / 2));
            r[1 + NF] = make_float4(n[0], n[2], n[4], -n[6]);
        }
    }
}

// the shared-harmonic form keeps 4 (64 registers, 8 bytes spilled outside the
// pair loop): 2110 Gpair-terms/s on the three-frequency RSI stage, 3 CTAs
// (77 registers, no spill) 2051
#ifndef RSI_MULTI_HARM_MIN_BLOCKS
#define RSI_MULTI_HARM_MIN_BLOCKS RSI_MULTI_PACKED_MIN_BLOCKS
#endif
template <int KIND, int NORM, int NF, int PK, int HM>
__global__ void __launch_bounds__(kThreads, PK ? (NF >= 4 ? 3 : HM ? RSI_MULTI_HARM_MIN_BLOCKS : RSI_MULTI_PACKED_MIN_BLOCKS) : 2)
    stage_multi_kernel(MultiArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * a.tile_bytes);
    init_barriers(bars);
    constexpr int RF4 = mrec_f4<KIND, NORM, NF, PK>();  // float4 per record in the tiles
    constexpr int URF4 = mrec_f4<KIND, NORM, NF, 0>();  // float4 per record in the scalar format
    constexpr int TPT = PK ? 1 : kMTpt;
    const int tid = threadIdx.x;
    // one-dimensional grid, the splits of a target block adjacent: they run
    // at about the same time, so their partial sums are still in L2 when the
    // last of them adds them up
    const int split = int(blockIdx.x % unsigned(a.splits));
    const int64_t tblock = int64_t(blockIdx.x / unsigned(a.splits));
    const int t_begin = split * a.tiles_per_split;
    const int ntile = max(0, min(a.n_tiles, t_begin + a.tiles_per_split) - t_begin);
    const uint32_t tb = uint32_t(a.tile_bytes);
    int64_t jt[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int64_t j = tblock * TPT * kThreads + int64_t(q) * kThreads + tid;
        jt[q] = j < a.n_tgt ? j : a.n_tgt - 1;
    }
    if (tid == 0)
        for (int s = 0; s < RSI_PIPE_STAGES && s < ntile; ++s) {
            const uint32_t bar = smem_u32(&bars[s]);
            mbar_expect_tx(bar, tb);
            bulk_g2s(smem_u32(smem + s * tb), a.tiles + size_t(t_begin + s) * tb, tb, bar);
        }
    float kv[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) kv[f] = a.kh[f];
    float hr[TPT][NF], lr[TPT][NF], hi[TPT][NF], li[TPT][NF];
#pragma unroll
    for (int q = 0; q < TPT; ++q)
#pragma unroll
        for (int f = 0; f < NF; ++f) hr[q][f] = lr[q][f] = hi[q][f] = li[q][f] = 0.0f;
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
        MRef ref[TPT];
        float ar[TPT][NF], ai[TPT][NF];
        const float far_min = 2.0f * hdr[6];
        bool far_lane = true;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t j = jt[q];
            ref[q] = multi_reference<NF>(__ldg(a.tgt.xh + j), __ldg(a.tgt.xl + j), __ldg(a.tgt.yh + j),
                                         __ldg(a.tgt.yl + j), __ldg(a.tgt.zh + j), __ldg(a.tgt.zl + j), hdr, a);
            far_lane = far_lane && ref[q].R > far_min && ref[q].R > 0.0f;
#pragma unroll
            for (int f = 0; f < NF; ++f) ar[q][f] = ai[q][f] = 0.0f;
        }
        if (PK && __all_sync(0xffffffffu, far_lane)) {
            float2 k2[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) k2[f] = make_float2(kv[f], kv[f]);
#pragma unroll
            for (int q = 0; q < TPT; ++q) {
                const MRef2 r2 = packed_mref<NF>(ref[q]);
                float2 acc[NF][4];
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int i = 0; i < a.S / 2; ++i) {
                    float4 pr[2 * RF4];
#pragma unroll
                    for (int m = 0; m < 2 * RF4; ++m) pr[m] = rec[i * 2 * RF4 + m];
                    mpair_far2<KIND, NORM, NF, HM>(r2, pr, k2, acc);
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (KIND == RSI_STAGE_PISTON) {
                        ar[q][f] = acc[f][0].x + acc[f][0].y;
                        ai[q][f] = acc[f][2].x + acc[f][2].y;
                        if (HM && f == NF - 1) {  // e^{2 i u_0} -> e^{i u_2}: turn by tau_2 - 2 tau_0
                            float st, ct;
                            __sincosf(fmaf(-2.0f, ref[q].tau[0], ref[q].tau[f]), &st, &ct);
                            const float xr = ar[q][f], xi = ai[q][f];
                            ar[q][f] = fmaf(ct, xr, -st * xi);
                            ai[q][f] = fmaf(st, xr, ct * xi);
                        }
                    } else {
                        // (-sum m h/r c - k sum m h s) + i (-sum m h/r s + k sum m h c), times e^{i tau}
                        const float sr = fmaf(-kv[f], acc[f][1].x + acc[f][1].y, -(acc[f][0].x + acc[f][0].y));
                        const float si = fmaf(kv[f], acc[f][3].x + acc[f][3].y, -(acc[f][2].x + acc[f][2].y));
                        float st, ct;
                        __sincosf(ref[q].tau[f], &st, &ct);
                        ar[q][f] = fmaf(ct, sr, -st * si);
                        ai[q][f] = fmaf(st, sr, ct * si);
                    }
                }
            }
        } else if (PK) {
            const float* tf = reinterpret_cast<const float*>(rec);
#pragma unroll 1
            for (int i = 0; i < a.S; ++i) {
                float4 r[URF4];  // unpacked: 1 + NF (+ 1) float4, polar amplitudes
                munpack<KIND, NORM, NF>(tf, i, r);
#pragma unroll
                for (int q = 0; q < TPT; ++q) mpair_near<KIND, NORM, NF, PK>(ref[q], r, kv, ar[q], ai[q]);
            }
        } else if (__all_sync(0xffffffffu, far_lane)) {
#pragma unroll 1
            for (int i = 0; i < a.S; ++i) {  // scalar records (PK = 0 only)
                float4 r[URF4];
#pragma unroll
                for (int m = 0; m < URF4; ++m) r[m] = rec[i * URF4 + m];
#pragma unroll
                for (int q = 0; q < TPT; ++q) mpair_far<KIND, NORM, NF>(ref[q], r, kv, ar[q], ai[q]);
            }
        } else {
#pragma unroll 1
            for (int i = 0; i < a.S; ++i) {
                float4 r[URF4];
#pragma unroll
                for (int m = 0; m < URF4; ++m) r[m] = rec[i * URF4 + m];
#pragma unroll
                for (int q = 0; q < TPT; ++q) mpair_near<KIND, NORM, NF, 0>(ref[q], r, kv, ar[q], ai[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q)
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                float s, e;
                two_sum(hr[q][f], ar[q][f], s, e);
                hr[q][f] = s;
                lr[q][f] = __fadd_rn(lr[q][f], e);
                two_sum(hi[q][f], ai[q][f], s, e);
                hi[q][f] = s;
                li[q][f] = __fadd_rn(li[q][f], e);
            }
        __syncthreads();
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
    double2* out = a.out + (a.splits > 1 ? size_t(split) * size_t(NF) * size_t(a.n_tgt) : 0);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int64_t j = tblock * TPT * kThreads + int64_t(q) * kThreads + tid;
        if (j < a.n_tgt)
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const double re = double(hr[q][f]) + double(lr[q][f]);
                const double im = double(hi[q][f]) + double(li[q][f]);
                if (a.splits == 1 && (!isfinite(re) || !isfinite(im))) atomicExch(a.status, RSI_DEV_NONFINITE);
                const int fo = a.splits == 1 ? a.perm[f] : f;  // partial sums stay in kernel order
                out[size_t(fo) * size_t(a.n_tgt) + size_t(j)] = make_double2(re, im);
            }
    }
    if (a.splits == 1) return;
    // The last split of this target block to finish adds the partial sums of
    // all splits in split order (Neumaier, FP64: the arithmetic of
    // reduce_partials_kernel), then drops their lines from L2 unwritten.  No
    // CTA waits for another: whichever finishes last does the sum.
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.done + tblock, 1u) == unsigned(a.splits - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int64_t j = tblock * TPT * kThreads + int64_t(q) * kThreads + tid;
        if (j >= a.n_tgt) continue;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
            for (int sp = 0; sp < a.splits; ++sp) {
                const double2 v = __ldcg(a.out + (size_t(sp) * NF + f) * size_t(a.n_tgt) + size_t(j));
                double t = sr + v.x;
                cr += (fabs(sr) >= fabs(v.x)) ? (sr - t) + v.x : (v.x - t) + sr;
                sr = t;
                t = si + v.y;
                ci += (fabs(si) >= fabs(v.y)) ? (si - t) + v.y : (v.y - t) + si;
                si = t;
            }
            const double re = sr + cr, im = si + ci;
            if (!isfinite(re) || !isfinite(im)) atomicExch(a.status, RSI_DEV_NONFINITE);
            a.field[size_t(a.perm[f]) * size_t(a.n_tgt) + size_t(j)] = make_double2(re, im);
        }
    }
    __syncthreads();
    // every split's partial sums of this block are read: discard their L2
    // lines (128 bytes = 8 targets) so that they are never written back
    const int64_t j0 = tblock * TPT * kThreads;
    const int64_t nj = min(int64_t(TPT * kThreads), a.n_tgt - j0);
    if ((j0 * int64_t(sizeof(double2))) % 128 == 0) {
        const int lines_f = int(nj / 8);  // whole lines of one (split, frequency) row
        for (int e = tid; e < a.splits * NF * lines_f; e += kThreads) {
            const int row = e / lines_f, ln = e - row * lines_f;
            const double2* ptr = a.out + size_t(row) * size_t(a.n_tgt) + size_t(j0) + size_t(ln) * 8;
            if ((reinterpret_cast<uintptr_t>(ptr) & 127) == 0)
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(ptr) : "memory");
        }
    }
}

// one CTA per tile: the geometry of stage_fp32_body.cuh's prep_tile, and one
// amplitude block per frequency
__global__ void mprep_kernel(int kind, int normals, int nf, int64_t n_src, PointsView src,
                             const double2* __restrict__ sigma, double amp_scale, MultiArgs a, uint8_t* tiles,
                             size_t tile_bytes) {
    __shared__ double red[32];
    const int S = blockDim.x;
    const int64_t tile = blockIdx.x;
    const int64_t i = tile * S + threadIdx.x;
    const bool valid = i < n_src;
    double c[3];
    const double* coord[3] = {src.x, src.y, src.z};
    for (int d = 0; d < 3; ++d) {
        const double v = valid ? coord[d][i] : 0.0;
        const double lo = block_reduce(valid ? v : INFINITY, false, red);
        const double hi = block_reduce(valid ? v : -INFINITY, true, red);
        c[d] = 0.5 * (lo + hi);
    }
    float ch[3], cl[3];
    for (int d = 0; d < 3; ++d) {
        ch[d] = __double2float_rn(c[d]);
        cl[d] = __double2float_rn(c[d] - double(ch[d]));
    }
    const int rf = 4 * mrec_f4_rt(kind, normals, nf, a.packed != 0);
    // field fi of this source: rec[fi * fs] (packed: pair-interleaved, see MRef2)
    const bool pk = a.packed != 0;
    const int fs = pk ? 2 : 1;
    float* rec = reinterpret_cast<float*>(tiles + size_t(tile) * tile_bytes + RSI_TILE_HDR_BYTES) +
                 (pk ? size_t(threadIdx.x >> 1) * 2 * rf + (threadIdx.x & 1) : size_t(threadIdx.x) * rf);
    float px = 4.0f, py = 4.0f, pz = 4.0f;
    if (valid) {
        float h, l;
        df_diff(src.xh[i], src.xl[i], ch[0], cl[0], h, l);
        px = h;
        df_diff(src.yh[i], src.yl[i], ch[1], cl[1], h, l);
        py = h;
        df_diff(src.zh[i], src.zl[i], ch[2], cl[2], h, l);
        pz = h;
    }
    const float sg = pk ? -1.0f : 1.0f;  // packed: -pz, -B, -n.p and |p|^2 / 2
    rec[0 * fs] = px;
    rec[1 * fs] = py;
    rec[2 * fs] = sg * pz;
    rec[3 * fs] = (pk ? 0.5f : 1.0f) * fmaf(px, px, fmaf(py, py, pz * pz));
    if (kind == RSI_STAGE_PISTON) {
        rec[4 * fs] = valid ? float(amp_scale * src.w[i]) : 0.0f;
        rec[5 * fs] = rec[6 * fs] = rec[7 * fs] = 0.0f;
    } else if (pk) {  // polar amplitudes (beta_f, m_f), padded to a whole float4
        const int nfp = 2 * ((nf + 1) / 2);
        for (int f = 0; f < nfp; ++f) {
            float* b = rec + (4 + 2 * f) * fs;
            // B_f = m_f e^{i beta_f}, beta_f = arg sigma_f, the signs of the
            // scale and the weight in m_f (reversed normals negate exactly)
            double2 sgm = make_double2(0.0, 0.0);
            double wa = 0.0;
            if (valid && f < nf) {
                sgm = sigma[size_t(a.perm[f]) * size_t(n_src) + size_t(i)];
                wa = amp_scale * src.w[i];
            }
            if (a.harm && f == nf) {
                // the padding slot: c = m_{nf-1} e^{i (beta_{nf-1} - 2 beta_0)} of the shared frequency
                double cr = 0.0, ci = 0.0;
                if (valid) {
                    const double2 s0 = sigma[size_t(a.perm[0]) * size_t(n_src) + size_t(i)];
                    const double2 s2 = sigma[size_t(a.perm[nf - 1]) * size_t(n_src) + size_t(i)];
                    const double g = atan2(s2.y, s2.x) - 2.0 * atan2(s0.y, s0.x);
                    const double m = amp_scale * src.w[i] * hypot(s2.x, s2.y);
                    cr = m * cos(g);
                    ci = m * sin(g);
                }
                b[0 * fs] = float(cr);
                b[1 * fs] = float(ci);
                continue;
            }
            b[0 * fs] = float(atan2(sgm.y, sgm.x));
            b[1 * fs] = float(wa * hypot(sgm.x, sgm.y));
        }
    } else {
        for (int f = 0; f < nf; ++f) {
            float* b = rec + (4 + 4 * f) * fs;
            if (valid) {
                const double k = double(a.kh[f]) + double(a.kl[f]);
                const double2 sgm = sigma[size_t(a.perm[f]) * size_t(n_src) + size_t(i)];
                const double br = amp_scale * src.w[i] * sgm.x, bi = amp_scale * src.w[i] * sgm.y;
                b[0 * fs] = float(br);
                b[1 * fs] = float(bi);
                b[2 * fs] = float(-k * bi);
                b[3 * fs] = float(k * br);
            } else {
                b[0 * fs] = b[1 * fs] = b[2 * fs] = b[3 * fs] = 0.0f;
            }
        }
    }
    if (kind != RSI_STAGE_PISTON) {
        if (normals == RSI_NORMALS_POINTS) {
            float* n = rec + (rf - 4) * fs;
            const float nx = valid ? float(src.nx[i]) : 0.0f, ny = valid ? float(src.ny[i]) : 0.0f,
                        nz = valid ? float(src.nz[i]) : 1.0f;
            n[0 * fs] = nx;
            n[1 * fs] = ny;
            n[2 * fs] = nz;
            n[3 * fs] = sg * fmaf(nx, px, fmaf(ny, py, nz * pz));
        }
    }
    const double rad = block_reduce(valid ? double(px * px + py * py + pz * pz) : 0.0, true, red);
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

size_t msmem(size_t tile_bytes) { return RSI_PIPE_STAGES * tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t); }

template <int KIND, int NORM, int NF, int PK, int HM = 0>
int mlaunch(const MultiArgs& a, cudaStream_t s, bool occ, int* occ_out) {
    auto kern = stage_multi_kernel<KIND, NORM, NF, PK, HM>;
    static RsiCtxOnce attr;
    if (attr.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                     "cudaFuncSetAttribute(stage_multi)");
        attr.done();
    }
    if (occ) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, msmem(a.tile_bytes)) != cudaSuccess)
            b = 1;
        *occ_out = b > 0 ? b : 1;
        return RSI_OK;
    }
    const int64_t per_block = int64_t(kThreads) * (PK ? 1 : kMTpt);
    const int64_t nblk = (a.n_tgt + per_block - 1) / per_block;
    dim3 grid(unsigned(nblk * a.splits));
    kern<<<grid, kThreads, msmem(a.tile_bytes), s>>>(a);
    RSI_CHECK_LAUNCH("stage_multi_kernel");
    return RSI_OK;
}

template <int KIND, int NORM, int PK>
int mdispatch_nf(const MultiArgs& a, cudaStream_t s, bool occ, int* o) {
    switch (a.nf) {
        case 2: return mlaunch<KIND, NORM, 2, PK>(a, s, occ, o);
        case 3:
            if constexpr (PK == 1)
                if (a.harm) return mlaunch<KIND, NORM, 3, 1, 1>(a, s, occ, o);
            return mlaunch<KIND, NORM, 3, PK>(a, s, occ, o);
        default: return mlaunch<KIND, NORM, 4, PK>(a, s, occ, o);
    }
}
template <int KIND, int NORM>
int mdispatch_pk(const MultiArgs& a, cudaStream_t s, bool occ, int* o) {
    return a.packed ? mdispatch_nf<KIND, NORM, 1>(a, s, occ, o) : mdispatch_nf<KIND, NORM, 0>(a, s, occ, o);
}

int mdispatch(const MultiArgs& a, cudaStream_t s, bool occ, int* o) {
    if (a.kind == RSI_STAGE_PISTON) return mdispatch_pk<RSI_STAGE_PISTON, RSI_NORMALS_Z>(a, s, occ, o);
    if (a.normals == RSI_NORMALS_POINTS) return mdispatch_pk<RSI_STAGE_RSI, RSI_NORMALS_POINTS>(a, s, occ, o);
    return mdispatch_pk<RSI_STAGE_RSI, RSI_NORMALS_Z>(a, s, occ, o);
}

struct MPlan {
    int S, n_tiles, tiles_per_split, splits;
    int64_t blocks;  // target blocks
    size_t tile_bytes, tiles_bytes, partial_bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int mplan(const rsi_stage& st, int nf, const double* ks, int64_t n_src, int64_t n_tgt, MPlan& p, MultiArgs& a) {
    if (st.kind != RSI_STAGE_PISTON && st.kind != RSI_STAGE_RSI)
        return rsi_fail(RSI_E_INVAL, "unknown stage kind %d", st.kind);
    if (st.precision != RSI_PREC_FP32C) return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi is FP32C only");
    if (nf < 2 || nf > kMaxNF) return rsi_fail(RSI_E_INVAL, "nf must be in 2..%d (got %d)", kMaxNF, nf);
    if (st.kind == RSI_STAGE_RSI && (st.normals < RSI_NORMALS_Z || st.normals > RSI_NORMALS_POINTS_NEG))
        return rsi_fail(RSI_E_INVAL, "unknown normals mode %d", st.normals);
    if (n_src < 1 || n_tgt < 1) return rsi_fail(RSI_E_INVAL, "empty source or target set");
    if (n_src > (int64_t(1) << 31) || n_tgt > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "more than 2^31 sources or targets");
    for (int f = 0; f < nf; ++f)
        if (!(ks[f] > 0) || !isfinite(ks[f])) return rsi_fail(RSI_E_INVAL, "wavenumbers must be finite and > 0");
    const int normals = st.kind == RSI_STAGE_RSI ? base_normals(st.normals) : RSI_NORMALS_Z;
    if (st.tile) {
        p.S = st.tile;
        if (p.S != 32 && p.S != 64 && p.S != 128 && p.S != 256)
            return rsi_fail(RSI_E_INVAL, "tile must be 32, 64, 128 or 256");
    } else {
        const int64_t cap = n_src / 64;
        p.S = 256;
        while (p.S > 32 && p.S > cap) p.S >>= 1;
    }
    p.n_tiles = int((n_src + p.S - 1) / p.S);
    if (st.variant != 0 && st.variant != 2 && st.variant != 3)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi: variant must be 0, 2 or 3");
    a.packed = st.variant != 2;  // 3 (and 0): two sources per f32x2 instruction; 2: scalar
    p.tile_bytes = RSI_TILE_HDR_BYTES + size_t(p.S) * 16 * size_t(mrec_f4_rt(st.kind, normals, nf, a.packed != 0));
    p.tiles_bytes = align256(size_t(p.n_tiles) * p.tile_bytes);
    a.kind = st.kind;
    a.normals = normals;
    a.nf = nf;
    a.S = p.S;
    a.n_tiles = p.n_tiles;
    a.n_tgt = n_tgt;
    a.tile_bytes = p.tile_bytes;
    // frequency order in the kernel: the caller's, or with a shared harmonic
    // (three frequencies, packed, k_j = 2 k_i to 2^-40) i first and j last
    for (int f = 0; f < kMaxNF; ++f) a.perm[f] = f < nf ? f : 0;
    a.harm = 0;
    if (nf == 3 && a.packed) {
        for (int i = 0; i < nf && !a.harm; ++i)
            for (int j = 0; j < nf && !a.harm; ++j)
                if (i != j && fabs(ks[j] - 2.0 * ks[i]) <= 0x1p-40 * ks[j]) {
                    a.harm = 1;
                    a.perm[0] = i;
                    a.perm[1] = 3 - i - j;
                    a.perm[2] = j;
                }
    }
    for (int f = 0; f < kMaxNF; ++f) {
        const double k = f < nf ? ks[a.perm[f]] : ks[0];
        a.kh[f] = float(k);
        a.kl[f] = float(k - double(a.kh[f]));
    }
    a.tp = two_pi_split();
    const int tpt = a.packed ? 1 : kMTpt;
    const int64_t blocks = (n_tgt + int64_t(kThreads) * tpt - 1) / (int64_t(kThreads) * tpt);
    int splits = st.splits;
    if (splits < 0) return rsi_fail(RSI_E_INVAL, "splits must be >= 0");
    if (splits == 0) {
        int occ = 1;
        mdispatch(a, nullptr, true, &occ);
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
    if (splits > 65535) return rsi_fail(RSI_E_INVAL, "too many splits");
    p.tiles_per_split = (p.n_tiles + splits - 1) / splits;
    p.splits = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    // partial sums [splits][nf][n_tgt], then one completion counter per target block
    p.partial_bytes = p.splits > 1 ? align256(size_t(p.splits) * size_t(nf) * size_t(n_tgt) * sizeof(double2)) +
                                         align256(size_t(blocks) * sizeof(unsigned))
                                   : 0;
    p.blocks = blocks;
    a.tiles_per_split = p.tiles_per_split;
    a.splits = p.splits;
    return RSI_OK;
}

}  // namespace

extern "C" size_t rsi_stage_multi_workspace_bytes(const rsi_stage* st, int32_t nf, const double* ks, int64_t n_src,
                                                  int64_t n_tgt) {
    if (!st || !ks) return 0;
    MPlan p;
    MultiArgs a = {};
    if (mplan(*st, nf, ks, n_src, n_tgt, p, a) != RSI_OK) return 0;
    return p.tiles_bytes + p.partial_bytes;
}

extern "C" int rsi_propagate_stage_multi(const rsi_stage* st, int32_t nf, const double* ks, const void* src_points,
                                         int64_t n_src, const double* src_sigma, const void* tgt_points,
                                         int64_t n_tgt, double* tgt_field, void* workspace, size_t workspace_bytes,
                                         void* stream) {
    if (!st || !ks || !src_points || !tgt_points || !tgt_field || !workspace)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi: null argument");
    if (st->kind == RSI_STAGE_RSI && !src_sigma)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi: RSI stage needs source densities");
    if (st->kind == RSI_STAGE_PISTON && !isfinite(st->v0))
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi: v0 must be finite");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 || reinterpret_cast<uintptr_t>(src_points) % 256 ||
        reinterpret_cast<uintptr_t>(tgt_points) % 256 || reinterpret_cast<uintptr_t>(tgt_field) % 16 ||
        (src_sigma && reinterpret_cast<uintptr_t>(src_sigma) % 16))
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage_multi: misaligned pointer");
    MPlan p;
    MultiArgs a = {};
    int rc = mplan(*st, nf, ks, n_src, n_tgt, p, a);
    if (rc != RSI_OK) return rc;
    if (workspace_bytes < p.tiles_bytes + p.partial_bytes)
        return rsi_fail(RSI_E_NOMEM, "rsi_propagate_stage_multi: workspace %zu < %zu bytes", workspace_bytes,
                        p.tiles_bytes + p.partial_bytes);
    int* status = rsi_status_ptr();
    if (!status) return RSI_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PointsView src = rsi_points_view(const_cast<void*>(src_points), n_src);
    PointsView tgt = rsi_points_view(const_cast<void*>(tgt_points), n_tgt);
    uint8_t* tiles = static_cast<uint8_t*>(workspace);
    mprep_kernel<<<p.n_tiles, p.S, 0, s>>>(a.kind, a.normals, nf, n_src, src,
                                           reinterpret_cast<const double2*>(src_sigma), stage_amp_scale(*st), a,
                                           tiles, p.tile_bytes);
    RSI_CHECK_LAUNCH("mprep_kernel");
    a.tiles = tiles;
    a.tgt = {tgt.xh, tgt.xl, tgt.yh, tgt.yl, tgt.zh, tgt.zl, tgt.x, tgt.y, tgt.z};
    double2* field = reinterpret_cast<double2*>(tgt_field);
    a.out = p.splits > 1 ? reinterpret_cast<double2*>(tiles + p.tiles_bytes) : field;
    a.field = field;
    a.done = nullptr;
    if (p.splits > 1) {
        const size_t part = align256(size_t(p.splits) * size_t(nf) * size_t(n_tgt) * sizeof(double2));
        a.done = reinterpret_cast<unsigned*>(tiles + p.tiles_bytes + part);
        RSI_CUDA_TRY(cudaMemsetAsync(a.done, 0, size_t(p.blocks) * sizeof(unsigned), s),
                     "rsi_propagate_stage_multi: clear the completion counters");
    }
    a.status = status;
    TimingScope tsc = timing_begin(s);
    int o = 0;
    rc = mdispatch(a, s, false, &o);
    if (rc != RSI_OK) return rc;
    timing_end(tsc, st->kind, double(nf) * double(n_src) * double(n_tgt), s);
    return RSI_OK;
}

extern "C" int rsi_stage_multi_shared_harmonic(const rsi_stage* st, int32_t nf, const double* ks) {
    if (!st || !ks) return rsi_fail(RSI_E_INVAL, "rsi_stage_multi_shared_harmonic: null argument");
    MPlan p;
    MultiArgs a = {};
    const int rc = mplan(*st, nf, ks, 1 << 12, 1 << 12, p, a);
    if (rc != RSI_OK) return rc;
    return a.harm;
}
