// stage_fp32.cu -- FP32C source x target kernel (steps a3, a5).
//
// Every target keeps, per source tile, a reference built in double-float
// arithmetic: D = Q - c (c = tile centre), R = |D| and the phase
// tau = k R mod 2 pi.  A pair then needs only FP32 work on small offsets
// p = P - c: r^2 = |D - p|^2 and t = |p|^2 - 2 D.p = r^2 - R^2 give
// r - R = t / (R + r) (or a Newton step on r^2 = R^2 + t) without
// cancellation, so the phase tau + k (r - R) is accurate to about
// 2^-23 k |r - R| <= 2^-23 k (tile radius) instead of 2^-24 k r.
// Tiles arrive in shared memory by bulk copy (cp.async.bulk) on mbarriers,
// RSI_PIPE_STAGES deep; each thread owns TPT targets and loops over the
// tile; tile sums are FP32 and are added into a double-float accumulator.
#include <math.h>

#include "stage.cuh"

namespace {

constexpr int kThreads = 256;
constexpr float kTwoPiInv = 0.159154943091895335768883763f;

struct TgtRef {
    float Dx, Dy, Dz, mx, my, mz, R, tau;
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
    t.tau = x;
    return t;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// one source (records a, b[, n]) onto one target reference
template <int KIND, int NORM, int VAR>
__device__ __forceinline__ void pair_term(const TgtRef& t, const float4& a, const float4& b, const float4& nr,
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
    float u = fmaf(k, dr, t.tau);
    float s, c;
    __sincosf(u, &s, &c);
    if (KIND == RSI_STAGE_PISTON) {
        float amp = b.x * ir;
        acc_r = fmaf(amp, c, acc_r);
        acc_i = fmaf(amp, s, acc_i);
    } else {
        float nd = (NORM == RSI_NORMALS_Z) ? dz : fmaf(nr.x, dx, fmaf(nr.y, dy, nr.z * dz));
        float h = nd * (ir * ir);  // cos(theta) / r
        float vr = fmaf(-ir, b.x, b.z);  // B (ik - 1/r)
        float vi = fmaf(-ir, b.y, b.w);
        float wr = fmaf(vr, c, -vi * s);
        float wi = fmaf(vr, s, vi * c);
        acc_r = fmaf(h, wr, acc_r);
        acc_i = fmaf(h, wi, acc_i);
    }
}

template <int KIND, int NORM, int TPT, int VAR>
__global__ void __launch_bounds__(kThreads, 2)
    stage_fp32_kernel(StageArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int t_begin = split * a.tiles_per_split;
    const int t_end = min(a.n_tiles, t_begin + a.tiles_per_split);
    const int ntile = max(0, t_end - t_begin);
    const uint32_t tile_bytes = uint32_t(a.tile_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * a.tile_bytes);
    const int rec_f4 = (KIND == RSI_STAGE_RSI && NORM == RSI_NORMALS_POINTS) ? 3 : 2;

    int64_t jt[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int64_t j = (int64_t(blockIdx.x) * TPT + q) * kThreads + tid;
        jt[q] = j < a.n_tgt ? j : a.n_tgt - 1;
    }

    if (tid == 0) {
        for (int s = 0; s < RSI_PIPE_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < RSI_PIPE_STAGES && s < ntile; ++s) {
            uint32_t bar = smem_u32(&bars[s]);
            mbar_expect_tx(bar, tile_bytes);
            bulk_g2s(smem_u32(smem + s * a.tile_bytes), a.tiles + size_t(t_begin + s) * a.tile_bytes, tile_bytes,
                     bar);
        }
    }

    float hr[TPT], lr[TPT], hi[TPT], li[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) hr[q] = lr[q] = hi[q] = li[q] = 0.0f;
    const float k = a.kh;
    int failed_at = -1;

    for (int it = 0; it < ntile; ++it) {
        const int buf = it % RSI_PIPE_STAGES;
        const uint32_t parity = uint32_t(it / RSI_PIPE_STAGES) & 1u;
        bool ok = mbar_wait_bounded(smem_u32(&bars[buf]), parity);
        if (__syncthreads_or(!ok)) {
            failed_at = it;
            break;
        }
        const uint8_t* tile = smem + buf * a.tile_bytes;
        const float* hdr = reinterpret_cast<const float*>(tile);
        const float4* rec = reinterpret_cast<const float4*>(tile + RSI_TILE_HDR_BYTES);
        TgtRef ref[TPT];
        float ar[TPT], ai[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            const int64_t j = jt[q];
            ref[q] = target_reference(__ldg(a.tgt.xh + j), __ldg(a.tgt.xl + j), __ldg(a.tgt.yh + j),
                                      __ldg(a.tgt.yl + j), __ldg(a.tgt.zh + j), __ldg(a.tgt.zl + j), hdr, a.kh,
                                      a.kl, a.tp);
            ar[q] = 0.0f;
            ai[q] = 0.0f;
        }
#pragma unroll 2
        for (int i = 0; i < a.S; ++i) {
            const float4 ra = rec[i * rec_f4];
            const float4 rb = rec[i * rec_f4 + 1];
            const float4 rn = (rec_f4 == 3) ? rec[i * rec_f4 + 2] : make_float4(0.f, 0.f, 1.f, 0.f);
#pragma unroll
            for (int q = 0; q < TPT; ++q) pair_term<KIND, NORM, VAR>(ref[q], ra, rb, rn, k, ar[q], ai[q]);
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
        if (tid == 0 && it + RSI_PIPE_STAGES < ntile) {
            uint32_t bar = smem_u32(&bars[buf]);
            mbar_expect_tx(bar, tile_bytes);
            bulk_g2s(smem_u32(smem + buf * a.tile_bytes),
                     a.tiles + size_t(t_begin + it + RSI_PIPE_STAGES) * a.tile_bytes, tile_bytes, bar);
        }
    }

    if (failed_at >= 0) {
        if (tid == 0) {
            atomicExch(a.status, RSI_DEV_TIMEOUT);
            // let the copies still in flight land (bounded) before the CTA's
            // shared memory is released
            for (int it = failed_at; it < ntile && it < failed_at + RSI_PIPE_STAGES; ++it)
                mbar_wait_bounded(smem_u32(&bars[it % RSI_PIPE_STAGES]), uint32_t(it / RSI_PIPE_STAGES) & 1u);
        }
        return;
    }

    double2* out = a.out + (a.splits > 1 ? size_t(split) * size_t(a.n_tgt) : 0);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int64_t j = (int64_t(blockIdx.x) * TPT + q) * kThreads + tid;
        if (j < a.n_tgt) {
            double re = double(hr[q]) + double(lr[q]);
            double im = double(hi[q]) + double(li[q]);
            if (!isfinite(re) || !isfinite(im)) atomicExch(a.status, RSI_DEV_NONFINITE);
            out[j] = make_double2(re, im);
        }
    }
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

__global__ void prep_fp32_kernel(int kind, int normals, int64_t n_src, PointsView src,
                                 const double2* __restrict__ sigma, double amp_scale, double k, uint8_t* tiles,
                                 size_t tile_bytes) {
    __shared__ double red[32];
    const int S = blockDim.x;
    const int64_t i = int64_t(blockIdx.x) * S + threadIdx.x;
    const bool valid = i < n_src;
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
    float* rec = reinterpret_cast<float*>(tiles + size_t(blockIdx.x) * tile_bytes + RSI_TILE_HDR_BYTES) +
                 size_t(threadIdx.x) * rec_f;
    float px = 4.0f, py = 4.0f, pz = 4.0f, radius2 = 0.0f;
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
    float nx = 0.f, ny = 0.f, nz = 1.f;
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
            nx = float(src.nx[i]);
            ny = float(src.ny[i]);
            nz = float(src.nz[i]);
        }
    }
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
        rec[11] = 0.0f;
    }
    double rad = block_reduce(double(radius2), true, red);
    if (threadIdx.x == 0) {
        float* hdr = reinterpret_cast<float*>(tiles + size_t(blockIdx.x) * tile_bytes);
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

template <int KIND, int NORM, int TPT, int VAR>
int launch_t(const StageArgs& a, cudaStream_t s) {
    size_t smem = RSI_PIPE_STAGES * a.tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t);
    static bool attr_set = false;
    if (!attr_set) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(stage_fp32_kernel<KIND, NORM, TPT, VAR>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                     "cudaFuncSetAttribute(stage_fp32)");
        attr_set = true;
    }
    int64_t per_block = int64_t(kThreads) * TPT;
    dim3 grid(unsigned((a.n_tgt + per_block - 1) / per_block), unsigned(a.splits));
    stage_fp32_kernel<KIND, NORM, TPT, VAR><<<grid, kThreads, smem, s>>>(a);
    RSI_CHECK_LAUNCH("stage_fp32_kernel");
    return RSI_OK;
}

template <int KIND, int NORM, int TPT, int VAR>
int occupancy_t(const StageArgs& a) {
    size_t smem = RSI_PIPE_STAGES * a.tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, stage_fp32_kernel<KIND, NORM, TPT, VAR>, kThreads,
                                                      smem) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

template <int KIND, int NORM>
int dispatch_tv(const StageArgs& a, cudaStream_t s, bool occ) {
    if (a.tpt == 4) {
        if (a.variant == 2) return occ ? occupancy_t<KIND, NORM, 4, 2>(a) : launch_t<KIND, NORM, 4, 2>(a, s);
        return occ ? occupancy_t<KIND, NORM, 4, 1>(a) : launch_t<KIND, NORM, 4, 1>(a, s);
    }
    if (a.variant == 2) return occ ? occupancy_t<KIND, NORM, 2, 2>(a) : launch_t<KIND, NORM, 2, 2>(a, s);
    return occ ? occupancy_t<KIND, NORM, 2, 1>(a) : launch_t<KIND, NORM, 2, 1>(a, s);
}

int dispatch(const StageArgs& a, cudaStream_t s, bool occ) {
    if (a.kind == RSI_STAGE_PISTON) return dispatch_tv<RSI_STAGE_PISTON, RSI_NORMALS_Z>(a, s, occ);
    if (a.normals == RSI_NORMALS_POINTS) return dispatch_tv<RSI_STAGE_RSI, RSI_NORMALS_POINTS>(a, s, occ);
    return dispatch_tv<RSI_STAGE_RSI, RSI_NORMALS_Z>(a, s, occ);
}

}  // namespace

size_t fp32_record_bytes(int kind, int normals) {
    return (kind == RSI_STAGE_RSI && normals == RSI_NORMALS_POINTS) ? 48 : 32;
}

int fp32_threads() { return kThreads; }

int launch_prep_fp32(const rsi_stage& st, const PointsView& src, int64_t n_src, const double2* sigma, int S,
                     uint8_t* tiles, size_t tile_bytes, int n_tiles, cudaStream_t s) {
    double amp_scale = (st.kind == RSI_STAGE_PISTON) ? -st.v0 / (2.0 * M_PI) : -1.0 / (2.0 * M_PI);
    prep_fp32_kernel<<<n_tiles, S, 0, s>>>(st.kind, st.normals, n_src, src, sigma, amp_scale, st.k, tiles,
                                           tile_bytes);
    RSI_CHECK_LAUNCH("prep_fp32_kernel");
    return RSI_OK;
}

int launch_stage_fp32(const StageArgs& a, cudaStream_t s) { return dispatch(a, s, false); }
int stage_occupancy_fp32(const StageArgs& a) { return dispatch(a, nullptr, true); }
