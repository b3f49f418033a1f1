// nn_net.cu -- the learned surrogate's coordinate network as whole calls:
// input rows (rsi_nn_rows), forward, backward, Adam and image inference
// (rsi_nn_infer), plus the training targets (rsi_nn_targets).  The hidden
// layers run on nn.cu's tensor-core GEMMs (rsi_nn_gemm: BF16 operands, FP32
// accumulation, bias + SiLU or SiLU' epilogues); this file adds the row
// inputs, the 3-output head and its gradient, the per-field assembly of an
// image, and the sequencing.  The network is defined in include/rsi.h.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "rsi_internal.cuh"

namespace {

using bf16 = __nv_bfloat16;
constexpr int kRaw = 16;   // raw inputs appended to the Fourier features (9 + 7 zeros)
constexpr int kHead = 3;   // head outputs: re, im, log rms
constexpr int kHeadRows = 128;  // rows per CTA of the head's backward
constexpr int kColRows = 64;    // rows per CTA of the column sums

int64_t seg(int64_t n) { return (n + 63) / 64 * 64; }
size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

struct Dims {
    int F, K0, W, D, R, npix;
};

int dims_of(const rsi_nn_net* n, Dims& d, const char* who) {
    if (!n) return rsi_fail(RSI_E_INVAL, "%s: null net", who);
    d.F = n->n_freq;
    d.K0 = 2 * n->n_freq + kRaw;
    d.W = n->width;
    d.D = n->depth;
    d.R = n->rows;
    d.npix = n->window.nx * n->window.nz;
    if (d.F < 1 || d.K0 % 128)
        return rsi_fail(RSI_E_INVAL, "%s: 2 n_freq + 16 must be a positive multiple of 128", who);
    if (d.W != 128 && d.W != 256 && d.W != 512 && d.W != 1024)
        return rsi_fail(RSI_E_INVAL, "%s: width must be 128, 256, 512 or 1024", who);
    if (d.D < 1 || d.D > RSI_NN_MAX_DEPTH) return rsi_fail(RSI_E_INVAL, "%s: depth outside 1..%d", who, RSI_NN_MAX_DEPTH);
    if (d.R < 128 || d.R % 128) return rsi_fail(RSI_E_INVAL, "%s: rows must be a multiple of 128", who);
    if (n->window.nx < 1 || n->window.nz < 1 || !(n->window.x1 > n->window.x0) || !(n->window.z1 > n->window.z0))
        return rsi_fail(RSI_E_INVAL, "%s: empty window", who);
    if (!(n->c1 > 0) || !(n->c2 > 0) || !(n->a > 0)) return rsi_fail(RSI_E_INVAL, "%s: bad media or radius", who);
    for (int k = 0; k < 4; ++k)
        if (!(n->box_hi[k] > n->box_lo[k])) return rsi_fail(RSI_E_INVAL, "%s: empty parameter box", who);
    if (n->engine != RSI_NN_ENGINE_TCGEN05 && n->engine != RSI_NN_ENGINE_MMA_SYNC)
        return rsi_fail(RSI_E_INVAL, "%s: unknown engine", who);
    return RSI_OK;
}

int in_of(const Dims& d, int l) { return l == 0 ? d.K0 : d.W; }

// element offsets of W_l and b_l in the flat parameter buffers
int64_t w_off(const Dims& d, int layer) {
    int64_t o = 0;
    for (int l = 0; l < layer; ++l) o += seg(int64_t(d.W) * in_of(d, l)) + seg(d.W);
    return o;
}
int64_t b_off(const Dims& d, int layer) {
    return w_off(d, layer) + seg(int64_t(layer == d.D ? kHead : d.W) * (layer == d.D ? d.W : in_of(d, layer)));
}
int64_t param_elems(const Dims& d) { return b_off(d, d.D) + seg(kHead); }

// split count of the weight-gradient GEMMs (M = width, N = in_l, K = rows):
// about two CTAs per SM over their few output tiles
int grad_splits(const Dims& d) {
    const int tiles = (d.W / 128) * (std::max(d.K0, d.W) / 128);
    int s = (2 * rsi_num_sms() + tiles - 1) / tiles;
    return std::max(1, std::min(s, d.R / 64));
}

struct Act {
    size_t h[RSI_NN_MAX_DEPTH + 1], z[RSI_NN_MAX_DEPTH + 1];
    size_t y, t, dz[2], work, part, colpart, lpart, env, p32, total;
    int splits, head_chunks;
};

Act act_layout(const Dims& d) {
    Act a = {};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = al256(o + bytes);
        return at;
    };
    a.h[0] = take(size_t(d.R) * d.K0 * sizeof(bf16));
    for (int l = 1; l <= d.D; ++l) {
        a.z[l] = take(size_t(d.R) * d.W * sizeof(float));
        a.h[l] = take(size_t(d.R) * d.W * sizeof(bf16));
    }
    a.y = take(size_t(d.R) * 4 * sizeof(float));
    a.t = take(size_t(d.R) * 4 * sizeof(float));
    a.dz[0] = take(size_t(d.R) * d.W * sizeof(bf16));
    a.dz[1] = take(size_t(d.R) * d.W * sizeof(bf16));
    a.splits = grad_splits(d);
    a.work = take(size_t(a.splits) * d.W * std::max(d.K0, d.W) * sizeof(float));
    a.head_chunks = d.R / kHeadRows;
    a.part = take(size_t(a.head_chunks) * (kHead * d.W + kHead + 1) * sizeof(float));
    a.colpart = take(size_t((d.R + kColRows - 1) / kColRows) * d.W * sizeof(float));
    a.lpart = take(1024 * sizeof(double));
    a.env = take(size_t(d.R) * 2 * sizeof(float));
    a.p32 = take(size_t(d.R) * 5 * sizeof(float));
    a.total = o;
    return a;
}

// ---------------------------------------------------------------------------
// kernel arguments: the row-input constants in FP32
// ---------------------------------------------------------------------------
struct RowK {
    int F, K0, nx, npix;
    float x0, dx, z0, dz, Wz, inv_S0, c21, a2_over_c1;
    float lo[4], inv_span[4];
    const float* fmat;
};

RowK row_consts(const rsi_nn_net& n, const Dims& d) {
    RowK k;
    k.F = d.F;
    k.K0 = d.K0;
    k.nx = n.window.nx;
    k.npix = d.npix;
    k.x0 = float(n.window.x0);
    k.dx = float((n.window.x1 - n.window.x0) / n.window.nx);
    k.z0 = float(n.window.z0);
    k.dz = float((n.window.z1 - n.window.z0) / n.window.nz);
    k.Wz = float(n.window.z1 - n.window.z0);
    k.inv_S0 = float(2.0 / (n.window.x1 - n.window.x0));
    k.c21 = float(n.c2 / n.c1);
    k.a2_over_c1 = float(n.a * n.a / n.c1);
    for (int i = 0; i < 4; ++i) {
        k.lo[i] = float(n.box_lo[i]);
        k.inv_span[i] = float(2.0 / (n.box_hi[i] - n.box_lo[i]));
    }
    k.fmat = n.fmat;
    return k;
}

// SplitMix64's output function (Steele, Lea & Flood 2014) at state s
__device__ __forceinline__ uint64_t splitmix64(uint64_t s) {
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// One warp per row: the (field, pixel) pair, the 9 inputs c, then columns
// [sin(pi B c) | cos(pi B c) | c, 0...] with the Fourier columns spread over
// the lanes (consecutive lanes write consecutive columns).
__global__ void __launch_bounds__(256) rows_kernel(RowK k, const double* __restrict__ params, int64_t n_fields,
                                                   int mode, uint64_t seed, const uint64_t* __restrict__ seed_dev,
                                                   int64_t first, const float* __restrict__ targets,
                                                   const float* __restrict__ log_rms, int R, bf16* __restrict__ h0,
                                                   float4* __restrict__ t_rows) {
    extern __shared__ float sB[];  // [F][9]
    for (int e = threadIdx.x; e < k.F * RSI_NN_IN; e += blockDim.x) sB[e] = k.fmat[e];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R) return;
    int64_t b, q;
    if (mode == RSI_NN_ROWS_RANDOM) {
        const uint64_t sd = seed_dev ? *seed_dev : seed;
        const uint64_t u = splitmix64(sd + 0x9E3779B97F4A7C15ull * uint64_t(r + 1));
        b = int64_t((uint64_t(uint32_t(u >> 32)) * uint64_t(n_fields)) >> 32);
        q = int64_t((uint64_t(uint32_t(u)) * uint64_t(k.npix)) >> 32);
    } else {
        int64_t g = first + r;
        const int64_t last = n_fields * int64_t(k.npix) - 1;
        g = g < last ? g : last;
        b = g / k.npix;
        q = g - b * k.npix;
    }
    const double* p = params + 5 * b;
    const float tilt = float(p[1]), L = float(p[2]), f = float(p[3]), d = float(p[4]);
    const int i = int(q % k.nx), j = int(q / k.nx);
    const float sg = tilt < 0.0f ? -1.0f : 1.0f;
    const float a1 = fabsf(tilt);
    const float xw = k.x0 + (float(i) + 0.5f) * k.dx;
    const float zw = k.z0 + (float(j) + 0.5f) * k.dz;
    const float x = sg * xw, z = d + zw;
    const float sth = fminf(1.0f, k.c21 * sinf(a1));
    const float cth = sqrtf(fmaxf(0.0f, 1.0f - sth * sth));
    const float s = x * sth + z * cth, t = x * cth - z * sth;
    const float fq = k.a2_over_c1 * f / (L + k.c21 * fmaxf(s, 0.0f));
    float c[RSI_NN_IN];
    c[0] = (a1 - k.lo[0]) * k.inv_span[0] - 1.0f;
    c[1] = (L - k.lo[1]) * k.inv_span[1] - 1.0f;
    c[2] = (f - k.lo[2]) * k.inv_span[2] - 1.0f;
    c[3] = (d - k.lo[3]) * k.inv_span[3] - 1.0f;
    c[4] = x * k.inv_S0;
    c[5] = 2.0f * (zw - k.z0) / k.Wz - 1.0f;
    c[6] = s * k.inv_S0;
    c[7] = t * k.inv_S0;
    c[8] = logf(fq);
    bf16* row = h0 + size_t(r) * k.K0;
    for (int fi = lane; fi < k.F; fi += 32) {
        const float* Bf = sB + fi * RSI_NN_IN;
        float arg = 0.0f;
#pragma unroll
        for (int m = 0; m < RSI_NN_IN; ++m) arg = fmaf(Bf[m], c[m], arg);
        float sn, cs;
        sincospif(arg, &sn, &cs);
        row[fi] = __float2bfloat16_rn(sn);
        row[k.F + fi] = __float2bfloat16_rn(cs);
    }
    if (lane < kRaw) row[2 * k.F + lane] = __float2bfloat16_rn(lane < RSI_NN_IN ? c[lane] : 0.0f);
    if (targets && lane == 0) {
        const float* tg = targets + 2 * (b * int64_t(k.npix) + q);
        t_rows[r] = make_float4(tg[0], tg[1], log_rms[b], 0.0f);
    }
}

// head forward, y = W_h h + b_h: each lane keeps its columns' head weights
// (lane l holds columns 8 l .. 8 l + 7 of every 256) in registers, and a warp
// walks rows with a stride of all the grid's warps, reading each row once
// (coalesced 16-byte loads) and reducing the three dot products by shuffles.
template <int NC>  // 256-column chunks per row: W = 256 NC (W = 128: half the lanes)
__global__ void __launch_bounds__(256) head_fwd_kernel(const bf16* __restrict__ H, int W, int R,
                                                       const float* __restrict__ Wh, const float* __restrict__ bh,
                                                       float4* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    float w[kHead][NC][8];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int col = c * 256 + lane * 8;
#pragma unroll
        for (int o = 0; o < kHead; ++o)
#pragma unroll
            for (int e = 0; e < 8; ++e) w[o][c][e] = col < W ? Wh[o * W + col + e] : 0.0f;
    }
    const float b0 = bh[0], b1 = bh[1], b2 = bh[2];
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
        const bf16* h = H + size_t(r) * W;
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int col = c * 256 + lane * 8;
            if (col >= W) continue;
            const uint4 v = *reinterpret_cast<const uint4*>(h + col);
            const bf16* hv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float x = __bfloat162float(hv[e]);
                a0 = fmaf(w[0][c][e], x, a0);
                a1 = fmaf(w[1][c][e], x, a1);
                a2 = fmaf(w[2][c][e], x, a2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) y[r] = make_float4(a0 + b0, a1 + b1, a2 + b2, 0.0f);
    }
}

__device__ __forceinline__ float silu_grad(float z) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));  // fast division: the result is rounded to bf16
    return s * (1.0f + z * (1.0f - s));
}

// head backward over kHeadRows rows per CTA of 256 threads: W / 8 column
// threads (8 columns each) times 256 / (W / 8) row groups.  dy = g (y - t)
// (first 3 outputs), dZ = (dy W_h) * silu'(Z) as bf16, and this CTA's partial
// sums of dy h (the head's weight gradient), of dy (its bias gradient) and of
// (y - t)^2, combined over the row groups in fixed order.
__global__ void __launch_bounds__(256) head_bwd_kernel(const bf16* __restrict__ H, const float* __restrict__ Z,
                                                       int W, const float4* __restrict__ y,
                                                       const float4* __restrict__ t, const float* __restrict__ Wh,
                                                       float g, bf16* __restrict__ dZ, float* __restrict__ part) {
    extern __shared__ float sm[];  // [3][W] weights, [kHeadRows][4] dy, [groups][3][W] partial sums
    const int ct = W / 8, groups = 256 / ct, rows_g = kHeadRows / groups;
    float* sW = sm;
    float* sdy = sW + kHead * W;
    float* sg = sdy + 4 * kHeadRows;
    __shared__ double sl[256];
    for (int e = threadIdx.x; e < kHead * W; e += blockDim.x) sW[e] = Wh[e];
    const int r0 = blockIdx.x * kHeadRows;
    double l2 = 0.0;
    for (int rr = threadIdx.x; rr < kHeadRows; rr += blockDim.x) {
        const float4 a = y[r0 + rr], b = t[r0 + rr];
        const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z;
        sdy[4 * rr] = g * e0;
        sdy[4 * rr + 1] = g * e1;
        sdy[4 * rr + 2] = g * e2;
        l2 += double(e0) * e0 + double(e1) * e1 + double(e2) * e2;
    }
    sl[threadIdx.x] = l2;
    __syncthreads();
    const int c0 = (threadIdx.x % ct) * 8, grp = threadIdx.x / ct;
    float gw[kHead][8];
#pragma unroll
    for (int o = 0; o < kHead; ++o)
#pragma unroll
        for (int e = 0; e < 8; ++e) gw[o][e] = 0.0f;
    for (int rr = grp * rows_g; rr < (grp + 1) * rows_g; ++rr) {
        const size_t off = size_t(r0 + rr) * W + c0;
        const uint4 hv4 = *reinterpret_cast<const uint4*>(H + off);
        const bf16* hv = reinterpret_cast<const bf16*>(&hv4);
        const float d0 = sdy[4 * rr], d1 = sdy[4 * rr + 1], d2 = sdy[4 * rr + 2];
        const float4 za = *reinterpret_cast<const float4*>(Z + off);
        const float4 zb = *reinterpret_cast<const float4*>(Z + off + 4);
        const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        uint4 outv;
        bf16* ov = reinterpret_cast<bf16*>(&outv);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float x = __bfloat162float(hv[e]);
            gw[0][e] = fmaf(d0, x, gw[0][e]);
            gw[1][e] = fmaf(d1, x, gw[1][e]);
            gw[2][e] = fmaf(d2, x, gw[2][e]);
            const float dh = fmaf(d0, sW[c0 + e], fmaf(d1, sW[W + c0 + e], d2 * sW[2 * W + c0 + e]));
            ov[e] = __float2bfloat16_rn(dh * silu_grad(zz[e]));
        }
        *reinterpret_cast<uint4*>(dZ + off) = outv;
    }
#pragma unroll
    for (int o = 0; o < kHead; ++o)
#pragma unroll
        for (int e = 0; e < 8; ++e) sg[(grp * kHead + o) * W + c0 + e] = gw[o][e];
    for (int st = 128; st > 0; st >>= 1) {
        __syncthreads();
        if (threadIdx.x < st) sl[threadIdx.x] += sl[threadIdx.x + st];
    }
    __syncthreads();
    float* out = part + size_t(blockIdx.x) * (kHead * W + kHead + 1);
    for (int e = threadIdx.x; e < kHead * W; e += blockDim.x) {
        float acc = 0.0f;
        for (int gq = 0; gq < groups; ++gq) acc += sg[gq * kHead * W + e];
        out[e] = acc;
    }
    if (threadIdx.x < kHead) {
        float sb = 0.0f;
        for (int rr = 0; rr < kHeadRows; ++rr) sb += sdy[4 * rr + threadIdx.x];
        out[kHead * W + threadIdx.x] = sb;
    }
    if (threadIdx.x == 0) out[kHead * W + kHead] = float(sl[0]);
}

// sum over chunks of per-chunk partial sums part[chunk][n], in a fixed order:
// 32 values per CTA, 8 lanes per value each taking every 8th chunk (FP64),
// the lanes added in lane order.  Values e < n_w go to out_w[e], the next
// n_b to out_b, a last one (if n > n_w + n_b) times last_scale to *last.
__global__ void __launch_bounds__(256) chunk_sum_kernel(const float* __restrict__ part, int chunks, int n, int n_w,
                                                        int n_b, float last_scale, float* __restrict__ out_w,
                                                        float* __restrict__ out_b, float* __restrict__ last) {
    __shared__ double red[8][33];
    const int e = blockIdx.x * 32 + threadIdx.x;
    double acc = 0.0;
    if (e < n)
        for (int c = threadIdx.y; c < chunks; c += 8) acc += double(part[size_t(c) * n + e]);
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y != 0 || e >= n) return;
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
    if (e < n_w)
        out_w[e] = float(t);
    else if (e < n_w + n_b)
        out_b[e - n_w] = float(t);
    else if (last)
        *last = float(t * double(last_scale));
}

// column sums of a bf16 [rows][cols] matrix (cols even), first pass: CTA
// (x, y) sums rows y kColRows .. + kColRows of columns 512 x .. + 512, two
// adjacent columns per thread, into part[y][cols]
__global__ void __launch_bounds__(256) colsum_part_kernel(const bf16* __restrict__ m, int rows, int cols,
                                                          float* __restrict__ part) {
    const int c = blockIdx.x * 512 + 2 * threadIdx.x;
    if (c >= cols) return;
    const int r0 = blockIdx.y * kColRows, r1 = min(rows, r0 + kColRows);
    float s0 = 0.0f, s1 = 0.0f;
    for (int r = r0; r < r1; ++r) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(m + size_t(r) * cols + c);
        s0 += __low2float(v);
        s1 += __high2float(v);
    }
    part[size_t(blockIdx.y) * cols + c] = s0;
    part[size_t(blockIdx.y) * cols + c + 1] = s1;
}

// per field (one CTA): the mean of the log-RMS outputs over its pixels, then
// exp(mean) (re, im) interleaved for the carrier pass
__global__ void __launch_bounds__(256) assemble_kernel(const float4* __restrict__ y, int npix,
                                                       float2* __restrict__ env) {
    __shared__ double red[256];
    const float4* yb = y + size_t(blockIdx.x) * npix;
    double s = 0.0;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) s += double(yb[p].z);
    red[threadIdx.x] = s;
    for (int st = 128; st > 0; st >>= 1) {
        __syncthreads();
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    }
    __syncthreads();
    const float amp = float(exp(red[0] / double(npix)));
    float2* eb = env + size_t(blockIdx.x) * npix;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) eb[p] = make_float2(amp * yb[p].x, amp * yb[p].y);
}

// training targets of one field (one CTA): the demodulated image over its RMS
// and the log of that RMS
__global__ void __launch_bounds__(256) targets_kernel(const float2* __restrict__ env, int npix,
                                                      float2* __restrict__ out, float* __restrict__ log_rms) {
    __shared__ double red[256];
    const float2* eb = env + size_t(blockIdx.x) * npix;
    double s = 0.0;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) s += double(eb[p].x) * eb[p].x + double(eb[p].y) * eb[p].y;
    red[threadIdx.x] = s;
    for (int st = 128; st > 0; st >>= 1) {
        __syncthreads();
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    }
    __syncthreads();
    const double rms = sqrt(red[0] / double(npix));
    const float inv = rms > 0.0 ? float(1.0 / rms) : 0.0f;
    float2* ob = out + size_t(blockIdx.x) * npix;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) ob[p] = make_float2(eb[p].x * inv, eb[p].y * inv);
    if (threadIdx.x == 0) log_rms[blockIdx.x] = rms > 0.0 ? float(log(rms)) : -1e30f;
}

template <typename T>
T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

int check_act(const Dims& d, void* act, size_t act_bytes, const char* who, Act& a) {
    a = act_layout(d);
    if (!act) return rsi_fail(RSI_E_INVAL, "%s: null workspace", who);
    if (reinterpret_cast<uintptr_t>(act) % 256) return rsi_fail(RSI_E_INVAL, "%s: workspace not 256-byte aligned", who);
    if (act_bytes < a.total) return rsi_fail(RSI_E_NOMEM, "%s: workspace %zu < %zu bytes", who, act_bytes, a.total);
    return RSI_OK;
}

int hidden_forward(const rsi_nn_net& n, const Dims& d, const Act& a, const bf16* w16, const float* w32, void* act,
                   cudaStream_t s) {
    for (int l = 0; l < d.D; ++l) {
        int rc = rsi_nn_gemm(RSI_NN_EPI_BIAS_SILU, n.engine, 0, at<bf16>(act, a.h[l]), w16 + w_off(d, l), d.R, d.W,
                             in_of(d, l), w32 + b_off(d, l), nullptr, at<float>(act, a.z[l + 1]),
                             at<bf16>(act, a.h[l + 1]), 1, nullptr, s);
        if (rc != RSI_OK) return rc;
    }
    // four CTAs of 8 warps per SM, each warp walking rows
    const unsigned blocks = unsigned(std::min<int64_t>((d.R + 7) / 8, int64_t(4) * rsi_num_sms()));
    const bf16* hD = at<bf16>(act, a.h[d.D]);
    const float *whd = w32 + w_off(d, d.D), *bhd = w32 + b_off(d, d.D);
    float4* yv = at<float4>(act, a.y);
    if (d.W <= 256)
        head_fwd_kernel<1><<<blocks, 256, 0, s>>>(hD, d.W, d.R, whd, bhd, yv);
    else if (d.W == 512)
        head_fwd_kernel<2><<<blocks, 256, 0, s>>>(hD, d.W, d.R, whd, bhd, yv);
    else
        head_fwd_kernel<4><<<blocks, 256, 0, s>>>(hD, d.W, d.R, whd, bhd, yv);
    RSI_CHECK_LAUNCH("head_fwd_kernel");
    return RSI_OK;
}

}  // namespace

extern "C" int64_t rsi_nn_param_elems(const rsi_nn_net* net) {
    Dims d;
    if (dims_of(net, d, "rsi_nn_param_elems") != RSI_OK) return -1;
    return param_elems(d);
}

extern "C" int64_t rsi_nn_param_offset(const rsi_nn_net* net, int32_t layer, int32_t bias) {
    Dims d;
    if (dims_of(net, d, "rsi_nn_param_offset") != RSI_OK) return -1;
    if (layer < 0 || layer > d.D || (bias != 0 && bias != 1)) return -1;
    return bias ? b_off(d, layer) : w_off(d, layer);
}

extern "C" size_t rsi_nn_act_bytes(const rsi_nn_net* net) {
    Dims d;
    if (dims_of(net, d, "rsi_nn_act_bytes") != RSI_OK) return 0;
    return act_layout(d).total;
}

extern "C" int rsi_nn_rows(const rsi_nn_net* net, const double* params, int64_t n_fields, int32_t mode,
                           uint64_t seed, const uint64_t* seed_dev, int64_t first, const float* targets,
                           const float* log_rms, void* act, size_t act_bytes, void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_rows");
    if (rc != RSI_OK) return rc;
    Act a;
    if ((rc = check_act(d, act, act_bytes, "rsi_nn_rows", a)) != RSI_OK) return rc;
    if (!params || !net->fmat || n_fields < 1 || n_fields > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_rows: bad parameters or Fourier matrix");
    if (mode != RSI_NN_ROWS_RANDOM && mode != RSI_NN_ROWS_PIXELS)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_rows: unknown mode %d", mode);
    if (mode == RSI_NN_ROWS_PIXELS && (first < 0 || first >= n_fields * int64_t(d.npix)))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_rows: first row outside the fields' pixels");
    if (bool(targets) != bool(log_rms)) return rsi_fail(RSI_E_INVAL, "rsi_nn_rows: targets need log_rms");
    const RowK k = row_consts(*net, d);
    const int warps = 8;
    const size_t smem = size_t(d.F) * RSI_NN_IN * sizeof(float);
    if (smem > 48 * 1024) return rsi_fail(RSI_E_INVAL, "rsi_nn_rows: n_freq too large");
    rows_kernel<<<unsigned((d.R + warps - 1) / warps), 32 * warps, smem, static_cast<cudaStream_t>(stream)>>>(
        k, params, n_fields, mode, seed, seed_dev, first, targets, log_rms, d.R, at<bf16>(act, a.h[0]),
        at<float4>(act, a.t));
    RSI_CHECK_LAUNCH("rows_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_forward(const rsi_nn_net* net, const void* w16, const float* w32, void* act, size_t act_bytes,
                              float* y, void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_forward");
    if (rc != RSI_OK) return rc;
    Act a;
    if ((rc = check_act(d, act, act_bytes, "rsi_nn_forward", a)) != RSI_OK) return rc;
    if (!w16 || !w32) return rsi_fail(RSI_E_INVAL, "rsi_nn_forward: null weights");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = hidden_forward(*net, d, a, static_cast<const bf16*>(w16), w32, act, s);
    if (rc != RSI_OK) return rc;
    if (y)
        RSI_CUDA_TRY(cudaMemcpyAsync(y, at<float>(act, a.y), size_t(d.R) * 4 * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s),
                     "rsi_nn_forward: copy of the outputs");
    return RSI_OK;
}

extern "C" int rsi_nn_backward(const rsi_nn_net* net, const void* w16, const float* w32, void* act, size_t act_bytes,
                               float* grad, float* loss_dev, void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_backward");
    if (rc != RSI_OK) return rc;
    Act a;
    if ((rc = check_act(d, act, act_bytes, "rsi_nn_backward", a)) != RSI_OK) return rc;
    if (!w16 || !w32 || !grad) return rsi_fail(RSI_E_INVAL, "rsi_nn_backward: null weights or gradient");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16* W16 = static_cast<const bf16*>(w16);
    // head: dZ_D and the head's gradients (loss = sum (y - t)^2 / (4 rows))
    const float g = 2.0f / (4.0f * float(d.R));
    int cur = 0;
    const size_t smem = (size_t(kHead) * d.W * (1 + 256 / (d.W / 8)) + 4 * kHeadRows) * sizeof(float);
    head_bwd_kernel<<<unsigned(a.head_chunks), 256, smem, s>>>(
        at<bf16>(act, a.h[d.D]), at<float>(act, a.z[d.D]), d.W, at<float4>(act, a.y), at<float4>(act, a.t),
        w32 + w_off(d, d.D), g, at<bf16>(act, a.dz[cur]), at<float>(act, a.part));
    RSI_CHECK_LAUNCH("head_bwd_kernel");
    const int n_part = kHead * d.W + kHead + 1;
    chunk_sum_kernel<<<unsigned((n_part + 31) / 32), dim3(32, 8), 0, s>>>(
        at<float>(act, a.part), a.head_chunks, n_part, kHead * d.W, kHead, 1.0f / (4.0f * float(d.R)),
        grad + w_off(d, d.D), grad + b_off(d, d.D), loss_dev);
    RSI_CHECK_LAUNCH("chunk_sum_kernel");
    // hidden layers, last to first: gW_l = dZ^T H_{l-1}, gb_l = colsum(dZ),
    // dZ_{l-1} = (dZ W_l) * silu'(Z_{l-1})
    for (int l = d.D - 1; l >= 0; --l) {
        const bf16* dZ = at<bf16>(act, a.dz[cur]);
        rc = rsi_nn_gemm(RSI_NN_EPI_F32, RSI_NN_ENGINE_TCGEN05, RSI_NN_A_T | RSI_NN_B_T, dZ, at<bf16>(act, a.h[l]),
                         d.W, in_of(d, l), d.R, nullptr, nullptr, grad + w_off(d, l), nullptr, a.splits,
                         at<float>(act, a.work), s);
        if (rc != RSI_OK) return rc;
        // bias gradient: column sums of dZ over the rows (two passes, fixed order)
        const int chunks = (d.R + kColRows - 1) / kColRows;
        colsum_part_kernel<<<dim3(unsigned((d.W + 511) / 512), unsigned(chunks)), 256, 0, s>>>(
            dZ, d.R, d.W, at<float>(act, a.colpart));
        RSI_CHECK_LAUNCH("colsum_part_kernel");
        chunk_sum_kernel<<<unsigned((d.W + 31) / 32), dim3(32, 8), 0, s>>>(
            at<float>(act, a.colpart), chunks, d.W, 0, d.W, 0.0f, nullptr, grad + b_off(d, l), nullptr);
        RSI_CHECK_LAUNCH("chunk_sum_kernel");
        if (l > 0) {
            rc = rsi_nn_gemm(RSI_NN_EPI_DSILU, RSI_NN_ENGINE_TCGEN05, RSI_NN_B_T, dZ, W16 + w_off(d, l), d.R,
                             in_of(d, l), d.W, nullptr, at<float>(act, a.z[l]), nullptr, at<bf16>(act, a.dz[1 - cur]),
                             1, nullptr, s);
            if (rc != RSI_OK) return rc;
            cur = 1 - cur;
        }
    }
    return RSI_OK;
}

extern "C" int rsi_nn_adam_step(const rsi_nn_net* net, float* w32, float* m, float* v, const float* grad, void* w16,
                                const float* hyper, float beta1, float beta2, float eps, void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_adam_step");
    if (rc != RSI_OK) return rc;
    return rsi_nn_adam_dev(w32, m, v, grad, param_elems(d), hyper, beta1, beta2, eps, w16, stream);
}

extern "C" int rsi_nn_targets(const rsi_nn_net* net, const double* params, int32_t n_fields, const float* images,
                              double* carrier, float* params_f32, float* env, float* targets, float* log_rms,
                              void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_targets");
    if (rc != RSI_OK) return rc;
    if (!params || !images || !carrier || !params_f32 || !env || !targets || !log_rms || n_fields < 1)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_targets: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = rsi_nn_carrier_coeffs(params, n_fields, net->c1, net->c2, carrier, params_f32, stream);
    if (rc != RSI_OK) return rc;
    rc = rsi_nn_carrier(carrier, n_fields, &net->window, -1, 1.0f, images, env, stream);
    if (rc != RSI_OK) return rc;
    targets_kernel<<<unsigned(n_fields), 256, 0, s>>>(reinterpret_cast<const float2*>(env), d.npix,
                                                      reinterpret_cast<float2*>(targets), log_rms);
    RSI_CHECK_LAUNCH("targets_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_infer(const rsi_nn_net* net, const void* w16, const float* w32, const double* params,
                            int32_t n_fields, void* act, size_t act_bytes, double* carrier, float* out, void* stream) {
    Dims d;
    int rc = dims_of(net, d, "rsi_nn_infer");
    if (rc != RSI_OK) return rc;
    Act a;
    if ((rc = check_act(d, act, act_bytes, "rsi_nn_infer", a)) != RSI_OK) return rc;
    if (!w16 || !w32 || !params || !carrier || !out || n_fields < 1)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_infer: bad arguments");
    if (d.R % d.npix) return rsi_fail(RSI_E_INVAL, "rsi_nn_infer: rows must be a multiple of the window's pixels");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int per = d.R / d.npix;  // fields per chunk
    for (int f0 = 0; f0 < n_fields; f0 += per) {
        const int nf = std::min(per, n_fields - f0);
        rc = rsi_nn_rows(net, params, n_fields, RSI_NN_ROWS_PIXELS, 0, nullptr, int64_t(f0) * d.npix, nullptr,
                         nullptr, act, act_bytes, stream);
        if (rc != RSI_OK) return rc;
        rc = hidden_forward(*net, d, a, static_cast<const bf16*>(w16), w32, act, s);
        if (rc != RSI_OK) return rc;
        assemble_kernel<<<unsigned(nf), 256, 0, s>>>(at<float4>(act, a.y), d.npix, at<float2>(act, a.env));
        RSI_CHECK_LAUNCH("assemble_kernel");
        rc = rsi_nn_carrier_coeffs(params + 5 * size_t(f0), nf, net->c1, net->c2, carrier + 4 * size_t(f0),
                                   at<float>(act, a.p32), stream);
        if (rc != RSI_OK) return rc;
        rc = rsi_nn_carrier(carrier + 4 * size_t(f0), nf, &net->window, +1, 1.0f, at<float>(act, a.env),
                            out + 2 * size_t(f0) * d.npix, stream);
        if (rc != RSI_OK) return rc;
    }
    return RSI_OK;
}
