// nn.cu -- step a9: kernels of the learned surrogate, a Fourier-feature MLP
// (not in the paper) that maps transducer offset, tilt, water path,
// frequency and image depth to the carrier-demodulated field image of the
// RSI chain, trained on fields the RSI kernels compute.
//
//   features   u = 2 (p - lo)/(hi - lo) - 1, h0 = [sin(pi B u), cos(pi B u)]  (bf16)
//   gemm       C[M x N] = A[M x K] B[N x K]^T on BF16 tensor cores with FP32
//              accumulation, two engines: tcgen05 (TMA-fed, 128-byte
//              swizzled stages, UMMA 128 x {256, 128, 64} x 16 into tensor
//              memory, a producer lane and an MMA lane on mbarriers) and
//              mma.sync (m16n8k16 fragments via ldmatrix, 3-stage cp.async
//              pipeline); both with split K and the fused epilogues:
//                F32        C (+ bias)                       -> f32
//                BIAS_SILU  z = C + bias -> f32 z, bf16 silu(z)
//                DSILU      C * silu'(aux)                   -> bf16   (backprop)
//              and, tcgen05 only, the output layer with the carrier:
//                CARRIER    scale exp(+-i psi) (C + bias)    -> f32   (inference)
//   transpose  bf16 [R x C] -> [C x R]
//   loss       mean (y - t)^2 and its gradient 2 (y - t)/n  -> bf16
//   colsum     bias gradients (column sums of a bf16 matrix)
//   adam       Kingma & Ba (2015) on FP32 master weights, bf16 copy out; the
//              schedule by value or from device memory (a replayed graph)
//   carrier    multiply an image by exp(+-i psi), psi = kx x + kz z + phi0;
//              the coefficients (kx, kz, phi0) from the parameters in FP64
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "rsi_internal.cuh"
#include "umma.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3, GEMM_THREADS = 256;
constexpr int LDS = BK + 8;  // padded smem row (bf16): 80 bytes, conflict-free ldmatrix
constexpr size_t GEMM_SMEM = size_t(STAGES) * (BM + BN) * LDS * sizeof(bf16);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, const void* smem) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(smem)));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// logistic sigmoid with the fast reciprocal division (a few ulp; the results
// are rounded to bf16): no IEEE division and its slow-path branch in the
// epilogue of every hidden layer.  Past z = -87 exp(-z) is infinite and the
// quotient the limit 0.
__device__ __forceinline__ float sigmoidf_(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_(float z) { return z * sigmoidf_(z); }
__device__ __forceinline__ float dsilu_(float z) {
    float s = sigmoidf_(z);
    return s * (1.0f + z * (1.0f - s));
}

// epilogue of one pair of neighbouring outputs (row, col), (row, col + 1)
template <int EPI>
__device__ __forceinline__ void epilogue2(float v0, float v1, size_t o, int col, const float* __restrict__ bias,
                                          const float* __restrict__ aux, float* __restrict__ outf,
                                          bf16* __restrict__ outh) {
    if (EPI == 0) {  // F32 (+ bias)
        if (bias) {
            v0 += bias[col];
            v1 += bias[col + 1];
        }
        *reinterpret_cast<float2*>(outf + o) = make_float2(v0, v1);
    } else if (EPI == 1) {  // BIAS_SILU
        v0 += bias[col];
        v1 += bias[col + 1];
        *reinterpret_cast<float2*>(outf + o) = make_float2(v0, v1);
        *reinterpret_cast<__nv_bfloat162*>(outh + o) = __floats2bfloat162_rn(silu_(v0), silu_(v1));
    } else {  // DSILU
        const float2 z = *reinterpret_cast<const float2*>(aux + o);
        *reinterpret_cast<__nv_bfloat162*>(outh + o) = __floats2bfloat162_rn(v0 * dsilu_(z.x), v1 * dsilu_(z.y));
    }
}

// M % 128 == 0, N % 128 == 0, K % 32 == 0 (checked on the host).  With
// gridDim.z > 1 (split K), CTA z covers k-tiles [z*kts, (z+1)*kts) and writes
// plain FP32 partial sums to outf + z*M*N; splitk_reduce_kernel finishes.
template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS)
    gemm_tn_kernel(const bf16* __restrict__ A, const bf16* __restrict__ B, int M, int N, int K,
                   const float* __restrict__ bias, const float* __restrict__ aux, float* __restrict__ outf,
                   bf16* __restrict__ outh, int kts) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    bf16* sA = reinterpret_cast<bf16*>(smem_raw);
    bf16* sB = sA + STAGES * BM * LDS;
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    auto load_stage = [&](int stage, int k0) {
#pragma unroll
        for (int c = tid; c < BM * BK / 8; c += GEMM_THREADS) {
            const int row = c >> 2, col = (c & 3) * 8;
            cp_async16(&sA[(stage * BM + row) * LDS + col], &A[size_t(bm + row) * K + k0 + col]);
            cp_async16(&sB[(stage * BN + row) * LDS + col], &B[size_t(bn + row) * K + k0 + col]);
        }
    };
    const int kt0 = blockIdx.z * kts;
    const int KT = min(K / BK - kt0, kts);
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < KT) load_stage(s, (kt0 + s) * BK);
        cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int nk = kt + STAGES - 1;
        if (nk < KT) load_stage(nk % STAGES, (kt0 + nk) * BK);
        cp_async_commit();
        const int st = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[4][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int row = wm + mi * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
                ldmatrix_x4(a[mi], &sA[(st * BM + row) * LDS + col]);
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int row = wn + nj * 16 + (lane >> 4) * 8 + (lane & 7), col = kk + ((lane >> 3) & 1) * 8;
                uint32_t r[4];
                ldmatrix_x4(r, &sB[(st * BN + row) * LDS + col]);
                b[2 * nj][0] = r[0];
                b[2 * nj][1] = r[1];
                b[2 * nj + 1][0] = r[2];
                b[2 * nj + 1][1] = r[3];
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
        }
    }
    cp_async_wait<0>();

#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int row = bm + wm + mi * 16 + (lane >> 2) + half * 8;
                const int col = bn + wn + ni * 8 + (lane & 3) * 2;
                const size_t o = size_t(row) * N + col;
                const float v0 = acc[mi][ni][2 * half], v1 = acc[mi][ni][2 * half + 1];
                if (gridDim.z > 1)
                    *reinterpret_cast<float2*>(outf + size_t(blockIdx.z) * M * N + o) = make_float2(v0, v1);
                else
                    epilogue2<EPI>(v0, v1, o, col, bias, aux, outf, outh);
            }
}

// sums the split-K partial sums in split order, then applies the epilogue
template <int EPI>
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M, int N,
                                     const float* __restrict__ bias, const float* __restrict__ aux,
                                     float* __restrict__ outf, bf16* __restrict__ outh) {
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // pair index
    const int64_t total = int64_t(M) * N / 2;
    if (q >= total) return;
    const size_t o = size_t(q) * 2;
    float v0 = 0.0f, v1 = 0.0f;
    for (int z = 0; z < splits; ++z) {
        const float2 p = *reinterpret_cast<const float2*>(part + size_t(z) * M * N + o);
        v0 += p.x;
        v1 += p.y;
    }
    epilogue2<EPI>(v0, v1, o, int(o % size_t(N)), bias, aux, outf, outh);
}

// epilogue of four neighbouring outputs (row, col .. col + 3); o, col % 4 == 0
template <int EPI>
__device__ __forceinline__ void epilogue4(float4 v, size_t o, int col, const float* __restrict__ bias,
                                          const float* __restrict__ aux, float* __restrict__ outf,
                                          bf16* __restrict__ outh) {
    if (EPI != 2 && bias) {
        const float4 b = *reinterpret_cast<const float4*>(bias + col);
        v.x += b.x;
        v.y += b.y;
        v.z += b.z;
        v.w += b.w;
    }
    if (EPI != 2) *reinterpret_cast<float4*>(outf + o) = v;
    if (EPI == 1) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(silu_(v.x), silu_(v.y));
        __nv_bfloat162 h1 = __floats2bfloat162_rn(silu_(v.z), silu_(v.w));
        uint2 u = make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1));
        *reinterpret_cast<uint2*>(outh + o) = u;
    } else if (EPI == 2) {
        const float4 z = *reinterpret_cast<const float4*>(aux + o);
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x * dsilu_(z.x), v.y * dsilu_(z.y));
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z * dsilu_(z.z), v.w * dsilu_(z.w));
        uint2 u = make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1));
        *reinterpret_cast<uint2*>(outh + o) = u;
    }
}

// ---------------------------------------------------------------------------
// tcgen05 engine: a persistent kernel, one CTA per SM, looping over output
// tiles of 128 x TBN (and, with split K, over K ranges).  Warp roles:
//   warp 0, one lane   TMA producer: A and B k-tiles (64 wide, 128 bytes of
//                      bf16 = one 128-byte swizzle row) into a ring of
//                      TC_STAGES shared-memory stages, completing on the
//                      stage's `full` barrier
//   warp 1, one lane   MMA issuer: waits for `full`, issues four
//                      128 x TBN x 16 tcgen05.mma into one of two tensor-
//                      memory accumulators, commits them to the stage's
//                      `empty` barrier (frees the stage) and, after a tile's
//                      last k-tile, to the accumulator's `acc_full` barrier
//   warps 2-9          epilogue, two warps per 32-lane quarter of tensor
//                      memory (each takes half the columns): tcgen05.ld of
//                      32 x 32 blocks into registers, then `acc_empty` frees
//                      the accumulator, so the epilogue of one tile overlaps
//                      the main loop of the next.  F32 output (and split-K
//                      partial sums) leave as TMA bulk stores of the block
//                      staged in the 128-byte-swizzled layout; the other
//                      epilogues go through shared memory into
//                      row-contiguous stores.
// Every wait is bounded; on a timeout all roles stop, the CTA drains its
// copies and MMAs, frees tensor memory and records RSI_DEV_TIMEOUT.
// ---------------------------------------------------------------------------
#ifndef RSI_TC_STAGES
#define RSI_TC_STAGES 4  // operand ring depth (4 x 48 KB with 256-wide tiles fills shared memory)
#endif
constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = RSI_TC_STAGES, TC_EPI_WARPS = 8,
              TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;
// epilogue staging: per warp 32 rows x 32 floats, 16-byte chunk j of row r
// stored at chunk j ^ (r & 7) (conflict-free row writes and column reads)
constexpr uint32_t TC_EPI_BYTES = TC_EPI_WARPS * 32 * 32 * 4;

// Output-layer epilogue with the carrier (EPI 3): each output row is one
// image of interleaved complex pixels on a window of nx columns; the epilogue
// multiplies pixel (ix, iz) of row b by scale exp(sign i psi_b(ix, iz)),
// psi_b / 2 pi = a_b + ix u_b + iz w_b (turns), with a, u, w from the
// row's coefficients (kx, kz, phi0) in FP64, as the carrier pass forms them.
struct CarrierArgs {
    const double* coef;  // [M][4] (kx, kz, phi0, unused)
    const float4* rows;  // [M][2]: each row's CarrierRow, formed once per call by carrier_rows_kernel
    int nx, sign;
    float scale;
    double x0, dx, z0, dz;
};
struct CarrierRow {
    float ah, al, uh, ul, wh, wl;  // turns, split into float pairs
    float rc, rs;                  // exp(2 pi i u): one pixel step in x
};
__device__ __forceinline__ float frac_mul_(float i, float h, float l) {
    const float p = i * h;
    const float e = fmaf(i, h, -p);
    return ((p - rintf(p)) + e) + i * l;
}
__device__ __forceinline__ CarrierRow carrier_row(const CarrierArgs& ca, int row) {
    const double* cb = ca.coef + 4 * size_t(row);
    const double inv2pi = 0.15915494309189535;  // 1 / (2 pi)
    double ad = (cb[2] + cb[0] * (ca.x0 + 0.5 * ca.dx) + cb[1] * (ca.z0 + 0.5 * ca.dz)) * inv2pi;
    ad -= rint(ad);
    double ud = cb[0] * ca.dx * inv2pi;
    const double wd = cb[1] * ca.dz * inv2pi;
    CarrierRow r;
    r.ah = float(ad);
    r.al = float(ad - double(r.ah));
    r.uh = float(ud);
    r.ul = float(ud - double(r.uh));
    r.wh = float(wd);
    r.wl = float(wd - double(r.wh));
    ud -= rint(ud);
    sincospif(2.0f * float(ud), &r.rs, &r.rc);  // accurate: the block's rotations build on it
    return r;
}
// exp(i 2 pi (a + ix u + iz w)) with the phase reduced as in the carrier pass
__device__ __forceinline__ void carrier_phase(const CarrierRow& r, int ix, int iz, float& c, float& s) {
    float t = (r.ah + frac_mul_(float(ix), r.uh, r.ul)) + frac_mul_(float(iz), r.wh, r.wl);
    t = (t - rintf(t)) + r.al;
    __sincosf(6.283185307179586f * t, &s, &c);
}

// the surrogate's carrier coefficients from its parameters (x-offset, tilt,
// water path, frequency, image depth), one row per sample, in FP64: the
// refracted plane wave's wavenumber components kx = k2 s, kz = k2 c and the
// phase phi0 = k1 L + k2 c depth at the window's origin, s = (c2/c1) sin(tilt),
// c = sqrt(max(0, 1 - s^2)); also the FP32 copy of the parameters
__global__ void carrier_coeffs_kernel(const double* __restrict__ p, int batch, double c1, double c2,
                                      double* __restrict__ coef, float* __restrict__ pf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double* q = p + 5 * size_t(b);
    const double twopi = 6.283185307179586;
    const double k1 = twopi * q[3] / c1, k2 = twopi * q[3] / c2;
    const double s = c2 / c1 * sin(q[1]);
    const double c = sqrt(fmax(1.0 - s * s, 0.0));
    coef[4 * size_t(b)] = k2 * s;
    coef[4 * size_t(b) + 1] = k2 * c;
    coef[4 * size_t(b) + 2] = k1 * q[2] + k2 * c * q[4];
    coef[4 * size_t(b) + 3] = 0.0;
    for (int j = 0; j < 5; ++j) pf[5 * size_t(b) + j] = float(q[j]);
}

// the per-row constants of the fused output layer, once per call
__global__ void carrier_rows_kernel(CarrierArgs ca, int M, float4* __restrict__ rows) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= M) return;
    const CarrierRow r = carrier_row(ca, b);
    rows[2 * b] = make_float4(r.ah, r.al, r.uh, r.ul);
    rows[2 * b + 1] = make_float4(r.wh, r.wl, r.rc, r.rs);
}

template <int TBN>
struct TcCfg {
    static constexpr uint32_t B_BYTES = TBN * TC_BK * 2;
    static constexpr uint32_t STAGE = TC_A_BYTES + B_BYTES;
    static constexpr size_t SMEM = size_t(TC_STAGES) * STAGE + TC_EPI_BYTES + 1024;  // + alignment slack
    static constexpr uint32_t IDESC = rsi_umma::idesc_bf16_f32(TC_BM, TBN);
};

struct TcTile {
    int m0, n0, kt0, KT, z;
};
// tile t -> (m, n, split): groups of up to 16 row blocks sweep N together so
// that CTAs running at the same time share A and B tiles in L2
__device__ __forceinline__ TcTile tc_tile(int t, int m_tiles, int n_tiles, int TBN, int kt_total, int kts) {
    const int mn = m_tiles * n_tiles;
    const int z = t / mn, r = t - z * mn;
    const int G = 16, g = r / (G * n_tiles), w = r - g * G * n_tiles;
    const int gm = min(G, m_tiles - g * G);
    TcTile T;
    T.m0 = (g * G + w % gm) * TC_BM;
    T.n0 = (w / gm) * TBN;
    T.z = z;
    T.kt0 = z * kts;
    T.KT = min(kt_total - T.kt0, kts);
    return T;
}

template <int EPI, int TBN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmH, int M, int N,
                   int K, int layout, const float* __restrict__ bias, const float* __restrict__ aux, int kts,
                   int splits, CarrierArgs car, int* status) {
    // layout bit 0: A is stored [K x M] (MN-major), bit 1: B is stored [K x N]
    const bool a_mn = layout & 1, b_mn = layout & 2;
    // outputs leave by TMA stores: f32 (F32, BIAS_SILU's z, split-K partial
    // sums) through tmC over [splits*M x N], bf16 (BIAS_SILU, DSILU) through tmH
    using C = TcCfg<TBN>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m_tiles = M / TC_BM, n_tiles = N / TBN, kt_total = K / TC_BK;
    const int total = m_tiles * n_tiles * splits;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;  // swizzle atoms need 1024-B alignment
    float* epi_buf = reinterpret_cast<float*>(smem_raw + (base - smem_u32(smem_raw)) + TC_STAGES * C::STAGE);

    if (warp == 0) {
        rsi_umma::tmem_alloc(smem_u32(&tmem_slot), 2 * TBN);
        rsi_umma::tmem_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&acc_full[a]), 1);
            mbar_init(smem_u32(&acc_empty[a]), TC_EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&done), 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (tid == 64) {
        rsi_umma::prefetch_tmap(&tmA);
        rsi_umma::prefetch_tmap(&tmB);
        if (EPI != 2 || splits > 1) rsi_umma::prefetch_tmap(&tmC);
        if ((EPI == 1 || EPI == 2) && splits == 1) rsi_umma::prefetch_tmap(&tmH);  // bf16 outputs only
    }
    rsi_umma::fence_before_sync();
    __syncthreads();
    rsi_umma::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // producer
            int it = 0;
            for (int t = blockIdx.x; t < total && !abort_flag; t += gridDim.x) {
                const TcTile T = tc_tile(t, m_tiles, n_tiles, TBN, kt_total, kts);
                for (int kt = 0; kt < T.KT; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    if (it >= TC_STAGES &&
                        !mbar_wait_bounded(smem_u32(&empty[s]), uint32_t(it / TC_STAGES - 1) & 1u)) {
                        abort_flag = 1;
                        break;
                    }
                    const uint32_t sa = base + uint32_t(s) * C::STAGE;
                    mbar_expect_tx(smem_u32(&full[s]), C::STAGE);
                    const int k0 = (T.kt0 + kt) * TC_BK;
                    if (a_mn)  // boxes of 64 M x 64 K, 8 KB apart
                        for (int j = 0; j < TC_BM / 64; ++j)
                            rsi_umma::tma_load_2d(sa + j * 8192u, &tmA, T.m0 + 64 * j, k0, smem_u32(&full[s]));
                    else
                        rsi_umma::tma_load_2d(sa, &tmA, k0, T.m0, smem_u32(&full[s]));
                    if (b_mn)
                        for (int j = 0; j < TBN / 64; ++j)
                            rsi_umma::tma_load_2d(sa + TC_A_BYTES + j * 8192u, &tmB, T.n0 + 64 * j, k0,
                                                  smem_u32(&full[s]));
                    else
                        rsi_umma::tma_load_2d(sa + TC_A_BYTES, &tmB, k0, T.n0, smem_u32(&full[s]));
                }
            }
            // the copies still in flight land before the CTA can exit
            for (int j = max(0, it - TC_STAGES); j < it; ++j)
                if (!mbar_wait_bounded(smem_u32(&full[j % TC_STAGES]), uint32_t(j / TC_STAGES) & 1u))
                    abort_flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = C::IDESC | (uint32_t(a_mn) << 15) | (uint32_t(b_mn) << 16);
            int it = 0, tc = 0;
            for (int t = blockIdx.x; t < total && !abort_flag; t += gridDim.x, ++tc) {
                const TcTile T = tc_tile(t, m_tiles, n_tiles, TBN, kt_total, kts);
                const int acc = tc & 1;
                if (tc >= 2 && !mbar_wait_bounded(smem_u32(&acc_empty[acc]), uint32_t(tc / 2 - 1) & 1u)) {
                    abort_flag = 1;
                    break;
                }
                rsi_umma::fence_after_sync();
                const uint32_t d = tmem + uint32_t(acc * TBN);
                bool ok = true;
                for (int kt = 0; kt < T.KT; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    if (!mbar_wait_bounded(smem_u32(&full[s]), uint32_t(it / TC_STAGES) & 1u)) {
                        ok = false;
                        break;
                    }
                    rsi_umma::fence_after_sync();
                    const uint32_t sa = base + uint32_t(s) * C::STAGE, sb = sa + TC_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        const uint64_t da = a_mn ? rsi_umma::smem_desc_mn_sw128(sa + kk * 2048, 8192)
                                                 : rsi_umma::smem_desc_sw128(sa + kk * 32);
                        const uint64_t db = b_mn ? rsi_umma::smem_desc_mn_sw128(sb + kk * 2048, 8192)
                                                 : rsi_umma::smem_desc_sw128(sb + kk * 32);
                        rsi_umma::mma_f16(d, da, db, idesc, (kt | kk) != 0);
                    }
                    rsi_umma::commit(smem_u32(&empty[s]));
                }
                if (!ok) {
                    abort_flag = 1;
                    break;
                }
                rsi_umma::commit(smem_u32(&acc_full[acc]));
            }
            rsi_umma::commit(smem_u32(&done));  // arrives when every MMA issued above has completed
        }
    } else {  // epilogue warps 2..9: TMEM lane quarter q = warp % 4, column half h
        const int q = warp & 3, h = (warp - 2) >> 2;
        float* buf = epi_buf + (warp - 2) * 32 * 32;
        int tc = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tc) {
            if (__any_sync(0xffffffffu, abort_flag)) break;  // warp-uniform: tcgen05.ld below is .sync.aligned
            const TcTile T = tc_tile(t, m_tiles, n_tiles, TBN, kt_total, kts);
            const int acc = tc & 1;
            // this warp's TBN/2 bias values, one float4 per lane, loaded before
            // the accumulator wait so that their latency (L2, under the full
            // load of the operand and output streams) hides behind it; each
            // block takes its 32 values from the lanes by shuffles
            const bool add_bias = EPI != 2 && splits == 1 && bias != nullptr;
            float4 bq = make_float4(0.f, 0.f, 0.f, 0.f);
            if (add_bias && 4 * lane < TBN / 2)
                bq = __ldg(reinterpret_cast<const float4*>(bias + T.n0 + h * (TBN / 2)) + lane);
            CarrierRow crow;  // this lane's image (row) constants, loaded while the MMAs run
            if (EPI == 3) {
                const float4 c0 = __ldg(car.rows + 2 * (T.m0 + q * 32 + lane));
                const float4 c1 = __ldg(car.rows + 2 * (T.m0 + q * 32 + lane) + 1);
                crow.ah = c0.x, crow.al = c0.y, crow.uh = c0.z, crow.ul = c0.w;
                crow.wh = c1.x, crow.wl = c1.y, crow.rc = c1.z, crow.rs = c1.w;
            }
            const bool ok = mbar_wait_bounded(smem_u32(&acc_full[acc]), uint32_t(tc / 2) & 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                abort_flag = 1;
                break;
            }
            rsi_umma::fence_after_sync();
            const uint32_t sbuf = smem_u32(buf);  // 1024-byte aligned: 32 rows of 128 B, 128-byte swizzle atoms
            const int row0 = T.m0 + q * 32;       // this warp's first output row; lane = row - row0
#pragma unroll 1
            for (int cb = h * (TBN / 2); cb < (h + 1) * (TBN / 2); cb += 32) {
                const int col0 = T.n0 + cb;
                float a[32];
                if (EPI == 2 && splits == 1) {  // the pre-activations this row's outputs need, ahead of the TMEM read
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 z = *reinterpret_cast<const float4*>(aux + size_t(row0 + lane) * N + col0 + 4 * i);
                        a[4 * i] = z.x;
                        a[4 * i + 1] = z.y;
                        a[4 * i + 2] = z.z;
                        a[4 * i + 3] = z.w;
                    }
                }
                float v[32];
                rsi_umma::ld_32x32b_x32(tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * TBN + cb), v);
                if (cb + 32 == (h + 1) * (TBN / 2)) {  // this warp's last read of the accumulator
                    rsi_umma::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
                }
                if (add_bias) {
                    const int src = (cb - h * (TBN / 2)) / 4;  // the lane holding columns col0 .. col0 + 3
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        v[4 * i] += __shfl_sync(0xffffffffu, bq.x, src + i);
                        v[4 * i + 1] += __shfl_sync(0xffffffffu, bq.y, src + i);
                        v[4 * i + 2] += __shfl_sync(0xffffffffu, bq.z, src + i);
                        v[4 * i + 3] += __shfl_sync(0xffffffffu, bq.w, src + i);
                    }
                }
                if (EPI == 3) {  // 16 complex pixels of this row's image: one exact phase, then rotations
                    int p = col0 >> 1;
                    int iz = p / car.nx, ix = p - iz * car.nx;  // the same for every lane (same columns)
                    // e = scale exp(sign i psi) as (c, s); a pixel's value (re, im) becomes
                    // re (c, s) + im (-s, c); one step in x multiplies e by (rc, sign rs).
                    // Both products run two lanes at a time (f32x2).
                    const float2 rot = make_float2(crow.rc, car.sign > 0 ? crow.rs : -crow.rs);
                    const float2 nrot = make_float2(-rot.y, rot.x);
                    float2 e;
                    carrier_phase(crow, ix, iz, e.x, e.y);
                    e = make_float2(e.x * car.scale, (car.sign > 0 ? e.y : -e.y) * car.scale);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float2 o = __ffma2_rn(make_float2(v[2 * k], v[2 * k]), e,
                                                    __fmul2_rn(make_float2(v[2 * k + 1], v[2 * k + 1]),
                                                               make_float2(-e.y, e.x)));
                        v[2 * k] = o.x;
                        v[2 * k + 1] = o.y;
                        if (k < 15) {
                            if (++ix == car.nx) {  // next image row: restart from the exact phase
                                ix = 0;
                                ++iz;
                                carrier_phase(crow, ix, iz, e.x, e.y);
                                e = make_float2(e.x * car.scale, (car.sign > 0 ? e.y : -e.y) * car.scale);
                            } else {
                                e = __ffma2_rn(make_float2(e.x, e.x), rot, __fmul2_rn(make_float2(e.y, e.y), nrot));
                            }
                        }
                    }
                }
                if (EPI != 2 || splits > 1) {  // f32 block: output, z, or partial sums of split T.z
                    if (lane == 0) rsi_umma::bulk_wait_read0();  // the previous block has left buf
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<float4*>(buf + lane * 32 + 4 * (i ^ (lane & 7))) =
                            make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    rsi_umma::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        rsi_umma::tma_store_2d(&tmC, col0, T.z * M + row0, sbuf);
                        rsi_umma::bulk_commit();
                    }
                }
                if ((EPI == 1 || EPI == 2) && splits == 1) {  // bf16 block (dense 64-byte rows): silu(z) or C * silu'(aux)
                    uint32_t hw[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float x0 = EPI == 1 ? silu_(v[2 * j]) : v[2 * j] * dsilu_(a[2 * j]);
                        const float x1 = EPI == 1 ? silu_(v[2 * j + 1]) : v[2 * j + 1] * dsilu_(a[2 * j + 1]);
                        __nv_bfloat162 p2 = __floats2bfloat162_rn(x0, x1);
                        hw[j] = *reinterpret_cast<uint32_t*>(&p2);
                    }
                    if (lane == 0) rsi_umma::bulk_wait_read0();
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(buf) + lane * 64 + 16 * c) =
                            make_uint4(hw[4 * c], hw[4 * c + 1], hw[4 * c + 2], hw[4 * c + 3]);
                    rsi_umma::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        rsi_umma::tma_store_2d(&tmH, col0, row0, sbuf);
                        rsi_umma::bulk_commit();
                    }
                }
            }
        }
    }
    if (warp >= 2 && lane == 0) rsi_umma::bulk_wait0();  // this warp's stores are complete
    __syncwarp();
    bool failed = !mbar_wait_bounded(smem_u32(&done), 0);
    failed = __syncthreads_or(failed || abort_flag);
    if (failed && tid == 0) atomicExch(status, RSI_DEV_TIMEOUT);
    rsi_umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) rsi_umma::tmem_dealloc(tmem, 2 * TBN);
}

__global__ void features_kernel(const float* __restrict__ p, const float* __restrict__ lo,
                                const float* __restrict__ hi, const float* __restrict__ Bm, int batch, int n_in,
                                int F, bf16* __restrict__ out) {
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= int64_t(batch) * F) return;
    const int b = int(q / F), f = int(q - int64_t(b) * F);
    // FP32 throughout: the features leave rounded to BF16 (2^-9), far above
    // the FP32 error of the scaled inputs and of sincospi
    float a = 0.0f;
    for (int j = 0; j < n_in; ++j) {
        const float u = fmaf(2.0f / (hi[j] - lo[j]), p[b * n_in + j] - lo[j], -1.0f);
        a = fmaf(Bm[f * n_in + j], u, a);
    }
    float s, c;
    sincospif(a, &s, &c);
    out[size_t(b) * 2 * F + f] = __float2bfloat16_rn(s);
    out[size_t(b) * 2 * F + F + f] = __float2bfloat16_rn(c);
}

__global__ void transpose_kernel(const bf16* __restrict__ in, int rows, int cols, bf16* __restrict__ out) {
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[dy][threadIdx.x] = in[size_t(r) * cols + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        int c = c0 + dy, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[size_t(c) * rows + r] = t[threadIdx.x][dy];
    }
}

// per-block partial sums of (y - t)^2 and the gradient scale * (y - t) in bf16
// n % 4 == 0.  Each thread sums its squared differences in FP32 (at most a
// few dozen terms), blocks combine in FP64; partial[blockIdx.x] = block sum.
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float gscale,
                            bf16* __restrict__ grad, double* __restrict__ partial) {
    __shared__ double red[32];
    float acc = 0.0f;
    const int64_t n4 = n / 4;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
        const float4 a = reinterpret_cast<const float4*>(y)[i];
        const float4 b = reinterpret_cast<const float4*>(t)[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
        if (grad) {
            __nv_bfloat162 g0 = __floats2bfloat162_rn(gscale * d0, gscale * d1);
            __nv_bfloat162 g1 = __floats2bfloat162_rn(gscale * d2, gscale * d3);
            reinterpret_cast<uint2*>(grad)[i] =
                make_uint2(*reinterpret_cast<uint32_t*>(&g0), *reinterpret_cast<uint32_t*>(&g1));
        }
    }
    double da = acc;
    for (int o = 16; o; o >>= 1) da += __shfl_xor_sync(0xffffffffu, da, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = da;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}
// one block of 256 threads: strided sums, then a fixed-order tree
__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double scale, float* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = float(red[0] * scale);
}
// out[c] = sum over rows of m[r][c]: blocks of 32 columns x 8 row lanes,
// each lane sums every 8th row, the 8 lane sums are added in a fixed order
__global__ void colsum_kernel(const bf16* __restrict__ m, int rows, int cols, float* __restrict__ out) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (c < cols)
        for (int r = threadIdx.y; r < rows; r += 8) s += __bfloat162float(m[size_t(r) * cols + c]);
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        out[c] = t;
    }
}
// one Adam element: m, v updated in place, returns the new weight
__device__ __forceinline__ float adam_elem(float w, float& m, float& v, float g, float lr, float b1, float b2,
                                          float eps, float c1, float c2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    return w - lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// hyper, when given, holds (lr, c1, c2) in device memory and overrides the
// scalar arguments (a schedule that a replayed CUDA graph can follow)
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2, const float* __restrict__ hyper, bf16* __restrict__ wh) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (hyper) {
        lr = hyper[0];
        c1 = hyper[1];
        c2 = hyper[2];
    }
    float mi = m[i], vi = v[i];
    const float wi = adam_elem(w[i], mi, vi, g[i], lr, b1, b2, eps, c1, c2);
    m[i] = mi;
    v[i] = vi;
    w[i] = wi;
    if (wh) wh[i] = __float2bfloat16_rn(wi);
}

// the same step four elements per thread (n % 4 == 0, 16-byte aligned arrays):
// the optimizer is bound by its 30 bytes of traffic per element
__global__ void adam4_kernel(float4* __restrict__ w, float4* __restrict__ m, float4* __restrict__ v,
                             const float4* __restrict__ g, int64_t n4, float lr, float b1, float b2, float eps,
                             float c1, float c2, const float* __restrict__ hyper, uint2* __restrict__ wh) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    if (hyper) {
        lr = hyper[0];
        c1 = hyper[1];
        c2 = hyper[2];
    }
    const float4 gi = g[i], wi = w[i];
    float4 mi = m[i], vi = v[i], wo;
    wo.x = adam_elem(wi.x, mi.x, vi.x, gi.x, lr, b1, b2, eps, c1, c2);
    wo.y = adam_elem(wi.y, mi.y, vi.y, gi.y, lr, b1, b2, eps, c1, c2);
    wo.z = adam_elem(wi.z, mi.z, vi.z, gi.z, lr, b1, b2, eps, c1, c2);
    wo.w = adam_elem(wi.w, mi.w, vi.w, gi.w, lr, b1, b2, eps, c1, c2);
    m[i] = mi;
    v[i] = vi;
    w[i] = wo;
    if (wh) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(wo.x, wo.y), h1 = __floats2bfloat162_rn(wo.z, wo.w);
        wh[i] = make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1));
    }
}

bool misaligned(const void* p, size_t a);

int launch_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2, float eps,
                float c1, float c2, const float* hyper, void* w_bf16, cudaStream_t s) {
    const bool vec = n % 4 == 0 && !misaligned(w, 16) && !misaligned(m, 16) && !misaligned(v, 16) &&
                     !misaligned(g, 16) && !misaligned(w_bf16, 8);
    if (vec) {
        const int64_t n4 = n / 4;
        adam4_kernel<<<unsigned((n4 + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<float4*>(w), reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v),
            reinterpret_cast<const float4*>(g), n4, lr, b1, b2, eps, c1, c2, hyper, static_cast<uint2*>(w_bf16));
        RSI_CHECK_LAUNCH("adam4_kernel");
    } else {
        adam_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2, hyper,
                                                               static_cast<bf16*>(w_bf16));
        RSI_CHECK_LAUNCH("adam_kernel");
    }
    return RSI_OK;
}

__global__ void cast_kernel(const float* __restrict__ in, int64_t n, bf16* __restrict__ out) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// img[b][j] (complex, float pairs) *= exp(sign * i psi_b(j)),
// psi = kx x_i + kz z_j + phi0; carrier[b] = (kx, kz, phi0, unused).
// In turns, psi / 2 pi = a + ix u + iz w with, per image,
//   a = (phi0 + kx (x0 + dx/2) + kz (z0 + dz/2)) / 2 pi  (reduced mod 1),
//   u = kx dx / 2 pi,  w = kz dz / 2 pi,
// formed once per block in FP64 (GB300's FP64 rate is low, so none of it is
// per pixel).  Per pixel ix u mod 1 is exact in FP32: with u = uh + ul (two
// floats), p = ix uh and its rounding error e = fma(ix, uh, -p) are exact,
// p - rint(p) is exact, and ix ul is a tiny correction; likewise iz w.  The
// sum lies within a few turns and is reduced once more, so the phase carries
// about 3e-7 turns (2e-6 rad) of error; the sine and cosine of the reduced
// angle (|angle| <= pi) come from the hardware approximation (absolute error
// about 4e-7).
__device__ __forceinline__ float frac_mul(float i, float h, float l) {
    const float p = i * h;
    const float e = fmaf(i, h, -p);
    return ((p - rintf(p)) + e) + i * l;
}

__global__ void __launch_bounds__(256) carrier_kernel(const double* __restrict__ carrier, int batch, int nx,
                                                      int per, double x0, double dx, double z0, double dz, int sign,
                                                      float scale, const float2* __restrict__ in,
                                                      float2* __restrict__ out) {
    __shared__ float k[6];  // ah, al, uh, ul, wh, wl
    for (int b = blockIdx.y; b < batch; b += gridDim.y) {
        __syncthreads();  // the previous image's constants are no longer read
        if (threadIdx.x == 0) {
            const double* cb = carrier + 4 * b;
            const double inv2pi = 0.15915494309189535;  // 1 / (2 pi)
            double ad = (cb[2] + cb[0] * (x0 + 0.5 * dx) + cb[1] * (z0 + 0.5 * dz)) * inv2pi;
            ad -= rint(ad);
            const double ud = cb[0] * dx * inv2pi, wd = cb[1] * dz * inv2pi;
            k[0] = float(ad);
            k[1] = float(ad - double(k[0]));
            k[2] = float(ud);
            k[3] = float(ud - double(k[2]));
            k[4] = float(wd);
            k[5] = float(wd - double(k[4]));
        }
        __syncthreads();
        const float ah = k[0], al = k[1], uh = k[2], ul = k[3], wh = k[4], wl = k[5];
        const float2* src = in + int64_t(b) * per;
        float2* dst = out + int64_t(b) * per;
        const int j0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
        const int sz = stride / nx, sx = stride - sz * nx;  // the stride in rows and columns
        int iz = j0 / nx, ix = j0 - iz * nx;
        for (int j = j0; j < per; j += stride) {
            float t = (ah + frac_mul(float(ix), uh, ul)) + frac_mul(float(iz), wh, wl);
            t = (t - rintf(t)) + al;
            float s, c;
            __sincosf(6.283185307179586f * t, &s, &c);
            ix += sx;
            iz += sz;
            if (ix >= nx) {
                ix -= nx;
                ++iz;
            }
            s = sign > 0 ? s * scale : -s * scale;
            c *= scale;
            const float2 v = src[j];
            dst[j] = make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
        }
    }
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// tensor map of a row-major matrix [rows x cols] of `type` (2 or 4 bytes):
// boxes of box_cols x box_rows, zero fill outside the matrix; with the
// 128-byte swizzle a box row is 128 bytes
int make_tmap(CUtensorMap* tm, CUtensorMapDataType type, size_t esize, const void* ptr, int64_t rows, int cols,
              int box_cols, int box_rows, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return rsi_fail(RSI_E_CUDA, "rsi_nn_gemm: cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(cols) * esize};
    const cuuint32_t box[2] = {cuuint32_t(box_cols), cuuint32_t(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, type, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return rsi_fail(RSI_E_CUDA, "rsi_nn_gemm: cuTensorMapEncodeTiled failed (%d)", int(r));
    return RSI_OK;
}

template <int EPI, int TBN>
int gemm_tc_launch_bn(const bf16* A, const bf16* B, int M, int N, int K, int layout, const float* bias,
                      const float* aux, float* outf, bf16* outh, int splits, float* work, cudaStream_t s,
                      const CarrierArgs& car = CarrierArgs{}) {
    using C = TcCfg<TBN>;
    static RsiCtxOnce attr;
    if (attr.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<EPI, TBN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(C::SMEM)),
                     "cudaFuncSetAttribute(gemm_tc)");
        attr.done();
    }
    int* status = rsi_status_ptr();
    if (!status) return RSI_E_CUDA;
    CUtensorMap ta, tb, tc, th;
    int rc = (layout & RSI_NN_A_T) ? make_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, K, M, 64, TC_BK)
                                   : make_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, M, K, TC_BK, TC_BM);
    if (rc) return rc;
    rc = (layout & RSI_NN_B_T) ? make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, K, N, 64, TC_BK)
                               : make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, N, K, TC_BK, TBN);
    if (rc) return rc;
    const int kt = K / TC_BK;
    const int kts = (kt + splits - 1) / splits;
    splits = (kt + kts - 1) / kts;
    memset(&tc, 0, sizeof(tc));
    memset(&th, 0, sizeof(th));
    if (EPI != 2 || splits > 1) {  // f32 blocks of 32 x 32: the output, z, or the partial sums
        rc = make_tmap(&tc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, splits > 1 ? static_cast<const void*>(work) : outf,
                       int64_t(splits) * M, N, 32, 32);
        if (rc) return rc;
    }
    if ((EPI == 1 || EPI == 2) && splits == 1) {  // bf16 blocks of 32 x 32, dense 64-byte rows in shared memory
        rc = make_tmap(&th, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, outh, M, N, 32, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (rc) return rc;
    }
    const int tiles = (M / TC_BM) * (N / TBN) * splits;
    const int grid = std::min(tiles, sm_count());
    gemm_tc_kernel<EPI, TBN><<<grid, TC_THREADS, C::SMEM, s>>>(ta, tb, tc, th, M, N, K, layout, bias, aux, kts,
                                                               splits, car, status);
    RSI_CHECK_LAUNCH("gemm_tc_kernel");
    if (splits > 1) {
        int64_t pairs = int64_t(M) * N / 2;
        splitk_reduce_kernel<EPI><<<unsigned((pairs + 255) / 256), 256, 0, s>>>(work, splits, M, N, bias, aux,
                                                                                 outf, outh);
        RSI_CHECK_LAUNCH("splitk_reduce_kernel");
    }
    return RSI_OK;
}

template <int EPI>
int gemm_tc_launch(const bf16* A, const bf16* B, int M, int N, int K, int layout, const float* bias,
                   const float* aux, float* outf, bf16* outh, int splits, float* work, cudaStream_t s,
                   const CarrierArgs& car = CarrierArgs{}) {
    // The widest output tile that still gives every SM a tile; else the
    // narrowest.  Small GEMMs (the hidden layers at batch 256) are latency-
    // bound: narrower tiles spread them over more SMs and shorten each CTA's
    // main loop and epilogue.
    const int64_t rows = M / TC_BM, sms = sm_count();
    const int kt = K / TC_BK, units = (kt + (kt + splits - 1) / splits - 1) / ((kt + splits - 1) / splits);
    if (N % 256 == 0 && rows * (N / 256) * units >= sms)
        return gemm_tc_launch_bn<EPI, 256>(A, B, M, N, K, layout, bias, aux, outf, outh, splits, work, s, car);
    if (N % 128 == 0 && rows * (N / 128) * units >= sms)
        return gemm_tc_launch_bn<EPI, 128>(A, B, M, N, K, layout, bias, aux, outf, outh, splits, work, s, car);
    return gemm_tc_launch_bn<EPI, 64>(A, B, M, N, K, layout, bias, aux, outf, outh, splits, work, s, car);
}

template <int EPI>
int gemm_launch(const bf16* A, const bf16* B, int M, int N, int K, const float* bias, const float* aux, float* outf,
                bf16* outh, int splits, float* work, cudaStream_t s) {
    static RsiCtxOnce attr;
    if (attr.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(gemm_tn_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(GEMM_SMEM)),
                     "cudaFuncSetAttribute(gemm)");
        attr.done();
    }
    const int kt = K / BK;
    const int kts = (kt + splits - 1) / splits;
    splits = (kt + kts - 1) / kts;
    dim3 grid(N / BN, M / BM, splits);
    gemm_tn_kernel<EPI><<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(A, B, M, N, K, bias, aux, splits > 1 ? work : outf,
                                                             outh, kts);
    RSI_CHECK_LAUNCH("gemm_tn_kernel");
    if (splits > 1) {
        int64_t pairs = int64_t(M) * N / 2;
        splitk_reduce_kernel<EPI><<<unsigned((pairs + 255) / 256), 256, 0, s>>>(work, splits, M, N, bias, aux,
                                                                                 outf, outh);
        RSI_CHECK_LAUNCH("splitk_reduce_kernel");
    }
    return RSI_OK;
}

bool misaligned(const void* p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) != 0; }

}  // namespace

extern "C" int rsi_nn_features(const float* params, const float* lo, const float* hi, const float* fmat,
                               int32_t batch, int32_t n_in, int32_t n_freq, void* out_bf16, void* stream) {
    if (!params || !lo || !hi || !fmat || !out_bf16 || batch < 1 || n_in < 1 || n_freq < 1)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_features: bad arguments");
    int64_t n = int64_t(batch) * n_freq;
    features_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        params, lo, hi, fmat, batch, n_in, n_freq, static_cast<bf16*>(out_bf16));
    RSI_CHECK_LAUNCH("features_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_gemm(int32_t epilogue, int32_t engine, int32_t layout, const void* A, const void* B, int32_t M,
                           int32_t N, int32_t K, const float* bias, const float* aux, float* out_f32, void* out_bf16,
                           int32_t splits, float* workspace, void* stream) {
    if (!A || !B || M < 1 || N < 1 || K < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: bad arguments");
    if (engine != RSI_NN_ENGINE_MMA_SYNC && engine != RSI_NN_ENGINE_TCGEN05)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: unknown engine %d", engine);
    if (layout & ~(RSI_NN_A_T | RSI_NN_B_T) || (layout && engine != RSI_NN_ENGINE_TCGEN05))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: layout %d needs the tcgen05 engine", layout);
    if (engine == RSI_NN_ENGINE_TCGEN05 && K % TC_BK)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: the tcgen05 engine needs K % 64 == 0 (got %d)", K);
    if (engine == RSI_NN_ENGINE_TCGEN05 && (misaligned(out_f32, 16) || misaligned(aux, 16) || misaligned(bias, 16) ||
                                            misaligned(out_bf16, 16) || misaligned(workspace, 16)))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: the tcgen05 engine needs 16-byte aligned outputs, bias and aux");
    if (splits < 1 || splits > K / BK || (splits > 1 && !workspace))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: splits must be in [1, K/32] and need a workspace");
    if (misaligned(workspace, 8)) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: misaligned workspace");
    if (M % BM || N % BN || K % BK)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: M, N must be multiples of 128 and K of 32 (got %d %d %d)", M, N,
                        K);
    if (misaligned(A, 16) || misaligned(B, 16) || misaligned(out_f32, 8) || misaligned(out_bf16, 4) ||
        misaligned(aux, 8))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: misaligned pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16* a = static_cast<const bf16*>(A);
    const bf16* b = static_cast<const bf16*>(B);
    bf16* oh = static_cast<bf16*>(out_bf16);
    const bool tc = engine == RSI_NN_ENGINE_TCGEN05;
    switch (epilogue) {
        case RSI_NN_EPI_F32:
            if (!out_f32) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: F32 epilogue needs out_f32");
            return tc ? gemm_tc_launch<0>(a, b, M, N, K, layout, bias, nullptr, out_f32, nullptr, splits, workspace, s)
                      : gemm_launch<0>(a, b, M, N, K, bias, nullptr, out_f32, nullptr, splits, workspace, s);
        case RSI_NN_EPI_BIAS_SILU:
            if (!out_f32 || !oh || !bias) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: BIAS_SILU needs bias and outputs");
            return tc ? gemm_tc_launch<1>(a, b, M, N, K, layout, bias, nullptr, out_f32, oh, splits, workspace, s)
                      : gemm_launch<1>(a, b, M, N, K, bias, nullptr, out_f32, oh, splits, workspace, s);
        case RSI_NN_EPI_DSILU:
            if (!aux || !oh) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: DSILU needs aux and out_bf16");
            return tc ? gemm_tc_launch<2>(a, b, M, N, K, layout, nullptr, aux, nullptr, oh, splits, workspace, s)
                      : gemm_launch<2>(a, b, M, N, K, nullptr, aux, nullptr, oh, splits, workspace, s);
        default:
            return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: unknown epilogue %d", epilogue);
    }
}

extern "C" int rsi_nn_gemm_carrier(const void* A, const void* B, int32_t M, int32_t N, int32_t K, const float* bias,
                                   const double* carrier, const rsi_grid* window, int32_t sign, float scale, float* out,
                                   float* workspace, void* stream) {
    if (!A || !B || !carrier || !window || !out || !workspace || M < 1 || N < 1 || K < 1 ||
        (sign != 1 && sign != -1) || !isfinite(scale))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm_carrier: bad arguments");
    if (M % TC_BM || N % 128 || K % TC_BK)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm_carrier: M, N must be multiples of 128 and K of 64 (got %d %d %d)",
                        M, N, K);
    if (window->nx < 1 || window->nz < 1 || int64_t(N) != 2 * int64_t(window->nx) * window->nz)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm_carrier: N must be 2 nx nz of the window (got %d)", N);
    if (int64_t(window->nx) * window->nz > (int64_t(1) << 24))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm_carrier: window exceeds 2^24 pixels");
    if (misaligned(A, 16) || misaligned(B, 16) || misaligned(out, 16) || misaligned(bias, 16) ||
        misaligned(carrier, 8) || misaligned(workspace, 16))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm_carrier: misaligned pointer");
    CarrierArgs car;
    car.coef = carrier;
    car.nx = window->nx;
    car.sign = sign;
    car.scale = scale;
    car.x0 = window->x0;
    car.dx = (window->x1 - window->x0) / window->nx;
    car.z0 = window->z0;
    car.dz = (window->z1 - window->z0) / window->nz;
    car.rows = reinterpret_cast<const float4*>(workspace);
    carrier_rows_kernel<<<unsigned((M + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        car, M, reinterpret_cast<float4*>(workspace));
    RSI_CHECK_LAUNCH("carrier_rows_kernel");
    return gemm_tc_launch<3>(static_cast<const bf16*>(A), static_cast<const bf16*>(B), M, N, K, 0, bias, nullptr,
                             out, nullptr, 1, nullptr, static_cast<cudaStream_t>(stream), car);
}

extern "C" int rsi_nn_carrier_coeffs(const double* params, int32_t batch, double c1, double c2, double* carrier,
                                     float* params_f32, void* stream) {
    if (!params || !carrier || !params_f32 || batch < 1 || !(c1 > 0) || !(c2 > 0))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier_coeffs: bad arguments");
    carrier_coeffs_kernel<<<unsigned((batch + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        params, batch, c1, c2, carrier, params_f32);
    RSI_CHECK_LAUNCH("carrier_coeffs_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_transpose(const void* in_bf16, int32_t rows, int32_t cols, void* out_bf16, void* stream) {
    if (!in_bf16 || !out_bf16 || rows < 1 || cols < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_transpose: bad arguments");
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const bf16*>(in_bf16), rows,
                                                                            cols, static_cast<bf16*>(out_bf16));
    RSI_CHECK_LAUNCH("transpose_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_loss(const float* y, const float* t, int64_t n, float grad_scale, void* grad_bf16,
                           double* partial, int32_t n_partial, float* loss_out, void* stream) {
    if (!y || !t || n < 1 || n % 4 || !partial || n_partial < 1 || !loss_out)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_loss: bad arguments (n must be a positive multiple of 4)");
    if (misaligned(y, 16) || misaligned(t, 16) || misaligned(grad_bf16, 8))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_loss: misaligned pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    loss_kernel<<<n_partial, 256, 0, s>>>(y, t, n, grad_scale, static_cast<bf16*>(grad_bf16), partial);
    RSI_CHECK_LAUNCH("loss_kernel");
    sum_partials_kernel<<<1, 256, 0, s>>>(partial, n_partial, 1.0 / double(n), loss_out);
    RSI_CHECK_LAUNCH("sum_partials_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_colsum(const void* m_bf16, int32_t rows, int32_t cols, float* out, void* stream) {
    if (!m_bf16 || !out || rows < 1 || cols < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_colsum: bad arguments");
    colsum_kernel<<<(cols + 31) / 32, dim3(32, 8), 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(m_bf16), rows, cols, out);
    RSI_CHECK_LAUNCH("colsum_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, float beta1,
                           float beta2, float eps, int32_t step, void* w_bf16, void* stream) {
    if (!w || !m || !v || !g || n < 1 || step < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_adam: bad arguments");
    float c1 = float(1.0 - pow(double(beta1), step)), c2 = float(1.0 - pow(double(beta2), step));
    return launch_adam(w, m, v, g, n, lr, beta1, beta2, eps, c1, c2, nullptr, w_bf16,
                       static_cast<cudaStream_t>(stream));
}

extern "C" int rsi_nn_adam_dev(float* w, float* m, float* v, const float* g, int64_t n, const float* hyper,
                               float beta1, float beta2, float eps, void* w_bf16, void* stream) {
    if (!w || !m || !v || !g || !hyper || n < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_adam_dev: bad arguments");
    return launch_adam(w, m, v, g, n, 0.0f, beta1, beta2, eps, 1.0f, 1.0f, hyper, w_bf16,
                       static_cast<cudaStream_t>(stream));
}

extern "C" int rsi_nn_cast_bf16(const float* in, int64_t n, void* out_bf16, void* stream) {
    if (!in || !out_bf16 || n < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_cast_bf16: bad arguments");
    cast_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, n,
                                                                                        static_cast<bf16*>(out_bf16));
    RSI_CHECK_LAUNCH("cast_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_carrier(const double* carrier, int32_t batch, const rsi_grid* window, int32_t sign,
                              float scale, const float* in, float* out, void* stream) {
    if (!carrier || !window || !in || !out || batch < 1 || (sign != 1 && sign != -1) || !isfinite(scale))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier: bad arguments");
    if (window->nx < 1 || window->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier: empty window");
    const int64_t per = int64_t(window->nx) * window->nz;
    if (per > (int64_t(1) << 24))  // pixel indices stay exact in FP32
        return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier: window of %lld pixels exceeds 2^24", (long long)per);
    double dx = (window->x1 - window->x0) / window->nx, dz = (window->z1 - window->z0) / window->nz;
    // about 4 pixels per thread, one row of blocks per image
    const unsigned bx = unsigned(std::max<int64_t>(1, std::min<int64_t>(256, (per + 1023) / 1024)));
    const dim3 grid(bx, unsigned(std::min(batch, 65535)));
    carrier_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        carrier, batch, window->nx, int(per), window->x0, dx, window->z0, dz, sign, scale,
        reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out));
    RSI_CHECK_LAUNCH("carrier_kernel");
    return RSI_OK;
}
