// nn.cu -- step a9: kernels of the learned surrogate, a Fourier-feature MLP
// (not in the paper) that maps transducer offset, tilt, water path,
// frequency and image depth to the carrier-demodulated field image of the
// RSI chain, trained on fields the RSI kernels compute.
//
//   features   u = 2 (p - lo)/(hi - lo) - 1, h0 = [sin(pi B u), cos(pi B u)]  (bf16)
//   gemm_tn    C[M x N] = A[M x K] B[N x K]^T on BF16 tensor cores (mma.sync
//              m16n8k16, FP32 accumulation), ldmatrix fragments, a 3-stage
//              cp.async pipeline, and fused epilogues:
//                F32        C (+ bias)                       -> f32
//                BIAS_SILU  z = C + bias -> f32 z, bf16 silu(z)
//                DSILU      C * silu'(aux)                   -> bf16   (backprop)
//   transpose  bf16 [R x C] -> [C x R]
//   loss       mean (y - t)^2 and its gradient 2 (y - t)/n  -> bf16
//   colsum     bias gradients (column sums of a bf16 matrix)
//   adam       Kingma & Ba (2015) on FP32 master weights, bf16 copy out
//   carrier    multiply an image by exp(+-i psi), psi = kx x + kz z + phi0
#include <cuda_bf16.h>
#include <math.h>

#include "rsi_internal.cuh"

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

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
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

__global__ void features_kernel(const float* __restrict__ p, const float* __restrict__ lo,
                                const float* __restrict__ hi, const float* __restrict__ Bm, int batch, int n_in,
                                int F, bf16* __restrict__ out) {
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= int64_t(batch) * F) return;
    const int b = int(q / F), f = int(q - int64_t(b) * F);
    double a = 0.0;
    for (int j = 0; j < n_in; ++j) {
        double u = 2.0 * (double(p[b * n_in + j]) - lo[j]) / (double(hi[j]) - lo[j]) - 1.0;
        a += double(Bm[f * n_in + j]) * u;
    }
    double s, c;
    sincospi(a, &s, &c);
    out[size_t(b) * 2 * F + f] = __float2bfloat16_rn(float(s));
    out[size_t(b) * 2 * F + F + f] = __float2bfloat16_rn(float(c));
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
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float gscale,
                            bf16* __restrict__ grad, double* __restrict__ partial) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float d = y[i] - t[i];
        acc += double(d) * d;
        if (grad) grad[i] = __float2bfloat16_rn(gscale * d);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double scale, float* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        *out = float(s * scale);
    }
}

__global__ void colsum_kernel(const bf16* __restrict__ m, int rows, int cols, float* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(m[size_t(r) * cols + c]);
    out[c] = s;
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2, bf16* __restrict__ wh) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wh) wh[i] = __float2bfloat16_rn(wi);
}

__global__ void cast_kernel(const float* __restrict__ in, int64_t n, bf16* __restrict__ out) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// img[b][j] (complex, float pairs) *= exp(sign * i psi_b(j)),
// psi = kx x_i + kz z_j + phi0; carrier[b] = (kx, kz, phi0, unused)
__global__ void carrier_kernel(const double* __restrict__ carrier, int batch, int nx, int nz, double x0,
                               double dx, double z0, double dz, int sign, const float2* __restrict__ in,
                               float2* __restrict__ out) {
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t per = int64_t(nx) * nz;
    if (q >= int64_t(batch) * per) return;
    const int b = int(q / per);
    const int64_t j = q - int64_t(b) * per;
    const int iz = int(j / nx), ix = int(j - int64_t(iz) * nx);
    const double* cb = carrier + 4 * b;
    double x = x0 + (ix + 0.5) * dx, z = z0 + (iz + 0.5) * dz;
    double psi = cb[0] * x + cb[1] * z + cb[2];
    double s, c;
    sincospi(psi / M_PI, &s, &c);
    s *= sign;
    float2 v = in[q];
    out[q] = make_float2(float(v.x * c - v.y * s), float(v.x * s + v.y * c));
}

template <int EPI>
int gemm_launch(const bf16* A, const bf16* B, int M, int N, int K, const float* bias, const float* aux, float* outf,
                bf16* outh, int splits, float* work, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(gemm_tn_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(GEMM_SMEM)),
                     "cudaFuncSetAttribute(gemm)");
        attr = true;
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

extern "C" int rsi_nn_gemm(int32_t epilogue, const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                           const float* bias, const float* aux, float* out_f32, void* out_bf16, int32_t splits,
                           float* workspace, void* stream) {
    if (!A || !B || M < 1 || N < 1 || K < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: bad arguments");
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
    switch (epilogue) {
        case RSI_NN_EPI_F32:
            if (!out_f32) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: F32 epilogue needs out_f32");
            return gemm_launch<0>(a, b, M, N, K, bias, nullptr, out_f32, nullptr, splits, workspace, s);
        case RSI_NN_EPI_BIAS_SILU:
            if (!out_f32 || !oh || !bias) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: BIAS_SILU needs bias and outputs");
            return gemm_launch<1>(a, b, M, N, K, bias, nullptr, out_f32, oh, splits, workspace, s);
        case RSI_NN_EPI_DSILU:
            if (!aux || !oh) return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: DSILU needs aux and out_bf16");
            return gemm_launch<2>(a, b, M, N, K, nullptr, aux, nullptr, oh, splits, workspace, s);
        default:
            return rsi_fail(RSI_E_INVAL, "rsi_nn_gemm: unknown epilogue %d", epilogue);
    }
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
    if (!y || !t || n < 1 || !partial || n_partial < 1 || !loss_out)
        return rsi_fail(RSI_E_INVAL, "rsi_nn_loss: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    loss_kernel<<<n_partial, 256, 0, s>>>(y, t, n, grad_scale, static_cast<bf16*>(grad_bf16), partial);
    RSI_CHECK_LAUNCH("loss_kernel");
    sum_partials_kernel<<<1, 32, 0, s>>>(partial, n_partial, 1.0 / double(n), loss_out);
    RSI_CHECK_LAUNCH("sum_partials_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_colsum(const void* m_bf16, int32_t rows, int32_t cols, float* out, void* stream) {
    if (!m_bf16 || !out || rows < 1 || cols < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_colsum: bad arguments");
    colsum_kernel<<<(cols + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const bf16*>(m_bf16), rows, cols, out);
    RSI_CHECK_LAUNCH("colsum_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, float beta1,
                           float beta2, float eps, int32_t step, void* w_bf16, void* stream) {
    if (!w || !m || !v || !g || n < 1 || step < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_adam: bad arguments");
    float c1 = float(1.0 - pow(double(beta1), step)), c2 = float(1.0 - pow(double(beta2), step));
    adam_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, m, v, g, n, lr, beta1, beta2, eps, c1, c2, static_cast<bf16*>(w_bf16));
    RSI_CHECK_LAUNCH("adam_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_cast_bf16(const float* in, int64_t n, void* out_bf16, void* stream) {
    if (!in || !out_bf16 || n < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_cast_bf16: bad arguments");
    cast_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, n,
                                                                                        static_cast<bf16*>(out_bf16));
    RSI_CHECK_LAUNCH("cast_kernel");
    return RSI_OK;
}

extern "C" int rsi_nn_carrier(const double* carrier, int32_t batch, const rsi_grid* window, int32_t sign,
                              const float* in, float* out, void* stream) {
    if (!carrier || !window || !in || !out || batch < 1 || (sign != 1 && sign != -1))
        return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier: bad arguments");
    if (window->nx < 1 || window->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_nn_carrier: empty window");
    int64_t n = int64_t(batch) * window->nx * window->nz;
    double dx = (window->x1 - window->x0) / window->nx, dz = (window->z1 - window->z0) / window->nz;
    carrier_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        carrier, batch, window->nx, window->nz, window->x0, dx, window->z0, dz, sign,
        reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out));
    RSI_CHECK_LAUNCH("carrier_kernel");
    return RSI_OK;
}
