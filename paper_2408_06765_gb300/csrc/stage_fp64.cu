// stage_fp64.cu -- double-precision source x target kernel (steps a3, a5),
// the path for runs validated at 1e-5 against the FP64 oracle.  Same tiling
// and bulk-copy pipeline as the FP32C kernel; per pair it evaluates the
// paper's terms directly in FP64 with Neumaier-compensated accumulation.
#include <math.h>

#include "stage.cuh"

namespace {

constexpr int kThreads = 128;

struct Neu {
    double s, c;
};
__device__ __forceinline__ void neu_add(Neu& a, double v) {
    double t = a.s + v;
    if (fabs(a.s) >= fabs(v))
        a.c += (a.s - t) + v;
    else
        a.c += (v - t) + a.s;
    a.s = t;
}

template <int KIND, int NORM>
__global__ void __launch_bounds__(kThreads)
    stage_fp64_kernel(StageArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int t_begin = split * a.tiles_per_split;
    const int t_end = min(a.n_tiles, t_begin + a.tiles_per_split);
    const int ntile = max(0, t_end - t_begin);
    const uint32_t tile_bytes = uint32_t(a.tile_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * a.tile_bytes);

    const int64_t j_raw = int64_t(blockIdx.x) * kThreads + tid;
    const int64_t j = j_raw < a.n_tgt ? j_raw : a.n_tgt - 1;
    const double qx = a.tgt.x[j], qy = a.tgt.y[j], qz = a.tgt.z[j];
    const double k = a.k;

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

    Neu re = {0.0, 0.0}, im = {0.0, 0.0};
    int failed_at = -1;
    for (int it = 0; it < ntile; ++it) {
        const int buf = it % RSI_PIPE_STAGES;
        const uint32_t parity = uint32_t(it / RSI_PIPE_STAGES) & 1u;
        bool ok = mbar_wait_bounded(smem_u32(&bars[buf]), parity);
        if (__syncthreads_or(!ok)) {
            failed_at = it;
            break;
        }
        const double* rec = reinterpret_cast<const double*>(smem + buf * a.tile_bytes + RSI_TILE_HDR_BYTES);
        for (int i = 0; i < a.S; ++i) {
            const double* r = rec + 8 * i;
            const double dx = qx - r[0], dy = qy - r[1], dz = qz - r[2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 >= 1e-24)) continue;  // pairs closer than 1e-12 m contribute nothing
            const double rr = sqrt(r2);
            const double ir = 1.0 / rr;
            double s, c;
            sincos(k * rr, &s, &c);
            if (KIND == RSI_STAGE_PISTON) {
                const double amp = r[3] * ir;  // -v0 w / (2 pi r)
                neu_add(re, amp * c);
                neu_add(im, amp * s);
            } else {
                const double nd = (NORM == RSI_NORMALS_Z) ? dz : (r[5] * dx + r[6] * dy + r[7] * dz);
                const double h = nd * ir * ir;  // cos(theta) / r
                // B (ik - 1/r) e^{ikr} cos(theta) / r,  B = -w sigma / (2 pi)
                const double vr = -ir * r[3] - k * r[4];
                const double vi = -ir * r[4] + k * r[3];
                neu_add(re, h * (vr * c - vi * s));
                neu_add(im, h * (vr * s + vi * c));
            }
        }
        __syncthreads();
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
            for (int it = failed_at; it < ntile && it < failed_at + RSI_PIPE_STAGES; ++it)
                mbar_wait_bounded(smem_u32(&bars[it % RSI_PIPE_STAGES]), uint32_t(it / RSI_PIPE_STAGES) & 1u);
        }
        return;
    }
    if (j_raw < a.n_tgt) {
        double2* out = a.out + (a.splits > 1 ? size_t(split) * size_t(a.n_tgt) : 0);
        double vr = re.s + re.c, vi = im.s + im.c;
        if (!isfinite(vr) || !isfinite(vi)) atomicExch(a.status, RSI_DEV_NONFINITE);
        out[j_raw] = make_double2(vr, vi);
    }
}

__global__ void prep_fp64_kernel(int kind, int normals, int64_t n_src, PointsView src,
                                 const double2* __restrict__ sigma, double amp_scale, uint8_t* tiles,
                                 size_t tile_bytes, int64_t n_slots) {
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n_slots) return;
    const int S = int((tile_bytes - RSI_TILE_HDR_BYTES) / 64);
    const int64_t tile = q / S, slot = q - tile * S;
    double* rec = reinterpret_cast<double*>(tiles + size_t(tile) * tile_bytes + RSI_TILE_HDR_BYTES) + 8 * slot;
    if (slot == 0) {
        double* hdr = reinterpret_cast<double*>(tiles + size_t(tile) * tile_bytes);
        hdr[0] = hdr[1] = hdr[2] = hdr[3] = 0.0;
    }
    if (q < n_src) {
        rec[0] = src.x[q];
        rec[1] = src.y[q];
        rec[2] = src.z[q];
        if (kind == RSI_STAGE_PISTON) {
            rec[3] = amp_scale * src.w[q];
            rec[4] = 0.0;
        } else {
            double2 sg = sigma[q];
            rec[3] = amp_scale * src.w[q] * sg.x;
            rec[4] = amp_scale * src.w[q] * sg.y;
        }
        rec[5] = src.nx[q];
        rec[6] = src.ny[q];
        rec[7] = src.nz[q];
    } else {
        rec[0] = rec[1] = rec[2] = 4.0;
        rec[3] = rec[4] = 0.0;
        rec[5] = rec[6] = 0.0;
        rec[7] = 1.0;
    }
    (void)normals;
}

template <int KIND, int NORM>
int launch_t(const StageArgs& a, cudaStream_t s) {
    size_t smem = RSI_PIPE_STAGES * a.tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t);
    static RsiCtxOnce attr_set;
    if (attr_set.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(stage_fp64_kernel<KIND, NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024),
                     "cudaFuncSetAttribute(stage_fp64)");
        attr_set.done();
    }
    dim3 grid(unsigned((a.n_tgt + kThreads - 1) / kThreads), unsigned(a.splits));
    stage_fp64_kernel<KIND, NORM><<<grid, kThreads, smem, s>>>(a);
    RSI_CHECK_LAUNCH("stage_fp64_kernel");
    return RSI_OK;
}

template <int KIND, int NORM>
int occupancy_t(const StageArgs& a) {
    size_t smem = RSI_PIPE_STAGES * a.tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, stage_fp64_kernel<KIND, NORM>, kThreads, smem) !=
        cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

int dispatch(const StageArgs& a, cudaStream_t s, bool occ) {
    if (a.kind == RSI_STAGE_PISTON)
        return occ ? occupancy_t<RSI_STAGE_PISTON, RSI_NORMALS_Z>(a) : launch_t<RSI_STAGE_PISTON, RSI_NORMALS_Z>(a, s);
    if (a.normals == RSI_NORMALS_POINTS)
        return occ ? occupancy_t<RSI_STAGE_RSI, RSI_NORMALS_POINTS>(a)
                   : launch_t<RSI_STAGE_RSI, RSI_NORMALS_POINTS>(a, s);
    return occ ? occupancy_t<RSI_STAGE_RSI, RSI_NORMALS_Z>(a) : launch_t<RSI_STAGE_RSI, RSI_NORMALS_Z>(a, s);
}

}  // namespace

size_t fp64_record_bytes() { return 64; }
int fp64_threads() { return kThreads; }

int launch_prep_fp64(const rsi_stage& st, const PointsView& src, int64_t n_src, const double2* sigma, int S,
                     uint8_t* tiles, size_t tile_bytes, int n_tiles, cudaStream_t s) {
    const double amp_scale = stage_amp_scale(st);
    const int normals = st.kind == RSI_STAGE_RSI ? base_normals(st.normals) : RSI_NORMALS_Z;
    int64_t n_slots = int64_t(n_tiles) * S;
    int threads = 256;
    unsigned blocks = unsigned((n_slots + threads - 1) / threads);
    prep_fp64_kernel<<<blocks, threads, 0, s>>>(st.kind, normals, n_src, src, sigma, amp_scale, tiles, tile_bytes,
                                                n_slots);
    RSI_CHECK_LAUNCH("prep_fp64_kernel");
    return RSI_OK;
}

int launch_stage_fp64(const StageArgs& a, cudaStream_t s) { return dispatch(a, s, false); }
int stage_occupancy_fp64(const StageArgs& a) { return dispatch(a, nullptr, true); }
