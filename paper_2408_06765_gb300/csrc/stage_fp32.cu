// stage_fp32.cu -- the FP32C source x target kernel of one stage (steps a3,
// a5): CTA (bx, split) handles targets [bx*TPT*256, (bx+1)*TPT*256) against
// the source tiles of its split.  The arithmetic is in stage_fp32_body.cuh.
#include "stage_fp32_body.cuh"

namespace {

using namespace rsi_fp32;

template <int KIND, int NORM, int TPT, int VAR>
__global__ void __launch_bounds__(kThreads, (min_blocks<KIND, TPT, VAR>()))
    stage_fp32_kernel(StageArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * a.tile_bytes);
    init_barriers(bars);
    const int split = blockIdx.y;
    BlockWork w;
    w.tiles = a.tiles;
    w.tile_bytes = uint32_t(a.tile_bytes);
    w.S = a.S;
    w.t_begin = split * a.tiles_per_split;
    w.ntile = max(0, min(a.n_tiles, w.t_begin + a.tiles_per_split) - w.t_begin);
    w.tgt = a.tgt;
    w.n_tgt = a.n_tgt;
    w.j0 = int64_t(blockIdx.x) * TPT * kThreads;
    w.kh = a.kh;
    w.kl = a.kl;
    w.tp = a.tp;
    w.out = a.out + (a.splits > 1 ? size_t(split) * size_t(a.n_tgt) : 0);
    w.status = a.status;
    uint32_t uses = 0;
    run_block<KIND, NORM, TPT, VAR>(w, smem, bars, uses);
}

__global__ void prep_fp32_kernel(int kind, int normals, int64_t n_src, PointsView src,
                                 const double2* __restrict__ sigma, double amp_scale, double k, uint8_t* tiles,
                                 size_t tile_bytes, int packed) {
    __shared__ double red[32];
    prep_tile(kind, normals, int(blockDim.x), n_src, src, sigma, amp_scale, k, tiles, tile_bytes,
              int64_t(blockIdx.x), red, packed != 0);
}

template <int KIND, int NORM, int TPT, int VAR>
int launch_t(const StageArgs& a, cudaStream_t s) {
    size_t smem = RSI_PIPE_STAGES * a.tile_bytes + RSI_PIPE_STAGES * sizeof(uint64_t);
    static RsiCtxOnce attr_set;
    if (attr_set.needed()) {
        RSI_CUDA_TRY(cudaFuncSetAttribute(stage_fp32_kernel<KIND, NORM, TPT, VAR>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                     "cudaFuncSetAttribute(stage_fp32)");
        attr_set.done();
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
    if (a.tpt == 1) {
        if (a.variant == 3) return occ ? occupancy_t<KIND, NORM, 1, 3>(a) : launch_t<KIND, NORM, 1, 3>(a, s);
        if (a.variant == 2) return occ ? occupancy_t<KIND, NORM, 1, 2>(a) : launch_t<KIND, NORM, 1, 2>(a, s);
        return occ ? occupancy_t<KIND, NORM, 1, 1>(a) : launch_t<KIND, NORM, 1, 1>(a, s);
    }
    if (a.tpt == 4) {
        if (a.variant == 3) return occ ? occupancy_t<KIND, NORM, 4, 3>(a) : launch_t<KIND, NORM, 4, 3>(a, s);
        if (a.variant == 2) return occ ? occupancy_t<KIND, NORM, 4, 2>(a) : launch_t<KIND, NORM, 4, 2>(a, s);
        return occ ? occupancy_t<KIND, NORM, 4, 1>(a) : launch_t<KIND, NORM, 4, 1>(a, s);
    }
    if (a.variant == 3) return occ ? occupancy_t<KIND, NORM, 2, 3>(a) : launch_t<KIND, NORM, 2, 3>(a, s);
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

double stage_amp_scale(const rsi_stage& st) {
    return (st.kind == RSI_STAGE_PISTON) ? -st.v0 / (2.0 * M_PI) : -normals_sign(st.normals) / (2.0 * M_PI);
}

int launch_prep_fp32(const rsi_stage& st, const PointsView& src, int64_t n_src, const double2* sigma, int S,
                     uint8_t* tiles, size_t tile_bytes, int n_tiles, cudaStream_t s, bool packed) {
    const int normals = st.kind == RSI_STAGE_RSI ? base_normals(st.normals) : RSI_NORMALS_Z;
    prep_fp32_kernel<<<n_tiles, S, 0, s>>>(st.kind, normals, n_src, src, sigma, stage_amp_scale(st), st.k, tiles,
                                           tile_bytes, packed ? 1 : 0);
    RSI_CHECK_LAUNCH("prep_fp32_kernel");
    return RSI_OK;
}

int launch_stage_fp32(const StageArgs& a, cudaStream_t s) { return dispatch(a, s, false); }
int stage_occupancy_fp32(const StageArgs& a) { return dispatch(a, nullptr, true); }
