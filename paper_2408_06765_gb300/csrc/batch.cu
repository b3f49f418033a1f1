// batch.cu -- step a8: many single-interface chains (piston -> interface ->
// image), e.g. the frequencies of a broadband pulse (Sec. 4: the multi-
// frequency field is a superposition of single-frequency fields) times the
// positions of a scan, with uneven QMC counts, run as ONE CUDA graph:
//
//   counters <- 0
//   points of every piston and interface, pixels of every distinct grid
//   piston tiles of every instance
//   persistent stage kernel over the work items of every piston stage
//   split reduction, transmission sigma = T12 phi, interface tiles
//   persistent stage kernel over the work items of every RSI stage
//   split reduction, images (complex64)
//
// A work item is (instance, block of 256*TPT targets, run of source tiles);
// items are sorted by size, largest first, and the resident CTAs of the
// persistent kernel take them from a global counter (longest-processing-
// time-first list scheduling), so uneven instances balance across the SMs.
// Each item writes its own partial-sum slot; the reduction adds the slots in
// a fixed order, so results do not depend on the schedule.
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "interface_body.cuh"
#include "qmc_body.cuh"
#include "stage_fp32_body.cuh"

namespace {

using rsi_fp32::kThreads;

struct BPointSet {
    rsi_qmc::SurfaceDev s;
    uint64_t k0, k1;
    int64_t n;
    PointsView out;
    int32_t scramble, pad;
};
struct BGrid {
    rsi_grid g;
    PointsView out;
};
struct BSeg {  // 256 consecutive elements of one set / instance
    int32_t set, pad;
    int64_t first;
};
struct BPrep {
    PointsView src;
    int64_t n_src;
    int32_t S, pad;
    const double2* sigma;
    uint8_t* tiles;
    size_t tile_bytes;
    double amp_scale, k;
    int32_t kind, normals;
};
struct BPrepTile {
    int32_t inst, pad;
    int64_t tile;
};
struct BStageInst {
    const uint8_t* tiles;
    size_t tile_bytes;
    int32_t S, n_tiles, tiles_per_split, splits;
    TgtView tgt;
    int64_t n_tgt;
    float kh, kl;
    double2* out;  // [splits][n_tgt] partial sums, or the field when splits == 1
};
struct BItem {
    int32_t inst, split;
    int64_t block;
};
struct BReduce {
    const double2* part;
    double2* out;
    int64_t n;
    int32_t splits, pad;
};
struct BTransmit {
    rsi_interface it;
    const double* nx;
    const double* nz;
    const double2* phi;
    double2* sigma;
    int64_t n;
};
struct BImage {
    const double2* field;
    float2* out;
    int64_t n;
    double scale;
};

constexpr int kSeg = 256;

__global__ void batch_points_kernel(const BPointSet* __restrict__ sets, const BSeg* __restrict__ segs,
                                    rsi_qmc::SobolDirs dirs) {
    const BSeg g = segs[blockIdx.x];
    const BPointSet& p = sets[g.set];
    int64_t i = g.first + threadIdx.x;
    if (i < p.n) rsi_qmc::make_point(p.s, dirs, p.k0, p.k1, p.scramble, i, p.n, p.out);
}

__global__ void batch_grid_kernel(const BGrid* __restrict__ grids, const BSeg* __restrict__ segs) {
    const BSeg g = segs[blockIdx.x];
    const BGrid& G = grids[g.set];
    int64_t q = g.first + threadIdx.x;
    if (q < int64_t(G.g.nx) * G.g.nz) rsi_qmc::make_grid_point(G.g, q, G.out);
}

__global__ void batch_prep_kernel(const BPrep* __restrict__ preps, const BPrepTile* __restrict__ tiles, int packed) {
    __shared__ double red[32];
    const BPrepTile t = tiles[blockIdx.x];
    const BPrep& p = preps[t.inst];
    // all instances share the CTA size; tiles of smaller instances use fewer
    // threads, and the extra threads take part only in the reductions
    rsi_fp32::prep_tile(p.kind, p.normals, p.S, p.n_src, p.src, p.sigma, p.amp_scale, p.k, p.tiles,
                        p.tile_bytes, t.tile, red, packed != 0);
}

// Resident CTAs per SM asked of the compiler for the persistent stage kernels:
// the packed RSI stage (variant 3) keeps its accumulators for two targets and
// the work-item state in registers at 2 CTAs per SM, where 3 spill;
// RSI_BATCH_RSI_MIN_BLOCKS overrides it.
#ifndef RSI_BATCH_RSI_MIN_BLOCKS
#define RSI_BATCH_RSI_MIN_BLOCKS 2
#endif
template <int KIND, int TPT, int VAR>
constexpr int batch_min_blocks() {
    return TPT == 1   ? RSI_FP32_TPT1_MIN_BLOCKS
           : TPT != 2 ? 2
           : (KIND == RSI_STAGE_RSI && VAR == 3) ? RSI_BATCH_RSI_MIN_BLOCKS
                                                  : RSI_FP32_MIN_BLOCKS;
}

template <int KIND, int NORM, int TPT, int VAR>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<KIND, TPT, VAR>())
    batch_stage_kernel(const BStageInst* __restrict__ insts, const BItem* __restrict__ items, int64_t n_items,
                       TwoPiSplit tp, size_t max_tile_bytes, unsigned long long* counter, int* status) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ long long s_item;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RSI_PIPE_STAGES * max_tile_bytes);
    rsi_fp32::init_barriers(bars);
    uint32_t uses = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();  // every thread has read the index before it is replaced
        if (it >= n_items) break;
        const BItem item = items[it];
        const BStageInst& I = insts[item.inst];
        rsi_fp32::BlockWork w;
        w.tiles = I.tiles;
        w.tile_bytes = uint32_t(I.tile_bytes);
        w.S = I.S;
        w.t_begin = item.split * I.tiles_per_split;
        w.ntile = max(0, min(I.n_tiles, w.t_begin + I.tiles_per_split) - w.t_begin);
        w.tgt = I.tgt;
        w.n_tgt = I.n_tgt;
        w.j0 = item.block * int64_t(TPT) * kThreads;
        w.kh = I.kh;
        w.kl = I.kl;
        w.tp = tp;
        w.out = I.out + (I.splits > 1 ? size_t(item.split) * size_t(I.n_tgt) : 0);
        w.status = status;
        if (!rsi_fp32::run_block<KIND, NORM, TPT, VAR>(w, smem, bars, uses)) return;
    }
}

__global__ void batch_reduce_kernel(const BReduce* __restrict__ red, const BSeg* __restrict__ segs, int* status) {
    const BSeg g = segs[blockIdx.x];
    const BReduce& R = red[g.set];
    int64_t j = g.first + threadIdx.x;
    if (j >= R.n) return;
    double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;  // Neumaier over the splits, in order
    for (int s = 0; s < R.splits; ++s) {
        double2 v = R.part[size_t(s) * size_t(R.n) + size_t(j)];
        double t = sr + v.x;
        cr += (fabs(sr) >= fabs(v.x)) ? (sr - t) + v.x : (v.x - t) + sr;
        sr = t;
        t = si + v.y;
        ci += (fabs(si) >= fabs(v.y)) ? (si - t) + v.y : (v.y - t) + si;
        si = t;
    }
    double re = sr + cr, im = si + ci;
    if (!isfinite(re) || !isfinite(im)) atomicExch(status, RSI_DEV_NONFINITE);
    R.out[j] = make_double2(re, im);
}

__global__ void batch_transmit_kernel(const BTransmit* __restrict__ tr, const BSeg* __restrict__ segs) {
    const BSeg g = segs[blockIdx.x];
    const BTransmit& T = tr[g.set];
    int64_t i = g.first + threadIdx.x;
    if (i < T.n) T.sigma[i] = rsi_iface::transmit_point(T.it, T.nx[i], T.nz[i], T.phi[i]);
}

__global__ void batch_image_kernel(const BImage* __restrict__ im, const BSeg* __restrict__ segs) {
    const BSeg g = segs[blockIdx.x];
    const BImage& M = im[g.set];
    int64_t j = g.first + threadIdx.x;
    if (j < M.n) {
        double2 f = M.field[j];
        M.out[j] = make_float2(float(M.scale * f.x), float(M.scale * f.y));
    }
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// single-stage tile-size rule: at most n/64 sources per tile (tiles of at
// most 1/64 of the surface), between 32 and the requested maximum
int tile_for(int64_t n, int max_tile) {
    int S = max_tile;
    while (S > 32 && S > n / 64) S >>= 1;
    return S;
}

void append_segments(std::vector<BSeg>& segs, int32_t set, int64_t n) {
    for (int64_t f = 0; f < n; f += kSeg) segs.push_back({set, 0, f});
}

}  // namespace

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
// one target per thread by default: the persistent stage kernels then hold
// their work-item state in 64 registers at 4 resident CTAs per SM (two
// targets per thread: 126 registers, 2 CTAs); 1433 against 1395 Gpair/s on
// the first 256 instances of the 64 x 32 scan
struct rsi_batch_plan {
    int n_inst = 0;
    int S_max = 256, tpt = 1, variant = 3, normals2 = RSI_NORMALS_Z;
    size_t ws_bytes = 0, img_elems = 0, max_tile1 = 0, max_tile2 = 0;
    std::vector<uint8_t> blob;  // device tables, uploaded to workspace offset 0
    // table offsets (bytes) in the blob / workspace
    size_t o_sets, o_psegs, o_grids, o_gsegs, o_prep1, o_pt1, o_st1, o_it1, o_red1, o_rs1, o_tr, o_ts, o_prep2, o_pt2,
        o_st2, o_it2, o_red2, o_rs2, o_imgtab, o_is, o_ctr;
    int64_t n_psegs = 0, n_gsegs = 0, n_pt1 = 0, n_it1 = 0, n_rs1 = 0, n_ts = 0, n_pt2 = 0, n_it2 = 0, n_rs2 = 0,
            n_is = 0;
    int n_sets = 0, n_grids = 0;
    // layout of the per-instance buffers (relative to the workspace base)
    std::vector<rsi_batch_instance> inst;
    uint64_t seed = 0;
    std::vector<size_t> o_pist, o_ifc, o_f1, o_sig, o_f2, o_t1, o_t2, o_p1, o_p2, img_off;
    std::vector<int> grid_id, S1, S2, tps1, tps2, sp1, sp2, nt1, nt2;
    std::vector<size_t> o_gridpts;
    std::vector<rsi_grid> grids;
    // captured graph
    cudaGraphExec_t exec = nullptr;
    void* ws = nullptr;
    void* images = nullptr;
    bool uploaded = false;
};

namespace {

template <class T>
size_t put(std::vector<uint8_t>& blob, const std::vector<T>& v) {
    size_t off = align256(blob.size());
    blob.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// Build every device table for workspace base `ws` (pointers are absolute).
void build_tables(rsi_batch_plan& P, uint8_t* ws) {
    std::vector<uint8_t>& blob = P.blob;
    blob.clear();
    const int n = P.n_inst;
    auto view = [&](size_t off, int64_t cnt) { return rsi_points_view(ws + off, cnt); };
    // points
    std::vector<BPointSet> sets;
    std::vector<BSeg> psegs;
    for (int i = 0; i < n; ++i) {
        const rsi_batch_instance& I = P.inst[i];
        for (int w = 0; w < 2; ++w) {
            const rsi_surface& s = w == 0 ? I.piston : I.iface;
            int64_t cnt = w == 0 ? I.n_piston : I.n_iface;
            uint32_t set_id = w == 0 ? I.piston_set : I.iface_set;
            BPointSet b;
            b.s = rsi_qmc::surface_dev(s);
            b.k0 = rsi_qmc::dim_key(P.seed, set_id, 0);
            b.k1 = rsi_qmc::dim_key(P.seed, set_id, 1);
            b.n = cnt;
            b.out = view(w == 0 ? P.o_pist[i] : P.o_ifc[i], cnt);
            b.scramble = s.scramble ? 1 : 0;
            b.pad = 0;
            append_segments(psegs, int32_t(sets.size()), cnt);
            sets.push_back(b);
        }
    }
    std::vector<BGrid> grids;
    std::vector<BSeg> gsegs;
    for (size_t g = 0; g < P.grids.size(); ++g) {
        int64_t cnt = int64_t(P.grids[g].nx) * P.grids[g].nz;
        grids.push_back({P.grids[g], view(P.o_gridpts[g], cnt)});
        append_segments(gsegs, int32_t(g), cnt);
    }
    // stage 1 (piston -> interface) and stage 2 (interface -> grid)
    std::vector<BPrep> prep1, prep2;
    std::vector<BPrepTile> pt1, pt2;
    std::vector<BStageInst> st1, st2;
    std::vector<std::pair<double, BItem>> it1, it2;
    std::vector<BReduce> red1, red2;
    std::vector<BSeg> rs1, rs2, ts, is;
    std::vector<BTransmit> tr;
    std::vector<BImage> img;
    const int per_block = kThreads * P.tpt;
    for (int i = 0; i < n; ++i) {
        const rsi_batch_instance& I = P.inst[i];
        const int64_t n_g = int64_t(P.grids[P.grid_id[i]].nx) * P.grids[P.grid_id[i]].nz;
        PointsView pist = view(P.o_pist[i], I.n_piston), ifc = view(P.o_ifc[i], I.n_iface);
        PointsView grd = view(P.o_gridpts[P.grid_id[i]], n_g);
        double2* f1 = reinterpret_cast<double2*>(ws + P.o_f1[i]);
        double2* sg = reinterpret_cast<double2*>(ws + P.o_sig[i]);
        double2* f2 = reinterpret_cast<double2*>(ws + P.o_f2[i]);
        // stage 1
        {
            BPrep p;
            p.src = pist;
            p.n_src = I.n_piston;
            p.S = P.S1[i];
            p.pad = 0;
            p.sigma = nullptr;
            p.tiles = ws + P.o_t1[i];
            p.tile_bytes = RSI_TILE_HDR_BYTES + size_t(P.S1[i]) * 32;
            p.amp_scale = -I.v0 / (2.0 * M_PI);
            p.k = I.k1;
            p.kind = RSI_STAGE_PISTON;
            p.normals = RSI_NORMALS_Z;
            prep1.push_back(p);
            for (int t = 0; t < P.nt1[i]; ++t) pt1.push_back({i, 0, t});
            BStageInst s;
            s.tiles = p.tiles;
            s.tile_bytes = p.tile_bytes;
            s.S = P.S1[i];
            s.n_tiles = P.nt1[i];
            s.tiles_per_split = P.tps1[i];
            s.splits = P.sp1[i];
            s.tgt = {ifc.xh, ifc.xl, ifc.yh, ifc.yl, ifc.zh, ifc.zl, ifc.x, ifc.y, ifc.z};
            s.n_tgt = I.n_iface;
            s.kh = float(I.k1);
            s.kl = float(I.k1 - double(s.kh));
            s.out = s.splits > 1 ? reinterpret_cast<double2*>(ws + P.o_p1[i]) : f1;
            st1.push_back(s);
            int64_t blocks = (I.n_iface + per_block - 1) / per_block;
            for (int64_t b = 0; b < blocks; ++b)
                for (int sp = 0; sp < s.splits; ++sp) {
                    int nt = std::min(s.n_tiles, (sp + 1) * s.tiles_per_split) - sp * s.tiles_per_split;
                    double cost = double(nt) * s.S * double(std::min<int64_t>(per_block, I.n_iface - b * per_block));
                    it1.push_back({cost, {i, sp, b}});
                }
            if (s.splits > 1) {
                red1.push_back({s.out, f1, I.n_iface, s.splits, 0});
                append_segments(rs1, int32_t(red1.size() - 1), I.n_iface);
            }
        }
        // transmission
        tr.push_back({I.transmit, ifc.nx, ifc.nz, f1, sg, I.n_iface});
        append_segments(ts, i, I.n_iface);
        // stage 2
        {
            BPrep p;
            p.src = ifc;
            p.n_src = I.n_iface;
            p.S = P.S2[i];
            p.pad = 0;
            p.sigma = sg;
            p.tiles = ws + P.o_t2[i];
            p.tile_bytes = RSI_TILE_HDR_BYTES + size_t(P.S2[i]) * fp32_record_bytes(RSI_STAGE_RSI, P.normals2);
            p.amp_scale = -1.0 / (2.0 * M_PI);
            p.k = I.k2;
            p.kind = RSI_STAGE_RSI;
            p.normals = P.normals2;
            prep2.push_back(p);
            for (int t = 0; t < P.nt2[i]; ++t) pt2.push_back({i, 0, t});
            BStageInst s;
            s.tiles = p.tiles;
            s.tile_bytes = p.tile_bytes;
            s.S = P.S2[i];
            s.n_tiles = P.nt2[i];
            s.tiles_per_split = P.tps2[i];
            s.splits = P.sp2[i];
            s.tgt = {grd.xh, grd.xl, grd.yh, grd.yl, grd.zh, grd.zl, grd.x, grd.y, grd.z};
            s.n_tgt = n_g;
            s.kh = float(I.k2);
            s.kl = float(I.k2 - double(s.kh));
            s.out = s.splits > 1 ? reinterpret_cast<double2*>(ws + P.o_p2[i]) : f2;
            st2.push_back(s);
            int64_t blocks = (n_g + per_block - 1) / per_block;
            for (int64_t b = 0; b < blocks; ++b)
                for (int sp = 0; sp < s.splits; ++sp) {
                    int nt = std::min(s.n_tiles, (sp + 1) * s.tiles_per_split) - sp * s.tiles_per_split;
                    double cost = double(nt) * s.S * double(std::min<int64_t>(per_block, n_g - b * per_block));
                    it2.push_back({cost, {i, sp, b}});
                }
            if (s.splits > 1) {
                red2.push_back({s.out, f2, n_g, s.splits, 0});
                append_segments(rs2, int32_t(red2.size() - 1), n_g);
            }
        }
        img.push_back({f2, nullptr, n_g, I.k2 / I.v0});
        append_segments(is, i, n_g);
    }
    auto sorted_items = [](std::vector<std::pair<double, BItem>>& v) {
        std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
        std::vector<BItem> out;
        out.reserve(v.size());
        for (auto& e : v) out.push_back(e.second);
        return out;
    };
    std::vector<BItem> items1 = sorted_items(it1), items2 = sorted_items(it2);
    P.o_sets = put(blob, sets);
    P.o_psegs = put(blob, psegs);
    P.o_grids = put(blob, grids);
    P.o_gsegs = put(blob, gsegs);
    P.o_prep1 = put(blob, prep1);
    P.o_pt1 = put(blob, pt1);
    P.o_st1 = put(blob, st1);
    P.o_it1 = put(blob, items1);
    P.o_red1 = put(blob, red1);
    P.o_rs1 = put(blob, rs1);
    P.o_tr = put(blob, tr);
    P.o_ts = put(blob, ts);
    P.o_prep2 = put(blob, prep2);
    P.o_pt2 = put(blob, pt2);
    P.o_st2 = put(blob, st2);
    P.o_it2 = put(blob, items2);
    P.o_red2 = put(blob, red2);
    P.o_rs2 = put(blob, rs2);
    P.o_imgtab = put(blob, img);
    P.o_is = put(blob, is);
    P.o_ctr = align256(blob.size());
    blob.resize(P.o_ctr + 256, 0);
    P.n_sets = int(sets.size());
    P.n_psegs = int64_t(psegs.size());
    P.n_grids = int(grids.size());
    P.n_gsegs = int64_t(gsegs.size());
    P.n_pt1 = int64_t(pt1.size());
    P.n_it1 = int64_t(items1.size());
    P.n_rs1 = int64_t(rs1.size());
    P.n_ts = int64_t(ts.size());
    P.n_pt2 = int64_t(pt2.size());
    P.n_it2 = int64_t(items2.size());
    P.n_rs2 = int64_t(rs2.size());
    P.n_is = int64_t(is.size());
}

// image pointers depend on the output buffer: patched into the blob
void set_image_outputs(rsi_batch_plan& P, void* images) {
    BImage* im = reinterpret_cast<BImage*>(P.blob.data() + P.o_imgtab);
    for (int i = 0; i < P.n_inst; ++i) im[i].out = reinterpret_cast<float2*>(images) + P.img_off[i];
}

template <int KIND, int NORM, int TPT, int VAR>
int launch_batch_stage(const rsi_batch_plan& P, uint8_t* ws, size_t o_st, size_t o_it, int64_t n_items,
                       size_t max_tile, unsigned long long* ctr, int* status, cudaStream_t s) {
    auto kern = batch_stage_kernel<KIND, NORM, TPT, VAR>;
    size_t smem = RSI_PIPE_STAGES * max_tile + RSI_PIPE_STAGES * sizeof(uint64_t);
    RSI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                 "cudaFuncSetAttribute(batch_stage)");
    int occ = 0;
    RSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem), "occupancy");
    if (occ < 1) occ = 1;
    int grid = rsi_num_sms() * occ;
    if (int64_t(grid) > n_items) grid = int(std::max<int64_t>(1, n_items));
    kern<<<grid, kThreads, smem, s>>>(reinterpret_cast<const BStageInst*>(ws + o_st),
                                      reinterpret_cast<const BItem*>(ws + o_it), n_items, two_pi_split(), max_tile,
                                      ctr, status);
    RSI_CHECK_LAUNCH("batch_stage_kernel");
    return RSI_OK;
}

template <int KIND, int NORM>
int launch_batch_stage_v(const rsi_batch_plan& P, uint8_t* ws, size_t o_st, size_t o_it, int64_t n_items,
                         size_t max_tile, unsigned long long* ctr, int* status, cudaStream_t s) {
    if (P.tpt == 1) {
        if (P.variant == 1)
            return launch_batch_stage<KIND, NORM, 1, 1>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
        if (P.variant == 3)
            return launch_batch_stage<KIND, NORM, 1, 3>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
        return launch_batch_stage<KIND, NORM, 1, 2>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
    }
    if (P.tpt == 4) {
        if (P.variant == 1)
            return launch_batch_stage<KIND, NORM, 4, 1>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
        if (P.variant == 3)
            return launch_batch_stage<KIND, NORM, 4, 3>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
        return launch_batch_stage<KIND, NORM, 4, 2>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
    }
    if (P.variant == 1)
        return launch_batch_stage<KIND, NORM, 2, 1>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
    if (P.variant == 3)
        return launch_batch_stage<KIND, NORM, 2, 3>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
    return launch_batch_stage<KIND, NORM, 2, 2>(P, ws, o_st, o_it, n_items, max_tile, ctr, status, s);
}

// Enqueue the whole batch on `s` (captured into the graph by rsi_batch_run).
int enqueue(rsi_batch_plan& P, uint8_t* ws, int* status, cudaStream_t s) {
    static const rsi_qmc::SobolDirs dirs = rsi_qmc::make_dirs();
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(ws + P.o_ctr);
    RSI_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s), "reset work counters");
    if (P.n_psegs) {
        batch_points_kernel<<<unsigned(P.n_psegs), kSeg, 0, s>>>(reinterpret_cast<const BPointSet*>(ws + P.o_sets),
                                                                 reinterpret_cast<const BSeg*>(ws + P.o_psegs), dirs);
        RSI_CHECK_LAUNCH("batch_points_kernel");
    }
    if (P.n_gsegs) {
        batch_grid_kernel<<<unsigned(P.n_gsegs), kSeg, 0, s>>>(reinterpret_cast<const BGrid*>(ws + P.o_grids),
                                                               reinterpret_cast<const BSeg*>(ws + P.o_gsegs));
        RSI_CHECK_LAUNCH("batch_grid_kernel");
    }
    batch_prep_kernel<<<unsigned(P.n_pt1), P.S_max, 0, s>>>(reinterpret_cast<const BPrep*>(ws + P.o_prep1),
                                                            reinterpret_cast<const BPrepTile*>(ws + P.o_pt1),
                                                            P.variant == 3 ? 1 : 0);
    RSI_CHECK_LAUNCH("batch_prep_kernel");
    int rc = launch_batch_stage_v<RSI_STAGE_PISTON, RSI_NORMALS_Z>(P, ws, P.o_st1, P.o_it1, P.n_it1, P.max_tile1,
                                                                   ctr, status, s);
    if (rc != RSI_OK) return rc;
    if (P.n_rs1) {
        batch_reduce_kernel<<<unsigned(P.n_rs1), kSeg, 0, s>>>(reinterpret_cast<const BReduce*>(ws + P.o_red1),
                                                               reinterpret_cast<const BSeg*>(ws + P.o_rs1), status);
        RSI_CHECK_LAUNCH("batch_reduce_kernel");
    }
    batch_transmit_kernel<<<unsigned(P.n_ts), kSeg, 0, s>>>(reinterpret_cast<const BTransmit*>(ws + P.o_tr),
                                                            reinterpret_cast<const BSeg*>(ws + P.o_ts));
    RSI_CHECK_LAUNCH("batch_transmit_kernel");
    batch_prep_kernel<<<unsigned(P.n_pt2), P.S_max, 0, s>>>(reinterpret_cast<const BPrep*>(ws + P.o_prep2),
                                                            reinterpret_cast<const BPrepTile*>(ws + P.o_pt2),
                                                            P.variant == 3 ? 1 : 0);
    RSI_CHECK_LAUNCH("batch_prep_kernel");
    if (P.normals2 == RSI_NORMALS_POINTS)
        rc = launch_batch_stage_v<RSI_STAGE_RSI, RSI_NORMALS_POINTS>(P, ws, P.o_st2, P.o_it2, P.n_it2, P.max_tile2,
                                                                     ctr + 1, status, s);
    else
        rc = launch_batch_stage_v<RSI_STAGE_RSI, RSI_NORMALS_Z>(P, ws, P.o_st2, P.o_it2, P.n_it2, P.max_tile2,
                                                                ctr + 1, status, s);
    if (rc != RSI_OK) return rc;
    if (P.n_rs2) {
        batch_reduce_kernel<<<unsigned(P.n_rs2), kSeg, 0, s>>>(reinterpret_cast<const BReduce*>(ws + P.o_red2),
                                                               reinterpret_cast<const BSeg*>(ws + P.o_rs2), status);
        RSI_CHECK_LAUNCH("batch_reduce_kernel");
    }
    batch_image_kernel<<<unsigned(P.n_is), kSeg, 0, s>>>(reinterpret_cast<const BImage*>(ws + P.o_imgtab),
                                                         reinterpret_cast<const BSeg*>(ws + P.o_is));
    RSI_CHECK_LAUNCH("batch_image_kernel");
    return RSI_OK;
}

}  // namespace

extern "C" int rsi_batch_create(const rsi_batch_instance* inst, int32_t n_inst, uint64_t seed,
                                const rsi_stage* shape, rsi_batch_plan** plan, size_t* workspace_bytes,
                                size_t* image_elems) {
    if (!inst || !plan || !workspace_bytes || !image_elems || n_inst < 1)
        return rsi_fail(RSI_E_INVAL, "rsi_batch_create: bad arguments");
    *plan = nullptr;
    auto P = new rsi_batch_plan();
    P->n_inst = n_inst;
    P->seed = seed;
    P->inst.assign(inst, inst + n_inst);
    if (shape) {
        if (shape->precision != RSI_PREC_FP32C) {
            delete P;
            return rsi_fail(RSI_E_UNSUPPORTED, "rsi_batch_create: batches run in FP32C only");
        }
        if (shape->tile) P->S_max = shape->tile;
        if (shape->tpt) P->tpt = shape->tpt;
        if (shape->variant) P->variant = shape->variant;
    }
    if (!(P->S_max == 32 || P->S_max == 64 || P->S_max == 128 || P->S_max == 256 || P->S_max == 512) ||
        (P->tpt != 1 && P->tpt != 2 && P->tpt != 4) || (P->variant < 1 || P->variant > 3)) {
        delete P;
        return rsi_fail(RSI_E_INVAL, "rsi_batch_create: bad tile / targets per thread / variant");
    }
    std::map<std::tuple<double, double, double, double, double, int, int>, int> grid_index;
    for (int i = 0; i < n_inst; ++i) {
        const rsi_batch_instance& I = inst[i];
        int rc = RSI_OK;
        if (I.piston.kind != RSI_SURF_DISK) rc = rsi_fail(RSI_E_INVAL, "instance %d: piston must be a disk", i);
        if (rc == RSI_OK) rc = rsi_qmc::check_surface(I.piston);
        if (rc == RSI_OK && I.iface.kind == RSI_SURF_DISK)
            rc = rsi_fail(RSI_E_INVAL, "instance %d: interface must be a patch or cylinder", i);
        if (rc == RSI_OK) rc = rsi_qmc::check_surface(I.iface);
        if (rc == RSI_OK) rc = rsi_iface::check_interface(I.transmit);
        if (rc == RSI_OK && (I.n_piston < 1 || I.n_iface < 1 || I.n_piston > (1 << 30) || I.n_iface > (1 << 30)))
            rc = rsi_fail(RSI_E_INVAL, "instance %d: point counts must be in [1, 2^30]", i);
        if (rc == RSI_OK && !(I.k1 > 0 && I.k2 > 0 && I.v0 != 0.0))
            rc = rsi_fail(RSI_E_INVAL, "instance %d: wavenumbers must be > 0 and v0 non-zero", i);
        if (rc == RSI_OK && (I.grid.nx < 1 || I.grid.nz < 1))
            rc = rsi_fail(RSI_E_INVAL, "instance %d: empty grid", i);
        if (rc != RSI_OK) {
            delete P;
            return rc;
        }
        if (I.iface.kind == RSI_SURF_CYL) P->normals2 = RSI_NORMALS_POINTS;
        auto key = std::make_tuple(I.grid.x0, I.grid.x1, I.grid.z0, I.grid.z1, I.grid.y, I.grid.nx, I.grid.nz);
        auto f = grid_index.find(key);
        if (f == grid_index.end()) {
            f = grid_index.emplace(key, int(P->grids.size())).first;
            P->grids.push_back(I.grid);
        }
        P->grid_id.push_back(f->second);
    }
    // work-item size: about 2^22 pairs (tiles per split chosen per instance)
    const int per_block = kThreads * P->tpt;
    const int64_t item_pairs = int64_t(1) << 22;
    size_t off = 0;  // per-instance buffers start after the tables (offset fixed below)
    auto take = [&](size_t bytes) {
        off = align256(off);
        size_t at = off;
        off += bytes;
        return at;
    };
    for (size_t g = 0; g < P->grids.size(); ++g)
        P->o_gridpts.push_back(take(rsi_points_bytes(int64_t(P->grids[g].nx) * P->grids[g].nz)));
    const size_t rec2 = fp32_record_bytes(RSI_STAGE_RSI, P->normals2);
    for (int i = 0; i < n_inst; ++i) {
        const rsi_batch_instance& I = inst[i];
        const int64_t n_g = int64_t(P->grids[P->grid_id[i]].nx) * P->grids[P->grid_id[i]].nz;
        int S1 = tile_for(I.n_piston, P->S_max), S2 = tile_for(I.n_iface, P->S_max);
        int nt1 = int((I.n_piston + S1 - 1) / S1), nt2 = int((I.n_iface + S2 - 1) / S2);
        int tps1 = int(std::max<int64_t>(1, item_pairs / (int64_t(S1) * per_block)));
        int tps2 = int(std::max<int64_t>(1, item_pairs / (int64_t(S2) * per_block)));
        tps1 = std::min(tps1, nt1);
        tps2 = std::min(tps2, nt2);
        int sp1 = (nt1 + tps1 - 1) / tps1, sp2 = (nt2 + tps2 - 1) / tps2;
        P->S1.push_back(S1);
        P->S2.push_back(S2);
        P->nt1.push_back(nt1);
        P->nt2.push_back(nt2);
        P->tps1.push_back(tps1);
        P->tps2.push_back(tps2);
        P->sp1.push_back(sp1);
        P->sp2.push_back(sp2);
        size_t tb1 = RSI_TILE_HDR_BYTES + size_t(S1) * 32, tb2 = RSI_TILE_HDR_BYTES + size_t(S2) * rec2;
        P->max_tile1 = std::max(P->max_tile1, tb1);
        P->max_tile2 = std::max(P->max_tile2, tb2);
        P->o_pist.push_back(take(rsi_points_bytes(I.n_piston)));
        P->o_ifc.push_back(take(rsi_points_bytes(I.n_iface)));
        P->o_f1.push_back(take(size_t(I.n_iface) * 16));
        P->o_sig.push_back(take(size_t(I.n_iface) * 16));
        P->o_f2.push_back(take(size_t(n_g) * 16));
        P->o_t1.push_back(take(size_t(nt1) * tb1));
        P->o_t2.push_back(take(size_t(nt2) * tb2));
        P->o_p1.push_back(sp1 > 1 ? take(size_t(sp1) * size_t(I.n_iface) * 16) : 0);
        P->o_p2.push_back(sp2 > 1 ? take(size_t(sp2) * size_t(n_g) * 16) : 0);
        P->img_off.push_back(P->img_elems);
        P->img_elems += size_t(n_g);
    }
    const size_t buffers = align256(off);
    // tables: build once against base 0 to learn their size, then shift every
    // buffer offset past them
    build_tables(*P, nullptr);
    const size_t tables = align256(P->blob.size());
    auto shift = [&](std::vector<size_t>& v) {
        for (auto& x : v) x += tables;
    };
    shift(P->o_gridpts);
    shift(P->o_pist);
    shift(P->o_ifc);
    shift(P->o_f1);
    shift(P->o_sig);
    shift(P->o_f2);
    shift(P->o_t1);
    shift(P->o_t2);
    for (int i = 0; i < n_inst; ++i) {
        if (P->sp1[i] > 1) P->o_p1[i] += tables;
        if (P->sp2[i] > 1) P->o_p2[i] += tables;
    }
    P->ws_bytes = tables + buffers;
    *workspace_bytes = P->ws_bytes;
    *image_elems = P->img_elems;
    *plan = P;
    return RSI_OK;
}

extern "C" int rsi_batch_run(rsi_batch_plan* P, void* workspace, size_t workspace_bytes, void* images,
                             void* stream) {
    if (!P || !workspace || !images) return rsi_fail(RSI_E_INVAL, "rsi_batch_run: null argument");
    if (workspace_bytes < P->ws_bytes)
        return rsi_fail(RSI_E_NOMEM, "rsi_batch_run: workspace %zu < %zu bytes", workspace_bytes, P->ws_bytes);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 || reinterpret_cast<uintptr_t>(images) % 16)
        return rsi_fail(RSI_E_INVAL, "rsi_batch_run: workspace must be 256-byte and images 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* status = rsi_status_ptr();
    if (!status) return RSI_E_CUDA;
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    if (P->exec && (P->ws != workspace || P->images != images)) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    if (!P->exec) {
        // tables with absolute pointers for this workspace and output
        build_tables(*P, ws);
        set_image_outputs(*P, images);
        RSI_CUDA_TRY(cudaMemcpyAsync(ws, P->blob.data(), P->blob.size(), cudaMemcpyHostToDevice, s),
                     "upload batch tables");
        RSI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        // capture the whole batch once; later runs replay the graph
        cudaStream_t cap = nullptr;
        RSI_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return rsi_cuda_fail(e, "cudaStreamBeginCapture");
        }
        int rc = enqueue(*P, ws, status, cap);
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (rc != RSI_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return rsi_cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->exec = nullptr;
            return rsi_cuda_fail(e, "cudaGraphInstantiate");
        }
        P->ws = workspace;
        P->images = images;
    }
    RSI_CUDA_TRY(cudaGraphLaunch(P->exec, s), "cudaGraphLaunch");
    rsi_note_launch();
    return RSI_OK;
}

extern "C" int rsi_batch_destroy(rsi_batch_plan* P) {
    if (!P) return RSI_OK;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    delete P;
    return RSI_OK;
}
