// stage.cu -- rsi_propagate_stage: resolves the launch shape, stages the
// source tiles, runs the FP32C or FP64 source x target kernel and, when the
// sources are split across CTAs, reduces the partial sums in a fixed order
// (step a6).
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stage.cuh"

// ---------------------------------------------------------------------------
// optional CUDA-event timing of the main source x target kernel
// ---------------------------------------------------------------------------
namespace {
struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;
    double pairs;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t pooled_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

extern "C" int rsi_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto& t : g_timed) {
        g_event_pool.push_back(t.a);
        g_event_pool.push_back(t.b);
    }
    g_timed.clear();
    g_timing = on != 0;
    return RSI_OK;
}

extern "C" int rsi_timing_read(int32_t kind, double* total_ms, int64_t* launches, double* pairs) {
    if (!total_ms || !launches || !pairs) return rsi_fail(RSI_E_INVAL, "rsi_timing_read: null argument");
    std::lock_guard<std::mutex> lk(g_tmu);
    double ms = 0.0, pr = 0.0;
    int64_t n = 0;
    for (auto& t : g_timed) {
        if (t.kind != kind) continue;
        RSI_CUDA_TRY(cudaEventSynchronize(t.b), "cudaEventSynchronize");
        float e = 0.0f;
        RSI_CUDA_TRY(cudaEventElapsedTime(&e, t.a, t.b), "cudaEventElapsedTime");
        ms += e;
        pr += t.pairs;
        ++n;
    }
    *total_ms = ms;
    *launches = n;
    *pairs = pr;
    return RSI_OK;
}

TwoPiSplit two_pi_split() {
    // Split 2 pi (double) into p1 + p2 + p3 with p1, p2 rounded to 11
    // significant bits (Cody & Waite 1980).
    const double two_pi = 2.0 * M_PI;
    auto trunc_bits = [](double v, int bits) {
        int e;
        double m = frexp(v, &e);  // v = m 2^e, 0.5 <= |m| < 1
        double scaled = ldexp(m, bits);
        return ldexp(trunc(scaled), e - bits);
    };
    TwoPiSplit t;
    double p1 = trunc_bits(two_pi, 11);
    double p2 = trunc_bits(two_pi - p1, 11);
    t.p1 = float(p1);
    t.p2 = float(p2);
    t.p3 = float(two_pi - p1 - p2);
    t.inv = float(1.0 / two_pi);
    return t;
}

namespace {

__global__ void reduce_partials_kernel(const double2* __restrict__ part, int splits, int64_t n,
                                       double2* __restrict__ out, int* status) {
    int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    // Neumaier summation over the splits in index order
    double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
    for (int s = 0; s < splits; ++s) {
        double2 v = part[size_t(s) * size_t(n) + size_t(j)];
        double t = sr + v.x;
        cr += (fabs(sr) >= fabs(v.x)) ? (sr - t) + v.x : (v.x - t) + sr;
        sr = t;
        t = si + v.y;
        ci += (fabs(si) >= fabs(v.y)) ? (si - t) + v.y : (v.y - t) + si;
        si = t;
    }
    double re = sr + cr, im = si + ci;
    if (!isfinite(re) || !isfinite(im)) atomicExch(status, RSI_DEV_NONFINITE);
    out[j] = make_double2(re, im);
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Plan {
    int S, tpt, variant, splits, tiles_per_split, n_tiles;
    size_t tile_bytes, tiles_bytes, partial_bytes;
};

bool valid_tile(int S) { return S == 32 || S == 64 || S == 128 || S == 256 || S == 512; }

// max_auto_splits bounds the automatic split count (st.splits == 0); the
// choice below it still minimises the busiest SM's work.
int make_plan(const rsi_stage& st, int64_t n_src, int64_t n_tgt, Plan& p, int max_auto_splits = 128) {
    if (st.kind != RSI_STAGE_PISTON && st.kind != RSI_STAGE_RSI)
        return rsi_fail(RSI_E_INVAL, "unknown stage kind %d", st.kind);
    if (st.precision != RSI_PREC_FP64 && st.precision != RSI_PREC_FP32C)
        return rsi_fail(RSI_E_INVAL, "unknown precision %d", st.precision);
    if (st.kind == RSI_STAGE_RSI && (st.normals < RSI_NORMALS_Z || st.normals > RSI_NORMALS_POINTS_NEG))
        return rsi_fail(RSI_E_INVAL, "unknown normals mode %d", st.normals);
    if (n_src < 1 || n_tgt < 1) return rsi_fail(RSI_E_INVAL, "empty source or target set");
    if (n_src > (int64_t(1) << 31) || n_tgt > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "more than 2^31 sources or targets");
    if (!(st.k > 0) || !isfinite(st.k)) return rsi_fail(RSI_E_INVAL, "wavenumber must be finite and > 0");
    const bool fp32 = st.precision == RSI_PREC_FP32C;
    if (st.tile) {
        p.S = st.tile;
    } else if (fp32) {
        // The FP32 offset term k (r - R) carries ~2^-23 k (tile radius) of
        // phase error.  Cell-ordered QMC tiles of S points cover S/n of the
        // surface, so keep S <= n/64 for small sets (tiles of at most 1/64 of
        // the surface), between 32 and 256 sources.
        int64_t cap = n_src / 64;
        p.S = 256;
        while (p.S > 32 && p.S > cap) p.S >>= 1;
    } else {
        p.S = 64;
    }
    if (!valid_tile(p.S)) return rsi_fail(RSI_E_INVAL, "tile must be 32, 64, 128, 256 or 512 (got %d)", st.tile);
    if (fp32) {
        // 2 targets per thread keeps 80 registers and 3 CTAs (24 warps) per SM;
        // it measured faster than 4 at every tile size
        p.tpt = st.tpt ? st.tpt : 2;
        if (p.tpt != 1 && p.tpt != 2 && p.tpt != 4)
            return rsi_fail(RSI_E_INVAL, "FP32C targets per thread must be 1, 2 or 4");
        p.variant = st.variant ? st.variant : 3;  // packed source pairs: ~10% faster than 2 on every shape
        if (p.variant < 1 || p.variant > 3) return rsi_fail(RSI_E_INVAL, "variant must be 1, 2 or 3");
    } else {
        p.tpt = 1;
        if (st.tpt && st.tpt != 1) return rsi_fail(RSI_E_INVAL, "FP64 targets per thread must be 1");
        p.variant = 0;
    }
    p.n_tiles = int((n_src + p.S - 1) / p.S);
    p.tile_bytes = RSI_TILE_HDR_BYTES +
                   size_t(p.S) * (fp32 ? fp32_record_bytes(st.kind, base_normals(st.normals)) : fp64_record_bytes());
    p.tiles_bytes = align256(size_t(p.n_tiles) * p.tile_bytes);

    const int threads = fp32 ? fp32_threads() : fp64_threads();
    const int64_t blocks = (n_tgt + int64_t(threads) * p.tpt - 1) / (int64_t(threads) * p.tpt);
    int splits = st.splits;
    if (splits < 0) return rsi_fail(RSI_E_INVAL, "splits must be >= 0");
    if (splits == 0) {
        StageArgs probe = {};
        probe.kind = st.kind;
        probe.normals = st.normals;
        probe.tpt = p.tpt;
        probe.variant = p.variant;
        probe.tile_bytes = p.tile_bytes;
        int occ = fp32 ? stage_occupancy_fp32(probe) : stage_occupancy_fp64(probe);
        int64_t slots = int64_t(rsi_num_sms()) * occ;
        // minimise (waves x tiles per CTA), the time of the busiest SM
        int64_t best_cost = INT64_MAX;
        splits = 1;
        for (int s = 1; s <= max_auto_splits && s <= p.n_tiles; ++s) {
            int64_t tps = (p.n_tiles + s - 1) / s;
            int64_t s_act = (p.n_tiles + tps - 1) / tps;
            int64_t waves = (blocks * s_act + slots - 1) / slots;
            int64_t cost = waves * tps;
            if (cost < best_cost) {
                best_cost = cost;
                splits = int(s_act);
            }
        }
    }
    if (splits > p.n_tiles) splits = p.n_tiles;
    if (splits > 65535) return rsi_fail(RSI_E_INVAL, "too many splits");
    p.tiles_per_split = (p.n_tiles + splits - 1) / splits;
    p.splits = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    p.partial_bytes = p.splits > 1 ? align256(size_t(p.splits) * size_t(n_tgt) * sizeof(double2)) : 0;
    return RSI_OK;
}

}  // namespace

extern "C" size_t rsi_stage_workspace_bytes(const rsi_stage* st, int64_t n_src, int64_t n_tgt) {
    if (!st) return 0;
    Plan p;
    if (make_plan(*st, n_src, n_tgt, p) != RSI_OK) return 0;
    return p.tiles_bytes + p.partial_bytes;
}

size_t rsi_stage_workspace_bytes_capped(const rsi_stage* st, int64_t n_src, int64_t n_tgt, int max_splits,
                                        int* splits) {
    if (!st || max_splits < 1) return 0;
    Plan p;
    if (make_plan(*st, n_src, n_tgt, p, max_splits) != RSI_OK) return 0;
    if (splits) *splits = p.splits;
    return p.tiles_bytes + p.partial_bytes;
}

extern "C" int rsi_propagate_stage(const rsi_stage* st, const void* src_points, int64_t n_src,
                                   const double* src_sigma, const void* tgt_points, int64_t n_tgt,
                                   double* tgt_field, void* workspace, size_t workspace_bytes, void* stream) {
    if (!st || !src_points || !tgt_points || !tgt_field || !workspace)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage: null argument");
    if (st->kind == RSI_STAGE_RSI && !src_sigma)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage: RSI stage needs a source density");
    if (st->kind == RSI_STAGE_PISTON && !isfinite(st->v0))
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage: v0 must be finite");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 || reinterpret_cast<uintptr_t>(src_points) % 256 ||
        reinterpret_cast<uintptr_t>(tgt_points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage: point sets and workspace must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(tgt_field) % 16 || (src_sigma && reinterpret_cast<uintptr_t>(src_sigma) % 16))
        return rsi_fail(RSI_E_INVAL, "rsi_propagate_stage: complex arrays must be 16-byte aligned");
    Plan p;
    int rc = make_plan(*st, n_src, n_tgt, p);
    if (rc != RSI_OK) return rc;
    if (workspace_bytes < p.tiles_bytes + p.partial_bytes)
        return rsi_fail(RSI_E_NOMEM, "rsi_propagate_stage: workspace %zu < %zu bytes", workspace_bytes,
                        p.tiles_bytes + p.partial_bytes);
    int* status = rsi_status_ptr();
    if (!status) return RSI_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp32 = st->precision == RSI_PREC_FP32C;
    PointsView src = rsi_points_view(const_cast<void*>(src_points), n_src);
    PointsView tgt = rsi_points_view(const_cast<void*>(tgt_points), n_tgt);
    uint8_t* tiles = static_cast<uint8_t*>(workspace);
    const double2* sigma = reinterpret_cast<const double2*>(src_sigma);
    rc = fp32 ? launch_prep_fp32(*st, src, n_src, sigma, p.S, tiles, p.tile_bytes, p.n_tiles, s, p.variant == 3)
              : launch_prep_fp64(*st, src, n_src, sigma, p.S, tiles, p.tile_bytes, p.n_tiles, s);
    if (rc != RSI_OK) return rc;

    StageArgs a = {};
    a.kind = st->kind;
    a.normals = st->kind == RSI_STAGE_RSI ? base_normals(st->normals) : RSI_NORMALS_Z;
    a.tpt = p.tpt;
    a.variant = p.variant;
    a.S = p.S;
    a.n_tiles = p.n_tiles;
    a.tiles_per_split = p.tiles_per_split;
    a.splits = p.splits;
    a.n_tgt = n_tgt;
    a.tile_bytes = p.tile_bytes;
    a.tiles = tiles;
    a.tgt = {tgt.xh, tgt.xl, tgt.yh, tgt.yl, tgt.zh, tgt.zl, tgt.x, tgt.y, tgt.z};
    a.k = st->k;
    a.kh = float(st->k);
    a.kl = float(st->k - double(a.kh));
    a.tp = two_pi_split();
    double2* field = reinterpret_cast<double2*>(tgt_field);
    a.out = p.splits > 1 ? reinterpret_cast<double2*>(tiles + p.tiles_bytes) : field;
    a.status = status;
    TimingScope tsc = timing_begin(s);
    rc = fp32 ? launch_stage_fp32(a, s) : launch_stage_fp64(a, s);
    if (rc != RSI_OK) return rc;
    timing_end(tsc, st->kind, double(n_src) * double(n_tgt), s);
    if (p.splits > 1) return launch_reduce_partials(a.out, p.splits, n_tgt, field, status, s);
    return RSI_OK;
}

TimingScope timing_begin(cudaStream_t s) {
    TimingScope t;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        if (!g_timing) return t;
        t.a = pooled_event();
        t.b = pooled_event();
    }
    if (t.a && t.b && cudaEventRecord(t.a, s) != cudaSuccess) t.a = t.b = nullptr;
    return t;
}

void timing_end(TimingScope& t, int kind, double pairs, cudaStream_t s) {
    if (!t.a || !t.b) return;
    if (cudaEventRecord(t.b, s) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timed.push_back({t.a, t.b, kind, pairs});
}

int launch_reduce_partials(const double2* part, int splits, int64_t n, double2* out, int* status, cudaStream_t s) {
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    reduce_partials_kernel<<<blocks, threads, 0, s>>>(part, splits, n, out, status);
    RSI_CHECK_LAUNCH("reduce_partials_kernel");
    return RSI_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, rsi_stage> g_tune_cache;

int ceil_log2(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) < v) ++b;
    return b;
}
}  // namespace

extern "C" int rsi_autotune_stage(const rsi_stage* st, const void* src_points, int64_t n_src,
                                  const double* src_sigma, const void* tgt_points, int64_t n_tgt,
                                  double* tgt_field, void* workspace, size_t workspace_bytes, void* stream,
                                  rsi_stage* best) {
    if (!st || !best) return rsi_fail(RSI_E_INVAL, "rsi_autotune_stage: null argument");
    Plan p0;
    int rc = make_plan(*st, n_src, n_tgt, p0);
    if (rc != RSI_OK) return rc;
    rsi_stage base = *st;
    base.tile = base.tpt = base.splits = base.variant = 0;
    if (st->precision != RSI_PREC_FP32C) {
        *best = base;
        return RSI_OK;
    }
    const auto key = std::make_tuple(st->kind, st->kind == RSI_STAGE_RSI ? base_normals(st->normals) : 0,
                                     ceil_log2(n_src),
                                     ceil_log2(n_tgt));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto f = g_tune_cache.find(key);
        if (f != g_tune_cache.end()) {
            *best = base;
            best->tile = f->second.tile;
            best->tpt = f->second.tpt;
            best->variant = f->second.variant;
            return RSI_OK;
        }
    }
    // largest tile the accuracy rule allows (the default plan's tile)
    const int cap = p0.S;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RSI_CUDA_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    RSI_CUDA_TRY(cudaEventCreate(&e1), "cudaEventCreate");
    float best_ms = 1e30f;
    rsi_stage win = base;
    for (int S = 32; S <= cap; S <<= 1)
        for (int tpt : {1, 2, 4})
            for (int var : {1, 2, 3}) {
                rsi_stage c = base;
                c.tile = S;
                c.tpt = tpt;
                c.variant = var;
                if (rsi_stage_workspace_bytes(&c, n_src, n_tgt) > workspace_bytes) continue;
                float t_best = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    RSI_CUDA_TRY(cudaEventRecord(e0, s), "cudaEventRecord");
                    rc = rsi_propagate_stage(&c, src_points, n_src, src_sigma, tgt_points, n_tgt, tgt_field,
                                             workspace, workspace_bytes, stream);
                    if (rc != RSI_OK) break;
                    RSI_CUDA_TRY(cudaEventRecord(e1, s), "cudaEventRecord");
                    RSI_CUDA_TRY(cudaEventSynchronize(e1), "cudaEventSynchronize");
                    float ms = 0.0f;
                    RSI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                    if (rep > 0) t_best = fminf(t_best, ms);
                }
                if (rc != RSI_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return rc;
                }
                if (t_best < best_ms) {
                    best_ms = t_best;
                    win = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f) return rsi_fail(RSI_E_NOMEM, "rsi_autotune_stage: no shape fits the workspace");
    win.splits = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = win;
    }
    *best = win;
    return RSI_OK;
}
