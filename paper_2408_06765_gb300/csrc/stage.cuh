// stage.cuh -- internal interface between the stage dispatcher (stage.cu) and
// the FP32C / FP64 source x target kernels (steps a3, a5, a6).
//
// Sources are staged as TILES: a 32-byte header followed by `S` fixed-size
// records, one tile per bulk copy into shared memory.
//   FP32C header : centre of the tile's bounding box as double-floats
//                  (xh, xl, yh, yl, zh, zl), tile radius, 0
//   FP32C record : p = P_i - centre (FP32, formed by df_diff exactly as the
//                  target offsets are), |p|^2, then
//                  PISTON  (A, 0, 0, 0)            A = -v0 w / (2 pi)
//                  RSI     (B.re, B.im, C.re, C.im) B = -w sigma / (2 pi), C = i k B
//                  [+ (nx, ny, nz, n.p) for per-point normals]
//   FP64 record  : (x, y, z, B.re, B.im, nx, ny, nz)  (PISTON: B = (A, 0))
// Padding records (past the last source) have zero amplitude and sit 4 m away.
#pragma once

#include "rsi_internal.cuh"

#define RSI_TILE_HDR_BYTES 32
#define RSI_PIPE_STAGES 3

struct TgtView {
    const float *xh, *xl, *yh, *yl, *zh, *zl;
    const double *x, *y, *z;
};

// Cody & Waite (1980) split of 2 pi into three floats; the first two carry 11
// significant bits so that n * P1 and n * P2 are exact for |n| < 2^13.
struct TwoPiSplit {
    float p1, p2, p3, inv;
};
TwoPiSplit two_pi_split();

struct StageArgs {
    int kind;      // RSI_STAGE_*
    int normals;   // RSI_NORMALS_*
    int tpt;       // targets per thread
    int variant;   // FP32C: 1 reciprocal, 2 Newton, 3 Newton on packed source pairs (f32x2)
    int S;         // sources per tile
    int n_tiles;
    int tiles_per_split;
    int splits;
    int64_t n_tgt;
    size_t tile_bytes;
    const uint8_t* tiles;
    TgtView tgt;
    double k;
    float kh, kl;
    TwoPiSplit tp;
    double2* out;  // [splits][n_tgt] partials, or the field when splits == 1
    int* status;
};

size_t fp32_record_bytes(int kind, int normals);
double stage_amp_scale(const rsi_stage& st);  // -v0/(2 pi) (piston) or -+1/(2 pi) (RSI)
// Reversed normals (RSI_NORMALS_NEG_Z, RSI_NORMALS_POINTS_NEG): cos(theta) is
// linear in the normal, so the kernels run with the stored normals and the
// sign goes into the source amplitudes (stage_amp_scale).
inline int base_normals(int n) {
    return n == RSI_NORMALS_NEG_Z ? RSI_NORMALS_Z : n == RSI_NORMALS_POINTS_NEG ? RSI_NORMALS_POINTS : n;
}
inline double normals_sign(int n) { return (n == RSI_NORMALS_NEG_Z || n == RSI_NORMALS_POINTS_NEG) ? -1.0 : 1.0; }
size_t fp64_record_bytes();

// packed: the pair-interleaved record layout of the packed kernel (variant 3)
int launch_prep_fp32(const rsi_stage& st, const PointsView& src, int64_t n_src, const double2* sigma,
                     int S, uint8_t* tiles, size_t tile_bytes, int n_tiles, cudaStream_t s, bool packed = false);
int launch_prep_fp64(const rsi_stage& st, const PointsView& src, int64_t n_src, const double2* sigma,
                     int S, uint8_t* tiles, size_t tile_bytes, int n_tiles, cudaStream_t s);
int launch_stage_fp32(const StageArgs& a, cudaStream_t s);
int launch_stage_fp64(const StageArgs& a, cudaStream_t s);
int fp32_threads();
int fp64_threads();
// resident CTAs per SM of the kernel a launch would use (>= 1)
int stage_occupancy_fp32(const StageArgs& a);
int stage_occupancy_fp64(const StageArgs& a);

// CUDA-event timing of a source x target kernel for rsi_timing_read: a no-op
// unless timing is enabled.  `kind` is RSI_STAGE_* or RSI_TIMING_RAYTRACE.
struct TimingScope {
    cudaEvent_t a = nullptr, b = nullptr;
};
TimingScope timing_begin(cudaStream_t s);
void timing_end(TimingScope& t, int kind, double pairs, cudaStream_t s);
// out[j] = sum over splits of part[split][j] (Neumaier, split order)
int launch_reduce_partials(const double2* part, int splits, int64_t n, double2* out, int* status, cudaStream_t s);
