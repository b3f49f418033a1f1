// qmc.cu -- steps a1-a2: integer Sobol points (dimensions 1-2) with a nested
// bit scramble, mapped onto the piston disk (Eq. circle_sampling), a flat
// patch (Eq. square_sampling) or a cylinder, written in cell order; and the
// cell-centred field-image grid as a target point set.
#include <math.h>

#include "rsi_internal.cuh"

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// SplitMix64 output function (Stafford's "Mix13" finaliser)
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t dim_key(uint64_t seed, uint32_t set_id, uint32_t dim) {
    uint64_t base = splitmix_out(seed + kGolden);
    return splitmix_out(base ^ ((uint64_t(set_id) << 1) | uint64_t(dim & 1u)));
}

struct SobolDirs {
    uint32_t v1[32];  // dimension 2 (polynomial x + 1); dimension 1 is bit reversal
};

SobolDirs make_dirs() {
    SobolDirs d;
    uint32_t m = 1u;  // m_1 = 1, m_j = (2 m_{j-1}) xor m_{j-1}
    for (int j = 1; j <= 32; ++j) {
        if (j > 1) m = (m << 1) ^ m;
        d.v1[j - 1] = m << (32 - j);
    }
    return d;
}

// digit b from the top is flipped by the top bit of the SplitMix64 output
// number (2^b + leading b digits) of the stream started at `key`
__device__ __forceinline__ uint32_t nested_scramble(uint32_t x, uint64_t key) {
    uint32_t flips = 0;
#pragma unroll 4
    for (int b = 0; b < 32; ++b) {
        uint64_t lead = b ? uint64_t(x >> (32 - b)) : 0ull;
        uint64_t node = (1ull << b) | lead;
        uint64_t h = splitmix_out(key + node * kGolden);
        flips |= uint32_t(h >> 63) << (31 - b);
    }
    return x ^ flips;
}

struct SurfaceDev {
    int kind;
    double cx, cy, cz, tilt_c, tilt_s, a, wx, wy, R;
};

__device__ __forceinline__ void split_hl(double v, float& h, float& l) {
    h = __double2float_rn(v);
    l = __double2float_rn(v - double(h));
}

// position of index i within its aligned power-of-two block of the n-point
// set (the blocks are the binary digits of n, largest first), and the block
__device__ __forceinline__ uint64_t cell_slot(uint64_t i, uint64_t n, uint32_t su, uint32_t sv) {
    int m = 63 - __clzll(static_cast<long long>(i ^ n));  // highest differing bit
    uint64_t start = n & ~((2ull << m) - 1ull);
    int a = (m + 1) >> 1, b = m >> 1;
    uint32_t cx = a ? (su >> (32 - a)) : 0u;
    uint32_t cy = b ? (sv >> (32 - b)) : 0u;
    uint64_t pos = 0;
    for (int q = 0; q < a; ++q) pos |= uint64_t((cx >> q) & 1u) << (2 * q);
    for (int q = 0; q < b; ++q) pos |= uint64_t((cy >> q) & 1u) << (2 * q + 1);
    return start + pos;
}

__global__ void qmc_points_kernel(SurfaceDev s, SobolDirs dirs, uint64_t k0, uint64_t k1, int scramble,
                                  int64_t n, PointsView out) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t ix = uint32_t(i);
    uint32_t x = __brev(ix);  // v_j = 2^(32-j): bit j-1 of i -> bit 32-j of x
    uint32_t y = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
        if ((ix >> j) & 1u) y ^= dirs.v1[j];
    if (scramble) {
        x = nested_scramble(x, k0);
        y = nested_scramble(y, k1);
    }
    const double u = (double(x) + 0.5) * (1.0 / 4294967296.0);
    const double v = (double(y) + 0.5) * (1.0 / 4294967296.0);
    double px, py, pz, nx, ny, nz, w;
    if (s.kind == RSI_SURF_DISK) {
        double r = s.a * sqrt(u);
        double sn, cs;
        sincospi(2.0 * v, &sn, &cs);
        double l1 = r * cs, l2 = r * sn;
        px = s.cx + l1 * s.tilt_c;
        py = s.cy + l2;
        pz = s.cz - l1 * s.tilt_s;
        nx = s.tilt_s;
        ny = 0.0;
        nz = s.tilt_c;
        w = M_PI * s.a * s.a / double(n);
    } else {
        double xi = s.wx * (u - 0.5);
        px = s.cx + xi;
        py = s.cy + s.wy * (v - 0.5);
        if (s.kind == RSI_SURF_CYL) {
            double q = sqrt(s.R * s.R - xi * xi);
            pz = s.cz + s.R - q;
            nx = -xi / s.R;
            ny = 0.0;
            nz = q / s.R;
            w = s.wx * s.wy / double(n) * (s.R / q);
        } else {
            pz = s.cz;
            nx = 0.0;
            ny = 0.0;
            nz = 1.0;
            w = s.wx * s.wy / double(n);
        }
    }
    uint64_t slot = cell_slot(uint64_t(i), uint64_t(n), x, y);
    out.idx[slot] = ix;
    out.su[slot] = x;
    out.sv[slot] = y;
    out.x[slot] = px;
    out.y[slot] = py;
    out.z[slot] = pz;
    out.nx[slot] = nx;
    out.ny[slot] = ny;
    out.nz[slot] = nz;
    out.w[slot] = w;
    split_hl(px, out.xh[slot], out.xl[slot]);
    split_hl(py, out.yh[slot], out.yl[slot]);
    split_hl(pz, out.zh[slot], out.zl[slot]);
}

__global__ void grid_points_kernel(rsi_grid g, PointsView out) {
    int64_t n = int64_t(g.nx) * g.nz;
    int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int64_t j = q / g.nx, i = q - j * g.nx;
    double px = g.x0 + (double(i) + 0.5) * ((g.x1 - g.x0) / double(g.nx));
    double pz = g.z0 + (double(j) + 0.5) * ((g.z1 - g.z0) / double(g.nz));
    out.idx[q] = uint32_t(q);
    out.su[q] = 0u;
    out.sv[q] = 0u;
    out.x[q] = px;
    out.y[q] = g.y;
    out.z[q] = pz;
    out.nx[q] = 0.0;
    out.ny[q] = 0.0;
    out.nz[q] = 1.0;
    out.w[q] = 0.0;
    split_hl(px, out.xh[q], out.xl[q]);
    split_hl(g.y, out.yh[q], out.yl[q]);
    split_hl(pz, out.zh[q], out.zl[q]);
}

}  // namespace

extern "C" int rsi_make_qmc_points(const rsi_surface* surf, uint64_t seed, uint32_t set_id, int64_t n,
                                   void* points, size_t points_bytes, void* stream) {
    if (!surf || !points) return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: null argument");
    if (n < 1 || n > (int64_t(1) << 31))
        return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: n = %lld outside [1, 2^31]", (long long)n);
    if (points_bytes < rsi_points_bytes(n))
        return rsi_fail(RSI_E_NOMEM, "rsi_make_qmc_points: buffer of %zu bytes < %zu", points_bytes,
                        rsi_points_bytes(n));
    if (reinterpret_cast<uintptr_t>(points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_make_qmc_points: buffer not 256-byte aligned");
    SurfaceDev s;
    s.kind = surf->kind;
    s.cx = surf->centre[0];
    s.cy = surf->centre[1];
    s.cz = surf->centre[2];
    s.tilt_c = cos(surf->tilt);
    s.tilt_s = sin(surf->tilt);
    s.a = surf->a;
    s.wx = surf->wx;
    s.wy = surf->wy;
    s.R = surf->R;
    switch (surf->kind) {
        case RSI_SURF_DISK:
            if (!(surf->a > 0)) return rsi_fail(RSI_E_INVAL, "disk radius must be > 0");
            break;
        case RSI_SURF_RECT:
            if (!(surf->wx > 0 && surf->wy > 0)) return rsi_fail(RSI_E_INVAL, "patch sides must be > 0");
            break;
        case RSI_SURF_CYL:
            if (!(surf->wx > 0 && surf->wy > 0 && surf->R > 0.5 * surf->wx))
                return rsi_fail(RSI_E_INVAL, "cylinder needs wx, wy > 0 and R > wx/2");
            break;
        default:
            return rsi_fail(RSI_E_INVAL, "unknown surface kind %d", surf->kind);
    }
    static const SobolDirs dirs = make_dirs();
    uint64_t k0 = dim_key(seed, set_id, 0), k1 = dim_key(seed, set_id, 1);
    PointsView v = rsi_points_view(points, n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    qmc_points_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(s, dirs, k0, k1,
                                                                               surf->scramble ? 1 : 0, n, v);
    RSI_CHECK_LAUNCH("qmc_points_kernel");
    return RSI_OK;
}

extern "C" int rsi_grid_points(const rsi_grid* g, void* points, size_t points_bytes, void* stream) {
    if (!g || !points) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: null argument");
    if (g->nx < 1 || g->nz < 1) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: empty grid");
    int64_t n = int64_t(g->nx) * g->nz;
    if (n > (int64_t(1) << 31)) return rsi_fail(RSI_E_INVAL, "rsi_grid_points: grid too large");
    if (points_bytes < rsi_points_bytes(n)) return rsi_fail(RSI_E_NOMEM, "rsi_grid_points: buffer too small");
    if (reinterpret_cast<uintptr_t>(points) % 256)
        return rsi_fail(RSI_E_INVAL, "rsi_grid_points: buffer not 256-byte aligned");
    PointsView v = rsi_points_view(points, n);
    int threads = 256;
    unsigned blocks = unsigned((n + threads - 1) / threads);
    grid_points_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(*g, v);
    RSI_CHECK_LAUNCH("grid_points_kernel");
    return RSI_OK;
}
