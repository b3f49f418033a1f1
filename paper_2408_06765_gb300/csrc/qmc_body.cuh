// qmc_body.cuh -- steps a1-a2 per point: integer Sobol digits (dimensions
// 1-2), the nested bit scramble, the surface maps and the cell-order slot;
// shared by the single-set kernel (qmc.cu) and the batched kernels (batch.cu).
#pragma once

#include <math.h>

#include "rsi_internal.cuh"

namespace rsi_qmc {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// SplitMix64 output function (Stafford's "Mix13" finaliser)
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline uint64_t dim_key(uint64_t seed, uint32_t set_id, uint32_t dim) {
    uint64_t base = splitmix_out(seed + kGolden);
    return splitmix_out(base ^ ((uint64_t(set_id) << 1) | uint64_t(dim & 1u)));
}

struct SobolDirs {
    uint32_t v1[32];  // dimension 2 (polynomial x + 1); dimension 1 is bit reversal
};

inline SobolDirs make_dirs() {
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
    int kind, seq;
    double cx, cy, cz, tilt_c, tilt_s, a, wx, wy, R, apod;
};

inline SurfaceDev surface_dev(const rsi_surface& s) {
    SurfaceDev d;
    d.kind = s.kind;
    d.cx = s.centre[0];
    d.cy = s.centre[1];
    d.cz = s.centre[2];
    d.tilt_c = cos(s.tilt);
    d.tilt_s = sin(s.tilt);
    d.a = s.a;
    d.wx = s.wx;
    d.wy = s.wy;
    d.R = s.R;
    d.seq = s.sequence;
    d.apod = s.apod;
    return d;
}

// host-side check of a surface description; RSI_OK or an RSI_E_INVAL message
inline int check_surface(const rsi_surface& s) {
    if (s.sequence != RSI_SEQ_SOBOL && s.sequence != RSI_SEQ_HALTON)
        return rsi_fail(RSI_E_INVAL, "unknown point sequence %d", s.sequence);
    if (s.sequence == RSI_SEQ_HALTON && s.scramble) return rsi_fail(RSI_E_INVAL, "Halton points are not scrambled");
    if (!(s.apod >= 0.0) || !isfinite(s.apod)) return rsi_fail(RSI_E_INVAL, "apodisation radius must be >= 0");
    switch (s.kind) {
        case RSI_SURF_DISK:
            if (!(s.a > 0)) return rsi_fail(RSI_E_INVAL, "disk radius must be > 0");
            return RSI_OK;
        case RSI_SURF_RECT:
            if (!(s.wx > 0 && s.wy > 0)) return rsi_fail(RSI_E_INVAL, "patch sides must be > 0");
            return RSI_OK;
        case RSI_SURF_CYL:
            if (!(s.wx > 0 && s.wy > 0 && s.R > 0.5 * s.wx))
                return rsi_fail(RSI_E_INVAL, "cylinder needs wx, wy > 0 and R > wx/2");
            return RSI_OK;
        case RSI_SURF_CAP:
            if (!(s.a > 0 && s.R > s.a)) return rsi_fail(RSI_E_INVAL, "spherical cap needs a > 0 and R > a");
            return RSI_OK;
        default:
            return rsi_fail(RSI_E_INVAL, "unknown surface kind %d", s.kind);
    }
}

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

// base-3 radical inverse of i < 3^20 as a fraction of 3^20 (digits reversed)
__device__ __forceinline__ uint32_t radical_inverse3(uint32_t i) {
    uint32_t r = 0;
#pragma unroll
    for (int d = 0; d < 20; ++d) {
        const uint32_t q = i / 3u;
        r = 3u * r + (i - 3u * q);
        i = q;
    }
    return r;
}

// point i (0 <= i < n) of a set, written to its slot (cell order for Sobol,
// index order for Halton)
__device__ __forceinline__ void make_point(const SurfaceDev& s, const SobolDirs& dirs, uint64_t k0, uint64_t k1,
                                           int scramble, int64_t i, int64_t n, const PointsView& out) {
    uint32_t ix = uint32_t(i);
    uint32_t x, y;
    double u, v;
    if (s.seq == RSI_SEQ_HALTON) {  // Halton point i + 1
        ix = uint32_t(i + 1);
        x = __brev(ix);
        y = radical_inverse3(ix);
        u = double(x) * (1.0 / 4294967296.0);
        v = double(y) / 3486784401.0;
    } else {
        x = __brev(ix);  // v_j = 2^(32-j): bit j-1 of i -> bit 32-j of x
        y = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if ((ix >> j) & 1u) y ^= dirs.v1[j];
        if (scramble) {
            x = nested_scramble(x, k0);
            y = nested_scramble(y, k1);
        }
        u = (double(x) + 0.5) * (1.0 / 4294967296.0);
        v = (double(y) + 0.5) * (1.0 / 4294967296.0);
    }
    double px, py, pz, nx, ny, nz, w;
    if (s.kind == RSI_SURF_DISK || s.kind == RSI_SURF_CAP) {
        double r = s.a * sqrt(u);
        double sn, cs;
        sincospi(2.0 * v, &sn, &cs);
        double l1 = r * cs, l2 = r * sn;
        w = M_PI * s.a * s.a / double(n);
        if (s.kind == RSI_SURF_DISK) {
            px = s.cx + l1 * s.tilt_c;
            py = s.cy + l2;
            pz = s.cz - l1 * s.tilt_s;
            nx = s.tilt_s;
            ny = 0.0;
            nz = s.tilt_c;
        } else {  // lifted onto the sphere; normal to the centre of curvature
            const double q = sqrt(s.R * s.R - r * r), h = s.R - q;
            px = s.cx + l1 * s.tilt_c + h * s.tilt_s;
            py = s.cy + l2;
            pz = s.cz - l1 * s.tilt_s + h * s.tilt_c;
            const double m1 = -l1 / s.R, m2 = -l2 / s.R, m3 = q / s.R;
            nx = m1 * s.tilt_c + m3 * s.tilt_s;
            ny = m2;
            nz = -m1 * s.tilt_s + m3 * s.tilt_c;
            w *= s.R / q;
        }
        if (s.apod > 0.0) w *= exp(-(r / s.apod) * (r / s.apod));
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
    const uint64_t slot = s.seq == RSI_SEQ_HALTON ? uint64_t(i) : cell_slot(uint64_t(i), uint64_t(n), x, y);
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

// pixel q of a cell-centred grid, row-major [nz][nx]
__device__ __forceinline__ void make_grid_point(const rsi_grid& g, int64_t q, const PointsView& out) {
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

}  // namespace rsi_qmc
