/*
 * rsi_oracle.c -- plain, slow FP64 CPU oracle for the quasi-Monte Carlo
 * Rayleigh-Sommerfeld-integral (RSI) beam model of Lello de Almeida, Png and
 * Lan, "Efficient numerical frameworks for modelling ultrasonic beams
 * propagating across interfaces" (arXiv 2408.06765).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path: its Sobol generator, scrambler, geometry and sums are written
 * here from the paper and from the published constructions named below.
 *
 * Every sum is a direct loop over sources in index order, in double
 * precision, with Neumaier compensation (Neumaier 1974).  Targets are
 * independent, so they are split across POSIX threads; this changes no
 * arithmetic.
 *
 * What each function follows:
 *   orc_sobol          QMC points (Sec. 2.3, Eq. monte_carlo).  The paper
 *                      draws Halton points; this build draws the first two
 *                      Sobol dimensions (Bratley & Fox 1988; Joe & Kuo 2008
 *                      construction), optionally with a nested (Owen 1995)
 *                      bit scramble keyed by a SplitMix64 stream (Steele, Lea
 *                      & Flood 2014; output mixer = Stafford 2011 "Mix13").
 *   orc_halton         the paper's own QMC points, the Halton sequence in
 *                      bases 2 and 3 (Sec. 2.3), as exact integer radical
 *                      inverses (index 0, the origin of every base, skipped).
 *   orc_map_disk       piston face sampling, Eq. circle_sampling (Sec. 2.3),
 *                      optionally with a Gaussian amplitude profile (the
 *                      apodised face Sec. 4 mentions).
 *   orc_map_cap        focused transducer: a spherical cap (Sec. 3.3, Fig.
 *                      transducer_system b), projected-disk sampling lifted
 *                      onto the sphere with the surface Jacobian.
 *   orc_map_rect       square interface sampling, Eq. square_sampling, with
 *                      the side length given explicitly.
 *   orc_map_cyl        cylindrical interface (projected-area sampling with the
 *                      surface Jacobian); the paper has no curved interface,
 *                      this is the multilayer workload's curved variant.
 *   orc_piston_field   incident field of a piston, Eq. incident_field (Sec. 2.1).
 *   orc_transmit       T12 of Eq. transmission_coefficient with Snell's
 *                      invariant of Eq. root_searching; the source density of
 *                      Eq. approximated_transmitted_field is T12 * phi_i since
 *                      (rho1/rho2)(1+R12) = T12 (Eq. reflection_coefficient).
 *   orc_reflect        source density of the reflected field in medium 1,
 *                      R12 * phi_i: the plane-wave approximation of the
 *                      reflected field on the interface (Sec. 2.1, with
 *                      Eq. reflection_coefficient), same incidence angles as
 *                      orc_transmit.
 *   orc_ray_path       the refracted ray between two points across a plane
 *                      interface: Snell's invariant C of Eq. ray_tracing
 *                      (Sec. 2.2, Eq. root_searching) by bisection, and the
 *                      path lengths and angles it fixes.
 *   orc_raytrace_field transmitted field of the ray-tracing model, Eq.
 *                      transmitted_ray_tracing (Sec. 2.2), over weighted
 *                      transducer points.
 *   orc_rsi_field      first Rayleigh-Sommerfeld solution, Eq. rayleigh_sommerfeld
 *                      (Sec. 2.1), over weighted source points; the sign of
 *                      its bracket is read as explained at rsi_range().
 *   orc_grid_points    cell-centred field-image grid (Sec. 3 uses a 2-D slice).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Counter-based hash: the SplitMix64 generator.  Its n-th output for initial
 * state s is mix64(s + n * GOLDEN).                                          */
/* ------------------------------------------------------------------------ */
#define ORC_GOLDEN 0x9E3779B97F4A7C15ULL

uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* key of one (seed, point set, dimension) triple */
uint64_t orc_scramble_key(uint64_t seed, uint32_t set_id, uint32_t dim)
{
    uint64_t base = orc_mix64(seed + ORC_GOLDEN);
    return orc_mix64(base ^ (((uint64_t)set_id << 1) | (uint64_t)(dim & 1u)));
}

/* Nested bit scramble: output bit b (counted from the most significant bit)
 * is input bit b XOR the top bit of the hash of the tree node formed by the
 * b leading input bits.  Node id = 2^b + (leading b bits). */
uint32_t orc_owen(uint32_t x, uint64_t key)
{
    uint32_t y = x;
    for (int b = 0; b < 32; ++b) {
        uint64_t prefix = (b == 0) ? 0u : (uint64_t)(x >> (32 - b));
        uint64_t node = ((uint64_t)1 << b) | prefix;
        uint64_t h = orc_mix64(key + node * ORC_GOLDEN);
        y ^= (uint32_t)(h >> 63) << (31 - b);
    }
    return y;
}

/* Direction numbers v_j = m_j 2^(32-j), j = 1..32.
 * dim 0: m_j = 1 (van der Corput in base 2).
 * dim 1: primitive polynomial x + 1 (degree 1), m_1 = 1, and the Sobol
 *        recurrence for degree 1: m_j = 2 m_{j-1} XOR m_{j-1}.            */
static void sobol_directions(uint32_t v[2][32])
{
    uint32_t m = 1u;
    for (int j = 1; j <= 32; ++j) {
        v[0][j - 1] = 1u << (32 - j);
        if (j > 1)
            m = (m << 1) ^ m;
        v[1][j - 1] = m << (32 - j);
    }
}

/* Points first .. first+n-1 of the 2-D Sobol sequence in natural index
 * order: x = XOR of v_j over the set bits j of the index (bit j-1 of i). */
void orc_sobol(uint64_t seed, uint32_t set_id, int64_t first, int64_t n,
               int scrambled, uint32_t *su, uint32_t *sv)
{
    uint32_t v[2][32];
    sobol_directions(v);
    uint64_t k0 = orc_scramble_key(seed, set_id, 0);
    uint64_t k1 = orc_scramble_key(seed, set_id, 1);
    for (int64_t q = 0; q < n; ++q) {
        uint64_t i = (uint64_t)(first + q);
        uint32_t x = 0, y = 0;
        for (int j = 1; j <= 32; ++j) {
            if ((i >> (j - 1)) & 1u) {
                x ^= v[0][j - 1];
                y ^= v[1][j - 1];
            }
        }
        if (scrambled) {
            x = orc_owen(x, k0);
            y = orc_owen(y, k1);
        }
        su[q] = x;
        sv[q] = y;
    }
}

/* Halton points first+1 .. first+n (Halton 1960): su = the base-2 radical
 * inverse of the index as a 32-bit fraction (its bits reversed), sv = the
 * base-3 radical inverse as a fraction of 3^20 (its 20 base-3 digits
 * reversed).  Indices stay below 2^31 < 3^20, so both are exact.          */
void orc_halton(int64_t first, int64_t n, uint32_t *su, uint32_t *sv)
{
    for (int64_t q = 0; q < n; ++q) {
        uint64_t i = (uint64_t)(first + q + 1);
        uint32_t r2 = 0;
        for (int b = 0; b < 32; ++b)
            if ((i >> b) & 1u)
                r2 |= 1u << (31 - b);
        uint64_t r3 = 0, k = i;
        for (int d = 0; d < 20; ++d) {
            r3 = 3 * r3 + k % 3;
            k /= 3;
        }
        su[q] = r2;
        sv[q] = (uint32_t)r3;
    }
}

/* unit value of a QMC coordinate.  seq 0 (Sobol): (x + 1/2) 2^-32.  seq 1
 * (Halton): dimension 0 is x 2^-32, dimension 1 is x / 3^20 -- the radical
 * inverses themselves.                                                     */
static double unit_of(int seq, int dim, uint32_t x)
{
    if (seq == 0)
        return ((double)x + 0.5) * (1.0 / 4294967296.0);
    if (dim == 0)
        return (double)x * (1.0 / 4294967296.0);
    return (double)x / 3486784401.0;
}

/* Piston face, Eq. circle_sampling: r = a sqrt(H), theta = 2 pi H (first
 * dimension radial, second angular).  The face is centred at c and tilted by
 * `tilt` radians about +y: in-plane axes e1 = (cos t, 0, -sin t), e2 = +y,
 * normal (sin t, 0, cos t).  Weight = face area / n (Eq. monte_carlo).    */
void orc_map_disk(int64_t n, int seq, const uint32_t *su, const uint32_t *sv,
                  double cx, double cy, double cz, double tilt, double a, double apod,
                  double *x, double *y, double *z,
                  double *nx, double *ny, double *nz, double *w)
{
    double ct = cos(tilt), st = sin(tilt);
    for (int64_t i = 0; i < n; ++i) {
        double r = a * sqrt(unit_of(seq, 0, su[i]));
        double th = 2.0 * M_PI * unit_of(seq, 1, sv[i]);
        double l1 = r * cos(th), l2 = r * sin(th);
        x[i] = cx + l1 * ct;
        y[i] = cy + l2;
        z[i] = cz - l1 * st;
        nx[i] = st;
        ny[i] = 0.0;
        nz[i] = ct;
        w[i] = M_PI * a * a / (double)n;
        if (apod > 0.0) /* Gaussian velocity profile v0 exp(-(r / apod)^2) */
            w[i] *= exp(-(r / apod) * (r / apod));
    }
}

/* Flat interface patch, Eq. square_sampling with sides wx, wy centred on c;
 * the interface normal is +z, toward the observation side (Sec. 2.1).    */
void orc_map_rect(int64_t n, int seq, const uint32_t *su, const uint32_t *sv,
                  double cx, double cy, double cz, double wx, double wy,
                  double *x, double *y, double *z,
                  double *nx, double *ny, double *nz, double *w)
{
    for (int64_t i = 0; i < n; ++i) {
        x[i] = cx + wx * (unit_of(seq, 0, su[i]) - 0.5);
        y[i] = cy + wy * (unit_of(seq, 1, sv[i]) - 0.5);
        z[i] = cz;
        nx[i] = 0.0;
        ny[i] = 0.0;
        nz[i] = 1.0;
        w[i] = wx * wy / (double)n;
    }
}

/* Cylindrical interface with axis parallel to y through (cx, ., cz + R):
 * z = cz + R - sqrt(R^2 - xi^2), xi = x - cx.  Points are uniform in the
 * projected (x, y) rectangle; the weight carries the surface Jacobian
 * R / sqrt(R^2 - xi^2).  The normal points toward the axis (+z side).     */
void orc_map_cyl(int64_t n, int seq, const uint32_t *su, const uint32_t *sv,
                 double cx, double cy, double cz, double wx, double wy, double R,
                 double *x, double *y, double *z,
                 double *nx, double *ny, double *nz, double *w)
{
    for (int64_t i = 0; i < n; ++i) {
        double xi = wx * (unit_of(seq, 0, su[i]) - 0.5);
        double s = sqrt(R * R - xi * xi);
        x[i] = cx + xi;
        y[i] = cy + wy * (unit_of(seq, 1, sv[i]) - 0.5);
        z[i] = cz + R - s;
        nx[i] = -xi / R;
        ny[i] = 0.0;
        nz[i] = s / R;
        w[i] = wx * wy / (double)n * (R / s);
    }
}

/* Focused transducer: the spherical cap of radius of curvature R over an
 * aperture of radius a, apex at c, centre of curvature R along the axis.
 * Points are uniform in the projected aperture (r = a sqrt(u), theta = 2 pi v,
 * as Eq. circle_sampling), lifted to the sphere at height
 * R - sqrt(R^2 - r^2); the weight carries the Jacobian R / sqrt(R^2 - r^2)
 * and the normal points to the centre of curvature.  The cap is tilted like
 * the disk: local (l1, l2, h) -> (l1 cos t + h sin t, l2, -l1 sin t + h cos t).
 * apod > 0 multiplies the weight by exp(-(r / apod)^2).                     */
void orc_map_cap(int64_t n, int seq, const uint32_t *su, const uint32_t *sv,
                 double cx, double cy, double cz, double tilt, double a, double R, double apod,
                 double *x, double *y, double *z,
                 double *nx, double *ny, double *nz, double *w)
{
    double ct = cos(tilt), st = sin(tilt);
    for (int64_t i = 0; i < n; ++i) {
        double r = a * sqrt(unit_of(seq, 0, su[i]));
        double th = 2.0 * M_PI * unit_of(seq, 1, sv[i]);
        double l1 = r * cos(th), l2 = r * sin(th);
        double q = sqrt(R * R - r * r);
        double h = R - q;
        x[i] = cx + l1 * ct + h * st;
        y[i] = cy + l2;
        z[i] = cz - l1 * st + h * ct;
        double m1 = -l1 / R, m2 = -l2 / R, m3 = q / R; /* toward the centre of curvature */
        nx[i] = m1 * ct + m3 * st;
        ny[i] = m2;
        nz[i] = -m1 * st + m3 * ct;
        w[i] = M_PI * a * a / (double)n * (R / q);
        if (apod > 0.0)
            w[i] *= exp(-(r / apod) * (r / apod));
    }
}

/* Cell-centred grid in the plane y = y0: x_i = x0 + (i + 1/2)(x1 - x0)/nx,
 * z_j = z0 + (j + 1/2)(z1 - z0)/nz, stored row-major [nz][nx].           */
void orc_grid_points(double x0, double x1, int64_t nxp, double z0, double z1,
                     int64_t nzp, double y0, double *x, double *y, double *z)
{
    double dx = (x1 - x0) / (double)nxp, dz = (z1 - z0) / (double)nzp;
    for (int64_t j = 0; j < nzp; ++j)
        for (int64_t i = 0; i < nxp; ++i) {
            int64_t q = j * nxp + i;
            x[q] = x0 + ((double)i + 0.5) * dx;
            y[q] = y0;
            z[q] = z0 + ((double)j + 0.5) * dz;
        }
}

/* ------------------------------------------------------------------------ */
/* Neumaier-compensated complex accumulator                                  */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

/* ------------------------------------------------------------------------ */
/* Thread fan-out over targets                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind; /* 0 piston, 1 rsi */
    int64_t ns;
    const double *sx, *sy, *sz, *snx, *sny, *snz, *sw, *sre, *sim;
    double v0, k;
    const double *tx, *ty, *tz;
    double *ore, *oim;
    int64_t t0, t1;
} field_job;

/* Eq. incident_field:  phi_i(P1) = -(v0 / 2 pi) sum_i w_i e^{i k r} / r      */
static void piston_range(const field_job *J)
{
    for (int64_t j = J->t0; j < J->t1; ++j) {
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t i = 0; i < J->ns; ++i) {
            double dx = J->tx[j] - J->sx[i];
            double dy = J->ty[j] - J->sy[i];
            double dz = J->tz[j] - J->sz[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < 1e-12)
                continue; /* coincident source and target: no contribution */
            double complex term = -(J->v0 / (2.0 * M_PI)) * J->sw[i] * cexp(I * J->k * r) / r;
            nsum_add(&re, creal(term));
            nsum_add(&im, cimag(term));
        }
        J->ore[j] = re.s + re.c;
        J->oim[j] = im.s + im.c;
    }
}

/* Eq. rayleigh_sommerfeld with the source density sigma = phi (or T12 phi_i
 * across an interface, Eq. approximated_transmitted_field):
 *   phi(Po) = -(i/lambda) sum_i w_i sigma_i e^{ikr}/r (1 - 1/(ikr)) cos(theta),
 * r from the source point P_i to Po, cos(theta) = n_i . (Po - P_i) / r with
 * n_i toward the observation side, lambda = 2 pi / k of the medium the field
 * propagates in.  The printed equation has the bracket as (1/(ikr) - 1); with
 * the paper's stated normal and r conventions that sign returns -phi for an
 * outgoing field, while the equation is named (and used in Sec. 3.1-3.2) as
 * the first Rayleigh-Sommerfeld solution, which must return +phi.  The
 * bracket is therefore read as (1 - 1/(ikr)), the standard solution.         */
static void rsi_range(const field_job *J)
{
    double lambda = 2.0 * M_PI / J->k;
    for (int64_t j = J->t0; j < J->t1; ++j) {
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t i = 0; i < J->ns; ++i) {
            double dx = J->tx[j] - J->sx[i];
            double dy = J->ty[j] - J->sy[i];
            double dz = J->tz[j] - J->sz[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < 1e-12)
                continue; /* coincident source and target: no contribution */
            double cos_theta = (J->snx[i] * dx + J->sny[i] * dy + J->snz[i] * dz) / r;
            double complex sigma = J->sre[i] + I * J->sim[i];
            double complex term = (-I / lambda) * J->sw[i] * sigma * cexp(I * J->k * r) / r
                                  * (1.0 - 1.0 / (I * J->k * r)) * cos_theta;
            nsum_add(&re, creal(term));
            nsum_add(&im, cimag(term));
        }
        J->ore[j] = re.s + re.c;
        J->oim[j] = im.s + im.c;
    }
}

static void *field_worker(void *arg)
{
    field_job *J = (field_job *)arg;
    if (J->kind == 0)
        piston_range(J);
    else
        rsi_range(J);
    return NULL;
}

static void run_field(field_job proto, int64_t nt, int nthreads)
{
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    if ((int64_t)nthreads > nt)
        nthreads = (int)(nt > 0 ? nt : 1);
    pthread_t th[256];
    int started[256];
    field_job jobs[256];
    int64_t chunk = (nt + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].t0 = (int64_t)t * chunk;
        jobs[t].t1 = jobs[t].t0 + chunk < nt ? jobs[t].t0 + chunk : nt;
        started[t] = 0;
        if (jobs[t].t0 >= jobs[t].t1)
            continue;
        if (nthreads > 1 && pthread_create(&th[t], NULL, field_worker, &jobs[t]) == 0)
            started[t] = 1;
        else
            field_worker(&jobs[t]); /* single thread, or no thread available */
    }
    for (int t = 0; t < nthreads; ++t)
        if (started[t])
            pthread_join(th[t], NULL);
}

void orc_piston_field(int64_t ns, const double *sx, const double *sy, const double *sz,
                      const double *sw, double v0, double k,
                      int64_t nt, const double *tx, const double *ty, const double *tz,
                      double *out_re, double *out_im, int nthreads)
{
    field_job J;
    memset(&J, 0, sizeof J);
    J.kind = 0;
    J.ns = ns;
    J.sx = sx; J.sy = sy; J.sz = sz; J.sw = sw;
    J.v0 = v0; J.k = k;
    J.tx = tx; J.ty = ty; J.tz = tz;
    J.ore = out_re; J.oim = out_im;
    run_field(J, nt, nthreads);
}

void orc_rsi_field(int64_t ns, const double *sx, const double *sy, const double *sz,
                   const double *snx, const double *sny, const double *snz,
                   const double *sw, const double *sig_re, const double *sig_im, double k,
                   int64_t nt, const double *tx, const double *ty, const double *tz,
                   double *out_re, double *out_im, int nthreads)
{
    field_job J;
    memset(&J, 0, sizeof J);
    J.kind = 1;
    J.ns = ns;
    J.sx = sx; J.sy = sy; J.sz = sz;
    J.snx = snx; J.sny = sny; J.snz = snz;
    J.sw = sw; J.sre = sig_re; J.sim = sig_im;
    J.k = k;
    J.tx = tx; J.ty = ty; J.tz = tz;
    J.ore = out_re; J.oim = out_im;
    run_field(J, nt, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Interface transmission                                                    */
/* ------------------------------------------------------------------------ */

/* cos of an angle whose sine is s (real): sqrt(1 - s^2) when |s| <= 1, else
 * the branch i sqrt(s^2 - 1) (Im >= 0: evanescent decay for e^{-i w t}).   */
static double complex cos_from_sin(double s)
{
    double q = 1.0 - s * s;
    if (q >= 0.0)
        return sqrt(q);
    return I * sqrt(-q);
}

/* Eq. transmission_coefficient:
 *   T12 = 2 rho1 c2 cos a1 / (rho2 c2 cos a1 + rho1 c1 cos a2).           */
double complex orc_T12(double rho1, double c1, double rho2, double c2,
                       double complex cos1, double complex cos2)
{
    return 2.0 * rho1 * c2 * cos1 / (rho2 * c2 * cos1 + rho1 * c1 * cos2);
}

/* Eq. reflection_coefficient, for the identity test (rho1/rho2)(1+R12) = T12. */
double complex orc_R12(double rho1, double c1, double rho2, double c2,
                       double complex cos1, double complex cos2)
{
    return (rho2 * c2 * cos1 - rho1 * c1 * cos2) / (rho2 * c2 * cos1 + rho1 * c1 * cos2);
}

/* ctypes-friendly wrappers (complex split into re/im) */
void orc_T12_ri(double rho1, double c1, double rho2, double c2,
                double cos1_re, double cos1_im, double cos2_re, double cos2_im,
                double *out)
{
    double complex t = orc_T12(rho1, c1, rho2, c2, cos1_re + I * cos1_im, cos2_re + I * cos2_im);
    out[0] = creal(t);
    out[1] = cimag(t);
}

void orc_R12_ri(double rho1, double c1, double rho2, double c2,
                double cos1_re, double cos1_im, double cos2_re, double cos2_im,
                double *out)
{
    double complex t = orc_R12(rho1, c1, rho2, c2, cos1_re + I * cos1_im, cos2_re + I * cos2_im);
    out[0] = creal(t);
    out[1] = cimag(t);
}

/* Source density on an interface, sigma_i = T12(alpha1_i) phi_i(P_i).
 * mode 0 (global): one incidence angle for the whole interface, fixed by
 *   Snell's invariant C = sin a / c (Eq. root_searching) of the beam axis:
 *   sin a1 = c1 C, sin a2 = c2 C.
 * mode 1 (local): the incidence angle at each point is the angle between
 *   the beam direction in medium 1, d = (c1 C, 0, sqrt(1 - (c1 C)^2)), and
 *   the local normal n_i: cos a1 = d . n_i (clamped at 0 from below),
 *   sin a2 = (c2 / c1) sin a1.
 * Writes T (re, im) when T_re/T_im are non-NULL.                            */
void orc_transmit(int64_t n, int mode, double rho1, double c1, double rho2, double c2,
                  double snell_C, const double *nx, const double *ny, const double *nz,
                  const double *phi_re, const double *phi_im,
                  double *sig_re, double *sig_im, double *T_re, double *T_im)
{
    double s1g = c1 * snell_C;
    double dxv = s1g, dyv = 0.0, dzv = sqrt(fmax(0.0, 1.0 - s1g * s1g));
    for (int64_t i = 0; i < n; ++i) {
        double complex cos1, cos2;
        if (mode == 0) {
            cos1 = cos_from_sin(c1 * snell_C);
            cos2 = cos_from_sin(c2 * snell_C);
        } else {
            double c = dxv * nx[i] + dyv * ny[i] + dzv * nz[i];
            if (c < 0.0)
                c = 0.0;
            if (c > 1.0)
                c = 1.0;
            double s = sqrt(1.0 - c * c);
            cos1 = c;
            cos2 = cos_from_sin(c2 / c1 * s);
        }
        double complex T = orc_T12(rho1, c1, rho2, c2, cos1, cos2);
        double complex phi = phi_re[i] + I * phi_im[i];
        double complex sig = T * phi;
        sig_re[i] = creal(sig);
        sig_im[i] = cimag(sig);
        if (T_re)
            T_re[i] = creal(T);
        if (T_im)
            T_im[i] = cimag(T);
    }
}

/* Source density of the reflected field, sigma_i = R12(alpha1_i) phi_i(P_i)
 * (the reflected field on the interface is taken as R12 times the incident
 * field, Sec. 2.1; R12 from Eq. reflection_coefficient).  The incidence
 * angles follow the same two modes as orc_transmit.  Writes R (re, im) when
 * R_re/R_im are non-NULL.                                                   */
void orc_reflect(int64_t n, int mode, double rho1, double c1, double rho2, double c2,
                 double snell_C, const double *nx, const double *ny, const double *nz,
                 const double *phi_re, const double *phi_im,
                 double *sig_re, double *sig_im, double *R_re, double *R_im)
{
    double s1g = c1 * snell_C;
    double dxv = s1g, dyv = 0.0, dzv = sqrt(fmax(0.0, 1.0 - s1g * s1g));
    for (int64_t i = 0; i < n; ++i) {
        double complex cos1, cos2;
        if (mode == 0) {
            cos1 = cos_from_sin(c1 * snell_C);
            cos2 = cos_from_sin(c2 * snell_C);
        } else {
            double c = dxv * nx[i] + dyv * ny[i] + dzv * nz[i];
            if (c < 0.0)
                c = 0.0;
            if (c > 1.0)
                c = 1.0;
            double s = sqrt(1.0 - c * c);
            cos1 = c;
            cos2 = cos_from_sin(c2 / c1 * s);
        }
        double complex R = orc_R12(rho1, c1, rho2, c2, cos1, cos2);
        double complex phi = phi_re[i] + I * phi_im[i];
        double complex sig = R * phi;
        sig_re[i] = creal(sig);
        sig_im[i] = cimag(sig);
        if (R_re)
            R_re[i] = creal(R);
        if (R_im)
            R_im[i] = cimag(R);
    }
}

/* ------------------------------------------------------------------------ */
/* Ray-tracing model (Sec. 2.2)                                              */
/* ------------------------------------------------------------------------ */
/* The ray from a point at height h1 above a plane interface (in medium 1,
 * speed c1) to a point at depth h2 below it (medium 2, speed c2), at
 * horizontal distance rho, obeys Eq. ray_tracing:
 *   rho = C h1 / sqrt(S1^2 - C^2) + C h2 / sqrt(S2^2 - C^2),  S = 1/c,
 * whose right side increases from 0 to infinity as C goes from 0 to
 * min(S1, S2), so the root is unique; it is found by bisection to the last
 * representable C.  out = {C, D1, D2, cos a1, cos a2}, with sin a = c C
 * (Eq. root_searching), D1 = h1 / cos a1, D2 = h2 / cos a2.               */
void orc_ray_path(double h1, double h2, double rho, double c1, double c2, double *out)
{
    double S1 = 1.0 / c1, S2 = 1.0 / c2;
    double lo = 0.0, hi = fmin(S1, S2);
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        double f = mid * h1 / sqrt(S1 * S1 - mid * mid) + mid * h2 / sqrt(S2 * S2 - mid * mid) - rho;
        if (f < 0.0)
            lo = mid;
        else
            hi = mid;
    }
    double C = 0.5 * (lo + hi);
    double s1 = c1 * C, s2 = c2 * C;
    double cos1 = sqrt(1.0 - s1 * s1), cos2 = sqrt(1.0 - s2 * s2);
    out[0] = C;
    out[1] = h1 / cos1;
    out[2] = h2 / cos2;
    out[3] = cos1;
    out[4] = cos2;
}

typedef struct {
    int64_t ns;
    const double *sx, *sy, *sz, *sw;
    double v0, rho1, c1, rho2, c2, zI, k1, k2;
    const double *tx, *ty, *tz;
    double *ore, *oim;
} ray_job;

typedef struct {
    const ray_job *J;
    int64_t t0, t1;
} ray_range_arg;

/* Eq. transmitted_ray_tracing: for every target,
 *   phi_t = -(v0 / 2 pi) sum_i w_i T12 e^{i (k1 D1 + k2 D2)}
 *           / sqrt((D1 + c2 cos^2 a1 / (c1 cos^2 a2) D2) (D1 + (c2 / c1) D2)),
 * T12 of Eq. transmission_coefficient at the ray's angles.                  */
static void *ray_range(void *argp)
{
    const ray_range_arg *a = (const ray_range_arg *)argp;
    const ray_job *J = a->J;
    const double pre = -J->v0 / (2.0 * M_PI);
    for (int64_t j = a->t0; j < a->t1; ++j) {
        double sre = 0.0, cre = 0.0, sim = 0.0, cim = 0.0;
        double h2 = J->tz[j] - J->zI;
        for (int64_t i = 0; i < J->ns; ++i) {
            double h1 = J->zI - J->sz[i];
            double rho = hypot(J->tx[j] - J->sx[i], J->ty[j] - J->sy[i]);
            double path[5];
            orc_ray_path(h1, h2, rho, J->c1, J->c2, path);
            double D1 = path[1], D2 = path[2], cos1 = path[3], cos2 = path[4];
            double complex T = orc_T12(J->rho1, J->c1, J->rho2, J->c2, cos1, cos2);
            double spread = sqrt((D1 + J->c2 * cos1 * cos1 / (J->c1 * cos2 * cos2) * D2) *
                                 (D1 + J->c2 / J->c1 * D2));
            double complex term = pre * J->sw[i] * T * cexp(I * (J->k1 * D1 + J->k2 * D2)) / spread;
            double v = creal(term), t = sre + v;
            cre += (fabs(sre) >= fabs(v)) ? (sre - t) + v : (v - t) + sre;
            sre = t;
            v = cimag(term);
            t = sim + v;
            cim += (fabs(sim) >= fabs(v)) ? (sim - t) + v : (v - t) + sim;
            sim = t;
        }
        J->ore[j] = sre + cre;
        J->oim[j] = sim + cim;
    }
    return NULL;
}

void orc_raytrace_field(int64_t ns, const double *sx, const double *sy, const double *sz, const double *sw,
                        double v0, double rho1, double c1, double rho2, double c2, double zI, double k1,
                        double k2, int64_t nt, const double *tx, const double *ty, const double *tz,
                        double *out_re, double *out_im, int nthreads)
{
    ray_job J = {ns, sx, sy, sz, sw, v0, rho1, c1, rho2, c2, zI, k1, k2, tx, ty, tz, out_re, out_im};
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    pthread_t th[256];
    ray_range_arg args[256];
    int64_t per = (nt + nthreads - 1) / nthreads;
    int used = 0;
    for (int q = 0; q < nthreads; ++q) {
        int64_t t0 = q * per, t1 = t0 + per < nt ? t0 + per : nt;
        if (t0 >= t1)
            break;
        args[q].J = &J;
        args[q].t0 = t0;
        args[q].t1 = t1;
        pthread_create(&th[q], NULL, ray_range, &args[q]);
        ++used;
    }
    for (int q = 0; q < used; ++q)
        pthread_join(th[q], NULL);
}
