/*
 * rsi.h -- C ABI of the GB300 (sm_103a) hot path of the quasi-Monte Carlo
 * Rayleigh-Sommerfeld-integral (RSI) beam model of Lello de Almeida, Png and
 * Lan (arXiv 2408.06765).
 *
 * Conventions shared by every call
 *   - Units are SI.  z is depth; the beam travels toward +z.  Complex values
 *     are interleaved (re, im) doubles; the time factor is e^{-i w t}, so an
 *     outgoing wave is e^{+ikr}/r (Sec. 2.1).
 *   - Pointers named *points, *field, *sigma, *out and *workspace are DEVICE
 *     pointers allocated and owned by the caller (for example torch tensors);
 *     structs passed by const pointer are HOST memory, read during the call
 *     only.  The library never frees caller memory and, apart from a small
 *     per-device status word, allocates no device memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     only enqueues work on it and returns; results are ready once the stream
 *     is synchronised.
 *   - Return value: RSI_OK (0) or a negative RSI_E_* code; rsi_last_error()
 *     then describes the failure (thread-local).  Invalid arguments are
 *     rejected before anything is enqueued.
 *   - Errors detected on the device (a bounded wait that expired, a
 *     non-finite result) are written to a per-device status word that
 *     rsi_sync_status() reads and clears.
 */
#ifndef RSI_H
#define RSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RSI_OK 0
#define RSI_E_INVAL (-1)       /* invalid argument (null pointer, size, kind)   */
#define RSI_E_CUDA (-2)        /* a CUDA runtime call failed                    */
#define RSI_E_TIMEOUT (-3)     /* a device-side bounded wait expired            */
#define RSI_E_NONFINITE (-4)   /* a result was NaN or infinite                  */
#define RSI_E_NOMEM (-5)       /* workspace or output buffer too small          */
#define RSI_E_UNSUPPORTED (-6) /* no kernel for this combination / device       */

int rsi_version(void);                 /* library ABI version (this header: 1) */
const char *rsi_last_error(void);      /* message of the last failure on this thread */

/* Wait for `stream`, then read and clear the device status word of the
 * current device.  Returns RSI_OK, RSI_E_TIMEOUT, RSI_E_NONFINITE or
 * RSI_E_CUDA (a CUDA error surfaced by the synchronisation). */
int rsi_sync_status(void *stream);

/* ---- point sets ---------------------------------------------------------- */
/* A point set of n points is ONE caller-allocated device buffer holding
 * structure-of-arrays fields, each starting on a 256-byte boundary at
 * rsi_points_offset(field, n); its total size is rsi_points_bytes(n).
 *   IDX, SU, SV    uint32  Sobol index of the point and its two 32-bit
 *                          (scrambled) coordinates
 *   X, Y, Z        double  position (m)
 *   NX, NY, NZ     double  unit normal pointing toward the observation side
 *   W              double  quadrature weight (area / n, times any Jacobian)
 *   XH..ZL         float   position split as hi = fl32(x), lo = fl32(x - hi)
 */
enum rsi_points_field {
    RSI_PF_IDX = 0, RSI_PF_SU, RSI_PF_SV,
    RSI_PF_X, RSI_PF_Y, RSI_PF_Z,
    RSI_PF_NX, RSI_PF_NY, RSI_PF_NZ,
    RSI_PF_W,
    RSI_PF_XH, RSI_PF_XL, RSI_PF_YH, RSI_PF_YL, RSI_PF_ZH, RSI_PF_ZL,
    RSI_PF_COUNT
};
size_t rsi_points_bytes(int64_t n);
int64_t rsi_points_offset(int32_t field, int64_t n); /* -1 for an unknown field */

enum rsi_surface_kind {
    RSI_SURF_DISK = 0, /* piston face: radius a, centre, tilt about +y          */
    RSI_SURF_RECT = 1, /* flat interface patch wx x wy at z = centre[2], normal +z */
    RSI_SURF_CYL = 2,  /* cylinder, axis parallel to y through (cx, ., cz + R)  */
    RSI_SURF_CAP = 3   /* focused transducer: spherical cap of aperture radius a
                          and radius of curvature R > a, apex at centre, centre
                          of curvature R along the (tilted) axis (Sec. 3.3)   */
};
enum rsi_sequence {
    RSI_SEQ_SOBOL = 0, /* scrambled (or plain) Sobol dimensions 1-2             */
    RSI_SEQ_HALTON = 1 /* the Halton points 1..n in bases 2 and 3 (Sec. 2.3)    */
};

typedef struct rsi_surface {
    int32_t kind;     /* enum rsi_surface_kind                                  */
    int32_t scramble; /* 1: nested bit scramble of the Sobol digits; 0: plain   */
    double centre[3]; /* DISK: face centre; RECT: patch centre; CYL, CAP: apex  */
    double tilt;      /* DISK, CAP: rotation about +y (rad), axis (sin t, 0, cos t) */
    double a;         /* DISK: radius; CAP: aperture radius (m)                 */
    double wx, wy;    /* RECT, CYL: side lengths of the (projected) patch (m)   */
    double R;         /* CYL, CAP: radius of curvature (m); CYL R > wx/2, CAP R > a */
    int32_t sequence; /* enum rsi_sequence (HALTON needs scramble = 0)          */
    int32_t reserved;
    double apod;      /* DISK, CAP: Gaussian profile radius g: weights times
                         exp(-(r/g)^2), r the radius in the aperture; 0 = uniform */
} rsi_surface;

/* Steps a1-a2.  Sobol points 0..n-1 of the set (seed, set_id), dimensions 1
 * and 2, optionally scrambled (digit b flipped by the top bit of SplitMix64's
 * (2^b + leading b digits)-th output for the dimension's key), mapped onto
 * the surface: DISK r = a sqrt(u), theta = 2 pi v (Eq. circle_sampling);
 * RECT x = cx + wx (u - 1/2), y = cy + wy (v - 1/2) (Eq. square_sampling);
 * CYL the same (x, y) with z = cz + R - sqrt(R^2 - (x - cx)^2) and Jacobian
 * R / sqrt(R^2 - (x - cx)^2) in the weight; CAP the disk's (r, theta) lifted
 * onto the sphere (height R - sqrt(R^2 - r^2), Jacobian R / sqrt(R^2 - r^2),
 * normal to the centre of curvature); u = (su + 1/2) 2^-32.  HALTON sets
 * hold points 1..n: su = the base-2 radical inverse as a 32-bit fraction,
 * sv = the base-3 one as a fraction of 3^20 (u = su 2^-32, v = sv / 3^20),
 * stored in index order (slot i = point i + 1).
 * Layout: points are stored in CELL ORDER, not index order: n is split into
 * aligned power-of-two blocks (its binary digits, largest first); within a
 * block of 2^m points, point i goes to slot block_start + morton(cx, cy) with
 * cx the top ceil(m/2) bits of su and cy the top floor(m/2) bits of sv (cx
 * on even bits).  Each block is a (0,m,2)-net, so this is a permutation and
 * consecutive slots are spatially compact.  IDX gives each slot's Sobol index.
 * Requires 1 <= n <= 2^31, points_bytes >= rsi_points_bytes(n).             */
int rsi_make_qmc_points(const rsi_surface *surf, uint64_t seed, uint32_t set_id, int64_t n,
                        void *points, size_t points_bytes, void *stream);

typedef struct rsi_grid {
    double x0, x1; /* x extent (m); pixel i at x0 + (i + 1/2)(x1 - x0)/nx      */
    double z0, z1; /* z extent (m); pixel j at z0 + (j + 1/2)(z1 - z0)/nz      */
    double y;      /* plane of the slice                                        */
    int32_t nx, nz;
} rsi_grid;

/* Step a7 (targets).  Writes the nx*nz cell-centred pixels of the grid as a
 * point set in row-major [nz][nx] order (IDX = pixel index, normals +z,
 * W = 0).  points_bytes >= rsi_points_bytes(nx * nz).                       */
int rsi_grid_points(const rsi_grid *g, void *points, size_t points_bytes, void *stream);

/* Slots [first, first + count) of a point set of n points, every field, as a
 * point set of `count` points in out_points (>= rsi_points_bytes(count)
 * bytes, 256-byte aligned, not overlapping the input).  A stage's targets
 * are independent of one another (each is its own sum in Eq. incident_field
 * and Eq. rayleigh_sommerfeld), so a stage can be evaluated on a contiguous
 * share of its target slots -- the unit of work of a target-sharded chain on
 * several GPUs.  Requires 0 <= first, 1 <= count, first + count <= n.      */
int rsi_points_slice(const void *points, int64_t n, int64_t first, int64_t count, void *out_points,
                     size_t out_bytes, void *stream);

/* ---- stage sums (steps a3, a5, a6) ------------------------------------- */
enum rsi_stage_kind {
    RSI_STAGE_PISTON = 0, /* Eq. incident_field: phi(Q) = -(v0/2pi) sum w e^{ikr}/r */
    RSI_STAGE_RSI = 1     /* Eq. rayleigh_sommerfeld: phi(Q) = -(i/lambda) sum w sigma
                               e^{ikr}/r (1 - 1/(ikr)) cos(theta), cos(theta) =
                               n.(Q - P)/r.  The printed bracket (1/(ikr) - 1)
                               would return -phi for an outgoing field; this is
                               the first Rayleigh-Sommerfeld solution itself.  */
};
enum rsi_precision {
    RSI_PREC_FP64 = 0, /* double precision throughout                          */
    RSI_PREC_FP32C = 1 /* FP32 pair arithmetic; per (target, source tile) a
                          double-float reference distance and phase k R mod 2 pi;
                          compensated accumulation across tiles              */
};
enum rsi_normals {
    RSI_NORMALS_Z = 0,          /* every source normal is +z (flat interface)  */
    RSI_NORMALS_POINTS = 1,     /* use the per-point normals                    */
    RSI_NORMALS_NEG_Z = 2,      /* every source normal is -z: a flat interface
                                   radiating back into the medium the field
                                   came from (the reflected field, Sec. 2.1)   */
    RSI_NORMALS_POINTS_NEG = 3  /* the per-point normals reversed              */
};

typedef struct rsi_stage {
    int32_t kind;      /* enum rsi_stage_kind                                   */
    int32_t precision; /* enum rsi_precision                                    */
    double k;          /* wavenumber of the medium the field propagates in (rad/m) */
    double v0;         /* PISTON: normal velocity amplitude (m/s)               */
    int32_t normals;   /* RSI: enum rsi_normals                                  */
    int32_t tile;      /* sources per shared-memory tile (64, 128, 256); 0 = auto */
    int32_t tpt;       /* targets per thread (FP32C: 1, 2 or 4; FP64: 1); 0 = auto */
    int32_t splits;    /* source splits (>= 1); 0 = auto                          */
    int32_t variant;   /* FP32C distance update: 0 = auto, 1 = reciprocal, 2 = Newton,
                          3 = Newton on two sources per packed f32x2 instruction */
    int32_t reserved;
} rsi_stage;

/* Workspace needed by rsi_propagate_stage for this stage and these sizes
 * (staged source tiles, plus split partial sums).  0 on invalid input.     */
size_t rsi_stage_workspace_bytes(const rsi_stage *st, int64_t n_src, int64_t n_tgt);

/* Steps a3/a5 (+a6).  For every target Q_j of `tgt_points`:
 *   PISTON  field[j] = -(v0 / 2 pi) sum_i w_i e^{ikr_ij} / r_ij
 *   RSI     field[j] = -(i / lambda) sum_i w_i sigma_i e^{ikr}/r (1 - 1/(ikr)) cos(theta_ij)
 * with lambda = 2 pi / k.  Pairs closer than 1e-12 m contribute nothing.
 * src_sigma: complex [n_src] in the source set's slot order (RSI only; NULL
 * for PISTON).  tgt_field: complex [n_tgt] in the target set's slot order,
 * overwritten.  workspace: >= rsi_stage_workspace_bytes(...), 256-byte
 * aligned; its contents are scratch.  Calls that share a workspace must be
 * ordered on one stream.                                                   */
int rsi_propagate_stage(const rsi_stage *st,
                        const void *src_points, int64_t n_src, const double *src_sigma,
                        const void *tgt_points, int64_t n_tgt, double *tgt_field,
                        void *workspace, size_t workspace_bytes, void *stream);

/* Steps a3/a5 (+a6) for nf frequencies at once on the same point sets: a
 * broadband field is the superposition of single-frequency fields (Sec. 4),
 * and frequencies that share the transducer and the interfaces share every
 * point.  The pair geometry (r - R, 1/r, the obliquity) is formed once per
 * pair and used by the nf sums; each frequency adds its phase, its sincos
 * and its source amplitude.  ks: the nf wavenumbers (st->k is not used);
 * src_sigma: complex [nf][n_src] (RSI; NULL for PISTON, whose amplitude does
 * not depend on the frequency); tgt_field: complex [nf][n_tgt], overwritten.
 * FP32C only, 2 <= nf <= 4; st->variant 0 or 3: two sources per packed
 * f32x2 instruction, 2: scalar.  Each frequency's result equals a
 * single-frequency rsi_propagate_stage to rounding; other conventions as
 * rsi_propagate_stage.  The workspace size depends on nf and the variant.
 * Shared harmonic: with nf = 3, the packed variant and one wavenumber twice
 * another (k_j = 2 k_i to a relative 2^-40; with one sound speed, one
 * frequency twice another), e^{i k_j (r - R)} is formed from e^{i k_i (r - R)}
 * by the double angle on pairs away from the tile, two MUFU operations per
 * pair fewer.  The doubled angle carries twice the sincos's angle error: on
 * 2.25, 5 and 10 MHz the 10 MHz image is 9.7e-7 from the FP64 oracle (5.5e-7
 * with its own sincos), far inside the FP32C tolerance.                    */
size_t rsi_stage_multi_workspace_bytes(const rsi_stage *st, int32_t nf, const double *ks, int64_t n_src,
                                       int64_t n_tgt);
int rsi_propagate_stage_multi(const rsi_stage *st, int32_t nf, const double *ks,
                              const void *src_points, int64_t n_src, const double *src_sigma,
                              const void *tgt_points, int64_t n_tgt, double *tgt_field,
                              void *workspace, size_t workspace_bytes, void *stream);
/* 1 if rsi_propagate_stage_multi shares a harmonic for these wavenumbers and
 * this stage (above), 0 if not, a negative status on invalid input.        */
int rsi_stage_multi_shared_harmonic(const rsi_stage *st, int32_t nf, const double *ks);

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot give the library device memory for scratch (a latency-bound
 * acquisition loop that must not call cudaMalloc, a plug-in whose host owns
 * every device allocation, a foreign-language host that only receives
 * finished buffers).  Same sums, arguments and results as
 * rsi_propagate_stage, but the scratch is a fixed area of
 * RSI_NOALLOC_SCRATCH_BYTES compiled into the library (held by every GPU that
 * loads it until the process exits); nothing is allocated.
 *   - The scratch a stage needs is its staged source tiles -- about 32 bytes
 *     per source for FP32C piston and flat-interface stages (some 2.1 million
 *     sources fit), 48 bytes with per-point normals (1.4 million) and 64
 *     bytes for FP64 (1.0 million) -- plus, when the sources are split
 *     across CTAs, 16 bytes per target for every split.  A stage that does
 *     not fit is rejected with RSI_E_NOMEM before anything is enqueued.  With
 *     splits = 0 the call first lowers the automatic split count to what
 *     fits (chosen, below that bound, as rsi_propagate_stage chooses it).
 *   - The first call on a device looks up the area's device address (with
 *     that device current) and keeps it for that device's context; a context
 *     created anew (after cudaDeviceReset) gets a fresh lookup.  Make the
 *     first call before any stream capture.
 *   - All calls on a device share the area: calls whose GPU work overlaps
 *     (other streams, other host threads) race; order them on one stream.
 *     No part of the area has to start at zero.                            */
#define RSI_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int rsi_propagate_stage_noalloc(const rsi_stage *st,
                                const void *src_points, int64_t n_src, const double *src_sigma,
                                const void *tgt_points, int64_t n_tgt, double *tgt_field,
                                void *stream);

/* ---- interface transmission (step a4) ------------------------------------ */
enum rsi_tmode {
    RSI_T_GLOBAL = 0, /* one incidence angle: sin a1 = c1 C, sin a2 = c2 C        */
    RSI_T_LOCAL = 1   /* per point: cos a1 = d . n_i, d = (c1 C, 0, sqrt(1-(c1 C)^2)),
                         sin a2 = (c2/c1) sin a1                                   */
};
typedef struct rsi_interface {
    int32_t mode;       /* enum rsi_tmode                                          */
    int32_t reserved;
    double rho1, c1;    /* medium the field arrives from                           */
    double rho2, c2;    /* medium the field is transmitted into                    */
    double snell_C;     /* Snell invariant sin(a)/c of the beam axis (s/m), Eq. root_searching */
} rsi_interface;

/* Step a4: sigma[i] = T12(a1_i) phi[i] with Eq. transmission_coefficient,
 *   T12 = 2 rho1 c2 cos a1 / (rho2 c2 cos a1 + rho1 c1 cos a2) = (rho1/rho2)(1 + R12),
 * cos a = i sqrt(sin^2 a - 1) past the critical angle.  phi and sigma are
 * complex [n] in slot order; sigma may alias phi.                           */
int rsi_interface_transmit(const rsi_interface *it, const void *points, int64_t n,
                           const double *phi, double *sigma, void *stream);

/* Source density of the reflected field in medium 1: sigma[i] = R12(a1_i)
 * phi[i], the reflected field on the interface taken as R12 times the
 * incident field (Sec. 2.1), R12 of Eq. reflection_coefficient,
 *   R12 = (rho2 c2 cos a1 - rho1 c1 cos a2) / (rho2 c2 cos a1 + rho1 c1 cos a2),
 * with the same incidence angles, modes and arguments as
 * rsi_interface_transmit.  It radiates into medium 1 through
 * rsi_propagate_stage (RSI, k of medium 1, normals reversed).               */
int rsi_interface_reflect(const rsi_interface *it, const void *points, int64_t n,
                          const double *phi, double *sigma, void *stream);

/* ---- ray-tracing model (Sec. 2.2) ------------------------------------------ */
typedef struct rsi_raytrace {
    double k1, k2;       /* wavenumbers of medium 1 (transducer side) and 2 (rad/m) */
    double rho1, c1;     /* medium 1: density, sound speed                          */
    double rho2, c2;     /* medium 2                                                */
    double z_interface;  /* the plane interface z = z_interface (m)                 */
    double v0;           /* piston normal velocity amplitude (m/s)                  */
    int32_t tile;        /* transducer points per tile (32, 64, 128, 256); 0 = auto */
    int32_t splits;      /* transducer-point splits (>= 1); 0 = auto                */
    int32_t newton;      /* Newton steps per pair for the crossing point after a
                            linear prediction from the tile's reference ray, before
                            the convergence test (safeguarded steps then continue,
                            at most 12, until the error bound of the last Newton
                            step, 1.5 max(1/D1, 1/D2) step^2, is < 1 nm); 0 = 1  */
    int32_t reserved;
} rsi_raytrace;

/* Workspace for rsi_raytrace_field (staged transducer tiles and split
 * partial sums); 0 on invalid input.                                      */
size_t rsi_raytrace_workspace_bytes(const rsi_raytrace *rt, int64_t n_src, int64_t n_tgt);

/* Eq. transmitted_ray_tracing: for every target Q_j (in medium 2, z > z_I)
 *   field[j] = -(v0 / 2 pi) sum_i w_i T12 e^{i (k1 D1 + k2 D2)}
 *              / sqrt((D1 + c2 cos^2 a1 / (c1 cos^2 a2) D2) (D1 + (c2 / c1) D2))
 * along the refracted ray from transducer point P_i (in medium 1, z < z_I)
 * to Q_j (Snell's law, Eq. root_searching; D1, D2 the path lengths in the two
 * media; T12 of Eq. transmission_coefficient at the ray's angles).  Points
 * on the wrong side of the interface break the model: their sums come out
 * non-finite (recorded in the status word).  Same conventions for point
 * sets, field, workspace and stream as rsi_propagate_stage.                */
int rsi_raytrace_field(const rsi_raytrace *rt, const void *src_points, int64_t n_src,
                       const void *tgt_points, int64_t n_tgt, double *tgt_field,
                       void *workspace, size_t workspace_bytes, void *stream);

/* ---- field image (step a7) ------------------------------------------------- */
enum rsi_image_format {
    RSI_IMG_C128 = 0, /* complex double [nz][nx]                                */
    RSI_IMG_C64 = 1,  /* complex float  [nz][nx]                                */
    RSI_IMG_ABS32 = 2 /* float |k phi / v0| [nz][nx]                            */
};
/* out[j] = (k / v0) field[j] for the grid's nx*nz pixels (normalised
 * velocity amplitude k phi / v0 of Fig. oblique_incidence).                */
int rsi_field_image(const rsi_grid *g, const double *field, double k, double v0,
                    int32_t format, void *out, void *stream);
/* out[j] = (k / v0) (field_a[j] + field_b[j]): the image of a medium holding
 * two fields at once, e.g. the incident plus the reflected field in medium 1
 * (Fig. rayleigh-sommerfeld_integral).  field_b may be NULL (then as
 * rsi_field_image).                                                        */
int rsi_field_image_sum(const rsi_grid *g, const double *field_a, const double *field_b, double k,
                        double v0, int32_t format, void *out, void *stream);

/* ---- autotuning of the launch shape --------------------------------------- */
/* Times the FP32C launch shapes of one stage on the given data -- tile size
 * (32 ... 512, capped by the accuracy rule of at most n_src/64 sources per
 * tile) x targets per thread {2, 4} x distance update {reciprocal, Newton},
 * each shape needing at most workspace_bytes -- and writes the fastest to
 * *best (kind, precision, k, v0 and normals copied from *st, splits = 0).
 * Each candidate runs once to warm up and twice timed (CUDA events on
 * `stream`); the call synchronises `stream` and leaves the last candidate's
 * field in tgt_field.  Shapes are cached for the process by (kind, normals,
 * ceil(log2 n_src), ceil(log2 n_tgt)); a cached shape returns at once.
 * FP64 stages have one shape and return it untimed.                        */
int rsi_autotune_stage(const rsi_stage *st,
                       const void *src_points, int64_t n_src, const double *src_sigma,
                       const void *tgt_points, int64_t n_tgt, double *tgt_field,
                       void *workspace, size_t workspace_bytes, void *stream, rsi_stage *best);

/* ---- batched chains in one CUDA graph (step a8) ---------------------------- */
/* One instance: piston -> one interface -> image grid (Eq. incident_field,
 * Eq. transmission_coefficient, Eq. approximated_transmitted_field), e.g. one
 * frequency of a broadband pulse (Sec. 4 superposes single-frequency fields)
 * at one scan position.                                                     */
typedef struct rsi_batch_instance {
    rsi_surface piston;       /* RSI_SURF_DISK                                 */
    rsi_surface iface;        /* RSI_SURF_RECT or RSI_SURF_CYL                 */
    int64_t n_piston, n_iface;/* QMC points (1 .. 2^30)                        */
    uint32_t piston_set, iface_set; /* Sobol point-set ids (with the batch seed) */
    rsi_interface transmit;   /* media and Snell invariant of the interface    */
    double k1, k2;            /* wavenumbers before / after the interface      */
    double v0;                /* piston velocity amplitude                     */
    rsi_grid grid;            /* image of this instance                        */
} rsi_batch_instance;

typedef struct rsi_batch_plan rsi_batch_plan; /* opaque, host memory */

/* Plans a batch (host work only, nothing enqueued): per-instance tile sizes
 * by the accuracy rule, work items of about 2^22 pairs sorted largest first,
 * and the workspace layout.  shape: NULL or an FP32C rsi_stage whose tile
 * (upper bound, default 256), tpt (1, 2 or 4, default 1) and variant
 * (default 3) fields override the defaults.  Returns the
 * workspace size and the number of complex64 image elements (the instances'
 * nx*nz, concatenated in instance order).                                  */
int rsi_batch_create(const rsi_batch_instance *inst, int32_t n_inst, uint64_t seed,
                     const rsi_stage *shape, rsi_batch_plan **plan,
                     size_t *workspace_bytes, size_t *image_elems);
/* Runs the whole batch on `stream`: points, piston stages, transmission, RSI
 * stages and images, with the two stage sums as persistent kernels that take
 * work items from a global counter.  The first run with a given workspace /
 * images pair uploads the plan's tables into the workspace (synchronously),
 * captures the work into a CUDA graph and instantiates it; every run then
 * launches that graph.  images: complex64 [image_elems], device.           */
int rsi_batch_run(rsi_batch_plan *plan, void *workspace, size_t workspace_bytes, void *images,
                  void *stream);
int rsi_batch_destroy(rsi_batch_plan *plan);

/* ---- learned surrogate (step a9; no counterpart in the paper) ------------- */
/* Building blocks of a Fourier-feature MLP that maps (x-offset, tilt, water
 * path, frequency, image depth) to the carrier-demodulated image of the RSI
 * chain; it is trained on fields the RSI kernels compute and falls back to
 * them when its held-out error is too large.  Matrices are row-major; bf16
 * arrays are passed as void* (IEEE bfloat16, 2 bytes per element).  All
 * pointers are device pointers; calls are asynchronous on `stream`.         */
enum rsi_nn_epilogue {
    RSI_NN_EPI_F32 = 0,       /* out_f32 = A B^T (+ bias)                              */
    RSI_NN_EPI_BIAS_SILU = 1, /* z = A B^T + bias: out_f32 = z, out_bf16 = silu(z)     */
    RSI_NN_EPI_DSILU = 2      /* out_bf16 = (A B^T) * silu'(aux)   (aux: f32, M x N)   */
};
/* out = [sin(pi B u), cos(pi B u)] (bf16, batch x 2F) with
 * u = 2 (p - lo)/(hi - lo) - 1; p: f32 batch x n_in, B: f32 F x n_in.     */
int rsi_nn_features(const float *params, const float *lo, const float *hi, const float *fmat,
                    int32_t batch, int32_t n_in, int32_t n_freq, void *out_bf16, void *stream);
enum rsi_nn_engine {
    RSI_NN_ENGINE_MMA_SYNC = 0, /* warp-level mma.sync m16n8k16 (K % 32 == 0)          */
    RSI_NN_ENGINE_TCGEN05 = 1   /* tcgen05.mma 128x128x16, accumulators in tensor memory
                                   (K % 64 == 0)                                      */
};
enum rsi_nn_layout {
    RSI_NN_A_T = 1, /* A is stored as [K x M] row-major (its transpose)       */
    RSI_NN_B_T = 2  /* B is stored as [K x N] row-major                       */
};
/* C[M x N] = A[M x K] B[N x K]^T on BF16 tensor cores with FP32 accumulation
 * and the chosen epilogue.  A, B row-major [M x K], [N x K] (K contiguous)
 * unless `layout` says otherwise (tcgen05 engine only).  M, N multiples of
 * 128; A, B 16-byte aligned (the tcgen05 engine: every pointer 16-byte
 * aligned).
 * bias: f32 [N] or NULL (F32 epilogue).  splits > 1 splits K across CTAs
 * (for few output tiles and long K): partial sums go to workspace
 * (f32 [splits][M][N], caller-allocated) and a second kernel adds them in
 * split order and applies the epilogue.                                    */
int rsi_nn_gemm(int32_t epilogue, int32_t engine, int32_t layout, const void *A, const void *B, int32_t M,
                int32_t N, int32_t K, const float *bias, const float *aux, float *out_f32, void *out_bf16,
                int32_t splits, float *workspace, void *stream);
/* out[c][r] = in[r][c] for a bf16 rows x cols matrix.                      */
int rsi_nn_transpose(const void *in_bf16, int32_t rows, int32_t cols, void *out_bf16, void *stream);
/* *loss_out = mean((y - t)^2) over n values (f32, n % 4 == 0, y and t
 * 16-byte aligned); grad_bf16 (may be NULL, 8-byte aligned) = grad_scale *
 * (y - t).  partial: f64 scratch [n_partial] (the number of CTAs of the
 * reduction).                                                              */
int rsi_nn_loss(const float *y, const float *t, int64_t n, float grad_scale, void *grad_bf16,
                double *partial, int32_t n_partial, float *loss_out, void *stream);
/* out[c] = sum over rows of a bf16 rows x cols matrix (bias gradients).    */
int rsi_nn_colsum(const void *m_bf16, int32_t rows, int32_t cols, float *out, void *stream);
/* One Adam step (Kingma & Ba 2015) on n FP32 master weights w with moments
 * m, v and gradient g at step >= 1; writes a bf16 copy to w_bf16 if given. */
int rsi_nn_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float beta1,
                float beta2, float eps, int32_t step, void *w_bf16, void *stream);
/* The same Adam step with its schedule in device memory: hyper points to
 * three floats (lr, 1 - beta1^t, 1 - beta2^t) that the kernel reads when it
 * runs, so that a training step captured in a CUDA graph can be replayed
 * while the caller updates the learning rate and step between replays.    */
int rsi_nn_adam_dev(float *w, float *m, float *v, const float *g, int64_t n, const float *hyper,
                    float beta1, float beta2, float eps, void *w_bf16, void *stream);
/* bf16 copy of an f32 array.                                               */
int rsi_nn_cast_bf16(const float *in, int64_t n, void *out_bf16, void *stream);
/* out = scale * in * exp(sign i psi) per pixel of batch images (complex f32
 * pairs, row-major [nz][nx] over `window`, relative coordinates), with
 * psi = kx x + kz z + phi0 and carrier[b] = (kx, kz, phi0, unused) (f64).
 * The phase carries about 2e-6 rad of error, its sine and cosine about 4e-7;
 * windows of more than 2^24
 * pixels and a non-finite scale return RSI_E_INVAL.                        */
int rsi_nn_carrier(const double *carrier, int32_t batch, const rsi_grid *window, int32_t sign,
                   float scale, const float *in, float *out, void *stream);
/* The output layer and the carrier in one kernel (tcgen05 engine):
 * out = scale * exp(sign i psi) * (A B^T + bias), row b of the M x N result
 * being image b of interleaved complex pixels over `window` (N = 2 nx nz)
 * and psi its carrier as in rsi_nn_carrier (carrier[b] = (kx, kz, phi0, .)).
 * A [M x K] and B [N x K] bf16, K-major; M % 128 == 0, N % 128 == 0,
 * K % 64 == 0; A, B, out, bias and workspace 16-byte aligned; workspace
 * holds M x 32 bytes (each row's phase constants, formed once per call).
 * Within a block of 16 pixels the carrier advances by rotation from one
 * exact phase, which adds up to about 2e-6 relative to rsi_nn_carrier's
 * per-pixel phase.  Fusing the two saves writing the layer's output and
 * reading it back.                                                          */
int rsi_nn_gemm_carrier(const void *a_bf16, const void *b_bf16, int32_t M, int32_t N, int32_t K,
                        const float *bias, const double *carrier, const rsi_grid *window, int32_t sign,
                        float scale, float *out, float *workspace, void *stream);
/* The surrogate's carrier coefficients on the device: for each of `batch`
 * parameter rows (x-offset, tilt, water path L, frequency f, image depth d;
 * f64, row-major [batch][5]) carrier[b] = (k2 s, k2 c, k1 L + k2 c d, 0),
 * k = 2 pi f / c_medium, s = (c2/c1) sin(tilt), c = sqrt(max(0, 1 - s^2))
 * (the refracted plane wave below the interface, Snell's law), in FP64; and
 * params_f32 = the rows rounded to f32 (the network's input).               */
int rsi_nn_carrier_coeffs(const double *params, int32_t batch, double c1, double c2, double *carrier,
                          float *params_f32, void *stream);

/* ---- the surrogate's coordinate network (step a9; not in the paper) ------- */
/* The surrogate evaluates one network row per (field, pixel): its inputs are
 * built from the field's parameters (x-offset, tilt, water path L, frequency
 * f, image depth d; f64 [field][5]) and the pixel's place in the window, its
 * three outputs are the pixel's carrier-demodulated field divided by the
 * field's RMS (re, im) and the log of that RMS.  Row inputs c (9 values),
 * with x from the point where the transducer axis meets the interface and z
 * below the interface (the window's top edge lies d below it):
 *   sg = sign(tilt), a1 = |tilt|, x = sg (window x), z = d + (window z),
 *   th = asin(min(1, (c2/c1) sin a1))                (Snell's law),
 *   s = x sin th + z cos th, t = x cos th - z sin th  (refracted-axis frame),
 *   q = a^2 f / (c1 (L + (c2/c1) max(s, 0)))          (Fresnel number),
 *   c = [n(a1), n(L), n(f), n(d), x/S0, 2 (zw - z0)/Wz - 1, s/S0, t/S0, ln q],
 * n(v) = 2 (v - lo)/(hi - lo) - 1 over box_lo/box_hi, S0 = (x1 - x0)/2; the
 * network input is [sin(pi B c), cos(pi B c), c, 0 x 7] (bf16, 2F + 16
 * wide), then `depth` SiLU layers of `width` and a linear head of 3.       */
#define RSI_NN_IN 9
#define RSI_NN_MAX_DEPTH 8
typedef struct rsi_nn_net {
    int32_t n_freq;      /* F: input rows are 2F + 16 wide, a multiple of 64     */
    int32_t width;       /* hidden width, a multiple of 128                        */
    int32_t depth;       /* hidden layers, 1 .. RSI_NN_MAX_DEPTH                   */
    int32_t rows;        /* rows per forward / backward call, a multiple of 128    */
    int32_t engine;      /* enum rsi_nn_engine (the hidden layers' GEMMs)          */
    int32_t reserved;
    double c1, c2;       /* sound speeds before / after the interface (m/s)        */
    double a;            /* piston radius (m)                                      */
    double box_lo[4], box_hi[4]; /* box of (|tilt|, L, f, d) for n()               */
    rsi_grid window;     /* window in relative coordinates (see above)             */
    const float *fmat;   /* device, f32 [F][9]: the Fourier matrix B               */
} rsi_nn_net;

/* Flat parameter buffers (f32 master weights, Adam moments, gradients: each
 * rsi_nn_param_elems() floats; their bf16 copy the same count of bf16):
 * layer l = 0 .. depth - 1 holds W_l [width][in_l] then b_l [width] (in_0 =
 * 2F + 16, else width), layer `depth` the head W [3][width] then b [3]; every
 * segment starts on a multiple of 64 elements.  rsi_nn_param_offset gives
 * the element offset of W (bias = 0) or b (bias = 1) of a layer; -1 if the
 * net or the layer is invalid.                                              */
int64_t rsi_nn_param_elems(const rsi_nn_net *net);
int64_t rsi_nn_param_offset(const rsi_nn_net *net, int32_t layer, int32_t bias);
/* Bytes of the activation workspace of one forward + backward of `rows`
 * rows (inputs, pre-activations, activations, head outputs, targets, the
 * backward's buffers and split-K partial sums); 0 for an invalid net.       */
size_t rsi_nn_act_bytes(const rsi_nn_net *net);

enum rsi_nn_rows_mode {
    RSI_NN_ROWS_RANDOM = 0, /* row r: a (field, pixel) pair drawn from SplitMix64
                               (Steele, Lea & Flood 2014) at (seed, r): uniform
                               over the n_fields x nx nz pairs               */
    RSI_NN_ROWS_PIXELS = 1  /* row r: pair first + r, field-major: field
                               (first + r) / (nx nz), pixel the remainder      */
};
/* Network input rows into the workspace `act`; with targets (f32
 * [n_fields][nx nz][2], the demodulated field over its RMS) and log_rms (f32
 * [n_fields]) also the rows' targets (re, im, log rms, 0) for
 * rsi_nn_backward.  seed_dev (device, optional) overrides `seed` with a
 * value read when the kernel runs, so that a captured training step draws new
 * rows on every replay.  Rows past the last pair (PIXELS mode) repeat it.    */
int rsi_nn_rows(const rsi_nn_net *net, const double *params, int64_t n_fields, int32_t mode, uint64_t seed,
                const uint64_t *seed_dev, int64_t first, const float *targets, const float *log_rms, void *act,
                size_t act_bytes, void *stream);
/* Forward pass of the rows in `act`: the hidden layers on the tensor cores
 * (bf16 weights w16, f32 biases from w32), the head in f32; head outputs
 * y (f32 [rows][4], the fourth 0) are written to `act` and, if y is not
 * NULL, copied to y.                                                        */
int rsi_nn_forward(const rsi_nn_net *net, const void *w16, const float *w32, void *act, size_t act_bytes,
                   float *y, void *stream);
/* Backward pass after rsi_nn_forward and rsi_nn_rows with targets: gradients
 * of loss = sum over rows and outputs of (y - t)^2 / (4 rows) into grad (f32,
 * flat, every parameter overwritten); *loss_dev (device f32) receives the
 * loss.  The backward's GEMMs read their operands transposed in place and so
 * run on the tcgen05 engine whatever net->engine says.                      */
int rsi_nn_backward(const rsi_nn_net *net, const void *w16, const float *w32, void *act, size_t act_bytes,
                    float *grad, float *loss_dev, void *stream);
/* One Adam step on every parameter (flat buffers) with the schedule in
 * device memory (hyper: lr, 1 - beta1^t, 1 - beta2^t); refreshes w16.       */
int rsi_nn_adam_step(const rsi_nn_net *net, float *w32, float *m, float *v, const float *grad, void *w16,
                     const float *hyper, float beta1, float beta2, float eps, void *stream);
/* Training targets of n_fields images (complex64 [n][nz][nx], e.g. from the
 * RSI path): each image times exp(-i psi) (psi as in rsi_nn_infer) divided by
 * its RMS over the window -> targets (f32 [n][nx nz][2]), and the log of that
 * RMS -> log_rms (f32 [n]).  carrier (f64 [n][4]), params_f32 (f32 [n][5])
 * and env (f32 [n][nx nz][2]) are scratch.                                  */
int rsi_nn_targets(const rsi_nn_net *net, const double *params, int32_t n_fields, const float *images,
                   double *carrier, float *params_f32, float *env, float *targets, float *log_rms, void *stream);
/* Images of n_fields parameter rows (f64 [n][5]): for each field, its
 * nx nz rows through the network (rows must be a multiple of nx nz), then
 * exp(mean log rms) (re + i im) exp(i psi) with psi the refracted plane
 * wave's phase k1 L + k2 (S x + C z) (S = (c2/c1) sin tilt, C = sqrt(max(0,
 * 1 - S^2))).  out: complex64 [n][nz][nx]; carrier: f64 [n][4] scratch.    */
int rsi_nn_infer(const rsi_nn_net *net, const void *w16, const float *w32, const double *params, int32_t n_fields,
                 void *act, size_t act_bytes, double *carrier, float *out, void *stream);

/* ---- measurement hooks (no counterpart in the paper) --------------------- */
/* Number of kernels this library has enqueued in this process.             */
uint64_t rsi_launch_count(void);

/* Per-kernel timing of the source x target kernels.  While enabled, every
 * rsi_propagate_stage and rsi_raytrace_field call brackets its main kernel
 * with CUDA events recorded on the call's stream.  rsi_timing_enable(1)
 * clears the record and starts; rsi_timing_enable(0) stops.
 * rsi_timing_read(kind, ...) synchronises with the recorded events and
 * returns, for the kernels of that kind (RSI_STAGE_PISTON, RSI_STAGE_RSI or
 * RSI_TIMING_RAYTRACE): the summed kernel time in ms, the number of launches
 * and the summed source x target pair count.                               */
#define RSI_TIMING_RAYTRACE 2
int rsi_timing_enable(int32_t on);
int rsi_timing_read(int32_t kind, double *total_ms, int64_t *launches, double *pairs);

/* Exercises the device-side failure path without a fault: one CTA waits on
 * an mbarrier that nothing completes, gives up after `cycles` SM clocks
 * (1 .. 2^32) exactly as the stage kernels' bounded waits do, records
 * RSI_E_TIMEOUT in the status word and exits; rsi_sync_status() then returns
 * RSI_E_TIMEOUT (and clears the word).                                      */
int rsi_selftest_wait_timeout(int64_t cycles, void *stream);

/* Throughput probes for the ALU roofline: `iters` iterations of 8
 * independent dependency chains per thread of one operation,
 *   RSI_UB_FFMA  fused multiply-add (FP32 pipe)
 *   RSI_UB_RSQRT rsqrt.approx.f32   (MUFU)
 *   RSI_UB_SIN   sin.approx.f32     (MUFU, after its range scaling)
 *   RSI_UB_DFMA  fused multiply-add in double precision (FP64 pipe)
 * over `blocks` CTAs of 256 threads; `sink` (device, >= blocks*256 floats)
 * receives one value per thread.  Time it with events on `stream`.         */
enum rsi_ubench_kind { RSI_UB_FFMA = 0, RSI_UB_RSQRT = 1, RSI_UB_SIN = 2, RSI_UB_DFMA = 3 };
int rsi_ubench(int32_t kind, int32_t blocks, int32_t iters, float *sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RSI_H */
