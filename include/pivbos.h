/*
 * pivbos -- ray-traced PIV/BOS image generation on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library libpivbos.so.  The calls follow the problem
 * statement of Rajendran, Bane & Vlachos, "PIV/BOS Synthetic Image Generation
 * in Variable Density Environments" (arXiv 1812.05902), Sec. 3: rays leave
 * sources (particles or BOS dots) toward the lens (Sec. 3.1), bend in a
 * refractive-index field built from density by the Gladstone-Dale relation
 * (Sec. 3.2, Eqs. 1-6), pass the optical elements (Sec. 3.3, Eq. 7) and
 * deposit a diffraction spot on the sensor (Sec. 3.4, Eq. 8).
 *
 * Conventions shared by every call:
 *  - SI units.  z is the optical axis, from the sources toward the sensor.
 *  - Every call returns a pivbos_status and never aborts the process; a
 *    message for the last failure on the calling thread is available from
 *    pivbos_last_error().
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream are asynchronous on it unless stated
 *    otherwise; device errors detected inside kernels are latched in a
 *    per-device status word that pivbos_sync() returns and clears.
 *  - Handles own their device memory, are immutable after creation except
 *    through pivbos_medium_refill(), and may be shared by renders on
 *    different streams of the device they were created on.
 *  - Device pointers must belong to the current device; host pointers may
 *    be pageable or pinned.
 */
#ifndef PIVBOS_H
#define PIVBOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIVBOS_OK = 0,
    PIVBOS_ERR_INVALID_ARG = 1,     /* NULL pointer, bad size, bad enum, wrong device */
    PIVBOS_ERR_OOM = 2,             /* device or host allocation failed */
    PIVBOS_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    PIVBOS_ERR_DEVICE_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    PIVBOS_ERR_OVERFLOW = 5,        /* more than 2^31 rays in one render */
    PIVBOS_ERR_UNSUPPORTED = 6      /* valid but outside what the kernels handle */
} pivbos_status;

/* Final state of a ray (pivbos_ray_state.status); also the index into the
 * per-render counters of pivbos_render(). */
enum {
    PIVBOS_RAY_REACHED = 0,     /* deposited on the sensor */
    PIVBOS_RAY_STOP = 1,        /* blocked by an aperture (Sec. 3.3, item 3) */
    PIVBOS_RAY_MISS = 2,        /* missed a surface or left its clear radius */
    PIVBOS_RAY_TIR = 3,         /* total internal reflection (Sec. 3.3, item 2) */
    PIVBOS_RAY_OFF_SENSOR = 4,  /* crossed the sensor plane outside the pixels */
    PIVBOS_RAY_MAXSTEP = 5,     /* integration step budget exhausted */
    PIVBOS_RAY_NSTATUS = 6
};

/* Optical element kinds (Sec. 3.3).  Elements are sequential along +z.  A
 * mirror reflects by the law of reflection (Sec. 3.3, item 1) and the system
 * is unfolded there: the reflected ray and every later element (and the
 * sensor) are described in the frame mirrored about the mirror's vertex
 * plane, z -> 2 z_vertex - z, so later elements sit at larger z.  Mirrors
 * are coaxial; the index the ray travels in does not change at a mirror. */
enum {
    PIVBOS_SURF_SPHERE = 0,     /* refracting sphere: vertex z, signed radius (centre at z + R) */
    PIVBOS_SURF_PLANE = 1,      /* flat refracting surface at z */
    PIVBOS_SURF_IDEAL_THIN = 2, /* ideal thin lens of focal length f at z (slopes u' = u - x/f) */
    PIVBOS_SURF_STOP = 3,       /* aperture: rays outside clear_radius at z are blocked */
    PIVBOS_SURF_MIRROR = 4,     /* mirror: vertex z, signed radius (0 = flat, square to the axis) */
    PIVBOS_SURF_LENS_ARRAY = 5  /* square array of ideal thin lenslets at z (Sec. 3.3: plenoptic camera):
                                   focal length f, lenslet pitch in `radius`, lenslet centres at
                                   (i pitch, j pitch); a ray uses the lenslet whose cell holds it:
                                   u' = u - (x - centre) / f */
};

/* Integrators of the ray equation (Sec. 3.2). */
enum {
    PIVBOS_EULER = 0,           /* first-order piecewise-linear scheme */
    PIVBOS_RK4 = 1              /* Runge-Kutta scheme of Sharma et al., Eqs. 3-6 */
};

#define PIVBOS_MAX_SURFACES 16
/* The spot window is at most this many pixels per axis: sigma/pitch must not
 * exceed (PIVBOS_MAX_WINDOW - 2) / 6. */
#define PIVBOS_MAX_WINDOW 12

typedef struct {
    int32_t type;          /* PIVBOS_SURF_* */
    int32_t reserved;      /* must be 0 */
    double z_vertex;       /* m, position of the vertex (or plane) on the axis */
    double radius;         /* m, signed radius of curvature (spheres, mirrors); lenslet pitch (lens arrays) */
    double focal;          /* m, focal length (ideal thin lens, lens array) */
    double n_after;        /* refractive index after the surface */
    double clear_radius;   /* m, clear (or stop) radius */
} pivbos_surface;

/* Per-ray result of pivbos_trace_exit_states (104 bytes, naturally aligned). */
typedef struct {
    double vol_pos[3];     /* where the ray left the density box (its source if it never entered) */
    double vol_dir[3];     /* unit direction there */
    double sensor_xy[2];   /* pixel coordinates on the sensor (valid if status is REACHED or OFF_SENSOR) */
    double sensor_dir[3];  /* unit direction at the sensor plane */
    int32_t status;        /* PIVBOS_RAY_* */
    int32_t steps;         /* integration steps taken inside the box */
    double opl;            /* optical path inside the box, integral of n ds (m): the integral of n^2 dt in
                              the parameter of Eqs. 3-5, by Simpson's rule on the RK4 stage points (the left
                              rule for the first-order scheme), summed in double-float; 0 if the ray never
                              enters the box */
} pivbos_ray_state;

typedef struct pivbos_medium pivbos_medium;
typedef struct pivbos_optics pivbos_optics;

/* ---------------------------------------------------------------------------
 * Medium (Sec. 3.2).  rho is a density grid [nz][ny][nx] (x fastest, float32,
 * kg/m^3) with nodes at origin + (i, j, k) * spacing.  The library stores
 * n - 1 = K_GD * rho (Eq. 1) and grad n at every node (second-order central
 * differences, second-order one-sided at the faces, two-point differences on
 * an axis with two nodes) as one float4 per node; rays are straight outside
 * the box [origin, origin + (n-1) * spacing] and inside it follow the ray
 * equation with n and grad n sampled trilinearly (clamped to the box).
 *
 * rho_on_device: 1 if rho is a device pointer on the current device, 0 for
 * host memory (copied).  The call does not keep rho.  nx, ny, nz >= 2;
 * spacing > 0; K_GD finite.  The grid build runs on `stream`; the handle is
 * usable by work later on that stream (or after pivbos_sync).
 * Errors: INVALID_ARG, OOM, CUDA.
 * ------------------------------------------------------------------------- */
pivbos_status pivbos_medium_create(const float* rho, int rho_on_device, int nx, int ny, int nz,
                                   const double origin[3], const double spacing[3], double K_GD,
                                   void* stream, pivbos_medium** out);

/* Rebuild the node field of an existing medium from a new density grid of
 * the same dimensions (time series, or one frame per step), on `stream`.
 * Renders enqueued earlier on other streams must be complete. */
pivbos_status pivbos_medium_refill(pivbos_medium* m, const float* rho, int rho_on_device, void* stream);

void pivbos_medium_destroy(pivbos_medium* m);

/* ---------------------------------------------------------------------------
 * Optics and sensor (Sec. 3.3-3.4).  `surfaces` are applied in order
 * (n_surfaces <= PIVBOS_MAX_SURFACES, may be 0); n_object is the refractive
 * index the rays travel in before the first surface.  Rays are aimed at points
 * drawn uniformly over the disk of radius aim_radius centred on the axis at
 * z = aim_z (Sec. 3.1: a ray joins its source to a point on the lens).  The
 * sensor is the plane z = sensor_z with width x height square pixels of
 * pixel_pitch; pixel (i, j) covers x/pitch + width/2 in [i, i+1) and
 * y/pitch + height/2 in [j, j+1).  The spot is a Gaussian of sigma = d_tau/4
 * with d_tau from Eq. 8: dtau_rule 0 uses the printed 2.44 pi f# (M+1) lambda,
 * dtau_rule 1 the textbook 2.44 f# (M+1) lambda.  The host arrays are copied.
 * Errors: INVALID_ARG; UNSUPPORTED if sigma/pitch exceeds
 * (PIVBOS_MAX_WINDOW - 2) / 6.
 * ------------------------------------------------------------------------- */
pivbos_status pivbos_optics_create(const pivbos_surface* surfaces, int n_surfaces, double n_object,
                                   double aim_z, double aim_radius,
                                   double f_number, double magnification, double wavelength,
                                   int dtau_rule, double sensor_z, double pixel_pitch,
                                   int width, int height, pivbos_optics** out);

/* A copy of `o` whose sensor is turned about its centre (0, 0, sensor_z):
 * first by tilt_x radians about the x axis, then by tilt_y about the y axis
 * (Fig. 1(d): perspective; the Scheimpflug arrangement).  Pixel (i, j) then
 * covers [i, i+1) x [j, j+1) along the turned x and y axes of the sensor,
 * the sensor centre at the array centre; a ray meets the sensor plane where
 * the line crosses it (a ray travelling away from the sensor's front, or
 * with the plane behind it, is a MISS).  The spot keeps its size in pixels.
 * Errors: INVALID_ARG (NULL, non-finite angles), OOM. */
pivbos_status pivbos_optics_tilt_sensor(const pivbos_optics* o, double tilt_x, double tilt_y, pivbos_optics** out);

/* Sec. 3.1: the radiance of a ray from a PIV particle follows Mie
 * scattering (the paper uses the method of Bohren & Huffman).  pivbos_mie
 * evaluates the series solution for a homogeneous sphere of `diameter` in a
 * medium of index n_medium lit at vacuum `wavelength`, with relative index
 * m = m_re + i m_im (m_im >= 0 absorbs): s12 (host double [n_angles][2])
 * receives |S1|^2 and |S2|^2 at theta_i = pi i / (n_angles - 1) from the
 * laser's direction; q (host double [4], may be NULL) receives Q_ext,
 * Q_sca, Re S(0) and the number of terms (x + 4 x^(1/3) + 2, size parameter
 * x = pi diameter n_medium / wavelength).  Runs on the current device,
 * synchronously (allocates its own scratch).  Errors: INVALID_ARG;
 * UNSUPPORTED for x > 20000; OOM; CUDA. */
pivbos_status pivbos_mie(double diameter, double wavelength, double n_medium, double m_re, double m_im,
                         int n_angles, double* s12, double* q);

/* A copy of `o` whose rays carry Mie radiance: a ray leaving its source
 * along d0 has theta = acos(d0 . laser_dir); |S1|^2 and |S2|^2 are
 * interpolated linearly in theta from the table s12 (host, as pivbos_mie
 * writes it, n_angles >= 2 covering 0..pi); its radiance is
 * |S2|^2 cos^2(phi) + |S1|^2 sin^2(phi) for a laser polarised along
 * `polarisation` (host double[3], normal to laser_dir; phi is its angle to
 * the scattering plane, which holds laser_dir and d0), or the mean of the
 * two for unpolarised light (polarisation NULL); divided by the largest
 * table entry, so weights lie in [0, 1].  A ray of weight w adds
 * round(w 2^32) to the image in all, spread like any spot.  The table is
 * held in FP32 on the device by the new handle.  Renders, batches and the
 * surrogate path use the weights; the BOS displacement means and the
 * per-ray exit states ignore them.  Errors: INVALID_ARG, OOM, CUDA. */
pivbos_status pivbos_optics_radiance(const pivbos_optics* o, const double laser_dir[3], const double* polarisation,
                                     const double* s12, int n_angles, pivbos_optics** out);

void pivbos_optics_destroy(pivbos_optics* o);

/* ---------------------------------------------------------------------------
 * Render (Sec. 3, all four steps; Sec. 3.5: one GPU thread per ray).
 * Traces rays_per_source rays from each of n_sources sources ([n][3] float64,
 * metres) and adds their spots into `image` ([height][width] int64, 32.32
 * fixed point: every ray that reaches the sensor adds exactly 2^32, so the
 * image is bit-identical from run to run and sums of partial renders equal
 * the whole render).  Ray k of source s draws its lens point from
 * Philox4x64-10 with counter (k, s, frame, 0) and key (seed, 0).  m may be
 * NULL (uniform medium everywhere).  integrator: PIVBOS_EULER or PIVBOS_RK4;
 * step: parameter step (t with dt = ds/n, so the arc length per step is about
 * n * step), > 0.
 *
 * sources_on_device / image_on_device: 1 for device pointers, 0 for host
 * memory.  With a host image the call copies it to the device, renders,
 * copies it back and synchronises `stream` before returning.  stats, if not
 * NULL, is a device array of PIVBOS_RAY_NSTATUS int64 counters that the call
 * adds the final status of every ray into.
 * Errors: INVALID_ARG; OVERFLOW if n_sources * rays_per_source > 2^31;
 * OOM; CUDA.
 * ------------------------------------------------------------------------- */
pivbos_status pivbos_render(const pivbos_medium* m, const pivbos_optics* o,
                            const double* sources, int64_t n_sources, int sources_on_device,
                            int32_t rays_per_source, uint64_t seed, uint32_t frame,
                            int integrator, double step,
                            int64_t* image, int image_on_device, int64_t* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Render without allocating (no counterpart in the paper: a library
 * facility).  For callers that cannot call cudaMalloc -- a host application
 * that has given the whole device to its own memory pool and forbids
 * allocations outside it, or a latency-critical loop in which the implicit
 * synchronisation of cudaMalloc/cudaFree would stall other streams.  Same
 * arguments and result as pivbos_render (the same kernels: the image and
 * stats are bit-identical), except that `sources` and `image` must be device
 * pointers (stats too, if not NULL) and the call never allocates or frees
 * memory.  Its scratch (Morton keys, the source permutation and a sorted
 * copy of the sources, ~4.5 MiB) is a fixed array in the library's device
 * image, held by every GPU that loads the library until the process exits.
 *  - n_sources above PIVBOS_NOALLOC_MAX_SOURCES: PIVBOS_ERR_UNSUPPORTED.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before capturing any stream.
 *  - Every call on a device uses the same array, which keeps the previous
 *    call's contents (the call rewrites what it reads).  Calls that overlap
 *    on the GPU (concurrent streams) race on it: serialise them.
 *  - Device-side errors land in the same per-device status word as every
 *    other call's (a fixed device array as well); pivbos_sync returns it.
 *  - Keep kernel timing (pivbos_timing_enable) off: timing creates CUDA
 *    events.
 * ------------------------------------------------------------------------- */
#define PIVBOS_NOALLOC_MAX_SOURCES (1 << 17)
pivbos_status pivbos_render_noalloc(const pivbos_medium* m, const pivbos_optics* o,
                                    const double* sources, int64_t n_sources, int32_t rays_per_source,
                                    uint64_t seed, uint32_t frame, int integrator, double step,
                                    int64_t* image, int64_t* stats, void* stream);

/* The render of sources [first_source, first_source + n_sources) of a larger
 * source set: `sources` points at that sub-range and ray k of local source s
 * draws its lens point with counter (k, first_source + s, frame, 0).  Renders
 * of disjoint ranges (on one GPU or on several) add up, bit for bit, to the
 * render of the whole set.  first_source + n_sources <= 2^32. */
pivbos_status pivbos_render_range(const pivbos_medium* m, const pivbos_optics* o,
                                  const double* sources, int64_t n_sources, int64_t first_source,
                                  int sources_on_device, int32_t rays_per_source, uint64_t seed,
                                  uint32_t frame, int integrator, double step,
                                  int64_t* image, int image_on_device, int64_t* stats, void* stream);

/* Per-ray exit states for the parity checks: the same tracing as
 * pivbos_render, without the deposit.  ray_ids (device, int64, may be NULL
 * for "all rays in order") lists flattened ids source * rays_per_source + k;
 * out (device) receives n_rays pivbos_ray_state.  Errors as pivbos_render. */
pivbos_status pivbos_trace_exit_states(const pivbos_medium* m, const pivbos_optics* o,
                                       const double* sources, int64_t n_sources, int sources_on_device,
                                       int32_t rays_per_source, uint64_t seed, uint32_t frame,
                                       int integrator, double step,
                                       const int64_t* ray_ids, int64_t n_rays,
                                       pivbos_ray_state* out, void* stream);

/* ---------------------------------------------------------------------------
 * Batched rendering (many frames of uneven size in one persistent launch).
 * A frame is one pivbos_render call's worth of arguments with device
 * buffers.  pivbos_batch_create validates the frames, allocates the
 * per-frame sort scratch and a device work queue, and orders the frames by
 * estimated work (largest first).  pivbos_batch_render enqueues, on
 * `stream`, the Morton ordering of every frame's sources and one persistent
 * kernel whose CTAs pop (frame, chunk of rays) items until all frames are
 * done; images and stats are accumulated into exactly as pivbos_render
 * would.  With tuning.use_graph the first call captures this sequence into
 * a CUDA graph (on a private stream) and every call launches that graph on
 * `stream` (the frames' buffers must stay at the same addresses; their
 * contents may change).
 * All frames of a batch share one integrator.  The batch does not own the
 * media, optics or buffers, which must outlive it.
 * Errors: as pivbos_render; INVALID_ARG for a frame with host buffers.
 * ------------------------------------------------------------------------- */
typedef struct {
    const pivbos_medium* medium;   /* NULL = uniform medium */
    const pivbos_optics* optics;
    const double* sources;         /* device [n_sources][3] */
    int64_t n_sources;
    int32_t rays_per_source;
    uint32_t frame;                /* Philox counter word of the frame */
    uint64_t seed;
    double step;                   /* integration parameter step, > 0 */
    int64_t* image;                /* device int64 [H][W] of the optics, accumulated into */
    int64_t* stats;                /* device int64 [PIVBOS_RAY_NSTATUS] or NULL */
} pivbos_frame_desc;

typedef struct {
    int32_t rays_per_cta;          /* rays per work item: 256..2048, multiple of 256 */
    int32_t cell_cache;            /* 1: keep the last cell's corners in registers */
    int32_t ctas_per_sm;           /* persistent CTAs per SM: 1..3 (1..2 with cell_cache) */
    int32_t use_graph;             /* 1: capture once per stream, then replay a CUDA graph */
} pivbos_tuning;

typedef struct pivbos_batch pivbos_batch;

/* Defaults: 2048 rays per item, no cell cache, 3 CTAs per SM, graphs on. */
pivbos_status pivbos_default_tuning(pivbos_tuning* out);

/* tuning NULL: the defaults, except that the cell cache (with 2 CTAs per
 * SM) is used when dense frames (>= 64 field evaluations per ray) whose
 * smallest grid spacing exceeds 4/3 of the step carry most of the estimated
 * work. */
pivbos_status pivbos_batch_create(const pivbos_frame_desc* frames, int n_frames, int integrator,
                                  const pivbos_tuning* tuning, pivbos_batch** out);
pivbos_status pivbos_batch_render(pivbos_batch* b, void* stream);
void pivbos_batch_destroy(pivbos_batch* b);

/* Autotuner for one frame (synchronous on `stream`; allocates its own
 * scratch, never writes the frame's image or stats).
 *  - step: starting from frame->step, the largest step (doubling, at most
 *    64x; halving, at most 64x, if the start is too coarse) whose estimated
 *    sensor error on n_sample_rays seeded rays stays within tol_px pixels;
 *    the error of step h is estimated from the traces with h and h/2
 *    (Richardson: x 16/15 for RK4, x 2 for the first-order scheme).  With
 *    no medium the step is returned unchanged.
 *  - tuning: the fastest of rays_per_cta in {512, 1024, 2048} with and
 *    without the cell cache, timed on a sub-frame of about 4e6 rays.
 * Results are only suggestions: the caller decides which step to render
 * with (the step changes the integration, hence the image). */
pivbos_status pivbos_autotune(const pivbos_frame_desc* frame, int integrator, double tol_px,
                              int32_t n_sample_rays, double* step_out, pivbos_tuning* tuning_out,
                              void* stream);

/* The surrogate's network parameters: PIVBOS_MLP_PARAMS floats, layer by
 * layer W [out][in] then b [out] (16 inputs -> 128 -> 128 -> 128 -> 128 -> 4). */
#define PIVBOS_MLP_PARAMS 52228

/* ---------------------------------------------------------------------------
 * Surrogate ray map (no counterpart in the paper: a learned part built on
 * the tracer of Sec. 3.2).  For a ray with entry state E -- where its
 * straight line meets z = max(box front, source z), and its slopes dx/dz,
 * dy/dz -- the surrogate predicts the residual of its exit line against the
 * straight ray (position difference on a reference plane, slope
 * difference) as
 *     r(E) = r_proj(E) + MLP(E, r_proj(E)),
 * where r_proj is the first-order (Born) residual: the ray equation's
 * dT/ds = grad n integrated along the unperturbed line, read from a table
 * of integrals of grad n along lines through the lens pupil centre (built
 * once per surrogate from the medium), the line cut into born_segments
 * pieces.  The network (BF16 16 -> 128 x 4 -> 4, ReLU, FP32 accumulation)
 * learns the correction from rays of the frame traced by the plain path
 * (Philox counter (sample, stream, frame, 2) picks them); training runs on
 * the GPU (tensor cores, Adam, cosine learning rate), the loss weighting
 * each output by its measured effect on the sensor.
 *
 * Confidence: on held-out rays the plain tracer judges the predictors at the
 * sensor, per entry-space bin (16 x 16 x 16 positions x 4 x 4 slopes).
 * With one predictor, bins are served in order of plain-path steps saved
 * per unit of squared sensor error while the summed error keeps the RMS over
 * all rays reaching the sensor within budget_margin * err_budget_px; with
 * the automatic choice each bin takes the least costly of the projection,
 * the corrected projection and the plain path under the same budget.  Rays
 * of bins not served are traced by the plain path at render time.  The report gives the same figures for
 * the projection alone and for the straight ray.  The surrogate is tied to
 * the frame's medium and optics (they must outlive it; a refill of the
 * medium makes later surrogate calls fail with INVALID_ARG) and needs the
 * lens after the box.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n_train;        /* training rays (<= 2^31) */
    int64_t n_val;          /* held-out rays for the confidence map (<= 2^31) */
    int32_t epochs;
    int32_t batch;          /* rows per step, 256..65536 */
    float lr;               /* peak learning rate (cosine decay to 1 %) */
    float err_budget_px;    /* RMS sensor error budget over all rays (px) */
    float budget_margin;    /* fraction of the budget the held-out estimate may use, (0, 1] */
    int32_t min_bin_count;  /* bins with fewer held-out rays are never served */
    uint64_t seed;
    double ref_plane_z;     /* residual reference plane z (m); NaN = box centre */
    int32_t born_segments;  /* 0..64; 0 = no projection (the network alone); -1 = the smallest of
                               1, 2, 4, ..., 32 whose projection alone keeps the pilot rays' RMS
                               sensor error within 0.8 * budget_margin * err_budget_px */
    int32_t use_network;    /* -1 (default) = automatic: the network is trained only if the projection
                               alone, served within the budget, would leave more than 1 % of the plain
                               path's integration steps to the fallback; then each bin is served by the
                               projection alone, the projection with the network's correction or the plain
                               path, whichever costs least under the budget.  1 = the network's
                               correction in every served bin; 0 = the projection alone */
    int32_t table_columns_per_cell;  /* projection-table columns per grid spacing across the box, 1..8, at
                                        most 2048 per axis; 0 = the densest of 4, 2, 1 whose table fits
                                        in 16 GiB */
    int32_t table_levels_per_cell;   /* table levels per grid spacing in depth, 1..4 (1); at most 1024 */
} pivbos_surrogate_cfg;

typedef struct {
    double train_loss;                 /* MSE of the last batch (scaled targets) */
    double train_steps;
    double val_rms_px;                 /* held-out RMS sensor error of the served predictor on every ray
                                          in the box (rays whose status matches the plain path's) */
    double val_rms_px_born;            /* the same for the projection alone */
    double val_rms_px_straight;        /* the same for the straight ray (no field) */
    double val_rms_px_served;          /* estimated RMS over all reaching rays with the chosen bins */
    double val_served_frac;            /* held-out box rays in served bins */
    double val_served_frac_born;       /* the same if the projection alone were served */
    double val_served_frac_straight;   /* the same if the straight ray were served */
    double steps_saved_frac;           /* plain-path steps of served rays / all steps */
    double steps_saved_frac_born;
    double steps_saved_frac_straight;
    double val_status_flip_frac;       /* box rays the predictor sends elsewhere (a stop, off the sensor) */
    double n_val_reached, n_val_box;   /* held-out rays reaching the sensor; those entering the box */
    double seconds_table, seconds_data, seconds_train, seconds_validate;
    double table_bytes;
    double born_segments;              /* segment count used */
    double table_columns_per_cell;     /* table columns per grid spacing used */
    double pilot_rms_px_born_k[6];     /* pilot RMS sensor error of the projection with 1, 2, 4, ..., 32 segments */
    double target_rms[4];              /* RMS residuals: x, y (m) on the reference plane, slope x, y */
    double correction_rms[4];          /* RMS of residual minus projection */
    double sensor_px_per_unit[4];      /* RMS sensor shift per unit of each residual (loss weights) */
    double network_trained;            /* 1 if the network was trained (use_network 1, or -1 when needed) */
    double val_served_frac_net;        /* held-out box rays served with the network's correction */
} pivbos_surrogate_report;

typedef struct pivbos_surrogate pivbos_surrogate;

pivbos_status pivbos_surrogate_default_cfg(pivbos_surrogate_cfg* cfg);
/* Train on `frame` (device buffers; its image and stats are not touched).
 * Synchronous on `stream`.  Errors: INVALID_ARG (arguments, configuration),
 * UNSUPPORTED (no medium, lens not after the box), OOM, CUDA. */
pivbos_status pivbos_surrogate_train(const pivbos_frame_desc* frame, int integrator,
                                     const pivbos_surrogate_cfg* cfg /* NULL = defaults */,
                                     pivbos_surrogate** out, pivbos_surrogate_report* report, void* stream);
/* Render `frame` (same medium and optics, any sources): each ray of a
 * served bin takes its bin's predictor (the projection, or the projection
 * with the network's correction), the rest the plain path; accumulates into
 * the frame's image and stats as pivbos_render does.  When no bin takes the
 * network the served rays are rendered in one pass with no intermediate
 * list; PIVBOS_SURR_DIRECT=0 in the environment (read per call) selects the
 * list-based kernels instead, with the same image bit for bit.  n_fallback
 * (may be NULL; if given, the call synchronises) receives the number of
 * plain-traced rays. */
pivbos_status pivbos_surrogate_render(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                      int64_t* n_fallback, void* stream);
/* The surrogate render of sources [first_source, first_source + n_sources)
 * of a larger source set (the frame's `sources` point at that range; ray k
 * of local source s draws its lens point with counter (k, first_source + s,
 * frame, 0)), for sharding one image across GPUs: renders of disjoint
 * ranges through the same trained surrogate add up, bit for bit, to the
 * render of the whole set.  first_source + n_sources <= 2^32. */
pivbos_status pivbos_surrogate_render_range(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                            int64_t first_source, int64_t* n_fallback, void* stream);
/* Per-ray sensor positions of the surrogate path for flat ray ids (device
 * int64 [n], source-major as in pivbos_trace_exit_states): sensor_xy
 * (device double [n][2]), flags (device int32 [n]: 0 the projection with the
 * network's correction, 3 the projection alone, 1 plain fallback, 2 never
 * enters the box) and status (device int32 [n]).  Synchronous. */
pivbos_status pivbos_surrogate_sensor(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                      const int64_t* ray_ids, int64_t n, double* sensor_xy, int32_t* flags,
                                      int32_t* status, void* stream);
pivbos_status pivbos_surrogate_report_get(const pivbos_surrogate* sg, pivbos_surrogate_report* out);
void pivbos_surrogate_destroy(pivbos_surrogate* sg);

/* ---------------------------------------------------------------------------
 * The simulated BOS experiment of Sec. 4.
 *
 * pivbos_bos_displacements: every ray of every dot (ray k of dot d draws its
 * lens point exactly as in pivbos_render: counter (k, d, frame, 0)) is traced
 * through the medium m and, with the same lens point, through the uniform
 * medium.  Over the rays that reach the sensor both times, per dot:
 * centroid (device double [n_dots][2]) = mean sensor position without the
 * medium, pixels; displacement (device double [n_dots][2]) = mean of (with -
 * without), pixels (Sec. 4: "the ray displacements corresponding to a single
 * dot are averaged"); n_pairs (device int32 [n_dots]) = the number of such
 * rays.  Dots without a pair get NaN.  Each of the three outputs may be
 * NULL.  The sums are taken in fixed point (2^-24 px, rounding error below
 * 3e-8 px in every mean), so results are bit-identical run to run.
 * dots: device [n_dots][3] float64.  Limits: rays_per_dot <= 2^22; sensor
 * at most 65536 pixels per side (else UNSUPPORTED); otherwise as
 * pivbos_render (m must not be NULL).  Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
pivbos_status pivbos_bos_displacements(const pivbos_medium* m, const pivbos_optics* o, const double* dots,
                                       int64_t n_dots, int32_t rays_per_dot, uint64_t seed, uint32_t frame,
                                       int integrator, double step, double* centroid, double* displacement,
                                       int32_t* n_pairs, void* stream);

/* The same for dots [first_dot, first_dot + n_dots) of a larger dot set:
 * `dots` points at that range and ray k of local dot d draws its lens point
 * with counter (k, first_dot + d, frame, 0), so ranges computed separately
 * (on one GPU or several) give, dot for dot and bit for bit, the results of
 * the whole set.  first_dot + n_dots <= 2^32. */
pivbos_status pivbos_bos_displacements_range(const pivbos_medium* m, const pivbos_optics* o, const double* dots,
                                             int64_t n_dots, int64_t first_dot, int32_t rays_per_dot, uint64_t seed,
                                             uint32_t frame, int integrator, double step, double* centroid,
                                             double* displacement, int32_t* n_pairs, void* stream);

/* Eq. 9 per dot, in pixels of the sensor frame:
 *     displacement = (M Z_D / n0) * integral of (dn/dx, dn/dy) dz / pitch,
 * with M, n0 (= n_object) and the pitch given to pivbos_optics_create, Z_D
 * from the dot to the mid-plane of the box, and the integral taken along the
 * dot's chief ray (the line to the centre of the aim disk at z = aim_z),
 * over its part inside the box, of the trilinearly sampled gradient the
 * tracer uses (exactly: piece by piece between node-plane crossings).  The
 * lens inverts the real image, so a ray bent toward +y moves the dot's
 * image toward +y in the (unflipped) sensor frame.  dots, displacement:
 * device [n_dots][3] and [n_dots][2] float64.  Asynchronous on `stream`. */
pivbos_status pivbos_bos_theory(const pivbos_medium* m, const pivbos_optics* o, const double* dots, int64_t n_dots,
                                double* displacement, void* stream);

/* Sec. 4: scattered values (per-dot displacements at their centroids) onto
 * a regular grid by bilinear interpolation.  Node (i, j) sits at
 * (x0 + i cell, y0 + j cell), i < grid_w, j < grid_h (both >= 2).  A point
 * (xy [n][2]) inside the grid gives the four nodes of its cell its value
 * (values [n][2]) with the bilinear weights; out[j][i] (device double
 * [grid_h][grid_w][2]) is the weighted mean at the node, NaN where the
 * summed weight is 0 or below min_weight; weight (device double
 * [grid_h][grid_w], may be NULL) receives the summed weight.  Points with a
 * non-finite coordinate or value, or outside the grid, are skipped.  Sums
 * are fixed point (weights 2^-40, weighted values 2^-32 px): bit-identical
 * run to run; the mean at a node that n points reach carries an absolute
 * error below n 2^-32 (1 + |mean|) / weight.  |value| must be below 256 px
 * per component (a larger one is skipped and the device status word reads
 * PIVBOS_ERR_OVERFLOW at the next pivbos_sync).  n <= 2^23.  Asynchronous. */
pivbos_status pivbos_regrid_bilinear(const double* xy, const double* values, int64_t n, int grid_w, int grid_h,
                                     double x0, double y0, double cell, double min_weight, double* out,
                                     double* weight, void* stream);

/* ---------------------------------------------------------------------------
 * Image pairs for displacement analysis and 16-bit images.
 *
 * pivbos_advect_sources: the particles of the second frame of a pair, the
 * first frame's sources (device double [n][3]) moved over dt by a velocity
 * field (device float [nz][ny][nx][3], m/s, nodes at origin + (i, j, k) *
 * spacing like a medium's; sampled trilinearly, the point clamped into the
 * grid) with the explicit midpoint rule: k = u(x), x' = x + dt u(x + dt k/2).
 * out: device double [n][3] (may not alias sources).  FP64.  Asynchronous.
 *
 * pivbos_image_u16: the 16 bits a camera writes (Sec. 3.4: about 1e4 rays per
 * particle give a 16-bit dynamic range): one count is d = llround(full_scale
 * 2^32 / 65535) units of the 32.32 image (full_scale rays read 65535);
 * counts = (image + floor(d/2)) / d in integers (rounded half up), clipped
 * to [0, 65535].  full_scale <= 2^14 * 65535 rays.  image (device int64) and
 * out (device uint16) 16-byte aligned.
 * Asynchronous.  Errors (both): INVALID_ARG, CUDA.
 * ------------------------------------------------------------------------- */
pivbos_status pivbos_advect_sources(const double* sources, int64_t n_sources, const float* velocity, int nx, int ny,
                                    int nz, const double origin[3], const double spacing[3], double dt,
                                    double* out, void* stream);
pivbos_status pivbos_image_u16(const int64_t* image, int64_t n_pixels, double full_scale, uint16_t* out,
                               void* stream);

/* Self-test of the failure detection (no counterpart in the paper): a
 * kernel waits, with the bounded wait the tensor-core kernels use, on an
 * mbarrier nothing arrives at; after `polls` polls (1..2^20) it gives up and
 * latches PIVBOS_ERR_DEVICE_TIMEOUT in the device status word, which the next
 * pivbos_sync returns (and clears).  The context stays usable.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
pivbos_status pivbos_selftest_wait_timeout(uint32_t polls, void* stream);

/* int64 32.32 image -> float32 intensity in rays (value * 2^-32).  Device
 * pointers, n_pixels >= 0. */
pivbos_status pivbos_image_finalize(const int64_t* image, int64_t n_pixels, float* out, void* stream);

/* Wait for `stream`, then return (and clear) the device status word of the
 * current device: PIVBOS_OK or the first device-side error latched since the
 * last call. */
pivbos_status pivbos_sync(void* stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char* pivbos_last_error(void);

/* Kernel timing for measurement: when enabled, every kernel the library
 * launches is bracketed by CUDA events on its stream.  pivbos_timing_read
 * waits for the recorded events and returns the summed milliseconds and the
 * launch count of kernels whose name starts with `prefix` since the last
 * reset. */
pivbos_status pivbos_timing_enable(int on);
pivbos_status pivbos_timing_reset(void);
pivbos_status pivbos_timing_read(const char* prefix, double* ms_total, int64_t* launches);

/* Number of kernels this library has launched in the process so far. */
int64_t pivbos_kernel_launches(void);

/* Library version string. */
const char* pivbos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PIVBOS_H */
