/*
 * pv3d.h -- C ABI of the GB300 shadow-sample library for PV shading losses.
 *
 * The method (Robledo, Leloux & Lorenzo, arXiv 1410.5780, Section 2) has four
 * steps: (1) import a 3D scene, (2) define the PV generator -- geometry and
 * electrical layout, (3) evaluate the shadows on the generator for every sun
 * position by drawing the scene from the sun into a depth buffer with an
 * orthographic view limited to the generator and depth-checking every sub-cell
 * point against it, (4) turn the shading into power and energy losses.  The
 * calls below follow those steps: pv3d_scene_load (1), pv3d_generator_define
 * and pv3d_set_poses (2), pv3d_set_sun and pv3d_evaluate / pv3d_submit (3, 4).
 *
 * Conventions
 *   * World frame: metres, x = east, y = north, z = up.
 *   * Every call returns PV3D_OK (0) or a negative PV3D_E_* status; the text of
 *     the last error of a context is available from pv3d_last_error.  The
 *     library never aborts or exits the process.
 *   * Input arrays are host pointers, copied to the device during the call; the
 *     caller may free them on return.  Output arrays of pv3d_result are caller
 *     allocated, host or device memory as its is_device field says.
 *   * A context is bound to one CUDA device and is not thread safe: use one
 *     context per host thread.
 */
#ifndef PV3D_H
#define PV3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PV3D_OK           0
#define PV3D_E_INVALID   -1  /* bad argument: NaN, degenerate geometry, |sun| != 1, bad layout ... */
#define PV3D_E_NOMEM     -2  /* device or host allocation failed */
#define PV3D_E_ADMISSION -3  /* request larger than the context's device-memory budget */
#define PV3D_E_OVERFLOW  -4  /* internal capacity could not be grown far enough */
#define PV3D_E_TIMEOUT   -5  /* a bounded wait ran out (pv3d_poll) */
#define PV3D_E_DEVICE    -6  /* CUDA runtime error */
#define PV3D_E_PENDING   -7  /* pv3d_poll: request not finished yet */
#define PV3D_E_NOTFOUND  -8  /* unknown scene, generator or request id */
#define PV3D_E_TOOBIG    -9  /* pv3d_module_shade_noalloc: map_res above PV3D_NOALLOC_MAX_RES */

/* ---- depth formats ------------------------------------------------------ */
#define PV3D_DEPTH_F32    0  /* FP32 depth, stored as order-preserving uint32 */
#define PV3D_DEPTH_U24    1  /* 24-bit unsigned fixed point over the window's depth range */

/* ---- evaluation paths ---------------------------------------------------
 * FUSED: each raster tile is built in shared memory and the samples that read
 *        it are depth-tested by the same CTA; no shadow map reaches HBM.
 * MAP:   raster tiles are stored to a shadow map in device memory and a second
 *        kernel gathers one texel per sample.  Same results, bit for bit. */
#define PV3D_PATH_FUSED   0
#define PV3D_PATH_MAP     1

/* ---- light windows (pv3d_eval_opts.window_groups) -------------------------
 * Section 2, step 3 limits the sun's field of view to the PV generator of
 * interest.  ONE: one window per sun step around all modules of the
 * generator.  The other modes give each group of modules its own window per
 * step (finer texels at the same map_res): the modules of one tracker, of one
 * series string (string_id) or of one inverter input (array_id); fixed
 * modules under PER_TRACKER form one group.  A group's modules must be
 * consecutive in module order (else PV3D_E_INVALID).  Every module of the
 * generator, in or out of the group, shades the group's samples.  map_res is
 * the side of each group's window; the steps per wave shrink so that a wave
 * holds at most 2^26 (group, step, tile) entries.  pv3d_evaluate only; string,
 * array and heat-map outputs are rejected with groups. */
#define PV3D_WINDOWS_ONE          0
#define PV3D_WINDOWS_PER_TRACKER  1
#define PV3D_WINDOWS_PER_STRING   2
#define PV3D_WINDOWS_PER_ARRAY    3

typedef struct pv3d_ctx pv3d_ctx;

/* Context options.  Zero fields take the defaults in brackets. */
typedef struct pv3d_opts {
    int32_t device;           /* CUDA device ordinal [0] */
    int32_t map_res;          /* default shadow-map side R, power of two, 64..16384 [4096] */
    int32_t tile;             /* rasteriser tile side: 32, 64 or 128 texels [64] */
    int32_t chunk_steps;      /* sun steps processed per wave, 1..256 [128] */
    int32_t depth_format;     /* PV3D_DEPTH_F32 or PV3D_DEPTH_U24 [F32] */
    int32_t max_inflight;     /* served requests resident on the device at once, 1..256 [64] */
    int64_t hbm_budget_bytes; /* device memory the context may use [90% of free memory] */
    int32_t wave_scratch_mb;  /* served waves: per-wave scratch target, MiB; requests take fewer steps per
                                 wave to stay under it [2048] */
    int32_t reserved0;
    int64_t bin_capacity;     /* initial (triangle, tile) pool entries; grown on overflow [4 Mi] */
    int32_t reserved[4];
} pv3d_opts;

/*
 * One PV module (Section 2, step 2): a planar grid of cells_u x cells_v square
 * cells of side `pitch`.  Cell (cu, cv) covers origin + a*u + b*v for
 * a in [cu, cu+1]*pitch, b in [cv, cv+1]*pitch; the front face is the side of
 * u x v.  For a tracked module (tracker >= 0) origin, u and v are given in the
 * tracker's rest frame relative to its pivot (rest = table horizontal, front
 * face up); otherwise in the world frame.  u and v must be unit, orthogonal.
 */
typedef struct pv3d_module {
    float origin[3];
    float u[3];
    float v[3];
    float pitch;        /* m */
    int32_t cells_u;    /* 1..64 */
    int32_t cells_v;    /* 1..64; cells_u * cells_v <= 1024 */
    int32_t layout;     /* index into the layouts of pv3d_generator_define */
    int32_t tracker;    /* index into the trackers, or -1 for a fixed module */
    int32_t string_id;  /* series string the module belongs to (string outputs of pv3d_evaluate) */
    int32_t array_id;   /* inverter input: strings whose modules share it are in parallel (array outputs);
                           all modules of a string carry the same array_id */
} pv3d_module;

/*
 * Bypass-diode layout (Section 2, step 2: cells in series, each cell related to
 * one by-pass diode).  cell_sub[cv * cells_u + cu] = substring index in
 * [0, n_sub); every substring must own at least one cell.  n_sub <= 64.
 */
typedef struct pv3d_layout {
    int32_t cells_u;
    int32_t cells_v;
    int32_t n_sub;
    int32_t reserved;
    const int32_t* cell_sub;  /* host pointer, cells_u * cells_v entries */
} pv3d_layout;

/* A two-axis tracker (Section 3.4): modules rotate rigidly about `pivot`. */
typedef struct pv3d_tracker {
    float pivot[3];
} pv3d_tracker;

/* Per-evaluation options.  Zero fields take the defaults in brackets. */
typedef struct pv3d_eval_opts {
    int32_t samples_per_side;  /* n: n x n sub-cell samples per cell, 1..15 [3] */
    int32_t map_res;           /* shadow-map side R [context default] */
    int64_t step_begin;        /* first sun step evaluated [0] */
    int64_t step_end;          /* one past the last step; 0 = all steps [0] */
    float i_ref;               /* cell current at 1000 W/m^2, A [9.0] */
    float v_cell;              /* cell voltage at the operating point, V [0.5] */
    float v_diode;             /* bypass-diode forward drop, V [0.5] */
    int32_t chunk_steps;       /* steps per wave [context default] */
    void* stream;              /* cudaStream_t to run on; NULL = the context's own stream */
    int32_t path;              /* PV3D_PATH_FUSED or PV3D_PATH_MAP [FUSED] */
    int32_t profile;           /* bit 0: time each stage with CUDA events; bit 1: count work (pv3d_last_profile) [0] */
    int32_t diffuse_shading;   /* 1: shade the diffuse term of each cell by its pv3d_sky_view fraction [0] */
    int32_t window_groups;     /* PV3D_WINDOWS_*: one light window, or one per tracker, string or array [ONE] */
    int32_t reserved[4];
} pv3d_eval_opts;

/*
 * Stage timings (profile bit 0) and work counts (profile bit 1) of the last
 * pv3d_evaluate run with opts->profile set.  Stages: 0 light window and module setup, 1 binning
 * (triangle bins, scan, receiver lists), 2 tiles (fused path: the depth tests
 * of the tiles taken one per warp; map path: tile rasterisation into the map),
 * 3 the tiles with many receivers or triangles (fused path, one per block,
 * rasterised in shared memory when they keep many triangles), 4 PV model
 * (with the texel gathers on the map path), 5 Kahan energy sums.  stage_ms
 * sums CUDA-event intervals over the waves, recorded on the evaluation's stream.
 */
typedef struct pv3d_profile {
    int32_t n_stages;
    int32_t waves;
    float stage_ms[8];
    float device_ms;
    int32_t reserved0;
    int64_t sample_tests;      /* sample depth tests performed against rasterised tiles */
    int64_t texel_visits;      /* texel-centre coverage tests */
    int64_t texel_writes;      /* fragments: (texel read by a sample, triangle covering its centre) pairs
                                  (rasterised dense tiles: every covered texel) */
    int64_t tris_culled;       /* (triangle, tile) pairs skipped: on or behind every receiver plane */
    int64_t nonempty_tiles;
    int64_t binned_tris;
    int64_t candidates;        /* receiver samples enumerated by the tile kernel (marking and testing) */
    int64_t dense_tiles;       /* tiles rasterised at every texel */
    int64_t sample_tiles;      /* tiles tested sample by sample against their few triangles (not rasterised) */
    int64_t pair_tests;        /* (sample, triangle) coverage tests made by the sample-driven test */
    int64_t heavy_tiles;       /* tiles with many receivers or triangles, taken one per block (stage 3) */
    int64_t heavy_sample_tests;   /* their share of sample_tests */
    int64_t heavy_texel_writes;   /* their share of texel_writes */
    int64_t heavy_why[3];      /* heavy tiles by cause: too many receivers, binned triangles, kept triangles */
} pv3d_profile;

/*
 * Results.  M = modules of the generator, C = their cells (module order, then
 * cv * cells_u + cu), S = step_end - step_begin.  Every array pointer may be
 * NULL when not wanted.  Energies are the FP32 Kahan-compensated sums of the
 * per-step values, returned as double.
 */
typedef struct pv3d_result {
    int32_t is_device;         /* 1: the arrays below are device pointers; 0: host */
    int32_t reserved0;
    double* energy;            /* [M] sum over steps of P_mpp * dt, Wh */
    double* energy_unshaded;   /* [M] same without shading, Wh */
    float* power;              /* [S x M] P_mpp per step, W */
    float* power_unshaded;     /* [S x M] */
    double* cell_beam_loss;    /* [C] sum over steps of DNI * max(0, cos i) * f_c * dt, Wh/m^2 */
    uint8_t* cell_counts;      /* [S x C] shaded samples per cell */
    uint64_t* sample_bits;     /* [S x C] bit k = j*n + i set if sample (i, j) is shaded; n <= 8 */
    /* filled by the library */
    int64_t tests;             /* sample depth tests performed (lit steps x samples per step) */
    int64_t steps_lit;         /* steps whose sun is above the horizon */
    float device_ms;           /* device time of the evaluation (CUDA events) */
    int32_t waves;             /* waves launched */
    int64_t nonempty_tiles;    /* rasterised (step, tile) pairs over the evaluation */
    int64_t binned_tris;       /* (triangle, tile) pairs binned over the evaluation */
    int64_t kernel_launches;   /* CUDA kernels launched by the evaluation */
    float latency_ms;          /* served requests: submit to results ready (host clock) */
    int32_t reserved1;
    /* series strings (pv3d_evaluate only): NS = pv3d_generator_strings' count,
     * strings in ascending string_id order.  One current flows through every
     * bypass substring of every module of a string, and the string runs at
     * its own maximum power point (Section 2: modules wired in series strings,
     * Fig. 2; the module outputs above keep one maximum power point per module). */
    double* string_energy;           /* [NS] sum over steps of the string's P_mpp * dt, Wh */
    double* string_energy_unshaded;  /* [NS] */
    float* string_power;             /* [S x NS] string P_mpp per step, W */
    float* string_power_unshaded;    /* [S x NS] */
    /* effective-shading map over the sky (pv3d_evaluate only; Section 3, Fig. 6:
     * the shading factor as a function of the sun's position): the evaluated
     * steps with the sun above the horizon, binned by compass azimuth
     * (heat_az_bins bins over [0, 360), clockwise from north) and zenith angle
     * (heat_zen_bins bins over [0, 90]); per bin, row-major [zen][az], the
     * generator's energy (sum over modules and the bin's steps of P_mpp * dt)
     * with and without shading, and the step count, summed in FP64 in step
     * order.  The bin's effective shading factor is
     * 1 - heat_energy / heat_energy_unshaded.  Set both bin counts (1..1024
     * each) and the three arrays, or leave them 0 / NULL. */
    int32_t heat_az_bins;
    int32_t heat_zen_bins;
    double* heat_energy;             /* [heat_zen_bins x heat_az_bins] Wh */
    double* heat_energy_unshaded;    /* [heat_zen_bins x heat_az_bins] Wh */
    int32_t* heat_steps;             /* [heat_zen_bins x heat_az_bins] */
    /* strings in parallel (pv3d_evaluate only): NA = pv3d_generator_arrays'
     * count, arrays in ascending array_id order.  One voltage is across every
     * string of an array and the array runs at its own maximum power point;
     * string s delivers the largest current at which its voltage still
     * reaches the array's (at most 512 bypass substrings per array). */
    double* array_energy;            /* [NA] sum over steps of the array's P_mpp * dt, Wh */
    double* array_energy_unshaded;   /* [NA] */
    float* array_power;              /* [S x NA] */
    float* array_power_unshaded;     /* [S x NA] */
} pv3d_result;

/* ---- context ------------------------------------------------------------ */

/* Create a context on opts->device (opts may be NULL). */
int pv3d_create(pv3d_ctx** out, const pv3d_opts* opts);

/* Release every device resource of the context.  NULL is accepted. */
void pv3d_destroy(pv3d_ctx* ctx);

/* Text of the last error reported by a call on `ctx` ("" if none). */
const char* pv3d_last_error(pv3d_ctx* ctx);

/* ---- step 1: scene (Section 2, step 1) ---------------------------------- */

/*
 * Load a triangle soup: xyz[3 * n_verts] floats, tri_idx[3 * n_tris] vertex
 * indices.  Triangles are two-sided.  Copied to the device; stays resident
 * until pv3d_release.  Errors: PV3D_E_INVALID for a non-finite coordinate or an
 * index out of range; n_tris may be 0.
 */
int pv3d_scene_load(pv3d_ctx* ctx, const float* xyz, int64_t n_verts,
                    const int32_t* tri_idx, int64_t n_tris, uint32_t* scene_id);

/* ---- step 2: generator (Section 2, step 2) ------------------------------ */

/*
 * Define a PV generator over a loaded scene.  The generator's modules are
 * occluders too (row-to-row and tracker-to-tracker shading), except a module
 * never shades itself.  One generator = one light window per sun step, the
 * bounding square of its modules as seen from the sun (Section 2, step 3).
 */
int pv3d_generator_define(pv3d_ctx* ctx, uint32_t scene_id,
                          const pv3d_module* mods, int32_t n_mods,
                          const pv3d_layout* layouts, int32_t n_layouts,
                          const pv3d_tracker* trackers, int32_t n_trackers,
                          uint32_t* gen_id);

/*
 * Clear-sky sun table computed on the device (the inputs of steps 3-4: the
 * paper takes TMY data, measured series or a clear-sky model it does not
 * name).  Solar time without longitude correction or equation of time;
 * declination of Cooper (1969), 23.45 deg * sin(360 deg * (284 + n) / 365) on
 * day n; hour angle 15 deg per hour from solar noon; unit vector toward the
 * sun in east-north-up axes; beam irradiance of Meinel & Meinel (1976),
 * DNI = 1353 * 0.7^(AM^0.678) W/m^2, with the air mass of Kasten & Young
 * (1989); DHI = dhi_fraction * DNI; step duration step_h hours.  All in FP64
 * on the device.  Replaces the generator's sun table like pv3d_set_sun; with
 * tracker_tilt_max_deg > 0 and trackers present, also sets every tracker to
 * the ideal two-axis pose of each step (compass azimuth of the sun, tilt =
 * zenith angle clamped to the maximum) like pv3d_set_poses.  *n_steps
 * (may be NULL) receives the table's length.  Errors: PV3D_E_INVALID (options
 * out of range, or daylight_only with no daylight step), PV3D_E_NOTFOUND,
 * PV3D_E_NOMEM, PV3D_E_DEVICE.
 */
typedef struct pv3d_sky_opts {
    double latitude_deg;         /* site latitude, degrees north, -89.9 .. 89.9 */
    double step_h;               /* hours between steps, (0, 24]; steps at solar hours 0, step_h, ... < 24 */
    int32_t day_first;           /* first day of the year, 1..366 */
    int32_t n_days;              /* days, 1..3660 */
    int32_t daylight_only;       /* 1: keep only the steps with the sun above the horizon */
    float dhi_fraction;          /* DHI / DNI [0.1] */
    float tracker_tilt_max_deg;  /* > 0: also set ideal tracker poses with this tilt limit [0: poses untouched] */
    int32_t reserved[5];
} pv3d_sky_opts;

int pv3d_set_sun_clear_sky(pv3d_ctx* ctx, uint32_t gen_id, const pv3d_sky_opts* opts, int64_t* n_steps);

/*
 * Copy the generator's sun table (set by pv3d_set_sun or
 * pv3d_set_sun_clear_sky) to host arrays of n_steps entries (its length):
 * sun_xyz[n_steps][3], dni, dhi, dt_h (any may be NULL).  Errors:
 * PV3D_E_INVALID (n_steps differs from the table's length), PV3D_E_NOTFOUND.
 */
int pv3d_sun_table(pv3d_ctx* ctx, uint32_t gen_id, double* sun_xyz, float* dni, float* dhi, float* dt_h,
                   int64_t n_steps);

/*
 * Diffuse shading (the paper leaves the isotropic diffuse term unshaded):
 * the share of each cell's cosine-weighted sky hidden by the scene.  The upper
 * hemisphere is cut into `rings` zenith bands of equal angle and `sectors`
 * azimuth sectors; every patch is represented by its centre direction, which
 * is evaluated like a sun step (depth map from that direction, the cell's n x n
 * samples tested), and weighted by its solid angle times the cosine to the
 * module's front normal.  A cell's fraction is sum_p W_p s_p / sum_p W_p (s_p
 * = its shaded samples toward patch p over n^2); 0 without obstructions.  The
 * fractions are kept with the generator and used by evaluations with
 * diffuse_shading = 1: G_c = DNI max(0, cos i)(1 - f_c) + DHI (1 + cos beta)/2
 * (1 - f_diffuse,c), cos beta the module's tilt at the step.
 *
 * Tracked generators (Section 3.4): a tracker's view of the sky changes with
 * its pose, so the fractions are taken per pose bin.  A step's pose bin is
 * that of the first tracker's pose (the plant tracks in unison): compass
 * azimuth in pose_az_bins equal sectors of [0, 360) deg, tilt in
 * pose_tilt_bins equal bands of [0, 90] deg, bin = tilt band * pose_az_bins +
 * azimuth sector.  For every bin that a lit step falls in, every tracker is
 * set to the bin's centre pose (the middle of both ranges) and the fractions
 * are taken as above with the modules' normals at that pose; a step then uses
 * the row of its bin.  The sun table and poses must be set first; a new sun
 * table or pose table drops the fractions (evaluate with diffuse_shading again
 * needs pv3d_sky_view).
 *
 * cell_fraction (host, may be NULL) receives bins x C floats, row-major by
 * bin (bins = 1 for a generator of fixed modules; rows of bins that no lit
 * step uses are 0).  Errors: PV3D_E_INVALID (options out of range, tracked
 * generator without poses), PV3D_E_NOTFOUND, PV3D_E_NOMEM, PV3D_E_DEVICE.
 */
typedef struct pv3d_sky_view_opts {
    int32_t rings;             /* zenith bands over [0, 90] deg, 1..90 [9] */
    int32_t sectors;           /* azimuth sectors, 1..360 [36] */
    int32_t samples_per_side;  /* n, 1..15 [3] */
    int32_t map_res;           /* shadow-map side [context default] */
    int32_t pose_az_bins;      /* tracked generators: azimuth sectors of the pose bins, 1..360 [12] */
    int32_t pose_tilt_bins;    /* tracked generators: tilt bands of the pose bins, 1..90 [6] */
    int32_t reserved[2];
} pv3d_sky_view_opts;

int pv3d_sky_view(pv3d_ctx* ctx, uint32_t gen_id, const pv3d_sky_view_opts* opts, float* cell_fraction);

/*
 * Series strings of a generator (Section 2: the modules are wired in series
 * strings, Fig. 2): modules with equal pv3d_module.string_id form one string.
 * *n_strings receives their number; string_ids (NULL, or room for
 * *n_strings entries) the distinct ids in ascending order, which is the order
 * of the string outputs of pv3d_result.  Errors: PV3D_E_NOTFOUND (unknown
 * generator), PV3D_E_INVALID (null context or count pointer).
 */
int pv3d_generator_strings(pv3d_ctx* ctx, uint32_t gen_id, int32_t* n_strings, int32_t* string_ids);

/* Arrays of a generator (strings in parallel at one inverter input): the number
 * and the distinct array_id values in ascending order, the order of the array
 * outputs of pv3d_result.  Errors as pv3d_generator_strings. */
int pv3d_generator_arrays(pv3d_ctx* ctx, uint32_t gen_id, int32_t* n_arrays, int32_t* array_ids);

/*
 * Tracker poses: az_tilt[(step * n_trackers + t) * 2 + {0, 1}] = compass
 * azimuth the table faces (radians from north, clockwise) and its tilt from
 * horizontal (radians).  A point x of the rest frame moves to
 * pivot + Rz(pi - az) * Rx(tilt) * x, so the front normal becomes
 * (sin tilt sin az, sin tilt cos az, cos tilt).  n_steps must equal the sun
 * table's length (either may be set first).
 */
int pv3d_set_poses(pv3d_ctx* ctx, uint32_t gen_id, const float* az_tilt, int64_t n_steps);

/* ---- step 3/4 inputs: sun and irradiance (Section 2, steps 3 and 4) ----- */

/*
 * Sun table: sun_xyz[3 * step] unit vector toward the sun (|s| = 1 +- 1e-6),
 * DNI and DHI in W/m^2, dt_h = duration represented by the step, hours.
 * Steps with s.z <= 0 receive no direct light and are skipped.
 */
int pv3d_set_sun(pv3d_ctx* ctx, uint32_t gen_id, const double* sun_xyz, const float* dni,
                 const float* dhi, const float* dt_h, int64_t n_steps);

/* ---- steps 3 and 4: evaluation -------------------------------------------
 *
 * For each lit sun step: depth-rasterise the scene and the generator's modules
 * from the sun into an R x R map over the generator's window, test each of the
 * n x n samples of every cell against the map (shaded iff its depth exceeds the
 * stored depth plus a slope-scaled bias), reduce to cell, substring and module
 * shaded fractions, and apply the bypass-diode model:
 *   G_c = DNI max(0, cos i)(1 - f_c) + DHI (1 + cos beta) / 2,   I_c = i_ref G_c / 1000,
 *   I_k = min_{c in k} I_c,  P(I) = I (sum_{I_k >= I} n_k v_cell - v_diode #{I_k < I}),
 *   P_mpp = max(0, max_k P(I_k)).
 * Energies are integrated over the steps (Section 2, step 4).
 */

/* Synchronous evaluation; returns when the results are in `out`. */
int pv3d_evaluate(pv3d_ctx* ctx, uint32_t gen_id, const pv3d_eval_opts* opts, pv3d_result* out);

/*
 * Served evaluation: enqueue the request and return at once with *req.  The
 * context keeps scenes resident and runs a worker thread: it admits queued
 * requests in arrival order while fewer than max_inflight are active and their
 * device-memory footprint (accumulators, host-output staging and their share of
 * the wave scratch) fits the budget, and every wave takes the next chunk of sun
 * steps of every active request (continuous batching: a request that arrives
 * while others run joins the next wave).  Results are bit-identical to
 * pv3d_evaluate of the same request.  PV3D_E_ADMISSION if the request alone
 * exceeds the budget.  The scene, generator and `out` must stay valid until
 * the request completes; pv3d_release refuses ids that queued or active
 * requests use.  Served requests use the fused path; they take every output
 * and option of pv3d_evaluate (series-string and array outputs, the diffuse
 * term) except sky-map outputs and window groups (PV3D_E_INVALID).
 */
int pv3d_submit(pv3d_ctx* ctx, uint32_t gen_id, const pv3d_eval_opts* opts, pv3d_result* out,
                uint64_t* req);

/*
 * Advance the served work and wait up to timeout_ms (0 = do not wait) for
 * request `req`: PV3D_OK when its results are in its pv3d_result,
 * PV3D_E_PENDING if still running, another status on failure.
 */
int pv3d_poll(pv3d_ctx* ctx, uint64_t req, int32_t timeout_ms);

/*
 * Evaluate n generators together: every request is submitted to the served
 * engine (its sun steps batched with the others' into shared waves) and the
 * call returns when all are done.  Returns the first failing status, or
 * PV3D_OK.  opts may be NULL (defaults for all).
 */
int pv3d_evaluate_batch(pv3d_ctx* ctx, int32_t n, const uint32_t* gen_ids, const pv3d_eval_opts* opts,
                        pv3d_result* outs);

/* Profile of the last profiled evaluation on `ctx` (PV3D_E_NOTFOUND if none). */
int pv3d_last_profile(pv3d_ctx* ctx, pv3d_profile* out);

/* Free a scene (and every generator defined on it) or a generator. */
int pv3d_release(pv3d_ctx* ctx, uint32_t scene_or_gen_id);

/* ---- measured raster roofline ------------------------------------------------
 *
 * The rasterising kernels draw a tile's depth in shared memory with atomicMin
 * of 32-bit order-preserving keys (Fig. 3: the depth buffer keeps the surface
 * nearest the sun).  Their roofline is this operation's throughput on the
 * device, measured here: 16 blocks of 128 threads per SM, each block a 32 x 32
 * shared tile of keys, warps updating strips of 32 consecutive texels (the
 * rasteriser's access pattern), best of 5 timed launches of 2^14 updates per
 * thread after a warm-up launch (CUDA events on a private stream).
 *   device         CUDA device ordinal; the caller's current device is restored
 *   atomics_per_s  out: shared-memory atomicMin updates per second, whole GPU
 *   best_ms        out (may be NULL): the best launch's duration
 * Allocates 4 bytes of device memory for the fold of the tiles and frees it.
 * Returns PV3D_OK, PV3D_E_INVALID (NULL output) or PV3D_E_DEVICE. */
int pv3d_raster_peak(int32_t device, double* atomics_per_s, double* best_ms);

/* ---- evaluation without device allocation --------------------------------
 *
 * The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory while they run -- a host loop that hands every byte
 * of the GPU to its own pool, a latency-critical loop that cannot take the
 * implicit synchronisation of cudaMalloc/cudaFree, or code recording into a
 * stream capture, where those calls are not permitted.  It needs no context.
 *
 * Shaded-sample counts of ONE fixed module for ONE sun direction: the
 * triangles are depth-rasterised from the sun into a map of map_res^2 texels
 * over the module's window and every one of the module's n x n samples per
 * cell is depth-tested against it.  The rules follow pv3d_evaluate's (light
 * frame, window of one texel padding, texel-centre coverage, slope-scaled
 * bias), but the frame is built in FP64 on the host for every elevation, the
 * coordinates are taken relative to the module's centre and each triangle is
 * rasterised by one warp: counts can differ from pv3d_evaluate's for samples
 * at texel edges (the tests accept one sample per cell and 0.1 % of all
 * samples), not bit for bit.
 *   tri_xyz       device pointer, 9 floats per triangle (three world vertices, m)
 *   module        host pointer; tracker must be -1; its layout is not used
 *   sun_xyz       host pointer, unit vector toward the sun; s.z <= 0 gives zeros
 *   map_res       power of two, 64..PV3D_NOALLOC_MAX_RES, else PV3D_E_INVALID or
 *                 PV3D_E_TOOBIG (above the maximum)
 *   cell_counts   device pointer, cells_u * cells_v uint32, overwritten with the
 *                 shaded samples per cell (c = cv * cells_u + cu)
 *   stream        cudaStream_t the work is queued on (NULL = legacy stream);
 *                 the call returns without waiting for it
 * The shadow map is one fixed array compiled into the library
 * (PV3D_NOALLOC_MAX_RES^2 x 4 bytes = 16 MiB per GPU, kept until the process
 * exits); the call allocates nothing itself.  With CUDA's lazy module loading
 * (the default) the array is reserved on a device when the library's module
 * is first loaded there, i.e. by the first call on that device: a caller
 * whose own pool takes all device memory should make one call before creating
 * the pool.  Each call looks up the array's device address for the current
 * device and context (after cudaDeviceReset the module loads again at a new
 * address); while `stream` is being captured no lookup is made and the address
 * found by the last uncaptured call on that device is used, so make one call
 * before any stream capture (else PV3D_E_DEVICE).  Launch failures of the
 * call's own kernels return PV3D_E_DEVICE; an earlier error of the caller's
 * is neither reported nor cleared.  All calls share the array: each clears the
 * part it uses, and calls that overlap on the GPU (different streams without
 * ordering) race on it.
 */
#define PV3D_NOALLOC_MAX_RES 2048
int pv3d_module_shade_noalloc(const float* tri_xyz, int64_t n_tris, const pv3d_module* module,
                              const double* sun_xyz, int32_t samples_per_side, int32_t map_res,
                              uint32_t* cell_counts, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PV3D_H */
