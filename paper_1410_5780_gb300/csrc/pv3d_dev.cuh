// pv3d_dev.cuh -- device-side data layout shared by the kernels and the host
// orchestration of the pv3d library (GB300 / sm_103a).
//
// Work is organised in waves.  A wave holds one or more jobs (a job = one
// generator evaluated over a chunk of consecutive sun steps).  Every kernel
// grid-strides over a flattened item space whose size it reads from the
// device-resident WaveDev, so one set of launches (or one captured CUDA graph)
// serves any mix of jobs: the plain per-scene evaluation is a wave with one
// job, batched and served evaluations put many jobs of uneven size in a wave.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pv3d {

constexpr int kMaxCellsPerModule = 1024;
constexpr int kMaxSub = 64;
constexpr int kBigTiles = 4;       // triangles over more tiles are binned by whole warps
constexpr int kWinPerItem = 256;   // modules reduced per window item

// Generator module in device memory (68 bytes).
struct ModuleDev {
    float o[3], u[3], v[3];
    float pitch;
    int32_t cu, cv, layout, tracker;
    int32_t cell_base;  // first cell of the module in the generator's cell numbering
    int32_t n_sub;      // substrings of its layout
    int32_t plane;      // plane group: modules with one id lie in one plane under every pose
};

constexpr uint32_t kPlaneNone = 0xFFFFFFFFu;   // t_plane: no receiver yet
constexpr uint32_t kPlaneMixed = 0xFFFFFFFEu;  // t_plane: receivers of several plane groups

// Light frame of one (job, step): orthographic view from the sun (Section 2,
// step 3).  Light-plane coordinates are taken relative to the job's reference
// point; texel coordinates are (lu - u0) * inv_delta, (lv - v0) * inv_delta.
struct LightParams {
    float ux, uy, uz;
    float vx, vy, vz;
    float sx, sy, sz;   // unit vector toward the sun; depth = -(x - ref) . s
    float u0, v0;
    float inv_delta, delta;
    float dni, dhi, dt;
    float dnear, qscale;  // 24-bit depth: q = (d - dnear) * qscale
    int32_t valid;       // sun above the horizon
    int32_t pad;
};

// One module at one step in texel space (48 bytes): a point a*U + b*V of the
// module (a, b in metres) maps to texel coordinates
// (tx0 + a*tax + b*tbx, ty0 + a*tay + b*tby) and depth d0 + a*da + b*db.
struct ModStep {
    float tx0, ty0, d0;
    float tax, tay, da;
    float tbx, tby, db;
    float cosi;   // cosine of incidence on the front face
    float bias;   // depth bias, metres
    float nz;     // z of the front normal (cos of the tilt)
};

struct JobDev {
    // scene (triangles relative to ref, 3 float4 each)
    const float4* tri;
    int32_t n_tris;
    int32_t n_mtris;  // module triangles rasterised: 2 per module, or 0 for a coplanar generator
    const float4* ml_box;  // scene meshlets (32 consecutive triangles, median-split order): world lo, hi
    int32_t n_ml;          // scene meshlets = ceil(n_tris / 32)
    int32_t pad_ml;
    // generator
    const ModuleDev* mods;
    int32_t n_mods;
    int32_t n_cells;
    const int32_t* cell_mod;  // [C] module of each cell
    const int32_t* lay_sub;   // concatenated cell -> substring maps
    const int32_t* lay_off;   // [layouts] offset into lay_sub
    const int32_t* lay_nk;    // concatenated cells per substring, same offsets as lay_sub's layouts
    const int32_t* lay_nk_off;
    const float* pivots;      // [n_trk][3] relative to ref
    int32_t n_trk;
    float ref[3];
    float scene_lo[3], scene_hi[3];  // relative to ref
    // sun table and poses
    const double* sun;
    const float* dni;
    const float* dhi;
    const float* dt;
    const float* poses;  // [steps][n_trk][2]
    int32_t step0;       // first sun step of this wave
    int32_t k;           // steps of this job in the wave
    int32_t out_row0;    // output row of step0
    // parameters
    int32_t R, tiles_x, n, nn;
    float i_ref, v_cell, v_diode;
    // wave-local bases
    int32_t js_base;  // (step) entries
    int32_t pad0;
    int64_t te_base;  // (step, tile) entries
    int64_t ms_base;  // (step, module) entries
    int64_t cs_base;  // (step, cell) entries
    // flattened item bases of this job, per kernel
    int64_t it_win, it_mod, it_tri, it_epi;
    // accumulators across the waves of one evaluation
    float2* kahan_mod;   // [M][2]  (E, comp), (E_unshaded, comp)
    float2* kahan_cell;  // [C]     (beam loss, comp); nullptr when the per-cell beam loss is not wanted
    // optional outputs, row = out_row0 + local step
    float* out_power;
    float* out_power_u;
    uint8_t* out_counts;
    unsigned long long* out_bits;
    // series strings (string outputs requested; n_str = 0 otherwise).  The
    // generator's bypass substrings are numbered string by string, so string
    // q owns substrings [str_sub[q], str_sub[q + 1]).
    int32_t n_str;
    int32_t n_sub_tot;        // substrings over all modules
    const int32_t* str_sub;   // [n_str + 1]
    const int32_t* sub_base;  // [M] first substring of each module
    const int32_t* sub_nk;    // [n_sub_tot] cells of each substring
    const int32_t* sub_mod;   // [n_sub_tot] module of each substring
    int64_t ss_base;          // (step, substring) entries
    int64_t sq_base;          // (step, string) entries
    int64_t it_str;           // string-kernel items
    float2* kahan_str;        // [n_str][2]  (E, comp), (E_unshaded, comp)
    float* out_str_power;     // [rows][n_str]
    float* out_str_power_u;
    // effective-shading map over the sky (heat_az * heat_zen bins, 0: none):
    // per bin, sums over the evaluation's steps (in step order, FP64)
    int32_t heat_az, heat_zen;
    int64_t it_heat;          // heat-kernel items (bins of the jobs before this one)
    double* heat_e;           // [bins]  sum of the generator's P_mpp * dt
    double* heat_eu;          // [bins]  same without shading
    int32_t* heat_n;          // [bins]  steps
    const float* fdiff;       // [bins][C] diffuse shading fraction per cell (pv3d_sky_view), or nullptr
    const int32_t* fbin;      // [steps] the step's pose bin (tracked generators), or nullptr (one bin)
    int64_t fstride;          // cells of the generator (one bin's row of fdiff)
    // strings in parallel (array outputs requested; n_arr = 0 otherwise):
    // array a holds strings arr_strs[arr_off[a] .. arr_off[a + 1])
    int32_t n_arr;
    int32_t pad_arr;
    const int32_t* arr_off;   // [n_arr + 1]
    const int32_t* arr_strs;  // [n_str]
    int64_t sa_base;          // (step, array) entries
    float2* kahan_arr;        // [n_arr][2]
    float* out_arr_power;     // [rows][n_arr]
    float* out_arr_power_u;
    // row strides of the per-step outputs: out_power rows hold out_mstride
    // modules, out_counts / out_bits rows out_cstride cells (a job over a
    // window group writes its columns of the generator's rows)
    int32_t out_mstride, out_cstride;
    // window groups: every module of the generator (occ_mods, n_occ) shades
    // the group's samples, as meshlets of 16 modules (32 triangles) with
    // world boxes that hold them under any pose (oml_box, n_oml meshlets,
    // tested like scene meshlets); their triangles follow the scene's.  The
    // group's own module triangles (n_mtris) are then 0.
    const ModuleDev* occ_mods;
    const float4* oml_box;    // [n_oml][2] world lo, hi
    int32_t n_occ, n_oml;
};

struct WaveDev {
    int32_t n_jobs;
    int32_t tile_sh;    // log2 of the tile side
    int32_t depth_u24;
    int32_t fused;      // 1: depth tests inside the tile CTA; 0: map in HBM + gather kernel
    int32_t want_bits;  // per-sample flags requested by some job of the wave
    int32_t profile;    // count work (texel visits, sample tests) into Counters
    int64_t tot_js, tot_te, tot_ms, tot_cs;
    int64_t tot_win, tot_mod, tot_tri, tot_epi;  // tot_tri: (group of 32 meshlets, step) warp items
    int64_t tot_ss, tot_sq;                      // (step, substring) and (step, string) entries
    int64_t tot_heat;                            // heat-map bins over the jobs
    int64_t tot_sa;                              // (step, array) entries
    int64_t bin_cap, map_cap_tiles, big_cap, recv_cap;
};

struct Counters {
    unsigned int n_big;
    unsigned int n_nonempty;
    unsigned int raster_next;
    unsigned int overflow;  // bit 0 bins, bit 1 map tiles, bit 2 big list, bit 3 receivers
    unsigned int n_heavy;     // tiles k_tile_warp hands to k_raster_test
    unsigned long long n_pairs;  // (tile, triangle) pairs appended by the binning kernels
    unsigned int heavy_next;  // k_raster_test's work counter
    unsigned long long tot_bins;
    unsigned long long tot_recv;
    unsigned long long need_recv;
    unsigned long long stat_nonempty;
    unsigned long long stat_bins;
    unsigned long long need_bins;    // max over waves of the bins a wave needed
    unsigned long long need_tiles;   // max over waves of the map tiles a wave needed
    unsigned long long need_big;
    // work counters, filled when WaveDev::profile is set
    unsigned long long prof_samples;   // sample depth tests in rasterised tiles
    unsigned long long prof_visits;    // texel coverage tests
    unsigned long long prof_writes;    // covered texels (depth atomicMin)
    unsigned long long prof_culled;    // (triangle, tile) pairs skipped by the receiver-plane test
    unsigned long long prof_cand;      // receiver samples enumerated (marking and testing passes)
    unsigned long long prof_tiles;     // tiles rasterised
    unsigned long long prof_dense;     // of which rasterised densely
    unsigned long long prof_tris;      // (triangle, tile) pairs set up
    unsigned long long prof_stiles;    // tiles tested sample by sample (not rasterised)
    unsigned long long prof_pairs;     // (sample, triangle) coverage tests of the sample-driven test
    unsigned long long prof_h_samples;  // of prof_samples, prof_writes and prof_tiles: the share of the
    unsigned long long prof_h_writes;   //   kernel that takes the heavy tiles (one block per tile)
    unsigned long long prof_h_tiles;
    unsigned long long prof_heavy_why[3];  // heavy because of: receivers, binned triangles, kept triangles
};

// Scratch and pools, sized by the host for the largest wave.
struct Buffers {
    LightParams* lp;         // [tot_js]
    uint32_t* win;           // [tot_js][4]
    ModStep* ms;             // [tot_ms]
    float* ms_p;             // [tot_ms]
    float* ms_pu;            // [tot_ms]
    float* ms_beam;          // [tot_ms]  DNI * max(0, cos i)
    float* ms_iu;            // [tot_ms]  unshaded cell current (string model)
    float* ss_i;             // [tot_ss]  substring current limit per (step, substring) (string model)
    float* sq_p;             // [tot_sq]  string MPP power per (step, string)
    float* sq_pu;            // [tot_sq]  same without shading
    float* sa_p;             // [tot_sa]  array MPP power per (step, array)
    float* sa_pu;            // [tot_sa]
    float* js_p;             // [tot_js]  the generator's P_mpp per step (heat map)
    float* js_pu;            // [tot_js]
    int32_t* js_bin;         // [tot_js]  sky bin of the step's sun, -1 below the horizon
    uint32_t* cs_cnt;        // [(tot_cs + 3) / 4]  shaded samples per (step, cell): one byte each (a count
                             //  is at most n^2 <= 225), four to a word for the tile kernels' atomics
    unsigned long long* cs_bits;  // [tot_cs] shaded flags per (step, cell), fused path with flags requested
    uint32_t* t_far;         // [tot_te]  far-plane key of the tile (0 = no sample)
    uint32_t* t_cnt;         // [tot_te]  triangles binned
    uint32_t* t_off;         // [tot_te]
    uint32_t* t_cur;         // [tot_te]
    uint32_t* t_slot;        // [tot_te]  index among the wave's non-empty tiles (= map slot)
    uint32_t* t_rcnt;        // [tot_te]  receiver modules touching the tile
    uint32_t* t_plane;       // [tot_te]  plane group of every receiver of the tile, or kPlaneMixed
    uint32_t* t_roff;        // [tot_te]
    uint32_t* t_rcur;        // [tot_te]
    uint32_t* nonempty;      // [tot_te]
    uint32_t* heavy;         // [tot_te]  tiles listed for the CTA-per-tile kernel (fused path)
    uint32_t* bins;          // [bin_cap]   triangle ids
    uint2* pairs;            // [bin_cap]   (tile entry, triangle) pairs in binning order
    uint32_t* recv;          // [recv_cap]  receiver module ids
    uint32_t* map;           // [map_cap_tiles << (2 * tile_sh)]  (map path)
    uint2* big;              // [big_cap]  (triangle, js)
    unsigned long long* block_sums;  // scan partials, 3 per scan tile
    Counters* ctr;
};

// ---- host launchers (kernels.cu) ------------------------------------------
struct LaunchCfg {
    int sm_count;
    int tile;     // 32, 64 or 128
    int fused;    // 1: k_raster_test + k_pv; 0: k_raster_map + k_sample
    int profile;  // counting kernels
    cudaStream_t stream;
    cudaEvent_t* ev;  // NULL, or kStages + 1 events recorded at the stage boundaries of the wave
    int extras;       // bit 0: series strings (k_string); bit 1: sky map (k_gen_step, k_heat); bit 2: arrays (k_array)
};

constexpr int kStages = 6;  // setup, bin, tile (warp per tile / map raster), heavy tiles, pv/sample, epilogue
constexpr int kLaunchesPerWave = 15;     // kernels launch_wave starts (fused path), plus 1 with
constexpr int kLaunchesPerWaveMap = 14;  // strings, 2 with the sky map, 1 with arrays; (map path)
constexpr int kMaxArraySub = 512;        // bypass substrings an array of parallel strings may hold

// once per context, before any launch: the block-per-tile kernels' dynamic shared tile
cudaError_t prepare_tile_kernels();
cudaError_t launch_wave(const WaveDev* d_wave, const JobDev* d_jobs, const Buffers& b,
                        const LaunchCfg& cfg, int64_t tot_te_host);
cudaError_t launch_finalize_pairs(const float2* kmod, int n_mods, const float2* kcell, int n_cells,
                                  double* energy, double* energy_u, double* cell_loss, cudaStream_t stream);
// clear-sky sun table: steps k * step_h (k < per_day) of n / per_day days from day_first;
// xyz toward the sun, DNI, DHI, duration and the lit flag per step
cudaError_t launch_sun_table(double lat_deg, int day_first, int64_t per_day, double step_h, double dhi_fraction,
                             int64_t n, double* xyz, float* dni, float* dhi, float* dt, uint8_t* lit,
                             cudaStream_t stream);
// keep steps idx[0, n) of the table (daylight only)
cudaError_t launch_gather_sun(const int64_t* idx, int64_t n, const double* xyz, const float* dni, const float* dhi,
                              double* oxyz, float* odni, float* odhi, cudaStream_t stream);
// sky patches (rings x sectors, centre directions) as a sun table: xyz, DNI 1, DHI 0, dt 1, solid angle
cudaError_t launch_sky_patches(int rings, int sectors, double* xyz, float* dni, float* dhi, float* dt, double* dom,
                               cudaStream_t stream);
// per cell: diffuse shading fraction from the counts [patch][cell] of fixed modules
cudaError_t launch_sky_fraction(const ModuleDev* mods, const int32_t* cell_mod, int n_cells, const double* xyz,
                                const double* dom, int n_patch, const uint8_t* counts, int nn, float* fdiff,
                                double az, double tilt, cudaStream_t st);
// two-axis trackers facing the sun: compass azimuth, tilt = zenith angle clamped to tilt_max
cudaError_t launch_ideal_poses(const double* sun, int64_t n_steps, int n_trk, float tilt_max, float* poses,
                               cudaStream_t stream);

}  // namespace pv3d
