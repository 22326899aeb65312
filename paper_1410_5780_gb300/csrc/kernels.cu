// kernels.cu -- the GB300 hot path of the 3DPV shadow-sample method.
//
// Per wave (a chunk of sun steps of one or more jobs), in stream order:
//   k_window      light window: bounding box of every module corner projected
//                 on the sun's light plane (Section 2, step 3: orthographic view
//                 from the sun, field of view limited to the generator)
//   k_light       light frame, texel size and origin per (job, step)
//   k_modsetup    each module at each step in texel space; marks the raster
//                 tiles that hold samples, their far plane (max sample depth +
//                 bias) and counts the receiver modules per tile
//   k_bin         (triangle, tile) pairs: one warp per 32 meshlets and step,
//                 meshlet boxes tested against the light window one per lane,
//                 then against the far planes of occupied tiles; the
//                 survivors' triangles transformed and binned one per lane;
//                 pairs counted per tile and appended to the wave's pair list
//   k_bin_big     same for triangles that span many tiles, one warp each
//   k_scan_*      bin offsets, the list of non-empty tiles, receiver offsets
//   k_scatter, k_recv_fill   write the bins and receiver lists
//   k_tile_warp   one warp per non-empty tile: the depth test of every sample
//                 that reads the tile against the tile's kept triangles (those
//                 in front of its receivers' planes), sub-block masks, one atomic
//                 per sample row for the cell tallies -- the same decision as a
//                 test against the tile's stored nearest depth (Fig. 3: the
//                 depth buffer keeps the surface nearest the sun)
//   k_raster_test one CTA per tile that a warp cannot take (many receivers or
//                 triangles): block-wide sample-driven test, or a shared-memory
//                 depth tile (texel-centre coverage, atomicMin of
//                 order-preserving depth keys) and the test of its samples
//   k_pv          per (step, module), one per lane: irradiance per cell,
//                 substring currents, bypass-diode maximum power point
//                 (Section 2, step 4)
//   k_string, k_array   series strings and strings in parallel (when asked)
//   k_gen_step, k_heat  sky map of the effective shading (when asked)
//   k_epilogue    Kahan-compensated FP32 sums over the wave's steps in step
//                 order, per module, string and array (energy) and per cell
//                 (beam loss, when asked)
// A job may cover one window group of a generator (its own light window);
// the generator's other modules then enter its map as occluder meshlets.
// The map path replaces the tile kernels + k_pv by k_raster_map (tiles stored
// to an HBM shadow map with 16-byte stores) + k_sample (texel gathers, ballot
// tallies, PV model).  Outside the waves: the clear-sky sun table and ideal
// tracker poses (k_sun_table, k_gather_sun, k_ideal_poses) and the diffuse
// sky view (k_sky_patches, then the waves over the patches, k_sky_fraction).
#include <cfloat>
#include <climits>
#include <cstdint>

#include "pv3d_dev.cuh"

namespace pv3d {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// Order-preserving map float -> uint32 (a < b  <=>  key(a) < key(b)).
__device__ __forceinline__ uint32_t okey(float d)
{
    uint32_t b = __float_as_uint(d);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey_inv(uint32_t k)
{
    uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(b);
}

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// Per-(step, cell) shaded-sample tallies, one byte per entry e (a count is at
// most n^2 <= 225), four bytes to a 32-bit word: the tile kernels add to a
// byte with a word atomic (no carry can leave the byte), the PV kernels read
// bytes.
__device__ __forceinline__ void tally_add(uint32_t* words, int64_t e, uint32_t cnt)
{
    atomicAdd(&words[e >> 2], cnt << (8 * (int)(e & 3)));
}
__device__ __forceinline__ uint32_t tally_get(const uint32_t* words, int64_t e)
{
    return reinterpret_cast<const uint8_t*>(words)[e];
}
__device__ __forceinline__ void tally_set(uint32_t* words, int64_t e, uint32_t v)
{
    reinterpret_cast<uint8_t*>(words)[e] = (uint8_t)v;
}

// Largest job index j with base(j) <= item (bases ascend with j).
template <typename F>
__device__ __forceinline__ int job_of(int n_jobs, int64_t item, F base)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Basis {
    float ux, uy, uz, vx, vy, vz, sx, sy, sz;
};

// Light frame from the sun vector: w = s, u = normalize(s x z) (x at the
// zenith), v = s x u.  Below 2 degrees of elevation the frame is built in FP64.
__device__ __forceinline__ Basis light_basis(const double* sp)
{
    Basis b;
    double sx = sp[0], sy = sp[1], sz = sp[2];
    if (sz < 0.03489949670250097) {  // sin(2 deg)
        double h2 = sx * sx + sy * sy;
        double ux = 1.0, uy = 0.0;
        if (h2 >= 1e-12) {
            double r = 1.0 / sqrt(h2);
            ux = sy * r;
            uy = -sx * r;
        }
        b.ux = (float)ux; b.uy = (float)uy; b.uz = 0.f;
        b.vx = (float)(-sz * uy);
        b.vy = (float)(sz * ux);
        b.vz = (float)(sx * uy - sy * ux);
    } else {
        float fx = (float)sx, fy = (float)sy, fz = (float)sz;
        float h2 = fx * fx + fy * fy;
        float ux = 1.f, uy = 0.f;
        if (h2 >= 1e-12f) {
            float r = rsqrtf(h2);
            ux = fy * r;
            uy = -fx * r;
        }
        b.ux = ux; b.uy = uy; b.uz = 0.f;
        b.vx = -fz * uy;
        b.vy = fz * ux;
        b.vz = fx * uy - fy * ux;
    }
    b.sx = (float)sx; b.sy = (float)sy; b.sz = (float)sz;
    return b;
}

// Posed module frame relative to the job's reference point.  Tracker rotation
// R = Rz(pi - az) * Rx(tilt) about the pivot (pv3d_set_poses).
__device__ __forceinline__ void posed_module(const JobDev& J, const ModuleDev& M, int step,
                                             float3& o, float3& u, float3& v)
{
    o = make_float3(M.o[0], M.o[1], M.o[2]);
    u = make_float3(M.u[0], M.u[1], M.u[2]);
    v = make_float3(M.v[0], M.v[1], M.v[2]);
    if (M.tracker >= 0) {
        const float* pz = J.poses + 2 * ((size_t)step * (size_t)J.n_trk + (size_t)M.tracker);
        float sb, cb, sa, ca;
        sincosf(pz[1], &sb, &cb);
        sincosf(pz[0], &sa, &ca);
        float cg = -ca, sg = sa;
        float r00 = cg, r01 = -sg * cb, r02 = sg * sb;
        float r10 = sg, r11 = cg * cb, r12 = -cg * sb;
        float r20 = 0.f, r21 = sb, r22 = cb;
        const float* pv = J.pivots + 3 * M.tracker;
        float3 oo = o, uu = u, vv = v;
        o = make_float3(pv[0] + r00 * oo.x + r01 * oo.y + r02 * oo.z,
                        pv[1] + r10 * oo.x + r11 * oo.y + r12 * oo.z,
                        pv[2] + r20 * oo.x + r21 * oo.y + r22 * oo.z);
        u = make_float3(r00 * uu.x + r01 * uu.y + r02 * uu.z, r10 * uu.x + r11 * uu.y + r12 * uu.z,
                        r20 * uu.x + r21 * uu.y + r22 * uu.z);
        v = make_float3(r00 * vv.x + r01 * vv.y + r02 * vv.z, r10 * vv.x + r11 * vv.y + r12 * vv.z,
                        r20 * vv.x + r21 * vv.y + r22 * vv.z);
    }
}

__device__ __forceinline__ float dot3(float3 a, float ax, float ay, float az)
{
    return a.x * ax + a.y * ay + a.z * az;
}

// Sample (I, J) of a module, I = cu * n + i and J = cv * n + j, sits at
// a = (I + 1/2) p/n, b = (J + 1/2) p/n along the module axes (Section 2,
// step 3: n x n areas per cell, centred).  Its texel-space position is the
// row's base (the b terms) plus a times the module's first axis, so the
// samples of a row share the base.  The rasteriser's needed-texel mask, the
// fused test and the map gather all evaluate this one rounding sequence, so
// they agree bit for bit on the texel every sample reads.
struct SampleRow {
    float x, y, d;
};
__device__ __forceinline__ SampleRow sample_row(const ModStep& s, int Jr, float p_over_n)
{
    const float b = __fmul_rn(__fadd_rn((float)Jr, 0.5f), p_over_n);
    return SampleRow{__fmaf_rn(b, s.tbx, s.tx0), __fmaf_rn(b, s.tby, s.ty0), __fmaf_rn(b, s.db, s.d0)};
}

// floor(x) clamped to [0, r_max] (r_max = R - 1 < 2^22) without a conversion
// instruction: x is clamped as a float (NaN goes to 0), then 1.5 * 2^23 is
// added rounding toward minus infinity, which leaves floor(x) in the low
// mantissa bits.
__device__ __forceinline__ int texel_floor(float x, float r_max)
{
    const float c = fminf(fmaxf(x, 0.f), r_max);
    return __float_as_int(__fadd_rd(c, 12582912.f)) - 0x4B400000;
}

// Texel (ix, iy) and depth d of sample I of a row; ih = I + 1/2 (exact).
__device__ __forceinline__ void sample_texel(const ModStep& s, const SampleRow& row, float ih, float p_over_n,
                                             float r_max, int& ix, int& iy, float& d)
{
    const float a = __fmul_rn(ih, p_over_n);
    ix = texel_floor(__fmaf_rn(a, s.tax, row.x), r_max);
    iy = texel_floor(__fmaf_rn(a, s.tay, row.y), r_max);
    d = __fmaf_rn(a, s.da, row.d);
}

// (float)k + 1/2 for 0 <= k < 2^22, by the same exponent trick.
__device__ __forceinline__ float texel_centre(int k)
{
    return __fadd_rn(__fadd_rn(__int_as_float(0x4B400000 | k), -12582912.f), 0.5f);
}

// Inclusive prefix sum over the lanes of a warp.
__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    return v;
}

// Edge function A px + B py + C of a set-up triangle at a texel centre, and
// its interpolated depth.  The rasteriser, the sample-driven test and the
// culling masks all evaluate them with this one rounding sequence, so the
// paths agree bit for bit on which triangles cover a texel and at what depth.
__device__ __forceinline__ float edge_at(float A, float Bc, float C, float px, float py)
{
    return __fmaf_rn(A, px, __fmaf_rn(Bc, py, C));
}
__device__ __forceinline__ float depth_at(float w0, float w1, float w2, float e0, float e1, float e2)
{
    return __fmaf_rn(w2, e2, __fmaf_rn(w1, e1, __fmul_rn(w0, e0)));
}

// Is a sample at depth d with bias b behind the stored depth key `key`
// (Section 2, step 3: shaded iff farther from the sun than the nearest
// surface; equality is lit)?
__device__ __forceinline__ bool behind_key(float d, float bias, uint32_t key, float dnear, float qscale,
                                           int u24)
{
    if (u24) return __fmul_rn(__fsub_rn(d, dnear), qscale) > __fmaf_rn(bias, qscale, (float)key);
    return d > __fadd_rn(okey_inv(key), bias);
}

// ---------------------------------------------------------------------------
// k_clear: reset the wave's accumulators (sizes read from the wave descriptor,
// so the whole wave can be replayed from one captured graph)
// ---------------------------------------------------------------------------
__global__ void k_clear(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i0 == 0) {
        B.ctr->n_big = 0u;
        B.ctr->n_nonempty = 0u;
        B.ctr->raster_next = 0u;
        B.ctr->n_heavy = 0u;
        B.ctr->n_pairs = 0ull;
        B.ctr->heavy_next = 0u;
    }
    const int64_t nw = 4 * W->tot_js, nt = W->tot_te;
    for (int64_t i = i0; i < nw; i += stride) B.win[i] = 0xFFFFFFFFu;
    for (int64_t i = i0; i < nt; i += stride) {
        B.t_far[i] = 0u;
        B.t_cnt[i] = 0u;
        B.t_rcnt[i] = 0u;
        B.t_plane[i] = kPlaneNone;
    }
    if (W->fused) {
        const int64_t nc = W->tot_cs, nw = (nc + 3) / 4;  // tallies, and their words
        for (int64_t i = i0; i < nw; i += stride) B.cs_cnt[i] = 0u;
        if (W->want_bits)
            for (int64_t i = i0; i < nc; i += stride) B.cs_bits[i] = 0ull;
    }
}

// ---------------------------------------------------------------------------
// k_window: projected bounding box of the generator per (job, step)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWinPerItem) k_window(const WaveDev* __restrict__ W,
                                                         const JobDev* __restrict__ jobs, Buffers B)
{
    __shared__ float red[4][kWinPerItem / 32];
    const int64_t tot = W->tot_win;
    const int nj = W->n_jobs;
    for (int64_t item = blockIdx.x; item < tot; item += gridDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_win; });
        const JobDev& J = jobs[j];
        int64_t li = item - J.it_win;
        int groups = (J.n_mods + kWinPerItem - 1) / kWinPerItem;
        int ls = (int)(li / groups), g = (int)(li % groups);
        const double* sp = J.sun + 3 * (size_t)(J.step0 + ls);
        if (!(sp[2] > 0.0)) continue;  // uniform over the block
        Basis bs = light_basis(sp);
        float umin = FLT_MAX, umax = -FLT_MAX, vmin = FLT_MAX, vmax = -FLT_MAX;
        int m = g * kWinPerItem + threadIdx.x;
        if (m < J.n_mods) {
            const ModuleDev& M = J.mods[m];
            float3 o, u, v;
            posed_module(J, M, J.step0 + ls, o, u, v);
            float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float a = (c == 1 || c == 2) ? lu : 0.f;
                float b = (c >= 2) ? lv : 0.f;
                float3 p = make_float3(o.x + a * u.x + b * v.x, o.y + a * u.y + b * v.y,
                                       o.z + a * u.z + b * v.z);
                float pu = dot3(p, bs.ux, bs.uy, bs.uz), pv = dot3(p, bs.vx, bs.vy, bs.vz);
                umin = fminf(umin, pu); umax = fmaxf(umax, pu);
                vmin = fminf(vmin, pv); vmax = fmaxf(vmax, pv);
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, off));
            umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, off));
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
        }
        int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[0][w] = umin; red[1][w] = -umax; red[2][w] = vmin; red[3][w] = -vmax;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            float r = red[threadIdx.x][0];
            for (int q = 1; q < kWinPerItem / 32; ++q) r = fminf(r, red[threadIdx.x][q]);
            if (r < FLT_MAX) atomicMin(&B.win[4 * (size_t)(J.js_base + ls) + threadIdx.x], okey(r));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_light: light frame, texel size delta = extent / (R - 2), window origin
// ---------------------------------------------------------------------------
__global__ void k_light(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs, Buffers B)
{
    const int64_t tot = W->tot_js;
    const int nj = W->n_jobs;
    for (int64_t js = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; js < tot;
         js += (int64_t)gridDim.x * blockDim.x) {
        int j = job_of(nj, js, [&](int q) { return (int64_t)jobs[q].js_base; });
        const JobDev& J = jobs[j];
        int ls = (int)(js - J.js_base);
        int step = J.step0 + ls;
        const double* sp = J.sun + 3 * (size_t)step;
        LightParams lp;
        Basis bs = light_basis(sp);
        lp.ux = bs.ux; lp.uy = bs.uy; lp.uz = bs.uz;
        lp.vx = bs.vx; lp.vy = bs.vy; lp.vz = bs.vz;
        lp.sx = bs.sx; lp.sy = bs.sy; lp.sz = bs.sz;
        lp.valid = sp[2] > 0.0;
        lp.dni = J.dni[step];
        lp.dhi = J.dhi[step];
        lp.dt = J.dt[step];
        lp.pad = 0;
        if (lp.valid) {
            float umin = okey_inv(B.win[4 * js + 0]), umax = -okey_inv(B.win[4 * js + 1]);
            float vmin = okey_inv(B.win[4 * js + 2]), vmax = -okey_inv(B.win[4 * js + 3]);
            float ext = fmaxf(fmaxf(umax - umin, vmax - vmin), 1e-6f);
            float delta = ext / (float)(J.R - 2);
            lp.delta = delta;
            lp.inv_delta = 1.f / delta;
            lp.u0 = 0.5f * (umin + umax) - 0.5f * J.R * delta;
            lp.v0 = 0.5f * (vmin + vmax) - 0.5f * J.R * delta;
            // depth range of everything (scene and generator bounds) for 24-bit depth
            float dmin = FLT_MAX, dmax = -FLT_MAX;
            for (int c = 0; c < 8; ++c) {
                float x = (c & 1) ? J.scene_hi[0] : J.scene_lo[0];
                float y = (c & 2) ? J.scene_hi[1] : J.scene_lo[1];
                float z = (c & 4) ? J.scene_hi[2] : J.scene_lo[2];
                float d = -(x * lp.sx + y * lp.sy + z * lp.sz);
                dmin = fminf(dmin, d); dmax = fmaxf(dmax, d);
            }
            float pad = 0.01f * (dmax - dmin) + 1.f;
            lp.dnear = dmin - pad;
            lp.qscale = 16777214.f / ((dmax + pad) - lp.dnear);
        } else {
            lp.delta = 0.f; lp.inv_delta = 0.f; lp.u0 = 0.f; lp.v0 = 0.f;
            lp.dnear = 0.f; lp.qscale = 0.f;
        }
        B.lp[js] = lp;
    }
}

// Depth key stored in the map for depth d (FP32 order bits, or 24-bit fixed point).
__device__ __forceinline__ uint32_t depth_store_key(float d, const LightParams& lp, int u24)
{
    if (!u24) return okey(d);
    float q = (d - lp.dnear) * lp.qscale;
    q = fminf(fmaxf(q, 0.f), 16777214.f);
    return (uint32_t)q;  // truncation: a surface is never stored farther than it is
}

// ---------------------------------------------------------------------------
// k_modsetup: module frames in texel space, bias, tile occupancy, far planes,
// receiver counts; k_recv_fill lists the receivers of the non-empty tiles
// ---------------------------------------------------------------------------
struct TileRange {
    int tx0, tx1, ty0, ty1;
    float dmax;
};

// Tiles touched by the bounding box of a module's corners in texel space.
__device__ __forceinline__ TileRange module_tiles(const ModStep& s, const ModuleDev& M, int R, int sh)
{
    const float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
    float xmin = FLT_MAX, xmax = -FLT_MAX, ymin = FLT_MAX, ymax = -FLT_MAX, dmax = -FLT_MAX;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float a = (k == 1 || k == 2) ? lu : 0.f;
        const float b = (k >= 2) ? lv : 0.f;
        const float x = s.tx0 + a * s.tax + b * s.tbx;
        const float y = s.ty0 + a * s.tay + b * s.tby;
        const float d = s.d0 + a * s.da + b * s.db;
        xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
        ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
        dmax = fmaxf(dmax, d);
    }
    TileRange t;
    t.tx0 = max(0, min(R - 1, (int)floorf(xmin))) >> sh;
    t.tx1 = max(0, min(R - 1, (int)floorf(xmax))) >> sh;
    t.ty0 = max(0, min(R - 1, (int)floorf(ymin))) >> sh;
    t.ty1 = max(0, min(R - 1, (int)floorf(ymax))) >> sh;
    t.dmax = dmax;
    return t;
}

__global__ void k_modsetup(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs, Buffers B)
{
    const int64_t tot = W->tot_mod;
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int u24 = W->depth_u24;
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_mod; });
        const JobDev& J = jobs[j];
        int64_t li = item - J.it_mod;
        int ls = (int)(li / J.n_mods), m = (int)(li % J.n_mods);
        int64_t js = J.js_base + ls;
        const LightParams& lp = B.lp[js];
        if (!lp.valid) continue;
        const ModuleDev& M = J.mods[m];
        float3 o, u, v;
        posed_module(J, M, J.step0 + ls, o, u, v);
        ModStep s;
        float lo_u = dot3(o, lp.ux, lp.uy, lp.uz), lo_v = dot3(o, lp.vx, lp.vy, lp.vz);
        s.tx0 = (lo_u - lp.u0) * lp.inv_delta;
        s.ty0 = (lo_v - lp.v0) * lp.inv_delta;
        s.d0 = -dot3(o, lp.sx, lp.sy, lp.sz);
        s.tax = dot3(u, lp.ux, lp.uy, lp.uz) * lp.inv_delta;
        s.tay = dot3(u, lp.vx, lp.vy, lp.vz) * lp.inv_delta;
        s.da = -dot3(u, lp.sx, lp.sy, lp.sz);
        s.tbx = dot3(v, lp.ux, lp.uy, lp.uz) * lp.inv_delta;
        s.tby = dot3(v, lp.vx, lp.vy, lp.vz) * lp.inv_delta;
        s.db = -dot3(v, lp.sx, lp.sy, lp.sz);
        float3 n = make_float3(u.y * v.z - u.z * v.y, u.z * v.x - u.x * v.z, u.x * v.y - u.y * v.x);
        float nl = rsqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
        n.x *= nl; n.y *= nl; n.z *= nl;
        float c = dot3(n, lp.sx, lp.sy, lp.sz);
        s.cosi = c;
        s.nz = n.z;
        // slope-scaled bias: half a texel diagonal times the receiver slope
        // (tan of incidence, clamped at 89 deg) plus 1/32 texel
        float cc = fmaxf(c, 0.017452406f);
        float tan_i = sqrtf(fmaxf(0.f, 1.f - cc * cc)) / cc;
        s.bias = lp.delta * (0.70710678f * tan_i + 0.03125f);
        if (u24) s.bias += 2.f / lp.qscale;
        B.ms[J.ms_base + li] = s;
        // A triangle shades a sample only where its depth is below the
        // sample's depth minus the bias, so a tile may drop every triangle whose
        // nearest point is not nearer than (max sample depth - bias).
        const TileRange tr = module_tiles(s, M, J.R, sh);
        const uint32_t far_key = u24 ? depth_store_key(tr.dmax - s.bias, lp, 1) + 2u : okey(tr.dmax - s.bias);
        const int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int ty = tr.ty0; ty <= tr.ty1; ++ty)
            for (int tx = tr.tx0; tx <= tr.tx1; ++tx) {
                const int64_t te = te0 + (int64_t)ty * J.tiles_x + tx;
                atomicMax(&B.t_far[te], far_key);
                atomicAdd(&B.t_rcnt[te], 1u);
                // the plane group shared by every receiver of the tile
                const uint32_t pl = (uint32_t)M.plane;
                const uint32_t old = atomicCAS(&B.t_plane[te], kPlaneNone, pl);
                if (old != kPlaneNone && old != pl && old != kPlaneMixed) atomicExch(&B.t_plane[te], kPlaneMixed);
            }
    }
}

// After the scan: list each module as a receiver of the non-empty tiles it touches.
__global__ void k_recv_fill(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs, Buffers B)
{
    const int64_t tot = W->tot_mod;
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int64_t cap = W->recv_cap;
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_mod; });
        const JobDev& J = jobs[j];
        int64_t li = item - J.it_mod;
        int ls = (int)(li / J.n_mods), m = (int)(li % J.n_mods);
        if (!B.lp[J.js_base + ls].valid) continue;
        const ModStep s = B.ms[J.ms_base + li];
        const TileRange tr = module_tiles(s, J.mods[m], J.R, sh);
        const int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int ty = tr.ty0; ty <= tr.ty1; ++ty)
            for (int tx = tr.tx0; tx <= tr.tx1; ++tx) {
                const int64_t te = te0 + (int64_t)ty * J.tiles_x + tx;
                if (B.t_cnt[te] == 0u) continue;
                const uint32_t pos = atomicAdd(&B.t_rcur[te], 1u);
                if (pos < (uint64_t)cap) B.recv[pos] = (uint32_t)m;
            }
    }
}

// ---------------------------------------------------------------------------
// triangles in texel space
// ---------------------------------------------------------------------------
struct TriT {
    float x[3], y[3], d[3];
};

// Light-space texel coordinates and depth of a point (world, relative to the
// job's reference), with every rounding written out: the tile kernels and
// the map path inline this in different contexts, and must get the same
// bits for the same vertex whatever the compiler would otherwise fuse.
__device__ __forceinline__ void project_point(const LightParams& lp, float x, float y, float z, float& tx, float& ty,
                                              float& d)
{
    tx = __fmul_rn(__fsub_rn(__fmaf_rn(z, lp.uz, __fmaf_rn(y, lp.uy, __fmul_rn(x, lp.ux))), lp.u0), lp.inv_delta);
    ty = __fmul_rn(__fsub_rn(__fmaf_rn(z, lp.vz, __fmaf_rn(y, lp.vy, __fmul_rn(x, lp.vx))), lp.v0), lp.inv_delta);
    d = -__fmaf_rn(z, lp.sz, __fmaf_rn(y, lp.sy, __fmul_rn(x, lp.sx)));
}

// Triangle `t` of job J (scene triangle, or module triangle after the scene's)
// at local step ls in texel coordinates.  Module triangles come from the
// job's own module frames (ModStep), or, for a window group, from every
// module of the generator posed for the step and projected like the scene.
__device__ __forceinline__ void tri_texel(const JobDev& J, const Buffers& B, const LightParams& lp,
                                          int ls, int t, TriT& T)
{
    if (t >= J.n_tris && J.occ_mods) {
        const int q = t - J.n_tris;
        float3 o, u, v;
        posed_module(J, J.occ_mods[q >> 1], J.step0 + ls, o, u, v);
        const ModuleDev& M = J.occ_mods[q >> 1];
        const float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
        // corners c0 = O, c1 = O + lu U, c2 = O + lu U + lv V, c3 = O + lv V;
        // triangles (c0, c1, c2) and (c0, c2, c3)
        const float a1 = lu, b1 = (q & 1) ? lv : 0.f;
        const float a2 = (q & 1) ? 0.f : lu, b2 = lv;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = k == 0 ? 0.f : (k == 1 ? a1 : a2), b = k == 0 ? 0.f : (k == 1 ? b1 : b2);
            const float x = __fmaf_rn(b, v.x, __fmaf_rn(a, u.x, o.x));
            const float y = __fmaf_rn(b, v.y, __fmaf_rn(a, u.y, o.y));
            const float z = __fmaf_rn(b, v.z, __fmaf_rn(a, u.z, o.z));
            project_point(lp, x, y, z, T.x[k], T.y[k], T.d[k]);
        }
        return;
    }
    if (t < J.n_tris) {
        const float4* p = J.tri + 3 * (size_t)t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 q = __ldg(p + k);
            project_point(lp, __fsub_rn(q.x, J.ref[0]), __fsub_rn(q.y, J.ref[1]), __fsub_rn(q.z, J.ref[2]), T.x[k],
                          T.y[k], T.d[k]);
        }
    } else {
        int q = t - J.n_tris;
        int m = q >> 1;
        const ModuleDev& M = J.mods[m];
        const ModStep s = B.ms[J.ms_base + (int64_t)ls * J.n_mods + m];
        float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
        // quad corners c0 = O, c1 = O + lu U, c2 = O + lu U + lv V, c3 = O + lv V;
        // triangles (c0, c1, c2) and (c0, c2, c3)
        float a1 = lu, b1 = (q & 1) ? lv : 0.f;
        float a2 = (q & 1) ? 0.f : lu, b2 = lv;
        T.x[0] = s.tx0; T.y[0] = s.ty0; T.d[0] = s.d0;
        T.x[1] = __fmaf_rn(b1, s.tbx, __fmaf_rn(a1, s.tax, s.tx0));
        T.y[1] = __fmaf_rn(b1, s.tby, __fmaf_rn(a1, s.tay, s.ty0));
        T.d[1] = __fmaf_rn(b1, s.db, __fmaf_rn(a1, s.da, s.d0));
        T.x[2] = __fmaf_rn(b2, s.tbx, __fmaf_rn(a2, s.tax, s.tx0));
        T.y[2] = __fmaf_rn(b2, s.tby, __fmaf_rn(a2, s.tay, s.ty0));
        T.d[2] = __fmaf_rn(b2, s.db, __fmaf_rn(a2, s.da, s.d0));
    }
}

// Plane group of triangle t if it is a module triangle (the job's own
// modules, or the generator's occluder modules of a window group), else
// kPlaneNone.  Modules of one plane group cannot shade one another, so a
// module triangle is not binned into a tile whose receivers all share its
// plane group (t_plane).
__device__ __forceinline__ uint32_t module_tri_plane(const JobDev& J, int t)
{
    if (t < J.n_tris) return kPlaneNone;
    const int m = (t - J.n_tris) >> 1;
    return (uint32_t)(J.occ_mods ? J.occ_mods[m].plane : J.mods[m].plane);
}

// Edge functions of a counter-clockwise triangle: E_k(p) = A_k px + B_k py + C_k,
// inside iff every E_k >= 0.  Returns false for a degenerate (edge-on) triangle.
struct Edges {
    float A[3], Bc[3], C[3];
    float area2;
};

__device__ __forceinline__ bool make_edges(TriT& T, Edges& e)
{
    float area2 = __fsub_rn(__fmul_rn(__fsub_rn(T.x[1], T.x[0]), __fsub_rn(T.y[2], T.y[0])),
                            __fmul_rn(__fsub_rn(T.y[1], T.y[0]), __fsub_rn(T.x[2], T.x[0])));
    if (!(fabsf(area2) > 0.f)) return false;
    if (area2 < 0.f) {
        float tx = T.x[1], ty = T.y[1], td = T.d[1];
        T.x[1] = T.x[2]; T.y[1] = T.y[2]; T.d[1] = T.d[2];
        T.x[2] = tx; T.y[2] = ty; T.d[2] = td;
        area2 = -area2;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // edge k is opposite vertex k: from vertex k+1 to vertex k+2
        int a = (k + 1) % 3, b = (k + 2) % 3;
        e.A[k] = -__fsub_rn(T.y[b], T.y[a]);
        e.Bc[k] = __fsub_rn(T.x[b], T.x[a]);
        e.C[k] = -__fadd_rn(__fmul_rn(e.A[k], T.x[a]), __fmul_rn(e.Bc[k], T.y[a]));
    }
    e.area2 = area2;
    return true;
}

// Could the triangle cover a texel centre of the rectangle [x0,x1] x [y0,y1]?
__device__ __forceinline__ bool rect_overlap(const Edges& e, float x0, float x1, float y0, float y1)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float x = e.A[k] > 0.f ? x1 : x0;
        float y = e.Bc[k] > 0.f ? y1 : y0;
        if (e.A[k] * x + e.Bc[k] * y + e.C[k] < 0.f) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// k_bin: (triangle, tile) pairs in one pass -- vertex transform batched over
// steps; each pair is counted into its tile and appended to the wave's pair
// list, which k_scatter distributes into the bins after the scan
// ---------------------------------------------------------------------------

// Append this lane's pairs (te[q], tri) for the set bits q of `valid` to the
// pair list: one atomic per warp.  Called by all 32 lanes together.
__device__ __forceinline__ void append_pairs(const Buffers& B, const WaveDev* W, const uint32_t* te, uint32_t valid,
                                             uint32_t tri)
{
    const int lane = threadIdx.x & 31;
    const int c = __popc(valid);
    const int inc = warp_incl_scan(c);
    const int tot = __shfl_sync(0xffffffffu, inc, 31);
    if (tot == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(&B.ctr->n_pairs, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned long long pos = base + (unsigned long long)(inc - c);
    const uint64_t cap = (uint64_t)W->bin_cap;
#pragma unroll
    for (int q = 0; q < kBigTiles; ++q)
        if (valid & (1u << q)) {
            if (pos < cap) B.pairs[pos] = make_uint2(te[q], tri);
            ++pos;
        }
}

constexpr int kLaneTiles = 16;  // a meshlet over at most this many tiles is tested by its own lane

__global__ void __launch_bounds__(256, 4) k_bin(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                             Buffers B)
{
    // One warp per (group of 32 meshlets, step), the step fastest so that
    // consecutive warps reuse the group's triangles from cache.  Each lane
    // first projects one scene meshlet's bounding box for the step and keeps
    // it if it overlaps the light window; the warp then tests each kept box
    // against the far planes of the tiles it covers (lanes over tiles): if no
    // tile can receive a shadow from the meshlet, its 32 triangles are
    // skipped together.  Otherwise each lane bins one of its triangles.
    // Generator module triangles follow the scene's, in meshlets of 32,
    // without the box test.  A triangle over more than kBigTiles tiles is
    // listed for k_bin_big.
    const int64_t tot = W->tot_tri;
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int TS = 1 << sh;
    const int u24 = W->depth_u24;
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < tot; item += n_warps) {
        const int j = job_of(nj, item, [&](int q) { return jobs[q].it_tri; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.it_tri;
        const int g = (int)(li / J.k), ls = (int)(li - (int64_t)g * J.k);
        const int R = J.R;
        const int64_t js = J.js_base + ls;
        const LightParams& lp = B.lp[js];
        if (!lp.valid) continue;
        const int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        // scene meshlets, then (window groups) occluder-module meshlets, both
        // with boxes, then the job's own module meshlets
        const int n_boxed = J.n_ml + J.n_oml;
        const int n_all = n_boxed + ((J.n_mtris + 31) >> 5);
        // this lane's boxed meshlet: window test, covered tiles, nearest depth key
        const int ml = g * 32 + lane;
        int btx0 = 0, btx1 = -1, bty0 = 0, bty1 = -1;
        uint32_t bkey = 0u;
        bool pass = false;
        if (ml < n_boxed) {
            const float4* box = ml < J.n_ml ? J.ml_box + 2 * ml : J.oml_box + 2 * (ml - J.n_ml);
            const float4 lo = box[0], hi = box[1];
            float xmin = FLT_MAX, xmax = -FLT_MAX, ymin = FLT_MAX, ymax = -FLT_MAX, dmin = FLT_MAX;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float x = ((c & 1) ? hi.x : lo.x) - J.ref[0];
                const float y = ((c & 2) ? hi.y : lo.y) - J.ref[1];
                const float z = ((c & 4) ? hi.z : lo.z) - J.ref[2];
                const float tx = (x * lp.ux + y * lp.uy + z * lp.uz - lp.u0) * lp.inv_delta;
                const float ty = (x * lp.vx + y * lp.vy + z * lp.vz - lp.v0) * lp.inv_delta;
                xmin = fminf(xmin, tx); xmax = fmaxf(xmax, tx);
                ymin = fminf(ymin, ty); ymax = fmaxf(ymax, ty);
                dmin = fminf(dmin, -(x * lp.sx + y * lp.sy + z * lp.sz));
            }
            pass = xmax >= 0.5f && ymax >= 0.5f && xmin <= R - 0.5f && ymin <= R - 0.5f;
            if (pass) {
                btx0 = max(0, (int)floorf(xmin - 0.5f)) >> sh;
                btx1 = min(R - 1, (int)ceilf(xmax)) >> sh;
                bty0 = max(0, (int)floorf(ymin - 0.5f)) >> sh;
                bty1 = min(R - 1, (int)ceilf(ymax)) >> sh;
                // the box's nearest point, less a margin for the rounding of
                // the projection
                bkey = depth_store_key(dmin - 1e-3f * (1.f + fabsf(dmin)), lp, u24);
            }
        } else {
            pass = ml < n_all;
        }
        // the meshlet's nearest point against the far plane of each tile it
        // covers: each lane tests its own meshlet's tiles (independent loads
        // across the warp), the warp together those of a meshlet over many
        // tiles
        bool keep_lane = false, coop = false;
        if (pass && ml < n_boxed) {
            const int ntl = (btx1 - btx0 + 1) * (bty1 - bty0 + 1);
            if (ntl <= kLaneTiles) {
                // no early exit: the loads of a row of tiles are issued together
                for (int ty = bty0; ty <= bty1; ++ty) {
                    const uint32_t* far_row = B.t_far + te0 + (int64_t)ty * J.tiles_x;
#pragma unroll 4
                    for (int tx = btx0; tx <= btx1; ++tx) keep_lane |= bkey < far_row[tx];
                }
            } else {
                coop = true;
            }
        } else if (pass) {
            keep_lane = true;  // module meshlets: no box
        }
        unsigned int kept = __ballot_sync(0xffffffffu, keep_lane);
        for (unsigned int cm = __ballot_sync(0xffffffffu, coop); cm; cm &= cm - 1u) {
            const int q = __ffs(cm) - 1;
            const int mx0 = __shfl_sync(0xffffffffu, btx0, q), mx1 = __shfl_sync(0xffffffffu, btx1, q);
            const int my0 = __shfl_sync(0xffffffffu, bty0, q), my1 = __shfl_sync(0xffffffffu, bty1, q);
            const uint32_t mkey = __shfl_sync(0xffffffffu, bkey, q);
            const int wx = mx1 - mx0 + 1, ntl = wx * (my1 - my0 + 1);
            bool keep = false;
            for (int q0 = 0; q0 < ntl && !keep; q0 += 32) {
                const int k = q0 + lane;
                bool kk = false;
                if (k < ntl) {
                    const int ty = my0 + k / wx, tx = mx0 + k % wx;
                    kk = mkey < B.t_far[te0 + (int64_t)ty * J.tiles_x + tx];
                }
                keep = __any_sync(0xffffffffu, kk);
            }
            if (keep) kept |= 1u << q;
        }
        for (unsigned int cand = kept; cand; cand &= cand - 1u) {
            const int q = __ffs(cand) - 1;
            const int mi = g * 32 + q;
            int t;
            bool act;
            if (mi < n_boxed) {
                if (mi < J.n_ml) {
                    t = mi * 32 + lane;
                    act = t < J.n_tris;
                } else {
                    t = J.n_tris + (mi - J.n_ml) * 32 + lane;
                    act = t < J.n_tris + 2 * J.n_occ;
                }
            } else {
                t = J.n_tris + (mi - n_boxed) * 32 + lane;
                act = t < J.n_tris + J.n_mtris;
            }
            // per lane: the tiles its triangle may shade (at most kBigTiles), in
            // registers until the warp appends them together
            uint32_t te[kBigTiles];
            uint32_t valid = 0u;
            if (act) {
                TriT T;
                tri_texel(J, B, lp, ls, t, T);
                const uint32_t tplane = module_tri_plane(J, t);
                Edges e;
                const float xmin = fminf(T.x[0], fminf(T.x[1], T.x[2])), xmax = fmaxf(T.x[0], fmaxf(T.x[1], T.x[2]));
                const float ymin = fminf(T.y[0], fminf(T.y[1], T.y[2])), ymax = fmaxf(T.y[0], fmaxf(T.y[1], T.y[2]));
                // covered texel centres (ix + 0.5) lie in [xmin, xmax]
                const int ix0 = max(0, (int)ceilf(xmin - 0.5f)), ix1 = min(R - 1, (int)floorf(xmax - 0.5f));
                const int iy0 = max(0, (int)ceilf(ymin - 0.5f)), iy1 = min(R - 1, (int)floorf(ymax - 0.5f));
                if (make_edges(T, e) && xmax >= 0.5f && ymax >= 0.5f && xmin <= R - 0.5f && ymin <= R - 0.5f &&
                    ix0 <= ix1 && iy0 <= iy1) {
                    const uint32_t dkey = depth_store_key(fminf(T.d[0], fminf(T.d[1], T.d[2])), lp, u24);
                    const int tx0 = ix0 >> sh, tx1 = ix1 >> sh, ty0 = iy0 >> sh, ty1 = iy1 >> sh;
                    const int wx = tx1 - tx0 + 1, ntiles = wx * (ty1 - ty0 + 1);
                    if (ntiles > kBigTiles) {
                        const unsigned int pos = atomicAdd(&B.ctr->n_big, 1u);
                        if (pos < (uint64_t)W->big_cap) B.big[pos] = make_uint2((uint32_t)t, (uint32_t)js);
                    } else {
#pragma unroll
                        for (int q = 0; q < kBigTiles; ++q) {
                            te[q] = 0u;
                            if (q >= ntiles) continue;
                            const int ty = ty0 + q / wx, tx = tx0 + q % wx;
                            if (ntiles > 1 && !rect_overlap(e, tx * TS + 0.5f, tx * TS + TS - 0.5f, ty * TS + 0.5f,
                                                            ty * TS + TS - 0.5f))
                                continue;
                            const uint32_t x = (uint32_t)(te0 + (int64_t)ty * J.tiles_x + tx);
                            // unoccupied tile (far 0) or triangle wholly behind its far plane
                            if (!(dkey < B.t_far[x])) continue;
                            // a module triangle in the plane of every receiver of the tile
                            if (tplane != kPlaneNone && B.t_plane[x] == tplane) continue;
                            atomicAdd(&B.t_cnt[x], 1u);
                            te[q] = x;
                            valid |= 1u << q;
                        }
                    }
                }
            }
            append_pairs(B, W, te, valid, (uint32_t)t);
        }
    }
}

// Triangles spanning more than kBigTiles tiles: one warp per triangle, lanes
// over its tiles.
__global__ void __launch_bounds__(256) k_bin_big(const WaveDev* __restrict__ W,
                                                 const JobDev* __restrict__ jobs, Buffers B)
{
    const unsigned int n_big = min((unsigned long long)B.ctr->n_big, (unsigned long long)W->big_cap);
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int TS = 1 << sh;
    const int u24 = W->depth_u24;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < n_big; e += n_warps) {
        uint2 en = B.big[e];
        int t = (int)en.x;
        int64_t js = en.y;
        int j = job_of(nj, js, [&](int q) { return (int64_t)jobs[q].js_base; });
        const JobDev& J = jobs[j];
        int ls = (int)(js - J.js_base);
        const LightParams lp = B.lp[js];
        TriT T;
        tri_texel(J, B, lp, ls, t, T);
        Edges ed;
        if (!make_edges(T, ed)) continue;
        const int R = J.R;
        float xmin = fminf(T.x[0], fminf(T.x[1], T.x[2])), xmax = fmaxf(T.x[0], fmaxf(T.x[1], T.x[2]));
        float ymin = fminf(T.y[0], fminf(T.y[1], T.y[2])), ymax = fmaxf(T.y[0], fmaxf(T.y[1], T.y[2]));
        int ix0 = max(0, (int)ceilf(xmin - 0.5f)), ix1 = min(R - 1, (int)floorf(xmax - 0.5f));
        int iy0 = max(0, (int)ceilf(ymin - 0.5f)), iy1 = min(R - 1, (int)floorf(ymax - 0.5f));
        if (ix0 > ix1 || iy0 > iy1) continue;
        float dmin = fminf(T.d[0], fminf(T.d[1], T.d[2]));
        uint32_t dkey = depth_store_key(dmin, lp, u24);
        const uint32_t tplane = module_tri_plane(J, t);
        int tx0 = ix0 >> sh, tx1 = ix1 >> sh, ty0 = iy0 >> sh, ty1 = iy1 >> sh;
        int wx = tx1 - tx0 + 1;
        int ntiles = wx * (ty1 - ty0 + 1);
        int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int q0 = 0; q0 < ntiles; q0 += 32) {
            const int q = q0 + lane;
            uint32_t te[kBigTiles];
            uint32_t valid = 0u;
            te[0] = 0u;
            if (q < ntiles) {
                const int tx = tx0 + q % wx, ty = ty0 + q / wx;
                const uint32_t x = (uint32_t)(te0 + (int64_t)ty * J.tiles_x + tx);
                if (rect_overlap(ed, tx * TS + 0.5f, tx * TS + TS - 0.5f, ty * TS + 0.5f, ty * TS + TS - 0.5f) &&
                    dkey < B.t_far[x] && !(tplane != kPlaneNone && B.t_plane[x] == tplane)) {
                    atomicAdd(&B.t_cnt[x], 1u);
                    te[0] = x;
                    valid = 1u;
                }
            }
            append_pairs(B, W, te, valid, (uint32_t)t);
        }
    }
}

// After the scan: each (tile, triangle) pair to its place in the tile's bin.
__global__ void __launch_bounds__(256) k_scatter(const WaveDev* __restrict__ W, Buffers B)
{
    const unsigned long long np = min(B.ctr->n_pairs, (unsigned long long)W->bin_cap);
    const uint64_t cap = (uint64_t)W->bin_cap;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < np;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 p = B.pairs[i];
        const uint32_t pos = atomicAdd(&B.t_cur[p.x], 1u);
        if (pos < cap) B.bins[pos] = p.y;
    }
}

// ---------------------------------------------------------------------------
// scan over the wave's tile entries: triangle-bin offsets, the list of
// non-empty tiles (= map slots) and receiver-list offsets of non-empty tiles
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

// Block-wide exclusive scan of three counters; returns the block totals.
__device__ __forceinline__ void block_scan3(unsigned long long v[3], unsigned long long tot[3])
{
    __shared__ unsigned long long ws[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, inc[q], off);
            if (lane >= off) inc[q] += y;
        }
    }
    if (lane == 31)
        for (int q = 0; q < 3; ++q) ws[q][w] = inc[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            unsigned long long x = lane < nw ? ws[q][lane] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            if (lane < nw) ws[q][lane] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        tot[q] = ws[q][nw - 1];
        v[q] = (w ? ws[q][w - 1] : 0ull) + inc[q] - v[q];
    }
    __syncthreads();
}

__device__ __forceinline__ void scan_values(const Buffers& B, int64_t i, unsigned long long v[3])
{
    const uint32_t c = B.t_cnt[i];
    v[0] = c;
    v[1] = c ? 1u : 0u;
    v[2] = c ? B.t_rcnt[i] : 0u;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_a(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    for (int64_t st = blockIdx.x; st < n_tiles; st += gridDim.x) {
        unsigned long long v[3] = {0, 0, 0};
        int64_t base = st * kScanTile + (int64_t)threadIdx.x * kScanPer;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            if (base + q < tot) {
                unsigned long long x[3];
                scan_values(B, base + q, x);
                v[0] += x[0]; v[1] += x[1]; v[2] += x[2];
            }
        }
        unsigned long long t[3];
        block_scan3(v, t);
        if (threadIdx.x == 0)
            for (int q = 0; q < 3; ++q) B.block_sums[3 * st + q] = t[q];
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_b(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    unsigned long long carry[3] = {0, 0, 0};
    for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        unsigned long long v[3], t[3];
        for (int q = 0; q < 3; ++q) v[q] = i < n_tiles ? B.block_sums[3 * i + q] : 0ull;
        block_scan3(v, t);
        if (i < n_tiles)
            for (int q = 0; q < 3; ++q) B.block_sums[3 * i + q] = v[q] + carry[q];
        for (int q = 0; q < 3; ++q) carry[q] += t[q];
    }
    if (threadIdx.x == 0) {
        Counters* c = B.ctr;
        c->tot_bins = carry[0];
        c->n_nonempty = (unsigned int)min(carry[1], 0xFFFFFFFFull);
        c->tot_recv = carry[2];
        c->stat_bins += carry[0];
        c->stat_nonempty += carry[1];
        if (carry[0] > c->need_bins) c->need_bins = carry[0];
        if (carry[1] > c->need_tiles) c->need_tiles = carry[1];
        if (carry[2] > c->need_recv) c->need_recv = carry[2];
        unsigned long long nb = c->n_big;
        if (nb > c->need_big) c->need_big = nb;
        if (carry[0] > (unsigned long long)W->bin_cap) c->overflow |= 1u;
        if (!W->fused && carry[1] > (unsigned long long)W->map_cap_tiles) c->overflow |= 2u;
        if (nb > (unsigned long long)W->big_cap) c->overflow |= 4u;
        if (carry[2] > (unsigned long long)W->recv_cap) c->overflow |= 8u;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_c(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    for (int64_t st = blockIdx.x; st < n_tiles; st += gridDim.x) {
        unsigned long long x[kScanPer][3];
        unsigned long long v[3] = {0, 0, 0};
        int64_t base = st * kScanTile + (int64_t)threadIdx.x * kScanPer;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            if (base + q < tot) scan_values(B, base + q, x[q]);
            else x[q][0] = x[q][1] = x[q][2] = 0ull;
            v[0] += x[q][0]; v[1] += x[q][1]; v[2] += x[q][2];
        }
        unsigned long long t[3];
        block_scan3(v, t);
        for (int q = 0; q < 3; ++q) v[q] += B.block_sums[3 * st + q];
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            int64_t i = base + q;
            // offsets of non-empty tiles only: every reader of t_off, t_cur,
            // t_slot, t_roff and t_rcur takes a tile from the non-empty list
            // or checks t_cnt first
            if (i < tot && x[q][1]) {
                B.t_off[i] = (uint32_t)min(v[0], 0xFFFFFFFFull);
                B.t_cur[i] = (uint32_t)min(v[0], 0xFFFFFFFFull);
                B.t_slot[i] = (uint32_t)min(v[1], 0xFFFFFFFFull);
                B.t_roff[i] = (uint32_t)min(v[2], 0xFFFFFFFFull);
                B.t_rcur[i] = (uint32_t)min(v[2], 0xFFFFFFFFull);
                B.nonempty[v[1]] = (uint32_t)i;
            }
            v[0] += x[q][0]; v[1] += x[q][1]; v[2] += x[q][2];
        }
    }
}

// ---------------------------------------------------------------------------
// per-tile work: receivers, the sample-driven depth test, and the tile
// rasteriser (shared by the fused and the map kernels)
// ---------------------------------------------------------------------------
constexpr int kRecvChunk = 64;  // receivers staged in shared memory at a time (two per lane of one warp)
constexpr int kTriBatchMax = 128;  // triangles set up in shared memory at a time by the rasteriser (one per thread)
constexpr int kMaxTri = 256;    // triangles a block-wide tile may keep for the sample-driven test
// Sub-blocks per tile side in the sample-driven test (4, 8 and 16 texels on
// 32-, 64- and 128-texel tiles; a 16 x 16 grid on 128-texel tiles tests fewer
// triangles per sample but costs more in its masks than it saves).
template <int TS>
struct SubGrid {
    static constexpr int side = 8;
    static constexpr int blocks = side * side;
};
// Triangles a heavy-tile block may keep for its sample-driven test: 32-texel
// tiles are always rasterised (k_raster_test), so their shared memory holds
// only a token list and more blocks fit an SM.
template <int TS>
struct HeavyKept {
    static constexpr int n = TS == 32 ? 32 : kMaxTri;
    static constexpr int words = n / 32;
};
static_assert(kRecvChunk == 64, "receiver prefix sums take two entries per lane of one warp");

// Exclusive prefix sum of up to 64 entries, two per lane; called by one full
// warp.  Returns the total in every lane.
__device__ __forceinline__ int warp_excl_scan64(int& a0, int& a1)
{
    const int s = a0 + a1;
    const int inc = warp_incl_scan(s);
    const int ex = inc - s;
    a1 = ex + a0;
    a0 = ex;
    return __shfl_sync(0xffffffffu, inc, 31);
}

// Exclusive prefix sum of n <= 32 K entries a[0, n), K consecutive entries
// per lane of one warp, in place; a[n] receives the total.  Called by one
// full warp.
template <int K>
__device__ __forceinline__ void warp_excl_scan_k(int* a, int n)
{
    const int lane = threadIdx.x & 31;
    int v[K], sum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        v[k] = i < n ? a[i] : 0;
        sum += v[k];
    }
    const int inc = warp_incl_scan(sum);
    int ex = inc - sum;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = lane * K + k;
        if (i < n) a[i] = ex;
        ex += v[k];
    }
    if (lane == 31) a[n] = inc;
}

// A triangle set up for one tile: edge functions, scaled depths, its texel
// box and the sub-blocks in which it may shade a sample (tri_sub_mask).  The
// rasteriser visits rows y0 .. y0 + rows - 1 of the box, one row per lane.
// 17 words: lanes reading different triangles' fields hit different banks.
struct TriSetup {
    float A[3], Bc[3], C[3];
    float e0, e1, e2;
    short x0, bw;
    int y0, rows;        // rows = 0: not kept
    uint32_t sm_lo, sm_hi;  // sub-block bits 0-31, 32-63
};
static_assert(sizeof(TriSetup) == 17 * 4, "odd word stride");

// A triangle set up for the sample-driven test (48 bytes, three 16-byte loads):
// edge functions k = 0..2 in tile-local texel coordinates and depths scaled by
// the inverse doubled area.
struct TriS {
    float4 p;  // A0, B0, C0, A1
    float4 q;  // B1, C1, A2, B2
    float4 r;  // C2, e0, e1, e2
};

// q / d for 0 <= q < 2^24 (one float estimate, one correction).
__device__ __forceinline__ int fdiv(int q, int d, float inv_d)
{
    int r = (int)((float)q * inv_d);
    const int rem = q - r * d;
    if (rem < 0) --r;
    else if (rem >= d) ++r;
    return r;
}

// A receiver module of the tile, staged in shared memory.  Its samples that
// may read the tile form the index box [I0, I1] x [J0, J1] (I = cu * n + i,
// J = cv * n + j), walked as (sample row, cell column) items; each item's
// samples are further clipped to the row's stretch that crosses the tile.
struct RecvSm {
    ModStep s;
    float p_over_n, inv_p;     // sample spacing along the module axes (m) and its inverse
    float pa, pb, pc;          // receiver depth plane d = pa x + pb y + pc in tile-local texel coordinates
    float cull_tol;            // plane tolerance (half the bias slack), or -1 if the plane may not cull
    float cx0, cy0;            // module origin, tile-local texel coordinates
    float inv_tax, inv_tay;    // inverse texels per metre along the module's U axis (0: no row clip by it)
    float xlo, xhi, ylo, yhi;  // the tile's texel range, tile-local (open towards the map border)
    float bx0, bx1, by0, by1;  // the module's texel-space bounding box, tile-local, one texel wider
    float inv_ncol;
    int cu;                    // cells across the module
    int cell_base;             // first cell of the module in the generator
    int I0, I1, J0;            // sample-index box (J1 = J0 + rows - 1)
    int cI0, ncol;             // cell columns of the box
    int item_pref;             // (row, cell column) items of the receivers staged before this one
};

// Threads of a k_raster_test block and its register budget (blocks an SM):
// 32-texel tiles have small shared tiles, and the plants with many heavy
// 32-texel tiles keep more of them in flight with 128-thread blocks (fewer
// threads wait at each of a tile's barriers).
template <int TS>
struct HeavyCfg {
    static constexpr int threads = TS == 32 ? 128 : 256;
    static constexpr int min_blocks = TS == 32 ? 9 : 4;  // 32: 53 registers, 9 x 24 KB shared
};

template <int TS>
struct RasterSm {
    uint32_t tile[TS * TS];  // depth keys of the tile
};

// Kept triangles of a tile for the sample-driven test, up to NT of them.
template <int TS, int NT, bool SEEN>
struct KeptSm {
    TriS tri[NT];
    uint32_t box[NT];                       // texel box x0 | y0 << 8 | x1 << 16 | y1 << 24
    float dmin[NT];                         // nearest vertex depth
    uint2 smask[NT];                        // strict keep: the sub-blocks (bit sb) it may shade a sample of
    float dlim[SubGrid<TS>::blocks];        // per sub-block: a triangle shades none of its samples
                                            // unless its nearest depth is below this
    uint32_t sbm[SubGrid<TS>::blocks][NT / 32];  // per sub-block: triangles that may shade one of its samples
    uint32_t seen[SEEN ? TS * TS / 32 : 1]; // work counting: texels whose fragments were counted
};
static_assert(SubGrid<32>::blocks == 64 && SubGrid<64>::blocks == 64 && SubGrid<128>::blocks == 64,
              "a triangle's sub-block set is one 64-bit mask");

// Summary of a tile's sub-block depth limits (sub_summary).
struct SubInfo {
    uint2 occ;   // sub-blocks some receiver meets
    float dlo;   // smallest limit among them
};

template <int TS>
struct TileSm {
    union {
        RasterSm<TS> r;
        KeptSm<TS, HeavyKept<TS>::n, true> s;
    } u;
    float dlim[SubGrid<TS>::blocks]; // per sub-block depth limit (sub_limits)
    SubInfo si;                      // their summary (sub_summary)
    uint32_t mask[TS * TS / 32];     // texels read by some sample (sparse tiles)
    int n_need;                      // how many (sparse tiles)
    RecvSm recv[kRecvChunk];
    int n_recv;                      // receivers staged
    int total_items;                 // (sample row, cell column) items over the staged receivers
    int any_write;                   // some texel of the tile received a depth
    int n_tri;                       // triangles kept by the sample-driven set-up
    TriSetup tri[kTriBatchMax];      // a batch of set-up triangles, one per thread
    int row_pref[kTriBatchMax + 1];  // prefix of their rows
};

// Stage receiver module m of tile (tx, ty): sample-index box (the tile
// corners mapped back onto the module plane, widened by one sample), row
// clipping, bounding box and depth plane.  item_pref receives the receiver's
// own item count.
template <int TS>
__device__ __forceinline__ void stage_one(RecvSm& R, const JobDev& J, const Buffers& B, int ls, int tx, int ty,
                                          int m)
{
    const ModuleDev& M = J.mods[m];
    const ModStep s = B.ms[J.ms_base + (int64_t)ls * J.n_mods + m];
    const int n = J.n;
    const float X0 = (float)(tx * TS), Y0 = (float)(ty * TS);
    R.s = s;
    R.p_over_n = __fdiv_rn(M.pitch, (float)n);
    R.inv_p = 1.f / R.p_over_n;
    R.cu = M.cu;
    R.cell_base = M.cell_base;
    R.cx0 = s.tx0 - X0;
    R.cy0 = s.ty0 - Y0;
    R.inv_tax = fabsf(s.tax) > 1e-6f ? 1.f / s.tax : 0.f;
    R.inv_tay = fabsf(s.tay) > 1e-6f ? 1.f / s.tay : 0.f;
    R.xlo = tx == 0 ? -FLT_MAX : 0.f;
    R.xhi = tx == J.tiles_x - 1 ? FLT_MAX : (float)TS;
    R.ylo = ty == 0 ? -FLT_MAX : 0.f;
    R.yhi = ty == J.tiles_x - 1 ? FLT_MAX : (float)TS;
    {
        const float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
        float x0 = FLT_MAX, x1 = -FLT_MAX, y0 = FLT_MAX, y1 = -FLT_MAX;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float a = (c & 1) ? lu : 0.f, b = (c & 2) ? lv : 0.f;
            const float x = R.cx0 + a * s.tax + b * s.tbx, y = R.cy0 + a * s.tay + b * s.tby;
            x0 = fminf(x0, x); x1 = fmaxf(x1, x);
            y0 = fminf(y0, y); y1 = fmaxf(y1, y);
        }
        R.bx0 = x0 - 1.f; R.bx1 = x1 + 1.f;
        R.by0 = y0 - 1.f; R.by1 = y1 + 1.f;
    }
    int I0 = 0, I1 = M.cu * n - 1, J0 = 0, J1 = M.cv * n - 1;
    const float det = s.tax * s.tby - s.tay * s.tbx;
    const bool planar = fabsf(det) > 1e-6f * (fabsf(s.tax * s.tby) + fabsf(s.tay * s.tbx));
    R.cull_tol = -1.f;
    R.pa = R.pb = R.pc = 0.f;
    if (planar) {
        const float inv_det = 1.f / det;
        float amin = FLT_MAX, amax = -FLT_MAX, bmin = FLT_MAX, bmax = -FLT_MAX;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float dx = ((c & 1) ? (float)TS : 0.f) - R.cx0;
            const float dy = ((c & 2) ? (float)TS : 0.f) - R.cy0;
            const float a = (dx * s.tby - dy * s.tbx) * inv_det;
            const float b = (dy * s.tax - dx * s.tay) * inv_det;
            amin = fminf(amin, a); amax = fmaxf(amax, a);
            bmin = fminf(bmin, b); bmax = fmaxf(bmax, b);
        }
        // samples at a = (I + 1/2) p/n: I in [a_min n/p - 1/2, a_max n/p - 1/2], one more each side
        I0 = max(I0, (int)fmaxf(floorf(amin * R.inv_p - 0.5f) - 1.f, -1.f));
        I1 = min(I1, (int)fminf(ceilf(amax * R.inv_p - 0.5f) + 1.f, 1e6f));
        J0 = max(J0, (int)fmaxf(floorf(bmin * R.inv_p - 0.5f) - 1.f, -1.f));
        J1 = min(J1, (int)fminf(ceilf(bmax * R.inv_p - 0.5f) + 1.f, 1e6f));
        // depth of the receiver plane over the tile: a triangle lying on or
        // behind the plane (by less than half the bias slack) shades none
        // of its samples, so it may be skipped for this receiver
        R.pa = (s.da * s.tby - s.db * s.tay) * inv_det;
        R.pb = (s.db * s.tax - s.da * s.tbx) * inv_det;
        R.pc = s.d0 - R.pa * R.cx0 - R.pb * R.cy0;
        if (s.cosi > 0.017452406f) R.cull_tol = B.lp[J.js_base + ls].delta * (1.f / 64.f);
    }
    R.I0 = I0;
    R.I1 = I1;
    R.J0 = J0;
    R.cI0 = I0 / n;
    R.ncol = (I0 <= I1) ? I1 / n - I0 / n + 1 : 0;
    R.inv_ncol = 1.f / (float)max(R.ncol, 1);
    R.item_pref = (I0 <= I1 && J0 <= J1) ? R.ncol * (J1 - J0 + 1) : 0;  // prefixed by the caller
}

// Stage receivers [r0, r0 + cnt) of tile (tx, ty) for the whole block (cnt <=
// kRecvChunk), with their item prefixes.
template <int TS>
__device__ void stage_receivers(TileSm<TS>& sm, const JobDev& J, const Buffers& B, int ls, int tx, int ty,
                                uint64_t r0, int cnt)
{
    const int tid = threadIdx.x;
    if (tid < cnt) stage_one<TS>(sm.recv[tid], J, B, ls, tx, ty, (int)B.recv[r0 + tid]);
    __syncthreads();
    if (tid < 32) {
        const int q0 = 2 * tid, q1 = q0 + 1;
        int i0 = q0 < cnt ? sm.recv[q0].item_pref : 0, i1 = q1 < cnt ? sm.recv[q1].item_pref : 0;
        const int ti = warp_excl_scan64(i0, i1);
        if (q0 < cnt) sm.recv[q0].item_pref = i0;
        if (q1 < cnt) sm.recv[q1].item_pref = i1;
        if (tid == 0) {
            sm.n_recv = cnt;
            sm.total_items = ti;
        }
    }
    __syncthreads();
}

// Receiver of staged item `it` (items prefixed in item_pref).
__device__ __forceinline__ int recv_of_item(const RecvSm* recv, int n_recv, int it)
{
    int lo = 0, hi = n_recv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (recv[mid].item_pref <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Clip [Ib, Ie] to the samples of row Jr whose texel may lie in the tile:
// the stretch of the row's line a -> (cx0 + a tax + b tbx, cy0 + a tay + b tby)
// inside the tile's texel range, widened by one sample each side (the exact
// test is the caller's, per sample).
__device__ __forceinline__ void row_range(const RecvSm& R, int Jr, int& Ib, int& Ie)
{
    const float b = __fmul_rn(__fadd_rn((float)Jr, 0.5f), R.p_over_n);
    float amin = -FLT_MAX, amax = FLT_MAX;
    if (R.inv_tax != 0.f) {
        const float c = fmaf(b, R.s.tbx, R.cx0);
        const float a0 = (R.xlo - c) * R.inv_tax, a1 = (R.xhi - c) * R.inv_tax;
        amin = fminf(a0, a1);
        amax = fmaxf(a0, a1);
    }
    if (R.inv_tay != 0.f) {
        const float c = fmaf(b, R.s.tby, R.cy0);
        const float a0 = (R.ylo - c) * R.inv_tay, a1 = (R.yhi - c) * R.inv_tay;
        amin = fmaxf(amin, fminf(a0, a1));
        amax = fminf(amax, fmaxf(a0, a1));
    }
    const float lo = floorf(amin * R.inv_p - 0.5f) - 1.f, hi = ceilf(amax * R.inv_p - 0.5f) + 1.f;
    Ib = max(Ib, (int)fminf(fmaxf(lo, -1.f), 1e7f));
    Ie = min(Ie, (int)fmaxf(fminf(hi, 1e7f), -2.f));
}

// Decode staged item `it`: receiver, sample row Jr, cell (cu, cv), row jj
// within the cell and the item's sample range [Ib, Ie].
__device__ __forceinline__ const RecvSm& decode_item(const RecvSm* recv, int n_recv, int it, int n, float inv_n,
                                                     int& Jr, int& cu, int& cv, int& jj, int& Ib, int& Ie)
{
    const RecvSm& R = recv[recv_of_item(recv, n_recv, it)];
    const int q = it - R.item_pref;
    const int row = fdiv(q, R.ncol, R.inv_ncol);
    cu = R.cI0 + q - row * R.ncol;
    Jr = R.J0 + row;
    cv = fdiv(Jr, n, inv_n);
    jj = Jr - cv * n;
    Ib = max(R.I0, cu * n);
    Ie = min(R.I1, cu * n + n - 1);
    row_range(R, Jr, Ib, Ie);
    return R;
}

// Visit the samples of the staged receivers that read tile (tx, ty): one
// thread per (sample row, cell column) item walks the row's samples inside
// the cell, the box and the row's stretch over the tile.  f(R, k, ix, iy, d)
// is called per sample inside the tile (k = j * n + i within the cell);
// g(R, cu, cv) after each item.
template <int TS, bool PROF, typename F, typename G>
__device__ __forceinline__ void for_tile_samples(const RecvSm* recv, int n_recv, int total_items, const JobDev& J,
                                                 int tx, int ty, int it_begin, int it_stride, unsigned int& cand,
                                                 F f, G g)
{
    constexpr int SH = TS == 128 ? 7 : (TS == 64 ? 6 : 5);
    const int n = J.n;
    const float r_max = (float)(J.R - 1);
    const float inv_n = 1.f / (float)n;
    for (int it = it_begin; it < total_items; it += it_stride) {
        int Jr, cu, cv, jj, Ib, Ie;
        const RecvSm& R = decode_item(recv, n_recv, it, n, inv_n, Jr, cu, cv, jj, Ib, Ie);
        if (PROF) cand += (unsigned int)max(0, Ie - Ib + 1);
        const SampleRow row = sample_row(R.s, Jr, R.p_over_n);
        float ih = (float)Ib + 0.5f;
        for (int I = Ib; I <= Ie; ++I, ih += 1.f) {
            float d;
            int ix, iy;
            sample_texel(R.s, row, ih, R.p_over_n, r_max, ix, iy, d);
            if ((ix >> SH) == tx && (iy >> SH) == ty) f(R, jj * n + (I - cu * n), ix, iy, d);
        }
        g(R, cu, cv);
    }
}

// Can triangle T (tile-local texel coordinates) shade a sample of a staged
// receiver?  False only if it lies on or behind every receiver's plane.
__device__ __forceinline__ bool may_shade(const RecvSm* recv, int n_recv, const TriT& T, bool cull_ok)
{
    if (!cull_ok) return true;
    for (int r = 0; r < n_recv; ++r) {
        const RecvSm& R = recv[r];
        if (R.cull_tol < 0.f) return true;
        float gap = FLT_MAX;
#pragma unroll
        for (int k = 0; k < 3; ++k) gap = fminf(gap, T.d[k] - (R.pa * T.x[k] + R.pb * T.y[k] + R.pc));
        if (!(gap >= -R.cull_tol)) return true;
    }
    return false;
}

// Tile-local texel-centre range [x0, x1] x [y0, y1] of a triangle's bounding box.
template <int TS>
__device__ __forceinline__ bool tri_box(const TriT& T, int& x0, int& x1, int& y0, int& y1)
{
    const float xmin = fminf(T.x[0], fminf(T.x[1], T.x[2])), xmax = fmaxf(T.x[0], fmaxf(T.x[1], T.x[2]));
    const float ymin = fminf(T.y[0], fminf(T.y[1], T.y[2])), ymax = fmaxf(T.y[0], fmaxf(T.y[1], T.y[2]));
    x0 = max(0, (int)ceilf(xmin - 0.5f));
    x1 = min(TS - 1, (int)floorf(xmax - 0.5f));
    y0 = max(0, (int)ceilf(ymin - 0.5f));
    y1 = min(TS - 1, (int)floorf(ymax - 0.5f));
    return x0 <= x1 && y0 <= y1;
}

// ---- sample-driven depth test ----------------------------------------------
// A tile with few triangles is not rasterised: each of its samples tests the
// triangles that may cover its texel directly.  The sample is shaded iff some
// triangle covers its texel centre at a depth it is behind -- the same
// decision as a depth test against the tile's stored minimum (the comparison
// is monotone in the stored depth), with the same arithmetic per triangle.

// Summary of a tile's sub-block depth limits, for tri_sub_mask's fast path:
// the sub-blocks that any receiver meets (limit above -inf) and the smallest
// limit among them.  Called by one full warp once the limits are written.
__device__ __forceinline__ SubInfo sub_summary(const float* dlim)
{
    const int lane = threadIdx.x & 31;
    const float a = dlim[lane], b = dlim[lane + 32];
    SubInfo si;
    si.occ.x = __ballot_sync(0xffffffffu, a > -FLT_MAX);
    si.occ.y = __ballot_sync(0xffffffffu, b > -FLT_MAX);
    float lo = fminf(a > -FLT_MAX ? a : FLT_MAX, b > -FLT_MAX ? b : FLT_MAX);
#pragma unroll
    for (int off = 16; off; off >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    si.dlo = lo;
    return si;
}

// The sub-blocks of the tile in which a set-up triangle may shade a sample
// (bit sb = sy * side + sx): its nearest vertex is nearer than the
// sub-block's depth limit, and each edge function is non-negative at the
// texel centre of (its texel box within the sub-block) farthest inside the
// edge -- exact, since edge_at is monotone in px and py, so a texel centre
// of the sub-block that the triangle covers implies a non-negative value
// there.  Row by row of sub-blocks: when every edge is non-negative at the
// row's corner farthest outside it, the triangle covers every texel centre
// of its box in that row, and when its nearest vertex is also nearer than the
// tile's smallest limit, the row's bits are the occupied sub-blocks of the
// box's columns.  A triangle with no such sub-block cannot shade any sample
// of the tile and is not kept.
template <int TS>
__device__ __forceinline__ uint64_t tri_sub_mask(const Edges& ed, int x0, int x1, int y0, int y1, float dmin,
                                                 const float* dlim, const SubInfo& si)
{
    constexpr int kSubSide = SubGrid<TS>::side;
    constexpr int SW = TS / kSubSide;  // sub-block side, texels
    static_assert(kSubSide == 8, "a row of sub-blocks is one byte of the mask");
    const uint64_t occ = (uint64_t)si.occ.x | ((uint64_t)si.occ.y << 32);
    const int sx0 = x0 / SW, sx1 = x1 / SW;
    const uint64_t cols = (uint64_t)((2u << sx1) - (1u << sx0));  // bits sx0..sx1 of a row
    const bool near_all = dmin < si.dlo;
    const float fxl = texel_centre(x0), fxh = texel_centre(x1);
    uint64_t m = 0ull;
    for (int sy = y0 / SW; sy <= y1 / SW; ++sy) {
        const float fy0 = texel_centre(max(y0, sy * SW)), fy1 = texel_centre(min(y1, sy * SW + SW - 1));
        float t[3];
        bool full = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t[k] = __fmaf_rn(ed.Bc[k], ed.Bc[k] > 0.f ? fy1 : fy0, ed.C[k]);
            full = full && edge_at(ed.A[k], ed.Bc[k], ed.C[k], ed.A[k] > 0.f ? fxl : fxh,
                                   ed.Bc[k] > 0.f ? fy0 : fy1) >= 0.f;
        }
        const uint64_t row = (cols << (8 * sy)) & occ;
        if (full && near_all) {
            m |= row;
            continue;
        }
        for (uint64_t r = row; r; r &= r - 1ull) {
            const int sb = __ffsll((long long)r) - 1;
            if (!(dmin < dlim[sb])) continue;
            if (!full) {
                const int sx = sb & 7;
                const float fx0 = texel_centre(max(x0, sx * SW)), fx1 = texel_centre(min(x1, sx * SW + SW - 1));
                bool in = true;
#pragma unroll
                for (int k = 0; k < 3; ++k) in = in && __fmaf_rn(ed.A[k], ed.A[k] > 0.f ? fx1 : fx0, t[k]) >= 0.f;
                if (!in) continue;
            }
            m |= 1ull << sb;
        }
    }
    return m;
}

// Set up binned triangle t of tile (ox, oy) for the sample-driven test: false
// if it lies behind every staged receiver or covers no texel centre of the
// tile; with `strict`, also if it may shade no sample of any sub-block
// (tri_sub_mask with the sub-block depth limits dlim), its sub-blocks in
// smask.  box and dmin feed sub_masks (loose keep).
template <int TS, bool PROF>
__device__ __forceinline__ bool setup_tri_s(const JobDev& J, const Buffers& B, const LightParams& lp, int ls, int t,
                                            float ox, float oy, const RecvSm* recv, int n_recv, bool cull_ok,
                                            bool strict, const float* dlim, const SubInfo& si, TriS& ts,
                                            uint32_t& box, float& dmin, uint64_t& smask, unsigned int& culled)
{
    TriT T;
    tri_texel(J, B, lp, ls, t, T);
#pragma unroll
    for (int k = 0; k < 3; ++k) { T.x[k] -= ox; T.y[k] -= oy; }
    if (!may_shade(recv, n_recv, T, cull_ok)) {
        if (PROF) ++culled;
        return false;
    }
    Edges ed;
    int x0, x1, y0, y1;
    if (!make_edges(T, ed) || !tri_box<TS>(T, x0, x1, y0, y1)) return false;
    dmin = fminf(T.d[0], fminf(T.d[1], T.d[2]));
    if (strict) {
        smask = tri_sub_mask<TS>(ed, x0, x1, y0, y1, dmin, dlim, si);
        if (smask == 0ull) return false;
    }
    const float inv_a = 1.f / ed.area2;
    ts.p = make_float4(ed.A[0], ed.Bc[0], ed.C[0], ed.A[1]);
    ts.q = make_float4(ed.Bc[1], ed.C[1], ed.A[2], ed.Bc[2]);
    ts.r = make_float4(ed.C[2], T.d[0] * inv_a, T.d[1] * inv_a, T.d[2] * inv_a);
    box = (uint32_t)x0 | ((uint32_t)y0 << 8) | ((uint32_t)x1 << 16) | ((uint32_t)y1 << 24);
    return true;
}

// Per sub-block, the depth below which a triangle must reach to shade one of
// its samples: the largest over the receivers whose box meets the sub-block
// of (receiver plane over the sub-block - bias), plus twice the plane
// tolerance and, for 24-bit depth, the one-step truncation of the stored
// key.  A sample at depth d is shaded only by a surface nearer than d - bias
// (less the truncation), and interpolated depths inside a triangle are no
// nearer than its nearest vertex (up to rounding, which the tolerance
// covers).  A sub-block with a receiver whose plane may not cull gets no
// limit; one that no receiver meets gets -inf.  Entries sb = q_begin,
// q_begin + q_stride, ... are written.
template <int TS>
__device__ __forceinline__ void sub_limits(const RecvSm* recv, int n_recv, float* dlim, float q1, int q_begin,
                                           int q_stride)
{
    constexpr int kSubSide = SubGrid<TS>::side, kSubBlocks = SubGrid<TS>::blocks;
    constexpr int SW = TS / kSubSide;
    for (int sb = q_begin; sb < kSubBlocks; sb += q_stride) {
        const float x0 = (float)((sb % kSubSide) * SW), x1 = x0 + (float)SW;
        const float y0 = (float)((sb / kSubSide) * SW), y1 = y0 + (float)SW;
        float lim = -FLT_MAX;
        for (int r = 0; r < n_recv; ++r) {
            const RecvSm& R = recv[r];
            if (R.bx1 < x0 || R.bx0 > x1 || R.by1 < y0 || R.by0 > y1) continue;
            if (R.cull_tol < 0.f) { lim = FLT_MAX; break; }
            const float pm = R.pc + fmaxf(R.pa * x0, R.pa * x1) + fmaxf(R.pb * y0, R.pb * y1);
            lim = fmaxf(lim, pm - R.s.bias + 2.f * R.cull_tol + q1);
        }
        dlim[sb] = lim;
    }
}

// Per sub-block of the tile, the kept triangles that may shade one of its
// samples: nearest depth below the sub-block's limit, box overlap, then each
// edge at the sub-block's texel centre farthest inside it (exact: edge_at is
// monotone in px and py, so a covered texel of the sub-block implies a
// non-negative value there).  Entries q = q_begin, q_begin + q_stride, ... <
// 64 * words(n) of sbm are written.
template <int TS, int WORDS>
__device__ __forceinline__ void sub_masks(const TriS* tri, const uint32_t* boxes, const float* dmin,
                                          const float* dlim, uint32_t (*sbm)[WORDS], int n, int q_begin, int q_stride)
{
    constexpr int kSubSide = SubGrid<TS>::side, kSubBlocks = SubGrid<TS>::blocks;
    constexpr int SW = TS / kSubSide;  // sub-block side, texels
    const int nw = (n + 31) >> 5;
    for (int q = q_begin; q < kSubBlocks * nw; q += q_stride) {
        const int sb = q & (kSubBlocks - 1), w = q / kSubBlocks;
        const int sx = (sb % kSubSide) * SW, sy = (sb / kSubSide) * SW;
        const float fx0 = (float)sx + 0.5f, fx1 = (float)(sx + SW - 1) + 0.5f;
        const float fy0 = (float)sy + 0.5f, fy1 = (float)(sy + SW - 1) + 0.5f;
        const float lim = dlim[sb];
        uint32_t m = 0u;
        const int kend = min(32, n - w * 32);
        for (int k = 0; k < kend; ++k) {
            const int t = w * 32 + k;
            if (!(dmin[t] < lim)) continue;
            const uint32_t bx = boxes[t];
            const int x0 = bx & 255u, y0 = (bx >> 8) & 255u, x1 = (bx >> 16) & 255u, y1 = bx >> 24;
            if (x0 > sx + SW - 1 || x1 < sx || y0 > sy + SW - 1 || y1 < sy) continue;
            const float4 p = tri[t].p, qq = tri[t].q, r = tri[t].r;
            if (edge_at(p.x, p.y, p.z, p.x > 0.f ? fx1 : fx0, p.y > 0.f ? fy1 : fy0) < 0.f) continue;
            if (edge_at(p.w, qq.x, qq.y, p.w > 0.f ? fx1 : fx0, qq.x > 0.f ? fy1 : fy0) < 0.f) continue;
            if (edge_at(qq.z, qq.w, r.x, qq.z > 0.f ? fx1 : fx0, qq.w > 0.f ? fy1 : fy0) < 0.f) continue;
            m |= 1u << k;
        }
        sbm[sb][w] = m;
    }
}

// Per sub-block of the tile, the kept triangles that may shade one of its
// samples (bit k of word w: kept triangle 32 w + k), transposed from the
// triangles' sub-block masks: for a few triangles each lane gathers its two
// sub-blocks' bits, else one ballot per sub-block.  Words w =
// w_begin, w_begin + w_stride, ... of the n kept triangles are written; called
// by whole warps.
template <int WORDS>
__device__ __forceinline__ void build_sbm(const uint2* smask, uint32_t (*sbm)[WORDS], int n, int w_begin,
                                          int w_stride)
{
    const int lane = threadIdx.x & 31;
    const int nw = (n + 31) >> 5;
    if (n <= 24) {
        // few triangles: each lane assembles its two sub-blocks' words
        if (w_begin != 0) return;
        uint32_t lo = 0u, hi = 0u;
        for (int t = 0; t < n; ++t) {
            const uint2 m = smask[t];
            lo |= ((m.x >> lane) & 1u) << t;
            hi |= ((m.y >> lane) & 1u) << t;
        }
        sbm[lane][0] = lo;
        sbm[lane + 32][0] = hi;
        return;
    }
    for (int w = w_begin; w < nw; w += w_stride) {
        const int t = (w << 5) | lane;
        const uint2 m = t < n ? smask[t] : make_uint2(0u, 0u);
        uint32_t lo = 0u, hi = 0u;
#pragma unroll
        for (int sb = 0; sb < 32; ++sb) {
            const uint32_t a = __ballot_sync(0xffffffffu, (m.x >> sb) & 1u);
            const uint32_t b = __ballot_sync(0xffffffffu, (m.y >> sb) & 1u);
            if (lane == sb) { lo = a; hi = b; }
        }
        sbm[lane][w] = lo;
        sbm[lane + 32][w] = hi;
    }
}

// Does kept triangle T cover texel centre (px, py) at a depth that the
// sample (depth d, bias) is behind?
__device__ __forceinline__ bool tri_shades(const TriS& T, float px, float py, float d, float bias,
                                           const LightParams& lp, int u24, bool& covers)
{
    const float4 p = T.p, q = T.q, r = T.r;
    const float w0 = edge_at(p.x, p.y, p.z, px, py);
    const float w1 = edge_at(p.w, q.x, q.y, px, py);
    const float w2 = edge_at(q.z, q.w, r.x, px, py);
    covers = w0 >= 0.f && w1 >= 0.f && w2 >= 0.f;
    if (!covers) return false;
    const float depth = depth_at(w0, w1, w2, r.y, r.z, r.w);
    if (u24) return behind_key(d, bias, depth_store_key(depth, lp, 1), lp.dnear, lp.qscale, 1);
    return d > __fadd_rn(depth, bias);  // = behind_key(d, bias, okey(depth), ...): okey is invertible
}

// Depth test of one sample (tile-local texel lx, ly) against the kept
// triangles of its sub-block; stops at the first that shades it.  With
// PROF, also counts the fragments a depth map needs at the texel (the kept
// triangles covering it) once per texel, using the `seen` bitmap.
template <int TS, int WORDS, bool PROF>
__device__ __forceinline__ bool sample_test(const TriS* tri, int n_kept, const uint32_t (*sbm)[WORDS], int nw,
                                            uint32_t* seen, int lx, int ly, float d, float bias,
                                            const LightParams& lp, int u24, unsigned int& pairs, unsigned int& frags)
{
    constexpr int kSubSide = SubGrid<TS>::side;
    const int sb = (ly / (TS / kSubSide)) * kSubSide + lx / (TS / kSubSide);
    const float px = texel_centre(lx), py = texel_centre(ly);
    const uint32_t* ms = sbm[sb];
    bool shaded = false;
    for (int w = 0; w < nw && !shaded; ++w) {
        uint32_t m = ms[w];
        while (m) {
            const int t = (w << 5) | (__ffs(m) - 1);
            m &= m - 1u;
            bool cov;
            if (PROF) ++pairs;
            if (tri_shades(tri[t], px, py, d, bias, lp, u24, cov)) {
                shaded = true;
                break;
            }
        }
    }
    if (PROF) {
        // the depth map's fragments at this texel: every kept triangle
        // covering it (before the sub-block depth limits)
        const uint32_t bit = 1u << (lx & 31);
        if (!(atomicOr(&seen[(ly * TS + lx) >> 5], bit) & bit)) {
            for (int t = 0; t < n_kept; ++t) {
                bool cov;
                tri_shades(tri[t], px, py, d, bias, lp, u24, cov);
                frags += cov ? 1u : 0u;
            }
        }
    }
    return shaded;
}

// Sub-blocks sx0..sx1 x sy0..sy1 of a tile as a mask (bit sy * 8 + sx).
__device__ __forceinline__ uint64_t sub_box(int sx0, int sx1, int sy0, int sy1)
{
    const uint64_t cols = (uint64_t)((2u << sx1) - (1u << sx0));
    const uint64_t rows = (0x0101010101010101ull >> (8 * (7 - (sy1 - sy0)))) << (8 * sy0);
    return rows * cols;  // bytes of rows are 0 or 1: no carries
}

// Depth-test the samples of staged receivers recv[0, n_recv) (items prefixed
// in item_pref, total_items in all) that read tile (tx, ty) against the kept
// triangles: items it_begin, it_begin + it_stride, ... one per thread.  Each
// item adds its shaded count to its (step, cell) tally with one atomic.  An
// item is skipped whole when no sub-block of the texel box of its end
// samples is in cand_sb (the sub-blocks in which some kept triangle may shade
// a sample; all ones: no skipping) -- exact, since a sample's texel is
// monotone in its index along the row (sample_texel), so every sample of the
// item reads a texel of that box.
template <int TS, int WORDS, bool PROF>
__device__ __forceinline__ void test_items(const RecvSm* recv, int n_recv, int total_items, const JobDev& J,
                                           const LightParams& lp, int u24, int tx, int ty, int it_begin,
                                           int it_stride, const TriS* tri, int n_kept,
                                           const uint32_t (*sbm)[WORDS], int nw, uint64_t cand_sb, uint32_t* seen,
                                           uint32_t* tally, int64_t tally0, unsigned long long* bits_row,
                                           int want_bits,
                                           unsigned int& cand, unsigned int& samples, unsigned int& pairs,
                                           unsigned int& frags)
{
    constexpr int SH = TS == 128 ? 7 : (TS == 64 ? 6 : 5);
    constexpr int SWS = SH - 3;  // log2 of the sub-block side (8 x 8 sub-blocks)
    static_assert(SubGrid<TS>::side == 8, "sub-block index by shifts");
    const int n = J.n;
    const float r_max = (float)(J.R - 1);
    const float inv_n = 1.f / (float)n;
    for (int it = it_begin; it < total_items; it += it_stride) {
        int Jr, cu, cv, jj, Ib, Ie;
        const RecvSm& R = decode_item(recv, n_recv, it, n, inv_n, Jr, cu, cv, jj, Ib, Ie);
        if (PROF) cand += (unsigned int)max(0, Ie - Ib + 1);
        if (Ib > Ie) continue;
        // the receiver's sample frame and the row's base in registers
        const ModStep s = R.s;
        const float p_over_n = R.p_over_n;
        const SampleRow row = sample_row(s, Jr, p_over_n);
        if (cand_sb != ~0ull) {
            float dq;
            int ax, ay, bx, by;
            sample_texel(s, row, (float)Ib + 0.5f, p_over_n, r_max, ax, ay, dq);
            sample_texel(s, row, (float)Ie + 0.5f, p_over_n, r_max, bx, by, dq);
            const int lx0 = max(min(ax, bx) - (tx << SH), 0), lx1 = min(max(ax, bx) - (tx << SH), TS - 1);
            const int ly0 = max(min(ay, by) - (ty << SH), 0), ly1 = min(max(ay, by) - (ty << SH), TS - 1);
            if (lx0 > lx1 || ly0 > ly1) continue;
            if (!(sub_box(lx0 >> SWS, lx1 >> SWS, ly0 >> SWS, ly1 >> SWS) & cand_sb)) continue;
        }
        const int i0 = cu * n;
        uint32_t bits = 0u;  // bit i: sample i of the item's row (within its cell) is shaded
        float ih = (float)Ib + 0.5f;
        for (int I = Ib; I <= Ie; ++I, ih += 1.f) {
            float d;
            int ix, iy;
            sample_texel(s, row, ih, p_over_n, r_max, ix, iy, d);
            if ((ix >> SH) != tx || (iy >> SH) != ty) continue;
            if (PROF) ++samples;
            if (sample_test<TS, WORDS, PROF>(tri, n_kept, sbm, nw, seen, ix & (TS - 1), iy & (TS - 1), d, s.bias,
                                             lp, u24, pairs, frags))
                bits |= 1u << (I - i0);
        }
        if (bits) {
            const int gcell = R.cell_base + cv * R.cu + cu;
            tally_add(tally, tally0 + gcell, (uint32_t)__popc(bits));
            // sample k = jj * n + i of the cell; flags kept for k < 64
            if (want_bits && jj * n < 64) atomicOr(&bits_row[gcell], (unsigned long long)bits << (jj * n));
        }
    }
}

// ---- tile rasteriser ------------------------------------------------------

// Narrow the texel range [lo, hi] of a row to the texels whose centre px
// has fma(A, px, t) >= 0 -- edge_at on that row, which is monotone in px,
// so the texels form an interval: an estimate of its end from the edge's
// root, corrected by evaluating the edge exactly as the per-texel test does
// (at most the range's width of steps, one or two in practice).
__device__ __forceinline__ void edge_span(float A, float t, int& lo, int& hi)
{
    if (lo > hi) return;
    if (A > 0.f) {
        const float f = ceilf(__fdividef(-t, A) - 0.5f);
        int i = (int)fminf(fmaxf(f, (float)lo), (float)(hi + 1));
        while (i > lo && __fmaf_rn(A, (float)(i - 1) + 0.5f, t) >= 0.f) --i;
        while (i <= hi && __fmaf_rn(A, (float)i + 0.5f, t) < 0.f) ++i;
        lo = i;
    } else if (A < 0.f) {
        const float f = floorf(__fdividef(-t, A) - 0.5f);
        int i = (int)fminf(fmaxf(f, (float)(lo - 1)), (float)hi);
        while (i < hi && __fmaf_rn(A, (float)(i + 1) + 0.5f, t) >= 0.f) ++i;
        while (i >= lo && __fmaf_rn(A, (float)i + 0.5f, t) < 0.f) --i;
        hi = i;
    } else if (!(t >= 0.f)) {
        hi = lo - 1;  // fma(0, px, t) = t for every texel of the row
    }
}

// Bits of the texels lo .. hi (tile-local) that fall in word w of a row.
__device__ __forceinline__ uint32_t span_word(int lo, int hi, int w)
{
    const int a = max(lo - 32 * w, 0), b = min(hi - 32 * w, 31);
    return b < a ? 0u : (0xFFFFFFFFu >> (31 - b)) & (0xFFFFFFFFu << a);
}

// Texel bits of word w of a row from the row's byte of sub-block bits (bit
// sx covers texels sx * TS / 8 .. sx * TS / 8 + TS / 8 - 1).
template <int TS>
__device__ __forceinline__ uint32_t sub_word(uint32_t sbyte, int w)
{
    if constexpr (TS == 32) {
        uint32_t x = sbyte;  // bit i -> bit 4 i, then a nibble each
        x = (x | (x << 12)) & 0x000F000Fu;
        x = (x | (x << 6)) & 0x03030303u;
        x = (x | (x << 3)) & 0x11111111u;
        return x * 0xFu;
    } else if constexpr (TS == 64) {
        uint32_t x = (sbyte >> (4 * w)) & 0xFu;  // bit i -> bit 8 i, then a byte each
        x = (x | (x << 14)) & 0x00030003u;
        x = (x | (x << 7)) & 0x01010101u;
        return x * 0xFFu;
    } else {
        uint32_t x = (sbyte >> (2 * w)) & 0x3u;  // bit i -> bit 16 i, then a half-word each
        x = (x | (x << 15)) & 0x00010001u;
        return x * 0xFFFFu;
    }
}

// Set up binned triangle t of tile (ox, oy) for the rasteriser in S and
// return its rows: 0 (not kept) if it lies behind every staged receiver's
// plane, covers no texel centre of the tile, or may shade no sample of any
// sub-block (tri_sub_mask with the sub-block depth limits dlim).
template <int TS, bool PROF>
__device__ __forceinline__ int setup_raster_tri(const JobDev& J, const Buffers& B, const LightParams& lp, int ls,
                                                int t, float ox, float oy, const RecvSm* recv, int n_recv,
                                                bool cull_ok, const float* dlim, const SubInfo& si, TriSetup& S,
                                                unsigned int& culled)
{
    constexpr int SWS = (TS == 128 ? 7 : (TS == 64 ? 6 : 5)) - 3;  // log2 of the sub-block side
    TriT T;
    tri_texel(J, B, lp, ls, t, T);
#pragma unroll
    for (int k = 0; k < 3; ++k) { T.x[k] -= ox; T.y[k] -= oy; }
    if (!may_shade(recv, n_recv, T, cull_ok)) {
        if (PROF) ++culled;
        return 0;
    }
    Edges ed;
    int x0, x1, y0, y1;
    if (!make_edges(T, ed) || !tri_box<TS>(T, x0, x1, y0, y1)) return 0;
    const uint64_t sb = tri_sub_mask<TS>(ed, x0, x1, y0, y1, fminf(T.d[0], fminf(T.d[1], T.d[2])), dlim, si);
    if (sb == 0ull) return 0;
    const float inv_a = 1.f / ed.area2;
#pragma unroll
    for (int k = 0; k < 3; ++k) { S.A[k] = ed.A[k]; S.Bc[k] = ed.Bc[k]; S.C[k] = ed.C[k]; }
    S.e0 = T.d[0] * inv_a; S.e1 = T.d[1] * inv_a; S.e2 = T.d[2] * inv_a;
    S.sm_lo = (uint32_t)sb;
    S.sm_hi = (uint32_t)(sb >> 32);
    S.x0 = (short)x0; S.bw = (short)(x1 - x0 + 1);
    // the box's rows within the sub-block rows it may shade
    const int sy0 = (__ffsll((long long)sb) - 1) >> 3, sy1 = (63 - __clzll((long long)sb)) >> 3;
    const int ry0 = max(y0, sy0 << SWS), ry1 = min(y1, (sy1 << SWS) + (1 << SWS) - 1);
    S.y0 = ry0;
    S.rows = ry1 - ry0 + 1;
    return S.rows;
}

// Draw rows [u_beg, u_end) of set-up triangles tri[0, nb) (rows prefixed in
// row_pref) into the depth tile, 32 at a time, one (triangle, row) per lane
// of the calling warp: the row's texels inside all three edges, exactly
// (edge_at on a row is fma(A, px, t_k), monotone in px: edge_span), within
// the triangle's sub-blocks and, unless mask is null, marked in mask.
template <int TS, bool PROF>
__device__ __forceinline__ void draw_rows(const TriSetup* tri, const int* row_pref, int nb, int u_beg, int u_end,
                                          const uint32_t* mask, uint32_t* tile, const LightParams& lp, int u24,
                                          bool& wrote, unsigned int& visits, unsigned int& writes)
{
    constexpr int WPR = TS / 32;
    constexpr int SWS = (TS == 128 ? 7 : (TS == 64 ? 6 : 5)) - 3;
    const int lane = threadIdx.x & 31;
    // a lane finds its triangle by walking forward from the last
    int t = 0;
    {
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_pref[mid] <= u_beg) lo = mid; else hi = mid - 1;
        }
        t = lo;
    }
    for (int ub = u_beg; ub < u_end; ub += 32) {
        const int u = ub + lane;
        if (u >= u_end) break;
        while (row_pref[t + 1] <= u) ++t;
        const TriSetup& S = tri[t];
        const int iy = S.y0 + (u - row_pref[t]);
        const int sy = iy >> SWS;
        const uint32_t sbyte = ((sy < 4 ? S.sm_lo : S.sm_hi) >> ((sy & 3) << 3)) & 0xFFu;
        if (sbyte == 0u) continue;
        if (mask) {
            uint32_t any = 0u;
#pragma unroll
            for (int w = 0; w < WPR; ++w) any |= mask[iy * WPR + w];
            if (any == 0u) continue;
        }
        const float py = (float)iy + 0.5f;
        const float A0 = S.A[0], A1 = S.A[1], A2 = S.A[2];
        const float t0 = __fmaf_rn(S.Bc[0], py, S.C[0]);
        const float t1 = __fmaf_rn(S.Bc[1], py, S.C[1]);
        const float t2 = __fmaf_rn(S.Bc[2], py, S.C[2]);
        int lo = S.x0, hi = S.x0 + S.bw - 1;
        edge_span(A0, t0, lo, hi);
        edge_span(A1, t1, lo, hi);
        edge_span(A2, t2, lo, hi);
        if (lo > hi) continue;
        const float e0 = S.e0, e1 = S.e1, e2 = S.e2;
        for (int w = lo >> 5; w <= (hi >> 5); ++w) {
            uint32_t bits = span_word(lo, hi, w) & sub_word<TS>(sbyte, w);
            if (mask) bits &= mask[iy * WPR + w];
            while (bits) {
                const int ix = (w << 5) + __ffs(bits) - 1;
                bits &= bits - 1u;
                const float px = (float)ix + 0.5f;
                const float w0 = __fmaf_rn(A0, px, t0);
                const float w1 = __fmaf_rn(A1, px, t1);
                const float w2 = __fmaf_rn(A2, px, t2);
                atomicMin(&tile[iy * TS + ix], depth_store_key(depth_at(w0, w1, w2, e0, e1, e2), lp, u24));
                wrote = true;
                if (PROF) { ++visits; ++writes; }
            }
        }
    }
}

// The tile's sub-block depth limits (sub_limits, or no limit when the
// receivers are staged in chunks) and their summary, for the whole block.
template <int TS>
__device__ __forceinline__ void tile_limits(TileSm<TS>& sm, const LightParams& lp, int u24, bool cull_ok)
{
    const int tid = threadIdx.x, bd = blockDim.x;
    if (cull_ok) sub_limits<TS>(sm.recv, sm.n_recv, sm.dlim, u24 ? 1.f / lp.qscale : 0.f, tid, bd);
    else
        for (int q = tid; q < SubGrid<TS>::blocks; q += bd) sm.dlim[q] = FLT_MAX;
    __syncthreads();
    if (tid < 32) {
        const SubInfo si = sub_summary(sm.dlim);
        if (tid == 0) sm.si = si;
    }
    __syncthreads();
}

// Rasterise the tile's triangles into sm.u.r.tile.  Sparse tiles (fewer samples
// than two per texel) are rasterised only at the texels their samples read.
// A triangle is drawn only in the sub-blocks where it may shade a sample
// (tri_sub_mask with the sub-block depth limits): the stored nearest depth
// may then differ at a texel, but never the decision of a sample there (the
// dropped triangles are behind every sample they cover, and "shaded" is
// "some covering triangle is nearer than the sample less its bias").  Each
// (triangle, row) goes to one lane, which visits only the texels of the row
// inside all three edges (edge_span), of the triangle's sub-blocks and, in
// sparse tiles, marked.  Receivers [r0, r0 + nrecv) must be staged (the
// first kRecvChunk of them) on entry.  Returns 0 if no sample reads the tile
// or nothing was drawn at a texel a sample reads.
template <int TS, bool PROF>
__device__ int tile_raster(TileSm<TS>& sm, const JobDev& J, const Buffers& B, const WaveDev* W, int ls, int tx,
                           int ty, int64_t te, uint64_t r0, int nrecv, bool limits_ready, unsigned int& visits,
                           unsigned int& writes, unsigned int& culled, unsigned int& cand, unsigned int& dense_n)
{
    constexpr int WPR = TS / 32;
    static_assert(SubGrid<TS>::side == 8, "sub-block index by shifts");
    const int tid = threadIdx.x, bd = blockDim.x;
    const int warp = tid >> 5, n_warps = bd >> 5;
    const int u24 = W->depth_u24;
    const LightParams& lp = B.lp[J.js_base + ls];
    const bool cull_ok = nrecv <= kRecvChunk;
    // samples reading the tile, at most (estimated from the staged receivers)
    const int64_t est = (int64_t)sm.total_items * J.n * ((nrecv + kRecvChunk - 1) / kRecvChunk);
    // dense only when the samples clearly outnumber the texels: marking costs
    // about as much per sample as a texel visit, and sparse tiles visit only
    // the texels that samples read
    const bool dense = est >= 2 * TS * TS;
    if (PROF && threadIdx.x == 0 && dense) ++dense_n;
    if (!limits_ready) tile_limits<TS>(sm, lp, u24, cull_ok);
    int n_need = TS * TS;
    if (!dense) {
        for (int q = tid; q < TS * WPR; q += bd) sm.mask[q] = 0u;
        __syncthreads();
        for (int c0 = 0; c0 < nrecv; c0 += kRecvChunk) {
            if (c0 > 0) stage_receivers<TS>(sm, J, B, ls, tx, ty, r0 + c0, min(kRecvChunk, nrecv - c0));
            for_tile_samples<TS, PROF>(
                sm.recv, sm.n_recv, sm.total_items, J, tx, ty, threadIdx.x, blockDim.x, cand,
                [&](const RecvSm&, int, int ix, int iy, float) {
                    atomicOr(&sm.mask[(iy & (TS - 1)) * WPR + ((ix & (TS - 1)) >> 5)], 1u << (ix & 31));
                },
                [&](const RecvSm&, int, int) {});
            __syncthreads();
        }
        if (nrecv > kRecvChunk) stage_receivers<TS>(sm, J, B, ls, tx, ty, r0, kRecvChunk);
        if (tid < 32) {
            unsigned int c = 0;
            for (int q = tid; q < TS * WPR; q += 32) c += __popc(sm.mask[q]);
            c = __reduce_add_sync(0xffffffffu, c);
            if (tid == 0) sm.n_need = (int)c;
        }
        __syncthreads();
        n_need = sm.n_need;
    }
    uint4* t4 = reinterpret_cast<uint4*>(sm.u.r.tile);
    for (int q = tid; q < TS * TS / 4; q += bd) t4[q] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
    if (tid == 0) sm.any_write = 0;
    __syncthreads();
    if (n_need == 0) return 0;
    bool wrote = false;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const uint64_t off = B.t_off[te];
    uint64_t cnt = B.t_cnt[te];
    const uint64_t cap = (uint64_t)W->bin_cap;
    if (off + cnt > cap) cnt = off < cap ? cap - off : 0;
    // triangles in batches of one per thread (at most kTriBatchMax): set-up,
    // then all warps share the batch's rows, one (triangle, row) per lane
    const int batch = min(bd, kTriBatchMax);
    for (uint64_t b0 = 0; b0 < cnt; b0 += batch) {
        const int nb = (int)min((uint64_t)batch, cnt - b0);
        if (tid < nb)
            sm.row_pref[tid] = setup_raster_tri<TS, PROF>(J, B, lp, ls, (int)B.bins[off + b0 + tid], ox, oy, sm.recv,
                                                          sm.n_recv, cull_ok, sm.dlim, sm.si, sm.tri[tid], culled);
        __syncthreads();
        if (tid < 32) warp_excl_scan_k<kTriBatchMax / 32>(sm.row_pref, nb);
        __syncthreads();
        // each warp takes a contiguous range of the batch's rows
        const int n_rows = sm.row_pref[nb];
        draw_rows<TS, PROF>(sm.tri, sm.row_pref, nb, (int)(((int64_t)n_rows * warp) / n_warps),
                            (int)(((int64_t)n_rows * (warp + 1)) / n_warps), dense ? nullptr : sm.mask, sm.u.r.tile,
                            lp, u24, wrote, visits, writes);
        __syncthreads();
    }
    if (wrote) sm.any_write = 1;
    __syncthreads();
    // no triangle reaches a texel that a sample reads: every sample is lit
    return sm.any_write ? n_need : 0;
}

// Add per-thread work counters to the global profile counters (warp-reduced).
__device__ __forceinline__ void flush_profile(const Buffers& B, unsigned int samples, unsigned int visits,
                                              unsigned int writes, unsigned int culled)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        samples += __shfl_xor_sync(0xffffffffu, samples, off);
        visits += __shfl_xor_sync(0xffffffffu, visits, off);
        writes += __shfl_xor_sync(0xffffffffu, writes, off);
        culled += __shfl_xor_sync(0xffffffffu, culled, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&B.ctr->prof_samples, (unsigned long long)samples);
        atomicAdd(&B.ctr->prof_visits, (unsigned long long)visits);
        atomicAdd(&B.ctr->prof_writes, (unsigned long long)writes);
        atomicAdd(&B.ctr->prof_culled, (unsigned long long)culled);
    }
}

__device__ __forceinline__ void flush_profile2(const Buffers& B, unsigned int cand, unsigned int tiles,
                                               unsigned int dense, unsigned int stiles, unsigned int pairs)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        cand += __shfl_xor_sync(0xffffffffu, cand, off);
        tiles += __shfl_xor_sync(0xffffffffu, tiles, off);
        dense += __shfl_xor_sync(0xffffffffu, dense, off);
        stiles += __shfl_xor_sync(0xffffffffu, stiles, off);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&B.ctr->prof_cand, (unsigned long long)cand);
        atomicAdd(&B.ctr->prof_tiles, (unsigned long long)tiles);
        atomicAdd(&B.ctr->prof_dense, (unsigned long long)dense);
        atomicAdd(&B.ctr->prof_stiles, (unsigned long long)stiles);
        atomicAdd(&B.ctr->prof_pairs, (unsigned long long)pairs);
    }
}

// The heavy-tile kernel's share of the work counters (also in the totals).
__device__ __forceinline__ void flush_heavy(const Buffers& B, unsigned int samples, unsigned int writes,
                                            unsigned int tiles)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        samples += __shfl_xor_sync(0xffffffffu, samples, off);
        writes += __shfl_xor_sync(0xffffffffu, writes, off);
        tiles += __shfl_xor_sync(0xffffffffu, tiles, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&B.ctr->prof_h_samples, (unsigned long long)samples);
        atomicAdd(&B.ctr->prof_h_writes, (unsigned long long)writes);
        atomicAdd(&B.ctr->prof_h_tiles, (unsigned long long)tiles);
    }
}

// Decode a non-empty tile entry.
__device__ __forceinline__ void decode_tile(const JobDev* jobs, int nj, uint32_t te, int& j, int& ls, int& tx,
                                            int& ty)
{
    j = job_of(nj, te, [&](int q) { return jobs[q].te_base; });
    const JobDev& J = jobs[j];
    const uint32_t lte = (uint32_t)(te - J.te_base);  // tile entries of a wave are numbered in 32 bits
    const uint32_t tps = (uint32_t)(J.tiles_x * J.tiles_x);
    ls = (int)(lte / tps);
    const uint32_t tl = lte - (uint32_t)ls * tps;
    ty = (int)(tl / (uint32_t)J.tiles_x);
    tx = (int)(tl - (uint32_t)ty * (uint32_t)J.tiles_x);
}

// Receivers of a tile entry, clamped to the receiver pool.
__device__ __forceinline__ void tile_receivers(const Buffers& B, const WaveDev* W, int64_t te, uint64_t& r0, int& n)
{
    r0 = B.t_roff[te];
    uint64_t r1 = r0 + B.t_rcnt[te];
    if (r1 > (uint64_t)W->recv_cap) r1 = (uint64_t)W->recv_cap;
    n = r1 > r0 ? (int)(r1 - r0) : 0;
}

// ---------------------------------------------------------------------------
// k_tile_warp: fused path -- one warp per non-empty tile: the depth test of
// every sample that reads the tile, sample by sample against the tile's kept
// triangles; shaded counts go to (step, cell).  A warp takes a tile with at
// most kWarpRecv receivers, kWarpBins binned (kWarpTri on 32-texel tiles,
// whose crowded tiles are rasterised anyway: handing them on before the keep
// loop saves the warp's set-up of triangles it would drop, measured on the
// tracker plant) and kWarpTri kept triangles; it lists any other tile for
// k_raster_test.  A tile is a small work item
// (hundreds of samples, a few triangles): one warp each keeps many tiles in
// flight per SM, which hides the chain of dependent loads that starts a tile.
// ---------------------------------------------------------------------------
constexpr int kWarpTri = 64;
constexpr int kWarpWords = kWarpTri / 32;
constexpr int kWarpRecv = 16;
constexpr int kWarpBins = 512;
constexpr int kTileWarps = 4;   // warps per block; 6 blocks per SM (80 registers a thread)

template <int TS, bool PROF>
struct WarpSm {
    KeptSm<TS, kWarpTri, PROF> k;
    RecvSm recv[kWarpRecv];
};

template <int TS, bool PROF>
__global__ void __launch_bounds__(kTileWarps * 32, 6) k_tile_warp(const WaveDev* __restrict__ W,
                                                                  const JobDev* __restrict__ jobs, Buffers B)
{
    __shared__ __align__(16) WarpSm<TS, PROF> sm_all[kTileWarps];
    unsigned int p_samples = 0, p_writes = 0, p_culled = 0, p_cand = 0, p_tiles = 0, p_stiles = 0, p_pairs = 0;
    unsigned int p_hr = 0, p_hb = 0, p_ht = 0;
    const int lane = threadIdx.x & 31;
    WarpSm<TS, PROF>& sm = sm_all[threadIdx.x >> 5];
    // the bins are incomplete when the pool overflowed: the wave is rerun
    // with a larger pool, so nothing here may read them
    const unsigned int n_ne = (B.ctr->overflow & 1u) ? 0u : B.ctr->n_nonempty;
    const int nj = W->n_jobs;
    const int want_bits = W->want_bits;
    const int u24 = W->depth_u24;
    const uint64_t bin_cap = (uint64_t)W->bin_cap;
    unsigned int next = 0;
    if (lane == 0) next = atomicAdd(&B.ctr->raster_next, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < n_ne) {
        const unsigned int item = next;
        if (lane == 0) next = atomicAdd(&B.ctr->raster_next, 1u);  // claim the following tile now
        const uint32_t te = B.nonempty[item];
        int j, ls, tx, ty;
        decode_tile(jobs, nj, te, j, ls, tx, ty);
        const JobDev& J = jobs[j];
        uint64_t r0;
        int nrecv;
        tile_receivers(B, W, te, r0, nrecv);
        const uint64_t off = B.t_off[te];
        uint64_t cnt = B.t_cnt[te];
        if (off + cnt > bin_cap) cnt = off < bin_cap ? bin_cap - off : 0;
        bool heavy = nrecv > kWarpRecv || cnt > (uint64_t)(TS == 32 ? kWarpTri : kWarpBins);
        if (PROF && lane == 0) {
            if (nrecv > kWarpRecv) ++p_hr;
            else if (heavy) ++p_hb;
        }
        if (!heavy) {
            const LightParams& lp = B.lp[J.js_base + ls];
            if (lane < nrecv) stage_one<TS>(sm.recv[lane], J, B, ls, tx, ty, (int)B.recv[r0 + lane]);
            if (PROF)
                for (int q = lane; q < TS * TS / 32; q += 32) sm.k.seen[q] = 0u;
            __syncwarp();
            const int c = lane < nrecv ? sm.recv[lane].item_pref : 0;
            const int inc = warp_incl_scan(c);
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            if (lane < nrecv) sm.recv[lane].item_pref = inc - c;
            sub_limits<TS>(sm.recv, nrecv, sm.k.dlim, u24 ? 1.f / lp.qscale : 0.f, lane, 32);
            __syncwarp();
            const float ox = (float)(tx * TS), oy = (float)(ty * TS);
            // strict keep (only the triangles that may shade a sample of some
            // sub-block, tri_sub_mask: fewer kept, tighter sub-block masks,
            // more set-up per triangle) on 32-texel tiles, whose samples are
            // dense over few texels, and on crowded tiles; otherwise the loose
            // keep (in front of some receiver's plane, covering a texel centre
            // of the tile), cheaper for the few large triangles of a 64- or
            // 128-texel tile (measured on the tracker plant and the facade)
            const bool strict = TS == 32 || cnt > (uint64_t)kWarpTri;
            SubInfo si{};
            if (strict) si = sub_summary(sm.k.dlim);
            int n = 0;
            for (uint64_t b0 = 0; b0 < cnt && n <= kWarpTri; b0 += 32) {
                TriS ts;
                uint32_t box = 0u;
                float dmin = 0.f;
                uint64_t smask = 0ull;
                const bool keep = b0 + lane < cnt &&
                                  setup_tri_s<TS, PROF>(J, B, lp, ls, (int)B.bins[off + b0 + lane], ox, oy, sm.recv,
                                                        nrecv, true, strict, sm.k.dlim, si, ts, box, dmin, smask,
                                                        p_culled);
                const unsigned int bal = __ballot_sync(0xffffffffu, keep);
                const int slot = n + __popc(bal & ((1u << lane) - 1u));
                if (keep && slot < kWarpTri) {
                    sm.k.tri[slot] = ts;
                    sm.k.box[slot] = box;
                    sm.k.dmin[slot] = dmin;
                    sm.k.smask[slot] = make_uint2((uint32_t)smask, (uint32_t)(smask >> 32));
                }
                n += __popc(bal);
            }
            heavy = n > kWarpTri;
            if (PROF && lane == 0 && heavy) ++p_ht;
            if (!heavy && n > 0) {
                __syncwarp();
                if (strict) build_sbm<kWarpWords>(sm.k.smask, sm.k.sbm, n, 0, 1);
                else sub_masks<TS, kWarpWords>(sm.k.tri, sm.k.box, sm.k.dmin, sm.k.dlim, sm.k.sbm, n, lane, 32);
                __syncwarp();
                const int C = J.n_cells;
                // sub-blocks in which some kept triangle may shade a sample
                uint32_t a0 = 0u, a1 = 0u;
                for (int w = 0; w < ((n + 31) >> 5); ++w) {
                    a0 |= sm.k.sbm[lane][w];
                    a1 |= sm.k.sbm[lane + 32][w];
                }
                const uint64_t cand_sb = (uint64_t)__ballot_sync(0xffffffffu, a0 != 0u) |
                                         ((uint64_t)__ballot_sync(0xffffffffu, a1 != 0u) << 32);
                test_items<TS, kWarpWords, PROF>(sm.recv, nrecv, total, J, lp, u24, tx, ty, lane, 32, sm.k.tri, n,
                                                 sm.k.sbm, (n + 31) >> 5, cand_sb, sm.k.seen,
                                                 B.cs_cnt, J.cs_base + (int64_t)ls * C,
                                                 B.cs_bits + J.cs_base + (int64_t)ls * C, want_bits, p_cand,
                                                 p_samples, p_pairs, p_writes);
            }
            if (PROF && lane == 0 && !heavy) { ++p_tiles; ++p_stiles; }
        }
        if (heavy && lane == 0) {
            const unsigned int pos = atomicAdd(&B.ctr->n_heavy, 1u);
            if (pos < (uint64_t)W->tot_te) B.heavy[pos] = te;
        }
        __syncwarp();  // the warp's shared memory may be reused
        next = __shfl_sync(0xffffffffu, next, 0);
    }
    if (PROF) {
        flush_profile(B, p_samples, 0u, p_writes, p_culled);
        flush_profile2(B, p_cand, p_tiles, 0u, p_stiles, p_pairs);
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            p_hr += __shfl_xor_sync(0xffffffffu, p_hr, off);
            p_hb += __shfl_xor_sync(0xffffffffu, p_hb, off);
            p_ht += __shfl_xor_sync(0xffffffffu, p_ht, off);
        }
        if (lane == 0) {
            atomicAdd(&B.ctr->prof_heavy_why[0], (unsigned long long)p_hr);
            atomicAdd(&B.ctr->prof_heavy_why[1], (unsigned long long)p_hb);
            atomicAdd(&B.ctr->prof_heavy_why[2], (unsigned long long)p_ht);
        }
    }
}

// ---------------------------------------------------------------------------
// k_raster_test: fused path, the tiles k_tile_warp listed (more receivers,
// binned or kept triangles than a warp takes) -- one CTA per tile.  On 64-
// and 128-texel tiles the binned triangles are first set up by the whole
// block, keeping those that may shade a sample of some sub-block
// (tri_sub_mask); with at most kMaxTri kept, every sample is tested against
// the kept triangles of its sub-block (few large triangles over sparse
// samples: most samples stop at their first occluder).  Otherwise, and always
// on 32-texel tiles, the tile is rasterised in shared memory (tile_raster:
// texel-centre coverage, atomicMin of order-preserving depth keys, only at
// the texels samples read and only where a triangle may shade) and the
// samples read it (many small triangles -- lattice members, grazing terrain
// -- each drawn once instead of tested by every sample near it; measured
// faster on the tracker plant for every kept count).  Both give the same
// decisions.
// ---------------------------------------------------------------------------

// Set up the tile's binned triangles that may shade a sample of a staged
// receiver (strict keep), for the whole block; the sub-block depth limits
// must be ready (tile_limits).  Returns how many were kept, or -1 if more than
// kMaxTri were.
template <int TS, bool PROF>
__device__ int setup_sample_tris(TileSm<TS>& sm, const JobDev& J, const Buffers& B, const WaveDev* W,
                                 const LightParams& lp, int ls, int tx, int ty, int64_t te, bool cull_ok,
                                 unsigned int& culled)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const uint64_t off = B.t_off[te];
    uint64_t cnt = B.t_cnt[te];
    const uint64_t cap = (uint64_t)W->bin_cap;
    if (off + cnt > cap) cnt = off < cap ? cap - off : 0;
    if (PROF)
        for (int q = tid; q < TS * TS / 32; q += blockDim.x) sm.u.s.seen[q] = 0u;
    if (tid == 0) sm.n_tri = 0;
    __syncthreads();
    const SubInfo si = sm.si;
    for (uint64_t b0 = 0; b0 < cnt; b0 += blockDim.x) {
        TriS ts;
        uint32_t box = 0u;
        float dmin = 0.f;
        uint64_t smask = 0ull;
        const bool keep = b0 + tid < cnt &&
                          setup_tri_s<TS, PROF>(J, B, lp, ls, (int)B.bins[off + b0 + tid], ox, oy, sm.recv,
                                                sm.n_recv, cull_ok, true, sm.dlim, si, ts, box, dmin, smask, culled);
        const unsigned int bal = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&sm.n_tri, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const int slot = base + __popc(bal & ((1u << lane) - 1u));
            if (slot < HeavyKept<TS>::n) {
                sm.u.s.tri[slot] = ts;
                sm.u.s.smask[slot] = make_uint2((uint32_t)smask, (uint32_t)(smask >> 32));
            }
        }
    }
    __syncthreads();
    const int n = sm.n_tri;
    return n > HeavyKept<TS>::n ? -1 : n;
}

template <int TS, bool PROF>
__global__ void __launch_bounds__(HeavyCfg<TS>::threads, HeavyCfg<TS>::min_blocks)
    k_raster_test(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs, Buffers B)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];  // sizeof(TileSm<TS>), set at launch
    TileSm<TS>& sm = *reinterpret_cast<TileSm<TS>*>(tile_smem);
    unsigned int p_samples = 0, p_visits = 0, p_writes = 0, p_culled = 0, p_cand = 0, p_dense = 0, p_tiles = 0;
    unsigned int p_stiles = 0, p_pairs = 0;
    __shared__ unsigned int s_item[2];
    // incomplete bins (pool overflow, the wave is rerun): nothing to read
    const unsigned int n_ne = (B.ctr->overflow & 1u) ? 0u : min(B.ctr->n_heavy, (unsigned int)W->tot_te);
    const int nj = W->n_jobs;
    const int u24 = W->depth_u24;
    const int want_bits = W->want_bits;
    const int tid = threadIdx.x;
    if (tid == 0) s_item[0] = atomicAdd(&B.ctr->heavy_next, 1u);
    __syncthreads();
    for (int par = 0;; par ^= 1) {
        // the next tile is claimed while this one runs; the barriers inside
        // the tile publish it
        const unsigned int item = s_item[par];
        if (item >= n_ne) break;
        if (tid == 0) s_item[par ^ 1] = atomicAdd(&B.ctr->heavy_next, 1u);
        const uint32_t te = B.heavy[item];
        int j, ls, tx, ty;
        decode_tile(jobs, nj, te, j, ls, tx, ty);
        const JobDev& J = jobs[j];
        uint64_t r0;
        int nrecv;
        tile_receivers(B, W, te, r0, nrecv);
        stage_receivers<TS>(sm, J, B, ls, tx, ty, r0, min(nrecv, kRecvChunk));
        if (PROF && tid == 0) ++p_tiles;
        const LightParams& lp = B.lp[J.js_base + ls];
        const int C = J.n_cells;
        const int64_t tally0 = J.cs_base + (int64_t)ls * C;
        unsigned long long* bits_row = B.cs_bits + J.cs_base + (int64_t)ls * C;
        const bool cull_ok = nrecv <= kRecvChunk;
        tile_limits<TS>(sm, lp, u24, cull_ok);
        // 32-texel tiles are always rasterised (dense samples over few
        // texels: each kept triangle drawn once beats every sample testing
        // it); larger tiles take the sample-driven test when at most kMaxTri
        // triangles are kept (few large triangles over sparse samples)
        const int nt = TS == 32 ? -1
                                : setup_sample_tris<TS, PROF>(sm, J, B, W, lp, ls, tx, ty, te, cull_ok, p_culled);
        const bool sample_driven = nt >= 0;
        if (sample_driven) {
            // sample-driven test (no triangle kept: every sample of the tile is lit)
            if (PROF && tid == 0) ++p_stiles;
            if (nt > 0) build_sbm<HeavyKept<TS>::words>(sm.u.s.smask, sm.u.s.sbm, nt, tid >> 5, blockDim.x >> 5);
            __syncthreads();
            for (int c0 = 0; nt > 0 && c0 < nrecv; c0 += kRecvChunk) {
                if (c0 > 0) {
                    __syncthreads();
                    stage_receivers<TS>(sm, J, B, ls, tx, ty, r0 + c0, min(kRecvChunk, nrecv - c0));
                }
                test_items<TS, HeavyKept<TS>::words, PROF>(sm.recv, sm.n_recv, sm.total_items, J, lp, u24, tx, ty, tid,
                                                blockDim.x, sm.u.s.tri, nt, sm.u.s.sbm, (nt + 31) >> 5, ~0ull,
                                                sm.u.s.seen, B.cs_cnt, tally0, bits_row, want_bits, p_cand, p_samples,
                                                p_pairs, p_writes);
            }
        } else if (tile_raster<TS, PROF>(sm, J, B, W, ls, tx, ty, te, r0, nrecv, true, p_visits, p_writes, p_culled,
                                         p_cand, p_dense) != 0) {
            for (int c0 = 0; c0 < nrecv; c0 += kRecvChunk) {
                if (c0 > 0) stage_receivers<TS>(sm, J, B, ls, tx, ty, r0 + c0, min(kRecvChunk, nrecv - c0));
                uint32_t cnt = 0;
                unsigned long long bits = 0ull;
                for_tile_samples<TS, PROF>(
                    sm.recv, sm.n_recv, sm.total_items, J, tx, ty, tid, blockDim.x, p_cand,
                    [&](const RecvSm& R, int k, int ix, int iy, float d) {
                        if (PROF) ++p_samples;
                        const uint32_t key = sm.u.r.tile[(iy & (TS - 1)) * TS + (ix & (TS - 1))];
                        if (key == kEmpty) return;
                        if (behind_key(d, R.s.bias, key, lp.dnear, lp.qscale, u24)) {
                            ++cnt;
                            if (k < 64) bits |= 1ull << k;
                        }
                    },
                    [&](const RecvSm& R, int cu, int cv) {
                        if (cnt) {
                            const int gcell = R.cell_base + cv * R.cu + cu;
                            tally_add(B.cs_cnt, tally0 + gcell, cnt);
                            if (want_bits) atomicOr(&bits_row[gcell], bits);
                        }
                        cnt = 0;
                        bits = 0ull;
                    });
                __syncthreads();
            }
        }
        __syncthreads();  // the tile's shared memory may be reused
    }
    if (PROF) {
        flush_profile(B, p_samples, p_visits, p_writes, p_culled);
        flush_profile2(B, p_cand, p_tiles, p_dense, p_stiles, p_pairs);
        flush_heavy(B, p_samples, p_writes, p_tiles);
    }
}

// ---------------------------------------------------------------------------
// k_raster_map: map path -- rasterise the tile and store it in HBM for the
// gather kernel (coalesced 16-byte stores)
// ---------------------------------------------------------------------------
template <int TS, bool PROF>
__global__ void __launch_bounds__(256) k_raster_map(const WaveDev* __restrict__ W,
                                                    const JobDev* __restrict__ jobs, Buffers B)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];  // sizeof(TileSm<TS>), set at launch
    TileSm<TS>& sm = *reinterpret_cast<TileSm<TS>*>(tile_smem);
    unsigned int p_visits = 0, p_writes = 0, p_culled = 0, p_cand = 0, p_dense = 0;
    __shared__ unsigned int s_item;
    // incomplete bins (pool overflow, the wave is rerun): nothing to read
    const unsigned int n_ne = (B.ctr->overflow & 1u) ? 0u : B.ctr->n_nonempty;
    const int64_t map_cap = W->map_cap_tiles;
    const int nj = W->n_jobs;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&B.ctr->raster_next, 1u);
        __syncthreads();
        const unsigned int item = s_item;
        __syncthreads();
        if (item >= n_ne || item >= map_cap) break;
        const uint32_t te = B.nonempty[item];
        int j, ls, tx, ty;
        decode_tile(jobs, nj, te, j, ls, tx, ty);
        const JobDev& J = jobs[j];
        uint64_t r0;
        int nrecv;
        tile_receivers(B, W, te, r0, nrecv);
        stage_receivers<TS>(sm, J, B, ls, tx, ty, r0, min(nrecv, kRecvChunk));
        // the tile is stored even when nothing was drawn: its samples read it
        tile_raster<TS, PROF>(sm, J, B, W, ls, tx, ty, te, r0, nrecv, false, p_visits, p_writes, p_culled, p_cand,
                              p_dense);
        const uint4* t4 = reinterpret_cast<const uint4*>(sm.u.r.tile);
        uint4* dst = reinterpret_cast<uint4*>(B.map + ((size_t)item * (TS * TS)));
        for (int q = tid; q < TS * TS / 4; q += bd) dst[q] = t4[q];
        __syncthreads();
    }
    if (PROF) flush_profile(B, 0u, p_visits, p_writes, p_culled);
}

// ---------------------------------------------------------------------------
// PV model per (step, module) from the cell tallies (Section 2, step 4)
// ---------------------------------------------------------------------------
constexpr int kPvThreads = 128;

// The diffuse shading fractions of local step ls: the row of its pose bin
// (tracked generators) or the generator's one row; nullptr when the diffuse
// term is not shaded.
__device__ __forceinline__ const float* diffuse_row(const JobDev& J, int ls)
{
    if (!J.fdiff) return nullptr;
    return J.fbin ? J.fdiff + (int64_t)J.fbin[J.step0 + ls] * J.fstride : J.fdiff;
}

// Irradiance per cell, substring currents, MPP over the bypass states.  All
// threads of the block call it with the cell counts in shared memory.
__device__ void module_pv(const JobDev& J, const ModuleDev& M, const ModStep& s, const LightParams& lp,
                          const uint32_t* s_cnt, uint32_t* s_imin, const Buffers& B, int64_t msi)
{
    const int ncell = M.cu * M.cv;
    const float beam = lp.dni * fmaxf(0.f, s.cosi);
    const float diff = lp.dhi * (1.f + s.nz) * 0.5f;
    const float inv_nn = 1.f / J.nn;
    const int* csub = J.lay_sub + J.lay_off[M.layout];
    const float* fd = diffuse_row(J, (int)((msi - J.ms_base) / J.n_mods));
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const float f = s_cnt[c] * inv_nn;
        const float gd = fd ? diff * (1.f - fd[M.cell_base + c]) : diff;
        const float G = beam * (1.f - f) + gd;
        const float I = J.i_ref * G * 1e-3f;
        atomicMin(&s_imin[csub[c]], __float_as_uint(I));  // I >= 0: uint order = float order
    }
    __syncthreads();
    if (J.n_str) {  // substring currents for the series-string model (k_string)
        const int ls = (int)((msi - J.ms_base) / J.n_mods);
        const int m = (int)(&M - J.mods);
        float* ss = B.ss_i + J.ss_base + (int64_t)ls * J.n_sub_tot + J.sub_base[m];
        for (int k = threadIdx.x; k < M.n_sub; k += blockDim.x) ss[k] = __uint_as_float(s_imin[k]);
        if (threadIdx.x == 0) B.ms_iu[msi] = J.i_ref * (beam + diff) * 1e-3f;
    }
    if (threadIdx.x == 0) {
        const int* nk = J.lay_nk + J.lay_nk_off[M.layout];
        const int ns = M.n_sub;
        float best = 0.f, vsum = 0.f;
        for (int k = 0; k < ns; ++k) {
            const float ik = __uint_as_float(s_imin[k]);
            float volt = 0.f;
            for (int q = 0; q < ns; ++q)
                volt += __uint_as_float(s_imin[q]) >= ik ? nk[q] * J.v_cell : -J.v_diode;
            best = fmaxf(best, ik * volt);
            vsum += nk[k] * J.v_cell;
        }
        B.ms_p[msi] = best;
        B.ms_pu[msi] = J.i_ref * (beam + diff) * 1e-3f * vsum;
        B.ms_beam[msi] = beam;
    }
}

__device__ __forceinline__ void zero_step_module(const JobDev& J, const ModuleDev& M, int ls, int64_t msi,
                                                 const Buffers& B)
{
    const int ncell = M.cu * M.cv, C = J.n_cells;
    const int64_t row = (int64_t)(J.out_row0 + ls);
    if (threadIdx.x == 0) { B.ms_p[msi] = 0.f; B.ms_pu[msi] = 0.f; B.ms_beam[msi] = 0.f; }
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        tally_set(B.cs_cnt, J.cs_base + (int64_t)ls * C + M.cell_base + c, 0u);
        if (J.out_counts) J.out_counts[row * J.out_cstride + M.cell_base + c] = 0;
        if (J.out_bits) J.out_bits[row * J.out_cstride + M.cell_base + c] = 0ull;
    }
}

// Fused path: the tallies were accumulated by the tile kernels.  The PV model
// of one (step, module) item by one warp: lanes over its cells into substring
// minima in shared memory, then over the candidate currents of the MPP.
// `imin` holds kMaxSub entries.
__device__ void pv_module_warp(const JobDev* jobs, int nj, int64_t item, const Buffers& B, uint32_t* imin)
{
    const int lane = threadIdx.x & 31;
    const int j = job_of(nj, item, [&](int q) { return jobs[q].it_mod; });
    const JobDev& J = jobs[j];
    const int64_t li = item - J.it_mod;
    const int ls = (int)(li / J.n_mods), m = (int)(li % J.n_mods);
    const int64_t msi = J.ms_base + li;
    const LightParams& lp = B.lp[J.js_base + ls];
    const ModuleDev& M = J.mods[m];
    const int ncell = M.cu * M.cv, C = J.n_cells;
    const int64_t row = (int64_t)(J.out_row0 + ls);
    const int64_t cbase = J.cs_base + (int64_t)ls * C + M.cell_base;
    if (!lp.valid) {
        if (lane == 0) { B.ms_p[msi] = 0.f; B.ms_pu[msi] = 0.f; B.ms_beam[msi] = 0.f; }
        for (int c = lane; c < ncell; c += 32) {
            tally_set(B.cs_cnt, cbase + c, 0u);
            if (J.out_counts) J.out_counts[row * J.out_cstride + M.cell_base + c] = 0;
            if (J.out_bits) J.out_bits[row * J.out_cstride + M.cell_base + c] = 0ull;
        }
        return;
    }
    const ModStep& s = B.ms[msi];
    const float beam = lp.dni * fmaxf(0.f, s.cosi);
    const float diff = lp.dhi * (1.f + s.nz) * 0.5f;
    const float inv_nn = 1.f / J.nn;
    const int* csub = J.lay_sub + J.lay_off[M.layout];
    const int ns = M.n_sub;
    for (int k = lane; k < ns; k += 32) imin[k] = 0x7F800000u;  // +inf
    __syncwarp();
    const float* fd = diffuse_row(J, ls);
    for (int c = lane; c < ncell; c += 32) {
        const uint32_t cnt = tally_get(B.cs_cnt, cbase + c);
        if (J.out_counts) J.out_counts[row * J.out_cstride + M.cell_base + c] = (uint8_t)cnt;
        if (J.out_bits) J.out_bits[row * J.out_cstride + M.cell_base + c] = B.cs_bits[cbase + c];
        const float gd = fd ? diff * (1.f - fd[M.cell_base + c]) : diff;
        const float G = beam * (1.f - cnt * inv_nn) + gd;
        const float I = J.i_ref * G * 1e-3f;
        atomicMin(&imin[csub[c]], __float_as_uint(I));  // I >= 0: uint order = float order
    }
    __syncwarp();
    if (J.n_str) {  // substring currents for the series-string model (k_string)
        float* ss = B.ss_i + J.ss_base + (int64_t)ls * J.n_sub_tot + J.sub_base[m];
        for (int k = lane; k < ns; k += 32) ss[k] = __uint_as_float(imin[k]);
        if (lane == 0) B.ms_iu[msi] = J.i_ref * (beam + diff) * 1e-3f;
    }
    const int* nk = J.lay_nk + J.lay_nk_off[M.layout];
    float best = 0.f, vsum = 0.f;
    for (int k = lane; k < ns; k += 32) {
        const float ik = __uint_as_float(imin[k]);
        float volt = 0.f;
        for (int q = 0; q < ns; ++q) volt += __uint_as_float(imin[q]) >= ik ? nk[q] * J.v_cell : -J.v_diode;
        best = fmaxf(best, ik * volt);
        vsum += nk[k] * J.v_cell;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
        vsum += __shfl_xor_sync(0xffffffffu, vsum, off);
    }
    if (lane == 0) {
        B.ms_p[msi] = best;
        B.ms_pu[msi] = J.i_ref * (beam + diff) * 1e-3f * vsum;
        B.ms_beam[msi] = beam;
    }
    __syncwarp();
}

// A warp takes bw consecutive (step, module) items, one per lane (bw = 32, or
// the smallest power of two that still covers the wave in one pass of the
// grid, so that small waves spread over all warps).  Each lane decodes its
// item (job, step, module, irradiance, cell layout); the warp then walks the
// items' cells one module at a time (lanes over its cells, the module's fields
// taken from its lane) into per-module substring minima in shared memory, and
// each lane evaluates its own module's MPP.  The arithmetic is that of
// pv_module_warp, operation for operation (a module's voltage sum is exact in
// either order), which the warp falls back to when one of its modules has
// more than kPvFastSub substrings.
constexpr int kPvWarps = kPvThreads / 32;
constexpr int kPvFastSub = 8;
constexpr int kPvUnroll = 4;
static_assert(32 * kPvFastSub >= kMaxSub, "the per-module path reuses the warp's minima");

__global__ void __launch_bounds__(kPvThreads) k_pv(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                                   Buffers B)
{
    __shared__ uint32_t s_imin[kPvWarps][32 * kPvFastSub];
    const int64_t tot = W->tot_mod;
    const int nj = W->n_jobs;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* imin = s_imin[wib];
    const int64_t n_warps = (int64_t)gridDim.x * kPvWarps;
    int bw = 32;
    while (bw > 1 && n_warps * (bw >> 1) >= tot) bw >>= 1;
    for (int64_t base = ((int64_t)blockIdx.x * kPvWarps + wib) * bw; base < tot; base += n_warps * bw) {
        const int64_t item = base + lane;
        const bool have = lane < bw && item < tot;
        int j = 0, ls = 0, m = 0, ncell = 0, ns = 0, cell0 = 0;
        int64_t msi = 0, cbase = 0;
        const int* csub = nullptr;
        bool lit = false;
        float beam = 0.f, diff = 0.f;
        if (have) {
            j = job_of(nj, item, [&](int q) { return jobs[q].it_mod; });
            const JobDev& J = jobs[j];
            const int64_t li = item - J.it_mod;
            ls = (int)(li / J.n_mods);
            m = (int)(li - (int64_t)ls * J.n_mods);
            msi = J.ms_base + li;
            const LightParams& lp = B.lp[J.js_base + ls];
            const ModuleDev& M = J.mods[m];
            ncell = M.cu * M.cv;
            ns = M.n_sub;
            cell0 = M.cell_base;
            cbase = J.cs_base + (int64_t)ls * J.n_cells + cell0;
            csub = J.lay_sub + J.lay_off[M.layout];
            lit = lp.valid != 0;
            if (lit) {
                const ModStep& s = B.ms[msi];
                beam = lp.dni * fmaxf(0.f, s.cosi);
                diff = lp.dhi * (1.f + s.nz) * 0.5f;
            }
        }
        if (__reduce_max_sync(0xffffffffu, ns) > kPvFastSub) {
            for (int q = 0; q < bw && base + q < tot; ++q) pv_module_warp(jobs, nj, base + q, B, imin);
            continue;
        }
        uint32_t* im = imin + lane * kPvFastSub;
        for (int k = 0; k < kPvFastSub; ++k) im[k] = 0x7F800000u;  // +inf
        if (bw == 32) {
            // a full batch: each lane walks its own module's cells (their
            // tallies are one byte each, consecutive per module: the warp's
            // lanes share the few cache lines of their modules), the
            // substring minima in its slice of shared memory
            if (have) {
                const JobDev& J = jobs[j];
                const int64_t row = (int64_t)(J.out_row0 + ls);
                if (!lit) {
                    for (int c = 0; c < ncell; ++c) {
                        tally_set(B.cs_cnt, cbase + c, 0u);
                        if (J.out_counts) J.out_counts[row * J.out_cstride + cell0 + c] = 0;
                        if (J.out_bits) J.out_bits[row * J.out_cstride + cell0 + c] = 0ull;
                    }
                } else {
                    const float* fd = diffuse_row(J, ls);
                    const float inv_nn = 1.f / J.nn;
                    for (int c = 0; c < ncell; ++c) {
                        const uint32_t cnt = tally_get(B.cs_cnt, cbase + c);
                        if (J.out_counts) J.out_counts[row * J.out_cstride + cell0 + c] = (uint8_t)cnt;
                        if (J.out_bits) J.out_bits[row * J.out_cstride + cell0 + c] = B.cs_bits[cbase + c];
                        const float gd = fd ? diff * (1.f - fd[cell0 + c]) : diff;
                        const float G = beam * (1.f - cnt * inv_nn) + gd;
                        const uint32_t I = __float_as_uint(J.i_ref * G * 1e-3f);  // I >= 0: uint order = float order
                        const int k = csub[c];
                        if (I < im[k]) im[k] = I;
                    }
                }
            }
        } else {
            // a short batch (a wave too small to fill the grid): the lanes
            // take the cells of one item after another, loads of 32 cells at
            // a time issued together before the minima are taken
            __syncwarp();
            for (unsigned int act = __ballot_sync(0xffffffffu, have); act; act &= act - 1u) {
                const int q = __ffs(act) - 1;
                const JobDev& J = jobs[__shfl_sync(0xffffffffu, j, q)];
                const int nc = __shfl_sync(0xffffffffu, ncell, q);
                const int c0 = __shfl_sync(0xffffffffu, cell0, q);
                const int64_t cb = __shfl_sync(0xffffffffu, cbase, q);
                const int* cs = reinterpret_cast<const int*>(
                    __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(csub), q));
                const int lsq = __shfl_sync(0xffffffffu, ls, q);
                const int64_t row = (int64_t)(J.out_row0 + lsq);
                const float* fd = diffuse_row(J, lsq);
                const bool litq = __shfl_sync(0xffffffffu, (int)lit, q) != 0;
                const float bq = __shfl_sync(0xffffffffu, beam, q), dq = __shfl_sync(0xffffffffu, diff, q);
                const float inv_nn = 1.f / J.nn;
                uint32_t* iq = imin + q * kPvFastSub;
                if (!litq) {
                    for (int c = lane; c < nc; c += 32) {
                        tally_set(B.cs_cnt, cb + c, 0u);
                        if (J.out_counts) J.out_counts[row * J.out_cstride + c0 + c] = 0;
                        if (J.out_bits) J.out_bits[row * J.out_cstride + c0 + c] = 0ull;
                    }
                    continue;
                }
                for (int cr = lane; cr < nc; cr += 32 * kPvUnroll) {
                    uint32_t cnt[kPvUnroll];
                    int sub[kPvUnroll];
#pragma unroll
                    for (int u = 0; u < kPvUnroll; ++u) {
                        const int c = cr + 32 * u;
                        cnt[u] = c < nc ? tally_get(B.cs_cnt, cb + c) : 0u;
                        sub[u] = c < nc ? cs[c] : 0;
                    }
#pragma unroll
                    for (int u = 0; u < kPvUnroll; ++u) {
                        const int c = cr + 32 * u;
                        if (c >= nc) continue;
                        if (J.out_counts) J.out_counts[row * J.out_cstride + c0 + c] = (uint8_t)cnt[u];
                        if (J.out_bits) J.out_bits[row * J.out_cstride + c0 + c] = B.cs_bits[cb + c];
                        const float gd = fd ? dq * (1.f - fd[c0 + c]) : dq;
                        const float G = bq * (1.f - cnt[u] * inv_nn) + gd;
                        const float I = J.i_ref * G * 1e-3f;
                        atomicMin(&iq[sub[u]], __float_as_uint(I));  // I >= 0: uint order = float order
                    }
                }
            }
        }
        __syncwarp();
        if (have) {
            const JobDev& J = jobs[j];
            if (!lit) {
                B.ms_p[msi] = 0.f;
                B.ms_pu[msi] = 0.f;
                B.ms_beam[msi] = 0.f;
            } else {
                const ModuleDev& M = J.mods[m];
                if (J.n_str) {  // substring currents for the series-string model (k_string)
                    float* ss = B.ss_i + J.ss_base + (int64_t)ls * J.n_sub_tot + J.sub_base[m];
                    for (int k = 0; k < ns; ++k) ss[k] = __uint_as_float(im[k]);
                    B.ms_iu[msi] = J.i_ref * (beam + diff) * 1e-3f;
                }
                const int* nk = J.lay_nk + J.lay_nk_off[M.layout];
                float best = 0.f, vsum = 0.f;
                for (int k = 0; k < ns; ++k) {
                    const float ik = __uint_as_float(im[k]);
                    float volt = 0.f;
                    for (int q = 0; q < ns; ++q) volt += __uint_as_float(im[q]) >= ik ? nk[q] * J.v_cell : -J.v_diode;
                    best = fmaxf(best, ik * volt);
                    vsum += nk[k] * J.v_cell;
                }
                B.ms_p[msi] = best;
                B.ms_pu[msi] = J.i_ref * (beam + diff) * 1e-3f * vsum;
                B.ms_beam[msi] = beam;
            }
        }
        __syncwarp();  // the warp's minima may be reset
    }
}

// ---------------------------------------------------------------------------
// k_sample: map path -- per (step, module) texel gathers from the HBM map,
// depth tests, warp-ballot cell tallies, then the PV model
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPvThreads) k_sample(const WaveDev* __restrict__ W,
                                                       const JobDev* __restrict__ jobs, Buffers B)
{
    __shared__ uint32_t s_cnt[kMaxCellsPerModule];
    __shared__ unsigned long long s_bits[kMaxCellsPerModule];
    __shared__ uint32_t s_imin[kMaxSub];
    const int64_t tot = W->tot_mod;
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int tmask = (1 << sh) - 1;
    const int64_t map_cap = W->map_cap_tiles;
    const int u24 = W->depth_u24;
    const int lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < tot; item += gridDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_mod; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.it_mod;
        const int ls = (int)(li / J.n_mods), m = (int)(li % J.n_mods);
        const int64_t msi = J.ms_base + li;
        const LightParams& lp = B.lp[J.js_base + ls];
        const ModuleDev& M = J.mods[m];
        if (!lp.valid) {
            zero_step_module(J, M, ls, msi, B);
            continue;
        }
        const int cu = M.cu, ncell = M.cu * M.cv;
        const int n = J.n, nn = J.nn;
        const int C = J.n_cells;
        const int64_t row = (int64_t)(J.out_row0 + ls);
        const ModStep s = B.ms[msi];
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) { s_cnt[c] = 0; s_bits[c] = 0ull; }
        if (threadIdx.x < kMaxSub) s_imin[threadIdx.x] = 0x7F800000u;
        __syncthreads();
        const int S = ncell * nn;
        const float p_over_n = __fdiv_rn(M.pitch, (float)n);
        const int R = J.R;
        const int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int g0 = 0; g0 < S; g0 += blockDim.x) {
            const int g = g0 + threadIdx.x;
            bool shaded = false;
            if (g < S) {
                int c = g / nn, k = g - c * nn;
                int jj = k / n, ii = k - jj * n;
                int cv_ = c / cu, cu_ = c - cv_ * cu;
                float d;
                int ix, iy;
                const int I = cu_ * n + ii;
                sample_texel(s, sample_row(s, cv_ * n + jj, p_over_n), (float)I + 0.5f, p_over_n,
                             (float)(R - 1), ix, iy, d);
                const int64_t te = te0 + (int64_t)(iy >> sh) * J.tiles_x + (ix >> sh);
                if (B.t_cnt[te] != 0u) {
                    const uint32_t slot = B.t_slot[te];
                    if (slot < map_cap) {
                        const uint32_t key = B.map[((size_t)slot << (2 * sh)) + ((iy & tmask) << sh) + (ix & tmask)];
                        if (key != kEmpty) shaded = behind_key(d, s.bias, key, lp.dnear, lp.qscale, u24);
                    }
                }
            }
            const unsigned int ball = __ballot_sync(0xffffffffu, shaded);
            if (lane == 0 && ball) {
                const int gw = g;  // first sample of this warp
                const int glast = min(gw + 31, S - 1);
                for (int c = gw / nn; c <= glast / nn; ++c) {
                    const int lo = max(c * nn, gw), hi = min((c + 1) * nn, glast + 1);
                    const unsigned int msk = (hi - lo >= 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
                    const unsigned int part = (ball >> (lo - gw)) & msk;
                    if (part) {
                        atomicAdd(&s_cnt[c], (uint32_t)__popc(part));
                        if (nn <= 64) atomicOr(&s_bits[c], (unsigned long long)part << (lo - c * nn));
                    }
                }
            }
        }
        __syncthreads();
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const uint32_t cnt = s_cnt[c];
            tally_set(B.cs_cnt, J.cs_base + (int64_t)ls * C + M.cell_base + c, cnt);
            if (J.out_counts) J.out_counts[row * J.out_cstride + M.cell_base + c] = (uint8_t)cnt;
            if (J.out_bits) J.out_bits[row * J.out_cstride + M.cell_base + c] = s_bits[c];
        }
        module_pv(J, M, s, lp, s_cnt, s_imin, B, msi);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_string: series strings (Section 2: the generator's modules wired in
// series strings, Fig. 2) -- one current through every bypass substring of
// every module of the string; P(I) = I (sum_{k: I_k >= I} V_k - v_diode
// #{k: I_k < I}) is linear between consecutive substring currents, so the
// string's maximum power point is the best of them.  One warp per (step,
// string): lanes over candidate currents, an inner loop over the string's
// substrings.  Without shading every substring of a module carries the
// module's unshaded current.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_string(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                                Buffers B)
{
    const int64_t tot = W->tot_sq;
    const int nj = W->n_jobs;
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < tot; item += n_warps) {
        const int j = job_of(nj, item, [&](int q) { return jobs[q].it_str; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.it_str;
        const int ls = (int)(li / J.n_str), q = (int)(li - (int64_t)ls * J.n_str);
        const int64_t sq = J.sq_base + li;
        const LightParams& lp = B.lp[J.js_base + ls];
        float best = 0.f, best_u = 0.f;
        if (lp.valid) {
            const int k0 = J.str_sub[q], k1 = J.str_sub[q + 1];
            const float* ik = B.ss_i + J.ss_base + (int64_t)ls * J.n_sub_tot;
            const float* iu = B.ms_iu + J.ms_base + (int64_t)ls * J.n_mods;
            for (int c = k0 + lane; c < k1; c += 32) {
                const float cur = ik[c], cur_u = iu[J.sub_mod[c]];
                float volt = 0.f, volt_u = 0.f;
                for (int k = k0; k < k1; ++k) {
                    const float vk = J.sub_nk[k] * J.v_cell;
                    volt += ik[k] >= cur ? vk : -J.v_diode;
                    volt_u += iu[J.sub_mod[k]] >= cur_u ? vk : -J.v_diode;
                }
                best = fmaxf(best, cur * volt);
                best_u = fmaxf(best_u, cur_u * volt_u);
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
                best_u = fmaxf(best_u, __shfl_xor_sync(0xffffffffu, best_u, off));
            }
        }
        if (lane == 0) {
            B.sq_p[sq] = best;
            B.sq_pu[sq] = best_u;
            const int64_t row = (int64_t)(J.out_row0 + ls);
            if (J.out_str_power) J.out_str_power[row * J.n_str + q] = best;
            if (J.out_str_power_u) J.out_str_power_u[row * J.n_str + q] = best_u;
        }
    }
}

// ---------------------------------------------------------------------------
// k_array: strings in parallel at one inverter input -- one voltage V across
// every string of the array; string s delivers the largest of its substring
// currents I_k whose string voltage V_s(I_k) = sum_{j: I_j >= I_k} V_j -
// v_diode #{j: I_j < I_k} still reaches V, and P(V) = V sum_s I_s(V) is
// linear between those voltages, so the array's maximum power point is the
// best of them.  One warp per (step, array): the array's substrings (current,
// string voltage at that current) staged in shared memory, then lanes over
// the candidate voltages.
// ---------------------------------------------------------------------------
constexpr int kArrayWarps = 4;

__global__ void __launch_bounds__(kArrayWarps * 32) k_array(const WaveDev* __restrict__ W,
                                                           const JobDev* __restrict__ jobs, Buffers B)
{
    __shared__ float s_i[kArrayWarps][kMaxArraySub], s_w[kArrayWarps][kMaxArraySub];
    __shared__ float s_iu[kArrayWarps][kMaxArraySub], s_wu[kArrayWarps][kMaxArraySub];
    __shared__ int s_str[kArrayWarps][kMaxArraySub];  // string of each staged substring (position in the array)
    const int64_t tot = W->tot_sa;
    const int nj = W->n_jobs;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * kArrayWarps;
    for (int64_t item = (int64_t)blockIdx.x * kArrayWarps + wib; item < tot; item += n_warps) {
        const int j = job_of(nj, item, [&](int q) { return jobs[q].sa_base; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.sa_base;
        const int ls = (int)(li / J.n_arr), a = (int)(li - (int64_t)ls * J.n_arr);
        const LightParams& lp = B.lp[J.js_base + ls];
        float best = 0.f, best_u = 0.f;
        if (lp.valid) {
            const float* ik = B.ss_i + J.ss_base + (int64_t)ls * J.n_sub_tot;
            const float* iu = B.ms_iu + J.ms_base + (int64_t)ls * J.n_mods;
            // stage the array's substrings string by string, with each one's string voltage
            int n = 0;
            for (int t = J.arr_off[a]; t < J.arr_off[a + 1]; ++t) {
                const int q = J.arr_strs[t];
                const int k0 = J.str_sub[q], k1 = J.str_sub[q + 1];
                for (int c = k0 + lane; c < k1; c += 32) {
                    const float cur = ik[c], cur_u = iu[J.sub_mod[c]];
                    float volt = 0.f, volt_u = 0.f;
                    for (int k = k0; k < k1; ++k) {
                        const float vk = J.sub_nk[k] * J.v_cell;
                        volt += ik[k] >= cur ? vk : -J.v_diode;
                        volt_u += iu[J.sub_mod[k]] >= cur_u ? vk : -J.v_diode;
                    }
                    const int pos = n + (c - k0);
                    if (pos < kMaxArraySub) {
                        s_i[wib][pos] = cur; s_w[wib][pos] = volt;
                        s_iu[wib][pos] = cur_u; s_wu[wib][pos] = volt_u;
                        s_str[wib][pos] = t;
                    }
                }
                n += k1 - k0;
            }
            n = min(n, kMaxArraySub);
            __syncwarp();
            for (int c = lane; c < n; c += 32) {
                const float V = s_w[wib][c], Vu = s_wu[wib][c];
                float cur = 0.f, cur_u = 0.f, is = 0.f, isu = 0.f;
                int prev = s_str[wib][0];
                for (int k = 0; k < n; ++k) {
                    if (s_str[wib][k] != prev) {  // next string: add the last one's current
                        cur += is; cur_u += isu;
                        is = 0.f; isu = 0.f;
                        prev = s_str[wib][k];
                    }
                    if (s_w[wib][k] >= V && s_i[wib][k] > is) is = s_i[wib][k];
                    if (s_wu[wib][k] >= Vu && s_iu[wib][k] > isu) isu = s_iu[wib][k];
                }
                cur += is; cur_u += isu;
                if (V > 0.f) best = fmaxf(best, V * cur);
                if (Vu > 0.f) best_u = fmaxf(best_u, Vu * cur_u);
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
                best_u = fmaxf(best_u, __shfl_xor_sync(0xffffffffu, best_u, off));
            }
            __syncwarp();
        }
        if (lane == 0) {
            B.sa_p[item] = best;
            B.sa_pu[item] = best_u;
            const int64_t row = (int64_t)(J.out_row0 + ls);
            if (J.out_arr_power) J.out_arr_power[row * J.n_arr + a] = best;
            if (J.out_arr_power_u) J.out_arr_power_u[row * J.n_arr + a] = best_u;
        }
    }
}

// ---------------------------------------------------------------------------
// sky map of the effective shading (Fig. 6: the shading factor over the sun's
// azimuth and zenith): k_gen_step sums the generator's power per step and
// bins the step's sun; k_heat adds each bin's steps in step order (FP64)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gen_step(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                                  Buffers B)
{
    const int64_t tot = W->tot_js;
    const int nj = W->n_jobs;
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t js = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; js < tot; js += n_warps) {
        const int j = job_of(nj, js, [&](int q) { return (int64_t)jobs[q].js_base; });
        const JobDev& J = jobs[j];
        if (J.heat_az == 0) continue;
        const int ls = (int)(js - J.js_base);
        float p = 0.f, pu = 0.f;
        for (int m = lane; m < J.n_mods; m += 32) {
            const int64_t msi = J.ms_base + (int64_t)ls * J.n_mods + m;
            p += B.ms_p[msi];
            pu += B.ms_pu[msi];
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, off);
            pu += __shfl_xor_sync(0xffffffffu, pu, off);
        }
        if (lane == 0) {
            B.js_p[js] = p;
            B.js_pu[js] = pu;
            const double* sp = J.sun + 3 * (size_t)(J.step0 + ls);
            int bin = -1;
            if (sp[2] > 0.0) {
                const double deg = 57.29577951308232;  // degrees per radian
                double az = atan2(sp[0], sp[1]) * deg;
                if (az < 0.0) az += 360.0;
                const double zen = acos(fmin(1.0, sp[2])) * deg;
                const int ia = min((int)(az / 360.0 * J.heat_az), J.heat_az - 1);
                const int iz = min((int)(zen / 90.0 * J.heat_zen), J.heat_zen - 1);
                bin = iz * J.heat_az + ia;
            }
            B.js_bin[js] = bin;
        }
    }
}

__global__ void __launch_bounds__(256) k_heat(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                              Buffers B)
{
    const int64_t tot = W->tot_heat;
    const int nj = W->n_jobs;
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int j = job_of(nj, item, [&](int q) { return jobs[q].it_heat; });
        const JobDev& J = jobs[j];
        const int bin = (int)(item - J.it_heat);
        double e = J.heat_e[bin], eu = J.heat_eu[bin];
        int cnt = J.heat_n[bin];
        for (int ls = 0; ls < J.k; ++ls) {
            const int64_t js = J.js_base + ls;
            if (B.js_bin[js] != bin) continue;
            const double dt = (double)B.lp[js].dt;
            e += (double)B.js_p[js] * dt;
            eu += (double)B.js_pu[js] * dt;
            ++cnt;
        }
        J.heat_e[bin] = e;
        J.heat_eu[bin] = eu;
        J.heat_n[bin] = cnt;
    }
}

// ---------------------------------------------------------------------------
// k_epilogue: Kahan sums over the wave's steps in step order
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kahan_add(float2& acc, float x)
{
    float y = x - acc.y;
    float t = acc.x + y;
    acc.y = (t - acc.x) - y;
    acc.x = t;
}

// One warp per item (cell, module or string): the lanes load 32 steps at a
// time, then every lane applies the same Kahan additions in step order from
// the shuffled values, so the sums equal a sequential loop over the steps
// while the loads of 32 steps overlap.
__global__ void __launch_bounds__(256) k_epilogue(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                                  Buffers B)
{
    const int64_t tot = W->tot_epi;
    const int nj = W->n_jobs;
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < tot; item += n_warps) {
        const int j = job_of(nj, item, [&](int q) { return jobs[q].it_epi; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.it_epi;
        // cell items only when the per-cell beam loss is wanted
        const int C = J.kahan_cell ? J.n_cells : 0, Mn = J.n_mods;
        const float inv_nn = 1.f / J.nn;
        // kind 0: cell c; 1: module m; 2: string q; 3: array
        const int kind = li < C ? 0 : (li < C + Mn ? 1 : (li < C + Mn + J.n_str ? 2 : 3));
        const int idx = kind == 0 ? (int)li
                                  : (kind == 1 ? (int)(li - C) : (kind == 2 ? (int)(li - C - Mn) : (int)(li - C - Mn - J.n_str)));
        const int m_cell = kind == 0 ? J.cell_mod[idx] : 0;
        float2 a, au = make_float2(0.f, 0.f);
        if (kind == 0) a = J.kahan_cell[idx];
        else if (kind == 1) { a = J.kahan_mod[2 * idx]; au = J.kahan_mod[2 * idx + 1]; }
        else if (kind == 2) { a = J.kahan_str[2 * idx]; au = J.kahan_str[2 * idx + 1]; }
        else { a = J.kahan_arr[2 * idx]; au = J.kahan_arr[2 * idx + 1]; }
        for (int l0 = 0; l0 < J.k; l0 += 32) {
            const int ls = l0 + lane;
            float x = 0.f, xu = 0.f;
            bool v = false;
            if (ls < J.k) {
                const LightParams& lp = B.lp[J.js_base + ls];
                v = lp.valid != 0;
                if (kind == 0) {
                    if (v) {
                        const float beam = B.ms_beam[J.ms_base + (int64_t)ls * Mn + m_cell];
                        const uint32_t cnt = tally_get(B.cs_cnt, J.cs_base + (int64_t)ls * C + idx);
                        x = beam * (cnt * inv_nn) * lp.dt;
                    }
                } else if (kind == 1) {
                    const int64_t msi = J.ms_base + (int64_t)ls * Mn + idx;
                    const float p = B.ms_p[msi], pu = B.ms_pu[msi];
                    if (J.out_power) J.out_power[(int64_t)(J.out_row0 + ls) * J.out_mstride + idx] = p;
                    if (J.out_power_u) J.out_power_u[(int64_t)(J.out_row0 + ls) * J.out_mstride + idx] = pu;
                    x = p * lp.dt;
                    xu = pu * lp.dt;
                } else if (v && kind == 2) {
                    const int64_t sq = J.sq_base + (int64_t)ls * J.n_str + idx;
                    x = B.sq_p[sq] * lp.dt;
                    xu = B.sq_pu[sq] * lp.dt;
                } else if (v) {
                    const int64_t sa = J.sa_base + (int64_t)ls * J.n_arr + idx;
                    x = B.sa_p[sa] * lp.dt;
                    xu = B.sa_pu[sa] * lp.dt;
                }
            }
            const unsigned int vm = __ballot_sync(0xffffffffu, v);
            const int n_here = min(32, J.k - l0);
            for (int q = 0; q < n_here; ++q) {
                const float xq = __shfl_sync(0xffffffffu, x, q);
                const float xuq = __shfl_sync(0xffffffffu, xu, q);
                if (!((vm >> q) & 1u)) continue;
                kahan_add(a, xq);
                if (kind != 0) kahan_add(au, xuq);
            }
        }
        if (lane == 0) {
            if (kind == 0) J.kahan_cell[idx] = a;
            else if (kind == 1) { J.kahan_mod[2 * idx] = a; J.kahan_mod[2 * idx + 1] = au; }
            else if (kind == 2) { J.kahan_str[2 * idx] = a; J.kahan_str[2 * idx + 1] = au; }
            else { J.kahan_arr[2 * idx] = a; J.kahan_arr[2 * idx + 1] = au; }
        }
    }
}

// Convert Kahan pairs (sum, compensation) to double results.
__global__ void k_finalize(const float2* __restrict__ kmod, int n_mods, const float2* __restrict__ kcell,
                           int n_cells, double* energy, double* energy_u, double* cell_loss)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_mods + n_cells; i += gridDim.x * blockDim.x) {
        if (i < n_mods) {
            const float2 e = kmod[2 * i], eu = kmod[2 * i + 1];
            if (energy) energy[i] = (double)e.x - (double)e.y;
            if (energy_u) energy_u[i] = (double)eu.x - (double)eu.y;
        } else {
            const int c = i - n_mods;
            const float2 h = kcell[c];
            if (cell_loss) cell_loss[c] = (double)h.x - (double)h.y;
        }
    }
}

// ---------------------------------------------------------------------------
// clear-sky sun table and ideal tracker poses, made on the device (the inputs
// of steps 3-4; the paper takes TMY data, measured series or an unnamed
// clear-sky model).  Solar time without longitude correction or equation of
// time; Cooper's (1969) declination; hour angle 15 deg per hour from noon;
// Meinel & Meinel's (1976) beam irradiance with Kasten & Young's (1989) air
// mass; all in FP64.
// ---------------------------------------------------------------------------
__global__ void k_sun_table(double lat_deg, int day_first, int64_t per_day, double step_h, double dhi_fraction,
                            int64_t n, double* __restrict__ xyz, float* __restrict__ dni, float* __restrict__ dhi,
                            float* __restrict__ dt, uint8_t* __restrict__ lit)
{
    const double deg = 0.017453292519943295;  // radians per degree
    const double phi = lat_deg * deg;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / per_day, k = i - d * per_day;
        const double day = (double)(day_first + d);
        const double delta = 23.45 * deg * sin(360.0 * deg * (284.0 + day) / 365.0);
        const double omega = 15.0 * deg * ((double)k * step_h - 12.0);
        double e = -cos(delta) * sin(omega);
        double no = sin(delta) * cos(phi) - cos(delta) * cos(omega) * sin(phi);
        double up = sin(delta) * sin(phi) + cos(delta) * cos(omega) * cos(phi);
        const double len = sqrt(e * e + no * no + up * up);
        e /= len; no /= len; up /= len;
        double b = 0.0;
        if (up > 0.0) {
            const double z = acos(up) / deg;
            const double am = 1.0 / (up + 0.50572 * pow(96.07995 - z, -1.6364));
            b = 1353.0 * pow(0.7, pow(am, 0.678));
        }
        xyz[3 * i] = e; xyz[3 * i + 1] = no; xyz[3 * i + 2] = up;
        dni[i] = (float)b;
        dhi[i] = (float)(dhi_fraction * b);
        dt[i] = (float)step_h;
        lit[i] = up > 0.0;
    }
}

__global__ void k_gather_sun(const int64_t* __restrict__ idx, int64_t n, const double* __restrict__ xyz,
                             const float* __restrict__ dni, const float* __restrict__ dhi, double* __restrict__ oxyz,
                             float* __restrict__ odni, float* __restrict__ odhi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx[i];
        oxyz[3 * i] = xyz[3 * k]; oxyz[3 * i + 1] = xyz[3 * k + 1]; oxyz[3 * i + 2] = xyz[3 * k + 2];
        odni[i] = dni[k];
        odhi[i] = dhi[k];
    }
}

// Diffuse shading: sky patches of equal zenith bands and azimuth sectors at
// their centre directions, solid angle (cos z0 - cos z1) 2 pi / sectors.
__global__ void k_sky_patches(int rings, int sectors, double* __restrict__ xyz, float* __restrict__ dni,
                              float* __restrict__ dhi, float* __restrict__ dt, double* __restrict__ dom)
{
    const double half_pi = 1.5707963267948966, two_pi = 6.283185307179586;
    const int n = rings * sectors;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i / sectors, k = i - r * sectors;
        const double z0 = half_pi * r / rings, z1 = half_pi * (r + 1) / rings;
        const double zc = 0.5 * (z0 + z1);
        const double a = two_pi * (k + 0.5) / sectors;
        xyz[3 * i] = sin(zc) * sin(a);
        xyz[3 * i + 1] = sin(zc) * cos(a);
        xyz[3 * i + 2] = cos(zc);
        dni[i] = 1.f;
        dhi[i] = 0.f;
        dt[i] = 1.f;
        dom[i] = (cos(z0) - cos(z1)) * two_pi / sectors;
    }
}

// Per cell: f = sum_p W_p s_p / sum_p W_p, W_p = solid angle x max(0, n . w_p)
// with the module's front normal n (a tracked module's at the pose (az,
// tilt) of the sky view: R = Rz(pi - az) Rx(tilt)), s_p = shaded samples
// toward patch p / n^2 (counts[p][c]); summed in patch order in FP64.
__global__ void k_sky_fraction(const ModuleDev* __restrict__ mods, const int32_t* __restrict__ cell_mod, int n_cells,
                               const double* __restrict__ xyz, const double* __restrict__ dom, int n_patch,
                               const uint8_t* __restrict__ counts, int nn, float* __restrict__ fdiff, double az,
                               double tilt)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const ModuleDev& M = mods[cell_mod[c]];
        double nx = (double)M.u[1] * M.v[2] - (double)M.u[2] * M.v[1];
        double ny = (double)M.u[2] * M.v[0] - (double)M.u[0] * M.v[2];
        double nz = (double)M.u[0] * M.v[1] - (double)M.u[1] * M.v[0];
        const double l = sqrt(nx * nx + ny * ny + nz * nz);
        nx /= l; ny /= l; nz /= l;
        if (M.tracker >= 0) {
            const double cb = cos(tilt), sb = sin(tilt), cg = -cos(az), sg = sin(az);
            const double yy = cb * ny - sb * nz, zz = sb * ny + cb * nz;
            const double xx = nx;
            nx = cg * xx - sg * yy;
            ny = sg * xx + cg * yy;
            nz = zz;
        }
        double num = 0.0, den = 0.0;
        for (int p = 0; p < n_patch; ++p) {
            const double w = dom[p] * fmax(0.0, nx * xyz[3 * p] + ny * xyz[3 * p + 1] + nz * xyz[3 * p + 2]);
            den += w;
            num += w * ((double)counts[(size_t)p * n_cells + c] / (double)nn);
        }
        fdiff[c] = den > 0.0 ? (float)(num / den) : 0.f;
    }
}

__global__ void k_ideal_poses(const double* __restrict__ sun, int64_t n_steps, int n_trk, float tilt_max,
                              float* __restrict__ poses)
{
    const int64_t n = n_steps * n_trk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / n_trk;
        const double* sp = sun + 3 * s;
        poses[2 * i] = (float)atan2(sp[0], sp[1]);
        poses[2 * i + 1] = fminf((float)acos(fmin(1.0, fmax(-1.0, sp[2]))), tilt_max);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline unsigned int grid_for(int64_t items, int per_block, int cap)
{
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned int)g;
}

// Blocks of the block-per-tile kernels per SM (their shared tile is dynamic:
// TileSm<128> holds a 64 KB depth tile).
template <int TS>
constexpr int tile_blocks() { return TS == 128 ? 2 : 4; }

template <int TS, bool PROF>
static cudaError_t allow_tile_smem()
{
    const int bytes = (int)sizeof(TileSm<TS>);
    cudaError_t e = cudaFuncSetAttribute(k_raster_test<TS, PROF>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_raster_map<TS, PROF>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t prepare_tile_kernels()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = allow_tile_smem<32, false>();
    if (e == cudaSuccess) e = allow_tile_smem<32, true>();
    if (e == cudaSuccess) e = allow_tile_smem<64, false>();
    if (e == cudaSuccess) e = allow_tile_smem<64, true>();
    if (e == cudaSuccess) e = allow_tile_smem<128, false>();
    if (e == cudaSuccess) e = allow_tile_smem<128, true>();
    return e;
}

template <int TS, bool PROF>
static void launch_tile_kernels(const WaveDev* W, const JobDev* d_jobs, const Buffers& b, const LaunchCfg& cfg)
{
    const int sm = cfg.sm_count;
    const size_t tsm = sizeof(TileSm<TS>);
    if (cfg.fused) {
        k_tile_warp<TS, PROF><<<sm * 6, kTileWarps * 32, 0, cfg.stream>>>(W, d_jobs, b);
        if (cfg.ev) cudaEventRecord(cfg.ev[3], cfg.stream);
        k_raster_test<TS, PROF><<<sm * (TS == 32 ? HeavyCfg<TS>::min_blocks : tile_blocks<TS>()), HeavyCfg<TS>::threads,
                                   tsm, cfg.stream>>>(W, d_jobs, b);
    } else {
        k_raster_map<TS, PROF><<<sm * tile_blocks<TS>(), 256, tsm, cfg.stream>>>(W, d_jobs, b);
        if (cfg.ev) cudaEventRecord(cfg.ev[3], cfg.stream);
    }
}

cudaError_t launch_wave(const WaveDev* d_wave, const JobDev* d_jobs, const Buffers& b, const LaunchCfg& cfg,
                        int64_t tot_te_host)
{
    const WaveDev* W = d_wave;
    cudaStream_t st = cfg.stream;
    const int sm = cfg.sm_count;
    (void)tot_te_host;
    if (cfg.ev) cudaEventRecord(cfg.ev[0], st);
    k_clear<<<sm * 8, 256, 0, st>>>(W, b);
    k_window<<<sm * 8, kWinPerItem, 0, st>>>(W, d_jobs, b);
    k_light<<<sm, 128, 0, st>>>(W, d_jobs, b);
    k_modsetup<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    if (cfg.ev) cudaEventRecord(cfg.ev[1], st);
    k_bin<<<sm * 16, 256, 0, st>>>(W, d_jobs, b);
    k_bin_big<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    k_scan_a<<<sm * 2, kScanThreads, 0, st>>>(W, b);
    k_scan_b<<<1, kScanThreads, 0, st>>>(W, b);
    k_scan_c<<<sm * 2, kScanThreads, 0, st>>>(W, b);
    k_scatter<<<sm * 8, 256, 0, st>>>(W, b);
    k_recv_fill<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    if (cfg.ev) cudaEventRecord(cfg.ev[2], st);
    if (cfg.tile == 32) {
        if (cfg.profile) launch_tile_kernels<32, true>(W, d_jobs, b, cfg);
        else launch_tile_kernels<32, false>(W, d_jobs, b, cfg);
    } else if (cfg.tile == 64) {
        if (cfg.profile) launch_tile_kernels<64, true>(W, d_jobs, b, cfg);
        else launch_tile_kernels<64, false>(W, d_jobs, b, cfg);
    } else {
        if (cfg.profile) launch_tile_kernels<128, true>(W, d_jobs, b, cfg);
        else launch_tile_kernels<128, false>(W, d_jobs, b, cfg);
    }
    if (cfg.ev) cudaEventRecord(cfg.ev[4], st);
    if (cfg.fused) k_pv<<<sm * 32, kPvThreads, 0, st>>>(W, d_jobs, b);
    else k_sample<<<sm * 16, kPvThreads, 0, st>>>(W, d_jobs, b);
    if (cfg.extras & 1) k_string<<<sm * 4, 256, 0, st>>>(W, d_jobs, b);
    if (cfg.extras & 4) k_array<<<sm * 4, kArrayWarps * 32, 0, st>>>(W, d_jobs, b);
    if (cfg.extras & 2) {
        k_gen_step<<<sm * 4, 256, 0, st>>>(W, d_jobs, b);
        k_heat<<<sm * 2, 256, 0, st>>>(W, d_jobs, b);
    }
    if (cfg.ev) cudaEventRecord(cfg.ev[5], st);
    k_epilogue<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    if (cfg.ev) cudaEventRecord(cfg.ev[6], st);
    return cudaGetLastError();
}

cudaError_t launch_sun_table(double lat_deg, int day_first, int64_t per_day, double step_h, double dhi_fraction,
                             int64_t n, double* xyz, float* dni, float* dhi, float* dt, uint8_t* lit, cudaStream_t st)
{
    k_sun_table<<<grid_for(n, 256, 4096), 256, 0, st>>>(lat_deg, day_first, per_day, step_h, dhi_fraction, n, xyz, dni,
                                                          dhi, dt, lit);
    return cudaGetLastError();
}

cudaError_t launch_gather_sun(const int64_t* idx, int64_t n, const double* xyz, const float* dni, const float* dhi,
                              double* oxyz, float* odni, float* odhi, cudaStream_t st)
{
    k_gather_sun<<<grid_for(n, 256, 4096), 256, 0, st>>>(idx, n, xyz, dni, dhi, oxyz, odni, odhi);
    return cudaGetLastError();
}

cudaError_t launch_sky_patches(int rings, int sectors, double* xyz, float* dni, float* dhi, float* dt, double* dom,
                               cudaStream_t st)
{
    k_sky_patches<<<grid_for((int64_t)rings * sectors, 256, 1024), 256, 0, st>>>(rings, sectors, xyz, dni, dhi, dt,
                                                                                 dom);
    return cudaGetLastError();
}

cudaError_t launch_sky_fraction(const ModuleDev* mods, const int32_t* cell_mod, int n_cells, const double* xyz,
                                const double* dom, int n_patch, const uint8_t* counts, int nn, float* fdiff,
                                double az, double tilt, cudaStream_t st)
{
    k_sky_fraction<<<grid_for(n_cells, 128, 4096), 128, 0, st>>>(mods, cell_mod, n_cells, xyz, dom, n_patch, counts,
                                                                  nn, fdiff, az, tilt);
    return cudaGetLastError();
}

cudaError_t launch_ideal_poses(const double* sun, int64_t n_steps, int n_trk, float tilt_max, float* poses,
                               cudaStream_t st)
{
    k_ideal_poses<<<grid_for(n_steps * n_trk, 256, 4096), 256, 0, st>>>(sun, n_steps, n_trk, tilt_max, poses);
    return cudaGetLastError();
}

cudaError_t launch_finalize_pairs(const float2* kmod, int n_mods, const float2* kcell, int n_cells,
                                  double* energy, double* energy_u, double* cell_loss, cudaStream_t st)
{
    int n = n_mods + n_cells;
    k_finalize<<<grid_for(n, 256, 1024), 256, 0, st>>>(kmod, n_mods, kcell, n_cells, energy, energy_u, cell_loss);
    return cudaGetLastError();
}

}  // namespace pv3d
