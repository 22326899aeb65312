// kernels.cu -- the GB300 hot path of the 3DPV shadow-sample method.
//
// Per wave (a chunk of sun steps of one or more jobs), in stream order:
//   k_window      light window: bounding box of every module corner projected
//                 on the sun's light plane (Section 2, step 3: orthographic view
//                 from the sun, field of view limited to the generator)
//   k_light       light frame, texel size and origin per (job, step)
//   k_modsetup    each module at each step in texel space; marks the raster
//                 tiles that hold samples and their far plane (max sample depth
//                 + bias) -- only those tiles are rasterised
//   k_bin<0>      count (triangle, tile) pairs: vertex transform batched over
//                 the job's steps (one read of a triangle serves k steps), cull
//                 against occupied tiles and their far planes
//   k_bin_big<0>  same for triangles that span many tiles, one warp each
//   k_scan_*      bin offsets and the list of non-empty tiles (= map slots)
//   k_bin<1>, k_bin_big<1>  write the bins
//   k_raster      one CTA per non-empty tile: shared-memory depth tile, texel-
//                 centre coverage, atomicMin of order-preserving depth keys,
//                 coalesced 16-byte stores of the finished tile (Fig. 3: the
//                 depth buffer keeps the surface nearest the sun)
//   k_sample      one CTA per (step, module): analytic sample positions, texel
//                 gather, depth test with slope-scaled bias, warp-ballot cell
//                 tallies, substring minima and the bypass-diode MPP (step 4)
//   k_epilogue    Kahan-compensated FP32 sums over the wave's steps in step
//                 order, per module (energy) and per cell (beam loss)
#include <cfloat>
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
// k_modsetup: module frames in texel space, bias, tile occupancy and far planes
// ---------------------------------------------------------------------------
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
        const LightParams lp = B.lp[js];
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
        // occupied tiles: bounding box of the corners in texel space
        float lu = M.cu * M.pitch, lv = M.cv * M.pitch;
        float xmin = FLT_MAX, xmax = -FLT_MAX, ymin = FLT_MAX, ymax = -FLT_MAX, dmax = -FLT_MAX;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float a = (k == 1 || k == 2) ? lu : 0.f;
            float b = (k >= 2) ? lv : 0.f;
            float x = s.tx0 + a * s.tax + b * s.tbx;
            float y = s.ty0 + a * s.tay + b * s.tby;
            float d = s.d0 + a * s.da + b * s.db;
            xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
            ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
            dmax = fmaxf(dmax, d);
        }
        int R = J.R;
        int ix0 = max(0, min(R - 1, (int)floorf(xmin))), ix1 = max(0, min(R - 1, (int)floorf(xmax)));
        int iy0 = max(0, min(R - 1, (int)floorf(ymin))), iy1 = max(0, min(R - 1, (int)floorf(ymax)));
        uint32_t far_key = u24 ? depth_store_key(dmax + s.bias, lp, 1) + 1u : okey(dmax + s.bias);
        int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int ty = iy0 >> sh; ty <= (iy1 >> sh); ++ty)
            for (int tx = ix0 >> sh; tx <= (ix1 >> sh); ++tx)
                atomicMax(&B.t_far[te0 + (int64_t)ty * J.tiles_x + tx], far_key);
    }
}

// ---------------------------------------------------------------------------
// triangles in texel space
// ---------------------------------------------------------------------------
struct TriT {
    float x[3], y[3], d[3];
};

// Triangle `t` of job J (scene triangle, or module triangle after the scene's)
// at local step ls in texel coordinates.
__device__ __forceinline__ void tri_texel(const JobDev& J, const Buffers& B, const LightParams& lp,
                                          int ls, int t, TriT& T)
{
    if (t < J.n_tris) {
        const float4* p = J.tri + 3 * (size_t)t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 q = __ldg(p + k);
            float x = q.x - J.ref[0], y = q.y - J.ref[1], z = q.z - J.ref[2];
            T.x[k] = (x * lp.ux + y * lp.uy + z * lp.uz - lp.u0) * lp.inv_delta;
            T.y[k] = (x * lp.vx + y * lp.vy + z * lp.vz - lp.v0) * lp.inv_delta;
            T.d[k] = -(x * lp.sx + y * lp.sy + z * lp.sz);
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
        T.x[1] = s.tx0 + a1 * s.tax + b1 * s.tbx;
        T.y[1] = s.ty0 + a1 * s.tay + b1 * s.tby;
        T.d[1] = s.d0 + a1 * s.da + b1 * s.db;
        T.x[2] = s.tx0 + a2 * s.tax + b2 * s.tbx;
        T.y[2] = s.ty0 + a2 * s.tay + b2 * s.tby;
        T.d[2] = s.d0 + a2 * s.da + b2 * s.db;
    }
}

// Edge functions of a counter-clockwise triangle: E_k(p) = A_k px + B_k py + C_k,
// inside iff every E_k >= 0.  Returns false for a degenerate (edge-on) triangle.
struct Edges {
    float A[3], Bc[3], C[3];
    float area2;
};

__device__ __forceinline__ bool make_edges(TriT& T, Edges& e)
{
    float area2 = (T.x[1] - T.x[0]) * (T.y[2] - T.y[0]) - (T.y[1] - T.y[0]) * (T.x[2] - T.x[0]);
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
        e.A[k] = -(T.y[b] - T.y[a]);
        e.Bc[k] = T.x[b] - T.x[a];
        e.C[k] = -(e.A[k] * T.x[a] + e.Bc[k] * T.y[a]);
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
// k_bin<FILL>: (triangle, tile) pairs, vertex transform batched over steps
// ---------------------------------------------------------------------------
template <int FILL>
__device__ __forceinline__ void bin_tile(const Buffers& B, int64_t te, uint32_t dkey, uint32_t tri,
                                         const WaveDev* W)
{
    uint32_t far = B.t_far[te];
    if (!(dkey < far)) return;  // unoccupied tile (far 0) or triangle wholly behind
    if (FILL == 0) {
        atomicAdd(&B.t_cnt[te], 1u);
    } else {
        uint32_t pos = atomicAdd(&B.t_cur[te], 1u);
        if (pos < (uint64_t)W->bin_cap) B.bins[pos] = tri;
    }
}

template <int FILL>
__global__ void __launch_bounds__(256) k_bin(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                             Buffers B)
{
    // item = (triangle, step) with the step fastest: the lanes of a warp take
    // consecutive sun steps of one triangle, so its three vertices are read
    // once (a broadcast load) and transformed for up to 32 steps.
    const int64_t tot = W->tot_tri;
    const int nj = W->n_jobs;
    const int sh = W->tile_sh;
    const int TS = 1 << sh;
    const int u24 = W->depth_u24;
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_tri; });
        const JobDev& J = jobs[j];
        const int64_t li = item - J.it_tri;
        const int t = (int)(li / J.k), ls = (int)(li - (int64_t)t * J.k);
        const int R = J.R;
        const int64_t js = J.js_base + ls;
        const LightParams& lp = B.lp[js];
        if (!lp.valid) continue;
        TriT T;
        tri_texel(J, B, lp, ls, t, T);
        Edges e;
        if (!make_edges(T, e)) continue;
        float xmin = fminf(T.x[0], fminf(T.x[1], T.x[2])), xmax = fmaxf(T.x[0], fmaxf(T.x[1], T.x[2]));
        float ymin = fminf(T.y[0], fminf(T.y[1], T.y[2])), ymax = fmaxf(T.y[0], fmaxf(T.y[1], T.y[2]));
        // covered texel centres (ix + 0.5) lie in [xmin, xmax]
        if (!(xmax >= 0.5f && ymax >= 0.5f && xmin <= R - 0.5f && ymin <= R - 0.5f)) continue;
        int ix0 = max(0, (int)ceilf(xmin - 0.5f)), ix1 = min(R - 1, (int)floorf(xmax - 0.5f));
        int iy0 = max(0, (int)ceilf(ymin - 0.5f)), iy1 = min(R - 1, (int)floorf(ymax - 0.5f));
        if (ix0 > ix1 || iy0 > iy1) continue;
        float dmin = fminf(T.d[0], fminf(T.d[1], T.d[2]));
        uint32_t dkey = depth_store_key(dmin, lp, u24);
        int tx0 = ix0 >> sh, tx1 = ix1 >> sh, ty0 = iy0 >> sh, ty1 = iy1 >> sh;
        int ntiles = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
        if (ntiles > kBigTiles) {
            if (FILL == 0) {
                unsigned int pos = atomicAdd(&B.ctr->n_big, 1u);
                if (pos < (uint64_t)W->big_cap) B.big[pos] = make_uint2((uint32_t)t, (uint32_t)js);
            }
            continue;
        }
        int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int ty = ty0; ty <= ty1; ++ty) {
            for (int tx = tx0; tx <= tx1; ++tx) {
                if (ntiles > 1 &&
                    !rect_overlap(e, tx * TS + 0.5f, tx * TS + TS - 0.5f, ty * TS + 0.5f, ty * TS + TS - 0.5f))
                    continue;
                bin_tile<FILL>(B, te0 + (int64_t)ty * J.tiles_x + tx, dkey, (uint32_t)t, W);
            }
        }
    }
}

// Triangles spanning more than kBigTiles tiles: one warp per triangle.
template <int FILL>
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
        int tx0 = ix0 >> sh, tx1 = ix1 >> sh, ty0 = iy0 >> sh, ty1 = iy1 >> sh;
        int wx = tx1 - tx0 + 1;
        int ntiles = wx * (ty1 - ty0 + 1);
        int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int q = lane; q < ntiles; q += 32) {
            int tx = tx0 + q % wx, ty = ty0 + q / wx;
            if (!rect_overlap(ed, tx * TS + 0.5f, tx * TS + TS - 0.5f, ty * TS + 0.5f, ty * TS + TS - 0.5f))
                continue;
            bin_tile<FILL>(B, te0 + (int64_t)ty * J.tiles_x + tx, dkey, (uint32_t)t, W);
        }
    }
}

// ---------------------------------------------------------------------------
// scan over the wave's tile entries: bin offsets, non-empty tile list
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

// Block-wide exclusive scan of (a, b) pairs; returns the block totals.
__device__ __forceinline__ void block_scan2(unsigned long long& a, unsigned long long& b,
                                            unsigned long long& tot_a, unsigned long long& tot_b)
{
    __shared__ unsigned long long wa[32], wb[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long ia = a, ib = b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned long long ya = __shfl_up_sync(0xffffffffu, ia, off);
        unsigned long long yb = __shfl_up_sync(0xffffffffu, ib, off);
        if (lane >= off) { ia += ya; ib += yb; }
    }
    if (lane == 31) { wa[w] = ia; wb[w] = ib; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        unsigned long long xa = lane < nw ? wa[lane] : 0ull, xb = lane < nw ? wb[lane] : 0ull;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long ya = __shfl_up_sync(0xffffffffu, xa, off);
            unsigned long long yb = __shfl_up_sync(0xffffffffu, xb, off);
            if (lane >= off) { xa += ya; xb += yb; }
        }
        if (lane < nw) { wa[lane] = xa; wb[lane] = xb; }
    }
    __syncthreads();
    unsigned long long pa = w ? wa[w - 1] : 0ull, pb = w ? wb[w - 1] : 0ull;
    tot_a = wa[(blockDim.x >> 5) - 1];
    tot_b = wb[(blockDim.x >> 5) - 1];
    a = pa + ia - a;
    b = pb + ib - b;
    __syncthreads();
}

__global__ void __launch_bounds__(kScanThreads) k_scan_a(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    for (int64_t st = blockIdx.x; st < n_tiles; st += gridDim.x) {
        unsigned long long a = 0, b = 0;
        int64_t base = st * kScanTile + (int64_t)threadIdx.x * kScanPer;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            int64_t i = base + q;
            if (i < tot) {
                uint32_t c = B.t_cnt[i];
                a += c;
                b += c ? 1u : 0u;
            }
        }
        unsigned long long ta, tb;
        block_scan2(a, b, ta, tb);
        if (threadIdx.x == 0) {
            B.block_sums[2 * st] = ta;
            B.block_sums[2 * st + 1] = tb;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_b(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    unsigned long long carry_a = 0, carry_b = 0;
    for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        unsigned long long a = i < n_tiles ? B.block_sums[2 * i] : 0ull;
        unsigned long long b = i < n_tiles ? B.block_sums[2 * i + 1] : 0ull;
        unsigned long long ta, tb;
        block_scan2(a, b, ta, tb);
        if (i < n_tiles) {
            B.block_sums[2 * i] = a + carry_a;
            B.block_sums[2 * i + 1] = b + carry_b;
        }
        carry_a += ta;
        carry_b += tb;
    }
    if (threadIdx.x == 0) {
        Counters* c = B.ctr;
        c->tot_bins = carry_a;
        c->n_nonempty = (unsigned int)min(carry_b, 0xFFFFFFFFull);
        c->stat_bins += carry_a;
        c->stat_nonempty += carry_b;
        if (carry_a > c->need_bins) c->need_bins = carry_a;
        if (carry_b > c->need_tiles) c->need_tiles = carry_b;
        unsigned long long nb = c->n_big;
        if (nb > c->need_big) c->need_big = nb;
        if (carry_a > (unsigned long long)W->bin_cap) c->overflow |= 1u;
        if (carry_b > (unsigned long long)W->map_cap_tiles) c->overflow |= 2u;
        if (nb > (unsigned long long)W->big_cap) c->overflow |= 4u;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_c(const WaveDev* __restrict__ W, Buffers B)
{
    const int64_t tot = W->tot_te;
    const int64_t n_tiles = (tot + kScanTile - 1) / kScanTile;
    for (int64_t st = blockIdx.x; st < n_tiles; st += gridDim.x) {
        uint32_t c[kScanPer];
        unsigned long long a = 0, b = 0;
        int64_t base = st * kScanTile + (int64_t)threadIdx.x * kScanPer;
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            int64_t i = base + q;
            c[q] = i < tot ? B.t_cnt[i] : 0u;
            a += c[q];
            b += c[q] ? 1u : 0u;
        }
        unsigned long long ta, tb;
        block_scan2(a, b, ta, tb);
        a += B.block_sums[2 * st];
        b += B.block_sums[2 * st + 1];
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) {
            int64_t i = base + q;
            if (i < tot) {
                B.t_off[i] = (uint32_t)min(a, 0xFFFFFFFFull);
                B.t_cur[i] = (uint32_t)min(a, 0xFFFFFFFFull);
                B.t_slot[i] = (uint32_t)min(b, 0xFFFFFFFFull);
                if (c[q]) B.nonempty[b] = (uint32_t)i;
            }
            a += c[q];
            b += c[q] ? 1u : 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// k_raster: shared-memory depth tile per non-empty (step, tile)
// ---------------------------------------------------------------------------
template <int TS>
__global__ void __launch_bounds__(256) k_raster(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs,
                                                Buffers B)
{
    __shared__ __align__(16) uint32_t tile[TS * TS];
    __shared__ unsigned int s_item;
    const unsigned int n_ne = B.ctr->n_nonempty;
    const int64_t map_cap = W->map_cap_tiles;
    const int64_t bin_cap = W->bin_cap;
    const int nj = W->n_jobs;
    const int u24 = W->depth_u24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&B.ctr->raster_next, 1u);
        __syncthreads();
        const unsigned int item = s_item;
        __syncthreads();
        if (item >= n_ne || item >= map_cap) break;
        const uint32_t te = B.nonempty[item];
        int j = job_of(nj, te, [&](int q) { return jobs[q].te_base; });
        const JobDev& J = jobs[j];
        const int64_t lte = te - J.te_base;
        const int tps = J.tiles_x * J.tiles_x;
        const int ls = (int)(lte / tps), tl = (int)(lte % tps);
        const int tx = tl % J.tiles_x, ty = tl / J.tiles_x;
        const LightParams lp = B.lp[J.js_base + ls];
        const float ox = (float)(tx * TS), oy = (float)(ty * TS);
        uint4* t4 = reinterpret_cast<uint4*>(tile);
        for (int q = threadIdx.x; q < TS * TS / 4; q += blockDim.x) t4[q] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
        __syncthreads();
        uint64_t off = B.t_off[te];
        uint64_t cnt = B.t_cnt[te];
        if (off + cnt > (uint64_t)bin_cap) cnt = off < (uint64_t)bin_cap ? bin_cap - off : 0;
        for (uint64_t e = warp; e < cnt; e += n_warps) {
            const int t = (int)B.bins[off + e];
            TriT T;
            tri_texel(J, B, lp, ls, t, T);
#pragma unroll
            for (int k = 0; k < 3; ++k) { T.x[k] -= ox; T.y[k] -= oy; }
            Edges ed;
            if (!make_edges(T, ed)) continue;
            float xmin = fminf(T.x[0], fminf(T.x[1], T.x[2])), xmax = fmaxf(T.x[0], fmaxf(T.x[1], T.x[2]));
            float ymin = fminf(T.y[0], fminf(T.y[1], T.y[2])), ymax = fmaxf(T.y[0], fmaxf(T.y[1], T.y[2]));
            int x0 = max(0, (int)ceilf(xmin - 0.5f)), x1 = min(TS - 1, (int)floorf(xmax - 0.5f));
            int y0 = max(0, (int)ceilf(ymin - 0.5f)), y1 = min(TS - 1, (int)floorf(ymax - 0.5f));
            if (x0 > x1 || y0 > y1) continue;
            const int bw = x1 - x0 + 1, bh = y1 - y0 + 1, n_px = bw * bh;
            const float inv_a = 1.f / ed.area2;
            const float inv_bw = 1.f / bw;
            // barycentric depth weights: d = sum_k w_k d_k / area2
            const float e0 = T.d[0] * inv_a, e1 = T.d[1] * inv_a, e2 = T.d[2] * inv_a;
            for (int q = lane; q < n_px; q += 32) {
                int ry = (int)((q + 0.5f) * inv_bw);  // exact: q < 2^12, bw <= 64
                int rx = q - ry * bw;
                if (rx < 0) { --ry; rx += bw; }
                if (rx >= bw) { ++ry; rx -= bw; }
                const int iy = y0 + ry, ix = x0 + rx;
                const float px = ix + 0.5f, py = iy + 0.5f;
                const float w0 = ed.A[0] * px + ed.Bc[0] * py + ed.C[0];
                const float w1 = ed.A[1] * px + ed.Bc[1] * py + ed.C[1];
                const float w2 = ed.A[2] * px + ed.Bc[2] * py + ed.C[2];
                if (w0 >= 0.f && w1 >= 0.f && w2 >= 0.f && ry < bh) {
                    const float d = w0 * e0 + w1 * e1 + w2 * e2;
                    atomicMin(&tile[iy * TS + ix], depth_store_key(d, lp, u24));
                }
            }
        }
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(B.map + ((size_t)item * (TS * TS)));
        for (int q = threadIdx.x; q < TS * TS / 4; q += blockDim.x) dst[q] = t4[q];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_sample: per (step, module) depth tests, cell tallies and the PV model
// ---------------------------------------------------------------------------
constexpr int kSampleThreads = 128;

__global__ void __launch_bounds__(kSampleThreads) k_sample(const WaveDev* __restrict__ W,
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
        const int64_t js = J.js_base + ls;
        const int64_t msi = J.ms_base + li;
        const LightParams lp = B.lp[js];
        const ModuleDev& M = J.mods[m];
        const int cu = M.cu, ncell = M.cu * M.cv;
        const int n = J.n, nn = J.nn;
        const int C = J.n_cells;
        const int64_t row = (int64_t)(J.out_row0 + ls);
        if (!lp.valid) {
            if (threadIdx.x == 0) { B.ms_p[msi] = 0.f; B.ms_pu[msi] = 0.f; B.ms_beam[msi] = 0.f; }
            for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
                B.cs_cnt[J.cs_base + (int64_t)ls * C + M.cell_base + c] = 0;
                if (J.out_counts) J.out_counts[row * C + M.cell_base + c] = 0;
                if (J.out_bits) J.out_bits[row * C + M.cell_base + c] = 0ull;
            }
            continue;
        }
        const ModStep s = B.ms[msi];
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) { s_cnt[c] = 0; s_bits[c] = 0ull; }
        if (threadIdx.x < kMaxSub) s_imin[threadIdx.x] = 0x7F800000u;  // +inf
        __syncthreads();
        const int S = ncell * nn;
        const float inv_n = 1.f / n;
        const float pitch = M.pitch;
        const int R = J.R;
        const int64_t te0 = J.te_base + (int64_t)ls * J.tiles_x * J.tiles_x;
        for (int g0 = 0; g0 < S; g0 += blockDim.x) {
            const int g = g0 + threadIdx.x;
            bool shaded = false;
            if (g < S) {
                int c = g / nn, k = g - c * nn;
                int jj = k / n, ii = k - jj * n;
                int cv_ = c / cu, cu_ = c - cv_ * cu;
                float a = (cu_ + (ii + 0.5f) * inv_n) * pitch;
                float b = (cv_ + (jj + 0.5f) * inv_n) * pitch;
                float tx = s.tx0 + a * s.tax + b * s.tbx;
                float ty = s.ty0 + a * s.tay + b * s.tby;
                float d = s.d0 + a * s.da + b * s.db;
                int ix = min(R - 1, max(0, (int)floorf(tx)));
                int iy = min(R - 1, max(0, (int)floorf(ty)));
                int64_t te = te0 + (int64_t)(iy >> sh) * J.tiles_x + (ix >> sh);
                if (B.t_cnt[te] != 0u) {
                    uint32_t slot = B.t_slot[te];
                    if (slot < map_cap) {
                        uint32_t key = B.map[((size_t)slot << (2 * sh)) + ((iy & tmask) << sh) + (ix & tmask)];
                        if (key != kEmpty) {
                            if (u24) {
                                float q = (d - lp.dnear) * lp.qscale;
                                shaded = q > (float)key + s.bias * lp.qscale;
                            } else {
                                shaded = d > okey_inv(key) + s.bias;
                            }
                        }
                    }
                }
            }
            unsigned int ball = __ballot_sync(0xffffffffu, shaded);
            if (lane == 0 && ball) {
                int gw = g;  // first sample of this warp
                int glast = min(gw + 31, S - 1);
                for (int c = gw / nn; c <= glast / nn; ++c) {
                    int lo = max(c * nn, gw), hi = min((c + 1) * nn, glast + 1);
                    unsigned int msk = (hi - lo >= 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
                    unsigned int part = (ball >> (lo - gw)) & msk;
                    if (part) {
                        atomicAdd(&s_cnt[c], (uint32_t)__popc(part));
                        if (nn <= 64) atomicOr(&s_bits[c], (unsigned long long)part << (lo - c * nn));
                    }
                }
            }
        }
        __syncthreads();
        const float beam = lp.dni * fmaxf(0.f, s.cosi);
        const float diff = lp.dhi * (1.f + s.nz) * 0.5f;
        const float inv_nn = 1.f / nn;
        const int* csub = J.lay_sub + J.lay_off[M.layout];
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            uint32_t cnt = s_cnt[c];
            float f = cnt * inv_nn;
            float G = beam * (1.f - f) + diff;
            float I = J.i_ref * G * 1e-3f;
            atomicMin(&s_imin[csub[c]], __float_as_uint(I));
            B.cs_cnt[J.cs_base + (int64_t)ls * C + M.cell_base + c] = (uint8_t)cnt;
            if (J.out_counts) J.out_counts[row * C + M.cell_base + c] = (uint8_t)cnt;
            if (J.out_bits) J.out_bits[row * C + M.cell_base + c] = s_bits[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int* nk = J.lay_nk + J.lay_nk_off[M.layout];
            const int ns = M.n_sub;
            float best = 0.f, vsum = 0.f;
            for (int k = 0; k < ns; ++k) {
                float ik = __uint_as_float(s_imin[k]);
                float volt = 0.f;
                for (int q = 0; q < ns; ++q) {
                    float iq = __uint_as_float(s_imin[q]);
                    volt += iq >= ik ? nk[q] * J.v_cell : -J.v_diode;
                }
                best = fmaxf(best, ik * volt);
                vsum += nk[k] * J.v_cell;
            }
            B.ms_p[msi] = best;
            B.ms_pu[msi] = J.i_ref * (beam + diff) * 1e-3f * vsum;
            B.ms_beam[msi] = beam;
        }
        __syncthreads();
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

__global__ void k_epilogue(const WaveDev* __restrict__ W, const JobDev* __restrict__ jobs, Buffers B)
{
    const int64_t tot = W->tot_epi;
    const int nj = W->n_jobs;
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < tot;
         item += (int64_t)gridDim.x * blockDim.x) {
        int j = job_of(nj, item, [&](int q) { return jobs[q].it_epi; });
        const JobDev& J = jobs[j];
        int64_t li = item - J.it_epi;
        const int C = J.n_cells, Mn = J.n_mods;
        const float inv_nn = 1.f / J.nn;
        if (li < C) {
            const int c = (int)li;
            const int m = J.cell_mod[c];
            float2 acc = J.kahan_cell[c];
            for (int ls = 0; ls < J.k; ++ls) {
                const LightParams& lp = B.lp[J.js_base + ls];
                if (!lp.valid) continue;
                float beam = B.ms_beam[J.ms_base + (int64_t)ls * Mn + m];
                uint32_t cnt = B.cs_cnt[J.cs_base + (int64_t)ls * C + c];
                kahan_add(acc, beam * (cnt * inv_nn) * lp.dt);
            }
            J.kahan_cell[c] = acc;
        } else {
            const int m = (int)(li - C);
            float2 e = J.kahan_mod[2 * m], eu = J.kahan_mod[2 * m + 1];
            for (int ls = 0; ls < J.k; ++ls) {
                const LightParams& lp = B.lp[J.js_base + ls];
                const int64_t msi = J.ms_base + (int64_t)ls * Mn + m;
                float p = B.ms_p[msi], pu = B.ms_pu[msi];
                if (J.out_power) J.out_power[(int64_t)(J.out_row0 + ls) * Mn + m] = p;
                if (J.out_power_u) J.out_power_u[(int64_t)(J.out_row0 + ls) * Mn + m] = pu;
                if (!lp.valid) continue;
                kahan_add(e, p * lp.dt);
                kahan_add(eu, pu * lp.dt);
            }
            J.kahan_mod[2 * m] = e;
            J.kahan_mod[2 * m + 1] = eu;
        }
    }
}

// Convert Kahan pairs (sum, compensation) to double results.
__global__ void k_finalize(const float2* __restrict__ kmod, int n_mods, const float2* __restrict__ kcell,
                           int n_cells, double* energy, double* energy_u, double* cell_loss)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_mods + n_cells; i += gridDim.x * blockDim.x) {
        if (i < n_mods) {
            float2 e = kmod[2 * i], eu = kmod[2 * i + 1];
            if (energy) energy[i] = (double)e.x - (double)e.y;
            if (energy_u) energy_u[i] = (double)eu.x - (double)eu.y;
        } else {
            int c = i - n_mods;
            float2 h = kcell[c];
            if (cell_loss) cell_loss[c] = (double)h.x - (double)h.y;
        }
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

cudaError_t launch_wave(const WaveDev* d_wave, const JobDev* d_jobs, const Buffers& b, const LaunchCfg& cfg,
                        int64_t tot_te_host)
{
    const WaveDev* W = d_wave;
    cudaStream_t st = cfg.stream;
    const int sm = cfg.sm_count;
    (void)tot_te_host;
    k_window<<<sm * 8, kWinPerItem, 0, st>>>(W, d_jobs, b);
    k_light<<<sm, 128, 0, st>>>(W, d_jobs, b);
    k_modsetup<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    k_bin<0><<<sm * 16, 256, 0, st>>>(W, d_jobs, b);
    k_bin_big<0><<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    k_scan_a<<<sm * 2, kScanThreads, 0, st>>>(W, b);
    k_scan_b<<<1, kScanThreads, 0, st>>>(W, b);
    k_scan_c<<<sm * 2, kScanThreads, 0, st>>>(W, b);
    k_bin<1><<<sm * 16, 256, 0, st>>>(W, d_jobs, b);
    k_bin_big<1><<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    if (cfg.tile == 32)
        k_raster<32><<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    else
        k_raster<64><<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
    k_sample<<<sm * 16, kSampleThreads, 0, st>>>(W, d_jobs, b);
    k_epilogue<<<sm * 8, 256, 0, st>>>(W, d_jobs, b);
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
