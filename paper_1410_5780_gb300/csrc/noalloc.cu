// noalloc.cu -- pv3d_module_shade_noalloc: shaded-sample counts of one module
// for one sun direction without any device allocation.
//
// Who needs it: callers that must not allocate device memory while they run --
// for example a host loop that owns every byte of the GPU through its own pool,
// a latency-critical loop where the implicit synchronisation of cudaMalloc and
// cudaFree would stall other streams, or code that records its work into a
// stream capture, where those calls are not permitted.  pv3d_evaluate needs
// pools that grow with the scene; this entry point instead works inside one
// fixed shadow map compiled into the library.
//
// The shadow map is the file-scope array g_noalloc_map below: kNoAllocMaxRes^2
// uint32 depth keys (16 MiB).  With CUDA's lazy module loading (the default)
// the array is reserved on a device when this file's module is first loaded
// there, i.e. by the first call on that device, and it is then kept until the
// process exits: a caller whose own pool takes all device memory should make
// one call before creating the pool.  Host code cannot use the array's name as
// a device address (in host code it names a host-side stand-in), so every call
// looks the address up with cudaGetSymbolAddress for the current device and
// context (a context made after cudaDeviceReset loads the module again at a new
// address).  While the stream is being captured the lookup is not made and the
// address found by the last call on that device is used, so one call must come
// before any stream capture.  All calls share the one array and it keeps the
// last call's contents: every call clears the part it uses first, and calls
// whose work overlaps on the GPU (different streams, no ordering) race on it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "pv3d.h"

namespace {

constexpr int kNoAllocMaxRes = PV3D_NOALLOC_MAX_RES;
constexpr int kMaxDevices = 64;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

static __device__ __align__(256) uint32_t g_noalloc_map[kNoAllocMaxRes * kNoAllocMaxRes];

std::mutex g_setup_mu;
uint32_t* g_map_ptr[kMaxDevices] = {};

__device__ __forceinline__ uint32_t na_key(float d)
{
    const uint32_t b = __float_as_uint(d);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float na_depth(uint32_t k)
{
    const uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(b);
}

// Light frame and window, computed on the host in FP64, used in FP32.
struct NaFrame {
    float ux, uy, uz, vx, vy, vz, sx, sy, sz;
    float refx, refy, refz;  // module centre; coordinates are taken relative to it
    float u0, v0, inv_delta, delta;
    int R;
};

// Clear the part of the map in use and the output tallies.
__global__ void na_clear(uint32_t* map, int64_t n_texels, uint32_t* counts, int n_cells)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_texels; i += stride) map[i] = kEmptyKey;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells; i += stride) counts[i] = 0u;
}

// One warp per triangle: texel-centre coverage (inclusive edges), barycentric
// depth, atomicMin of the order-preserving depth key into the map.
__global__ void na_raster(const float* __restrict__ tri, int64_t n_tris, NaFrame f, uint32_t* map)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < n_tris; t += n_warps) {
        float x[3], y[3], d[3];
        for (int k = 0; k < 3; ++k) {
            const float px = tri[9 * t + 3 * k] - f.refx, py = tri[9 * t + 3 * k + 1] - f.refy,
                        pz = tri[9 * t + 3 * k + 2] - f.refz;
            x[k] = (px * f.ux + py * f.uy + pz * f.uz - f.u0) * f.inv_delta;
            y[k] = (px * f.vx + py * f.vy + pz * f.vz - f.v0) * f.inv_delta;
            d[k] = -(px * f.sx + py * f.sy + pz * f.sz);
        }
        float area2 = (x[1] - x[0]) * (y[2] - y[0]) - (y[1] - y[0]) * (x[2] - x[0]);
        if (!(fabsf(area2) > 0.f)) continue;
        if (area2 < 0.f) {
            float t0 = x[1], t1 = y[1], t2 = d[1];
            x[1] = x[2]; y[1] = y[2]; d[1] = d[2];
            x[2] = t0; y[2] = t1; d[2] = t2;
            area2 = -area2;
        }
        const float xmin = fminf(x[0], fminf(x[1], x[2])), xmax = fmaxf(x[0], fmaxf(x[1], x[2]));
        const float ymin = fminf(y[0], fminf(y[1], y[2])), ymax = fmaxf(y[0], fmaxf(y[1], y[2]));
        if (!(xmax >= 0.5f && ymax >= 0.5f && xmin <= f.R - 0.5f && ymin <= f.R - 0.5f)) continue;
        const int x0 = max(0, (int)ceilf(xmin - 0.5f)), x1 = min(f.R - 1, (int)floorf(xmax - 0.5f));
        const int y0 = max(0, (int)ceilf(ymin - 0.5f)), y1 = min(f.R - 1, (int)floorf(ymax - 0.5f));
        if (x0 > x1 || y0 > y1) continue;
        float A[3], Bc[3], C[3];
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            A[k] = -(y[b] - y[a]);
            Bc[k] = x[b] - x[a];
            C[k] = -(A[k] * x[a] + Bc[k] * y[a]);
        }
        const float inv_a = 1.f / area2;
        const int bw = x1 - x0 + 1;
        const int64_t n_px = (int64_t)bw * (y1 - y0 + 1);
        for (int64_t q = lane; q < n_px; q += 32) {
            const int iy = y0 + (int)(q / bw), ix = x0 + (int)(q % bw);
            const float px = ix + 0.5f, py = iy + 0.5f;
            const float w0 = A[0] * px + Bc[0] * py + C[0];
            const float w1 = A[1] * px + Bc[1] * py + C[1];
            const float w2 = A[2] * px + Bc[2] * py + C[2];
            if (w0 >= 0.f && w1 >= 0.f && w2 >= 0.f)
                atomicMin(&map[(int64_t)iy * f.R + ix], na_key((w0 * d[0] + w1 * d[1] + w2 * d[2]) * inv_a));
        }
    }
}

// One thread per sample: texel lookup, depth test with slope-scaled bias,
// shaded count per cell.
__global__ void na_sample(NaFrame f, const uint32_t* __restrict__ map, float3 o, float3 u, float3 v, float pitch,
                          int cells_u, int n_cells, int n, float bias, uint32_t* counts)
{
    const int nn = n * n;
    const int64_t total = (int64_t)n_cells * nn;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(g / nn), k = (int)(g % nn);
        const int j = k / n, i = k % n;
        const int cv = c / cells_u, cu = c % cells_u;
        const float a = (cu + (i + 0.5f) / n) * pitch, b = (cv + (j + 0.5f) / n) * pitch;
        const float px = o.x + a * u.x + b * v.x, py = o.y + a * u.y + b * v.y, pz = o.z + a * u.z + b * v.z;
        const float tx = (px * f.ux + py * f.uy + pz * f.uz - f.u0) * f.inv_delta;
        const float ty = (px * f.vx + py * f.vy + pz * f.vz - f.v0) * f.inv_delta;
        const float d = -(px * f.sx + py * f.sy + pz * f.sz);
        const int ix = min(f.R - 1, max(0, (int)floorf(tx))), iy = min(f.R - 1, max(0, (int)floorf(ty)));
        const uint32_t key = map[(int64_t)iy * f.R + ix];
        if (key != kEmptyKey && d > na_depth(key) + bias) atomicAdd(&counts[c], 1u);
    }
}

}  // namespace

extern "C" int pv3d_module_shade_noalloc(const float* tri_xyz, int64_t n_tris, const pv3d_module* module,
                                         const double* sun_xyz, int32_t samples_per_side, int32_t map_res,
                                         uint32_t* cell_counts, void* stream)
{
    if (!module || !sun_xyz || !cell_counts || n_tris < 0 || (n_tris > 0 && !tri_xyz)) return PV3D_E_INVALID;
    if (map_res > kNoAllocMaxRes) return PV3D_E_TOOBIG;
    if (map_res < 64 || (map_res & (map_res - 1))) return PV3D_E_INVALID;
    const int n = samples_per_side;
    if (n < 1 || n > 15) return PV3D_E_INVALID;
    const pv3d_module& M = *module;
    if (M.tracker != -1 || M.cells_u < 1 || M.cells_v < 1 || M.cells_u > 64 || M.cells_v > 64 || !(M.pitch > 0.f))
        return PV3D_E_INVALID;
    const double sx = sun_xyz[0], sy = sun_xyz[1], sz = sun_xyz[2];
    const double sl = std::sqrt(sx * sx + sy * sy + sz * sz);
    if (!std::isfinite(sl) || std::fabs(sl - 1.0) > 1e-6) return PV3D_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_cells = M.cells_u * M.cells_v;

    // device address of the map for the current device and context; under
    // stream capture, the address the last call on this device found
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PV3D_E_DEVICE;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return PV3D_E_DEVICE;
    uint32_t* map = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_map) != cudaSuccess || !p) return PV3D_E_DEVICE;
            g_map_ptr[dev] = (uint32_t*)p;
        }
        map = g_map_ptr[dev];
    }
    if (!map) return PV3D_E_DEVICE;  // captured before any call on this device

    // light frame (w = s, u = normalize(s x z), x at the zenith, v = s x u) and
    // window: bounding square of the module's corners, one texel of padding
    double ux = 1.0, uy = 0.0;
    const double h2 = sx * sx + sy * sy;
    if (h2 >= 1e-12) {
        const double r = 1.0 / std::sqrt(h2);
        ux = sy * r;
        uy = -sx * r;
    }
    const double vx = -sz * uy, vy = sz * ux, vz = sx * uy - sy * ux;
    const double lu = M.cells_u * (double)M.pitch, lv = M.cells_v * (double)M.pitch;
    double cx[4][3];
    for (int k = 0; k < 4; ++k) {
        const double a = (k == 1 || k == 2) ? lu : 0.0, b = (k >= 2) ? lv : 0.0;
        for (int q = 0; q < 3; ++q) cx[k][q] = M.origin[q] + a * M.u[q] + b * M.v[q];
    }
    double ref[3];
    for (int q = 0; q < 3; ++q) {
        double lo = cx[0][q], hi = cx[0][q];
        for (int k = 1; k < 4; ++k) { lo = std::fmin(lo, cx[k][q]); hi = std::fmax(hi, cx[k][q]); }
        ref[q] = (float)(0.5 * (lo + hi));
    }
    double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
    for (int k = 0; k < 4; ++k) {
        const double px = cx[k][0] - ref[0], py = cx[k][1] - ref[1], pz = cx[k][2] - ref[2];
        const double pu = px * ux + py * uy, pv = px * vx + py * vy + pz * vz;
        umin = std::fmin(umin, pu); umax = std::fmax(umax, pu);
        vmin = std::fmin(vmin, pv); vmax = std::fmax(vmax, pv);
    }
    const double ext = std::fmax(std::fmax(umax - umin, vmax - vmin), 1e-6);
    const double delta = ext / (map_res - 2);
    NaFrame f;
    f.ux = (float)ux; f.uy = (float)uy; f.uz = 0.f;
    f.vx = (float)vx; f.vy = (float)vy; f.vz = (float)vz;
    f.sx = (float)sx; f.sy = (float)sy; f.sz = (float)sz;
    f.refx = (float)ref[0]; f.refy = (float)ref[1]; f.refz = (float)ref[2];
    f.delta = (float)delta;
    f.inv_delta = (float)(1.0 / delta);
    f.u0 = (float)(0.5 * (umin + umax) - 0.5 * map_res * delta);
    f.v0 = (float)(0.5 * (vmin + vmax) - 0.5 * map_res * delta);
    f.R = map_res;
    // depth bias: half a texel diagonal times the receiver slope (tan of
    // incidence, clamped at 89 deg) plus 1/32 texel
    double nx = (double)M.u[1] * M.v[2] - (double)M.u[2] * M.v[1];
    double ny = (double)M.u[2] * M.v[0] - (double)M.u[0] * M.v[2];
    double nz = (double)M.u[0] * M.v[1] - (double)M.u[1] * M.v[0];
    const double nl = std::sqrt(nx * nx + ny * ny + nz * nz);
    const double ci = std::fmax((nx * sx + ny * sy + nz * sz) / nl, 0.017452406);
    const float bias = (float)(delta * (0.70710678 * std::sqrt(std::fmax(0.0, 1.0 - ci * ci)) / ci + 0.03125));

    const int64_t n_texels = (int64_t)map_res * map_res;
    // each launch's status comes from its own cudaLaunchKernel call, so an
    // earlier error of the caller's is neither reported nor cleared here
    void* a_clear[] = {&map, (void*)&n_texels, &cell_counts, (void*)&n_cells};
    if (cudaLaunchKernel((const void*)na_clear, dim3(512), dim3(256), a_clear, 0, st) != cudaSuccess)
        return PV3D_E_DEVICE;
    if (sz > 0.0) {
        if (n_tris > 0) {
            const int64_t blocks = std::min<int64_t>((n_tris + 7) / 8, 4096);
            void* a_raster[] = {(void*)&tri_xyz, &n_tris, &f, &map};
            if (cudaLaunchKernel((const void*)na_raster, dim3((unsigned)blocks), dim3(256), a_raster, 0, st) !=
                cudaSuccess)
                return PV3D_E_DEVICE;
        }
        float3 o = make_float3((float)(M.origin[0] - ref[0]), (float)(M.origin[1] - ref[1]),
                               (float)(M.origin[2] - ref[2]));
        float3 u = make_float3(M.u[0], M.u[1], M.u[2]), v = make_float3(M.v[0], M.v[1], M.v[2]);
        float pitch = M.pitch;
        int cells_u = M.cells_u, nc = n_cells, nside = n;
        float b = bias;
        const int64_t total = (int64_t)n_cells * n * n;
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, 4096);
        const uint32_t* cmap = map;
        void* a_sample[] = {&f, &cmap, &o, &u, &v, &pitch, &cells_u, &nc, &nside, &b, &cell_counts};
        if (cudaLaunchKernel((const void*)na_sample, dim3((unsigned)blocks), dim3(256), a_sample, 0, st) !=
            cudaSuccess)
            return PV3D_E_DEVICE;
    }
    return PV3D_OK;
}
