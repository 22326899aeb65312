// peaks.cu -- pv3d_raster_peak: the measured throughput of shared-memory
// atomicMin on 32-bit depth keys, the second roofline of the rasterising
// kernels (the first is HBM bandwidth).  Each block holds a 32 x 32 tile of
// keys in shared memory, as k_raster_test does, and its warps draw strips of
// 32 consecutive texels (one per lane, a chunk of a triangle's texel visits)
// with atomicMin of a varying key; the tile is folded into one word per block
// at the end so that no update can be optimised away.
#include <cstdint>

#include "pv3d.h"

namespace {

constexpr int kPeakTile = 32 * 32;
constexpr int kPeakThreads = 128;
constexpr int kPeakBlocksPerSm = 16;

__global__ void __launch_bounds__(kPeakThreads) k_atomic_min_peak(int iters, uint32_t* out)
{
    __shared__ uint32_t tile[kPeakTile];
    for (int q = threadIdx.x; q < kPeakTile; q += blockDim.x) tile[q] = 0xFFFFFFFFu;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t key = 0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    // strip origin walks the tile row by row; lanes take consecutive texels
    int base = (warp * 256) & (kPeakTile - 1);
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        atomicMin(&tile[(base + lane) & (kPeakTile - 1)], key);
        key = key * 1664525u + 1013904223u;
        base = (base + 96) & (kPeakTile - 1);
    }
    __syncthreads();
    uint32_t v = 0xFFFFFFFFu;
    for (int q = threadIdx.x; q < kPeakTile; q += blockDim.x) v = min(v, tile[q]);
    for (int off = 16; off; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) atomicMin(out, v);
}

}  // namespace

extern "C" int pv3d_raster_peak(int32_t device, double* atomics_per_s, double* best_ms)
{
    if (!atomics_per_s) return PV3D_E_INVALID;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return PV3D_E_DEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return PV3D_E_DEVICE;
    int rc = PV3D_OK;
    int sms = 0;
    uint32_t* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const int iters = 1 << 14;
    float best = 1e30f;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&out, sizeof(uint32_t)) != cudaSuccess || cudaStreamCreate(&st) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = PV3D_E_DEVICE;
    } else {
        const unsigned grid = (unsigned)(sms * kPeakBlocksPerSm);
        for (int rep = 0; rep < 6 && rc == PV3D_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(a, st);
            k_atomic_min_peak<<<grid, kPeakThreads, 0, st>>>(iters, out);
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess) { rc = PV3D_E_DEVICE; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;
        }
        if (rc == PV3D_OK) {
            const double ops = (double)grid * kPeakThreads * iters;
            *atomics_per_s = ops / (best * 1e-3);
            if (best_ms) *best_ms = best;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    return rc;
}
