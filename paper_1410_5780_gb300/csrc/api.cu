// api.cu -- host side of the pv3d C ABI: contexts, resident scenes and
// generators, wave planning, workspace pools and the served request loop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pv3d.h"
#include "pv3d_dev.cuh"

using namespace pv3d;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct SceneH {
    float4* d_tri = nullptr;
    float4* d_ml = nullptr;  // meshlet boxes, 2 per meshlet
    int32_t n_tris = 0;
    int32_t n_ml = 0;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    size_t bytes = 0;
};

struct GenH {
    uint32_t scene_id = 0;
    int32_t M = 0, C = 0, n_trk = 0;
    int32_t max_cells = 0;
    bool coplanar = false;
    float ref[3] = {0, 0, 0};
    float glo[3], ghi[3];  // generator bounds (world), tracker reach included
    std::vector<ModuleDev> mods_h;
    ModuleDev* d_mods = nullptr;
    int32_t* d_cell_mod = nullptr;
    int32_t* d_lay_sub = nullptr;
    int32_t* d_lay_off = nullptr;
    int32_t* d_lay_nk = nullptr;
    int32_t* d_lay_nk_off = nullptr;
    float* d_pivots = nullptr;
    // sun table
    int64_t n_steps = 0;
    double* d_sun = nullptr;
    float* d_dni = nullptr;
    float* d_dhi = nullptr;
    float* d_dt = nullptr;
    std::vector<uint8_t> lit;  // host copy: s.z > 0
    // poses
    int64_t n_pose_steps = 0;
    float* d_poses = nullptr;
    // series strings: distinct string ids in ascending order; substrings
    // numbered string by string (module order within a string)
    std::vector<int32_t> str_ids;
    int32_t n_sub_tot = 0;
    int32_t* d_str_sub = nullptr;   // [n_str + 1]
    int32_t* d_sub_base = nullptr;  // [M]
    int32_t* d_sub_nk = nullptr;    // [n_sub_tot]
    int32_t* d_sub_mod = nullptr;   // [n_sub_tot]
    float* d_fdiff = nullptr;       // [bins][C] diffuse shading fraction per cell (pv3d_sky_view)
    int32_t* d_fbin = nullptr;      // [n_steps] pose bin of each step (tracked generators)
    int32_t fdiff_bins = 0;         // rows of d_fdiff
    // arrays of parallel strings: distinct array ids ascending; their strings
    std::vector<int32_t> arr_ids;
    int32_t max_arr_sub = 0;        // substrings of the largest array
    int32_t* d_arr_off = nullptr;   // [n_arr + 1]
    int32_t* d_arr_strs = nullptr;  // [n_str]
    // window groups: each module's string and array ids, and the world boxes of
    // the occluder meshlets (16 modules each, boxes that hold them under any pose)
    std::vector<int32_t> mod_string, mod_array;
    float4* d_oml = nullptr;
    int32_t n_oml = 0;
    // per grouping mode: group g holds modules [m0[g], m0[g + 1]) and cells
    // [c0[g], c0[g + 1]); module tables with group-local cell numbers
    struct WinGroups {
        std::vector<int32_t> m0, c0;
        ModuleDev* d_mods = nullptr;
        int32_t* d_cell_mod = nullptr;
    };
    std::map<int, WinGroups> wgroups;
    size_t bytes = 0;
};

// One evaluation split into waves of consecutive steps.
struct Plan {
    std::vector<WaveDev> waves;
    std::vector<JobDev> jobs;  // one job per wave for a plain evaluation
    int64_t max_js = 0, max_te = 0, max_ms = 0, max_cs = 0;
};

}  // namespace

struct pv3d_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    pv3d_opts opts{};
    std::string err;
    std::map<uint32_t, SceneH> scenes;
    std::map<uint32_t, GenH> gens;
    uint32_t next_id = 1;
    // workspace pools
    DevBuf lp, win, ms, ms_p, ms_pu, ms_beam, ms_iu, ss_i, sq_p, sq_pu, kahan_str, js_p, js_pu, js_bin, heat, sa_p, sa_pu,
        kahan_arr, cs_cnt, cs_bits, t_far, t_cnt, t_off, t_cur, t_slot, t_rcnt, t_plane, t_roff, t_rcur, nonempty, heavy, bins, pairs, recv, map,
        big, block_sums, ctr, waves, jobs, kahan_mod, kahan_cell, staging;
    int64_t bin_cap = 0, map_cap_tiles = 0, big_cap = 0, recv_cap = 0;
    uint64_t bufgen = 0;  // bumped whenever a pool is reallocated (captured graphs hold its pointers)
    // captured wave graph: the kernels read the wave from fixed descriptor slots
    DevBuf wave_slot, jobs_slot;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_key = 0;
    bool use_graphs = true;
    void* h_stage = nullptr;  // pinned staging for descriptors
    size_t h_stage_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> prof_ev;  // stage-boundary events, kStages + 1 per wave
    pv3d_profile last_prof{};
    bool have_prof = false;
    // served requests: a worker thread runs waves built from every admitted
    // request (continuous batching); admission by device-memory footprint
    struct Request;
    std::mutex gpu_mu;  // one wave or plain evaluation at a time on the workspace
    std::mutex mu;      // request tables
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> active;
    size_t rr = 0;              // round-robin start of the next wave
    int64_t reserved = 0;       // footprint of admitted requests
    uint64_t next_req = 1;
    std::vector<DevBuf> free_bufs;  // request buffers for reuse
    cudaStream_t serve_stream = nullptr;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int fail(pv3d_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CUDA_TRY(ctx, call)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? PV3D_E_NOMEM : PV3D_E_DEVICE, \
                        "%s: %s", #call, cudaGetErrorString(e_));                              \
    } while (0)

static int ensure(pv3d_ctx* c, DevBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return PV3D_OK;
    ++c->bufgen;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, PV3D_E_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.bytes = want;
    return PV3D_OK;
}

static void release_buf(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b = DevBuf{};
}

template <typename T>
static int upload(pv3d_ctx* c, T** dst, const T* src, size_t n)
{
    *dst = nullptr;
    size_t bytes = std::max<size_t>(n * sizeof(T), 16);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return fail(c, PV3D_E_NOMEM, "cudaMalloc(%zu) failed", bytes);
    }
    if (n) {
        e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(c, PV3D_E_DEVICE, "upload: %s", cudaGetErrorString(e));
    }
    return PV3D_OK;
}

static bool finite3(const float* p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

static void free_gen(GenH& g)
{
    void* ps[] = {g.d_mods, g.d_cell_mod, g.d_lay_sub, g.d_lay_off, g.d_lay_nk, g.d_lay_nk_off, g.d_pivots,
                  g.d_sun, g.d_dni, g.d_dhi, g.d_dt, g.d_poses, g.d_str_sub, g.d_sub_base, g.d_sub_nk,
                  g.d_sub_mod, g.d_fdiff, g.d_fbin, g.d_arr_off, g.d_arr_strs, g.d_oml};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (auto& kv : g.wgroups) {
        if (kv.second.d_mods) cudaFree(kv.second.d_mods);
        if (kv.second.d_cell_mod) cudaFree(kv.second.d_cell_mod);
    }
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int pv3d_create(pv3d_ctx** out, const pv3d_opts* opts)
{
    if (!out) return PV3D_E_INVALID;
    *out = nullptr;
    std::unique_ptr<pv3d_ctx> c(new (std::nothrow) pv3d_ctx());
    if (!c) return PV3D_E_NOMEM;
    if (opts) c->opts = *opts;
    pv3d_opts& o = c->opts;
    if (o.map_res == 0) o.map_res = 4096;
    if (o.tile == 0) o.tile = 64;
    if (o.chunk_steps == 0) o.chunk_steps = 128;
    if (o.max_inflight == 0) o.max_inflight = 64;
    if (o.max_inflight < 1 || o.max_inflight > 256) return PV3D_E_INVALID;  // jobs per wave
    if (o.wave_scratch_mb == 0) o.wave_scratch_mb = 2048;
    if (o.wave_scratch_mb < 1) return PV3D_E_INVALID;
    if (o.bin_capacity < 0 || o.bin_capacity > (1ll << 32)) return PV3D_E_INVALID;
    if (o.bin_capacity > 0) c->bin_cap = o.bin_capacity;
    if (o.tile != 32 && o.tile != 64 && o.tile != 128) return PV3D_E_INVALID;
    if (o.map_res < 64 || o.map_res > 16384 || (o.map_res & (o.map_res - 1))) return PV3D_E_INVALID;
    if (o.chunk_steps < 1 || o.chunk_steps > 256) return PV3D_E_INVALID;
    if (o.depth_format != PV3D_DEPTH_F32 && o.depth_format != PV3D_DEPTH_U24) return PV3D_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PV3D_E_DEVICE;
    }
    if (o.device < 0 || o.device >= ndev) return PV3D_E_INVALID;
    c->device = o.device;
    if (cudaSetDevice(c->device) != cudaSuccess) return PV3D_E_DEVICE;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return PV3D_E_DEVICE;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return PV3D_E_DEVICE;
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return PV3D_E_DEVICE;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return PV3D_E_DEVICE;
    if (prepare_tile_kernels() != cudaSuccess) return PV3D_E_DEVICE;
    if (o.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        o.hbm_budget_bytes = (int64_t)(0.9 * (double)fr);
    }
    *out = c.release();
    return PV3D_OK;
}

extern "C" const char* pv3d_last_error(pv3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------
// Order of the triangles (3 float4 vertices each in tv) for 32-triangle
// meshlets: the set is split at the median centroid of its longest centroid
// extent, at a multiple of 32 triangles, until each part is one meshlet, so a
// meshlet is a compact patch and its box stays tight.  The two parts of a
// split are independent: host threads take parts from a shared stack (the
// order is the same whatever the threads' timing, since parts never overlap).
static std::vector<uint32_t> meshlet_order(const std::vector<float4>& tv, int64_t n_tris)
{
    struct Rec {
        float c[3];
        uint32_t t;
    };
    std::vector<Rec> r((size_t)n_tris);
    for (int64_t t = 0; t < n_tris; ++t) {
        const float4 a = tv[3 * t], b = tv[3 * t + 1], d = tv[3 * t + 2];
        r[t] = Rec{{(a.x + b.x + d.x) / 3.f, (a.y + b.y + d.y) / 3.f, (a.z + b.z + d.z) / 3.f}, (uint32_t)t};
    }
    // split [b, e) once; its parts of more than one meshlet go to `out`
    auto split = [&r](int64_t b, int64_t e, std::vector<std::pair<int64_t, int64_t>>& out) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = b; i < e; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], r[i].c[a]);
                hi[a] = std::max(hi[a], r[i].c[a]);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
        // b is a multiple of 32, so every part starts on a meshlet
        const int64_t mid = b + ((e - b + 31) / 32 / 2) * 32;
        std::nth_element(r.begin() + b, r.begin() + mid, r.begin() + e,
                         [ax](const Rec& x, const Rec& y) { return x.c[ax] < y.c[ax]; });
        if (mid - b > 32) out.push_back({b, mid});
        if (e - mid > 32) out.push_back({mid, e});
    };
    constexpr int64_t kSerial = 1 << 14;  // a part this small is finished by one thread
    std::vector<std::pair<int64_t, int64_t>> todo;
    if (n_tris > 32) todo.push_back({0, n_tris});
    std::mutex mu;
    std::condition_variable cv;
    int busy = 0;
    auto worker = [&]() {
        std::vector<std::pair<int64_t, int64_t>> local;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return !todo.empty() || busy == 0; });
            if (todo.empty()) break;  // nothing queued and nobody splitting: done
            const auto part = todo.back();
            todo.pop_back();
            ++busy;
            lk.unlock();
            local.clear();
            split(part.first, part.second, local);
            std::vector<std::pair<int64_t, int64_t>> out;
            for (const auto& q : local) {
                if (q.second - q.first > kSerial) {
                    out.push_back(q);
                    continue;
                }
                std::vector<std::pair<int64_t, int64_t>> stack{q};
                while (!stack.empty()) {
                    const auto c = stack.back();
                    stack.pop_back();
                    split(c.first, c.second, stack);
                }
            }
            lk.lock();
            for (const auto& q : out) todo.push_back(q);
            --busy;
            cv.notify_all();
        }
    };
    const int n_threads = n_tris > 4 * kSerial ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
    std::vector<std::thread> pool;
    for (int k = 1; k < n_threads; ++k) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    std::vector<uint32_t> order((size_t)n_tris);
    for (int64_t t = 0; t < n_tris; ++t) order[t] = r[t].t;
    return order;
}

extern "C" int pv3d_scene_load(pv3d_ctx* c, const float* xyz, int64_t n_verts, const int32_t* tri_idx,
                               int64_t n_tris, uint32_t* scene_id)
{
    if (!c || !scene_id) return PV3D_E_INVALID;
    if (n_verts < 0 || n_tris < 0 || n_tris > (1ll << 30)) return fail(c, PV3D_E_INVALID, "bad sizes");
    if ((n_tris > 0 && (!xyz || !tri_idx))) return fail(c, PV3D_E_INVALID, "null arrays");
    cudaSetDevice(c->device);
    SceneH s;
    s.n_tris = (int32_t)n_tris;
    std::vector<float4> tv((size_t)n_tris * 3);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < n_tris; ++t) {
        for (int k = 0; k < 3; ++k) {
            int64_t vi = tri_idx[3 * t + k];
            if (vi < 0 || vi >= n_verts) return fail(c, PV3D_E_INVALID, "triangle %lld: index out of range", (long long)t);
            const float* p = xyz + 3 * vi;
            if (!finite3(p)) return fail(c, PV3D_E_INVALID, "vertex %lld not finite", (long long)vi);
            tv[3 * t + k] = make_float4(p[0], p[1], p[2], 0.f);
            for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
        }
    }
    if (n_tris == 0)
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 0.f;
    memcpy(s.lo, lo, sizeof(lo));
    memcpy(s.hi, hi, sizeof(hi));
    // triangles grouped 32 at a time into meshlets with world bounding boxes
    // (the binning culls whole meshlets), in meshlet_order
    {
        const std::vector<uint32_t> order = meshlet_order(tv, n_tris);
        std::vector<float4> sorted(tv.size());
        for (int64_t t = 0; t < n_tris; ++t)
            for (int k = 0; k < 3; ++k) sorted[3 * t + k] = tv[3 * order[t] + k];
        tv.swap(sorted);
        s.n_ml = (int32_t)((n_tris + 31) / 32);
        std::vector<float4> boxes((size_t)s.n_ml * 2);
        for (int32_t m = 0; m < s.n_ml; ++m) {
            float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t t = (int64_t)m * 32; t < std::min<int64_t>(n_tris, (int64_t)m * 32 + 32); ++t)
                for (int k = 0; k < 3; ++k) {
                    const float4 p = tv[3 * t + k];
                    blo[0] = std::min(blo[0], p.x); bhi[0] = std::max(bhi[0], p.x);
                    blo[1] = std::min(blo[1], p.y); bhi[1] = std::max(bhi[1], p.y);
                    blo[2] = std::min(blo[2], p.z); bhi[2] = std::max(bhi[2], p.z);
                }
            boxes[2 * m] = make_float4(blo[0], blo[1], blo[2], 0.f);
            boxes[2 * m + 1] = make_float4(bhi[0], bhi[1], bhi[2], 0.f);
        }
        int rc0 = upload(c, &s.d_ml, boxes.data(), boxes.size());
        if (rc0) return rc0;
    }
    int rc = upload(c, &s.d_tri, tv.data(), tv.size());
    if (rc) return rc;
    s.bytes = std::max<size_t>(tv.size() * sizeof(float4), 16) + (size_t)s.n_ml * 32;
    uint32_t id = c->next_id++;
    c->scenes[id] = s;
    *scene_id = id;
    return PV3D_OK;
}

// ---------------------------------------------------------------------------
// generator
// ---------------------------------------------------------------------------
extern "C" int pv3d_generator_define(pv3d_ctx* c, uint32_t scene_id, const pv3d_module* mods, int32_t n_mods,
                                     const pv3d_layout* layouts, int32_t n_layouts, const pv3d_tracker* trackers,
                                     int32_t n_trackers, uint32_t* gen_id)
{
    if (!c || !gen_id) return PV3D_E_INVALID;
    auto sit = c->scenes.find(scene_id);
    if (sit == c->scenes.end()) return fail(c, PV3D_E_NOTFOUND, "unknown scene %u", scene_id);
    if (n_mods < 1 || !mods) return fail(c, PV3D_E_INVALID, "a generator needs at least one module");
    if (n_layouts < 1 || !layouts) return fail(c, PV3D_E_INVALID, "a generator needs at least one layout");
    if (n_trackers < 0 || (n_trackers > 0 && !trackers)) return fail(c, PV3D_E_INVALID, "bad trackers");
    cudaSetDevice(c->device);
    GenH g;
    g.scene_id = scene_id;
    g.M = n_mods;
    g.n_trk = n_trackers;
    // layouts
    std::vector<int32_t> lay_sub, lay_off, lay_nk, lay_nk_off;
    for (int32_t l = 0; l < n_layouts; ++l) {
        const pv3d_layout& L = layouts[l];
        int nc = L.cells_u * L.cells_v;
        if (L.cells_u < 1 || L.cells_v < 1 || nc > kMaxCellsPerModule || L.n_sub < 1 || L.n_sub > kMaxSub ||
            !L.cell_sub)
            return fail(c, PV3D_E_INVALID, "layout %d: bad size", l);
        lay_off.push_back((int32_t)lay_sub.size());
        lay_nk_off.push_back((int32_t)lay_nk.size());
        std::vector<int32_t> nk(L.n_sub, 0);
        for (int k = 0; k < nc; ++k) {
            int s = L.cell_sub[k];
            if (s < 0 || s >= L.n_sub) return fail(c, PV3D_E_INVALID, "layout %d: substring index out of range", l);
            nk[s]++;
            lay_sub.push_back(s);
        }
        for (int s = 0; s < L.n_sub; ++s)
            if (nk[s] == 0) return fail(c, PV3D_E_INVALID, "layout %d: substring %d owns no cell", l, s);
        lay_nk.insert(lay_nk.end(), nk.begin(), nk.end());
    }
    for (int32_t t = 0; t < n_trackers; ++t)
        if (!finite3(trackers[t].pivot)) return fail(c, PV3D_E_INVALID, "tracker %d: pivot not finite", t);
    // modules
    double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
    std::vector<int32_t> cell_mod;
    g.mods_h.resize(n_mods);
    std::vector<double> mlo((size_t)3 * n_mods), mhi((size_t)3 * n_mods);  // module world boxes
    int32_t cell = 0;
    for (int32_t m = 0; m < n_mods; ++m) {
        const pv3d_module& P = mods[m];
        g.mod_string.push_back(P.string_id);
        g.mod_array.push_back(P.array_id);
        if (!finite3(P.origin) || !finite3(P.u) || !finite3(P.v) || !std::isfinite(P.pitch) || !(P.pitch > 0))
            return fail(c, PV3D_E_INVALID, "module %d: non-finite geometry", m);
        double uu = (double)P.u[0] * P.u[0] + (double)P.u[1] * P.u[1] + (double)P.u[2] * P.u[2];
        double vv = (double)P.v[0] * P.v[0] + (double)P.v[1] * P.v[1] + (double)P.v[2] * P.v[2];
        double uv = (double)P.u[0] * P.v[0] + (double)P.u[1] * P.v[1] + (double)P.u[2] * P.v[2];
        if (std::fabs(uu - 1) > 1e-4 || std::fabs(vv - 1) > 1e-4 || std::fabs(uv) > 1e-4)
            return fail(c, PV3D_E_INVALID, "module %d: u and v must be orthonormal", m);
        if (P.cells_u < 1 || P.cells_v < 1 || P.cells_u > 64 || P.cells_v > 64 ||
            P.cells_u * P.cells_v > kMaxCellsPerModule)
            return fail(c, PV3D_E_INVALID, "module %d: bad cell grid", m);
        if (P.layout < 0 || P.layout >= n_layouts) return fail(c, PV3D_E_INVALID, "module %d: bad layout", m);
        const pv3d_layout& L = layouts[P.layout];
        if (L.cells_u != P.cells_u || L.cells_v != P.cells_v)
            return fail(c, PV3D_E_INVALID, "module %d: layout grid differs from the module's", m);
        if (P.tracker < -1 || P.tracker >= n_trackers) return fail(c, PV3D_E_INVALID, "module %d: bad tracker", m);
        ModuleDev& D = g.mods_h[m];
        for (int a = 0; a < 3; ++a) { D.o[a] = P.origin[a]; D.u[a] = P.u[a]; D.v[a] = P.v[a]; }
        D.pitch = P.pitch;
        D.cu = P.cells_u; D.cv = P.cells_v; D.layout = P.layout; D.tracker = P.tracker;
        D.cell_base = cell;
        D.n_sub = L.n_sub;
        for (int k = 0; k < P.cells_u * P.cells_v; ++k) cell_mod.push_back(m);
        cell += P.cells_u * P.cells_v;
        g.max_cells = std::max(g.max_cells, P.cells_u * P.cells_v);
        // bounds: corners (fixed) or pivot +- reach (tracked)
        double lu = P.cells_u * (double)P.pitch, lv = P.cells_v * (double)P.pitch;
        double cx[4][3];
        for (int k = 0; k < 4; ++k) {
            double a = (k == 1 || k == 2) ? lu : 0, b = (k >= 2) ? lv : 0;
            for (int q = 0; q < 3; ++q) cx[k][q] = P.origin[q] + a * P.u[q] + b * P.v[q];
        }
        if (P.tracker < 0) {
            for (int q = 0; q < 3; ++q) { mlo[3 * m + q] = INFINITY; mhi[3 * m + q] = -INFINITY; }
            for (int k = 0; k < 4; ++k)
                for (int q = 0; q < 3; ++q) {
                    mlo[3 * m + q] = std::min(mlo[3 * m + q], cx[k][q]);
                    mhi[3 * m + q] = std::max(mhi[3 * m + q], cx[k][q]);
                }
        } else {
            double reach = 0;
            for (int k = 0; k < 4; ++k)
                reach = std::max(reach, std::sqrt(cx[k][0] * cx[k][0] + cx[k][1] * cx[k][1] + cx[k][2] * cx[k][2]));
            const float* pv = trackers[P.tracker].pivot;
            for (int q = 0; q < 3; ++q) {
                mlo[3 * m + q] = pv[q] - reach;
                mhi[3 * m + q] = pv[q] + reach;
            }
        }
        for (int q = 0; q < 3; ++q) {
            glo[q] = std::min(glo[q], mlo[3 * m + q]);
            ghi[q] = std::max(ghi[q], mhi[3 * m + q]);
        }
    }
    g.C = cell;
    for (int q = 0; q < 3; ++q) {
        g.ref[q] = (float)(0.5 * (glo[q] + ghi[q]));
        g.glo[q] = (float)glo[q];
        g.ghi[q] = (float)ghi[q];
    }
    // coplanar generator: every module fixed, one plane, one facing -> modules
    // cannot shade one another and are left out of the depth map
    {
        bool cop = true;
        double n0[3] = {0, 0, 0};
        for (int32_t m = 0; m < n_mods && cop; ++m) {
            const pv3d_module& P = mods[m];
            if (P.tracker >= 0) { cop = false; break; }
            double n[3] = {(double)P.u[1] * P.v[2] - (double)P.u[2] * P.v[1],
                           (double)P.u[2] * P.v[0] - (double)P.u[0] * P.v[2],
                           (double)P.u[0] * P.v[1] - (double)P.u[1] * P.v[0]};
            double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            for (int q = 0; q < 3; ++q) n[q] /= l;
            if (m == 0) {
                for (int q = 0; q < 3; ++q) n0[q] = n[q];
                continue;
            }
            double dn = n[0] * n0[0] + n[1] * n0[1] + n[2] * n0[2];
            double off = 0;
            for (int q = 0; q < 3; ++q) off += n0[q] * ((double)P.origin[q] - mods[0].origin[q]);
            if (dn < 1.0 - 1e-9 || std::fabs(off) > 1e-4) cop = false;
        }
        g.coplanar = cop;
    }
    // plane groups: the modules of one tracker that share one plane in the
    // tracker's frame (a pose moves them together), and fixed modules that
    // share one plane in the world, lie in one plane under every pose and
    // cannot shade one another (a ray leaving a plane does not meet it again)
    {
        struct PlaneKey {
            int32_t tracker;
            double n[3], off;
        };
        std::vector<PlaneKey> groups;
        std::map<std::pair<int32_t, long long>, std::vector<int32_t>> index;  // (tracker, offset bucket) -> groups
        for (int32_t m = 0; m < n_mods; ++m) {
            const pv3d_module& P = mods[m];
            double n[3] = {(double)P.u[1] * P.v[2] - (double)P.u[2] * P.v[1],
                           (double)P.u[2] * P.v[0] - (double)P.u[0] * P.v[2],
                           (double)P.u[0] * P.v[1] - (double)P.u[1] * P.v[0]};
            const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            for (int q = 0; q < 3; ++q) n[q] /= l;
            const double off = n[0] * P.origin[0] + n[1] * P.origin[1] + n[2] * P.origin[2];
            const std::pair<int32_t, long long> key(P.tracker, (long long)std::floor(off * 1e3));
            int32_t id = -1;
            for (int32_t cand : index[key]) {
                const PlaneKey& G = groups[(size_t)cand];
                const double dn = n[0] * G.n[0] + n[1] * G.n[1] + n[2] * G.n[2];
                if (dn >= 1.0 - 1e-12 && std::fabs(off - G.off) <= 1e-6) { id = cand; break; }
            }
            if (id < 0) {
                id = (int32_t)groups.size();
                groups.push_back(PlaneKey{P.tracker, {n[0], n[1], n[2]}, off});
                index[key].push_back(id);
            }
            g.mods_h[m].plane = id;
        }
    }
    // positions relative to the reference point
    for (auto& D : g.mods_h)
        if (D.tracker < 0)
            for (int a = 0; a < 3; ++a) D.o[a] -= g.ref[a];
    std::vector<float> piv((size_t)n_trackers * 3);
    for (int32_t t = 0; t < n_trackers; ++t)
        for (int a = 0; a < 3; ++a) piv[3 * t + a] = trackers[t].pivot[a] - g.ref[a];
    // series strings: rank the string ids, number the substrings string by string
    std::vector<int32_t> str_sub, sub_base(n_mods), sub_nk, sub_mod;
    {
        for (int32_t m = 0; m < n_mods; ++m) g.str_ids.push_back(mods[m].string_id);
        std::sort(g.str_ids.begin(), g.str_ids.end());
        g.str_ids.erase(std::unique(g.str_ids.begin(), g.str_ids.end()), g.str_ids.end());
        std::vector<std::vector<int32_t>> members(g.str_ids.size());
        for (int32_t m = 0; m < n_mods; ++m) {
            const size_t q = std::lower_bound(g.str_ids.begin(), g.str_ids.end(), mods[m].string_id) - g.str_ids.begin();
            members[q].push_back(m);
        }
        for (auto& mem : members) {
            str_sub.push_back((int32_t)sub_nk.size());
            for (int32_t m : mem) {
                sub_base[m] = (int32_t)sub_nk.size();
                const int32_t lay = mods[m].layout;
                for (int k = 0; k < layouts[lay].n_sub; ++k) {
                    sub_nk.push_back(lay_nk[lay_nk_off[lay] + k]);
                    sub_mod.push_back(m);
                }
            }
        }
        str_sub.push_back((int32_t)sub_nk.size());
        g.n_sub_tot = (int32_t)sub_nk.size();
    }
    // arrays of parallel strings: every module of a string names the same array
    std::vector<int32_t> arr_off, arr_strs;
    {
        const size_t NS = g.str_ids.size();
        std::vector<int32_t> str_arr(NS, INT32_MIN);
        for (int32_t m = 0; m < n_mods; ++m) {
            const size_t q = std::lower_bound(g.str_ids.begin(), g.str_ids.end(), mods[m].string_id) - g.str_ids.begin();
            if (str_arr[q] == INT32_MIN) str_arr[q] = mods[m].array_id;
            else if (str_arr[q] != mods[m].array_id)
                return fail(c, PV3D_E_INVALID, "string %d: its modules name different array_id values",
                            mods[m].string_id);
        }
        g.arr_ids = str_arr;
        std::sort(g.arr_ids.begin(), g.arr_ids.end());
        g.arr_ids.erase(std::unique(g.arr_ids.begin(), g.arr_ids.end()), g.arr_ids.end());
        std::vector<std::vector<int32_t>> members(g.arr_ids.size());
        for (size_t q = 0; q < NS; ++q)
            members[std::lower_bound(g.arr_ids.begin(), g.arr_ids.end(), str_arr[q]) - g.arr_ids.begin()].push_back((int32_t)q);
        for (auto& mem : members) {
            arr_off.push_back((int32_t)arr_strs.size());
            int32_t nsub = 0;
            for (int32_t q : mem) {
                arr_strs.push_back(q);
                nsub += str_sub[q + 1] - str_sub[q];
            }
            g.max_arr_sub = std::max(g.max_arr_sub, nsub);
        }
        arr_off.push_back((int32_t)arr_strs.size());
    }
    // occluder meshlets for window groups: modules 16q .. 16q + 15 (triangles
    // 32q .. 32q + 31), boxes widened by a millimetre for the rounding of poses
    g.n_oml = (n_mods + 15) / 16;
    std::vector<float4> oml((size_t)2 * g.n_oml);
    for (int32_t q = 0; q < g.n_oml; ++q) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t m = 16 * q; m < std::min(n_mods, 16 * q + 16); ++m)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], mlo[3 * m + a]);
                hi[a] = std::max(hi[a], mhi[3 * m + a]);
            }
        oml[2 * q] = make_float4((float)(lo[0] - 1e-3), (float)(lo[1] - 1e-3), (float)(lo[2] - 1e-3), 0.f);
        oml[2 * q + 1] = make_float4((float)(hi[0] + 1e-3), (float)(hi[1] + 1e-3), (float)(hi[2] + 1e-3), 0.f);
    }
    int rc;
    if ((rc = upload(c, &g.d_oml, oml.data(), oml.size())) ||
        (rc = upload(c, &g.d_mods, g.mods_h.data(), g.mods_h.size())) ||
        (rc = upload(c, &g.d_cell_mod, cell_mod.data(), cell_mod.size())) ||
        (rc = upload(c, &g.d_lay_sub, lay_sub.data(), lay_sub.size())) ||
        (rc = upload(c, &g.d_lay_off, lay_off.data(), lay_off.size())) ||
        (rc = upload(c, &g.d_lay_nk, lay_nk.data(), lay_nk.size())) ||
        (rc = upload(c, &g.d_lay_nk_off, lay_nk_off.data(), lay_nk_off.size())) ||
        (rc = upload(c, &g.d_pivots, piv.data(), piv.size())) ||
        (rc = upload(c, &g.d_str_sub, str_sub.data(), str_sub.size())) ||
        (rc = upload(c, &g.d_sub_base, sub_base.data(), sub_base.size())) ||
        (rc = upload(c, &g.d_sub_nk, sub_nk.data(), sub_nk.size())) ||
        (rc = upload(c, &g.d_sub_mod, sub_mod.data(), sub_mod.size())) ||
        (rc = upload(c, &g.d_arr_off, arr_off.data(), arr_off.size())) ||
        (rc = upload(c, &g.d_arr_strs, arr_strs.data(), arr_strs.size()))) {
        free_gen(g);
        return rc;
    }
    g.bytes = g.mods_h.size() * sizeof(ModuleDev) + cell_mod.size() * 4 + lay_sub.size() * 8 + piv.size() * 4 +
              (str_sub.size() + sub_base.size() + 2 * sub_nk.size()) * 4 + oml.size() * sizeof(float4);
    uint32_t id = c->next_id++;
    c->gens[id] = std::move(g);
    *gen_id = id;
    return PV3D_OK;
}

extern "C" int pv3d_generator_strings(pv3d_ctx* c, uint32_t gen_id, int32_t* n_strings, int32_t* string_ids)
{
    if (!c || !n_strings) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    *n_strings = (int32_t)it->second.str_ids.size();
    if (string_ids) std::copy(it->second.str_ids.begin(), it->second.str_ids.end(), string_ids);
    return PV3D_OK;
}

extern "C" int pv3d_generator_arrays(pv3d_ctx* c, uint32_t gen_id, int32_t* n_arrays, int32_t* array_ids)
{
    if (!c || !n_arrays) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    *n_arrays = (int32_t)it->second.arr_ids.size();
    if (array_ids) std::copy(it->second.arr_ids.begin(), it->second.arr_ids.end(), array_ids);
    return PV3D_OK;
}

// Diffuse fractions of a tracked generator are tied to the poses and steps
// they were binned with: a new pose or sun table drops them.
static void drop_tracked_diffuse(GenH& g)
{
    if (!g.n_trk) return;
    if (g.d_fdiff) cudaFree(g.d_fdiff);
    if (g.d_fbin) cudaFree(g.d_fbin);
    g.d_fdiff = nullptr;
    g.d_fbin = nullptr;
    g.fdiff_bins = 0;
}

extern "C" int pv3d_set_poses(pv3d_ctx* c, uint32_t gen_id, const float* az_tilt, int64_t n_steps)
{
    if (!c) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    GenH& g = it->second;
    if (n_steps < 1 || !az_tilt) return fail(c, PV3D_E_INVALID, "empty pose table");
    if (g.n_steps && n_steps != g.n_steps) return fail(c, PV3D_E_INVALID, "pose table length differs from the sun table");
    size_t n = (size_t)n_steps * (size_t)g.n_trk * 2;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(az_tilt[k])) return fail(c, PV3D_E_INVALID, "pose %zu not finite", k / 2);
    cudaSetDevice(c->device);
    drop_tracked_diffuse(g);
    if (g.d_poses) cudaFree(g.d_poses);
    g.d_poses = nullptr;
    int rc = upload(c, &g.d_poses, az_tilt, n);
    if (rc) return rc;
    g.n_pose_steps = n_steps;
    return PV3D_OK;
}

extern "C" int pv3d_set_sun(pv3d_ctx* c, uint32_t gen_id, const double* sun_xyz, const float* dni, const float* dhi,
                            const float* dt_h, int64_t n_steps)
{
    if (!c) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    GenH& g = it->second;
    if (n_steps < 1 || n_steps > (1ll << 30) || !sun_xyz || !dni || !dhi || !dt_h)
        return fail(c, PV3D_E_INVALID, "bad sun table");
    if (g.n_pose_steps && g.n_trk && n_steps != g.n_pose_steps)
        return fail(c, PV3D_E_INVALID, "sun table length differs from the pose table");
    std::vector<uint8_t> lit((size_t)n_steps);
    for (int64_t k = 0; k < n_steps; ++k) {
        const double* s = sun_xyz + 3 * k;
        if (!std::isfinite(s[0]) || !std::isfinite(s[1]) || !std::isfinite(s[2]))
            return fail(c, PV3D_E_INVALID, "sun %lld not finite", (long long)k);
        double l = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        if (std::fabs(l - 1.0) > 1e-6) return fail(c, PV3D_E_INVALID, "sun %lld: |s| = %.9f is not 1", (long long)k, l);
        if (!std::isfinite(dni[k]) || !std::isfinite(dhi[k]) || !std::isfinite(dt_h[k]) || dni[k] < 0 || dhi[k] < 0 ||
            dt_h[k] < 0)
            return fail(c, PV3D_E_INVALID, "irradiance or duration %lld invalid", (long long)k);
        lit[k] = s[2] > 0.0;
    }
    cudaSetDevice(c->device);
    drop_tracked_diffuse(g);
    void* olds[] = {g.d_sun, g.d_dni, g.d_dhi, g.d_dt};
    for (void* p : olds)
        if (p) cudaFree(p);
    g.d_sun = nullptr; g.d_dni = g.d_dhi = g.d_dt = nullptr;
    int rc;
    if ((rc = upload(c, &g.d_sun, sun_xyz, (size_t)n_steps * 3)) || (rc = upload(c, &g.d_dni, dni, (size_t)n_steps)) ||
        (rc = upload(c, &g.d_dhi, dhi, (size_t)n_steps)) || (rc = upload(c, &g.d_dt, dt_h, (size_t)n_steps)))
        return rc;
    g.n_steps = n_steps;
    g.lit = std::move(lit);
    return PV3D_OK;
}

extern "C" int pv3d_sun_table(pv3d_ctx* c, uint32_t gen_id, double* sun_xyz, float* dni, float* dhi, float* dt_h,
                              int64_t n_steps)
{
    if (!c) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    const GenH& g = it->second;
    if (n_steps != g.n_steps || n_steps < 1) return fail(c, PV3D_E_INVALID, "the sun table has %lld steps",
                                                          (long long)g.n_steps);
    cudaSetDevice(c->device);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (sun_xyz) CUDA_TRY(c, cudaMemcpy(sun_xyz, g.d_sun, (size_t)n_steps * 24, cudaMemcpyDeviceToHost));
    if (dni) CUDA_TRY(c, cudaMemcpy(dni, g.d_dni, (size_t)n_steps * 4, cudaMemcpyDeviceToHost));
    if (dhi) CUDA_TRY(c, cudaMemcpy(dhi, g.d_dhi, (size_t)n_steps * 4, cudaMemcpyDeviceToHost));
    if (dt_h) CUDA_TRY(c, cudaMemcpy(dt_h, g.d_dt, (size_t)n_steps * 4, cudaMemcpyDeviceToHost));
    return PV3D_OK;
}

extern "C" int pv3d_set_sun_clear_sky(pv3d_ctx* c, uint32_t gen_id, const pv3d_sky_opts* o, int64_t* n_steps)
{
    if (!c || !o) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    GenH& g = it->second;
    if (!(std::fabs(o->latitude_deg) <= 89.9) || !(o->step_h > 0.0 && o->step_h <= 24.0) || o->day_first < 1 ||
        o->day_first > 366 || o->n_days < 1 || o->n_days > 3660 || !(o->dhi_fraction >= 0.f) ||
        !(o->tracker_tilt_max_deg >= 0.f && o->tracker_tilt_max_deg <= 90.f))
        return fail(c, PV3D_E_INVALID, "clear-sky options out of range");
    int64_t per_day = 0;
    while ((double)per_day * o->step_h < 24.0 - 1e-9) ++per_day;
    const int64_t n_all = per_day * o->n_days;
    if (n_all > (1ll << 30)) return fail(c, PV3D_E_INVALID, "sun table too long");
    const double dhi_f = o->dhi_fraction > 0.f ? o->dhi_fraction : 0.1;
    cudaSetDevice(c->device);
    drop_tracked_diffuse(g);
    cudaStream_t st = c->stream;
    double* d_xyz = nullptr;
    float *d_dni = nullptr, *d_dhi = nullptr, *d_dt = nullptr, *d_poses = nullptr;
    uint8_t* d_lit = nullptr;
    int64_t* d_idx = nullptr;
    auto cleanup = [&]() {
        void* ps[] = {d_xyz, d_dni, d_dhi, d_dt, d_lit, d_idx, d_poses};
        for (void* p : ps)
            if (p) cudaFree(p);
    };
    if (cudaMalloc(&d_xyz, (size_t)n_all * 24) != cudaSuccess || cudaMalloc(&d_dni, (size_t)n_all * 4) != cudaSuccess ||
        cudaMalloc(&d_dhi, (size_t)n_all * 4) != cudaSuccess || cudaMalloc(&d_dt, (size_t)n_all * 4) != cudaSuccess ||
        cudaMalloc(&d_lit, (size_t)n_all) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(c, PV3D_E_NOMEM, "sun table of %lld steps", (long long)n_all);
    }
    std::vector<uint8_t> lit((size_t)n_all);
    if (launch_sun_table(o->latitude_deg, o->day_first, per_day, o->step_h, dhi_f, n_all, d_xyz, d_dni, d_dhi, d_dt,
                         d_lit, st) != cudaSuccess ||
        cudaMemcpyAsync(lit.data(), d_lit, (size_t)n_all, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cleanup();
        return fail(c, PV3D_E_DEVICE, "sun table kernel: %s", cudaGetErrorString(cudaGetLastError()));
    }
    int64_t n = n_all;
    if (o->daylight_only) {
        std::vector<int64_t> idx;
        for (int64_t k = 0; k < n_all; ++k)
            if (lit[k]) idx.push_back(k);
        n = (int64_t)idx.size();
        if (n == 0) {
            cleanup();
            return fail(c, PV3D_E_INVALID, "no daylight step in the requested period");
        }
        double* k_xyz = nullptr;
        float *k_dni = nullptr, *k_dhi = nullptr;
        if (cudaMalloc(&d_idx, (size_t)n * 8) != cudaSuccess || cudaMalloc(&k_xyz, (size_t)n * 24) != cudaSuccess ||
            cudaMalloc(&k_dni, (size_t)n * 4) != cudaSuccess || cudaMalloc(&k_dhi, (size_t)n * 4) != cudaSuccess) {
            if (k_xyz) cudaFree(k_xyz);
            if (k_dni) cudaFree(k_dni);
            if (k_dhi) cudaFree(k_dhi);
            cleanup();
            cudaGetLastError();
            return fail(c, PV3D_E_NOMEM, "sun table");
        }
        if (cudaMemcpyAsync(d_idx, idx.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            launch_gather_sun(d_idx, n, d_xyz, d_dni, d_dhi, k_xyz, k_dni, k_dhi, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaFree(k_xyz); cudaFree(k_dni); cudaFree(k_dhi);
            cleanup();
            return fail(c, PV3D_E_DEVICE, "sun table gather: %s", cudaGetErrorString(cudaGetLastError()));
        }
        cudaFree(d_xyz); cudaFree(d_dni); cudaFree(d_dhi);
        d_xyz = k_xyz; d_dni = k_dni; d_dhi = k_dhi;
        lit.assign((size_t)n, 1);  // d_dt holds step_h in its first n entries
    }
    const bool poses = o->tracker_tilt_max_deg > 0.f && g.n_trk > 0;
    if (poses) {
        if (cudaMalloc(&d_poses, (size_t)n * g.n_trk * 8) != cudaSuccess) {
            cleanup();
            cudaGetLastError();
            return fail(c, PV3D_E_NOMEM, "pose table");
        }
        if (launch_ideal_poses(d_xyz, n, g.n_trk, o->tracker_tilt_max_deg * 0.017453292519943295f, d_poses, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            return fail(c, PV3D_E_DEVICE, "pose kernel: %s", cudaGetErrorString(cudaGetLastError()));
        }
    } else if (g.n_trk > 0 && g.n_pose_steps && g.n_pose_steps != n) {
        cleanup();
        return fail(c, PV3D_E_INVALID, "sun table length differs from the pose table");
    }
    void* olds[] = {g.d_sun, g.d_dni, g.d_dhi, g.d_dt};
    for (void* p : olds)
        if (p) cudaFree(p);
    g.d_sun = d_xyz; g.d_dni = d_dni; g.d_dhi = d_dhi; g.d_dt = d_dt;
    g.n_steps = n;
    g.lit = std::move(lit);
    if (poses) {
        if (g.d_poses) cudaFree(g.d_poses);
        g.d_poses = d_poses;
        g.n_pose_steps = n;
    }
    if (d_lit) cudaFree(d_lit);
    if (d_idx) cudaFree(d_idx);
    if (n_steps) *n_steps = n;
    return PV3D_OK;
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------
namespace {

struct EvalSetup {
    int n, R, K, tile, fused, profile, count, strings, heat, diffuse, arrays, groups;
    int64_t b, e;
    float i_ref, v_cell, v_diode;
};

}  // namespace

static int check_eval(pv3d_ctx* c, const GenH& g, const pv3d_eval_opts* o, const pv3d_result* out, EvalSetup& es)
{
    pv3d_eval_opts d{};
    if (o) d = *o;
    es.n = d.samples_per_side ? d.samples_per_side : 3;
    es.R = d.map_res ? d.map_res : c->opts.map_res;
    es.K = d.chunk_steps ? d.chunk_steps : c->opts.chunk_steps;
    es.tile = c->opts.tile;
    if (d.path != PV3D_PATH_FUSED && d.path != PV3D_PATH_MAP) return fail(c, PV3D_E_INVALID, "unknown path");
    es.fused = d.path == PV3D_PATH_FUSED;
    es.profile = (d.profile & 1) != 0;  // stage events
    es.count = (d.profile & 2) != 0;    // work counters
    es.i_ref = d.i_ref > 0 ? d.i_ref : 9.0f;
    es.v_cell = d.v_cell > 0 ? d.v_cell : 0.5f;
    es.v_diode = d.v_diode > 0 ? d.v_diode : 0.5f;
    if (es.n < 1 || es.n > 15) return fail(c, PV3D_E_INVALID, "samples_per_side must be 1..15");
    if (es.R < 64 || es.R > 16384 || (es.R & (es.R - 1))) return fail(c, PV3D_E_INVALID, "map_res must be a power of two in 64..16384");
    if (es.K < 1 || es.K > 256) return fail(c, PV3D_E_INVALID, "chunk_steps must be 1..256");
    if (g.n_steps < 1) return fail(c, PV3D_E_INVALID, "no sun table set");
    if (g.n_trk > 0 && g.n_pose_steps != g.n_steps) return fail(c, PV3D_E_INVALID, "tracker poses missing");
    es.b = d.step_begin;
    es.e = d.step_end ? d.step_end : g.n_steps;
    if (es.b < 0 || es.e > g.n_steps || es.b >= es.e) return fail(c, PV3D_E_INVALID, "bad step range");
    if (!out) return fail(c, PV3D_E_INVALID, "null result");
    if (out->sample_bits && es.n > 8) return fail(c, PV3D_E_INVALID, "sample_bits needs samples_per_side <= 8");
    es.diffuse = d.diffuse_shading != 0;
    if (es.diffuse && !g.d_fdiff) return fail(c, PV3D_E_INVALID, "diffuse_shading needs pv3d_sky_view first");
    es.arrays = out->array_energy || out->array_energy_unshaded || out->array_power || out->array_power_unshaded;
    if (es.arrays && g.max_arr_sub > kMaxArraySub)
        return fail(c, PV3D_E_INVALID, "an array holds %d bypass substrings (at most %d)", g.max_arr_sub, kMaxArraySub);
    es.strings = out->string_energy || out->string_energy_unshaded || out->string_power || out->string_power_unshaded ||
                 es.arrays;
    es.heat = out->heat_az_bins > 0 || out->heat_zen_bins > 0 || out->heat_energy || out->heat_energy_unshaded ||
              out->heat_steps;
    if (es.heat && (out->heat_az_bins < 1 || out->heat_az_bins > 1024 || out->heat_zen_bins < 1 ||
                    out->heat_zen_bins > 1024 || !out->heat_energy || !out->heat_energy_unshaded || !out->heat_steps))
        return fail(c, PV3D_E_INVALID, "heat map: bin counts 1..1024 and all three arrays");
    es.groups = d.window_groups;
    if (es.groups < PV3D_WINDOWS_ONE || es.groups > PV3D_WINDOWS_PER_ARRAY)
        return fail(c, PV3D_E_INVALID, "unknown window_groups mode %d", es.groups);
    if (es.groups && (es.strings || es.heat))
        return fail(c, PV3D_E_INVALID, "window groups: string, array and heat-map outputs are not supported");
    return PV3D_OK;
}

// The window groups of generator g under `mode` (PV3D_WINDOWS_PER_*): runs of
// consecutive modules with the same tracker, string or array id.  Built on
// first use and kept with the generator.
static int window_groups(pv3d_ctx* c, GenH& g, int mode, const GenH::WinGroups** out)
{
    auto it = g.wgroups.find(mode);
    if (it != g.wgroups.end()) {
        *out = &it->second;
        return PV3D_OK;
    }
    auto key = [&](int32_t m) {
        return mode == PV3D_WINDOWS_PER_TRACKER ? std::max(g.mods_h[m].tracker, -1)
                                                : (mode == PV3D_WINDOWS_PER_STRING ? g.mod_string[m] : g.mod_array[m]);
    };
    GenH::WinGroups wg;
    std::vector<int32_t> seen;
    for (int32_t m = 0; m < g.M; ++m)
        if (m == 0 || key(m) != key(m - 1)) {
            if (std::find(seen.begin(), seen.end(), key(m)) != seen.end())
                return fail(c, PV3D_E_INVALID, "window groups: the modules of group %d are not consecutive", key(m));
            seen.push_back(key(m));
            wg.m0.push_back(m);
            wg.c0.push_back(g.mods_h[m].cell_base);
        }
    wg.m0.push_back(g.M);
    wg.c0.push_back(g.C);
    // module tables and cell -> module maps numbered within each group
    std::vector<ModuleDev> local = g.mods_h;
    std::vector<int32_t> cell_mod((size_t)g.C);
    for (size_t q = 0; q + 1 < wg.m0.size(); ++q)
        for (int32_t m = wg.m0[q]; m < wg.m0[q + 1]; ++m) {
            local[m].cell_base -= wg.c0[q];
            for (int32_t k = 0; k < local[m].cu * local[m].cv; ++k)
                cell_mod[(size_t)g.mods_h[m].cell_base + k] = m - wg.m0[q];
        }
    int rc;
    if ((rc = upload(c, &wg.d_mods, local.data(), local.size())) ||
        (rc = upload(c, &wg.d_cell_mod, cell_mod.data(), cell_mod.size()))) {
        if (wg.d_mods) cudaFree(wg.d_mods);
        return rc;
    }
    g.bytes += local.size() * sizeof(ModuleDev) + cell_mod.size() * 4;
    *out = &(g.wgroups[mode] = std::move(wg));
    return PV3D_OK;
}

// Fill a JobDev for generator g over steps [step0, step0 + k).
static JobDev make_job(pv3d_ctx* c, const GenH& g, const SceneH& s, const EvalSetup& es, int64_t step0, int k,
                       float2* kmod, float2* kcell, float* pw, float* pwu, uint8_t* cnt, unsigned long long* bits,
                       float2* kstr = nullptr, float* spw = nullptr, float* spwu = nullptr, double* heat_e = nullptr,
                       double* heat_eu = nullptr, int32_t* heat_n = nullptr, int heat_az = 0, int heat_zen = 0,
                       float2* karr = nullptr, float* apw = nullptr, float* apwu = nullptr)
{
    JobDev J{};
    J.tri = s.d_tri;
    J.n_tris = s.n_tris;
    J.ml_box = s.d_ml;
    J.n_ml = s.n_ml;
    J.n_mtris = g.coplanar ? 0 : 2 * g.M;
    J.mods = g.d_mods;
    J.n_mods = g.M;
    J.n_cells = g.C;
    J.cell_mod = g.d_cell_mod;
    J.lay_sub = g.d_lay_sub;
    J.lay_off = g.d_lay_off;
    J.lay_nk = g.d_lay_nk;
    J.lay_nk_off = g.d_lay_nk_off;
    J.pivots = g.d_pivots;
    J.n_trk = g.n_trk;
    for (int a = 0; a < 3; ++a) {
        J.ref[a] = g.ref[a];
        float lo = s.n_tris ? std::min(s.lo[a], g.glo[a]) : g.glo[a];
        float hi = s.n_tris ? std::max(s.hi[a], g.ghi[a]) : g.ghi[a];
        J.scene_lo[a] = lo - g.ref[a];
        J.scene_hi[a] = hi - g.ref[a];
    }
    J.sun = g.d_sun;
    J.dni = g.d_dni;
    J.dhi = g.d_dhi;
    J.dt = g.d_dt;
    J.poses = g.d_poses;
    J.step0 = (int32_t)step0;
    J.k = k;
    J.out_row0 = (int32_t)(step0 - es.b);
    J.R = es.R;
    J.tiles_x = es.R / es.tile;
    J.n = es.n;
    J.nn = es.n * es.n;
    J.i_ref = es.i_ref;
    J.v_cell = es.v_cell;
    J.v_diode = es.v_diode;
    J.kahan_mod = kmod;
    J.kahan_cell = kcell;
    J.out_power = pw;
    J.out_power_u = pwu;
    J.out_counts = cnt;
    J.out_bits = bits;
    J.out_mstride = g.M;
    J.out_cstride = g.C;
    if (es.strings) {
        J.n_str = (int32_t)g.str_ids.size();
        J.n_sub_tot = g.n_sub_tot;
        J.str_sub = g.d_str_sub;
        J.sub_base = g.d_sub_base;
        J.sub_nk = g.d_sub_nk;
        J.sub_mod = g.d_sub_mod;
        J.kahan_str = kstr;
        J.out_str_power = spw;
        J.out_str_power_u = spwu;
    }
    J.fdiff = es.diffuse ? g.d_fdiff : nullptr;
    J.fbin = es.diffuse ? g.d_fbin : nullptr;
    J.fstride = g.C;
    if (es.arrays) {
        J.n_arr = (int32_t)g.arr_ids.size();
        J.arr_off = g.d_arr_off;
        J.arr_strs = g.d_arr_strs;
        J.kahan_arr = karr;
        J.out_arr_power = apw;
        J.out_arr_power_u = apwu;
    }
    if (heat_e) {
        J.heat_az = heat_az;
        J.heat_zen = heat_zen;
        J.heat_e = heat_e;
        J.heat_eu = heat_eu;
        J.heat_n = heat_n;
    }
    (void)c;
    return J;
}

// Lay out jobs[first, last) as one wave: bases and item offsets.
static WaveDev pack_wave(std::vector<JobDev>& jobs, size_t first, size_t last, int tile_sh, int u24, int fused,
                         int profile)
{
    WaveDev W{};
    W.profile = profile;
    W.n_jobs = (int32_t)(last - first);
    W.tile_sh = tile_sh;
    W.depth_u24 = u24;
    W.fused = fused;
    for (size_t q = first; q < last; ++q) {
        JobDev& J = jobs[q];
        J.js_base = (int32_t)W.tot_js;
        J.te_base = W.tot_te;
        J.ms_base = W.tot_ms;
        J.cs_base = W.tot_cs;
        J.it_win = W.tot_win;
        J.it_mod = W.tot_mod;
        J.it_tri = W.tot_tri;
        J.it_epi = W.tot_epi;
        J.ss_base = W.tot_ss;
        J.sq_base = W.tot_sq;
        J.it_str = W.tot_sq;
        J.it_heat = W.tot_heat;
        J.sa_base = W.tot_sa;
        int64_t groups = (J.n_mods + kWinPerItem - 1) / kWinPerItem;
        W.tot_js += J.k;
        W.tot_te += (int64_t)J.k * J.tiles_x * J.tiles_x;
        W.tot_ms += (int64_t)J.k * J.n_mods;
        W.tot_cs += (int64_t)J.k * J.n_cells;
        W.tot_win += (int64_t)J.k * groups;
        W.tot_mod += (int64_t)J.k * J.n_mods;
        W.tot_tri += (((int64_t)J.n_ml + J.n_oml + (J.n_mtris + 31) / 32 + 31) / 32) * J.k;  // groups of 32 meshlets
        W.tot_epi += (J.kahan_cell ? (int64_t)J.n_cells : 0) + J.n_mods + J.n_str + J.n_arr;
        W.tot_sa += (int64_t)J.k * J.n_arr;
        W.tot_ss += (int64_t)J.k * (J.n_str ? J.n_sub_tot : 0);
        W.tot_sq += (int64_t)J.k * J.n_str;
        W.tot_heat += (int64_t)J.heat_az * J.heat_zen;
        if (J.out_bits) W.want_bits = 1;
    }
    return W;
}

static int ensure_workspace(pv3d_ctx* c, int64_t js, int64_t te, int64_t ms, int64_t cs, int tile, bool fused,
                            bool want_bits, int64_t ss = 0, int64_t sq = 0, int64_t sa = 0)
{
    int rc;
    if (sa > 0 && ((rc = ensure(c, c->sa_p, sa * 4)) || (rc = ensure(c, c->sa_pu, sa * 4)))) return rc;
    if ((rc = ensure(c, c->js_p, js * 4)) || (rc = ensure(c, c->js_pu, js * 4)) || (rc = ensure(c, c->js_bin, js * 4)))
        return rc;
    if (sq > 0 && ((rc = ensure(c, c->ms_iu, ms * 4)) || (rc = ensure(c, c->ss_i, ss * 4)) ||
                   (rc = ensure(c, c->sq_p, sq * 4)) || (rc = ensure(c, c->sq_pu, sq * 4))))
        return rc;
    int64_t scan_tiles = (te + 4095) / 4096 + 1;
    if ((rc = ensure(c, c->lp, js * sizeof(LightParams))) || (rc = ensure(c, c->win, js * 16)) ||
        (rc = ensure(c, c->ms, ms * sizeof(ModStep))) || (rc = ensure(c, c->ms_p, ms * 4)) ||
        (rc = ensure(c, c->ms_pu, ms * 4)) || (rc = ensure(c, c->ms_beam, ms * 4)) ||
        (rc = ensure(c, c->cs_cnt, (cs + 3) / 4 * 4)) || (rc = ensure(c, c->t_far, te * 4)) ||
        (rc = ensure(c, c->t_cnt, te * 4)) || (rc = ensure(c, c->t_off, te * 4)) ||
        (rc = ensure(c, c->t_cur, te * 4)) || (rc = ensure(c, c->t_slot, te * 4)) ||
        (rc = ensure(c, c->t_rcnt, te * 4)) || (rc = ensure(c, c->t_plane, te * 4)) ||
        (rc = ensure(c, c->t_roff, te * 4)) ||
        (rc = ensure(c, c->t_rcur, te * 4)) || (rc = ensure(c, c->nonempty, te * 4)) || (rc = ensure(c, c->heavy, te * 4)) ||
        (rc = ensure(c, c->block_sums, scan_tiles * 24)) || (rc = ensure(c, c->ctr, sizeof(Counters))))
        return rc;
    if (fused && want_bits && (rc = ensure(c, c->cs_bits, cs * 8))) return rc;
    if (c->bin_cap == 0) c->bin_cap = 1 << 22;
    if (c->big_cap == 0) c->big_cap = 1 << 18;
    if (c->recv_cap == 0) c->recv_cap = 1 << 20;
    if ((rc = ensure(c, c->bins, c->bin_cap * 4)) || (rc = ensure(c, c->pairs, c->bin_cap * 8)) ||
        (rc = ensure(c, c->big, c->big_cap * 8)) ||
        (rc = ensure(c, c->recv, c->recv_cap * 4)))
        return rc;
    if (!fused) {
        if (c->map_cap_tiles == 0) c->map_cap_tiles = std::max<int64_t>(256, te / 8);
        c->map_cap_tiles = std::min<int64_t>(c->map_cap_tiles, te);
        if ((rc = ensure(c, c->map, (size_t)c->map_cap_tiles * tile * tile * 4))) return rc;
    }
    return PV3D_OK;
}

static Buffers buffers_of(pv3d_ctx* c)
{
    Buffers B;
    B.lp = (LightParams*)c->lp.p;
    B.win = (uint32_t*)c->win.p;
    B.ms = (ModStep*)c->ms.p;
    B.ms_p = (float*)c->ms_p.p;
    B.ms_pu = (float*)c->ms_pu.p;
    B.ms_beam = (float*)c->ms_beam.p;
    B.ms_iu = (float*)c->ms_iu.p;
    B.ss_i = (float*)c->ss_i.p;
    B.sq_p = (float*)c->sq_p.p;
    B.sq_pu = (float*)c->sq_pu.p;
    B.js_p = (float*)c->js_p.p;
    B.sa_p = (float*)c->sa_p.p;
    B.sa_pu = (float*)c->sa_pu.p;
    B.js_pu = (float*)c->js_pu.p;
    B.js_bin = (int32_t*)c->js_bin.p;
    B.cs_cnt = (uint32_t*)c->cs_cnt.p;
    B.cs_bits = (unsigned long long*)c->cs_bits.p;
    B.t_far = (uint32_t*)c->t_far.p;
    B.t_cnt = (uint32_t*)c->t_cnt.p;
    B.t_off = (uint32_t*)c->t_off.p;
    B.t_cur = (uint32_t*)c->t_cur.p;
    B.t_slot = (uint32_t*)c->t_slot.p;
    B.nonempty = (uint32_t*)c->nonempty.p;
    B.heavy = (uint32_t*)c->heavy.p;
    B.t_rcnt = (uint32_t*)c->t_rcnt.p;
    B.t_plane = (uint32_t*)c->t_plane.p;
    B.t_roff = (uint32_t*)c->t_roff.p;
    B.t_rcur = (uint32_t*)c->t_rcur.p;
    B.recv = (uint32_t*)c->recv.p;
    B.bins = (uint32_t*)c->bins.p;
    B.pairs = (uint2*)c->pairs.p;
    B.map = (uint32_t*)c->map.p;
    B.big = (uint2*)c->big.p;
    B.block_sums = (unsigned long long*)c->block_sums.p;
    B.ctr = (Counters*)c->ctr.p;
    return B;
}

static int stage_descriptors(pv3d_ctx* c, const std::vector<WaveDev>& waves, const std::vector<JobDev>& jobs,
                             cudaStream_t st)
{
    size_t wb = waves.size() * sizeof(WaveDev), jb = jobs.size() * sizeof(JobDev);
    int rc;
    if ((rc = ensure(c, c->waves, wb)) || (rc = ensure(c, c->jobs, jb))) return rc;
    if (c->h_stage_bytes < wb + jb) {
        if (c->h_stage) {
            cudaStreamSynchronize(st);
            cudaFreeHost(c->h_stage);
        }
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        size_t want = (wb + jb) * 2 + 4096;
        if (cudaMallocHost(&c->h_stage, want) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PV3D_E_NOMEM, "pinned staging allocation failed");
        }
        c->h_stage_bytes = want;
    } else {
        // the previous evaluation's copies must have left the staging buffer
        cudaStreamSynchronize(st);
    }
    memcpy(c->h_stage, waves.data(), wb);
    memcpy((char*)c->h_stage + wb, jobs.data(), jb);
    CUDA_TRY(c, cudaMemcpyAsync(c->waves.p, c->h_stage, wb, cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->jobs.p, (char*)c->h_stage + wb, jb, cudaMemcpyHostToDevice, st));
    return PV3D_OK;
}

// The wave sequence captured once as a CUDA graph; re-captured when a pool or
// the launch configuration changes.
static int wave_graph(pv3d_ctx* c, const LaunchCfg& cfg0, int max_jobs, cudaGraphExec_t* out)
{
    int rc;
    if ((rc = ensure(c, c->wave_slot, sizeof(WaveDev))) ||
        (rc = ensure(c, c->jobs_slot, (size_t)std::max(max_jobs, 1) * sizeof(JobDev))))
        return rc;
    const uint64_t key = (c->bufgen << 10) ^ ((uint64_t)cfg0.extras << 8) ^ ((uint64_t)cfg0.tile << 3) ^
                         ((uint64_t)cfg0.fused << 1) ^ (uint64_t)cfg0.profile;
    if (c->graph_exec && c->graph_key == key) {
        *out = c->graph_exec;
        return PV3D_OK;
    }
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    LaunchCfg cfg = cfg0;
    cfg.stream = c->cap_stream;
    cfg.ev = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_wave((const WaveDev*)c->wave_slot.p, (const JobDev*)c->jobs_slot.p, buffers_of(c), cfg, 0);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(c, PV3D_E_DEVICE, "wave graph capture failed: %s / %s", cudaGetErrorString(le),
                    cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph_exec = nullptr;
        return fail(c, PV3D_E_DEVICE, "wave graph instantiation failed: %s", cudaGetErrorString(ie));
    }
    c->graph_key = key;
    *out = c->graph_exec;
    return PV3D_OK;
}

// Run the planned waves: for each, copy its descriptors into the fixed slots
// and replay the captured graph (or launch the kernels when stage events are
// recorded).
static int run_waves(pv3d_ctx* c, const std::vector<WaveDev>& waves, cudaStream_t st, int tile, bool fused,
                     bool profile, bool count, int extras = 0)
{
    LaunchCfg cfg;
    cfg.extras = extras;
    cfg.sm_count = c->sm_count;
    cfg.tile = tile;
    cfg.fused = fused ? 1 : 0;
    cfg.profile = count ? 1 : 0;
    cfg.stream = st;
    cfg.ev = nullptr;
    if (profile) {
        const size_t need = waves.size() * (kStages + 1);
        while (c->prof_ev.size() < need) {
            cudaEvent_t e;
            CUDA_TRY(c, cudaEventCreate(&e));
            c->prof_ev.push_back(e);
        }
    }
    int max_jobs = 1;
    for (const WaveDev& W : waves) max_jobs = std::max(max_jobs, (int)W.n_jobs);
    cudaGraphExec_t exec = nullptr;
    int rc;
    const bool graph = c->use_graphs && !profile;
    if (graph) {
        if ((rc = wave_graph(c, cfg, max_jobs, &exec))) return rc;
    } else if ((rc = ensure(c, c->wave_slot, sizeof(WaveDev))) ||
               (rc = ensure(c, c->jobs_slot, (size_t)max_jobs * sizeof(JobDev)))) {
        return rc;
    }
    const Buffers B = buffers_of(c);
    const char* dW = (const char*)c->waves.p;
    const char* dJ = (const char*)c->jobs.p;
    size_t job0 = 0;
    for (size_t w = 0; w < waves.size(); ++w) {
        const WaveDev& W = waves[w];
        CUDA_TRY(c, cudaMemcpyAsync(c->wave_slot.p, dW + w * sizeof(WaveDev), sizeof(WaveDev),
                                    cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(c, cudaMemcpyAsync(c->jobs_slot.p, dJ + job0 * sizeof(JobDev), (size_t)W.n_jobs * sizeof(JobDev),
                                    cudaMemcpyDeviceToDevice, st));
        if (graph) {
            CUDA_TRY(c, cudaGraphLaunch(exec, st));
        } else {
            if (profile) cfg.ev = &c->prof_ev[w * (kStages + 1)];
            CUDA_TRY(c, launch_wave((const WaveDev*)c->wave_slot.p, (const JobDev*)c->jobs_slot.p, B, cfg, W.tot_te));
        }
        job0 += (size_t)W.n_jobs;
    }
    return PV3D_OK;
}

static int evaluate_plain(pv3d_ctx* c, uint32_t gen_id, const pv3d_eval_opts* o, pv3d_result* out)
{
    if (!c) return PV3D_E_INVALID;
    auto git = c->gens.find(gen_id);
    if (git == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    GenH& g = git->second;
    auto sit = c->scenes.find(g.scene_id);
    if (sit == c->scenes.end()) return fail(c, PV3D_E_NOTFOUND, "scene of generator %u is gone", gen_id);
    const SceneH& s = sit->second;
    EvalSetup es{};
    int rc = check_eval(c, g, o, out, es);
    if (rc) return rc;
    cudaSetDevice(c->device);
    cudaStream_t st = (o && o->stream) ? (cudaStream_t)o->stream : c->stream;
    const int64_t S = es.e - es.b;
    const int tile_sh = es.tile == 32 ? 5 : (es.tile == 64 ? 6 : 7);
    const int u24 = c->opts.depth_format == PV3D_DEPTH_U24;

    // result staging: device outputs are written in place, host outputs are
    // copied back from a device staging area at the end
    const bool dev = out->is_device != 0;
    size_t off_e = 0, off_eu = 0, off_cl = 0, off_p = 0, off_pu = 0, off_cnt = 0, off_bits = 0, tot = 0;
    size_t off_se = 0, off_seu = 0, off_sp = 0, off_spu = 0, off_ae = 0, off_aeu = 0, off_ap = 0, off_apu = 0;
    const int32_t NS = (int32_t)g.str_ids.size(), NA = (int32_t)g.arr_ids.size();
    auto take = [&](size_t bytes) {
        size_t o_ = tot;
        tot += (bytes + 255) & ~size_t(255);
        return o_;
    };
    if (!dev) {
        if (out->energy) off_e = take(g.M * 8);
        if (out->energy_unshaded) off_eu = take(g.M * 8);
        if (out->cell_beam_loss) off_cl = take((size_t)g.C * 8);
        if (out->power) off_p = take((size_t)S * g.M * 4);
        if (out->power_unshaded) off_pu = take((size_t)S * g.M * 4);
        if (out->cell_counts) off_cnt = take((size_t)S * g.C);
        if (out->sample_bits) off_bits = take((size_t)S * g.C * 8);
        if (out->string_energy) off_se = take((size_t)NS * 8);
        if (out->string_energy_unshaded) off_seu = take((size_t)NS * 8);
        if (out->string_power) off_sp = take((size_t)S * NS * 4);
        if (out->string_power_unshaded) off_spu = take((size_t)S * NS * 4);
        if (out->array_energy) off_ae = take((size_t)NA * 8);
        if (out->array_energy_unshaded) off_aeu = take((size_t)NA * 8);
        if (out->array_power) off_ap = take((size_t)S * NA * 4);
        if (out->array_power_unshaded) off_apu = take((size_t)S * NA * 4);
        if ((rc = ensure(c, c->staging, tot))) return rc;
    }
    char* sb = (char*)c->staging.p;
    double* d_e = dev ? out->energy : (out->energy ? (double*)(sb + off_e) : nullptr);
    double* d_eu = dev ? out->energy_unshaded : (out->energy_unshaded ? (double*)(sb + off_eu) : nullptr);
    double* d_cl = dev ? out->cell_beam_loss : (out->cell_beam_loss ? (double*)(sb + off_cl) : nullptr);
    float* d_p = dev ? out->power : (out->power ? (float*)(sb + off_p) : nullptr);
    float* d_pu = dev ? out->power_unshaded : (out->power_unshaded ? (float*)(sb + off_pu) : nullptr);
    uint8_t* d_cnt = dev ? out->cell_counts : (out->cell_counts ? (uint8_t*)(sb + off_cnt) : nullptr);
    unsigned long long* d_bits =
        dev ? (unsigned long long*)out->sample_bits : (out->sample_bits ? (unsigned long long*)(sb + off_bits) : nullptr);
    double* d_se = dev ? out->string_energy : (out->string_energy ? (double*)(sb + off_se) : nullptr);
    double* d_seu = dev ? out->string_energy_unshaded : (out->string_energy_unshaded ? (double*)(sb + off_seu) : nullptr);
    float* d_sp = dev ? out->string_power : (out->string_power ? (float*)(sb + off_sp) : nullptr);
    float* d_spu = dev ? out->string_power_unshaded : (out->string_power_unshaded ? (float*)(sb + off_spu) : nullptr);
    double* d_ae = dev ? out->array_energy : (out->array_energy ? (double*)(sb + off_ae) : nullptr);
    double* d_aeu = dev ? out->array_energy_unshaded : (out->array_energy_unshaded ? (double*)(sb + off_aeu) : nullptr);
    float* d_ap = dev ? out->array_power : (out->array_power ? (float*)(sb + off_ap) : nullptr);
    float* d_apu = dev ? out->array_power_unshaded : (out->array_power_unshaded ? (float*)(sb + off_apu) : nullptr);

    const int64_t n_bins = es.heat ? (int64_t)out->heat_az_bins * out->heat_zen_bins : 0;
    if ((rc = ensure(c, c->kahan_mod, (size_t)g.M * 2 * sizeof(float2))) ||
        (rc = ensure(c, c->kahan_cell, (size_t)g.C * sizeof(float2))) ||
        (es.strings && (rc = ensure(c, c->kahan_str, (size_t)NS * 2 * sizeof(float2)))) ||
        (es.arrays && (rc = ensure(c, c->kahan_arr, (size_t)NA * 2 * sizeof(float2)))) ||
        (es.heat && (rc = ensure(c, c->heat, (size_t)n_bins * 20))))
        return rc;
    double* h_e = es.heat ? (double*)c->heat.p : nullptr;
    double* h_eu = es.heat ? h_e + n_bins : nullptr;
    int32_t* h_n = es.heat ? (int32_t*)(h_eu + n_bins) : nullptr;

    // plan: a wave per chunk of steps, one job per window group (or one job)
    const GenH::WinGroups* wg = nullptr;
    if (es.groups && (rc = window_groups(c, g, es.groups, &wg))) return rc;
    const int n_groups = wg ? (int)wg->m0.size() - 1 : 1;
    int64_t K = es.K;
    if (wg) {  // at most 2^26 (group, step, tile) entries a wave
        const int64_t tiles = (int64_t)(es.R / es.tile) * (es.R / es.tile);
        K = std::max<int64_t>(1, std::min<int64_t>(K, (int64_t(1) << 26) / ((int64_t)n_groups * tiles)));
    }
    std::vector<JobDev> jobs;
    std::vector<WaveDev> waves;
    for (int64_t s0 = es.b; s0 < es.e; s0 += K) {
        int k = (int)std::min<int64_t>(K, es.e - s0);
        const size_t first = jobs.size();
        for (int q = 0; q < n_groups; ++q) {
            JobDev J = make_job(c, g, s, es, s0, k, (float2*)c->kahan_mod.p, d_cl ? (float2*)c->kahan_cell.p : nullptr,
                                d_p, d_pu,
                                d_cnt, d_bits, (float2*)c->kahan_str.p, d_sp, d_spu, h_e, h_eu, h_n,
                                es.heat ? out->heat_az_bins : 0, es.heat ? out->heat_zen_bins : 0,
                                (float2*)c->kahan_arr.p, d_ap, d_apu);
            if (wg) {
                // the group's modules and cells; every module of the generator
                // is an occluder (none when the generator is one plane)
                const int32_t m0 = wg->m0[q], c0 = wg->c0[q];
                J.mods = wg->d_mods + m0;
                J.n_mods = wg->m0[q + 1] - m0;
                J.n_cells = wg->c0[q + 1] - c0;
                J.cell_mod = wg->d_cell_mod + c0;
                J.kahan_mod += 2 * m0;
                if (J.kahan_cell) J.kahan_cell += c0;
                if (J.out_power) J.out_power += m0;
                if (J.out_power_u) J.out_power_u += m0;
                if (J.out_counts) J.out_counts += c0;
                if (J.out_bits) J.out_bits += c0;
                if (J.fdiff) J.fdiff += c0;
                J.n_mtris = 0;
                if (!g.coplanar) {
                    J.occ_mods = g.d_mods;
                    J.n_occ = g.M;
                    J.oml_box = g.d_oml;
                    J.n_oml = g.n_oml;
                }
            }
            jobs.push_back(J);
        }
        waves.push_back(pack_wave(jobs, first, jobs.size(), tile_sh, u24, es.fused, es.count));
    }
    int64_t mjs = 0, mte = 0, mms = 0, mcs = 0, mss = 0, msq = 0, msa = 0;
    for (auto& W : waves) {
        mjs = std::max(mjs, W.tot_js); mte = std::max(mte, W.tot_te);
        mms = std::max(mms, W.tot_ms); mcs = std::max(mcs, W.tot_cs);
        mss = std::max(mss, W.tot_ss); msq = std::max(msq, W.tot_sq); msa = std::max(msa, W.tot_sa);
    }
    const int extras = (es.strings ? 1 : 0) | (es.heat ? 2 : 0) | (es.arrays ? 4 : 0);
    Counters hc{};
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((rc = ensure_workspace(c, mjs, mte, mms, mcs, es.tile, es.fused, d_bits != nullptr, mss, msq, msa)))
            return rc;
        for (auto& W : waves) {
            W.bin_cap = c->bin_cap;
            W.map_cap_tiles = c->map_cap_tiles;
            W.big_cap = c->big_cap;
            W.recv_cap = c->recv_cap;
        }
        if ((rc = stage_descriptors(c, waves, jobs, st))) return rc;
        CUDA_TRY(c, cudaMemsetAsync(c->ctr.p, 0, sizeof(Counters), st));
        CUDA_TRY(c, cudaMemsetAsync(c->kahan_mod.p, 0, (size_t)g.M * 2 * sizeof(float2), st));
        CUDA_TRY(c, cudaMemsetAsync(c->kahan_cell.p, 0, (size_t)g.C * sizeof(float2), st));
        if (es.strings) CUDA_TRY(c, cudaMemsetAsync(c->kahan_str.p, 0, (size_t)NS * 2 * sizeof(float2), st));
        if (es.arrays) CUDA_TRY(c, cudaMemsetAsync(c->kahan_arr.p, 0, (size_t)NA * 2 * sizeof(float2), st));
        if (es.heat) CUDA_TRY(c, cudaMemsetAsync(c->heat.p, 0, (size_t)n_bins * 20, st));
        CUDA_TRY(c, cudaEventRecord(c->ev0, st));
        if ((rc = run_waves(c, waves, st, es.tile, es.fused, es.profile, es.count, extras))) return rc;
        CUDA_TRY(c, launch_finalize_pairs((const float2*)c->kahan_mod.p, g.M, (const float2*)c->kahan_cell.p,
                                          d_cl ? g.C : 0,
                                          d_e, d_eu, d_cl, st));
        if (es.strings)
            CUDA_TRY(c, launch_finalize_pairs((const float2*)c->kahan_str.p, NS, nullptr, 0, d_se, d_seu, nullptr, st));
        if (es.arrays)
            CUDA_TRY(c, launch_finalize_pairs((const float2*)c->kahan_arr.p, NA, nullptr, 0, d_ae, d_aeu, nullptr, st));
        if (es.heat) {
            const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CUDA_TRY(c, cudaMemcpyAsync(out->heat_energy, h_e, (size_t)n_bins * 8, kind, st));
            CUDA_TRY(c, cudaMemcpyAsync(out->heat_energy_unshaded, h_eu, (size_t)n_bins * 8, kind, st));
            CUDA_TRY(c, cudaMemcpyAsync(out->heat_steps, h_n, (size_t)n_bins * 4, kind, st));
        }
        CUDA_TRY(c, cudaEventRecord(c->ev1, st));
        CUDA_TRY(c, cudaMemcpyAsync(&hc, c->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        if (!hc.overflow) break;
        if (attempt == 3) return fail(c, PV3D_E_OVERFLOW, "bin/map capacity could not be grown far enough");
        if (hc.overflow & 1u) c->bin_cap = (int64_t)(hc.need_bins * 5 / 4 + 1024);
        if (hc.overflow & 2u) c->map_cap_tiles = (int64_t)(hc.need_tiles * 5 / 4 + 16);
        if (hc.overflow & 4u) c->big_cap = (int64_t)(hc.need_big * 5 / 4 + 1024);
        if (hc.overflow & 8u) c->recv_cap = (int64_t)(hc.need_recv * 5 / 4 + 1024);
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    if (!dev) {
        if (out->energy) CUDA_TRY(c, cudaMemcpy(out->energy, d_e, g.M * 8, cudaMemcpyDeviceToHost));
        if (out->energy_unshaded) CUDA_TRY(c, cudaMemcpy(out->energy_unshaded, d_eu, g.M * 8, cudaMemcpyDeviceToHost));
        if (out->cell_beam_loss) CUDA_TRY(c, cudaMemcpy(out->cell_beam_loss, d_cl, (size_t)g.C * 8, cudaMemcpyDeviceToHost));
        if (out->power) CUDA_TRY(c, cudaMemcpy(out->power, d_p, (size_t)S * g.M * 4, cudaMemcpyDeviceToHost));
        if (out->power_unshaded)
            CUDA_TRY(c, cudaMemcpy(out->power_unshaded, d_pu, (size_t)S * g.M * 4, cudaMemcpyDeviceToHost));
        if (out->cell_counts) CUDA_TRY(c, cudaMemcpy(out->cell_counts, d_cnt, (size_t)S * g.C, cudaMemcpyDeviceToHost));
        if (out->sample_bits)
            CUDA_TRY(c, cudaMemcpy(out->sample_bits, d_bits, (size_t)S * g.C * 8, cudaMemcpyDeviceToHost));
        if (out->string_energy) CUDA_TRY(c, cudaMemcpy(out->string_energy, d_se, (size_t)NS * 8, cudaMemcpyDeviceToHost));
        if (out->string_energy_unshaded)
            CUDA_TRY(c, cudaMemcpy(out->string_energy_unshaded, d_seu, (size_t)NS * 8, cudaMemcpyDeviceToHost));
        if (out->string_power)
            CUDA_TRY(c, cudaMemcpy(out->string_power, d_sp, (size_t)S * NS * 4, cudaMemcpyDeviceToHost));
        if (out->string_power_unshaded)
            CUDA_TRY(c, cudaMemcpy(out->string_power_unshaded, d_spu, (size_t)S * NS * 4, cudaMemcpyDeviceToHost));
        if (out->array_energy) CUDA_TRY(c, cudaMemcpy(out->array_energy, d_ae, (size_t)NA * 8, cudaMemcpyDeviceToHost));
        if (out->array_energy_unshaded)
            CUDA_TRY(c, cudaMemcpy(out->array_energy_unshaded, d_aeu, (size_t)NA * 8, cudaMemcpyDeviceToHost));
        if (out->array_power) CUDA_TRY(c, cudaMemcpy(out->array_power, d_ap, (size_t)S * NA * 4, cudaMemcpyDeviceToHost));
        if (out->array_power_unshaded)
            CUDA_TRY(c, cudaMemcpy(out->array_power_unshaded, d_apu, (size_t)S * NA * 4, cudaMemcpyDeviceToHost));
    }
    int64_t lit = 0;
    for (int64_t k = es.b; k < es.e; ++k) lit += g.lit[k];
    out->steps_lit = lit;
    out->tests = lit * (int64_t)g.C * es.n * es.n;
    out->device_ms = ms;
    out->waves = (int32_t)waves.size();
    out->nonempty_tiles = (int64_t)hc.stat_nonempty;
    out->binned_tris = (int64_t)hc.stat_bins;
    out->kernel_launches = (int64_t)waves.size() * ((es.fused ? kLaunchesPerWave : kLaunchesPerWaveMap) +
                                                    (es.strings ? 1 : 0) + (es.heat ? 2 : 0) + (es.arrays ? 1 : 0)) +
                           1 + (es.strings ? 1 : 0) + (es.arrays ? 1 : 0);
    if (es.profile || es.count) {
        pv3d_profile& P = c->last_prof;
        P = pv3d_profile{};
        P.n_stages = kStages;
        P.waves = (int32_t)waves.size();
        for (size_t w = 0; es.profile && w < waves.size(); ++w)
            for (int k = 0; k < kStages; ++k) {
                float t = 0;
                cudaEventElapsedTime(&t, c->prof_ev[w * (kStages + 1) + k], c->prof_ev[w * (kStages + 1) + k + 1]);
                P.stage_ms[k] += t;
            }
        P.device_ms = ms;
        P.sample_tests = (int64_t)hc.prof_samples;
        P.texel_visits = (int64_t)hc.prof_visits;
        P.texel_writes = (int64_t)hc.prof_writes;
        P.tris_culled = (int64_t)hc.prof_culled;
        P.candidates = (int64_t)hc.prof_cand;
        P.dense_tiles = (int64_t)hc.prof_dense;
        P.sample_tiles = (int64_t)hc.prof_stiles;
        P.pair_tests = (int64_t)hc.prof_pairs;
        P.heavy_tiles = (int64_t)hc.prof_h_tiles;
        P.heavy_sample_tests = (int64_t)hc.prof_h_samples;
        P.heavy_texel_writes = (int64_t)hc.prof_h_writes;
        for (int k = 0; k < 3; ++k) P.heavy_why[k] = (int64_t)hc.prof_heavy_why[k];
        P.nonempty_tiles = (int64_t)hc.stat_nonempty;
        P.binned_tris = (int64_t)hc.stat_bins;
        c->have_prof = true;
    }
    return PV3D_OK;
}

extern "C" int pv3d_last_profile(pv3d_ctx* c, pv3d_profile* out)
{
    if (!c || !out) return PV3D_E_INVALID;
    if (!c->have_prof) return fail(c, PV3D_E_NOTFOUND, "no profiled evaluation yet");
    *out = c->last_prof;
    return PV3D_OK;
}

extern "C" int pv3d_evaluate(pv3d_ctx* c, uint32_t gen_id, const pv3d_eval_opts* o, pv3d_result* out)
{
    if (!c) return PV3D_E_INVALID;
    std::lock_guard<std::mutex> g(c->gpu_mu);
    return evaluate_plain(c, gen_id, o, out);
}

// Pose bin of a tracker pose: compass azimuth in n_az equal sectors of
// [0, 2 pi), tilt in n_tilt equal bands of [0, pi/2]; bin = tilt band * n_az +
// azimuth sector.  Its centre pose is the middle of both ranges.
static int pose_bin(float az, float tilt, int n_az, int n_tilt)
{
    const double two_pi = 6.283185307179586, half_pi = 1.5707963267948966;
    double a = std::fmod((double)az, two_pi);
    if (a < 0) a += two_pi;
    const int ia = std::min(n_az - 1, std::max(0, (int)std::floor(a / two_pi * n_az)));
    const double t = std::min(half_pi, std::max(0.0, (double)tilt));
    const int it = std::min(n_tilt - 1, std::max(0, (int)std::floor(t / half_pi * n_tilt)));
    return it * n_az + ia;
}

extern "C" int pv3d_sky_view(pv3d_ctx* c, uint32_t gen_id, const pv3d_sky_view_opts* o, float* cell_fraction)
{
    if (!c) return PV3D_E_INVALID;
    auto it = c->gens.find(gen_id);
    if (it == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    GenH& g = it->second;
    pv3d_sky_view_opts d{};
    if (o) d = *o;
    const int rings = d.rings ? d.rings : 9, sectors = d.sectors ? d.sectors : 36;
    const int n = d.samples_per_side ? d.samples_per_side : 3;
    if (rings < 1 || rings > 90 || sectors < 1 || sectors > 360 || n < 1 || n > 15)
        return fail(c, PV3D_E_INVALID, "sky view: rings 1..90, sectors 1..360, samples_per_side 1..15");
    const bool tracked = g.n_trk > 0;
    const int n_az = tracked ? (d.pose_az_bins ? d.pose_az_bins : 12) : 1;
    const int n_tilt = tracked ? (d.pose_tilt_bins ? d.pose_tilt_bins : 6) : 1;
    if (n_az < 1 || n_az > 360 || n_tilt < 1 || n_tilt > 90)
        return fail(c, PV3D_E_INVALID, "sky view: pose_az_bins 1..360, pose_tilt_bins 1..90");
    if (tracked && (!g.d_poses || g.n_pose_steps != g.n_steps || g.n_steps < 1))
        return fail(c, PV3D_E_INVALID, "sky view of tracked modules: set the sun table and the poses first");
    const int nb = n_az * n_tilt;
    const int P = rings * sectors;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    // the pose bin of every step (tracked): the first tracker's pose
    std::vector<int32_t> bins;
    std::vector<int> used;
    if (tracked) {
        std::vector<float> p0((size_t)g.n_steps * 2);
        if (cudaMemcpy2D(p0.data(), 8, g.d_poses, (size_t)g.n_trk * 8, 8, (size_t)g.n_steps, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return fail(c, PV3D_E_DEVICE, "sky view: pose read-back: %s", cudaGetErrorString(cudaGetLastError()));
        bins.resize((size_t)g.n_steps);
        std::vector<char> seen((size_t)nb, 0);
        for (int64_t k = 0; k < g.n_steps; ++k) {
            bins[(size_t)k] = pose_bin(p0[2 * k], p0[2 * k + 1], n_az, n_tilt);
            if (g.lit[(size_t)k] && !seen[(size_t)bins[(size_t)k]]) {
                seen[(size_t)bins[(size_t)k]] = 1;
                used.push_back(bins[(size_t)k]);
            }
        }
        std::sort(used.begin(), used.end());
    } else {
        used.push_back(0);
    }
    double *xyz = nullptr, *dom = nullptr;
    float *dni = nullptr, *dhi = nullptr, *dt = nullptr, *bposes = nullptr, *fdiff = nullptr;
    int32_t* fbin = nullptr;
    uint8_t* counts = nullptr;
    auto cleanup = [&]() {
        void* ps[] = {xyz, dom, dni, dhi, dt, counts, bposes, fdiff, fbin};
        for (void* p : ps)
            if (p) cudaFree(p);
    };
    if (cudaMalloc(&xyz, (size_t)P * 24) != cudaSuccess || cudaMalloc(&dom, (size_t)P * 8) != cudaSuccess ||
        cudaMalloc(&dni, (size_t)P * 4) != cudaSuccess || cudaMalloc(&dhi, (size_t)P * 4) != cudaSuccess ||
        cudaMalloc(&dt, (size_t)P * 4) != cudaSuccess || cudaMalloc(&counts, (size_t)P * g.C) != cudaSuccess ||
        cudaMalloc(&fdiff, (size_t)nb * g.C * 4) != cudaSuccess ||
        (tracked && (cudaMalloc(&bposes, (size_t)P * g.n_trk * 8) != cudaSuccess ||
                     cudaMalloc(&fbin, (size_t)g.n_steps * 4) != cudaSuccess))) {
        cleanup();
        cudaGetLastError();
        return fail(c, PV3D_E_NOMEM, "sky view buffers");
    }
    if (cudaMemsetAsync(fdiff, 0, (size_t)nb * g.C * 4, st) != cudaSuccess ||
        (tracked && cudaMemcpy(fbin, bins.data(), bins.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
        launch_sky_patches(rings, sectors, xyz, dni, dhi, dt, dom, st) != cudaSuccess) {
        cleanup();
        return fail(c, PV3D_E_DEVICE, "sky patches: %s", cudaGetErrorString(cudaGetLastError()));
    }
    const double two_pi = 6.283185307179586, half_pi = 1.5707963267948966;
    int rc = PV3D_OK;
    for (int b : used) {
        const double az_c = (b % n_az + 0.5) * two_pi / n_az, tilt_c = (b / n_az + 0.5) * half_pi / n_tilt;
        if (tracked) {
            std::vector<float> pz((size_t)P * g.n_trk * 2);
            for (size_t k = 0; k < pz.size(); k += 2) { pz[k] = (float)az_c; pz[k + 1] = (float)tilt_c; }
            if (cudaMemcpy(bposes, pz.data(), pz.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = fail(c, PV3D_E_DEVICE, "sky view: pose upload");
                break;
            }
        }
        // the patches stand in for the sun table (and every tracker takes the
        // bin's centre pose) while their depth tests run
        double* s_sun = g.d_sun;
        float *s_dni = g.d_dni, *s_dhi = g.d_dhi, *s_dt = g.d_dt, *s_poses = g.d_poses;
        const int64_t s_n = g.n_steps, s_np = g.n_pose_steps;
        std::vector<uint8_t> s_lit = std::move(g.lit);
        g.d_sun = xyz; g.d_dni = dni; g.d_dhi = dhi; g.d_dt = dt;
        g.n_steps = P;
        if (tracked) { g.d_poses = bposes; g.n_pose_steps = P; }
        g.lit.assign((size_t)P, 1);
        pv3d_eval_opts eo{};
        eo.samples_per_side = n;
        eo.map_res = d.map_res;
        pv3d_result r{};
        r.is_device = 1;
        r.cell_counts = counts;
        rc = evaluate_plain(c, gen_id, &eo, &r);
        g.d_sun = s_sun; g.d_dni = s_dni; g.d_dhi = s_dhi; g.d_dt = s_dt;
        g.n_steps = s_n;
        g.d_poses = s_poses;
        g.n_pose_steps = s_np;
        g.lit = std::move(s_lit);
        if (rc) break;
        if (launch_sky_fraction(g.d_mods, g.d_cell_mod, g.C, xyz, dom, P, counts, n * n, fdiff + (size_t)b * g.C,
                                tracked ? az_c : 0.0, tracked ? tilt_c : 0.0, st) != cudaSuccess) {
            rc = fail(c, PV3D_E_DEVICE, "sky fraction: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
    }
    if (!rc && (cudaStreamSynchronize(st) != cudaSuccess ||
                (cell_fraction &&
                 cudaMemcpy(cell_fraction, fdiff, (size_t)nb * g.C * 4, cudaMemcpyDeviceToHost) != cudaSuccess)))
        rc = fail(c, PV3D_E_DEVICE, "sky fraction: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc) {
        cleanup();
        return rc;
    }
    if (g.d_fdiff) cudaFree(g.d_fdiff);
    if (g.d_fbin) cudaFree(g.d_fbin);
    g.d_fdiff = fdiff;
    g.d_fbin = fbin;
    g.fdiff_bins = nb;
    fdiff = nullptr;
    fbin = nullptr;
    cleanup();
    return PV3D_OK;
}

// ---------------------------------------------------------------------------
// served requests (queue; executed in arrival order on poll)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// served requests: continuous batching over waves
// ---------------------------------------------------------------------------
struct pv3d_ctx::Request {
    uint64_t id = 0;
    uint32_t gen_id = 0;
    pv3d_eval_opts opts{};
    pv3d_result* out = nullptr;
    EvalSetup es{};
    int status = PV3D_E_PENDING;
    int64_t next = 0;          // next sun step to evaluate
    DevBuf kmod, kcell, kstr, karr, stage; // Kahan pairs and the staging of host outputs
    double* d_e = nullptr;
    double* d_eu = nullptr;
    double* d_cl = nullptr;
    float* d_p = nullptr;
    float* d_pu = nullptr;
    uint8_t* d_cnt = nullptr;
    unsigned long long* d_bits = nullptr;
    double *d_se = nullptr, *d_seu = nullptr, *d_ae = nullptr, *d_aeu = nullptr;  // string and array energies
    float *d_sp = nullptr, *d_spu = nullptr, *d_ap = nullptr, *d_apu = nullptr;   // string and array powers
    int64_t footprint = 0;
    int64_t waves = 0;
    float device_ms = 0.f;
    bool admitted = false;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

static int64_t per_step_scratch(const GenH& g, const EvalSetup& es)
{
    const int64_t tiles = (int64_t)(es.R / es.tile) * (es.R / es.tile);
    return tiles * 4 * 10 + (int64_t)g.C * 12 + (int64_t)g.M * (sizeof(ModStep) + 12) + sizeof(LightParams) + 16;
}

static int64_t request_bytes(const GenH& g, const EvalSetup& es, const pv3d_result* out, int64_t S)
{
    int64_t b = (int64_t)g.M * 16 + (int64_t)g.C * 8;
    if (!out->is_device) {
        if (out->energy) b += g.M * 8;
        if (out->energy_unshaded) b += g.M * 8;
        if (out->cell_beam_loss) b += (int64_t)g.C * 8;
        if (out->power) b += S * g.M * 4;
        if (out->power_unshaded) b += S * g.M * 4;
        if (out->cell_counts) b += S * g.C;
        if (out->sample_bits) b += S * g.C * 8;
        const int64_t NS = (int64_t)g.str_ids.size(), NA = (int64_t)g.arr_ids.size();
        if (out->string_energy) b += NS * 8;
        if (out->string_energy_unshaded) b += NS * 8;
        if (out->string_power) b += S * NS * 4;
        if (out->string_power_unshaded) b += S * NS * 4;
        if (out->array_energy) b += NA * 8;
        if (out->array_energy_unshaded) b += NA * 8;
        if (out->array_power) b += S * NA * 4;
        if (out->array_power_unshaded) b += S * NA * 4;
    }
    if (es.strings) b += (int64_t)g.str_ids.size() * 16;
    if (es.arrays) b += (int64_t)g.arr_ids.size() * 16;
    return b;
}

static int64_t resident_bytes(pv3d_ctx* c)
{
    int64_t b = 0;
    for (auto& kv : c->scenes) b += (int64_t)kv.second.bytes;
    for (auto& kv : c->gens) b += (int64_t)kv.second.bytes + kv.second.n_steps * 36;
    return b;
}

// Take a device buffer of at least `bytes` from the free list (or allocate).
static int take_buf(pv3d_ctx* c, DevBuf& dst, size_t bytes)
{
    bytes = std::max<size_t>(bytes, 16);
    size_t best = (size_t)-1;
    for (size_t k = 0; k < c->free_bufs.size(); ++k)
        if (c->free_bufs[k].bytes >= bytes && (best == (size_t)-1 || c->free_bufs[k].bytes < c->free_bufs[best].bytes))
            best = k;
    if (best != (size_t)-1) {
        dst = c->free_bufs[best];
        c->free_bufs.erase(c->free_bufs.begin() + best);
        return PV3D_OK;
    }
    DevBuf b;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PV3D_E_NOMEM, "request buffer allocation failed");
    }
    b.bytes = bytes;
    dst = b;
    return PV3D_OK;
}

static void give_buf(pv3d_ctx* c, DevBuf& b)
{
    if (b.p) c->free_bufs.push_back(b);
    b = DevBuf{};
}

// Allocate the request's buffers and point its outputs (worker thread, mu held).
static int admit(pv3d_ctx* c, pv3d_ctx::Request& r)
{
    const GenH& g = c->gens.at(r.gen_id);
    const int64_t S = r.es.e - r.es.b;
    int rc;
    const size_t NS = g.str_ids.size(), NA = g.arr_ids.size();
    if ((rc = take_buf(c, r.kmod, (size_t)g.M * 2 * sizeof(float2))) ||
        (rc = take_buf(c, r.kcell, (size_t)g.C * sizeof(float2))) ||
        (r.es.strings && (rc = take_buf(c, r.kstr, NS * 2 * sizeof(float2)))) ||
        (r.es.arrays && (rc = take_buf(c, r.karr, NA * 2 * sizeof(float2)))))
        return rc;
    pv3d_result* out = r.out;
    if (out->is_device) {
        r.d_e = out->energy; r.d_eu = out->energy_unshaded; r.d_cl = out->cell_beam_loss;
        r.d_p = out->power; r.d_pu = out->power_unshaded; r.d_cnt = out->cell_counts;
        r.d_bits = (unsigned long long*)out->sample_bits;
        r.d_se = out->string_energy; r.d_seu = out->string_energy_unshaded;
        r.d_sp = out->string_power; r.d_spu = out->string_power_unshaded;
        r.d_ae = out->array_energy; r.d_aeu = out->array_energy_unshaded;
        r.d_ap = out->array_power; r.d_apu = out->array_power_unshaded;
    } else {
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
        size_t oe = out->energy ? take(g.M * 8) : 0, oeu = out->energy_unshaded ? take(g.M * 8) : 0;
        size_t ocl = out->cell_beam_loss ? take((size_t)g.C * 8) : 0;
        size_t op = out->power ? take((size_t)S * g.M * 4) : 0, opu = out->power_unshaded ? take((size_t)S * g.M * 4) : 0;
        size_t oc = out->cell_counts ? take((size_t)S * g.C) : 0, ob = out->sample_bits ? take((size_t)S * g.C * 8) : 0;
        size_t ose = out->string_energy ? take(NS * 8) : 0, oseu = out->string_energy_unshaded ? take(NS * 8) : 0;
        size_t osp = out->string_power ? take((size_t)S * NS * 4) : 0;
        size_t ospu = out->string_power_unshaded ? take((size_t)S * NS * 4) : 0;
        size_t oae = out->array_energy ? take(NA * 8) : 0, oaeu = out->array_energy_unshaded ? take(NA * 8) : 0;
        size_t oap = out->array_power ? take((size_t)S * NA * 4) : 0;
        size_t oapu = out->array_power_unshaded ? take((size_t)S * NA * 4) : 0;
        if ((rc = take_buf(c, r.stage, off))) return rc;
        char* b = (char*)r.stage.p;
        r.d_e = out->energy ? (double*)(b + oe) : nullptr;
        r.d_eu = out->energy_unshaded ? (double*)(b + oeu) : nullptr;
        r.d_cl = out->cell_beam_loss ? (double*)(b + ocl) : nullptr;
        r.d_p = out->power ? (float*)(b + op) : nullptr;
        r.d_pu = out->power_unshaded ? (float*)(b + opu) : nullptr;
        r.d_cnt = out->cell_counts ? (uint8_t*)(b + oc) : nullptr;
        r.d_bits = out->sample_bits ? (unsigned long long*)(b + ob) : nullptr;
        r.d_se = out->string_energy ? (double*)(b + ose) : nullptr;
        r.d_seu = out->string_energy_unshaded ? (double*)(b + oseu) : nullptr;
        r.d_sp = out->string_power ? (float*)(b + osp) : nullptr;
        r.d_spu = out->string_power_unshaded ? (float*)(b + ospu) : nullptr;
        r.d_ae = out->array_energy ? (double*)(b + oae) : nullptr;
        r.d_aeu = out->array_energy_unshaded ? (double*)(b + oaeu) : nullptr;
        r.d_ap = out->array_power ? (float*)(b + oap) : nullptr;
        r.d_apu = out->array_power_unshaded ? (float*)(b + oapu) : nullptr;
    }
    CUDA_TRY(c, cudaMemsetAsync(r.kmod.p, 0, (size_t)g.M * 2 * sizeof(float2), c->serve_stream));
    CUDA_TRY(c, cudaMemsetAsync(r.kcell.p, 0, (size_t)g.C * sizeof(float2), c->serve_stream));
    if (r.es.strings) CUDA_TRY(c, cudaMemsetAsync(r.kstr.p, 0, NS * 2 * sizeof(float2), c->serve_stream));
    if (r.es.arrays) CUDA_TRY(c, cudaMemsetAsync(r.karr.p, 0, NA * 2 * sizeof(float2), c->serve_stream));
    r.next = r.es.b;
    r.admitted = true;
    return PV3D_OK;
}

// Finish a request: Kahan pairs to its outputs, host copies (worker thread).
static int finish(pv3d_ctx* c, pv3d_ctx::Request& r)
{
    const GenH& g = c->gens.at(r.gen_id);
    const int64_t S = r.es.e - r.es.b;
    cudaStream_t st = c->serve_stream;
    CUDA_TRY(c, launch_finalize_pairs((const float2*)r.kmod.p, g.M, (const float2*)r.kcell.p, r.d_cl ? g.C : 0, r.d_e,
                                      r.d_eu,
                                      r.d_cl, st));
    const int NS = (int)g.str_ids.size(), NA = (int)g.arr_ids.size();
    if (r.es.strings)
        CUDA_TRY(c, launch_finalize_pairs((const float2*)r.kstr.p, NS, nullptr, 0, r.d_se, r.d_seu, nullptr, st));
    if (r.es.arrays)
        CUDA_TRY(c, launch_finalize_pairs((const float2*)r.karr.p, NA, nullptr, 0, r.d_ae, r.d_aeu, nullptr, st));
    pv3d_result* out = r.out;
    if (!out->is_device) {
        auto cp = [&](void* dst, const void* src, size_t bytes) {
            return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
        };
        CUDA_TRY(c, cp(out->energy, r.d_e, g.M * 8));
        CUDA_TRY(c, cp(out->energy_unshaded, r.d_eu, g.M * 8));
        CUDA_TRY(c, cp(out->cell_beam_loss, r.d_cl, (size_t)g.C * 8));
        CUDA_TRY(c, cp(out->power, r.d_p, (size_t)S * g.M * 4));
        CUDA_TRY(c, cp(out->power_unshaded, r.d_pu, (size_t)S * g.M * 4));
        CUDA_TRY(c, cp(out->cell_counts, r.d_cnt, (size_t)S * g.C));
        CUDA_TRY(c, cp(out->sample_bits, r.d_bits, (size_t)S * g.C * 8));
        CUDA_TRY(c, cp(out->string_energy, r.d_se, (size_t)NS * 8));
        CUDA_TRY(c, cp(out->string_energy_unshaded, r.d_seu, (size_t)NS * 8));
        CUDA_TRY(c, cp(out->string_power, r.d_sp, (size_t)S * NS * 4));
        CUDA_TRY(c, cp(out->string_power_unshaded, r.d_spu, (size_t)S * NS * 4));
        CUDA_TRY(c, cp(out->array_energy, r.d_ae, (size_t)NA * 8));
        CUDA_TRY(c, cp(out->array_energy_unshaded, r.d_aeu, (size_t)NA * 8));
        CUDA_TRY(c, cp(out->array_power, r.d_ap, (size_t)S * NA * 4));
        CUDA_TRY(c, cp(out->array_power_unshaded, r.d_apu, (size_t)S * NA * 4));
    }
    CUDA_TRY(c, cudaStreamSynchronize(st));
    int64_t lit = 0;
    for (int64_t k = r.es.b; k < r.es.e; ++k) lit += g.lit[k];
    out->steps_lit = lit;
    out->tests = lit * (int64_t)g.C * r.es.n * r.es.n;
    out->device_ms = r.device_ms;
    out->waves = (int32_t)r.waves;
    out->kernel_launches = r.waves * kLaunchesPerWave + 1 + (r.es.strings ? 1 : 0) + (r.es.arrays ? 1 : 0);
    r.t_done = std::chrono::steady_clock::now();
    out->latency_ms = (float)std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
    return PV3D_OK;
}

static void release_request_bufs(pv3d_ctx* c, pv3d_ctx::Request& r)
{
    give_buf(c, r.kmod);
    give_buf(c, r.kcell);
    give_buf(c, r.kstr);
    give_buf(c, r.karr);
    give_buf(c, r.stage);
}

// One wave over the active requests; returns the requests it advanced.
static int serve_wave(pv3d_ctx* c, std::unique_lock<std::mutex>& lk)
{
    // admission: FIFO while slots and device memory allow
    const int64_t budget = c->opts.hbm_budget_bytes - resident_bytes(c);
    while (!c->pending.empty() && (int)c->active.size() < c->opts.max_inflight) {
        pv3d_ctx::Request& r = *c->reqs.at(c->pending.front());
        if (!c->active.empty() && c->reserved + r.footprint > budget) break;
        c->pending.pop_front();
        int rc = admit(c, r);
        if (rc) {
            r.status = rc;
            release_request_bufs(c, r);
            c->cv_done.notify_all();
            continue;
        }
        c->reserved += r.footprint;
        c->active.push_back(r.id);
    }
    if (c->active.empty()) return 0;
    // wave: the next chunk of every active request, within the scratch limits
    // the wave's tile and cell arrays are kept near the scratch target (the
    // L2-sized working set decides the binning and tally speed); the first
    // request of the wave shortens its chunk if it alone is over the target
    const int64_t scratch_cap = std::min<int64_t>((int64_t)c->opts.wave_scratch_mb << 20, std::max<int64_t>(budget / 4, 1));
    std::vector<JobDev> jobs;
    std::vector<pv3d_ctx::Request*> in_wave;
    std::vector<int> ks;
    int64_t scratch = 0;
    bool want_bits = false;
    int extras = 0;  // string (1) and array (4) kernels in the wave
    const size_t na = c->active.size();
    for (size_t q = 0; q < na; ++q) {
        pv3d_ctx::Request& r = *c->reqs.at(c->active[(c->rr + q) % na]);
        const GenH& g = c->gens.at(r.gen_id);
        const SceneH& sc = c->scenes.at(g.scene_id);
        int k = (int)std::min<int64_t>(r.es.K, r.es.e - r.next);
        const int64_t per_step = per_step_scratch(g, r.es);
        if (jobs.empty()) k = (int)std::max<int64_t>(1, std::min<int64_t>(k, scratch_cap / std::max<int64_t>(per_step, 1)));
        const int64_t need = per_step * k;
        if (!jobs.empty() && scratch + need > scratch_cap) break;
        scratch += need;
        jobs.push_back(make_job(c, g, sc, r.es, r.next, k, (float2*)r.kmod.p, r.d_cl ? (float2*)r.kcell.p : nullptr,
                                r.d_p, r.d_pu, r.d_cnt, r.d_bits, (float2*)r.kstr.p, r.d_sp, r.d_spu, nullptr, nullptr,
                                nullptr, 0, 0, (float2*)r.karr.p, r.d_ap, r.d_apu));
        in_wave.push_back(&r);
        ks.push_back(k);
        want_bits = want_bits || r.d_bits;
        extras |= (r.es.strings ? 1 : 0) | (r.es.arrays ? 4 : 0);
    }
    c->rr = (c->rr + jobs.size()) % std::max<size_t>(na, 1);
    lk.unlock();
    std::vector<WaveDev> waves{pack_wave(jobs, 0, jobs.size(), c->opts.tile == 32 ? 5 : (c->opts.tile == 64 ? 6 : 7),
                                         c->opts.depth_format == PV3D_DEPTH_U24, 1, 0)};
    WaveDev& W = waves[0];
    Counters hc{};
    int rc = PV3D_OK;
    float ms = 0.f;
    {
        std::lock_guard<std::mutex> g(c->gpu_mu);
        cudaSetDevice(c->device);
        cudaStream_t st = c->serve_stream;
        rc = ensure_workspace(c, W.tot_js, W.tot_te, W.tot_ms, W.tot_cs, c->opts.tile, true, want_bits, W.tot_ss,
                              W.tot_sq, W.tot_sa);
        if (!rc) {
            W.bin_cap = c->bin_cap; W.map_cap_tiles = c->map_cap_tiles;
            W.big_cap = c->big_cap; W.recv_cap = c->recv_cap;
            rc = stage_descriptors(c, waves, jobs, st);
        }
        if (!rc && cudaMemsetAsync(c->ctr.p, 0, sizeof(Counters), st) != cudaSuccess) rc = PV3D_E_DEVICE;
        if (!rc && cudaEventRecord(c->ev0, st) != cudaSuccess) rc = PV3D_E_DEVICE;
        if (!rc) rc = run_waves(c, waves, st, c->opts.tile, true, false, false, extras);
        if (!rc && cudaEventRecord(c->ev1, st) != cudaSuccess) rc = PV3D_E_DEVICE;
        if (!rc && cudaMemcpyAsync(&hc, c->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = PV3D_E_DEVICE;
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = PV3D_E_DEVICE;
        if (!rc) cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        if (!rc && hc.overflow) {
            // grow the pools and restart the requests of this wave from their first step
            if (hc.overflow & 1u) c->bin_cap = (int64_t)(hc.need_bins * 5 / 4 + 1024);
            if (hc.overflow & 4u) c->big_cap = (int64_t)(hc.need_big * 5 / 4 + 1024);
            if (hc.overflow & 8u) c->recv_cap = (int64_t)(hc.need_recv * 5 / 4 + 1024);
            for (auto* r : in_wave) {
                const GenH& g = c->gens.at(r->gen_id);
                cudaMemsetAsync(r->kmod.p, 0, (size_t)g.M * 2 * sizeof(float2), st);
                cudaMemsetAsync(r->kcell.p, 0, (size_t)g.C * sizeof(float2), st);
                if (r->kstr.p) cudaMemsetAsync(r->kstr.p, 0, g.str_ids.size() * 2 * sizeof(float2), st);
                if (r->karr.p) cudaMemsetAsync(r->karr.p, 0, g.arr_ids.size() * 2 * sizeof(float2), st);
            }
            cudaStreamSynchronize(st);
        }
    }
    lk.lock();
    if (rc) {
        for (auto* r : in_wave) r->status = rc;
    } else {
        for (size_t q = 0; q < in_wave.size(); ++q) {
            pv3d_ctx::Request& r = *in_wave[q];
            if (hc.overflow) {
                r.next = r.es.b;
                continue;
            }
            r.next += ks[q];
            r.waves += 1;
            r.device_ms += ms;
            if (r.next >= r.es.e) {
                std::lock_guard<std::mutex> g(c->gpu_mu);
                r.status = finish(c, r);
            }
        }
    }
    // retire finished or failed requests
    for (auto it = c->active.begin(); it != c->active.end();) {
        pv3d_ctx::Request& r = *c->reqs.at(*it);
        if (r.status != PV3D_E_PENDING) {
            c->reserved -= r.footprint;
            release_request_bufs(c, r);
            it = c->active.erase(it);
        } else {
            ++it;
        }
    }
    c->cv_done.notify_all();
    return (int)in_wave.size();
}

static void serve_loop(pv3d_ctx* c)
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(c->mu);
    while (!c->stop) {
        if (c->pending.empty() && c->active.empty()) {
            c->cv_work.wait(lk);
            continue;
        }
        serve_wave(c, lk);
    }
}

extern "C" int pv3d_submit(pv3d_ctx* c, uint32_t gen_id, const pv3d_eval_opts* o, pv3d_result* out, uint64_t* req)
{
    if (!c || !out || !req) return PV3D_E_INVALID;
    std::unique_lock<std::mutex> lk(c->mu);
    auto git = c->gens.find(gen_id);
    if (git == c->gens.end()) return fail(c, PV3D_E_NOTFOUND, "unknown generator %u", gen_id);
    const GenH& g = git->second;
    if (c->scenes.find(g.scene_id) == c->scenes.end()) return fail(c, PV3D_E_NOTFOUND, "scene is gone");
    std::unique_ptr<pv3d_ctx::Request> r(new pv3d_ctx::Request());
    int rc = check_eval(c, g, o, out, r->es);
    if (rc) return rc;
    if (o && o->path == PV3D_PATH_MAP) return fail(c, PV3D_E_INVALID, "served requests use the fused path");
    if (r->es.heat) return fail(c, PV3D_E_INVALID, "sky-map outputs are produced by pv3d_evaluate only");
    if (r->es.groups) return fail(c, PV3D_E_INVALID, "window groups are evaluated by pv3d_evaluate only");
    r->gen_id = gen_id;
    r->opts = o ? *o : pv3d_eval_opts{};
    r->out = out;
    const int64_t S = r->es.e - r->es.b;
    r->footprint = request_bytes(g, r->es, out, S) + per_step_scratch(g, r->es) * r->es.K;
    if (r->footprint > c->opts.hbm_budget_bytes - resident_bytes(c))
        return fail(c, PV3D_E_ADMISSION, "request needs %lld bytes, budget leaves %lld", (long long)r->footprint,
                    (long long)(c->opts.hbm_budget_bytes - resident_bytes(c)));
    r->t_submit = std::chrono::steady_clock::now();
    const uint64_t id = c->next_req++;
    r->id = id;
    c->reqs[id] = std::move(r);
    c->pending.push_back(id);
    if (!c->worker.joinable()) {
        if (!c->serve_stream && cudaStreamCreateWithFlags(&c->serve_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, PV3D_E_DEVICE, "stream creation failed");
        c->stop = false;
        c->worker = std::thread(serve_loop, c);
    }
    c->cv_work.notify_one();
    *req = id;
    return PV3D_OK;
}

extern "C" int pv3d_poll(pv3d_ctx* c, uint64_t req, int32_t timeout_ms)
{
    if (!c) return PV3D_E_INVALID;
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->reqs.find(req);
    if (it == c->reqs.end()) return fail(c, PV3D_E_NOTFOUND, "unknown request %llu", (unsigned long long)req);
    pv3d_ctx::Request* r = it->second.get();
    if (r->status == PV3D_E_PENDING && timeout_ms != 0) {
        auto pred = [&] { return r->status != PV3D_E_PENDING; };
        if (timeout_ms < 0) c->cv_done.wait(lk, pred);
        else c->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    const int s = r->status;
    if (s != PV3D_E_PENDING) c->reqs.erase(it);
    return s;
}

extern "C" int pv3d_evaluate_batch(pv3d_ctx* c, int32_t n, const uint32_t* gen_ids, const pv3d_eval_opts* opts,
                                   pv3d_result* outs)
{
    if (!c || n < 0 || (n > 0 && (!gen_ids || !outs))) return PV3D_E_INVALID;
    std::vector<uint64_t> ids((size_t)n, 0);
    int first = PV3D_OK;
    for (int32_t k = 0; k < n; ++k) {
        int rc = pv3d_submit(c, gen_ids[k], opts ? &opts[k] : nullptr, &outs[k], &ids[k]);
        if (rc && first == PV3D_OK) first = rc;
    }
    for (int32_t k = 0; k < n; ++k) {
        if (!ids[k]) continue;
        int rc = pv3d_poll(c, ids[k], -1);
        if (rc && first == PV3D_OK) first = rc;
    }
    return first;
}

extern "C" int pv3d_release(pv3d_ctx* c, uint32_t id)
{
    if (!c) return PV3D_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (auto& kv : c->reqs) {
            const uint32_t gid = kv.second->gen_id;
            auto git = c->gens.find(gid);
            if (gid == id || (git != c->gens.end() && git->second.scene_id == id))
                return fail(c, PV3D_E_INVALID, "id %u is used by request %llu", id, (unsigned long long)kv.first);
        }
    }
    std::lock_guard<std::mutex> gl(c->gpu_mu);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    auto git = c->gens.find(id);
    if (git != c->gens.end()) {
        free_gen(git->second);
        c->gens.erase(git);
        return PV3D_OK;
    }
    auto sit = c->scenes.find(id);
    if (sit == c->scenes.end()) return fail(c, PV3D_E_NOTFOUND, "unknown id %u", id);
    for (auto it = c->gens.begin(); it != c->gens.end();) {
        if (it->second.scene_id == id) {
            free_gen(it->second);
            it = c->gens.erase(it);
        } else {
            ++it;
        }
    }
    if (sit->second.d_tri) cudaFree(sit->second.d_tri);
    if (sit->second.d_ml) cudaFree(sit->second.d_ml);
    c->scenes.erase(sit);
    return PV3D_OK;
}

extern "C" void pv3d_destroy(pv3d_ctx* c)
{
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv_work.notify_all();
    if (c->worker.joinable()) c->worker.join();
    cudaSetDevice(c->device);
    for (auto& kv : c->reqs) release_request_bufs(c, *kv.second);
    for (DevBuf& b : c->free_bufs) release_buf(b);
    if (c->serve_stream) cudaStreamDestroy(c->serve_stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->scenes) {
        if (kv.second.d_tri) cudaFree(kv.second.d_tri);
        if (kv.second.d_ml) cudaFree(kv.second.d_ml);
    }
    for (auto& kv : c->gens) free_gen(kv.second);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    release_buf(c->wave_slot);
    release_buf(c->jobs_slot);
    DevBuf* bufs[] = {&c->lp, &c->win, &c->ms, &c->ms_p, &c->ms_pu, &c->ms_beam, &c->ms_iu, &c->ss_i, &c->sq_p,
                      &c->sq_pu, &c->kahan_str, &c->js_p, &c->js_pu, &c->js_bin, &c->heat, &c->sa_p, &c->sa_pu, &c->kahan_arr, &c->cs_cnt, &c->cs_bits, &c->t_far,
                      &c->t_cnt, &c->t_off, &c->t_cur, &c->t_slot, &c->t_rcnt, &c->t_plane, &c->t_roff, &c->t_rcur, &c->nonempty, &c->heavy,
                      &c->bins, &c->pairs, &c->recv, &c->map, &c->big,
                      &c->block_sums, &c->ctr, &c->waves, &c->jobs, &c->kahan_mod, &c->kahan_cell, &c->staging};
    for (DevBuf* b : bufs) release_buf(*b);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}
