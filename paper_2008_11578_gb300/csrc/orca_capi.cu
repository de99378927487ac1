// orca_capi.cu -- the C ABI of liborca (declared in include/orca.h).
//
// Host side of the ORCA step: argument validation, workspace layout, and
// the launch sequence of one step (bin_count, scan x3, scatter, solve)
// bracketed by a load and an unload kernel per call.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "orca.h"
#include "orca_step_kernels.cuh"

using namespace orca;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace carve-up (device, caller owned).
struct Layout {
    size_t err, count, start, bsum, key, slot, pos0, vel0, pos1, vel1;
    size_t rad[2], typ[2], orig[2];
    size_t total;
};

Layout make_layout(size_t n, size_t ncells) {
    Layout L{};
    size_t nb = (ncells + kScanChunk - 1) / kScanChunk;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.err = take(16);
    L.count = take(ncells * 4);
    L.start = take((ncells + 1) * 4);
    L.bsum = take((nb + 1) * 4);
    L.key = take(n * 4);
    L.slot = take(n * 4);
    L.pos0 = take(n * 8);
    L.vel0 = take(n * 8);
    L.pos1 = take(n * 8);
    L.vel1 = take(n * 8);
    for (int b = 0; b < 2; ++b) {
        L.rad[b] = take(n * 4);
        L.typ[b] = take(n);
        L.orig[b] = take(n * 4);
    }
    L.total = o;
    return L;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }

int check_params(const orca_params* p) {
    if (!p) return ORCA_ERR_INVALID_ARG;
    if (!finite_pos(p->neighbor_dist) || !finite_pos(p->time_horizon) || !finite_pos(p->dt) ||
        !finite_pos(p->cell_size))
        return ORCA_ERR_INVALID_ARG;
    if (!std::isfinite(p->origin_x) || !std::isfinite(p->origin_y)) return ORCA_ERR_INVALID_ARG;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (!std::isfinite(p->f[a][b])) return ORCA_ERR_INVALID_ARG;
    if (p->max_neighbors < 0) return ORCA_ERR_INVALID_ARG;
    if (p->max_neighbors > ORCA_MAX_NEIGHBORS) return ORCA_ERR_CAPACITY;
    if (p->grid_nx < 1 || p->grid_ny < 1) return ORCA_ERR_INVALID_ARG;
    if ((long long)p->grid_nx * (long long)p->grid_ny > (long long)ORCA_MAX_CELLS)
        return ORCA_ERR_CAPACITY;
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 128 || p->block_size % 32))
        return ORCA_ERR_INVALID_ARG;
    return ORCA_OK;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

int check_agents(const orca_agents* a) {
    if (!a || a->n_agents < 0) return ORCA_ERR_INVALID_ARG;
    if (a->n_agents == 0) return ORCA_OK;
    if (!a->pos || !a->vel || !a->goal || !a->radius || !a->max_speed || !a->type)
        return ORCA_ERR_INVALID_ARG;
    if (!aligned(a->pos, 8) || !aligned(a->vel, 8) || !aligned(a->goal, 8) ||
        !aligned(a->radius, 4) || !aligned(a->max_speed, 4))
        return ORCA_ERR_INVALID_ARG;
    if (a->route) {
        if (!a->waypoints || !a->wp_idx || a->n_waypoints < 1 || a->n_waypoints > 255 ||
            a->n_routes < 1 || !aligned(a->waypoints, 8) || !aligned(a->route, 4))
            return ORCA_ERR_INVALID_ARG;
    }
    return ORCA_OK;
}

// ring-search margin: computed cell coordinates differ from exact ones by a
// relative 3u (two roundings and the rounded inverse); 16u of the largest
// coordinate covers both agents with room to spare
float ring_delta_for(int nx, int ny) {
    double u = std::ldexp(1.0, -24);
    return (float)(16.0 * u * (double)(std::max(nx, ny) + 2));
}

SceneDev scene_dev(const orca_params* p, int agent_off, int n, int cell_off) {
    SceneDev s{};
    s.agent_off = agent_off;
    s.n_agents = n;
    s.cell_off = cell_off;
    s.nx = p->grid_nx;
    s.ny = p->grid_ny;
    s.origin_x = p->origin_x;
    s.origin_y = p->origin_y;
    s.cell_size = p->cell_size;
    volatile float one = 1.0f;
    s.inv_cell = one / p->cell_size;
    s.ring_delta = ring_delta_for(p->grid_nx, p->grid_ny);
    volatile float R = p->neighbor_dist;
    s.R2 = R * R;
    s.k = p->max_neighbors;
    s.inv_tau = one / p->time_horizon;
    s.inv_dt = one / p->dt;
    s.dt = p->dt;
    s.f00 = p->f[0][0];
    s.f01 = p->f[0][1];
    s.f10 = p->f[1][0];
    s.f11 = p->f[1][1];
    return s;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ORCA_OK : ORCA_ERR_CUDA; }

template <class SRC>
void launch_solve(int kcap, bool count, int grid, int block, size_t smem, cudaStream_t st, int n,
                  SRC src, const float2* pos, const float2* vel, const float* rad,
                  const uint8_t* typ, const int32_t* orig, const uint32_t* start, AgentIn ain,
                  const float2* vpd, float2* out_pos, float2* out_vel, DebugOut dbg,
                  unsigned long long* counters) {
    // more than 48 KB of dynamic shared memory needs an explicit opt-in
#define ORCA_SOLVE(K, C)                                                                  \
    do {                                                                                  \
        if (smem > 48 * 1024)                                                             \
            cudaFuncSetAttribute(solve_kernel<K, SRC, C>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        solve_kernel<K, SRC, C><<<grid, block, smem, st>>>(n, src, pos, vel, rad, typ,    \
                                                            orig, start, ain, vpd,        \
                                                            out_pos, out_vel, dbg,        \
                                                            counters);                    \
    } while (0)
    if (kcap == 16) {
        if (count) ORCA_SOLVE(16, true);
        else ORCA_SOLVE(16, false);
    } else {
        if (count) ORCA_SOLVE(32, true);
        else ORCA_SOLVE(32, false);
    }
#undef ORCA_SOLVE
}

}  // namespace

struct orca_scene {
    orca_params params;
    orca_agents agents;
    int n;
    int ncells;
    int nblocks;
    Layout lay;
    char* ws;
    SceneDev dev;
    DebugOut dbg;
    int kcap;
    int block;
    cudaEvent_t ev_begin;
    cudaEvent_t ev_end;
    unsigned long long* counters;
};

extern "C" {

const char* orca_status_string(int status) {
    switch (status) {
        case ORCA_OK: return "ok";
        case ORCA_ERR_INVALID_ARG: return "invalid argument";
        case ORCA_ERR_CUDA: return "CUDA error";
        case ORCA_ERR_TIMEOUT: return "bounded device wait timed out";
        case ORCA_ERR_NONFINITE: return "non-finite position or velocity";
        case ORCA_ERR_CAPACITY: return "capacity exceeded";
        default: return "unknown status";
    }
}

int orca_abi_version(void) { return 1; }

int orca_workspace_bytes(const orca_params* params, int n_agents, size_t* out_bytes) {
    int st = check_params(params);
    if (st != ORCA_OK) return st;
    if (n_agents < 0 || !out_bytes) return ORCA_ERR_INVALID_ARG;
    size_t ncells = (size_t)params->grid_nx * (size_t)params->grid_ny;
    *out_bytes = make_layout((size_t)n_agents, ncells).total;
    return ORCA_OK;
}

int orca_scene_create(const orca_params* params, const orca_agents* agents, void* workspace,
                      size_t workspace_bytes, orca_scene** out) {
    if (!out) return ORCA_ERR_INVALID_ARG;
    *out = nullptr;
    int st = check_params(params);
    if (st != ORCA_OK) return st;
    st = check_agents(agents);
    if (st != ORCA_OK) return st;
    size_t ncells = (size_t)params->grid_nx * (size_t)params->grid_ny;
    Layout lay = make_layout((size_t)agents->n_agents, ncells);
    if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total)
        return ORCA_ERR_INVALID_ARG;
    orca_scene* s = new (std::nothrow) orca_scene;
    if (!s) return ORCA_ERR_CAPACITY;
    s->params = *params;
    s->agents = *agents;
    s->n = agents->n_agents;
    s->ncells = (int)ncells;
    s->nblocks = (int)((ncells + kScanChunk - 1) / kScanChunk);
    s->lay = lay;
    s->ws = (char*)workspace;
    s->dev = scene_dev(params, 0, s->n, 0);
    s->dbg = DebugOut{nullptr, nullptr, nullptr, nullptr, nullptr, params->max_neighbors};
    s->kcap = params->max_neighbors <= 16 ? 16 : 32;
    s->block = params->block_size ? params->block_size : 128;
    s->ev_begin = nullptr;
    s->ev_end = nullptr;
    s->counters = nullptr;
    if (cudaMemset(s->ws + lay.err, 0, 16) != cudaSuccess) {
        delete s;
        return ORCA_ERR_CUDA;
    }
    *out = s;
    return ORCA_OK;
}

int orca_scene_set_debug(orca_scene* s, int32_t* cell, int32_t* nbr, int32_t* cnt,
                         uint8_t* flags, float* tstar) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    s->dbg = DebugOut{cell, nbr, cnt, flags, tstar, s->params.max_neighbors};
    return ORCA_OK;
}

int orca_scene_set_solve_events(orca_scene* s, void* begin, void* end) {
    if (!s || ((begin == nullptr) != (end == nullptr))) return ORCA_ERR_INVALID_ARG;
    s->ev_begin = (cudaEvent_t)begin;
    s->ev_end = (cudaEvent_t)end;
    return ORCA_OK;
}

int orca_scene_set_counters(orca_scene* s, unsigned long long* counters) {
    if (!s || (counters && !aligned(counters, 8))) return ORCA_ERR_INVALID_ARG;
    s->counters = counters;
    return ORCA_OK;
}

int orca_step_launch_count(const orca_scene* s, int n_steps) {
    if (!s || n_steps < 0) return -1;
    if (s->n == 0 || n_steps == 0) return 0;
    return 2 + 6 * n_steps;
}

int orca_step(orca_scene* s, int n_steps, const float* vpref_delta, void* stream) {
    if (!s || n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    if (s->n == 0 || n_steps == 0) return ORCA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = s->n;
    const Layout& L = s->lay;
    char* w = s->ws;
    int* err = (int*)(w + L.err);
    uint32_t* count = (uint32_t*)(w + L.count);
    uint32_t* start = (uint32_t*)(w + L.start);
    uint32_t* bsum = (uint32_t*)(w + L.bsum);
    uint32_t* key = (uint32_t*)(w + L.key);
    uint32_t* slot = (uint32_t*)(w + L.slot);
    float2* pos0 = (float2*)(w + L.pos0);
    float2* vel0 = (float2*)(w + L.vel0);
    float2* pos1 = (float2*)(w + L.pos1);
    float2* vel1 = (float2*)(w + L.vel1);
    float* rad[2] = {(float*)(w + L.rad[0]), (float*)(w + L.rad[1])};
    uint8_t* typ[2] = {(uint8_t*)(w + L.typ[0]), (uint8_t*)(w + L.typ[1])};
    int32_t* orig[2] = {(int32_t*)(w + L.orig[0]), (int32_t*)(w + L.orig[1])};

    const orca_agents& A = s->agents;
    const int tb = 256;
    const int gb = (n + tb - 1) / tb;
    {
        int g = (std::max(n, s->ncells) + tb - 1) / tb;
        g = std::min(g, 152 * 16);
        load_kernel<<<g, tb, 0, st>>>(n, (const float2*)A.pos, (const float2*)A.vel, A.radius,
                                      A.type, pos0, vel0, rad[0], typ[0], orig[0], count,
                                      s->ncells, err);
    }
    AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                A.n_waypoints, A.wp_idx};
    OneScene src{s->dev};
    int cur = 0;
    const int sb = s->block;
    const int sgrid = (n + sb - 1) / sb;
    const size_t smem = (size_t)s->kcap * sb * sizeof(float4);
    for (int t = 0; t < n_steps; ++t) {
        bin_count_kernel<OneScene><<<gb, tb, 0, st>>>(n, src, pos0, key, slot, count);
        scan_blocks_kernel<<<s->nblocks, kScanThreads, 0, st>>>(count, start, bsum, s->ncells);
        scan_bsum_kernel<<<1, 1024, 0, st>>>(bsum, s->nblocks);
        scan_add_kernel<<<(s->ncells + 255) / 256, 256, 0, st>>>(start, bsum, s->ncells,
                                                                 s->nblocks);
        scatter_kernel<<<gb, tb, 0, st>>>(n, key, slot, start, pos0, vel0, rad[cur], typ[cur],
                                          orig[cur], pos1, vel1, rad[1 - cur], typ[1 - cur],
                                          orig[1 - cur]);
        cur = 1 - cur;
        const float2* vpd =
            vpref_delta ? (const float2*)vpref_delta + (size_t)t * (size_t)n : nullptr;
        if (s->ev_begin) cudaEventRecord(s->ev_begin, st);
        launch_solve(s->kcap, s->counters != nullptr, sgrid, sb, smem, st, n, src, pos1, vel1,
                     rad[cur], typ[cur], orig[cur], start, ain, vpd, pos0, vel0, s->dbg,
                     s->counters);
        if (s->ev_end) cudaEventRecord(s->ev_end, st);
    }
    unload_kernel<<<gb, tb, 0, st>>>(n, orig[cur], pos0, vel0, (float2*)A.pos, (float2*)A.vel);
    return cuda_status(cudaGetLastError());
}

int orca_scene_sync_status(orca_scene* s) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return ORCA_ERR_CUDA;
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, s->ws + s->lay.err, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ORCA_ERR_CUDA;
    if (cudaMemset(s->ws + s->lay.err, 0, 16) != cudaSuccess) return ORCA_ERR_CUDA;
    if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
    if (h[0] & ERR_BIT_TIMEOUT) return ORCA_ERR_TIMEOUT;
    return ORCA_OK;
}

void orca_scene_destroy(orca_scene* s) { delete s; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free step (orca_step_noalloc): the workspace is a fixed scratch
// array compiled into the library instead of caller memory.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

// The scratch area.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ORCA_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
char* g_noalloc_base[kNoallocMaxDevices] = {};

// Device address of the scratch area on the current device, looked up once
// per device.  Returns nullptr on failure.
char* noalloc_base(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_base[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return nullptr;
        g_noalloc_base[dev] = (char*)p;
    }
    return g_noalloc_base[dev];
}

}  // namespace

extern "C" int orca_step_noalloc(const orca_params* params, const orca_agents* agents,
                                 int n_steps, const float* vpref_delta, void* stream,
                                 int synchronize) {
    int st = check_params(params);
    if (st != ORCA_OK) return st;
    st = check_agents(agents);
    if (st != ORCA_OK) return st;
    if (n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    const size_t ncells = (size_t)params->grid_nx * (size_t)params->grid_ny;
    const Layout L = make_layout((size_t)agents->n_agents, ncells);
    if (L.total > (size_t)ORCA_NOALLOC_SCRATCH_BYTES) return ORCA_ERR_CAPACITY;
    const int n = agents->n_agents;
    if (n == 0 || n_steps == 0) return ORCA_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ORCA_ERR_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return ORCA_ERR_CAPACITY;
    char* w = noalloc_base(dev);
    if (w == nullptr) return ORCA_ERR_CUDA;
    cudaStream_t stm = (cudaStream_t)stream;

    int* err = (int*)(w + L.err);
    uint32_t* count = (uint32_t*)(w + L.count);
    uint32_t* start = (uint32_t*)(w + L.start);
    uint32_t* bsum = (uint32_t*)(w + L.bsum);
    uint32_t* key = (uint32_t*)(w + L.key);
    uint32_t* slot = (uint32_t*)(w + L.slot);
    float2* pos0 = (float2*)(w + L.pos0);
    float2* vel0 = (float2*)(w + L.vel0);
    float2* pos1 = (float2*)(w + L.pos1);
    float2* vel1 = (float2*)(w + L.vel1);
    float* rad[2] = {(float*)(w + L.rad[0]), (float*)(w + L.rad[1])};
    uint8_t* typ[2] = {(uint8_t*)(w + L.typ[0]), (uint8_t*)(w + L.typ[1])};
    int32_t* orig[2] = {(int32_t*)(w + L.orig[0]), (int32_t*)(w + L.orig[1])};

    // the error word and the cell counts must start at zero; the load
    // kernel clears the counts, the error word is cleared here
    if (cudaMemsetAsync(err, 0, 16, stm) != cudaSuccess) return ORCA_ERR_CUDA;
    const int ncell = (int)ncells;
    const int nblocks = (int)((ncells + kScanChunk - 1) / kScanChunk);
    const orca_agents& A = *agents;
    const int tb = 256;
    const int gb = (n + tb - 1) / tb;
    {
        int g = (std::max(n, ncell) + tb - 1) / tb;
        g = std::min(g, 152 * 16);
        load_kernel<<<g, tb, 0, stm>>>(n, (const float2*)A.pos, (const float2*)A.vel, A.radius,
                                       A.type, pos0, vel0, rad[0], typ[0], orig[0], count, ncell,
                                       err);
    }
    AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                A.n_waypoints, A.wp_idx};
    OneScene src{scene_dev(params, 0, n, 0)};
    const DebugOut dbg{nullptr, nullptr, nullptr, nullptr, nullptr, params->max_neighbors};
    const int kcap = params->max_neighbors <= 16 ? 16 : 32;
    const int sb = params->block_size ? params->block_size : 128;
    const int sgrid = (n + sb - 1) / sb;
    const size_t smem = (size_t)kcap * sb * sizeof(float4);
    int cur = 0;
    for (int t = 0; t < n_steps; ++t) {
        bin_count_kernel<OneScene><<<gb, tb, 0, stm>>>(n, src, pos0, key, slot, count);
        scan_blocks_kernel<<<nblocks, kScanThreads, 0, stm>>>(count, start, bsum, ncell);
        scan_bsum_kernel<<<1, 1024, 0, stm>>>(bsum, nblocks);
        scan_add_kernel<<<(ncell + 255) / 256, 256, 0, stm>>>(start, bsum, ncell, nblocks);
        scatter_kernel<<<gb, tb, 0, stm>>>(n, key, slot, start, pos0, vel0, rad[cur], typ[cur],
                                           orig[cur], pos1, vel1, rad[1 - cur], typ[1 - cur],
                                           orig[1 - cur]);
        cur = 1 - cur;
        const float2* vpd =
            vpref_delta ? (const float2*)vpref_delta + (size_t)t * (size_t)n : nullptr;
        launch_solve(kcap, false, sgrid, sb, smem, stm, n, src, pos1, vel1, rad[cur], typ[cur],
                     orig[cur], start, ain, vpd, pos0, vel0, dbg, nullptr);
    }
    unload_kernel<<<gb, tb, 0, stm>>>(n, orig[cur], pos0, vel0, (float2*)A.pos, (float2*)A.vel);
    if (cudaGetLastError() != cudaSuccess) return ORCA_ERR_CUDA;
    if (synchronize) {
        if (cudaStreamSynchronize(stm) != cudaSuccess) return ORCA_ERR_CUDA;
        int h[4] = {0, 0, 0, 0};
        if (cudaMemcpy(h, err, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return ORCA_ERR_CUDA;
        if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
        if (h[0] & ERR_BIT_TIMEOUT) return ORCA_ERR_TIMEOUT;
    }
    return ORCA_OK;
}
