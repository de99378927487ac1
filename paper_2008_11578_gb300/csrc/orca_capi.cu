// orca_capi.cu -- the C ABI of liborca (declared in include/orca.h).
//
// Host side of the ORCA step: argument validation, workspace layout, and
// the launch sequence of one step (bin_count, scan x3, scatter, solve)
// bracketed by a load and an unload kernel per call.
//
// A single scene and a batch of independent scenes run the same kernels.  A
// batch concatenates its scenes' agents (scene 0 first) and their grid cells
// into one index space; every agent finds the constants of its scene through
// a scene table in the workspace, so one launch per phase serves all scenes.
// Because the cells of scene s precede those of scene s+1, the global
// counting sort keeps every scene's agents inside the scene's own slot range.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "orca.h"
#include "orca_step_kernels.cuh"

using namespace orca;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace carve-up (device, caller owned).  The scene table and the scene
// id of every slot exist only for batches (n_scenes > 0).
struct Layout {
    size_t err, count, start, bsum, key, slot, pos0, vel0, pos1, vel1;
    size_t rad[2], typ[2], orig[2];
    size_t scenes, sid;
    size_t total;
};

Layout make_layout(size_t n, size_t ncells, size_t n_scenes) {
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
    if (n_scenes > 0) {
        L.scenes = take(n_scenes * sizeof(SceneDev));
        L.sid = take(n * 4);
    }
    L.total = o;
    return L;
}

// Device pointers of one workspace.
struct Buffers {
    int* err;
    uint32_t *count, *start, *bsum, *key, *slot;
    float2 *pos0, *vel0, *pos1, *vel1;
    float* rad[2];
    uint8_t* typ[2];
    int32_t* orig[2];
    SceneDev* scenes;
    int32_t* sid;
};

Buffers carve(char* w, const Layout& L, bool batch) {
    Buffers b{};
    b.err = (int*)(w + L.err);
    b.count = (uint32_t*)(w + L.count);
    b.start = (uint32_t*)(w + L.start);
    b.bsum = (uint32_t*)(w + L.bsum);
    b.key = (uint32_t*)(w + L.key);
    b.slot = (uint32_t*)(w + L.slot);
    b.pos0 = (float2*)(w + L.pos0);
    b.vel0 = (float2*)(w + L.vel0);
    b.pos1 = (float2*)(w + L.pos1);
    b.vel1 = (float2*)(w + L.vel1);
    for (int i = 0; i < 2; ++i) {
        b.rad[i] = (float*)(w + L.rad[i]);
        b.typ[i] = (uint8_t*)(w + L.typ[i]);
        b.orig[i] = (int32_t*)(w + L.orig[i]);
    }
    b.scenes = batch ? (SceneDev*)(w + L.scenes) : nullptr;
    b.sid = batch ? (int32_t*)(w + L.sid) : nullptr;
    return b;
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

int kcap_for(int k) { return k <= 16 ? 16 : 32; }

// More than 48 KB of dynamic shared memory needs an explicit opt-in, set
// once per scene/batch on its device (outside any stream capture).
template <class SRC>
cudaError_t prepare_solve(int kcap, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (kcap == 16) {
        e = cudaFuncSetAttribute(solve_kernel<16, SRC, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(solve_kernel<16, SRC, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
        e = cudaFuncSetAttribute(solve_kernel<32, SRC, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(solve_kernel<32, SRC, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    return e;
}

template <class SRC>
void launch_solve(int kcap, bool count, int grid, int block, size_t smem, cudaStream_t st, int n,
                  SRC src, const float2* pos, const float2* vel, const float* rad,
                  const uint8_t* typ, const int32_t* orig, const uint32_t* start, AgentIn ain,
                  const float2* vpd, float2* out_pos, float2* out_vel, DebugOut dbg,
                  unsigned long long* counters) {
#define ORCA_SOLVE(K, C)                                                                   \
    solve_kernel<K, SRC, C><<<grid, block, smem, st>>>(n, src, pos, vel, rad, typ, orig,    \
                                                        start, ain, vpd, out_pos, out_vel, \
                                                        dbg, counters)
    if (kcap == 16) {
        if (count) ORCA_SOLVE(16, true);
        else ORCA_SOLVE(16, false);
    } else {
        if (count) ORCA_SOLVE(32, true);
        else ORCA_SOLVE(32, false);
    }
#undef ORCA_SOLVE
}

// Everything one call of the step pipeline needs: the caller's arrays, the
// workspace and the launch shape.  n_scenes == 0 is a single scene (its
// constants passed by value), otherwise a batch.
struct Pipeline {
    orca_agents agents;
    int n;
    int ncells;
    int nblocks;
    int kcap;
    int block;
    int n_scenes;
    Layout lay;
    char* ws;
    Buffers buf;
    SceneDev one;
    DebugOut dbg;
    cudaEvent_t ev_begin;
    cudaEvent_t ev_end;
    unsigned long long* counters;
    cudaGraphExec_t graph;
    int graph_steps;
};

size_t solve_smem(const Pipeline& P) { return (size_t)P.kcap * P.block * sizeof(float4); }

template <class SRC>
void enqueue_steps(const Pipeline& P, SRC src, int n_steps, const float* vpref_delta,
                   cudaStream_t st) {
    const int n = P.n;
    const Buffers& B = P.buf;
    const orca_agents& A = P.agents;
    const int tb = 256;
    const int gb = (n + tb - 1) / tb;
    {
        int g = (std::max(n, P.ncells) + tb - 1) / tb;
        g = std::min(g, 152 * 16);
        load_kernel<<<g, tb, 0, st>>>(n, (const float2*)A.pos, (const float2*)A.vel, A.radius,
                                      A.type, B.pos0, B.vel0, B.rad[0], B.typ[0], B.orig[0],
                                      B.count, P.ncells, B.err);
    }
    AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                A.n_waypoints, A.wp_idx};
    int cur = 0;
    const int sb = P.block;
    const int sgrid = (n + sb - 1) / sb;
    const size_t smem = solve_smem(P);
    for (int t = 0; t < n_steps; ++t) {
        bin_count_kernel<SRC><<<gb, tb, 0, st>>>(n, src, B.pos0, B.key, B.slot, B.count);
        scan_blocks_kernel<<<P.nblocks, kScanThreads, 0, st>>>(B.count, B.start, B.bsum,
                                                               P.ncells);
        scan_bsum_kernel<<<1, 1024, 0, st>>>(B.bsum, P.nblocks);
        scan_add_kernel<<<(P.ncells + 255) / 256, 256, 0, st>>>(B.start, B.bsum, P.ncells,
                                                                P.nblocks);
        scatter_kernel<<<gb, tb, 0, st>>>(n, B.key, B.slot, B.start, B.pos0, B.vel0,
                                          B.rad[cur], B.typ[cur], B.orig[cur], B.pos1, B.vel1,
                                          B.rad[1 - cur], B.typ[1 - cur], B.orig[1 - cur]);
        cur = 1 - cur;
        const float2* vpd =
            vpref_delta ? (const float2*)vpref_delta + (size_t)t * (size_t)n : nullptr;
        if (P.ev_begin) cudaEventRecord(P.ev_begin, st);
        launch_solve(P.kcap, P.counters != nullptr, sgrid, sb, smem, st, n, src, B.pos1, B.vel1,
                     B.rad[cur], B.typ[cur], B.orig[cur], B.start, ain, vpd, B.pos0, B.vel0,
                     P.dbg, P.counters);
        if (P.ev_end) cudaEventRecord(P.ev_end, st);
    }
    unload_kernel<<<gb, tb, 0, st>>>(n, B.orig[cur], B.pos0, B.vel0, (float2*)A.pos,
                                     (float2*)A.vel);
}

int run_steps(const Pipeline& P, int n_steps, const float* vpref_delta, cudaStream_t st) {
    if (P.n_scenes == 0) enqueue_steps(P, OneScene{P.one}, n_steps, vpref_delta, st);
    else enqueue_steps(P, ManyScenes{P.buf.scenes, P.buf.sid}, n_steps, vpref_delta, st);
    return cuda_status(cudaGetLastError());
}

int prepare(const Pipeline& P) {
    const size_t smem = solve_smem(P);
    cudaError_t e = P.n_scenes == 0 ? prepare_solve<OneScene>(P.kcap, smem)
                                    : prepare_solve<ManyScenes>(P.kcap, smem);
    return cuda_status(e);
}

int read_status(const Pipeline& P) {
    if (cudaDeviceSynchronize() != cudaSuccess) return ORCA_ERR_CUDA;
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, P.buf.err, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return ORCA_ERR_CUDA;
    if (cudaMemset(P.buf.err, 0, 16) != cudaSuccess) return ORCA_ERR_CUDA;
    if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
    if (h[0] & ERR_BIT_TIMEOUT) return ORCA_ERR_TIMEOUT;
    return ORCA_OK;
}

int launch_count(const Pipeline& P, int n_steps) {
    if (n_steps < 0) return -1;
    if (P.n == 0 || n_steps == 0) return 0;
    return 2 + 6 * n_steps;
}

void drop_graph(Pipeline& P) {
    if (P.graph) cudaGraphExecDestroy(P.graph);
    P.graph = nullptr;
    P.graph_steps = 0;
}

// Record n_steps of the pipeline into a CUDA graph.  Capture runs on a
// private non-blocking stream (capture executes nothing), so the caller's
// stream may be any stream, the legacy default one included.  Timing events
// and counters are left out of the graph.
int capture_graph(Pipeline& P, int n_steps, const float* vpref_delta) {
    drop_graph(P);
    if (P.n == 0 || n_steps == 0) return ORCA_OK;
    int st = prepare(P);
    if (st != ORCA_OK) return st;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ORCA_ERR_CUDA;
    cudaEvent_t eb = P.ev_begin, ee = P.ev_end;
    unsigned long long* cn = P.counters;
    P.ev_begin = P.ev_end = nullptr;
    P.counters = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = run_steps(P, n_steps, vpref_delta, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (st == ORCA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&P.graph, g, 0);
    }
    P.ev_begin = eb;
    P.ev_end = ee;
    P.counters = cn;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != ORCA_OK) return st;
    if (e != cudaSuccess) {
        P.graph = nullptr;
        return ORCA_ERR_CUDA;
    }
    P.graph_steps = n_steps;
    return ORCA_OK;
}

int launch_graph(Pipeline& P, cudaStream_t st) {
    if (P.n == 0 || P.graph_steps == 0) return ORCA_OK;
    if (!P.graph) return ORCA_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(P.graph, st));
}

void init_pipeline(Pipeline& P, const orca_agents* agents, int ncells, int kcap, int block,
                   int n_scenes, const Layout& lay, void* workspace, int k_stride) {
    P.agents = *agents;
    P.n = agents->n_agents;
    P.ncells = ncells;
    P.nblocks = (ncells + kScanChunk - 1) / kScanChunk;
    P.kcap = kcap;
    P.block = block ? block : 128;
    P.n_scenes = n_scenes;
    P.lay = lay;
    P.ws = (char*)workspace;
    P.buf = carve(P.ws, lay, n_scenes > 0);
    P.one = SceneDev{};
    P.dbg = DebugOut{nullptr, nullptr, nullptr, nullptr, nullptr, k_stride};
    P.ev_begin = P.ev_end = nullptr;
    P.counters = nullptr;
    P.graph = nullptr;
    P.graph_steps = 0;
}

// Host-side checks of a batch description; fills the total cell count and
// the largest k.
int check_batch(const orca_params* params, int n_scenes, const int* offsets, int n_agents,
                size_t* ncells_out, int* kmax_out) {
    if (!params || !offsets || n_scenes < 1) return ORCA_ERR_INVALID_ARG;
    if (n_scenes > ORCA_MAX_SCENES) return ORCA_ERR_CAPACITY;
    if (offsets[0] != 0 || offsets[n_scenes] != n_agents) return ORCA_ERR_INVALID_ARG;
    size_t ncells = 0;
    int kmax = 0;
    for (int s = 0; s < n_scenes; ++s) {
        int st = check_params(params + s);
        if (st != ORCA_OK) return st;
        if (offsets[s + 1] < offsets[s]) return ORCA_ERR_INVALID_ARG;
        if (params[s].block_size != params[0].block_size ||
            params[s].debug_flags != params[0].debug_flags)
            return ORCA_ERR_INVALID_ARG;
        ncells += (size_t)params[s].grid_nx * (size_t)params[s].grid_ny;
        if (ncells > (size_t)ORCA_MAX_CELLS) return ORCA_ERR_CAPACITY;
        kmax = std::max(kmax, params[s].max_neighbors);
    }
    *ncells_out = ncells;
    *kmax_out = kmax;
    return ORCA_OK;
}

}  // namespace

struct orca_scene {
    orca_params params;
    Pipeline p;
};

struct orca_batch {
    int n_scenes;
    int kmax;
    Pipeline p;
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

int orca_abi_version(void) { return 2; }

int orca_workspace_bytes(const orca_params* params, int n_agents, size_t* out_bytes) {
    int st = check_params(params);
    if (st != ORCA_OK) return st;
    if (n_agents < 0 || !out_bytes) return ORCA_ERR_INVALID_ARG;
    size_t ncells = (size_t)params->grid_nx * (size_t)params->grid_ny;
    *out_bytes = make_layout((size_t)n_agents, ncells, 0).total;
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
    Layout lay = make_layout((size_t)agents->n_agents, ncells, 0);
    if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total)
        return ORCA_ERR_INVALID_ARG;
    orca_scene* s = new (std::nothrow) orca_scene;
    if (!s) return ORCA_ERR_CAPACITY;
    s->params = *params;
    init_pipeline(s->p, agents, (int)ncells, kcap_for(params->max_neighbors),
                  params->block_size, 0, lay, workspace, params->max_neighbors);
    s->p.one = scene_dev(params, 0, s->p.n, 0);
    if (cudaMemset(s->p.buf.err, 0, 16) != cudaSuccess || prepare(s->p) != ORCA_OK) {
        delete s;
        return ORCA_ERR_CUDA;
    }
    *out = s;
    return ORCA_OK;
}

int orca_scene_set_debug(orca_scene* s, int32_t* cell, int32_t* nbr, int32_t* cnt,
                         uint8_t* flags, float* tstar) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    s->p.dbg = DebugOut{cell, nbr, cnt, flags, tstar, s->params.max_neighbors};
    return ORCA_OK;
}

int orca_scene_set_solve_events(orca_scene* s, void* begin, void* end) {
    if (!s || ((begin == nullptr) != (end == nullptr))) return ORCA_ERR_INVALID_ARG;
    s->p.ev_begin = (cudaEvent_t)begin;
    s->p.ev_end = (cudaEvent_t)end;
    return ORCA_OK;
}

int orca_scene_set_counters(orca_scene* s, unsigned long long* counters) {
    if (!s || (counters && !aligned(counters, 8))) return ORCA_ERR_INVALID_ARG;
    s->p.counters = counters;
    return ORCA_OK;
}

int orca_step_launch_count(const orca_scene* s, int n_steps) {
    if (!s) return -1;
    return launch_count(s->p, n_steps);
}

int orca_step(orca_scene* s, int n_steps, const float* vpref_delta, void* stream) {
    if (!s || n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    if (s->p.n == 0 || n_steps == 0) return ORCA_OK;
    return run_steps(s->p, n_steps, vpref_delta, (cudaStream_t)stream);
}

int orca_scene_graph_capture(orca_scene* s, int n_steps, const float* vpref_delta) {
    if (!s || n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    return capture_graph(s->p, n_steps, vpref_delta);
}

int orca_scene_graph_launch(orca_scene* s, void* stream) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    return launch_graph(s->p, (cudaStream_t)stream);
}

int orca_scene_sync_status(orca_scene* s) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    return read_status(s->p);
}

void orca_scene_destroy(orca_scene* s) {
    if (!s) return;
    drop_graph(s->p);
    delete s;
}

// ------------------------------------------------------------- batches ----

int orca_batch_workspace_bytes(const orca_params* params, int n_scenes, const int* offsets,
                               size_t* out_bytes) {
    if (!out_bytes || !offsets || n_scenes < 1) return ORCA_ERR_INVALID_ARG;
    size_t ncells = 0;
    int kmax = 0;
    int st = check_batch(params, n_scenes, offsets, offsets[n_scenes], &ncells, &kmax);
    if (st != ORCA_OK) return st;
    if (offsets[n_scenes] < 0) return ORCA_ERR_INVALID_ARG;
    *out_bytes = make_layout((size_t)offsets[n_scenes], ncells, (size_t)n_scenes).total;
    return ORCA_OK;
}

int orca_batch_create(const orca_params* params, int n_scenes, const int* offsets,
                      const orca_agents* agents, void* workspace, size_t workspace_bytes,
                      orca_batch** out) {
    if (!out) return ORCA_ERR_INVALID_ARG;
    *out = nullptr;
    int st = check_agents(agents);
    if (st != ORCA_OK) return st;
    size_t ncells = 0;
    int kmax = 0;
    st = check_batch(params, n_scenes, offsets, agents->n_agents, &ncells, &kmax);
    if (st != ORCA_OK) return st;
    const int n = agents->n_agents;
    Layout lay = make_layout((size_t)n, ncells, (size_t)n_scenes);
    if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total)
        return ORCA_ERR_INVALID_ARG;
    std::vector<SceneDev> table((size_t)n_scenes);
    std::vector<int32_t> sid((size_t)n);
    int cell_off = 0;
    for (int s = 0; s < n_scenes; ++s) {
        table[s] = scene_dev(params + s, offsets[s], offsets[s + 1] - offsets[s], cell_off);
        cell_off += params[s].grid_nx * params[s].grid_ny;
        for (int i = offsets[s]; i < offsets[s + 1]; ++i) sid[i] = s;
    }
    orca_batch* b = new (std::nothrow) orca_batch;
    if (!b) return ORCA_ERR_CAPACITY;
    b->n_scenes = n_scenes;
    b->kmax = kmax;
    init_pipeline(b->p, agents, (int)ncells, kcap_for(kmax), params[0].block_size, n_scenes, lay,
                  workspace, kmax);
    bool ok = cudaMemset(b->p.buf.err, 0, 16) == cudaSuccess &&
              cudaMemcpy(b->p.buf.scenes, table.data(), table.size() * sizeof(SceneDev),
                         cudaMemcpyHostToDevice) == cudaSuccess &&
              (n == 0 || cudaMemcpy(b->p.buf.sid, sid.data(), sid.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice) == cudaSuccess) &&
              prepare(b->p) == ORCA_OK;
    if (!ok) {
        delete b;
        return ORCA_ERR_CUDA;
    }
    *out = b;
    return ORCA_OK;
}

int orca_batch_set_debug(orca_batch* b, int32_t* cell, int32_t* nbr, int32_t* cnt,
                         uint8_t* flags, float* tstar) {
    if (!b) return ORCA_ERR_INVALID_ARG;
    b->p.dbg = DebugOut{cell, nbr, cnt, flags, tstar, b->kmax};
    return ORCA_OK;
}

int orca_step_batched(orca_batch* b, int n_steps, const float* vpref_delta, void* stream) {
    if (!b || n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    if (b->p.n == 0 || n_steps == 0) return ORCA_OK;
    return run_steps(b->p, n_steps, vpref_delta, (cudaStream_t)stream);
}

int orca_batch_launch_count(const orca_batch* b, int n_steps) {
    if (!b) return -1;
    return launch_count(b->p, n_steps);
}

int orca_batch_graph_capture(orca_batch* b, int n_steps, const float* vpref_delta) {
    if (!b || n_steps < 0) return ORCA_ERR_INVALID_ARG;
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    return capture_graph(b->p, n_steps, vpref_delta);
}

int orca_batch_graph_launch(orca_batch* b, void* stream) {
    if (!b) return ORCA_ERR_INVALID_ARG;
    return launch_graph(b->p, (cudaStream_t)stream);
}

int orca_batch_sync_status(orca_batch* b) {
    if (!b) return ORCA_ERR_INVALID_ARG;
    return read_status(b->p);
}

void orca_batch_destroy(orca_batch* b) {
    if (!b) return;
    drop_graph(b->p);
    delete b;
}

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
    const Layout L = make_layout((size_t)agents->n_agents, ncells, 0);
    if (L.total > (size_t)ORCA_NOALLOC_SCRATCH_BYTES) return ORCA_ERR_CAPACITY;
    const int n = agents->n_agents;
    if (n == 0 || n_steps == 0) return ORCA_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ORCA_ERR_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return ORCA_ERR_CAPACITY;
    char* w = noalloc_base(dev);
    if (w == nullptr) return ORCA_ERR_CUDA;
    cudaStream_t stm = (cudaStream_t)stream;

    // a pipeline over the scratch area, held on the host stack
    Pipeline P;
    init_pipeline(P, agents, (int)ncells, kcap_for(params->max_neighbors), params->block_size,
                  0, L, w, params->max_neighbors);
    P.one = scene_dev(params, 0, n, 0);
    st = prepare(P);
    if (st != ORCA_OK) return st;
    // the error word and the cell counts must start at zero; the load
    // kernel clears the counts, the error word is cleared here
    if (cudaMemsetAsync(P.buf.err, 0, 16, stm) != cudaSuccess) return ORCA_ERR_CUDA;
    st = run_steps(P, n_steps, vpref_delta, stm);
    if (st != ORCA_OK) return st;
    if (synchronize) {
        if (cudaStreamSynchronize(stm) != cudaSuccess) return ORCA_ERR_CUDA;
        int h[4] = {0, 0, 0, 0};
        if (cudaMemcpy(h, P.buf.err, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return ORCA_ERR_CUDA;
        if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
        if (h[0] & ERR_BIT_TIMEOUT) return ORCA_ERR_TIMEOUT;
    }
    return ORCA_OK;
}
