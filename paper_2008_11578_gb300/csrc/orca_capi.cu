// orca_capi.cu -- the C ABI of liborca (declared in include/orca.h).
//
// Host side of the ORCA step: argument validation, workspace layout, and
// the launch sequence: per step one cooperative binning kernel (on a call's
// first step it reads the caller's arrays) and the solve kernel (which bins
// the new positions for the next step, and writes the last step's results
// straight into the caller's arrays).
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

#include <nvtx3/nvToolsExt.h>

#include "orca.h"
#include "orca_adjoint.cuh"
#include "orca_step_kernels.cuh"

using namespace orca;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace carve-up (device, caller owned).  The scene table and the scene
// id of every slot exist only for batches (n_scenes > 0).
struct Layout {
    size_t err, count, start, bsum, key, slot, hint, xrank, pos0, vel0, pos1, vel1;
    size_t aux[2];
    size_t scenes, sid;
    size_t total;
};

Layout make_layout(size_t n, size_t ncells, size_t n_scenes) {
    Layout L{};
    // block sums of the binning kernel's scan (one per launch block), and of
    // the agent scan of orca_scene_remove_arrived
    size_t nb = std::max((std::max(ncells, n) + kScanChunk - 1) / kScanChunk,
                         (size_t)kBinGridMax);
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
    L.slot = take((n + 1) * 4);   // + the total of the agent scan
    L.hint = take(n * 4);
    L.xrank = take(n * 16);
    L.pos0 = take(n * 8);
    L.vel0 = take(n * 8);
    L.pos1 = take(n * 8);
    L.vel1 = take(n * 8);
    for (int b = 0; b < 2; ++b) {
        L.aux[b] = take(n * 8);
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
    uint32_t *count, *start, *bsum, *key, *slot, *hint;
    uint4* xrank;
    float2 *pos0, *vel0, *pos1, *vel1;
    uint2* aux[2];
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
    b.hint = (uint32_t*)(w + L.hint);
    b.xrank = (uint4*)(w + L.xrank);
    b.pos0 = (float2*)(w + L.pos0);
    b.vel0 = (float2*)(w + L.vel0);
    b.pos1 = (float2*)(w + L.pos1);
    b.vel1 = (float2*)(w + L.vel1);
    for (int i = 0; i < 2; ++i) {
        b.aux[i] = (uint2*)(w + L.aux[i]);
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
    if (!std::isfinite(p->cell_height) || p->cell_height < 0.0f) return ORCA_ERR_INVALID_ARG;
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
    const unsigned schemes = ORCA_FLAG_LP_WORK_UNITS | ORCA_FLAG_LP_ENUMERATION |
                             ORCA_FLAG_LP_WARP | ORCA_DEBUG_CHECKED;
    if (p->debug_flags & ~(schemes | ORCA_DEBUG_BARRIER_TIMEOUT)) return ORCA_ERR_INVALID_ARG;
    const unsigned scheme = p->debug_flags & schemes;
    if (scheme & (scheme - 1u)) return ORCA_ERR_INVALID_ARG;   // one LP scheme at a time
    if (!std::isfinite(p->vehicle_turn_rate) || !std::isfinite(p->vehicle_accel) ||
        p->vehicle_turn_rate < 0.0f || p->vehicle_accel < 0.0f ||
        (double)p->vehicle_turn_rate * (double)p->dt >= 1.5707963267948966)
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

// row-bound margin of the neighbour search: computed cell coordinates differ
// from exact ones by a relative 3u (two roundings and the rounded inverse);
// 16u of the largest coordinate covers both agents with room to spare
float ring_delta_for(int nx, int ny) {
    double u = std::ldexp(1.0, -24);
    return (float)(16.0 * u * (double)(std::max(nx, ny) + 2));
}

float cell_height(const orca_params* p) {
    return p->cell_height > 0.0f ? p->cell_height : p->cell_size;
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
    volatile float one = 1.0f;
    s.cell_w = p->cell_size;
    s.cell_h = cell_height(p);
    s.inv_cell_x = one / s.cell_w;
    s.inv_cell_y = one / s.cell_h;
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
    const double th = (double)p->vehicle_turn_rate * (double)p->dt;
    s.kin_turn = p->vehicle_turn_rate > 0.0f;
    s.kin_accel = p->vehicle_accel > 0.0f;
    s.cos_turn = (float)std::cos(th);
    s.sin_turn = (float)std::sin(th);
    volatile float a = p->vehicle_accel;
    s.accel_dt = a * p->dt;
    return s;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ORCA_OK : ORCA_ERR_CUDA; }

// float4 slots per thread: the neighbour list, then the lines (plus the
// vehicles' kinematic half-planes)
int kcap_for(int k, bool kin) { return std::max(k, 1) + (kin ? kKinLines : 0); }
bool kinematic(const orca_params* p) {
    return p->vehicle_turn_rate > 0.0f || p->vehicle_accel > 0.0f;
}

// More than 48 KB of dynamic shared memory needs an explicit opt-in, set
// once per scene/batch on its device (outside any stream capture).
template <class SRC>
cudaError_t prepare_solve(size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_PLAIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_COUNT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_RECORD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_PLAIN, LP_WORK_UNITS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_PLAIN, LP_ENUMERATION>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_PLAIN, LP_WARP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<SRC, MODE_CHECK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

template <class SRC>
void launch_solve(int mode, int grid, int block, size_t smem, cudaStream_t st, int n, SRC src,
                  const float2* pos, const float2* vel, const uint2* aux, const uint32_t* start,
                  AgentIn ain, const float2* vpd, StepOut out, DebugOut dbg,
                  unsigned long long* counters, int* err) {
#define ORCA_SOLVE(M, W)                                                                    \
    solve_kernel<SRC, M, W><<<grid, block, smem, st>>>(n, src, pos, vel, aux, start, ain, vpd, \
                                                        out, dbg, counters, err)
    if (mode == MODE_COUNT) ORCA_SOLVE(MODE_COUNT, LP_INCREMENTAL);
    else if (mode == MODE_RECORD) ORCA_SOLVE(MODE_RECORD, LP_INCREMENTAL);
    else if (mode == MODE_WORK_UNITS) ORCA_SOLVE(MODE_PLAIN, LP_WORK_UNITS);
    else if (mode == MODE_ENUMERATION) ORCA_SOLVE(MODE_PLAIN, LP_ENUMERATION);
    else if (mode == MODE_WARP_LP) ORCA_SOLVE(MODE_PLAIN, LP_WARP);
    else if (mode == MODE_CHECK) ORCA_SOLVE(MODE_CHECK, LP_INCREMENTAL);
    else ORCA_SOLVE(MODE_PLAIN, LP_INCREMENTAL);
#undef ORCA_SOLVE
}

// Everything one call of the step pipeline needs: the caller's arrays, the
// workspace and the launch shape.  n_scenes == 0 is a single scene (its
// constants passed by value), otherwise a batch.
struct Pipeline {
    orca_agents agents;
    int n;
    int ncells;
    int kcap;
    int block;
    int n_scenes;
    unsigned flags;   // orca_params.debug_flags
    Layout lay;
    char* ws;
    Buffers buf;
    SceneDev one;
    DebugOut dbg;
    cudaEvent_t ev_begin;
    cudaEvent_t ev_end;
    cudaEvent_t bin_begin;
    cudaEvent_t bin_end;
    unsigned long long* counters;
    cudaGraphExec_t graph;
    int graph_steps;
    int bin_grid_max;   // co-resident blocks of the binning kernel on this device
};

size_t solve_smem(const Pipeline& P) { return (size_t)P.kcap * P.block * sizeof(float4); }

// The solve variant and diagnostics of an ordinary step.
struct SameDebug {
    DebugOut d;
    __host__ DebugOut operator()(int) const { return d; }
};

int step_mode(const Pipeline& P) {
    if (P.counters != nullptr) return MODE_COUNT;
    if (P.dbg.act != nullptr) return MODE_RECORD;
    if (P.flags & ORCA_FLAG_LP_WORK_UNITS) return MODE_WORK_UNITS;
    if (P.flags & ORCA_FLAG_LP_WARP) return MODE_WARP_LP;
    if (P.flags & ORCA_DEBUG_CHECKED) return MODE_CHECK;
    return (P.flags & ORCA_FLAG_LP_ENUMERATION) ? MODE_ENUMERATION : MODE_PLAIN;
}

// The binning kernel of one step (cooperative launch, grid sized to what is
// resident at once on this device).  first: from the caller's arrays.
template <class SRC>
void launch_bin(const Pipeline& P, SRC src, bool first, int cur, cudaStream_t st) {
    const Buffers& B = P.buf;
    const orca_agents& A = P.agents;
    const BinArgs a{P.n, P.ncells, (const float2*)A.pos, (const float2*)A.vel, A.radius, A.type,
                    B.pos0, B.vel0, B.aux[cur], B.pos0, B.vel0, B.aux[cur], B.key, B.slot,
                    B.count, B.start, B.bsum, B.xrank,
                    B.pos1, B.vel1, B.aux[1 - cur], B.err, B.hint,
                    (P.flags & ORCA_DEBUG_BARRIER_TIMEOUT) ? 1 : 0};
    const long long work = std::max((long long)P.n, (long long)P.ncells / 4);
    const int grid = (int)std::max(
        1LL, std::min((long long)P.bin_grid_max, (work + kBinThreads - 1) / kBinThreads));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBinThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (first) cudaLaunchKernelEx(&cfg, bin_kernel<SRC, true>, src, a);
    else cudaLaunchKernelEx(&cfg, bin_kernel<SRC, false>, src, a);
}

// Enqueue n_steps steps.  dbg_for(t) gives the solve
// kernel's optional outputs of step t.
template <class SRC, class DBG>
void enqueue_steps(const Pipeline& P, SRC src, int n_steps, const float* vpref_delta,
                   cudaStream_t st, DBG dbg_for, int mode) {
    const int n = P.n;
    const Buffers& B = P.buf;
    const orca_agents& A = P.agents;
    AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                A.n_waypoints, A.wp_idx};
    int cur = 0;
    const int sb = P.block;
    const int sgrid = (n + sb - 1) / sb;
    const size_t smem = solve_smem(P);
    // NVTX ranges (host side: the enqueue of each step and its two kernels)
    nvtxRangePushA("orca_step");
    for (int t = 0; t < n_steps; ++t) {
        nvtxRangePushA("orca_step/binning");
        if (P.bin_begin) cudaEventRecord(P.bin_begin, st);
        // step 0 bins the caller's state; later steps were binned by the
        // previous step's solve kernel
        launch_bin(P, src, t == 0, cur, st);
        cur = 1 - cur;
        if (P.bin_end) cudaEventRecord(P.bin_end, st);
        nvtxRangePop();
        nvtxRangePushA("orca_step/solve");
        const float2* vpd =
            vpref_delta ? (const float2*)vpref_delta + (size_t)t * (size_t)n : nullptr;
        if (P.ev_begin) cudaEventRecord(P.ev_begin, st);
        const bool last = t == n_steps - 1;
        const StepOut out = last ? StepOut{(float2*)A.pos, (float2*)A.vel, true, nullptr, nullptr,
                                           nullptr, B.hint, B.err + 1}
                                 : StepOut{B.pos0, B.vel0, false, B.key, B.slot, B.count,
                                           nullptr, nullptr};
        launch_solve(mode, sgrid, sb, smem, st, n, src, B.pos1, B.vel1, B.aux[cur], B.start,
                     ain, vpd, out, dbg_for(t), P.counters, B.err);
        if (P.ev_end) cudaEventRecord(P.ev_end, st);
        nvtxRangePop();
    }
    nvtxRangePop();
}

int run_steps(const Pipeline& P, int n_steps, const float* vpref_delta, cudaStream_t st) {
    const SameDebug dbg{P.dbg};
    const int mode = step_mode(P);
    if (P.n_scenes == 0) enqueue_steps(P, OneScene{P.one}, n_steps, vpref_delta, st, dbg, mode);
    else
        enqueue_steps(P, ManyScenes{P.buf.scenes, P.buf.sid}, n_steps, vpref_delta, st, dbg,
                      mode);
    return cuda_status(cudaGetLastError());
}

// Blocks of the binning kernel that are resident at once on the current
// device (both variants), at most kBinGridMax.
template <class SRC>
cudaError_t bin_grid_max(int* out) {
    int dev = 0, sms = 0, b0 = 0, b1 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, bin_kernel<SRC, false>, kBinThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, bin_kernel<SRC, true>, kBinThreads, 0);
    if (e == cudaSuccess && std::min(b0, b1) < 1) e = cudaErrorInvalidConfiguration;
    *out = std::max(1, std::min(kBinGridMax, std::min(b0, b1) * sms));
    return e;
}

int prepare(Pipeline& P) {
    const size_t smem = solve_smem(P);
    cudaError_t e = P.n_scenes == 0 ? prepare_solve<OneScene>(smem)
                                    : prepare_solve<ManyScenes>(smem);
    if (e == cudaSuccess)
        e = P.n_scenes == 0 ? bin_grid_max<OneScene>(&P.bin_grid_max)
                            : bin_grid_max<ManyScenes>(&P.bin_grid_max);
    return cuda_status(e);
}

int read_status(const Pipeline& P) {
    if (cudaDeviceSynchronize() != cudaSuccess) return ORCA_ERR_CUDA;
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, P.buf.err, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return ORCA_ERR_CUDA;
    if (h[0] == 0) return ORCA_OK;   // nothing to clear; the recorded cell order stays
    // clears the status bits, the recorded cell order and the binning
    // kernel's barrier words; after a barrier gave up, the cell counts may be
    // left mid-step, so clear them too
    if (cudaMemset(P.buf.err, 0, 16) != cudaSuccess) return ORCA_ERR_CUDA;
    if ((h[0] & (ERR_BIT_TIMEOUT | ERR_BIT_STATE)) &&
        cudaMemset(P.buf.count, 0, (size_t)P.ncells * 4) != cudaSuccess)
        return ORCA_ERR_CUDA;
    if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
    if (h[0] & (ERR_BIT_TIMEOUT | ERR_BIT_STATE)) return ORCA_ERR_TIMEOUT;
    if (h[0] & ERR_BIT_CHECK) return ORCA_ERR_CHECK;
    return ORCA_OK;
}

int launch_count(const Pipeline& P, int n_steps) {
    if (n_steps < 0) return -1;
    if (P.n == 0 || n_steps == 0) return 0;
    return 2 * n_steps;   // binning + solve per step
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
    cudaEvent_t eb = P.ev_begin, ee = P.ev_end, bb = P.bin_begin, be = P.bin_end;
    unsigned long long* cn = P.counters;
    P.ev_begin = P.ev_end = P.bin_begin = P.bin_end = nullptr;
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
    P.bin_begin = bb;
    P.bin_end = be;
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
                   int n_scenes, const Layout& lay, void* workspace, int k_stride,
                   unsigned flags) {
    P.agents = *agents;
    P.flags = flags;
    P.n = agents->n_agents;
    P.ncells = ncells;
    P.kcap = kcap;
    P.block = block ? block : 128;
    P.n_scenes = n_scenes;
    P.lay = lay;
    P.ws = (char*)workspace;
    P.buf = carve(P.ws, lay, n_scenes > 0);
    P.one = SceneDev{};
    P.dbg = DebugOut{};
    P.dbg.k_stride = k_stride;
    P.ev_begin = P.ev_end = nullptr;
    P.bin_begin = P.bin_end = nullptr;
    P.counters = nullptr;
    P.graph = nullptr;
    P.graph_steps = 0;
    P.bin_grid_max = 1;
}

// Host-side checks of a batch description; fills the total cell count and
// the largest k.
int check_batch(const orca_params* params, int n_scenes, const int* offsets, int n_agents,
                size_t* ncells_out, int* kmax_out, bool* kin_out = nullptr) {
    if (!params || !offsets || n_scenes < 1) return ORCA_ERR_INVALID_ARG;
    if (n_scenes > ORCA_MAX_SCENES) return ORCA_ERR_CAPACITY;
    if (offsets[0] != 0 || offsets[n_scenes] != n_agents) return ORCA_ERR_INVALID_ARG;
    size_t ncells = 0;
    int kmax = 0;
    bool kin = false;
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
        kin = kin || kinematic(params + s);
    }
    *ncells_out = ncells;
    *kmax_out = kmax;
    if (kin_out) *kin_out = kin;
    return ORCA_OK;
}

// Adjoint workspace (caller owned): checkpoints of the rollout, the state
// a segment is replayed from, what the replay records for each step of a
// segment, and three rotating pairs of state cotangents.
struct AdjLayout {
    int n_ck;
    size_t ck_pos, ck_vel, ck_wp;
    size_t rp_pos, rp_vel, rp_wp;
    size_t r_pos, r_vel, r_nbr, r_act, r_wp, r_vnew;
    size_t bar_p[3], bar_v[3];
    size_t total;
};

AdjLayout make_adj_layout(size_t n, int k, int n_steps, int K) {
    AdjLayout L{};
    L.n_ck = (n_steps + K - 1) / K;
    const size_t ck = (size_t)std::max(L.n_ck, 1);
    const size_t kk = (size_t)std::max(k, 1);
    const size_t seg = (size_t)std::min(std::max(n_steps, 1), K);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.ck_pos = take(ck * n * 8);
    L.ck_vel = take(ck * n * 8);
    L.ck_wp = take(ck * n);
    L.rp_pos = take(n * 8);
    L.rp_vel = take(n * 8);
    L.rp_wp = take(n);
    L.r_pos = take(seg * n * 8);
    L.r_vel = take(seg * n * 8);
    L.r_nbr = take(seg * n * kk * 4);
    L.r_act = take(seg * n * 4);
    L.r_wp = take(seg * n);
    L.r_vnew = take(seg * n * 8);
    for (int b = 0; b < 3; ++b) {
        L.bar_p[b] = take(n * 8);
        L.bar_v[b] = take(n * 8);
    }
    L.total = o;
    return L;
}

}  // namespace

struct orca_scene {
    orca_params params;
    Pipeline p;
    // the last orca_rollout: its length, checkpoint interval and workspace
    int adj_steps;
    int adj_every;
    void* adj_ws;
};

namespace {

int check_adjoint_args(const orca_scene* s, int n_steps, int ckpt_every, void* adj_ws,
                       size_t adj_bytes, const float* vpref_delta) {
    if (!s || n_steps < 0 || ckpt_every < 1) return ORCA_ERR_INVALID_ARG;
    if (kinematic(&s->params)) return ORCA_ERR_INVALID_ARG;   // not differentiated
    if (vpref_delta && !aligned(vpref_delta, 8)) return ORCA_ERR_INVALID_ARG;
    const AdjLayout L = make_adj_layout((size_t)s->p.n, s->params.max_neighbors, n_steps,
                                        ckpt_every);
    if (!adj_ws || !aligned(adj_ws, kAlign) || adj_bytes < L.total) return ORCA_ERR_INVALID_ARG;
    return ORCA_OK;
}

// Per-step outputs of the checkpointing forward: the new velocity of every
// step, and the state at the start of every ckpt_every-th step.
struct RolloutDebug {
    DebugOut base;
    float2* vel_traj;
    float2* ck_pos;
    float2* ck_vel;
    uint8_t* ck_wp;
    int n;
    int every;
    __host__ DebugOut operator()(int t) const {
        DebugOut d = base;
        d.vnew = vel_traj ? vel_traj + (size_t)t * n : nullptr;
        if (t % every == 0) {
            const size_t c = (size_t)(t / every) * n;
            d.spos = ck_pos + c;
            d.svel = ck_vel + c;
            d.swp = ck_wp ? ck_wp + c : nullptr;
        }
        return d;
    }
};

// Per-step records of a replayed segment for the adjoint kernel.
struct ReplayDebug {
    DebugOut base;
    float2* r_pos;
    float2* r_vel;
    int32_t* r_nbr;
    uint32_t* r_act;
    uint8_t* r_wp;
    float2* r_vnew;
    int n;
    int k;
    __host__ DebugOut operator()(int t) const {
        DebugOut d = base;
        const size_t o = (size_t)t * n;
        d.spos = r_pos + o;
        d.svel = r_vel + o;
        d.nbr = r_nbr + o * (size_t)k;
        d.act = r_act + o;
        d.wp_used = r_wp ? r_wp + o : nullptr;
        d.vnew = r_vnew + o;
        return d;
    }
};

}  // namespace

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
        case ORCA_ERR_CHECK: return "checked step: invariant violated";
        default: return "unknown status";
    }
}

int orca_abi_version(void) { return 5; }

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
    init_pipeline(s->p, agents, (int)ncells, kcap_for(params->max_neighbors, kinematic(params)),
                  params->block_size, 0, lay, workspace, params->max_neighbors,
                  params->debug_flags);
    s->p.one = scene_dev(params, 0, s->p.n, 0);
    s->adj_steps = -1;
    s->adj_every = 0;
    s->adj_ws = nullptr;
    // the binning kernel expects zero cell counts on entry
    if (cudaMemset(s->p.buf.err, 0, 16) != cudaSuccess ||
        cudaMemset(s->p.buf.count, 0, ncells * 4) != cudaSuccess || prepare(s->p) != ORCA_OK) {
        delete s;
        return ORCA_ERR_CUDA;
    }
    *out = s;
    return ORCA_OK;
}

int orca_scene_set_debug(orca_scene* s, int32_t* cell, int32_t* nbr, int32_t* cnt,
                         uint8_t* flags, float* tstar) {
    if (!s) return ORCA_ERR_INVALID_ARG;
    s->p.dbg.cell = cell;
    s->p.dbg.nbr = nbr;
    s->p.dbg.cnt = cnt;
    s->p.dbg.flags = flags;
    s->p.dbg.tstar = tstar;
    return ORCA_OK;
}

int orca_scene_set_solve_events(orca_scene* s, void* begin, void* end) {
    if (!s || ((begin == nullptr) != (end == nullptr))) return ORCA_ERR_INVALID_ARG;
    s->p.ev_begin = (cudaEvent_t)begin;
    s->p.ev_end = (cudaEvent_t)end;
    return ORCA_OK;
}

int orca_scene_set_bin_events(orca_scene* s, void* begin, void* end) {
    if (!s || ((begin == nullptr) != (end == nullptr))) return ORCA_ERR_INVALID_ARG;
    s->p.bin_begin = (cudaEvent_t)begin;
    s->p.bin_end = (cudaEvent_t)end;
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

int orca_scene_remove_arrived(orca_scene* s, int* n_kept, int32_t* kept_index, void* stream) {
    if (!s || !n_kept) return ORCA_ERR_INVALID_ARG;
    if (kept_index && !aligned(kept_index, 4)) return ORCA_ERR_INVALID_ARG;
    Pipeline& P = s->p;
    const int n = P.n;
    *n_kept = n;
    if (n == 0) return ORCA_OK;
    if ((size_t)n > (size_t)kScanChunk * 1024 * 16) return ORCA_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    const Buffers& B = P.buf;
    const orca_agents& A = P.agents;
    const int tb = 256, gb = (n + tb - 1) / tb;
    const int nb = (n + kScanChunk - 1) / kScanChunk;
    // keep flags -> exclusive scan (destinations) -> gather into the step
    // buffers -> copy back to the front of the caller's arrays
    arrived_kernel<<<gb, tb, 0, st>>>(n, (const float2*)A.pos, (const float2*)A.goal, A.radius,
                                      A.route, (const float2*)A.waypoints, A.n_waypoints,
                                      A.wp_idx, B.key);
    scan_blocks_kernel<<<nb, kScanThreads, 0, st>>>(B.key, B.slot, B.bsum, n);
    scan_bsum_kernel<<<1, 1024, 0, st>>>(B.bsum, nb);
    scan_add_kernel<<<(n / 4 + 256) / 256, 256, 0, st>>>(B.slot, B.bsum, n, nb);
    compact_gather_kernel<<<gb, tb, 0, st>>>(n, B.slot, (const float2*)A.pos, (const float2*)A.vel,
                                             (const float2*)A.goal, A.radius, A.max_speed, A.type,
                                             A.route, A.wp_idx, B.pos0, B.vel0, B.pos1, B.vel1,
                                             B.aux[0], B.aux[1]);
    uint32_t kept = 0;
    if (cudaMemcpyAsync(&kept, B.slot + n, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ORCA_ERR_CUDA;
    if (kept > 0)
        compact_scatter_kernel<<<((int)kept + tb - 1) / tb, tb, 0, st>>>(
            (int)kept, B.pos0, B.vel0, B.pos1, B.vel1, B.aux[0], B.aux[1], (float2*)A.pos,
            (float2*)A.vel, (float2*)A.goal, (float*)A.radius, (float*)A.max_speed,
            (uint8_t*)A.type, (int32_t*)A.route, A.wp_idx, kept_index);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return ORCA_ERR_CUDA;
    // the recorded sorted order names the old indices: bin the next call in
    // the caller's order
    if (cudaMemsetAsync(B.err + 1, 0, 4, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ORCA_ERR_CUDA;
    P.n = (int)kept;
    drop_graph(P);   // a graph recorded for the old count is stale
    s->adj_steps = -1;
    *n_kept = (int)kept;
    return ORCA_OK;
}

int orca_scene_set_debug_active(orca_scene* s, uint32_t* act) {
    if (!s || (act && !aligned(act, 4))) return ORCA_ERR_INVALID_ARG;
    s->p.dbg.act = act;
    return ORCA_OK;
}

// ------------------------------------------------------------- adjoint ----

int orca_adjoint_workspace_bytes(const orca_scene* s, int n_steps, int ckpt_every,
                                 size_t* out_bytes) {
    if (!s || !out_bytes || n_steps < 0 || ckpt_every < 1) return ORCA_ERR_INVALID_ARG;
    *out_bytes =
        make_adj_layout((size_t)s->p.n, s->params.max_neighbors, n_steps, ckpt_every).total;
    return ORCA_OK;
}

int orca_rollout(orca_scene* s, int n_steps, int ckpt_every, const float* vpref_delta,
                 void* adj_ws, size_t adj_bytes, float* vel_traj, void* stream) {
    int st = check_adjoint_args(s, n_steps, ckpt_every, adj_ws, adj_bytes, vpref_delta);
    if (st != ORCA_OK) return st;
    if (vel_traj && !aligned(vel_traj, 8)) return ORCA_ERR_INVALID_ARG;
    s->adj_steps = -1;
    const int n = s->p.n;
    if (n > 0 && n_steps > 0) {
        const AdjLayout L = make_adj_layout((size_t)n, s->params.max_neighbors, n_steps,
                                            ckpt_every);
        char* w = (char*)adj_ws;
        RolloutDebug dbg{DebugOut{}, (float2*)vel_traj, (float2*)(w + L.ck_pos),
                         (float2*)(w + L.ck_vel),
                         s->p.agents.route ? (uint8_t*)(w + L.ck_wp) : nullptr, n, ckpt_every};
        dbg.base.k_stride = s->params.max_neighbors;
        enqueue_steps(s->p, OneScene{s->p.one}, n_steps, vpref_delta, (cudaStream_t)stream, dbg,
                      MODE_PLAIN);
        st = cuda_status(cudaGetLastError());
        if (st != ORCA_OK) return st;
    }
    s->adj_steps = n_steps;
    s->adj_every = ckpt_every;
    s->adj_ws = adj_ws;
    return ORCA_OK;
}

int orca_adjoint(orca_scene* s, int n_steps, int ckpt_every, const float* vpref_delta,
                 void* adj_ws, size_t adj_bytes, const float* dl_dpos, const float* dl_dvel_traj,
                 float* dl_dvpref_delta, float* dl_dwaypoints, float* dl_dpos0, float* dl_dvel0,
                 void* stream) {
    int st = check_adjoint_args(s, n_steps, ckpt_every, adj_ws, adj_bytes, vpref_delta);
    if (st != ORCA_OK) return st;
    if (s->adj_steps != n_steps || s->adj_every != ckpt_every || s->adj_ws != adj_ws)
        return ORCA_ERR_INVALID_ARG;
    const int n = s->p.n;
    if (n > 0 && !dl_dpos) return ORCA_ERR_INVALID_ARG;
    const void* ptrs[] = {dl_dpos, dl_dvel_traj, dl_dvpref_delta, dl_dwaypoints, dl_dpos0,
                          dl_dvel0};
    for (const void* q : ptrs)
        if (q && !aligned(q, 8)) return ORCA_ERR_INVALID_ARG;
    const orca_agents& A = s->p.agents;
    if (dl_dwaypoints && !A.route) return ORCA_ERR_INVALID_ARG;
    cudaStream_t stm = (cudaStream_t)stream;
    const size_t nb = (size_t)n * 8;
    if (dl_dwaypoints &&
        cudaMemsetAsync(dl_dwaypoints, 0, (size_t)A.n_routes * A.n_waypoints * 8, stm) !=
            cudaSuccess)
        return ORCA_ERR_CUDA;
    if (n == 0) return ORCA_OK;
    if (n_steps == 0) {
        if (dl_dpos0 && cudaMemcpyAsync(dl_dpos0, dl_dpos, nb, cudaMemcpyDeviceToDevice, stm))
            return ORCA_ERR_CUDA;
        if (dl_dvel0 && cudaMemsetAsync(dl_dvel0, 0, nb, stm)) return ORCA_ERR_CUDA;
        return ORCA_OK;
    }
    const int k = s->params.max_neighbors;
    const AdjLayout L = make_adj_layout((size_t)n, k, n_steps, ckpt_every);
    char* w = (char*)adj_ws;
    float2* bp[3] = {(float2*)(w + L.bar_p[0]), (float2*)(w + L.bar_p[1]),
                     (float2*)(w + L.bar_p[2])};
    float2* bv[3] = {(float2*)(w + L.bar_v[0]), (float2*)(w + L.bar_v[1]),
                     (float2*)(w + L.bar_v[2])};
    bool ok = cudaMemcpyAsync(bp[0], dl_dpos, nb, cudaMemcpyDeviceToDevice, stm) == cudaSuccess &&
              cudaMemsetAsync(bv[0], 0, nb, stm) == cudaSuccess &&
              cudaMemsetAsync(bp[1], 0, nb, stm) == cudaSuccess &&
              cudaMemsetAsync(bv[1], 0, nb, stm) == cudaSuccess;
    if (!ok) return ORCA_ERR_CUDA;

    // the replay pipeline: the scene's kernels over the replay state arrays
    Pipeline R = s->p;
    R.agents.pos = (float*)(w + L.rp_pos);
    R.agents.vel = (float*)(w + L.rp_vel);
    if (A.route) R.agents.wp_idx = (uint8_t*)(w + L.rp_wp);
    R.ev_begin = R.ev_end = R.bin_begin = R.bin_end = nullptr;
    R.counters = nullptr;
    R.graph = nullptr;
    ReplayDebug rec{DebugOut{}, (float2*)(w + L.r_pos), (float2*)(w + L.r_vel),
                    (int32_t*)(w + L.r_nbr), (uint32_t*)(w + L.r_act),
                    A.route ? (uint8_t*)(w + L.r_wp) : nullptr, (float2*)(w + L.r_vnew), n,
                    std::max(k, 1)};
    rec.base.k_stride = std::max(k, 1);
    const AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                      A.n_waypoints, A.wp_idx};
    int nx = 0, cu = 1, sp = 2;
    const int ab = 128, ag = (n + ab - 1) / ab;
    for (int seg = L.n_ck - 1; seg >= 0; --seg) {
        const int t0 = seg * ckpt_every;
        const int t1 = std::min(n_steps, t0 + ckpt_every);
        const size_t c = (size_t)seg * n;
        ok = cudaMemcpyAsync(R.agents.pos, (float2*)(w + L.ck_pos) + c, nb,
                             cudaMemcpyDeviceToDevice, stm) == cudaSuccess &&
             cudaMemcpyAsync(R.agents.vel, (float2*)(w + L.ck_vel) + c, nb,
                             cudaMemcpyDeviceToDevice, stm) == cudaSuccess &&
             (!A.route || cudaMemcpyAsync(R.agents.wp_idx, (uint8_t*)(w + L.ck_wp) + c, n,
                                          cudaMemcpyDeviceToDevice, stm) == cudaSuccess);
        if (!ok) return ORCA_ERR_CUDA;
        const float* vpd0 = vpref_delta ? vpref_delta + (size_t)t0 * n * 2 : nullptr;
        enqueue_steps(R, OneScene{R.one}, t1 - t0, vpd0, stm, rec, MODE_RECORD);
        for (int t = t1 - 1; t >= t0; --t) {
            const size_t o = (size_t)(t - t0) * n;
            const size_t tn = (size_t)t * n;
            // the kernel reads the scene's radius/type in caller order
            adjoint_kernel<<<ag, ab, 0, stm>>>(
                n, s->p.one, rec.r_pos + o, rec.r_vel + o, A.radius, A.type,
                rec.r_nbr + o * rec.k, rec.k, rec.r_act + o, rec.r_wp ? rec.r_wp + o : nullptr,
                rec.r_vnew + o, ain, vpref_delta ? (const float2*)vpref_delta + tn : nullptr,
                bp[nx], bv[nx], dl_dvel_traj ? (const float2*)dl_dvel_traj + tn : nullptr,
                bp[cu], bv[cu], bp[sp], bv[sp],
                dl_dvpref_delta ? (float2*)dl_dvpref_delta + tn : nullptr,
                (float2*)dl_dwaypoints, s->p.buf.err);
            const int old_nx = nx;
            nx = cu;
            cu = sp;
            sp = old_nx;
        }
    }
    if (dl_dpos0 &&
        cudaMemcpyAsync(dl_dpos0, bp[nx], nb, cudaMemcpyDeviceToDevice, stm) != cudaSuccess)
        return ORCA_ERR_CUDA;
    if (dl_dvel0 &&
        cudaMemcpyAsync(dl_dvel0, bv[nx], nb, cudaMemcpyDeviceToDevice, stm) != cudaSuccess)
        return ORCA_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

int orca_step_vjp(orca_scene* s, void* adj_ws, size_t adj_bytes, const float* pos,
                  const float* vel, const uint8_t* wp_idx, const float* vpref_delta,
                  const float* dl_dpos_next, const float* dl_dvel_next, float* dl_dpos,
                  float* dl_dvel, float* dl_dvpref_delta, float* dl_dwaypoints, void* stream) {
    int st = check_adjoint_args(s, 1, 1, adj_ws, adj_bytes, vpref_delta);
    if (st != ORCA_OK) return st;
    const int n = s->p.n;
    if (n == 0) return ORCA_OK;
    const orca_agents& A = s->p.agents;
    const void* ptrs[] = {pos, vel, dl_dpos_next, dl_dvel_next, dl_dpos, dl_dvel,
                          dl_dvpref_delta, dl_dwaypoints};
    for (const void* q : ptrs)
        if (q && !aligned(q, 8)) return ORCA_ERR_INVALID_ARG;
    if (!pos || !vel || !dl_dpos_next || !dl_dvel_next || !dl_dpos || !dl_dvel)
        return ORCA_ERR_INVALID_ARG;
    if ((A.route != nullptr) != (wp_idx != nullptr)) return ORCA_ERR_INVALID_ARG;
    if (dl_dwaypoints && !A.route) return ORCA_ERR_INVALID_ARG;
    cudaStream_t stm = (cudaStream_t)stream;
    const int k = s->params.max_neighbors;
    const AdjLayout L = make_adj_layout((size_t)n, k, 1, 1);
    char* w = (char*)adj_ws;
    const size_t nb = (size_t)n * 8;
    Pipeline R = s->p;
    R.agents.pos = (float*)(w + L.rp_pos);
    R.agents.vel = (float*)(w + L.rp_vel);
    if (A.route) R.agents.wp_idx = (uint8_t*)(w + L.rp_wp);
    R.ev_begin = R.ev_end = R.bin_begin = R.bin_end = nullptr;
    R.counters = nullptr;
    R.graph = nullptr;
    bool ok = cudaMemcpyAsync(R.agents.pos, pos, nb, cudaMemcpyDeviceToDevice, stm) ==
                  cudaSuccess &&
              cudaMemcpyAsync(R.agents.vel, vel, nb, cudaMemcpyDeviceToDevice, stm) ==
                  cudaSuccess &&
              (!A.route || cudaMemcpyAsync(R.agents.wp_idx, wp_idx, n,
                                           cudaMemcpyDeviceToDevice, stm) == cudaSuccess);
    float2* bp[3] = {(float2*)(w + L.bar_p[0]), (float2*)(w + L.bar_p[1]),
                     (float2*)(w + L.bar_p[2])};
    float2* bv[3] = {(float2*)(w + L.bar_v[0]), (float2*)(w + L.bar_v[1]),
                     (float2*)(w + L.bar_v[2])};
    ok = ok && cudaMemsetAsync(bp[1], 0, nb, stm) == cudaSuccess &&
         cudaMemsetAsync(bv[1], 0, nb, stm) == cudaSuccess;
    if (!ok) return ORCA_ERR_CUDA;
    ReplayDebug rec{DebugOut{}, (float2*)(w + L.r_pos), (float2*)(w + L.r_vel),
                    (int32_t*)(w + L.r_nbr), (uint32_t*)(w + L.r_act),
                    A.route ? (uint8_t*)(w + L.r_wp) : nullptr, (float2*)(w + L.r_vnew), n,
                    std::max(k, 1)};
    rec.base.k_stride = std::max(k, 1);
    enqueue_steps(R, OneScene{R.one}, 1, vpref_delta, stm, rec, MODE_RECORD);
    const AgentIn ain{(const float2*)A.goal, A.max_speed, A.route, (const float2*)A.waypoints,
                      A.n_waypoints, A.wp_idx};
    const int ab = 128, ag = (n + ab - 1) / ab;
    adjoint_kernel<<<ag, ab, 0, stm>>>(
        n, s->p.one, rec.r_pos, rec.r_vel, A.radius, A.type, rec.r_nbr, rec.k, rec.r_act,
        rec.r_wp, rec.r_vnew, ain, (const float2*)vpref_delta, (const float2*)dl_dpos_next,
        (const float2*)dl_dvel_next, nullptr, bp[1], bv[1], bp[2], bv[2],
        (float2*)dl_dvpref_delta, (float2*)dl_dwaypoints, s->p.buf.err);
    ok = cudaMemcpyAsync(dl_dpos, bp[1], nb, cudaMemcpyDeviceToDevice, stm) == cudaSuccess &&
         cudaMemcpyAsync(dl_dvel, bv[1], nb, cudaMemcpyDeviceToDevice, stm) == cudaSuccess;
    if (!ok) return ORCA_ERR_CUDA;
    return cuda_status(cudaGetLastError());
}

int orca_adjoint_launch_count(const orca_scene* s, int n_steps, int ckpt_every) {
    if (!s || n_steps < 0 || ckpt_every < 1) return -1;
    if (s->p.n == 0 || n_steps == 0) return 0;
    return 2 * n_steps + n_steps;   // replayed steps (binning + solve) + adjoint kernels
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
    bool kin = false;
    st = check_batch(params, n_scenes, offsets, agents->n_agents, &ncells, &kmax, &kin);
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
    init_pipeline(b->p, agents, (int)ncells, kcap_for(kmax, kin), params[0].block_size, n_scenes, lay,
                  workspace, kmax, params[0].debug_flags);
    bool ok = cudaMemset(b->p.buf.err, 0, 16) == cudaSuccess &&
              cudaMemset(b->p.buf.count, 0, (size_t)ncells * 4) == cudaSuccess &&
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
    b->p.dbg.cell = cell;
    b->p.dbg.nbr = nbr;
    b->p.dbg.cnt = cnt;
    b->p.dbg.flags = flags;
    b->p.dbg.tstar = tstar;
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

// Device address of the scratch area on the current device.  Outside a
// stream capture it is looked up on every call (after a reset of the
// device's primary context the module is loaded again, at a new address);
// while the stream is capturing the lookup, which may load the module, is
// not made and the last address found is returned (nullptr if none, or on
// failure).
char* noalloc_base(int dev, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return nullptr;
    if (cs == cudaStreamCaptureStatusNone) {
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
    cudaStream_t stm = (cudaStream_t)stream;
    char* w = noalloc_base(dev, stm);
    if (w == nullptr) return ORCA_ERR_CUDA;

    // a pipeline over the scratch area, held on the host stack
    Pipeline P;
    init_pipeline(P, agents, (int)ncells, kcap_for(params->max_neighbors, kinematic(params)),
                  params->block_size,
                  0, L, w, params->max_neighbors, params->debug_flags);
    P.one = scene_dev(params, 0, n, 0);
    st = prepare(P);
    if (st != ORCA_OK) return st;
    // the error word, the barrier words and the cell counts start at zero
    if (cudaMemsetAsync(P.buf.err, 0, 16, stm) != cudaSuccess ||
        cudaMemsetAsync(P.buf.count, 0, ncells * 4, stm) != cudaSuccess)
        return ORCA_ERR_CUDA;
    st = run_steps(P, n_steps, vpref_delta, stm);
    if (st != ORCA_OK) return st;
    if (synchronize) {
        if (cudaStreamSynchronize(stm) != cudaSuccess) return ORCA_ERR_CUDA;
        int h[4] = {0, 0, 0, 0};
        if (cudaMemcpy(h, P.buf.err, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return ORCA_ERR_CUDA;
        if (h[0] & ERR_BIT_NONFINITE) return ORCA_ERR_NONFINITE;
        if (h[0] & (ERR_BIT_TIMEOUT | ERR_BIT_STATE)) return ORCA_ERR_TIMEOUT;
        if (h[0] & ERR_BIT_CHECK) return ORCA_ERR_CHECK;
    }
    return ORCA_OK;
}
