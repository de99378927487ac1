// orca_step_kernels.cuh -- device kernels of the ORCA step (sm_103a).
//
// The binning kernel is one cooperative launch per step (counting sort by
// cell in four phases); the solve kernel is one thread
// per agent in cell-sorted order, so the 32 agents of a warp come from a few
// neighbouring cells and read the same candidate cells through L1.
#pragma once

#include "orca_kernels.cuh"

namespace orca {

// ------------------------------------------------------------------ scan ----
// Exclusive scan of the cell counts into cell starts, three phases: per-block
// scan of kScanChunk cells (writing block totals), scan of the block totals
// (one block), and adding the block offsets.  Phase 1 also zeroes the counts
// for the next step.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* warp_sums,
                                                    uint32_t& total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t pre = wid ? warp_sums[wid - 1] : 0u;
    total = warp_sums[nw - 1];
    __syncthreads();
    return pre + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(uint32_t* __restrict__ count, uint32_t* __restrict__ start,
                   uint32_t* __restrict__ bsum, int ncells) {
    __shared__ uint32_t ws[32];
    static_assert(kScanItems == 16, "four 16-byte vectors per thread");
    const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
    const bool whole = base + kScanItems <= ncells;   // 64-byte aligned full chunk
    if (whole) {
        uint4* c4 = reinterpret_cast<uint4*>(count + base);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 x = c4[q];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) c4[q] = make_uint4(0u, 0u, 0u, 0u);
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const int c = base + j;
            v[j] = c < ncells ? count[c] : 0u;
            if (c < ncells) count[c] = 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) s += v[j];
    uint32_t total;
    uint32_t pre = block_excl_scan(s, ws, total);
    uint32_t o[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        o[j] = pre;
        pre += v[j];
    }
    if (whole) {
        uint4* s4 = reinterpret_cast<uint4*>(start + base);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            s4[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (base + j < ncells) start[base + j] = o[j];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_bsum_kernel(uint32_t* __restrict__ bsum, int nb) {
    __shared__ uint32_t ws[32];
    constexpr int kItems = 16;   // 1024 * 16 block totals = 2^26 cells
    int base = threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        v[j] = base + j < nb ? bsum[base + j] : 0u;
        s += v[j];
    }
    uint32_t total;
    uint32_t pre = block_excl_scan(s, ws, total);
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (base + j < nb) bsum[base + j] = pre;
        pre += v[j];
    }
    if (threadIdx.x == 0) bsum[nb] = total;
}

// one thread per four cells (16-byte aligned vectors; kScanChunk is a
// multiple of 4, so the four share one block offset)
__global__ void scan_add_kernel(uint32_t* __restrict__ start, const uint32_t* __restrict__ bsum,
                                int ncells, int nb) {
    const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (c + 4 <= ncells) {
        const uint32_t b = bsum[c / kScanChunk];
        uint4* s4 = reinterpret_cast<uint4*>(start + c);
        uint4 x = *s4;
        x.x += b;
        x.y += b;
        x.z += b;
        x.w += b;
        *s4 = x;
    } else {
        for (int q = c; q < ncells && q < c + 4; ++q) start[q] += bsum[q / kScanChunk];
    }
    if (c == 0) start[ncells] = bsum[nb];
}

// ------------------------------------------------------------- binning ----
// One cooperative launch per step sorts the agents by cell (counting sort):
//   A  (first step of a call only) cell key and counter slot of every agent,
//      from the caller's positions: one atomic increment of its cell count;
//   B  every block sums the counts of its contiguous range of cells;
//   C  every block adds up the sums of the blocks before it and scans its
//      range into cell starts, clearing the counts for the next step;
//   D  every agent's state moves to slot start[cell] + counter slot.
// Later steps skip A: the solve kernel bins the new positions as it writes
// them.  Grid barriers separate the phases.  The cooperative launch keeps
// every block resident; a barrier that waits longer than about half a second
// flags ERR_BIT_TIMEOUT and every block leaves the kernel.
// The cell counts are zero on entry: the workspace is cleared once when a
// scene is created, and phase C clears them again every step.  Should they
// not sum to the agent count (a step cut short by a barrier that gave up, or
// two calls on one workspace at once), the starts are clamped to the agent
// count, agents whose slot falls outside are not moved, and ERR_BIT_STATE is
// flagged: the step is wrong but stays inside its buffers.
constexpr int kBinThreads = 256;
constexpr int kBinUnroll = 4;        // agents in flight per thread in A and D
constexpr int kBinGridMax = 4096;    // launch blocks at most (block-sum slots)
constexpr unsigned kBarrierSpins = 1u << 22;

struct BinArgs {
    int n, ncells;
    const float2* __restrict__ upos;   // caller arrays, caller order (first step)
    const float2* __restrict__ uvel;
    const float* __restrict__ urad;
    const uint8_t* __restrict__ utype;
    const float2* __restrict__ pos0;   // the previous solve's output (later steps)
    const float2* __restrict__ vel0;
    const uint2* __restrict__ aux0;
    float2* __restrict__ stage_pos;    // first step: the caller's state in binning order
    float2* __restrict__ stage_vel;
    uint2* __restrict__ stage_aux;
    uint32_t* __restrict__ key;
    uint32_t* __restrict__ slot;
    uint32_t* __restrict__ count;
    uint32_t* __restrict__ start;
    uint32_t* __restrict__ bsum;
    float2* __restrict__ pos1;         // sorted state
    float2* __restrict__ vel1;
    uint2* __restrict__ aux1;
    int* __restrict__ err;             // [0] status bits, [1] hint valid; [2] arrivals, [3] generation
    const uint32_t* __restrict__ hint; // first step: original index per previous sorted slot
    int test_skip_arrival;             // ORCA_DEBUG_BARRIER_TIMEOUT
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier: bar[0] counts arrivals (the last block to arrive resets
// it), bar[1] is the generation that the waiting blocks watch.  Returns false
// in every thread of a block whose wait gave up.
__device__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned gen = ld_acquire_gpu(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicExch(bar + 1, gen + 1u);
        } else {
            unsigned it = 0;
            while (ld_acquire_gpu(bar + 1) == gen) {
                if (++it > kBarrierSpins) {
                    atomicOr(err, ERR_BIT_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <class SRC, bool FIRST>
__global__ void __launch_bounds__(kBinThreads, 4) bin_kernel(SRC src, BinArgs a) {
    __shared__ uint32_t ws[32];
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int gs = gridDim.x * blockDim.x;
    unsigned* bar = reinterpret_cast<unsigned*>(a.err + 2);
    if (a.test_skip_arrival && blockIdx.x == 0) {
        // failure-detection test: this block never arrives, the others' waits
        // give up (a one-block grid flags the timeout itself)
        if (threadIdx.x == 0) atomicOr(a.err, ERR_BIT_TIMEOUT);
        return;
    }

    // Order of the first step's agents: the previous call's sorted order
    // when its last step recorded it (the agents have barely moved, so
    // neighbouring threads share cells), else the caller's order.  Any
    // permutation gives the same result; indices are checked all the same.
    const uint32_t* __restrict__ hint = nullptr;
    if (FIRST && __ldcg(a.err + 1) != 0) hint = a.hint;
    const int lane = threadIdx.x & 31;

    // ---- A: cell key and slot in the uniform grid (Sec. 1, grid-partitioned messaging) ----
    // The caller's state is staged in this order (pos0, vel0, aux0), so the
    // scatter below reads it sequentially, as on later steps.
    if (FIRST) {
        bool lost = false, bad = false;
        // i0 - lane is the same in a whole warp, so every lane runs the loop
        // and the warp-wide votes below see all of them
        for (int i0 = gt; i0 - lane < a.n; i0 += kBinUnroll * gs) {
            int oi[kBinUnroll];
            float2 p[kBinUnroll], v[kBinUnroll];
            float rad[kBinUnroll];
            int typ[kBinUnroll];
#pragma unroll
            for (int u = 0; u < kBinUnroll; ++u) {
                const int i = i0 + u * gs;
                oi[u] = -1;
                if (i < a.n) {
                    const uint32_t o = hint ? __ldg(hint + i) : (uint32_t)i;
                    if (o < (uint32_t)a.n) {
                        oi[u] = (int)o;
                        p[u] = a.upos[o];
                        v[u] = a.uvel[o];
                        rad[u] = a.urad[o];
                        typ[u] = a.utype[o];
                    } else {
                        lost = true;
                    }
                }
            }
            uint32_t c[kBinUnroll], grp[kBinUnroll], base[kBinUnroll];
#pragma unroll
            for (int u = 0; u < kBinUnroll; ++u) {
                const bool valid = oi[u] >= 0;
                const unsigned vm = __ballot_sync(0xffffffffu, valid);
                c[u] = 0xffffffffu;
                grp[u] = 0u;
                if (valid) {
                    const SceneDev& sc = src.get(oi[u]);
                    const int cx = cell_axis(p[u].x, sc.origin_x, sc.inv_cell, sc.nx);
                    const int cy = cell_axis(p[u].y, sc.origin_y, sc.inv_cell, sc.ny);
                    c[u] = (uint32_t)(sc.cell_off + cy * sc.nx + cx);
                    grp[u] = __match_any_sync(vm, c[u]);
                }
            }
            // one counter increment per distinct cell of the warp; all of a
            // thread's increments are issued before any result is used
#pragma unroll
            for (int u = 0; u < kBinUnroll; ++u) {
                base[u] = 0u;
                if (grp[u] != 0u && lane == __ffs(grp[u]) - 1)
                    base[u] = atomicAdd(a.count + c[u], (uint32_t)__popc(grp[u]));
            }
#pragma unroll
            for (int u = 0; u < kBinUnroll; ++u) {
                const int i = i0 + u * gs;
                if (grp[u] != 0u) {
                    const uint32_t b0 = __shfl_sync(grp[u], base[u], __ffs(grp[u]) - 1);
                    a.key[i] = c[u];
                    a.slot[i] = b0 + (uint32_t)__popc(grp[u] & ((1u << lane) - 1u));
                    bad |= !(isfinite(p[u].x) && isfinite(p[u].y) && isfinite(v[u].x) &&
                             isfinite(v[u].y));
                    a.stage_pos[i] = p[u];
                    a.stage_vel[i] = v[u];
                    a.stage_aux[i] = aux_pack(rad[u], typ[u], oi[u]);
                } else if (i < a.n) {
                    a.key[i] = 0xffffffffu;   // out-of-range order entry: not moved
                }
            }
        }
        if (lost) atomicOr(a.err, ERR_BIT_STATE);
        if (bad) atomicOr(a.err, ERR_BIT_NONFINITE);
        if (!grid_barrier(bar, a.err)) return;
    }

    // ---- B: block sums over contiguous cell ranges (multiples of 4) ----
    const int chunk = (((a.ncells + (int)gridDim.x - 1) / (int)gridDim.x) + 3) & ~3;
    const int c_lo = min((int)blockIdx.x * chunk, a.ncells);
    const int c_hi = min(c_lo + chunk, a.ncells);
    {
        uint32_t sum = 0;
        for (int c = c_lo + 4 * threadIdx.x; c < c_hi; c += 4 * blockDim.x) {
            if (c + 4 <= c_hi) {
                const uint4 x = __ldcg(reinterpret_cast<const uint4*>(a.count + c));
                sum += x.x + x.y + x.z + x.w;
            } else {
                for (int q = c; q < c_hi; ++q) sum += __ldcg(a.count + q);
            }
        }
        uint32_t total;
        block_excl_scan(sum, ws, total);
        if (threadIdx.x == 0) a.bsum[blockIdx.x] = total;
    }
    if (!grid_barrier(bar, a.err)) return;

    // ---- C: cell starts (exclusive scan), counts cleared ----
    {
        uint32_t before = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) before += __ldcg(a.bsum + b);
        uint32_t carry;
        block_excl_scan(before, ws, carry);
        for (int c0 = c_lo; c0 < c_hi; c0 += 4 * blockDim.x) {
            const int c = c0 + 4 * threadIdx.x;
            const bool whole = c + 4 <= c_hi;
            uint32_t v[4] = {0u, 0u, 0u, 0u};
            if (whole) {
                uint4* p4 = reinterpret_cast<uint4*>(a.count + c);
                const uint4 x = __ldcg(p4);
                v[0] = x.x;
                v[1] = x.y;
                v[2] = x.z;
                v[3] = x.w;
                *p4 = make_uint4(0u, 0u, 0u, 0u);
            } else {
                for (int q = 0; q < 4; ++q)
                    if (c + q < c_hi) {
                        v[q] = __ldcg(a.count + c + q);
                        a.count[c + q] = 0u;
                    }
            }
            uint32_t tile;
            uint32_t o = carry + block_excl_scan(v[0] + v[1] + v[2] + v[3], ws, tile);
            uint32_t st[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                st[q] = min(o, (uint32_t)a.n);
                o += v[q];
            }
            if (whole) {
                *reinterpret_cast<uint4*>(a.start + c) = make_uint4(st[0], st[1], st[2], st[3]);
            } else {
                for (int q = 0; q < 4; ++q)
                    if (c + q < c_hi) a.start[c + q] = st[q];
            }
            carry += tile;
        }
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
            a.start[a.ncells] = min(carry, (uint32_t)a.n);
            if (carry != (uint32_t)a.n) atomicOr(a.err, ERR_BIT_STATE);
        }
    }
    if (!grid_barrier(bar, a.err)) return;

    // ---- D: scatter the state to sorted slots ----
    bool lost = false;
    const float2* __restrict__ spos = FIRST ? a.stage_pos : a.pos0;
    const float2* __restrict__ svel = FIRST ? a.stage_vel : a.vel0;
    const uint2* __restrict__ saux = FIRST ? a.stage_aux : a.aux0;
    for (int i0 = gt; i0 < a.n; i0 += kBinUnroll * gs) {
        uint32_t d[kBinUnroll];
#pragma unroll
        for (int u = 0; u < kBinUnroll; ++u) {
            const int i = i0 + u * gs;
            d[u] = 0xffffffffu;
            if (i < a.n) {
                const uint32_t c = a.key[i];
                if (c < (uint32_t)a.ncells) d[u] = __ldcg(a.start + c) + a.slot[i];
            }
        }
        float2 p[kBinUnroll], v[kBinUnroll];
        uint2 x[kBinUnroll];
#pragma unroll
        for (int u = 0; u < kBinUnroll; ++u) {
            const int i = i0 + u * gs;
            if (i < a.n && d[u] < (uint32_t)a.n) {
                // staged by this thread in phase A on a first step
                p[u] = spos[i];
                v[u] = svel[i];
                x[u] = saux[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kBinUnroll; ++u) {
            const int i = i0 + u * gs;
            if (i < a.n) {
                if (d[u] < (uint32_t)a.n) {
                    a.pos1[d[u]] = p[u];
                    a.vel1[d[u]] = v[u];
                    a.aux1[d[u]] = x[u];
                } else {
                    lost = true;
                }
            }
        }
    }
    if (lost) atomicOr(a.err, ERR_BIT_STATE);
}

// ------------------------------------------------------- removal at goal ----
// keep[i] = 0 when agent i has arrived: |g - p|^2 <= r^2 in FP32, each
// difference, product and the sum rounded in that order, where g is its goal,
// or for an agent on a route its last waypoint once that is the current one.
__global__ void arrived_kernel(int n, const float2* __restrict__ pos,
                               const float2* __restrict__ goal, const float* __restrict__ radius,
                               const int32_t* __restrict__ route,
                               const float2* __restrict__ waypoints, int n_waypoints,
                               const uint8_t* __restrict__ wp_idx, uint32_t* __restrict__ keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 p = pos[i];
    float2 g = goal[i];
    bool final_target = true;
    if (route != nullptr && route[i] >= 0) {
        const int wi = wp_idx[i];
        final_target = wi == n_waypoints - 1;
        g = waypoints[(size_t)route[i] * n_waypoints + wi];
    }
    const float dx = __fsub_rn(g.x, p.x), dy = __fsub_rn(g.y, p.y);
    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    const float r = radius[i];
    keep[i] = (final_target && d2 <= __fmul_rn(r, r)) ? 0u : 1u;
}

// Kept agent i moves to dest[i]: its fields are gathered into the step
// buffers (packed), then copied back to the front of the caller's arrays.
__global__ void compact_gather_kernel(int n, const uint32_t* __restrict__ dest,
                                      const float2* __restrict__ pos,
                                      const float2* __restrict__ vel,
                                      const float2* __restrict__ goal,
                                      const float* __restrict__ radius,
                                      const float* __restrict__ max_speed,
                                      const uint8_t* __restrict__ type,
                                      const int32_t* __restrict__ route,
                                      const uint8_t* __restrict__ wp_idx, float2* __restrict__ t_pos,
                                      float2* __restrict__ t_vel, float2* __restrict__ t_goal,
                                      float2* __restrict__ t_rv, uint2* __restrict__ t_misc,
                                      uint2* __restrict__ t_orig) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t d = dest[i];
    if (dest[i + 1] == d) return;   // not kept (exclusive scan did not advance)
    t_pos[d] = pos[i];
    t_vel[d] = vel[i];
    t_goal[d] = goal[i];
    t_rv[d] = make_float2(radius[i], max_speed[i]);
    t_misc[d] = make_uint2(route ? (uint32_t)route[i] : 0u,
                           (uint32_t)type[i] | ((wp_idx ? (uint32_t)wp_idx[i] : 0u) << 8));
    t_orig[d] = make_uint2((uint32_t)i, 0u);
}

__global__ void compact_scatter_kernel(int kept, const float2* __restrict__ t_pos,
                                       const float2* __restrict__ t_vel,
                                       const float2* __restrict__ t_goal,
                                       const float2* __restrict__ t_rv,
                                       const uint2* __restrict__ t_misc,
                                       const uint2* __restrict__ t_orig, float2* __restrict__ pos,
                                       float2* __restrict__ vel, float2* __restrict__ goal,
                                       float* __restrict__ radius, float* __restrict__ max_speed,
                                       uint8_t* __restrict__ type, int32_t* __restrict__ route,
                                       uint8_t* __restrict__ wp_idx,
                                       int32_t* __restrict__ kept_index) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= kept) return;
    pos[d] = t_pos[d];
    vel[d] = t_vel[d];
    goal[d] = t_goal[d];
    const float2 rv = t_rv[d];
    radius[d] = rv.x;
    max_speed[d] = rv.y;
    const uint2 m = t_misc[d];
    type[d] = (uint8_t)(m.y & 0xffu);
    if (route != nullptr) {
        route[d] = (int32_t)m.x;
        wp_idx[d] = (uint8_t)(m.y >> 8);
    }
    if (kept_index != nullptr) kept_index[d] = (int32_t)t_orig[d].x;
}

// ----------------------------------------------------------------- solve ----
// One thread per agent (sorted slot s).  The neighbour list and then the
// lines are kept in dynamic shared memory (k float4 slots per thread), slot i
// of thread t at [i * blockDim.x + t] (conflict-free float4).
// MODE_COUNT adds work tallies (algorithmic FLOP accounting) and
// MODE_RECORD the LP's active set; both are dead code in MODE_PLAIN.
// LP selects the velocity-LP scheme: the incremental per-thread LP, or for
// comparison only the paper's block-cooperative work units, the
// warp-cooperative LP (with both, every thread of the block takes part to the
// end of the LP, lanes past the last agent shadowing it and writing nothing)
// or active-set enumeration.
template <class SRC, int MODE, int LP = LP_INCREMENTAL>
__global__ void __launch_bounds__(128)
solve_kernel(int n, SRC src, const float2* __restrict__ pos, const float2* __restrict__ vel,
             const uint2* __restrict__ aux, const uint32_t* __restrict__ cstart,
             AgentIn ain, const float2* __restrict__ vpd, StepOut out, DebugOut dbg,
             unsigned long long* __restrict__ counters, int* __restrict__ err) {
    extern __shared__ float4 smem_lines[];
    // after a binning kernel that gave up or found inconsistent counts the
    // sorted state is not valid: leave everything as it is (the status call
    // reports the error)
    if (__ldcg(err) & (ERR_BIT_TIMEOUT | ERR_BIT_STATE)) return;
    const int stride = blockDim.x;
    float4* L = smem_lines + threadIdx.x;
    const int s_raw = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr bool WORK_UNITS = LP == LP_WORK_UNITS;
    constexpr bool ALL_LANES = WORK_UNITS || LP == LP_WARP;
    if (!ALL_LANES && s_raw >= n) return;
    const bool active = s_raw < n;
    const int s = active ? s_raw : n - 1;
    const SceneDev& sc = src.get(s);
    const float2 p = pos[s];
    const float2 v = vel[s];
    const uint2 as = aux[s];
    const float r = aux_rad(as);
    const int ta = aux_type(as);
    const int o = aux_orig(as);
    if (MODE == MODE_CHECK && o >= n) {   // bounds check of the original index
        atomicOr(err, ERR_BIT_CHECK);
        return;
    }
    const int cx = cell_axis(p.x, sc.origin_x, sc.inv_cell, sc.nx);
    const int cy = cell_axis(p.y, sc.origin_y, sc.inv_cell, sc.ny);

    // ---- k nearest by (d^2, index), exact ring search over the grid ----
    // The list lives in the thread's line slots, sorted ascending by
    // (d^2, original index): slot m = (d^2, sorted slot j, original index).
    // An admitted candidate shifts only the entries behind it.
    const int k = sc.k;
    float thr_d = CUDART_INF_F;   // key of the k-th entry once the list is full
    // (d^2, original index) as one 64-bit key: d^2 >= 0, so its bits order
    // like the value, and the index breaks ties in the low word
    unsigned long long thr_key = ~0ull;
    int cnt = 0;
    int n_cand = 0, work = 0;
    const float R2 = sc.R2;
    const uint32_t* __restrict__ cs = cstart + sc.cell_off;

    // candidate j at key distance d2: admitted when within R_n and its
    // (d^2, original index) key is below the k-th; the entries behind it shift
    auto consider = [&](int j, float d2) {
        if (d2 < R2 && d2 <= thr_d && j != s) {
            const int oj = aux_orig(__ldg(aux + j));
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)oj;
            if (key < thr_key) {
                int at = min(cnt, k - 1);
                while (at > 0) {
                    const float4 e = L[(at - 1) * stride];
                    const unsigned long long ek =
                        ((unsigned long long)__float_as_uint(e.x) << 32) | __float_as_uint(e.z);
                    if (ek < key) break;
                    L[at * stride] = e;
                    --at;
                }
                L[at * stride] = make_float4(d2, __int_as_float(j), __int_as_float(oj), 0.0f);
                cnt = min(cnt + 1, k);
                if (cnt == k) {
                    const float4 e = L[(k - 1) * stride];
                    thr_d = e.x;
                    thr_key =
                        ((unsigned long long)__float_as_uint(e.x) << 32) | __float_as_uint(e.z);
                }
            }
        }
    };

    if (k > 0) {
        const int nx = sc.nx, ny = sc.ny;
        const int mmax = max(max(cx, nx - 1 - cx), max(cy, ny - 1 - cy));
        const float prx = __fsub_rn(p.x, sc.origin_x), pry = __fsub_rn(p.y, sc.origin_y);
        for (int m = 0; m <= mmax; ++m) {
            // ring m = row cy-m, row cy+m (each one contiguous run of cells)
            // and the two side cells of every row strictly between them
            const int x0 = max(cx - m, 0), x1 = min(cx + m, nx - 1);
            const int ylo = cy - m, yhi = cy + m;
            const int ya = max(ylo + 1, 0), yb = min(yhi - 1, ny - 1);
            const int nr = (m == 0) ? 1 : 2 + 2 * max(0, yb - ya + 1);
            for (int rr = 0; rr < nr; ++rr) {
                int ry, rx0, rx1;
                if (rr < 2) {
                    ry = rr ? yhi : ylo;
                    if (ry < 0 || ry >= ny) continue;
                    rx0 = x0;
                    rx1 = x1;
                } else {
                    const int q = rr - 2;
                    ry = ya + (q >> 1);
                    rx0 = rx1 = (q & 1) ? cx + m : cx - m;
                    if (rx0 < 0 || rx0 >= nx) continue;
                }
                if (m > 0) {
                    // No agent of cells rx0..rx1 of row ry can enter the list
                    // when the run's box is beyond the k-th key (or R_n).  The
                    // box is taken relative to the grid origin, like the cell
                    // assignment, widened by the same cell-rounding margin as
                    // the ring bound, and unbounded toward the grid edge (agents
                    // outside the box are clamped into edge cells).
                    const float cz = sc.cell_size, mg = sc.ring_delta * cz;
                    const float bx0 = rx0 == 0 ? -CUDART_INF_F : (float)rx0 * cz - mg;
                    const float bx1 = rx1 == nx - 1 ? CUDART_INF_F : (float)(rx1 + 1) * cz + mg;
                    const float by0 = ry == 0 ? -CUDART_INF_F : (float)ry * cz - mg;
                    const float by1 = ry == ny - 1 ? CUDART_INF_F : (float)(ry + 1) * cz + mg;
                    const float ex = fmaxf(fmaxf(bx0 - prx, prx - bx1), 0.0f);
                    const float ey = fmaxf(fmaxf(by0 - pry, pry - by1), 0.0f);
                    const float bd2 = (ex * ex + ey * ey) * 0.99999f;
                    if (bd2 >= R2 || (cnt >= k && bd2 > thr_d)) continue;
                }
                const int c0 = ry * nx + rx0, c1 = ry * nx + rx1;
                const int jb = (int)__ldg(cs + c0), je = (int)__ldg(cs + c1 + 1);
                if (MODE == MODE_CHECK && !(0 <= jb && jb <= je && je <= n)) {
                    atomicOr(err, ERR_BIT_CHECK);   // bounds check of the run
                    continue;
                }
                n_cand += je - jb;
                // two candidates per iteration: both position loads in flight
                for (int j = jb; j < je; j += 2) {
                    const int j1 = min(j + 1, je - 1);
                    const float2 q0 = pos[j], q1 = pos[j1];
                    const float d0 = key_d2(p.x, p.y, q0.x, q0.y);
                    const float d1 = j + 1 < je ? key_d2(p.x, p.y, q1.x, q1.y) : CUDART_INF_F;
                    consider(j, d0);
                    consider(j + 1, d1);
                }
            }
            // every agent outside rings 0..m is farther than (m - delta) cells
            const float D = ((float)m - sc.ring_delta) * sc.cell_size;
            if (D > 0.0f) {
                const float D2 = D * D * 0.99999f;
                if (D2 >= R2) break;
                if (cnt >= k && thr_d < D2) break;
            }
        }
    }

    if (MODE == MODE_CHECK && active) {
        // the k-list: sorted by (d^2, original index), within R_n, no self;
        // and this agent inside the slot range of its own cell
        bool bad = cnt > k;
        unsigned long long prev = 0ull;
        for (int m = 0; m < cnt; ++m) {
            const float4 e = L[m * stride];
            const int j = __float_as_int(e.y);
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(e.x) << 32) | __float_as_uint(e.z);
            bad |= j < 0 || j >= n || j == s || !(e.x < R2) || (m > 0 && key <= prev);
            prev = key;
        }
        const int own = cy * sc.nx + cx;
        bad |= !((int)__ldg(cs + own) <= s && s < (int)__ldg(cs + own + 1));
        if (bad) {
            atomicOr(err, ERR_BIT_CHECK);
            cnt = 0;   // no neighbour access through a list that failed its check
        }
    }

    // ---- preferred velocity toward the goal or the current waypoint ----
    float2 g = ain.goal[o];
    const float vmax = ain.max_speed[o];
    if (ain.route != nullptr) {
        const int rt = ain.route[o];
        if (rt >= 0) {
            int wi = ain.wp_idx[o];
            if (MODE == MODE_CHECK && wi >= ain.n_waypoints) {   // bounds check
                atomicOr(err, ERR_BIT_CHECK);
                wi = ain.n_waypoints - 1;
            }
            if (active && dbg.swp != nullptr) dbg.swp[o] = (uint8_t)wi;
            const float2* W = ain.waypoints + (size_t)rt * ain.n_waypoints;
            float2 w = W[wi];
            float wdx = __fsub_rn(w.x, p.x), wdy = __fsub_rn(w.y, p.y);
            float w2 = __fadd_rn(__fmul_rn(wdx, wdx), __fmul_rn(wdy, wdy));
            if (wi < ain.n_waypoints - 1 && w2 <= __fmul_rn(r, r)) ++wi;
            g = W[wi];
            if (active) {
                ain.wp_idx[o] = (uint8_t)wi;
                if (dbg.wp_used != nullptr) dbg.wp_used[o] = (uint8_t)wi;
            }
        }
    }
    float vpx = 0.0f, vpy = 0.0f;
    {
        float gx = g.x - p.x, gy = g.y - p.y;
        float gl = sqrtf(gx * gx + gy * gy);
        if (gl > 0.0f) {
            float f = fminf(vmax / gl, sc.inv_dt);
            vpx = gx * f;
            vpy = gy * f;
        }
        if (vpd != nullptr) {
            float2 dl = vpd[o];
            vpx += dl.x;
            vpy += dl.y;
        }
    }

    // ---- one ORCA half-plane per neighbour (Sec. 3.1) ----
    // Constraint m is the m-th nearest; its line replaces its list entry.
    if (active && dbg.nbr != nullptr) {
        int32_t* nb = dbg.nbr + (size_t)o * dbg.k_stride;
        for (int m = 0; m < dbg.k_stride; ++m)
            nb[m] = m < cnt ? __float_as_int(L[m * stride].z) : -1;
    }
    bool any_overlap = false;
    uint32_t capbits = 0u, ovbits = 0u;   // per-line construction (MODE_RECORD)
    for (int i = 0; i < cnt; ++i) {
        const float4 e = L[i * stride];
        const int j = __float_as_int(e.y);
        const float2 pj = pos[j], vj = vel[j];
        const uint2 aj = aux[j];
        const float rj = aux_rad(aj);
        const int tb = aux_type(aj);
        const float rs = __fadd_rn(r, rj);
        const bool ov = e.x <= __fmul_rn(rs, rs);
        any_overlap |= ov;
        const float f = tb ? (ta ? sc.f11 : sc.f01) : (ta ? sc.f10 : sc.f00);
        bool cap;
        L[i * stride] = orca_line(p.x, p.y, v.x, v.y, r, pj.x, pj.y, vj.x, vj.y, rj, f,
                                  sc.inv_tau, sc.inv_dt, ov, cap);
        if (MODE == MODE_RECORD) {
            ovbits |= (ov ? 1u : 0u) << i;
            capbits |= (cap ? 1u : 0u) << i;
        }
    }

    // ---- vehicles' kinematic half-planes (off unless the scene sets limits) ----
    int nlines = cnt;
    if (ta != 0 && (sc.kin_turn || sc.kin_accel)) {
        const float sp2 = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
        const bool moving = sp2 >= 0.01f;   // |v| >= 0.1 m/s: the heading is defined
        float hx = 0.0f, hy = 0.0f, sp = 0.0f;
        if (moving) {
            sp = sqrtf(sp2);
            hx = v.x / sp;
            hy = v.y / sp;
        } else {
            const float pl = sqrtf(vpx * vpx + vpy * vpy);
            if (pl > 0.0f) {
                hx = vpx / pl;
                hy = vpy / pl;
            }
        }
        if (moving && sc.kin_turn) {
            // the heading may turn by at most +-theta: the wedge between the
            // rays R(+theta) h and R(-theta) h, two half-planes through 0
            const float lx = sc.cos_turn * hx - sc.sin_turn * hy;
            const float ly = sc.sin_turn * hx + sc.cos_turn * hy;
            L[nlines++ * stride] = make_float4(0.0f, 0.0f, -lx, -ly);
            const float rx = sc.cos_turn * hx + sc.sin_turn * hy;
            const float ry = -sc.sin_turn * hx + sc.cos_turn * hy;
            L[nlines++ * stride] = make_float4(0.0f, 0.0f, rx, ry);
        }
        if (sc.kin_accel && (hx != 0.0f || hy != 0.0f)) {
            // forward speed gain at most accel * dt: v . h <= |v| + accel dt
            const float smax = sp + sc.accel_dt;
            L[nlines++ * stride] = make_float4(smax * hx, smax * hy, -hy, hx);
        }
    }

    // ---- velocity LP, least-penetration fallback ----
    float vx, vy, tstar;
    uint32_t act = 0u;
    const int infeasible =
        WORK_UNITS ? solve_velocity_work_units(smem_lines, active ? nlines : 0, vmax, vpx, vpy,
                                               vx, vy, tstar, work)
        : LP == LP_WARP
            ? solve_velocity_warp(smem_lines, (int)(threadIdx.x & ~31u), active ? nlines : 0, vmax,
                                  vpx, vpy, vx, vy, tstar, work)
        : LP == LP_ENUMERATION
            ? solve_velocity_enumeration(L, stride, nlines, vmax, vpx, vpy, vx, vy, tstar, work)
            : solve_velocity(L, stride, nlines, vmax, vpx, vpy, vx, vy, tstar, work, act);
    if (!active) return;
    const uint8_t flags = (uint8_t)(infeasible | (any_overlap ? 4 : 0));
    if (MODE == MODE_CHECK) {
        // the LP result: finite, inside the speed disc, and inside every
        // half-plane (feasible) or at the least penetration t* (fallback),
        // each up to rounding at the scale of the line's data
        bool bad = !(isfinite(vx) && isfinite(vy)) ||
                   vx * vx + vy * vy > vmax * vmax * (1.0f + 1e-5f) + 1e-5f;
        float tmax = -CUDART_INF_F;
        for (int i = 0; i < nlines; ++i) {
            const float4 li = L[i * stride];
            const float pi = penetration(li, vx, vy);
            const float tol = 1e-4f * (1.0f + vmax + fabsf(li.x) + fabsf(li.y));
            if (!infeasible) bad |= pi > tol;
            tmax = fmaxf(tmax, pi - tol);
        }
        if (infeasible) bad |= tstar < -1e-4f * (1.0f + vmax) || tmax > tstar;
        if (bad) atomicOr(err, ERR_BIT_CHECK);
    }

    // ---- integrate ----
    const float2 pn = make_float2(__fadd_rn(p.x, __fmul_rn(sc.dt, vx)),
                                  __fadd_rn(p.y, __fmul_rn(sc.dt, vy)));
    if (MODE == MODE_CHECK && !(isfinite(pn.x) && isfinite(pn.y))) atomicOr(err, ERR_BIT_CHECK);
    const int w = out.caller_order ? o : s;
    out.vel[w] = make_float2(vx, vy);
    out.pos[w] = pn;
    if (out.hint != nullptr) {
        out.hint[s] = (uint32_t)o;
        if (s == 0) *out.hint_ok = 1;
    }
    if (out.key != nullptr) {
        // bin the new position for the next step (as the binning kernel's
        // cell-key phase does on a call's first step)
        const int ncx = cell_axis(pn.x, sc.origin_x, sc.inv_cell, sc.nx);
        const int ncy = cell_axis(pn.y, sc.origin_y, sc.inv_cell, sc.ny);
        const uint32_t c = (uint32_t)(sc.cell_off + ncy * sc.nx + ncx);
        out.key[s] = c;
        out.slot[s] = atomicAdd(out.count + c, 1u);
    }

    if (dbg.spos != nullptr) dbg.spos[o] = p;
    if (dbg.svel != nullptr) dbg.svel[o] = v;
    if (dbg.vnew != nullptr) dbg.vnew[o] = make_float2(vx, vy);
    if (MODE == MODE_RECORD && dbg.act != nullptr) {
        const int nl = act_nlines(act);
        for (int m = 0; m < nl; ++m) {
            const int li = act_line(act, m);
            act |= ((capbits >> li) & 1u) << (13 + 8 * m);
            act |= ((ovbits >> li) & 1u) << (14 + 8 * m);
        }
        dbg.act[o] = act;
    }

    if (MODE == MODE_COUNT) {
        unsigned long long c[kNumCounters] = {(unsigned long long)n_cand,
                                              (unsigned long long)cnt,
                                              (unsigned long long)work,
                                              (unsigned long long)(flags & 1), 1ull};
#pragma unroll
        for (int q = 0; q < kNumCounters; ++q) atomicAdd(counters + q, c[q]);
    }
    if (dbg.cell != nullptr) dbg.cell[o] = cy * sc.nx + cx;
    if (dbg.cnt != nullptr) dbg.cnt[o] = cnt;
    if (dbg.flags != nullptr) dbg.flags[o] = flags;
    if (dbg.tstar != nullptr) dbg.tstar[o] = tstar;
}

}  // namespace orca
