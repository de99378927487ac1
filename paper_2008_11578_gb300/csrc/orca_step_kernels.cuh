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
// One cooperative launch per step sorts the agents by cell (counting sort),
// then by x inside every cell:
//   A  (first step of a call only) cell key and counter slot of every agent,
//      from the caller's positions: one atomic increment of its cell count;
//   B  every block sums the counts of its contiguous range of cells;
//   C  every block adds up the sums of the blocks before it and scans its
//      range into cell starts, clearing the counts for the next step;
//   D  every agent's x key and pre-sort index go to slot
//      start[cell] + counter slot;
//   E  every slot counts the slots of its cell with a smaller (x key, slot)
//      and moves its agent's state there.
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
constexpr int kRankPerThread = 4;    // slots per thread and chunk in E
constexpr int kRankChunk = kBinThreads * kRankPerThread;
constexpr int kRankHalo = 128;       // keys staged on either side of a chunk in E
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
    uint4* __restrict__ xrank;         // cell order: x as an ordered key, pre-sort index, cell range
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
                    const int cx = cell_axis(p[u].x, sc.origin_x, sc.inv_cell_x, sc.nx);
                    const int cy = cell_axis(p[u].y, sc.origin_y, sc.inv_cell_y, sc.ny);
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

    // ---- D: cell order: every agent's x key, pre-sort index and cell range ----
    bool lost = false;
    const float2* __restrict__ spos = FIRST ? a.stage_pos : a.pos0;
    const float2* __restrict__ svel = FIRST ? a.stage_vel : a.vel0;
    const uint2* __restrict__ saux = FIRST ? a.stage_aux : a.aux0;
    for (int i0 = gt; i0 < a.n; i0 += kBinUnroll * gs) {
        uint32_t d[kBinUnroll], cb[kBinUnroll], ce[kBinUnroll];
        float x[kBinUnroll];
#pragma unroll
        for (int u = 0; u < kBinUnroll; ++u) {
            const int i = i0 + u * gs;
            d[u] = 0xffffffffu;
            if (i < a.n) {
                const uint32_t c = a.key[i];
                // staged by this thread in phase A on a first step
                x[u] = spos[i].x;
                if (c < (uint32_t)a.ncells) {
                    cb[u] = __ldcg(a.start + c);
                    ce[u] = __ldcg(a.start + c + 1);
                    d[u] = cb[u] + a.slot[i];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kBinUnroll; ++u) {
            const int i = i0 + u * gs;
            if (i < a.n) {
                if (d[u] < (uint32_t)a.n)
                    a.xrank[d[u]] = make_uint4(x_order_key(x[u]), (uint32_t)i, cb[u], ce[u]);
                else
                    lost = true;
            }
        }
    }
    if (lost) atomicOr(a.err, ERR_BIT_STATE);
    if (!grid_barrier(bar, a.err)) return;

    // ---- E: inside every cell, order by x (ties by slot); move the state ----
    // The rank of slot t among the slots of its cell by (x key, slot) is its
    // place in the cell, so each grid row becomes one run sorted by x, which
    // the neighbour search scans outward from an agent's x.  Every block
    // takes an equal contiguous range of slots, in chunks whose x keys it
    // stages in shared memory together with kRankHalo keys on either side: a
    // cell's slots are consecutive, so the rank loop reads global memory only
    // for a cell that reaches beyond the halo.  O(m) per agent for a cell of
    // m agents.
    __shared__ uint32_t skey[kRankChunk + 2 * kRankHalo];
    constexpr int kStage = (kRankChunk + 2 * kRankHalo + kBinThreads - 1) / kBinThreads;
    lost = false;
    const int blo = (int)((long long)a.n * blockIdx.x / gridDim.x);
    const int bhi = (int)((long long)a.n * (blockIdx.x + 1) / gridDim.x);
    for (int c0 = blo; c0 < bhi; c0 += kRankChunk) {   // block-uniform
        const int c1 = min(c0 + kRankChunk, bhi);
        const int s0 = max(c0 - kRankHalo, 0), s1 = min(c1 + kRankHalo, a.n);
        // every read of the chunk is issued before the first result is used:
        // the slots' records, the keys to stage, then the agents' state
        uint4 e[kRankPerThread];
#pragma unroll
        for (int u = 0; u < kRankPerThread; ++u) {
            const int t = c0 + (int)threadIdx.x + u * kBinThreads;
            e[u] = t < c1 ? __ldcg(a.xrank + t) : make_uint4(0u, 0xffffffffu, 0u, 0u);
        }
        uint32_t kv[kStage];
#pragma unroll
        for (int q = 0; q < kStage; ++q) {
            const int t = s0 + (int)threadIdx.x + q * kBinThreads;
            kv[q] = t < s1 ? __ldcg(&a.xrank[t].x) : 0u;
        }
        float2 sp[kRankPerThread], sv[kRankPerThread];
        uint2 sa[kRankPerThread];
#pragma unroll
        for (int u = 0; u < kRankPerThread; ++u) {
            const uint32_t i = e[u].y;
            if (i < (uint32_t)a.n) {
                sp[u] = spos[i];
                sv[u] = svel[i];
                sa[u] = saux[i];
            }
        }
#pragma unroll
        for (int q = 0; q < kStage; ++q) {
            const int t = s0 + (int)threadIdx.x + q * kBinThreads;
            if (t < s1) skey[t - s0] = kv[q];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kRankPerThread; ++u) {
            const uint32_t t = (uint32_t)(c0 + (int)threadIdx.x + u * kBinThreads);
            const uint32_t b = e[u].z, en = e[u].w, x = e[u].x;
            if (t >= (uint32_t)c1 || e[u].y >= (uint32_t)a.n || en > (uint32_t)a.n) {
                lost |= t < (uint32_t)c1;
                continue;
            }
            uint32_t r = 0u;
            for (uint32_t v = b; v < en; ++v) {
                const uint32_t xv = (v >= (uint32_t)s0 && v < (uint32_t)s1)
                                        ? skey[v - (uint32_t)s0] : __ldcg(&a.xrank[v].x);
                r += (xv < x || (xv == x && v < t)) ? 1u : 0u;
            }
            const uint32_t dst = b + r;
            if (dst >= en) {
                lost = true;
                continue;
            }
            a.pos1[dst] = sp[u];
            a.vel1[dst] = sv[u];
            a.aux1[dst] = sa[u];
        }
        __syncthreads();   // before the next chunk overwrites the staged keys
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
    // A checked step never hands its slot order to the next call: a slot that
    // fails a bounds check leaves its entry unwritten, so the next call bins
    // in the caller's order instead (the flag is cleared before any slot can
    // return early).
    if (MODE == MODE_CHECK && s_raw == 0 && out.hint_ok != nullptr) *out.hint_ok = 0;
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
    const int cx = cell_axis(p.x, sc.origin_x, sc.inv_cell_x, sc.nx);
    const int cy = cell_axis(p.y, sc.origin_y, sc.inv_cell_y, sc.ny);
    // the counting variant also records the thread's clock at the phase
    // boundaries (search, half-planes, LP, the rest)
    long long clk[4] = {0, 0, 0, 0};
    if (MODE == MODE_COUNT) clk[0] = clock64();

    // ---- k nearest by (d^2, index), exact search over the x-sorted grid rows ----
    // The list lives in the thread's line slots, sorted ascending by
    // (d^2, original index): slot m = (d^2, sorted slot j, original index).
    // An admitted candidate shifts only the entries behind it.
    const int k = sc.k;
    const float R2 = sc.R2;
    // d^2 of the k-th entry once the list is full; before, the largest float
    // below R_n^2, so one comparison admits a candidate (d^2 < R_n^2 and
    // below the k-th key) and stops a row cursor
    float thr_d = R2 > 0.0f ? __int_as_float(__float_as_int(R2) - 1) : -1.0f;
    // (d^2, original index) as one 64-bit key: d^2 >= 0, so its bits order
    // like the value, and the index breaks ties in the low word
    unsigned long long thr_key = ~0ull;
    int cnt = 0;
    int n_cand = 0, work = 0;
    int n_adm = 0, n_shift = 0, n_rows = 0, n_iter = 0;   // search tallies (MODE_COUNT)
    const uint32_t* __restrict__ cs = cstart + sc.cell_off;

    // candidate j at key distance d2: admitted when within R_n and its
    // (d^2, original index) key is below the k-th; the entries behind it
    // shift.  aj is the word of aux[j] that holds its original index (loaded
    // with the position, so an admission does not wait on a load).  The
    // agent itself is never a candidate: its own row is scanned from its
    // neighbouring slots.
    const uint32_t* __restrict__ aux_idx = reinterpret_cast<const uint32_t*>(aux) + 1;
    auto consider = [&](int j, float d2, uint32_t aj) {
        if (d2 <= thr_d) {
            const int oj = aux_orig(make_uint2(0u, aj));
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)oj;
            if (key < thr_key) {
                if (MODE == MODE_COUNT) ++n_adm;
                int at = min(cnt, k - 1);
                while (at > 0) {
                    if (MODE == MODE_COUNT) ++n_shift;
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

    if (k > 0 && isfinite(p.x) && isfinite(p.y)) {   // (a non-finite state is an error)
        // Every grid row is one run of slots sorted by x (the binning kernel
        // orders each cell by x, and cells of a row are consecutive in x).
        // A row is scanned outward from the agent's x with two cursors: the
        // right one stops at the first candidate right of the agent whose
        // fl(dx^2 + g2) exceeds the threshold (the k-th key, or the float
        // below R_n^2 while the list fills), the left one likewise on the
        // left, where g2 is the row's
        // lower bound of dy^2; every candidate farther along has a larger
        // dx^2, and d^2 = fl(dx^2 + dy^2) >= fl(dx^2 + g2) (rounding is
        // monotone), so none of them can enter the list.
        // Any start slot is valid (candidates on the wrong side of the agent
        // never stop a cursor); a good start only saves candidate tests.
        // Rows are visited nearest first (the agent's own row, then one row
        // on each side in turn, the nearer of the two first) and a side ends
        // at the first row whose y gap is beyond the k-th key (or R_n).
        const int nx = sc.nx, ny = sc.ny;
        const float ch = sc.cell_h, mg = sc.ring_delta * ch;
        const float pry = __fsub_rn(p.y, sc.origin_y);
        // lower bound of dy^2 for every agent binned into row ry (widened by
        // the cell-rounding margin, open toward the grid edge), with the
        // 1e-5 relative slack of the key comparison
        auto row_gap2 = [&](int ry) {
            const float by0 = ry == 0 ? -CUDART_INF_F : (float)ry * ch - mg;
            const float by1 = ry == ny - 1 ? CUDART_INF_F : (float)(ry + 1) * ch + mg;
            const float ey = fmaxf(fmaxf(by0 - pry, pry - by1), 0.0f);
            return ey * ey * 0.99999f;
        };
        // start slot of row ry: the agent's x interpolated inside the row's
        // cell of column cx (x-sorted, so agents spread roughly evenly)
        const float fx = fminf(fmaxf(__fmul_rn(__fsub_rn(p.x, sc.origin_x), sc.inv_cell_x) -
                                         (float)cx, 0.0f), 1.0f);
        // scan row ry leftward from jl and rightward from jr while
        // fl(dx^2 + g2) stays within the threshold; g2 is the row's lower
        // bound of dy^2 (0 for the own row)
        auto scan = [&](int jr, int jl, int ry, float g2) {
            const int rb = (int)__ldg(cs + ry * nx), re = (int)__ldg(cs + ry * nx + nx);
            bool ron = jr < re, lon = jl >= rb;
            if (MODE == MODE_CHECK && (rb < 0 || re > n || rb > re)) {
                atomicOr(err, ERR_BIT_CHECK);   // bounds check of the row
                ron = lon = false;
            }
            if (MODE == MODE_COUNT) ++n_rows;
            while (ron || lon) {
                if (MODE == MODE_COUNT) ++n_iter;
                float2 qr = make_float2(0.0f, 0.0f), ql = make_float2(0.0f, 0.0f);
                uint32_t ar = 0u, al = 0u;
                if (ron) {
                    qr = pos[jr];
                    ar = __ldg(aux_idx + 2 * jr);
                }
                if (lon) {
                    ql = pos[jl];
                    al = __ldg(aux_idx + 2 * jl);
                }
                const float lim = thr_d;
                if (ron) {
                    const float dx = __fsub_rn(qr.x, p.x);
                    const float dxx = __fmul_rn(dx, dx);
                    if (dx > 0.0f && __fadd_rn(dxx, g2) > lim) {
                        ron = false;
                    } else {
                        const float dy = __fsub_rn(qr.y, p.y);
                        ++n_cand;
                        consider(jr, __fadd_rn(dxx, __fmul_rn(dy, dy)), ar);
                        ron = ++jr < re;
                    }
                }
                if (lon) {
                    const float dx = __fsub_rn(ql.x, p.x);
                    const float dxx = __fmul_rn(dx, dx);
                    if (dx < 0.0f && __fadd_rn(dxx, g2) > lim) {
                        lon = false;
                    } else {
                        const float dy = __fsub_rn(ql.y, p.y);
                        ++n_cand;
                        consider(jl, __fadd_rn(dxx, __fmul_rn(dy, dy)), al);
                        lon = --jl >= rb;
                    }
                }
            }
        };
        // Rows in visiting order, through one call site of the row scan: the
        // agent's own row (ring 0) from its neighbouring slots, then ring by
        // ring the nearer of rows cy - m and cy + m first, each from the
        // agent's x interpolated inside the row's cell of column cx.  A side
        // ends at the grid edge or at the first row whose y gap is beyond the
        // threshold.
        bool up = true, down = true;   // rows cy + m / cy - m left to visit
        int m = 0, so = 2;             // ring, and the next of its two sides
        float gd = 0.0f, gu = 0.0f;    // the ring's y gaps below and above
        int first = 0;
        int ry = cy, jr = s + 1, jl = s - 1;
        float g2 = 0.0f;
        for (;;) {
            scan(jr, jl, ry, g2);
            bool found = false;
            while (!found && (up || down)) {
                if (so == 2) {
                    ++m;
                    so = 0;
                    gd = row_gap2(cy - m);
                    gu = row_gap2(cy + m);
                    first = gu < gd ? 1 : 0;
                }
                const int side = so ^ first;
                ++so;
                if (!(side == 0 ? down : up)) continue;
                ry = side == 0 ? cy - m : cy + m;
                g2 = side == 0 ? gd : gu;
                if (ry < 0 || ry >= ny || g2 > thr_d) {
                    if (side == 0) down = false;
                    else up = false;
                    continue;
                }
                found = true;
            }
            if (!found) break;
            const int c = ry * nx + cx;
            const int b = (int)__ldg(cs + c), e = (int)__ldg(cs + c + 1);
            jr = min(b + (int)(fx * (float)(e - b)), e);
            jl = jr - 1;
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
            if (j < 0 || j >= n) {   // no index read through an out-of-range slot
                bad = true;
                continue;
            }
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(e.x) << 32) | __float_as_uint(e.z);
            bad |= j == s || !(e.x < R2) || (m > 0 && key <= prev);
            prev = key;
        }
        const int own = cy * sc.nx + cx;
        bad |= !((int)__ldg(cs + own) <= s && s < (int)__ldg(cs + own + 1));
        if (bad) {
            atomicOr(err, ERR_BIT_CHECK);
            cnt = 0;   // no neighbour access through a list that failed its check
        }
    }

    if (MODE == MODE_COUNT) clk[1] = clock64();

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

    // ---- constraint order of the LP ----
    // Half-planes in decreasing penetration at the agent's current velocity:
    // the least-penetration optimum usually rests on the most violated ones,
    // so fewer of the later lines force a re-solve.  The two most violated
    // go first (swaps: slot 0 <-> sw0, then slot 1 <-> sw1); with at most 16
    // lines the rest follow in sorted order (insertion sort, ties keep their
    // order).  The LP's result does not depend on the order beyond rounding;
    // the recorded active set is mapped back to the neighbour order below,
    // through perm (slot -> neighbour index, 4 bits per slot) when sorted.
    int sw0 = 0, sw1 = 1;
    if (nlines > 1) {
        float pm0 = -CUDART_INF_F, pm1 = -CUDART_INF_F;
        int im0 = -1, im1 = -1;
        for (int i = 0; i < nlines; ++i) {
            const float pv = penetration(L[i * stride], v.x, v.y);
            if (pv > pm0) {
                pm1 = pm0;
                im1 = im0;
                pm0 = pv;
                im0 = i;
            } else if (pv > pm1) {
                pm1 = pv;
                im1 = i;
            }
        }
        if (im0 > 0) {
            const float4 a = L[0];
            L[0] = L[im0 * stride];
            L[im0 * stride] = a;
            sw0 = im0;
        }
        if (im1 >= 0 && nlines > 2) {
            const int b = im1 == 0 ? sw0 : im1;   // where the second line is now (>= 1)
            if (b > 1) {
                const float4 a = L[stride];
                L[stride] = L[b * stride];
                L[b * stride] = a;
                sw1 = b;
            }
        }
    }
    auto nib = [](uint64_t q, int i) { return (uint32_t)((q >> (4 * i)) & 15ull); };
    auto put = [](uint64_t q, int i, uint32_t x) {
        return (q & ~(15ull << (4 * i))) | ((uint64_t)x << (4 * i));
    };
    uint64_t perm = 0ull;
    if (MODE == MODE_RECORD && nlines <= 16) {
        perm = 0xFEDCBA9876543210ull;
        const uint32_t a0 = nib(perm, sw0);
        perm = put(put(perm, sw0, nib(perm, 0)), 0, a0);
        const uint32_t a1 = nib(perm, sw1);
        perm = put(put(perm, sw1, nib(perm, 1)), 1, a1);
    }
    if (nlines <= 16) {
        for (int m = 3; m < nlines; ++m) {
            const float4 e = L[m * stride];
            const float pe = penetration(e, v.x, v.y);
            const uint32_t em = MODE == MODE_RECORD ? nib(perm, m) : 0u;
            int at = m;
            while (at > 2) {
                const float4 f = L[(at - 1) * stride];
                if (!(penetration(f, v.x, v.y) < pe)) break;
                L[at * stride] = f;
                if (MODE == MODE_RECORD) perm = put(perm, at, nib(perm, at - 1));
                --at;
            }
            L[at * stride] = e;
            if (MODE == MODE_RECORD) perm = put(perm, at, em);
        }
    }

    if (MODE == MODE_COUNT) clk[2] = clock64();

    // ---- velocity LP, least-penetration fallback ----
    float vx, vy, tstar;
    uint32_t act = 0u;
    const int infeasible =
        WORK_UNITS ? solve_velocity_work_units(smem_lines, active ? nlines : 0, vmax, vpx, vpy,
                                               v.x, v.y, vx, vy, tstar, work)
        : LP == LP_WARP
            ? solve_velocity_warp(smem_lines, (int)(threadIdx.x & ~31u), active ? nlines : 0, vmax,
                                  vpx, vpy, vx, vy, tstar, work)
        : LP == LP_ENUMERATION
            ? solve_velocity_enumeration(L, stride, nlines, vmax, vpx, vpy, vx, vy, tstar, work)
            : solve_velocity(L, stride, nlines, vmax, vpx, vpy, v.x, v.y, vx, vy, tstar, work,
                             act);
    if (MODE == MODE_COUNT) clk[3] = clock64();
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
        if (s == 0 && MODE != MODE_CHECK) *out.hint_ok = 1;
    }
    if (out.key != nullptr) {
        // bin the new position for the next step (as the binning kernel's
        // cell-key phase does on a call's first step)
        const int ncx = cell_axis(pn.x, sc.origin_x, sc.inv_cell_x, sc.nx);
        const int ncy = cell_axis(pn.y, sc.origin_y, sc.inv_cell_y, sc.ny);
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
            // the LP's line index in the neighbour order
            int li = act_line(act, m);
            if (nlines <= 16) {
                li = (int)nib(perm, li);
            } else {   // undo the two swaps
                li = li == 1 ? sw1 : (li == sw1 ? 1 : li);
                li = li == 0 ? sw0 : (li == sw0 ? 0 : li);
            }
            act = (act & ~(31u << (8 + 8 * m))) | ((uint32_t)li << (8 + 8 * m));
            act |= ((capbits >> li) & 1u) << (13 + 8 * m);
            act |= ((ovbits >> li) & 1u) << (14 + 8 * m);
        }
        dbg.act[o] = act;
    }

    if (MODE == MODE_COUNT) {
        const long long end = clock64();
        unsigned long long c[kNumCounters] = {(unsigned long long)n_cand,
                                              (unsigned long long)cnt,
                                              (unsigned long long)work,
                                              (unsigned long long)(flags & 1), 1ull,
                                              (unsigned long long)(clk[1] - clk[0]),
                                              (unsigned long long)(clk[2] - clk[1]),
                                              (unsigned long long)(clk[3] - clk[2]),
                                              (unsigned long long)(end - clk[0]),
                                              (unsigned long long)n_adm,
                                              (unsigned long long)n_shift,
                                              (unsigned long long)n_rows,
                                              (unsigned long long)n_iter};
#pragma unroll
        for (int q = 0; q < kNumCounters; ++q) atomicAdd(counters + q, c[q]);
    }
    if (dbg.cell != nullptr) dbg.cell[o] = cy * sc.nx + cx;
    if (dbg.cnt != nullptr) dbg.cnt[o] = cnt;
    if (dbg.flags != nullptr) dbg.flags[o] = flags;
    if (dbg.tstar != nullptr) dbg.tstar[o] = tstar;
}

}  // namespace orca
