// orca_kernels.cuh -- kernels of one ORCA step over one or many scenes.
//
// Data layout (device, structure of arrays):
//   caller order     user pos/vel/goal/radius/max_speed/type/route/wp_idx
//   "state" order    pos0/vel0: output of the solve kernel, in the cell order
//                    of the step that produced it (on a call's first step
//                    the binning kernel stages the caller's state here)
//   sorted order     pos1/vel1 + aux (radius, type, original index): agents
//                    grouped by grid cell, cells in row-major order, scenes
//                    one after another, and inside a cell ordered by x, so
//                    that every grid row is one run sorted by x
// One step: the binning kernel (cell keys and per-cell slots on a call's
// first step -- later steps get them from the previous solve -- then the
// exclusive scan of the cell counts, the scatter into cell order and the
// ordering by x inside every cell) ->
// solve (one thread per agent: k-nearest search over the x-sorted grid rows,
// ORCA lines, LP, integrate) writing pos0/vel0 in sorted order, which becomes the state
// order of the next step; the last step of a call writes the caller's
// arrays instead.
#pragma once

#include <climits>

#include "orca_math.cuh"

namespace orca {

// per-scene constants
struct SceneDev {
    int agent_off;     // first sorted slot of the scene
    int n_agents;
    int cell_off;      // first global cell of the scene
    int nx, ny;
    float origin_x, origin_y;
    float inv_cell_x;  // fl32(1 / cell width)
    float inv_cell_y;  // fl32(1 / cell height)
    float cell_w, cell_h;
    float ring_delta;  // cell-rounding margin of the row bounds, in cells
    float R2;          // fl32(R_n * R_n)
    int k;
    float inv_tau, inv_dt, dt;
    float f00, f01, f10, f11;
    // vehicles' kinematic half-planes (off when both flags are false)
    bool kin_turn, kin_accel;
    float cos_turn, sin_turn;   // of the largest heading change per step
    float accel_dt;             // largest forward speed gain per step
};

// kinematic half-planes a vehicle can add to its LP
constexpr int kKinLines = 3;

struct OneScene {
    SceneDev s;
    __device__ __forceinline__ const SceneDev& get(int) const { return s; }
};

struct ManyScenes {
    const SceneDev* __restrict__ s;
    const int* __restrict__ sid;   // scene of every sorted slot (fixed)
    __device__ __forceinline__ const SceneDev& get(int i) const { return s[__ldg(sid + i)]; }
};

// caller-order per-agent inputs of the solve kernel
struct AgentIn {
    const float2* __restrict__ goal;
    const float* __restrict__ max_speed;
    const int32_t* __restrict__ route;     // may be null
    const float2* __restrict__ waypoints;
    int n_waypoints;
    uint8_t* __restrict__ wp_idx;          // may be null when route is null
};

// Per-agent constants of the sorted state, packed in 8 bytes so that the
// scatter moves one word for them: the radius, and the original index with
// the agent type (0 pedestrian, 1 vehicle) in its top bit.
__host__ __device__ __forceinline__ uint2 aux_pack(float r, int type, int orig) {
    union { float f; uint32_t u; } c;
    c.f = r;
    return make_uint2(c.u, (uint32_t)orig | (type ? 0x80000000u : 0u));
}
__device__ __forceinline__ float aux_rad(uint2 a) { return __uint_as_float(a.x); }
__device__ __forceinline__ int aux_orig(uint2 a) { return (int)(a.y & 0x7fffffffu); }
__device__ __forceinline__ int aux_type(uint2 a) { return (int)(a.y >> 31); }

// Where the solve kernel writes the new state.  Ordinary steps write pos/vel
// in sorted order (the next step's state order) and, when key is set, the
// next step's cell key and counter slot, so that step's binning skips its
// cell-key phase.  The last step of a call writes straight to the caller's
// arrays at the original index instead (caller_order), so no separate kernel
// has to copy the results back to the caller's order.  It also records the
// original index of every sorted slot (hint) and raises *hint_ok: the next
// call bins its agents in that order, which is nearly the new cell order.
struct StepOut {
    float2* pos;
    float2* vel;
    bool caller_order;
    uint32_t* key;
    uint32_t* slot;
    uint32_t* count;
    uint32_t* hint;
    int* hint_ok;
};

// Optional per-agent outputs of the solve kernel, caller order, any of them
// null.  The first group is diagnostics; the second records what the adjoint
// needs: the state at step start, the waypoint index before and after the
// advance, the new velocity and the LP's active set (solve MODE_RECORD only).
struct DebugOut {
    int32_t* cell;
    int32_t* nbr;
    int32_t* cnt;
    uint8_t* flags;
    float* tstar;
    int k_stride;
    float2* spos;
    float2* svel;
    uint8_t* swp;
    uint8_t* wp_used;
    float2* vnew;
    uint32_t* act;
};

// Variants of the solve kernel: plain, with work tallies, with the active set,
// and the checked step (plain plus on-device certificates of its results)
constexpr int MODE_PLAIN = 0, MODE_COUNT = 1, MODE_RECORD = 2, MODE_CHECK = 6;
// host-side choice of the plain variant with the paper's work-unit LP, or
// with active-set enumeration
constexpr int MODE_WORK_UNITS = 3, MODE_ENUMERATION = 4, MODE_WARP_LP = 5;
// the solve kernel's velocity-LP scheme
constexpr int LP_INCREMENTAL = 0, LP_WORK_UNITS = 1, LP_ENUMERATION = 2, LP_WARP = 3;

// Work tallies of the counting variant of the solve kernel:
// [0] candidate key tests, [1] ORCA lines built, [2] LP pair evaluations
// (one constraint against another inside a 1D or bisector sub-problem),
// [3] agents that took the least-penetration fallback, [4] agents;
// thread clock cycles (clock64) summed over agents: [5] neighbour search,
// [6] preferred velocity and half-planes, [7] velocity LP, [8] the whole
// thread from the search on (the rest is integration and output); neighbour
// search: [9] k-list admissions, [10] k-list entries shifted by them,
// [11] grid rows scanned, [12] iterations of the rows' two-cursor loop.
constexpr int kNumCounters = 13;

// Device error word bits.  ERR_BIT_STATE: the binning kernel found cell
// counts that do not sum to the agent count (reported as a timeout: the only
// in-library cause is a step cut short by a barrier that gave up).
// ERR_BIT_CHECK: a checked step (MODE_CHECK) found a broken invariant.
enum : int { ERR_BIT_NONFINITE = 1, ERR_BIT_TIMEOUT = 2, ERR_BIT_STATE = 4, ERR_BIT_CHECK = 8 };

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;   // cells per scan block

}  // namespace orca
