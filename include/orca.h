/*
 * orca.h -- C ABI of liborca, the GB300 (sm_103a) implementation of the
 * per-time-step ORCA update for pedestrians and autonomous vehicles
 * (Charlton et al., "Simulating Crowds and Autonomous Vehicles").
 *
 * One step moves every agent once, all agents reading the state of step t
 * (paper Sec. 3, overview paragraph):
 *   1. bin agents into a uniform grid (Sec. 1, grid-partitioned messaging);
 *   2. each agent observes the radius, position and velocity of its k
 *      nearest neighbours within the neighbour distance (Sec. 3);
 *   3. one ORCA half-plane per neighbour, placed at v_opt + f_{A|B} u with
 *      the responsibility factor of the ordered pair of agent types
 *      (Sec. 3.1, Fig. 1c);
 *   4. the admissible velocity closest to the preferred velocity (Sec. 3,
 *      LP paragraphs); when no velocity is admissible, the velocity of least
 *      penetration (Sec. 3, infeasible-set paragraph);
 *   5. position update with the new velocity.
 *
 * Conventions shared by every entry point
 *   - All agent arrays are DEVICE memory owned by the caller, in the
 *     caller's agent order.  Arrays of 2D vectors are interleaved (x, y)
 *     float pairs ("float2"), 8-byte aligned.  The library keeps non-owning
 *     pointers to them; they must outlive the scene.
 *   - The workspace is device memory owned by the caller, at least
 *     orca_workspace_bytes() bytes, 256-byte aligned.  The library never
 *     allocates device memory in a step.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls that take a stream are asynchronous on it.
 *   - Every function returns an int status (ORCA_OK = 0).  Nothing throws.
 *     Argument errors are detected on the host before any launch.  Errors
 *     raised inside kernels (non-finite inputs, a bounded wait that gave up)
 *     are recorded in a device error word that orca_scene_sync_status()
 *     reads and clears.
 *   - Agent types: 0 = pedestrian, 1 = vehicle.  Both run the same code;
 *     only radius, max speed and the f table entries differ (Sec. 3.1).
 */
#ifndef ORCA_H_
#define ORCA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORCA_OK 0
#define ORCA_ERR_INVALID_ARG 1   /* bad pointer, size, parameter or alignment */
#define ORCA_ERR_CUDA 2          /* a CUDA runtime call or launch failed */
#define ORCA_ERR_TIMEOUT 3       /* a bounded device wait gave up */
#define ORCA_ERR_NONFINITE 4     /* a position or velocity was NaN/Inf */
#define ORCA_ERR_CAPACITY 5      /* k above ORCA_MAX_NEIGHBORS, grid too large */
#define ORCA_ERR_CHECK 6         /* a checked step found a broken invariant */

/* largest max_neighbors the kernels are compiled for */
#define ORCA_MAX_NEIGHBORS 32
/* largest number of grid cells of one scene, and of all scenes of a batch */
#define ORCA_MAX_CELLS (1 << 26)
/* largest number of scenes in one batch */
#define ORCA_MAX_SCENES (1 << 20)

/* debug_flags bits */
#define ORCA_DEBUG_NONE 0u
/* Solve the 2D LPs with the batch-LP load balancing the paper uses (Sec. 3,
   LP paragraphs: re-solves split into work units that every thread of a
   block shares) instead of one thread per LP.  Results agree to FP32
   rounding. */
#define ORCA_FLAG_LP_WORK_UNITS 2u
/* Test hook for failure detection: the first block of every binning kernel
   leaves without arriving at the grid barrier, so the other blocks' bounded
   waits run out.  The step then reports ORCA_ERR_TIMEOUT through
   orca_scene_sync_status() and leaves the caller's arrays untouched. */
#define ORCA_DEBUG_BARRIER_TIMEOUT 4u
/* Solve the velocity LPs by active-set enumeration instead (every candidate
   optimum of the 2D LP, then of the least-penetration LP, built and tested;
   O(k^3) per agent, loops fixed by k).  For comparison; results agree with
   the incremental LP to FP32 rounding.  One LP-scheme flag at a time. */
#define ORCA_FLAG_LP_ENUMERATION 8u
/* Solve the velocity LPs warp-cooperatively instead (a warp takes its 32
   agents' LPs one after another, its lanes splitting the constraints of each
   1D sub-problem, merged by warp min/max reductions).  For comparison;
   results agree with the incremental LP to FP32 rounding.  One LP-scheme
   flag at a time. */
#define ORCA_FLAG_LP_WARP 16u
/* Checked mode: every step certifies its own results on the device and
   records ORCA_ERR_CHECK (read by orca_scene_sync_status) when one fails:
   each neighbour list is sorted by (d^2, index), within R_n, without the
   agent itself; the agent lies in its slot's cell range; the new velocity is
   finite, inside the speed disc and, when the half-planes are feasible,
   inside every one of them (else its largest penetration is t*); the new
   position is finite (all up to FP32 rounding).  The results agree with the
   plain step to FP32 rounding; the checks cost time.  Not with an LP-scheme
   flag. */
#define ORCA_DEBUG_CHECKED 32u

/*
 * Global parameters of one scene (Sec. 3 and 3.1).
 *   neighbor_dist   R_n: agents closer than this are neighbour candidates
 *   time_horizon    tau: look-ahead of the velocity obstacles, seconds
 *   dt              step length, seconds
 *   max_neighbors   k: the k nearest candidates become constraints
 *                   (0 <= k <= ORCA_MAX_NEIGHBORS)
 *   f[a][b]         responsibility factor f_{A|B} of an agent of type a
 *                   avoiding one of type b (paper default 1/2, 1, 0, 1/2)
 *   cell_size       grid cell width (along x); any positive value gives
 *                   identical results (the neighbour search is exact), only
 *                   speed changes
 *   cell_height     grid cell height (along y), 0 = cell_size (square
 *                   cells); also a speed knob only.  Thin, wide cells suit
 *                   the search: it scans each grid row outward from the
 *                   agent's x, so the row height sets how far beyond the
 *                   k-th nearest neighbour it looks
 *   origin_x/y, grid_nx/ny   grid box; agents outside clamp to edge cells
 *   block_size      threads per block of the solve kernel (0 = 128)
 *   debug_flags     ORCA_DEBUG_NONE, or one of ORCA_FLAG_LP_WORK_UNITS,
 *                   ORCA_FLAG_LP_ENUMERATION, ORCA_FLAG_LP_WARP and
 *                   ORCA_DEBUG_CHECKED, and/or ORCA_DEBUG_BARRIER_TIMEOUT
 *   vehicle_turn_rate, vehicle_accel   kinematic limits of vehicles (type 1),
 *                   rad/s and m/s^2, 0 = off (default).  The paper names such
 *                   extra linear constraints as its extension for vehicles
 *                   (Sec. 5).  A vehicle moving at |v| >= 0.1 m/s gets two
 *                   half-planes through the origin that keep the new
 *                   velocity within +-turn_rate*dt of its heading (turn_rate*dt
 *                   < pi/2), and one half-plane v . h <= |v| + accel*dt along its
 *                   heading h; a slower vehicle gets only the latter, along
 *                   its preferred velocity.  They enter the same LP (and the
 *                   least-penetration fallback) after the ORCA half-planes.
 *                   Not differentiated: orca_rollout/orca_adjoint refuse them.
 */
typedef struct orca_params {
    float neighbor_dist;
    float time_horizon;
    float dt;
    int max_neighbors;
    float f[2][2];
    float cell_size;
    float origin_x;
    float origin_y;
    int grid_nx;
    int grid_ny;
    int block_size;
    unsigned debug_flags;
    float vehicle_turn_rate;
    float vehicle_accel;
    float cell_height;
} orca_params;

/*
 * Agents of one scene (Sec. 3: start, goal, radius, speeds).  Device
 * pointers, caller's order, N = n_agents.
 *   pos, vel        float2[N], read at step start, written at the end
 *   goal            float2[N]
 *   radius          float[N]  (> 0)
 *   max_speed       float[N]  (>= 0); the preferred velocity points at the
 *                   goal with this speed, capped so as not to overshoot
 *   type            uint8[N]  (0 pedestrian, 1 vehicle)
 *   route           int32[N] or NULL: row of `waypoints` the agent follows,
 *                   -1 = follow `goal`
 *   waypoints       float2[n_routes * n_waypoints] (row-major), or NULL
 *   wp_idx          uint8[N] current waypoint of each agent, read and
 *                   written by every step; required when route != NULL
 */
typedef struct orca_agents {
    int n_agents;
    float *pos;
    float *vel;
    const float *goal;
    const float *radius;
    const float *max_speed;
    const uint8_t *type;
    const int32_t *route;
    const float *waypoints;
    int n_routes;
    int n_waypoints;
    uint8_t *wp_idx;
} orca_agents;

typedef struct orca_scene orca_scene;
typedef struct orca_batch orca_batch;

/* Human-readable name of a status code (static string). */
const char *orca_status_string(int status);

/* ABI version of this header (increments on any signature change). */
int orca_abi_version(void);

/*
 * Workspace bytes a scene of n_agents agents with these parameters needs.
 * Returns ORCA_ERR_INVALID_ARG / ORCA_ERR_CAPACITY on bad parameters.
 */
int orca_workspace_bytes(const orca_params *params, int n_agents, size_t *out_bytes);

/*
 * Create a scene over caller-owned agent arrays and workspace.  Validates
 * everything that can be checked on the host (sizes, alignment, parameter
 * ranges), clears the workspace's error word and cell counts (synchronous
 * memsets) and launches no kernel.  *out receives a host object that
 * orca_scene_destroy() frees.
 */
int orca_scene_create(const orca_params *params, const orca_agents *agents,
                      void *workspace, size_t workspace_bytes, orca_scene **out);

/*
 * Optional per-agent diagnostics written by every following step (for the
 * last step of a call), caller's order; any pointer may be NULL:
 *   cell[N]        int32 grid cell id cy * nx + cx of the agent at step start
 *   nbr[N * k]     int32 neighbour indices in constraint order, -1 padded
 *   cnt[N]         int32 number of neighbours
 *   flags[N]       uint8 bit0 = half-planes infeasible (least-penetration
 *                  fallback taken), bit2 = overlaps a neighbour
 *   tstar[N]       float least penetration t* (only for bit0 agents, else 0)
 */
int orca_scene_set_debug(orca_scene *scene, int32_t *cell, int32_t *nbr,
                         int32_t *cnt, uint8_t *flags, float *tstar);

/*
 * Advance the scene n_steps synchronous steps (n_steps >= 0).  pos, vel and
 * wp_idx are updated in place.  vpref_delta is NULL or float2[n_steps * N]:
 * an offset added to the preferred velocity of agent i at step t at
 * vpref_delta[t * N + i] (the leaf of the adjoint).
 * Launches 2 kernels per step (binning, solve).  The last step of a call
 * also records, in the workspace, the cell order it used; the next call
 * bins its first step in that order, which only changes memory access
 * patterns.  Results never depend on it: the caller may change or reorder
 * any array between calls.
 */
int orca_step(orca_scene *scene, int n_steps, const float *vpref_delta, void *stream);

/*
 * Record two caller-created CUDA events (cudaEvent_t passed as void*, or
 * NULL to stop) on the step's stream right before and right after the solve
 * kernel of every following step, so a caller can time that kernel alone.
 * With n_steps > 1 the events bracket the last step's solve kernel.
 */
int orca_scene_set_solve_events(orca_scene *scene, void *begin, void *end);

/*
 * The same for the binning phase (cell keys, the scan of the cell counts and
 * the scatter into cell order, one cooperative kernel per step): begin and
 * end bracket that kernel.  On the first step of a call it also reads the
 * caller's arrays (later steps read the state the solve kernel wrote).
 */
int orca_scene_set_bin_events(orca_scene *scene, void *begin, void *end);

/*
 * Work tallies for FLOP accounting, or NULL to stop.  counters is device
 * memory, uint64[13], accumulated (never cleared) by every following step:
 *   [0] candidate key tests of the neighbour search
 *   [1] ORCA half-planes built
 *   [2] LP pair evaluations (a constraint tested against another inside a
 *       1D sub-problem or a bisector sub-problem)
 *   [3] agents whose half-planes were infeasible
 *   [4] agent updates
 *   [5] .. [8] thread clock cycles (clock64) summed over agents: neighbour
 *       search; preferred velocity and half-planes; velocity LP; the whole
 *       solve thread from the search on.  Shares of [8] give the phase split
 *       of the solve kernel (time a thread spends in each phase, stalls
 *       included).
 *   [9] candidates admitted to the sorted k-nearest list
 *   [10] list entries shifted by those admissions
 *   [11] grid rows scanned
 *   [12] iterations of the row scans' two-cursor loop (one candidate of
 *        each live cursor per iteration)
 * A scene with counters set runs a separate, slower kernel variant.
 */
int orca_scene_set_counters(orca_scene *scene, unsigned long long *counters);

/* Number of kernel launches one orca_step call of n_steps makes. */
int orca_step_launch_count(const orca_scene *scene, int n_steps);

/*
 * Record n_steps of orca_step (same arguments) into a CUDA graph kept by the
 * scene, replacing an earlier one.  Capture runs on a private stream and
 * executes nothing; orca_scene_graph_launch() then replays the recorded
 * launches on any stream with one call.  The graph holds the pointers of
 * this call (vpref_delta included), so each replay reads the same arrays.
 * Timing events and work counters are not recorded into the graph.
 */
int orca_scene_graph_capture(orca_scene *scene, int n_steps, const float *vpref_delta);

/* Replay the captured graph on `stream` (ORCA_ERR_INVALID_ARG if none). */
int orca_scene_graph_launch(orca_scene *scene, void *stream);

/*
 * Synchronise the device, then read and clear the scene's device error
 * word.  Returns ORCA_OK or the first recorded error status.
 * ORCA_ERR_TIMEOUT: a grid barrier of the binning kernel waited longer than
 * about half a second, or a later step found the cell counts such a step
 * left behind (or two calls ran on one scene at once); the results of those
 * steps are invalid.  This call also resets the barrier and the cell counts,
 * so the scene can step again.
 */
int orca_scene_sync_status(orca_scene *scene);

/* Free the host object and its graph (the caller's memory is untouched). */
void orca_scene_destroy(orca_scene *scene);

/*
 * Remove the agents that have arrived (Sec. 4: agents leave the scene at
 * their goal; a run ends when all have arrived).  Agent i has arrived when
 * |g - p|^2 <= r^2, evaluated in FP32 with each difference, product and the
 * sum rounded in that order, where p is its position now, r its radius and
 * g its goal, or, for an agent on a route, its last waypoint once that is
 * its current waypoint.  The kept agents move, in order, to the front of
 * EVERY agent array of the scene (pos, vel, goal, radius, max_speed, type,
 * route, wp_idx: the library writes the caller's arrays, including those the
 * struct declares const), and the scene's agent count becomes *n_kept.
 * kept_index (device int32[N], or NULL) receives the previous index of each
 * kept agent in its first *n_kept entries.  The call synchronises `stream`
 * (the host needs the new count) and drops a captured graph.  Scenes only.
 */
int orca_scene_remove_arrived(orca_scene *scene, int *n_kept, int32_t *kept_index,
                              void *stream);

/*
 * Record the velocity LP's active set of every agent in every following
 * step (NULL to stop): act[N] uint32, caller order, packed as
 *   bits 0-1   0 = projection of the preferred velocity onto the admissible
 *              set, 1 = least-penetration vertex, 2 = projection onto the
 *              mid-line of two exactly opposite half-planes (valley)
 *   bit 2      the speed circle |v| = max_speed is active
 *   bits 3-4   number of active half-planes (0-3)
 *   bits 8-12, 16-20, 24-28   their constraint indices (positions in nbr)
 *   bits 13/21/29   that half-plane was built on the cut-off circle
 *   bits 14/22/30   that half-plane belongs to an overlapping pair
 * The active set decides how the adjoint differentiates the LP.
 */
int orca_scene_set_debug_active(orca_scene *scene, uint32_t *act);

/*
 * ---------------------------------------------------------------------------
 * Differentiable rollouts.  The paper runs the ORCA update forward only; the
 * adjoint below is an addition of this library.  A rollout of n_steps steps
 * maps the preferred-velocity offsets delta[t][i] (the vpref_delta of
 * orca_step) and the waypoint table to the trajectory.  orca_adjoint
 * returns the gradient of a scalar loss L from dL/dpos after the last step
 * and dL/dvel after every step.  Each LP is differentiated through its
 * active half-planes and speed circle (implicit function on the active set);
 * neighbour sets, active sets, leg/cut-off choices and waypoint switches are
 * held fixed (no gradient through discrete choices).  Memory: the state is
 * checkpointed every ckpt_every steps and each segment is recomputed.
 * ---------------------------------------------------------------------------
 */

/* Bytes of the caller-owned adjoint workspace of a rollout. */
int orca_adjoint_workspace_bytes(const orca_scene *scene, int n_steps, int ckpt_every,
                                 size_t *out_bytes);

/*
 * orca_step over n_steps steps that also stores checkpoints in adj_ws
 * (device, 256-byte aligned, orca_adjoint_workspace_bytes bytes) and, when
 * vel_traj != NULL, writes the velocity after every step into vel_traj
 * (float2[n_steps * N], step-major, caller order).  The scene's pos, vel and
 * wp_idx advance as with orca_step.
 */
int orca_rollout(orca_scene *scene, int n_steps, int ckpt_every, const float *vpref_delta,
                 void *adj_ws, size_t adj_bytes, float *vel_traj, void *stream);

/*
 * Gradient of L through the last orca_rollout of this scene (same n_steps,
 * ckpt_every, vpref_delta and adj_ws, else ORCA_ERR_INVALID_ARG; the scene's
 * current state is not used).  Inputs (device, caller order):
 *   dl_dpos          float2[N]  dL/dpos after the last step (required)
 *   dl_dvel_traj     float2[n_steps * N] dL/d(velocity after step t), or NULL
 * Outputs (device, overwritten, any may be NULL):
 *   dl_dvpref_delta  float2[n_steps * N]
 *   dl_dwaypoints    float2[n_routes * n_waypoints] (scene needs routes)
 *   dl_dpos0, dl_dvel0  float2[N] gradient w.r.t. the rollout's start state
 * Neighbour cotangents are summed with atomics, so the last bits of the
 * result can vary between runs.
 */
int orca_adjoint(orca_scene *scene, int n_steps, int ckpt_every, const float *vpref_delta,
                 void *adj_ws, size_t adj_bytes, const float *dl_dpos,
                 const float *dl_dvel_traj, float *dl_dvpref_delta, float *dl_dwaypoints,
                 float *dl_dpos0, float *dl_dvel0, void *stream);

/*
 * Vector-Jacobian product of ONE step at a given state, for callers that
 * build their own reverse loops (or linearise along another trajectory).
 * Inputs (device, caller order): the state at the step's start pos, vel
 * (float2[N]) and wp_idx (uint8[N], required exactly when the scene has
 * routes), vpref_delta (float2[N] or NULL), and the cotangents of the state
 * after the step dl_dpos_next, dl_dvel_next (float2[N]; add any direct loss
 * term on the new velocity to dl_dvel_next).  Outputs: dl_dpos, dl_dvel
 * (float2[N], overwritten), dl_dvpref_delta (float2[N], overwritten, or
 * NULL) and dl_dwaypoints (ACCUMULATED into, or NULL).  adj_ws must hold
 * orca_adjoint_workspace_bytes(scene, 1, 1) bytes.  The scene's own state is
 * not touched.
 */
int orca_step_vjp(orca_scene *scene, void *adj_ws, size_t adj_bytes, const float *pos,
                  const float *vel, const uint8_t *wp_idx, const float *vpref_delta,
                  const float *dl_dpos_next, const float *dl_dvel_next, float *dl_dpos,
                  float *dl_dvel, float *dl_dvpref_delta, float *dl_dwaypoints, void *stream);

/* Kernel launches of one orca_adjoint call (replays and adjoint kernels). */
int orca_adjoint_launch_count(const orca_scene *scene, int n_steps, int ckpt_every);

/*
 * ---------------------------------------------------------------------------
 * Batches: many independent scenes of uneven size advanced by one launch per
 * phase of the step.  The paper simulates one scene at a time (Sec. 4);
 * every scene of a batch computes exactly what orca_step computes for it
 * alone, bit for bit.
 *
 * The agents of all scenes are concatenated, scene 0 first, into ONE
 * orca_agents (n_agents = total).  offsets is a HOST int array of
 * n_scenes + 1 entries: scene s owns agents [offsets[s], offsets[s + 1]),
 * offsets[0] = 0 and offsets[n_scenes] = n_agents.  params is a HOST array
 * of n_scenes orca_params (each scene has its own grid box, neighbour
 * distance, k, tau, dt and f table); block_size and debug_flags must be the
 * same in all of them.  route entries index rows of the one concatenated
 * waypoints array.  Agents of different scenes never interact.
 * ---------------------------------------------------------------------------
 */

/* Workspace bytes of a batch (the agent total is offsets[n_scenes]). */
int orca_batch_workspace_bytes(const orca_params *params, int n_scenes, const int *offsets,
                               size_t *out_bytes);

/*
 * Create a batch over caller-owned arrays and workspace.  Validates on the
 * host, then copies the scene table (n_scenes * 80 bytes) and the scene id
 * of every agent (4 bytes each) into the workspace with cudaMemcpy.
 */
int orca_batch_create(const orca_params *params, int n_scenes, const int *offsets,
                      const orca_agents *agents, void *workspace, size_t workspace_bytes,
                      orca_batch **out);

/* Per-agent diagnostics as orca_scene_set_debug; nbr rows have max_k
   entries (the largest k of the batch) and hold concatenated indices; cell
   ids are local to each scene's grid. */
int orca_batch_set_debug(orca_batch *batch, int32_t *cell, int32_t *nbr, int32_t *cnt,
                         uint8_t *flags, float *tstar);

/* Advance every scene n_steps steps; vpref_delta is NULL or
   float2[n_steps * n_agents] in the concatenated order. */
int orca_step_batched(orca_batch *batch, int n_steps, const float *vpref_delta, void *stream);

/* Number of kernel launches one orca_step_batched call of n_steps makes
   (independent of the number of scenes). */
int orca_batch_launch_count(const orca_batch *batch, int n_steps);

/* CUDA graph of n_steps batched steps, as orca_scene_graph_capture. */
int orca_batch_graph_capture(orca_batch *batch, int n_steps, const float *vpref_delta);
int orca_batch_graph_launch(orca_batch *batch, void *stream);

/* Device error word of the batch, as orca_scene_sync_status. */
int orca_batch_sync_status(orca_batch *batch);

/* Free the host object and its graph. */
void orca_batch_destroy(orca_batch *batch);

/*
 * Bytes of the library's built-in scratch area used by orca_step_noalloc()
 * (2 MiB, held in device memory by every GPU that loads the library, until
 * the process exits).
 */
#define ORCA_NOALLOC_SCRATCH_BYTES (2u << 20)

/*
 * orca_step for callers that cannot allocate device memory themselves: code
 * running inside another framework's memory pool, a plugin that may not
 * call cudaMalloc, or a real-time loop that must never allocate.  The paper
 * has no counterpart; it is a convenience of this library.
 *
 * Same inputs, outputs and step as creating a scene and calling orca_step,
 * but no scene object and no caller workspace: the scratch lives in a fixed
 * area inside the library.  This call performs no cudaMalloc, cudaFree or
 * any other allocation.
 *   - Size limit: the call is refused with ORCA_ERR_CAPACITY when
 *     orca_workspace_bytes(params, agents->n_agents) exceeds
 *     ORCA_NOALLOC_SCRATCH_BYTES (about 20,000 agents on a 256 x 256 grid).
 *   - Each call made outside a stream capture looks up the scratch area's
 *     device address on the current device (cudaGetSymbolAddress), so the
 *     next such call after a reset of the device's primary context
 *     (cudaDeviceReset) finds the area at its new address.  Make the first
 *     call on a device before any stream capture: while the stream is
 *     capturing the lookup is not made and the last address found on that
 *     device is used (ORCA_ERR_CUDA if there is none).
 *   - Every call, from every thread and stream, shares the one scratch area
 *     and it keeps the last call's contents; the call clears what has to
 *     start at zero.  Calls that overlap on the GPU race with each other:
 *     serialise them (one stream, or events between streams).
 *   - synchronize != 0 waits for the stream and also reports errors found
 *     on the device (ORCA_ERR_NONFINITE); with 0 the call is asynchronous
 *     and only host-side errors are returned.
 */
int orca_step_noalloc(const orca_params *params, const orca_agents *agents, int n_steps,
                      const float *vpref_delta, void *stream, int synchronize);

#ifdef __cplusplus
}
#endif

#endif /* ORCA_H_ */
