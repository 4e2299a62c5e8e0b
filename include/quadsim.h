/*
 * quadsim.h -- C ABI of the batched quadrotor simulator (libquadsim.so).
 *
 * One step of a swarm of N nonlinear quadrotors, computed on the GPU, one
 * thread per agent:
 *   - rigid-body dynamics, Eq. (qd1)-(qd4) of arXiv 2308.12698, Sec. III-B:
 *       p' = v,  v' = R(q)[0,0,f_c]/m - (c_d/m) v + [0,0,-g],
 *       q' = 1/2 q o [0, omega],  omega' = I^-1(-omega x I omega + tau);
 *   - rotor thrust/torque, Eq. (2): f_i = kt Omega_i^2, tau_i = kq Omega_i^2;
 *   - allocation, Eq. (3): [f_c, tau_x, tau_y, tau_z] = G [f_1..f_4], with G
 *     rows (1,1,1,1), L sin(a)(1,-1,-1,1), L cos(a)(-1,-1,1,1), kq/kt(1,-1,1,-1);
 *   - first-order rotor lag Omega' = (Omega_cmd - Omega)/tau_m;
 *   - classical RK4 with the command held over the four stages (Sec. III-B,
 *     last paragraph);
 *   - closed loop: a cascaded controller evaluated once per step (position PD
 *     with per-axis acceleration clamp and gravity feed-forward -> desired
 *     attitude from thrust direction and heading -> attitude P on the error
 *     quaternion -> body-rate P scaled by the axis torque limit -> G^-1 ->
 *     per-rotor clamp of Omega^2 to [0, omega_max^2] -> sqrt).  The paper
 *     names only the inner body-rate loop (Sec. III-B); the cascade above is
 *     this library's definition of it;
 *   - closed loop with a PID body-rate loop (the paper's "PID body rate
 *     controller", Sec. III-B; it gives no gains): the rate loop's torque
 *     becomes taumax_i (krate_i e_i + kI_i xi_i - kD_i omega'_i), e = omega_des
 *     - omega, omega' of Eq. (qd4) at the step start (derivative on the
 *     measurement), and xi, the integral of e, is three more state components
 *     advanced once per step: xi <- clamp(xi + dt e, +-xi_max);
 *   - two more agent types in the same launch (the paper's simulator runs
 *     fixed-wing drones, quadrotors and cars, Sec. III-B, and cites their
 *     models without equations), chosen per parameter group, closed loop:
 *       car: kinematic bicycle on the rear axle, p' = v (cos psi, sin psi),
 *         v' = a, psi' = v kappa, steered by pure pursuit towards the
 *         waypoint (kappa = 2 sin(alpha) / max(distance, l_min) for any
 *         bearing alpha, |kappa| <= tan(delta_max) / L_w) and
 *         a = clamp(k_v (v_c - v), +-a_max);
 *       fixed-wing: coordinated-turn guidance model without wind,
 *         p' = V (cos chi, sin chi), chi' = g tan(phi) / V,
 *         phi' = b_phi (phi_c - phi), h'' = -b_hd h' + b_h (h_c - h),
 *         V' = b_V (V_c - V), phi_c = clamp(k_chi * course error, +-phi_max).
 *
 * Conventions
 *   State of one agent, 17 floats: p(3) v(3) q(4: w,x,y,z, Hamilton,
 *   body->inertial) omega(3, body) Omega(4, rad/s).  Frames ENU / FLU.
 *   Rotors: 1 front-left, 2 front-right, 3 rear-right, 4 rear-left.
 *
 *   SIM_CLOSED_LOOP_PID adds xi(3), the body-rate error integral: 20 floats.
 *   Cars and fixed-wing drones use components of the same 17: position
 *   0-2 (a car's height is held), speed 3 (v or airspeed V), climb rate 5
 *   (fixed-wing), heading or course as a unit vector (cos, sin) 6-7, bank 10
 *   (fixed-wing); the other components are left unchanged.  Their commands:
 *   car (x_c, y_c, unused, v_c), fixed-wing (x_c, y_c, h_c, V_c).
 *
 *   State buffers are PLANAR ("SoA of float4"): for N agents, 17*N floats,
 *     plane k = 0..3 : N float4 holding components 4k..4k+3 of every agent,
 *                      at float offset 4*k*N;
 *     plane 4        : N floats holding component 16, at float offset 16*N.
 *   In SIM_CLOSED_LOOP_PID, 20*N floats: plane 4 is N float4 holding
 *   components 16..19 (Omega_4, xi_x, xi_y, xi_z) at float offset 16*N.
 *   The base pointer must be 16-byte aligned.
 *   Commands: N float4 (16-byte aligned).  Closed loop: waypoint x, y, z and
 *   heading psi (rad).  Open loop: the four rotor speed commands (rad/s).
 *
 * Execution and ownership
 *   Every pointer named d_* is device memory owned by the caller; h_* is host
 *   memory owned by the caller.  The library owns only the handle, its device
 *   copy of the parameter groups and a per-agent status byte array, all
 *   allocated in sim_create and freed in sim_destroy.  Calls that take a
 *   stream enqueue asynchronous work on it and return without synchronising
 *   (unless stated) and allocate nothing, so sim_step can be captured in a
 *   CUDA graph.  A stream argument is a cudaStream_t passed as void*
 *   (NULL = the legacy default stream).
 *
 * Threads
 *   Calls on one handle must not overlap in time from several host threads:
 *   the handle holds the launch settings, the host pipeline's streams and
 *   events and a pinned status word.  Different handles may be used from
 *   different threads at once, except by sim_rollout_backward_noalloc, whose
 *   scratch is one per device.
 *
 * Errors
 *   Every int-returning call returns SIM_OK (0) or a negative SIM_ERR_*.
 *   Arguments are checked on the host before anything is enqueued.  No call
 *   raises, traps or asserts on the device.  An agent whose state becomes
 *   non-finite is marked dead in the status array (1) and left at its last
 *   finite state, whatever substeps_K: the stepping calls check each agent at
 *   the end of a launch, and one more pass at the end of the call steps
 *   again, one step at a time, the agents that went non-finite in the middle
 *   of a K-step launch.  Dead agents (any nonzero status byte) are skipped by
 *   every later call (cf. Sec. III-A: agents marked dead are excluded from
 *   the system).  A status of 3 marks, inside a call, an agent waiting for
 *   that pass; it can outlast a call only if the call returned an error.
 *   The controller's clamps also bound a non-finite command component in the
 *   closed-loop modes; commands should be finite.
 */
#ifndef QUADSIM_H
#define QUADSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIM_OK 0
#define SIM_ERR_ARG (-1)       /* bad pointer, size, alignment or value */
#define SIM_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define SIM_ERR_WORKSPACE (-3) /* workspace too small */
#define SIM_ERR_TIMEOUT (-4)   /* a bounded host wait ran out */
#define SIM_ERR_GROUP (-5)     /* a group id >= n_groups was found */
#define SIM_ERR_STALE (-6)     /* a graph captured before the handle's agent order changed */

#define SIM_OPEN_LOOP 0
#define SIM_CLOSED_LOOP 1
#define SIM_CLOSED_LOOP_PID 2 /* closed loop, PID body-rate loop, 20-float state */

#define SIM_TYPE_QUADROTOR 0  /* agent types of a parameter group */
#define SIM_TYPE_CAR 1
#define SIM_TYPE_FIXED_WING 2

#define SIM_MAX_GROUPS 32 /* parameter groups per handle */
#define SIM_NTHETA 16     /* differentiable parameters per group */

/* One parameter group (homogeneous airframe + controller).  Units SI, rad. */
typedef struct {
  float m, Jxx, Jyy, Jzz;               /* kg; principal inertias kg m^2 (Eq. qd4) */
  float L, alpha;                       /* arm length m; arm angle from body x (Eq. 3) */
  float kt, kq;                         /* Eq. 2 coefficients N/(rad/s)^2, N m/(rad/s)^2 */
  float tau_m, c_d, omega_max, g;       /* rotor lag s; drag N s/m; rotor clamp rad/s; m/s^2 */
  float kp[3], kd[3], katt[3], krate[3]; /* position PD, attitude P, normalised rate P */
  float a_max;                          /* per-axis acceleration clamp m/s^2 (INFINITY = off) */
  float kI[3], kD[3];                   /* PID rate loop: integral (1/rad), derivative (s^2/rad), */
  float xi_max[3];                      /* normalised like krate; integrator limit rad (INFINITY = off) */
  int32_t type;                         /* SIM_TYPE_*; a car or fixed-wing group reads only g, L (its */
                                        /* collision radius) and veh */
  float veh[8];                         /* car: L_w m, tan(delta_max), a_max m/s^2, k_v 1/s, l_min m; */
                                        /* fixed-wing: b_phi 1/s, phi_max rad, k_chi, b_hd 1/s, */
                                        /* b_h 1/s^2, b_V 1/s */
} sim_group_params_t;

typedef struct sim_s* sim_handle_t;
typedef struct sim_graph_s* sim_graph_t;

/* Create a simulator for n_agents agents in n_groups parameter groups.
 * d_group_id: device array of n_agents uint8 group ids, or NULL when
 * n_groups == 1.  The handle keeps the pointer (the caller keeps the buffer
 * alive and unchanged); sim_create checks every id once (synchronously) and
 * returns SIM_ERR_GROUP if one is out of range.  It also reads the ids once to
 * see whether each group's agents form one contiguous range (sorted ids, or
 * contiguous blocks in any order): if so, the fused steps run as one kernel
 * launch per group range with the group's constants in the kernel's
 * parameters, the launches side by side on streams the handle creates (one
 * per group; forked from the caller's stream by an event and joined back to
 * it before the call's later work), which is faster than the general form
 * (the results are the same bit for bit).
 * When the groups interleave (and n_agents < 2^32), the handle keeps a
 * group-sorted order of the agents (4 bytes per agent, device memory it owns)
 * and the fused steps reach the agents through it, still one group per block:
 * always when the groups mix agent types (a warp of mixed types would run
 * every type's model), and for launches of 32 fused steps or more otherwise
 * (below that, the order's scattered loads cost more than they save).  The
 * caller's buffers keep their layout.  mode: SIM_OPEN_LOOP,
 * SIM_CLOSED_LOOP or SIM_CLOSED_LOOP_PID (kI, kD, xi_max are read only in the
 * last; they must be finite, xi_max >= 0, in every mode).  Groups of car or
 * fixed-wing type need SIM_CLOSED_LOOP; such a handle steps (sim_step and
 * the calls built on it, collisions) but has no checkpointed rollout or
 * adjoint (SIM_ERR_ARG).  Runs on the current CUDA device.  A handle's calls
 * come from one host thread at a time: its calls reuse streams and events the
 * handle owns. */
int sim_create(const sim_group_params_t* groups, int n_groups, int64_t n_agents, const uint8_t* d_group_id,
               int mode, sim_handle_t* out);

/* Replace the parameter groups (same count; vehicle types need the handle's
 * mode to be SIM_CLOSED_LOOP).  Every group is checked first; on
 * SIM_ERR_ARG nothing changes.  Synchronous on the host, but it does not wait for work
 * of this handle already enqueued on other streams: synchronise those first,
 * or a launch in flight may see some blocks with the old groups and some
 * with the new.  CUDA graphs captured before keep the kernels and the group
 * parameters their launches carry (one group, and the groups that run as a
 * launch per range or through an order): capture them again after this
 * call. */
int sim_set_params(sim_handle_t h, const sim_group_params_t* groups, int n_groups);

/* Advance every live agent nsteps RK4 steps of length dt, in place.
 * substeps_K: steps fused per launch (state stays in registers between
 * them and touches HBM once per launch); 0 = the handle's tuned value.
 * nsteps % K remainder steps run as one shorter launch.  nsteps >= 0 (0
 * enqueues nothing), dt > 0 and finite, d_state and d_cmd 16-byte aligned;
 * otherwise SIM_ERR_ARG. */
int sim_step(sim_handle_t h, float* d_state, const float* d_cmd, float dt, int64_t nsteps, int substeps_K,
             void* stream);

/* sim_step for callers whose state lives in host memory: copies h_state and
 * h_cmd into the caller's device buffers d_state / d_cmd, steps, copies the
 * state back into h_state, then waits for `stream` (bounded wait).  The agents
 * are processed in up to 32 chunks whose host-to-device copies, steps (over 4
 * compute streams) and device-to-host copies run on library-owned streams, so
 * copies overlap compute; the call is ordered after earlier work on `stream`.  Host buffers
 * should be pinned for the copies to be asynchronous.  Not capturable in a
 * CUDA graph (it waits).  On SIM_ERR_TIMEOUT the copies may still be running:
 * keep every buffer alive until `stream` is idle. */
int sim_step_host(sim_handle_t h, float* h_state, const float* h_cmd, float* d_state, float* d_cmd, float dt,
                  int64_t nsteps, int substeps_K, void* stream);

/* Decision rounds with the algorithm side outside the physics loop (Sec.
 * III-A: the physical world runs on between decisions).  Runs `rounds` rounds
 * of steps_per_round RK4 steps (substeps_K fused per launch; 0 = tuned).
 * Round r uses the commands h_cmds + r * 4 N (pinned host memory, float4 per
 * agent): they are copied into one of the two device command planes of
 * d_cmd2 (2 * 4 N floats) on a library copy stream while round r - 1 runs.
 * After round r the positions plane (plane 0: px, py, pz, vx per agent) is
 * snapshotted into one of the two planes of d_obs2 (2 * 4 N floats, may be
 * NULL with h_obs NULL) and copied to h_obs + r * 4 N on another copy stream
 * while round r + 1 runs.  d_state is updated in place.  The call is ordered
 * after earlier work on `stream` and returns when the last round and its
 * observations are done (bounded wait).  Not capturable (it waits).  On
 * SIM_ERR_TIMEOUT the copies may still be running: keep every buffer alive
 * until `stream` is idle. */
int sim_run_rounds(sim_handle_t h, float* d_state, float* d_cmd2, const float* h_cmds, float* d_obs2, float* h_obs,
                   float dt, int64_t steps_per_round, int64_t rounds, int substeps_K, void* stream);

/* Forward rollout with checkpoints, one launch (nsteps >= 1; ckpt_C >= 0,
 * 0 = the handle's tuned interval).  Reads d_state0, writes
 * S+1 planar states into d_ckpt (S = ceil(nsteps/ckpt_C)): x_0, x_C, ...,
 * x_{(S-1)C}, then x_nsteps last.  State s starts at float offset s*P, with
 * P = 17*N (20*N in SIM_CLOSED_LOOP_PID) rounded up to a multiple of 4, so
 * that each state starts 16-byte aligned; d_ckpt holds S*P + 17*N (20*N)
 * floats, which is (S+1)*17*N when N is a multiple of 4.  d_run_cost (N floats, may be NULL)
 * receives, per agent, the sum over step ends n = 1..nsteps of
 * sum_i Omega_{n,i}^2. */
int sim_rollout_forward(sim_handle_t h, const float* d_state0, const float* d_cmd, float dt, int64_t nsteps,
                        int ckpt_C, float* d_ckpt, float* d_run_cost, void* stream);

/* Bytes of workspace sim_rollout_backward needs for this handle, its
 * current launch configuration and checkpoint interval ckpt_C. */
size_t sim_workspace_bytes(sim_handle_t h, int ckpt_C);

/* Discrete adjoint of the rollout of sim_rollout_forward (same dt, nsteps,
 * ckpt_C, d_cmd).  For the loss L = l(x_T) + sum_a w_a * run_cost_a it takes
 *   d_dL_dxT : planar 17*N (20*N in SIM_CLOSED_LOOP_PID), dl/dx_T;
 *   d_w_run  : N floats, w_a (NULL = no running cost);
 * and writes
 *   d_dL_dx0          : planar like d_dL_dxT, dL/dx_0;
 *   d_dL_dtheta       : n_groups*16 floats, dL/dtheta per group, theta =
 *                       (kp[3], kd[3], katt[3], krate[3], m, Jxx, Jyy, Jzz);
 *   d_dL_dtheta_agent : N*16 floats of per-agent contributions, or NULL.
 * Segments are recomputed from the checkpoints into the workspace and swept
 * backwards.  Subgradients: clamps pass the gradient on their closed
 * interval, sqrt(0) has derivative 0, branch choices are constants.  The
 * per-group sums are deterministic (fixed reduction order, no atomics).
 * d_workspace must hold sim_workspace_bytes(h, ckpt_C) bytes, 256-byte
 * aligned.  In SIM_CLOSED_LOOP_PID the integrator's clamp passes the gradient
 * on its closed interval too; kI, kD and xi_max are not differentiated.
 * Agents marked dead when the call runs are frozen over the rollout, as
 * sim_rollout_forward treats them (x_T = x_0, running cost 0): their dL/dx_0
 * is their dL/dx_T, their per-agent rows are 0 and they add nothing to
 * d_dL_dtheta.  (An agent whose state turned non-finite during the forward
 * rollout is marked by it and gets the same frozen gradient, which then has
 * no meaning.) */
int sim_rollout_backward(sim_handle_t h, const float* d_ckpt, const float* d_cmd, float dt, int64_t nsteps,
                         int ckpt_C, const float* d_dL_dxT, const float* d_w_run, float* d_dL_dx0,
                         float* d_dL_dtheta, float* d_dL_dtheta_agent, void* d_workspace, size_t ws_bytes,
                         void* stream);

/* Workspace-free variant of sim_rollout_backward (the paper has no
 * counterpart; it exists for this library's callers).  Some callers may not
 * allocate device memory once they are running -- for example a real-time
 * control loop that reserves all of its memory at start-up, or a plug-in
 * whose host application owns every device allocation and hands out no
 * workspace -- so they cannot provide the workspace sim_rollout_backward
 * needs.  This entry point takes the same arguments minus the workspace and
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * call): its scratch is a fixed array of SIM_NOALLOC_SCRATCH_BYTES (32 MiB)
 * inside the library, which every GPU that loads the library holds until the
 * process exits.
 *   - The grid is capped so that its scratch fits in the array, possibly
 *     slower.  Per-agent outputs equal sim_rollout_backward's bit for bit.
 *     The per-group sums equal them up to FP32 summation-order rounding: a
 *     capped grid partitions the agents over fewer blocks, so each block's
 *     grid-stride loop, its per-warp accumulation and the final reduction
 *     add the agents' terms in another order.
 *   - SIM_ERR_WORKSPACE if even one block does not fit, i.e. when
 *     ckpt_C * (68 B, 80 B in the PID mode) * (adjoint block size) + n_groups * 64 B exceeds
 *     32 MiB (ckpt_C above about 3,800 with the default 128-thread adjoint
 *     block).
 *   - The first call on a device looks up the array's device address for
 *     that device (cudaGetSymbolAddress); make that first call before any
 *     stream capture.
 *   - Every call shares the one array: calls whose work overlaps on the GPU
 *     (other streams, other threads) race and corrupt each other's results.
 *     Serialise them. */
#define SIM_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int sim_rollout_backward_noalloc(sim_handle_t h, const float* d_ckpt, const float* d_cmd, float dt, int64_t nsteps,
                                 int ckpt_C, const float* d_dL_dxT, const float* d_w_run, float* d_dL_dx0,
                                 float* d_dL_dtheta, float* d_dL_dtheta_agent, void* stream);

/* Collision detection (Sec. III-A: the collision/detection module marks
 * colliding agents as dead and excludes them from the whole system).  Two
 * live agents collide when their centres are closer than the sum of their
 * bounding radii, radius = (arm length L of the agent's group) *
 * radius_scale; the decision is taken in FP32 as d2 < (r_i + r_j)^2 with
 * d2 = (dx*dx + dy*dy) + dz*dz, each operation rounded separately.  Every
 * colliding live agent is marked dead (status 2) and frozen by later calls.
 * Method: a uniform grid of cells of side 1.01 x twice the largest contact
 * distance (4.04 max radius), hashed into a power-of-two table of >= 4
 * n_agents buckets (spatial hash of Teschner et al., 2003), one linked list
 * per bucket of 32-byte records (position, radius, link) built with atomic
 * exchanges.  A pair in contact is then less than half a cell apart on every
 * axis, so each agent searches the 2 x 2 x 2 cells on the side of its own
 * cell it lies nearer to (cell coordinates computed in FP64).  The outcome
 * does not depend on the order of the lists.
 * d_state: planar state (only positions are read).  d_workspace:
 * sim_collide_workspace_bytes(h) bytes (about 16 + 32 + 1 bytes per agent),
 * 256-byte aligned.  radius_scale > 0.
 * Up to 2^31 - 1 agents.  The call may run on a stream other than the
 * stepping stream ("outside the main loop"): an agent marked while a step is
 * in flight is frozen from the next launch on. */
size_t sim_collide_workspace_bytes(sim_handle_t h);
int sim_collide(sim_handle_t h, const float* d_state, float radius_scale, void* d_workspace, size_t ws_bytes,
                void* stream);
/* Copies the per-agent status bytes (0 alive, 1 non-finite, 2 collided) into
 * the caller's device buffer of n_agents bytes. */
int sim_copy_status(sim_handle_t h, uint8_t* d_status_out, void* stream);

/* Replaces the per-agent status bytes with the caller's device buffer of
 * n_agents bytes (any nonzero byte marks the agent dead; the library itself
 * writes 1 for a non-finite state and 2 for a collision).  The planar state
 * (the caller's buffer), the parameter groups and the status are the whole
 * of a swarm's state: saving the state and sim_copy_status, then restoring
 * both with a copy and sim_load_status, resumes a run bit for bit
 * (checkpoint / resume).  Stream-ordered, allocates nothing. */
int sim_load_status(sim_handle_t h, const uint8_t* d_status_in, void* stream);

/* Launch configuration: threads per block of the forward kernels (a
 * multiple of 32, <= 256) and of the adjoint kernel (a multiple of 32,
 * <= 128), and the defaults used when a call passes 0 for the steps fused
 * per launch (K) or the checkpoint interval (C).  A 0 argument leaves that
 * value unchanged; anything else out of range returns SIM_ERR_ARG.
 * sim_create sets the block sizes to the largest of 128, 64 and 32 (forward
 * and adjoint alike) that gives every SM at least one block, and to 32
 * for a swarm too small for that, so that a small swarm spreads one warp per
 * SM instead of sharing the schedulers of a few SMs.  Forward results do not
 * depend on the block size; group sums of the adjoint are summed in another
 * order (within rounding). */
int sim_set_launch(sim_handle_t h, int block_fwd, int block_adj, int K, int C);
int sim_get_launch(sim_handle_t h, int* block_fwd, int* block_adj, int* K, int* C);

/* Number of agents marked dead (non-finite state).  Synchronises the stream
 * with a bounded wait (SIM_ERR_TIMEOUT after timeout_ms). */
int sim_status(sim_handle_t h, int64_t* n_dead, int timeout_ms, void* stream);
/* Marks every agent alive again (and drops a sim_compact order). */
int sim_reset_status(sim_handle_t h, void* stream);

/* Per-group diagnostics of the swarm in d_state (planar, 16-byte aligned): for
 * each group g, h_out[6 g .. 6 g + 5] = the number of live agents, of agents
 * frozen non-finite (status 1), of agents marked collided (status 2), and the
 * mean position x, y, z of the live agents (0 when none is live; z is the
 * altitude).  FP64 sums reduced in a fixed order (the same result on every
 * run); ordered after earlier work on `stream`, then waits for it (bounded).
 * h_out: host memory of 6 n_groups doubles. */
int sim_group_stats(sim_handle_t h, const float* d_state, double* h_out, void* stream);

/* Steps only the live agents from now on (Sec. III-A: agents marked dead are
 * excluded from the computation).  Dead agents are otherwise skipped by the
 * thread that holds them, so a swarm whose dead agents are spread over the ids
 * (after collisions, say) keeps its full launch time: with half of 1e6 agents
 * dead at random, half the throughput per live agent.  sim_compact builds,
 * from the status bytes, an order of the live agents alone, sorted by group
 * (4 bytes per agent of device memory the handle owns): two passes on the
 * device ordered after earlier work on `stream`, with one bounded wait for
 * the per-group counts between them and one at the end (0.14 ms for 1e6
 * agents).  Fused launches of 2 steps or more (any number when the groups mix
 * agent types), over the whole swarm or whole sim_step_host chunks, then step
 * only those agents, one group per block; sim_rollout_forward and the adjoint
 * (sim_rollout_backward, sim_rollout_backward_noalloc) sweep only those agents
 * too, and a memory-bound pass writes the frozen results of the dead ones
 * (their checkpoints, dL/dx0 = dL/dx_T, zero theta rows).  Results are the same bit for bit.
 * Agents that die later are skipped as before; sim_reset_status and
 * sim_load_status drop the order (dead agents may come alive).  Each of these
 * changes of the order makes graphs captured before it stale: sim_graph_launch
 * refuses them with SIM_ERR_STALE (capture again).  Work of this handle on
 * other streams must be finished first.  More than 2^32 agents: no order,
 * SIM_OK. */
int sim_compact(sim_handle_t h, void* stream);

/* Capture ceil(nsteps/K) sim_step launches on d_state/d_cmd into a CUDA
 * graph (stream capture on `stream`, which must not be the legacy default
 * stream); sim_graph_launch replays them on any stream, or returns
 * SIM_ERR_STALE when sim_compact (or a status reset that dropped its order)
 * has changed the handle's agent order since the capture.  A graph must not
 * outlive its handle. */
int sim_graph_create(sim_handle_t h, float* d_state, const float* d_cmd, float dt, int64_t nsteps, int substeps_K,
                     void* stream, sim_graph_t* out);
int sim_graph_launch(sim_graph_t g, void* stream);
void sim_graph_destroy(sim_graph_t g);

/* Number of kernel launches one sim_step call makes for these arguments:
 * ceil(nsteps / K) fused step launches, each one kernel launch per group
 * range when several groups run by range or order (contiguous ids, a
 * group-sorted order, or sim_compact's live order: one launch per group with
 * agents there, each on a stream of the handle's own, forked from and joined
 * back to the caller's stream), plus one pass that replays agents which went
 * non-finite in the middle of a launch (none when every launch is a single
 * step of one open- or P-closed-loop quadrotor group).  An upper bound: a
 * launch over no agent is skipped, and counted as if each group had agents. */
int64_t sim_step_launches(sim_handle_t h, int64_t nsteps, int substeps_K);

void sim_destroy(sim_handle_t h);
const char* sim_error_string(int code);

/* Device bounds checks (a stand-in for a memory checker).  The library can be
 * built a second time with its kernels' index checks compiled in
 * (libquadsim_checked.so): each instrumented access first tests its index
 * against the extent of its buffer; a failed test records the first failure
 * in a device word, site << 48 | index (low 48 bits), and skips the access --
 * no trap, no assert, so the context stays usable.  sim_bounds_checks waits
 * for the device, stores that word in *first_failure (0: no failure) and
 * clears it, and returns 1; the product library returns 0 with
 * *first_failure = 0.  Sites: 1-3 planar state loads, stores and prefetches,
 * 4 agent indices, 5 group ids, 6-7 range-kernel ranges and order entries,
 * 8 checkpoint indices, 9 adjoint scratch steps and theta rows, 10 collision
 * records, 11 live-order positions, 12 partial sums. */
int sim_bounds_checks(uint64_t* first_failure);

#ifdef __cplusplus
}
#endif
#endif /* QUADSIM_H */
