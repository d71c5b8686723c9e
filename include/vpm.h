/*
 * vpm.h - C ABI of the B300 vortex-particle-model (VPM) rollout library.
 *
 * The library advances batches of 2-D VPM models of a flat-plate glider, each carrying its own
 * field of regularised point vortices, and reduces rollout costs to MPPI weights, as defined in
 * "Real-Time Maneuver Planning for Fixed-Wing UAVs in Unsteady Flows Using a GPU-Accelerated
 * Vortex Particle Model": the model of §III-A (Eqs. 2-17), the glider of §III-B (Eqs. 18-22),
 * the terminal cost of §IV-A (Eq. 24) and the MPPI reweighting of §IV-A (Eq. 25).
 *
 * Conventions shared by every call
 *  - Coordinates are (x, z) in chord units, z up. Positive circulation and positive pitch are
 *    counter-clockwise (nose up). A particle is (x, z, Gamma).
 *  - Pointers named d_* are device pointers (for example from torch tensors); h_* are host
 *    pointers. The caller owns every buffer it passes. The library owns vpm_state handles.
 *  - Every call that takes a cudaStream_t enqueues its work on that stream and returns without
 *    waiting, unless it says otherwise. Calls on one state must not overlap on the device.
 *  - Every call returns a vpm_status. VPM_OK is 0. vpm_last_error() gives a message for the
 *    last failing call of the calling host thread. Invalid arguments are rejected on the host
 *    before anything is enqueued; device-side failures (non-finite values) latch into the
 *    state's error word, which vpm_state_status() reads.
 *  - The library builds for sm_103a only and keeps no CPU fallback: without a CUDA device every
 *    call that needs one returns VPM_ERR_CUDA.
 */
#ifndef VPM_H
#define VPM_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VPM_OK = 0,
    VPM_ERR_INVALID = 1,     /* bad argument (null, negative size, non-finite parameter)   */
    VPM_ERR_OOM = 2,         /* device allocation failed                                    */
    VPM_ERR_CAPACITY = 3,    /* particles would exceed the state's capacity or shared memory */
    VPM_ERR_NONFINITE = 4,   /* a NaN or Inf appeared in a model quantity                   */
    VPM_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                               */
    VPM_ERR_CUDA = 6,        /* a CUDA runtime call failed (message in vpm_last_error)       */
    VPM_ERR_BUSY = 7,        /* resource in use                                             */
    VPM_ERR_SINGULAR = 8     /* the surface-circulation system is singular                  */
} vpm_status;

/* Kernel applied by wake and shed vortices. Bound vortices always use the singular kernel
 * (§III-A: Eq. 4 for bound vortices, Eq. 5 for wake vortices). */
typedef enum {
    VPM_KERNEL_SINGULAR = 0, /* Eq. 4: K = -1/(2 pi r^2) [[0,1],[-1,0]] dr                   */
    VPM_KERNEL_VATISTAS = 1, /* Eq. 5: Eq. 4 times (r/r_core)^2 / sqrt(1 + (r/r_core)^4)     */
    VPM_KERNEL_GAUSSIAN = 2  /* Eq. 4 times 1 - exp(-r^2 / r_core^2)                          */
} vpm_kernel;

/* Arithmetic of the particle sums and positions. VPM_FP32: binary32 pair sums with
 * compensated accumulation across source tiles and double-length (hi + lo) positions;
 * the surface solve, Kelvin sum, loads and glider stay binary64. VPM_FP64: binary64
 * throughout. */
typedef enum { VPM_FP32 = 0, VPM_FP64 = 1 } vpm_precision;

/* Separation gate of §III-A. */
typedef enum {
    VPM_GATE_OFF = 0,        /* LEV and TEV shed every step                                 */
    VPM_GATE_BOTH = 1,       /* nothing is shed while |alpha| <= alpha_crit                  */
    VPM_GATE_LEV = 2         /* TEV every step, LEV only while |alpha| > alpha_crit          */
} vpm_gate;

/* Model parameters. Field meanings follow §III-A and §III-B. */
typedef struct {
    int n_b;                 /* bound vortices N_b (collocation points N_c = N_b + 1), 2..32  */
    double chord, span, rho; /* chord c, span s, air density                                 */
    int wake_kernel;         /* vpm_kernel of wake and shed vortices                         */
    double r_core;           /* core radius of the wake kernel                               */
    double shed_offset;      /* delta_s / c: LEV at LE - delta_s e_t, TEV at TE + delta_s e_t  */
    double gamma_decay;      /* gamma of Eq. 17; Gamma <- Gamma exp(-gamma dt) each step      */
    int shed_gate;           /* vpm_gate                                                     */
    double alpha_crit;       /* critical angle of attack (rad)                               */
    int n_wake_max;          /* merge the two oldest particles while N > n_wake_max; 0 = off  */
    double u_inf[2];         /* uniform free stream (0 in still air)                         */
    double dt;               /* time step (explicit Euler)                                   */
    int fixed_plate;         /* 1: the plate is held at the initial glider pose, never moves  */
    double mass, inertia, g; /* glider mass, pitch inertia, gravity                          */
    double l, l_w, l_e, s_e; /* body length, wing offset, elevator length and area (Eq. 18)   */
    double q[7];             /* diagonal of Q (Eq. 24)                                        */
    double x_d[7];           /* desired final state x_d (Eq. 24)                              */
    int precision;           /* vpm_precision                                                */
} vpm_params;

typedef struct vpm_state vpm_state;

/* Message describing the last failure of the calling host thread ("" if none). */
const char *vpm_last_error(void);

/* Library version string. */
const char *vpm_version(void);

/*
 * Creates a resident model: glider state x_g = [x, z, theta, phi, xdot, zdot, thetadot]
 * (§III-B, Eq. 23) and n wake particles, with room for `capacity` particles. h_particles is
 * n x 3 row-major binary64 (x, z, Gamma). The previous-step circulations used by the time
 * derivatives of Eq. 13 start unset (the first step's derivatives are zero). Synchronises
 * `stream` before returning.
 * Errors: VPM_ERR_INVALID (null pointers, n < 0, capacity < n, bad parameters),
 * VPM_ERR_NONFINITE (non-finite input), VPM_ERR_CAPACITY (capacity beyond the shared memory
 * of one block), VPM_ERR_OOM, VPM_ERR_SINGULAR (surface system singular for these
 * parameters), VPM_ERR_CUDA (no device).
 */
vpm_status vpm_state_create(const vpm_params *params, const double *h_particles, int n,
                            int capacity, const double *h_glider7, vpm_state **out,
                            cudaStream_t stream);

/* Frees the state's device memory (synchronises the device first). */
vpm_status vpm_state_destroy(vpm_state *state);

/*
 * Sets the previous-step bound circulations h_gb_prev[n_b], the previous LEV circulation and
 * whether they are valid (has_prev = 0 makes the next step's derivatives zero). Synchronises
 * `stream`. The previous LEV circulation is kept with the state for the caller's records;
 * the pressure of Eq. 13 does not use it: each step sheds a new LEV, and the derivative of
 * the leading-edge circulation in Eq. 13 is that new LEV's circulation over dt.
 */
vpm_status vpm_state_set_history(vpm_state *state, const double *h_gb_prev, double glev_prev,
                                 int has_prev, cudaStream_t stream);

/*
 * Copies the state to the host and synchronises `stream`: *n_out particles into
 * h_particles (capacity x 3 binary64; on the binary32 path x and z are hi + lo), the glider
 * state h_glider7, and optionally (if non-null) h_hist[n_b + 2] = [Gamma_b of the previous
 * step (n_b), Gamma_LEV of the previous step, has_prev]. Returns the latched device error.
 */
vpm_status vpm_state_read(const vpm_state *state, double *h_particles, int *n_out,
                          double *h_glider7, double *h_hist, cudaStream_t stream);

/* Replaces the glider state (x, z, theta, phi, xdot, zdot, thetadot) by h_x7, e.g. with an
 * observed one (the tracking instance of §IV-C follows the observed rigid-body state).
 * Synchronises `stream`. Errors: VPM_ERR_INVALID (null), VPM_ERR_NONFINITE. */
vpm_status vpm_state_set_glider(vpm_state *state, const double *h_x7, cudaStream_t stream);

/*
 * Puts a disturbance pair (§V: two opposite vortices standing for a vortex ring) in front of the
 * state's wake: h_pair = (x1, z1, Gamma1, x2, z2, Gamma2). The pair occupies the first two
 * slots, is convected with the wake by every step and rollout, is left out of merging, and is
 * removed when, after a step's glider update, the segment joining it crosses the chord line
 * moved by 2 % of the chord against the normal (the termination at the wing of §V).
 * Errors: VPM_ERR_INVALID (null, a pair already present), VPM_ERR_NONFINITE,
 * VPM_ERR_CAPACITY (no room for two more particles), VPM_ERR_CUDA.
 */
vpm_status vpm_state_inject_pair(vpm_state *state, const double *h_pair, cudaStream_t stream);

/* *h_n_dist = 2 while the state's disturbance pair is present, else 0 (synchronises). */
vpm_status vpm_state_disturbance(const vpm_state *state, int *h_n_dist, cudaStream_t stream);

/* Copies the glider state to h_x7 (synchronises `stream`). */
vpm_status vpm_state_get_glider(const vpm_state *state, double *h_x7, cudaStream_t stream);

/* Device-side copy of src (particles, count, glider state, previous circulations) into dst,
 * asynchronous on `stream`. Both states must have the same precision and n_b, and dst's
 * capacity must hold src's particles. Errors: VPM_ERR_INVALID. */
vpm_status vpm_state_copy(vpm_state *dst, const vpm_state *src, cudaStream_t stream);

/*
 * Advances the state in place by `steps` steps under the tracking policy of §IV-B: at step k
 * the control is ubar_j - H_j . (x_k - xbar_j), j = offset + k, x_k the state's own glider
 * state (one launch; the projection over the replanning time of §IV-C). Policy arrays as in
 * vpm_rollout_batch_policy. Errors: VPM_ERR_INVALID, VPM_ERR_CAPACITY, VPM_ERR_CUDA.
 */
vpm_status vpm_state_advance_policy(vpm_state *state, int steps, const double *d_gains,
                                    const double *d_xbar, const float *d_ubar, int offset,
                                    cudaStream_t stream);

/* Reads and clears the state's latched device error word (synchronises `stream`). */
vpm_status vpm_state_status(vpm_state *state, cudaStream_t stream);

/* Serialises the complete state into a host buffer (synchronises `stream`). With h_buf null,
 * *bytes receives the size needed. */
vpm_status vpm_state_save(const vpm_state *state, void *h_buf, size_t *bytes,
                          cudaStream_t stream);

/* Restores a state saved by vpm_state_save into a state created with the same precision,
 * n_b and capacity (synchronises `stream`). */
vpm_status vpm_state_load(vpm_state *state, const void *h_buf, size_t bytes,
                          cudaStream_t stream);

/*
 * Advances the resident model by one step under elevator rate u (the tracking instance of
 * §IV-C), in the order: geometry, relative velocity at the plate (Eq. 12), surface solve
 * (Eq. 11), pressure and loads (Eqs. 13-15), glider update, shedding, convection (Eq. 16),
 * Euler advection, decay (Eq. 17), merging. Optional device outputs (null to skip):
 *   d_fm[3]              wing load F_w,x, F_w,z, M_w of this step
 *   d_gamma_s[n_b+2]     surface circulations [Gamma_b, Gamma_LEV, Gamma_TEV] (0 if not shed)
 *   d_vel[2*(n+2)]       convection velocity (u, w) of every particle of the enlarged wake
 *   d_vtilde[2*(2n_b+1)] relative velocity of Eq. 12 at the collocation then bound points
 * Errors: VPM_ERR_CAPACITY if the step could overflow the capacity, VPM_ERR_CUDA.
 */
vpm_status vpm_step(vpm_state *state, double u, double *d_fm, double *d_gamma_s, double *d_vel,
                    double *d_vtilde, cudaStream_t stream);

/*
 * Device bytes of the pair-sum scratch that a batch of K rollouts of H steps from this state
 * allocates while it runs (0 for binary64 states and fields that stay within 128 particles).
 * Each block of the binary32 rollout kernel keeps, per step, the sums formed when one
 * evaluation of a particle pair serves both particles: about cap^2 / 256 float2 slots for a
 * field that can reach cap particles. Errors: VPM_ERR_INVALID (null, K or H < 1).
 */
vpm_status vpm_rollout_scratch_bytes(const vpm_state *state, int K, int H, size_t *bytes);

/* The same for K rollout blocks whose fields can reach `capacity` particles, without a state
 * (precision VPM_FP32 or VPM_FP64; host only). Errors: VPM_ERR_INVALID (null, K < 1,
 * capacity < 0, unknown precision). */
vpm_status vpm_rollout_scratch_bytes_cap(int precision, int capacity, int K, size_t *bytes);

/* The binary32 rollout kernel's own scratch index (host only; the paper has no counterpart: it
 * serves checks of the scratch layout). For a block whose fields can reach `capacity` particles,
 * in float2 slots from the block's scratch start: kind 0 gives the first of the two slots that
 * hold the compensated forward sum of target `particle` (a particle of an off-diagonal row,
 * particle < 128 (ceil(capacity / 128) - 1)); kind 1 gives the slot of the reverse sum of source
 * `particle` over the targets of off-diagonal row `row` (particle >= 128 (row + 1)). The rows
 * are the 128-particle rows of the pair phase. Errors: VPM_ERR_INVALID (null, or no such slot). */
vpm_status vpm_rollout_scratch_slot(int capacity, int kind, int row, int particle, long long *slot);

/*
 * K independent rollouts of H steps from the root model, which is not modified. Rollout i
 * applies elevator rates d_controls[i*H + k] (binary32, K x H row-major). One thread block
 * holds one rollout's field in shared memory for the whole horizon. Binary32 launches of a few
 * rollouts whose fields can exceed 2300 particles (Vatistas kernel, H > 1) instead spread each
 * rollout over a thread-block cluster of C CTAs, the largest C in {4, 2} with K C <= the SM count
 * (every CTA holds the field; the pair work is split between them): the same bits, faster when
 * K alone would leave SMs idle; VPM_ROLLOUT_CLUSTERS=0 in the environment keeps one block per
 * rollout. A launch made while `stream` is being captured into a CUDA graph uses clusters only
 * for a launch shape (field capacity, and the cluster size the rule picks) that an earlier launch
 * outside capture has used, and one block per rollout otherwise. Outputs (device):
 *   d_costs[K]               terminal cost J_i of Eq. 24 (computed in binary64, stored binary32;
 *                            NaN if the rollout produced a non-finite value)
 *   d_final_glider[K*7]      final glider states (binary64), or null
 *   d_traj[K*H*7]            glider state after every step (binary64), or null
 *   d_field[K*capacity*3]    final wake (x, z, Gamma) per rollout (binary64), or null
 *   d_count[K]               final particle count per rollout, or null
 * Binary32 roots whose field can grow past 128 particles need device scratch for the pair
 * sums (vpm_rollout_scratch_bytes); it is allocated on `stream` from the library's own memory
 * pool for the launch and freed after it (stream-ordered; see vpm_pool_trim). The device's
 * default pool is not touched.
 * Errors: VPM_ERR_INVALID (K, H < 1, null controls/costs), VPM_ERR_CAPACITY (the count could
 * exceed the capacity within H steps), VPM_ERR_CUDA.
 */
vpm_status vpm_rollout_batch(const vpm_state *root, int K, int H, const float *d_controls,
                             float *d_costs, double *d_final_glider, double *d_traj,
                             double *d_field, int *d_count, cudaStream_t stream);

/*
 * vpm_rollout_batch with a separate initial glider state per rollout: d_x0[K*7] (binary64,
 * row i = rollout i) replaces the root's glider state; the wake and the previous circulations
 * are the root's. These are the perturbed initial states X^0 of the policy synthesis of §IV-B.
 * Errors as vpm_rollout_batch, and VPM_ERR_INVALID for a null d_x0.
 */
vpm_status vpm_rollout_batch_x0(const vpm_state *root, int K, int H, const double *d_x0,
                                const float *d_controls, float *d_costs, double *d_final_glider,
                                double *d_traj, double *d_field, int *d_count,
                                cudaStream_t stream);

/*
 * Closed-loop rollouts under the tracking policy of §IV-B: at step k of rollout i the control is
 *   u = ubar_j - H_j . (x_k - xbar_j),  j = offset + k  (+ d_controls[i*H + k] if given),
 * with x_k the rollout's own glider state. d_gains[(offset+H)*7], d_xbar[(offset+H)*7] (binary64)
 * and d_ubar[offset+H] (binary32) hold the policy (as from vpm_tvlqr and the nominal
 * trajectory); d_x0[K*7] per-rollout initial states or null (the root's). Outputs as
 * vpm_rollout_batch. Used to project the state over the replanning time and to evaluate a policy
 * over perturbed initial conditions. Errors: VPM_ERR_INVALID (null policy or costs, K, H < 1,
 * offset < 0), VPM_ERR_CAPACITY, VPM_ERR_CUDA.
 */
vpm_status vpm_rollout_batch_policy(const vpm_state *root, int K, int H, const double *d_x0,
                                    const double *d_gains, const double *d_xbar,
                                    const float *d_ubar, int offset, const float *d_controls,
                                    float *d_costs, double *d_final_glider, double *d_traj,
                                    cudaStream_t stream);

/*
 * Least-squares synthesis of the glider's time-varying Jacobians from perturbed rollouts
 * (§IV-B, the least-squares problem for df/dx, df/du). For each step k < H:
 *   rows i < K:  regressors (x^i_k - xbar_k) at (theta, phi, xdot, zdot, thetadot) and
 *                u^i_k - ubar_k;  targets the deviation of the accelerations
 *                (xddot, zddot, thetaddot) from the nominal, the derivative of every trajectory
 *                being its explicit-Euler increment (x_{k+1} - x_k) / dt;
 *   solution:    A_hat_k (3 x 5) and B_hat_k (3 x 1), the unknown blocks of A_k and B_k.
 * Inputs (device, binary64 unless stated): d_x0[K*7] initial states x^i_0, d_traj[K*H*7] the
 * states after every step (as written by vpm_rollout_batch_x0), d_controls[K*H] binary32 the
 * rollouts' controls, d_xbar[(H+1)*7] nominal states, d_ubar[H] binary32 nominal controls.
 * Outputs: d_ahat[H*15] (row-major 3 x 5 per step), d_bhat[H*3], and d_info[H] (or null):
 * 0, or 1 where the normal equations are singular (that step's outputs are NaN). Solved in
 * binary64 by the normal equations with column equilibration and Cholesky factorisation.
 * Errors: VPM_ERR_INVALID (K < 6, H < 1, dt <= 0, a null input or output), VPM_ERR_CUDA.
 */
vpm_status vpm_ls_jacobians(int K, int H, double dt, const double *d_x0, const double *d_traj,
                            const float *d_controls, const double *d_xbar, const float *d_ubar,
                            double *d_ahat, double *d_bhat, int *d_info, cudaStream_t stream);

/*
 * TVLQR gains of §IV-B from identified Jacobians: A_k, B_k are assembled from A_hat_k, B_hat_k
 * with the known structure (kinematic rows on the velocity columns, phidot = u), discretised by
 * explicit Euler (I + dt A_k, dt B_k), and the discrete Riccati recursion runs backwards from
 * S_H = Q_f with S_k formed from S_{k+1}; the gain is
 *   H_k = (R_c + B_k' S_{k+1} B_k)^-1 B_k' S_{k+1} A_k,   u_k = ubar_k - H_k (x_k - xbar_k).
 * h_qc[7], h_qf[7]: host diagonals of Q_c and Q_f; rc > 0 the scalar R_c. Outputs (device,
 * binary64): d_gains[H*7], d_s0[49] (S_0 row-major) or null. One warp, binary64.
 * Errors: VPM_ERR_INVALID (H < 1, dt <= 0, rc <= 0, null or non-finite weights, null gains),
 * VPM_ERR_CUDA.
 */
vpm_status vpm_tvlqr(int H, double dt, const double *d_ahat, const double *d_bhat,
                     const double *h_qc, const double *h_qf, double rc, double *d_gains,
                     double *d_s0, cudaStream_t stream);

/*
 * Same results as vpm_rollout_batch computed in the plain one-rollout-per-launch form: every
 * step of every rollout is its own single-block launch (H x K launches) and each rollout's
 * field lives in global memory between launches. Kept as the comparison baseline for the
 * persistent form. Uses library-allocated scratch (stream-ordered allocation).
 */
vpm_status vpm_rollout_batch_per_launch(const vpm_state *root, int K, int H,
                                        const float *d_controls, float *d_costs,
                                        double *d_final_glider, cudaStream_t stream);

/*
 * MPPI weights of §IV-A, Eq. 25: w_i = eta exp(-(J_i - J_min) / lambda), eta normalising the
 * sum to 1. d_costs[K] binary32 in, d_weights[K] binary32 out; exponentials and sums in
 * binary64 in a fixed order (deterministic). J_min and the sum run over the finite costs; a
 * cost that is NaN or infinite (vpm_rollout_batch stores NaN for a rollout that diverged) gets
 * weight 0, the limit of Eq. 25 as its cost grows without bound. If no cost is finite every
 * weight is NaN. Errors: VPM_ERR_INVALID (K < 1, lambda <= 0).
 */
vpm_status mppi_weights(const float *d_costs, int K, float lambda, float *d_weights,
                        cudaStream_t stream);

/* Reweighted control sequence of Eq. 25: d_mu[k] = sum_i d_weights[i] d_controls[i*H + k]
 * (binary64 sums, fixed order). */
vpm_status mppi_update(const float *d_weights, const float *d_controls, int K, int H,
                       float *d_mu, cudaStream_t stream);

/* Sampled control sequences xi_i = mu + eps_i (§IV-A): d_controls[i*H + k] =
 * d_mu[k] + d_eps[i*H + k]. The noise is an input so that it can be drawn anywhere. */
vpm_status mppi_perturb(const float *d_mu, const float *d_eps, int K, int H,
                        float *d_controls, cudaStream_t stream);

/*
 * Free-field velocities (Eq. 3 with the chosen kernel, self term excluded) of n particles
 * d_particles[n*4] = (x, z, Gamma, unused) binary32; d_vel[n*2] receives (u, w). Binary32
 * pair sums, compensated across source tiles. One evaluation of each particle pair serves both
 * particles; every particle's partial sums are added exactly into a fixed-point accumulator per
 * velocity component (a 128-bit integer held as three 64-bit digit words), so the result does
 * not depend on the order in which the partial sums arrive. The call allocates
 * vpm_freefield_scratch_bytes(n) bytes (48 n + 64) of device scratch on `stream` from the
 * library's memory pool and frees it after it (stream-ordered). Non-finite input gives NaN
 * velocities. Errors: VPM_ERR_INVALID, VPM_ERR_CAPACITY (n > 2^30, where the digit words could
 * overflow), VPM_ERR_CUDA (including an allocation that does not fit).
 */
vpm_status vpm_freefield_velocity(const float *d_particles, int n, int kernel, double r_core,
                                  float *d_vel, cudaStream_t stream);

/* Device bytes of scratch one free-field velocity evaluation of n particles uses: two
 * accumulators of three 64-bit words per particle and the call's scale (48 n + 64; 0 for
 * n = 0). Errors: VPM_ERR_INVALID (n < 0, null). */
vpm_status vpm_freefield_scratch_bytes(int n, size_t *bytes);

/*
 * `steps` Heun (explicit trapezoidal RK2) steps of a free field in place:
 * v1 = V(r), r* = r + dt v1, v2 = V(r*), r <- r + dt (v1 + v2) / 2. d_particles as above.
 * Uses 24 n bytes plus vpm_freefield_scratch_bytes(n) bytes of library-allocated scratch
 * (stream-ordered allocation); vpm_freefield_heun_noalloc allocates nothing. n <= 2^30
 * (VPM_ERR_CAPACITY beyond).
 */
vpm_status vpm_freefield_heun(float *d_particles, int n, int kernel, double r_core, double dt,
                              int steps, cudaStream_t stream);

/*
 * The library's stream-ordered scratch (rollout pair sums, pacing tables, free-field
 * accumulators, serving buffers) comes from a memory pool of its own on each device, separate
 * from the device's default pool, which it leaves untouched. Freed scratch stays reserved in
 * that pool for the library's next launches. vpm_pool_trim gives the current device's reserved,
 * unused pool memory back to the device (memory still in use is not affected) and writes the
 * bytes the pool still holds to *bytes_held if non-null. Errors: VPM_ERR_CUDA.
 */
vpm_status vpm_pool_trim(size_t *bytes_held);

/*
 * Host-only checks of the free-field accumulators (no device needed; the paper has no
 * counterpart). vpm_fixed_sum converts h_v[count] to fixed point with unit 2^-e, splits each into
 * the kernels' digits (bits 0-41, 42-83, 84-127 of the 128-bit integer, signed), adds them word by
 * word in the given order as the kernels' 64-bit reductions do, combines the three words into the
 * 128-bit total and returns it as a double in *h_sum (*h_bad = 1 if a value was NaN or infinite). vpm_fixed_exponent gives the e the kernels use for n particles whose
 * largest |Gamma| is gmax: with B = n gmax kappa (kappa = 1 / r_core for the regularised kernels,
 * 2^40 for the singular one) and B < 2^eb, e = 125 - eb. Errors: VPM_ERR_INVALID.
 */
vpm_status vpm_fixed_sum(const float *h_v, int count, int e, double *h_sum, int *h_bad);
vpm_status vpm_fixed_exponent(float gmax, int n, int kernel, double r_core, int *h_e);

/* ------------------------------------------------------------------ uneven batches
 * Rollouts from many different roots at once: the MPPI step of §IV-A applied to R scenarios
 * whose fields have different particle counts (one rollout per root). Roots are grouped by
 * the shared memory their fields can need into classes; each class runs as one persistent
 * launch (blocks claim rollouts largest-first) on its own stream, forked from and joined back
 * into the caller's stream, or, if the autotuner finds it faster, all rollouts run in one
 * persistent launch sized for the largest field. A rollout's result does not depend on the
 * class, the block size, the diagonal-unit size or the order of execution.
 */
typedef struct vpm_batch vpm_batch;

/*
 * Creates a batch of R roots: h_counts[R] particle counts, h_particles the concatenated fields
 * (sum of counts x 3, binary64 x, z, Gamma in root order), h_gliders[R x 7] glider states.
 * max_horizon bounds the H of later rollouts (capacities are counts + 2 max_horizon).
 * Synchronises `stream`. Errors: VPM_ERR_INVALID, VPM_ERR_NONFINITE, VPM_ERR_CAPACITY (a field
 * would not fit one block's shared memory: about 9300 particles on the binary32 path, 4500 on
 * the binary64 path), VPM_ERR_OOM, VPM_ERR_CUDA.
 */
vpm_status vpm_batch_create(const vpm_params *params, int R, const int *h_counts,
                            const double *h_particles, const double *h_gliders, int max_horizon,
                            vpm_batch **out, cudaStream_t stream);

vpm_status vpm_batch_destroy(vpm_batch *batch);

/*
 * One rollout of H steps per root under d_controls[R x H]; d_costs[R] receives the terminal
 * costs (Eq. 24), d_count[R] (or null) the final particle counts, d_final_glider[R x 7] (or
 * null) the final glider states. With use_graph = 1 the class launches of this (H, buffers)
 * combination are captured once into a CUDA graph on a library stream and replayed on
 * `stream` afterwards; changing H or a buffer recaptures.
 */
vpm_status vpm_batch_rollout(vpm_batch *batch, int H, const float *d_controls, float *d_costs,
                             int *d_count, double *d_final_glider, int use_graph,
                             cudaStream_t stream);

/*
 * Autotuner over the launch shape. Each class, and the merged class that runs every rollout in
 * one persistent launch sized for the largest field, is timed alone over min(H, 3) steps for
 * each block size that fits (128, 256, 512 threads) and each diagonal pair-unit size (32, 64 or
 * 128 targets, i.e. 1, 2 or 4 per lane; Vatistas kernel only, others keep 2), keeping its
 * fastest. A class whose fields can exceed 2300 particles (Vatistas kernel) is then timed at
 * that shape with each rollout spread over a thread-block cluster of 2 and of 4 CTAs (every CTA
 * holds the field; the step's pair units are split between them and the advected records are
 * exchanged through distributed shared memory), and keeps the fastest of 1, 2 and 4 CTAs per
 * rollout; cluster choices are kept only if the whole batch of class launches runs faster with
 * them than with one CTA per rollout (a class alone can leave SMs idle that clusters fill; side
 * by side the classes fill the GPU anyway). Then the whole batch is timed as the class launches
 * side by side and as the one merged launch, each over the whole horizon H as a captured CUDA
 * graph (median of three replays), and the faster is kept. It
 * changes speed only, never results. Synchronises `stream`.
 */
vpm_status vpm_batch_tune(vpm_batch *batch, int H, const float *d_controls, cudaStream_t stream);

/* The schedule: the number of launches it runs and, per launch, the capacity, threads per
 * block, number of rollouts, tuned time (ms, 0 before tuning), targets per lane of the
 * diagonal pair units and CTAs per rollout (any output array may be null; arrays hold up to 5
 * entries); *h_merged (if non-null) is 1 when all rollouts run in one launch. */
vpm_status vpm_batch_schedule(const vpm_batch *batch, int *h_nclasses, int *h_cap, int *h_nt,
                              int *h_items, float *h_tuned_ms, int *h_diag_t, int *h_ctas,
                              int *h_merged);

/* The tuner's times (ms, H steps of the whole batch, graph replay) of the class launches side by side
 * and of the one merged launch (0 before tuning or with a single class). */
vpm_status vpm_batch_tuned_modes(const vpm_batch *batch, float *h_split_ms, float *h_merged_ms);

/* Sets the schedule by hand: merged = 1 selects the one-launch schedule, then launch `cls` of
 * that schedule (as vpm_batch_schedule lists them) gets nt threads (128, 256, 512) and diag_t
 * targets per lane (1, 2, 4; 2 unless the wake kernel is Vatistas; binary64 batches: 128 and
 * 2). Results do not depend on it. Errors: VPM_ERR_INVALID (a size that does not fit). */
vpm_status vpm_batch_set_schedule(vpm_batch *batch, int merged, int cls, int nt, int diag_t);

/* Sets CTAs per rollout by hand for launch `cls` of the schedule selected by `merged` (as in
 * vpm_batch_set_schedule): 1, or a cluster of 2 or 4 CTAs per rollout (binary32 batches with the
 * Vatistas kernel of Eq. 5 only), keeping the launch's threads and diagonal-unit size. The
 * batch rollout over a cluster is the same computation as on one CTA (§III-A steps; Eq. 16's
 * pair sums split between the CTAs by unit), so results are the same bits. Errors:
 * VPM_ERR_INVALID (another count, another precision or kernel, or a cluster that does not fit
 * the launch's shared memory and threads). */
vpm_status vpm_batch_set_ctas(vpm_batch *batch, int merged, int cls, int ctas);

/* Reads and clears the batch's device error word (synchronises `stream`). */
vpm_status vpm_batch_status(vpm_batch *batch, cudaStream_t stream);

/* ------------------------------------------------------------------ replanning server
 * Serves replanning requests (§IV-C: re-running the MPPI iteration of §IV-A from each
 * scenario's current vortex state) from many scenarios at once. Each scenario's field stays
 * resident on the device between requests. A worker thread admits queued requests (in arrival
 * order, or least estimated work first: vpm_server_config.policy) whenever a slot is free, the
 * scenario has nothing on the device, and the request's device buffers fit the memory budget;
 * admitted requests run on their own streams and overlap on the GPU. A newer request for a scenario supersedes its older request still in the queue
 * (that one completes with VPM_ERR_BUSY). Results do not depend on what else runs.
 */
typedef struct vpm_server vpm_server;

typedef struct {
    int max_inflight;     /* requests on the device at once; 1 gives the plain per-request form */
    size_t hbm_budget;    /* cap on the device bytes of requests in flight; 0: no cap. Either
                             way a request is admitted only while the device has its bytes free
                             at that moment (cudaMemGetInfo plus the library pool's idle memory,
                             less a reserve of max(1 GiB, 2 % of device memory)), so memory other
                             code takes after the server was made delays admission              */
    int max_rollouts;     /* largest K accepted                                                 */
    int max_horizon;      /* largest H accepted                                                 */
    int max_inflight_rollouts;  /* rollouts on the device at once; a request is admitted while the
                                   total stays within it or when nothing else runs. 0: the rollout
                                   blocks the device holds at once (SMs x 7), beyond which more
                                   concurrency only adds latency                                */
    int policy;           /* admission order: VPM_ADMIT_ARRIVAL (0) admits queued requests in
                             arrival order; VPM_ADMIT_LEAST_WORK (1) admits, among the queued
                             requests whose scenario is idle and whose bytes fit, the one with the
                             fewest estimated pair interactions (K H n^2, n the scenario's
                             particle count at mid-horizon) first                              */
    double max_wait_ms;   /* with VPM_ADMIT_LEAST_WORK: a request queued longer than this is
                             admitted first, in arrival order (<= 0: no such bound)              */
    int small_rollouts;   /* with VPM_ADMIT_LEAST_WORK: requests of at most this many rollouts
                             take a lane of their own, admitted while that lane's rollouts stay
                             within max_inflight_rollouts whatever the other requests hold, on
                             streams of the highest priority, so that their blocks start ahead of
                             the waiting blocks of larger launches. 0: no such lane              */
} vpm_server_config;

enum { VPM_ADMIT_ARRIVAL = 0, VPM_ADMIT_LEAST_WORK = 1 };

typedef struct {
    int status;           /* VPM_OK, VPM_ERR_BUSY (superseded), or the error that stopped it     */
    int scenario, K, H;
    double t_submit_ms, t_start_ms, t_done_ms;   /* host clock, ms since the server was created   */
    float j_min;          /* smallest rollout cost of the iteration                              */
} vpm_server_result;

vpm_status vpm_server_create(const vpm_server_config *cfg, vpm_server **out);

/* Adds a scenario with a resident field (as vpm_state_create, default stream); *scenario
 * receives its index. */
vpm_status vpm_server_add_scenario(vpm_server *server, const vpm_params *params,
                                   const double *h_particles, int n, int capacity,
                                   const double *h_glider7, int *scenario);

/*
 * Queues one MPPI iteration on a scenario: controls h_mu[H] (null: zeros) plus noise
 * h_eps[K x H] (both copied before return), temperature lambda; before the rollouts the
 * scenario's field is advanced by advance_steps committed steps at elevator rate advance_u.
 * *ticket identifies the request. Errors: VPM_ERR_INVALID, VPM_ERR_CAPACITY (the request can
 * never fit the memory budget).
 */
vpm_status vpm_server_submit(vpm_server *server, int scenario, int K, int H, const float *h_mu,
                             const float *h_eps, float lambda, int advance_steps,
                             float advance_u, long long *ticket);

/* Waits up to timeout_ms (-1: forever, 0: no wait) for a request; on completion fills *out and
 * h_mu_out[H] (the reweighted controls, if non-null) and forgets the ticket. Returns
 * VPM_ERR_BUSY (not done, no wait) or VPM_ERR_TIMEOUT when it is not done yet. */
vpm_status vpm_server_poll(vpm_server *server, long long ticket, int timeout_ms,
                           vpm_server_result *out, float *h_mu_out);

/* Device bytes that admission counts for a request of K rollouts over H steps on `scenario`
 * taken after advance_steps committed steps: its own buffers (noise, controls, costs, weights,
 * reweighted controls) plus the rollouts' pair-sum scratch (vpm_rollout_scratch_bytes). */
vpm_status vpm_server_request_bytes(vpm_server *server, int scenario, int K, int H,
                                    int advance_steps, size_t *bytes);

/* Rollouts completed so far, requests queued, requests and bytes on the device. */
vpm_status vpm_server_stats(vpm_server *server, long long *completed_rollouts, int *queued,
                            int *in_flight, size_t *in_flight_bytes);

/* Copies a scenario's resident field and glider state to the host once it is idle
 * (h_particles must hold its capacity x 3 values). */
vpm_status vpm_server_read_scenario(vpm_server *server, int scenario, double *h_particles,
                                    int *n_out, double *h_glider7);

/* Stops the worker, waits for the device, frees everything. */
vpm_status vpm_server_destroy(vpm_server *server);

/*
 * The same Heun steps as vpm_freefield_heun for callers that must not let the library
 * allocate device memory, such as a control loop whose memory is fixed before it starts or a
 * host that gives all device memory to another owner. It evaluates every pair once per target
 * (vpm_freefield_heun evaluates each pair once for both particles and adds the partial sums into
 * exact accumulators), so the two agree to binary32 rounding, not bit for bit. The paper has no counterpart; it is a
 * deployment variant. Its scratch is one device array of fixed size built into the library
 * (6 MiB, held on every device where it has been taken until the process exits), so n is
 * limited to 262144 particles; larger n returns VPM_ERR_CAPACITY without launching anything.
 * Every call looks up that array's device address (cudaGetSymbolAddress) with the caller's
 * device current. CUDA loads a library's device code lazily by default, so the array's 6 MiB
 * are taken from the device on the first call on that device (n >= 1 and steps >= 1; calls
 * with n = 0 or steps = 0 return before the lookup), and that first call can fail with
 * VPM_ERR_CUDA if other owners already hold all device memory. Make one such warm-up call
 * (n = 1, steps = 1 is enough) before fixing the process's memory, handing device memory to
 * another owner, or capturing the stream into a graph. Every call on a device uses the same
 * array: calls whose work overlaps on the GPU (other streams, other host threads) race on it
 * and must be serialised by the caller. Nothing in the array needs clearing between calls:
 * each step writes it fully before reading it. No cudaMalloc, cudaFree or other allocating
 * routine is called.
 */
vpm_status vpm_freefield_heun_noalloc(float *d_particles, int n, int kernel, double r_core,
                                      double dt, int steps, cudaStream_t stream);

/*
 * Feedback NMPC of §IV-C over a manoeuvre of `horizon` steps. A tracking instance of the model
 * (created from h_particles, h_x0) follows the observed glider state. The first control call
 * plans from the tracking instance (with any pair injected before it); then every `replan_every` steps (t > 0, t + latency < horizon, while
 * draws remain) a plan starts from a copy of the tracking instance with the observed glider
 * state, projected `latency` steps ahead under the current policy. A plan is `iterations` MPPI
 * reweightings (Eq. 25) of `rollouts` rollouts over the remaining steps, warm-started from the
 * previous nominal controls, and the least-squares / TVLQR synthesis (§IV-B) around the new
 * nominal; its policy takes effect `latency` steps after the replan started, before a replan
 * due at that same step begins (so that replan projects under the new policy).
 * threaded = 0: the plan runs inside vpm_nmpc_control (deterministic);
 * threaded = 1: a planning thread with its own stream runs it while control continues (the
 *               two-thread split of §IV-C); a replan that falls due while the planner is still
 *               busy is skipped.
 */
typedef struct {
    int horizon;          /* N: steps of the manoeuvre */
    int replan_every;     /* P: steps between replans */
    int latency;          /* L: projection steps (the replanning time), 0 <= L <= P
                             (a longer latency would replace a plan before it took effect;
                             VPM_ERR_INVALID) */
    int rollouts;         /* K: MPPI and synthesis rollouts per plan (>= 6) */
    int iterations;       /* MPPI iterations per plan */
    float lambda;         /* MPPI temperature */
    double qc[7], qf[7];  /* TVLQR weights (diagonals) */
    double rc;            /* TVLQR control weight */
    int threaded;
} vpm_nmpc_config;

typedef struct vpm_nmpc vpm_nmpc;

/*
 * Random draws are inputs (host arrays, copied): for plan p < n_plans (plan 0 is the initial
 * one), MPPI perturbations h_eps[p][iterations][rollouts][horizon] (binary32; a plan from step t0
 * uses the first horizon - t0 columns), synthesis initial-state perturbations
 * h_xi[p][rollouts][7] and control perturbations h_zeta[p][rollouts][horizon] (binary32).
 * h_mu0[horizon]: initial nominal controls. The model's precision is params->precision.
 * Errors: VPM_ERR_INVALID (null, horizon < 2, rollouts < 6, lambda or rc <= 0, ...), those of
 * vpm_state_create, VPM_ERR_SINGULAR (a least-squares step singular), VPM_ERR_OOM,
 * VPM_ERR_CUDA.
 */
vpm_status vpm_nmpc_create(const vpm_nmpc_config *cfg, const vpm_params *params,
                           const double *h_particles, int n, int capacity, const double *h_x0,
                           const float *h_mu0, int n_plans, const float *h_eps,
                           const double *h_xi, const float *h_zeta, vpm_nmpc **out);

/*
 * Control step t (0 <= t < horizon, called in order) with the observed glider state h_x_obs[7]:
 * starts a replan if one is due, installs a finished plan whose first step has come, writes the
 * control *h_u = ubar_t - H_t (x_obs - xbar_t), and advances the tracking instance by one step
 * under it from the observed state. Errors: VPM_ERR_INVALID, and any error of a plan.
 */
vpm_status vpm_nmpc_control(vpm_nmpc *nmpc, int t, const double *h_x_obs, double *h_u);

/* Puts a disturbance pair (see vpm_state_inject_pair) into the tracking instance: plans started
 * afterwards account for it (the compensated case of §V). */
vpm_status vpm_nmpc_inject_pair(vpm_nmpc *nmpc, const double *h_pair);

/* The policy in effect: its first step *t0 (-1 before the first control call), h_gains[horizon*7]
 * and h_ubar[horizon] by absolute step, h_xbar[(horizon+1)*7] (rows before t0 unused). Any
 * pointer may be null. */
vpm_status vpm_nmpc_policy(vpm_nmpc *nmpc, int *t0, double *h_gains, double *h_xbar,
                           float *h_ubar);

/* Plans finished (the initial one included), replans skipped while the planner was busy, and the
 * wall time of the last and the longest replan (projection + MPPI + synthesis) in ms. */
vpm_status vpm_nmpc_stats(vpm_nmpc *nmpc, int *plans_done, int *plans_skipped,
                          double *last_plan_ms, double *max_plan_ms);

/* Stops the planner, waits for the device, frees everything. */
vpm_status vpm_nmpc_destroy(vpm_nmpc *nmpc);

/*
 * Throughput probe. The paper has no counterpart: it is a measurement aid that states, from
 * this device, the ceiling the pair kernels run against. One timed launch of blocks_per_sm x
 * (SM count) blocks of 128 threads writes to *h_rate:
 *   VPM_PROBE_FFMA      binary32 fused multiply-adds per second (lane operations),
 *   VPM_PROBE_RSQRT     MUFU reciprocal square roots per second,
 *   VPM_PROBE_EX2       MUFU base-2 exponentials per second,
 *   VPM_PROBE_PAIRS_T1/T2/T4  pair interactions per second of the rollout kernel's binary32
 *                       pair loop (Vatistas kernel) with 1, 2 or 4 targets per lane, every block
 *                       summing a 1024-particle field held in its shared memory, every pair
 *                       evaluated once per target;
 *   VPM_PROBE_PAIRS_SYM pair interactions per second (n^2 per field) of the rollout kernel's
 *                       binary32 pair phase as it runs: one evaluation per particle pair across
 *                       128-particle rows, diagonal groups, partial sums combined per particle.
 * blocks_per_sm must lie in 1..7. The call allocates and frees its own device scratch, runs on
 * the legacy default stream of the current device and synchronises it. Errors:
 * VPM_ERR_INVALID for an unknown probe or block count, VPM_ERR_CUDA for a CUDA failure.
 */
typedef enum {
    VPM_PROBE_FFMA = 0,
    VPM_PROBE_RSQRT = 1,
    VPM_PROBE_EX2 = 2,
    VPM_PROBE_PAIRS_T1 = 3,
    VPM_PROBE_PAIRS_T2 = 4,
    VPM_PROBE_PAIRS_T4 = 5,
    VPM_PROBE_PAIRS_SYM = 6
} vpm_probe;

vpm_status vpm_probe_rate(int probe, int blocks_per_sm, double *h_rate);

#ifdef __cplusplus
}
#endif
#endif /* VPM_H */
