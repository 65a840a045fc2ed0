/*
 * wave.h -- C ABI of the GB300 time-tiled acoustic wave library (libwavetile).
 *
 * The library solves the isotropic acoustic wave equation
 *
 *     m u_tt + damp u_t - lap u = f            (m = 1/v^2, km, s units)
 *
 * on a 3D grid with leapfrog time stepping and an order-`space_order` central
 * Laplacian (radius r = space_order/2), point sources injected and receivers
 * interpolated every step.  The paper it follows (N. Sim, "Optimising finite-
 * difference methods for PDEs through parameterised time-tiling in Devito",
 * 2018) tiles this sweep in time: Sec. 4.1 skews space by the stencil radius
 * per time step, Sec. 4.2 tiles the skewed space-time, Sec. 5.8 applies it to
 * the acoustic operator at space orders 4..16.  The paper states no
 * discretisation; the one implemented here is:
 *
 *   u^{n+1} = u^n + B (u^n - u^{n-1}) + C (L u^n + f^n)
 *     B = (m - eta)/(m + eta),  C = dt^2/(m + eta),  eta = damp dt / 2
 *   which is the centred-damping leapfrog  m(u^{n+1}-2u^n+u^{n-1})/dt^2
 *   + damp(u^{n+1}-u^{n-1})/(2 dt) - L u^n = f^n  solved for u^{n+1};
 *   L u = sum_a h_a^-2 [c_0 u + sum_{k=1..r} c_k (u(+k e_a) + u(-k e_a))],
 *   u = 0 outside the grid, u^0 = u^{-1} = 0;
 *   f^n[p] = sum_s w_{s,p} q_s^n (trilinear weights over the 8 corners of the
 *   cell holding source s, no 1/h^3 factor);
 *   d^n[r] = sum_p w_{r,p} u^{n+1}[p]   (receivers record the new level).
 *
 * Conventions for every entry point
 *   - Arrays are float32, C order [nx][ny][nz] (z contiguous), as in the
 *     paper's generated code (Sec. 3.2.1).  Traces are [nt][npts].
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory, read during the call only.
 *   - The library never allocates device memory.  The caller passes a device
 *     workspace of at least wave_workspace_bytes(...) bytes (256-byte aligned)
 *     that the call may overwrite; it must not be shared by calls that can
 *     overlap on the GPU.
 *   - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and return without waiting, except the first call for a new
 *     problem shape with tuning.time_tile == 0, which times candidate tilings
 *     on `stream` before it returns.  wave_status() waits for the stream and
 *     reports device-side errors recorded in the workspace.
 *   - Return value: WAVE_OK or a negative WAVE_E* code; nothing is enqueued
 *     when an argument check fails.  No C++ exception crosses the ABI.
 */
#ifndef WAVETILE_WAVE_H
#define WAVETILE_WAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WAVE_OK 0
#define WAVE_EINVAL (-1)      /* bad argument: space order, shape, pointer, point outside grid */
#define WAVE_EUNSTABLE (-2)   /* dt above the von Neumann limit (see wave_cfl_dt)             */
#define WAVE_ECUDA (-3)       /* a CUDA runtime call failed                                  */
#define WAVE_ETIMEOUT (-4)    /* a bounded device-side wait gave up                           */
#define WAVE_ENOSPACE (-5)    /* workspace smaller than wave_workspace_bytes()                */
#define WAVE_EUNSUPPORTED (-6)/* requested tiling not compiled into this library              */

/* wave_workspace_bytes `op` values */
#define WAVE_OP_FWD 0
#define WAVE_OP_ADJ 1
#define WAVE_OP_GRAD 2
#define WAVE_OP_REVOLVE 3 /* wave_grad_revolve; the ckpt_every argument is nslots */
#define WAVE_OP_BORN 4    /* wave_born */

/* wave_tuning.flags */
#define WAVE_ALLOW_UNSTABLE 1 /* skip the dt <= CFL check                              */
#define WAVE_TIME_SWEEPS 2    /* record CUDA events around the sweep launches of the call
                                 (read back with wave_sweep_stats)                       */
#define WAVE_AUTOTUNE_SHAPE 4 /* with time_tile = T >= 1: time the compiled variants of
                                 depth T (tile, vec, x-chunk) and keep the fastest       */
#define WAVE_BORN_TWO_SWEEPS 8 /* wave_born: the background and perturbation sweeps as two
                                 launches per step (the form of every order) instead of
                                 the fused sweep                                        */
#define WAVE_TEST_WITHHOLD 256 /* test hook: the sweep's producer issues no loads, so
                                 every bounded wait of the call runs out (about 2 s per
                                 launch) and wave_status reports WAVE_ETIMEOUT; the
                                 CUDA context stays usable.  Results are undefined.     */

typedef struct wave_grid {
    int32_t n[3];        /* nx, ny, nz >= space_order + 1 each; ny * nz < 2^31      */
    float h[3];          /* grid spacing per axis (km), > 0                          */
    float dt;            /* time step (s), > 0                                       */
    int32_t nt;          /* number of time steps, >= 1                               */
    int32_t space_order; /* even, 2..16 (paper: 4, 6, 8, 12, 16, Sec. 5.8.1)         */
} wave_grid;

typedef struct wave_points {
    int32_t npts;        /* number of points, >= 0                                   */
    const float *xyz;    /* HOST, [npts][3] physical coordinates (km) inside
                            [0, (n_a - 1) h_a] on every axis                         */
} wave_points;

/* Sweep configuration.  Zero fields mean "choose automatically".
 *   time_tile : 0 = autotune, 1 = untiled sweep (one step per launch),
 *               T >= 2 = T steps per launch (time-tile depth, Sec. 4.2).
 *   tile_y    : output rows per block (0 = any compiled variant).
 *   tile_x    : x-chunk length streamed by one block (0 = default).
 *   vec       : z points per thread, 2, 4 or 8 (0 = any compiled variant).
 *   flags     : WAVE_ALLOW_UNSTABLE | WAVE_TIME_SWEEPS | WAVE_AUTOTUNE_SHAPE.
 *   tile_z    : output columns per block (0 = the first compiled variant
 *               matching the other fields).
 *   kernel    : sweep kernel family (0 = any): WAVE_KERNEL_SHARED, every time
 *               step of a tile on the same warps; WAVE_KERNEL_STAGED, each
 *               time step of a tile on its own warps (T = 1 or 2).  All
 *               families and shapes give bitwise the same results.
 *   rows      : output rows per thread (0 = any; the shared family has 1). */
typedef struct wave_tuning {
    int32_t time_tile;
    int32_t tile_y;
    int32_t tile_x;
    int32_t vec;
    int32_t flags;
    int32_t tile_z;
    int32_t kernel;
    int32_t rows;
} wave_tuning;

#define WAVE_KERNEL_SHARED 1 /* wave_tuning.kernel: stages of a time tile share warps */
#define WAVE_KERNEL_STAGED 2 /* wave_tuning.kernel: one group of warps per stage      */

/* Library version (major*10000 + minor*100 + patch). */
int32_t wave_version(void);

/* Message for a WAVE_* code; never NULL, static storage. */
const char *wave_strerror(int32_t code);

/* Stencil coefficients c_0..c_r (unit spacing) of the order-`space_order`
 * central second derivative, c_k = 2(-1)^(k+1)(r!)^2 / (k^2 (r-k)! (r+k)!),
 * c_0 = -2 sum_{k>=1} c_k.  The paper derives its stencils from Taylor's
 * theorem (Sec. 2.1).  c_out (HOST) receives space_order/2 + 1 doubles.
 * Returns WAVE_OK or WAVE_EINVAL. */
int32_t wave_fd_coefficients(int32_t space_order, double *c_out);

/* Largest stable dt of the undamped scheme (von Neumann, periodic):
 *   dt = 2 / (v_max sqrt(sum_a S / h_a^2)),  S = |c_0 + 2 sum_k (-1)^k c_k|.
 * Returns a negative value on bad arguments. */
double wave_cfl_dt(int32_t space_order, const float *h /* HOST [3] */, float v_max);

/* Device workspace needed by one call of operation `op` (WAVE_OP_*).
 * nsrc/nrec are the source and receiver counts of that call; ckpt_every is
 * the checkpoint interval k for WAVE_OP_GRAD (and ignored otherwise).
 * tuning may be NULL.  Returns 0 for invalid arguments. */
size_t wave_workspace_bytes(const wave_grid *g, int32_t op, int32_t nsrc, int32_t nrec,
                            int32_t ckpt_every, const wave_tuning *tuning);

/* Size in bytes of the checkpoint buffer that wave_fwd fills and wave_grad
 * reads: ceil(nt / ckpt_every) states of two levels each, in the library's
 * internal (z-padded) layout.  Returns 0 on invalid arguments. */
size_t wave_ckpt_bytes(const wave_grid *g, int32_t ckpt_every);

/* Forward modelling (Sec. 5.8: the acoustic operator, with the source and
 * receiver loops of Sec. 4.5.1 fused into the time-tiled sweep).
 *   m, damp      device [nx][ny][nz]; m > 0 (s^2/km^2), damp >= 0 (1/s)
 *   src          host points; src_traces device [nt][nsrc] (q_s^n), may be
 *                NULL when nsrc == 0
 *   rec          host points; rec_traces device [nt][nrec] out (d^n), may be
 *                NULL when nrec == 0
 *   u_last       device [2][nx][ny][nz] out (u^nt, u^{nt-1}) or NULL
 *   ckpt         device, wave_ckpt_bytes(g, ckpt_every) bytes out, or NULL;
 *                state c holds (u^{c k}, u^{c k - 1})
 *   ckpt_every   k >= 1 when ckpt != NULL
 *   tuning       NULL = autotune
 *   ws, ws_bytes device workspace (WAVE_OP_FWD)
 *   stream       cudaStream_t
 * The time-tiled and untiled sweeps give bitwise identical results. */
int32_t wave_fwd(const wave_grid *g, const float *m, const float *damp,
                 const wave_points *src, const float *src_traces,
                 const wave_points *rec, float *rec_traces,
                 float *u_last, float *ckpt, int32_t ckpt_every,
                 const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream);

/* Adjoint modelling: the transpose of wave_fwd's source-to-receiver map.
 * With a residual res = dJ/dd (device [nt][nrec]) it returns
 *   src_adj  device [nt][nsrc] out: dJ/dq_s^n = sum_p w_{s,p} nu^{n+1}[p]
 *   v_last   device [2][nx][ny][nz] out (nu^1, nu^2) or NULL,
 * where nu^k = C lambda^k and lambda^k = dJ/du^k.  nu obeys the forward
 * scheme run backwards in time with res injected at the receivers, which is
 * how it is computed (the same time-tiled sweep).  Workspace: WAVE_OP_ADJ. */
int32_t wave_adj(const wave_grid *g, const float *m, const float *damp,
                 const wave_points *rec, const float *rec_resid,
                 const wave_points *src, float *src_adj, float *v_last,
                 const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream);

/* Gradient of J with respect to m for a fixed residual res = dJ/dd:
 *   grad = dJ/dm = -(1/dt^2) sum_{n=0}^{nt-1} nu^{n+1} (u^{n+1} - 2u^n + u^{n-1})
 * (device [nx][ny][nz] out, overwritten).  u comes from the checkpoints of a
 * previous wave_fwd call with the same grid, m, damp, sources and ckpt_every:
 * each segment of ckpt_every steps is recomputed from its checkpoint with the
 * second difference stored per step, then the adjoint sweep of that segment
 * accumulates the imaging condition.  Workspace: WAVE_OP_GRAD.
 * The recompute and adjoint sweeps each run on the compiled shape measured
 * fastest for that phase on this grid (a few steps of every candidate, once
 * per grid, forward plan and point counts); every shape gives the same bits.
 * Test hook: the environment variable WAVE_GRAD_PIN="i,j" makes this call
 * (and wave_grad_revolve) run recompute candidate i and adjoint candidate j
 * untimed, and return WAVE_EUNSUPPORTED when either index is past the end. */
int32_t wave_grad(const wave_grid *g, const float *m, const float *damp,
                  const wave_points *src, const float *src_traces,
                  const wave_points *rec, const float *rec_resid,
                  const float *ckpt, int32_t ckpt_every, float *grad,
                  const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream);

/* The same gradient as wave_grad, without a previous wave_fwd: binomial
 * checkpointing (revolve; A. Griewank, Optim. Methods Softw. 1, 1992;
 * A. Griewank and A. Walther, ACM TOMS 26, 2000) reverses the nt steps with
 * nslots stored states (0 <= nslots <= nt) in the workspace.  The paper uses
 * uniform checkpoints; this schedule needs far less memory for long runs at
 * the price of recomputed forward steps, the fewest possible for nslots
 * states: wave_revolve_forward_steps(nt, nslots) of them in all, counting
 * the recomputation inside each reversed step (2 nt - 1 when nslots >=
 * nt - 1, as wave_fwd plus wave_grad less one; nt (nt + 1) / 2 with
 * nslots = 0).  Each reversed step n
 * recomputes u^{n+1} from a restored or current state with D^n stored, then
 * runs the adjoint step of n with the imaging condition, so the result is
 * wave_grad's, bit for bit, for any checkpoint interval.  Arguments as
 * wave_grad; workspace: wave_workspace_bytes(g, WAVE_OP_REVOLVE, nsrc, nrec,
 * nslots, tuning). */
int32_t wave_grad_revolve(const wave_grid *g, const float *m, const float *damp,
                          const wave_points *src, const float *src_traces,
                          const wave_points *rec, const float *rec_resid, int32_t nslots,
                          float *grad, const wave_tuning *tuning, void *ws, size_t ws_bytes,
                          void *stream);

/* Born (linearised) modelling: the derivative of the receiver traces of
 * wave_fwd with respect to m in the direction dm (not in the paper; the
 * linearisation of its scheme).  With D^n = u^{n+1} - 2u^n + u^{n-1} of the
 * background wavefield u (sources as wave_fwd) and alpha = 1 / (m + eta),
 *   du^{n+1} = alpha (2 m du^n - (m - eta) du^{n-1} + dt^2 L du^n) - alpha dm D^n,
 *   du^0 = du^-1 = 0,   rec_traces[n][r] = sum_p w_{r,p} du^{n+1}[p].
 * Its adjoint is wave_grad: <born(dm), r> = <dm, grad(r)>.  Each step
 * advances both fields in one fused sweep (where compiled for the order):
 * the background with D^n kept in registers, the perturbation adding
 * C (P D^n) with P = -dm / dt^2 (C = alpha dt^2) to its new level, reading
 * u^n, u^{n-1}, du^n, du^{n-1}, B, C, E, P and writing two levels (40 B per
 * point-update).  With WAVE_BORN_TWO_SWEEPS, or at an order without the
 * fused sweep, the background sweep stores D^n and a second sweep runs the
 * perturbation (56 B); both forms give the same bits.
 *   m, damp, dm  device [nx][ny][nz]
 *   src / src_traces, rec   as wave_fwd
 *   rec_traces   device [nt][nrec] out (linearised data)
 *   du_last      device [2][nx][ny][nz] out (du^nt, du^{nt-1}), or NULL
 *   tuning       as wave_fwd: the plan of the background sweep; the
 *                perturbation sweep runs the one untiled variant of its order
 *   ws, ws_bytes wave_workspace_bytes(g, WAVE_OP_BORN, nsrc, nrec, 0, tuning)
 * Returns WAVE_OK or a WAVE_E* code; device status as wave_fwd. */
int32_t wave_born(const wave_grid *g, const float *m, const float *damp, const float *dm,
                  const wave_points *src, const float *src_traces, const wave_points *rec,
                  float *rec_traces, float *du_last, const wave_tuning *tuning, void *ws,
                  size_t ws_bytes, void *stream);

/* Forward steps (recomputations included, one per reversed step) of the
 * schedule wave_grad_revolve runs for nt steps and nslots states, or -1 for
 * invalid arguments.  Host only. */
int64_t wave_revolve_forward_steps(int32_t nt, int32_t nslots);

/* The schedule itself, host only: returns the number of actions and writes
 * the first min(cap, count) as (kind, a, b) triples into actions (HOST):
 *   0 ADVANCE a b   forward from the current state (step a) to step b
 *   1 TAKESHOT a k  store the current state (step a) in slot k
 *   2 RESTORE a k   make the state of step a in slot k current (k = -1: the
 *                   zero initial state of step 0)
 *   3 YOUTURN a 0   one forward step from the current state (step a) storing
 *                   D^a, then the adjoint step of time index a
 * The run starts with the zero state of step 0 current.  WAVE_EINVAL for
 * invalid arguments. */
int32_t wave_revolve_schedule(int32_t nt, int32_t nslots, int32_t *actions, int32_t cap);

/* The heat (Laplace) operator of Sec. 5.7 through the same time-tiled sweep:
 * explicit Euler for u_t = kappa (lap u + f),
 *   u^{n+1} = u^n + dt kappa (L u^n + f^n),   n = 0 .. nt-1,
 * with L the order-so Laplacian of wave_fwd (zero outside the grid) and f^n
 * the trilinear spread of the source traces at step n.  It is the leapfrog
 * update with B = 0 and C = dt kappa, so every tiling gives the same bits.
 *   kappa        device [nx][ny][nz] diffusivity >= 0, or NULL for 1
 *   u0           device [nx][ny][nz] initial field
 *   src / src_traces, rec / rec_traces   as wave_fwd (rec_traces[n] holds
 *                the interpolated u^{n+1})
 *   u_out        device [nx][ny][nz] out: u^nt
 *   tuning       as wave_fwd (NULL = autotune); WAVE_ALLOW_UNSTABLE skips the
 *                stability check dt kappa |L| <= 2, else WAVE_EUNSTABLE is
 *                reported through the status word
 *   ws, ws_bytes workspace of WAVE_OP_FWD for the same points
 * g->dt and g->nt give the step and the number of steps. */
int32_t wave_heat(const wave_grid *g, const float *kappa, const float *u0,
                  const wave_points *src, const float *src_traces,
                  const wave_points *rec, float *rec_traces, float *u_out,
                  const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream);

/* A multi-step form of the same operator (a time dependence of two levels,
 * the larger time dependences the paper names for further work: multi-step
 * linear methods such as Adams-Bashforth, Sec. 6): the two-step
 * Adams-Bashforth scheme for u_t = kappa (lap u + f),
 *   F^n = L u^n + f^n,  u^{n+1} = u^n + dt kappa (3/2 F^n - 1/2 F^{n-1}),
 * with an Euler first step u^1 = u^0 + dt kappa F^0.  The sweep carries the
 * rate F in place of the leapfrog's level n-1, so an untiled step moves 20 B
 * per point (read u^n, F^{n-1}, C; write u^{n+1}, F^n) and a depth-2 tile 10
 * (the new level and rate only; level n+1 stays on chip), against 12 for a
 * depth-2 leapfrog tile.  Arguments as wave_heat; depth 2 runs when compiled
 * for the order (so 2, 4, 8) and tuning->time_tile is not 1 (a depth-2
 * launch does not store the level between its steps: its second stage
 * records the receivers of that level from registers).
 * Stability: dt kappa |L| <= 1, else WAVE_EUNSTABLE through the status word
 * (unless WAVE_ALLOW_UNSTABLE).  Workspace: WAVE_OP_FWD. */
int32_t wave_heat_ab2(const wave_grid *g, const float *kappa, const float *u0,
                      const wave_points *src, const float *src_traces,
                      const wave_points *rec, float *rec_traces, float *u_out,
                      const wave_tuning *tuning, void *ws, size_t ws_bytes, void *stream);

/* Wait for `stream`, then read the device status word that kernels of the
 * last call using workspace `ws` may have set.  Returns WAVE_OK,
 * WAVE_ETIMEOUT or WAVE_ECUDA. */
int32_t wave_status(const void *ws, void *stream);

/* Timing of the sweep launches of the last wave_fwd / wave_adj / wave_grad
 * call made on this host thread with WAVE_TIME_SWEEPS set: events recorded on
 * that call's stream just before its first sweep launch and just after its
 * last.  Waits for the second event.  ms (HOST) receives the elapsed time,
 * launches (HOST) the number of sweep kernel launches and steps the number of
 * time steps they advanced.  Returns WAVE_OK, WAVE_EINVAL (no such call) or
 * WAVE_ECUDA. */
int32_t wave_sweep_stats(float *ms, int32_t *launches, int32_t *steps);

/* Compiled sweep variants for `space_order`: writes up to `max` records of
 * eight int32 each to out (HOST) -- time_tile, tile_y, tile_z, vec, TMA
 * prefetch distance, threads per block, kernel family (WAVE_KERNEL_*), rows
 * per thread -- and returns the number of variants (negative WAVE_EINVAL on
 * bad arguments). */
int32_t wave_list_variants(int32_t space_order, int32_t *out, int32_t max);

/* Counts of the last autotuner run on this host thread: *candidates (HOST) the
 * (variant, x-chunk) plans it considered, *pruned (HOST) those it did not time
 * because their runtime bound (wave_plan_bound) exceeded the best time it had
 * already measured -- the paper's proposal to prune the auto-tuner's search
 * space with a bound that assumes perfect scheduling (Sec. 6.3.3).  Candidates
 * are timed in order of their bound; WAVE_TUNE_NOPRUNE=1 in the environment
 * times every one.  Returns WAVE_OK, or WAVE_EINVAL when the last call on this
 * thread that needed an autotuned plan took it from a cache (or none did). */
int32_t wave_autotune_stats(int32_t *candidates, int32_t *pruned);

/* Lower bound, in milliseconds per time step, on the sweep of the plan that
 * `tuning` selects (time_tile >= 1) for grid g, assuming perfect scheduling:
 * the larger of (a) the compulsory DRAM bytes -- 20 per point-update untiled,
 * 24/T for depth T -- at hbm_gbs GB/s, counted when five fields exceed twice
 * l2_bytes (l2_bytes < 0: always), and (b) the bytes the kernel's code moves
 * through the SM's shared-memory (LSU) pipe for every point each stage
 * computes, the recomputed halo, x-chunk margins and overhanging tiles
 * included, at lsu_gbs GB/s.  Arguments <= 0 (l2_bytes == 0) take the current
 * device's figures: theoretical memory bandwidth, 128 bytes per clock per SM at
 * the maximum SM clock, its L2 size.  *ms (HOST) receives the bound.  Returns
 * WAVE_OK, WAVE_EINVAL, WAVE_EUNSUPPORTED or WAVE_ECUDA. */
int32_t wave_plan_bound(const wave_grid *g, const wave_tuning *tuning, double hbm_gbs, double lsu_gbs,
                        double l2_bytes, double *ms);

/* Sweep variant the library would run for grid g with `tuning` (the cached
 * autotuned plan when tuning->time_tile == 0 and the autotuner already ran
 * for this shape, otherwise the untiled default): out[0..7] = time_tile,
 * tile_y, tile_x, tile_z, vec, TMA prefetch distance, kernel family
 * (WAVE_KERNEL_*), rows per thread.  Returns WAVE_OK or a WAVE_E* code. */
int32_t wave_describe_plan(const wave_grid *g, const wave_tuning *tuning, int32_t *out);

/* The shapes a wave_grad call with these arguments (grid, tuning, source and
 * receiver counts, checkpoint interval) runs its gradient sweeps on, as
 * timed by the first such call on this device: out[0..7] the recompute sweeps
 * storing second differences, out[8..15] the adjoint sweeps with the imaging
 * condition, each laid out as wave_describe_plan's out (the x-chunk is the
 * one the sweeps run).  A host-side query; WAVE_EUNSUPPORTED when no such
 * call has run yet, WAVE_EINVAL on bad arguments. */
int32_t wave_describe_grad_plan(const wave_grid *g, const wave_tuning *tuning, int32_t nsrc, int32_t nrec,
                                int32_t ckpt_every, int32_t *out);

/* ------------------------------------------------------------------------
 * Batched shots.  A seismic survey runs many independent shots over one
 * model; each shot here is a window of the global grid (its own sources and
 * receivers), and the FWI gradient of the survey is the sum of the shots'
 * window gradients scattered into the global grid.  The paper times one
 * operator at a time (Sec. 5.8); batching is how the same sweep fills a GPU
 * whose one shot of a realistic survey leaves most SMs idle.
 * ------------------------------------------------------------------------ */
typedef struct wave_shot {
    int32_t origin[3];   /* first global cell of the window, >= 0 per axis          */
    int32_t n[3];        /* window extent; origin + n <= global n, n >= so + 1      */
    wave_points src;     /* HOST coordinates relative to the window origin (km)     */
    wave_points rec;
} wave_shot;

/* Device workspace for wave_fwd_batched (ckpt_every == 0) or
 * wave_grad_batched (ckpt_every = k >= 1) with `concurrency` shots in flight
 * (1..16; 0 = 4).  g is the global grid (nt, dt, h, space order shared by all
 * shots).  Returns 0 on invalid arguments. */
size_t wave_batch_workspace_bytes(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                                  int32_t ckpt_every, int32_t concurrency);

/* Forward modelling of every shot.  m, damp: device, global [nx][ny][nz].
 * src_traces: device, the shots' [nt][nsrc_s] blocks one after another (shot
 * order); rec_traces: device out, the shots' [nt][nrec_s] blocks likewise.
 * Shots run in groups of `concurrency` consecutive shots; the window of m
 * and damp of each is copied into the workspace first.  The shots of a group
 * advance in lockstep on `stream` when a batched kernel runs the plan: one
 * launch covers every shot of the group per time step (batched kernel of the
 * shared-warp family) or per T steps (batched stage-specialised kernel).
 *   - tuning NULL or time_tile 0: the group times the forward kernel (the
 *     shared-warp batched kernel and every batched stage-specialised shape
 *     whose depth divides nt and ckpt_every) on its own shots for a few
 *     steps, once per device, order and group shape, and caches the choice;
 *   - kernel WAVE_KERNEL_STAGED with time_tile T: the batched
 *     stage-specialised shape of depth T (and tile_y, tile_z, vec, rows where
 *     given), if compiled and T divides nt and ckpt_every;
 *   - time_tile 1 with the default shape: the shared-warp batched kernel.
 * Any other plan runs wave_fwd per shot on library-owned streams that wait
 * for `stream` at the start and that `stream` waits for at the end.  tuning
 * applies to every shot; the per-shape autotuning flags are ignored.  The
 * gradient's recompute and adjoint phases run on a batched
 * stage-specialised gradient shape (the first of the named depth, or the
 * fastest timed one) or on the shared-warp batched kernel.
 * wave_status(ws, stream) reports the most severe device status of all
 * shots.  Results equal wave_fwd on each window, bit for bit, whichever
 * kernel runs. */
int32_t wave_fwd_batched(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                         const float *m, const float *damp, const float *src_traces,
                         float *rec_traces, int32_t concurrency, const wave_tuning *tuning,
                         void *ws, size_t ws_bytes, void *stream);

/* Gradient of J = sum over shots of J_s with respect to the global m, for
 * fixed residuals rec_resid (device, the shots' [nt][nrec_s] blocks of
 * dJ/dd_s, shot order).  Per shot: the forward with checkpoints every
 * ckpt_every steps on the window, then the gradient on the window (the steps
 * of wave_grad), grouped and launched as in wave_fwd_batched.  The window
 * gradients are added into grad (device, global [nx][ny][nz], overwritten;
 * zero outside every window) in shot order, so the result is deterministic
 * and independent of `concurrency`. */
int32_t wave_grad_batched(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                          const float *m, const float *damp, const float *src_traces,
                          const float *rec_resid, int32_t ckpt_every, float *grad,
                          int32_t concurrency, const wave_tuning *tuning, void *ws,
                          size_t ws_bytes, void *stream);

/* The kernels the first group of a batched call with these arguments runs:
 * out[0..7] the forward phases' kernel as wave_describe_plan (time_tile,
 * tile_y, 0, tile_z, vec, prefetch, kernel family, rows), out[8] = 1 for
 * lockstep groups, and for the gradient (ckpt_every >= 1) the family and
 * depth of the recompute and adjoint phases' kernel in out[9] and out[10].
 * All are 0 when the plan runs shot by shot, and out[0] is 0 while an
 * autotuned group (time_tile 0) has not been timed yet on the current
 * device.  out: HOST, 11 ints.  Returns WAVE_OK, WAVE_EINVAL or WAVE_ECUDA.
 * No device work is queued. */
int32_t wave_describe_batch_plan(const wave_grid *g, int32_t nshots, const wave_shot *shots,
                                 int32_t ckpt_every, int32_t concurrency, const wave_tuning *tuning,
                                 int32_t *out);

/* Size in bytes of the static device workspace behind wave_fwd_noalloc. */
#define WAVE_NOALLOC_MAX_BYTES (32u * 1024u * 1024u)

/* Forward modelling without a caller workspace.  The paper has no counterpart:
 * this is a calling convention of this library, not part of the method.
 *
 * For callers that cannot allocate device memory: a C or Fortran host program
 * with no device allocator of its own, a process whose device memory is
 * handed in full to another allocator's pool, or a loop that must not pay the
 * implicit device synchronisation of cudaMalloc / cudaFree.  The workspace is
 * a static device array of WAVE_NOALLOC_MAX_BYTES in this library, reserved
 * when CUDA loads the library's module on a device; the call itself
 * allocates and frees no device memory.
 *
 * Arguments and results as wave_fwd (same kernels, same plan for the same
 * tuning), without checkpoints.  `status` (HOST) may be NULL: then the call
 * returns once the work is queued on `stream`; otherwise it waits for
 * `stream` and stores the device status word there (the value wave_status
 * would return).  If that wait or the read of the word fails, the call returns
 * WAVE_ECUDA and leaves *status unchanged, so *status never holds a host-side
 * error.
 *
 * Set-up: the first call in each CUDA context (normally the primary context
 * of each device), with that context current, takes the array's address
 * (cudaGetSymbolAddress) and keeps it, keyed by the driver's unique context
 * id.  A context created later for the same device (for example after
 * cudaDeviceReset) is set up again by its own first call.  Make each
 * context's first call before any stream capture in it.
 *
 * Sharing: every call on a device uses the same array.  Each call clears, in
 * stream order before its first kernel, what must start at zero (the status
 * words and the wavefield levels) and writes everything else before reading
 * it.  Calls whose work overlaps on the GPU (different streams, or host
 * threads without ordering between them) race on the array and give
 * undefined results: issue them on one stream, or order them.
 *
 * Returns WAVE_ENOSPACE when wave_workspace_bytes(g, WAVE_OP_FWD, nsrc, nrec,
 * 0, tuning) exceeds WAVE_NOALLOC_MAX_BYTES (roughly grids up to 100^3 with
 * few receivers; the receiver buffer takes 32 * nt * nrec bytes), before
 * anything is enqueued; otherwise the codes of wave_fwd.  With a NULL tuning
 * the first call for a shape runs the autotuner, which creates and destroys
 * two CUDA events. */
int32_t wave_fwd_noalloc(const wave_grid *g, const float *m, const float *damp,
                         const wave_points *src, const float *src_traces,
                         const wave_points *rec, float *rec_traces, float *u_last,
                         const wave_tuning *tuning, void *stream, int32_t *status);

#ifdef __cplusplus
}
#endif
#endif /* WAVETILE_WAVE_H */
