/*
 * wf.h - C ABI of the GB300 quasi-implicit ADS wildfire time step.
 *
 * The library advances the temperature T and fuel phi of the reduced
 * energy-balance wildfire model (paper Sec. 2, Eq. energy) on a 2-D
 * tensor-product B-spline space of degree p (Sec. 3.1, "Matrix
 * formulation": open uniform knots, n elements per direction, N = n + p
 * coefficients per direction).  One time step is either
 *
 *   Peaceman-Rachford (Sec. 3.1, Eq. matrixPR):
 *     (X(tau/2,+) (x) M^y) T*      = (M^x (x) Y(tau/2,-)) T^n + tau/2 F
 *     (M^x (x) Y(tau/2,+)) T^{n+1} = (X(tau/2,-) (x) M^y) T*  + tau/2 F
 *   or Strang splitting with Crank-Nicolson (Sec. 3.2, Eq. matrixCN),
 *
 * with X(theta,+-) = M^x +- theta (C_d K^x + c_W b_x G^x + c_chi M^x),
 * Y(theta,+-) = M^y +- theta (C_d K^y + c_W b_y G^y), F the Gauss-quadrature
 * load vector of the explicit nonlinear terms (Sec. 3, normalised form;
 * Sec. 7 listing "compute_rhs") and the fuel advanced by the explicit Euler
 * L2 projection of the same listing.  Every 2-D solve is done as
 * independent 1-D banded solves along x and then along y (Sec. 4).
 *
 * Conventions common to every call
 *  - Return value: WF_OK (0) on success, a negative WF_E* code on failure,
 *    WF_PENDING (> 0) from wf_poll while a request runs.  wf_strerror()
 *    names every code.  No call aborts the process.
 *  - Host arrays are row-major [Ny][Nx] float64 with Nx = nx + p, x fastest.
 *    The caller owns them; the library copies what it needs before
 *    returning (or, for wf_step, never touches host memory).
 *  - The library owns all device memory it allocates and one CUDA stream
 *    per handle (or the caller's stream, see wf_set_stream).
 *  - A handle is not thread-safe: one thread at a time per handle.  The
 *    server calls (wf_submit, wf_poll, wf_server_stats) are thread-safe.
 */
#ifndef WF_H
#define WF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define WF_OK 0
#define WF_PENDING 1         /* wf_poll: request admitted or queued, not finished */
#define WF_EINVAL (-1)       /* invalid argument */
#define WF_ENOMEM (-2)       /* device allocation failed or HBM budget exhausted */
#define WF_ESINGULAR (-3)    /* a 1-D operator had a pivot below 1e-300 * ||A|| */
#define WF_EUNSTABLE (-4)    /* a temperature became non-finite or exceeded 1e5 K */
#define WF_ETIMEOUT (-5)     /* a bounded device wait gave up */
#define WF_ECUDA (-6)        /* a CUDA runtime call failed (no device, launch error, ...) */
#define WF_ETRUNC (-7)       /* the chunked line solve could not reach its truncation tolerance */
#define WF_ENOTFOUND (-8)    /* unknown request ticket */

/* ---- choices ----------------------------------------------------------- */
#define WF_PR 0              /* Peaceman-Rachford, Sec. 3.1 */
#define WF_STRANG_CN 1       /* Strang splitting + Crank-Nicolson, Sec. 3.2 */
#define WF_EXPLICIT 2        /* explicit L2 projection: every term at T^n, mass solves (the
                                explicit dynamics of Sec. 6, the scheme the Sec. 7 listing runs) */
#define WF_FP32 0            /* FP32 quadrature and substitution, FP64 1-D factorisation */
#define WF_FP64 1            /* everything in FP64 (verification mode) */
#define WF_F_ONCE 0          /* PR: F(T^n, phi^n) used in both substeps (default) */
#define WF_F_PER_SUBSTEP 1   /* PR: F(T*, phi^n) in the second substep */

/*
 * Model parameters.  Defaults (wf_params_default) are the paper's Table
 * "Model parameters" (Sec. 2.2) plus these readings: A_r = 1e-4,
 * M/M_1 = 1, T_a = 300 K (exponent of the normalised form), heat scale
 * 1e4 and fuel rate 300 (listing of Sec. 7), fuel threshold 0.2 with a
 * 1e-6 guard, heat release not scaled by fuel.  Lx, Ly are the physical
 * extents in metres; the mean wind (wind_x, wind_y) is treated
 * implicitly in the 1-D operators.
 */
typedef struct wf_params {
    double Lx, Ly;
    double rho, cp, kappa, sigma, eps, ch, hc, cW, chi, T_amb, T_ig, delta_x, delta_z;
    double A_r, M_ratio, T_a, heat_scale, fuel_rate, fuel_thresh, thresh_guard;
    double wind_x, wind_y;
    int scheme;              /* WF_PR | WF_STRANG_CN | WF_EXPLICIT */
    int precision;           /* WF_FP32 | WF_FP64 */
    int F_timing;            /* WF_F_ONCE | WF_F_PER_SUBSTEP (PR only) */
    int scale_heat_by_fuel;  /* 0 (default) or 1 */
} wf_params;

typedef struct wf_handle wf_handle;

/* Fill *p with the defaults above (the Table of Sec. 2.2 plus the stated readings) and
 * Lx = Ly = 100 (m).  Errors: WF_EINVAL for p == NULL, else none. */
int wf_params_default(wf_params* p);

/*
 * Create a simulation on nx x ny elements of degree p (1..3) with time
 * step dt > 0.  Builds, on the GPU and in FP64, the Gauss tables, the 1-D
 * matrices M, K, G (Sec. 3.1) and the banded LU factors of every 1-D
 * operator of the chosen scheme.  The state is zero until wf_set_state.
 * Errors: WF_EINVAL (sizes, p, dt, params), WF_ENOMEM, WF_ESINGULAR,
 * WF_ETRUNC, WF_ECUDA.  On error *out is NULL.
 */
int wf_create(int nx, int ny, int p, double dt, const wf_params* params, wf_handle** out);

/*
 * Copy the state from host arrays T and fuel, each n = Nx*Ny float64
 * values ([Ny][Nx]): the B-spline coefficients of temperature (K) and fuel
 * fraction (Sec. 3.1; the initial state of Sec. 5 and 7 is given in this
 * form).  Converts to the handle's precision on the device.
 * Waits for earlier work on the handle's stream.  Errors: WF_EINVAL
 * (NULL pointer or n != Nx*Ny), WF_ECUDA.
 */
int wf_set_state(wf_handle* h, const double* T, const double* fuel, size_t n);

/*
 * wf_set_state with float32 host arrays (n = Nx*Ny values each, [Ny][Nx];
 * no counterpart in the paper):
 * half the bytes over the host link for a handle that computes in FP32
 * (an FP64 handle widens them).  The arrays are the caller's; pinned
 * memory makes the copy asynchronous to the host.  Same waiting and
 * errors as wf_set_state.
 */
int wf_set_state_f32(wf_handle* h, const float* T, const float* fuel, size_t n);

/*
 * Set the explicit, spatially varying part b'(x, y) of the wind (the wind
 * term c_W b.grad T of Sec. 2, split as in Sec. 3: the mean wind b is
 * implicit in the 1-D operators, the variation b' enters F):
 *   b'_x(x,y) = sum_r fx_r(x) gx_r(y),  b'_y(x,y) = sum_r fy_r(x) gy_r(y),
 * r < rank (0..4), each factor a 1-D spline of the handle's degree and
 * knots given by its coefficients.  `factors` holds, in this order,
 * fx (rank*Nx), gx (rank*Ny), fy (rank*Nx), gy (rank*Ny) float64 values.
 * rank 0 (factors may be NULL) removes the variation.
 * Errors: WF_EINVAL, WF_ECUDA.
 */
int wf_set_wind(wf_handle* h, int rank, const double* factors);

/*
 * Enqueue nsteps >= 0 time steps (Sec. 3.1 / 3.2 / the explicit scheme of
 * Sec. 6, per the handle's scheme) on the handle's stream and return
 * without waiting.  Steps are replayed from a CUDA graph captured on the
 * first call.  Errors: WF_EINVAL, WF_ECUDA (launch failure).
 */
int wf_step(wf_handle* h, int nsteps);

/*
 * Wait for all enqueued work and report device status since the last
 * wf_sync: WF_ETIMEOUT if a bounded device wait gave up in any slot (the
 * output of that step is invalid for every slot of the handle: a CTA that
 * gives up leaves its lines unsolved), else WF_EUNSTABLE if an active
 * slot's temperature became non-finite or exceeded 1e5 K, else WF_OK.
 * The flags are cleared by the call.  No counterpart in the paper.
 */
int wf_sync(wf_handle* h);

/*
 * Limit of every bounded wait inside the library's kernels (the staging
 * barrier of the x pass, the arrival counters of the persistent step), in
 * seconds of the GPU's global timer: 0..60, default 1.  A wait that reaches
 * it gives up, drains its copies in flight, sets the timeout bit of its
 * slot and returns, so the device stays usable and wf_sync reports
 * WF_ETIMEOUT.  0 gives up without waiting (for tests of that path).
 * Captured step graphs are dropped.  Errors: WF_EINVAL.  No counterpart
 * in the paper.
 */
int wf_set_wait_limit(wf_handle* h, double seconds);

/*
 * Wait for enqueued work and copy the state (B-spline coefficients of T and
 * fuel, Sec. 3.1) into host arrays T and fuel (n = Nx*Ny float64 each;
 * either may be NULL to skip it).  Errors: WF_EINVAL, WF_ECUDA.
 */
int wf_get_state(wf_handle* h, double* T, double* fuel, size_t n);

/*
 * wf_get_state into float32 host arrays (n = Nx*Ny values each; either
 * may be NULL; no counterpart in the paper).  An FP64 handle's state is
 * rounded to float32.  Same waiting and errors as wf_get_state.
 */
int wf_get_state_f32(wf_handle* h, float* T, float* fuel, size_t n);

/* Grid sizes of a handle (Nx = nx + p, Ny = ny + p coefficients per direction, Sec. 3.1; any
 * pointer may be NULL).  Errors: WF_EINVAL. */
int wf_get_dims(const wf_handle* h, int* Nx, int* Ny, int* p, int* precision);

/*
 * Use the caller's CUDA stream (a cudaStream_t passed as void*; NULL
 * restores the handle's own stream; no counterpart in the paper).  The captured step graph is kept;
 * it is launched on whichever stream is current.  Errors: WF_EINVAL.
 */
int wf_set_stream(wf_handle* h, void* stream);

/*
 * Per-kernel timing (no counterpart in the paper).  With on != 0, wf_step launches its kernels
 * directly (no graph) with a CUDA event pair around each launch, on the
 * launching stream; wf_kernel_times then returns, per kernel class k <
 * max_k, the summed milliseconds ms[k], the launch count counts[k] and a
 * NUL-terminated name (names[k], up to 47 characters, may be NULL), and
 * resets the sums.  Returns the number of classes (>= 0) or an error:
 * WF_EINVAL (NULL handle, max_k < 0), WF_ECUDA (an event failed).
 */
int wf_set_profiling(wf_handle* h, int on);
int wf_kernel_times(wf_handle* h, double* ms, int* counts, char (*names)[48], int max_k);

/*
 * Change the mean wind b (m/s) of a slot between steps (slot 0 for a handle of
 * wf_create), keeping its state: the runs of Sec. 7 change the wind direction
 * part-way (the Gran Canaria run: a south-westerly, then a westerly wind).  The
 * slot's implicit operators and their chunked factors are rebuilt on the GPU
 * (FP64); the call waits for the handle's stream first.  Captured step graphs
 * stay valid (they address the factors, not their values).
 * Errors: WF_EINVAL, WF_ESINGULAR / WF_ETRUNC (the new operators cannot be
 * factored with the chunk length chosen at creation; the slot keeps its
 * previous wind), WF_ECUDA.
 */
int wf_set_mean_wind(wf_handle* h, int slot, double wind_x, double wind_y);

/*
 * Manufactured-solution forcing for the convergence study of Sec. 6 ("Stability
 * and order of the time integration scheme").  With m != NULL every
 * right-hand side of a step gains the load vector of
 *   f = u_t - C_d lap u + c_W b.grad u + c_chi u
 *       - [c_chi T_amb + c_rad (T_amb^4 - u^4) + C_nld (u^3 lap u + 3 u^2 |grad u|^2)]
 * evaluated at the exact solution
 *   u*(x, y, t) = base + sum_{k < nmodes} amp[k] (1 - cos(2 pi kx[k] x / Lx))
 *                                        (1 - cos(2 pi ky[k] y / Ly)) exp(-lambda[k] t)
 * (the paper: base 300, modes (80, 1, 1, 3), (30, 2, 1, 5), (110, 2, 2, 1.5) on
 * [0, 100]^2), at the start time of the step, scaled like the scheme's F; the
 * time starts at t0 and advances by dt every step (kept on the device).  The
 * model's combustion and wind variation are not part of f: run the study with
 * heat_scale = 0 and no wind variation.  m == NULL switches the forcing off.
 * Single-scenario handles only.  Captured graphs are dropped.
 * Errors: WF_EINVAL (batch handle, nmodes outside 0..4, non-finite values),
 * WF_ECUDA.  wf_get_time reads the current time (waits for the stream).
 */
typedef struct wf_mms {
    int nmodes;
    double amp[4], kx[4], ky[4], lambda[4];
    double base;
    double t0;
} wf_mms;
int wf_set_mms(wf_handle* h, const wf_mms* m);
int wf_get_time(wf_handle* h, double* t);

/*
 * (No counterpart in the paper.)  Number of time-step kernels the library has launched in this process (every
 * handle, eager launches and graph captures alike; a replayed graph launches
 * again the kernels it captured).  For measurement: the difference over eager
 * steps is the number of kernels one step launches.  Errors: WF_EINVAL.
 */
int wf_launch_count(unsigned long long* n);

/*
 * Launch-shape autotuner (no counterpart in the paper, whose solver runs on
 * CPU threads).  Eight values are tuned (int shape[8]):
 *   shape[0]  lines per CTA of the first x pass of a step (rows staged per
 *             CTA; at most 8 warps' worth); lines per tile of both x passes of
 *             the persistent step,
 *   shape[1]  lines per CTA of the y pass (columns per CTA, bounded by
 *             lines x chunks <= 256 threads); columns per tile of the
 *             persistent step's y passes,
 *   shape[2]  element rows per segment of the streaming quadrature kernel,
 *   shape[3]  lines per warp of the x passes (1, 2 or 4; at most 32 / chunks
 *             per line, which is also the default),
 *   shape[4]  lines per CTA of the second x pass,
 *   shape[5]  where Peaceman-Rachford with one F per step forms the right-hand
 *             side of its second x pass: 1 inside that pass (from staged rows
 *             of T* and F), 2 in a streaming matvec kernel before it (one more
 *             pass over R, but every thread busy on short lines);
 *   shape[6]  step form: 1 one launch per pass (seven or eight per step), 2 one
 *             persistent launch per step over every active slot (Peaceman-
 *             Rachford with one F per step, FP32, p <= 2, wind rank <= 2,
 *             no manufactured forcing; elsewhere the per-pass form runs),
 *             3 the per-pass launches over two groups of slots (the first
 *             and the second half) on two streams, the second group's
 *             quadrature of a step starting when the first group's ends, so
 *             that one group's quadrature runs beside the other group's line
 *             passes; the groups join at the end of each wf_step call (and
 *             of each captured graph of steps).  Batches of two or more
 *             slots without manufactured forcing; profiled steps and
 *             wf_step_noalloc run the per-pass form;
 *   shape[7]  slots per group of the persistent step's work order (the order
 *             keeps about six groups' fields live, sized for the L2 cache);
 * 0 selects the built-in rule (shape[5]: inside the pass; shape[6]: the
 * per-pass launches).
 * Every value changes the schedule only: both right-hand-side placements and
 * every step form perform the same operations in the same order, so the
 * results are the same bits.  wf_autotune tunes one value at a
 * time (two sweeps, the others held at their best values): each candidate
 * is timed in three rounds (the candidates in alternating order, so that a
 * drift of the clocks favours none), each round about reps steps (graphs
 * of up to four steps, after one warm-up graph) of the handle's active
 * slots; the value whose fastest round took least device time is kept,
 * and restores every slot's device state afterwards, so the trajectory is
 * unchanged.  It needs a temporary device copy of the slot blocks
 * (S x the per-slot bytes, freed before return; WF_ENOMEM if it cannot be
 * had), synchronises the handle's stream, drops the captured graphs (they
 * are captured again by the next wf_step) and discards kernel times
 * collected under wf_set_profiling.  No active slot: WF_OK, nothing tuned.
 * Errors: WF_EINVAL (reps outside 1..100), WF_ENOMEM, WF_ECUDA.
 * wf_get_tuning / wf_set_tuning read and write the eight values
 * (wf_set_tuning: shape[5] 0..2, shape[6] 0..3, the others 0..1024, else
 * WF_EINVAL).
 */
int wf_autotune(wf_handle* h, int reps);
int wf_get_tuning(const wf_handle* h, int* shape);
int wf_set_tuning(wf_handle* h, const int* shape);

/*
 * ---- batches of scenarios ------------------------------------------------
 * A batch handle holds `capacity` independent scenarios (slots) of one grid
 * (nx, ny, p, dt and model parameters shared).  Each slot has its own state,
 * mean wind (which sets its implicit 1-D operators) and wind variation.  A
 * wf_step on a batch advances every active slot with one launch per kernel
 * of the step (the slots are the third grid dimension); inactive slots cost
 * nothing.  Slots can be filled, activated and drained between steps; the
 * step graph is not re-captured for that.  wf_create is a batch of capacity
 * 1 whose slot 0 is active; the single-scenario calls (wf_set_state,
 * wf_set_wind, wf_get_state) address slot 0.  This extends Sec. 4's
 * independent line solves across scenarios; the paper runs one scenario.
 */

/* Create a batch of `capacity` (1..65535) inactive slots, all with the mean wind
 * of `params` (the tables and operators of wf_create, Sec. 3.1, per slot; batches
 * extend Sec. 4 as above).  Errors as wf_create.  The device memory it holds is reported by
 * wf_device_bytes. */
int wf_batch_create(int nx, int ny, int p, double dt, const wf_params* params, int capacity, wf_handle** out);

/* (Batches extend Sec. 4 as above.) Load slot `slot`: state T, fuel ([Ny][Nx]
 * float64 each), mean wind (wind_x, wind_y) and wind variation of rank 0..4 (factors
 * as in wf_set_wind, NULL for rank 0). A new mean wind refactors the slot's
 * operators on the GPU. Clears the slot's guard flag; does not change whether the
 * slot is active. Waits for earlier work on the handle's stream. Errors: WF_EINVAL,
 * WF_ETRUNC, WF_ESINGULAR, WF_ECUDA. */
int wf_batch_set_slot(wf_handle* h, int slot, const double* T, const double* fuel, double wind_x, double wind_y,
                      int wind_rank, const double* wind_factors);

/* Copy slot `slot`'s state (B-spline coefficients, Sec. 3.1) into host arrays
 * (either may be NULL); waits.  Errors: WF_EINVAL, WF_ECUDA. */
int wf_batch_get_slot(wf_handle* h, int slot, double* T, double* fuel);

/*
 * Every slot's state in one call (no counterpart in the paper): T and fuel are host arrays of
 * n = S*Nx*Ny values each, slot-major ([S][Ny][Nx]), float64 or (the _f32
 * calls) float32; one copy per field and one conversion over all slots,
 * through a device staging area that the first call allocates (2*n values
 * of the host type) and the handle keeps.  Slots' winds, activity and
 * guard flags are untouched.  The get calls wait for enqueued work; either
 * array may be NULL to skip it.  The arrays are the caller's (pinned memory
 * makes the copies asynchronous to the host).
 * Errors: WF_EINVAL (NULL handle or set array, n != S*Nx*Ny), WF_ENOMEM
 * (staging), WF_ECUDA.
 */
int wf_batch_set_states(wf_handle* h, const double* T, const double* fuel, size_t n);
int wf_batch_set_states_f32(wf_handle* h, const float* T, const float* fuel, size_t n);
int wf_batch_get_states(wf_handle* h, double* T, double* fuel, size_t n);
int wf_batch_get_states_f32(wf_handle* h, float* T, float* fuel, size_t n);

/*
 * End-to-end run from host arrays (no counterpart in the paper): every
 * slot's state from T_in, fuel_in, `steps` steps of every active slot, every
 * slot's state into T_out, fuel_out (slot-major [S][Ny][Nx], float64 or,
 * the _f32 call, float32; out may equal in).  The slots are taken in `groups`
 * groups of consecutive slots (1..8, at most S) pipelined over four streams
 * (upload, download, and two compute streams that the groups alternate on):
 * group g's upload overlaps the steps of groups g-1 and g-2 and the downloads
 * of earlier groups, so that the host copies hide behind the steps, and
 * neighbouring groups' steps run side by side (each group's first quadrature
 * after the previous group's).  Each group's steps are
 * the per-pass launches over its slots (the same operations as wf_step: the
 * results are bit for bit those of wf_batch_set_states, wf_step,
 * wf_batch_get_states).  Uses the staging area of the calls above; waits for
 * completion; the caller's arrays should be pinned for the copies to overlap.
 * Errors: WF_EINVAL (NULL handle or array, n != S*Nx*Ny, steps < 0, groups
 * outside 1..8), WF_ENOMEM, WF_ECUDA.
 */
int wf_batch_run(wf_handle* h, const double* T_in, const double* fuel_in, double* T_out, double* fuel_out,
                 size_t n, int steps, int groups);
int wf_batch_run_f32(wf_handle* h, const float* T_in, const float* fuel_in, float* T_out, float* fuel_out,
                     size_t n, int steps, int groups);

/* Include (on != 0) or exclude a slot from the following wf_step calls (a host
 * flag, uploaded with the next step; no counterpart in the paper).
 * Errors: WF_EINVAL. */
int wf_batch_activate(wf_handle* h, int slot, int on);

/* (The guards have no counterpart in the paper.) Waits and writes, per slot, its
 * flag word since the last call into status[0 .. capacity-1] (n >= capacity), and
 * clears the flags: WF_STATUS_UNSTABLE a temperature became non-finite or exceeded
 * 1e5 K; WF_STATUS_TIMEOUT a bounded device wait gave up (the step's output is
 * invalid for every slot of the handle); 0 when neither happened. Errors: WF_EINVAL,
 * WF_ECUDA. */
#define WF_STATUS_UNSTABLE 1
#define WF_STATUS_TIMEOUT 4
int wf_batch_status(wf_handle* h, int* status, int n);

/* Step budget of a slot: it takes part in at most `steps` more steps
 * (counted on the device at the end of each step it takes part in), then
 * every launch skips it until a budget is set again, so that one
 * wf_step(h, n) with n at least the largest budget advances every slot by
 * its own count; steps < 0 removes the budget (the default: unlimited),
 * 0 stops the slot now.  Independent of wf_batch_activate (a slot steps when
 * it is active and its budget is not spent).  Waits for the handle's
 * stream.  The first budget set on a handle drops its captured graphs.
 * Errors: WF_EINVAL, WF_ECUDA.  No counterpart in the paper: it lets a
 * server run one quantum for slots with different step counts left. */
int wf_batch_set_budget(wf_handle* h, int slot, int steps);

/* Number of slots of a handle (>= 1), or WF_EINVAL.  No counterpart in the paper. */
int wf_batch_capacity(const wf_handle* h);

/* Device bytes held by the handle (the layout of its slots and tables).  Errors:
 * WF_EINVAL.  No counterpart in the paper. */
int wf_device_bytes(const wf_handle* h, size_t* bytes);

/* Upper bound of the device bytes wf_batch_create would allocate for these
 * arguments (the largest layout over every chunk length the creation may
 * settle on), computed on the host without touching the device: lets a
 * caller admit work by memory budget before allocating.  The whole-batch
 * state calls' staging (2 x capacity x Nx x Ny host-type values, allocated
 * on their first use) is not included.  Errors: WF_EINVAL (as
 * wf_batch_create's argument checks).  No counterpart in the paper. */
int wf_batch_bytes(int nx, int ny, int p, double dt, const wf_params* params, int capacity, size_t* bytes);

/*
 * ---- serving ---------------------------------------------------------------
 * A server runs fire-scenario requests of any grid size, degree, precision and
 * step count on one GPU.  A worker thread admits requests, first come first
 * served, into slots of batch handles (one per class of requests that can share
 * a launch: same nx, ny, p, dt and parameters apart from the mean wind), creating
 * a class's handle when the device-memory budget allows; it advances every class
 * by quanta of at most 25 steps, all classes enqueued before any is waited for,
 * and retires finished requests.  Requests join and leave running batches at
 * quantum boundaries (continuous batching); a request's result does not depend
 * on the other requests it ran beside.  The paper has no serving layer.
 */
typedef struct wf_request {
    int nx, ny, p, steps;        /* grid, degree (1..3), time steps (>= 0) */
    double dt;                   /* time step (> 0) */
    wf_params params;            /* precision, scheme, extents, mean wind, model constants */
    const double* T0;            /* [Ny][Nx] initial temperature: copied by wf_submit */
    const double* fuel0;         /* [Ny][Nx] initial fuel: copied by wf_submit */
    int wind_rank;               /* 0..4 */
    const double* wind_factors;  /* as in wf_set_wind (NULL for rank 0): copied by wf_submit */
    double* T_out;               /* [Ny][Nx]: written before wf_poll reports completion; */
    double* fuel_out;            /*   the caller keeps both alive until then */
} wf_request;

typedef struct wf_result {
    int status;        /* WF_OK or the request's error (WF_EUNSTABLE, WF_ENOMEM, ...) */
    double latency_s;  /* submit -> result written */
    double queue_s;    /* submit -> admitted into a slot */
    double run_s;      /* admitted -> result written */
} wf_result;

typedef struct wf_server wf_server;

/* Start a server (see the section note: no counterpart in the paper) on the current
 * device with a device-memory budget (bytes) and at most max_slots (1..4096) slots
 * per class.  Errors: WF_EINVAL, WF_ENOMEM, WF_ECUDA. */
int wf_server_create(size_t hbm_budget_bytes, int max_slots, wf_server** out);

/* Queue a request (its steps are those of wf_step for its scheme, Sec. 3); copies its inputs
 * and returns a ticket.  Thread-safe.  Errors: WF_EINVAL. */
int wf_submit(wf_server* s, const wf_request* req, uint64_t* ticket);

/* (Serving layer, no counterpart in the paper.) WF_PENDING while the request is
 * queued or running; otherwise fills *res (may be NULL), forgets the ticket and
 * returns the request's status (WF_OK once T_out and fuel_out hold the result).
 * WF_ENOTFOUND for an unknown or already reported ticket. Thread-safe, never blocks
 * on the GPU. */
int wf_poll(wf_server* s, uint64_t ticket, wf_result* res);

/* (Serving layer, no counterpart in the paper.) Completed DOF-steps ((nx+p)(ny+p) x
 * steps summed over finished requests), number of finished requests and device bytes
 * held by the server's batch handles (any pointer may be NULL). Thread-safe. Errors:
 * WF_EINVAL (NULL server). */
int wf_server_stats(wf_server* s, double* dof_steps, uint64_t* completed, size_t* hbm_used);

/* Stop the worker (running requests are abandoned) and free everything (NULL is
 * accepted).  No return value.  No counterpart in the paper. */
void wf_server_destroy(wf_server* s);

/*
 * Advance a caller-owned FP32 state by nsteps time steps without allocating any
 * device memory.  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc while they step, e.g. a process whose device memory is
 * all owned by another allocator (a framework's pool or an arena sized at start
 * up), or a latency-critical loop that must not pay cudaMalloc's implicit device
 * synchronisation.  The handle h (created earlier, FP32 precision) supplies the
 * tables and factors; T and fuel are device arrays of Ny rows with a row pitch of
 * `pitch` >= Nx float elements, updated in place.  The intermediate fields of
 * the step live in one static device array that the library reserves on every
 * GPU it is loaded on (6 MiB, held until the process exits); pitch * Ny must not
 * exceed 524288 (512 x 512 elements of degree 2 fit).  The first call on a
 * device looks up that array's device address; make that first call before any
 * stream capture.  All calls share the array: two calls whose work overlaps on
 * the GPU (other streams, other threads) race and corrupt each other's results.
 * Work is enqueued on the handle's stream (wf_set_stream) without waiting; use
 * wf_sync to wait and read the guard status.  No CUDA graph is used.
 * Errors: WF_EINVAL (NULL pointer, FP64 handle, pitch < Nx, pitch * Ny above the
 * limit, nsteps < 0, manufactured-solution forcing switched on: its clock belongs
 * to the handle's own state), WF_ECUDA.
 */
int wf_step_noalloc(wf_handle* h, void* T, void* fuel, int pitch, int nsteps);
/* (wf_step_noalloc takes single-scenario handles only: capacity 1.) */

/*
 * Measure this GPU's rate of plain fused multiply-adds (TFLOP/s, one FMA =
 * 2 flops) in `precision` (WF_FP32: the faster of scalar and packed-pair
 * FMAs; WF_FP64): every SM runs independent FMA chains for a few ms,
 * timed with CUDA events, best of three.  The roofline denominator of the
 * quadrature and the line solves, which use these pipes, not tensor cores.
 * Allocates and frees a small device buffer and a stream; synchronises.
 * Errors: WF_EINVAL, WF_ENOMEM, WF_ECUDA.  No counterpart in the paper.
 */
int wf_measure_fma_peak(int precision, double* tflops);

/*
 * Measure the copy rate (GB/s) between pinned host memory and this GPU:
 * host_in -> device (gbs_h2d), device -> host_out (gbs_d2h), and both at
 * once on two streams (gbs_both: the bytes of both directions over the
 * time of the pair).  host_in and host_out: caller-owned page-locked
 * arrays of `bytes` bytes each (host_out is overwritten); best of three
 * copies after a warm-up, CUDA events.  The bound of an end-to-end step
 * whose states come from and return to host memory.  Allocates and frees
 * two device buffers of `bytes`, two streams and two events; synchronises.
 * Errors: WF_EINVAL (a NULL pointer, bytes = 0), WF_ENOMEM, WF_ECUDA.  No
 * counterpart in the paper.
 */
int wf_measure_host_link(const void* host_in, void* host_out, size_t bytes, double* gbs_h2d, double* gbs_d2h,
                         double* gbs_both);

/* Free every resource of the handle (NULL is accepted).  No return value; the
 * handle must not be used afterwards.  No counterpart in the paper. */
void wf_destroy(wf_handle* h);

/* Static text for a status code (unknown codes included); never NULL.  No
 * counterpart in the paper. */
const char* wf_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* WF_H */
