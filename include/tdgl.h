/*
 * tdgl.h - C ABI of libtdgl: one explicit time step of the time-dependent Ginzburg-Landau
 * (Landau-Khalatnikov) equation for the three-component polarization P of a ferroelectric on a
 * 3D finite-difference grid, after arxiv 2605.28800 ("A GPU-based Solver for Polarization
 * Dynamics in Ferroelectric Materials"), on NVIDIA B300 (sm_103a).
 *
 * What one step computes (Sec. 2, Eqs. 1-7):
 *   dP/dt = -L dF/dP,  L = 1 s^-1 m^-2 C^2 N^-1,   F = F_Land + F_Grad + F_Elec + F_Ext,
 *   h = h_Land (Eq. 3) + h_Grad (Eq. 4) + E_el (Eqs. 5-6, open boundary, P = 0 outside)
 *       + E_ext (Eq. 7),
 *   P <- P + dt L h  (forward Euler; vacuum cells keep P = 0).
 * Units at this boundary are SI: metres, kelvin, seconds, V/m, C/m^2, joules.
 *
 * Conventions common to every call:
 *  - Return value: TDGL_OK (0) or a negative TDGL_E* code; a human-readable message is kept per
 *    context and returned by tdgl_last_error().
 *  - Arrays of cells are float32, "SoA", shape [3][nz][ny][nx] for vectors and [nz][ny][nx] for
 *    scalars, x fastest.  Component order x, y, z.
 *  - `where` says where a caller buffer lives: TDGL_HOST (ordinary or pinned host memory) or
 *    TDGL_DEVICE (device memory of the context's GPU, e.g. a torch CUDA tensor's data_ptr()).
 *    Data are always copied; the library never keeps a pointer to a caller buffer.
 *  - The library owns every device buffer it allocates.  All work is ordered on the context's
 *    stream.  Calls that return data to the host synchronize that stream; others do not.
 *  - Not thread safe: one context (and its sims) must be used from one host thread at a time.
 */
#ifndef TDGL_H
#define TDGL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------- */
#define TDGL_OK              0
#define TDGL_EINVAL         -1   /* bad argument: null pointer, size, id, dt, ...               */
#define TDGL_ENOMEM         -2   /* a device or host allocation failed                           */
#define TDGL_ECUDA          -3   /* a CUDA runtime call failed (message has the CUDA error)     */
#define TDGL_EDIVERGED      -4   /* NaN or |P| above the divergence bound after a step          */
#define TDGL_ENOTCONVERGED  -5   /* relaxation hit its step cap before reaching the tolerance   */
#define TDGL_ESTATE         -6   /* call not valid in the current state (e.g. no material)      */
#define TDGL_ETOOBIG        -7   /* grid too large for tdgl_elec_field_static's fixed scratch   */
#define TDGL_ETIMEOUT       -8   /* a bounded device wait (a pipeline barrier of a tensor copy)
                                    gave up; the kernel returned and the device stays usable     */

#define TDGL_HOST   0
#define TDGL_DEVICE 1

/* energy terms (Eq. 2); also used as the on/off flags of Sec. 3 ("flags allow users to turn
 * different contributions on or off") */
#define TDGL_TERM_LANDAU 1u
#define TDGL_TERM_GRAD   2u
#define TDGL_TERM_ELEC   4u
#define TDGL_TERM_EXT    8u
#define TDGL_TERM_ALL    15u

#define TDGL_MAX_MATERIALS 16    /* material ids 1..15; id 0 is vacuum (P = 0)                  */
#define TDGL_MAX_DIM       1024  /* largest nx, ny, nz                                          */

typedef struct tdgl_ctx   tdgl_ctx;
typedef struct tdgl_sim   tdgl_sim;
typedef struct tdgl_batch tdgl_batch;
typedef struct tdgl_unet  tdgl_unet;

/* Material coefficients, SI (Table 1 forms; the z quadratic coefficient is r_s * alpha1,
 * the strain form of Sec. 4.4):
 *   a1_form 0: alpha1 = a0 (T - T0)
 *   a1_form 1: alpha1 = coth_A (coth(coth_Ts/T) - coth(coth_Ts/coth_T1))   (SrTiO3 form)
 *   a1_form 2: alpha1 = a0                                                  (constant)
 *   alpha11  = a11_0  + a11_T  (T - a11_Tref)        alpha12, alpha112, alpha123 constant
 *   alpha111 = a111_0 + a111_T (T - a111_Tref)       G11, G12, G44, G44p (= G'44) of Eq. 4 */
typedef struct {
    int    a1_form;
    double a0, T0, coth_A, coth_Ts, coth_T1;
    double a11_0, a11_T, a11_Tref, a12;
    double a111_0, a111_T, a111_Tref, a112, a123;
    double G11, G12, G44, G44p;
    double r_s;
} tdgl_material;

/* Energy terms of Eq. 2, joules, accumulated in float64 (Eqs. 3, 4 (discrete), 5, 7). */
typedef struct {
    double land, grad, elec, ext, total;
} tdgl_energies;

/* ---- context --------------------------------------------------------------------------------
 * tdgl_ctx_create: bind to CUDA device `device` and to `stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream; NULL = the library creates and owns a stream).
 * The caller keeps ownership of a stream it passes.  *out receives the context.
 * tdgl_ctx_destroy also destroys the context's remaining batches and sims (their handles become
 * invalid).  DEVICE-side results are ordered on the context's stream: synchronize it (or pass
 * your own stream here) before reading them on another stream. */
int  tdgl_ctx_create(tdgl_ctx **out, int device, void *stream);
void tdgl_ctx_destroy(tdgl_ctx *ctx);
/* last error message of the context (never NULL; "" when none); valid until the next call */
const char *tdgl_last_error(const tdgl_ctx *ctx);
/* number of libtdgl kernel launches issued on this context so far (graph replays included) */
long tdgl_launch_count(const tdgl_ctx *ctx);

/* ---- simulation (Sec. 3: P uniform in each cell of a finite-difference grid) -----------------
 * tdgl_sim_create: grid nx*ny*nz (1..TDGL_MAX_DIM each) of dx*dy*dz cells (metres, > 0).
 * All cells start as vacuum (id 0) until a map or layers are set; P starts at zero.
 * The electrostatic field uses a zero-padded FFT of size >= 2n-1 per axis (open boundary). */
int  tdgl_sim_create(tdgl_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                     tdgl_sim **out);
void tdgl_sim_destroy(tdgl_sim *sim);

/* Padded transform lengths of the open-boundary convolution (Eqs. 5-6; any length >= 2n - 1 gives
 * the same linear convolution).  Defaults: the smallest 2^a 3^b >= 2n - 1 along x (even), y and z,
 * except that along z a length with a factor 3 gives way to the next power of two when that is 128,
 * 256 or 512 and at most 4/3 of it (96 -> 128, 192 -> 256, 384 -> 512), whose tuned z pass finishes
 * first, and along y and z a length the specialized transforms (16, 32, 48, 64, 96, 128, 192, 256,
 * 512) do not cover gives way to the smallest one they cover within 4/3 (81 -> 96, 162 -> 192).
 * Along x, for rows a multiple of 4 cells long whose half-length is not specialized, twice the
 * smallest specialized half-length >= nx within 4/3 (80 cells: 162 -> 192): such rows, and any rows
 * of nx <= Mx / 2 cells with nx a multiple of 4, run in the tiled step kernel.
 * tdgl_fft_pad reports them; tdgl_set_fft_pad sets them (0 = the default
 * for that axis): each must be 2^a 3^b, >= 2n - 1 and <= 4 TDGL_MAX_DIM, Mx even, else TDGL_EINVAL.
 * Setting new lengths waits for the context's stream, frees the sim's spectra and tensor spectrum
 * (rebuilt on the next call that needs the field) and drops its captured step graphs. */
int tdgl_fft_pad(tdgl_sim *sim, int *Mx, int *My, int *Mz);
int tdgl_set_fft_pad(tdgl_sim *sim, int Mx, int My, int Mz);

/* Define (or redefine) material `id` (1..15) from Table 1-style coefficients (Sec. 3:
 * spatially varying material parameters at the cell level). */
int tdgl_material_define(tdgl_sim *sim, int id, const tdgl_material *m);
/* Per-cell material ids, uint8 [nz][ny][nx]; 0 = vacuum.  Every non-zero id must be defined
 * before the first step.  Cells that become vacuum get P = 0. */
int tdgl_set_material_map(tdgl_sim *sim, const uint8_t *ids, int where);
/* Layers along z: cells with z0[i] <= z < z1[i] get id[i] (later entries win); others vacuum. */
int tdgl_set_layers(tdgl_sim *sim, int n, const int *z0, const int *z1, const int *id);
/* Background permittivity eps_B of Eq. 6 (> 0; a free parameter in the paper). Default 1. */
int tdgl_set_eps_b(tdgl_sim *sim, double eps_b);
/* Enabled terms, a mask of TDGL_TERM_*.  Default TDGL_TERM_ALL. */
int tdgl_set_terms(tdgl_sim *sim, unsigned mask);
/* Temperature (kelvin, > 0) at which Table 1 coefficients are evaluated.  Default 300. */
int tdgl_set_temperature(tdgl_sim *sim, double T);
/* Uniform applied field E_ext of Eq. 7, V/m.  Default 0. */
int tdgl_set_field(tdgl_sim *sim, double Ex, double Ey, double Ez);

/* Time-dependent excitation (Sec. 3 "time-dependent external excitations"; Sec. 4.4 AC loops):
 * the applied field becomes E_ext(t) = (Ex, Ey, Ez) + (Ax, Ay, Az) sin(2 pi freq_hz t + phase), V/m,
 * evaluated at the time of each step (t advances by dt per step; explicit Euler uses E_ext(t_n)).
 * Amplitude 0 (the default) turns it off. */
int tdgl_set_field_ac(tdgl_sim *sim, double Ax, double Ay, double Az, double freq_hz, double phase);
/* Time integrator of Eq. 1 (Sec. 3 lists Heun, RK45 and AB3M2):
 *   TDGL_EULER (default)  P <- P + dt h(P, t)
 *   TDGL_HEUN             P~ = P + dt h(P, t);  P <- P + dt/2 (h(P, t) + h(P~, t + dt))
 *   TDGL_RK45             Runge-Kutta-Fehlberg 4(5): six field evaluations, P advances with the
 *                         fourth-order solution; the fifth-order one gives the local error
 *                         max |P5 - P4| / P0, which drives the step size when tdgl_set_adaptive
 *                         has set a tolerance
 *   TDGL_AB3M2            Adams-Bashforth 3-step predictor, Adams-Moulton 2-step corrector (PECE:
 *                         two field evaluations per step); its first two steps use the 1- and
 *                         2-step pairs (the first is Heun's method).  Any change of P, time,
 *                         fields, terms, materials or temperature restarts the history.
 * Heun costs 12 bytes per cell of device memory, RK45 and AB3M2 72.  The sims of a batch must use
 * one integrator, Euler or Heun. */
#define TDGL_EULER 0
#define TDGL_HEUN  1
#define TDGL_RK45  2
#define TDGL_AB3M2 3
int tdgl_set_integrator(tdgl_sim *sim, int method);
/* RK45 step-size control: err_tol > 0 makes tdgl_step and tdgl_relax adaptive (a step whose local
 * error exceeds err_tol is retried with a smaller dt; after an accepted step dt grows or shrinks by
 * 0.9 (err_tol / err)^(1/5), within [0.2, 5] per step and [dt_min, dt_max] overall, dt_max 0 = no
 * bound); err_tol = 0 returns to fixed steps.  tdgl_step(sim, n, dt) then takes n accepted steps,
 * starting from dt on the first call and from the controller's dt afterwards; tdgl_relax checks
 * max |dP| / P0 of the last step scaled by dt / dt_step.  tdgl_get_dt returns the next dt (s). */
int tdgl_set_adaptive(tdgl_sim *sim, double err_tol, double dt_min, double dt_max);
int tdgl_get_dt(tdgl_sim *sim, double *dt);

/* Radix-schedule autotuning of the z pass (the transform along z, the 3x3 tensor multiply and the
 * inverse transform) for 128-, 256- and 512-point lines.  Variants: 0, 16 elements per thread
 * (radices 16 x 8, 16 x 16, 16 x 16 x 2); 1, 8 elements per thread (8 x 8 x 2, 8 x 8 x 4,
 * 8 x 8 x 8) with twice the warps per SM; 2 (128 and 256 only), variant 1 with the block's rows of
 * the tensor spectrum copied into shared memory at the start, overlapping the forward transforms;
 * 3 (128 and 256 only), variant 2 with the three components' transforms run together (one
 * shared-memory exchange serves all three) and the tensor multiply on registers.
 * The first time a context prepares a sim with such lines it times every variant of the length on
 * that sim's buffers (no state changes) and keeps the fastest.  tdgl_zpass_variant reads the
 * choice (-1 = not tuned yet) and, if us is not NULL, writes TDGL_ZPASS_VARIANTS doubles: the
 * measured microseconds per launch of each variant (0 for a variant the length does not have);
 * tdgl_set_zpass_variant forces one (-1 tunes again).  All variants compute the same field up to
 * FP32 rounding. */
#define TDGL_ZPASS_VARIANTS 4
int tdgl_zpass_variant(tdgl_ctx *ctx, int length, int *variant, double *us);
int tdgl_set_zpass_variant(tdgl_ctx *ctx, int length, int variant);
/* Row-tile autotuning of the fused step kernel (the x-rows kernel: x transforms, Landau, gradient,
 * update) for a sim run alone.  A block takes a tile of consecutive rows of one z plane; up to
 * TDGL_ROW_CANDIDATES tile heights (the kernel's maximum, its half and quarter, and the height that
 * gives about one block per SM) are timed the first time a context prepares a sim of that shape
 * (x half-length, ny, nz, electrostatics on or off), three step launches each on scratch copies of
 * the sim's buffers (no state changes), and the fastest is kept for the context.  Sims of the
 * generic (any-length) row kernel keep one row per block group as before.  Batch members use the
 * kernel's maximum tile.  tdgl_row_tile reports the sim's tile (0 = not tuned) and, if not NULL,
 * the candidates and their microseconds per launch (0 for unused slots). */
#define TDGL_ROW_CANDIDATES 4
int tdgl_row_tile(tdgl_sim *sim, int *rows, int *candidates, double *us);
/* Forces the sim's row tile to `rows` rows per block (clamped to the kernel's maximum; the
 * autotuner then leaves the sim alone), or with rows = 0 returns it to the autotuner.  For runs
 * whose timings cannot be trusted, e.g. under a profiler that serializes launches.  Waits for the
 * context's stream and drops the sim's captured step graphs (they are captured again on the next
 * use).  TDGL_EINVAL for rows < 0. */
int tdgl_set_row_tile(tdgl_sim *sim, int rows);
/* Simulated time t (s) of the sim: 0 at creation, advanced by n dt by every step call. */
int tdgl_set_time(tdgl_sim *sim, double t);
int tdgl_get_time(tdgl_sim *sim, double *t);

/* Internal normalization (Table 2): P* = P/P0, tau = alpha_ref L t, E* = E/(alpha_ref P0).
 * Defaults, fixed at the first step unless set here: alpha_ref = |alpha1| of the lowest defined
 * material id at 300 K; P0 = that material's tetragonal spontaneous polarization at 300 K
 * (1 C/m^2 if it has none).  Relaxation tolerances are in units of P0.  Setting the scales
 * keeps the physical P. */
int tdgl_set_scales(tdgl_sim *sim, double P0, double alpha_ref);
int tdgl_get_scales(tdgl_sim *sim, double *P0, double *alpha_ref);

/* P in C/m^2, float32 [3][nz][ny][nx].  set_P zeroes vacuum cells. */
int tdgl_set_P(tdgl_sim *sim, const float *P, int where);
int tdgl_get_P(tdgl_sim *sim, float *out, int where);

/* Pipelined host I/O (Sec. 3: the solver records P at user-chosen intervals while it runs).  These
 * calls queue work and return without waiting for it:
 *  - tdgl_set_P_async copies P (C/m^2, float32 [3][nz][ny][nx] in host memory) into the sim on the
 *    context's upload stream; the sim's later work waits for it.
 *  - tdgl_step_async queues n steps like tdgl_step (forward Euler or Heun; TDGL_EINVAL for RK45 and
 *    AB3M2, which read their error estimates on the host) without reading their status.
 *  - tdgl_get_P_async queues the copy of the sim's P at that point of its work into `out` (host
 *    memory, same layout) on the context's download stream.
 *  - tdgl_sync waits until every call above on this sim has completed, then reports the status of
 *    the steps queued since the last check: TDGL_EDIVERGED or TDGL_ETIMEOUT as tdgl_step would.
 * Uploads and downloads go through device staging buffers, two per direction used in turn
 * (allocated on first use, 4 x 12 bytes per cell), so consecutive set / step / get calls overlap:
 * the next input's upload and the last result's download run while the current steps compute, and
 * the copies of one direction follow each other back to back.  Host buffers must be
 * page-locked for the copies to overlap (pageable memory works, with the copies staged by the
 * driver); a buffer passed to tdgl_set_P_async must not change, and one passed to tdgl_get_P_async
 * must not be read, until tdgl_sync returns.  Not for use inside a stream capture. */
int tdgl_set_P_async(tdgl_sim *sim, const float *P);
int tdgl_step_async(tdgl_sim *sim, int n, double dt);
int tdgl_get_P_async(tdgl_sim *sim, float *out);
int tdgl_sync(tdgl_sim *sim);
/* Fill P with independent uniform values in [-amp, amp] C/m^2 from a Philox4x32-10 stream:
 * value (c, cell) uses counter (cell, c, 0, 0) and key (seed & 0xffffffff, seed >> 32); the
 * first 32-bit output u maps to amp * (2 (u + 0.5) / 2^32 - 1).  Vacuum cells stay 0. */
int tdgl_init_random(tdgl_sim *sim, uint64_t seed, double amp);

/* Effective-field contributions of the current P for the terms in `mask` (V/m, float32
 * [3][nz][ny][nx], zero on vacuum cells): h_Land, h_Grad, E_el, E_ext of Eqs. 3-7. */
int tdgl_get_field(tdgl_sim *sim, unsigned mask, float *out, int where);

/* n >= 0 steps of Eq. 1 (forward Euler unless tdgl_set_integrator chose Heun) with time step dt
 * (seconds, > 0).  Returns
 * TDGL_EDIVERGED (state left as computed) if any step produced NaN or |P_i| > 1e3 P0. */
int tdgl_step(tdgl_sim *sim, int n, double dt);
/* max over cells and components of |P_new - P_old| of the most recent step, in units of P0. */
int tdgl_last_max_dP(tdgl_sim *sim, double *out);
/* Relaxation (Sec. 4: equilibrium as the steady state of Eq. 1): step with dt until the
 * max |dP| of a step, checked every `check_every` steps (>= 1), is below tol * P0, or until
 * max_steps.  *steps_taken (may be NULL) receives the steps done.  Returns TDGL_OK on
 * convergence, TDGL_ENOTCONVERGED at the cap, TDGL_EDIVERGED on divergence.  For forward Euler
 * with an even check_every, and for Heun, without a time-dependent applied field, the check runs
 * on the device inside one CUDA graph (the host waits once per call); the steps taken and the
 * result are the same as with a host check every check_every steps. */
int tdgl_relax(tdgl_sim *sim, double dt, double tol, long max_steps, int check_every,
               long *steps_taken);
/* Energy terms of Eq. 2 for the current P (joules, float64 accumulation). */
int tdgl_energy(tdgl_sim *sim, tdgl_energies *out);

/* ---- batches (Sec. 3: many independent simulations run in parallel on one GPU) --------------
 * A batch groups n sims of one context (any sizes) so that each kernel of a step is one launch
 * over all of them.  The sims stay usable on their own; a sim may belong to one batch at a time;
 * destroying a sim removes it from its batch (per-sim arrays then follow the remaining order). */
int  tdgl_batch_create(tdgl_ctx *ctx, int n, tdgl_sim *const *sims, tdgl_batch **out);
void tdgl_batch_destroy(tdgl_batch *b);
/* n steps of every sim; dt[i] (seconds) per sim. */
int  tdgl_batch_step(tdgl_batch *b, int n, const double *dt);
/* Relax every sim to its own tolerance (tol in units of each sim's P0, one value for all);
 * converged sims leave the batch's work list.  steps_taken[i] (may be NULL) per sim.
 * Returns TDGL_OK when all converged, else TDGL_ENOTCONVERGED / TDGL_EDIVERGED. */
int  tdgl_batch_relax(tdgl_batch *b, const double *dt, double tol, long max_steps,
                      int check_every, long *steps_taken);
/* tdgl_batch_relax that also reports how each sim ended, in state[i] (may be NULL): converged,
 * still above the tolerance after max_steps, diverged, or a bounded device wait timed out.  With
 * it a caller can run a long relaxation in slices of max_steps (a multiple of check_every keeps
 * the check steps of one uninterrupted call) and refill the slots of finished sims between slices:
 * a sim that converges exactly at a slice's last check is told apart from one that did not. */
#define TDGL_RELAX_CONVERGED 0
#define TDGL_RELAX_AT_CAP 1
#define TDGL_RELAX_DIVERGED 2
#define TDGL_RELAX_TIMEOUT 3
int  tdgl_batch_relax_state(tdgl_batch *b, const double *dt, double tol, long max_steps,
                            int check_every, long *steps_taken, int *state);

/* ---- field without allocation ------------------------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot call cudaMalloc:
 * plug-ins whose host application owns all device memory through its own pool allocator, and
 * real-time loops that must not wait on the driver's allocator (cudaMalloc can synchronize the
 * device).  The arithmetic is that of tdgl_get_field with TDGL_TERM_ELEC alone, run through the
 * library's generic (any-length) kernels; the FP64 tensor spectrum is rebuilt on every call, so a
 * call costs more GPU time than a tdgl_get_field on a prepared sim.
 *
 * tdgl_elec_field_static computes the open-boundary electrostatic field E_el of P (the same
 * quantity as tdgl_get_field with TDGL_TERM_ELEC) on an nx*ny*nz grid of dx*dy*dz cells:
 *   P     device, float32 [3][nz][ny][nx], C/m^2 (caller-owned input; must be 0 on vacuum cells)
 *   mat   device, uint8 [nz][ny][nx], 0 = vacuum, or NULL for an all-material box
 *   E     device, float32 [3][nz][ny][nx], V/m (caller-owned output; 0 on vacuum cells)
 *   stream  cudaStream_t to enqueue on (NULL = legacy default stream); the call returns once the
 *           work is enqueued.
 * It allocates nothing: every intermediate lives in one static device array of
 * TDGL_STATIC_SCRATCH_BYTES that each GPU loading this library holds until the process exits.
 * Grids whose intermediates do not fit return TDGL_ETOOBIG (a 36x36x36 cube fits, 40x40x40 does
 * not; 32x32x32 needs about 8 MiB); bad
 * arguments return TDGL_EINVAL.  The first call on a device looks up the array's device address
 * with that device current (set-up done once per device): make that first call before any stream
 * capture begins.  All calls share the array and each call overwrites it completely, so calls
 * whose work overlaps on the GPU (other streams, other host threads) race and must be serialized
 * by the caller. */
#define TDGL_STATIC_SCRATCH_BYTES (16u << 20)
int tdgl_elec_field_static(int nx, int ny, int nz, double dx, double dy, double dz, double eps_b,
                           const float *P, const uint8_t *mat, float *E, void *stream);

/* ---- measurement -----------------------------------------------------------------------------
 * tdgl_profile(ctx, 1) records a CUDA event pair around every kernel launch on the context's
 * stream; tdgl_profile_read(ctx, k, &ms, &n) synchronizes and returns the summed device time and
 * the launch count of kernel kind k since the last reset (then resets kind k).  Kinds: */
#define TDGL_K_STEP   0   /* fused x-inverse + Landau + gradient + update + x-forward  */
#define TDGL_K_YFWD   1   /* y forward FFT of the zero-padded x-spectrum               */
#define TDGL_K_ZCONV  2   /* z FFT, 3x3 tensor multiply, inverse z FFT                  */
#define TDGL_K_YINV   3   /* inverse y FFT                                             */
#define TDGL_K_XFWD   4   /* x forward real FFT of P (prologue)                        */
#define TDGL_K_OTHER  5   /* energy, field readback, tensor build, copies              */
#define TDGL_K_UNET   6   /* learned warm start: convolutions, their gradients, Adam     */
#define TDGL_K_COUNT  7
int tdgl_profile(tdgl_ctx *ctx, int enable);
int tdgl_profile_read(tdgl_ctx *ctx, int kind, double *total_ms, long *launches);

/* Timeout path check.  Every wait of the library's kernels on an mbarrier (the arrival of a tensor
 * copy, a tensor-core commit) is bounded: after its poll limit the waiting thread sets a status flag,
 * the kernel finishes and the call returns TDGL_ETIMEOUT, with the context still usable.
 * tdgl_wait_probe runs that path on purpose and safely: one thread of a one-block kernel waits for
 * an mbarrier on which nothing is pending and nothing will arrive (no copy in flight), for at most
 * `polls` polls (1 .. 2^24), then records the timeout.  Returns TDGL_ETIMEOUT (the expected result),
 * TDGL_EINVAL for a bad count, TDGL_ECUDA if the launch failed. */
int tdgl_wait_probe(tdgl_ctx *ctx, long polls);

/* Measurement helper (it computes nothing of the paper's method): the device's FP32 fused
 * multiply-add throughput, the denominator of the FP32-ALU roofline of the transform kernels.  One
 * launch of 8 independent FMA chains per thread on every SM (a warm-up launch, then three timed with
 * CUDA events on the context's stream); *tflops receives 2 flops per FMA over the mean launch time,
 * in TFLOP/s.  Uses a 4-byte device buffer that it allocates and frees.  Returns TDGL_ECUDA on a
 * CUDA error. */
int tdgl_fp32_fma_peak(tdgl_ctx *ctx, double *tflops);

/* ---- learned warm start ----------------------------------------------------------------------
 * The relaxation starts from a proposal instead of a random state (a data-driven model trained on
 * solver-made textures, the use Sec. 5 names for the solver): a 3D U-Net maps per-cell inputs (material indicators,
 * temperature, applied field) to a polarization texture, and the plain relaxation to the same
 * tolerance then judges it.  The network: `levels` resolution levels with chans[l] channels,
 * two 3x3x3 convolutions + ReLU per level, 2x2x2 average pooling down, nearest-neighbour
 * upsampling + skip concatenation up, a 1x1x1 output convolution.  BF16 weights and activations
 * on the tensor cores (tcgen05, FP32 accumulation in tensor memory), FP32 master weights, Adam.
 *
 * Tensors at this boundary are float32 [B][C][nz][ny][nx] (x fastest), the layout of P.
 * Parameters travel as one float32 vector in the order of the layers (encoder level 0 a, b, ...,
 * decoder level levels-2 a, b, ..., level 0 a, b, head); per layer the weights w[o][i][dz][dy][dx]
 * (offsets -1..1, or a single tap for the head) then the biases b[o].
 *
 * tdgl_unet_create: cin input channels (1..8), cout outputs (1..16), 2 <= levels <= 5, chans[l]
 *   multiples of 16 in 16..128; grid: nx a multiple of 8 * 2^(levels-1), ny and nz multiples of
 *   2^(levels-1); max_batch >= 1 samples per call.  Weights He-normal (std sqrt(2 / fan-in)) from a
 *   counter-based generator (Philox4x32-10) keyed by seed, biases 0.  Returns TDGL_EINVAL on bad
 *   shapes, TDGL_ENOMEM if the buffers do not fit.
 * tdgl_unet_param_count: number of floats of the parameter vector.
 * tdgl_unet_set_params / tdgl_unet_get_params: host float32 vector (caller-owned), resets Adam.
 * tdgl_unet_forward: x (B*cin*N floats) -> y (B*cout*N), where = TDGL_HOST or TDGL_DEVICE for both.
 * tdgl_unet_loss_grad: mean-squared loss of forward(x) against target t and its gradient with
 *   respect to every parameter (grads: caller-owned, param_count floats, same order), no update.
 * tdgl_unet_train_step: forward, loss, backward and one Adam step (lr; beta1 0.9, beta2 0.999,
 *   eps 1e-8, bias-corrected with the net's own step counter).  *loss receives the loss before the
 *   update.  Returns TDGL_ETIMEOUT if a tensor-core pipeline wait timed out (the device stays usable).
 * All calls are ordered on the context's stream and return after the results are in place. */
int  tdgl_unet_create(tdgl_ctx *ctx, int cin, int cout, int levels, const int *chans, int nx, int ny, int nz,
                      int max_batch, uint64_t seed, tdgl_unet **out);
void tdgl_unet_destroy(tdgl_unet *net);
long tdgl_unet_param_count(const tdgl_unet *net);
int  tdgl_unet_set_params(tdgl_unet *net, const float *params);
int  tdgl_unet_get_params(tdgl_unet *net, float *params);
int  tdgl_unet_forward(tdgl_unet *net, const float *x, float *y, int batch, int where);
int  tdgl_unet_loss_grad(tdgl_unet *net, const float *x, const float *t, int batch, double *loss, float *grads,
                         int where);
int  tdgl_unet_train_step(tdgl_unet *net, const float *x, const float *t, int batch, double lr, double *loss,
                          int where);

/* The convolution primitives of the network, for checking them one by one.  x [B][ci][nz][ny][nx],
 * w [co][ci][k][k][k] (k = 3 or 1), b [co], all host float32; operands are rounded to BF16, sums
 * are FP32.  tdgl_conv3d: y [B][co][...] = conv(x, w) + b (relu != 0: max(., 0)).
 * tdgl_conv3d_backward: for upstream gradient dy [B][co][...] returns dx [B][ci][...], dw, db.
 * Channel counts: ci a multiple of 8 up to 192 (forward) and up to 128 for co; nx a multiple of 8. */
int tdgl_conv3d(tdgl_ctx *ctx, const float *x, const float *w, const float *b, float *y, int batch, int ci, int co,
                int k, int nx, int ny, int nz, int relu);
int tdgl_conv3d_backward(tdgl_ctx *ctx, const float *x, const float *w, const float *dy, float *dx, float *dw,
                         float *db, int batch, int ci, int co, int k, int nx, int ny, int nz);

#ifdef __cplusplus
}
#endif
#endif /* TDGL_H */
