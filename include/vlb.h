/*
 * vlb.h -- C ABI of the GB300 vielbein lattice-Boltzmann + Cahn-Hilliard solver.
 *
 * Method: Ambrus, Busuioc, Wagner, Paillusson & Kusumaatmaja, "Multicomponent flow on curved
 * surfaces: a vielbein lattice Boltzmann approach" (arXiv:1904.10070).
 *
 * The solver advances, on a periodic (theta, varphi) grid of a torus of radii R > r (or of a
 * flat periodic L_x x L_y = 2 pi R x 2 pi r domain):
 *   - 16 fluid distributions f_ij on the Q = 4 Gauss-Hermite velocity set (Sec. 2.3, Eq. vmatrix),
 *     obeying the torus Boltzmann equation with BGK collisions (Eq. boltz_tor, Eq. feq),
 *   - the order parameter phi, obeying the Cahn-Hilliard equation solved by finite differences
 *     (Eq. CH with the chemical potential of Eq. mu and the force of Eq. pbin).
 * Space: conservative flux form, linear 3rd-order upwind ("UW3") or WENO5-JS face values.
 * Time: three-stage SSP Runge-Kutta.  One fused CUDA kernel per Runge-Kutta stage.
 *
 * Conventions for every call:
 *   - Host arrays are [N_theta][N_phi] row-major doubles (varphi fastest) and belong to the
 *     caller; they are only accessed during the call.  f16 arrays are [16][N_theta][N_phi] with
 *     population k = 4 i + j, i the theta-hat velocity index and j the varphi-hat index, v_i
 *     ordered as in Eq. vmatrix (v_1 < v_2 < v_3 < v_4).
 *   - Velocities are vielbein (orthonormal-frame) components; rho is the number density n (m = 1).
 *   - Device memory is owned by the caller: one workspace of vlb_workspace_bytes() bytes, at
 *     least 256-byte aligned, which the library sub-allocates and never frees.  The handle
 *     itself is allocated by the library and released by vlb_destroy().
 *   - All GPU work is issued on the caller's stream (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  Calls that return host data synchronise that stream.
 *   - Every call returns a vlb_status; nothing aborts, throws or traps.  vlb_last_error()
 *     gives a message for the last failure (per handle, or per thread for handle-less calls).
 *   - A handle is not thread-safe.
 */
#ifndef VLB_H
#define VLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vlb_handle vlb_handle;

typedef enum {
  VLB_OK = 0,
  VLB_ERR_ARG = -1,       /* invalid argument or parameter                                 */
  VLB_ERR_CUDA = -2,      /* a CUDA runtime call failed (message in vlb_last_error)         */
  VLB_ERR_UNSTABLE = -3,  /* a diagnostic found a non-finite value or |u| > 2 (blow-up)      */
  VLB_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up                             */
  VLB_ERR_WORKSPACE = -5  /* workspace missing, too small or misaligned                     */
} vlb_status;

enum { VLB_TORUS = 0, VLB_FLAT = 1 };
enum { VLB_FP64 = 0, VLB_FP32 = 1 };
enum { VLB_UW3 = 0, VLB_WENO5 = 1 };
enum { VLB_HYDRO = 0, VLB_DIFFUSIVE = 1 };

/* Problem definition.  Sec. 2 (Eqs. Landau, mu, CH, boltz_tor, nu) and App. A (Eq. torus).
 * tau may be +infinity (no collisions).  Flat geometry: J = 1, Gamma = 0, dx = 2 pi R / N_phi,
 * dy = 2 pi r / N_theta.  Nodes sit at theta_q = q 2pi/N_theta, varphi_s = s 2pi/N_phi.
 * ch_stab = 1 advances phi in every Runge-Kutta stage by P(dt L_phi) instead of dt L_phi, with the
 * fixed preconditioner P = J^{-1} (I + dt M kappa D^2)^{-1} J, D the constant-coefficient periodic
 * five-point Laplacian at the finest spacings (r dtheta and (R - r) dvarphi; R dvarphi flat), applied
 * by FFTs on the device.  P damps the stiff kappa Delta^2 modes, conserves the integral of phi sqrt(g)
 * and tends to the identity as dt -> 0 (a first-order change of the time derivative). */
typedef struct {
  int32_t geometry;    /* VLB_TORUS or VLB_FLAT                                            */
  int32_t n_theta;     /* N_theta >= 4 (>= 6 for WENO5)                                    */
  int32_t n_phi;       /* N_phi >= 1 (1 = azimuthally symmetric)                           */
  int32_t precision;   /* VLB_FP64 or VLB_FP32 (FP32 state; FP64 coefficients and sums)    */
  int32_t advection;   /* VLB_UW3 or VLB_WENO5                                             */
  int32_t ch_mode;     /* VLB_HYDRO, or VLB_DIFFUSIVE: no CH advection and no force (Sec. 4.1.1) */
  int32_t diag_every;  /* steps between finiteness checks inside vlb_step; 0 = never       */
  int32_t ch_stab;     /* 0: explicit Cahn-Hilliard (the paper's scheme); 1: stabilised semi-
                          implicit stages (not in the paper; N_theta, N_phi powers of two in
                          4 .. 4096, solver handles only), see vlb_max_stable_dt             */
  double R, r;         /* torus radii, R > r > 0 (flat: domain 2 pi R x 2 pi r)            */
  double dt;           /* time step > 0                                                     */
  double tau;          /* BGK relaxation time > 0 (nu = tau, Eq. nu)                        */
  double M;            /* mobility >= 0 (Eq. CH)                                            */
  double A, kappa;     /* free-energy parameters (Eq. Landau), A >= 0, kappa >= 0           */
} vlb_params;

/* Bytes of device workspace that vlb_create needs for these parameters; 0 if they are invalid. */
size_t vlb_workspace_bytes(const vlb_params* p);

/* Largest time step the explicit scheme is expected to be stable at (host-only, no GPU):
 * min over (a) advection  dt <= 1 / (v_max (1/h_theta + 1/h_phi,min)), v_max = sqrt(3 + sqrt 6);
 *          (b) BGK        dt <= 2.5 tau  (SSP-RK3 reaches -2.51 on the real axis);
 *          (c) Cahn-Hilliard  dt <= 2.5 / (M lambda (kappa lambda + 2 A)),
 *              lambda = 4/h_theta^2 + 4/h_phi,min^2, h_phi,min = (R - r) dvarphi on the torus;
 *              with ch_stab the stiff part is damped and (c) becomes dt <= 6.25 kappa / (A^2 M)
 *              (the largest preconditioned rate of the spinodal term, A sqrt(dt M / kappa), at 2.5);
 *          (d) relaxation and advection together: the largest dt at which one SSP-RK3 step of
 *              dg/dt = -(v_i/h_theta) D(k_theta) g - (v_j/h_phi,min) D(k_phi) g - g/tau has
 *              |1 + z + z^2/2 + z^3/6| <= 1 on a 64 x 64 grid of Fourier modes and all velocity
 *              pairs (D: the symbol of the UW3 difference, or of the fifth-order linear scheme
 *              for WENO5).  It binds when dt/tau approaches 2 and advection is not negligible.
 * The paper leaves the time integrator to its supplement; these are properties of SSP-RK3.
 * Returns VLB_ERR_ARG for invalid parameters (dt itself is not checked). */
vlb_status vlb_max_stable_dt(const vlb_params* p, double* dt_out);

/* Create a solver on the current CUDA device.  d_workspace: caller-owned device memory of at
 * least vlb_workspace_bytes(p) bytes, 256-byte aligned.  cuda_stream: cudaStream_t or NULL.
 * The state is zero until vlb_set_fields or vlb_set_state. */
vlb_status vlb_create(const vlb_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                      vlb_handle** out);

/* Release the handle (not the workspace).  NULL is accepted. */
vlb_status vlb_destroy(vlb_handle* h);

/* Initialise from macroscopic fields (host [N_theta][N_phi] doubles): f_k := f^eq_k(rho, u)
 * (Eq. feq, the initialisation of Sec. 4), phi := phi.  Synchronous. */
vlb_status vlb_set_fields(vlb_handle* h, const double* rho, const double* u_th, const double* u_ph,
                          const double* phi);

/* Checkpoint / restore of the full state: f16 is [16][N_theta][N_phi], phi [N_theta][N_phi].
 * A state written by vlb_get_state and read back by vlb_set_state (on this or a new handle with
 * the same parameters) continues bit for bit.  Synchronous. */
vlb_status vlb_set_state(vlb_handle* h, const double* f16, const double* phi);
vlb_status vlb_get_state(vlb_handle* h, double* f16, double* phi);

/* Advance nsteps SSP-RK3 steps (3 fused-stage launches per step), asynchronously on the stream.
 * Axisymmetric grids (N_phi = 1, N_theta <= 4096) run up to 256 whole steps per launch of a
 * single-CTA kernel instead.  With the wavefront schedule (vlb_set_schedule) up to 4096 whole steps
 * run per persistent launch, whose bounded dependency waits raise the same flag as the bulk-copy
 * waits below.  The result does not depend on how the steps are grouped or scheduled (bit for bit).
 * With diag_every > 0 the totals are checked every diag_every steps and at the end, the
 * stream is synchronised, and VLB_ERR_UNSTABLE is returned if a value was non-finite or
 * max |u| exceeded 2.
 * Every wait of a stage kernel on a bulk copy is bounded; one that gives up skips its tile and
 * raises the handle's device flag.  vlb_step with diag_every > 0, and every synchronous call below
 * (vlb_get_state, vlb_get_fields, vlb_get_totals, vlb_interface_length), read that flag and then
 * return VLB_ERR_TIMEOUT (the state is invalid; the call's outputs are still written).  The flag
 * stays raised until vlb_set_fields or vlb_set_state. */
vlb_status vlb_step(vlb_handle* h, int64_t nsteps);

/* Test hook for the status path (not part of the method): sets the device flag of handle h to
 * `value` (0 = clear, 1 = unstable, 2 = a bounded wait gave up) as a failing kernel would, so that
 * the statuses above can be checked without making a GPU wait run out.  h == NULL sets the
 * device-wide flag of the tensor-core convolutions on the current device instead (0 or 1; see
 * vlb_conv_status).  Synchronous. */
vlb_status vlb_test_raise_flag(vlb_handle* h, int32_t value);

/* Macroscopic fields (host [N_theta][N_phi] doubles; any pointer may be NULL to skip):
 * rho = n, u = vielbein velocity (Sec. 2.3 moments), phi, and
 * mu = -A phi (1 - phi^2) - kappa Delta phi (Eq. mu, second-order Laplace-Beltrami).  Synchronous. */
vlb_status vlb_get_fields(vlb_handle* h, double* rho, double* u_th, double* u_ph, double* phi,
                          double* mu);

/* Conserved totals and diagnostics, reduced in FP64 on the GPU:
 * out[0] = sum n sqrt(g) dtheta dvarphi, out[1] = sum phi sqrt(g) dtheta dvarphi,
 * out[2] = Psi (Eq. Landau, central differences), out[3] = max |u|.  Synchronous. */
vlb_status vlb_get_totals(vlb_handle* h, double out[4]);

/* Total interface length L_I (Sec. 4: every neighbour pair with phi phi' < 0 adds the shared
 * edge, r dtheta across varphi and (R + r cos theta_{q+1/2}) dvarphi across theta), reduced in
 * FP64 on the GPU; the domain length is L_d = 4 pi^2 r R / L_I (Eq. cart_scaling_L0).  Synchronous. */
vlb_status vlb_interface_length(vlb_handle* h, double* out);

/* Structure-factor length L_S = 2 pi sum S(k) / sum |k| S(k) over k != 0 (a Fourier measure of the
 * coarsening domain size beside Sec. 4.1's L_d), with S(m, n) = |sum phi e^{-2 pi i (m q / N_theta +
 * n s / N_phi)}|^2 on the index grid and wavenumbers k = (m'/r, n'/R), m' and n' the signed frequencies
 * (the physical side lengths 2 pi r along theta and 2 pi R along varphi; on the torus R is the mean
 * circumference over 2 pi).  The transform and both sums run in FP64 on the GPU (phi in FP32 is
 * read as hi + lo); the strip sums are added on the host in a fixed order.  *out = +inf for a
 * uniform phi.  n_theta and n_phi must be powers of two in [4, 4096] (VLB_ERR_ARG otherwise).  Uses
 * the handle's staging area.  Synchronous. */
vlb_status vlb_structure_length(vlb_handle* h, double* out);

/* Device pointer of the resident state (for zero-copy readers on the same device): arrays of
 * n_theta*n_phi elements spaced *stride elements apart -- 16 population deviations
 * g_k = f_k - n0 w_i w_j (n0: the area-weighted mean density at the last set call, rounded to
 * 20 significant bits), then phi; in FP32 mode phi is the float pair (hi at 16 * stride, lo at
 * 17 * stride).  Elements are double (FP64) or float (FP32).  Valid until vlb_destroy; reading
 * it while a vlb_step is in flight on another stream races. */
vlb_status vlb_state_device(vlb_handle* h, void** f, int64_t* stride);

/* Steps taken since the last set call. */
vlb_status vlb_steps_done(const vlb_handle* h, int64_t* out);

/* Execution schedule of vlb_step on a solver handle (not part of the method; the results are the
 * same bit for bit).  VLB_SCHED_STAGES: one launch per Runge-Kutta stage, every stage streaming the
 * whole state through HBM.  VLB_SCHED_WAVE: whole steps in one persistent cooperative launch whose
 * CTAs take 16 x 32 tiles of all three stages in a skewed band order (a stage of a band runs once
 * the previous stage has finished the band and its two neighbours), so that the intermediate
 * stages are read back from L2 and only the state itself crosses HBM; it needs an FP32 UW3
 * explicit grid with N_theta a multiple of 16 and >= 176 and N_phi a multiple of 32 (VLB_ERR_ARG
 * otherwise).  VLB_SCHED_AUTO (the default) takes the per-stage launches: the stage is bound by
 * instruction issue rather than HBM, and the wavefront's per-tile dependency waits cost more than the
 * HBM traffic it saves (measured on GB300: 0.469 against 0.236 ms per step at 1024 x 2048).
 * vlb_get_schedule writes the schedule vlb_step takes (STAGES or WAVE). */
enum { VLB_SCHED_AUTO = 0, VLB_SCHED_STAGES = 1, VLB_SCHED_WAVE = 2 };
vlb_status vlb_set_schedule(vlb_handle* h, int32_t schedule);
vlb_status vlb_get_schedule(const vlb_handle* h, int32_t* active);

/* Host-only self-check of the wavefront ticket order (no GPU needed): VLB_OK if, for n_bands bands,
 * the given lag and nsteps steps, every band item appears exactly once and after every band item it
 * depends on; VLB_ERR_ARG otherwise (also when n_bands <= 2 lag + 2 or lag < 3). */
vlb_status vlb_test_wave_schedule(int32_t n_bands, int32_t lag, int32_t nsteps);

/* Test hook of the wavefront timeout path (not part of the method): CTA skip_cta (-1: none) of every
 * later wavefront launch on h never reports its finished tiles, and each dependency wait gives up
 * after `budget` SM cycles (0: the default, about a second).  The waits that depend on the skipped
 * tiles then run out, raise the handle's flag (2) and end the launch, so vlb_step with diag_every > 0
 * and the synchronous readers return VLB_ERR_TIMEOUT; the context stays usable.  (-1, 0) restores
 * normal operation. */
vlb_status vlb_test_wave_timeout(vlb_handle* h, int32_t skip_cta, int64_t budget);

/* Message of the last failure on h (or of the calling thread's last handle-less failure when
 * h is NULL).  Never NULL; empty when there was none. */
const char* vlb_last_error(const vlb_handle* h);

/* ---- Ensembles: many tori stepped together ----
 * Members are independent problems (own geometry, grid, time step, seed) in FP32 with UW3
 * advection and one common ch_mode.  The tiles of all members form one work list of (member, tile)
 * items, run in one of two ways:
 *   - batched: each Runge-Kutta stage of all members is one launch over the work list;
 *   - persistent: one cooperative launch runs whole steps; its CTAs (all resident at once) take
 *     the items of a stage round-robin and meet at a grid barrier before the next stage.  A CTA
 *     waits at the barrier for a bounded number of SM clock cycles; on expiry it raises the
 *     ensemble's device flag and every CTA returns, so a lost CTA ends the launch with
 *     VLB_ERR_TIMEOUT on the next synchronous call of a member view, never with a hang.
 * The mode and the tile height (16 or 8 theta rows) are chosen on the first vlb_ensemble_step by
 * timing the four candidates on the ensemble (or taken from vlb_ensemble_configure); the choice is
 * cached per process and, if the environment variable VLB_AUTOTUNE_CACHE names a file, in that file
 * (one JSON object per line, keyed by the members' grids, ch_mode and the device's SM count).  The
 * per-step launch sequence is then recorded into CUDA graphs (1 and 32 steps) and replayed on the
 * caller's stream; a launch that cannot be captured runs eagerly instead. */
enum { VLB_ENS_AUTO = 0, VLB_ENS_BATCHED = 1, VLB_ENS_PERSISTENT = 2 };
typedef struct {
  int32_t mode;            /* VLB_ENS_AUTO (timed and chosen), VLB_ENS_BATCHED or VLB_ENS_PERSISTENT */
  int32_t tile_rows;       /* 0 (chosen with the mode), 16 or 8 */
  int32_t ctas_per_sm;     /* persistent launches: 0 = as many as fit, else 1 .. that limit */
  int32_t test_skip_cta;   /* -1; a CTA index of the persistent launch that skips its barrier arrivals
                              (a test of the timeout path: the launch then ends with the flag raised) */
  int64_t barrier_budget;  /* SM clock cycles a CTA waits at a grid barrier; 0 = 2^31 (about a second) */
} vlb_ensemble_config;

/* Workspace bytes for an ensemble of `count` members p[0..count-1]; 0 if invalid. */
size_t vlb_ensemble_workspace_bytes(const vlb_params* p, int32_t count);

/* Create an ensemble handle over a caller-owned workspace (see vlb_create for the conventions). */
vlb_status vlb_ensemble_create(const vlb_params* p, int32_t count, void* d_workspace, size_t bytes,
                               void* cuda_stream, vlb_handle** out);

/* Advance every member by nsteps steps of its own dt, asynchronously on the stream.  The first
 * call synchronises once (autotuning and graph recording; it also takes the first step eagerly).
 * diag_every is not applied: read the totals of members through their views. */
vlb_status vlb_ensemble_step(vlb_handle* h, int64_t nsteps);

/* A view of member idx, usable with vlb_set_fields, vlb_set_state, vlb_get_state, vlb_get_fields,
 * vlb_get_totals, vlb_interface_length, vlb_state_device and vlb_step (which then advances that
 * member alone with per-member launches).  Views are owned by the ensemble: vlb_destroy on a view
 * is a no-op, vlb_destroy on the ensemble releases them. */
vlb_status vlb_ensemble_member(vlb_handle* h, int32_t idx, vlb_handle** view);

/* The chosen tile height (16 or 8; 0 before the first vlb_ensemble_step) and the autotuner's time of
 * one batched first-stage pass for 16- and 8-row tiles (ms; either pointer may be NULL). */
vlb_status vlb_ensemble_tile_rows(const vlb_handle* h, int32_t* rows, float* ms16, float* ms8);

/* Request a mode, tile height, persistent CTAs per SM, barrier budget or the skip test hook (fields
 * left 0 are chosen by timing on the next vlb_ensemble_step).  Synchronises the stream; the next
 * step re-chooses and re-records its graphs. */
vlb_status vlb_ensemble_configure(vlb_handle* h, const vlb_ensemble_config* c);
/* The execution in use (mode 0 before the first step) and the autotuner's times of one first-stage
 * pass per candidate, ms[4] = {batched 16 rows, batched 8, persistent 16, persistent 8} (0 = not
 * timed; ms may be NULL). */
vlb_status vlb_ensemble_get_config(const vlb_handle* h, vlb_ensemble_config* c, float ms[4]);

/* ---- Snapshots: device FP32 [N][4] = (phi, n, u_theta, u_phi), node-major ----
 * vlb_get_snapshot: moments of the state (Sec. 2.3) and phi; asynchronous on the handle's stream.
 * vlb_set_snapshot: restart from a snapshot (n', u', phi').  phi := phi'; keep_nonequilibrium == 0:
 * f := f^eq(n', u') (Eq. feq), which drops the non-equilibrium part of f; keep_nonequilibrium != 0:
 * f := f + f^eq(n', u') - f^eq(n, u) with (n, u) the moments of the current f, which keeps
 * f - f^eq(n, u) (it relaxes on the time scale tau, longer than a surrogate window when tau >> dt).
 * If conserve != NULL, n' and phi' are first shifted uniformly so that sum n' sqrt(g) dtheta dvarphi =
 * conserve[0] and sum phi' sqrt(g) dtheta dvarphi = conserve[1] (reduced on the device).
 * Arithmetic in the state's precision.  Asynchronous on the handle's stream; d_snap is read in that
 * stream's order. */
vlb_status vlb_get_snapshot(vlb_handle* h, float* d_snap);
vlb_status vlb_set_snapshot(vlb_handle* h, const float* d_snap, const double* conserve, int32_t keep_nonequilibrium);

/* ---- Surrogate network kernels (not in the paper) ----
 * A periodic-padding CNN that stands in for blocks of solver steps.  Tensors are device NHWC
 * [H][W][C] (H = N_theta rows, W = N_phi columns, W a multiple of 128), bf16 unless named f32;
 * weights [C_out][3][3][C_in] bf16, biases f32.  Supported (C_in, C_out): (16, 64), (64, 64),
 * (64, 16).  All calls are asynchronous on cuda_stream and accumulate in FP32 on the tensor cores.
 *
 * y = act(conv3x3(x, w) + bias): tap t = 3 (dy + 1) + (dx + 1) reads x at (y + dy, x + dx) mod
 * (H, W); bias may be NULL; relu != 0 clamps at 0; if mask != NULL (same shape as y) outputs where
 * mask <= 0 are zeroed; y_bf16 and/or y_f32 receive the result.
 * Backward data of a layer is this call on dY with the flipped weights of vlb_conv3x3_flip
 * (w'[ci][8 - t][co] = w[co][t][ci]) and mask = the layer's input activation (ReLU derivative). */
vlb_status vlb_conv3x3_fwd(int32_t H, int32_t W, int32_t cin, int32_t cout, const void* x, const void* w,
                           const float* bias, const void* mask, int32_t relu, void* y_bf16, float* y_f32,
                           void* cuda_stream);
vlb_status vlb_conv3x3_flip(int32_t cin, int32_t cout, const void* w, void* w_flipped, void* cuda_stream);
/* dw[co][t][ci] = sum_p dy[p][co] x[p + d_t][ci] and db[co] = sum_p dy[p][co] (db may be NULL), in
 * FP32, with partial sums reduced in a fixed order; workspace of vlb_conv3x3_wgrad_workspace_bytes. */
size_t vlb_conv3x3_wgrad_workspace_bytes(int32_t H, int32_t W, int32_t cin, int32_t cout);
vlb_status vlb_conv3x3_bwd_weight(int32_t H, int32_t W, int32_t cin, int32_t cout, const void* x, const void* dy,
                                  float* dw, float* db, void* workspace, size_t bytes, void* cuda_stream);
/* Status of the tensor-core convolutions: every wait inside their kernels is bounded, and one that
 * gives up raises a device-wide flag (the kernel winds down and its outputs are invalid) instead of
 * hanging.  This call synchronises cuda_stream, reads the flag of the current device, clears it if
 * `clear` != 0, and returns VLB_ERR_TIMEOUT if it was raised, else VLB_OK.  The convolution calls
 * themselves are asynchronous and do not read it: check at the points where you synchronise. */
vlb_status vlb_conv_status(void* cuda_stream, int32_t clear);
/* Scratch (bytes) that vlb_channel_sums and vlb_mse_loss need in d_work. */
size_t vlb_reduce_workspace_bytes(void);
/* Snapshot statistics for the network, on the device, without a host read-back:
 * d_norm8[0..3] = {n_mean, s_phi, s_n, s_u} with n_mean the mean of n, s_phi = rms(phi),
 * s_n = rms(n - n_mean) and s_u = rms(|u|) / sqrt 2 unless the fixed values s_n_fixed / s_u_fixed are
 * > 0 (each scale floored at 1e-12; a non-finite snapshot gives NaNs), and
 * d_norm8[4..7] = {g[0] s_phi, g[1] s_n, g[2] s_u, g[3] s_u}, the output scales (g NULL: all 1).
 * d_work: vlb_reduce_workspace_bytes of scratch; d_sums: 8 doubles of scratch. */
vlb_status vlb_surrogate_norm(int64_t npix, const float* snap, float s_n_fixed, float s_u_fixed, const float g[4],
                              double* d_work, double* d_sums, float* d_norm8, void* cuda_stream);
/* Network input from a snapshot: 16 bf16 channels per node -- phi/s_phi, (n - n_mean)/s_n,
 * u_theta/s_u, u_phi/s_u with d_norm = {n_mean, s_phi, s_n, s_u} (a device array), then
 * J = 1 + a cos theta (sqrt(g)/(r R)), R Gamma = sin theta / J, sin theta, cos theta, 1/J, a = r/R,
 * then zeros (App. A geometry; row q has theta = 2 pi q / H). */
vlb_status vlb_surrogate_features(int32_t H, int32_t W, double r_over_R, const float* snap, const float* d_norm,
                                  void* out_bf16, void* cuda_stream);
/* target[p][c] = (after[p][c] - before[p][c]) / d_scale[c] for the 4 snapshot channels (d_scale on
 * the device). */
vlb_status vlb_surrogate_targets(int64_t npix, const float* before, const float* after, const float* d_scale,
                                 float* target, void* cuda_stream);
/* after[p][c] = before[p][c] + d_scale[c] * pred16[p][c] (first 4 of 16 f32 channels; d_scale on the
 * device). */
vlb_status vlb_surrogate_apply(int64_t npix, const float* before, const float* pred16, const float* d_scale,
                               float* after, void* cuda_stream);
/* Error of a predicted snapshot a against a reference b in phi: d_out4 = {max_p |a.phi - b.phi|,
 * max_p |b.phi|, sum_p (a.phi - b.phi)^2, sum_p b.phi^2} (FP64; sums in a fixed order, maxima exact).
 * A non-finite value in a or b makes d_out4[0] and d_out4[2] +inf.  d_work: vlb_reduce_workspace_bytes. */
vlb_status vlb_snapshot_compare(int64_t npix, const float* a, const float* b, double* d_work, double* d_out4,
                                void* cuda_stream);
/* d_out[c] = sum_p x[p][c], d_out[C + c] = sum_p x[p][c]^2 in FP64 (C <= 16). */
vlb_status vlb_channel_sums(int64_t npix, int32_t C, const float* x, double* d_work, double* d_out, void* cuda_stream);
/* *d_loss = mean over p and c < 4 of (pred16[p][c] - target4[p][c])^2 (FP64); if grad16_bf16 != NULL
 * it receives d loss / d pred (zero in channels 4..15). */
vlb_status vlb_mse_loss(int64_t npix, const float* pred16, const float* target4, void* grad16_bf16, double* d_work,
                        double* d_loss, void* cuda_stream);
/* One Adam step (Kingma & Ba 2015, step t >= 1) on FP32 parameters; p_bf16 (may be NULL) receives
 * the updated parameters rounded to bf16. */
vlb_status vlb_adam_step(int64_t n, float* p, const float* g, float* m, float* v, int64_t t, float lr, float b1,
                         float b2, float eps, void* p_bf16, void* cuda_stream);
vlb_status vlb_to_bf16(int64_t n, const float* x, void* y, void* cuda_stream);

/* ---- Surrogate-accelerated stepping (not in the paper) ----
 * A learned network stands in for windows of solver steps, with the solver as judge and fallback.
 * The network is the 8-layer periodic 3 x 3 CNN of the kernels above: 16 -> 64, six 64 -> 64 and
 * 64 -> 16 channels, ReLU between layers; input = vlb_surrogate_features of the solver's snapshot
 * scaled by vlb_surrogate_norm (with s_n, s_u, g below); output = the window's change, applied by
 * vlb_surrogate_apply.  It is trained elsewhere (the kernels above; paper_1904_10070_gb300/surrogate.py). */
typedef struct {
  const void* weights_bf16;  /* the layers' weights, bf16 [C_out][3][3][C_in], concatenated in layer
                                order (239616 values); host or device memory, copied at create */
  const float* biases;       /* the layers' FP32 biases, concatenated (464 values); host or device */
  float s_n, s_u;            /* fixed input scales of n - mean(n) and of u (> 0) */
  float g[4];                /* output ratios: change of channel c = g[c] * (input scale of c) * output c */
  int32_t window;            /* solver steps that one prediction stands for (> 0) */
  int32_t reserved;          /* must be 0 */
} vlb_surrogate_net;

/* Window kinds reported by vlb_surrogate_advance. */
enum { VLB_WINDOW_SURROGATE = 0, VLB_WINDOW_CHECKED = 1, VLB_WINDOW_FALLBACK = 2, VLB_WINDOW_SOLVER = 3 };
/* Options of vlb_surrogate_advance (bit flags). */
enum { VLB_SUR_JUDGE_LINF = 1, VLB_SUR_NO_GRAPH = 2 };

/* Workspace bytes of a surrogate for the solver grid `geom` (FP32, N_theta even, N_phi a multiple of
 * 128); 0 if invalid.  About 60 MB at 256 x 512. */
size_t vlb_surrogate_workspace_bytes(const vlb_params* geom);

/* Create a surrogate handle for solvers with the grid and radii of geom, over a caller-owned device
 * workspace (256-byte aligned).  The network is copied into the workspace (synchronous on cuda_stream).
 * Release with vlb_destroy. */
vlb_status vlb_surrogate_create(const vlb_params* geom, const vlb_surrogate_net* net, void* d_workspace,
                                size_t bytes, void* cuda_stream, vlb_handle** out);

/* Advance the FP32 solver (a solver handle or an ensemble member view with the network's grid) by
 * nwindows windows of net->window steps, on the solver's stream.  Window k (counted from the first
 * call on this solver) is
 *   - judged when check_every > 0 and k % check_every == 0 (k from 1): the network predicts the
 *     window and the solver runs it from the same state; their phi fields are compared by the
 *     relative L2 error ||phi_net - phi_solver||_2 / ||phi_solver||_2, or with VLB_SUR_JUDGE_LINF by
 *     the relative L-infinity error max|phi_net - phi_solver| / max|phi_solver|.  Within phi_tol the
 *     solver's result is kept (VLB_WINDOW_CHECKED).  Otherwise (or if a value is not finite) the state
 *     returns to the last judged one, the solver redoes the windows since then and this one, and runs
 *     the next check_every windows alone (VLB_WINDOW_FALLBACK, then VLB_WINDOW_SOLVER);
 *   - otherwise predicted (VLB_WINDOW_SURROGATE): snapshot, network, and a restart of the solver from
 *     the prediction that keeps the non-equilibrium part of f (vlb_set_snapshot, keep_nonequilibrium)
 *     with the totals int n sqrt(g) and int phi sqrt(g) held at their values when the surrogate was
 *     bound to this solver.  Nothing is read back to the host; on a stream other than the default
 *     streams the second and later predicted windows replay one captured CUDA graph (VLB_SUR_NO_GRAPH:
 *     always eager).
 * The first call with a given solver binds the surrogate to it (reads its totals, synchronous); a call
 * with another solver starts a new binding.  The solver's step count advances by the window per
 * window (a rollback restores it).  kinds (nwindows ints) and errors (2 nwindows doubles: relative L2
 * and L-infinity error of judged windows, NaN otherwise) may be NULL; *fell_back (may be NULL)
 * receives the number of fallbacks in this call.  Judged windows synchronise the stream; a raised
 * tensor-core flag (see vlb_conv_status) returns VLB_ERR_TIMEOUT there.  Errors of the solver calls
 * inside are returned with their message on the surrogate handle. */
vlb_status vlb_surrogate_advance(vlb_handle* solver, vlb_handle* sur, int32_t nwindows, int32_t check_every,
                                 double phi_tol, int32_t options, int32_t* kinds, double* errors,
                                 int32_t* fell_back);

/* Counters of the current binding: out[0] windows, out[1] predicted windows, out[2] fallbacks,
 * out[3] 1 if a predicted window has been captured as a CUDA graph. */
vlb_status vlb_surrogate_stats(const vlb_handle* sur, int64_t out[4]);

/* Fixed size, in bytes, of the device scratch that vlb_step_noalloc uses. */
#define VLB_NOALLOC_SCRATCH_BYTES (24u * 1024u * 1024u)

/* vlb_step without any device allocation.  The paper has no counterpart: this is a deployment
 * variant for callers that cannot allocate device memory where they step -- plug-ins that may only
 * use the buffers their host application hands them (the host owns the device memory budget), and
 * loops that cannot afford cudaMalloc's implicit device synchronisation.
 *
 * Advances the caller's device state in place by nsteps SSP-RK3 steps on cuda_stream (NULL: the
 * legacy default stream), asynchronously.  d_state (256-byte aligned) holds arrays spaced stride
 * elements apart (stride >= n_theta * n_phi, a multiple of 64): 16 population deviations
 * g_k = f_k - n0 w_i w_j (k = 4 i + j, w the weights of Sec. 2.3), then phi; in FP32 mode phi is
 * the float pair hi (array 16) + lo (array 17).  Elements are double (FP64) or float (FP32).
 * n0 > 0 is the caller's reference density (any value near the mean density keeps the FP32
 * resolution).  diag_every is ignored; nothing is read back.
 *
 * The two intermediate Runge-Kutta states and the row coefficients live in one file-scope device
 * array of VLB_NOALLOC_SCRATCH_BYTES that every device loading the library holds until exit; the
 * call needs 2 * (17 or 18) * stride * element-size bytes plus the tables, and a larger grid is
 * rejected with VLB_ERR_ARG (about 170 k nodes in FP32, 90 k in FP64), and so is a stride beyond
 * that limit, before any size arithmetic.  The first call on each device does the one-time set-up:
 * it looks up the array's device address (cudaGetSymbolAddress) with that device current, raises
 * the stage kernels' shared-memory limit (cudaFuncSetAttribute) and builds their constant
 * velocity tables; so that first call should come before any stream capture.  All calls share the array, which keeps
 * the previous call's contents: calls whose GPU work overlaps (other streams, other host threads
 * on the same device) race.  No cudaMalloc, cudaFree or other allocating routine is called.
 * On failure *error (if not NULL) points to a thread-local message. */
vlb_status vlb_step_noalloc(const vlb_params* p, void* d_state, int64_t stride, double n0, int64_t nsteps,
                            void* cuda_stream, const char** error);

#ifdef __cplusplus
}
#endif

#endif /* VLB_H */
