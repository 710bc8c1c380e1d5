// Internal declarations shared by the translation units of libvlb (not part of the C ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (type only: the encoder is looked up in the driver at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vlb.h"

namespace vlb {

constexpr int NPOP = 16;  // Q^2 populations, k = 4 i + j
constexpr int NARR = 17;  // host/staging layout: 16 populations + phi
// Device state arrays: 16 population deviations, phi, and in FP32 mode the low part of phi.
constexpr int state_arrays(size_t esize) { return esize == 4 ? NARR + 1 : NARR; }

// Per-theta-row coefficient tables, one array of n_theta entries per field (SoA).
// Computed in FP64 on the host (App. A geometry) and rounded once to the state precision.
enum RowCoef : int {
  C_J = 0,   // J_q = 1 + a cos theta_q                       (sqrt g = r R J)
  C_JP,      // J_{q+1/2}
  C_JM,      // J_{q-1/2}
  C_CT,      // 1 / (r J_q dtheta)        theta-divergence prefactor
  C_CP,      // 1 / (R J_q dvarphi)       varphi-divergence prefactor
  C_GAM,     // Gamma_q = sin theta_q / (R J_q)   (Eq. conn_torus)
  C_LT,      // 1 / (r^2 J_q dtheta^2)    Laplace-Beltrami, theta part
  C_LP,      // 1 / (R^2 J_q^2 dvarphi^2) Laplace-Beltrami, varphi part
  C_GP,      // 1 / (2 R J_q dvarphi)     central varphi gradient
  C_EP,      // rest-state residual for v_i > 0 (see below)
  C_EN,      // rest-state residual for v_i < 0
  C_DA,      // sqrt(g) dtheta dvarphi    area element (kept in FP64 only)
  C_EDGE,    // (R + r cos theta_{q+1/2}) dvarphi   interface edge across theta (FP64 only)
  NCOEF
};

// Storage: the populations are kept as g_k = f_k - n0 w_i w_j, the deviation from the rest
// equilibrium at a reference density n0 (fixed at set time).  Every term of the right-hand side is
// linear in f except the BGK equilibrium and the WENO weights, so the reference part is carried
// through exact identities of the Q = 4 kernel: (K w)_i = -v_i w_i and (K (v w))_i = w_i (1 - v_i^2).
// The reference part of the force, inertial and UW3 advection terms then collapses to
//   n0 w_i w_j [ v_i (E_sign(v_i)(q) + F^theta) + v_j F^phi ],
// with E_pos/neg(q) = -D_pos/neg[J](q) / (r J_q dtheta) - Gamma_q the discrete residual of the
// continuum cancellation between the J-flux and the inertial term (E = -Gamma for WENO5, whose
// theta-advection acts on the full J f).  The state therefore keeps FP32 resolution on the
// small deviations that carry the dynamics instead of on f ~ n w_i w_j.
//
// In FP32 mode phi is stored as hi + lo (two FP32 arrays, |lo| <= ulp(hi)/2): the kappa Delta phi
// term multiplies the storage rounding of phi by 4 kappa / h^2, and with a single FP32 array that
// rounding alone sets the FP32-vs-FP64 difference of the velocity.  The arithmetic stays FP32: hi
// differences of neighbouring nodes are exact, lo enters the Laplacian and, to first order, the
// cubic term of mu, and the Runge-Kutta update is an error-free float sum.

// Velocity-space constants (Sec. 2.3): roots v, weights w, derivative kernel K (K~ = K diag v).
struct VelocityConsts {
  double v[4];
  double w[4];
  double K[4][4];
};
VelocityConsts velocity_consts();  // computed from the Hermite definitions in FP64

template <typename T>
struct StageArgs {
  const T* fin;     // state read by the right-hand side (17 arrays)
  const T* f0;      // U^n for the Runge-Kutta combination (NULL in the first stage)
  T* fout;          // output state (may alias f0 at the same node)
  const T* coef;    // [NCOEF][n_theta]
  int nt, ns;
  int64_t stride;   // elements between consecutive arrays
  T b, dt;         // U_out = U0 + b (U_in - U0 + dt L(U_in)); without U0: U_in + dt L(U_in)
  T inv_tau, M, A, kappa, gt;  // gt = 1 / (2 r dtheta)
  T n0;             // reference density of the stored deviations
  int* err;         // device flag raised if a bounded wait on a bulk copy gives up (may be NULL)
  int ahead;        // tensor-map path: CTAs resident at once; each prefetches the tile this many ahead
  T* dphi = nullptr;  // stabilised Cahn-Hilliard: receives dt L_phi per node, and phi is not written
                      // (launch_ch_stab forms it); NULL: the stage writes phi itself
};

// Tensor maps of the FP32 UW3 stage kernel over the 18 state arrays: the halo box of the stage
// input (fin) and the U^n tile (f0).  With them, interior tiles are staged by the tensor-memory-
// access unit (cp.async.bulk.tensor) instead of per-thread copies.
struct StageMaps {
  CUtensorMap box;
  CUtensorMap tile;
};
// Whether a grid takes the tensor-map path (FP32 UW3 with n_phi % 4 == 0 and a grid at least one
// box large).
bool stage_maps_apply(int nt, int ns);
cudaError_t make_stage_maps(const float* fin, const float* f0, int nt, int ns, int64_t stride, StageMaps* out);

// Ensemble member as seen by the batched stage kernel (FP32 state).
struct EnsembleMember {
  float* U[3];        // U^n, U^(1), U^(2)
  const float* coef;  // [NCOEF][n_theta]
  int nt, ns;
  int64_t stride;
  float dt, inv_tau, M, A, kappa, gt, n0;
  int maps;  // index of the member's first tensor map in EnsembleMaps, or -1 (per-thread copies)
};

// Tensor maps of the first kEnsMapMembers ensemble members, passed as one __grid_constant__ kernel
// parameter (coherent for each launch, no proxy fence): per member the boxes of U^n, U^(1), U^(2)
// and the U^n tile, for 16-row tiles.  28 KB, inside the 32 KB kernel-parameter limit.
constexpr int kEnsMapMembers = 56;
struct EnsembleMaps {
  CUtensorMap m[4 * kEnsMapMembers];
};

// Host launchers (vlb_stage.cu).
// One stage (0, 1, 2) of every ensemble member; items[b] = (member, tile index), tile_rows 16 or 8.
// err: the ensemble's device flag, raised (2) if a bounded wait on a bulk copy gives up.
cudaError_t launch_ensemble_stage(const EnsembleMember* members, const int2* items, int nitems, int stage,
                                  int tile_rows, int ch_mode, int* err, cudaStream_t s, const EnsembleMaps* maps);
// Persistent ensemble: one cooperative launch over the same work list runs nsteps steps (with only0,
// nsteps passes of the first stage alone), with a grid barrier between stages that gives up after
// `budget` SM cycles and raises err (2).  bar: two unsigned words in device memory (arrival counter,
// generation).  skip_cta >= 0 makes that CTA skip its arrivals (a test of the timeout path).
// ctas_per_sm 0 = the occupancy limit; *grid_out = the grid used.
cudaError_t launch_ensemble_persistent(const EnsembleMember* members, const int2* items, int nitems, int nsteps,
                                       int only0, int tile_rows, int ch_mode, unsigned* bar, int* err, long long budget,
                                       int skip_cta, int ctas_per_sm, cudaStream_t s, const EnsembleMaps* maps,
                                       int* grid_out);
// Wavefront schedule of whole steps in one persistent cooperative launch (FP32 UW3 one torus; see
// wave_kernel): grids with wave_apply, up to kWaveMaxSteps steps per launch.  cnt: wave_counter_words
// unsigned words of device scratch (zeroed by the launcher).  A dependency wait that exceeds `budget`
// SM cycles raises a.err (2) and ends the launch.  stage_maps: the three stages' tensor maps.
// skip_cta >= 0 makes that CTA never report its tiles (a test of the timeout path).
constexpr int kWaveLag = 4;
constexpr int kWaveMaxSteps = 4096;
bool wave_apply(int nt, int ns);
bool wave_schedule_ok(int nb, int lag, int nsteps);  // host check of the ticket order
int wave_counter_words(int nt);
cudaError_t launch_wave(const StageArgs<float>& a, int ch_mode, float* U0, float* U1, float* U2, int nsteps,
                        unsigned* cnt, long long budget, int skip_cta, cudaStream_t st, const StageMaps* stage_maps,
                        int* grid_out);
// maps: tensor maps for this stage's fin / f0 (FP32 UW3 only), or NULL for per-thread copies.
template <typename T>
cudaError_t launch_stage(const StageArgs<T>& a, int advection, int ch_mode, cudaStream_t s,
                         const StageMaps* maps = nullptr);
// Axisymmetric grids (n_phi = 1, n_theta <= kAxiMaxRows): `steps` whole SSP-RK3 steps of the
// column in one single-CTA launch, on the buffers U0 (U^n, updated in place), U1, U2.  a.fin, a.f0,
// a.fout and a.b are set per stage inside the kernel.
constexpr int kAxiMaxRows = 4096;
template <typename T>
cudaError_t launch_axi(const StageArgs<T>& a, int advection, int ch_mode, T* U0, T* U1, T* U2, int steps,
                       cudaStream_t s);

// Stabilised semi-implicit Cahn-Hilliard (vlb_chsolve.cu): phi_out = phi^n + b (phi_in - phi^n +
// P(dphi)) with P = J^{-1} (I + dt M kappa D^2)^{-1} J (D: the constant-coefficient periodic Laplacian
// at the finest spacings); phi0 NULL in the first stage (phi^n = phi_in).  FP32: phi is a float pair,
// the low word lo_off elements after the high word.  buf: ch_stab_buffer_bytes of scratch whose tail
// holds the factor tables of lambda and the twiddles of both transform lengths, written once by
// ch_stab_tables (host, FP64 then rounded to esize) and copied to the device by the caller.
bool ch_stab_shape_ok(int nt, int ns);
size_t ch_stab_buffer_bytes(int nt, int ns, size_t esize);
size_t ch_stab_table_offset(int nt, int ns, size_t esize);  // bytes from buf to the tables
size_t ch_stab_table_elems(int nt, int ns);                   // elements of esize in the tables
void ch_stab_tables(int nt, int ns, double h_t, double h_p, size_t esize, void* host_out);
template <typename T>
cudaError_t launch_ch_stab(int nt, int ns, double dt_m_kappa, const double* J, const T* dphi, void* buf, const T* phin,
                           const T* phi0, T* phiout, int64_t lo_off, T b, cudaStream_t st);

// Structure-factor sums (vlb_chsolve.cu, same power-of-two shapes): FP64 transform of phi (+ phi_lo
// when not NULL) into buf (n_theta * n_phi complex doubles), then structure_blocks(nt, ns) CTAs write
// part[2 b] = sum S and part[2 b + 1] = sum |k| S over their strips (k = (m'/r, n'/R), mean mode left out).
int structure_blocks(int nt, int ns);
template <typename T>
cudaError_t launch_structure_sums(int nt, int ns, double r, double R, const T* phi, const T* phi_lo, void* buf,
                                  double* part, cudaStream_t st);

// Auxiliary kernels (vlb_aux.cu).  Staging arrays are FP64 [n_theta][n_phi].
// out[q] = the sum of row q of x (FP64 [nt][ns]), in a fixed order.
cudaError_t launch_row_sums(const double* x, int nt, int ns, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_init_feq(T* state, int64_t stride, const double* rho, const double* ut,
                            const double* up, const double* phi, int64_t n, double n0, cudaStream_t s);
template <typename T>
cudaError_t launch_convert_in(T* state, int64_t stride, const double* src, int64_t n, double n0, cudaStream_t s);
template <typename T>
cudaError_t launch_convert_out(double* dst, const T* state, int64_t stride, int64_t n, double n0, cudaStream_t s);
template <typename T>
cudaError_t launch_fields(const T* state, int64_t stride, const double* coefd, int nt, int ns, double A,
                          double kappa, double n0, double* rho, double* ut, double* up, double* phi, double* mu,
                          cudaStream_t s);
// partials: n_blocks x 8 doubles; out: 8 doubles
// out[0] mass, out[1] phi total, out[2] Psi, out[3] max|u|, out[4] non-finite count, out[5] L_I
template <typename T>
cudaError_t launch_totals(const T* state, int64_t stride, const double* coefd, int nt, int ns, double R,
                          double r, double A, double kappa, double n0, int geometry, double* partials,
                          int n_blocks, double* out, cudaStream_t s);
int totals_blocks();

// Solver snapshots (vlb_aux.cu): FP32 [N][4] = (phi, n, u_theta, u_phi) on the device.
template <typename T>
cudaError_t launch_snapshot_out(const T* state, int64_t stride, int64_t n, double n0, float* snap, cudaStream_t s);
template <typename T>
cudaError_t launch_snapshot_in(T* state, int64_t stride, int64_t n, double n0, const float* snap, const double* shift,
                               int keep_neq, cudaStream_t s);
// shift[0..1] := the uniform shifts of n and phi that give the snapshot the totals (mass, phi_total)
cudaError_t launch_snapshot_shift(const float* snap, const double* coefd, int nt, int ns, double mass,
                                  double phi_total, double inv_area, double* partials, double* shift, cudaStream_t s);

// Surrogate network kernels (vlb_conv.cu, vlb_surrogate.cu).
bool conv_shape_ok(int H, int W, int cin, int cout, const char** why);
size_t conv_wgrad_workspace_bytes(int H, int W, int cin, int cout);
// the forward on the tcgen05 tensor cores (vlb_conv_tc.cu)
cudaError_t conv_fwd_tc(int H, int W, int cin, int cout, const void* x, const void* w, const float* b,
                        const void* mask, int relu, void* y, float* yf, cudaStream_t st);
// partial[group][tap][co][ci] of a weight gradient on tcgen05 (vlb_conv_tc.cu; (c_in, c_out) = (64, 64),
// (16, 64) or (64, 16)); group g covers row segments (128 pixels) g * segs_per_group ..  With bpart,
// also bpart[group][co] = the group's sum of dY[p][co] (the bias gradient's partials).
cudaError_t conv_wgrad_tc(int H, int W, int cin, int cout, const void* x, const void* dy, float* partial, float* bpart,
                          int segs_per_group, cudaStream_t st);
// The device-wide flag raised (1) when a bounded wait of a tensor-core convolution gives up: read
// after synchronising st (and cleared if `clear`); conv_tc_raise sets it (tests of the status path).
cudaError_t conv_tc_status(cudaStream_t st, int clear, int* raised);
cudaError_t conv_tc_raise(int value);
cudaError_t conv_flip(int cin, int cout, const void* w, void* wf, cudaStream_t st);
cudaError_t conv_wgrad(int H, int W, int cin, int cout, const void* x, const void* dy, float* dw, float* db,
                       float* partial, cudaStream_t st);
cudaError_t sur_norm(int64_t n, const float* snap, float s_n, float s_u, const float* g4, double* part, double* sums,
                     float* norm8, cudaStream_t st);
cudaError_t sur_features(int H, int W, double a, const float* snap, const float* norm4, void* out, cudaStream_t st);
cudaError_t sur_compare(int64_t n, const float* a, const float* b, double* part, double* out4, cudaStream_t st);
cudaError_t sur_targets(int64_t n, const float* before, const float* after, const float* scale4, float* target,
                        cudaStream_t st);
cudaError_t sur_apply(int64_t n, const float* before, const float* pred, const float* scale4, float* after,
                      cudaStream_t st);
cudaError_t sur_stats(int64_t n, int C, const float* x, double* part, double* out, cudaStream_t st);
cudaError_t sur_mse(int64_t n, const float* pred, const float* target, void* grad, double* part, double* loss,
                    cudaStream_t st);
cudaError_t sur_adam(int64_t n, float* p, const float* g, float* m, float* v, int64_t t, float lr, float b1, float b2,
                     float eps, void* pb, cudaStream_t st);
cudaError_t sur_to_bf16(int64_t n, const float* x, void* y, cudaStream_t st);
size_t sur_reduce_doubles();

}  // namespace vlb
