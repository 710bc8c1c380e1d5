// The handle behind the C ABI's opaque vlb_handle (internal to libvlb).  One struct serves the
// four kinds of handle: a solver, an ensemble, a member view of an ensemble, and a surrogate.
#pragma once

#include "vlb_internal.cuh"

struct vlb_handle {
  vlb_params p;
  cudaStream_t stream;
  int device;
  int64_t N;       // n_theta * n_phi
  int64_t stride;  // elements between state arrays
  size_t esize;    // 4 or 8
  unsigned char* ws;
  size_t ws_bytes;
  void* U[3];          // U^n, U^(1), U^(2)
  void* coefT;         // [NCOEF][n_theta] in state precision
  double* coefD;       // [NCOEF][n_theta] FP64
  double* staging;     // 17 N doubles
  double* partials;    // totals_blocks() * 8
  double* totals;      // 8 doubles (read-out)
  double* diag;        // 8 doubles (last in-step diagnostic)
  int* flag;           // device flag: diagnostics found an unstable state (1) or a bulk copy gave up (2)
  void* dphi = nullptr;  // stabilised Cahn-Hilliard: dt L_phi of a stage (state precision, N)
  void* fft = nullptr;   // stabilised Cahn-Hilliard: complex spectrum (N complex)
  vlb::StageMaps* maps = nullptr;  // FP32 UW3: tensor maps of the three stage inputs (NULL: per-thread copies)
  unsigned* wave_cnt = nullptr;    // FP32 UW3: counters of the wavefront schedule (NULL: not available)
  int sched = 0;                   // VLB_SCHED_AUTO / STAGES / WAVE (vlb_set_schedule)
  int wave_skip = -1;              // test hook: a wavefront CTA that never reports its tiles
  long long wave_budget = 0;       // wavefront dependency-wait budget in SM cycles (0 = default)
  vlb::EnsembleMaps* ens_maps = nullptr;  // ensemble: members' tensor maps, passed to each launch
  double n0;           // reference density of the stored deviations g = f - n0 w_i w_j
  int64_t steps_done;
  char err[512];
  // ensembles
  int kind = 0;                              // 0 solver, 1 ensemble, 2 member view, 3 surrogate
  vlb_handle* parent = nullptr;              // view: its ensemble
  int index = 0;                             // view: member index
  int count = 0;                             // ensemble: members
  vlb_handle** views = nullptr;              // ensemble: one view per member
  vlb::EnsembleMember* d_members = nullptr;  // ensemble: device descriptors
  int2* d_items[2] = {nullptr, nullptr};     // ensemble: work lists for tile rows 16 and 8
  int nitems[2] = {0, 0};
  int tile_rows = 0;                         // ensemble: autotuner's choice, 0 = not tuned yet
  float tune_ms[2] = {0.0f, 0.0f};
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_1 = nullptr, graph_32 = nullptr;  // one step, 32 steps
  // ensemble execution: mode 1 = one batched launch per stage, 2 = one persistent cooperative launch
  // per block of steps (grid barrier between stages); 0 = not chosen yet
  int ens_mode = 0, ens_ctas = 0, ens_grid = 0;
  int ens_req_mode = 0, ens_req_rows = 0, ens_req_ctas = 0;  // requested by vlb_ensemble_configure (0 = tune)
  int ens_skip = -1;                 // test hook: a persistent CTA that skips its barrier arrivals
  long long ens_budget = 0;          // grid-barrier budget in SM cycles (0 = default)
  unsigned* ens_bar = nullptr;       // grid barrier: arrival counter, generation
  float ens_ms[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // autotuner: batched 16 / 8, persistent 16 / 8
  int ens_from_cache = 0;
  bool ens_graphs = true;            // false if the launch could not be captured (replayed eagerly)
  // surrogate (kind 3): the network, its buffers in the workspace and the state of the advance loop
  int sur_H = 0, sur_W = 0, sur_window = 0;
  double sur_r_over_R = 0.0;
  float sur_s_n = 0.0f, sur_s_u = 0.0f, sur_g[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  void* sur_w = nullptr;       // the 8 layers' bf16 weights, concatenated
  float* sur_b = nullptr;      // their FP32 biases, concatenated
  void* sur_act[3] = {nullptr, nullptr, nullptr};  // input features (16 ch), two 64-channel buffers
  float* sur_out = nullptr;    // last layer, FP32 16 channels
  float* sur_snap = nullptr;   // snapshot of the solver, prediction, solver's check: FP32 [N][4]
  float* sur_pred = nullptr;
  float* sur_check = nullptr;
  float* sur_norm = nullptr;   // 8 floats: input statistics and output scales
  double* sur_cmp = nullptr;   // 4 doubles: comparison of prediction and check
  double* sur_red = nullptr;   // reduction scratch
  double* sur_sums = nullptr;  // 8 doubles
  void* sur_good = nullptr;    // the last judged state of the bound solver
  vlb_handle* sur_bound = nullptr;  // the solver the advance loop follows
  double sur_conserve[2] = {0.0, 0.0};
  int64_t sur_count = 0, sur_predicted = 0, sur_fallbacks = 0, sur_good_steps = 0;
  int sur_solver_only = 0, sur_since_good = 0;
  cudaGraphExec_t sur_graph = nullptr;  // one predicted window, replayed on the bound solver's stream
  cudaStream_t sur_graph_stream = nullptr;
};

// Records msg as the last error of h (or of the calling thread when h is NULL) and returns st.
vlb_status vlb_internal_fail(vlb_handle* h, vlb_status st, const char* msg);
