// Surrogate-accelerated stepping behind the C ABI (not part of the paper's method).
//
// A surrogate handle holds the learned network (an 8-layer periodic 3 x 3 CNN, 16 -> 64, six
// 64 -> 64, 64 -> 16 channels, BF16 weights, FP32 biases) and the buffers of one prediction.  It
// advances an FP32 solver by windows of `window` steps: most windows are predicted by the network,
// and every check_every-th window is judged by the solver, which runs the window from the same state.
// The judge compares phi (relative L2 or relative L-infinity error); a prediction within phi_tol
// keeps the solver's result, a larger error (or a non-finite value) rolls the state back to the last
// judged one, lets the solver redo the windows since, and runs the next check_every windows with
// the solver alone.  A taken prediction (n', u', phi') replaces f by f + f^eq(n', u') - f^eq(n, u),
// keeping the non-equilibrium part, with int n sqrt(g) and int phi sqrt(g) restored to their values
// when the handle was bound to the solver.  Between judged windows nothing is read back to the host,
// and on a stream that can be captured a predicted window replays as one CUDA graph.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "vlb_handle.cuh"

namespace {

constexpr int kLayers = 8;
constexpr int kCin[kLayers] = {16, 64, 64, 64, 64, 64, 64, 64};
constexpr int kCout[kLayers] = {64, 64, 64, 64, 64, 64, 64, 16};

constexpr size_t weight_count() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)kCout[l] * 9 * kCin[l];
  return n;
}
constexpr size_t bias_count() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)kCout[l];
  return n;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

struct SurLayout {
  size_t off_w, off_b, off_act[3], off_out, off_snap, off_pred, off_check, off_norm, off_cmp, off_red, off_sums,
      off_good, total;
};

SurLayout sur_layout(const vlb_params* p) {
  SurLayout L;
  const size_t N = (size_t)p->n_theta * p->n_phi;
  const size_t stride = (N + 63) / 64 * 64;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = a256(off + bytes);
    return o;
  };
  L.off_w = take(2 * weight_count());
  L.off_b = take(4 * bias_count());
  L.off_act[0] = take(N * 16 * 2);
  L.off_act[1] = take(N * 64 * 2);
  L.off_act[2] = take(N * 64 * 2);
  L.off_out = take(N * 16 * 4);
  L.off_snap = take(N * 16);
  L.off_pred = take(N * 16);
  L.off_check = take(N * 16);
  L.off_norm = take(8 * 4);
  L.off_cmp = take(4 * 8);
  L.off_red = take(sizeof(double) * vlb::sur_reduce_doubles());
  L.off_sums = take(8 * 8);
  L.off_good = take((size_t)vlb::state_arrays(4) * stride * 4);
  L.total = off;
  return L;
}

bool sur_params_ok(const vlb_params* p, char* why, size_t n) {
  if (!p) return snprintf(why, n, "geometry params are NULL"), false;
  if (p->precision != VLB_FP32) return snprintf(why, n, "the surrogate advances FP32 solvers"), false;
  const char* w = nullptr;
  if (!vlb::conv_shape_ok(p->n_theta, p->n_phi, 16, 64, &w)) return snprintf(why, n, "grid: %s", w), false;
  if (!(p->R > 0.0) || !(p->r > 0.0)) return snprintf(why, n, "radii must be > 0"), false;
  return true;
}

vlb_status fail(vlb_handle* h, vlb_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
vlb_status fail(vlb_handle* h, vlb_status st, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  return vlb_internal_fail(h, st, msg);
}

#define SUR_CUDA(h, call)                                                                                  \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return fail((h), VLB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// A failed public call on the solver: its message is carried over to the surrogate handle.
vlb_status relay(vlb_handle* sur, vlb_handle* solver, vlb_status st, const char* what) {
  if (st == VLB_OK) return st;
  return fail(sur, st, "%s: %s", what, vlb_last_error(solver));
}

// pred := the network's estimate of snap one window ahead (all on the device, on st)
vlb_status predict(vlb_handle* h, const float* snap, float* pred, cudaStream_t st) {
  const int H = h->sur_H, W = h->sur_W;
  const int64_t N = (int64_t)H * W;
  SUR_CUDA(h, vlb::sur_norm(N, snap, h->sur_s_n, h->sur_s_u, h->sur_g, h->sur_red, h->sur_sums, h->sur_norm, st));
  SUR_CUDA(h, vlb::sur_features(H, W, h->sur_r_over_R, snap, h->sur_norm, h->sur_act[0], st));
  const unsigned char* w = static_cast<const unsigned char*>(h->sur_w);
  const float* b = h->sur_b;
  const void* x = h->sur_act[0];
  for (int l = 0; l < kLayers; ++l) {
    const bool last = l == kLayers - 1;
    void* y = last ? nullptr : h->sur_act[1 + (l & 1)];
    SUR_CUDA(h, vlb::conv_fwd_tc(H, W, kCin[l], kCout[l], x, w, b, nullptr, last ? 0 : 1, y,
                                 last ? h->sur_out : nullptr, st));
    w += 2 * (size_t)kCout[l] * 9 * kCin[l];
    b += kCout[l];
    x = y;
  }
  SUR_CUDA(h, vlb::sur_apply(N, snap, h->sur_out, h->sur_norm + 4, pred, st));
  return VLB_OK;
}

// One predicted window: snapshot, prediction, restart of the solver from it (conserving the totals).
vlb_status predicted_body(vlb_handle* h, vlb_handle* s, cudaStream_t st) {
  vlb_status r = relay(h, s, vlb_get_snapshot(s, h->sur_snap), "vlb_get_snapshot");
  if (r) return r;
  if ((r = predict(h, h->sur_snap, h->sur_pred, st))) return r;
  return relay(h, s, vlb_set_snapshot(s, h->sur_pred, h->sur_conserve, 1), "vlb_set_snapshot");
}

bool capturable(cudaStream_t st) { return (uintptr_t)st > 2; }  // not the legacy or per-thread default stream

vlb_status predicted_window(vlb_handle* h, vlb_handle* s, cudaStream_t st, bool use_graph) {
  h->sur_predicted++;
  // the first predicted window of a binding runs eagerly (one-time set-up of the kernels happens
  // outside any capture); later ones replay a graph captured on the solver's stream
  if (!use_graph || !capturable(st) || h->sur_predicted == 1) return predicted_body(h, s, st);
  if (h->sur_graph && h->sur_graph_stream != st) {
    cudaGraphExecDestroy(h->sur_graph);
    h->sur_graph = nullptr;
  }
  if (!h->sur_graph) {
    cudaGraph_t g = nullptr;
    SUR_CUDA(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    vlb_status r = predicted_body(h, s, st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (r != VLB_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return fail(h, VLB_ERR_CUDA, "capture of a predicted window: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->sur_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->sur_graph = nullptr;
      return fail(h, VLB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    h->sur_graph_stream = st;
  }
  SUR_CUDA(h, cudaGraphLaunch(h->sur_graph, st));
  return VLB_OK;
}

vlb_status save_state(vlb_handle* h, vlb_handle* s, cudaStream_t st, int64_t* saved_steps) {
  const size_t bytes = (size_t)vlb::state_arrays(4) * s->stride * 4;
  SUR_CUDA(h, cudaMemcpyAsync(h->sur_good, s->U[0], bytes, cudaMemcpyDeviceToDevice, st));
  h->sur_since_good = 0;
  *saved_steps = s->steps_done;
  return VLB_OK;
}

vlb_status bind(vlb_handle* h, vlb_handle* s) {
  double t[4];
  vlb_status r = relay(h, s, vlb_get_totals(s, t), "vlb_get_totals");
  if (r) return r;
  h->sur_bound = s;
  h->sur_conserve[0] = t[0];
  h->sur_conserve[1] = t[1];
  h->sur_count = h->sur_predicted = h->sur_fallbacks = 0;
  h->sur_solver_only = h->sur_since_good = 0;
  if (h->sur_graph) {
    cudaGraphExecDestroy(h->sur_graph);
    h->sur_graph = nullptr;
  }
  return VLB_OK;
}

}  // namespace

extern "C" {

size_t vlb_surrogate_workspace_bytes(const vlb_params* geom) {
  char why[256];
  if (!sur_params_ok(geom, why, sizeof why)) {
    fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_workspace_bytes: %s", why);
    return 0;
  }
  return sur_layout(geom).total;
}

vlb_status vlb_surrogate_create(const vlb_params* geom, const vlb_surrogate_net* net, void* d_workspace, size_t bytes,
                                void* cuda_stream, vlb_handle** out) {
  char why[256];
  if (!out) return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: out is NULL");
  *out = nullptr;
  if (!sur_params_ok(geom, why, sizeof why)) return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: %s", why);
  if (!net || !net->weights_bf16 || !net->biases) return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: no network");
  if (net->window < 1 || net->reserved != 0) return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: window must be > 0");
  if (!(net->s_n > 0.0f) || !(net->s_u > 0.0f) || !isfinite(net->s_n) || !isfinite(net->s_u))
    return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: input scales must be finite and > 0");
  for (int c = 0; c < 4; ++c)
    if (!(net->g[c] > 0.0f) || !isfinite(net->g[c]))
      return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_create: output ratios must be finite and > 0");
  const SurLayout L = sur_layout(geom);
  if (!d_workspace) return fail(nullptr, VLB_ERR_WORKSPACE, "vlb_surrogate_create: workspace is NULL");
  if (((uintptr_t)d_workspace) % 256 != 0)
    return fail(nullptr, VLB_ERR_WORKSPACE, "vlb_surrogate_create: workspace not 256-byte aligned");
  if (bytes < L.total)
    return fail(nullptr, VLB_ERR_WORKSPACE, "vlb_surrogate_create: workspace too small: %zu < %zu bytes", bytes,
                L.total);
  vlb_handle* h = new (std::nothrow) vlb_handle();
  if (!h) return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  unsigned char* ws = (unsigned char*)d_workspace;
  h->kind = 3;
  h->p = *geom;
  h->stream = (cudaStream_t)cuda_stream;
  h->ws = ws;
  h->ws_bytes = bytes;
  h->esize = 4;
  h->N = (int64_t)geom->n_theta * geom->n_phi;
  h->stride = (h->N + 63) / 64 * 64;
  h->err[0] = 0;
  h->sur_H = geom->n_theta;
  h->sur_W = geom->n_phi;
  h->sur_window = net->window;
  h->sur_r_over_R = geom->r / geom->R;
  h->sur_s_n = net->s_n;
  h->sur_s_u = net->s_u;
  for (int c = 0; c < 4; ++c) h->sur_g[c] = net->g[c];
  h->sur_w = ws + L.off_w;
  h->sur_b = (float*)(ws + L.off_b);
  for (int k = 0; k < 3; ++k) h->sur_act[k] = ws + L.off_act[k];
  h->sur_out = (float*)(ws + L.off_out);
  h->sur_snap = (float*)(ws + L.off_snap);
  h->sur_pred = (float*)(ws + L.off_pred);
  h->sur_check = (float*)(ws + L.off_check);
  h->sur_norm = (float*)(ws + L.off_norm);
  h->sur_cmp = (double*)(ws + L.off_cmp);
  h->sur_red = (double*)(ws + L.off_red);
  h->sur_sums = (double*)(ws + L.off_sums);
  h->sur_good = ws + L.off_good;
  cudaError_t e = cudaGetDevice(&h->device);
  // the network is copied in: the caller's buffers (host or device memory) may be released afterwards
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->sur_w, net->weights_bf16, 2 * weight_count(), cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->sur_b, net->biases, 4 * bias_count(), cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, VLB_ERR_CUDA, "vlb_surrogate_create: %s", cudaGetErrorString(e));
  }
  *out = h;
  return VLB_OK;
}

vlb_status vlb_surrogate_advance(vlb_handle* solver, vlb_handle* sur, int32_t nwindows, int32_t check_every,
                                 double phi_tol, int32_t options, int32_t* kinds, double* errors, int32_t* fell_back) {
  if (fell_back) *fell_back = 0;
  if (!sur || sur->kind != 3) return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: not a surrogate handle");
  vlb_handle* s = solver;
  if (!s || (s->kind != 0 && s->kind != 2))
    return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: not a solver handle (or an ensemble member view)");
  if (s->esize != 4) return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: the surrogate advances FP32 solvers");
  if (s->p.n_theta != sur->sur_H || s->p.n_phi != sur->sur_W)
    return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: the solver's grid is not the network's (%d x %d)", sur->sur_H,
                sur->sur_W);
  if (nwindows < 0 || check_every < 0 || isnan(phi_tol) || phi_tol < 0.0)
    return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: nwindows, check_every >= 0 and phi_tol >= 0 required");
  if (options & ~(VLB_SUR_JUDGE_LINF | VLB_SUR_NO_GRAPH))
    return fail(sur, VLB_ERR_ARG, "vlb_surrogate_advance: unknown option bits");
  int dev = -1;
  SUR_CUDA(sur, cudaGetDevice(&dev));
  if (dev != sur->device) SUR_CUDA(sur, cudaSetDevice(sur->device));
  cudaStream_t st = s->stream;
  vlb_status r;
  if (sur->sur_bound != s && (r = bind(sur, s))) return r;
  const int w = sur->sur_window;
  const int64_t N = s->N;
  const bool use_graph = !(options & VLB_SUR_NO_GRAPH);
  int64_t& saved_steps = sur->sur_good_steps;  // the bound solver's step count at the last judged state
  for (int32_t k = 0; k < nwindows; ++k) {
    int kind;
    double e2 = NAN, einf = NAN;
    if (sur->sur_count == 0 && (r = save_state(sur, s, st, &saved_steps))) return r;
    sur->sur_count++;
    if (sur->sur_solver_only > 0) {
      if ((r = relay(sur, s, vlb_step(s, w), "vlb_step"))) return r;
      sur->sur_solver_only--;
      sur->sur_since_good++;
      if (sur->sur_solver_only == 0 && (r = save_state(sur, s, st, &saved_steps))) return r;
      kind = VLB_WINDOW_SOLVER;
    } else if (check_every > 0 && sur->sur_count % check_every == 0) {
      // judged window: the network's prediction and the solver's window from the same state
      if ((r = relay(sur, s, vlb_get_snapshot(s, sur->sur_snap), "vlb_get_snapshot"))) return r;
      if ((r = predict(sur, sur->sur_snap, sur->sur_pred, st))) return r;
      if ((r = relay(sur, s, vlb_step(s, w), "vlb_step"))) return r;
      if ((r = relay(sur, s, vlb_get_snapshot(s, sur->sur_check), "vlb_get_snapshot"))) return r;
      SUR_CUDA(sur, vlb::sur_compare(N, sur->sur_pred, sur->sur_check, sur->sur_red, sur->sur_cmp, st));
      double c[4];
      SUR_CUDA(sur, cudaMemcpyAsync(c, sur->sur_cmp, sizeof c, cudaMemcpyDeviceToHost, st));
      int raised = 0;
      SUR_CUDA(sur, vlb::conv_tc_status(st, 0, &raised));  // synchronises st
      if (raised)
        return fail(sur, VLB_ERR_TIMEOUT, "vlb_surrogate_advance: a bounded wait of a tensor-core convolution gave up");
      einf = c[1] > 0.0 ? c[0] / c[1] : INFINITY;
      e2 = c[3] > 0.0 ? sqrt(c[2] / c[3]) : INFINITY;
      const double err = (options & VLB_SUR_JUDGE_LINF) ? einf : e2;
      if (err <= phi_tol) {  // NaN fails too
        if ((r = save_state(sur, s, st, &saved_steps))) return r;
        kind = VLB_WINDOW_CHECKED;
      } else {
        // back to the last judged state; the solver redoes the windows since, then runs alone
        const size_t bytes = (size_t)vlb::state_arrays(4) * s->stride * 4;
        SUR_CUDA(sur, cudaMemcpyAsync(s->U[0], sur->sur_good, bytes, cudaMemcpyDeviceToDevice, st));
        s->steps_done = saved_steps;
        if ((r = relay(sur, s, vlb_step(s, (int64_t)w * (sur->sur_since_good + 1)), "vlb_step"))) return r;
        sur->sur_solver_only = check_every;
        if ((r = save_state(sur, s, st, &saved_steps))) return r;
        kind = VLB_WINDOW_FALLBACK;
        sur->sur_fallbacks++;
        if (fell_back) (*fell_back)++;
      }
    } else {
      if ((r = predicted_window(sur, s, st, use_graph))) return r;
      s->steps_done += w;  // the state stands for the window's end
      sur->sur_since_good++;
      kind = VLB_WINDOW_SURROGATE;
    }
    if (kinds) kinds[k] = kind;
    if (errors) {
      errors[2 * k] = e2;
      errors[2 * k + 1] = einf;
    }
  }
  return VLB_OK;
}

vlb_status vlb_surrogate_stats(const vlb_handle* sur, int64_t out[4]) {
  if (!sur || sur->kind != 3 || !out)
    return fail(const_cast<vlb_handle*>(sur), VLB_ERR_ARG, "vlb_surrogate_stats: bad argument");
  out[0] = sur->sur_count;
  out[1] = sur->sur_predicted;
  out[2] = sur->sur_fallbacks;
  out[3] = sur->sur_graph ? 1 : 0;
  return VLB_OK;
}

}  // extern "C"
