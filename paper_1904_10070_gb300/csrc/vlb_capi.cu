// C ABI of libvlb: parameter validation, geometry tables, workspace layout and the step driver.
//
// Geometry (App. A): x = (R + r cos theta) cos varphi, y = (R + r cos theta) sin varphi,
// z = r sin theta; metric g_phiphi = (R + r cos theta)^2, g_thth = r^2; vielbein
// e_phi = 1/(R + r cos theta), e_theta = 1/r; the only connection coefficient is
// Gamma = sin theta / (R + r cos theta) (Eq. conn_torus).  The tables below are evaluated in
// FP64 per theta row and rounded once to the state precision.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vlb_handle.cuh"

// Raises the handle's device flag when a diagnostic vector shows an unstable state.
cudaError_t vlb_internal_flag(const double* diag, int* flag, cudaStream_t s);

// struct vlb_handle is defined in vlb_handle.cuh.

namespace {

thread_local char g_err[512] = "";

vlb_status fail(vlb_handle* h, vlb_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
vlb_status fail(vlb_handle* h, vlb_status st, const char* fmt, ...) {
  char* dst = h ? h->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define VLB_CUDA(h, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail((h), VLB_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                       \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool params_ok(const vlb_params* p, char* why, size_t n) {
  if (!p) return snprintf(why, n, "params is NULL"), false;
  if (p->geometry != VLB_TORUS && p->geometry != VLB_FLAT) return snprintf(why, n, "geometry must be 0 or 1"), false;
  if (p->precision != VLB_FP64 && p->precision != VLB_FP32) return snprintf(why, n, "precision must be 0 or 1"), false;
  if (p->advection != VLB_UW3 && p->advection != VLB_WENO5) return snprintf(why, n, "advection must be 0 or 1"), false;
  if (p->ch_mode != VLB_HYDRO && p->ch_mode != VLB_DIFFUSIVE) return snprintf(why, n, "ch_mode must be 0 or 1"), false;
  const int nt_min = p->advection == VLB_WENO5 ? 6 : 4;
  if (p->n_theta < nt_min) return snprintf(why, n, "n_theta must be >= %d", nt_min), false;
  if (p->n_phi < 1) return snprintf(why, n, "n_phi must be >= 1"), false;
  if (p->n_theta > 65535 * 16) return snprintf(why, n, "n_theta must be <= %d", 65535 * 16), false;
  if ((int64_t)p->n_theta * p->n_phi > (int64_t)1 << 31) return snprintf(why, n, "grid larger than 2^31 nodes"), false;
  if (p->diag_every < 0) return snprintf(why, n, "diag_every must be >= 0"), false;
  if (p->ch_stab != 0 && p->ch_stab != 1) return snprintf(why, n, "ch_stab must be 0 or 1"), false;
  if (p->ch_stab && !vlb::ch_stab_shape_ok(p->n_theta, p->n_phi))
    return snprintf(why, n, "ch_stab needs n_theta and n_phi powers of two in 4 .. 4096"), false;
  if (!(p->r > 0.0) || !(p->R > 0.0) || !isfinite(p->r) || !isfinite(p->R))
    return snprintf(why, n, "radii must be finite and positive"), false;
  if (p->geometry == VLB_TORUS && !(p->R > p->r)) return snprintf(why, n, "torus needs R > r"), false;
  if (!(p->dt > 0.0) || !isfinite(p->dt)) return snprintf(why, n, "dt must be finite and > 0"), false;
  if (!(p->tau > 0.0)) return snprintf(why, n, "tau must be > 0 (inf allowed)"), false;
  if (!(p->M >= 0.0) || !(p->A >= 0.0) || !(p->kappa >= 0.0) || !isfinite(p->M) || !isfinite(p->A) ||
      !isfinite(p->kappa))
    return snprintf(why, n, "M, A, kappa must be finite and >= 0"), false;
  return true;
}

struct Layout {
  int64_t N, stride;
  size_t esize;
  size_t off_coefT, off_coefD, off_U[3], off_staging, off_partials, off_totals, off_diag, off_flag, off_dphi, off_fft,
      off_wave, total;
};

Layout layout(const vlb_params* p) {
  Layout L;
  L.N = (int64_t)p->n_theta * p->n_phi;
  L.stride = (int64_t)align_up((size_t)L.N, 64);
  L.esize = p->precision == VLB_FP64 ? 8 : 4;
  size_t off = 0;
  L.off_coefT = off;
  off = align_up(off + (size_t)vlb::NCOEF * p->n_theta * L.esize, 256);
  L.off_coefD = off;
  off = align_up(off + (size_t)vlb::NCOEF * p->n_theta * 8, 256);
  for (int k = 0; k < 3; ++k) {
    L.off_U[k] = off;
    off = align_up(off + (size_t)vlb::state_arrays(L.esize) * L.stride * L.esize, 256);
  }
  L.off_staging = off;
  off = align_up(off + (size_t)vlb::NARR * L.N * 8, 256);
  L.off_partials = off;
  off = align_up(off + (size_t)vlb::totals_blocks() * 8 * 8, 256);
  L.off_totals = off;
  off = align_up(off + 8 * 8, 256);
  L.off_diag = off;
  off = align_up(off + 8 * 8, 256);
  L.off_flag = off;
  off = align_up(off + 256, 256);
  L.off_dphi = L.off_fft = 0;
  if (p->ch_stab) {  // dt L_phi of a stage and the complex spectrum of the stabilised solve
    L.off_dphi = off;
    off = align_up(off + (size_t)L.N * L.esize, 256);
    L.off_fft = off;
    off = align_up(off + vlb::ch_stab_buffer_bytes(p->n_theta, p->n_phi, L.esize), 256);
  }
  L.off_wave = 0;
  if (L.esize == 4 && p->advection == VLB_UW3 && !p->ch_stab && vlb::wave_apply(p->n_theta, p->n_phi)) {
    L.off_wave = off;  // band counters and the ticket of the wavefront schedule
    off = align_up(off + sizeof(unsigned) * vlb::wave_counter_words(p->n_theta), 256);
  }
  L.total = off;
  return L;
}

// Row tables in FP64 (see RowCoef for the meaning of each entry).
void row_tables(const vlb_params* p, double* out) {
  const int nt = p->n_theta;
  const double dth = 2.0 * M_PI / nt, dph = 2.0 * M_PI / p->n_phi;
  const bool torus = p->geometry == VLB_TORUS;
  const double a = torus ? p->r / p->R : 0.0;
  for (int q = 0; q < nt; ++q) {
    const double th = q * dth;
    const double J = 1.0 + a * cos(th);
    const double Jp = 1.0 + a * cos(th + 0.5 * dth);
    const double Jm = 1.0 + a * cos(th - 0.5 * dth);
    out[vlb::C_J * nt + q] = J;
    out[vlb::C_JP * nt + q] = Jp;
    out[vlb::C_JM * nt + q] = Jm;
    out[vlb::C_CT * nt + q] = 1.0 / (p->r * J * dth);
    out[vlb::C_CP * nt + q] = 1.0 / (p->R * J * dph);
    out[vlb::C_GAM * nt + q] = torus ? sin(th) / (p->R * J) : 0.0;
    out[vlb::C_LT * nt + q] = 1.0 / (p->r * p->r * J * dth * dth);
    out[vlb::C_LP * nt + q] = 1.0 / (p->R * p->R * J * J * dph * dph);
    out[vlb::C_GP * nt + q] = 1.0 / (2.0 * p->R * J * dph);
    // Rest-state residual E(q) = -D[J](q) / (r J dtheta) - Gamma (UW3 flux differences of the
    // J row values, v > 0 and v < 0); WENO5 advects the full J f, leaving E = -Gamma.
    const double gam = out[vlb::C_GAM * nt + q];
    if (p->advection == VLB_UW3) {
      auto Jat = [&](int d) { return 1.0 + a * cos(th + d * dth); };
      const double dpos = (Jat(-2) - 6.0 * Jat(-1) + 3.0 * Jat(0) + 2.0 * Jat(1)) / 6.0;
      const double dneg = (-2.0 * Jat(-1) - 3.0 * Jat(0) + 6.0 * Jat(1) - Jat(2)) / 6.0;
      out[vlb::C_EP * nt + q] = -dpos / (p->r * J * dth) - gam;
      out[vlb::C_EN * nt + q] = -dneg / (p->r * J * dth) - gam;
    } else {
      out[vlb::C_EP * nt + q] = -gam;
      out[vlb::C_EN * nt + q] = -gam;
    }
    out[vlb::C_DA * nt + q] = p->r * p->R * J * dth * dph;
    out[vlb::C_EDGE * nt + q] = torus ? (p->R + p->r * cos(th + 0.5 * dth)) * dph : p->R * dph;
  }
}

// The reference density n0 of the stored deviations from the row sums of n: the area-weighted mean
// sum_q J_q row_q / sum_q J_q N_phi (J_q = 1 + (r/R) cos theta_q), rounded to 20 significant bits so
// that it is exact in FP32.  False if it is not finite and positive.
bool reference_density_rows(const vlb_params& p, const double* rows, double* out) {
  const double dth = 2.0 * M_PI / p.n_theta;
  const double a = p.geometry == VLB_TORUS ? p.r / p.R : 0.0;
  double num = 0.0, den = 0.0;
  for (int q = 0; q < p.n_theta; ++q) {
    const double J = 1.0 + a * cos(q * dth);
    num += J * rows[q];
    den += J * p.n_phi;
  }
  const double mean = num / den;
  if (!isfinite(mean) || !(mean > 0.0)) return false;
  int e = 0;
  const double m = frexp(mean, &e);
  *out = ldexp(nearbyint(ldexp(m, 20)), e - 20);
  return true;
}

// Reference density n0 of the stored deviations: the area-weighted mean density
// sum_q J_q sum_s n_qs / (N_phi sum_q J_q), rounded to 20 significant bits.  The scheme conserves
// sum n sqrt(g), so a state restored from a checkpoint reproduces the same n0 (and bitwise the same
// stored deviations).  `n_at(q, s)` returns the density at a node.
template <typename F>
bool reference_density(const vlb_params& p, F n_at, double* out) {
  std::vector<double> rows((size_t)p.n_theta);
  for (int q = 0; q < p.n_theta; ++q) {
    // four interleaved partial sums (a fixed order), so the row sum is not one serial chain of adds
    double r4[4] = {0.0, 0.0, 0.0, 0.0};
    int s = 0;
    for (; s + 4 <= p.n_phi; s += 4)
      for (int k = 0; k < 4; ++k) r4[k] += n_at(q, s + k);
    for (; s < p.n_phi; ++s) r4[0] += n_at(q, s);
    rows[q] = (r4[0] + r4[1]) + (r4[2] + r4[3]);
  }
  return reference_density_rows(p, rows.data(), out);
}

// Uploads the FP64 and state-precision row tables of h (synchronous on h's stream).
vlb_status upload_tables(vlb_handle* h) {
  const vlb_params* p = &h->p;
  const int nt = p->n_theta;
  double* tab = (double*)malloc(sizeof(double) * vlb::NCOEF * nt);
  void* tabT = malloc(h->esize * vlb::NCOEF * nt);
  if (!tab || !tabT) {
    free(tab);
    free(tabT);
    return fail(h, VLB_ERR_ARG, "out of host memory");
  }
  row_tables(p, tab);
  for (int i = 0; i < vlb::NCOEF * nt; ++i) {
    if (h->esize == 8)
      ((double*)tabT)[i] = tab[i];
    else
      ((float*)tabT)[i] = (float)tab[i];
  }
  cudaError_t e = cudaMemcpyAsync(h->coefD, tab, sizeof(double) * vlb::NCOEF * nt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->coefT, tabT, h->esize * vlb::NCOEF * nt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(tab);
  free(tabT);
  if (e != cudaSuccess) return fail(h, VLB_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
  return VLB_OK;
}

// A member view's reference density lives in the ensemble's device descriptor too.
vlb_status sync_member_n0(vlb_handle* h) {
  if (h->kind != 2) return VLB_OK;
  const float n0 = (float)h->n0;
  VLB_CUDA(h, cudaMemcpyAsync(&h->parent->d_members[h->index].n0, &n0, sizeof(float), cudaMemcpyHostToDevice,
                              h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  return VLB_OK;
}

constexpr long long kWaveBudget = 1ll << 31;  // SM clock cycles per dependency wait, about a second

// Whether vlb_step takes the wavefront schedule: only when asked for (VLB_SCHED_WAVE) on a grid that
// has its counters and the stage tensor maps.  VLB_SCHED_AUTO takes the per-stage launches, which
// measured faster on GB300 (0.236 against 0.469 ms per step at 1024 x 2048).
bool wave_active(const vlb_handle* h) {
  return h->kind == 0 && h->wave_cnt && h->maps && h->sched == VLB_SCHED_WAVE;
}

template <typename T>
vlb_status run_steps(vlb_handle* h, int64_t nsteps) {
  const vlb_params& p = h->p;
  vlb::StageArgs<T> a;
  a.coef = (const T*)h->coefT;
  a.nt = p.n_theta;
  a.ns = p.n_phi;
  a.stride = h->stride;
  a.dt = (T)p.dt;
  a.inv_tau = (T)(1.0 / p.tau);
  a.M = (T)p.M;
  a.A = (T)p.A;
  a.kappa = (T)p.kappa;
  a.gt = (T)(1.0 / (2.0 * p.r * (2.0 * M_PI / p.n_theta)));
  a.n0 = (T)h->n0;
  a.err = h->flag;
  T* U0 = (T*)h->U[0];
  T* U1 = (T*)h->U[1];
  T* U2 = (T*)h->U[2];
  if (p.n_phi == 1 && p.n_theta <= vlb::kAxiMaxRows && !p.ch_stab) {
    // axisymmetric grid: up to 256 steps per single-CTA launch, cut at the diagnostic steps
    int64_t n = 0;
    while (n < nsteps) {
      int64_t chunk = std::min<int64_t>(nsteps - n, 256);
      if (p.diag_every > 0) chunk = std::min<int64_t>(chunk, p.diag_every - h->steps_done % p.diag_every);
      VLB_CUDA(h, vlb::launch_axi<T>(a, p.advection, p.ch_mode, U0, U1, U2, (int)chunk, h->stream));
      h->steps_done += chunk;
      n += chunk;
      if (p.diag_every > 0 && (h->steps_done % p.diag_every == 0 || n == nsteps)) {
        VLB_CUDA(h, vlb::launch_totals<T>(U0, h->stride, h->coefD, p.n_theta, p.n_phi, p.R, p.r, p.A, p.kappa,
                                          h->n0, p.geometry, h->partials, vlb::totals_blocks(), h->diag, h->stream));
        VLB_CUDA(h, vlb_internal_flag(h->diag, h->flag, h->stream));
      }
    }
    return VLB_OK;
  }
  // stabilised Cahn-Hilliard: the stage kernel writes dt L_phi, the Fourier solve forms phi
  T* dphi = p.ch_stab ? (T*)h->dphi : nullptr;
  a.dphi = dphi;
  const double* Jrow = h->coefD + (size_t)vlb::C_J * p.n_theta;
  auto solve = [&](const T* fin, const T* f0, T* fout, T b) -> cudaError_t {
    if (!dphi) return cudaSuccess;
    return vlb::launch_ch_stab<T>(p.n_theta, p.n_phi, p.dt * p.M * p.kappa, Jrow, dphi, h->fft,
                                  fin + vlb::NPOP * h->stride, f0 ? f0 + vlb::NPOP * h->stride : nullptr,
                                  fout + vlb::NPOP * h->stride, h->stride, b, h->stream);
  };
  if constexpr (sizeof(T) == 4) {
    if (wave_active(h)) {
      // whole steps per persistent launch (the wavefront schedule), cut at the diagnostic steps
      int64_t n = 0;
      while (n < nsteps) {
        int64_t chunk = std::min<int64_t>(nsteps - n, vlb::kWaveMaxSteps);
        if (p.diag_every > 0) chunk = std::min<int64_t>(chunk, p.diag_every - h->steps_done % p.diag_every);
        VLB_CUDA(h, vlb::launch_wave(a, p.ch_mode, U0, U1, U2, (int)chunk, h->wave_cnt,
                                     h->wave_budget > 0 ? h->wave_budget : kWaveBudget, h->wave_skip, h->stream,
                                     h->maps, nullptr));
        h->steps_done += chunk;
        n += chunk;
        if (p.diag_every > 0 && (h->steps_done % p.diag_every == 0 || n == nsteps)) {
          VLB_CUDA(h, vlb::launch_totals<T>(U0, h->stride, h->coefD, p.n_theta, p.n_phi, p.R, p.r, p.A, p.kappa,
                                            h->n0, p.geometry, h->partials, vlb::totals_blocks(), h->diag, h->stream));
          VLB_CUDA(h, vlb_internal_flag(h->diag, h->flag, h->stream));
        }
      }
      return VLB_OK;
    }
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    // SSP-RK3 (Shu & Osher 1988): U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
    // U <- 1/3 U + 2/3 (U2 + dt L(U2))
    const vlb::StageMaps* m = h->maps;
    a.fin = U0; a.f0 = nullptr; a.fout = U1; a.b = (T)1;
    VLB_CUDA(h, vlb::launch_stage<T>(a, p.advection, p.ch_mode, h->stream, m ? m + 0 : nullptr));
    VLB_CUDA(h, solve(U0, nullptr, U1, (T)1));
    a.fin = U1; a.f0 = U0; a.fout = U2; a.b = (T)0.25;
    VLB_CUDA(h, vlb::launch_stage<T>(a, p.advection, p.ch_mode, h->stream, m ? m + 1 : nullptr));
    VLB_CUDA(h, solve(U1, U0, U2, (T)0.25));
    a.fin = U2; a.f0 = U0; a.fout = U0; a.b = (T)(2.0 / 3.0);
    VLB_CUDA(h, vlb::launch_stage<T>(a, p.advection, p.ch_mode, h->stream, m ? m + 2 : nullptr));
    VLB_CUDA(h, solve(U2, U0, U0, (T)(2.0 / 3.0)));
    h->steps_done++;
    if (p.diag_every > 0 && (h->steps_done % p.diag_every == 0 || n + 1 == nsteps)) {
      VLB_CUDA(h, vlb::launch_totals<T>(U0, h->stride, h->coefD, p.n_theta, p.n_phi, p.R, p.r, p.A, p.kappa,
                                        h->n0, p.geometry, h->partials, vlb::totals_blocks(), h->diag, h->stream));
      VLB_CUDA(h, vlb_internal_flag(h->diag, h->flag, h->stream));
    }
  }
  return VLB_OK;
}

template <typename T>
vlb_status totals_impl(vlb_handle* h) {
  const vlb_params& p = h->p;
  VLB_CUDA(h, vlb::launch_totals<T>((const T*)h->U[0], h->stride, h->coefD, p.n_theta, p.n_phi, p.R, p.r, p.A,
                                    p.kappa, h->n0, p.geometry, h->partials, vlb::totals_blocks(), h->totals,
                                    h->stream));
  return VLB_OK;
}

vlb_status check_handle(vlb_handle* h, bool ensemble_ok = false) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (h->kind == 3) return fail(h, VLB_ERR_ARG, "surrogate handle: pass it to vlb_surrogate_advance");
  if (h->kind == 1 && !ensemble_ok)
    return fail(h, VLB_ERR_ARG, "ensemble handle: use vlb_ensemble_step, or a member view from vlb_ensemble_member");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(h, VLB_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != h->device) {
    e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail(h, VLB_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  return VLB_OK;
}

// Reads the handle's device flag in the stream order of the work issued so far, synchronises, and
// turns a raised flag into a status: 2 = a bounded wait on a bulk copy gave up and a tile was
// skipped (the state is no longer a solution: VLB_ERR_TIMEOUT), 1 = a diagnostic found a non-finite
// value or |u| > 2 (VLB_ERR_UNSTABLE, reported only when `unstable_too`).  The flag stays raised
// until the next vlb_set_fields / vlb_set_state.
vlb_status sync_and_check(vlb_handle* h, const char* what, bool unstable_too) {
  int flag = 0;
  VLB_CUDA(h, cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (flag == 2)
    return fail(h, VLB_ERR_TIMEOUT, "%s: a bounded device wait on a bulk copy gave up after %lld steps; a tile was "
                "skipped and the state is invalid (reset it with vlb_set_fields or vlb_set_state)", what,
                (long long)h->steps_done);
  if (flag == 1 && unstable_too)
    return fail(h, VLB_ERR_UNSTABLE, "%s: unstable state: non-finite value or |u| > 2 after %lld steps", what,
                (long long)h->steps_done);
  return VLB_OK;
}

}  // namespace

vlb_status vlb_internal_fail(vlb_handle* h, vlb_status st, const char* msg) { return fail(h, st, "%s", msg); }

// Flags an unstable state: non-finite values or |u| > 2 in the diagnostic vector.
__global__ void vlb_flag_kernel(const double* diag, int* flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double m = diag[0], um = diag[3], bad = diag[4];
    if ((bad > 0.0 || !(um <= 2.0) || !isfinite(m)) && *flag == 0) *flag = 1;  // a timeout (2) takes precedence
  }
}

cudaError_t vlb_internal_flag(const double* diag, int* flag, cudaStream_t s) {
  vlb_flag_kernel<<<1, 32, 0, s>>>(diag, flag);
  return cudaGetLastError();
}

namespace vlb {

// Velocity set of Eq. vmatrix, weights w_k = Q!/He_{Q+1}(v_k)^2 and the derivative kernel
// K_{i,m} = -w_i sum_{l<Q} He_{l+1}(v_i) He_l(v_m) / l!  (Sec. 2.3), in FP64.
static double he(int n, double x) {
  double a = 1.0, b = x;
  if (n == 0) return a;
  for (int m = 1; m < n; ++m) {
    const double c = x * b - m * a;
    a = b;
    b = c;
  }
  return b;
}

VelocityConsts velocity_consts() {
  VelocityConsts c;
  const double s6 = sqrt(6.0);
  c.v[0] = -sqrt(3.0 + s6);
  c.v[1] = -sqrt(3.0 - s6);
  c.v[2] = sqrt(3.0 - s6);
  c.v[3] = sqrt(3.0 + s6);
  for (int i = 0; i < 4; ++i) {
    const double h5 = he(5, c.v[i]);
    c.w[i] = 24.0 / (h5 * h5);
  }
  for (int i = 0; i < 4; ++i)
    for (int m = 0; m < 4; ++m) {
      double s = 0.0, fact = 1.0;
      for (int l = 0; l < 4; ++l) {
        if (l > 0) fact *= l;
        s += he(l + 1, c.v[i]) * he(l, c.v[m]) / fact;
      }
      c.K[i][m] = -c.w[i] * s;
    }
  return c;
}

}  // namespace vlb

extern "C" {

size_t vlb_workspace_bytes(const vlb_params* p) {
  char why[256];
  if (!params_ok(p, why, sizeof why)) {
    fail(nullptr, VLB_ERR_ARG, "%s", why);
    return 0;
  }
  return layout(p).total;
}

namespace {

// Largest dt for which one SSP-RK3 step of the linearised per-population model
//   dg/dt = -(v_i / h_theta) D(k_theta) g - (v_j / h_phi) D(k_phi) g - g / tau
// has amplification |R(z)| = |1 + z + z^2/2 + z^3/6| <= 1 on every Fourier mode of a 64 x 64 grid
// over [-pi, pi)^2 and every velocity pair.  D is the symbol of the upwind difference per unit
// spacing (UW3, or the fifth-order linear scheme WENO5 reduces to on smooth data).  A velocity of
// the opposite sign has the symbol of mode -k, so |v| in {v_2, v_3} covers all 16 pairs.  With
// dt / tau near 2 the relaxation shifts the advective eigenvalues to where the stability region of
// RK3 is narrow, which the separate limits on advection and relaxation miss.
double combined_rk3_dt(double ht, double hp, double tau, int advection, bool phi_dir, double vmax) {
  constexpr int NK = 64;
  double re[NK], im[NK];
  for (int n = 0; n < NK; ++n) {
    const double k = -M_PI + 2.0 * M_PI * n / NK;
    if (advection == VLB_WENO5) {  // (-2 e^{-3ik} + 15 e^{-2ik} - 60 e^{-ik} + 20 + 30 e^{ik} - 3 e^{2ik}) / 60
      re[n] = (-2.0 * cos(3 * k) + 15.0 * cos(2 * k) - 60.0 * cos(k) + 20.0 + 30.0 * cos(k) - 3.0 * cos(2 * k)) / 60.0;
      im[n] = (2.0 * sin(3 * k) - 15.0 * sin(2 * k) + 60.0 * sin(k) + 30.0 * sin(k) - 3.0 * sin(2 * k)) / 60.0;
    } else {  // (2 e^{ik} + 3 - 6 e^{-ik} + e^{-2ik}) / 6
      re[n] = (2.0 * cos(k) + 3.0 - 6.0 * cos(k) + cos(2 * k)) / 6.0;
      im[n] = (2.0 * sin(k) + 6.0 * sin(k) - sin(2 * k)) / 6.0;
    }
  }
  const double s6 = sqrt(6.0), va[2] = {sqrt(3.0 - s6), sqrt(3.0 + s6)};
  const double rel = isfinite(tau) ? 1.0 / tau : 0.0;
  auto stable = [&](double dt) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < (phi_dir ? 2 : 1); ++b)
        for (int m = 0; m < NK; ++m)
          for (int n = 0; n < (phi_dir ? NK : 1); ++n) {
            double zr = -va[a] / ht * re[m] - rel, zi = -va[a] / ht * im[m];
            if (phi_dir) {
              zr -= va[b] / hp * re[n];
              zi -= va[b] / hp * im[n];
            }
            zr *= dt;
            zi *= dt;
            // R(z) = 1 + z (1 + z (1/2 + z / 6)) in complex arithmetic
            double tr = 0.5 + zr / 6.0, ti = zi / 6.0;
            double ur = 1.0 + (zr * tr - zi * ti), ui = zr * ti + zi * tr;
            const double rr = 1.0 + (zr * ur - zi * ui), ri = zr * ui + zi * ur;
            if (rr * rr + ri * ri > 1.0 + 1e-12) return false;
          }
    return true;
  };
  // bracket: the advective CFL limit of RK3 is below 3 / (v_max (1/h_theta + 1/h_phi)) and the
  // real-axis limit below 2.52 tau
  double hi = 3.0 / (vmax * (1.0 / ht + (phi_dir ? 1.0 / hp : 0.0)));
  if (isfinite(tau)) hi = fmin(hi, 2.52 * tau);
  double lo = 0.0;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (stable(mid))
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

}  // namespace

vlb_status vlb_max_stable_dt(const vlb_params* p, double* dt_out) {
  char why[256];
  if (!dt_out) return fail(nullptr, VLB_ERR_ARG, "dt_out is NULL");
  vlb_params q = p ? *p : vlb_params{};
  if (p) q.dt = 1.0;  // dt itself is not validated here
  if (!params_ok(p ? &q : nullptr, why, sizeof why)) return fail(nullptr, VLB_ERR_ARG, "%s", why);
  const double dth = 2.0 * M_PI / p->n_theta, dph = 2.0 * M_PI / p->n_phi;
  const double ht = p->r * dth;
  const double hp = (p->geometry == VLB_TORUS ? (p->R - p->r) : p->R) * dph;
  const double vmax = sqrt(3.0 + sqrt(6.0));
  double dt = 1.0 / (vmax * (1.0 / ht + (p->n_phi > 1 ? 1.0 / hp : 0.0)));
  if (isfinite(p->tau)) dt = fmin(dt, 2.5 * p->tau);
  dt = fmin(dt, combined_rk3_dt(ht, hp, p->tau, p->advection, p->n_phi > 1, vmax));
  const double lam = 4.0 / (ht * ht) + (p->n_phi > 1 ? 4.0 / (hp * hp) : 0.0);
  if (p->ch_stab) {
    // preconditioned spinodal rate dt 2 M A lam / (1 + dt M kappa lam^2) peaks at A sqrt(dt M / kappa)
    if (p->A > 0.0 && p->M > 0.0) dt = fmin(dt, 6.25 * p->kappa / (p->A * p->A * p->M));
  } else {
    const double ch = p->M * lam * (p->kappa * lam + 2.0 * p->A);
    if (ch > 0.0) dt = fmin(dt, 2.5 / ch);
  }
  *dt_out = dt;
  return VLB_OK;
}

vlb_status vlb_create(const vlb_params* p, void* d_workspace, size_t bytes, void* cuda_stream, vlb_handle** out) {
  char why[256];
  if (!out) return fail(nullptr, VLB_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params_ok(p, why, sizeof why)) return fail(nullptr, VLB_ERR_ARG, "%s", why);
  const Layout L = layout(p);
  if (!d_workspace) return fail(nullptr, VLB_ERR_WORKSPACE, "workspace is NULL");
  if (((uintptr_t)d_workspace) % 256 != 0) return fail(nullptr, VLB_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (bytes < L.total)
    return fail(nullptr, VLB_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", bytes, L.total);
  vlb_handle* h = new (std::nothrow) vlb_handle();
  if (!h) return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  h->p = *p;
  h->stream = (cudaStream_t)cuda_stream;
  h->N = L.N;
  h->stride = L.stride;
  h->esize = L.esize;
  h->ws = (unsigned char*)d_workspace;
  h->ws_bytes = bytes;
  h->coefT = h->ws + L.off_coefT;
  h->coefD = (double*)(h->ws + L.off_coefD);
  for (int k = 0; k < 3; ++k) h->U[k] = h->ws + L.off_U[k];
  h->staging = (double*)(h->ws + L.off_staging);
  h->partials = (double*)(h->ws + L.off_partials);
  h->totals = (double*)(h->ws + L.off_totals);
  h->diag = (double*)(h->ws + L.off_diag);
  h->flag = (int*)(h->ws + L.off_flag);
  h->dphi = p->ch_stab ? h->ws + L.off_dphi : nullptr;
  h->fft = p->ch_stab ? h->ws + L.off_fft : nullptr;
  h->wave_cnt = L.off_wave ? (unsigned*)(h->ws + L.off_wave) : nullptr;
  h->steps_done = 0;
  h->n0 = 1.0;
  h->err[0] = 0;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, VLB_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  // geometry tables
  const int nt = p->n_theta;
  double* tab = (double*)malloc(sizeof(double) * vlb::NCOEF * nt);
  void* tabT = malloc(L.esize * vlb::NCOEF * nt);
  if (!tab || !tabT) {
    free(tab);
    free(tabT);
    delete h;
    return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  }
  row_tables(p, tab);
  for (int i = 0; i < vlb::NCOEF * nt; ++i) {
    if (L.esize == 8)
      ((double*)tabT)[i] = tab[i];
    else
      ((float*)tabT)[i] = (float)tab[i];
  }
  e = cudaMemcpyAsync(h->coefD, tab, sizeof(double) * vlb::NCOEF * nt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->coefT, tabT, L.esize * vlb::NCOEF * nt, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.off_U[0], 0, L.off_staging - L.off_U[0], h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
  std::vector<double> lam;
  if (e == cudaSuccess && p->ch_stab) {
    // the stabiliser's tables after the spectrum: the factors of lambda at the finest spacings
    // (r dtheta; (R - r) dvarphi on the torus, R dvarphi flat) and the twiddles
    const double h_t = p->r * (2.0 * M_PI / p->n_theta);
    const double h_p = (p->geometry == VLB_TORUS ? p->R - p->r : p->R) * (2.0 * M_PI / p->n_phi);
    lam.resize(vlb::ch_stab_table_elems(p->n_theta, p->n_phi));
    vlb::ch_stab_tables(p->n_theta, p->n_phi, h_t, h_p, L.esize, lam.data());
    e = cudaMemcpyAsync((unsigned char*)h->fft + vlb::ch_stab_table_offset(p->n_theta, p->n_phi, L.esize), lam.data(),
                        L.esize * lam.size(), cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(tab);
  free(tabT);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, VLB_ERR_CUDA, "vlb_create upload: %s", cudaGetErrorString(e));
  }
  if (h->esize == 4 && p->advection == VLB_UW3 && vlb::stage_maps_apply(p->n_theta, p->n_phi)) {
    h->maps = new (std::nothrow) vlb::StageMaps[3];
    for (int k = 0; k < 3 && h->maps; ++k)
      if (vlb::make_stage_maps((const float*)h->U[k], (const float*)h->U[0], p->n_theta, p->n_phi, h->stride,
                               h->maps + k) != cudaSuccess) {
        delete[] h->maps;  // the driver has no tensor-map encoder: per-thread copies only
        h->maps = nullptr;
      }
  }
  *out = h;
  return VLB_OK;
}

vlb_status vlb_destroy(vlb_handle* h) {
  if (!h || h->kind == 2) return VLB_OK;  // member views are owned by their ensemble
  if (h->kind == 3 && h->sur_graph) cudaGraphExecDestroy(h->sur_graph);
  if (h->kind == 1) {
    if (h->graph_1) cudaGraphExecDestroy(h->graph_1);
    if (h->graph_32) cudaGraphExecDestroy(h->graph_32);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (int i = 0; i < h->count; ++i) delete h->views[i];
    delete[] h->views;
  }
  delete[] h->maps;
  delete h->ens_maps;
  delete h;
  return VLB_OK;
}

vlb_status vlb_set_fields(vlb_handle* h, const double* rho, const double* u_th, const double* u_ph, const double* phi) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!rho || !u_th || !u_ph || !phi) return fail(h, VLB_ERR_ARG, "vlb_set_fields: NULL input");
  const int ns = h->p.n_phi;
  const size_t nb = sizeof(double) * h->N;
  double* s = h->staging;
  VLB_CUDA(h, cudaMemcpyAsync(s, rho, nb, cudaMemcpyHostToDevice, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(s + h->N, u_th, nb, cudaMemcpyHostToDevice, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(s + 2 * h->N, u_ph, nb, cudaMemcpyHostToDevice, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(s + 3 * h->N, phi, nb, cudaMemcpyHostToDevice, h->stream));
  // the reference density from row sums formed on the device (one small read-back) rather than a
  // pass of the host over the caller's array
  std::vector<double> rows((size_t)h->p.n_theta);
  double* row_sums = s + 4 * h->N;  // the staging area holds 17 N doubles
  VLB_CUDA(h, vlb::launch_row_sums(s, h->p.n_theta, ns, row_sums, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(rows.data(), row_sums, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost,
                              h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!reference_density_rows(h->p, rows.data(), &h->n0))
    return fail(h, VLB_ERR_ARG, "vlb_set_fields: density must be finite with a positive mean");
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_init_feq<double>((double*)h->U[0], h->stride, s, s + h->N, s + 2 * h->N, s + 3 * h->N,
                                             h->N, h->n0, h->stream));
  else
    VLB_CUDA(h, vlb::launch_init_feq<float>((float*)h->U[0], h->stride, s, s + h->N, s + 2 * h->N, s + 3 * h->N,
                                            h->N, h->n0, h->stream));
  VLB_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->steps_done = 0;
  return sync_member_n0(h);
}

vlb_status vlb_set_state(vlb_handle* h, const double* f16, const double* phi) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!f16 || !phi) return fail(h, VLB_ERR_ARG, "vlb_set_state: NULL input");
  const int ns = h->p.n_phi;
  const int64_t N = h->N;
  auto dens = [&](int q, int s) {
    double x = 0.0;
    for (int k = 0; k < 16; ++k) x += f16[k * N + (int64_t)q * ns + s];
    return x;
  };
  if (!reference_density(h->p, dens, &h->n0))
    return fail(h, VLB_ERR_ARG, "vlb_set_state: populations must be finite with a positive mean density");
  const size_t nb = sizeof(double) * h->N;
  VLB_CUDA(h, cudaMemcpyAsync(h->staging, f16, 16 * nb, cudaMemcpyHostToDevice, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(h->staging + 16 * h->N, phi, nb, cudaMemcpyHostToDevice, h->stream));
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_convert_in<double>((double*)h->U[0], h->stride, h->staging, h->N, h->n0, h->stream));
  else
    VLB_CUDA(h, vlb::launch_convert_in<float>((float*)h->U[0], h->stride, h->staging, h->N, h->n0, h->stream));
  VLB_CUDA(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->steps_done = 0;
  return sync_member_n0(h);
}

vlb_status vlb_get_state(vlb_handle* h, double* f16, double* phi) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!f16 || !phi) return fail(h, VLB_ERR_ARG, "vlb_get_state: NULL output");
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_convert_out<double>(h->staging, (const double*)h->U[0], h->stride, h->N, h->n0,
                                                h->stream));
  else
    VLB_CUDA(h, vlb::launch_convert_out<float>(h->staging, (const float*)h->U[0], h->stride, h->N, h->n0,
                                               h->stream));
  const size_t nb = sizeof(double) * h->N;
  VLB_CUDA(h, cudaMemcpyAsync(f16, h->staging, 16 * nb, cudaMemcpyDeviceToHost, h->stream));
  VLB_CUDA(h, cudaMemcpyAsync(phi, h->staging + 16 * h->N, nb, cudaMemcpyDeviceToHost, h->stream));
  return sync_and_check(h, "vlb_get_state", false);
}

vlb_status vlb_step(vlb_handle* h, int64_t nsteps) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (nsteps < 0) return fail(h, VLB_ERR_ARG, "nsteps must be >= 0");
  st = h->esize == 8 ? run_steps<double>(h, nsteps) : run_steps<float>(h, nsteps);
  if (st) return st;
  if (h->p.diag_every > 0 && nsteps > 0) return sync_and_check(h, "vlb_step", true);
  return VLB_OK;
}

vlb_status vlb_get_fields(vlb_handle* h, double* rho, double* u_th, double* u_ph, double* phi, double* mu) {
  vlb_status st = check_handle(h);
  if (st) return st;
  const vlb_params& p = h->p;
  double* s = h->staging;
  const int64_t N = h->N;
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_fields<double>((const double*)h->U[0], h->stride, h->coefD, p.n_theta, p.n_phi, p.A,
                                           p.kappa, h->n0, s, s + N, s + 2 * N, s + 3 * N, s + 4 * N, h->stream));
  else
    VLB_CUDA(h, vlb::launch_fields<float>((const float*)h->U[0], h->stride, h->coefD, p.n_theta, p.n_phi, p.A,
                                          p.kappa, h->n0, s, s + N, s + 2 * N, s + 3 * N, s + 4 * N, h->stream));
  double* outs[5] = {rho, u_th, u_ph, phi, mu};
  for (int k = 0; k < 5; ++k)
    if (outs[k])
      VLB_CUDA(h, cudaMemcpyAsync(outs[k], s + k * N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  return sync_and_check(h, "vlb_get_fields", false);
}

vlb_status vlb_get_totals(vlb_handle* h, double out[4]) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!out) return fail(h, VLB_ERR_ARG, "out is NULL");
  st = h->esize == 8 ? totals_impl<double>(h) : totals_impl<float>(h);
  if (st) return st;
  double t[8];
  VLB_CUDA(h, cudaMemcpyAsync(t, h->totals, sizeof t, cudaMemcpyDeviceToHost, h->stream));
  st = sync_and_check(h, "vlb_get_totals", false);
  for (int k = 0; k < 4; ++k) out[k] = t[k];
  return st;
}

vlb_status vlb_interface_length(vlb_handle* h, double* out) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!out) return fail(h, VLB_ERR_ARG, "out is NULL");
  st = h->esize == 8 ? totals_impl<double>(h) : totals_impl<float>(h);
  if (st) return st;
  double t[8];
  VLB_CUDA(h, cudaMemcpyAsync(t, h->totals, sizeof t, cudaMemcpyDeviceToHost, h->stream));
  st = sync_and_check(h, "vlb_interface_length", false);
  *out = t[5];
  return st;
}

vlb_status vlb_set_schedule(vlb_handle* h, int32_t schedule) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (h->kind != 0) return fail(h, VLB_ERR_ARG, "vlb_set_schedule: solver handles only");
  if (schedule != VLB_SCHED_AUTO && schedule != VLB_SCHED_STAGES && schedule != VLB_SCHED_WAVE)
    return fail(h, VLB_ERR_ARG, "vlb_set_schedule: unknown schedule %d", (int)schedule);
  if (schedule == VLB_SCHED_WAVE && !(h->wave_cnt && h->maps))
    return fail(h, VLB_ERR_ARG, "vlb_set_schedule: the wavefront schedule needs an FP32 UW3 explicit grid with "
                                "n_theta a multiple of 16 (at least 176) and n_phi a multiple of 32");
  h->sched = schedule;
  return VLB_OK;
}

vlb_status vlb_get_schedule(const vlb_handle* h, int32_t* active) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (!active) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "NULL output");
  *active = wave_active(h) ? VLB_SCHED_WAVE : VLB_SCHED_STAGES;
  return VLB_OK;
}

vlb_status vlb_test_wave_timeout(vlb_handle* h, int32_t skip_cta, int64_t budget) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (h->kind != 0) return fail(h, VLB_ERR_ARG, "vlb_test_wave_timeout: solver handles only");
  if (budget < 0) return fail(h, VLB_ERR_ARG, "vlb_test_wave_timeout: budget < 0");
  h->wave_skip = skip_cta < 0 ? -1 : skip_cta;
  h->wave_budget = budget;
  return VLB_OK;
}

vlb_status vlb_test_wave_schedule(int32_t n_bands, int32_t lag, int32_t nsteps) {
  return vlb::wave_schedule_ok(n_bands, lag, nsteps) ? VLB_OK
                                                     : fail(nullptr, VLB_ERR_ARG, "wavefront ticket order invalid");
}

vlb_status vlb_structure_length(vlb_handle* h, double* out) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!out) return fail(h, VLB_ERR_ARG, "out is NULL");
  const vlb_params& p = h->p;
  if (!vlb::ch_stab_shape_ok(p.n_theta, p.n_phi))
    return fail(h, VLB_ERR_ARG, "vlb_structure_length: n_theta and n_phi must be powers of two in [4, 4096]");
  // scratch: the FP64 staging area (17 N doubles) holds the spectrum (2 N) and the strip sums
  double* spec = h->staging;
  double* part = h->staging + 2 * h->N;
  const int nb = vlb::structure_blocks(p.n_theta, p.n_phi);
  if (h->esize == 8) {
    const double* phi = (const double*)h->U[0] + 16 * h->stride;
    VLB_CUDA(h, vlb::launch_structure_sums<double>(p.n_theta, p.n_phi, p.r, p.R, phi, nullptr, spec, part,
                                                   h->stream));
  } else {
    const float* phi = (const float*)h->U[0] + 16 * h->stride;
    VLB_CUDA(h, vlb::launch_structure_sums<float>(p.n_theta, p.n_phi, p.r, p.R, phi, phi + h->stride, spec, part,
                                                  h->stream));
  }
  std::vector<double> sums((size_t)2 * nb);
  VLB_CUDA(h, cudaMemcpyAsync(sums.data(), part, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  st = sync_and_check(h, "vlb_structure_length", false);
  double s_sum = 0.0, k_sum = 0.0;
  for (int b = 0; b < nb; ++b) {
    s_sum += sums[2 * b];
    k_sum += sums[2 * b + 1];
  }
  // a uniform phi has no domains: its length is infinite
  *out = k_sum > 0.0 ? 2.0 * M_PI * s_sum / k_sum : INFINITY;
  return st;
}

vlb_status vlb_state_device(vlb_handle* h, void** f, int64_t* stride) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (h->kind == 1) return fail(h, VLB_ERR_ARG, "ensemble handle: use a member view");
  if (!f || !stride) return fail(h, VLB_ERR_ARG, "NULL output");
  *f = h->U[0];
  *stride = h->stride;
  return VLB_OK;
}

vlb_status vlb_steps_done(const vlb_handle* h, int64_t* out) {
  if (!h) return fail(nullptr, VLB_ERR_ARG, "handle is NULL");
  if (!out) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "NULL output");
  *out = h->steps_done;
  return VLB_OK;
}

const char* vlb_last_error(const vlb_handle* h) { return h ? h->err : g_err; }

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Ensembles: many tori advanced by one batched launch per Runge-Kutta stage.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr int kTileRows[2] = {16, 8};

struct EnsLayout {
  size_t off_staging, off_partials, off_totals, off_diag, off_flag, off_bar, off_members, off_items[2];
  std::vector<size_t> off_member;  // start of member m's region: coefT, coefD, U0, U1, U2
  std::vector<Layout> member;
  int nitems[2];
  size_t total;
};

bool ensemble_params_ok(const vlb_params* p, int count, char* why, size_t n) {
  if (!p) return snprintf(why, n, "params is NULL"), false;
  if (count < 1 || count > 65536) return snprintf(why, n, "count must be in 1..65536"), false;
  for (int m = 0; m < count; ++m) {
    char w2[200];
    if (!params_ok(&p[m], w2, sizeof w2)) return snprintf(why, n, "member %d: %s", m, w2), false;
    if (p[m].precision != VLB_FP32 || p[m].advection != VLB_UW3)
      return snprintf(why, n, "member %d: ensembles run FP32 UW3", m), false;
    if (p[m].ch_mode != p[0].ch_mode) return snprintf(why, n, "member %d: all members share ch_mode", m), false;
    if (p[m].ch_stab) return snprintf(why, n, "member %d: ensembles run the explicit Cahn-Hilliard step", m), false;
  }
  return true;
}

EnsLayout ens_layout(const vlb_params* p, int count) {
  EnsLayout E;
  int64_t maxN = 0;
  E.nitems[0] = E.nitems[1] = 0;
  for (int m = 0; m < count; ++m) {
    E.member.push_back(layout(&p[m]));
    maxN = std::max(maxN, E.member.back().N);
    const int ts = (p[m].n_phi + 31) / 32;
    for (int k = 0; k < 2; ++k) E.nitems[k] += ts * ((p[m].n_theta + kTileRows[k] - 1) / kTileRows[k]);
  }
  size_t off = 0;
  E.off_staging = off;
  off = align_up(off + (size_t)vlb::NARR * maxN * 8, 256);
  E.off_partials = off;
  off = align_up(off + (size_t)vlb::totals_blocks() * 8 * 8, 256);
  E.off_totals = off;
  off = align_up(off + 64, 256);
  E.off_diag = off;
  off = align_up(off + 64, 256);
  E.off_flag = off;
  off = align_up(off + 256, 256);
  E.off_bar = off;
  off = align_up(off + 256, 256);
  E.off_members = off;
  off = align_up(off + sizeof(vlb::EnsembleMember) * count, 256);
  for (int k = 0; k < 2; ++k) {
    E.off_items[k] = off;
    off = align_up(off + sizeof(int2) * E.nitems[k], 256);
  }
  for (int m = 0; m < count; ++m) {
    const Layout& L = E.member[m];
    E.off_member.push_back(off);
    off += L.off_staging - L.off_coefT;  // coefT, coefD and the three state buffers of a solver layout
    off = align_up(off, 256);
  }
  E.total = off;
  return E;
}

constexpr long long kBarrierBudget = 1ll << 31;  // SM clock cycles, about a second at 2 GHz

// nsteps steps of every member in the chosen mode (rows_idx: 0 = 16-row tiles, 1 = 8-row tiles).
vlb_status ens_launch_steps(vlb_handle* h, int mode, int rows_idx, int nsteps, cudaStream_t st) {
  if (mode == 2) {
    VLB_CUDA(h, vlb::launch_ensemble_persistent(h->d_members, h->d_items[rows_idx], h->nitems[rows_idx], nsteps, 0,
                                                kTileRows[rows_idx], h->p.ch_mode, h->ens_bar, h->flag,
                                                h->ens_budget > 0 ? h->ens_budget : kBarrierBudget, h->ens_skip,
                                                h->ens_ctas, st, h->ens_maps, &h->ens_grid));
    return VLB_OK;
  }
  for (int n = 0; n < nsteps; ++n)
    for (int stage = 0; stage < 3; ++stage)
      VLB_CUDA(h, vlb::launch_ensemble_stage(h->d_members, h->d_items[rows_idx], h->nitems[rows_idx], stage,
                                            kTileRows[rows_idx], h->p.ch_mode, h->flag, st, h->ens_maps));
  return VLB_OK;
}

// One timing of a candidate: three passes of the first Runge-Kutta stage (which writes only the
// scratch U^(1), so the state does not advance), after a warm-up pass.  Batched: three launches;
// persistent: one launch with grid barriers between the passes.
vlb_status ens_time(vlb_handle* h, int mode, int rows_idx, float* ms) {
  cudaEvent_t e0, e1;
  VLB_CUDA(h, cudaEventCreate(&e0));
  VLB_CUDA(h, cudaEventCreate(&e1));
  auto pass = [&](int reps) -> cudaError_t {
    if (mode == 2)
      return vlb::launch_ensemble_persistent(h->d_members, h->d_items[rows_idx], h->nitems[rows_idx], reps, 1,
                                             kTileRows[rows_idx], h->p.ch_mode, h->ens_bar, h->flag, kBarrierBudget,
                                             -1, h->ens_ctas, h->stream, h->ens_maps, nullptr);
    for (int r = 0; r < reps; ++r) {
      cudaError_t e = vlb::launch_ensemble_stage(h->d_members, h->d_items[rows_idx], h->nitems[rows_idx], 0,
                                                 kTileRows[rows_idx], h->p.ch_mode, h->flag, h->stream, h->ens_maps);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  VLB_CUDA(h, pass(1));
  VLB_CUDA(h, cudaEventRecord(e0, h->stream));
  VLB_CUDA(h, pass(3));
  VLB_CUDA(h, cudaEventRecord(e1, h->stream));
  VLB_CUDA(h, cudaEventSynchronize(e1));
  float t = 0.0f;
  VLB_CUDA(h, cudaEventElapsedTime(&t, e0, e1));
  *ms = t / 3.0f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return VLB_OK;
}

// ---- autotune cache: one JSON object per line, keyed by the members' grids, ch_mode and SM count.
// The file is VLB_AUTOTUNE_CACHE if that is set; every process also keeps its own entries.
struct EnsChoice {
  int mode, rows, ctas;
  float ms[4];
};
std::mutex g_tune_mu;
std::map<std::string, EnsChoice> g_tune;

std::string ens_key(const vlb_handle* h, int sms) {
  uint64_t x = 1469598103934665603ull;  // FNV-1a over the members' grids
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      x ^= (v >> (8 * b)) & 0xFF;
      x *= 1099511628211ull;
    }
  };
  mix((uint64_t)h->count);
  mix((uint64_t)h->p.ch_mode);
  for (int m = 0; m < h->count; ++m) {
    mix((uint64_t)h->views[m]->p.n_theta);
    mix((uint64_t)h->views[m]->p.n_phi);
  }
  char buf[64];
  snprintf(buf, sizeof buf, "%016llx-%d", (unsigned long long)x, sms);
  return buf;
}

bool cache_lookup(const std::string& key, EnsChoice* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) {
    *out = it->second;
    return true;
  }
  const char* path = getenv("VLB_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  FILE* fh = fopen(path, "r");
  if (!fh) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, fh)) {
    char k[64];
    EnsChoice c;
    int sms = 0, members = 0;
    if (sscanf(line,
               "{\"key\": \"%63[^\"]\", \"kind\": \"ensemble\", \"sms\": %d, \"members\": %d, \"mode\": %d, "
               "\"tile_rows\": %d, \"ctas_per_sm\": %d, \"ms\": [%f, %f, %f, %f]}",
               k, &sms, &members, &c.mode, &c.rows, &c.ctas, &c.ms[0], &c.ms[1], &c.ms[2], &c.ms[3]) == 10 &&
        key == k && (c.mode == 1 || c.mode == 2) && (c.rows == 16 || c.rows == 8)) {
      *out = c;  // the last entry for a key wins
      found = true;
    }
  }
  fclose(fh);
  if (found) g_tune[key] = *out;
  return found;
}

void cache_store(const std::string& key, const EnsChoice& c, int sms, int members) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = c;
  const char* path = getenv("VLB_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* fh = fopen(path, "a");
  if (!fh) return;  // an unwritable cache only costs a re-tune
  fprintf(fh,
          "{\"key\": \"%s\", \"kind\": \"ensemble\", \"sms\": %d, \"members\": %d, \"mode\": %d, \"tile_rows\": %d, "
          "\"ctas_per_sm\": %d, \"ms\": [%.6f, %.6f, %.6f, %.6f]}\n",
          key.c_str(), sms, members, c.mode, c.rows, c.ctas, c.ms[0], c.ms[1], c.ms[2], c.ms[3]);
  fclose(fh);
}

// Chooses the execution of the ensemble: the requested mode and tile height, or the fastest of
// batched and persistent launches with 16- and 8-row tiles (cached).
vlb_status ens_choose(vlb_handle* h) {
  int dev = 0, sms = 0;
  VLB_CUDA(h, cudaGetDevice(&dev));
  VLB_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->ens_ctas = h->ens_req_ctas;
  if (h->ens_req_mode != 0 && h->ens_req_rows != 0) {
    h->ens_mode = h->ens_req_mode;
    h->tile_rows = h->ens_req_rows;
    return VLB_OK;
  }
  const std::string key = ens_key(h, sms);
  EnsChoice c;
  const bool any = h->ens_req_mode == 0 && h->ens_req_rows == 0 && h->ens_req_ctas == 0;
  if (any && cache_lookup(key, &c)) {
    h->ens_mode = c.mode;
    h->tile_rows = c.rows;
    h->ens_ctas = c.ctas;
    for (int k = 0; k < 4; ++k) h->ens_ms[k] = c.ms[k];
    h->tune_ms[0] = c.ms[0];
    h->tune_ms[1] = c.ms[1];
    h->ens_from_cache = 1;
    return VLB_OK;
  }
  float best = 1e30f;
  for (int mode = 1; mode <= 2; ++mode)
    for (int k = 0; k < 2; ++k) {
      float& ms = h->ens_ms[2 * (mode - 1) + k];
      ms = 0.0f;
      if ((h->ens_req_mode && h->ens_req_mode != mode) || (h->ens_req_rows && h->ens_req_rows != kTileRows[k]))
        continue;
      vlb_status st = ens_time(h, mode, k, &ms);
      if (st) return st;
      if (ms < best) {
        best = ms;
        h->ens_mode = mode;
        h->tile_rows = kTileRows[k];
      }
    }
  h->tune_ms[0] = h->ens_ms[0];
  h->tune_ms[1] = h->ens_ms[1];
  if (any) {
    c.mode = h->ens_mode;
    c.rows = h->tile_rows;
    c.ctas = h->ens_ctas;
    for (int k = 0; k < 4; ++k) c.ms[k] = h->ens_ms[k];
    cache_store(key, c, sms, h->count);
  }
  return VLB_OK;
}

vlb_status ens_capture(vlb_handle* h, int steps, cudaGraphExec_t* out) {
  const int k = h->tile_rows == kTileRows[0] ? 0 : 1;
  cudaGraph_t g = nullptr;
  VLB_CUDA(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  vlb_status st = ens_launch_steps(h, h->ens_mode, k, steps, h->capture_stream);
  cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
  if (st != VLB_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // a launch that cannot be captured is replayed eagerly instead
    h->ens_graphs = false;
    *out = nullptr;
    return VLB_OK;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ens_graphs = false;
    *out = nullptr;
  }
  return VLB_OK;
}

void ens_drop_graphs(vlb_handle* h) {
  if (h->graph_1) cudaGraphExecDestroy(h->graph_1);
  if (h->graph_32) cudaGraphExecDestroy(h->graph_32);
  h->graph_1 = h->graph_32 = nullptr;
  h->ens_graphs = true;
}

}  // namespace

extern "C" {

size_t vlb_ensemble_workspace_bytes(const vlb_params* p, int32_t count) {
  char why[256];
  if (!ensemble_params_ok(p, count, why, sizeof why)) {
    fail(nullptr, VLB_ERR_ARG, "%s", why);
    return 0;
  }
  return ens_layout(p, count).total;
}

vlb_status vlb_ensemble_create(const vlb_params* p, int32_t count, void* d_workspace, size_t bytes, void* cuda_stream,
                               vlb_handle** out) {
  char why[256];
  if (!out) return fail(nullptr, VLB_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ensemble_params_ok(p, count, why, sizeof why)) return fail(nullptr, VLB_ERR_ARG, "%s", why);
  const EnsLayout E = ens_layout(p, count);
  if (!d_workspace) return fail(nullptr, VLB_ERR_WORKSPACE, "workspace is NULL");
  if (((uintptr_t)d_workspace) % 256 != 0) return fail(nullptr, VLB_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (bytes < E.total) return fail(nullptr, VLB_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", bytes, E.total);
  unsigned char* ws = (unsigned char*)d_workspace;
  vlb_handle* h = new (std::nothrow) vlb_handle();
  if (!h) return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  h->kind = 1;
  h->p = p[0];
  h->stream = (cudaStream_t)cuda_stream;
  h->ws = ws;
  h->ws_bytes = bytes;
  h->esize = 4;
  h->staging = (double*)(ws + E.off_staging);
  h->partials = (double*)(ws + E.off_partials);
  h->totals = (double*)(ws + E.off_totals);
  h->diag = (double*)(ws + E.off_diag);
  h->flag = (int*)(ws + E.off_flag);
  h->ens_bar = (unsigned*)(ws + E.off_bar);
  h->d_members = (vlb::EnsembleMember*)(ws + E.off_members);
  for (int k = 0; k < 2; ++k) {
    h->d_items[k] = (int2*)(ws + E.off_items[k]);
    h->nitems[k] = E.nitems[k];
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, VLB_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  h->count = count;
  h->views = new (std::nothrow) vlb_handle*[count]();
  if (!h->views) {
    delete h;
    return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  }
  std::vector<vlb::EnsembleMember> desc(count);
  h->ens_maps = new (std::nothrow) vlb::EnsembleMaps();
  if (!h->ens_maps) {
    vlb_destroy(h);
    return fail(nullptr, VLB_ERR_ARG, "out of host memory");
  }
  std::vector<int2> items[2];
  for (int m = 0; m < count; ++m) {
    vlb_handle* v = new (std::nothrow) vlb_handle();
    if (!v) {
      vlb_destroy(h);
      return fail(nullptr, VLB_ERR_ARG, "out of host memory");
    }
    h->views[m] = v;
    const Layout& L = E.member[m];
    unsigned char* base = ws + E.off_member[m] - L.off_coefT;  // so that base + L.off_* lands in the region
    v->kind = 2;
    v->parent = h;
    v->index = m;
    v->p = p[m];
    v->stream = h->stream;
    v->device = h->device;
    v->N = L.N;
    v->stride = L.stride;
    v->esize = 4;
    v->ws = ws;
    v->ws_bytes = bytes;
    v->coefT = base + L.off_coefT;
    v->coefD = (double*)(base + L.off_coefD);
    for (int k = 0; k < 3; ++k) v->U[k] = base + L.off_U[k];
    v->staging = h->staging;
    v->partials = h->partials;
    v->totals = h->totals;
    v->diag = h->diag;
    v->flag = h->flag;
    v->n0 = 1.0;
    v->steps_done = 0;
    vlb_status st = upload_tables(v);
    if (st == VLB_OK) {
      e = cudaMemsetAsync(v->U[0], 0, L.off_staging - L.off_U[0], h->stream);
      if (e != cudaSuccess) st = fail(nullptr, VLB_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    } else {
      fail(nullptr, st, "member %d: %s", m, v->err);
    }
    if (st != VLB_OK) {
      vlb_destroy(h);
      return st;
    }
    vlb::EnsembleMember& d = desc[m];
    for (int k = 0; k < 3; ++k) d.U[k] = (float*)v->U[k];
    d.coef = (const float*)v->coefT;
    d.nt = p[m].n_theta;
    d.ns = p[m].n_phi;
    d.stride = L.stride;
    d.dt = (float)p[m].dt;
    d.inv_tau = (float)(1.0 / p[m].tau);
    d.M = (float)p[m].M;
    d.A = (float)p[m].A;
    d.kappa = (float)p[m].kappa;
    d.gt = (float)(1.0 / (2.0 * p[m].r * (2.0 * M_PI / p[m].n_theta)));
    d.n0 = 1.0f;
    d.maps = -1;  // members beyond kEnsMapMembers, or without an encoder, take per-thread copies
    if (m < vlb::kEnsMapMembers && vlb::stage_maps_apply(p[m].n_theta, p[m].n_phi)) {
      bool ok = true;
      for (int k = 0; k < 3 && ok; ++k) {
        vlb::StageMaps sm;
        ok = vlb::make_stage_maps((const float*)v->U[k], (const float*)v->U[0], p[m].n_theta, p[m].n_phi, L.stride,
                                  &sm) == cudaSuccess;
        h->ens_maps->m[4 * m + k] = sm.box;
        if (k == 0) h->ens_maps->m[4 * m + 3] = sm.tile;
      }
      if (ok) d.maps = 4 * m;
    }
    const int ts = (p[m].n_phi + 31) / 32;
    for (int k = 0; k < 2; ++k) {
      const int tq = (p[m].n_theta + kTileRows[k] - 1) / kTileRows[k];
      for (int t = 0; t < ts * tq; ++t) items[k].push_back(make_int2(m, t));
    }
  }
  e = cudaMemcpyAsync(h->d_members, desc.data(), sizeof(vlb::EnsembleMember) * count, cudaMemcpyHostToDevice,
                      h->stream);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(h->d_items[k], items[k].data(), sizeof(int2) * items[k].size(), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ens_bar, 0, 256, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    vlb_destroy(h);
    return fail(nullptr, VLB_ERR_CUDA, "ensemble set-up: %s", cudaGetErrorString(e));
  }
  *out = h;
  return VLB_OK;
}

vlb_status vlb_ensemble_step(vlb_handle* h, int64_t nsteps) {
  vlb_status st = check_handle(h, true);
  if (st) return st;
  if (h->kind != 1) return fail(h, VLB_ERR_ARG, "not an ensemble handle");
  if (nsteps < 0) return fail(h, VLB_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return VLB_OK;
  int64_t left = nsteps;
  if (!h->ens_mode) {
    // first call (or after vlb_ensemble_configure): choose the execution, take one step eagerly (every
    // kernel variant is then set up outside any capture), and record the 1-step and 32-step graphs
    if ((st = ens_choose(h))) return st;
    const int k = h->tile_rows == kTileRows[0] ? 0 : 1;
    if ((st = ens_launch_steps(h, h->ens_mode, k, 1, h->stream))) return st;
    VLB_CUDA(h, cudaStreamSynchronize(h->stream));
    --left;
    ens_drop_graphs(h);
    if ((st = ens_capture(h, 1, &h->graph_1))) return st;
    if (h->ens_graphs && (st = ens_capture(h, 32, &h->graph_32))) return st;
  }
  const int k = h->tile_rows == kTileRows[0] ? 0 : 1;
  if (h->ens_graphs && h->graph_1 && h->graph_32) {
    for (; left >= 32; left -= 32) VLB_CUDA(h, cudaGraphLaunch(h->graph_32, h->stream));
    for (; left > 0; --left) VLB_CUDA(h, cudaGraphLaunch(h->graph_1, h->stream));
  } else {
    while (left > 0) {
      const int chunk = (int)std::min<int64_t>(left, 256);
      if ((st = ens_launch_steps(h, h->ens_mode, k, chunk, h->stream))) return st;
      left -= chunk;
    }
  }
  h->steps_done += nsteps;
  for (int m = 0; m < h->count; ++m) h->views[m]->steps_done += nsteps;
  return VLB_OK;
}

vlb_status vlb_ensemble_configure(vlb_handle* h, const vlb_ensemble_config* c) {
  if (!h || !c) return fail(h, VLB_ERR_ARG, "vlb_ensemble_configure: NULL argument");
  if (h->kind != 1) return fail(h, VLB_ERR_ARG, "not an ensemble handle");
  if (c->mode < VLB_ENS_AUTO || c->mode > VLB_ENS_PERSISTENT)
    return fail(h, VLB_ERR_ARG, "vlb_ensemble_configure: mode must be VLB_ENS_AUTO, _BATCHED or _PERSISTENT");
  if (c->tile_rows != 0 && c->tile_rows != 16 && c->tile_rows != 8)
    return fail(h, VLB_ERR_ARG, "vlb_ensemble_configure: tile_rows must be 0, 16 or 8");
  if (c->ctas_per_sm < 0 || c->ctas_per_sm > 32 || c->test_skip_cta < -1 || c->barrier_budget < 0)
    return fail(h, VLB_ERR_ARG, "vlb_ensemble_configure: bad ctas_per_sm, test_skip_cta or barrier_budget");
  vlb_status st = check_handle(h, true);
  if (st) return st;
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->ens_req_mode = c->mode;
  h->ens_req_rows = c->tile_rows;
  h->ens_req_ctas = c->ctas_per_sm;
  h->ens_skip = c->test_skip_cta;
  h->ens_budget = c->barrier_budget;
  h->ens_mode = 0;  // re-chosen (and the graphs re-recorded) by the next vlb_ensemble_step
  h->ens_from_cache = 0;
  ens_drop_graphs(h);
  return VLB_OK;
}

vlb_status vlb_ensemble_get_config(const vlb_handle* h, vlb_ensemble_config* c, float ms[4]) {
  if (!h || !c) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "vlb_ensemble_get_config: NULL argument");
  if (h->kind != 1) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "not an ensemble handle");
  c->mode = h->ens_mode;
  c->tile_rows = h->tile_rows;
  c->ctas_per_sm = h->ens_ctas;
  c->test_skip_cta = h->ens_skip;
  c->barrier_budget = h->ens_budget > 0 ? h->ens_budget : kBarrierBudget;
  if (ms)
    for (int k = 0; k < 4; ++k) ms[k] = h->ens_ms[k];
  return VLB_OK;
}

vlb_status vlb_ensemble_member(vlb_handle* h, int32_t idx, vlb_handle** view) {
  if (!h || !view) return fail(h, VLB_ERR_ARG, "NULL argument");
  if (h->kind != 1) return fail(h, VLB_ERR_ARG, "not an ensemble handle");
  if (idx < 0 || idx >= h->count) return fail(h, VLB_ERR_ARG, "member index %d out of range", idx);
  *view = h->views[idx];
  return VLB_OK;
}

vlb_status vlb_ensemble_tile_rows(const vlb_handle* h, int32_t* rows, float* ms16, float* ms8) {
  if (!h || !rows) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "NULL argument");
  if (h->kind != 1) return fail(const_cast<vlb_handle*>(h), VLB_ERR_ARG, "not an ensemble handle");
  *rows = h->tile_rows;
  if (ms16) *ms16 = h->tune_ms[0];
  if (ms8) *ms8 = h->tune_ms[1];
  return VLB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Snapshots (device FP32 (phi, n, u_theta, u_phi)) and the surrogate network's kernels.
// ------------------------------------------------------------------------------------------------
extern "C" {

vlb_status vlb_get_snapshot(vlb_handle* h, float* d_snap) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!d_snap) return fail(h, VLB_ERR_ARG, "snapshot pointer is NULL");
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_snapshot_out<double>((const double*)h->U[0], h->stride, h->N, h->n0, d_snap, h->stream));
  else
    VLB_CUDA(h, vlb::launch_snapshot_out<float>((const float*)h->U[0], h->stride, h->N, h->n0, d_snap, h->stream));
  return VLB_OK;
}

vlb_status vlb_set_snapshot(vlb_handle* h, const float* d_snap, const double* conserve, int32_t keep_nonequilibrium) {
  vlb_status st = check_handle(h);
  if (st) return st;
  if (!d_snap) return fail(h, VLB_ERR_ARG, "snapshot pointer is NULL");
  const vlb_params& p = h->p;
  double* shift = nullptr;
  if (conserve) {
    shift = h->totals + 6;  // two spare slots of the totals read-out
    const double inv_area = 1.0 / (4.0 * M_PI * M_PI * p.r * p.R);  // sum of the area elements, torus or flat
    VLB_CUDA(h, vlb::launch_snapshot_shift(d_snap, h->coefD, p.n_theta, p.n_phi, conserve[0], conserve[1], inv_area,
                                           h->partials, shift, h->stream));
  }
  const int keep = keep_nonequilibrium ? 1 : 0;
  if (h->esize == 8)
    VLB_CUDA(h, vlb::launch_snapshot_in<double>((double*)h->U[0], h->stride, h->N, h->n0, d_snap, shift, keep,
                                                h->stream));
  else
    VLB_CUDA(h, vlb::launch_snapshot_in<float>((float*)h->U[0], h->stride, h->N, h->n0, d_snap, shift, keep,
                                               h->stream));
  return VLB_OK;
}

vlb_status vlb_conv3x3_fwd(int32_t H, int32_t W, int32_t cin, int32_t cout, const void* x, const void* w,
                           const float* bias, const void* mask, int32_t relu, void* y_bf16, float* y_f32,
                           void* cuda_stream) {
  const char* why = nullptr;
  if (!vlb::conv_shape_ok(H, W, cin, cout, &why)) return fail(nullptr, VLB_ERR_ARG, "vlb_conv3x3_fwd: %s", why);
  if (!x || !w || (!y_bf16 && !y_f32)) return fail(nullptr, VLB_ERR_ARG, "vlb_conv3x3_fwd: NULL tensor");
  VLB_CUDA(nullptr, vlb::conv_fwd_tc(H, W, cin, cout, x, w, bias, mask, relu, y_bf16, y_f32, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_conv3x3_flip(int32_t cin, int32_t cout, const void* w, void* w_flipped, void* cuda_stream) {
  if (!w || !w_flipped || cin < 1 || cout < 1) return fail(nullptr, VLB_ERR_ARG, "vlb_conv3x3_flip: bad argument");
  VLB_CUDA(nullptr, vlb::conv_flip(cin, cout, w, w_flipped, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

size_t vlb_conv3x3_wgrad_workspace_bytes(int32_t H, int32_t W, int32_t cin, int32_t cout) {
  const char* why = nullptr;
  if (!vlb::conv_shape_ok(H, W, cin, cout, &why)) return 0;
  return vlb::conv_wgrad_workspace_bytes(H, W, cin, cout);
}

vlb_status vlb_conv3x3_bwd_weight(int32_t H, int32_t W, int32_t cin, int32_t cout, const void* x, const void* dy,
                                  float* dw, float* db, void* workspace, size_t bytes, void* cuda_stream) {
  const char* why = nullptr;
  if (!vlb::conv_shape_ok(H, W, cin, cout, &why)) return fail(nullptr, VLB_ERR_ARG, "vlb_conv3x3_bwd_weight: %s", why);
  if (!x || !dy || !dw || !workspace) return fail(nullptr, VLB_ERR_ARG, "vlb_conv3x3_bwd_weight: NULL tensor");
  if (bytes < vlb::conv_wgrad_workspace_bytes(H, W, cin, cout))
    return fail(nullptr, VLB_ERR_WORKSPACE, "vlb_conv3x3_bwd_weight: workspace too small");
  VLB_CUDA(nullptr, vlb::conv_wgrad(H, W, cin, cout, x, dy, dw, db, (float*)workspace, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_conv_status(void* cuda_stream, int32_t clear) {
  int raised = 0;
  VLB_CUDA(nullptr, vlb::conv_tc_status((cudaStream_t)cuda_stream, clear, &raised));
  if (raised)
    return fail(nullptr, VLB_ERR_TIMEOUT, "a bounded wait of a tensor-core convolution gave up: outputs of the "
                "convolution calls since the last clear are invalid");
  return VLB_OK;
}

vlb_status vlb_test_raise_flag(vlb_handle* h, int32_t value) {
  if (value < 0 || value > 2) return fail(h, VLB_ERR_ARG, "vlb_test_raise_flag: value must be 0, 1 or 2");
  if (!h) {
    VLB_CUDA(nullptr, vlb::conv_tc_raise(value));
    return VLB_OK;
  }
  vlb_status st = check_handle(h, true);
  if (st) return st;
  const int v = value;
  VLB_CUDA(h, cudaMemcpyAsync(h->flag, &v, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  VLB_CUDA(h, cudaStreamSynchronize(h->stream));
  return VLB_OK;
}

size_t vlb_reduce_workspace_bytes(void) { return sizeof(double) * vlb::sur_reduce_doubles(); }

vlb_status vlb_surrogate_norm(int64_t npix, const float* snap, float s_n_fixed, float s_u_fixed, const float g[4],
                              double* d_work, double* d_sums, float* d_norm8, void* cuda_stream) {
  if (npix < 1 || !snap || !d_work || !d_sums || !d_norm8)
    return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_norm: bad argument");
  const float ones[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  VLB_CUDA(nullptr, vlb::sur_norm(npix, snap, s_n_fixed, s_u_fixed, g ? g : ones, d_work, d_sums, d_norm8,
                                  (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_surrogate_features(int32_t H, int32_t W, double r_over_R, const float* snap, const float* d_norm,
                                  void* out_bf16, void* cuda_stream) {
  if (H < 1 || W < 1 || !snap || !out_bf16 || !d_norm)
    return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_features: bad argument");
  VLB_CUDA(nullptr, vlb::sur_features(H, W, r_over_R, snap, d_norm, out_bf16, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_surrogate_targets(int64_t npix, const float* before, const float* after, const float* d_scale,
                                 float* target, void* cuda_stream) {
  if (npix < 1 || !before || !after || !d_scale || !target)
    return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_targets: bad argument");
  VLB_CUDA(nullptr, vlb::sur_targets(npix, before, after, d_scale, target, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_surrogate_apply(int64_t npix, const float* before, const float* pred16, const float* d_scale,
                               float* after, void* cuda_stream) {
  if (npix < 1 || !before || !pred16 || !d_scale || !after)
    return fail(nullptr, VLB_ERR_ARG, "vlb_surrogate_apply: bad argument");
  VLB_CUDA(nullptr, vlb::sur_apply(npix, before, pred16, d_scale, after, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_snapshot_compare(int64_t npix, const float* a, const float* b, double* d_work, double* d_out4,
                                void* cuda_stream) {
  if (npix < 1 || !a || !b || !d_work || !d_out4) return fail(nullptr, VLB_ERR_ARG, "vlb_snapshot_compare: bad argument");
  VLB_CUDA(nullptr, vlb::sur_compare(npix, a, b, d_work, d_out4, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_channel_sums(int64_t npix, int32_t C, const float* x, double* d_work, double* d_out,
                            void* cuda_stream) {
  if (npix < 1 || C < 1 || C > 16 || !x || !d_work || !d_out)
    return fail(nullptr, VLB_ERR_ARG, "vlb_channel_sums: bad argument");
  VLB_CUDA(nullptr, vlb::sur_stats(npix, C, x, d_work, d_out, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_mse_loss(int64_t npix, const float* pred16, const float* target4, void* grad16_bf16, double* d_work,
                        double* d_loss, void* cuda_stream) {
  if (npix < 1 || !pred16 || !target4 || !d_work || !d_loss)
    return fail(nullptr, VLB_ERR_ARG, "vlb_mse_loss: bad argument");
  VLB_CUDA(nullptr, vlb::sur_mse(npix, pred16, target4, grad16_bf16, d_work, d_loss, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_adam_step(int64_t n, float* p, const float* g, float* m, float* v, int64_t t, float lr, float b1,
                         float b2, float eps, void* p_bf16, void* cuda_stream) {
  if (n < 1 || !p || !g || !m || !v || t < 1) return fail(nullptr, VLB_ERR_ARG, "vlb_adam_step: bad argument");
  VLB_CUDA(nullptr, vlb::sur_adam(n, p, g, m, v, t, lr, b1, b2, eps, p_bf16, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

vlb_status vlb_to_bf16(int64_t n, const float* x, void* y, void* cuda_stream) {
  if (n < 1 || !x || !y) return fail(nullptr, VLB_ERR_ARG, "vlb_to_bf16: bad argument");
  VLB_CUDA(nullptr, vlb::sur_to_bf16(n, x, y, (cudaStream_t)cuda_stream));
  return VLB_OK;
}

}  // extern "C"
