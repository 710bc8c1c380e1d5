// vlb_step_noalloc: the SSP-RK3 step without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need to advance a state:
// plug-ins whose host application hands out only pre-sized device buffers from its own arena (the
// host owns the memory budget), and latency-critical loops where cudaMalloc's implicit device
// synchronisation is not acceptable.  For them this entry point keeps the two
// intermediate Runge-Kutta states and the per-row coefficient tables in one file-scope device
// array of fixed size; the caller passes only the state it owns.
//
// The array is a device symbol: host code cannot use its name as a device address.  Its address
// is obtained with cudaGetSymbolAddress once per device (with that device current) and cached.
// Every call shares the array, so two calls whose work overlaps on the GPU (different streams,
// or different host threads on one device) race; calls on one stream are ordered.  Nothing in it
// needs to start at zero: the coefficient tables are rewritten by every call, and each Runge-
// Kutta stage writes every node of its output buffer before the next stage reads it.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "vlb_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[VLB_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
thread_local char g_noalloc_err[256] = "";

// Device address of the scratch array on the current device (set-up on the first call per device).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Row coefficient tables (the same quantities the handle API precomputes on the host), evaluated
// in FP64 on the device and rounded once to T.
template <typename T>
__global__ void noalloc_tables(T* coef, int nt, int nphi, int geometry, int advection, double R, double r) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  const double pi = 3.14159265358979323846;
  const double dth = 2.0 * pi / nt, dph = 2.0 * pi / nphi;
  const bool torus = geometry == VLB_TORUS;
  const double a = torus ? r / R : 0.0;
  const double th = q * dth;
  auto Jat = [&](int d) { return 1.0 + a * cos(th + d * dth); };
  const double J = Jat(0);
  const double gam = torus ? sin(th) / (R * J) : 0.0;
  coef[vlb::C_J * nt + q] = (T)J;
  coef[vlb::C_JP * nt + q] = (T)(1.0 + a * cos(th + 0.5 * dth));
  coef[vlb::C_JM * nt + q] = (T)(1.0 + a * cos(th - 0.5 * dth));
  coef[vlb::C_CT * nt + q] = (T)(1.0 / (r * J * dth));
  coef[vlb::C_CP * nt + q] = (T)(1.0 / (R * J * dph));
  coef[vlb::C_GAM * nt + q] = (T)gam;
  coef[vlb::C_LT * nt + q] = (T)(1.0 / (r * r * J * dth * dth));
  coef[vlb::C_LP * nt + q] = (T)(1.0 / (R * R * J * J * dph * dph));
  coef[vlb::C_GP * nt + q] = (T)(1.0 / (2.0 * R * J * dph));
  if (advection == VLB_UW3) {
    const double dpos = (Jat(-2) - 6.0 * Jat(-1) + 3.0 * Jat(0) + 2.0 * Jat(1)) / 6.0;
    const double dneg = (-2.0 * Jat(-1) - 3.0 * Jat(0) + 6.0 * Jat(1) - Jat(2)) / 6.0;
    coef[vlb::C_EP * nt + q] = (T)(-dpos / (r * J * dth) - gam);
    coef[vlb::C_EN * nt + q] = (T)(-dneg / (r * J * dth) - gam);
  } else {
    coef[vlb::C_EP * nt + q] = (T)(-gam);
    coef[vlb::C_EN * nt + q] = (T)(-gam);
  }
}

const char* check_params(const vlb_params* p) {
  if (!p) return "params is NULL";
  if (p->geometry != VLB_TORUS && p->geometry != VLB_FLAT) return "geometry must be 0 or 1";
  if (p->precision != VLB_FP64 && p->precision != VLB_FP32) return "precision must be 0 or 1";
  if (p->advection != VLB_UW3 && p->advection != VLB_WENO5) return "advection must be 0 or 1";
  if (p->ch_mode != VLB_HYDRO && p->ch_mode != VLB_DIFFUSIVE) return "ch_mode must be 0 or 1";
  if (p->n_theta < (p->advection == VLB_WENO5 ? 6 : 4) || p->n_phi < 1) return "grid too small";
  if (p->n_theta > 65535 * 16) return "n_theta too large";
  if (!(p->r > 0.0) || !(p->R > 0.0) || !isfinite(p->r) || !isfinite(p->R)) return "radii must be finite and > 0";
  if (p->geometry == VLB_TORUS && !(p->R > p->r)) return "torus needs R > r";
  if (!(p->dt > 0.0) || !isfinite(p->dt) || !(p->tau > 0.0)) return "dt must be finite and > 0, tau > 0";
  if (!(p->M >= 0.0) || !(p->A >= 0.0) || !(p->kappa >= 0.0)) return "M, A, kappa must be >= 0";
  if (p->ch_stab != 0) return "the no-allocation step runs the explicit Cahn-Hilliard step (ch_stab must be 0)";
  return nullptr;
}

template <typename T>
cudaError_t run(const vlb_params* p, T* state, int64_t stride, double n0, int64_t nsteps, unsigned char* scratch,
                cudaStream_t st) {
  const int nt = p->n_theta;
  T* coef = reinterpret_cast<T*>(scratch);
  T* U1 = reinterpret_cast<T*>(scratch + align256(sizeof(T) * vlb::NCOEF * nt));
  T* U2 = U1 + (size_t)vlb::state_arrays(sizeof(T)) * stride;
  noalloc_tables<T><<<(nt + 127) / 128, 128, 0, st>>>(coef, nt, p->n_phi, p->geometry, p->advection, p->R, p->r);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vlb::StageArgs<T> a;
  a.coef = coef;
  a.nt = nt;
  a.ns = p->n_phi;
  a.stride = stride;
  a.dt = (T)p->dt;
  a.inv_tau = (T)(1.0 / p->tau);
  a.M = (T)p->M;
  a.A = (T)p->A;
  a.kappa = (T)p->kappa;
  a.gt = (T)(1.0 / (2.0 * p->r * (2.0 * M_PI / nt)));
  a.n0 = (T)n0;
  a.err = nullptr;
  for (int64_t n = 0; n < nsteps; ++n) {
    a.fin = state; a.f0 = nullptr; a.fout = U1; a.b = (T)1;
    if ((e = vlb::launch_stage<T>(a, p->advection, p->ch_mode, st)) != cudaSuccess) return e;
    a.fin = U1; a.f0 = state; a.fout = U2; a.b = (T)0.25;
    if ((e = vlb::launch_stage<T>(a, p->advection, p->ch_mode, st)) != cudaSuccess) return e;
    a.fin = U2; a.f0 = state; a.fout = state; a.b = (T)(2.0 / 3.0);
    if ((e = vlb::launch_stage<T>(a, p->advection, p->ch_mode, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

vlb_status vlb_step_noalloc(const vlb_params* p, void* d_state, int64_t stride, double n0, int64_t nsteps,
                            void* cuda_stream, const char** error) {
  static const char* kOk = "";
  if (error) *error = kOk;
  auto fail = [&](vlb_status s, const char* msg) {
    snprintf(g_noalloc_err, sizeof g_noalloc_err, "vlb_step_noalloc: %s", msg);
    if (error) *error = g_noalloc_err;
    return s;
  };
  if (const char* why = check_params(p)) return fail(VLB_ERR_ARG, why);
  if (!d_state) return fail(VLB_ERR_ARG, "state is NULL");
  if (((uintptr_t)d_state) % 256 != 0) return fail(VLB_ERR_ARG, "state must be 256-byte aligned");
  const int64_t N = (int64_t)p->n_theta * p->n_phi;
  if (stride < N || stride % 64 != 0) return fail(VLB_ERR_ARG, "stride must be >= n_theta * n_phi and a multiple of 64");
  if (nsteps < 0) return fail(VLB_ERR_ARG, "nsteps must be >= 0");
  if (!(n0 > 0.0) || !isfinite(n0)) return fail(VLB_ERR_ARG, "n0 must be finite and > 0");
  const size_t esize = p->precision == VLB_FP64 ? 8 : 4;
  // bound the stride first, so that the size arithmetic below cannot wrap around
  const int64_t max_stride = (int64_t)(VLB_NOALLOC_SCRATCH_BYTES / (2 * (size_t)vlb::state_arrays(esize) * esize));
  if (stride > max_stride) {
    char msg[160];
    snprintf(msg, sizeof msg, "stride %lld exceeds %lld elements, the most the fixed scratch (VLB_NOALLOC_SCRATCH_BYTES) holds",
             (long long)stride, (long long)max_stride);
    return fail(VLB_ERR_ARG, msg);
  }
  const size_t need = align256(esize * vlb::NCOEF * p->n_theta) +
                      2 * (size_t)vlb::state_arrays(esize) * (size_t)stride * esize;
  if (need > VLB_NOALLOC_SCRATCH_BYTES) {
    char msg[160];
    snprintf(msg, sizeof msg, "grid needs %zu bytes of scratch, more than the fixed %zu (VLB_NOALLOC_SCRATCH_BYTES)",
             need, (size_t)VLB_NOALLOC_SCRATCH_BYTES);
    return fail(VLB_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(VLB_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(VLB_ERR_CUDA, "device index out of range");
  void* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) return fail(VLB_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  e = esize == 8 ? run<double>(p, (double*)d_state, stride, n0, nsteps, (unsigned char*)scratch, st)
                 : run<float>(p, (float*)d_state, stride, n0, nsteps, (unsigned char*)scratch, st);
  if (e != cudaSuccess) return fail(VLB_ERR_CUDA, cudaGetErrorString(e));
  return VLB_OK;
}

}  // extern "C"
