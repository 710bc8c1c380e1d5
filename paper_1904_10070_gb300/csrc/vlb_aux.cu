// Initialisation, state conversion, field read-out and FP64 diagnostic reductions.
//
// These kernels run once per set/get call or once per diagnostic, not per time step.  All of
// their arithmetic is done in FP64 (the FP32 state is widened on load), so the read-outs and the
// conserved totals carry no FP32 rounding beyond that of the state itself.
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

constexpr int TOTAL_BLOCKS = 512;
constexpr int TOTAL_THREADS = 256;
constexpr int NSUM = 8;

struct VD {
  double v[4], w[4];
};

VD make_vd() {
  const VelocityConsts c = velocity_consts();
  VD d;
  for (int i = 0; i < 4; ++i) {
    d.v[i] = c.v[i];
    d.w[i] = c.w[i];
  }
  return d;
}

__device__ __forceinline__ int wrapi(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

// phi as stored: one array in FP64 mode, hi + lo in FP32 mode.
template <typename T>
__device__ __forceinline__ void store_phi(T* state, int64_t stride, int64_t idx, double v) {
  const T hi = (T)v;
  state[NPOP * stride + idx] = hi;
  if (sizeof(T) == 4) state[(NPOP + 1) * stride + idx] = (T)(v - (double)hi);
}

template <typename T>
__device__ __forceinline__ double load_phi(const T* state, int64_t stride, int64_t idx) {
  double v = (double)state[NPOP * stride + idx];
  if (sizeof(T) == 4) v += (double)state[(NPOP + 1) * stride + idx];
  return v;
}

// f := f^eq(rho, u) (Eq. feq), phi := phi, stored as the deviation g = f^eq - n0 w_i w_j
// = w_i w_j ((n - n0) + n (poly - 1)).  FP64 state: evaluated in FP64.  FP32 state: n - n0 is formed in
// FP64 (exact enough that its rounding to FP32 is the only error), the Hermite polynomial and the
// product in FP32 -- every term is small next to the stored value's own rounding -- so the
// initialisation does not run on GB300's FP64 units.
template <typename T>
__global__ void init_feq_kernel(T* state, int64_t stride, const double* rho, const double* ut, const double* up,
                                const double* phi, int64_t n, double n0, VD vd) {
  using C = T;  // arithmetic of the polynomial: the state precision
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const double nn = rho[idx];
    const C a = (C)ut[idx], b = (C)up[idx], dn = (C)(nn - n0), nc = (C)nn;
    const C usq = a * a + b * b;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const C xi = (C)vd.v[i] * a + (C)vd.v[j] * b;
        const C pm1 = xi + C(0.5) * (xi * xi - usq) + xi * (xi * xi - C(3) * usq) * C(1.0 / 6.0);
        state[(4 * i + j) * stride + idx] = (T)((C)(vd.w[i] * vd.w[j]) * (dn + nc * pm1));
      }
    store_phi(state, stride, idx, phi[idx]);
  }
}

__device__ __forceinline__ double ref_pop(int k, double n0, const VD& vd) {
  return k < NPOP ? n0 * vd.w[k >> 2] * vd.w[k & 3] : 0.0;
}

template <typename T>
__global__ void convert_in_kernel(T* state, int64_t stride, const double* src, int64_t n, double n0, VD vd) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * NARR;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx / n, i = idx - k * n;
    if (k == NPOP)
      store_phi(state, stride, i, src[idx]);
    else
      state[k * stride + i] = (T)(src[idx] - ref_pop((int)k, n0, vd));
  }
}

template <typename T>
__global__ void convert_out_kernel(double* dst, const T* state, int64_t stride, int64_t n, double n0, VD vd) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * NARR;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx / n, i = idx - k * n;
    dst[idx] = k == NPOP ? load_phi(state, stride, i) : (double)state[k * stride + i] + ref_pop((int)k, n0, vd);
  }
}

template <typename T>
__device__ __forceinline__ void node_moments(const T* state, int64_t stride, int64_t idx, const VD& vd, double n0,
                                             double& n, double& ut, double& up) {
  double row[4] = {0, 0, 0, 0}, col[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double x = (double)state[(4 * i + j) * stride + idx];
      row[i] += x;
      col[j] += x;
    }
  n = n0 + ((row[0] + row[1]) + (row[2] + row[3]));
  const double inv_n = 1.0 / n;  // one FP64 division per node
  ut = (vd.v[0] * row[0] + vd.v[1] * row[1] + vd.v[2] * row[2] + vd.v[3] * row[3]) * inv_n;
  up = (vd.v[0] * col[0] + vd.v[1] * col[1] + vd.v[2] * col[2] + vd.v[3] * col[3]) * inv_n;
}

// rho, u (Sec. 2.3 moments), phi and mu (Eq. mu) in FP64; one CTA row per theta row (blockIdx.y).
template <typename T>
__global__ void fields_kernel(const T* state, int64_t stride, const double* coefd, int nt, int ns, double A,
                              double kappa, double n0, double* rho, double* ut, double* up, double* phi, double* mu, VD vd) {
  const int q = blockIdx.y, s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int64_t idx = (int64_t)q * ns + s;
  double nn, a, b;
  node_moments(state, stride, idx, vd, n0, nn, a, b);
  rho[idx] = nn;
  ut[idx] = a;
  up[idx] = b;
  const int qn = q + 1 == nt ? 0 : q + 1, qs = q == 0 ? nt - 1 : q - 1;
  const int se = s + 1 == ns ? 0 : s + 1, sw = s == 0 ? ns - 1 : s - 1;
  const double p0 = load_phi(state, stride, idx);
  const double pn = load_phi(state, stride, (int64_t)qn * ns + s);
  const double ps = load_phi(state, stride, (int64_t)qs * ns + s);
  const double pe = load_phi(state, stride, (int64_t)q * ns + se);
  const double pw = load_phi(state, stride, (int64_t)q * ns + sw);
  const double lap = coefd[C_LT * nt + q] * (coefd[C_JP * nt + q] * (pn - p0) - coefd[C_JM * nt + q] * (p0 - ps)) +
                     coefd[C_LP * nt + q] * (pe - 2.0 * p0 + pw);
  phi[idx] = p0;
  mu[idx] = -A * p0 * (1.0 - p0 * p0) - kappa * lap;
}

// Per-block FP64 partial sums: mass, phi total, Psi (Eq. Landau), max |u|, non-finite count, L_I.
template <typename T>
__global__ void __launch_bounds__(TOTAL_THREADS) totals_kernel(const T* state, int64_t stride, const double* coefd,
                                                               int nt, int ns, double r, double A, double kappa,
                                                               double n0, double gt, double edge_p, double* partials,
                                                               VD vd) {
  const int64_t n = (int64_t)nt * ns;
  double acc[NSUM] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / ns), s = (int)(idx - (int64_t)q * ns);
    double nn, a, b;
    node_moments(state, stride, idx, vd, n0, nn, a, b);
    const double dA = coefd[C_DA * nt + q];
    const double p0 = load_phi(state, stride, idx);
    const double pn = load_phi(state, stride, (int64_t)wrapi(q + 1, nt) * ns + s);
    const double ps = load_phi(state, stride, (int64_t)wrapi(q - 1, nt) * ns + s);
    const double pe = load_phi(state, stride, (int64_t)q * ns + wrapi(s + 1, ns));
    const double pw = load_phi(state, stride, (int64_t)q * ns + wrapi(s - 1, ns));
    const double g1 = (pn - ps) * gt, g2 = (pe - pw) * coefd[C_GP * nt + q];
    const double om = 1.0 - p0 * p0;
    acc[0] += nn * dA;
    acc[1] += p0 * dA;
    acc[2] += (0.25 * A * om * om + 0.5 * kappa * (g1 * g1 + g2 * g2)) * dA;
    const double umag = sqrt(a * a + b * b);
    acc[3] = fmax(acc[3], umag);
    if (!isfinite(nn) || !isfinite(umag) || !isfinite(p0)) acc[4] += 1.0;
    if (p0 * pe < 0.0) acc[5] += edge_p;                     // neighbour across varphi: r dtheta
    if (p0 * pn < 0.0) acc[5] += coefd[C_EDGE * nt + q];     // neighbour across theta
  }
  // warp then block reduction in a fixed order
  __shared__ double red[TOTAL_THREADS / 32][NSUM];
#pragma unroll
  for (int k = 0; k < NSUM; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = (k == 3) ? fmax(x, y) : x + y;
    }
    acc[k] = x;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < NSUM; ++k) red[wid][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < NSUM) {
    const int k = threadIdx.x;
    double x = (k == 3) ? 0.0 : 0.0;
    for (int w = 0; w < TOTAL_THREADS / 32; ++w) x = (k == 3) ? fmax(x, red[w][k]) : x + red[w][k];
    partials[blockIdx.x * NSUM + k] = x;
  }
}

// Fixed-order sum (or max) of part[b * stride + k] over b < nb by one warp: lane l takes b = l, l + 32,
// ... in order, then a shuffle tree; the result depends only on nb, not on scheduling.
__device__ __forceinline__ double warp_fold(const double* part, int nb, int stride, int k, bool is_max) {
  const int lane = threadIdx.x & 31;
  double x = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const double v = part[b * stride + k];
    x = is_max ? fmax(x, v) : x + v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_down_sync(0xffffffffu, x, o);
    x = is_max ? fmax(x, y) : x + y;
  }
  return x;
}

// one warp per output k (blockDim = 32 NSUM)
__global__ void totals_final_kernel(const double* partials, int nb, double* out) {
  const int k = threadIdx.x >> 5;
  const double x = warp_fold(partials, nb, NSUM, k, k == 3);
  if ((threadIdx.x & 31) == 0) out[k] = x;
}

__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

// The surrogate's snapshot kernels work in the state's own precision T (they run once per window).
template <typename T>
__device__ __forceinline__ void node_moments_t(const T* state, int64_t stride, int64_t idx, const VD& vd, T n0, T& n,
                                               T& ut, T& up) {
  T row[4] = {0, 0, 0, 0}, col[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T x = state[(4 * i + j) * stride + idx];
      row[i] += x;
      col[j] += x;
    }
  n = n0 + ((row[0] + row[1]) + (row[2] + row[3]));
  ut = ((T)vd.v[0] * row[0] + (T)vd.v[1] * row[1] + (T)vd.v[2] * row[2] + (T)vd.v[3] * row[3]) / n;
  up = ((T)vd.v[0] * col[0] + (T)vd.v[1] * col[1] + (T)vd.v[2] * col[2] + (T)vd.v[3] * col[3]) / n;
}

// (phi, n, u_theta, u_phi) per node, from the state, as FP32.
template <typename T>
__global__ void snapshot_out_kernel(const T* state, int64_t stride, int64_t n, T n0, float* snap, VD vd) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    T nn, a, b;
    node_moments_t(state, stride, idx, vd, n0, nn, a, b);
    reinterpret_cast<float4*>(snap)[idx] =
        make_float4((float)load_phi(state, stride, idx), (float)nn, (float)a, (float)b);
  }
}

// Per-block FP64 partial sums of n dA and phi dA over a snapshot (dA the row's area element).
__global__ void __launch_bounds__(TOTAL_THREADS) snapshot_sums_kernel(const float* snap, const double* coefd, int nt,
                                                                      int ns, double* partials) {
  const int64_t n = (int64_t)nt * ns;
  double sn = 0.0, sp = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = reinterpret_cast<const float4*>(snap)[idx];
    const double dA = coefd[C_DA * nt + (int)(idx / ns)];
    sn += (double)v.y * dA;
    sp += (double)v.x * dA;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sn += __shfl_down_sync(0xffffffffu, sn, o);
    sp += __shfl_down_sync(0xffffffffu, sp, o);
  }
  __shared__ double red[2][TOTAL_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = sn;
    red[1][wid] = sp;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double x = 0.0;
    for (int w = 0; w < TOTAL_THREADS / 32; ++w) x += red[threadIdx.x][w];
    partials[blockIdx.x * NSUM + threadIdx.x] = x;
  }
}

// shift[0] = (mass - sum n dA) / area, shift[1] = (phi_total - sum phi dA) / area (Sec. 2.5 totals);
// one warp per total (blockDim = 64).
__global__ void snapshot_shift_kernel(const double* partials, int nb, double mass, double phi_total, double inv_area,
                                      double* shift) {
  const int k = threadIdx.x >> 5;
  const double x = warp_fold(partials, nb, NSUM, k, false);
  if ((threadIdx.x & 31) == 0) shift[k] = ((k == 0 ? mass : phi_total) - x) * inv_area;
}

// The surrogate restart from a snapshot (n', u', phi'), with n' += shift[0] and phi' += shift[1] when
// shift != NULL.  keep_neq == 0: f := f^eq(n', u') (Eq. feq).  keep_neq != 0: f := f + f^eq(n', u') -
// f^eq(n, u) with (n, u) the moments of the current f, which keeps the non-equilibrium part f - f^eq
// of the state and gives f the moments (n', u').  In the deviation storage g = f - n0 w_i w_j:
// f^eq - n0 w_i w_j = w_i w_j ((n - n0) + n P(u)), P(u) = xi + (xi^2 - u^2)/2 + xi (xi^2 - 3 u^2)/6.
template <typename T>
__global__ void snapshot_in_kernel(T* state, int64_t stride, int64_t n, T n0, const float* snap, const double* shift,
                                   int keep_neq, VD vd) {
  const T dn = shift ? (T)shift[0] : (T)0, dphi = shift ? (T)shift[1] : (T)0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const float4 s = reinterpret_cast<const float4*>(snap)[idx];
    const T nn = (T)s.y + dn, a = (T)s.z, b = (T)s.w;
    const T usq = a * a + b * b;
    T n1 = 0, a1 = 0, b1 = 0, usq1 = 0;
    if (keep_neq) {
      node_moments_t(state, stride, idx, vd, n0, n1, a1, b1);
      usq1 = a1 * a1 + b1 * b1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const T vi = (T)vd.v[i], vj = (T)vd.v[j], ww = (T)(vd.w[i] * vd.w[j]);
        const T xi = vi * a + vj * b;
        const T pm = xi + (T)0.5 * (xi * xi - usq) + xi * (xi * xi - (T)3 * usq) / (T)6;
        T* g = state + (4 * i + j) * stride + idx;
        if (keep_neq) {
          const T xi1 = vi * a1 + vj * b1;
          const T pm1 = xi1 + (T)0.5 * (xi1 * xi1 - usq1) + xi1 * (xi1 * xi1 - (T)3 * usq1) / (T)6;
          // rounded products (no contraction): the state's own moments give exactly zero change
          *g = *g + ww * ((nn - n1) + (mul_rn(nn, pm) - mul_rn(n1, pm1)));
        } else {
          *g = ww * ((nn - n0) + nn * pm);
        }
      }
    store_phi(state, stride, idx, (double)s.x + (double)dphi);
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int totals_blocks() { return TOTAL_BLOCKS; }

// out[q] = sum over s of x[q][s], one CTA per row: each thread adds its strided elements in order,
// then a fixed-order tree in shared memory (deterministic).
__global__ void __launch_bounds__(256) row_sums_kernel(const double* x, int ns, double* out) {
  __shared__ double red[256];
  const double* row = x + (int64_t)blockIdx.x * ns;
  double acc = 0.0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) acc += row[s];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

cudaError_t launch_row_sums(const double* x, int nt, int ns, double* out, cudaStream_t s) {
  row_sums_kernel<<<nt, 256, 0, s>>>(x, ns, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_feq(T* state, int64_t stride, const double* rho, const double* ut, const double* up,
                            const double* phi, int64_t n, double n0, cudaStream_t s) {
  init_feq_kernel<T><<<grid_for(n), 256, 0, s>>>(state, stride, rho, ut, up, phi, n, n0, make_vd());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_in(T* state, int64_t stride, const double* src, int64_t n, double n0, cudaStream_t s) {
  convert_in_kernel<T><<<grid_for(n * NARR), 256, 0, s>>>(state, stride, src, n, n0, make_vd());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_out(double* dst, const T* state, int64_t stride, int64_t n, double n0, cudaStream_t s) {
  convert_out_kernel<T><<<grid_for(n * NARR), 256, 0, s>>>(dst, state, stride, n, n0, make_vd());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fields(const T* state, int64_t stride, const double* coefd, int nt, int ns, double A, double kappa,
                          double n0, double* rho, double* ut, double* up, double* phi, double* mu, cudaStream_t s) {
  fields_kernel<T><<<dim3((ns + 255) / 256, nt), 256, 0, s>>>(state, stride, coefd, nt, ns, A, kappa, n0, rho, ut, up,
                                                             phi, mu, make_vd());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_totals(const T* state, int64_t stride, const double* coefd, int nt, int ns, double R, double r,
                          double A, double kappa, double n0, int geometry, double* partials, int n_blocks,
                          double* out, cudaStream_t s) {
  (void)R;
  (void)geometry;
  const double dth = 2.0 * M_PI / nt;
  const double gt = 1.0 / (2.0 * r * dth);
  const double edge_p = r * dth;
  totals_kernel<T><<<n_blocks, TOTAL_THREADS, 0, s>>>(state, stride, coefd, nt, ns, r, A, kappa, n0, gt, edge_p,
                                                      partials, make_vd());
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  totals_final_kernel<<<1, 32 * NSUM, 0, s>>>(partials, n_blocks, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_snapshot_out(const T* state, int64_t stride, int64_t n, double n0, float* snap, cudaStream_t s) {
  snapshot_out_kernel<T><<<grid_for(n), 256, 0, s>>>(state, stride, n, (T)n0, snap, make_vd());
  return cudaGetLastError();
}

cudaError_t launch_snapshot_shift(const float* snap, const double* coefd, int nt, int ns, double mass,
                                  double phi_total, double inv_area, double* partials, double* shift, cudaStream_t s) {
  snapshot_sums_kernel<<<TOTAL_BLOCKS, TOTAL_THREADS, 0, s>>>(snap, coefd, nt, ns, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  snapshot_shift_kernel<<<1, 64, 0, s>>>(partials, TOTAL_BLOCKS, mass, phi_total, inv_area, shift);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_snapshot_in(T* state, int64_t stride, int64_t n, double n0, const float* snap, const double* shift,
                               int keep_neq, cudaStream_t s) {
  snapshot_in_kernel<T><<<grid_for(n), 256, 0, s>>>(state, stride, n, (T)n0, snap, shift, keep_neq, make_vd());
  return cudaGetLastError();
}

#define VLB_INST(T)                                                                                              \
  template cudaError_t launch_init_feq<T>(T*, int64_t, const double*, const double*, const double*,              \
                                          const double*, int64_t, double, cudaStream_t);                          \
  template cudaError_t launch_convert_in<T>(T*, int64_t, const double*, int64_t, double, cudaStream_t);         \
  template cudaError_t launch_convert_out<T>(double*, const T*, int64_t, int64_t, double, cudaStream_t);        \
  template cudaError_t launch_fields<T>(const T*, int64_t, const double*, int, int, double, double, double,     \
                                        double*, double*, double*, double*, double*, cudaStream_t);               \
  template cudaError_t launch_totals<T>(const T*, int64_t, const double*, int, int, double, double, double,      \
                                        double, double, int, double*, int, double*, cudaStream_t);               \
  template cudaError_t launch_snapshot_out<T>(const T*, int64_t, int64_t, double, float*, cudaStream_t);        \
  template cudaError_t launch_snapshot_in<T>(T*, int64_t, int64_t, double, const float*, const double*, int,   \
                                             cudaStream_t);
VLB_INST(float)
VLB_INST(double)
#undef VLB_INST

}  // namespace vlb
