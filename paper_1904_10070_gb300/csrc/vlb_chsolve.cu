// Stabilised semi-implicit Cahn-Hilliard stage (not part of the paper's method, which advances Eq. CH
// explicitly; the explicit step is limited to dt ~ h^4 / (M kappa)).
//
// With the stabilisation the phi part of every SSP-RK3 stage reads
//   phi_out = phi^n + b (phi_in - phi^n + P(dt L_phi(phi_in))),   (first stage: phi^n = phi_in, b = 1)
// with the fixed preconditioner P = J^{-1} (I + dt M kappa D^2)^{-1} J, D the constant-coefficient
// periodic five-point Laplacian at the finest spacings of the grid (h_theta = r dtheta, h_phi =
// (R - r) dvarphi on the torus, R dvarphi flat).  P is diagonal in the discrete Fourier basis of J x:
// a mode (m, n) is divided by 1 + dt M kappa lambda(m, n) with lambda = ((4/h_theta^2) sin^2(pi m/N_theta)
// + (4/h_phi^2) sin^2(pi n/N_phi))^2; the mean (m = n = 0) is kept, so P conserves sum J x (the
// integral of x sqrt(g)).  The stage kernel writes dt L_phi into a scratch array; three kernels then
//   1. transform every theta row of J dt L_phi (complex FFT of real data, one CTA per row),
//   2. transform strips of columns, divide by 1 + dt M kappa lambda and transform them back,
//   3. transform every row back, take the real part / (N_theta N_phi J), and form phi_out (in FP32 as
//      the float pair hi + lo with an error-free sum, as the stage kernel does).
// The FFTs are in-place radix-2 (decimation in time, bit-reversed load) in shared memory, in the
// state's precision, with twiddles from sincospi; N_theta and N_phi are powers of two <= 4096.  The
// two factors of lambda, (4/h_theta^2) sin^2(pi m/N_theta) and (4/h_phi^2) sin^2(pi n/N_phi), are
// tabulated once in FP64 on the host (ch_stab_tables) and rounded to the state precision, so the
// division runs in that precision with no transcendental per mode; so are the twiddles of both
// transform lengths, which each CTA copies from global memory (L2) into shared memory.
#include <math.h>

#include <vector>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

template <typename T>
struct C2 {
  T x, y;
};

__device__ __forceinline__ void sincospi_t(double a, double* s, double* c) { sincospi(a, s, c); }
__device__ __forceinline__ void sincospi_t(float a, float* s, float* c) { sincospif(a, s, c); }

__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// Twiddles stored level by level, so that the butterflies of one level read consecutive entries
// (a single table indexed by j n / 2^l puts a warp's reads on one shared-memory bank at the middle
// levels): tw[2^(l-1) - 1 + j] = exp(-2 pi i j / 2^l), j < 2^(l-1), l = 1 .. log2 n; n - 1 entries.
template <typename T>
__device__ void twiddles(C2<T>* tw, int n) {
  for (int k = threadIdx.x; k < n - 1; k += blockDim.x) {
    const int half = 1 << (31 - __clz(k + 1));  // 2^(l-1), the level's first entry is half - 1
    const int j = k + 1 - half;
    T s, c;
    sincospi_t((T)(-(double)j / half), &s, &c);  // -2 pi j / 2^l = -pi j / half
    tw[k].x = c;
    tw[k].y = s;
  }
}

// Shared-memory position of element e of a row transform: one pad element every 2^sh elements, so
// that the bit-reversed scatter of 32 consecutive indices (multiples of n / 32) and the butterflies
// spread over the banks.  Column strips use sh = 31 (no padding).
__device__ __forceinline__ int padded(int e, int sh) { return e + (e >> sh); }
__host__ __device__ inline int row_pad_shift(int logn) { return logn >= 5 ? logn - 5 : 31; }

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> v, C2<T> t) {
  return {v.x * t.x - v.y * t.y, v.x * t.y + v.y * t.x};
}

// In-place FFT along the first index of a[i * w + c] (w = 2^logw interleaved sequences of length n,
// loaded in bit-reversed order of i; element e stored at padded(e, sh)), decimation in time: the
// radix-2 levels l = 1 .. log2 n, taken two at a time as one radix-4 pass (one radix-2 pass first when
// log2 n is odd), which halves the shared-memory passes and barriers.  A radix-4 group of levels
// (l, l + 1) holds the elements i0 + {0, 1, 2, 3} h (h = 2^(l-1), i0 = 4h (g / h) + g % h, j = g % h):
// level l pairs (0, 1) and (2, 3) with twiddle t1 = W_2h^j, level l + 1 pairs (0, 2) with
// t2 = W_4h^j and (1, 3) with W_4h^(j + h) = -i t2 (+i t2 for the inverse).  inverse: conjugate
// twiddles (unnormalised).
template <typename T>
__device__ void fft_strided(C2<T>* a, int n, int logn, int logw, int sh, const C2<T>* tw, bool inverse) {
  const int w = 1 << logw;
  int l = 1;
  if (logn & 1) {  // level 1 alone: pairs (2 g, 2 g + 1), twiddle 1
    const int nb = (n >> 1) << logw;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
      const int g = idx >> logw, c = idx & (w - 1);
      const int e0 = padded(((2 * g) << logw) + c, sh), e1 = padded(((2 * g + 1) << logw) + c, sh);
      const C2<T> u = a[e0], v = a[e1];
      a[e0] = {u.x + v.x, u.y + v.y};
      a[e1] = {u.x - v.x, u.y - v.y};
    }
    __syncthreads();
    l = 2;
  }
  const int nq = (n >> 2) << logw;
  for (; l < logn; l += 2) {
    const int h = 1 << (l - 1);
    for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
      const int g = idx >> logw, c = idx & (w - 1);
      const int j = g & (h - 1);
      const int i0 = ((g >> (l - 1)) << (l + 1)) + j;
      C2<T> t1 = tw[h - 1 + j], t2 = tw[2 * h - 1 + j];
      if (inverse) {
        t1.y = -t1.y;
        t2.y = -t2.y;
      }
      const int e0 = padded((i0 << logw) + c, sh), e1 = padded(((i0 + h) << logw) + c, sh);
      const int e2 = padded(((i0 + 2 * h) << logw) + c, sh), e3 = padded(((i0 + 3 * h) << logw) + c, sh);
      const C2<T> a0 = a[e0], a1 = cmul(a[e1], t1), a2 = a[e2], a3 = cmul(a[e3], t1);
      const C2<T> b0 = {a0.x + a1.x, a0.y + a1.y}, b1 = {a0.x - a1.x, a0.y - a1.y};
      const C2<T> b2 = cmul(C2<T>{a2.x + a3.x, a2.y + a3.y}, t2);
      C2<T> b3 = cmul(C2<T>{a2.x - a3.x, a2.y - a3.y}, t2);
      b3 = inverse ? C2<T>{-b3.y, b3.x} : C2<T>{b3.y, -b3.x};  // times +i / -i
      a[e0] = {b0.x + b2.x, b0.y + b2.y};
      a[e2] = {b0.x - b2.x, b0.y - b2.y};
      a[e1] = {b1.x + b3.x, b1.y + b3.y};
      a[e3] = {b1.x - b3.x, b1.y - b3.y};
    }
    __syncthreads();
  }
}

constexpr int kBatch = 8;  // global loads a thread keeps in flight before it stores them

// the n - 1 per-level twiddles of a transform, from the host-computed table
template <typename T>
__device__ __forceinline__ void load_twiddles(C2<T>* tw, const C2<T>* table, int n) {
  for (int k0 = threadIdx.x; k0 < n - 1; k0 += kBatch * blockDim.x) {
    C2<T> v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int k = k0 + u * blockDim.x;
      if (k < n - 1) v[u] = table[k];
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int k = k0 + u * blockDim.x;
      if (k < n - 1) tw[k] = v[u];
    }
  }
}

// 1. Row q: F_phi[J_q dt L_phi(q, .)] -> buf row q.
template <typename T>
__global__ void __launch_bounds__(256) row_fwd_kernel(int ns, int logns, const T* dphi, const double* J,
                                                      const C2<T>* tw_s, C2<T>* buf) {
  extern __shared__ __align__(16) unsigned char raw[];
  C2<T>* a = reinterpret_cast<C2<T>*>(raw);
  const int sh = row_pad_shift(logns);
  C2<T>* tw = a + padded(ns, sh);
  const int q = blockIdx.x;
  const T jq = (T)J[q];
  const T* row = dphi + (int64_t)q * ns;
  for (int s0 = threadIdx.x; s0 < ns; s0 += kBatch * blockDim.x) {
    T v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < ns) v[u] = row[s];
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < ns) a[padded(bitrev(s, logns), sh)] = {jq * v[u], T(0)};
    }
  }
  load_twiddles(tw, tw_s, ns);
  __syncthreads();
  fft_strided(a, ns, logns, 0, sh, tw, false);
  for (int s = threadIdx.x; s < ns; s += blockDim.x) buf[(int64_t)q * ns + s] = a[padded(s, sh)];
}

// 2. Columns n0 .. n0 + cw - 1: F_theta, division by 1 + s lambda(m, n), inverse F_theta.
template <typename T>
__global__ void __launch_bounds__(256) col_solve_kernel(int nt, int lognt, int ns, int lcw, T sfac, const T* lam_t,
                                                        const T* lam_p, const C2<T>* tw_t, C2<T>* buf) {
  extern __shared__ __align__(16) unsigned char raw[];
  C2<T>* a = reinterpret_cast<C2<T>*>(raw);
  const int cw = 1 << lcw;
  C2<T>* tw = a + ((size_t)nt << lcw);
  const int n0 = blockIdx.x << lcw;
  const int total = nt << lcw;
  for (int i0 = threadIdx.x; i0 < total; i0 += kBatch * blockDim.x) {
    C2<T> v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) v[u] = buf[(int64_t)(idx >> lcw) * ns + n0 + (idx & (cw - 1))];
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) a[(bitrev(idx >> lcw, lognt) << lcw) + (idx & (cw - 1))] = v[u];
    }
  }
  load_twiddles(tw, tw_t, nt);
  __syncthreads();
  fft_strided(a, nt, lognt, lcw, 31, tw, false);
  const T lp = lam_p[n0 + (threadIdx.x & (cw - 1))];  // a thread keeps its column (blockDim % cw == 0)
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int m = idx >> lcw;
    const T lap = lam_t[m] + lp;
    const T g = T(1) / (T(1) + sfac * lap * lap);
    a[idx].x *= g;
    a[idx].y *= g;
  }
  __syncthreads();
  // back to bit-reversed order for the inverse transform: in-place swaps of the pairs (m, rev(m))
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int m = idx >> lcw, c = idx & (cw - 1), r = bitrev(m, lognt);
    if (m < r) {
      const C2<T> t = a[idx];
      a[idx] = a[(r << lcw) + c];
      a[(r << lcw) + c] = t;
    }
  }
  __syncthreads();
  fft_strided(a, nt, lognt, lcw, 31, tw, true);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int q = idx >> lcw, c = idx & (cw - 1);
    buf[(int64_t)q * ns + n0 + c] = a[idx];
  }
}

// (hi, lo) <- (base, base_lo) + inc with an error-free sum, renormalised (FP32 float pair)
__device__ __forceinline__ void pair_add(float base, float base_lo, float inc, float& hi, float& lo) {
  const float s1 = base + inc;
  const float bb = s1 - base;
  const float err = (base - (s1 - bb)) + (inc - bb);
  const float lo2 = base_lo + err;
  hi = s1 + lo2;
  lo = lo2 - (hi - s1);
}

// 3. Row q: inverse F_phi, y = Re / (N J_q), phi_out = phi^n + b (phi_in - phi^n + y).
template <typename T>
__global__ void __launch_bounds__(256) row_inv_kernel(int ns, int logns, double inv_n, const double* J,
                                                      const C2<T>* tw_s, const C2<T>* buf, const T* phin,
                                                      const T* phi0, T* phiout, int64_t lo_off, T b) {
  constexpr bool DF = sizeof(T) == 4;  // phi as a float pair
  constexpr int U = 4;                 // nodes per batch of loads (four state words each)
  extern __shared__ __align__(16) unsigned char raw[];
  C2<T>* a = reinterpret_cast<C2<T>*>(raw);
  const int sh = row_pad_shift(logns);
  C2<T>* tw = a + padded(ns, sh);
  const int q = blockIdx.x;
  const C2<T>* row = buf + (int64_t)q * ns;
  for (int s0 = threadIdx.x; s0 < ns; s0 += kBatch * blockDim.x) {
    C2<T> v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < ns) v[u] = row[s];
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < ns) a[padded(bitrev(s, logns), sh)] = v[u];
    }
  }
  load_twiddles(tw, tw_s, ns);
  __syncthreads();
  fft_strided(a, ns, logns, 0, sh, tw, true);
  const T scale = (T)(inv_n / J[q]);
  for (int s0 = threadIdx.x; s0 < ns; s0 += U * blockDim.x) {
    T ph[U], lo[U], base[U], base_lo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s < ns) {
        const int64_t g = (int64_t)q * ns + s;
        ph[u] = phin[g];
        lo[u] = DF ? phin[g + lo_off] : T(0);
        base[u] = phi0 ? phi0[g] : ph[u];
        base_lo[u] = phi0 ? (DF ? phi0[g + lo_off] : T(0)) : lo[u];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * blockDim.x;
      if (s >= ns) continue;
      const int64_t g = (int64_t)q * ns + s;
      const T y = a[padded(s, sh)].x * scale;
      const T inc = phi0 ? b * (((ph[u] - base[u]) + (lo[u] - base_lo[u])) + y) : y;
      if constexpr (DF) {
        float hi_o, lo_o;
        pair_add(base[u], base_lo[u], inc, hi_o, lo_o);
        phiout[g] = hi_o;
        phiout[g + lo_off] = lo_o;
      } else {
        phiout[g] = base[u] + inc;
      }
    }
  }
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes, int& mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (mask & (1 << dev))) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 32) mask |= 1 << dev;
  return e;
}

constexpr size_t kColBudget = 96 * 1024;  // shared bytes of a column strip (without twiddles)

}  // namespace

bool ch_stab_shape_ok(int nt, int ns) {
  auto pow2 = [](int n) { return n >= 4 && n <= 4096 && (n & (n - 1)) == 0; };
  return pow2(nt) && pow2(ns);
}

// the complex spectrum, then the tables: the two factors of lambda (N_theta + N_phi values) and the
// per-level twiddles of both transform lengths ((N_theta - 1) + (N_phi - 1) complex values)
size_t ch_stab_table_elems(int nt, int ns) { return (size_t)(nt + ns) + 2 * (size_t)(nt - 1 + ns - 1); }
size_t ch_stab_buffer_bytes(int nt, int ns, size_t esize) {
  return ((size_t)nt * ns * 2 + ch_stab_table_elems(nt, ns)) * esize;
}
size_t ch_stab_table_offset(int nt, int ns, size_t esize) { return (size_t)nt * ns * 2 * esize; }

void ch_stab_tables(int nt, int ns, double h_t, double h_p, size_t esize, void* host_out) {
  std::vector<double> v;
  v.reserve(ch_stab_table_elems(nt, ns));
  for (int i = 0; i < nt + ns; ++i) {
    const bool th = i < nt;
    const double sn = sin(M_PI * (th ? i : i - nt) / (th ? nt : ns));
    v.push_back((th ? 4.0 / (h_t * h_t) : 4.0 / (h_p * h_p)) * sn * sn);
  }
  // twiddles level by level: entry 2^(l-1) - 1 + j = exp(-2 pi i j / 2^l), j < 2^(l-1)
  for (int n : {nt, ns})
    for (int half = 1; half < n; half *= 2)
      for (int j = 0; j < half; ++j) {
        v.push_back(cos(M_PI * j / half));
        v.push_back(-sin(M_PI * j / half));
      }
  for (size_t i = 0; i < v.size(); ++i) {
    if (esize == 8)
      ((double*)host_out)[i] = v[i];
    else
      ((float*)host_out)[i] = (float)v[i];
  }
}

template <typename T>
cudaError_t launch_ch_stab(int nt, int ns, double dt_m_kappa, const double* J, const T* dphi, void* buf, const T* phin,
                           const T* phi0, T* phiout, int64_t lo_off, T b, cudaStream_t st) {
  if (!ch_stab_shape_ok(nt, ns)) return cudaErrorInvalidValue;
  const int lognt = ilog2(nt), logns = ilog2(ns);
  C2<T>* cb = reinterpret_cast<C2<T>*>(buf);
  const T* lam = reinterpret_cast<const T*>(buf) + (size_t)nt * ns * 2;  // ch_stab_tables
  const C2<T>* tw_t = reinterpret_cast<const C2<T>*>(lam + nt + ns);      // 8- or 16-byte aligned
  const C2<T>* tw_s = tw_t + (nt - 1);
  const size_t row_bytes = sizeof(C2<T>) * ((size_t)ns * 2 + 32);  // data (with its pads) and twiddles
  // column strips of 2^lcw columns: wide enough for whole 32-byte segments, narrow enough that the
  // launch keeps at least 512 CTAs (about three per SM) when the grid allows
  int lcw = 0;
  while (lcw < 5 && (2 << lcw) <= ns && ((size_t)nt << lcw) * 2 * sizeof(C2<T>) <= kColBudget &&
         (lcw < 2 || (ns >> (lcw + 1)) >= 512))
    ++lcw;
  const size_t col_bytes = sizeof(C2<T>) * (((size_t)nt << lcw) + nt);
  // the attribute is set once per device to the largest size any grid needs (setting it to a
  // smaller size would cap later launches on larger grids)
  constexpr size_t row_max = sizeof(C2<T>) * (4096 * 2 + 32);
  constexpr size_t col_max = kColBudget + sizeof(C2<T>) * 4096;
  static int m1 = 0, m2 = 0, m3 = 0;
  cudaError_t e;
  if ((e = smem_attr(row_fwd_kernel<T>, row_max, m1)) != cudaSuccess) return e;
  if ((e = smem_attr(col_solve_kernel<T>, col_max, m2)) != cudaSuccess) return e;
  if ((e = smem_attr(row_inv_kernel<T>, row_max, m3)) != cudaSuccess) return e;
  row_fwd_kernel<T><<<nt, 256, row_bytes, st>>>(ns, logns, dphi, J, tw_s, cb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  col_solve_kernel<T><<<ns >> lcw, 256, col_bytes, st>>>(nt, lognt, ns, lcw, (T)dt_m_kappa, lam, lam + nt, tw_t, cb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  row_inv_kernel<T><<<nt, 256, row_bytes, st>>>(ns, logns, 1.0 / ((double)nt * ns), J, tw_s, cb, phin, phi0, phiout,
                                               lo_off, b);
  return cudaGetLastError();
}

namespace {

// ---- Structure factor S(m, n) = |F phi|^2 and its two sums (the L_S diagnostic) --------------------
// The same radix-2 transforms in FP64 whatever the state's precision (phi in FP32 is the float pair
// hi + lo, exact in a double): rows first, then strips of columns, whose CTA sums S and |k| S over its
// strip (k = (m'/r, n'/R), m' and n' the signed frequencies; the mean mode m = n = 0 is left out) and
// writes the two sums to part[2 b], part[2 b + 1].

template <typename T>
__global__ void __launch_bounds__(256) sf_row_kernel(int ns, int logns, const T* phi, const T* phi_lo,
                                                     C2<double>* buf) {
  extern __shared__ __align__(16) unsigned char raw[];
  C2<double>* a = reinterpret_cast<C2<double>*>(raw);
  C2<double>* tw = a + ns;
  const int q = blockIdx.x;
  twiddles(tw, ns);
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const int64_t g = (int64_t)q * ns + s;
    const double v = (double)phi[g] + (phi_lo ? (double)phi_lo[g] : 0.0);
    a[bitrev(s, logns)] = {v, 0.0};
  }
  __syncthreads();
  fft_strided(a, ns, logns, 0, 31, tw, false);
  for (int s = threadIdx.x; s < ns; s += blockDim.x) buf[(int64_t)q * ns + s] = a[s];
}

__global__ void __launch_bounds__(256) sf_col_kernel(int nt, int lognt, int ns, int cw, double kt, double kp,
                                                     const C2<double>* buf, double* part) {
  extern __shared__ __align__(16) unsigned char raw[];
  C2<double>* a = reinterpret_cast<C2<double>*>(raw);
  C2<double>* tw = a + (size_t)nt * cw;
  __shared__ double red[2][8];
  const int n0 = blockIdx.x * cw;
  twiddles(tw, nt);
  for (int idx = threadIdx.x; idx < nt * cw; idx += blockDim.x) {
    const int q = idx / cw, c = idx - q * cw;
    a[bitrev(q, lognt) * cw + c] = buf[(int64_t)q * ns + n0 + c];
  }
  __syncthreads();
  fft_strided(a, nt, lognt, __ffs(cw) - 1, 31, tw, false);  // cw is a power of two
  double s_sum = 0.0, k_sum = 0.0;
  for (int idx = threadIdx.x; idx < nt * cw; idx += blockDim.x) {
    const int m = idx / cw, n = n0 + idx - m * cw;
    if (m == 0 && n == 0) continue;
    const int ms = m <= nt / 2 ? m : m - nt, nsg = n <= ns / 2 ? n : n - ns;
    const double S = a[idx].x * a[idx].x + a[idx].y * a[idx].y;
    const double k = sqrt((ms * kt) * (ms * kt) + (nsg * kp) * (nsg * kp));
    s_sum += S;
    k_sum += k * S;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_sum += __shfl_xor_sync(0xffffffffu, s_sum, o);
    k_sum += __shfl_xor_sync(0xffffffffu, k_sum, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = s_sum;
    red[1][warp] = k_sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a0 += red[0][w];
      a1 += red[1][w];
    }
    part[2 * blockIdx.x] = a0;
    part[2 * blockIdx.x + 1] = a1;
  }
}

}  // namespace

int structure_blocks(int nt, int ns) {
  int cw = 1;
  while (cw < 32 && cw * 2 <= ns && (size_t)nt * cw * 2 * sizeof(C2<double>) <= kColBudget) cw *= 2;
  return ns / cw;
}

template <typename T>
cudaError_t launch_structure_sums(int nt, int ns, double r, double R, const T* phi, const T* phi_lo, void* buf,
                                  double* part, cudaStream_t st) {
  if (!ch_stab_shape_ok(nt, ns)) return cudaErrorInvalidValue;
  const int lognt = ilog2(nt), logns = ilog2(ns);
  const int cw = ns / structure_blocks(nt, ns);
  C2<double>* cb = reinterpret_cast<C2<double>*>(buf);
  const size_t row_bytes = sizeof(C2<double>) * (size_t)ns * 2;
  const size_t col_bytes = sizeof(C2<double>) * ((size_t)nt * cw + nt);
  constexpr size_t row_max = sizeof(C2<double>) * 4096 * 2;
  constexpr size_t col_max = kColBudget + sizeof(C2<double>) * 4096;
  static int m1 = 0, m2 = 0;
  cudaError_t e;
  if ((e = smem_attr(sf_row_kernel<T>, row_max, m1)) != cudaSuccess) return e;
  if ((e = smem_attr(sf_col_kernel, col_max, m2)) != cudaSuccess) return e;
  sf_row_kernel<T><<<nt, 256, row_bytes, st>>>(ns, logns, phi, phi_lo, cb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  sf_col_kernel<<<ns / cw, 256, col_bytes, st>>>(nt, lognt, ns, cw, 1.0 / r, 1.0 / R, cb, part);
  return cudaGetLastError();
}

template cudaError_t launch_structure_sums<float>(int, int, double, double, const float*, const float*, void*,
                                                  double*, cudaStream_t);
template cudaError_t launch_structure_sums<double>(int, int, double, double, const double*, const double*, void*,
                                                   double*, cudaStream_t);

template cudaError_t launch_ch_stab<float>(int, int, double, const double*, const float*, void*, const float*,
                                           const float*, float*, int64_t, float, cudaStream_t);
template cudaError_t launch_ch_stab<double>(int, int, double, const double*, const double*, void*, const double*,
                                            const double*, double*, int64_t, double, cudaStream_t);

}  // namespace vlb
