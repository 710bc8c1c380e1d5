// Kernels of the learned surrogate other than the convolutions: input features, training targets,
// channel statistics, the MSE loss and its gradient, and the Adam update.  Snapshots are FP32
// [H][W][4] arrays (phi, n, u_theta, u_phi) on the device; network tensors are NHWC.
#include <cuda_bf16.h>
#include <math.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

using bf16 = __nv_bfloat16;

// Input channels: 0 phi/s_phi, 1 (n - n_mean)/s_n, 2 u_theta/s_u, 3 u_phi/s_u (norm = {n_mean, s_phi, s_n,
// s_u} on the device), then the geometry of the row (App. A): 4 J = 1 + a cos theta (sqrt(g)/(r R)),
// 5 R Gamma = sin theta / J (Eq. conn_torus), 6 sin theta, 7 cos theta, 8 1/J, 9 a = r/R; 10-15 zero.
__global__ void features_kernel(int H, int W, double a, const float* snap, const float* norm, bf16* out) {
  const int64_t n = (int64_t)H * W;
  const float n_mean = norm[0], i_phi = 1.0f / norm[1], i_n = 1.0f / norm[2], i_u = 1.0f / norm[3];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(p / W);
    float sn, cs;
    sincospif(2.0f * (float)q / (float)H, &sn, &cs);  // theta = 2 pi q / H
    const float af = (float)a, J = 1.0f + af * cs, iJ = 1.0f / J;
    const float4 s = reinterpret_cast<const float4*>(snap)[p];
    float c[16] = {s.x * i_phi, (s.y - n_mean) * i_n, s.z * i_u, s.w * i_u, J, sn * iJ, sn, cs, iJ, af,
                   0, 0, 0, 0, 0, 0};
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + p * 16);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __floats2bfloat162_rn(c[2 * k], c[2 * k + 1]);
  }
}

// target[p][c] = (after[p][c] - before[p][c]) / scale[c]
__global__ void targets_kernel(int64_t n, const float* before, const float* after, const float* scale, float* target) {
  const float4 sc = make_float4(1.0f / scale[0], 1.0f / scale[1], 1.0f / scale[2], 1.0f / scale[3]);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 b = reinterpret_cast<const float4*>(before)[p], f = reinterpret_cast<const float4*>(after)[p];
    reinterpret_cast<float4*>(target)[p] =
        make_float4((f.x - b.x) * sc.x, (f.y - b.y) * sc.y, (f.z - b.z) * sc.z, (f.w - b.w) * sc.w);
  }
}

// after[p][c] = before[p][c] + scale[c] * pred[p][c]  (pred: the first 4 of 16 FP32 channels)
__global__ void apply_kernel(int64_t n, const float* before, const float* pred, const float* scale, float* after) {
  const float4 sc = make_float4(scale[0], scale[1], scale[2], scale[3]);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 b = reinterpret_cast<const float4*>(before)[p];
    const float4 d = *reinterpret_cast<const float4*>(pred + p * 16);
    reinterpret_cast<float4*>(after)[p] =
        make_float4(b.x + sc.x * d.x, b.y + sc.y * d.y, b.z + sc.z * d.z, b.w + sc.w * d.w);
  }
}

// norm8 = {n_mean, s_phi, s_n, s_u, g0 s_phi, g1 s_n, g2 s_u, g3 s_u} from the FP64 channel sums of a
// snapshot (sums[c], sums[4 + c] = sum of x_c, x_c^2); fixed s_n / s_u when > 0.
__global__ void norm_kernel(int64_t n, const double* sums, float s_n_fixed, float s_u_fixed, float4 g, float* norm8) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool finite = true;
  for (int c = 0; c < 8; ++c) finite = finite && isfinite(sums[c]);
  const double inv = 1.0 / (double)n;
  const double mean_n = sums[1] * inv;
  double s_phi = sqrt(fmax(sums[4] * inv, 0.0));
  double s_n = s_n_fixed > 0.0f ? (double)s_n_fixed : sqrt(fmax(sums[5] * inv - mean_n * mean_n, 0.0));
  double s_u = s_u_fixed > 0.0f ? (double)s_u_fixed : sqrt(fmax(0.5 * (sums[6] + sums[7]) * inv, 0.0));
  s_phi = fmax(s_phi, 1e-12);
  s_n = fmax(s_n, 1e-12);
  s_u = fmax(s_u, 1e-12);
  const float v[8] = {(float)mean_n, (float)s_phi, (float)s_n, (float)s_u,
                      (float)(g.x * s_phi), (float)(g.y * s_n), (float)(g.z * s_u), (float)(g.w * s_u)};
  for (int c = 0; c < 8; ++c) norm8[c] = finite ? v[c] : __int_as_float(0x7fc00000);
}

constexpr int RED_BLOCKS = 256;

// Fixed-order fold of part[b * stride + k] over b < nb by one warp (lane l takes b = l, l + 32, ...,
// then a shuffle tree): the result depends only on nb, not on scheduling.
__device__ __forceinline__ double warp_sum(const double* part, int nb, int stride, int k) {
  const int lane = threadIdx.x & 31;
  double x = 0.0;
  for (int b = lane; b < nb; b += 32) x += part[b * stride + k];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// per-block FP64 sums of x[p][c] and x[p][c]^2 for c < C (C <= 16); squares in FP64 too, since a
// variance sum(x^2)/n - mean^2 of a density near 1 cancels most of its digits
__global__ void stats_kernel(int64_t n, int C, const float* x, double* part) {
  double s[16], s2[16];
  for (int c = 0; c < 16; ++c) s[c] = s2[c] = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < C; ++c) {
      const double v = x[p * C + c];
      s[c] += v;
      s2[c] += v * v;
    }
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < 2 * C; ++c) {
    double v = c < C ? s[c] : s2[c - C];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * C) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    part[blockIdx.x * 32 + threadIdx.x] = v;
  }
}

// phi of two snapshots a (prediction) and b (reference): per-block FP64 partial sums of (a - b)^2 and
// b^2 into part[block * 32 + {0, 1}], and the maxima of |a - b| and |b| as non-negative float bit
// patterns (integer max: exact, independent of the order of the atomics) into max2, zeroed before.
// A non-finite value in a or b makes the difference +inf.
__global__ void compare_kernel(int64_t n, const float* a, const float* b, double* part, unsigned* max2) {
  float d = 0.0f, m = 0.0f;
  double s2 = 0.0, r2 = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 x = reinterpret_cast<const float4*>(a)[p], y = reinterpret_cast<const float4*>(b)[p];
    const bool ok = isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w) && isfinite(y.x) &&
                    isfinite(y.y) && isfinite(y.z) && isfinite(y.w);
    const double e = (double)x.x - (double)y.x;
    d = ok ? fmaxf(d, fabsf(x.x - y.x)) : INFINITY;
    m = ok ? fmaxf(m, fabsf(y.x)) : m;
    s2 += ok ? e * e : (double)INFINITY;
    r2 += ok ? (double)y.x * y.x : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(max2, __float_as_uint(d));
    atomicMax(max2 + 1, __float_as_uint(m));
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = s2;
  red[1][threadIdx.x] = r2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x * 32] = red[0][0];
    part[blockIdx.x * 32 + 1] = red[1][0];
  }
}

// out4 = {max |a - b|, max |b|, sum (a - b)^2, sum b^2} from compare_kernel's results, in a fixed order
// (one warp per sum, blockDim = 64).
__global__ void compare_final_kernel(int nb, const double* part, const unsigned* max2, double* out4) {
  const int k = threadIdx.x >> 5;
  const double v = warp_sum(part, nb, 32, k);
  if ((threadIdx.x & 31) == 0) out4[2 + k] = v;
  if (threadIdx.x == 0) {
    out4[0] = (double)__uint_as_float(max2[0]);
    out4[1] = (double)__uint_as_float(max2[1]);
  }
}

__global__ void stats_final_kernel(int nb, int C, const double* part, double* out) {
  const int c = threadIdx.x >> 5;
  const double v = warp_sum(part, nb, 32, c);
  if ((threadIdx.x & 31) == 0 && c < 2 * C) out[c] = v;
}

// loss partials of (pred[p][c] - target[p][c])^2 over c < 4; grad[p][c] = 2 (pred - target) / (4 n)
__global__ void mse_kernel(int64_t n, const float* pred, const float* target, bf16* grad, double* part) {
  double s = 0.0;
  const float inv = 2.0f / (4.0f * (float)n);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float4 y = *reinterpret_cast<const float4*>(pred + p * 16);
    const float4 t = reinterpret_cast<const float4*>(target)[p];
    const float d0 = y.x - t.x, d1 = y.y - t.y, d2 = y.z - t.z, d3 = y.w - t.w;
    s += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2 + (double)d3 * d3;
    if (grad) {
      __nv_bfloat162* g = reinterpret_cast<__nv_bfloat162*>(grad + p * 16);
      g[0] = __floats2bfloat162_rn(inv * d0, inv * d1);
      g[1] = __floats2bfloat162_rn(inv * d2, inv * d3);
#pragma unroll
      for (int k = 2; k < 8; ++k) g[k] = __floats2bfloat162_rn(0.0f, 0.0f);
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sum_final_kernel(int nb, const double* part, double scale, double* out) {
  const double v = warp_sum(part, nb, 1, 0);
  if (threadIdx.x == 0) *out = v * scale;
}

// Adam (Kingma & Ba 2015) on FP32 master parameters; optionally refreshes a BF16 copy.
__global__ void adam_kernel(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2, bf16* pb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float pi = p[i] - upd;
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(int64_t n, const float* x, bf16* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

}  // namespace

cudaError_t sur_features(int H, int W, double a, const float* snap, const float* norm4, void* out, cudaStream_t st) {
  features_kernel<<<blocks_for((int64_t)H * W), 256, 0, st>>>(H, W, a, snap, norm4, (bf16*)out);
  return cudaGetLastError();
}

cudaError_t sur_targets(int64_t n, const float* before, const float* after, const float* scale4, float* target,
                        cudaStream_t st) {
  targets_kernel<<<blocks_for(n), 256, 0, st>>>(n, before, after, scale4, target);
  return cudaGetLastError();
}

cudaError_t sur_apply(int64_t n, const float* before, const float* pred, const float* scale4, float* after,
                      cudaStream_t st) {
  apply_kernel<<<blocks_for(n), 256, 0, st>>>(n, before, pred, scale4, after);
  return cudaGetLastError();
}

cudaError_t sur_compare(int64_t n, const float* a, const float* b, double* part, double* out4, cudaStream_t st) {
  // the two maxima live in the last two slots of the partials (RED_BLOCKS * 32 doubles, 2 used per block)
  unsigned* max2 = reinterpret_cast<unsigned*>(part + RED_BLOCKS * 32 - 1);
  cudaError_t e = cudaMemsetAsync(max2, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  compare_kernel<<<RED_BLOCKS, 256, 0, st>>>(n, a, b, part, max2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  compare_final_kernel<<<1, 64, 0, st>>>(RED_BLOCKS, part, max2, out4);
  return cudaGetLastError();
}

cudaError_t sur_stats(int64_t n, int C, const float* x, double* part, double* out, cudaStream_t st) {
  stats_kernel<<<RED_BLOCKS, 256, 0, st>>>(n, C, x, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stats_final_kernel<<<1, 64 * C, 0, st>>>(RED_BLOCKS, C, part, out);
  return cudaGetLastError();
}

cudaError_t sur_norm(int64_t n, const float* snap, float s_n, float s_u, const float* g4, double* part, double* sums,
                     float* norm8, cudaStream_t st) {
  cudaError_t e = sur_stats(n, 4, snap, part, sums, st);
  if (e != cudaSuccess) return e;
  norm_kernel<<<1, 32, 0, st>>>(n, sums, s_n, s_u, make_float4(g4[0], g4[1], g4[2], g4[3]), norm8);
  return cudaGetLastError();
}

cudaError_t sur_mse(int64_t n, const float* pred, const float* target, void* grad, double* part, double* loss,
                    cudaStream_t st) {
  mse_kernel<<<RED_BLOCKS, 256, 0, st>>>(n, pred, target, (bf16*)grad, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_final_kernel<<<1, 32, 0, st>>>(RED_BLOCKS, part, 1.0 / (4.0 * (double)n), loss);
  return cudaGetLastError();
}

cudaError_t sur_adam(int64_t n, float* p, const float* g, float* m, float* v, int64_t t, float lr, float b1, float b2,
                     float eps, void* pb, cudaStream_t st) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  adam_kernel<<<blocks_for(n), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2, (bf16*)pb);
  return cudaGetLastError();
}

cudaError_t sur_to_bf16(int64_t n, const float* x, void* y, cudaStream_t st) {
  to_bf16_kernel<<<blocks_for(n), 256, 0, st>>>(n, x, (bf16*)y);
  return cudaGetLastError();
}

size_t sur_reduce_doubles() { return RED_BLOCKS * 32; }

}  // namespace vlb
