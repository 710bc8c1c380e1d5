// 3x3 periodic convolutions on BF16 NHWC tensors for the learned surrogate: the fixed-order reduction
// of the weight and bias gradients (whose per-group partial sums come from the tcgen05 kernels of
// vlb_conv_tc.cu) and the weight flip that turns the backward-data convolution into a forward one.
// The forward and the weight gradient themselves run on the tcgen05 tensor cores (vlb_conv_tc.cu).
//
// Layouts: activations [H][W][C] (C contiguous), weights [C_out][3][3][C_in], both bf16; the torus
// is periodic in both directions, so the padding wraps.  Tap t = 3 (dy + 1) + (dx + 1) reads the
// input at (y + dy, x + dx).
//
//   forward        Y[p][co] = act( sum_{t,ci} X[p + d_t][ci] W[co][t][ci] + b[co] )
//   backward data  dX[p][ci] = mask(p, ci) * sum_{t,co} dY[p - d_t][co] W[co][t][ci]
//                  = a forward convolution of dY with W'[ci][8 - t][co] (vlb_conv3x3_flip)
//   backward wts   dW[co][t][ci] = sum_p dY[p][co] X[p + d_t][ci],  db[co] = sum_p dY[p][co]
#include <cuda_bf16.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

constexpr int CPX = 128;     // pixels per row segment
constexpr int WG_SEGS = 16;  // row segments per weight-gradient CTA (a group)

using bf16 = __nv_bfloat16;

// W'[ci][8 - t][co] = W[co][t][ci]
__global__ void flip_kernel(int cin, int cout, const bf16* w, bf16* wf) {
  const int n = cout * 9 * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i / (9 * cin), rem = i - co * 9 * cin, t = rem / cin, ci = rem - t * cin;
    wf[((size_t)ci * 9 + (8 - t)) * cout + co] = w[i];
  }
}

// dW[co][t][ci] = sum over groups of partial[group][t][co][ci] and db[co] = sum over groups of
// bpart[group][co], in a fixed order.  A 256-thread block takes 32 consecutive entries (blocks past the
// weights take the biases): warp j adds groups j, j + 8, ... (each load 128 contiguous bytes), and the
// eight warp sums are folded in warp order through shared memory.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(int groups, int cin, int cout, const float* partial,
                                                           float* dw, const float* bpart, float* db) {
  __shared__ float part[8][32];
  const int nw = 9 * cout * cin, wblocks = (nw + 31) / 32, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool bias = (int)blockIdx.x >= wblocks;
  const int n = bias ? cout : nw;
  const float* src = bias ? bpart : partial;
  const int i = (bias ? (int)blockIdx.x - wblocks : (int)blockIdx.x) * 32 + lane;
  float s = 0.0f;
  if (i < n) {
    int gp = j;
    for (; gp + 24 < groups; gp += 32) {
      const float a0 = src[(size_t)gp * n + i], a1 = src[(size_t)(gp + 8) * n + i];
      const float a2 = src[(size_t)(gp + 16) * n + i], a3 = src[(size_t)(gp + 24) * n + i];
      s += a0;
      s += a1;
      s += a2;
      s += a3;
    }
    for (; gp < groups; gp += 8) s += src[(size_t)gp * n + i];
  }
  part[j][lane] = s;
  __syncthreads();
  if (j == 0 && i < n) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    if (bias) {
      db[i] = t;
    } else {
      const int tap = i / (cout * cin), rem = i - tap * cout * cin, co = rem / cin, ci = rem - co * cin;
      dw[((size_t)co * 9 + tap) * cin + ci] = t;
    }
  }
}

bool shape_ok(int H, int W, int cin, int cout, const char** why) {
  if (H < 2 || H % 2 != 0) return *why = "H must be a positive multiple of 2", false;
  if (W < CPX || W % CPX != 0) return *why = "W must be a positive multiple of 128", false;
  if (!((cin == 16 && cout == 64) || (cin == 64 && cout == 64) || (cin == 64 && cout == 16)))
    return *why = "(c_in, c_out) must be (16, 64), (64, 64) or (64, 16)", false;
  return true;
}

}  // namespace

// the weight partials [groups][9][cout][cin], then the bias partials [groups][cout]
size_t conv_wgrad_workspace_bytes(int H, int W, int cin, int cout) {
  const int groups = (H * (W / CPX) + WG_SEGS - 1) / WG_SEGS;
  return sizeof(float) * (size_t)groups * (9 * cin * cout + cout);
}

cudaError_t conv_flip(int cin, int cout, const void* w, void* wf, cudaStream_t st) {
  flip_kernel<<<(9 * cin * cout + 255) / 256, 256, 0, st>>>(cin, cout, (const bf16*)w, (bf16*)wf);
  return cudaGetLastError();
}

cudaError_t conv_wgrad(int H, int W, int cin, int cout, const void* x, const void* dy, float* dw, float* db,
                       float* partial, cudaStream_t st) {
  // on tcgen05 (vlb_conv_tc.cu) with the bias sums folded in, then one fixed-order reduction over
  // the groups for both
  const int groups = (H * (W / CPX) + WG_SEGS - 1) / WG_SEGS;
  float* bpart = db ? partial + (size_t)groups * 9 * cin * cout : nullptr;
  cudaError_t e = conv_wgrad_tc(H, W, cin, cout, x, dy, partial, bpart, WG_SEGS, st);
  if (e != cudaSuccess) return e;
  const int blocks = (9 * cin * cout + 31) / 32 + (db ? (cout + 31) / 32 : 0);
  wgrad_reduce_kernel<<<blocks, 256, 0, st>>>(groups, cin, cout, partial, dw, bpart, db);
  return cudaGetLastError();
}

bool conv_shape_ok(int H, int W, int cin, int cout, const char** why) { return shape_ok(H, W, cin, cout, why); }

}  // namespace vlb
