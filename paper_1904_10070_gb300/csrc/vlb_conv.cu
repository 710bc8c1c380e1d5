// 3x3 periodic convolutions on BF16 NHWC tensors for the learned surrogate: the weight gradient
// (mma.sync m16n8k16 tensor-core tiles, FP32 accumulation), the bias gradient and the weight flip
// that turns the backward-data convolution into a forward one.  The forward itself runs on the
// tcgen05 tensor cores (vlb_conv_tc.cu).
//
// Layouts: activations [H][W][C] (C contiguous), weights [C_out][3][3][C_in], both bf16; the torus
// is periodic in both directions, so the padding wraps.  Tap t = 3 (dy + 1) + (dx + 1) reads the
// input at (y + dy, x + dx).
//
//   forward        Y[p][co] = act( sum_{t,ci} X[p + d_t][ci] W[co][t][ci] + b[co] )
//   backward data  dX[p][ci] = mask(p, ci) * sum_{t,co} dY[p - d_t][co] W[co][t][ci]
//                  = a forward convolution of dY with W'[ci][8 - t][co] (vlb_conv3x3_flip)
//   backward wts   dW[co][t][ci] = sum_p dY[p][co] X[p + d_t][ci],  db[co] = sum_p dY[p][co]
//
// Weight gradient: a CTA (4 warps) owns one tap and a group of row segments; per segment it stages
// the shifted input row and dY in shared memory and accumulates dY^T X_t with both operands loaded
// by ldmatrix.trans; per-group partial sums are reduced in a fixed order by a second kernel.
#include <cuda_bf16.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

constexpr int CPX = 128;  // pixels per CTA (one row segment)
constexpr int NWARP = 4;
constexpr int NTHR = NWARP * 32;
constexpr int WG_SEGS = 16;  // row segments per weight-gradient CTA

using bf16 = __nv_bfloat16;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src));
}

__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

// W'[ci][8 - t][co] = W[co][t][ci]
__global__ void flip_kernel(int cin, int cout, const bf16* w, bf16* wf) {
  const int n = cout * 9 * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i / (9 * cin), rem = i - co * 9 * cin, t = rem / cin, ci = rem - t * cin;
    wf[((size_t)ci * 9 + (8 - t)) * cout + co] = w[i];
  }
}

template <int CIN, int COUT>
constexpr size_t wg_smem() {
  return sizeof(bf16) * CPX * ((CIN + 8) + (COUT + 8));
}

// Partial weight gradients of tap blockIdx.y over the row segments of group blockIdx.x.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR) conv_wgrad_kernel(int H, int W, const bf16* __restrict__ x,
                                                          const bf16* __restrict__ dy, float* partial) {
  constexpr int XS = CIN + 8, DS = COUT + 8, MT = COUT / 16, NT8 = CIN / 8;
  // warps split the (m-tile, n-tile pair) grid: MT m-tiles x NT8/2 n-pairs
  constexpr int WORK = MT * (NT8 / 2);
  constexpr int PER = (WORK + NWARP - 1) / NWARP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16* xs = reinterpret_cast<bf16*>(smem_raw);
  bf16* ds = xs + CPX * XS;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tap = blockIdx.y, ddy = tap / 3 - 1, ddx = tap % 3 - 1;
  const int segs_row = W / CPX, nseg = H * segs_row;
  float acc[PER][2][4];
#pragma unroll
  for (int u = 0; u < PER; ++u)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[u][h][e] = 0.0f;
  const int j = lane / 8, i8 = lane % 8;
#pragma unroll 1
  for (int sg = blockIdx.x * WG_SEGS; sg < (blockIdx.x + 1) * WG_SEGS && sg < nseg; ++sg) {
    const int row = sg / segs_row, x0 = (sg % segs_row) * CPX;
    int gy = row + ddy;
    gy += gy < 0 ? H : (gy >= H ? -H : 0);
    __syncthreads();  // the previous segment's tiles are consumed
    for (int idx = tid; idx < CPX * (CIN / 8); idx += NTHR) {
      const int pc = idx / (CIN / 8), ch = idx - pc * (CIN / 8);
      int gx = x0 + pc + ddx;
      gx += gx < 0 ? W : (gx >= W ? -W : 0);
      cp16(xs + pc * XS + ch * 8, x + ((size_t)gy * W + gx) * CIN + ch * 8);
    }
    for (int idx = tid; idx < CPX * (COUT / 8); idx += NTHR) {
      const int pc = idx / (COUT / 8), ch = idx - pc * (COUT / 8);
      cp16(ds + pc * DS + ch * 8, dy + ((size_t)row * W + x0 + pc) * COUT + ch * 8);
    }
    cp_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int kb = 0; kb < CPX; kb += 16) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int wi = warp + NWARP * u;
        if (wi < WORK) {
          const int mt = wi % MT, np = wi / MT;
          uint32_t a[4], b[4];
          // A = dY^T (m = co, k = pixel) from ds[pixel][co]: blocks (k 0-7|8-15, m 0-7|8-15)
          ldsm4t(a, ds + (kb + i8 + 8 * (j / 2)) * DS + mt * 16 + 8 * (j % 2));
          // B = X_t (k = pixel, n = ci) from xs[pixel][ci]: blocks (k 0-7|8-15, n 0-7|8-15)
          ldsm4t(b, xs + (kb + i8 + 8 * (j % 2)) * XS + np * 16 + 8 * (j / 2));
          mma16816(acc[u][0], a, b[0], b[1]);
          mma16816(acc[u][1], a, b[2], b[3]);
        }
      }
    }
  }
  // partial[group][tap][co][ci]
  const int g = lane / 4, t4 = lane % 4;
  float* out = partial + ((size_t)blockIdx.x * 9 + tap) * COUT * CIN;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int wi = warp + NWARP * u;
    if (wi < WORK) {
      const int mt = wi % MT, np = wi / MT;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int co = mt * 16 + g + 8 * r, ci = np * 16 + 8 * h + 2 * t4;
          out[co * CIN + ci] = acc[u][h][2 * r];
          out[co * CIN + ci + 1] = acc[u][h][2 * r + 1];
        }
    }
  }
}

// dW[co][t][ci] = sum over groups of partial[group][t][co][ci] in a fixed order. A 256-thread block
// takes 32 consecutive weights: warp j adds groups j, j + 8, ... (each load 128 contiguous bytes), and
// the eight warp sums are folded in warp order through shared memory.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(int groups, int cin, int cout, const float* partial,
                                                           float* dw) {
  __shared__ float part[8][32];
  const int n = 9 * cout * cin, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.0f;
  if (i < n) {
    int gp = j;
    for (; gp + 24 < groups; gp += 32) {
      const float a0 = partial[(size_t)gp * n + i], a1 = partial[(size_t)(gp + 8) * n + i];
      const float a2 = partial[(size_t)(gp + 16) * n + i], a3 = partial[(size_t)(gp + 24) * n + i];
      s += a0;
      s += a1;
      s += a2;
      s += a3;
    }
    for (; gp < groups; gp += 8) s += partial[(size_t)gp * n + i];
  }
  part[j][lane] = s;
  __syncthreads();
  if (j == 0 && i < n) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    const int tap = i / (cout * cin), rem = i - tap * cout * cin, co = rem / cin, ci = rem - co * cin;
    dw[((size_t)co * 9 + tap) * cin + ci] = t;
  }
}

// db[co] = sum_p dY[p][co] in two passes with a fixed order.  Pass 1: BG_BLOCKS blocks; thread t
// takes the 8-channel chunk t % (cout / 8) of every (256 / (cout / 8))-th pixel of its block's share
// (16-byte loads, whole 128-byte rows per 8 or 2 lanes); the pixel lanes of a block are then summed
// in shared memory.
constexpr int BG_BLOCKS = 608;  // 4 per SM of GB300; a multiple of 32 for the final warp fold

__global__ void __launch_bounds__(256) bias_partial_kernel(int npix, int cout, const bf16* dy, float* part) {
  __shared__ float red[256 * 8];
  const int chunks = cout / 8, lanes = blockDim.x / chunks;
  const int ch = threadIdx.x % chunks, pl = threadIdx.x / chunks;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  auto add = [&](const uint4& v) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      s[2 * i] += f.x;
      s[2 * i + 1] += f.y;
    }
  };
  const int step = gridDim.x * lanes;
  int p = blockIdx.x * lanes + pl;
  for (; p + 3 * step < npix; p += 4 * step) {  // four loads in flight, added in pixel order
    const uint4 v0 = reinterpret_cast<const uint4*>(dy + (size_t)p * cout)[ch];
    const uint4 v1 = reinterpret_cast<const uint4*>(dy + (size_t)(p + step) * cout)[ch];
    const uint4 v2 = reinterpret_cast<const uint4*>(dy + (size_t)(p + 2 * step) * cout)[ch];
    const uint4 v3 = reinterpret_cast<const uint4*>(dy + (size_t)(p + 3 * step) * cout)[ch];
    add(v0);
    add(v1);
    add(v2);
    add(v3);
  }
  for (; p < npix; p += step) add(reinterpret_cast<const uint4*>(dy + (size_t)p * cout)[ch]);
#pragma unroll
  for (int i = 0; i < 8; ++i) red[pl * cout + 8 * ch + i] = s[i];
  __syncthreads();
  if (threadIdx.x < cout) {
    float t = 0.0f;
    for (int l = 0; l < lanes; ++l) t += red[l * cout + threadIdx.x];
    part[blockIdx.x * cout + threadIdx.x] = t;
  }
}

// Pass 2: db[co] = sum over the blocks' partials in a fixed order, one warp per channel (lane l adds
// blocks l, l + 32, ... in order, then a shuffle tree); all loads of a channel are in flight together.
__global__ void bias_final_kernel(int cout, const float* part, float* db) {
  const int co = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (co >= cout) return;
  float v[BG_BLOCKS / 32];
#pragma unroll
  for (int i = 0; i < BG_BLOCKS / 32; ++i) v[i] = part[(lane + 32 * i) * cout + co];
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < BG_BLOCKS / 32; ++i) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) db[co] = s;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CIN, int COUT>
cudaError_t wg_launch(int H, int W, const void* x, const void* dy, float* partial, float* dw, cudaStream_t st) {
  constexpr size_t S = wg_smem<CIN, COUT>();
  cudaError_t e = allow_smem(conv_wgrad_kernel<CIN, COUT>, S);
  if (e != cudaSuccess) return e;
  const int groups = (H * (W / CPX) + WG_SEGS - 1) / WG_SEGS;
  conv_wgrad_kernel<CIN, COUT><<<dim3(groups, 9), NTHR, S, st>>>(H, W, (const bf16*)x, (const bf16*)dy, partial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wgrad_reduce_kernel<<<(9 * CIN * COUT + 31) / 32, 256, 0, st>>>(groups, CIN, COUT, partial, dw);
  return cudaGetLastError();
}

bool shape_ok(int H, int W, int cin, int cout, const char** why) {
  if (H < 2 || H % 2 != 0) return *why = "H must be a positive multiple of 2", false;
  if (W < CPX || W % CPX != 0) return *why = "W must be a positive multiple of 128", false;
  if (!((cin == 16 && cout == 64) || (cin == 64 && cout == 64) || (cin == 64 && cout == 16)))
    return *why = "(c_in, c_out) must be (16, 64), (64, 64) or (64, 16)", false;
  return true;
}

}  // namespace

size_t conv_wgrad_workspace_bytes(int H, int W, int cin, int cout) {
  const int groups = (H * (W / CPX) + WG_SEGS - 1) / WG_SEGS;
  const size_t wg = (size_t)groups * 9 * cin * cout, bg = (size_t)BG_BLOCKS * cout;
  return sizeof(float) * (wg > bg ? wg : bg);
}

cudaError_t conv_flip(int cin, int cout, const void* w, void* wf, cudaStream_t st) {
  flip_kernel<<<(9 * cin * cout + 255) / 256, 256, 0, st>>>(cin, cout, (const bf16*)w, (bf16*)wf);
  return cudaGetLastError();
}

cudaError_t conv_wgrad(int H, int W, int cin, int cout, const void* x, const void* dy, float* dw, float* db,
                       float* partial, cudaStream_t st) {
  cudaError_t e;
  if (cin == 16)
    e = wg_launch<16, 64>(H, W, x, dy, partial, dw, st);
  else if (cout == 64) {  // on tcgen05 (vlb_conv_tc.cu), then the same fixed-order reduction
    e = conv_wgrad_tc64(H, W, x, dy, partial, WG_SEGS, st);
    if (e == cudaSuccess) {
      const int groups = (H * (W / CPX) + WG_SEGS - 1) / WG_SEGS;
      wgrad_reduce_kernel<<<(9 * 64 * 64 + 31) / 32, 256, 0, st>>>(groups, 64, 64, partial, dw);
      e = cudaGetLastError();
    }
  }
  else
    e = wg_launch<64, 16>(H, W, x, dy, partial, dw, st);
  if (e != cudaSuccess || !db) return e;
  // the weight partials are consumed by now: their workspace (sized for both, see
  // conv_wgrad_workspace_bytes) holds the BG_BLOCKS x cout bias partials
  bias_partial_kernel<<<BG_BLOCKS, 256, 0, st>>>(H * W, cout, (const bf16*)dy, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bias_final_kernel<<<(cout + 7) / 8, 256, 0, st>>>(cout, partial, db);
  return cudaGetLastError();
}

bool conv_shape_ok(int H, int W, int cin, int cout, const char** why) { return shape_ok(H, W, cin, cout, why); }

}  // namespace vlb
