// 3x3 periodic convolution forward on the 5th-generation tensor cores (tcgen05.mma, BF16 x BF16 ->
// FP32 accumulators in tensor memory), for the learned surrogate.  Y[p][co] = act(sum_{t,ci}
// X[p + d_t][ci] W[co][t][ci] + b[co]) on NHWC bf16 tensors, periodic in both directions, with the
// optional bias, ReLU, mask (outputs where mask <= 0 are zeroed) and bf16 / f32 outputs.  The
// backward-data convolution is this kernel on flipped weights.
//
// Implicit GEMM.  A work item is one output row segment of 128 pixels: D[m][n] (m = pixel, n =
// output channel, M = 128, N = C_out) accumulates over K = 9 taps x C_in,
//   A_t[m][k] = X[pixel m shifted by tap t][k],  B_t[n][k] = W[n][t][k],  D = sum_t A_t B_t^T.
// The input patch (3 rows x 130 pixels) is staged once per item; the A matrix of tap (dy, dx) is the
// same buffer with its descriptor start shifted by whole pixel rows, so a shifted window needs no
// copy.  The weights are staged once per CTA (the CTA is persistent over work items).
//
// One 192-thread CTA per SM with six warps in fixed roles: warps 0-3 run the epilogue (warp w reads
// tensor-memory lanes 32w .. 32w + 31, i.e. those pixels: bias, ReLU, mask, bf16/f32 stores), warp 4
// allocates tensor memory and one of its threads issues the MMAs, warp 5 issues the copies (the
// weights once, then one patch per item, three deep, and the periodic fix-ups of edge items).  Two
// accumulators let the epilogue of one item overlap the MMAs of the next.  Hand-offs are mbarriers
// and every wait is bounded.
#include <cuda_bf16.h>
#include <string.h>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

using bf16 = __nv_bfloat16;

constexpr int TPX = 128;                 // pixels per work item (the MMA's M)
constexpr int TPR = 3, TPW = TPX + 2;    // patch rows, patch columns
// Warp roles: 0-3 epilogue (warp w reads tensor-memory lanes 32w .. 32w + 31), 4 MMA issue and
// tensor-memory allocation, 5 issues the tensor-map copies (waiting only for a free buffer), 6
// completes them (waits for a copy to land, applies the periodic fix-ups of edge items and hands the
// buffer to the MMA warp), so that the latency of the fix-ups never delays the next copy.
constexpr int TTHR = 224;
constexpr int MMA_WARP = 4, LOAD_WARP = 5, FIX_WARP = 6;

template <int CIN, int COUT>
struct TcLay {
  // C_in = 64: 128-byte pixel rows in the 128-byte-swizzled K-major layout (fast row copies);
  // C_in = 16: the no-swizzle chunk-major layout [16-byte chunk][patch row][patch column]
  static constexpr bool SW = CIN == 64;
  static constexpr int CH = CIN / 8;                         // 16-byte channel chunks per pixel
  static constexpr int NBUF = 3;                             // patch buffers
  static constexpr int WTS = 9 * CH * COUT * 16;             // weight bytes
  static constexpr int PATCH_RAW = CH * TPR * TPW * 16;      // patch bytes
  static constexpr int PATCH = SW ? (PATCH_RAW + 1023) / 1024 * 1024 : (PATCH_RAW + 127) / 128 * 128;
  static constexpr int W_OFF = 0, P_OFF = WTS, BAR_OFF = WTS + NBUF * PATCH;
  static constexpr int NBAR = 3 * NBUF + 5;                  // tma, pfull, pempty (x NBUF), afull, aempty (x 2), w
  static constexpr int TSLOT_OFF = BAR_OFF + 8 * NBAR;       // tensor-memory address
  static constexpr int BIAS_OFF = TSLOT_OFF + 16;
  static constexpr int BYTES = BIAS_OFF + 4 * COUT;
  static constexpr int ACC = COUT;                           // accumulator columns of one work item
  static constexpr int COLS = 2 * ACC <= 32 ? 32 : (2 * ACC <= 64 ? 64 : (2 * ACC <= 128 ? 128 : 256));
  static constexpr uint32_t LBO_A = TPR * TPW * 16;          // next channel chunk of the patch
  static constexpr uint32_t LBO_B = COUT * 16;               // next channel chunk of a tap's weights
  static_assert(SW ? (WTS % 1024 == 0 && PATCH % 1024 == 0) : (WTS % 128 == 0 && PATCH % 128 == 0),
                "operand buffers stay aligned to the swizzle atom (1024 bytes) or the core matrix (128 bytes)");
  static_assert(BYTES <= 232448, "fits the opt-in shared memory of one CTA");
  static_assert(COUT % 16 == 0 && COUT <= 256 && CIN % 16 == 0, "MMA shape M = 128, N = C_out, K = 16");
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch: the convolutions are launched so that a kernel's CTAs may start (tensor
// memory, mbarriers) while the previous kernel of the stream drains; every global access comes after
// the wait, which returns once the previous kernel has completed and its memory is visible.  The
// trigger lets the next convolution start the same way.
__device__ __forceinline__ void pdl_wait_and_trigger() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(su32(dst)), "l"(src));
}
// copies written by this thread become visible to the tensor core (the async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
// the box at (0, x, y) of a 3-D tensor map into shared memory (1024-byte aligned), completing on bar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];\n" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(0), "r"(x), "r"(y)
      : "memory");
}
// the box at (0, x, y, 0) of a 4-D tensor map into shared memory (128-byte aligned), completing on bar
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
      "%6}], [%2];\n" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(0), "r"(x), "r"(y), "r"(0)
      : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {  // bounded: a commit that never arrives cannot hang the GPU
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (K-direction core-matrix) and stride (M/N-direction
// core-matrix) byte offsets, each encoded >> 4 in 14 bits; bits 46-47 = 1 (tcgen05 descriptor);
// base offset 0; layout 0 = no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// 128-byte swizzle (layout 2 in bits 61-63): 8-row groups of 128-byte rows 1024 bytes apart, the
// 16-byte chunk c of row r stored at chunk c ^ (r % 8) counted from the 1024-byte-aligned atom.  The
// tensor core applies the swizzle to absolute shared-memory address bits, as the tensor-map copy
// does, so a start address inside an atom (a window shifted by whole pixel rows, or a K step of 32
// bytes) needs no base offset (bits 49-51 stay 0; measured on GB300).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int N>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TPX >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's lane (asynchronous: tmem_wait_ld before use)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Shared-memory offset of 16-byte chunk c of patch pixel (pr, pc) in a patch buffer.
template <int CIN>
__device__ __forceinline__ int patch_off(int c, int pr, int pc) {
  if constexpr (CIN == 64) {
    const int j = pr * TPW + pc;  // 128-byte pixel row; buffers are 1024-byte aligned
    return j * 128 + ((c ^ (j & 7)) << 4);
  } else {
    return ((c * TPR + pr) * TPW + pc) * 16;
  }
}

// Periodic fix-up of an edge item's patch after its tensor-map copy (which zero-fills out-of-range
// positions): out-of-range patch rows get whole wrapped rows, out-of-range columns the wrapped pixel.
// Run by the 32 lanes of the load warp; returns whether anything was copied.
template <int CIN>
__device__ __forceinline__ bool fix_patch(unsigned char* dst, const bf16* x, int H, int W, int row, int x0, int lane) {
  constexpr int CH = CIN / 8;
  const bool top = row == 0, bottom = row + 1 == H, left = x0 == 0, right = x0 + TPX == W;
  if (!(top || bottom || left || right)) return false;
  for (int pr = 0; pr < TPR; ++pr) {
    const int yy = row + pr - 1;
    const int gy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
    if (gy != yy) {  // a whole wrapped row
      for (int i = lane; i < TPW * CH; i += 32) {
        const int c = i % CH, pc = i / CH, xx = x0 + pc - 1;
        const int gx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
        cp16(dst + patch_off<CIN>(c, pr, pc), x + ((size_t)gy * W + gx) * CIN + c * 8);
      }
    } else {  // at most the two edge pixels
      for (int i = lane; i < 2 * CH; i += 32) {
        const int c = i % CH, side = i / CH;
        if ((side == 0 && left) || (side == 1 && right)) {
          const int pc = side == 0 ? 0 : TPW - 1, gx = side == 0 ? W - 1 : 0;
          cp16(dst + patch_off<CIN>(c, pr, pc), x + ((size_t)gy * W + gx) * CIN + c * 8);
        }
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  return true;
}

// Epilogue of work item `item` (row item % H, segment item / H: consecutive items of a CTA fall in
// different segments) from the accumulator at column `col0`: thread (warp, lane) owns pixel
// x0 + 32 warp + lane of the item's row; all C_out columns are read before one wait.
template <int COUT>
__device__ __forceinline__ void epilogue(uint32_t tmem, uint32_t col0, int H, int W, int item, int warp, int lane,
                                         const float* sbias, const bf16* mask, int relu, bf16* y, float* yf) {
  const int row = item % H, x0 = (item / H) * TPX;
  const size_t p = (size_t)row * W + x0 + 32 * warp + lane;
  uint32_t raw[COUT];
#pragma unroll
  for (int j = 0; j < COUT / 16; ++j)
    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + col0 + (uint32_t)(16 * j), raw + 16 * j);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < COUT / 16; ++j) {
    float v[16];
    const int co = 16 * j;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(raw[co + i]) + sbias[co + i];
    if (relu) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
    }
    if (mask) {
      const uint4* mp = reinterpret_cast<const uint4*>(mask + p * COUT + co);
      const uint4 m0 = mp[0], m1 = mp[1];
      const __nv_bfloat162* mh = reinterpret_cast<const __nv_bfloat162*>(&m0);
      const __nv_bfloat162* mh1 = reinterpret_cast<const __nv_bfloat162*>(&m1);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!(__low2float(mh[i]) > 0.0f)) v[2 * i] = 0.0f;
        if (!(__high2float(mh[i]) > 0.0f)) v[2 * i + 1] = 0.0f;
        if (!(__low2float(mh1[i]) > 0.0f)) v[8 + 2 * i] = 0.0f;
        if (!(__high2float(mh1[i]) > 0.0f)) v[8 + 2 * i + 1] = 0.0f;
      }
    }
    if (y) {
      uint4 o[2];
      __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
      for (int i = 0; i < 8; ++i) oh[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      uint4* yp = reinterpret_cast<uint4*>(y + p * COUT + co);
      yp[0] = o[0];
      yp[1] = o[1];
    }
    if (yf) {
      float4* fp = reinterpret_cast<float4*>(yf + p * COUT + co);
#pragma unroll
      for (int i = 0; i < 4; ++i) fp[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
  }
}

// Persistent over work items item_k = blockIdx.x + k gridDim.x with warp-specialised roles: patch
// buffer k % 3 and accumulator k % 2 serve item k.  The load warp copies patch k while the MMA warp
// works on earlier items and the epilogue warps drain the accumulator of item k - 2.  Hand-offs are
// mbarriers: tma[b] (copy landed), pfull[b] (patch ready, fix-ups included), pempty[b] (its MMAs are
// done), afull[a] (accumulator ready), aempty[a] (accumulator read, 4 arrivals), w (weights landed).
template <int CIN, int COUT>
__global__ void __launch_bounds__(TTHR, 1)
    conv_fwd_tc_kernel(int H, int W, const bf16* __restrict__ x, const bf16* __restrict__ w,
                       const float* __restrict__ bias, const bf16* __restrict__ mask, int relu, bf16* y, float* yf,
                       int* err, const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap) {
  using L = TcLay<CIN, COUT>;
  constexpr int NB = L::NBUF;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::BAR_OFF);
  uint64_t *tma = bars, *pfull = bars + NB, *pempty = bars + 2 * NB, *afull = bars + 3 * NB,
           *aempty = bars + 3 * NB + 2, *wbar = bars + 3 * NB + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::TSLOT_OFF);
  float* sbias = reinterpret_cast<float*>(sm + L::BIAS_OFF);
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                 "r"(L::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < NB; ++b) {
      mbar_init(tma + b, 1);
      mbar_init(pfull + b, 1);
      mbar_init(pempty + b, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(afull + a, 1);
      mbar_init(aempty + a, 4);
    }
    mbar_init(wbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  pdl_wait_and_trigger();
  for (int i = tid; i < COUT; i += TTHR) sbias[i] = bias ? bias[i] : 0.0f;
  if constexpr (!L::SW) {
    // 16-channel weights (18 KB), chunk-major [t][c][co]: per-thread copies before the roles split
    for (int i = tid; i < COUT * 9 * L::CH; i += TTHR) {
      const int c = i % L::CH, t = (i / L::CH) % 9, co = i / (9 * L::CH);
      cp16(sm + L::W_OFF + ((t * L::CH + c) * COUT + co) * 16, w + ((size_t)co * 9 + t) * CIN + c * 8);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    fence_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int segs = W / TPX, nitems = H * segs;
  const int nmine = blockIdx.x < nitems ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool ok = true;
  if (warp == LOAD_WARP) {
    if constexpr (L::SW) {
      // 64-channel weights (72 KB): nine tensor-map copies, one per tap, of the box (64 c_in, 1 tap,
      // C_out), each landing as C_out rows of 128 bytes with the 128-byte swizzle at [tap][c_out]; they
      // overlap the first patch copies
      if (lane == 0) {
        mbar_expect_tx(wbar, L::WTS);
        for (int t = 0; t < 9; ++t)
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
              "%5}], [%2];\n" ::"r"(su32(sm + L::W_OFF + t * COUT * 128)),
              "l"(reinterpret_cast<uint64_t>(&wmap)), "r"(su32(wbar)), "r"(0), "r"(t), "r"(0)
              : "memory");
      }
    }
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NB, use = k / NB, item = blockIdx.x + k * gridDim.x;
      const int row = item % H, x0 = (item / H) * TPX;
      if (k >= NB) ok = mbar_wait(pempty + b, (use - 1) & 1);  // the MMAs of item k - NB read it
      if (!ok) break;
      if (lane == 0) {
        unsigned char* dst = sm + L::P_OFF + b * L::PATCH;
        mbar_expect_tx(tma + b, L::PATCH_RAW);
        if constexpr (L::SW)
          tma_load_3d(dst, &xmap, tma + b, x0 - 1, row - 1);
        else
          tma_load_4d(dst, &xmap, tma + b, x0 - 1, row - 1);
      }
      __syncwarp();
    }
    if (L::SW && nmine == 0 && lane == 0) mbar_wait(wbar, 0);  // the weight copy lands before the CTA exits
  } else if (warp == FIX_WARP) {
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NB, item = blockIdx.x + k * gridDim.x;
      const int row = item % H, x0 = (item / H) * TPX;
      unsigned char* dst = sm + L::P_OFF + b * L::PATCH;
      const bool left = x0 == 0, right = x0 + TPX == W;
      const bool slow = row == 0 || row + 1 == H || (left && right);  // wrapped rows, or both sides wrap
      // column wrap of an edge segment: the TPR x CH 16-byte chunks of the wrapped pixel, loaded into
      // registers before the copy lands (their latency overlaps the copy), stored after it
      uint4 v = make_uint4(0, 0, 0, 0);
      const bool col_fix = (left || right) && !slow && lane < TPR * L::CH;
      const int pr = lane / L::CH, c = lane % L::CH, pc = left ? 0 : TPW - 1;
      if (col_fix) {
        const int gx = left ? W - 1 : 0, gy = row + pr - 1;
        v = *reinterpret_cast<const uint4*>(x + ((size_t)gy * W + gx) * CIN + c * 8);
      }
      ok = mbar_wait(tma + b, (k / NB) & 1);
      if (!ok) break;
      if (slow) {  // the first or last row of the grid, or a one-segment-wide grid (rare)
        if (fix_patch<CIN>(dst, x, H, W, row, x0, lane)) fence_async_smem();
      } else if (left || right) {
        if (col_fix) *reinterpret_cast<uint4*>(dst + patch_off<CIN>(c, pr, pc)) = v;
        fence_async_smem();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(pfull + b);
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      constexpr uint32_t ID = idesc<COUT>();
      if (L::SW && nmine > 0) ok = mbar_wait(wbar, 0);
      const uint64_t bd0 = sdesc(su32(sm + L::W_OFF), L::LBO_B, 128);
      for (int k = 0; k < nmine && ok; ++k) {
        const int b = k % NB, a = k & 1;
        ok = mbar_wait(pfull + b, (k / NB) & 1);
        if (ok && k >= 2) ok = mbar_wait(aempty + a, ((k - 2) >> 1) & 1);  // epilogue of item k - 2
        if (!ok) break;
        tc_fence_after();
        // descriptors differ only in the start address (low 14 bits, 16-byte units): constant offsets
        const uint32_t pb = su32(sm + L::P_OFF + b * L::PATCH), wb = su32(sm + L::W_OFF);
        const uint64_t ad0 = sdesc(pb, L::LBO_A, 128);
        const uint32_t acc = tmem + (uint32_t)(a * L::ACC);
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
          for (int s2 = 0; s2 < CIN / 16; ++s2) {
            uint64_t ad, bdd;
            if constexpr (L::SW) {  // rows (t / 3) * TPW + t % 3 + m; K step s2 is 32 bytes into the row
              ad = sdesc_sw128(pb + (uint32_t)(((t / 3) * TPW + t % 3) * 128 + 32 * s2));
              bdd = sdesc_sw128(wb + (uint32_t)(t * COUT * 128 + 32 * s2));
            } else {
              ad = ad0 + (uint32_t)(((2 * s2) * TPR + t / 3) * TPW + t % 3);
              bdd = bd0 + (uint32_t)((t * L::CH + 2 * s2) * COUT);
            }
            umma(acc, ad, bdd, ID, (t | s2) != 0);
          }
        umma_commit(pempty + b);
        umma_commit(afull + a);
      }
    }
    __syncwarp();
  } else {  // epilogue warps 0-3
    for (int k = 0; k < nmine && ok; ++k) {
      const int a = k & 1;
      ok = mbar_wait(afull + a, (k >> 1) & 1);
      if (!ok) break;
      tc_fence_after();
      epilogue<COUT>(tmem, (uint32_t)(a * L::ACC), H, W, blockIdx.x + k * gridDim.x, warp, lane, sbias, mask, relu,
                     y, yf);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty + a);
    }
  }
  if (!ok && lane == 0 && err) atomicExch(err, 1);  // a wait gave up: flagged, the CTA winds down
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Weight gradient of a 64 -> 64 layer: for tap t, D_t[co][ci] = sum_p dY[p][co] X[p + d_t][ci]
// (M = 64 output channels, N = 64 input channels, K = pixels, 16 per MMA).  Both operands stay
// pixel-major as they lie in memory: 128-byte pixel rows (64 channels) with the 128-byte swizzle,
// i.e. the MN-major layout (transpose bits 15 and 16 set; K steps of 16 pixels are 2048 bytes).  An
// M = 64 accumulator puts row m in tensor-memory lane 32 (m / 16) + m % 16 (measured on GB300).
// A CTA owns a group of row segments (128 pixels) and one tap row dy (taps 3 dy .. 3 dy + 2): the
// K window of each of its taps lies in the single input row y + dy - 1, so a step copies the dY
// segment and that one 130-pixel row (two tensor-map boxes, plus the periodic fix-ups), three deep.
// Warps 0-3 read the three accumulators at the end and write the group's partial sums (reduced over
// groups in a fixed order by a second kernel); warp 4 issues the MMAs; warp 5 copies.
struct WgLay {
  static constexpr int NSTAGE = 3;
  static constexpr int DY = TPX * 128;                        // dY segment: 128 pixel rows of 128 B
  static constexpr int XR = (TPW * 128 + 1023) / 1024 * 1024;  // one input row of 130 pixels
  static constexpr int STAGE = DY + XR;
  static constexpr int BAR_OFF = NSTAGE * STAGE;              // tma, full, empty (x NSTAGE), done
  static constexpr int TSLOT_OFF = BAR_OFF + 8 * (3 * NSTAGE + 1);
  static constexpr int BYTES = TSLOT_OFF + 16;
  static_assert(DY % 1024 == 0 && XR % 1024 == 0, "swizzle atoms stay aligned");
};

// Bias gradient folded into the weight-gradient kernels: in the CTAs of tap row 1 (every pixel row
// once) the epilogue warps, idle until the accumulators are done, add up the staged dY segments.
// Thread t (0 .. 127) sums channel t % DC over the pixels t / DC, t / DC + 128 / DC, ... of a segment
// (DC = 64: 128-byte rows, chunk c at c ^ (j % 8); DC = 16: 32-byte rows, chunk c at c ^ ((j / 4) % 2)),
// then releases the stage together with the MMAs (the stage's empty barrier counts both).
template <int DC>
__device__ __forceinline__ float dy_column_sum(const unsigned char* dyb, int t) {
  const int c = t % DC, j0 = t / DC;
  float s = 0.0f;
#pragma unroll 8
  for (int j = j0; j < TPX; j += 128 / DC) {
    const int chunk = DC == 64 ? ((c >> 3) ^ (j & 7)) : ((c >> 3) ^ ((j >> 2) & 1));
    s += __bfloat162float(*reinterpret_cast<const bf16*>(dyb + j * (DC * 2) + (chunk << 4) + (c & 7) * 2));
  }
  return s;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

// the epilogue warps' share of a bias-gradient CTA: per segment, wait for its stage (one thread
// waits, the outcome is broadcast), add it up, release it; returns false if a wait gave up
template <int DC, int NS>
__device__ __forceinline__ bool bias_segments(const unsigned char* sm, int stage_bytes, uint64_t* full,
                                              uint64_t* empty, int nmine, int tid, uint32_t* flag, float& acc) {
  for (int k = 0; k < nmine; ++k) {
    const int b = k % NS;
    if (tid == 0) *flag = mbar_wait(full + b, (k / NS) & 1) ? 1u : 0u;
    epi_sync();
    if (!*flag) return false;
    acc += dy_column_sum<DC>(sm + b * stage_bytes, tid);
    epi_sync();
    if (tid == 0) mbar_arrive(empty + b);
  }
  return true;
}

// the CTA's partial bias sums, once every MMA is done (stage 0 serves as scratch): bpart[group][co]
template <int DC>
__device__ __forceinline__ void bias_store(unsigned char* sm, float acc, int tid, float* bpart) {
  float* red = reinterpret_cast<float*>(sm);
  red[tid] = acc;
  epi_sync();
  if (tid < DC) {
    float t = 0.0f;
    for (int r = 0; r < 128 / DC; ++r) t += red[r * DC + tid];
    bpart[(size_t)blockIdx.x * DC + tid] = t;
  }
}

// MN-major, 128-byte swizzle: 8-pixel groups of 128-byte rows 1024 bytes apart (one 64-wide atom in MN)
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__global__ void __launch_bounds__(TTHR)
    conv_wgrad_tc_kernel(int H, int W, int segs_per_group, const bf16* __restrict__ x, float* partial, float* bpart,
                         int* err,
                         const __grid_constant__ CUtensorMap dymap, const __grid_constant__ CUtensorMap xmap) {
  using L = WgLay;
  constexpr int NS = L::NSTAGE;
  constexpr uint32_t COLS = 256;  // three 64-column accumulators
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::BAR_OFF);
  uint64_t *tma = bars, *full = bars + NS, *empty = bars + 2 * NS, *done = bars + 3 * NS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::TSLOT_OFF);
  const int dyr = blockIdx.y;  // tap row: taps 3 dyr + dx
  const bool bias = bpart != nullptr && dyr == 1;
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)), "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < NS; ++b) {
      mbar_init(tma + b, 1);
      mbar_init(full + b, 1);
      mbar_init(empty + b, bias ? 2 : 1);  // the MMAs (and the bias sums) release a stage
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  pdl_wait_and_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int segs_row = W / TPX, nseg = H * segs_row;
  const int seg0 = blockIdx.x * segs_per_group;
  const int nmine = seg0 < nseg ? min(segs_per_group, nseg - seg0) : 0;
  bool ok = true;
  if (warp == LOAD_WARP) {
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NS, use = k / NS, sg = seg0 + k, row = sg / segs_row, x0 = (sg % segs_row) * TPX;
      if (k >= NS) ok = mbar_wait(empty + b, (use - 1) & 1);  // the MMAs of step k - NS read it
      if (!ok) break;
      const int yy = row + dyr - 1, gy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
      if (lane == 0) {
        unsigned char* dyb = sm + b * L::STAGE;
        mbar_expect_tx(tma + b, L::DY + TPW * 128);
        tma_load_3d(dyb, &dymap, tma + b, x0, row);
        tma_load_3d(dyb + L::DY, &xmap, tma + b, x0 - 1, gy);  // the row index is wrapped here already
      }
      __syncwarp();
    }
  } else if (warp == FIX_WARP) {
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NS, use = k / NS, sg = seg0 + k, row = sg / segs_row, x0 = (sg % segs_row) * TPX;
      unsigned char* xb = sm + b * L::STAGE + L::DY;
      const int yy = row + dyr - 1, gy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
      // the edge pixels of a wrapped segment (pixel j, chunk c at c ^ (j % 8)), loaded into registers
      // before the copy lands so that their latency overlaps it: lanes 0-7 the left wrap (pixel
      // j = 0 <- column W - 1), lanes 8-15 the right wrap (j = TPW - 1 <- column 0)
      const bool left = x0 == 0, right = x0 + TPX == W;
      const int c = lane % 8, side = lane / 8, j = side == 0 ? 0 : TPW - 1;
      const bool mine = lane < 16 && ((side == 0 && left) || (side == 1 && right));
      uint4 v = make_uint4(0, 0, 0, 0);
      if (mine) v = *reinterpret_cast<const uint4*>(x + ((size_t)gy * W + (side == 0 ? W - 1 : 0)) * 64 + c * 8);
      ok = mbar_wait(tma + b, use & 1);
      if (!ok) break;
      if (left || right) {
        if (mine) *reinterpret_cast<uint4*>(xb + j * 128 + ((c ^ (j & 7)) << 4)) = v;
        fence_async_smem();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(full + b);
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((64u >> 3) << 17) |
                              ((64u >> 4) << 24);
      for (int k = 0; k < nmine && ok; ++k) {
        const int b = k % NS;
        ok = mbar_wait(full + b, (k / NS) & 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dyb = su32(sm + b * L::STAGE), xb = dyb + L::DY;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
          for (int s2 = 0; s2 < TPX / 16; ++s2)
            umma(tmem + 64u * dx, sdesc_mn_sw128(dyb + 2048u * s2), sdesc_mn_sw128(xb + 128u * dx + 2048u * s2), ID,
                 (k | s2) != 0);
        umma_commit(empty + b);
      }
      if (ok) umma_commit(done);
    }
    __syncwarp();
  } else {  // warps 0-3: the bias sums as the segments arrive, then this group's partial sums
    float bacc = 0.0f;
    if (bias) ok = bias_segments<64, NS>(sm, L::STAGE, full, empty, nmine, tid, tslot + 1, bacc);
    ok = ok && (nmine == 0 || mbar_wait(done, 0));
    if (ok && bias) bias_store<64>(sm, bacc, tid, bpart);
    if (ok && nmine > 0) {
      tc_fence_after();
      for (int dx = 0; dx < 3; ++dx) {
        uint32_t raw[64];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 64u * dx + 16u * q, raw + 16 * q);
        tmem_wait_ld();
        if (lane < 16) {  // lanes 0-15 of warp w hold output channels 16 w .. 16 w + 15
          const int co = 16 * warp + lane;
          float4* dst =
              reinterpret_cast<float4*>(partial + (((size_t)blockIdx.x * 9 + 3 * dyr + dx) * 64 + co) * 64);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            dst[q] = make_float4(__uint_as_float(raw[4 * q]), __uint_as_float(raw[4 * q + 1]),
                                 __uint_as_float(raw[4 * q + 2]), __uint_as_float(raw[4 * q + 3]));
        }
      }
    }
  }
  if (!ok && lane == 0 && err) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Weight gradient of the 16 -> 64 (first) and 64 -> 16 (last) layers, the same scheme as the 64 -> 64
// kernel with the 64-channel tensor as the M = 64 operand and the 16-channel one as N = 16:
//   16 -> 64 (XC = 16, DC = 64): D_t[co][ci] = sum_p dY[p][co] X[p + d_t][ci],  A = dY, B = X_t;
//   64 -> 16 (XC = 64, DC = 16): D_t[ci][co] = sum_p X[p + d_t][ci] dY[p][co],  A = X_t, B = dY,
// written transposed.  Both operands stay pixel-major (MN-major): 64-channel pixel rows of 128 bytes
// with the 128-byte swizzle (SBO = 1024), 16-channel rows of 32 bytes with the 32-byte swizzle
// (SBO = 256: eight pixels); a tap's shift moves the X operand's start by whole pixel rows.
// ---------------------------------------------------------------------------------------------
template <int XC, int DC>
struct Wg16Lay {
  static constexpr int NSTAGE = 3;
  static constexpr int DY = (TPX * DC * 2 + 1023) / 1024 * 1024;  // dY segment
  static constexpr int XR = (TPW * XC * 2 + 1023) / 1024 * 1024;  // one input row of 130 pixels
  static constexpr int STAGE = DY + XR;
  static constexpr int BAR_OFF = NSTAGE * STAGE;
  static constexpr int TSLOT_OFF = BAR_OFF + 8 * (3 * NSTAGE + 1);
  static constexpr int BYTES = TSLOT_OFF + 16;
  static_assert((XC == 16 && DC == 64) || (XC == 64 && DC == 16), "one 16-channel and one 64-channel side");
};

// MN-major, 32-byte swizzle: 8-pixel groups of 32-byte rows 256 bytes apart (one 16-wide atom in MN)
__device__ __forceinline__ uint64_t sdesc_mn_sw32(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

template <int XC, int DC>
__global__ void __launch_bounds__(TTHR)
    conv_wgrad16_tc_kernel(int H, int W, int segs_per_group, const bf16* __restrict__ x, float* partial,
                           float* bpart, int* err,
                           const __grid_constant__ CUtensorMap dymap, const __grid_constant__ CUtensorMap xmap) {
  using L = Wg16Lay<XC, DC>;
  constexpr int NS = L::NSTAGE;
  constexpr uint32_t COLS = 64;  // three 16-column accumulators
  constexpr int XROW = XC * 2;   // bytes of one input pixel row
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::BAR_OFF);
  uint64_t *tma = bars, *full = bars + NS, *empty = bars + 2 * NS, *done = bars + 3 * NS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::TSLOT_OFF);
  const int dyr = blockIdx.y;  // tap row: taps 3 dyr + dx
  const bool bias = bpart != nullptr && dyr == 1;
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)), "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < NS; ++b) {
      mbar_init(tma + b, 1);
      mbar_init(full + b, 1);
      mbar_init(empty + b, bias ? 2 : 1);  // the MMAs (and the bias sums) release a stage
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  pdl_wait_and_trigger();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int segs_row = W / TPX, nseg = H * segs_row;
  const int seg0 = blockIdx.x * segs_per_group;
  const int nmine = seg0 < nseg ? min(segs_per_group, nseg - seg0) : 0;
  bool ok = true;
  if (warp == LOAD_WARP) {
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NS, use = k / NS, sg = seg0 + k, row = sg / segs_row, x0 = (sg % segs_row) * TPX;
      if (k >= NS) ok = mbar_wait(empty + b, (use - 1) & 1);  // the MMAs of step k - NS read it
      if (!ok) break;
      const int yy = row + dyr - 1, gy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
      if (lane == 0) {
        unsigned char* dyb = sm + b * L::STAGE;
        mbar_expect_tx(tma + b, TPX * DC * 2 + TPW * XROW);
        tma_load_3d(dyb, &dymap, tma + b, x0, row);
        tma_load_3d(dyb + L::DY, &xmap, tma + b, x0 - 1, gy);  // the row index is wrapped here already
      }
      __syncwarp();
    }
  } else if (warp == FIX_WARP) {
    constexpr int CPP = XROW / 16;  // 16-byte chunks per input pixel (2 or 8)
    for (int k = 0; k < nmine && ok; ++k) {
      const int b = k % NS, use = k / NS, sg = seg0 + k, row = sg / segs_row, x0 = (sg % segs_row) * TPX;
      unsigned char* xb = sm + b * L::STAGE + L::DY;
      const int yy = row + dyr - 1, gy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
      // the edge pixels of a wrapped segment, loaded into registers before the copy lands: lanes
      // 0 .. CPP-1 the left wrap (pixel j = 0 <- column W - 1), CPP .. 2 CPP - 1 the right wrap
      // (j = TPW - 1 <- column 0).  Chunk c of pixel j sits at chunk c ^ (j % 8) of its 128-byte row
      // (128-byte swizzle) or c ^ ((j / 4) % 2) of its 32-byte row (32-byte swizzle).
      const bool left = x0 == 0, right = x0 + TPX == W;
      const int c = lane % CPP, side = lane / CPP, j = side == 0 ? 0 : TPW - 1;
      const bool mine = lane < 2 * CPP && ((side == 0 && left) || (side == 1 && right));
      uint4 v = make_uint4(0, 0, 0, 0);
      if (mine) v = *reinterpret_cast<const uint4*>(x + ((size_t)gy * W + (side == 0 ? W - 1 : 0)) * XC + c * 8);
      ok = mbar_wait(tma + b, use & 1);
      if (!ok) break;
      if (left || right) {
        const int cs = XC == 64 ? (c ^ (j & 7)) : (c ^ ((j >> 2) & 1));
        if (mine) *reinterpret_cast<uint4*>(xb + j * XROW + (cs << 4)) = v;
        fence_async_smem();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(full + b);
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      // BF16 x BF16 -> F32, both operands MN-major (transpose bits 15, 16), N = 16, M = 64
      constexpr uint32_t ID = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((16u >> 3) << 17) |
                              ((64u >> 4) << 24);
      for (int k = 0; k < nmine && ok; ++k) {
        const int b = k % NS;
        ok = mbar_wait(full + b, (k / NS) & 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dyb = su32(sm + b * L::STAGE), xb = dyb + L::DY;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
          for (int s2 = 0; s2 < TPX / 16; ++s2) {
            uint64_t da, db;
            if (XC == 16) {  // A = dY (64 channels), B = the shifted X window (16 channels)
              da = sdesc_mn_sw128(dyb + 2048u * s2);
              db = sdesc_mn_sw32(xb + 32u * dx + 512u * s2);
            } else {         // A = the shifted X window (64 channels), B = dY (16 channels)
              da = sdesc_mn_sw128(xb + 128u * dx + 2048u * s2);
              db = sdesc_mn_sw32(dyb + 512u * s2);
            }
            umma(tmem + 16u * dx, da, db, ID, (k | s2) != 0);
          }
        umma_commit(empty + b);
      }
      if (ok) umma_commit(done);
    }
    __syncwarp();
  } else {  // warps 0-3: the bias sums as the segments arrive, then this group's partial sums
    float bacc = 0.0f;
    if (bias) ok = bias_segments<DC, NS>(sm, L::STAGE, full, empty, nmine, tid, tslot + 1, bacc);
    ok = ok && (nmine == 0 || mbar_wait(done, 0));
    if (ok && bias) bias_store<DC>(sm, bacc, tid, bpart);
    if (ok && nmine > 0) {
      tc_fence_after();
      uint32_t raw[48];
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16u * dx, raw + 16 * dx);
      tmem_wait_ld();
      if (lane < 16) {  // lanes 0-15 of warp w hold rows m = 16 w .. 16 w + 15 of the M = 64 side
        const int m = 16 * warp + lane;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          float* tap = partial + ((size_t)blockIdx.x * 9 + 3 * dyr + dx) * 64 * 16;  // [co][ci]
          if (XC == 16) {  // m = co, n = ci: 16 consecutive floats
            float4* dst = reinterpret_cast<float4*>(tap + (size_t)m * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              dst[q] = make_float4(__uint_as_float(raw[16 * dx + 4 * q]), __uint_as_float(raw[16 * dx + 4 * q + 1]),
                                   __uint_as_float(raw[16 * dx + 4 * q + 2]),
                                   __uint_as_float(raw[16 * dx + 4 * q + 3]));
          } else {  // m = ci, n = co: partial[co][ci], consecutive lanes on consecutive ci
#pragma unroll
            for (int n = 0; n < 16; ++n) tap[(size_t)n * 64 + m] = __uint_as_float(raw[16 * dx + n]);
          }
        }
      }
    }
  }
  if (!ok && lane == 0 && err) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(COLS) : "memory");
  }
}

__device__ int g_conv_tc_err = 0;  // raised if a bounded wait on the tensor cores gives up

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

cudaLaunchConfig_t pdl_config(dim3 grid, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(TTHR);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cfg;
}

void pdl_attr(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

template <int CIN, int COUT>
cudaError_t tc_launch(int H, int W, const void* x, const void* w, const float* b, const void* mask, int relu, void* y,
                      float* yf, cudaStream_t st) {
  using L = TcLay<CIN, COUT>;
  static int ready[32] = {0};
  static int grid_max[32] = {0};
  static int* err[32] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 32) return cudaErrorInvalidDevice;
  if (!ready[dev]) {
    e = cudaFuncSetAttribute(conv_fwd_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_fwd_tc_kernel<CIN, COUT>, TTHR, L::BYTES);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // at most 512 / COLS CTAs of this kernel share an SM's tensor memory
    const int tmem_cap = 512 / L::COLS;
    grid_max[dev] = sms * (per_sm < tmem_cap ? per_sm : tmem_cap);
    if ((e = cudaGetSymbolAddress((void**)&err[dev], g_conv_tc_err)) != cudaSuccess) return e;
    ready[dev] = 1;
  }
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  alignas(64) CUtensorMap xmap, wmap;
  memset(&wmap, 0, sizeof wmap);
  CUresult r;
  if (L::SW) {
    // input (64 channels = one 128-byte row, W, H), box 64 x 130 x 3, 128-byte swizzle
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint64_t dims[3] = {(cuuint64_t)CIN, (cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[2] = {(cuuint64_t)CIN * 2, (cuuint64_t)W * CIN * 2};
    const cuuint32_t box[3] = {(cuuint32_t)CIN, (cuuint32_t)TPW, (cuuint32_t)TPR};
    r = enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // weights [c_out][tap][c_in] as (c_in, tap, c_out): the box (64, 1, C_out) of tap t lands as C_out
    // rows of 128 bytes, 128-byte swizzle (the B operand of tap t)
    const cuuint64_t wdims[3] = {(cuuint64_t)CIN, 9, (cuuint64_t)COUT};
    const cuuint64_t wstrides[2] = {(cuuint64_t)CIN * 2, (cuuint64_t)9 * CIN * 2};
    const cuuint32_t wbox[3] = {(cuuint32_t)CIN, 1, (cuuint32_t)COUT};
    r = enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(w), wdims, wstrides, wbox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {  // (8 channels of a chunk, W, H, chunk): the box 8 x 130 x 3 x CH lands chunk-major
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint64_t dims[4] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)L::CH};
    const cuuint64_t strides[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)W * CIN * 2, 16};
    const cuuint32_t box[4] = {8, (cuuint32_t)TPW, (cuuint32_t)TPR, (cuuint32_t)L::CH};
    r = enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int nitems = H * (W / TPX);
  const int grid = nitems < grid_max[dev] ? nitems : grid_max[dev];
  cudaLaunchConfig_t cfg = pdl_config(dim3(grid), L::BYTES, st);
  cudaLaunchAttribute attr[1];
  pdl_attr(cfg, attr);
  return cudaLaunchKernelEx(&cfg, conv_fwd_tc_kernel<CIN, COUT>, H, W, (const bf16*)x, (const bf16*)w, b,
                            (const bf16*)mask, relu, (bf16*)y, yf, err[dev], xmap, wmap);
}

cudaError_t wg64_launch(int H, int W, const void* x, const void* dy, float* partial, float* bpart, int segs_per_group,
                        cudaStream_t st) {
  static int ready[32] = {0};
  static int* err[32] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 32) return cudaErrorInvalidDevice;
  if (!ready[dev]) {
    e = cudaFuncSetAttribute(conv_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WgLay::BYTES);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&err[dev], g_conv_tc_err)) != cudaSuccess) return e;
    ready[dev] = 1;
  }
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  alignas(64) CUtensorMap dymap, xmap;
  const cuuint64_t dims[3] = {64, (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[2] = {128, (cuuint64_t)W * 128};
  const cuuint32_t box_dy[3] = {64, (cuuint32_t)TPX, 1}, box_x[3] = {64, (cuuint32_t)TPW, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&dymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(dy), dims, strides, box_dy, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box_x, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int nseg = H * (W / TPX), groups = (nseg + segs_per_group - 1) / segs_per_group;
  cudaLaunchConfig_t cfg = pdl_config(dim3(groups, 3), WgLay::BYTES, st);
  cudaLaunchAttribute attr[1];
  pdl_attr(cfg, attr);
  return cudaLaunchKernelEx(&cfg, conv_wgrad_tc_kernel, H, W, segs_per_group, (const bf16*)x, partial, bpart, err[dev],
                            dymap, xmap);
}

template <int XC, int DC>
cudaError_t wg16_launch(int H, int W, const void* x, const void* dy, float* partial, float* bpart, int segs_per_group,
                        cudaStream_t st) {
  using L = Wg16Lay<XC, DC>;
  static int ready[32] = {0};
  static int* err[32] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 32) return cudaErrorInvalidDevice;
  if (!ready[dev]) {
    e = cudaFuncSetAttribute(conv_wgrad16_tc_kernel<XC, DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&err[dev], g_conv_tc_err)) != cudaSuccess) return e;
    ready[dev] = 1;
  }
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  alignas(64) CUtensorMap dymap, xmap;
  const cuuint64_t ddims[3] = {(cuuint64_t)DC, (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t dstr[2] = {(cuuint64_t)DC * 2, (cuuint64_t)W * DC * 2};
  const cuuint64_t xdims[3] = {(cuuint64_t)XC, (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t xstr[2] = {(cuuint64_t)XC * 2, (cuuint64_t)W * XC * 2};
  const cuuint32_t box_dy[3] = {(cuuint32_t)DC, (cuuint32_t)TPX, 1}, box_x[3] = {(cuuint32_t)XC, (cuuint32_t)TPW, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapSwizzle dsw = DC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B;
  const CUtensorMapSwizzle xsw = XC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B;
  if (enc(&dymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(dy), ddims, dstr, box_dy, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, dsw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), xdims, xstr, box_x, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, xsw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int nseg = H * (W / TPX), groups = (nseg + segs_per_group - 1) / segs_per_group;
  cudaLaunchConfig_t cfg = pdl_config(dim3(groups, 3), L::BYTES, st);
  cudaLaunchAttribute attr[1];
  pdl_attr(cfg, attr);
  return cudaLaunchKernelEx(&cfg, conv_wgrad16_tc_kernel<XC, DC>, H, W, segs_per_group, (const bf16*)x, partial, bpart,
                            err[dev], dymap, xmap);
}

}  // namespace

cudaError_t conv_fwd_tc(int H, int W, int cin, int cout, const void* x, const void* w, const float* b,
                        const void* mask, int relu, void* y, float* yf, cudaStream_t st) {
  if (cin == 16) return tc_launch<16, 64>(H, W, x, w, b, mask, relu, y, yf, st);
  if (cout == 64) return tc_launch<64, 64>(H, W, x, w, b, mask, relu, y, yf, st);
  return tc_launch<64, 16>(H, W, x, w, b, mask, relu, y, yf, st);
}

cudaError_t conv_wgrad_tc(int H, int W, int cin, int cout, const void* x, const void* dy, float* partial, float* bpart,
                          int segs_per_group, cudaStream_t st) {
  if (cin == 64 && cout == 64) return wg64_launch(H, W, x, dy, partial, bpart, segs_per_group, st);
  if (cin == 16 && cout == 64) return wg16_launch<16, 64>(H, W, x, dy, partial, bpart, segs_per_group, st);
  if (cin == 64 && cout == 16) return wg16_launch<64, 16>(H, W, x, dy, partial, bpart, segs_per_group, st);
  return cudaErrorInvalidValue;
}

cudaError_t conv_tc_status(cudaStream_t st, int clear, int* raised) {
  int* flag = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&flag, g_conv_tc_err);
  if (e != cudaSuccess) return e;
  int v = 0;
  if ((e = cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  *raised = v;
  if (clear && v) {
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t conv_tc_raise(int value) {
  int* flag = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&flag, g_conv_tc_err);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(flag, &value, sizeof(int), cudaMemcpyHostToDevice);
}

}  // namespace vlb
