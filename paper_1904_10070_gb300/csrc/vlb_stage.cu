// Fused Runge-Kutta stage of the vielbein LB + Cahn-Hilliard solver (arXiv:1904.10070).
//
// One launch evaluates, for every node of the periodic (theta, varphi) grid,
//   L_f   = right-hand side of Eq. boltz_tor with BGK collisions (Sec. 2.3),
//   L_phi = right-hand side of Eq. CH with mu from Eq. mu and the force of Eq. pbin,
// and writes U_out = U^n + b (U_in - U^n + dt L(U_in)) -- one stage of SSP-RK3 in Shu-Osher form
// (b = 1, 1/4, 2/3), written so that the weights only multiply small increments.  The populations
// are stored as deviations g = f - n0 w_i w_j from the rest equilibrium, and in FP32 mode phi is
// carried as an unevaluated float pair hi + lo (vlb_internal.cuh explains both).
//
// Work unit: a tile of TQ theta rows x 32 varphi columns.  For a tile the CTA
//   1. stages, with asynchronous global->shared copies (cp.async), a box of H rows (2 for UW3,
//      3 for WENO5) and HS columns around the tile for the 16 populations and phi, the tile's
//      U^n values and the per-row coefficients;
//   2. computes the moments and mu on the tile plus a halo of 1;
//   3. computes the right-hand sides and the Runge-Kutta combination and stores the tile.
// One 256-thread CTA per 16 x 32 tile, two CTAs per SM.  For FP32 UW3 grids with n_phi % 4 == 0 (the
// production path) step 3 runs on adjacent node pairs in packed FP32x2 arithmetic, two lanes of
// one float2 per thread; every other case (FP64, WENO5, odd or tiny grids) runs step 3 in scalar
// arithmetic, two nodes per thread.  A persistent double-buffered variant (next tile copied in
// while the current one computes, one 384-thread CTA per SM) measured 1.6x slower on GB300: with
// 12 warps per SM and all warps issuing copies and shared loads in the same phase, the memory-
// input queue throttled issue to 30%.
// Periodic wrap-around is resolved on the copy addresses, so ragged tiles need no special case.
#include <vector>

#include "vlb_internal.cuh"

namespace vlb {

namespace {

constexpr int TS = 32;   // tile width along varphi
constexpr int NCT = 11;  // coefficient rows staged in shared memory (C_J .. C_EN)

template <typename T>
struct VConst {
  T v[4], w[4], K[4][4];
  T ww[4][4];  // w_i w_j
};

// Shared-memory layout of one CTA.  Offsets are in elements of T.
template <typename T, int H_, int TQ_, int HS_, int NTH_, int NBUF_>
struct Lay {
  static constexpr bool DF = sizeof(T) == 4;       // phi as a float pair
  static constexpr int H = H_, TQ = TQ_, HS = HS_, NTH = NTH_, NBUF = NBUF_;
  static constexpr int NST = DF ? NARR + 1 : NARR;  // state arrays (= staged boxes)
  static constexpr int BQ = TQ + 2 * H, BS = TS + 2 * HS;
  static constexpr int BOX = NST * BQ * BS;          // populations, phi (, phi lo)
  static constexpr int MQ = TQ + 2, MS = TS + 4;     // moment / mu box: halo 1, column origin -2
  static constexpr int CO = (NCT * BQ + 15) / 16 * 16;  // padded: sub-buffers stay 16-byte aligned
  static constexpr int VEC = 16 / sizeof(T);              // elements per 16-byte chunk
  // each box row starts HS columns left of the tile: shift the buffers so that the tile columns
  // (and every 16-byte chunk copied into them) start on a 16-byte boundary
  static constexpr int BOX_OFF = (VEC - HS % VEC) % VEC;
  static constexpr int CO_OFF = (BOX_OFF + NBUF * BOX + VEC - 1) / VEC * VEC;
  static constexpr int U0_OFF = CO_OFF + NBUF * CO;
  static constexpr int N_OFF = U0_OFF + NST * TQ * TS;
  static constexpr int UT_OFF = N_OFF + MQ * MS;
  static constexpr int UP_OFF = UT_OFF + MQ * MS;
  static constexpr int MU_OFF = UP_OFF + MQ * MS;
  static constexpr int MB_OFF = (MU_OFF + MQ * MS + 1) / 2 * 2;  // two 8-byte mbarriers
  static constexpr int TOTAL = MB_OFF + 16 / (int)sizeof(T);
  static constexpr size_t BYTES = sizeof(T) * (size_t)TOTAL;
  static_assert((BOX * sizeof(T)) % 16 == 0 && (BS * sizeof(T)) % 16 == 0 && (BQ * BS * sizeof(T)) % 16 == 0,
                "box rows and arrays keep 16-byte alignment");
  static_assert(((BOX_OFF + HS) * sizeof(T)) % 16 == 0, "tile columns start on a 16-byte boundary");
  static_assert((BOX_OFF * sizeof(T)) % 8 == 0, "edge chunks are 8-byte aligned");
  static_assert((CO_OFF * sizeof(T)) % 16 == 0 && (U0_OFF * sizeof(T)) % 16 == 0, "16-byte aligned sub-buffers");
};

template <typename T, int ADV>
using GenericLay = Lay<T, (ADV == VLB_UW3 ? 2 : 3), 16, 4, 256, 1>;

__device__ __forceinline__ int wrap(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Programmatic dependent launch: a stage may start while the previous kernel in the stream drains.
// pdl_wait() blocks until that kernel has completed and its writes are visible (a no-op without a
// programmatic launch); pdl_trigger() lets the next stage's CTAs be scheduled.  Every global
// access (state buffers and coefficient tables) comes after pdl_wait(); only shared-memory set-up
// runs before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// mbarrier and bulk tensor copy (TMA) primitives.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after 2^22 polls (each poll may suspend the thread for a while), so that a
// copy that never lands cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Copy the box {x, y, z} .. + box dims of a 3-D tensor map into shared memory (128-byte aligned),
// completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Prefetch the box {x, y, z} .. + box dims of a 3-D tensor map into L2 (a hint: no shared memory).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Fifth-order WENO-JS face value between g2 and g3 of the window g0..g4, upwind from g0's side.
template <typename T>
__device__ __forceinline__ T weno5(T g0, T g1, T g2, T g3, T g4) {
  const T c13_12 = T(13) / T(12), sixth = T(1) / T(6), eps = T(1e-6);
  T q0 = (T(2) * g0 - T(7) * g1 + T(11) * g2) * sixth;
  T q1 = (-g1 + T(5) * g2 + T(2) * g3) * sixth;
  T q2 = (T(2) * g2 + T(5) * g3 - g4) * sixth;
  T d0 = g0 - T(2) * g1 + g2, e0 = g0 - T(4) * g1 + T(3) * g2;
  T d1 = g1 - T(2) * g2 + g3, e1 = g1 - g3;
  T d2 = g2 - T(2) * g3 + g4, e2 = T(3) * g2 - T(4) * g3 + g4;
  T b0 = c13_12 * d0 * d0 + T(0.25) * e0 * e0;
  T b1 = c13_12 * d1 * d1 + T(0.25) * e1 * e1;
  T b2 = c13_12 * d2 * d2 + T(0.25) * e2 * e2;
  T a0 = T(0.1) / ((eps + b0) * (eps + b0));
  T a1 = T(0.6) / ((eps + b1) * (eps + b1));
  T a2 = T(0.3) / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// WENO5 flux difference face_{+1/2} - face_{-1/2} at the centre x[3] of a 7-point window.
template <typename T, bool POS>
__device__ __forceinline__ T weno_diff(const T (&x)[7]) {
  if (POS) return weno5(x[1], x[2], x[3], x[4], x[5]) - weno5(x[0], x[1], x[2], x[3], x[4]);
  return weno5(x[6], x[5], x[4], x[3], x[2]) - weno5(x[5], x[4], x[3], x[2], x[1]);
}

// Whether the chunked copy path applies: rows wrap at most once and columns come in aligned
// 16-byte chunks that never straddle the periodic seam.
template <typename L>
__host__ __device__ inline bool chunked(int nt, int ns) {
  constexpr int VEC = 16 / (L::DF ? 4 : 8);
  return ns % VEC == 0 && ns >= L::BS && nt >= L::BQ;
}

// ---------------------------------------------------------------------------------------------
// Step 1: asynchronous copies of the box (populations and phi of U_in) with its row coefficients,
// and of the tile's U^n.
// ---------------------------------------------------------------------------------------------
template <typename L, typename T>
__device__ __forceinline__ void issue_co(const StageArgs<T>& a, T* co, int q0, int tid) {
  for (int idx = tid; idx < NCT * L::BQ; idx += L::NTH) {
    const int k = idx / L::BQ, r = idx - k * L::BQ;
    cp_async_small<sizeof(T)>(co + idx, a.coef + (int64_t)k * a.nt + wrap(q0 + r - L::H, a.nt));
  }
}

template <typename L, typename T>
__device__ __forceinline__ void issue_box(const StageArgs<T>& a, T* box, T* co, int q0, int s0, int tid) {
  constexpr int H = L::H, BQ = L::BQ, BS = L::BS, HS = L::HS;
  constexpr int VEC = 16 / sizeof(T);
  const int nt = a.nt, ns = a.ns;
  const int64_t stride = a.stride;
  if (chunked<L>(nt, ns)) {
    // chunk c of a box row: with HS % VEC == 0 all chunks are VEC wide; otherwise the two edge
    // chunks are HS wide (8-byte copies) and the interior ones VEC wide.
    constexpr bool EDGE = HS % VEC != 0;
    constexpr int CPR = EDGE ? TS / VEC + 2 : BS / VEC;
    for (int pos = tid; pos < BQ * CPR; pos += L::NTH) {
      const int r = pos / CPR, ch = pos - r * CPR;
      int gq = q0 + r - H;
      gq += gq < 0 ? nt : (gq >= nt ? -nt : 0);
      int col, width;
      if (EDGE) {
        col = ch == 0 ? 0 : (ch == CPR - 1 ? HS + TS : HS + (ch - 1) * VEC);
        width = (ch == 0 || ch == CPR - 1) ? HS : VEC;
      } else {
        col = ch * VEC;
        width = VEC;
      }
      int gs = s0 - HS + col;
      gs += gs < 0 ? ns : (gs >= ns ? -ns : 0);
      const T* src = a.fin + (int64_t)gq * ns + gs;
      T* dst = box + r * BS + col;
      if (width == VEC) {
#pragma unroll
        for (int k = 0; k < L::NST; ++k) cp_async16(dst + k * BQ * BS, src + k * stride);
      } else {
#pragma unroll
        for (int k = 0; k < L::NST; ++k) cp_async_small<8>(dst + k * BQ * BS, src + k * stride);
      }
    }
  } else {
    for (int idx = tid; idx < L::NST * BQ * BS; idx += L::NTH) {
      const int k = idx / (BQ * BS);
      const int rem = idx - k * (BQ * BS);
      const int r = rem / BS, c = rem - r * BS;
      const int gq = wrap(q0 + r - H, nt), gs = wrap(s0 + c - HS, ns);
      cp_async_small<sizeof(T)>(box + (k * BQ + r) * BS + c, a.fin + k * stride + (int64_t)gq * ns + gs);
    }
  }
}

template <typename L, typename T>
__device__ __forceinline__ void issue_u0(const StageArgs<T>& a, T* su0, int q0, int s0, int tid) {
  constexpr int TQ = L::TQ, VEC = 16 / sizeof(T);
  const int nt = a.nt, ns = a.ns;
  const int64_t stride = a.stride;
  if (chunked<L>(nt, ns)) {
    // TQ x TS/VEC chunk positions; the arrays are split between groups of threads
    constexpr int CT = TS / VEC, NPOS = TQ * CT;
    constexpr int GROUPS = L::NTH / NPOS > 0 ? L::NTH / NPOS : 1;
    constexpr int PER = (L::NST + GROUPS - 1) / GROUPS;
    for (int t = tid; t < NPOS * GROUPS; t += L::NTH) {
      const int pos = t % NPOS, grp = t / NPOS;
      const int r = pos / CT, ch = pos - r * CT;
      const int gq = q0 + r, gs = s0 + ch * VEC;
      if (gq < nt && gs < ns) {
        const T* src = a.f0 + (int64_t)gq * ns + gs;
        T* dst = su0 + r * TS + ch * VEC;
        const int k0 = grp * PER, k1 = k0 + PER < L::NST ? k0 + PER : L::NST;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) cp_async16(dst + k * TQ * TS, src + k * stride);
      }
    }
  } else {
    for (int idx = tid; idx < L::NST * TQ * TS; idx += L::NTH) {
      const int k = idx / (TQ * TS);
      const int rem = idx - k * (TQ * TS);
      const int r = rem / TS, c = rem - r * TS;
      const int gq = q0 + r, gs = s0 + c;
      if (gq < nt && gs < ns)
        cp_async_small<sizeof(T)>(su0 + (k * TQ + r) * TS + c, a.f0 + k * stride + (int64_t)gq * ns + gs);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Step 2: moments (Sec. 2.3) and mu (Eq. mu) on the tile plus a halo of 1 (cross-shaped).
// Moment-box position (mr, mc) is tile node (mr - 1, mc - 2).
// ---------------------------------------------------------------------------------------------
// Moments and mu at moment-box position (mr, mc).
template <typename L, typename T>
__device__ __forceinline__ void moment_point(const StageArgs<T>& a, const VConst<T>& vc, const T* box, const T* co,
                                             T* sm, int mr, int mc) {
  constexpr int H = L::H, BQ = L::BQ, BS = L::BS, HS = L::HS, MS = L::MS;
  const T* sf = box;
  const T* sphi = box + NPOP * BQ * BS;
  const T* sphl = box + (NPOP + 1) * BQ * BS;
  const int bi = (mr + H - 1) * BS + (mc - 2 + HS);  // box index of this position
  const T* fp = sf + bi;
  T row[4] = {T(0), T(0), T(0), T(0)}, col[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T x = fp[(4 * i + j) * BQ * BS];
      row[i] += x;
      col[j] += x;
    }
  // n = n0 + sum g (the reference part carries no momentum); v_1 = -v_4, v_2 = -v_3
  const T dn = (row[0] + row[1]) + (row[2] + row[3]);
  const T mt = vc.v[3] * (row[3] - row[0]) + vc.v[2] * (row[2] - row[1]);
  const T mp = vc.v[3] * (col[3] - col[0]) + vc.v[2] * (col[2] - col[1]);
  const int mi = mr * MS + mc;
  const T inv_n = recip(a.n0 + dn);
  sm[L::N_OFF + mi] = dn;
  sm[L::UT_OFF + mi] = mt * inv_n;
  sm[L::UP_OFF + mi] = mp * inv_n;
  const T* pp = sphi + bi;
  const int cr = mr + H - 1;
  const T ph = pp[0];
  // neighbour differences of phi = hi + lo: the hi differences are exact for nearby values
  T dN = pp[BS] - ph, dS = ph - pp[-BS], dE = pp[1] - ph, dW = ph - pp[-1], lo = T(0);
  if (L::DF) {
    const T* pl = sphl + bi;
    lo = pl[0];
    dN += pl[BS] - lo;
    dS += lo - pl[-BS];
    dE += pl[1] - lo;
    dW += lo - pl[-1];
  }
  const T lap = co[C_LT * BQ + cr] * (co[C_JP * BQ + cr] * dN - co[C_JM * BQ + cr] * dS) +
                co[C_LP * BQ + cr] * (dE - dW);
  // phi (1 - phi^2) at hi + lo, to first order in lo
  const T cubic = ph * (T(1) - ph * ph) + (T(1) - T(3) * ph * ph) * lo;
  sm[L::MU_OFF + mi] = -a.A * cubic - a.kappa * lap;
}

template <typename L, typename T>
__device__ __forceinline__ void phase2(const StageArgs<T>& a, const VConst<T>& vc, const T* box, const T* co,
                                       T* sm, int tid) {
  constexpr int MQ = L::MQ, TQ = L::TQ;
  constexpr int MS2 = TS + 2;  // tile columns -1 .. TS in the rows of the tile
  constexpr int PA = TQ * MS2;
  constexpr int PM = PA + 2 * TS;
  for (int idx = tid; idx < PM; idx += L::NTH) {
    int mr, mc;
    if (idx < PA) {
      mr = 1 + idx / MS2;
      mc = 1 + (idx - (mr - 1) * MS2);
    } else {
      const int j = idx - PA;
      mr = (j < TS) ? 0 : MQ - 1;
      mc = 2 + (j < TS ? j : j - TS);
    }
    moment_point<L>(a, vc, box, co, sm, mr, mc);
  }
}

// ---------------------------------------------------------------------------------------------
// Step 3, scalar: right-hand sides and the Runge-Kutta combination for node (lr, lc) of the tile.
// ---------------------------------------------------------------------------------------------
template <typename L, typename T, int ADV, int CH, bool F0>
__device__ __forceinline__ void phase3_node(const StageArgs<T>& a, const VConst<T>& vc, const T* box, const T* co,
                                            const T* sm, int lr, int lc, int q, int s) {
  constexpr bool DF = L::DF;
  constexpr int H = L::H, BQ = L::BQ, BS = L::BS, HS = L::HS, MS = L::MS, TQ = L::TQ;
  const T* sf = box;
  const T* sphi = box + NPOP * BQ * BS;
  const T* sphl = box + (NPOP + 1) * BQ * BS;
  const T* su0 = sm + L::U0_OFF;
  const T* sn = sm + L::N_OFF;
  const T* sut = sm + L::UT_OFF;
  const T* sup = sm + L::UP_OFF;
  const T* smu = sm + L::MU_OFF;
  const int64_t stride = a.stride;
  const T sixth = T(1) / T(6);
  const int fr = lr + H, fc = lc + HS;
  const int bi = fr * BS + fc;
  const int mi = (lr + 1) * MS + (lc + 2);
  const int ui = lr * TS + lc;

  const T dn = sn[mi], ut = sut[mi], up = sup[mi], ph = sphi[bi];
  const T n = a.n0 + dn;
  const T ct = co[C_CT * BQ + fr], cp = co[C_CP * BQ + fr], gam = co[C_GAM * BQ + fr];
  const T mu_c = smu[mi], mu_n = smu[mi + MS], mu_s = smu[mi - MS], mu_e = smu[mi + 1], mu_w = smu[mi - 1];

  // Cahn-Hilliard: M Delta mu - div(u phi) (Eq. CH), flux form with mean face values
  T Lphi = a.M * (co[C_LT * BQ + fr] * (co[C_JP * BQ + fr] * (mu_n - mu_c) - co[C_JM * BQ + fr] * (mu_c - mu_s)) +
                  co[C_LP * BQ + fr] * (mu_e - T(2) * mu_c + mu_w));
  T Ft = T(0), Fp = T(0);
  if (CH == VLB_HYDRO) {
    const T Xn = co[C_J * BQ + fr + 1] * sut[mi + MS] * sphi[bi + BS];
    const T Xs = co[C_J * BQ + fr - 1] * sut[mi - MS] * sphi[bi - BS];
    const T Ye = sup[mi + 1] * sphi[bi + 1];
    const T Yw = sup[mi - 1] * sphi[bi - 1];
    Lphi -= T(0.5) * (ct * (Xn - Xs) + cp * (Ye - Yw));
    // n F = -phi grad mu (Eq. pbin), central differences
    const T pn = ph * recip(n);
    Ft = -pn * (mu_n - mu_s) * a.gt;
    Fp = -pn * (mu_e - mu_w) * co[C_GP * BQ + fr];
  }

  const int64_t gidx = (int64_t)q * a.ns + s;
  if (a.dphi) {
    a.dphi[gidx] = Lphi * a.dt;  // the stabilised Cahn-Hilliard solve forms phi
  } else {
    const T lo = DF ? sphl[bi] : T(0);
    T base = ph, base_lo = lo, inc = Lphi * a.dt;
    if (F0) {
      base = su0[NPOP * TQ * TS + ui];
      base_lo = DF ? su0[(NPOP + 1) * TQ * TS + ui] : T(0);
      inc = a.b * (((ph - base) + (lo - base_lo)) + inc);
    }
    if (DF) {
      // (hi, lo) <- (base, base_lo) + inc with an error-free sum, then renormalised
      const T s1 = base + inc;
      const T bb = s1 - base;
      const T err = (base - (s1 - bb)) + (inc - bb);
      const T lo2 = base_lo + err;
      const T hi_out = s1 + lo2;
      a.fout[NPOP * stride + gidx] = hi_out;
      a.fout[(NPOP + 1) * stride + gidx] = lo2 - (hi_out - s1);
    } else {
      a.fout[NPOP * stride + gidx] = base + inc;
    }
  }

  // population deviations at the node
  T g[NPOP];
#pragma unroll
  for (int k = 0; k < NPOP; ++k) g[k] = sf[k * BQ * BS + bi];

  // UW3 advection weights: the theta flux difference of G = J g with ct/6 folded in, over
  // d = -2..1 (v > 0) and d = -1..2 (v < 0); the varphi difference is scaled by cp/6.
  const T ct6 = ct * sixth, cp6 = cp * sixth;
  const T Jm1 = co[C_J * BQ + fr - 1], J0 = co[C_J * BQ + fr], Jp1 = co[C_J * BQ + fr + 1];
  const T wp0 = ct6 * co[C_J * BQ + fr - 2], wp1 = T(-6) * ct6 * Jm1, wp2 = T(3) * ct6 * J0, wp3 = T(2) * ct6 * Jp1;
  const T wn0 = T(-2) * ct6 * Jm1, wn1 = T(-3) * ct6 * J0, wn2 = T(6) * ct6 * Jp1, wn3 = -ct6 * co[C_J * BQ + fr + 2];

  const T usq = ut * ut + up * up;
  const T c0 = T(1) - T(0.5) * usq;
  const T hu = T(-0.5) * usq;
  const T ntau = n * a.inv_tau, dntau = dn * a.inv_tau;
  const T Ep = co[C_EP * BQ + fr], En = co[C_EN * BQ + fr];

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // varphi-derivative operands h_m = (-F^phi - Gamma v_i v_m) g_{i m}; K~ = K diag(v) (Sec. 2.3)
    const T gvi = gam * vc.v[i];
    T h[4];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) h[mm] = (-Fp - gvi * vc.v[mm]) * g[4 * i + mm];
    const T ai = vc.v[i] * ut;
    // The BGK relaxation and the closed-form reference part share the factor w_i w_j:
    //   (f^eq - n0 w w)/tau + n0 w w [v_i (E(q) + F^theta) + v_j F^phi]
    //   = w_i w_j [ (dn + n (poly - 1))/tau + n0 v_i (E + F^theta) + n0 v_j F^phi ]
    const T ci = dntau + a.n0 * vc.v[i] * ((i >= 2 ? Ep : En) + Ft);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * i + j;
      const T* fk = sf + k * BQ * BS + bi;
      T rhs;
      if (ADV == VLB_UW3) {
        const T Dt = (i >= 2) ? wp0 * fk[-2 * BS] + wp1 * fk[-BS] + wp2 * g[k] + wp3 * fk[BS]
                              : wn0 * fk[-BS] + wn1 * g[k] + wn2 * fk[BS] + wn3 * fk[2 * BS];
        const T Dp = (j >= 2) ? (fk[-2] - T(6) * fk[-1] + T(3) * g[k] + T(2) * fk[1])
                              : (T(-2) * fk[-1] - T(3) * g[k] + T(6) * fk[1] - fk[2]);
        rhs = -(vc.v[i] * Dt) - (vc.v[j] * cp6) * Dp;
      } else {
        // WENO5 is nonlinear: theta reconstruction of the full G = J (g + n0 w_i w_j); along
        // varphi the reference part is a constant, which the reconstruction passes through.
        const T fref = a.n0 * vc.ww[i][j];
        T xt[7], xp[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) {
          xt[d] = co[C_J * BQ + fr + d - 3] * (fk[(d - 3) * BS] + fref);
          xp[d] = fk[d - 3];
        }
        const T Dt = (i >= 2) ? weno_diff<T, true>(xt) : weno_diff<T, false>(xt);
        const T Dp = (j >= 2) ? weno_diff<T, true>(xp) : weno_diff<T, false>(xp);
        rhs = -(vc.v[i] * ct) * Dt - (vc.v[j] * cp) * Dp;
      }
      // force and inertial terms on the deviation: (Gamma v_j^2 - F^theta) dg/dv_theta + sum_m K_jm h_m
      T dvt = T(0), dvp = T(0);
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        dvt += vc.K[i][mm] * g[4 * mm + j];
        dvp += vc.K[j][mm] * h[mm];
      }
      rhs += (gam * vc.v[j] * vc.v[j] - Ft) * dvt + dvp;
      // BGK towards the third-order Hermite equilibrium (Eq. feq) plus the reference part
      const T xi = ai + vc.v[j] * up;
      const T pm1 = xi * (c0 + xi * (T(0.5) + xi * sixth)) + hu;
      const T X = ntau * pm1 + (ci + a.n0 * vc.v[j] * Fp);
      rhs += vc.ww[i][j] * X - a.inv_tau * g[k];
      T o;
      if (F0) {
        const T g0 = su0[k * TQ * TS + ui];
        o = g0 + a.b * ((g[k] - g0) + rhs * a.dt);
      } else {
        o = rhs * a.dt + g[k];
      }
      a.fout[k * stride + gidx] = o;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Step 3, packed FP32 pairs: two horizontally adjacent nodes per thread, one float2 lane each, so
// the per-population arithmetic issues as FFMA2/FADD2/FMUL2 and shared/global accesses are 8 bytes.
// Same arithmetic as phase3_node, lane by lane.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// (hi, lo) <- (base, base_lo) + inc with an error-free sum, renormalised (one lane)
__device__ __forceinline__ void df_add(float base, float base_lo, float inc, float& hi, float& lo) {
  const float s1 = base + inc;
  const float bb = s1 - base;
  const float err = (base - (s1 - bb)) + (inc - bb);
  const float lo2 = base_lo + err;
  hi = s1 + lo2;
  lo = lo2 - (hi - s1);
}

// Step 2 on packed node pairs (FP32): moment-box positions (mr, mc) and (mr, mc + 1), mc even, in
// FP32x2 arithmetic; lanes: bit 0 stores the first, bit 1 the second.
template <typename L>
__device__ __forceinline__ void pair_point(const StageArgs<float>& a, const VConst<float>& vc, const float* box,
                                           const float* co, float* sm, int mr, int mc, int lanes) {
  constexpr int H = L::H, BQ = L::BQ, BS = L::BS, HS = L::HS, MS = L::MS;
  static_assert(HS % 2 == 0 && BS % 2 == 0 && MS % 2 == 0 && L::N_OFF % 2 == 0 && L::UT_OFF % 2 == 0 &&
                    L::UP_OFF % 2 == 0 && L::MU_OFF % 2 == 0,
                "pair alignment");
  const int bi = (mr + H - 1) * BS + (mc - 2 + HS);  // even
  const float* fp = box + bi;
  float2 row[4] = {f2(0.0f), f2(0.0f), f2(0.0f), f2(0.0f)}, col[4] = {f2(0.0f), f2(0.0f), f2(0.0f), f2(0.0f)};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 x = ld2(fp + (4 * i + j) * BQ * BS);
      row[i] = add2(row[i], x);
      col[j] = add2(col[j], x);
    }
  // n = n0 + sum g (the reference part carries no momentum); v_1 = -v_4, v_2 = -v_3
  const float2 dn = add2(add2(row[0], row[1]), add2(row[2], row[3]));
  const float2 mt = fma2(f2(vc.v[3]), sub2(row[3], row[0]), mul2(f2(vc.v[2]), sub2(row[2], row[1])));
  const float2 mp = fma2(f2(vc.v[3]), sub2(col[3], col[0]), mul2(f2(vc.v[2]), sub2(col[2], col[1])));
  const float2 nn = add2(f2(a.n0), dn);
  const float2 inv_n = make_float2(__frcp_rn(nn.x), __frcp_rn(nn.y));
  const float2 ut = mul2(mt, inv_n), up = mul2(mp, inv_n);
  const int cr = mr + H - 1;
  const float* pp = box + NPOP * BQ * BS + bi;
  const float* pl = box + (NPOP + 1) * BQ * BS + bi;
  const float2 ph = ld2(pp), lo = ld2(pl);
  const float2 phW = ld2(pp - 2), phE = ld2(pp + 2), loW = ld2(pl - 2), loE = ld2(pl + 2);
  // neighbour differences of phi = hi + lo: the hi differences are exact for nearby values
  float2 dN = sub2(ld2(pp + BS), ph), dS = sub2(ph, ld2(pp - BS));
  float2 dE = sub2(make_float2(ph.y, phE.x), ph), dW = sub2(ph, make_float2(phW.y, ph.x));
  dN = add2(dN, sub2(ld2(pl + BS), lo));
  dS = add2(dS, sub2(lo, ld2(pl - BS)));
  dE = add2(dE, sub2(make_float2(lo.y, loE.x), lo));
  dW = add2(dW, sub2(lo, make_float2(loW.y, lo.x)));
  const float2 lap = fma2(f2(co[C_LP * BQ + cr]), sub2(dE, dW),
                          mul2(f2(co[C_LT * BQ + cr]),
                               sub2(mul2(f2(co[C_JP * BQ + cr]), dN), mul2(f2(co[C_JM * BQ + cr]), dS))));
  // phi (1 - phi^2) at hi + lo, to first order in lo
  const float2 ph2 = mul2(ph, ph);
  const float2 cubic = fma2(sub2(f2(1.0f), mul2(f2(3.0f), ph2)), lo, mul2(ph, sub2(f2(1.0f), ph2)));
  const float2 mu = sub2(mul2(f2(-a.A), cubic), mul2(f2(a.kappa), lap));
  const int mi = mr * MS + mc;  // even
  if (lanes == 3) {
    st2(sm + L::N_OFF + mi, dn);
    st2(sm + L::UT_OFF + mi, ut);
    st2(sm + L::UP_OFF + mi, up);
    st2(sm + L::MU_OFF + mi, mu);
  } else {
    const int o = lanes == 1 ? 0 : 1;
    sm[L::N_OFF + mi + o] = o ? dn.y : dn.x;
    sm[L::UT_OFF + mi + o] = o ? ut.y : ut.x;
    sm[L::UP_OFF + mi + o] = o ? up.y : up.x;
    sm[L::MU_OFF + mi + o] = o ? mu.y : mu.x;
  }
}

// Step 2 on packed node pairs: tile columns 0 .. TS-1 of every moment row two at a time; the halo
// columns -1 and TS of the tile rows inside the aligned pairs (-2, -1) and (TS, TS + 1), keeping
// one lane, so that every column takes the same sequence of FP32 operations (an axisymmetric
// state stays bitwise axisymmetric).  The pairs' other lanes read box columns -4 .. TS + 3, inside
// the HS = 4 halo.
template <typename L>
__device__ __forceinline__ void phase2_pair(const StageArgs<float>& a, const VConst<float>& vc, const float* box,
                                            const float* co, float* sm, int tid) {
  constexpr int MQ = L::MQ, TQ = L::TQ, NP = MQ * (TS / 2), NSGL = 2 * TQ;
  static_assert(L::HS >= 4, "the halo pairs read two columns beyond the halo column");
  for (int idx = tid; idx < NP + NSGL; idx += L::NTH) {
    int mr, mc, lanes = 3;
    if (idx < NP) {
      mr = idx / (TS / 2);
      mc = 2 + 2 * (idx - mr * (TS / 2));
    } else {  // column TS: first lane of (TS, TS + 1); column -1: second lane of (-2, -1)
      const int j = idx - NP;
      mr = 1 + (j >> 1);
      mc = (j & 1) ? TS + 2 : 0;
      lanes = (j & 1) ? 1 : 2;
    }
    pair_point<L>(a, vc, box, co, sm, mr, mc, lanes);
  }
}

template <typename L, int CH, bool F0>
__device__ __forceinline__ void phase3_pair(const StageArgs<float>& a, const VConst<float>& vc, const float* box,
                                            const float* co, const float* sm, int lr, int lc, int q, int s) {
  constexpr int H = L::H, BQ = L::BQ, BS = L::BS, HS = L::HS, MS = L::MS, TQ = L::TQ;
  static_assert(HS % 2 == 0 && BS % 2 == 0 && MS % 2 == 0, "pair alignment");
  const float* sf = box;
  const float* sphi = box + NPOP * BQ * BS;
  const float* sphl = box + (NPOP + 1) * BQ * BS;
  const float* su0 = sm + L::U0_OFF;
  const float* sn = sm + L::N_OFF;
  const float* sut = sm + L::UT_OFF;
  const float* sup = sm + L::UP_OFF;
  const float* smu = sm + L::MU_OFF;
  const int64_t stride = a.stride;
  const int fr = lr + H;
  const int bi = fr * BS + lc + HS;       // even: 8-byte aligned pairs
  const int mi = (lr + 1) * MS + lc + 2;  // even
  const int ui = lr * TS + lc;
  const float sixth = 1.0f / 6.0f;

  const float2 dn = ld2(sn + mi), ut = ld2(sut + mi), up = ld2(sup + mi), ph = ld2(sphi + bi);
  const float2 n = add2(dn, f2(a.n0));
  const float ct = co[C_CT * BQ + fr], cp = co[C_CP * BQ + fr], gam = co[C_GAM * BQ + fr];
  const float lt = co[C_LT * BQ + fr], lp = co[C_LP * BQ + fr];
  const float Jp = co[C_JP * BQ + fr], Jm = co[C_JM * BQ + fr];
  const float2 muC = ld2(smu + mi), muN = ld2(smu + mi + MS), muS = ld2(smu + mi - MS);
  const float2 muL = ld2(smu + mi - 2), muR = ld2(smu + mi + 2);
  const float2 muE = make_float2(muC.y, muR.x), muW = make_float2(muL.y, muC.x);

  // Cahn-Hilliard: M Delta mu - div(u phi) (Eq. CH), flux form with mean face values
  float2 lapmu = mul2(f2(lt), sub2(mul2(f2(Jp), sub2(muN, muC)), mul2(f2(Jm), sub2(muC, muS))));
  lapmu = fma2(f2(lp), add2(sub2(muE, muC), sub2(muW, muC)), lapmu);
  float2 Lphi = mul2(f2(a.M), lapmu);
  float2 Ft = f2(0.0f), Fp = f2(0.0f);
  if (CH == VLB_HYDRO) {
    const float2 Xn = mul2(f2(co[C_J * BQ + fr + 1]), mul2(ld2(sut + mi + MS), ld2(sphi + bi + BS)));
    const float2 Xs = mul2(f2(co[C_J * BQ + fr - 1]), mul2(ld2(sut + mi - MS), ld2(sphi + bi - BS)));
    const float2 upL = ld2(sup + mi - 2), upR = ld2(sup + mi + 2);
    const float2 phL = ld2(sphi + bi - 2), phR = ld2(sphi + bi + 2);
    const float2 Ye = mul2(make_float2(up.y, upR.x), make_float2(ph.y, phR.x));
    const float2 Yw = mul2(make_float2(upL.y, up.x), make_float2(phL.y, ph.x));
    Lphi = sub2(Lphi, mul2(f2(0.5f), fma2(f2(ct), sub2(Xn, Xs), mul2(f2(cp), sub2(Ye, Yw)))));
    // n F = -phi grad mu (Eq. pbin), central differences
    const float2 mpn = make_float2(-ph.x * __frcp_rn(n.x), -ph.y * __frcp_rn(n.y));
    Ft = mul2(mul2(mpn, sub2(muN, muS)), f2(a.gt));
    Fp = mul2(mul2(mpn, sub2(muE, muW)), f2(co[C_GP * BQ + fr]));
  }

  const int64_t gidx = (int64_t)q * a.ns + s;  // even
  if (a.dphi) {
    st2(a.dphi + gidx, mul2(Lphi, f2(a.dt)));  // the stabilised Cahn-Hilliard solve forms phi
  } else {
    const float2 lo = ld2(sphl + bi);
    float2 base = ph, base_lo = lo, inc = mul2(Lphi, f2(a.dt));
    if (F0) {
      base = ld2(su0 + NPOP * TQ * TS + ui);
      base_lo = ld2(su0 + (NPOP + 1) * TQ * TS + ui);
      inc = mul2(f2(a.b), fma2(Lphi, f2(a.dt), add2(sub2(ph, base), sub2(lo, base_lo))));
    }
    float2 hi_o, lo_o;
    df_add(base.x, base_lo.x, inc.x, hi_o.x, lo_o.x);
    df_add(base.y, base_lo.y, inc.y, hi_o.y, lo_o.y);
    st2(a.fout + NPOP * stride + gidx, hi_o);
    st2(a.fout + (NPOP + 1) * stride + gidx, lo_o);
  }

  float2 g[NPOP];
#pragma unroll
  for (int k = 0; k < NPOP; ++k) g[k] = ld2(sf + k * BQ * BS + bi);

  // UW3 theta weights with ct/6 folded in (same row for both lanes)
  const float ct6 = ct * sixth, cp6 = cp * sixth;
  const float Jm1 = co[C_J * BQ + fr - 1], J0 = co[C_J * BQ + fr], Jp1 = co[C_J * BQ + fr + 1];
  const float wp0 = ct6 * co[C_J * BQ + fr - 2], wp1 = -6.0f * ct6 * Jm1, wp2 = 3.0f * ct6 * J0, wp3 = 2.0f * ct6 * Jp1;
  const float wn0 = -2.0f * ct6 * Jm1, wn1 = -3.0f * ct6 * J0, wn2 = 6.0f * ct6 * Jp1, wn3 = -ct6 * co[C_J * BQ + fr + 2];

  const float2 usq = fma2(ut, ut, mul2(up, up));
  const float2 hu = mul2(f2(-0.5f), usq);
  const float2 c0 = add2(f2(1.0f), hu);
  const float2 ntau = mul2(n, f2(a.inv_tau)), dntau = mul2(dn, f2(a.inv_tau));
  const float Ep = co[C_EP * BQ + fr], En = co[C_EN * BQ + fr];
  float2 cj[4], nFp[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cj[j] = sub2(f2(gam * vc.v[j] * vc.v[j]), Ft);  // Gamma v_j^2 - F^theta
    nFp[j] = mul2(f2(a.n0 * vc.v[j]), Fp);           // n0 v_j F^phi
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // h_m = (-F^phi - Gamma v_i v_m) g_{i m}  (K~ = K diag v, Sec. 2.3)
    float2 h[4];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) h[mm] = mul2(sub2(f2(-gam * vc.v[i] * vc.v[mm]), Fp), g[4 * i + mm]);
    const float2 ai = mul2(f2(vc.v[i]), ut);
    // BGK relaxation and the closed-form reference part share w_i w_j
    const float2 ci = fma2(f2(a.n0 * vc.v[i]), add2(f2(i >= 2 ? Ep : En), Ft), dntau);
    // theta-advection weights of this velocity row with -v_i folded in (upwind side by sign(v_i))
    const float mvi = -vc.v[i];
    const float t0 = mvi * (i >= 2 ? wp0 : wn0), t1 = mvi * (i >= 2 ? wp1 : wn1);
    const float t2 = mvi * (i >= 2 ? wp2 : wn2), t3 = mvi * (i >= 2 ? wp3 : wn3);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * i + j;
      const float* fk = sf + k * BQ * BS + bi;
      const float2 gk = g[k];
      float2 rhs;  // -v_i (theta flux difference) - v_j (varphi flux difference) / (R J dvarphi)
      if (i >= 2)
        rhs = fma2(f2(t3), ld2(fk + BS), fma2(f2(t2), gk, fma2(f2(t1), ld2(fk - BS), mul2(f2(t0), ld2(fk - 2 * BS)))));
      else
        rhs = fma2(f2(t3), ld2(fk + 2 * BS), fma2(f2(t2), ld2(fk + BS), fma2(f2(t1), gk, mul2(f2(t0), ld2(fk - BS)))));
      const float2 A = ld2(fk - 2), C = ld2(fk + 2);
      const float2 M1 = make_float2(A.y, gk.x), M2 = make_float2(gk.y, C.x);
      float2 Dp;
      if (j >= 2)
        Dp = fma2(f2(2.0f), M2, fma2(f2(3.0f), gk, fma2(f2(-6.0f), M1, A)));
      else
        Dp = sub2(fma2(f2(6.0f), M2, fma2(f2(-3.0f), gk, mul2(f2(-2.0f), M1))), C);
      rhs = fma2(f2(-vc.v[j] * cp6), Dp, rhs);
      float2 dvt = mul2(f2(vc.K[i][0]), g[j]);
#pragma unroll
      for (int mm = 1; mm < 4; ++mm) dvt = fma2(f2(vc.K[i][mm]), g[4 * mm + j], dvt);
      rhs = fma2(cj[j], dvt, rhs);
      // the K~ term accumulates straight into the right-hand side
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) rhs = fma2(f2(vc.K[j][mm]), h[mm], rhs);
      // BGK towards the third-order Hermite equilibrium (Eq. feq) plus the reference part
      const float2 xi = fma2(f2(vc.v[j]), up, ai);
      const float2 pm1 = fma2(xi, fma2(xi, fma2(xi, f2(sixth), f2(0.5f)), c0), hu);
      const float2 X = fma2(ntau, pm1, add2(ci, nFp[j]));
      rhs = fma2(f2(-a.inv_tau), gk, fma2(f2(vc.ww[i][j]), X, rhs));
      float2 o;
      if (F0) {
        const float2 g0 = ld2(su0 + k * TQ * TS + ui);
        o = fma2(f2(a.b), fma2(rhs, f2(a.dt), sub2(gk, g0)), g0);
      } else {
        o = fma2(rhs, f2(a.dt), gk);
      }
      st2(a.fout + k * stride + gidx, o);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------------

// Steps 1-3 for one tile.  PM: 0 = scalar step 3 (two or more nodes per thread), 1 = packed node
// pairs, 2 = decided at run time from the grid (pairs when the chunked layout applies, FP32 UW3).
template <typename L, typename T, int ADV, int CH, bool F0, int PM>
__device__ __forceinline__ void tile_body(const StageArgs<T>& a, const VConst<T>& vc, T* sm, int tid, int q0, int s0) {
  T* box = sm + L::BOX_OFF;
  T* co = sm + L::CO_OFF;
  pdl_wait();  // the coefficients too may come from the previous kernel (the scratch tables of vlb_step_noalloc)
  issue_co<L>(a, co, q0, tid);
  issue_box<L>(a, box, co, q0, s0, tid);
  cp_async_commit();
  if (F0) issue_u0<L>(a, sm + L::U0_OFF, q0, s0, tid);
  cp_async_commit();
  cp_async_wait<1>();  // the box; U^n may still be in flight
  __syncthreads();
  bool pair = PM == 1;
  if constexpr (PM == 2) pair = chunked<L>(a.nt, a.ns);
  if constexpr (PM != 0 && sizeof(T) == 4 && ADV == VLB_UW3) {
    if (pair)
      phase2_pair<L>(a, vc, box, co, sm, tid);
    else
      phase2<L>(a, vc, box, co, sm, tid);
  } else {
    phase2<L>(a, vc, box, co, sm, tid);
  }
  cp_async_wait<0>();
  __syncthreads();
  pdl_trigger();
  if constexpr (PM != 0 && sizeof(T) == 4 && ADV == VLB_UW3) {
    if (pair) {
      static_assert(L::NTH == L::TQ * (TS / 2), "one node pair per thread");
      const int lr = tid / (TS / 2), lc = 2 * (tid % (TS / 2));
      const int q = q0 + lr, s = s0 + lc;  // n_phi is even, so s + 1 < n_phi whenever s < n_phi
      if (q < a.nt && s < a.ns) phase3_pair<L, CH, F0>(a, vc, box, co, sm, lr, lc, q, s);
      return;
    }
  }
  constexpr int ROWS = L::NTH / TS;  // thread rows; each thread takes TQ / ROWS nodes of its column
#pragma unroll 1
  for (int m = 0; m < L::TQ / ROWS; ++m) {
    const int lr = tid / TS + ROWS * m, lc = tid % TS;
    const int q = q0 + lr, s = s0 + lc;
    if (q < a.nt && s < a.ns) phase3_node<L, T, ADV, CH, F0>(a, vc, box, co, sm, lr, lc, q, s);
  }
}

// Steps 1-3 for an interior tile (box inside the grid, no wrap-around) of the FP32 UW3 pair path,
// with the box and the U^n tile staged by two tensor-map copies issued by one thread and
// completing on two mbarriers.  The layout in shared memory is the one issue_box / issue_u0 produce.
// A persistent CTA (which stages many tiles) initialises the two mbarriers once and passes init =
// false with the parity of each barrier's current phase.
template <typename L, int CH, bool F0>
__device__ __forceinline__ void tile_body_tma(const StageArgs<float>& a, const VConst<float>& vc, float* sm, int tid,
                                              int q0, int s0, const CUtensorMap* tmb, const CUtensorMap* tmu,
                                              bool init = true, unsigned ph_box = 0, unsigned ph_u0 = 0) {
  constexpr unsigned BOX_BYTES = sizeof(float) * L::NST * L::BQ * L::BS;
  constexpr unsigned U0_BYTES = sizeof(float) * L::NST * L::TQ * TS;
  static_assert((L::BOX_OFF * sizeof(float)) % 128 == 0 && (L::U0_OFF * sizeof(float)) % 128 == 0,
                "tensor-map destinations are 128-byte aligned");
  static_assert((L::MB_OFF * sizeof(float)) % 8 == 0, "mbarriers are 8-byte aligned");
  float* box = sm + L::BOX_OFF;
  float* co = sm + L::CO_OFF;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::MB_OFF);
  if (init) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  pdl_wait();
  issue_co<L>(a, co, q0, tid);
  cp_async_commit();
  if (tid == 0) {
    mbar_expect_tx(bar, BOX_BYTES);
    tma_load_3d(box, tmb, bar, s0 - L::HS, q0 - L::H, 0);
    if (F0) {
      mbar_expect_tx(bar + 1, U0_BYTES);
      tma_load_3d(sm + L::U0_OFF, tmu, bar + 1, s0, q0, 0);
    }
    // Software pipelining through L2: the CTA that starts a.ahead tiles later (linear tile index,
    // about half a wave) will find its box and U^n tile already on chip.
    const int tiles_s = (a.ns + TS - 1) / TS;
    const int nxt = (q0 / L::TQ) * tiles_s + s0 / TS + a.ahead;
    const int qn = (nxt / tiles_s) * L::TQ, sn = (nxt % tiles_s) * TS;
    if (a.ahead > 0 && qn >= L::H && qn + L::TQ + L::H <= a.nt && sn >= L::HS && sn + TS + L::HS <= a.ns) {
      tma_prefetch_3d(tmb, sn - L::HS, qn - L::H, 0);
      if (F0) tma_prefetch_3d(tmu, sn, qn, 0);
    }
  }
  cp_async_wait<0>();
  bool ok = mbar_wait(bar, ph_box);
  if (__syncthreads_or(!ok)) {  // a copy did not land: flag it, let the copies settle, skip the tile
    if (tid == 0) {
      if (a.err) atomicExch(a.err, 2);
      mbar_wait(bar, ph_box);
      if (F0) mbar_wait(bar + 1, ph_u0);
    }
    return;
  }
  phase2_pair<L>(a, vc, box, co, sm, tid);
  ok = F0 ? mbar_wait(bar + 1, ph_u0) : true;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      if (a.err) atomicExch(a.err, 2);
      mbar_wait(bar + 1, ph_u0);
    }
    return;
  }
  pdl_trigger();
  const int lr = tid / (TS / 2), lc = 2 * (tid % (TS / 2));
  phase3_pair<L, CH, F0>(a, vc, box, co, sm, lr, lc, q0 + lr, s0 + lc);
}

// One CTA per 16 x 32 tile.
// F0: the stage combines with U^n (stages 2 and 3); the first stage writes U_in + dt L(U_in).
// PAIR: step 3 on packed node pairs (FP32, UW3, chunked layout); otherwise two scalar nodes per
// thread (rows lr and lr + 8).
// TMA: interior tiles are staged by tensor-map copies (tmb: the box of fin, tmu: the tile of f0);
// tiles whose box wraps around the grid take the per-thread copies.
template <typename T, int ADV, int CH, bool F0, bool PAIR, bool TMA>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    stage_kernel(StageArgs<T> a, VConst<T> vc, const __grid_constant__ CUtensorMap tmb,
                 const __grid_constant__ CUtensorMap tmu) {
  using L = GenericLay<T, ADV>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int q0 = blockIdx.y * L::TQ, s0 = blockIdx.x * TS;
  if constexpr (TMA && sizeof(T) == 4 && ADV == VLB_UW3 && PAIR) {
    if (q0 >= L::H && q0 + L::TQ + L::H <= a.nt && s0 >= L::HS && s0 + TS + L::HS <= a.ns) {
      tile_body_tma<L, CH, F0>(a, vc, sm, threadIdx.x, q0, s0, &tmb, &tmu);
      return;
    }
  }
  tile_body<L, T, ADV, CH, F0, PAIR ? 1 : 0>(a, vc, sm, threadIdx.x, q0, s0);
}

// Ensemble: one launch per stage over the tiles of every member (FP32, UW3).  Block b takes work
// item items[b] = (member, tile index within the member); the member's buffers, grid and scalars
// come from its descriptor, so members of different sizes, aspect ratios and time steps share the
// launch.  TQR is the tile height chosen by the autotuner (16 or 8 rows).
template <int TQR>
using EnsLay = Lay<float, 2, TQR, 4, TQR * (TS / 2), 1>;

// With 16-row tiles, interior tiles of members that have tensor maps are staged by the bulk copies
// of tile_body_tma, and each block prefetches into L2 the work item `ahead` blocks later.
template <int TQR, int CH, bool F0>
__global__ void __launch_bounds__(TQR * (TS / 2)) ensemble_stage_kernel(const EnsembleMember* members,
                                                                       const int2* items, int nitems, int ahead,
                                                                       int stage, int* err, VConst<float> vc,
                                                                       const __grid_constant__ EnsembleMaps maps) {
  using L = EnsLay<TQR>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int2 it = items[blockIdx.x];
  const EnsembleMember& d = members[it.x];
  StageArgs<float> a;
  a.fin = d.U[stage == 0 ? 0 : stage];  // stage 0 reads U^n, 1 reads U^(1), 2 reads U^(2)
  a.f0 = F0 ? d.U[0] : nullptr;
  a.fout = d.U[stage == 2 ? 0 : stage + 1];
  a.coef = d.coef;
  a.nt = d.nt;
  a.ns = d.ns;
  a.stride = d.stride;
  a.b = stage == 0 ? 1.0f : (stage == 1 ? 0.25f : 2.0f / 3.0f);
  a.dt = d.dt;
  a.inv_tau = d.inv_tau;
  a.M = d.M;
  a.A = d.A;
  a.kappa = d.kappa;
  a.gt = d.gt;
  a.n0 = d.n0;
  a.err = err;
  a.ahead = 0;
  const int tiles_s = (d.ns + TS - 1) / TS;
  const int q0 = (it.y / tiles_s) * TQR, s0 = (it.y % tiles_s) * TS;
  if constexpr (TQR == 16) {
    if (threadIdx.x == 0 && ahead > 0 && blockIdx.x + ahead < nitems) {
      const int2 nx = items[blockIdx.x + ahead];
      const EnsembleMember& e = members[nx.x];
      const int ts = (e.ns + TS - 1) / TS, qn = (nx.y / ts) * TQR, sn = (nx.y % ts) * TS;
      if (e.maps >= 0 && qn >= L::H && qn + TQR + L::H <= e.nt && sn >= L::HS && sn + TS + L::HS <= e.ns) {
        tma_prefetch_3d(&maps.m[e.maps + stage], sn - L::HS, qn - L::H, 0);
        if (F0) tma_prefetch_3d(&maps.m[e.maps + 3], sn, qn, 0);
      }
    }
    if (d.maps >= 0 && q0 >= L::H && q0 + TQR + L::H <= d.nt && s0 >= L::HS && s0 + TS + L::HS <= d.ns) {
      tile_body_tma<L, CH, F0>(a, vc, sm, threadIdx.x, q0, s0, &maps.m[d.maps + stage], &maps.m[d.maps + 3]);
      return;
    }
  }
  tile_body<L, float, VLB_UW3, CH, F0, 2>(a, vc, sm, threadIdx.x, q0, s0);
}

// ---------------------------------------------------------------------------------------------
// Persistent ensemble: one cooperative launch runs whole steps.  Its CTAs (all resident at once)
// take the work items of a stage from a ticket counter and meet at a grid barrier before the next
// stage.
// The barrier is a counter and a generation word in global memory; a CTA waits for the generation
// to change for at most `budget` SM clock cycles.  On expiry it raises the ensemble's flag (2), and
// every CTA that sees the flag raised while waiting returns, so a CTA that never arrives (a lost
// CTA, or the test hook skip_cta) ends the launch with an error status instead of a hang.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
// ordering between this thread's generic-proxy accesses and later bulk (async-proxy) copies
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;\n" ::: "memory"); }

// bar[0]: arrivals, bar[1]: generation, bar[2 + k]: the work-item tickets of stages k = 0, 1 (mod 2).
// The last CTA to arrive resets the ticket counter `reset` for the stage after the barrier before it
// releases the others.  Returns false if the barrier gave up (flag raised).
__device__ bool grid_barrier(unsigned* bar, int* err, long long budget, bool skip, int* s_ok, int reset) {
  fence_proxy_async_all();  // this thread's stores of the stage, before the next stage's bulk copies
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire_u32(bar + 1);  // the generation cannot change before this CTA arrives
    __threadfence();                              // the CTA's stores (ordered by the CTA barrier) first
    if (!skip && atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      atomicExch(bar + 2 + reset, 0u);
      st_release_u32(bar + 1, g + 1u);
    }
    const long long t0 = clock64();
    while (ld_acquire_u32(bar + 1) == g) {
      if (ld_volatile_i32(err) == 2) {  // another CTA gave up
        ok = 0;
        break;
      }
      if (clock64() - t0 > budget) {
        atomicCAS(err, 0, 2);
        atomicCAS(err, 1, 2);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    fence_proxy_async_all();  // the other CTAs' stores, before this CTA's bulk copies read them
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ StageArgs<float> member_args(const EnsembleMember& d, int stage, int* err) {
  StageArgs<float> a;
  a.fin = d.U[stage == 0 ? 0 : stage];  // stage 0 reads U^n, 1 reads U^(1), 2 reads U^(2)
  a.f0 = stage == 0 ? nullptr : d.U[0];
  a.fout = d.U[stage == 2 ? 0 : stage + 1];
  a.coef = d.coef;
  a.nt = d.nt;
  a.ns = d.ns;
  a.stride = d.stride;
  a.b = stage == 0 ? 1.0f : (stage == 1 ? 0.25f : 2.0f / 3.0f);
  a.dt = d.dt;
  a.inv_tau = d.inv_tau;
  a.M = d.M;
  a.A = d.A;
  a.kappa = d.kappa;
  a.gt = d.gt;
  a.n0 = d.n0;
  a.err = err;
  a.ahead = 0;
  return a;
}

// nsteps whole steps, or with only0 nsteps passes of the first stage alone (which writes only the
// scratch U^(1), so the autotuner can time it without advancing the state).
template <int TQR, int CH>
__global__ void __launch_bounds__(TQR * (TS / 2), TQR == 16 ? 2 : 3) ensemble_persistent_kernel(
    const EnsembleMember* members, const int2* items, int nitems, int nsteps, int only0, unsigned* bar, int* err,
    long long budget, int skip_cta, VConst<float> vc, const __grid_constant__ EnsembleMaps maps) {
  using L = EnsLay<TQR>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_ok;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x;
  if (TQR == 16 && tid == 0) {
    uint64_t* mb = reinterpret_cast<uint64_t*>(sm + L::MB_OFF);
    mbar_init(mb, 1);
    mbar_init(mb + 1, 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned ph_box = 0, ph_u0 = 0;
  const bool skip = (int)blockIdx.x == skip_cta;
  __shared__ int s_next, s_next2;
  int gstage = 0;  // stages run so far in this launch: the ticket counter alternates between two words
  for (int n = 0; n < nsteps; ++n) {
    for (int stage = 0; stage <= (only0 ? 0 : 2); ++stage, ++gstage) {
      if (gstage > 0 && !grid_barrier(bar, err, budget, skip, &s_ok, gstage & 1)) return;
      unsigned* tickets = bar + 2 + (gstage & 1);
      // work items are handed out by a ticket counter: a CTA holds the tickets of its current and its
      // next item, so that the next item's box can be prefetched into L2 and the counter's latency
      // overlaps the current tile
      if (tid == 0) {
        s_next = (int)atomicAdd(tickets, 1u);
        s_next2 = (int)atomicAdd(tickets, 1u);
      }
      __syncthreads();
      int w = s_next, nxw = s_next2;
      while (w < nitems) {
        fence_proxy_async_all();  // the previous tile's shared-memory reads, before new copies land
        __syncthreads();          // ... and every thread has read s_next
        const int2 it = items[w];
        const EnsembleMember& d = members[it.x];
        const StageArgs<float> a = member_args(d, stage, err);
        const int tiles_s = (d.ns + TS - 1) / TS;
        const int q0 = (it.y / tiles_s) * TQR, s0 = (it.y % tiles_s) * TS;
        int after = 0;
        if (tid == 0) {
          after = (int)atomicAdd(tickets, 1u);  // used only at the end of the tile
          if (TQR == 16 && nxw < nitems) {      // the next tile of this CTA, into L2
            const int2 nx = items[nxw];
            const EnsembleMember& e = members[nx.x];
            const int ts = (e.ns + TS - 1) / TS, qn = (nx.y / ts) * TQR, sn = (nx.y % ts) * TS;
            if (e.maps >= 0 && qn >= L::H && qn + TQR + L::H <= e.nt && sn >= L::HS && sn + TS + L::HS <= e.ns) {
              tma_prefetch_3d(&maps.m[e.maps + stage], sn - L::HS, qn - L::H, 0);
              if (stage > 0) tma_prefetch_3d(&maps.m[e.maps + 3], sn, qn, 0);
            }
          }
        }
        bool tma = false;
        if constexpr (TQR == 16) {
          tma = d.maps >= 0 && q0 >= L::H && q0 + TQR + L::H <= d.nt && s0 >= L::HS && s0 + TS + L::HS <= d.ns;
          if (tma) {
            if (stage == 0)
              tile_body_tma<L, CH, false>(a, vc, sm, tid, q0, s0, &maps.m[d.maps], &maps.m[d.maps + 3], false, ph_box,
                                          ph_u0);
            else
              tile_body_tma<L, CH, true>(a, vc, sm, tid, q0, s0, &maps.m[d.maps + stage], &maps.m[d.maps + 3], false,
                                         ph_box, ph_u0);
            ph_box ^= 1u;
            if (stage > 0) ph_u0 ^= 1u;
          }
        }
        if (!tma) {
          if (stage == 0)
            tile_body<L, float, VLB_UW3, CH, false, 2>(a, vc, sm, tid, q0, s0);
          else
            tile_body<L, float, VLB_UW3, CH, true, 2>(a, vc, sm, tid, q0, s0);
        }
        if (tid == 0) s_next = after;
        __syncthreads();
        w = nxw;
        nxw = s_next;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Wavefront schedule (FP32 UW3, one torus): `nsteps` whole SSP-RK3 steps in one persistent launch,
// so that the two intermediate stages of a step are consumed from L2 instead of HBM.
//
// A band is the 16 rows of one row of tiles (nb = n_theta / 16 bands, tiles_s tiles each).  Sweep
// sigma = 3 n + k (step n, stage k) visits the bands in the rotated order b = (sigma + i) mod nb,
// i = 0 .. nb - 1, and stage k of band b may run once stage k - 1 (stage 2 of step n - 1 for k = 0)
// has finished bands b - 1, b, b + 1 (the stencil reaches 2 rows, under one band).  The rotation
// makes position i of a sweep depend only on positions i .. i + 2 of the previous sweep, also across
// the periodic seam.  Band item (n, k, i) is placed in slot n nb + k lag + i, and CTAs take tiles from
// one ticket counter in slot order (stage 2 first within a slot), so that the three sweeps of a step
// trail each other by `lag` bands: the U^(1) and U^(2) a band produces is read again within about
// 2 lag bands of work, while the state U^n is read once and written once per step from HBM.
// Every dependency sits in an earlier slot when lag >= 3 and nb > 2 lag + 2, and the CTAs are all
// resident (cooperative launch), so the CTA holding the oldest unfinished ticket can always proceed.
//
// cnt[k nb + b] counts the finished tiles of stage k in band b over the launch (monotone); a wait
// polls it with acquire loads for at most `budget` SM cycles, then raises err (2) and returns, and
// every CTA that sees err == 2 while waiting returns too.  Once no reader of an intermediate band is
// left (stage 2 of band b has waited for stage 1 of b - 1 .. b + 1; stage 0 of the next step for
// stage 2 of the previous one), its lines are discarded from L2 without write-back.
// ---------------------------------------------------------------------------------------------
struct WaveMaps {
  CUtensorMap box[3];  // halo boxes of U^n, U^(1), U^(2)
  CUtensorMap tile;    // the U^n tile
};

// Band item j (0 <= j < 3 nsteps nb) in ticket order -> (n, k, i).  Slots [0, lag) hold stage 0
// only, [lag, 2 lag) stages 1, 0, [2 lag, nsteps nb) stages 2, 1, 0, then stages 2, 1 for lag
// slots and stage 2 alone for lag slots (requires nsteps nb >= 2 lag).
__host__ __device__ __forceinline__ void wave_decode(int j, int nb, int lag, int nsteps, int& n, int& k, int& i) {
  int s;
  const int steady_end = 3 * lag + 3 * (nsteps * nb - 2 * lag);
  if (j < lag) {
    s = j;
    k = 0;
  } else if (j < 3 * lag) {
    s = lag + (j - lag) / 2;
    k = 1 - (j - lag) % 2;
  } else if (j < steady_end) {
    s = 2 * lag + (j - 3 * lag) / 3;
    k = 2 - (j - 3 * lag) % 3;
  } else {
    const int jj = j - steady_end;
    if (jj < 2 * lag) {
      s = nsteps * nb + jj / 2;
      k = 2 - jj % 2;
    } else {
      s = nsteps * nb + lag + (jj - 2 * lag);
      k = 2;
    }
  }
  const int x = s - k * lag;
  n = x / nb;
  i = x - n * nb;
}

// waits until *c >= need; false if the wait gave up or another CTA did
__device__ __forceinline__ bool wave_wait(const unsigned* c, unsigned need, int* err, long long budget) {
  if (ld_acquire_u32(c) >= need) return true;
  const long long t0 = clock64();
  while (ld_acquire_u32(c) < need) {
    if (ld_volatile_i32(err) == 2) return false;
    if (clock64() - t0 > budget) {
      atomicCAS(err, 0, 2);
      atomicCAS(err, 1, 2);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// the 18 state arrays of one 16 x 32 tile (128-byte row segments) leave L2 without write-back
__device__ __forceinline__ void discard_tile(const float* U, int64_t stride, int ns, int q0, int s0, int tid) {
  constexpr int LINES = (NARR + 1) * 16;
  for (int l = tid; l < LINES; l += 256) {
    const int arr = l / 16, row = l % 16;
    const float* p = U + arr * stride + (int64_t)(q0 + row) * ns + s0;
    asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p) : "memory");
  }
}

template <int CH>
__global__ void __launch_bounds__(256, 2) wave_kernel(StageArgs<float> base, float* U0, float* U1, float* U2,
                                                      int nsteps, int lag, unsigned* cnt, int* err, long long budget,
                                                      int skip_cta, VConst<float> vc,
                                                      const __grid_constant__ WaveMaps maps) {
  using L = GenericLay<float, VLB_UW3>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_item[2], s_go;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x;
  const int nb = base.nt / L::TQ, tiles_s = base.ns / TS;
  const int total = 3 * nsteps * nb * tiles_s;
  unsigned* tickets = cnt + 3 * nb;
  if (tid == 0) {
    uint64_t* mb = reinterpret_cast<uint64_t*>(sm + L::MB_OFF);
    mbar_init(mb, 1);
    mbar_init(mb + 1, 1);
    fence_mbar_init();
    s_item[0] = (int)atomicAdd(tickets, 1u);
    s_item[1] = (int)atomicAdd(tickets, 1u);
  }
  __syncthreads();
  unsigned ph_box = 0, ph_u0 = 0;
  int t = s_item[0], tn = s_item[1];
  while (t < total) {
    const int j = t / tiles_s, c = t - j * tiles_s;
    int n, k, i;
    wave_decode(j, nb, lag, nsteps, n, k, i);
    const int b = (3 * n + k + i) % nb;
    const int q0 = b * L::TQ, s0 = c * TS;
    if (tid == 0) {
      // dependencies: the previous sweep on bands b - 1, b, b + 1
      bool ok = true;
      const int kp = k == 0 ? 2 : k - 1;
      const unsigned need = (unsigned)((k == 0 ? n : n + 1) * tiles_s);
      if (k > 0 || n > 0) {
        for (int d = -1; d <= 1 && ok; ++d) ok = wave_wait(cnt + kp * nb + (b + d + nb) % nb, need, err, budget);
      }
      fence_proxy_async_all();  // the other CTAs' stores, before this CTA's bulk copies read them
      // the next tile of this CTA, into L2 (a hint: its inputs may not be final yet)
      if (ok && tn < total) {
        const int jn = tn / tiles_s, cn = tn - jn * tiles_s;
        int nn, kn, in_;
        wave_decode(jn, nb, lag, nsteps, nn, kn, in_);
        const int qn = ((3 * nn + kn + in_) % nb) * L::TQ, sn = cn * TS;
        if (qn >= L::H && qn + L::TQ + L::H <= base.nt && sn >= L::HS && sn + TS + L::HS <= base.ns) {
          tma_prefetch_3d(&maps.box[kn], sn - L::HS, qn - L::H, 0);
          if (kn > 0) tma_prefetch_3d(&maps.tile, sn, qn, 0);
        }
      }
      s_go = ok;
      s_item[0] = (int)atomicAdd(tickets, 1u);  // the ticket after next, used at the end of the tile
    }
    __syncthreads();
    if (!s_go) return;
    // no reader of these intermediate bands is left
    if (k == 2) discard_tile(U1, base.stride, base.ns, q0, s0, tid);
    if (k == 0 && n > 0) discard_tile(U2, base.stride, base.ns, q0, s0, tid);
    StageArgs<float> a = base;
    a.fin = k == 0 ? U0 : (k == 1 ? U1 : U2);
    a.f0 = k == 0 ? nullptr : U0;
    a.fout = k == 0 ? U1 : (k == 1 ? U2 : U0);
    a.b = k == 0 ? 1.0f : (k == 1 ? 0.25f : 2.0f / 3.0f);
    a.ahead = 0;
    a.err = err;
    const bool tma = q0 >= L::H && q0 + L::TQ + L::H <= a.nt && s0 >= L::HS && s0 + TS + L::HS <= a.ns;
    if (tma) {
      if (k == 0)
        tile_body_tma<L, CH, false>(a, vc, sm, tid, q0, s0, &maps.box[0], &maps.tile, false, ph_box, ph_u0);
      else
        tile_body_tma<L, CH, true>(a, vc, sm, tid, q0, s0, &maps.box[k], &maps.tile, false, ph_box, ph_u0);
      ph_box ^= 1u;
      if (k > 0) ph_u0 ^= 1u;
    } else {
      if (k == 0)
        tile_body<L, float, VLB_UW3, CH, false, 1>(a, vc, sm, tid, q0, s0);
      else
        tile_body<L, float, VLB_UW3, CH, true, 1>(a, vc, sm, tid, q0, s0);
    }
    // this tile's stores, before the consumers' bulk copies; the CTA's shared-memory reads, before
    // the next tile's copies land
    fence_proxy_async_all();
    __syncthreads();
    if (ld_volatile_i32(err) == 2) return;  // a copy of this CTA (or another) gave up
    if (tid == 0 && (int)blockIdx.x != skip_cta) {  // skip_cta: test hook, a CTA that never reports
      __threadfence();
      red_release_add(cnt + k * nb + b, 1u);
    }
    t = tn;
    tn = s_item[0];
    __syncthreads();  // every thread has read s_item before thread 0 rewrites it
  }
}

// ---------------------------------------------------------------------------------------------
// Axisymmetric special case, n_phi = 1.  With one varphi column every varphi difference is zero:
// the varphi flux of f and of u^phi phi, the varphi part of the Laplace-Beltrami operator and the
// force component F^phi all vanish, while u^phi itself (a swirl) and the inertial terms through
// Gamma and K~ remain.  One CTA holds the column: per Runge-Kutta stage it computes the moments
// and mu of every node into shared memory, synchronises, then computes the right-hand sides and
// the stage update of every node, and synchronises again, for `steps` steps per launch.  The
// arithmetic is that of the tile kernels (steps 2 and 3) with the varphi terms removed; nodes are
// strided over the threads.
// ---------------------------------------------------------------------------------------------
// threads of the CTA: FP64 keeps 256 so that a thread's node fits in registers
template <typename T>
constexpr int axi_threads() { return sizeof(T) == 8 ? 256 : 512; }

template <typename T>
__device__ __forceinline__ T axi_co(const StageArgs<T>& a, int c, int q) {
  return a.coef[(int64_t)c * a.nt + wrap(q, a.nt)];
}
template <typename T>
__device__ __forceinline__ T axi_f(const StageArgs<T>& a, const T* f, int k, int q) {
  return f[k * a.stride + wrap(q, a.nt)];
}

// Moments and mu of node q of fin into mom = [dn | u^theta | u^phi | mu], each nt long.
template <typename T>
__device__ __forceinline__ void axi_moments(const StageArgs<T>& a, const VConst<T>& vc, const T* fin, T* mom, int q) {
  constexpr bool DF = sizeof(T) == 4;  // phi as a float pair in FP32 storage
  const int nt = a.nt;
  T row[4] = {T(0), T(0), T(0), T(0)}, col[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T x = fin[(4 * i + j) * a.stride + q];
      row[i] += x;
      col[j] += x;
    }
  const T dn = (row[0] + row[1]) + (row[2] + row[3]);
  const T mt = vc.v[3] * (row[3] - row[0]) + vc.v[2] * (row[2] - row[1]);
  const T mp = vc.v[3] * (col[3] - col[0]) + vc.v[2] * (col[2] - col[1]);
  const T inv_n = recip(a.n0 + dn);
  mom[q] = dn;
  mom[nt + q] = mt * inv_n;
  mom[2 * nt + q] = mp * inv_n;
  const T ph = fin[NPOP * a.stride + q];
  T dN = axi_f(a, fin, NPOP, q + 1) - ph, dS = ph - axi_f(a, fin, NPOP, q - 1), lo = T(0);
  if (DF) {
    lo = fin[(NPOP + 1) * a.stride + q];
    dN += axi_f(a, fin, NPOP + 1, q + 1) - lo;
    dS += lo - axi_f(a, fin, NPOP + 1, q - 1);
  }
  const T lap = axi_co(a, C_LT, q) * (axi_co(a, C_JP, q) * dN - axi_co(a, C_JM, q) * dS);
  const T cubic = ph * (T(1) - ph * ph) + (T(1) - T(3) * ph * ph) * lo;
  mom[3 * nt + q] = -a.A * cubic - a.kappa * lap;
}

// Right-hand side and Runge-Kutta combination of node q: fout = f0 + b (fin - f0 + dt L(fin)), or
// fin + dt L(fin) without f0 (first stage).
template <typename T, int ADV, int CH, bool F0>
__device__ __forceinline__ void axi_node(const StageArgs<T>& a, const VConst<T>& vc, const T* fin, const T* f0,
                                         T* fout, const T* mom, int q) {
  constexpr bool DF = sizeof(T) == 4;
  const int nt = a.nt;
  const int64_t stride = a.stride;
  const T sixth = T(1) / T(6);
  const int qn = q + 1 < nt ? q + 1 : q + 1 - nt, qs = q > 0 ? q - 1 : nt - 1;
  const T dn = mom[q], ut = mom[nt + q], up = mom[2 * nt + q];
  const T mu_c = mom[3 * nt + q], mu_n = mom[3 * nt + qn], mu_s = mom[3 * nt + qs];
  const T ph = fin[NPOP * stride + q];
  const T n = a.n0 + dn;
  const T ct = axi_co(a, C_CT, q), gam = axi_co(a, C_GAM, q);

  // Cahn-Hilliard (Eq. CH): M Delta mu - div(u phi), theta parts only
  T Lphi = a.M * (axi_co(a, C_LT, q) * (axi_co(a, C_JP, q) * (mu_n - mu_c) - axi_co(a, C_JM, q) * (mu_c - mu_s)));
  T Ft = T(0);
  if (CH == VLB_HYDRO) {
    const T Xn = axi_co(a, C_J, q + 1) * mom[nt + qn] * fin[NPOP * stride + qn];
    const T Xs = axi_co(a, C_J, q - 1) * mom[nt + qs] * fin[NPOP * stride + qs];
    Lphi -= T(0.5) * (ct * (Xn - Xs));
    Ft = -(ph * recip(n)) * (mu_n - mu_s) * a.gt;  // n F^theta = -phi d_theta mu (Eq. pbin)
  }
  {
    const T lo = DF ? fin[(NPOP + 1) * stride + q] : T(0);
    T base = ph, base_lo = lo, inc = Lphi * a.dt;
    if (F0) {
      base = f0[NPOP * stride + q];
      base_lo = DF ? f0[(NPOP + 1) * stride + q] : T(0);
      inc = a.b * (((ph - base) + (lo - base_lo)) + inc);
    }
    if (DF) {  // (hi, lo) <- (base, base_lo) + inc, error-free sum, renormalised
      const T s1 = base + inc;
      const T bb = s1 - base;
      const T err = (base - (s1 - bb)) + (inc - bb);
      const T lo2 = base_lo + err;
      const T hi_out = s1 + lo2;
      fout[NPOP * stride + q] = hi_out;
      fout[(NPOP + 1) * stride + q] = lo2 - (hi_out - s1);
    } else {
      fout[NPOP * stride + q] = base + inc;
    }
  }

  T g[NPOP];
#pragma unroll
  for (int k = 0; k < NPOP; ++k) g[k] = fin[k * stride + q];
  const T ct6 = ct * sixth;
  const T Jm1 = axi_co(a, C_J, q - 1), J0 = axi_co(a, C_J, q), Jp1 = axi_co(a, C_J, q + 1);
  const T wp0 = ct6 * axi_co(a, C_J, q - 2), wp1 = T(-6) * ct6 * Jm1, wp2 = T(3) * ct6 * J0, wp3 = T(2) * ct6 * Jp1;
  const T wn0 = T(-2) * ct6 * Jm1, wn1 = T(-3) * ct6 * J0, wn2 = T(6) * ct6 * Jp1, wn3 = -ct6 * axi_co(a, C_J, q + 2);
  const T usq = ut * ut + up * up;
  const T c0 = T(1) - T(0.5) * usq, hu = T(-0.5) * usq;
  const T ntau = n * a.inv_tau, dntau = dn * a.inv_tau;
  const T Ep = axi_co(a, C_EP, q), En = axi_co(a, C_EN, q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T gvi = gam * vc.v[i];
    T h[4];  // (-F^phi - Gamma v_i v_m) g_{im} with F^phi = 0
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) h[mm] = (-gvi * vc.v[mm]) * g[4 * i + mm];
    const T ai = vc.v[i] * ut;
    const T ci = dntau + a.n0 * vc.v[i] * ((i >= 2 ? Ep : En) + Ft);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * i + j;
      T rhs;
      if (ADV == VLB_UW3) {
        const T Dt = (i >= 2) ? wp0 * axi_f(a, fin, k, q - 2) + wp1 * axi_f(a, fin, k, q - 1) + wp2 * g[k] +
                                    wp3 * axi_f(a, fin, k, q + 1)
                              : wn0 * axi_f(a, fin, k, q - 1) + wn1 * g[k] + wn2 * axi_f(a, fin, k, q + 1) +
                                    wn3 * axi_f(a, fin, k, q + 2);
        rhs = -(vc.v[i] * Dt);
      } else {
        const T fref = a.n0 * vc.ww[i][j];
        T xt[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) xt[d] = axi_co(a, C_J, q + d - 3) * (axi_f(a, fin, k, q + d - 3) + fref);
        const T Dt = (i >= 2) ? weno_diff<T, true>(xt) : weno_diff<T, false>(xt);
        rhs = -(vc.v[i] * ct) * Dt;
      }
      T dvt = T(0), dvp = T(0);
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        dvt += vc.K[i][mm] * g[4 * mm + j];
        dvp += vc.K[j][mm] * h[mm];
      }
      rhs += (gam * vc.v[j] * vc.v[j] - Ft) * dvt + dvp;
      const T xi = ai + vc.v[j] * up;
      const T pm1 = xi * (c0 + xi * (T(0.5) + xi * sixth)) + hu;
      rhs += vc.ww[i][j] * (ntau * pm1 + ci) - a.inv_tau * g[k];
      T o;
      if (F0) {
        const T g0 = f0[k * stride + q];
        o = g0 + a.b * ((g[k] - g0) + rhs * a.dt);
      } else {
        o = rhs * a.dt + g[k];
      }
      fout[k * stride + q] = o;
    }
  }
}

// `steps` SSP-RK3 steps of the whole column in one CTA, in the Shu-Osher form of run_steps:
// U1 = U + dt L(U); U2 = U + 1/4 (U1 - U + dt L(U1)); U <- U + 2/3 (U2 - U + dt L(U2)).  The third
// stage writes U in place: each node's U is read by its own thread before it is overwritten, and no
// thread reads another node's U in that stage.
template <typename T, int ADV, int CH>
__global__ void __launch_bounds__(axi_threads<T>()) axi_kernel(StageArgs<T> a, VConst<T> vc, T* U0, T* U1, T* U2,
                                                          int steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* mom = reinterpret_cast<T*>(smem_raw);  // 4 x nt
  const int nt = a.nt;
  for (int n = 0; n < steps; ++n) {
#pragma unroll 1
    for (int st = 0; st < 3; ++st) {
      const T* fin = st == 0 ? U0 : (st == 1 ? U1 : U2);
      T* fout = st == 0 ? U1 : (st == 1 ? U2 : U0);
      a.b = st == 0 ? T(1) : (st == 1 ? T(0.25) : T(2.0 / 3.0));
      for (int q = threadIdx.x; q < nt; q += blockDim.x) axi_moments(a, vc, fin, mom, q);
      __syncthreads();
      for (int q = threadIdx.x; q < nt; q += blockDim.x) {
        if (st == 0)
          axi_node<T, ADV, CH, false>(a, vc, fin, nullptr, fout, mom, q);
        else
          axi_node<T, ADV, CH, true>(a, vc, fin, U0, fout, mom, q);
      }
      __syncthreads();
    }
  }
}

template <typename T>
VConst<T> make_vconst() {
  const VelocityConsts d = velocity_consts();
  VConst<T> c;
  for (int i = 0; i < 4; ++i) {
    c.v[i] = (T)d.v[i];
    c.w[i] = (T)d.w[i];
    for (int m = 0; m < 4; ++m) {
      c.K[i][m] = (T)d.K[i][m];
      c.ww[i][m] = (T)(d.w[i] * d.w[m]);
    }
  }
  return c;
}

// Per-device, per-kernel one-time set-up (dynamic shared memory opt-in).
template <typename K>
cudaError_t ensure_smem(K kernel, size_t bytes, int& mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (mask & (1 << dev))) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 32) mask |= (1 << dev);
  return e;
}

template <typename T, int ADV, int CH, bool F0, bool PAIR, bool TMA>
cudaError_t launch_generic(const StageArgs<T>& a, cudaStream_t st, const StageMaps* maps) {
  using L = GenericLay<T, ADV>;
  static int mask = 0;
  cudaError_t e = ensure_smem(stage_kernel<T, ADV, CH, F0, PAIR, TMA>, L::BYTES, mask);
  if (e != cudaSuccess) return e;
  static const VConst<T> vc = make_vconst<T>();
  static const StageMaps none = {};
  const StageMaps& m = maps ? *maps : none;
  StageArgs<T> args = a;
  args.ahead = 0;
  if (TMA) {
    static int resident[32] = {0};  // CTAs of this kernel resident at once, per device
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev < 32 && resident[dev] == 0) {
      int per_sm = 0, sms = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel<T, ADV, CH, F0, PAIR, TMA>, 256,
                                                             L::BYTES)) != cudaSuccess)
        return e;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      resident[dev] = per_sm * sms;
    }
    // half a wave ahead (about the next tile started on the same SM) measured best on GB300: 0.237 ms
    // per step on 1024 x 2048 against 0.244 (one wave), 0.268 (two) and 0.254 (no prefetch)
    args.ahead = dev < 32 ? resident[dev] / 2 : 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.ns + TS - 1) / TS, (a.nt + L::TQ - 1) / L::TQ);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, stage_kernel<T, ADV, CH, F0, PAIR, TMA>, args, vc, m.box, m.tile);
}

template <int TQR, int CH, bool F0>
cudaError_t launch_ens(const EnsembleMember* members, const int2* items, int nitems, int stage, int* err,
                       cudaStream_t st, const EnsembleMaps& maps) {
  using L = EnsLay<TQR>;
  static int mask = 0;
  cudaError_t e = ensure_smem(ensemble_stage_kernel<TQR, CH, F0>, L::BYTES, mask);
  if (e != cudaSuccess) return e;
  static const VConst<float> vc = make_vconst<float>();
  static int resident[32] = {0};  // blocks of this kernel resident at once, per device
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 32 && resident[dev] == 0) {
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_stage_kernel<TQR, CH, F0>, L::NTH,
                                                           L::BYTES)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    resident[dev] = per_sm * sms;
  }
  const int ahead = dev < 32 ? resident[dev] / 2 : 0;  // half a wave, as for a single torus
  ensemble_stage_kernel<TQR, CH, F0><<<nitems, L::NTH, L::BYTES, st>>>(members, items, nitems, ahead, stage, err, vc,
                                                                     maps);
  return cudaGetLastError();
}

template <int TQR, int CH>
cudaError_t launch_pers(const EnsembleMember* members, const int2* items, int nitems, int nsteps, int only0,
                        unsigned* bar, int* err, long long budget, int skip_cta, int ctas_per_sm, cudaStream_t st,
                        const EnsembleMaps& maps, int* grid_out) {
  using L = EnsLay<TQR>;
  static int mask = 0;
  cudaError_t e = ensure_smem(ensemble_persistent_kernel<TQR, CH>, L::BYTES, mask);
  if (e != cudaSuccess) return e;
  static const VConst<float> vc = make_vconst<float>();
  static int occ[32] = {0}, sms[32] = {0};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev >= 32) return cudaErrorInvalidDevice;
  if (occ[dev] == 0) {
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], ensemble_persistent_kernel<TQR, CH>, L::NTH,
                                                           L::BYTES)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (occ[dev] < 1) return cudaErrorInvalidConfiguration;
  }
  const int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ[dev] ? ctas_per_sm : occ[dev];
  int grid = per_sm * sms[dev];
  if (grid > nitems) grid = nitems;
  if (grid_out) *grid_out = grid;
  if (grid < 1 || nsteps < 1) return cudaSuccess;
  // the arrival counter and both ticket counters start at zero (a launch that gave up may have left
  // arrivals or tickets behind); the generation word keeps counting
  if ((e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(bar + 2, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(L::NTH);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident at once: the grid barrier is safe
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ensemble_persistent_kernel<TQR, CH>, members, items, nitems, nsteps, only0, bar, err,
                            budget, skip_cta, vc, maps);
}

template <int TQR>
cudaError_t launch_ens_rows(const EnsembleMember* members, const int2* items, int nitems, int stage, int ch_mode,
                            int* err, cudaStream_t st, const EnsembleMaps& maps) {
  if (ch_mode == VLB_HYDRO)
    return stage == 0 ? launch_ens<TQR, VLB_HYDRO, false>(members, items, nitems, stage, err, st, maps)
                      : launch_ens<TQR, VLB_HYDRO, true>(members, items, nitems, stage, err, st, maps);
  return stage == 0 ? launch_ens<TQR, VLB_DIFFUSIVE, false>(members, items, nitems, stage, err, st, maps)
                    : launch_ens<TQR, VLB_DIFFUSIVE, true>(members, items, nitems, stage, err, st, maps);
}


template <typename T, int ADV, int CH>
cudaError_t launch_axi_t(const StageArgs<T>& a, T* U0, T* U1, T* U2, int steps, cudaStream_t st) {
  static int mask = 0;
  cudaError_t e = ensure_smem(axi_kernel<T, ADV, CH>, sizeof(T) * 4 * (size_t)kAxiMaxRows, mask);
  if (e != cudaSuccess) return e;
  static const VConst<T> vc = make_vconst<T>();
  axi_kernel<T, ADV, CH><<<1, axi_threads<T>(), sizeof(T) * 4 * (size_t)a.nt, st>>>(a, vc, U0, U1, U2, steps);
  return cudaGetLastError();
}

template <typename T, int ADV, int CH>
cudaError_t launch_one(const StageArgs<T>& a, cudaStream_t st, const StageMaps* maps) {
  if constexpr (sizeof(T) == 4 && ADV == VLB_UW3) {
    if (chunked<GenericLay<T, ADV>>(a.nt, a.ns)) {  // n_phi % 4 == 0: packed node pairs
      if (maps)
        return a.f0 ? launch_generic<T, ADV, CH, true, true, true>(a, st, maps)
                    : launch_generic<T, ADV, CH, false, true, true>(a, st, maps);
      return a.f0 ? launch_generic<T, ADV, CH, true, true, false>(a, st, nullptr)
                  : launch_generic<T, ADV, CH, false, true, false>(a, st, nullptr);
    }
  }
  return a.f0 ? launch_generic<T, ADV, CH, true, false, false>(a, st, nullptr)
              : launch_generic<T, ADV, CH, false, false, false>(a, st, nullptr);
}

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

// 3-D map over the 18 FP32 state arrays: (varphi, theta, array), box bx x by x 18.
cudaError_t encode_state_map(CUtensorMap* m, const float* base, int nt, int ns, int64_t stride, int bx, int by) {
  EncodeTiled fn = encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)ns, (cuuint64_t)nt, (cuuint64_t)(NARR + 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)ns * sizeof(float), (cuuint64_t)stride * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)(NARR + 1)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool stage_maps_apply(int nt, int ns) { return chunked<GenericLay<float, VLB_UW3>>(nt, ns); }

cudaError_t make_stage_maps(const float* fin, const float* f0, int nt, int ns, int64_t stride, StageMaps* out) {
  using L = GenericLay<float, VLB_UW3>;
  if (!stage_maps_apply(nt, ns) || stride % 4 != 0 || ((uintptr_t)fin) % 16 != 0 || ((uintptr_t)f0) % 16 != 0)
    return cudaErrorInvalidValue;
  cudaError_t e = encode_state_map(&out->box, fin, nt, ns, stride, L::BS, L::BQ);
  if (e == cudaSuccess) e = encode_state_map(&out->tile, f0, nt, ns, stride, TS, L::TQ);
  return e;
}

template <typename T>
cudaError_t launch_stage(const StageArgs<T>& a, int advection, int ch_mode, cudaStream_t s, const StageMaps* maps) {
  if (advection == VLB_UW3)
    return ch_mode == VLB_HYDRO ? launch_one<T, VLB_UW3, VLB_HYDRO>(a, s, maps)
                                : launch_one<T, VLB_UW3, VLB_DIFFUSIVE>(a, s, maps);
  return ch_mode == VLB_HYDRO ? launch_one<T, VLB_WENO5, VLB_HYDRO>(a, s, nullptr)
                              : launch_one<T, VLB_WENO5, VLB_DIFFUSIVE>(a, s, nullptr);
}

cudaError_t launch_ensemble_stage(const EnsembleMember* members, const int2* items, int nitems, int stage,
                                  int tile_rows, int ch_mode, int* err, cudaStream_t s, const EnsembleMaps* maps) {
  if (nitems <= 0) return cudaSuccess;
  static const EnsembleMaps none = {};
  const EnsembleMaps& m = maps ? *maps : none;
  if (tile_rows == 8) return launch_ens_rows<8>(members, items, nitems, stage, ch_mode, err, s, m);
  return launch_ens_rows<16>(members, items, nitems, stage, ch_mode, err, s, m);
}

cudaError_t launch_ensemble_persistent(const EnsembleMember* members, const int2* items, int nitems, int nsteps,
                                       int only0, int tile_rows, int ch_mode, unsigned* bar, int* err, long long budget,
                                       int skip_cta, int ctas_per_sm, cudaStream_t s, const EnsembleMaps* maps,
                                       int* grid_out) {
  if (nitems <= 0) return cudaSuccess;
  static const EnsembleMaps none = {};
  const EnsembleMaps& m = maps ? *maps : none;
  if (tile_rows == 8)
    return ch_mode == VLB_HYDRO ? launch_pers<8, VLB_HYDRO>(members, items, nitems, nsteps, only0, bar, err, budget,
                                                             skip_cta, ctas_per_sm, s, m, grid_out)
                                : launch_pers<8, VLB_DIFFUSIVE>(members, items, nitems, nsteps, only0, bar, err, budget,
                                                                 skip_cta, ctas_per_sm, s, m, grid_out);
  return ch_mode == VLB_HYDRO ? launch_pers<16, VLB_HYDRO>(members, items, nitems, nsteps, only0, bar, err, budget,
                                                            skip_cta, ctas_per_sm, s, m, grid_out)
                              : launch_pers<16, VLB_DIFFUSIVE>(members, items, nitems, nsteps, only0, bar, err, budget,
                                                                skip_cta, ctas_per_sm, s, m, grid_out);
}

bool wave_schedule_ok(int nb, int lag, int nsteps) {
  if (lag < 3 || nb <= 2 * lag + 2 || nsteps < 1) return false;
  // every band item's dependencies sit in earlier tickets (checked by enumeration for small launches)
  if ((int64_t)3 * nsteps * nb > (int64_t)1 << 20) return true;
  std::vector<int> pos((size_t)3 * nsteps * nb, -1);  // ticket position of (n, k, band)
  for (int j = 0; j < 3 * nsteps * nb; ++j) {
    int n, k, i;
    wave_decode(j, nb, lag, nsteps, n, k, i);
    if (n < 0 || n >= nsteps || k < 0 || k > 2 || i < 0 || i >= nb) return false;
    const size_t at = ((size_t)n * 3 + k) * nb + (3 * n + k + i) % nb;
    if (pos[at] != -1) return false;  // each band item exactly once
    pos[at] = j;
  }
  for (int n = 0; n < nsteps; ++n)
    for (int k = 0; k < 3; ++k)
      for (int b = 0; b < nb; ++b) {
        if (k == 0 && n == 0) continue;
        const int np = k == 0 ? n - 1 : n, kp = k == 0 ? 2 : k - 1;
        for (int d = -1; d <= 1; ++d)
          if (pos[((size_t)np * 3 + kp) * nb + (b + d + nb) % nb] >= pos[((size_t)n * 3 + k) * nb + b]) return false;
      }
  return true;
}

bool wave_apply(int nt, int ns) {
  using L = GenericLay<float, VLB_UW3>;
  return stage_maps_apply(nt, ns) && nt % L::TQ == 0 && ns % TS == 0 && nt / L::TQ > 2 * kWaveLag + 2;
}

int wave_counter_words(int nt) { return 3 * (nt / 16) + 1; }

template <int CH>
cudaError_t launch_wave_t(const StageArgs<float>& a, float* U0, float* U1, float* U2, int nsteps, unsigned* cnt,
                          long long budget, int skip_cta, cudaStream_t st, const WaveMaps& maps, int* grid_out) {
  using L = GenericLay<float, VLB_UW3>;
  static int mask = 0;
  cudaError_t e = ensure_smem(wave_kernel<CH>, L::BYTES, mask);
  if (e != cudaSuccess) return e;
  static const VConst<float> vc = make_vconst<float>();
  static int occ[32] = {0}, sms[32] = {0};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev >= 32) return cudaErrorInvalidDevice;
  if (occ[dev] == 0) {
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], wave_kernel<CH>, 256, L::BYTES)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (occ[dev] < 1) return cudaErrorInvalidConfiguration;
  }
  const int nb = a.nt / L::TQ, tiles = nb * (a.ns / TS);
  int grid = occ[dev] * sms[dev];
  if (grid > 3 * tiles) grid = 3 * tiles;
  if (grid_out) *grid_out = grid;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * wave_counter_words(a.nt), st)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every ticket holder is resident: the waits end
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, wave_kernel<CH>, a, U0, U1, U2, nsteps, kWaveLag, cnt, a.err, budget, skip_cta, vc,
                            maps);
}

cudaError_t launch_wave(const StageArgs<float>& a, int ch_mode, float* U0, float* U1, float* U2, int nsteps,
                        unsigned* cnt, long long budget, int skip_cta, cudaStream_t st, const StageMaps* stage_maps,
                        int* grid_out) {
  if (!wave_apply(a.nt, a.ns) || !stage_maps || nsteps < 1 || nsteps > kWaveMaxSteps) return cudaErrorInvalidValue;
  for (float* u : {U0, U1, U2})
    if (((uintptr_t)u) % 128 != 0 || a.stride % 32 != 0) return cudaErrorInvalidValue;  // discarded lines
  WaveMaps m;
  m.box[0] = stage_maps[0].box;
  m.box[1] = stage_maps[1].box;
  m.box[2] = stage_maps[2].box;
  m.tile = stage_maps[1].tile;
  return ch_mode == VLB_HYDRO
             ? launch_wave_t<VLB_HYDRO>(a, U0, U1, U2, nsteps, cnt, budget, skip_cta, st, m, grid_out)
             : launch_wave_t<VLB_DIFFUSIVE>(a, U0, U1, U2, nsteps, cnt, budget, skip_cta, st, m, grid_out);
}

template <typename T>
cudaError_t launch_axi(const StageArgs<T>& a, int advection, int ch_mode, T* U0, T* U1, T* U2, int steps,
                       cudaStream_t s) {
  if (a.ns != 1 || a.nt < 1 || a.nt > kAxiMaxRows || steps < 0) return cudaErrorInvalidValue;
  if (steps == 0) return cudaSuccess;
  if (advection == VLB_UW3)
    return ch_mode == VLB_HYDRO ? launch_axi_t<T, VLB_UW3, VLB_HYDRO>(a, U0, U1, U2, steps, s)
                                : launch_axi_t<T, VLB_UW3, VLB_DIFFUSIVE>(a, U0, U1, U2, steps, s);
  return ch_mode == VLB_HYDRO ? launch_axi_t<T, VLB_WENO5, VLB_HYDRO>(a, U0, U1, U2, steps, s)
                              : launch_axi_t<T, VLB_WENO5, VLB_DIFFUSIVE>(a, U0, U1, U2, steps, s);
}

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, cudaStream_t, const StageMaps*);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, cudaStream_t, const StageMaps*);
template cudaError_t launch_axi<float>(const StageArgs<float>&, int, int, float*, float*, float*, int, cudaStream_t);
template cudaError_t launch_axi<double>(const StageArgs<double>&, int, int, double*, double*, double*, int,
                                        cudaStream_t);

}  // namespace vlb
