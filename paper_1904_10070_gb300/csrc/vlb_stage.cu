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
// Tiling: a CTA owns a 16 (theta) x 32 (varphi) tile; 256 threads, each thread two nodes.
// Shared memory holds, for the tile plus its halo:
//   - the 16 populations on the cross-shaped region the upwind stencils reach (halo 2 for UW3,
//     3 for WENO5) -- every global element is read once per CTA with coalesced loads;
//   - phi with a halo of 2 (corners included: mu is needed one node outside the tile);
//   - the moments n, u and the chemical potential mu on the tile plus a halo of 1;
//   - the per-row geometric coefficients of the rows the CTA touches.
// Periodic wrap-around is done on the load indices, so tiles may be ragged and grids tiny.
#include "vlb_internal.cuh"

namespace vlb {

namespace {

constexpr int TS = 32;       // tile width along varphi (one warp)
constexpr int TYT = 8;       // thread rows
constexpr int NQ = 2;        // nodes per thread along theta
constexpr int TQ = TYT * NQ; // tile height along theta
constexpr int NTHREADS = TS * TYT;
constexpr int NCT = 11;      // coefficient rows staged in shared memory (C_J .. C_EN)

template <typename T>
struct VConst {
  T v[4], w[4], K[4][4];
};

template <int ADV>
struct Halo { static constexpr int H = (ADV == VLB_UW3) ? 2 : 3; };

template <typename T, int ADV>
struct Smem {
  static constexpr int H = Halo<ADV>::H;
  static constexpr int BQ = TQ + 2 * H, BS = TS + 2 * H;  // population box
  static constexpr int PQ = TQ + 4, PS = TS + 4;          // phi box (halo 2)
  static constexpr int MQ = TQ + 2, MS = TS + 2;          // moment / mu box (halo 1)
  static constexpr int F_OFF = 0;
  static constexpr int PHI_OFF = F_OFF + NPOP * BQ * BS;
  static constexpr int N_OFF = PHI_OFF + PQ * PS;
  static constexpr int UT_OFF = N_OFF + MQ * MS;
  static constexpr int UP_OFF = UT_OFF + MQ * MS;
  static constexpr int MU_OFF = UP_OFF + MQ * MS;
  static constexpr int PHL_OFF = MU_OFF + MQ * MS;                       // phi low part (FP32 only)
  static constexpr int CO_OFF = PHL_OFF + (sizeof(T) == 4 ? PQ * PS : 0);
  static constexpr int TOTAL = CO_OFF + NCT * BQ;
  static constexpr size_t BYTES = sizeof(T) * (size_t)TOTAL;
};

__device__ __forceinline__ int wrap(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

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

// Flux difference g_{+1/2} - g_{-1/2} at the centre of a 7-point window x[0..6] (centre x[3]).
template <typename T, int ADV, bool POS>
__device__ __forceinline__ T flux_diff(const T (&x)[7]) {
  if (ADV == VLB_UW3) {
    // UW3 faces (-x_{i-1} + 5 x_i + 2 x_{i+1})/6 (v > 0), mirrored for v < 0, differenced.
    if (POS) return (x[1] - T(6) * x[2] + T(3) * x[3] + T(2) * x[4]) * (T(1) / T(6));
    return (-T(2) * x[2] - T(3) * x[3] + T(6) * x[4] - x[5]) * (T(1) / T(6));
  } else {
    if (POS) return weno5(x[1], x[2], x[3], x[4], x[5]) - weno5(x[0], x[1], x[2], x[3], x[4]);
    return weno5(x[6], x[5], x[4], x[3], x[2]) - weno5(x[5], x[4], x[3], x[2], x[1]);
  }
}

template <typename T, int ADV, int CH>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? (ADV == VLB_UW3 ? 3 : 2) : 1) stage_kernel(StageArgs<T> a, VConst<T> vc) {
  using S = Smem<T, ADV>;
  constexpr int H = S::H, BQ = S::BQ, BS = S::BS, PQ = S::PQ, PS = S::PS, MQ = S::MQ, MS = S::MS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sf = sm + S::F_OFF;
  T* sphi = sm + S::PHI_OFF;
  T* sn = sm + S::N_OFF;
  T* sut = sm + S::UT_OFF;
  T* sup = sm + S::UP_OFF;
  T* smu = sm + S::MU_OFF;
  T* sco = sm + S::CO_OFF;
  T* sphl = sm + S::PHL_OFF;
  constexpr bool DF = sizeof(T) == 4;  // phi as a float pair

  const int nt = a.nt, ns = a.ns;
  const int64_t stride = a.stride;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TS + tx;
  const int s0 = blockIdx.x * TS, q0 = blockIdx.y * TQ;

  // ---- phase 1: stage populations (cross), phi (box) and row coefficients ----
  {
    constexpr int PA = TQ * BS;            // interior rows, full width
    constexpr int PF = PA + 2 * H * TS;    // + halo rows, interior columns
    for (int idx = tid; idx < PF; idx += NTHREADS) {
      int r, c;
      if (idx < PA) {
        r = H + idx / BS;
        c = idx % BS;
      } else {
        const int j = idx - PA, hr = j / TS;
        c = H + j % TS;
        r = hr < H ? hr : hr + TQ;
      }
      const int gq = wrap(q0 + r - H, nt), gs = wrap(s0 + c - H, ns);
      const T* src = a.fin + (int64_t)gq * ns + gs;
      T* dst = sf + r * BS + c;
#pragma unroll
      for (int k = 0; k < NPOP; ++k) dst[k * BQ * BS] = __ldg(src + k * stride);
    }
    const T* phin = a.fin + NPOP * stride;
    for (int idx = tid; idx < PQ * PS; idx += NTHREADS) {
      const int r = idx / PS, c = idx % PS;
      const int gq = wrap(q0 + r - 2, nt), gs = wrap(s0 + c - 2, ns);
      sphi[idx] = __ldg(phin + (int64_t)gq * ns + gs);
      if (DF) sphl[idx] = __ldg(phin + stride + (int64_t)gq * ns + gs);
    }
    for (int idx = tid; idx < NCT * BQ; idx += NTHREADS) {
      const int k = idx / BQ, r = idx % BQ;
      sco[idx] = __ldg(a.coef + (int64_t)k * nt + wrap(q0 + r - H, nt));
    }
  }
  __syncthreads();

  // ---- phase 2: moments (Sec. 2.3) and mu (Eq. mu) on the tile plus a halo of 1 (cross) ----
  {
    constexpr int PA = TQ * MS;
    constexpr int PM = PA + 2 * TS;
    for (int idx = tid; idx < PM; idx += NTHREADS) {
      int mr, mc;
      if (idx < PA) {
        mr = 1 + idx / MS;
        mc = idx % MS;
      } else {
        const int j = idx - PA;
        mr = (j < TS) ? 0 : MQ - 1;
        mc = 1 + j % TS;
      }
      const T* fp = sf + (mr + H - 1) * BS + (mc + H - 1);
      T row[4] = {T(0), T(0), T(0), T(0)}, col[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T x = fp[(4 * i + j) * BQ * BS];
          row[i] += x;
          col[j] += x;
        }
      // n = n0 + sum g (the reference part carries no momentum: sum_k w_i w_j v = 0)
      const T dn = (row[0] + row[1]) + (row[2] + row[3]);
      const T mt = vc.v[0] * row[0] + vc.v[1] * row[1] + vc.v[2] * row[2] + vc.v[3] * row[3];
      const T mp = vc.v[0] * col[0] + vc.v[1] * col[1] + vc.v[2] * col[2] + vc.v[3] * col[3];
      const int mi = mr * MS + mc;
      const T n = a.n0 + dn;
      sn[mi] = dn;
      sut[mi] = mt / n;
      sup[mi] = mp / n;
      const int pidx = (mr + 1) * PS + (mc + 1);
      const T* pp = sphi + pidx;
      const int cr = mr + H - 1;
      const T ph = pp[0];
      // neighbour differences of phi = hi + lo: the hi differences are exact for nearby values
      T dN = pp[PS] - ph, dS = ph - pp[-PS], dE = pp[1] - ph, dW = ph - pp[-1], lo = T(0);
      if (DF) {
        const T* pl = sphl + pidx;
        lo = pl[0];
        dN += pl[PS] - lo;
        dS += lo - pl[-PS];
        dE += pl[1] - lo;
        dW += lo - pl[-1];
      }
      const T lap = sco[C_LT * BQ + cr] * (sco[C_JP * BQ + cr] * dN - sco[C_JM * BQ + cr] * dS) +
                    sco[C_LP * BQ + cr] * (dE - dW);
      // phi (1 - phi^2) at hi + lo, to first order in lo
      const T cubic = ph * (T(1) - ph * ph) + (T(1) - T(3) * ph * ph) * lo;
      smu[mi] = -a.A * cubic - a.kappa * lap;
    }
  }
  __syncthreads();

  // ---- phase 3: right-hand sides and the Runge-Kutta combination, per node ----
#pragma unroll 1
  for (int m = 0; m < NQ; ++m) {
    const int lr = ty + TYT * m, lc = tx;
    const int q = q0 + lr, s = s0 + lc;
    if (q >= nt || s >= ns) continue;
    const int fr = lr + H, fc = lc + H;
    const int mi = (lr + 1) * MS + (lc + 1);
    const int pi = (lr + 2) * PS + (lc + 2);

    const T dn = sn[mi], ut = sut[mi], up = sup[mi], ph = sphi[pi];
    const T n = a.n0 + dn;
    const T ct = sco[C_CT * BQ + fr], cp = sco[C_CP * BQ + fr], gam = sco[C_GAM * BQ + fr];
    const T Ep = sco[C_EP * BQ + fr], En = sco[C_EN * BQ + fr];
    const T mu_c = smu[mi], mu_n = smu[mi + MS], mu_s = smu[mi - MS], mu_e = smu[mi + 1], mu_w = smu[mi - 1];

    // Cahn-Hilliard: M Delta mu - div(u phi) (Eq. CH), flux form with mean face values
    T Lphi = a.M * (sco[C_LT * BQ + fr] * (sco[C_JP * BQ + fr] * (mu_n - mu_c) - sco[C_JM * BQ + fr] * (mu_c - mu_s)) +
                    sco[C_LP * BQ + fr] * (mu_e - T(2) * mu_c + mu_w));
    T Ft = T(0), Fp = T(0);
    if (CH == VLB_HYDRO) {
      const T Xn = sco[C_J * BQ + fr + 1] * sut[mi + MS] * sphi[pi + PS];
      const T Xs = sco[C_J * BQ + fr - 1] * sut[mi - MS] * sphi[pi - PS];
      const T Ye = sup[mi + 1] * sphi[pi + 1];
      const T Yw = sup[mi - 1] * sphi[pi - 1];
      Lphi -= T(0.5) * (ct * (Xn - Xs) + cp * (Ye - Yw));
      // n F = -phi grad mu (Eq. pbin), central differences
      const T pn = ph / n;
      Ft = -pn * (mu_n - mu_s) * a.gt;
      Fp = -pn * (mu_e - mu_w) * sco[C_GP * BQ + fr];
    }

    const int64_t gidx = (int64_t)q * ns + s;
    {
      const T lo = DF ? sphl[pi] : T(0);
      T base = ph, base_lo = lo, inc = Lphi * a.dt;
      if (a.f0) {
        base = a.f0[NPOP * stride + gidx];
        base_lo = DF ? a.f0[(NPOP + 1) * stride + gidx] : T(0);
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
    for (int k = 0; k < NPOP; ++k) g[k] = sf[k * BQ * BS + fr * BS + fc];

    // theta-direction weights J_{q+d}, d = -3..3
    T Jw[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) Jw[d] = (d >= 3 - H && d <= 3 + H) ? sco[C_J * BQ + fr + d - 3] : T(0);

    const T usq = ut * ut + up * up;
    const T c0 = T(1) - T(0.5) * usq;
    const T sixth = T(1) / T(6);

#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // varphi-derivative operands h_m = (-F^phi - Gamma v_i v_m) g_{i m}; K~ = K diag(v) (Sec. 2.3)
      const T gvi = gam * vc.v[i];
      T h[4];
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) h[mm] = (-Fp - gvi * vc.v[mm]) * g[4 * i + mm];
      const T ai = vc.v[i] * ut;
      const T n0wi = a.n0 * vc.w[i];
      // reference part: v_i (E(q) + F^theta) per row and sign
      const T refi = vc.v[i] * ((i >= 2 ? Ep : En) + Ft);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * i + j;
        const T fref = n0wi * vc.w[j];
        // advection along theta of G = J f and along varphi of f (Eq. boltz_tor); the reference
        // part of f is constant in varphi and, for UW3, handled through E(q)
        T xt[7], xp[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) {
          const bool in = (d >= 3 - H && d <= 3 + H);
          const T gt_d = sf[k * BQ * BS + (fr + d - 3) * BS + fc];
          xt[d] = in ? Jw[d] * (ADV == VLB_UW3 ? gt_d : gt_d + fref) : T(0);
          xp[d] = in ? sf[k * BQ * BS + fr * BS + fc + d - 3] : T(0);
        }
        const T Dt = (i >= 2) ? flux_diff<T, ADV, true>(xt) : flux_diff<T, ADV, false>(xt);
        const T Dp = (j >= 2) ? flux_diff<T, ADV, true>(xp) : flux_diff<T, ADV, false>(xp);
        T rhs = -(vc.v[i] * ct) * Dt - (vc.v[j] * cp) * Dp;
        // force and inertial terms on the deviation: (Gamma v_j^2 - F^theta) dg/dv_theta + sum_m K_jm h_m
        T dvt = T(0), dvp = T(0);
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
          dvt += vc.K[i][mm] * g[4 * mm + j];
          dvp += vc.K[j][mm] * h[mm];
        }
        rhs += (gam * vc.v[j] * vc.v[j] - Ft) * dvt + dvp;
        // same terms (and UW3 theta-advection) on the reference part n0 w_i w_j, in closed form
        rhs += fref * (refi + vc.v[j] * Fp);
        // BGK towards the third-order Hermite equilibrium (Eq. feq):
        // f^eq - n0 w_i w_j = w_i w_j (dn + n (poly - 1))
        const T xi = ai + vc.v[j] * up;
        const T pm1 = xi * (c0 + xi * (T(0.5) + xi * sixth)) - T(0.5) * usq;
        const T geq = vc.w[i] * vc.w[j] * (dn + n * pm1);
        rhs += a.inv_tau * (geq - g[k]);
        T o = rhs * a.dt + g[k];
        if (a.f0) {
          const T g0 = a.f0[k * stride + gidx];
          o = g0 + a.b * ((g[k] - g0) + rhs * a.dt);
        }
        a.fout[k * stride + gidx] = o;
      }
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
    for (int m = 0; m < 4; ++m) c.K[i][m] = (T)d.K[i][m];
  }
  return c;
}

template <typename T, int ADV, int CH>
cudaError_t launch_one(const StageArgs<T>& a, cudaStream_t st) {
  using S = Smem<T, ADV>;
  static int configured_mask = 0;  // one bit per device id < 32
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 32 || !(configured_mask & (1 << dev))) {
    e = cudaFuncSetAttribute(stage_kernel<T, ADV, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::BYTES);
    if (e != cudaSuccess) return e;
    if (dev < 32) configured_mask |= (1 << dev);
  }
  static const VConst<T> vc = make_vconst<T>();
  dim3 grid((a.ns + TS - 1) / TS, (a.nt + TQ - 1) / TQ);
  stage_kernel<T, ADV, CH><<<grid, dim3(TS, TYT), S::BYTES, st>>>(a, vc);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_stage(const StageArgs<T>& a, int advection, int ch_mode, cudaStream_t s) {
  if (advection == VLB_UW3)
    return ch_mode == VLB_HYDRO ? launch_one<T, VLB_UW3, VLB_HYDRO>(a, s) : launch_one<T, VLB_UW3, VLB_DIFFUSIVE>(a, s);
  return ch_mode == VLB_HYDRO ? launch_one<T, VLB_WENO5, VLB_HYDRO>(a, s) : launch_one<T, VLB_WENO5, VLB_DIFFUSIVE>(a, s);
}

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, cudaStream_t);

}  // namespace vlb
