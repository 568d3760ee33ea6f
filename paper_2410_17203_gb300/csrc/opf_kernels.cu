// Proximal message passing for contingency-constrained DC OPF -- sm_103a kernels.
//
// One cooperative persistent launch runs many iterations of the message-passing
// form of ADMM (Section 3.2).  Each iteration has three phases separated by
// grid-wide barriers with a bounded spin:
//
//   A  prox phase (Section 3.2 steps 1-2, Section 4.2):
//        - every (contingency k, line l, time chunk) applies the line prox to
//          (p~ - u, theta_bar - v) gathered from its two end nodes, and folds in
//          the deferred phase-dual update v += theta - theta_bar of the
//          previous iteration;
//        - every generator / load applies its closed-form prox with weight
//          (K+1) rho_p to p_d - avg_k(pbar + u);
//        - ramp-limited generators and batteries run the inner ADMM of
//          Appendix D, one warp per device, lanes over time steps, with the
//          x-update as a tridiagonal solve done by a warp-wide scan;
//   B  node phase (Eq. average-op, Section 3.2 step 3, Section 3.3): every
//      (node, time chunk) walks the node's terminals in CSR-by-node order,
//      for each contingency forms pbar, theta_bar and u += pbar with plain
//      register sums (no atomics), accumulates sum_k pbar and sum_k u for the
//      next step A, and the FP64 residual partial sums;
//   C  every CTA reduces the per-CTA FP64 partials in the same order and takes
//      the same stopping / adaptive-penalty decision (Section 3.5), so no third
//      barrier is needed.
//
// Memory layout and the deferred v update are described in opf_internal.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "opf_internal.h"

namespace opfk {

constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;
constexpr int ST_TIMEOUT = 4;    // opf_status values used on the device
constexpr int ST_NONFINITE = 5;

// ---------------------------------------------------------------------------
// small vector helpers: VW consecutive time steps per thread (4 -> 128-bit I/O)
// ---------------------------------------------------------------------------
template <int VW>
struct FV {
  float v[VW];
};

template <int VW>
__device__ __forceinline__ FV<VW> ldv(const float *p) {
  FV<VW> r;
  if constexpr (VW == 4) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
    r.v[0] = *p;
  }
  return r;
}

// streaming load/store (read or written once per phase: evict first)
template <int VW>
__device__ __forceinline__ FV<VW> ldv_cs(const float *p) {
  FV<VW> r;
  if constexpr (VW == 4) {
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
    r.v[0] = __ldcs(p);
  }
  return r;
}

template <int VW>
__device__ __forceinline__ void stv(float *p, const FV<VW> &r) {
  if constexpr (VW == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    *p = r.v[0];
  }
}

template <int VW>
__device__ __forceinline__ void stv_cs(float *p, const FV<VW> &r) {
  if constexpr (VW == 4) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
  } else {
    __stcs(p, r.v[0]);
  }
}

// ---------------------------------------------------------------------------
// grid barrier with a bounded spin.  On timeout the CTA records ST_TIMEOUT in
// *err and returns false; every CTA that sees *err set returns false too, so
// the whole grid leaves the iteration loop and the kernel ends.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(const Params &p, int *s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned *vgen = p.bar_gen;
    volatile int *verr = p.err;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(p.bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      *p.bar_count = 0;
      __threadfence();
      atomicAdd(p.bar_gen, 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == g) {
        if (*verr) { ok = 0; break; }
        if (clock64() - t0 > p.barrier_budget) {
          atomicCAS(p.err, 0, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    if (*verr) ok = 0;
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// ---------------------------------------------------------------------------
// tridiagonal systems with constant off-diagonal `off` and diagonal d_end at
// both ends, d_mid inside (every x-update of Appendix D reduces to one).
// Factor: pivots q_i = d_i - off^2 / q_{i-1} (Thomas); the solve divides by
// the pivots (correctly rounded) rather than multiplying by rounded
// reciprocals, which would bias every solve of a device the same way.
// ---------------------------------------------------------------------------
__device__ void tri_factor(float *q, int n, float d_end, float d_mid, float off) {
  float prev = 0.f;
  for (int i = 0; i < n; ++i) {
    const float d = (i == 0 || i == n - 1) ? d_end : d_mid;
    const float qi = (i == 0) ? d : d - off * (off / prev);
    q[i] = qi;
    prev = qi;
  }
}

// Solve in place (buf: right-hand side in, solution out; shared memory).
// Forward  y_i = A_i y_{i-1} + r_i / q_i  and backward  x_i = A_i x_{i+1} + y_i
// with A_i = -off / q_i are first-order linear recurrences; each lane composes
// the affine maps of a contiguous chunk, a 5-step shuffle scan composes the
// chunks across the warp, then each lane applies the prefix to its chunk.
__device__ void warp_tri_solve(const float *__restrict__ q, float off, float *buf, int n,
                               int lane) {
  const int cs = (n + 31) >> 5;
  const int i0 = min(lane * cs, n), i1 = min(i0 + cs, n);
  // forward
  float Ac = 1.f, Bc = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float qi = q[i];
    const float Ai = (i == 0) ? 0.f : -off / qi;
    Bc = fmaf(Ai, Bc, buf[i] / qi);
    Ac = Ai * Ac;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_up_sync(0xffffffffu, Ac, d);
    const float Bp = __shfl_up_sync(0xffffffffu, Bc, d);
    if (lane >= d) {
      Bc = fmaf(Ac, Bp, Bc);
      Ac = Ac * Ap;
    }
  }
  float prev = __shfl_up_sync(0xffffffffu, Bc, 1);
  if (lane == 0) prev = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float qi = q[i];
    const float Ai = (i == 0) ? 0.f : -off / qi;
    prev = fmaf(Ai, prev, buf[i] / qi);
    buf[i] = prev;
  }
  __syncwarp();
  // backward
  Ac = 1.f;
  Bc = 0.f;
  for (int i = i1 - 1; i >= i0; --i) {
    const float Ci = (i == n - 1) ? 0.f : -off / q[i];
    Bc = fmaf(Ci, Bc, buf[i]);
    Ac = Ci * Ac;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_down_sync(0xffffffffu, Ac, d);
    const float Bp = __shfl_down_sync(0xffffffffu, Bc, d);
    if (lane + d < 32) {
      Bc = fmaf(Ac, Bp, Bc);
      Ac = Ac * Ap;
    }
  }
  float nxt = __shfl_down_sync(0xffffffffu, Bc, 1);
  if (lane == 31) nxt = 0.f;
  for (int i = i1 - 1; i >= i0; --i) {
    const float Ci = (i == n - 1) ? 0.f : -off / q[i];
    nxt = fmaf(Ci, nxt, buf[i]);
    buf[i] = nxt;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Appendix D inner ADMM, ramp-limited generator (one warp, lanes over t).
// Rows: p_t <= pmax_t, -p_t <= -pmin_t, p_{t+1} - p_t <= R, p_t - p_{t+1} <= R.
// x-update matrix (2a + rho + 2 omega) I + 2 omega D'D is tridiagonal.
// ---------------------------------------------------------------------------
__device__ void ramp_prox(const Params &p, int r, float rho, float su, float kpf,
                          float *sm, bool resid, int lane) {
  const int T = p.T;
  const int d = p.ramp_ids[r];
  const int n = p.dev_node[d];
  const float a = p.dev_a[d], b = p.dev_b[d], R = p.ramp_R[r];
  const float om = rho;
  float *lam = p.ramp_lam + (size_t)r * RG_N * T;
  float *bet = p.ramp_beta + (size_t)r * RG_N * T;
  float *mf = p.ramp_m + (size_t)r * T;
  const float *lo = p.dev_lo + (size_t)d * T;
  const float *hi = p.dev_hi + (size_t)d * T;
  float *pd = p.PD + (size_t)d * T;
  float *X = sm, *W = sm + (T + 1), *Z = sm + 2 * (T + 1);

  // keep the unscaled inner duals omega * lam when omega changes; refactor
  const float rho_old = p.ramp_rho[r];
  if (rho_old != rho) {
    const float ls = (rho_old == 0.f) ? 1.f : fabsf(rho_old) / rho;
    for (int t = lane; t < RG_N * T; t += 32) lam[t] *= ls;
    if (lane == 0) {
      tri_factor(mf, T, 2.f * a + rho + 4.f * om, 2.f * a + rho + 6.f * om, -2.f * om);
      p.ramp_rho[r] = rho;
    }
    __syncwarp();
  }
  for (int t = lane; t < T; t += 32) {
    size_t o = (size_t)n * T + t;
    X[t] = pd[t] - (p.SPBAR[o] + su * p.SU[o]) / kpf;
  }
  __syncwarp();
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    for (int t = lane; t < T - 1; t += 32)
      W[t] = (bet[RG_RU * T + t] - lam[RG_RU * T + t]) - (bet[RG_RD * T + t] - lam[RG_RD * T + t]);
    __syncwarp();
    for (int t = lane; t < T; t += 32) {
      float atr = (hi[t] + bet[RG_UP * T + t] - lam[RG_UP * T + t]) -
                  (-lo[t] + bet[RG_LO * T + t] - lam[RG_LO * T + t]);
      if (t >= 1) atr += W[t - 1];
      if (t <= T - 2) atr -= W[t];
      Z[t] = rho * X[t] - b + om * atr;
    }
    __syncwarp();
    warp_tri_solve(mf, -2.f * om, Z, T, lane);
    for (int t = lane; t < T; t += 32) {
      const float pt = Z[t];
      float al, nb;
      al = pt - hi[t];
      nb = fminf(al + lam[RG_UP * T + t], 0.f);
      lam[RG_UP * T + t] += al - nb;
      bet[RG_UP * T + t] = nb;
      al = lo[t] - pt;
      nb = fminf(al + lam[RG_LO * T + t], 0.f);
      lam[RG_LO * T + t] += al - nb;
      bet[RG_LO * T + t] = nb;
      if (t < T - 1) {
        const float pn = Z[t + 1];
        al = pn - pt - R;
        nb = fminf(al + lam[RG_RU * T + t], 0.f);
        lam[RG_RU * T + t] += al - nb;
        bet[RG_RU * T + t] = nb;
        al = pt - pn - R;
        nb = fminf(al + lam[RG_RD * T + t], 0.f);
        lam[RG_RD * T + t] += al - nb;
        bet[RG_RD * T + t] = nb;
      }
    }
    __syncwarp();
  }
  for (int t = lane; t < T; t += 32) {
    const float pn = Z[t];
    if (resid) p.DPD[(size_t)d * T + t] = pn - pd[t];
    pd[t] = pn;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Appendix D inner ADMM, battery (one warp, lanes over t).  Variables
// (p, c, delta, s), rows as in opf.h.  The x-update eliminates p_t, then
// (c_t, delta_t) per step (a 2x2 Schur complement), leaving a tridiagonal
// system of size T + 1 in the state of charge s.
// ---------------------------------------------------------------------------
__device__ void stor_prox(const Params &p, int sidx, float rho, float su, float kpf,
                          float *sm, bool resid, int lane) {
  const int T = p.T, Tp = T + 1;
  const int d = p.stor_ids[sidx];
  const int n = p.dev_node[d];
  const float eta = p.stor_eff[sidx], Pm = p.stor_P[sidx], Em = p.stor_dur[sidx] * Pm;
  const float q = p.stor_cost[sidx];
  const float om = rho;
  float *lam = p.stor_lam + (size_t)sidx * SG_N * Tp;
  float *bet = p.stor_beta + (size_t)sidx * SG_N * Tp;
  float *mf = p.stor_m + (size_t)sidx * Tp;
  float *pd = p.PD + (size_t)d * T;
  float *dl_out = p.stor_delta + (size_t)sidx * T;
  float *X = sm, *TAU = sm + Tp, *S = sm + 2 * Tp;

  // 2x2 block of (c, delta) after eliminating p; constants of the reduction
  const float kap = rho * om / (rho + om);
  const float h00 = kap + 2.f * om + om * eta * eta, h01 = -kap - om * eta, h11 = kap + 3.f * om;
  const float det = h00 * h11 - h01 * h01;
  const float i00 = h11 / det, i01 = -h01 / det, i11 = h00 / det;
  const float f1c = om * eta, f1d = -om;
  const float w0 = i00 * f1c + i01 * f1d, w1 = i01 * f1c + i11 * f1d;
  const float gam = om - (f1c * w0 + f1d * w1);

  const float rho_old = p.stor_rho[sidx];
  if (rho_old != rho) {
    const float ls = (rho_old == 0.f) ? 1.f : fabsf(rho_old) / rho;
    for (int t = lane; t < SG_N * Tp; t += 32) lam[t] *= ls;
    if (lane == 0) {
      tri_factor(mf, Tp, gam + 3.f * om, 2.f * gam + 2.f * om, -gam);
      p.stor_rho[sidx] = rho;
    }
    __syncwarp();
  }
  for (int t = lane; t < T; t += 32) {
    size_t o = (size_t)n * T + t;
    X[t] = pd[t] - (p.SPBAR[o] + su * p.SU[o]) / kpf;
  }
  __syncwarp();
#define LAM(g, t) lam[(g) * Tp + (t)]
#define BET(g, t) bet[(g) * Tp + (t)]
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    for (int t = lane; t < T; t += 32) {
      const float r1 = -LAM(SG_E1, t), r2 = -LAM(SG_E2, t);
      const float mc = 0.5f * ((Pm + BET(SG_CU, t) - LAM(SG_CU, t)) - (BET(SG_CL, t) - LAM(SG_CL, t)));
      const float md = 0.5f * ((Pm + BET(SG_DU, t) - LAM(SG_DU, t)) - (BET(SG_DL, t) - LAM(SG_DL, t)));
      const float e1 = r1 - X[t];
      const float f0c = kap * e1 + 2.f * om * mc;
      const float f0d = -kap * e1 - q + 2.f * om * md;
      TAU[t] = r2 + (w0 * f0c + w1 * f0d) / gam;
    }
    __syncwarp();
    for (int j = lane; j < Tp; j += 32) {
      const float ms = 0.5f * ((Em + BET(SG_SU, j) - LAM(SG_SU, j)) - (BET(SG_SL, j) - LAM(SG_SL, j)));
      float rhs = 2.f * om * ms;
      if (j >= 1) rhs += gam * TAU[j - 1];
      if (j <= T - 1) rhs -= gam * TAU[j];
      if (j == 0) rhs -= om * LAM(SG_E3, 0);
      if (j == T) rhs -= om * LAM(SG_E3, 1);
      S[j] = rhs;
    }
    __syncwarp();
    warp_tri_solve(mf, -gam, S, Tp, lane);
    for (int t = lane; t < T; t += 32) {
      const float r1 = -LAM(SG_E1, t), r2 = -LAM(SG_E2, t);
      const float mc = 0.5f * ((Pm + BET(SG_CU, t) - LAM(SG_CU, t)) - (BET(SG_CL, t) - LAM(SG_CL, t)));
      const float md = 0.5f * ((Pm + BET(SG_DU, t) - LAM(SG_DU, t)) - (BET(SG_DL, t) - LAM(SG_DL, t)));
      const float e1 = r1 - X[t];
      const float f0c = kap * e1 + 2.f * om * mc;
      const float f0d = -kap * e1 - q + 2.f * om * md;
      const float s0 = S[t], s1 = S[t + 1];
      const float g = s1 - s0 - r2;
      const float fc = f0c + g * f1c, fd = f0d + g * f1d;
      const float c = i00 * fc + i01 * fd;
      const float dl = i01 * fc + i11 * fd;
      const float pt = (rho * X[t] + om * (r1 - c + dl)) / (rho + om);
      TAU[t] = pt;  // TAU is consumed; keep p_t for the end
      dl_out[t] = dl;
      float al, nb;
      LAM(SG_E1, t) += pt + c - dl;                  // equality rows: beta = 0
      LAM(SG_E2, t) += s1 - s0 - eta * c + dl;
      al = c - Pm;  nb = fminf(al + LAM(SG_CU, t), 0.f); LAM(SG_CU, t) += al - nb; BET(SG_CU, t) = nb;
      al = -c;      nb = fminf(al + LAM(SG_CL, t), 0.f); LAM(SG_CL, t) += al - nb; BET(SG_CL, t) = nb;
      al = dl - Pm; nb = fminf(al + LAM(SG_DU, t), 0.f); LAM(SG_DU, t) += al - nb; BET(SG_DU, t) = nb;
      al = -dl;     nb = fminf(al + LAM(SG_DL, t), 0.f); LAM(SG_DL, t) += al - nb; BET(SG_DL, t) = nb;
    }
    for (int j = lane; j < Tp; j += 32) {
      const float sj = S[j];
      float al, nb;
      if (j == 0) LAM(SG_E3, 0) += sj;
      if (j == T) LAM(SG_E3, 1) += sj;
      al = sj - Em; nb = fminf(al + LAM(SG_SU, j), 0.f); LAM(SG_SU, j) += al - nb; BET(SG_SU, j) = nb;
      al = -sj;     nb = fminf(al + LAM(SG_SL, j), 0.f); LAM(SG_SL, j) += al - nb; BET(SG_SL, j) = nb;
    }
    __syncwarp();
  }
#undef LAM
#undef BET
  for (int t = lane; t < T; t += 32) {
    const float pn = TAU[t];
    if (resid) p.DPD[(size_t)d * T + t] = pn - pd[t];
    pd[t] = pn;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// the persistent iteration kernel
// ---------------------------------------------------------------------------
template <int VW>
__global__ void __launch_bounds__(BLOCK, 2) iteration_kernel(Params p) {
  extern __shared__ float smem[];
  __shared__ double red[WARPS][NSLOT];
  __shared__ double dec[8];
  __shared__ int s_flag;

  const int T = p.T, TV = T / VW, Kp = p.Kp, L = p.L, N = p.N;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * WARPS + wib, nwarp = gridDim.x * WARPS;
  const long long gthr = (long long)blockIdx.x * BLOCK + threadIdx.x;
  const long long nthr = (long long)gridDim.x * BLOCK;
  float *wsm = smem + wib * 3 * (T + 1);

  const DevScalars sc0 = *p.sc;
  double rho_p = sc0.rho_p, rho_th = sc0.rho_th, su = sc0.su, sv = sc0.sv;
  double res[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) res[j] = sc0.res[j];
  long long it = sc0.it;
  int v_fresh = sc0.v_fresh, converged = sc0.converged, status = 0, dual_valid = sc0.dual_valid;
  const float kpf = (float)Kp;
  const int n_inner = p.n_stor + p.n_ramp;
  const long long n_closed_items = (long long)p.n_closed * TV;
  const long long n_line_items = (long long)Kp * L * TV;

  // a sticky device error (timeout, non-finite) leaves the state as it is
  const int n_iters = sc0.status ? 0 : p.n_iters;
  for (int i = 0; i < n_iters; ++i) {
    const long long itn = it + 1;
    const bool last = (i == n_iters - 1);
    const bool adapt_now = p.adapt_every > 0 && (itn % p.adapt_every) == 0;
    const bool check_now = p.eps > 0 && p.check_every > 0 && (itn % p.check_every) == 0;
    const bool resid = adapt_now || check_now || last;
    const int par = (int)(itn & 1);
    const float frp = (float)rho_p, frt = (float)rho_th;
    const float fsu = (float)su, fsv = (float)sv;
    const float rho_dev = (float)(Kp * rho_p);
    // per-thread partial sums in FP32; FP64 from the block reduction on
    float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f};

    // ---------------- phase A: proxes ----------------
    for (int w = gwarp; w < n_inner; w += nwarp) {
      if (w < p.n_stor)
        stor_prox(p, w, rho_dev, fsu, kpf, wsm, resid, lane);
      else
        ramp_prox(p, w - p.n_stor, rho_dev, fsu, kpf, wsm, resid, lane);
    }
    for (long long item = gthr; item < n_closed_items + n_line_items; item += nthr) {
      if (item < n_closed_items) {
        const int ci = (int)(item / TV), tc = (int)(item % TV);
        const int d = p.closed_ids[ci];
        const int nd = p.dev_node[d];
        const size_t od = (size_t)d * T + tc * VW, on = (size_t)nd * T + tc * VW;
        FV<VW> pd = ldv<VW>(p.PD + od);
        const FV<VW> sp = ldv<VW>(p.SPBAR + on), sum_u = ldv<VW>(p.SU + on);
        const FV<VW> lo = ldv<VW>(p.dev_lo + od), hi = ldv<VW>(p.dev_hi + od);
        const float a = p.dev_a[d], b = p.dev_b[d];
        const float den = 2.f * a + rho_dev;
        FV<VW> dpd;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const float x = pd.v[e] - (sp.v[e] + fsu * sum_u.v[e]) / kpf;
          const float pn = fminf(fmaxf((rho_dev * x - b) / den, lo.v[e]), hi.v[e]);
          dpd.v[e] = pn - pd.v[e];
          pd.v[e] = pn;
        }
        stv<VW>(p.PD + od, pd);
        if (resid) stv<VW>(p.DPD + od, dpd);
      } else {
        const long long li = item - n_closed_items;
        const int k = (int)(li / ((long long)L * TV));
        const long long rem = li - (long long)k * L * TV;
        const int l = (int)(rem / TV), tc = (int)(rem % TV);
        const int n1 = p.line_n1[l], n2 = p.line_n2[l];
        const bool act = p.out_line[k] != l;
        const size_t ol = ((size_t)k * L + l) * T + tc * VW;
        const size_t o1 = ((size_t)k * N + n1) * T + tc * VW;
        const size_t o2 = ((size_t)k * N + n2) * T + tc * VW;
        FV<VW> P = ldv_cs<VW>(p.P + ol), A1 = ldv_cs<VW>(p.TH1 + ol), A2 = ldv_cs<VW>(p.TH2 + ol);
        FV<VW> V1 = ldv_cs<VW>(p.V1 + ol), V2 = ldv_cs<VW>(p.V2 + ol);
        const FV<VW> U1 = ldv<VW>(p.U + o1), U2 = ldv<VW>(p.U + o2);
        const FV<VW> B1 = ldv<VW>(p.PBAR + o1), B2 = ldv<VW>(p.PBAR + o2);
        const FV<VW> G1 = ldv<VW>(p.THBAR + o1), G2 = ldv<VW>(p.THBAR + o2);
        // line prox (Section 4.2 closed form, denominator as derived in the oracle)
        float tb = 1.f, den = 1.f, ulim = 0.f;
        if (act) {
          const float bb = p.line_b[l];
          ulim = p.line_u[l];
          tb = 2.f * bb;
          den = 2.f * frp + frt / (tb * bb);
        }
        FV<VW> DPv;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const float x1 = -P.v[e] - B1.v[e] - fsu * U1.v[e];
          const float x2 = P.v[e] - B2.v[e] - fsu * U2.v[e];
          const float v1 = v_fresh ? fsv * V1.v[e] : fsv * (V1.v[e] + (A1.v[e] - G1.v[e]));
          const float v2 = v_fresh ? fsv * V2.v[e] : fsv * (V2.v[e] + (A2.v[e] - G2.v[e]));
          const float y1 = G1.v[e] - v1, y2 = G2.v[e] - v2;
          float pn, t1, t2;
          if (act) {
            const float num = frp * (x2 - x1) + frt * (y1 - y2) / tb;
            pn = fminf(fmaxf(num / den, -ulim), ulim);
            const float mid = 0.5f * (y1 + y2);
            const float h = pn / tb;
            t1 = mid + h;
            t2 = mid - h;
          } else {
            pn = 0.f;
            t1 = y1;
            t2 = y2;
          }
          DPv.v[e] = pn - P.v[e];
          P.v[e] = pn;
          A1.v[e] = t1;
          A2.v[e] = t2;
          V1.v[e] = v1;
          V2.v[e] = v2;
        }
        stv_cs<VW>(p.P + ol, P);
        stv_cs<VW>(p.TH1 + ol, A1);
        stv_cs<VW>(p.TH2 + ol, A2);
        stv_cs<VW>(p.V1 + ol, V1);
        stv_cs<VW>(p.V2 + ol, V2);
        if (resid) stv_cs<VW>(p.DP + ol, DPv);
      }
    }
    if (!grid_barrier(p, &s_flag)) { status = ST_TIMEOUT; break; }

    // ---------------- phase B: node averages, prices, residual partials ----------------
    for (long long item = gthr; item < (long long)N * TV; item += nthr) {
      const int n = (int)(item / TV), tc = (int)(item % TV);
      const int l0 = p.lcsr_ptr[n], l1 = p.lcsr_ptr[n + 1];
      const int d0 = p.dcsr_ptr[n], d1 = p.dcsr_ptr[n + 1];
      const float cp = p.cnt_p[n], ct = p.cnt_th[n];
      FV<VW> devsum;
#pragma unroll
      for (int e = 0; e < VW; ++e) devsum.v[e] = 0.f;
      for (int j = d0; j < d1; ++j) {
        const FV<VW> x = ldv<VW>(p.PD + (size_t)p.dcsr_idx[j] * T + tc * VW);
#pragma unroll
        for (int e = 0; e < VW; ++e) devsum.v[e] += x.v[e];
      }
      FV<VW> sumpb, sumu;
#pragma unroll
      for (int e = 0; e < VW; ++e) { sumpb.v[e] = 0.f; sumu.v[e] = 0.f; }
      for (int k = 0; k < Kp; ++k) {
        FV<VW> sp = devsum, st;
#pragma unroll
        for (int e = 0; e < VW; ++e) st.v[e] = 0.f;
        const size_t kb = (size_t)k * L * T + tc * VW;
        for (int j = l0; j < l1; ++j) {
          const int code = p.lcsr_idx[j];
          const size_t ol = kb + (size_t)(code >> 1) * T;
          const FV<VW> pl = ldv<VW>(p.P + ol);
          const FV<VW> th = ldv<VW>(((code & 1) ? p.TH2 : p.TH1) + ol);
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            sp.v[e] += (code & 1) ? pl.v[e] : -pl.v[e];
            st.v[e] += th.v[e];
          }
        }
        const size_t on = ((size_t)k * N + n) * T + tc * VW;
        FV<VW> u = ldv<VW>(p.U + on), pb, tbar, dpb;
        FV<VW> pb_old, tb_old;
        if (resid) {
          pb_old = ldv<VW>(p.PBAR + on);
          tb_old = ldv<VW>(p.THBAR + on);
        }
        float a_pp = 0.f, a_pt = 0.f, a_dp = 0.f, a_dt = 0.f, a_nf = 0.f;
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          pb.v[e] = sp.v[e] / cp;                              // Eq. (average-op)
          tbar.v[e] = ct > 0.f ? st.v[e] / ct : 0.f;
          u.v[e] = fsu * u.v[e] + pb.v[e];                      // u += pbar
          sumpb.v[e] += pb.v[e];
          sumu.v[e] += u.v[e];
          a_pp += cp * pb.v[e] * pb.v[e];
          if (!isfinite(u.v[e]) || !isfinite(tbar.v[e])) a_nf += 1.f;
          if (resid) {
            dpb.v[e] = pb.v[e] - pb_old.v[e];
            const float ddt = tbar.v[e] - tb_old.v[e];
            a_dt += ct * ddt * ddt;
          }
        }
        // second pass over the terminals (rows are L1-resident): theta~ and p~ change
        for (int j = l0; j < l1; ++j) {
          const int code = p.lcsr_idx[j];
          const size_t ol = kb + (size_t)(code >> 1) * T;
          const FV<VW> th = ldv<VW>(((code & 1) ? p.TH2 : p.TH1) + ol);
#pragma unroll
          for (int e = 0; e < VW; ++e) {
            const float r = th.v[e] - tbar.v[e];
            a_pt += r * r;
          }
          if (resid) {
            const FV<VW> dl = ldv<VW>(p.DP + ol);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
              const float r = ((code & 1) ? dl.v[e] : -dl.v[e]) - dpb.v[e];
              a_dp += r * r;
            }
          }
        }
        if (resid) {
          for (int j = d0; j < d1; ++j) {
            const FV<VW> dd = ldv<VW>(p.DPD + (size_t)p.dcsr_idx[j] * T + tc * VW);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
              const float r = dd.v[e] - dpb.v[e];
              a_dp += r * r;
            }
          }
        }
        acc[SL_PP] += a_pp;
        acc[SL_PT] += a_pt;
        acc[SL_DP] += a_dp;
        acc[SL_DT] += a_dt;
        acc[SL_NF] += a_nf;
        stv<VW>(p.U + on, u);
        stv<VW>(p.PBAR + on, pb);
        stv<VW>(p.THBAR + on, tbar);
      }
      stv<VW>(p.SPBAR + (size_t)n * T + tc * VW, sumpb);
      stv<VW>(p.SU + (size_t)n * T + tc * VW, sumu);
    }
    // block reduction of the partials in FP64
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      double v = (double)acc[s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wib][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
      double v = 0.0;
      for (int w = 0; w < WARPS; ++w) v += red[w][threadIdx.x];
      p.partials[((size_t)par * gridDim.x + blockIdx.x) * NSLOT + threadIdx.x] = v;
    }
    if (!grid_barrier(p, &s_flag)) { status = ST_TIMEOUT; break; }

    // ---------------- phase C: residuals and decisions (same in every CTA) ----------------
    if (wib == 0) {
      double tot[NSLOT];
#pragma unroll
      for (int s = 0; s < NSLOT; ++s) tot[s] = 0.0;
      const double *base = p.partials + (size_t)par * gridDim.x * NSLOT;
      for (int b = lane; b < (int)gridDim.x; b += 32) {
        double v[NSLOT];
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) v[s] = __ldcg(base + (size_t)b * NSLOT + s);
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) tot[s] += v[s];
      }
#pragma unroll
      for (int s = 0; s < NSLOT; ++s) {
        double v = tot[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        tot[s] = v;
      }
      if (lane == 0) {
        const double r_pp = sqrt(fmax(tot[SL_PP], 0.0));
        const double r_pt = sqrt(fmax(tot[SL_PT], 0.0));
        const double r_dp = rho_p * sqrt(fmax(tot[SL_DP], 0.0));
        const double r_dt = rho_th * sqrt(fmax(tot[SL_DT], 0.0));
        const double rp = sqrt(r_pp * r_pp + r_pt * r_pt);
        const double rd = sqrt(r_dp * r_dp + r_dt * r_dt);
        double stop = 0.0, st = 0.0, nrp = rho_p, nrt = rho_th;
        if (!isfinite(rp) || (resid && !isfinite(rd)) || tot[SL_NF] != 0.0) {
          st = ST_NONFINITE;
          stop = 1.0;
        } else {
          if (check_now && fmax(rp, rd) <= p.tol) stop = 2.0;
          if (adapt_now) {
            if (r_pp > p.mu * r_dp) nrp = rho_p * p.gamma;
            else if (r_dp > p.mu * r_pp) nrp = rho_p / p.gamma;
            if (r_pt > p.mu * r_dt) nrt = rho_th * p.gamma;
            else if (r_dt > p.mu * r_pt) nrt = rho_th / p.gamma;
          }
        }
        dec[0] = rp; dec[1] = resid ? rd : res[1];
        dec[2] = r_pp; dec[3] = r_pt;
        dec[4] = resid ? r_dp : res[4]; dec[5] = resid ? r_dt : res[5];
        dec[6] = stop + 4.0 * st;
        red[0][0] = nrp;
        red[0][1] = nrt;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 6; ++j) res[j] = dec[j];
    const int code = (int)dec[6];
    const double nrp = red[0][0], nrt = red[0][1];
    __syncthreads();  // red is rewritten in the next iteration
    su = rho_p / nrp;
    sv = rho_th / nrt;
    rho_p = nrp;
    rho_th = nrt;
    it = itn;
    v_fresh = 0;
    dual_valid = resid ? 1 : 0;
    if ((code & 3) == 2) converged = 1;
    if (code >= 4) status = code >> 2;
    if (code != 0) break;
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevScalars sc = sc0;
    sc.rho_p = rho_p;
    sc.rho_th = rho_th;
    sc.su = su;
    sc.sv = sv;
    for (int j = 0; j < 6; ++j) sc.res[j] = res[j];
    sc.it = it;
    sc.converged = converged;
    int e = *(volatile int *)p.err;
    sc.status = status ? status : (e ? e : sc0.status);
    sc.v_fresh = v_fresh;
    sc.dual_valid = dual_valid;
    *p.sc = sc;
  }
}

// ---------------------------------------------------------------------------
// auxiliary kernels: averages after a state import, deferred-v export,
// prices, v projection on import
// ---------------------------------------------------------------------------
__global__ void node_average_kernel(Params p) {
  const int T = p.T, N = p.N, L = p.L;
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x; item < (long long)N * T;
       item += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(item / T), t = (int)(item % T);
    float devsum = 0.f;
    for (int j = p.dcsr_ptr[n]; j < p.dcsr_ptr[n + 1]; ++j) devsum += p.PD[(size_t)p.dcsr_idx[j] * T + t];
    float sumpb = 0.f, sumu = 0.f;
    for (int k = 0; k < p.Kp; ++k) {
      float sp = devsum, st = 0.f;
      for (int j = p.lcsr_ptr[n]; j < p.lcsr_ptr[n + 1]; ++j) {
        const int code = p.lcsr_idx[j];
        const size_t ol = ((size_t)k * L + (code >> 1)) * T + t;
        sp += (code & 1) ? p.P[ol] : -p.P[ol];
        st += (code & 1) ? p.TH2[ol] : p.TH1[ol];
      }
      const size_t on = ((size_t)k * N + n) * T + t;
      const float pb = sp / p.cnt_p[n];
      p.PBAR[on] = pb;
      p.THBAR[on] = p.cnt_th[n] > 0.f ? st / p.cnt_th[n] : 0.f;
      sumpb += pb;
      sumu += p.U[on];
    }
    p.SPBAR[(size_t)n * T + t] = sumpb;
    p.SU[(size_t)n * T + t] = sumu;
  }
}

// v projected onto v_bar = 0 per node and contingency (Appendix C)
__global__ void project_v_kernel(Params p) {
  const int T = p.T, N = p.N, L = p.L;
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
       item < (long long)p.Kp * N * T; item += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(item / ((long long)N * T));
    const long long rem = item - (long long)k * N * T;
    const int n = (int)(rem / T), t = (int)(rem % T);
    const int l0 = p.lcsr_ptr[n], l1 = p.lcsr_ptr[n + 1];
    if (l1 == l0) continue;
    float s = 0.f;
    for (int j = l0; j < l1; ++j) {
      const int code = p.lcsr_idx[j];
      const size_t ol = ((size_t)k * L + (code >> 1)) * T + t;
      s += (code & 1) ? p.V2[ol] : p.V1[ol];
    }
    const float m = s / p.cnt_th[n];
    for (int j = l0; j < l1; ++j) {
      const int code = p.lcsr_idx[j];
      const size_t ol = ((size_t)k * L + (code >> 1)) * T + t;
      if (code & 1) p.V2[ol] -= m; else p.V1[ol] -= m;
    }
  }
}

// current v = sv * (V + theta - theta_bar) (deferred update), or sv * V when fresh
__global__ void export_v_kernel(Params p, float *v1, float *v2) {
  const DevScalars sc = *p.sc;
  const float sv = (float)sc.sv;
  const int T = p.T, N = p.N, L = p.L;
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
       item < (long long)p.Kp * L * T; item += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(item / ((long long)L * T));
    const long long rem = item - (long long)k * L * T;
    const int l = (int)(rem / T), t = (int)(rem % T);
    const size_t ol = item;
    float a = p.V1[ol], b = p.V2[ol];
    if (!sc.v_fresh) {
      a += p.TH1[ol] - p.THBAR[((size_t)k * N + p.line_n1[l]) * T + t];
      b += p.TH2[ol] - p.THBAR[((size_t)k * N + p.line_n2[l]) * T + t];
    }
    if (v1) v1[ol] = sv * a;
    if (v2) v2[ol] = sv * b;
  }
}

__global__ void export_u_kernel(Params p, float *u) {
  const float su = (float)p.sc->su;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)p.Kp * p.N * p.T;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = su * p.U[i];
}

// price_{n,t} = -rho_p * sum_k u_{k,n,t} with the pending rescale applied
__global__ void price_kernel(Params p, float *price) {
  const DevScalars sc = *p.sc;
  const double f = -sc.rho_p * sc.su;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)p.N * p.T;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < p.Kp; ++k) s += p.U[(size_t)k * p.N * p.T + i];
    price[i] = (float)(f * s);
  }
}

__global__ void set_rho_kernel(DevScalars *sc, double rho) {
  DevScalars s = *sc;
  s.su *= s.rho_p / rho;
  s.sv *= s.rho_th / rho;
  s.rho_p = rho;
  s.rho_th = rho;
  *sc = s;
}

static size_t iteration_smem(int T) { return (size_t)WARPS * 3 * (T + 1) * sizeof(float); }

}  // namespace opfk

using namespace opfk;

int opfk_max_grid(int T, int *grid) {
  int dev = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  cudaError_t e;
  if (T % 4 == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<4>, BLOCK, iteration_smem(T));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<1>, BLOCK, iteration_smem(T));
  if (e != cudaSuccess || nb < 1) return -1;
  *grid = nb * sms;
  return 0;
}

int opfk_iteration_launch(const Params &p, void *stream, int *grid_used, char *msg, int msglen) {
  cudaStream_t s = (cudaStream_t)stream;
  int grid = *grid_used;
  size_t sm = iteration_smem(p.T);
  if (sm > 48 * 1024) {
    cudaError_t e = (p.T % 4 == 0)
        ? cudaFuncSetAttribute(iteration_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
        : cudaFuncSetAttribute(iteration_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) {
      snprintf(msg, msglen, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return -1;
    }
  }
  Params pp = p;
  void *args[] = {&pp};
  cudaError_t e = (p.T % 4 == 0)
      ? cudaLaunchCooperativeKernel((void *)iteration_kernel<4>, dim3(grid), dim3(BLOCK), args, sm, s)
      : cudaLaunchCooperativeKernel((void *)iteration_kernel<1>, dim3(grid), dim3(BLOCK), args, sm, s);
  if (e != cudaSuccess) {
    snprintf(msg, msglen, "cudaLaunchCooperativeKernel: %s", cudaGetErrorString(e));
    return -1;
  }
  return 0;
}

static int aux_grid(long long work) {
  long long g = (work + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int opfk_node_average_launch(const Params &p, void *stream) {
  node_average_kernel<<<aux_grid((long long)p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_project_v_launch(const Params &p, void *stream) {
  project_v_kernel<<<aux_grid((long long)p.Kp * p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_export_v_launch(const Params &p, float *v1, float *v2, void *stream) {
  export_v_kernel<<<aux_grid((long long)p.Kp * p.L * p.T), 256, 0, (cudaStream_t)stream>>>(p, v1, v2);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_export_u_launch(const Params &p, float *u, void *stream) {
  export_u_kernel<<<aux_grid((long long)p.Kp * p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p, u);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_price_launch(const Params &p, float *price, void *stream) {
  price_kernel<<<aux_grid((long long)p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p, price);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_set_rho_launch(DevScalars *sc, double rho, void *stream) {
  set_rho_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(sc, rho);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
