// Proximal message passing for contingency-constrained DC OPF -- sm_103a kernels.
//
// One iteration of the message-passing form of ADMM (Section 3.2) is seven
// kernels replayed from CUDA graphs; each reads the iteration's scalars
// (penalties, pending rescales, buffer parity, whether residuals are read)
// from the device, so the same graph serves every iteration:
//   xs     step 2 input: avg_k(pbar + u) from the stored pbar + u at every
//          node with devices (a node's K+1 rows are one run), and the
//          closed-form prox with weight (K+1) rho_p of its generators/loads;
//   inner  step 2, one warp per ramp-limited generator, battery or HVDC link:
//          the inner ADMM of Appendix D (lanes over time steps, tridiagonal
//          x-updates by warp-wide scans) or the link's closed form;
//   dsum   the node sums of device powers and their Welford change state;
//   line   step 1, one thread per (line, contingency, 4 time steps): the line
//          prox from the previous iterate at both ends (second stream, beside
//          xs, inner and dsum), the deferred v update, over-relaxed blends;
//   node   step 3 where the residuals are read (stopping test, adaptation,
//          end of a call): pbar, theta_bar, u += pbar as register sums over
//          the node's terminals in CSR order (no atomics), the residual
//          partial sums (one-pass Welford sums); node_lean does step 3 alone
//          on the other iterations (each returns at once on the other's);
//   decide FP64 reduction of the partial sums in a fixed order, stopping
//          test and adaptive penalty (Section 3.5); advances the counter.
//
// Splitting the phases lets each kernel run at its own register budget.
// There is no spin-wait on the device: ordering comes from kernel boundaries
// and graph edges.  Every kernel body also serves a batch of independent
// instances: the batch entry points take the instances' parameters and a
// CTA schedule, so one launch per phase covers all instances.
//
// Memory layout (line- and node-major), numbering and the deferred v
// update: opf_internal.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "opf_internal.h"

namespace opfk {

constexpr int WARPS = BLOCK / 32;
constexpr int ST_NONFINITE = 5;  // opf_status value set on the device
constexpr int NODE_VW = 4;       // time steps per node item
constexpr int NODE_MIN_CTAS = 2; // resident CTAs per SM the node kernel is compiled for
constexpr int LINE_IPT = 4;      // line items per thread (CTA-sized blocks of items)
constexpr int N_SLABS = 1;       // contingency slabs per iteration (line / node overlap)
constexpr int NODE_LEAN_CTAS = 4;  // resident CTAs per SM of the residual-free node pass
constexpr int NODE_LEAN_NB = 2;    // line terminals it gathers together
constexpr int REG_T = 127;         // longest horizon of the register-resident inner ADMM (T + 1 <= 4 x 32)

// shared floats per warp of the shared-memory inner ADMM: 3 (T+1) for the
// work arrays, plus room for one device's (lam, beta) while the horizon is
// short enough
__host__ __device__ inline int warp_smem_floats(int T) {
  const int work = 3 * (T + 1), state = 2 * SG_N * (T + 1);
  return T <= 128 ? work + state : work;
}

// register chunk of the inner ADMM at horizon T: a battery's T + 1 elements
// over 32 lanes (1 .. 4); 0 beyond REG_T (the shared-memory path)
__host__ __device__ inline int inner_chunk(int T) { return T <= REG_T ? (T + 32) >> 5 : 0; }

// ---------------------------------------------------------------------------
// The inner ADMM (Appendix D) writes every product, sum and quotient with its
// rounding (__fmul_rn, __fadd_rn, __fmaf_rn, ...), which the compiler may not
// contract or reorder: its shared-memory and register forms, and each kernel
// that inlines them (one instance, a batch), compute the same bits.
// ---------------------------------------------------------------------------
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// one projected dual step of an inequality row (Appendix D): lam += al - nb,
// beta = nb = min(al + lam, 0)
__device__ __forceinline__ void ineq_step(float al, float &lam, float &bet) {
  const float nb = fminf(radd(al, lam), 0.f);
  lam = radd(lam, rsub(al, nb));
  bet = nb;
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
    const float qi = (i == 0) ? d : rsub(d, rmul(off, rdiv(off, prev)));
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
  const float noff = -off;
  // forward (r_i = buf_i / q_i is kept in buf for the second pass)
  float Ac = 1.f, Bc = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float ri = rdiv(buf[i], q[i]);
    const float Ai = (i == 0) ? 0.f : rdiv(noff, q[i]);
    buf[i] = ri;
    Bc = rfma(Ai, Bc, ri);
    Ac = rmul(Ai, Ac);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_up_sync(FULL, Ac, d);
    const float Bp = __shfl_up_sync(FULL, Bc, d);
    if (lane >= d) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float prev = __shfl_up_sync(FULL, Bc, 1);
  if (lane == 0) prev = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float Ai = (i == 0) ? 0.f : rdiv(noff, q[i]);
    prev = rfma(Ai, prev, buf[i]);
    buf[i] = prev;
  }
  __syncwarp();
  // backward
  Ac = 1.f;
  Bc = 0.f;
  for (int i = i1 - 1; i >= i0; --i) {
    const float Ci = (i == n - 1) ? 0.f : rdiv(noff, q[i]);
    Bc = rfma(Ci, Bc, buf[i]);
    Ac = rmul(Ci, Ac);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_down_sync(FULL, Ac, d);
    const float Bp = __shfl_down_sync(FULL, Bc, d);
    if (lane + d < 32) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float nxt = __shfl_down_sync(FULL, Bc, 1);
  if (lane == 31) nxt = 0.f;
  for (int i = i1 - 1; i >= i0; --i) {
    const float Ci = (i == n - 1) ? 0.f : rdiv(noff, q[i]);
    nxt = rfma(Ci, nxt, buf[i]);
    buf[i] = nxt;
  }
  __syncwarp();
}

// sums over contingencies k of two node arrays (pbar + u and u; u_o may be
// NULL, giving 0) at one (node, t) offset o, with 8 independent loads in
// flight per step
__device__ __forceinline__ void ksum(const float *pbar_o, const float *u_o, size_t o, size_t stride, int Kp,
                                     float &sp, float &sq) {
  float a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) { a[j] = 0.f; b[j] = 0.f; }
  int k = 0;
  for (; k + 8 <= Kp; k += 8) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] += pbar_o[(size_t)(k + j) * stride + o];
      b[j] += u_o ? u_o[(size_t)(k + j) * stride + o] : 0.f;
    }
  }
  for (; k < Kp; ++k) {
    a[0] += pbar_o[(size_t)k * stride + o];
    b[0] += u_o ? u_o[(size_t)k * stride + o] : 0.f;
  }
  sp = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  sq = ((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + (b[6] + b[7]));
}

// The same sums for four consecutive time steps (o 16-byte aligned): one
// 128-bit load per row, two rows of each array in flight per step.
__device__ __forceinline__ void ksum4(const float *pbar_o, const float *u_o, size_t o, size_t stride, int Kp,
                                      float4 &sp, float4 &sq) {
  float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
  int k = 0;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (; k + 2 <= Kp; k += 2) {
    const float4 x0 = *reinterpret_cast<const float4 *>(pbar_o + (size_t)k * stride + o);
    const float4 x1 = *reinterpret_cast<const float4 *>(pbar_o + (size_t)(k + 1) * stride + o);
    const float4 y0 = u_o ? *reinterpret_cast<const float4 *>(u_o + (size_t)k * stride + o) : z;
    const float4 y1 = u_o ? *reinterpret_cast<const float4 *>(u_o + (size_t)(k + 1) * stride + o) : z;
    a0.x += x0.x; a0.y += x0.y; a0.z += x0.z; a0.w += x0.w;
    a1.x += x1.x; a1.y += x1.y; a1.z += x1.z; a1.w += x1.w;
    b0.x += y0.x; b0.y += y0.y; b0.z += y0.z; b0.w += y0.w;
    b1.x += y1.x; b1.y += y1.y; b1.z += y1.z; b1.w += y1.w;
  }
  if (k < Kp) {
    const float4 x = *reinterpret_cast<const float4 *>(pbar_o + (size_t)k * stride + o);
    const float4 y = u_o ? *reinterpret_cast<const float4 *>(u_o + (size_t)k * stride + o) : z;
    a0.x += x.x; a0.y += x.y; a0.z += x.z; a0.w += x.w;
    b0.x += y.x; b0.y += y.y; b0.z += y.z; b0.w += y.w;
  }
  sp = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
  sq = make_float4(b0.x + b1.x, b0.y + b1.y, b0.z + b1.z, b0.w + b1.w);
}

// X[t] = p_d[t] - avg_k(pbar + u) at the device's node n, t in [0, T), by
// one warp (Section 3.2 step 2 input); the average was formed this iteration
// by the node-average items into XS
// Over-relaxation (Section 3.6) in the form kept on the device: the stored
// schedules are the relaxed P = alpha p + (1 - alpha) P_prev, whose node
// averages are the copies' complements (z = P - avg_n P, xi = avg_n Theta);
// alpha = 1 returns p exactly.
__device__ __forceinline__ float relaxed(float alpha, float pnew, float pold) {
  return rfma(alpha, pnew, rmul(rsub(1.f, alpha), pold));
}

__device__ __forceinline__ void device_x(const Params &p, int n, const float *pd, float *X, int lane) {
  const int T = p.T;
  const float *xs = p.XS + (size_t)n * T;
  for (int t = lane; t < T; t += 32) X[t] = rsub(pd[t], __ldcg(xs + t));
  __syncwarp();
}

// The warp's inner-ADMM state (lam, beta) lives in shared memory during the
// inner iterations when it fits (lam_sh != nullptr), else in global memory.
__device__ __forceinline__ void stage_in(float *&lam, float *&bet, float *lam_sh, int n, int lane) {
  if (!lam_sh) return;
  float *bsh = lam_sh + n;
  for (int i = lane; i < n; i += 32) {
    lam_sh[i] = lam[i];
    bsh[i] = bet[i];
  }
  __syncwarp();
  lam = lam_sh;
  bet = bsh;
}

__device__ __forceinline__ void stage_out(float *lam_g, float *bet_g, const float *lam_sh, int n, int lane) {
  if (!lam_sh) return;
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    lam_g[i] = lam_sh[i];
    bet_g[i] = lam_sh[n + i];
  }
}

// ---------------------------------------------------------------------------
// Appendix D inner ADMM, ramp-limited generator (one warp, lanes over t).
// Rows: p_t <= pmax_t, -p_t <= -pmin_t, p_{t+1} - p_t <= R, p_t - p_{t+1} <= R.
// x-update matrix (2a + rho + 2 omega) I + 2 omega D'D is tridiagonal.
// ---------------------------------------------------------------------------
__device__ void ramp_prox(const Params &p, int r, float rho, float *sm, float *state_sh, int lane) {
  const int T = p.T;
  const int d = p.ramp_ids[r];
  const int n = p.dev_node[d];
  const float a = p.dev_a[d], b = p.dev_b[d], R = p.ramp_R[r];
  const float om = rho, om2 = rmul(2.f, om);
  float *const lam_g = p.ramp_lam + (size_t)r * RG_N * T;
  float *const bet_g = p.ramp_beta + (size_t)r * RG_N * T;
  float *lam = lam_g, *bet = bet_g;
  stage_in(lam, bet, state_sh, RG_N * T, lane);
  float *mf = p.ramp_q + (size_t)r * T;
  const float *lo = p.dev_lo + (size_t)d * T;
  const float *hi = p.dev_hi + (size_t)d * T;
  float *pd = p.PD + (size_t)d * T;
  float *X = sm, *W = sm + (T + 1), *Z = sm + 2 * (T + 1);

  // keep the unscaled inner duals omega * lam when omega changes; refactor
  // (2a + rho + 2 omega) I + 2 omega D'D
  const float rho_old = p.ramp_rho[r];
  if (rho_old != rho) {
    const float ls = (rho_old == 0.f) ? 1.f : rdiv(fabsf(rho_old), rho);
    for (int t = lane; t < RG_N * T; t += 32) lam[t] = rmul(lam[t], ls);
    if (lane == 0) {
      const float base = radd(rmul(2.f, a), rho);
      tri_factor(mf, T, radd(base, rmul(4.f, om)), radd(base, rmul(6.f, om)), -om2);
      p.ramp_rho[r] = rho;
    }
    __syncwarp();
  }
  device_x(p, n, pd, X, lane);   // p_d - avg_k(pbar + u)
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    for (int t = lane; t < T - 1; t += 32)
      W[t] = rsub(rsub(bet[RG_RU * T + t], lam[RG_RU * T + t]), rsub(bet[RG_RD * T + t], lam[RG_RD * T + t]));
    __syncwarp();
    for (int t = lane; t < T; t += 32) {
      float atr = rsub(rsub(radd(hi[t], bet[RG_UP * T + t]), lam[RG_UP * T + t]),
                       rsub(radd(-lo[t], bet[RG_LO * T + t]), lam[RG_LO * T + t]));
      if (t >= 1) atr = radd(atr, W[t - 1]);
      if (t <= T - 2) atr = rsub(atr, W[t]);
      Z[t] = rfma(om, atr, rfma(rho, X[t], -b));
    }
    __syncwarp();
    warp_tri_solve(mf, -om2, Z, T, lane);
    for (int t = lane; t < T; t += 32) {
      const float pt = Z[t];
      ineq_step(rsub(pt, hi[t]), lam[RG_UP * T + t], bet[RG_UP * T + t]);
      ineq_step(rsub(lo[t], pt), lam[RG_LO * T + t], bet[RG_LO * T + t]);
      if (t < T - 1) {
        const float pn = Z[t + 1];
        ineq_step(rsub(rsub(pn, pt), R), lam[RG_RU * T + t], bet[RG_RU * T + t]);
        ineq_step(rsub(rsub(pt, pn), R), lam[RG_RD * T + t], bet[RG_RD * T + t]);
      }
    }
    __syncwarp();
  }
  stage_out(lam_g, bet_g, state_sh, RG_N * T, lane);
  for (int t = lane; t < T; t += 32) {
    const float pn = relaxed(p.alpha, Z[t], pd[t]);
    p.DPD[(size_t)d * T + t] = rsub(pn, pd[t]);
    pd[t] = pn;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// HVDC link (one warp, lanes over t): with x_i = p_i - avg_k(pbar + u) at
// terminal i, p2 = clip((x2 - x1) / 2, -u, u) and p1 = -p2 (the minimiser
// of the two squared distances over p1 + p2 = 0, clipped to the limit)
// ---------------------------------------------------------------------------
__device__ void hvdc_prox(const Params &p, int h, int lane) {
  const int T = p.T;
  const int d1 = p.hvdc0 + 2 * h, d2 = d1 + 1;
  const float u = p.hvdc_u[h];
  const float *xs1 = p.XS + (size_t)p.dev_node[d1] * T, *xs2 = p.XS + (size_t)p.dev_node[d2] * T;
  float *pd1 = p.PD + (size_t)d1 * T, *pd2 = p.PD + (size_t)d2 * T;
  for (int t = lane; t < T; t += 32) {
    const float q1 = pd1[t], q2 = pd2[t];
    const float x1 = q1 - __ldcg(xs1 + t), x2 = q2 - __ldcg(xs2 + t);
    const float f = fminf(fmaxf(0.5f * (x2 - x1), -u), u);
    const float r1 = relaxed(p.alpha, -f, q1), r2 = relaxed(p.alpha, f, q2);
    p.DPD[(size_t)d1 * T + t] = r1 - q1;
    p.DPD[(size_t)d2 * T + t] = r2 - q2;
    pd1[t] = r1;
    pd2[t] = r2;
  }
}

// ---------------------------------------------------------------------------
// Appendix D inner ADMM, battery (one warp, lanes over t).  Variables
// (p, c, delta, s), rows as in opf.h.  The x-update eliminates p_t, then
// (c_t, delta_t) per step (a 2x2 Schur complement), leaving a tridiagonal
// system of size T + 1 in the state of charge s.
// ---------------------------------------------------------------------------
__device__ void stor_prox(const Params &p, int sidx, float rho, float *sm, float *state_sh, int lane) {
  const int T = p.T, Tp = T + 1;
  const int d = p.stor_ids[sidx];
  const int n = p.dev_node[d];
  const float eta = p.stor_eff[sidx], Pm = p.stor_P[sidx], Em = rmul(p.stor_dur[sidx], Pm);
  const float q = p.stor_cost[sidx];
  const float om = rho, om2 = rmul(2.f, om);
  float *const lam_g = p.stor_lam + (size_t)sidx * SG_N * Tp;
  float *const bet_g = p.stor_beta + (size_t)sidx * SG_N * Tp;
  float *lam = lam_g, *bet = bet_g;
  stage_in(lam, bet, state_sh, SG_N * Tp, lane);
  float *mf = p.stor_q + (size_t)sidx * Tp;
  float *pd = p.PD + (size_t)d * T;
  float *dl_out = p.stor_delta + (size_t)sidx * T;
  float *X = sm, *TAU = sm + Tp, *S = sm + 2 * Tp;

  // 2x2 block of (c, delta) after eliminating p; constants of the reduction
  const float kap = rdiv(rmul(rho, om), radd(rho, om));
  const float h00 = radd(radd(kap, om2), rmul(rmul(om, eta), eta));
  const float h01 = rsub(-kap, rmul(om, eta)), h11 = radd(kap, rmul(3.f, om));
  const float det = rsub(rmul(h00, h11), rmul(h01, h01));
  const float i00 = rdiv(h11, det), i01 = rdiv(-h01, det), i11 = rdiv(h00, det);
  const float f1c = rmul(om, eta), f1d = -om;
  const float w0 = radd(rmul(i00, f1c), rmul(i01, f1d)), w1 = radd(rmul(i01, f1c), rmul(i11, f1d));
  const float gam = rsub(om, radd(rmul(f1c, w0), rmul(f1d, w1)));
  const float rpo = radd(rho, om);

  const float rho_old = p.stor_rho[sidx];
  if (rho_old != rho) {
    const float ls = (rho_old == 0.f) ? 1.f : rdiv(fabsf(rho_old), rho);
    for (int t = lane; t < SG_N * Tp; t += 32) lam[t] = rmul(lam[t], ls);
    if (lane == 0) {
      tri_factor(mf, Tp, radd(gam, rmul(3.f, om)), radd(rmul(2.f, gam), om2), -gam);
      p.stor_rho[sidx] = rho;
    }
    __syncwarp();
  }
  device_x(p, n, pd, X, lane);   // p_d - avg_k(pbar + u)
#define LAM(g, t) lam[(g) * Tp + (t)]
#define BET(g, t) bet[(g) * Tp + (t)]
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    for (int t = lane; t < T; t += 32) {
      const float r1 = -LAM(SG_E1, t), r2 = -LAM(SG_E2, t);
      const float mc = rmul(0.5f, rsub(rsub(radd(Pm, BET(SG_CU, t)), LAM(SG_CU, t)), rsub(BET(SG_CL, t), LAM(SG_CL, t))));
      const float md = rmul(0.5f, rsub(rsub(radd(Pm, BET(SG_DU, t)), LAM(SG_DU, t)), rsub(BET(SG_DL, t), LAM(SG_DL, t))));
      const float e1 = rsub(r1, X[t]);
      const float f0c = rfma(kap, e1, rmul(om2, mc));
      const float f0d = rfma(om2, md, rsub(rmul(-kap, e1), q));
      TAU[t] = radd(r2, rdiv(rfma(w0, f0c, rmul(w1, f0d)), gam));
    }
    __syncwarp();
    for (int j = lane; j < Tp; j += 32) {
      const float ms = rmul(0.5f, rsub(rsub(radd(Em, BET(SG_SU, j)), LAM(SG_SU, j)), rsub(BET(SG_SL, j), LAM(SG_SL, j))));
      float rhs = rmul(om2, ms);
      if (j >= 1) rhs = rfma(gam, TAU[j - 1], rhs);
      if (j <= T - 1) rhs = rfma(-gam, TAU[j], rhs);
      if (j == 0) rhs = rfma(-om, LAM(SG_E3, 0), rhs);
      if (j == T) rhs = rfma(-om, LAM(SG_E3, 1), rhs);
      S[j] = rhs;
    }
    __syncwarp();
    warp_tri_solve(mf, -gam, S, Tp, lane);
    for (int t = lane; t < T; t += 32) {
      const float r1 = -LAM(SG_E1, t), r2 = -LAM(SG_E2, t);
      const float mc = rmul(0.5f, rsub(rsub(radd(Pm, BET(SG_CU, t)), LAM(SG_CU, t)), rsub(BET(SG_CL, t), LAM(SG_CL, t))));
      const float md = rmul(0.5f, rsub(rsub(radd(Pm, BET(SG_DU, t)), LAM(SG_DU, t)), rsub(BET(SG_DL, t), LAM(SG_DL, t))));
      const float e1 = rsub(r1, X[t]);
      const float f0c = rfma(kap, e1, rmul(om2, mc));
      const float f0d = rfma(om2, md, rsub(rmul(-kap, e1), q));
      const float s0 = S[t], s1 = S[t + 1];
      const float ds = rsub(s1, s0);
      const float g = rsub(ds, r2);
      const float fc = rfma(g, f1c, f0c), fd = rfma(g, f1d, f0d);
      const float c = rfma(i00, fc, rmul(i01, fd));
      const float dl = rfma(i01, fc, rmul(i11, fd));
      const float pt = rdiv(rfma(om, radd(rsub(r1, c), dl), rmul(rho, X[t])), rpo);
      TAU[t] = pt;  // TAU is consumed; keep p_t for the end
      dl_out[t] = dl;
      LAM(SG_E1, t) = radd(LAM(SG_E1, t), rsub(radd(pt, c), dl));   // equality rows: beta = 0
      LAM(SG_E2, t) = radd(LAM(SG_E2, t), radd(rfma(-eta, c, ds), dl));
      ineq_step(rsub(c, Pm), LAM(SG_CU, t), BET(SG_CU, t));
      ineq_step(-c, LAM(SG_CL, t), BET(SG_CL, t));
      ineq_step(rsub(dl, Pm), LAM(SG_DU, t), BET(SG_DU, t));
      ineq_step(-dl, LAM(SG_DL, t), BET(SG_DL, t));
    }
    for (int j = lane; j < Tp; j += 32) {
      const float sj = S[j];
      if (j == 0) LAM(SG_E3, 0) = radd(LAM(SG_E3, 0), sj);
      if (j == T) LAM(SG_E3, 1) = radd(LAM(SG_E3, 1), sj);
      ineq_step(rsub(sj, Em), LAM(SG_SU, j), BET(SG_SU, j));
      ineq_step(-sj, LAM(SG_SL, j), BET(SG_SL, j));
    }
    __syncwarp();
  }
#undef LAM
#undef BET
  stage_out(lam_g, bet_g, state_sh, SG_N * Tp, lane);
  for (int t = lane; t < T; t += 32) {
    const float pn = relaxed(p.alpha, TAU[t], pd[t]);
    p.DPD[(size_t)d * T + t] = rsub(pn, pd[t]);
    pd[t] = pn;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The same inner ADMM with the device's state in registers, for horizons of
// at most REG_T steps: lane l holds the C = ceil(n / 32) consecutive
// elements l C .. l C + C - 1 of each vector (the solve's chunks), so the
// inner iterations touch no memory; neighbours across a chunk boundary come
// by one shuffle.  Every product, sum and quotient is written with its
// rounding (__fmul_rn, __fadd_rn, __fmaf_rn, ...), which the compiler may
// not contract or reorder, so each kernel that inlines this path (one
// instance, a batch) computes the same bits.
// ---------------------------------------------------------------------------

// warp_tri_solve on a chunk held in registers (element i = lane C + j, valid
// while i < n), a[j] = -off / q[j]
template <int C>
__device__ __forceinline__ void warp_tri_solve_r(const float (&q)[C], const float (&a)[C], float (&x)[C], int n,
                                                 int lane) {
  const int i0 = lane * C;
  float r[C];
  float Ac = 1.f, Bc = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int i = i0 + j;
    if (i < n) {
      r[j] = rdiv(x[j], q[j]);
      const float Ai = (i == 0) ? 0.f : a[j];
      Bc = rfma(Ai, Bc, r[j]);
      Ac = rmul(Ai, Ac);
    }
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_up_sync(FULL, Ac, d);
    const float Bp = __shfl_up_sync(FULL, Bc, d);
    if (lane >= d) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float prev = __shfl_up_sync(FULL, Bc, 1);
  if (lane == 0) prev = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int i = i0 + j;
    if (i < n) {
      const float Ai = (i == 0) ? 0.f : a[j];
      prev = rfma(Ai, prev, r[j]);
      x[j] = prev;
    }
  }
  Ac = 1.f;
  Bc = 0.f;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    const int i = i0 + j;
    if (i < n) {
      const float Ci = (i == n - 1) ? 0.f : a[j];
      Bc = rfma(Ci, Bc, x[j]);
      Ac = rmul(Ci, Ac);
    }
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_down_sync(FULL, Ac, d);
    const float Bp = __shfl_down_sync(FULL, Bc, d);
    if (lane + d < 32) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float nxt = __shfl_down_sync(FULL, Bc, 1);
  if (lane == 31) nxt = 0.f;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    const int i = i0 + j;
    if (i < n) {
      const float Ci = (i == n - 1) ? 0.f : a[j];
      nxt = rfma(Ci, nxt, x[j]);
      x[j] = nxt;
    }
  }
}


template <int C>
__device__ void ramp_prox_r(const Params &p, int r, float rho, int lane) {
  const int T = p.T, t0 = lane * C;
  const int d = p.ramp_ids[r];
  const int n = p.dev_node[d];
  const float a = p.dev_a[d], b = p.dev_b[d], R = p.ramp_R[r];
  const float om = rho, om2 = rmul(2.f, om);
  float *const lam_g = p.ramp_lam + (size_t)r * RG_N * T;
  float *const bet_g = p.ramp_beta + (size_t)r * RG_N * T;
  float *mf = p.ramp_q + (size_t)r * T;
  // keep the unscaled inner duals omega * lam when omega changes; refactor
  // (2a + rho + 2 omega) I + 2 omega D'D
  const float rho_old = p.ramp_rho[r];
  const bool rescale = rho_old != rho;
  const float ls = (rho_old == 0.f) ? 1.f : rdiv(fabsf(rho_old), rho);
  if (rescale) {
    if (lane == 0) {
      const float base = radd(rmul(2.f, a), rho);
      tri_factor(mf, T, radd(base, rmul(4.f, om)), radd(base, rmul(6.f, om)), -om2);
      p.ramp_rho[r] = rho;
    }
    __syncwarp();
  }
  float lam[RG_N][C], bet[RG_N][C], hi[C], lo[C], X[C], pd[C], qv[C], av[C], Z[C];
  const float *xs = p.XS + (size_t)n * T;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int t = t0 + j;
    const bool in = t < T;
#pragma unroll
    for (int g = 0; g < RG_N; ++g) {
      lam[g][j] = in ? lam_g[g * T + t] : 0.f;
      bet[g][j] = in ? bet_g[g * T + t] : 0.f;
      if (rescale) lam[g][j] = rmul(lam[g][j], ls);
    }
    hi[j] = in ? p.dev_hi[(size_t)d * T + t] : 0.f;
    lo[j] = in ? p.dev_lo[(size_t)d * T + t] : 0.f;
    pd[j] = in ? p.PD[(size_t)d * T + t] : 0.f;
    X[j] = in ? rsub(pd[j], __ldcg(xs + t)) : 0.f;   // p_d - avg_k(pbar + u)
    qv[j] = in ? mf[t] : 1.f;
    av[j] = rdiv(om2, qv[j]);                         // -off / q with off = -2 omega
    Z[j] = 0.f;
  }
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    float W[C];
#pragma unroll
    for (int j = 0; j < C; ++j)
      W[j] = rsub(rsub(bet[RG_RU][j], lam[RG_RU][j]), rsub(bet[RG_RD][j], lam[RG_RD][j]));
    const float wprev = __shfl_up_sync(FULL, W[C - 1], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      if (t < T) {
        float atr = rsub(rsub(radd(hi[j], bet[RG_UP][j]), lam[RG_UP][j]),
                         rsub(radd(-lo[j], bet[RG_LO][j]), lam[RG_LO][j]));
        if (t >= 1) atr = radd(atr, (j == 0) ? wprev : W[j - 1]);
        if (t <= T - 2) atr = rsub(atr, W[j]);
        Z[j] = rfma(om, atr, rfma(rho, X[j], -b));
      }
    }
    warp_tri_solve_r<C>(qv, av, Z, T, lane);
    const float znext = __shfl_down_sync(FULL, Z[0], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      if (t < T) {
        const float pt = Z[j];
        ineq_step(rsub(pt, hi[j]), lam[RG_UP][j], bet[RG_UP][j]);
        ineq_step(rsub(lo[j], pt), lam[RG_LO][j], bet[RG_LO][j]);
        if (t < T - 1) {
          const float pn = (j == C - 1) ? znext : Z[j + 1];
          ineq_step(rsub(rsub(pn, pt), R), lam[RG_RU][j], bet[RG_RU][j]);
          ineq_step(rsub(rsub(pt, pn), R), lam[RG_RD][j], bet[RG_RD][j]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int t = t0 + j;
    if (t < T) {
#pragma unroll
      for (int g = 0; g < RG_N; ++g) {
        lam_g[g * T + t] = lam[g][j];
        bet_g[g * T + t] = bet[g][j];
      }
      const float pn = relaxed(p.alpha, Z[j], pd[j]);
      p.DPD[(size_t)d * T + t] = rsub(pn, pd[j]);
      p.PD[(size_t)d * T + t] = pn;
    }
  }
}

template <int C>
__device__ void stor_prox_r(const Params &p, int sidx, float rho, int lane) {
  const int T = p.T, Tp = T + 1, t0 = lane * C;
  const int d = p.stor_ids[sidx];
  const int n = p.dev_node[d];
  const float eta = p.stor_eff[sidx], Pm = p.stor_P[sidx], Em = rmul(p.stor_dur[sidx], Pm);
  const float q = p.stor_cost[sidx];
  const float om = rho, om2 = rmul(2.f, om);
  float *const lam_g = p.stor_lam + (size_t)sidx * SG_N * Tp;
  float *const bet_g = p.stor_beta + (size_t)sidx * SG_N * Tp;
  float *mf = p.stor_q + (size_t)sidx * Tp;

  // 2x2 block of (c, delta) after eliminating p; constants of the reduction
  const float kap = rdiv(rmul(rho, om), radd(rho, om));
  const float h00 = radd(radd(kap, om2), rmul(rmul(om, eta), eta));
  const float h01 = rsub(-kap, rmul(om, eta)), h11 = radd(kap, rmul(3.f, om));
  const float det = rsub(rmul(h00, h11), rmul(h01, h01));
  const float i00 = rdiv(h11, det), i01 = rdiv(-h01, det), i11 = rdiv(h00, det);
  const float f1c = rmul(om, eta), f1d = -om;
  const float w0 = radd(rmul(i00, f1c), rmul(i01, f1d)), w1 = radd(rmul(i01, f1c), rmul(i11, f1d));
  const float gam = rsub(om, radd(rmul(f1c, w0), rmul(f1d, w1)));
  const float rpo = radd(rho, om);

  const float rho_old = p.stor_rho[sidx];
  const bool rescale = rho_old != rho;
  const float ls = (rho_old == 0.f) ? 1.f : rdiv(fabsf(rho_old), rho);
  if (rescale) {
    if (lane == 0) {
      tri_factor(mf, Tp, radd(gam, rmul(3.f, om)), radd(rmul(2.f, gam), om2), -gam);
      p.stor_rho[sidx] = rho;
    }
    __syncwarp();
  }
  // element e = t0 + j: step t = e of (p, c, delta) while e < T, state of
  // charge s_e while e < T + 1
  float lE1[C], lE2[C], lCU[C], lCL[C], lDU[C], lDL[C], lSU[C], lSL[C];
  float bCU[C], bCL[C], bDU[C], bDL[C], bSU[C], bSL[C];
  float X[C], pd[C], qv[C], av[C], S[C], TAU[C], DL[C];
  float e3a = lam_g[SG_E3 * Tp], e3b = lam_g[SG_E3 * Tp + 1];   // s_0 and s_T rows
  if (rescale) {
    e3a = rmul(e3a, ls);
    e3b = rmul(e3b, ls);
  }
  const float *xs = p.XS + (size_t)n * T;
#define LD_L(arr, g) arr[j] = in ? (rescale ? rmul(lam_g[(g) * Tp + e], ls) : lam_g[(g) * Tp + e]) : 0.f
#define LD_B(arr, g) arr[j] = in ? bet_g[(g) * Tp + e] : 0.f
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int e = t0 + j;
    const bool in = e < Tp;
    LD_L(lE1, SG_E1); LD_L(lE2, SG_E2); LD_L(lCU, SG_CU); LD_L(lCL, SG_CL);
    LD_L(lDU, SG_DU); LD_L(lDL, SG_DL); LD_L(lSU, SG_SU); LD_L(lSL, SG_SL);
    LD_B(bCU, SG_CU); LD_B(bCL, SG_CL); LD_B(bDU, SG_DU); LD_B(bDL, SG_DL);
    LD_B(bSU, SG_SU); LD_B(bSL, SG_SL);
    const bool st = e < T;
    pd[j] = st ? p.PD[(size_t)d * T + e] : 0.f;
    X[j] = st ? rsub(pd[j], __ldcg(xs + e)) : 0.f;   // p_d - avg_k(pbar + u)
    qv[j] = in ? mf[e] : 1.f;
    av[j] = rdiv(gam, qv[j]);                         // -off / q with off = -gam
    S[j] = TAU[j] = DL[j] = 0.f;
  }
#undef LD_L
#undef LD_B
  for (int itn = 0; itn < p.inner_iters; ++itn) {
    float f0c[C], f0d[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      f0c[j] = f0d[j] = 0.f;
      if (t0 + j < T) {
        const float r1 = -lE1[j], r2 = -lE2[j];
        const float mc = rmul(0.5f, rsub(rsub(radd(Pm, bCU[j]), lCU[j]), rsub(bCL[j], lCL[j])));
        const float md = rmul(0.5f, rsub(rsub(radd(Pm, bDU[j]), lDU[j]), rsub(bDL[j], lDL[j])));
        const float e1 = rsub(r1, X[j]);
        f0c[j] = rfma(kap, e1, rmul(om2, mc));
        f0d[j] = rfma(om2, md, rsub(rmul(-kap, e1), q));
        TAU[j] = radd(r2, rdiv(rfma(w0, f0c[j], rmul(w1, f0d[j])), gam));
      }
    }
    const float tprev = __shfl_up_sync(FULL, TAU[C - 1], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      if (e < Tp) {
        const float ms = rmul(0.5f, rsub(rsub(radd(Em, bSU[j]), lSU[j]), rsub(bSL[j], lSL[j])));
        float rhs = rmul(om2, ms);
        if (e >= 1) rhs = rfma(gam, (j == 0) ? tprev : TAU[j - 1], rhs);
        if (e <= T - 1) rhs = rfma(-gam, TAU[j], rhs);
        if (e == 0) rhs = rfma(-om, e3a, rhs);
        if (e == T) rhs = rfma(-om, e3b, rhs);
        S[j] = rhs;
      }
    }
    warp_tri_solve_r<C>(qv, av, S, Tp, lane);
    const float snext = __shfl_down_sync(FULL, S[0], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (t0 + j < T) {
        const float r1 = -lE1[j], r2 = -lE2[j];
        const float s0 = S[j], s1 = (j == C - 1) ? snext : S[j + 1];
        const float ds = rsub(s1, s0);
        const float g = rsub(ds, r2);
        const float fc = rfma(g, f1c, f0c[j]), fd = rfma(g, f1d, f0d[j]);
        const float c = rfma(i00, fc, rmul(i01, fd));
        const float dl = rfma(i01, fc, rmul(i11, fd));
        const float pt = rdiv(rfma(om, radd(rsub(r1, c), dl), rmul(rho, X[j])), rpo);
        TAU[j] = pt;   // TAU is consumed; keep p_t for the end
        DL[j] = dl;
        lE1[j] = radd(lE1[j], rsub(radd(pt, c), dl));   // equality rows: beta = 0
        lE2[j] = radd(lE2[j], radd(rfma(-eta, c, ds), dl));
        ineq_step(rsub(c, Pm), lCU[j], bCU[j]);
        ineq_step(-c, lCL[j], bCL[j]);
        ineq_step(rsub(dl, Pm), lDU[j], bDU[j]);
        ineq_step(-dl, lDL[j], bDL[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      if (e < Tp) {
        const float sj = S[j];
        if (e == 0) e3a = radd(e3a, sj);
        if (e == T) e3b = radd(e3b, sj);
        ineq_step(rsub(sj, Em), lSU[j], bSU[j]);
        ineq_step(-sj, lSL[j], bSL[j]);
      }
    }
  }
#define ST_L(arr, g) lam_g[(g) * Tp + e] = arr[j]
#define ST_B(arr, g) bet_g[(g) * Tp + e] = arr[j]
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int e = t0 + j;
    if (e < T) {
      ST_L(lE1, SG_E1); ST_L(lE2, SG_E2); ST_L(lCU, SG_CU); ST_L(lCL, SG_CL);
      ST_L(lDU, SG_DU); ST_L(lDL, SG_DL);
      ST_B(bCU, SG_CU); ST_B(bCL, SG_CL); ST_B(bDU, SG_DU); ST_B(bDL, SG_DL);
      const float pn = relaxed(p.alpha, TAU[j], pd[j]);
      p.DPD[(size_t)d * T + e] = rsub(pn, pd[j]);
      p.PD[(size_t)d * T + e] = pn;
      p.stor_delta[(size_t)sidx * T + e] = DL[j];
    }
    if (e < Tp) {
      ST_L(lSU, SG_SU); ST_L(lSL, SG_SL);
      ST_B(bSU, SG_SU); ST_B(bSL, SG_SL);
      if (e == 0) lam_g[SG_E3 * Tp] = e3a;
      if (e == T) lam_g[SG_E3 * Tp + 1] = e3b;
    }
  }
#undef ST_L
#undef ST_B
}

// ---------------------------------------------------------------------------
// VW consecutive time steps per thread (4 -> 128-bit accesses when T % 4 == 0)
// ---------------------------------------------------------------------------
template <int VW>
struct FV {
  float v[VW];
};

template <int VW>
__device__ __forceinline__ FV<VW> ldv(const float *p) {
  FV<VW> r;
  if constexpr (VW == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (VW == 2) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = *p;
  }
  return r;
}

// streaming load (read once per iteration: evict first)
template <int VW>
__device__ __forceinline__ FV<VW> ldv_cs(const float *p) {
  FV<VW> r;
  if constexpr (VW == 4) {
    const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (VW == 2) {
    const float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = __ldcs(p);
  }
  return r;
}

template <int VW>
__device__ __forceinline__ void stv(float *p, const FV<VW> &r) {
  if constexpr (VW == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else if constexpr (VW == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(r.v[0], r.v[1]);
  } else {
    *p = r.v[0];
  }
}

// streaming store (not read again in this iteration: evict first)
template <int VW>
__device__ __forceinline__ void stv_cs(float *p, const FV<VW> &r) {
  if constexpr (VW == 4) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
  } else if constexpr (VW == 2) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(r.v[0], r.v[1]));
  } else {
    __stcs(p, r.v[0]);
  }
}

// one-pass sum of squared deviations from the mean (Welford)
template <int VW>
struct Welf {
  float n;
  float mean[VW], m2[VW];
  __device__ __forceinline__ void reset() {
    n = 0.f;
#pragma unroll
    for (int e = 0; e < VW; ++e) { mean[e] = 0.f; m2[e] = 0.f; }
  }
  __device__ __forceinline__ void add(const float *x) {
    n += 1.f;
    const float r = __frcp_rn(n);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const float d = x[e] - mean[e];
      mean[e] = fmaf(d, r, mean[e]);
      m2[e] = fmaf(d, x[e] - mean[e], m2[e]);
    }
  }
};

// one-pass sums of two series over a node's terminals (Welford with the
// co-moment): means, centred second moments and sum (x - mean_x)(y - mean_y)
template <int VW>
struct Welf2 {
  float n;
  float mx[VW], my[VW], m2x[VW], m2y[VW], cxy[VW];
  __device__ __forceinline__ void reset() {
    n = 0.f;
#pragma unroll
    for (int e = 0; e < VW; ++e) { mx[e] = my[e] = m2x[e] = m2y[e] = cxy[e] = 0.f; }
  }
  __device__ __forceinline__ void add(const float *x, const float *y) {
    n += 1.f;
    const float r = __frcp_rn(n);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const float dx = x[e] - mx[e], dy = y[e] - my[e];
      mx[e] = fmaf(dx, r, mx[e]);
      my[e] = fmaf(dy, r, my[e]);
      m2x[e] = fmaf(dx, x[e] - mx[e], m2x[e]);
      m2y[e] = fmaf(dy, y[e] - my[e], m2y[e]);
      cxy[e] = fmaf(dx, y[e] - my[e], cxy[e]);
    }
  }
};

// x / c given r = 1/c rounded to nearest: one FMA correction step gives the
// correctly rounded quotient for these well-scaled operands (a plain x * r
// would carry the rounding bias of r into every node average, iteration
// after iteration).
__device__ __forceinline__ float div_rn(float x, float c, float r) {
  const float q = x * r;
  return fmaf(fmaf(-q, c, x), r, q);
}

// Index (a, b, c) of a row-major [.][B][C] item space, advanced by a fixed
// stride with carries instead of 64-bit divisions per item.
struct Idx3 {
  int a, b, c;
  __device__ __forceinline__ void set(unsigned x, int B, int C) {
    c = (int)(x % (unsigned)C);
    const unsigned q = x / (unsigned)C;
    b = (int)(q % (unsigned)B);
    a = (int)(q / (unsigned)B);
  }
  __device__ __forceinline__ void step(const Idx3 &d, int B, int C) {
    c += d.c;
    if (c >= C) { c -= C; ++b; }
    b += d.b;
    if (b >= B) { b -= B; ++a; }
    a += d.a;
  }
};

// ---------------------------------------------------------------------------
// line prox item (Section 3.2 step 1, Section 2.1 f^ac, Section 4.2): one
// (contingency k, line l, VW time steps).  x = p~ - u and y = theta_bar - v at
// both terminals from the previous iterate; the deferred phase-dual update
// v += theta - theta_bar of the previous iteration is applied on the way.
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void line_item(const Params &p, int old, int nw, int k, int l, int toff, float frp,
                                          float frt, float fsu, float fsv, bool v_fresh) {
  // offsets of the line and its end nodes' rows: lidx / nidx
  const int n1 = p.line_n1[l], n2 = p.line_n2[l];
  const bool act = p.out_line[k] != l;
  const size_t ol = lidx(p, k, l, toff);
  const size_t o1 = nidx(p, k, n1, toff), o2 = nidx(p, k, n2, toff);
  // p stays cached: the node sums read its old value again
  FV<VW> P = ldv<VW>(p.P[old] + ol), M = ldv_cs<VW>(p.MID[old] + ol);
  FV<VW> V1 = ldv_cs<VW>(p.V1[old] + ol), V2 = ldv_cs<VW>(p.V2[old] + ol);
  // pbar + s u at both ends from PU = pbar + u; u itself only while a
  // penalty rescale s != 1 is pending (an adaptation iteration)
  const FV<VW> B1 = ldv<VW>(p.PU[old] + o1), B2 = ldv<VW>(p.PU[old] + o2);
  FV<VW> U1, U2;
  const bool rescale = fsu != 1.f;
  if (rescale) {
    U1 = ldv<VW>(p.U[old] + o1);
    U2 = ldv<VW>(p.U[old] + o2);
  }
  const FV<VW> G1 = ldv<VW>(p.THBAR[old] + o1), G2 = ldv<VW>(p.THBAR[old] + o2);
  float tb = 1.f, den = 1.f, ulim = 0.f;
  if (act) {
    const float bb = p.line_b[l];
    ulim = p.line_u[l];
    tb = 2.f * bb;
    den = 2.f * frp + frt / (tb * bb);   // 2 rho_p + rho_theta / (2 b^2), Section 4.2 (reading of the garbled print)
  }
  const float rden = __frcp_rn(den), rtb = __frcp_rn(tb);
  const float al = p.alpha, oma = 1.f - p.alpha;
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    // the previous prox's terminal values (stored as p and the mean angle;
    // relaxed values when alpha != 1, Section 3.6)
    const float po = act ? P.v[e] : 0.f;
    const float ho = act ? div_rn(P.v[e], tb, rtb) : P.v[e];
    const float a1 = M.v[e] + ho, a2 = M.v[e] - ho;
    const float w1 = rescale ? fmaf(fsu - 1.f, U1.v[e], B1.v[e]) : B1.v[e];   // pbar + s u
    const float w2 = rescale ? fmaf(fsu - 1.f, U2.v[e], B2.v[e]) : B2.v[e];
    const float x1 = -po - w1;                              // p~ - u at terminal 1 (z - u relaxed)
    const float x2 = po - w2;                               // p~ - u at terminal 2
    const float r1 = a1 - G1.v[e], r2 = a2 - G2.v[e];       // theta - theta_bar (Theta - xi relaxed)
    const float v1 = v_fresh ? fsv * V1.v[e] : fsv * (V1.v[e] + r1);
    const float v2 = v_fresh ? fsv * V2.v[e] : fsv * (V2.v[e] + r2);
    const float y1 = G1.v[e] - v1, y2 = G2.v[e] - v2;       // theta_bar - v
    const float mo = M.v[e], sto = P.v[e];
    M.v[e] = fmaf(al, 0.5f * (y1 + y2), oma * mo);
    if (act) {
      const float num = frp * (x2 - x1) + div_rn(frt * (y1 - y2), tb, rtb);
      P.v[e] = fminf(fmaxf(div_rn(num, den, rden), -ulim), ulim);   // theta_{1,2} = mid +- p / (2b)
    } else {
      P.v[e] = 0.5f * (y1 - y2);   // outaged line: p = 0, the terminals decouple, theta = y
    }
    P.v[e] = fmaf(al, P.v[e], oma * sto);
    // v' = v - (Theta - xi) is what the next pass completes:
    // v'_new = v + alpha theta~_new - (Theta_new - xi_new) = v - (1 - alpha) (Theta - xi)
    V1.v[e] = fmaf(-oma, r1, v1);
    V2.v[e] = fmaf(-oma, r2, v2);
  }
  // p and the mean angle are read back by the node sums; v is not
  stv<VW>(p.P[nw] + ol, P);
  stv<VW>(p.MID[nw] + ol, M);
  stv_cs<VW>(p.V1[nw] + ol, V1);
  stv_cs<VW>(p.V2[nw] + ol, V2);
}

// ---------------------------------------------------------------------------
// node item (Section 3.2 step 3, Eq. average-op, Section 3.3): one
// (contingency k, node n, VW time steps).  Sums the node's terminals in CSR
// order (no atomics), forms pbar, theta_bar, u += pbar, and the residual
// partial sums: ||pbar||^2, ||theta~||^2 and ||p~ - p~_prev||^2 by one-pass
// Welford sums over the terminals, ||theta_bar - theta_bar_prev||^2.  The
// terminal codes come four at a time so that a node's row loads issue
// together.
// ---------------------------------------------------------------------------
// res = 0: the iteration's residuals are not read, so the node sums skip the
// inputs only they need (old p and theta_bar rows, the device Welford state)
// and their accumulation; the relaxed variant always needs the mean change.
// ILD: where the pass forms no residuals, whether it sums the device powers
// itself (0 never, 1 always, 2 as Params::dsum_lean says)
template <int VW, bool RELAX, int NB = 4, int ILD = 2>
__device__ __forceinline__ void node_item(const Params &p, int old, int nw, int k, int n, int toff, float fsu,
                                          float *acc, bool res) {
  const int T = p.T;
  if constexpr (RELAX) res = true;
  // level 1: the node record, the node's old rows and its device sums
  const int4 r0 = p.nrec[3 * n], r1 = p.nrec[3 * n + 1], r2 = p.nrec[3 * n + 2];
  const float cp = __int_as_float(r0.x), ct = __int_as_float(r0.y);
  const float rcp = __int_as_float(r0.z), rct = __int_as_float(r0.w);
  const size_t on = nidx(p, k, n, toff), os = (size_t)n * T + toff;
  const FV<VW> uo = ldv_cs<VW>(p.U[old] + on);
  FV<VW> go;
  if (res) go = ldv_cs<VW>(p.THBAR[old] + on);
  // device terminals first: the sum and the Welford state after them, the
  // same in every contingency -- from dsum_kernel, or (dsum_lean, where no
  // residuals are formed) summed here over the node's devices in its order
  FV<VW> sp, st;
  if (res || ILD == 0 || (ILD == 2 && !p.dsum_lean)) {
    sp = ldv<VW>(p.DSP + os);
  } else {
#pragma unroll
    for (int e = 0; e < VW; ++e) sp.v[e] = 0.f;
    for (int j = r2.w; j < r2.w + r2.z; ++j) {
      const FV<VW> pd = ldv<VW>(p.PD + (size_t)p.dcsr_idx[j] * T + toff);
#pragma unroll
      for (int e = 0; e < VW; ++e) sp.v[e] += pd.v[e];
    }
  }
  Welf<VW> wdp, wth;
  Welf2<VW> wrx;   // RELAX: (Theta_new, Theta_new - Theta_old) over the line terminals
  if constexpr (RELAX) wrx.reset();
  if (res) {
    const FV<VW> m = ldv<VW>(p.DSM + os), q = ldv<VW>(p.DSQ + os);
    wdp.n = (float)r2.z;
#pragma unroll
    for (int e = 0; e < VW; ++e) { wdp.mean[e] = m.v[e]; wdp.m2[e] = q.v[e]; }
  }
  wth.reset();
#pragma unroll
  for (int e = 0; e < VW; ++e) st.v[e] = 0.f;
  // level 2: the rows of the line terminals, four at a time; a terminal's
  // angle is mid +- p / (2b) (mid +- the stored value on the outaged line)
  const size_t kb = (size_t)k * T + toff, lrow = (size_t)p.Kp * T;   // line l's row of k: l * lrow + kb
  const int lout = p.out_line[k];
  int4 c4 = r1;
  for (int j = r2.x - 4;;) {
    const int code4[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll 1
    for (int half = 0; half < 4; half += NB) {
    int code[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) code[q] = code4[half + q];
    FV<VW> pn[NB], po[NB], mq[NB], mo[RELAX ? NB : 1];
    float bq[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (code[q] >= 0) {
        const int l = code[q] >> 1;
        const size_t ol = (size_t)l * lrow + kb;
        pn[q] = ldv<VW>(p.P[nw] + ol);
        if (res) po[q] = ldv<VW>(p.P[old] + ol);   // kept in L2 for the line's other end
        mq[q] = ldv<VW>(p.MID[nw] + ol);
        if constexpr (RELAX) mo[q] = ldv<VW>(p.MID[old] + ol);
        bq[q] = p.line_b[l];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (code[q] >= 0) {
        const bool t2 = code[q] & 1, act = (code[q] >> 1) != lout;
        const float tb = 2.f * bq[q], rtb = __frcp_rn(tb);
        float dpo[VW], th[VW], dth[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const float pv = act ? pn[q].v[e] : 0.f, pov = (act && res) ? po[q].v[e] : 0.f;
          const float h = act ? div_rn(pn[q].v[e], tb, rtb) : pn[q].v[e];
          th[e] = t2 ? mq[q].v[e] - h : mq[q].v[e] + h;
          sp.v[e] += t2 ? pv : -pv;
          st.v[e] += th[e];
          dpo[e] = t2 ? pv - pov : pov - pv;
          if constexpr (RELAX) {
            const float ho = act ? div_rn(po[q].v[e], tb, rtb) : po[q].v[e];
            dth[e] = th[e] - (t2 ? mo[q].v[e] - ho : mo[q].v[e] + ho);
          }
        }
        if (res) {
          wdp.add(dpo);
          if constexpr (RELAX) wrx.add(th, dth);
          else wth.add(th);
        }
      }
    }
    }
    j += 4;
    if (j >= r2.y) break;
    c4 = *reinterpret_cast<const int4 *>(p.tcode + j);   // terminals beyond the first four
  }
  FV<VW> pb, tbar, un;
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    pb.v[e] = div_rn(sp.v[e], cp, rcp);                      // Eq. (average-op)
    tbar.v[e] = ct > 0.f ? div_rn(st.v[e], ct, rct) : 0.f;
    if (!res) {
      un.v[e] = fsu * uo.v[e] + pb.v[e];                     // u += pbar
      continue;
    }
    const float dt = tbar.v[e] - go.v[e];
    if constexpr (RELAX) {
      // stored values are relaxed: pb = Q = avg_n P, tbar = xi.  The actual
      // iterate is P + c dP with c = (1 - alpha) / alpha, so
      //   u += alpha pbar_actual = alpha Q + (1 - alpha) dQ,
      //   ||p - z||^2 = c^2 sum (dP - dQ)^2 + |n| (Q + c dQ)^2,
      //   ||theta - xi||^2 = sum (Theta - xi + c dTheta)^2 by the co-moment
      const float a = p.alpha, c = (1.f - a) / a, dq = wdp.mean[e];
      un.v[e] = fsu * uo.v[e] + fmaf(a, pb.v[e], (1.f - a) * dq);
      const float qc = fmaf(c, dq, pb.v[e]);
      acc[SL_PP] += fmaf(c * c, wdp.m2[e], cp * qc * qc);
      acc[SL_PT] += wrx.m2x[e] + c * (2.f * wrx.cxy[e] + c * fmaf(wrx.n * wrx.my[e], wrx.my[e], wrx.m2y[e]));
    } else {
      un.v[e] = fsu * uo.v[e] + pb.v[e];                     // u += pbar
      acc[SL_PP] += cp * pb.v[e] * pb.v[e];
      acc[SL_PT] += wth.m2[e];
    }
    acc[SL_DP] += wdp.m2[e];
    acc[SL_DT] += ct * dt * dt;
    if (!isfinite(un.v[e]) || !isfinite(tbar.v[e])) acc[SL_NF] += 1.f;
  }
  // the new node rows are read in the next iteration only
  stv_cs<VW>(p.U[nw] + on, un);
  FV<VW> pu;
#pragma unroll
  for (int e = 0; e < VW; ++e) pu.v[e] = pb.v[e] + un.v[e];
  stv_cs<VW>(p.PU[nw] + on, pu);
  stv_cs<VW>(p.THBAR[nw] + on, tbar);
}

// ---------------------------------------------------------------------------
// the persistent iteration kernel
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// the scalars of the current iteration, read once per CTA.  A context that
// stopped in this call (passed stopping test) or holds a sticky error makes
// every kernel return at once.
// ---------------------------------------------------------------------------
struct Iter {
  float frp, frt, fsu, fsv, rho_dev;
  int old, nw, v_fresh, skip;
  int res;   // this iteration's residuals are read (stopping test, adaptation, end of the call)
};

// whether the penalties may still change after iteration itn (1-based):
// adaptation on, within opf_options.adapt_until, not fixed by the stall rule
__device__ __forceinline__ bool adapting(const Params &p, const DevScalars &sc, long long itn) {
  return p.adapt_every > 0 && (p.adapt_until <= 0 || itn <= p.adapt_until) && sc.frozen_at == 0;
}
// iteration itn adapts the penalties (Section 3.5, every adapt_every iterations)
__device__ __forceinline__ bool adapt_at(const Params &p, const DevScalars &sc, long long itn) {
  return adapting(p, sc, itn) && itn % p.adapt_every == 0;
}

__device__ __forceinline__ Iter iter_scalars(const Params &p) {
  __shared__ Iter s;
  if (threadIdx.x == 0) {
    const DevScalars sc = *p.sc;
    Iter r;
    r.frp = (float)sc.rho_p;
    r.frt = (float)sc.rho_th;
    r.fsu = (float)sc.su;
    r.fsv = (float)sc.sv;
    r.rho_dev = (float)(p.Kp_glob * sc.rho_p);   // rho' = (K+1) rho_p
    r.old = (int)(sc.it & 1);
    r.nw = r.old ^ 1;
    r.v_fresh = sc.v_fresh;
    r.skip = (sc.status != 0 || sc.stop != 0) ? 1 : 0;
    const long long itn = sc.it + 1;
    r.res = adapt_at(p, sc, itn) || (p.eps > 0 && p.check_every > 0 && itn % p.check_every == 0) ||
            itn >= sc.it_last;
    s = r;
  }
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// xs: avg_k(pbar + u) at each node with devices, one (node, VW time steps)
// item per thread; the node's closed-form devices are updated on the spot
// (Section 4.2), nodes with inner-ADMM devices keep the average in XS
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void xs_body(const Params &p, unsigned bid, unsigned nblk) {
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  const int T = p.T, TV = T / VW, Kp = p.Kp;
  const float kpf = (float)p.Kp_glob, rkp = __frcp_rn(kpf);
  const size_t KT = (size_t)Kp * T;    // a node's K+1 rows are contiguous
  // avg_k(pbar + s u) = (sum_k PU + (s - 1) sum_k u) / (K+1); u is read only
  // while a penalty rescale s != 1 is pending
  const float *Uo = p.U[q.old], *Wo = p.PU[q.old];
  const bool rescale = q.fsu != 1.f;
  const float sm1 = q.fsu - 1.f;
  const unsigned n_xv = (unsigned)p.n_dnode * (unsigned)TV;
  for (unsigned item = bid * BLOCK + threadIdx.x; item < n_xv; item += nblk * BLOCK) {
    const int ci = (int)(item / (unsigned)TV), t0 = (int)(item % (unsigned)TV) * VW;
    const size_t on = (size_t)p.dnode_ids[ci] * T + t0, ok = (size_t)p.dnode_ids[ci] * KT + t0;
    FV<VW> xs;
    if (p.slice) {
      // a contingency slice: the sums over every slice's k, exchanged
      const double *esp = p.xsum + (size_t)ci * T + t0, *esq = p.xsum + (size_t)(p.n_dnode + ci) * T + t0;
#pragma unroll
      for (int e = 0; e < VW; ++e) xs.v[e] = div_rn(fmaf(sm1, (float)esq[e], (float)esp[e]), kpf, rkp);
    } else if constexpr (VW == 4) {
      float4 sp, sq;
      ksum4(Wo, rescale ? Uo : nullptr, ok, T, Kp, sp, sq);   // sum_k PU, sum_k u
      xs.v[0] = div_rn(fmaf(sm1, sq.x, sp.x), kpf, rkp);
      xs.v[1] = div_rn(fmaf(sm1, sq.y, sp.y), kpf, rkp);
      xs.v[2] = div_rn(fmaf(sm1, sq.z, sp.z), kpf, rkp);
      xs.v[3] = div_rn(fmaf(sm1, sq.w, sp.w), kpf, rkp);
    } else {
      float sp, sq;
      ksum(Wo, rescale ? Uo : nullptr, ok, T, Kp, sp, sq);
      xs.v[0] = div_rn(fmaf(sm1, sq, sp), kpf, rkp);
    }
    if (p.dnode_keep[ci]) stv<VW>(p.XS + on, xs);
    for (int j = p.dnode_ptr[ci]; j < p.dnode_ptr[ci + 1]; ++j) {
      const int d = p.dnode_dev[j];
      const size_t od = (size_t)d * T + t0;
      const float den = 2.f * p.dev_a[d] + q.rho_dev, rden = __frcp_rn(den), bd = p.dev_b[d];
      const FV<VW> pd = ldv<VW>(p.PD + od), lo = ldv<VW>(p.dev_lo + od), hi = ldv<VW>(p.dev_hi + od);
      FV<VW> pn, dp;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const float x = pd.v[e] - xs.v[e];                 // p_d - avg_k(pbar + u)
        pn.v[e] = relaxed(p.alpha, fminf(fmaxf(div_rn(q.rho_dev * x - bd, den, rden), lo.v[e]), hi.v[e]),
                          pd.v[e]);
        dp.v[e] = pn.v[e] - pd.v[e];
      }
      stv<VW>(p.DPD + od, dp);
      stv<VW>(p.PD + od, pn);
    }
  }
}

// the register path at the device's own chunk (cs, cr <= C)
template <int C>
__device__ __forceinline__ void stor_r(const Params &p, int sidx, float rho, int lane, int cs) {
  if constexpr (C > 1) {
    if (cs < C) {
      stor_r<C - 1>(p, sidx, rho, lane, cs);
      return;
    }
  }
  stor_prox_r<C>(p, sidx, rho, lane);
}

template <int C>
__device__ __forceinline__ void ramp_r(const Params &p, int r, float rho, int lane, int cr) {
  if constexpr (C > 1) {
    if (cr < C) {
      ramp_r<C - 1>(p, r, rho, lane, cr);
      return;
    }
  }
  ramp_prox_r<C>(p, r, rho, lane);
}

// ---------------------------------------------------------------------------
// inner: one warp per battery, then per ramp-limited generator (Appendix D).
// C > 0: the register path, for horizons of at most REG_T steps (chunks of
// at most C); C = 0: the shared-memory path.  MIXED (batches): the
// instance's horizon chooses, beyond REG_T the shared-memory path.
// ---------------------------------------------------------------------------
template <int C, bool MIXED>
__device__ __forceinline__ void inner_body(const Params &p, unsigned bid, unsigned nblk, float *smem) {
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int T = p.T;
  const int n_inner = p.n_stor + p.n_ramp + p.n_hvdc;
  constexpr bool HAS_SMEM = C == 0 || MIXED, HAS_REG = C > 0;
  const bool reg = HAS_REG && (!HAS_SMEM || T <= REG_T);
  float *wsm = nullptr, *state_sh = nullptr;
  if (HAS_SMEM && !reg) {
    const int wfl = warp_smem_floats(T);
    wsm = smem + (size_t)wib * wfl;
    state_sh = (wfl > 3 * (T + 1)) ? wsm + 3 * (T + 1) : nullptr;
  }
  const int cs = (T + 32) >> 5, cr = (T + 31) >> 5;   // chunks of T + 1 and T elements
  for (int w = bid * nw + wib; w < n_inner; w += nblk * nw) {
    if (w < p.n_stor) {
      if constexpr (HAS_REG) {
        if (reg) {
          stor_r<C>(p, w, q.rho_dev, lane, cs);
          continue;
        }
      }
      if constexpr (HAS_SMEM) stor_prox(p, w, q.rho_dev, wsm, state_sh, lane);
    } else if (w < p.n_stor + p.n_ramp) {
      if constexpr (HAS_REG) {
        if (reg) {
          ramp_r<C>(p, w - p.n_stor, q.rho_dev, lane, cr);
          continue;
        }
      }
      if constexpr (HAS_SMEM) ramp_prox(p, w - p.n_stor, q.rho_dev, wsm, state_sh, lane);
    } else {
      hvdc_prox(p, w - p.n_stor - p.n_ramp, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// dsum: per (node, VW time steps), the sum of the node's device powers and
// the Welford state of their changes, in device order (the node sums of
// every contingency start from it), on the iterations that form residuals
// (and every iteration of the over-relaxed form)
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void dsum_body(const Params &p, unsigned bid, unsigned nblk) {
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  // with dsum_lean the node passes that form no residuals sum the device
  // powers themselves
  if (p.dsum_lean && !q.res && p.alpha == 1.f) return;
  const int T = p.T, TV = T / VW;
  const unsigned n_items = (unsigned)p.N * (unsigned)TV;
  for (unsigned item = bid * BLOCK + threadIdx.x; item < n_items; item += nblk * BLOCK) {
    const int n = (int)(item / (unsigned)TV), t0 = (int)(item % (unsigned)TV) * VW;
    FV<VW> sp;
    Welf<VW> w;
    w.reset();
#pragma unroll
    for (int e = 0; e < VW; ++e) sp.v[e] = 0.f;
    for (int j = p.dcsr_ptr[n]; j < p.dcsr_ptr[n + 1]; ++j) {
      const size_t od = (size_t)p.dcsr_idx[j] * T + t0;
      const FV<VW> pd = ldv<VW>(p.PD + od), dpd = ldv<VW>(p.DPD + od);
#pragma unroll
      for (int e = 0; e < VW; ++e) sp.v[e] += pd.v[e];
      w.add(dpd.v);
    }
    FV<VW> m, q2;
#pragma unroll
    for (int e = 0; e < VW; ++e) { m.v[e] = w.mean[e]; q2.v[e] = w.m2[e]; }
    const size_t os = (size_t)n * T + t0;
    stv<VW>(p.DSP + os, sp);
    stv<VW>(p.DSM + os, m);
    stv<VW>(p.DSQ + os, q2);
  }
}

// ---------------------------------------------------------------------------
// line: step 1 for every (contingency, line, VW time steps)
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void line_body(const Params &p, int k0, int k1, unsigned bid) {
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  const int L = p.L, TV = p.T / VW;
  const unsigned n = (unsigned)(k1 - k0) * (unsigned)L * (unsigned)TV;
  // each CTA takes LINE_IPT consecutive blocks of BLOCK items, so CTAs are
  // short-lived and the device kernels' CTAs find room beside them
  const unsigned base = bid * (unsigned)(BLOCK * LINE_IPT) + threadIdx.x;
  // items (line, contingency, step block): a line's K+1 rows are contiguous
  const int KK = k1 - k0;
  Idx3 ix, dx;
  ix.set(base, KK, TV);
  dx.set(BLOCK, KK, TV);
#pragma unroll 1
  for (int j = 0; j < LINE_IPT; ++j, ix.step(dx, KK, TV)) {
    if (base + (unsigned)(j * BLOCK) < n)
      line_item<VW>(p, q.old, q.nw, k0 + ix.b, ix.a, ix.c * VW, q.frp, q.frt, q.fsu, q.fsv, q.v_fresh);
  }
}

// ---------------------------------------------------------------------------
// node: step 3 for every (contingency, node, VW time steps), and the CTA's
// residual partial sums: FP32 per thread, FP64 across warps
// ---------------------------------------------------------------------------
// LEAN: the variant for iterations that form no residuals (it returns at
// once on the others); the general variant returns at once on those when a
// lean launch covers them.
template <int VW, bool RELAX, bool LEAN = false, int ILD = 2>
__device__ __forceinline__ void node_body(const Params &p, int k0, int k1, int first, unsigned bid,
                                          unsigned nblk, bool lean_split = false) {
  __shared__ double red[WARPS][NSLOT];
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  if constexpr (LEAN) {
    if (q.res) return;
  } else {
    if (lean_split && !q.res) return;
  }
  const int N = p.N, TV = p.T / VW;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned n = (unsigned)(k1 - k0) * (unsigned)N * (unsigned)TV;
  const unsigned stride = nblk * BLOCK;
  unsigned item = bid * BLOCK + threadIdx.x;
  float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f};
  // items (node, contingency, step block): a node's K+1 rows are contiguous,
  // and so are the K+1 rows of each line it gathers
  const int KK = k1 - k0;
  Idx3 ix, dx;
  ix.set(item, KK, TV);
  dx.set(stride, KK, TV);
  for (; item < n; item += stride, ix.step(dx, KK, TV))
    node_item<VW, RELAX, LEAN ? NODE_LEAN_NB : 4, ILD>(p, q.old, q.nw, k0 + ix.b, ix.a, ix.c * VW, q.fsu, acc,
                                                  LEAN ? false : q.res != 0);
  if constexpr (!LEAN) {
    if (!q.res) return;   // nothing reads this iteration's partial sums
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      float v = acc[s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wib][s] = (double)v;
    }
    __syncthreads();
    // the slabs of one iteration run in order on one stream: the first one
    // sets the CTA's partial sums, the others add to them
    if (threadIdx.x < NSLOT) {
      double v = first ? 0.0 : p.partials[(size_t)bid * NSLOT + threadIdx.x];
      for (int w = 0; w < WARPS; ++w) v += red[w][threadIdx.x];
      p.partials[(size_t)bid * NSLOT + threadIdx.x] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// decide: residuals (Section 3.3) from the node kernel's n_part CTA partials
// in FP64 and a fixed order, the stopping test of Eq. (converge) and the
// adaptive penalty (Section 3.5); advances the iteration counter.
// ---------------------------------------------------------------------------
// the node kernel's n_part CTA partial sums reduced in FP64 and a fixed
// order; thread 0 returns true with the totals
__device__ __forceinline__ bool reduce_partials(const Params &p, int n_part, double tot[NSLOT],
                                                double (*red)[NSLOT]) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) tot[s] = 0.0;
  for (int b = threadIdx.x; b < n_part; b += BLOCK) {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) tot[s] += p.partials[(size_t)b * NSLOT + s];
  }
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    double v = tot[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wib][s] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    double v = 0.0;
    for (int w = 0; w < WARPS; ++w) v += red[w][s];
    tot[s] = v;
  }
  return true;
}

__device__ __forceinline__ void decide_body(const Params &p, int n_part) {
  __shared__ double red[WARPS][NSLOT];
  const Iter q = iter_scalars(p);
  if (q.skip) return;
  if (!q.res) {
    // nothing reads this iteration's residuals (a non-finite value is caught
    // at the next iteration that forms them): advance
    if (threadIdx.x == 0) {
      DevScalars sc = *p.sc;
      sc.su = 1.0;
      sc.sv = 1.0;
      sc.it = sc.it + 1;
      sc.v_fresh = 0;
      *p.sc = sc;
    }
    return;
  }
  double tot[NSLOT];
  if (p.slice) {
    // a contingency slice: the residual sums of every slice, exchanged
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) tot[s] = p.xsum[(size_t)2 * p.n_dnode * p.T + s];
  } else {
    if (!reduce_partials(p, n_part, tot, red)) return;
  }
  DevScalars sc = *p.sc;
  const long long itn = sc.it + 1;
  const bool check_now = p.eps > 0 && p.check_every > 0 && (itn % p.check_every) == 0;
  const double rho_p = sc.rho_p, rho_th = sc.rho_th;
  int flags = 0;
  const double r_pp = sqrt(fmax(tot[SL_PP], 0.0));
  const double r_pt = sqrt(fmax(tot[SL_PT], 0.0));
  const double r_dp = rho_p * sqrt(fmax(tot[SL_DP], 0.0));
  const double r_dt = rho_th * sqrt(fmax(tot[SL_DT], 0.0));
  const double rp = sqrt(r_pp * r_pp + r_pt * r_pt);
  const double rd = sqrt(r_dp * r_dp + r_dt * r_dt);
  double nrp = rho_p, nrt = rho_th;
  if (!isfinite(rp) || !isfinite(rd) || tot[SL_NF] != 0.0) {
    sc.status = ST_NONFINITE;
    sc.stop = 1;
    flags |= HF_NONFINITE;
  } else {
    const double m = fmax(rp, rd);
    if (check_now && m <= p.tol) {
      sc.converged = 1;
      sc.stop = 1;
      flags |= HF_CONVERGED;
    } else if (check_now && p.stall_window > 0) {
      // stall rule (include/opf.h, opf_options): progress is a fall of the
      // best m by 1 %; without it for stall_window iterations, fix adapting
      // penalties, else stop with a stall
      if (m < 0.99 * sc.stall_ref) {
        sc.stall_ref = m;
        sc.stall_it = itn;
      } else if (itn - sc.stall_it >= p.stall_window) {
        if (adapting(p, sc, itn)) {
          sc.frozen_at = itn;
          sc.stall_ref = m;
          sc.stall_it = itn;
          flags |= HF_FROZEN;
        } else {
          sc.stalled = 1;
          sc.stop = 1;
          flags |= HF_STALLED;
        }
      }
    }
    if (adapt_at(p, sc, itn)) {   // Section 3.5 (strict comparisons, FP64)
      if (r_pp > p.mu * r_dp) nrp = rho_p * p.gamma;
      else if (r_dp > p.mu * r_pp) nrp = rho_p / p.gamma;
      if (r_pt > p.mu * r_dt) nrt = rho_th * p.gamma;
      else if (r_dt > p.mu * r_pt) nrt = rho_th / p.gamma;
      if (nrp != rho_p || nrt != rho_th) flags |= HF_ADAPTED;
    }
  }
  if (p.hist_cap > 0) {   // residual history ring (opf_history)
    double *row = p.hist + (size_t)(sc.hist_n % p.hist_cap) * HIST_COLS;
    row[0] = (double)itn;
    row[1] = rp;
    row[2] = rd;
    row[3] = r_pp;
    row[4] = r_pt;
    row[5] = r_dp;
    row[6] = r_dt;
    row[7] = rho_p;
    row[8] = rho_th;
    row[9] = (double)flags;
    sc.hist_n += 1;
  }
  sc.res[0] = rp; sc.res[1] = rd; sc.res[2] = r_pp; sc.res[3] = r_pt; sc.res[4] = r_dp; sc.res[5] = r_dt;
  sc.su = rho_p / nrp;   // pending rescale of u and v (Section 3.5), applied on their next read
  sc.sv = rho_th / nrt;
  sc.rho_p = nrp;
  sc.rho_th = nrt;
  sc.it = itn;
  sc.v_fresh = 0;
  *p.sc = sc;
}

// ---------------------------------------------------------------------------
// kernel entry points: one instance (parameters in the constant bank), or a
// batch of instances (each CTA looks up its instance, its block index within
// the instance and the instance's block count in a schedule, and works on a
// shared-memory copy of that instance's parameters)
// ---------------------------------------------------------------------------
template <int VW>
__global__ void __launch_bounds__(BLOCK) xs_kernel(Params p) { xs_body<VW>(p, blockIdx.x, gridDim.x); }

template <int C>
__global__ void __launch_bounds__(BLOCK) inner_kernel(Params p) {
  extern __shared__ float smem[];
  inner_body<C, false>(p, blockIdx.x, gridDim.x, smem);
}

template <int VW>
__global__ void __launch_bounds__(BLOCK) dsum_kernel(Params p) { dsum_body<VW>(p, blockIdx.x, gridDim.x); }

template <int VW>
__global__ void __launch_bounds__(BLOCK, 4) line_kernel(Params p, int k0, int k1) {
  line_body<VW>(p, k0, k1, blockIdx.x);
}

// the over-relaxed variant carries more per-terminal state: it takes the
// registers of one CTA per SM rather than spill
template <int VW, bool RELAX>
__global__ void __launch_bounds__(BLOCK, RELAX ? 1 : NODE_MIN_CTAS) node_kernel(Params p, int k0, int k1, int first) {
  node_body<VW, RELAX>(p, k0, k1, first, blockIdx.x, gridDim.x, !RELAX && VW == NODE_VW);
}

// the residual-free node pass: fewer live values, more CTAs per SM
// ILD: the plan's dsum_lean, fixed at compile time for this pass
template <int ILD>
__global__ void __launch_bounds__(BLOCK, NODE_LEAN_CTAS) node_kernel_lean(Params p, int k0, int k1, int first) {
  node_body<NODE_VW, false, true, ILD>(p, k0, k1, first, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(BLOCK) decide_kernel(Params p, int n_part) { decide_body(p, n_part); }

// A contingency slice's contributions to the exchange (after its node
// sums): sum over its k of pbar + u at every node with devices, the same of
// u on adaptation iterations (whose decision may rescale u before the next
// device prox reads it), and its residual partial sums on iterations that
// form residuals.  A stopped context (and `prime`, before the first
// iteration) contributes the sums of its current state, so that the
// caller's exchange always sums fresh contributions of every slice.
__global__ void __launch_bounds__(BLOCK) slice_sums_kernel(Params p, int prime) {
  __shared__ double red[WARPS][NSLOT];
  __shared__ int s_buf, s_with_u, s_res;
  if (threadIdx.x == 0) {
    const DevScalars sc = *p.sc;
    const long long itn = sc.it + 1;
    const bool stopped = sc.status != 0 || sc.stop != 0;
    const bool current = prime || stopped;
    const int old = (int)(sc.it & 1);
    s_buf = current ? old : old ^ 1;
    s_with_u = current || adapt_at(p, sc, itn);
    s_res = !current && ((p.adapt_every > 0 && adapt_at(p, sc, itn)) ||
                         (p.eps > 0 && p.check_every > 0 && itn % p.check_every == 0) || itn >= sc.it_last);
  }
  __syncthreads();
  const int T = p.T, Kp = p.Kp;
  const size_t KT = (size_t)Kp * T;
  const float *W = p.PU[s_buf], *U = p.U[s_buf];
  const bool with_u = s_with_u != 0;
  double *esp = p.xsum, *esq = p.xsum + (size_t)p.n_dnode * T;
  for (long long i = (long long)blockIdx.x * BLOCK + threadIdx.x; i < (long long)p.n_dnode * T;
       i += (long long)gridDim.x * BLOCK) {
    const int ci = (int)(i / T), t = (int)(i % T);
    float sp, sq;
    ksum(W, with_u ? U : nullptr, (size_t)p.dnode_ids[ci] * KT + t, T, Kp, sp, sq);
    esp[i] = (double)sp;
    esq[i] = (double)sq;
  }
  if (blockIdx.x == 0) {
    double tot[NSLOT];
    double *tail = p.xsum + (size_t)2 * p.n_dnode * T;
    if (s_res) {
      if (reduce_partials(p, p.node_grid, tot, red))
        for (int s = 0; s < NSLOT; ++s) tail[s] = tot[s];
    } else if (threadIdx.x < NSLOT) {
      tail[threadIdx.x] = 0.0;
    }
  }
}

// the instance of this CTA: its parameters copied to shared memory, and
// (block, blocks) within the instance
__device__ __forceinline__ const Params &batch_params(const Params *ps, const int4 *sched, Params &sp,
                                                      unsigned &bid, unsigned &nblk) {
  const int4 e = sched[blockIdx.x];
  static_assert(sizeof(Params) % 4 == 0, "Params is copied as 32-bit words");
  const int *src = reinterpret_cast<const int *>(ps + e.x);
  int *dst = reinterpret_cast<int *>(&sp);
  for (int i = threadIdx.x; i < (int)(sizeof(Params) / 4); i += BLOCK) dst[i] = src[i];
  __syncthreads();
  bid = (unsigned)e.y;
  nblk = (unsigned)e.z;
  return sp;
}

template <int VW>
__global__ void __launch_bounds__(BLOCK) xs_kernel_b(const Params *ps, const int4 *sched) {
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  xs_body<VW>(p, bid, nblk);
}

// batches keep the GPU full of inner-ADMM warps: on the shared-memory path
// alone 64 registers, 4 CTAs per SM; C: the largest register chunk of the
// batch's instances (0: every horizon beyond REG_T), any longer horizon on
// the shared-memory path
template <int C>
__global__ void __launch_bounds__(BLOCK, C == 0 ? 4 : 1) inner_kernel_b(const Params *ps, const int4 *sched) {
  extern __shared__ float smem[];
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  inner_body<C, true>(p, bid, nblk, smem);
}

template <int VW>
__global__ void __launch_bounds__(BLOCK) dsum_kernel_b(const Params *ps, const int4 *sched) {
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  dsum_body<VW>(p, bid, nblk);
}

template <int VW>
__global__ void __launch_bounds__(BLOCK, 4) line_kernel_b(const Params *ps, const int4 *sched) {
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  line_body<VW>(p, 0, p.Kp, bid);
}

template <int VW, bool RELAX>
__global__ void __launch_bounds__(BLOCK, RELAX ? 1 : NODE_MIN_CTAS) node_kernel_b(const Params *ps, const int4 *sched) {
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  node_body<VW, RELAX>(p, 0, p.Kp, 1, bid, nblk);
}

__global__ void __launch_bounds__(BLOCK) decide_kernel_b(const Params *ps, const int4 *sched) {
  __shared__ Params sp;
  unsigned bid, nblk;
  const Params &p = batch_params(ps, sched, sp, bid, nblk);
  decide_body(p, p.node_grid);
}

// A line's terminal values from its stored (p, mid) at contingency k:
// p2 (0 on the outaged line) and theta_{1,2} = mid +- h, h = p / (2b) on an
// active line and the stored value itself on the outaged line.
// the actual iterate from two relaxed ones: (P - (1 - alpha) P_prev) / alpha
__device__ __forceinline__ float actual(float alpha, float cur, float prev) {
  return (cur - (1.f - alpha) * prev) / alpha;
}

__device__ __forceinline__ void line_terminals(const Params &p, int cur, int k, int l, size_t i, float &p2,
                                               float &th1, float &th2) {
  const float ps = p.P[cur][i], m = p.MID[cur][i];
  float h = ps;
  p2 = 0.f;
  if (p.out_line[k] != l) {
    const float tb = 2.f * p.line_b[l];
    h = div_rn(ps, tb, __frcp_rn(tb));
    p2 = ps;
  }
  th1 = m + h;
  th2 = m - h;
}

// ---------------------------------------------------------------------------
// import / export between internal and caller numbering
// ---------------------------------------------------------------------------
__global__ void import_kernel(Params p, int cur, const float *pl, const float *a1, const float *a2,
                              const float *v1, const float *v2, const float *u) {
  const int T = p.T, L = p.L, N = p.N;
  const long long nl = (long long)p.Kp * L * T, nn = (long long)p.Kp * N * T;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nl + nn;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nl) {
      const int k = (int)(i / ((long long)L * T));
      const long long rem = i - (long long)k * L * T;
      const int l = (int)(rem / T), t = (int)(rem % T);
      const size_t src = ((size_t)k * L + p.line_perm[l]) * T + t, dst = lidx(p, k, l, t);
      // stored as p and the mean angle; the outaged line keeps its half
      // angle difference in p's place (its p is 0)
      const float x1 = a1 ? a1[src] : 0.f, x2 = a2 ? a2[src] : 0.f;
      const bool act = p.out_line[k] != l;
      p.P[cur][dst] = act ? (pl ? pl[src] : 0.f) : 0.5f * (x1 - x2);
      p.MID[cur][dst] = 0.5f * (x1 + x2);
      p.V1[cur][dst] = v1 ? v1[src] : 0.f;
      p.V2[cur][dst] = v2 ? v2[src] : 0.f;
    } else {
      const long long j = i - nl;
      const int k = (int)(j / ((long long)N * T));
      const long long rem = j - (long long)k * N * T;
      const int n = (int)(rem / T), t = (int)(rem % T);
      p.U[cur][nidx(p, k, n, t)] = u ? u[((size_t)k * N + p.node_perm[n]) * T + t] : 0.f;
    }
  }
}

// A starting state from node rows in the caller's numbering, rows[(t N + n)
// stride + 0] = price / price_scale and [+ 1] = node angle: u_k = -price /
// (rho_p (K+1)) in every contingency (prices are -rho_p sum_k u_k), every
// line terminal at its node's angle, line power b (theta1 - theta2) clipped
// to the limit (0 on the outaged line of a contingency, whose terminals keep
// their angles), v = 0.  The same construction as a host-built state
// imported through import_kernel.
__global__ void start_from_nodes_kernel(Params p, int cur, const float *rows, int stride, float price_scale,
                                        float u_scale) {
  const int T = p.T, L = p.L, N = p.N;
  const long long nl = (long long)p.Kp * L * T, nn = (long long)p.Kp * N * T;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nl + nn;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nl) {
      const int k = (int)(i / ((long long)L * T));
      const long long rem = i - (long long)k * L * T;
      const int l = (int)(rem / T), t = (int)(rem % T);
      const float x1 = rows[((size_t)t * N + p.node_perm[p.line_n1[l]]) * stride + 1];
      const float x2 = rows[((size_t)t * N + p.node_perm[p.line_n2[l]]) * stride + 1];
      const bool act = p.out_line[k] != l;
      const float u = p.line_u[l];
      const size_t dst = lidx(p, k, l, t);
      p.P[cur][dst] = act ? fminf(fmaxf(p.line_b[l] * (x1 - x2), -u), u) : 0.5f * (x1 - x2);
      p.MID[cur][dst] = 0.5f * (x1 + x2);
      p.V1[cur][dst] = 0.f;
      p.V2[cur][dst] = 0.f;
    } else {
      const long long j = i - nl;
      const int k = (int)(j / ((long long)N * T));
      const long long rem = j - (long long)k * N * T;
      const int n = (int)(rem / T), t = (int)(rem % T);
      const float price = rows[((size_t)t * N + p.node_perm[n]) * stride] * price_scale;
      p.U[cur][nidx(p, k, n, t)] = -price * u_scale;
    }
  }
}

// node averages from the stored terminal values (after import)
__global__ void node_average_kernel(Params p, int cur) {
  const int T = p.T, N = p.N;
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x; item < (long long)N * T;
       item += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(item / T), t = (int)(item % T);
    float devsum = 0.f;
    for (int j = p.dcsr_ptr[n]; j < p.dcsr_ptr[n + 1]; ++j) devsum += p.PD[(size_t)p.dcsr_idx[j] * T + t];
    for (int k = 0; k < p.Kp; ++k) {
      float sp = devsum, st = 0.f;
      for (int j = p.lcsr_ptr[n]; j < p.lcsr_ptr[n + 1]; ++j) {
        const int code = p.lcsr[j].x;
        const size_t ol = lidx(p, k, code >> 1, t);
        float p2, th1, th2;
        line_terminals(p, cur, k, code >> 1, ol, p2, th1, th2);
        sp += (code & 1) ? p2 : -p2;
        st += (code & 1) ? th2 : th1;
      }
      const size_t on = nidx(p, k, n, t);
      const float pb = sp / p.cnt_p[n];
      p.PU[cur][on] = pb + p.U[cur][on];   // u was imported before
      p.THBAR[cur][on] = p.cnt_th[n] > 0.f ? st / p.cnt_th[n] : 0.f;
    }
  }
}

// v projected onto v_bar = 0 per node and contingency (Appendix C)
__global__ void project_v_kernel(Params p, int cur) {
  const int T = p.T, N = p.N;
  for (long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
       item < (long long)p.Kp * N * T; item += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(item / ((long long)N * T));
    const long long rem = item - (long long)k * N * T;
    const int n = (int)(rem / T), t = (int)(rem % T);
    const int l0 = p.lcsr_ptr[n], l1 = p.lcsr_ptr[n + 1];
    if (l1 == l0) continue;
    float s = 0.f;
    for (int j = l0; j < l1; ++j) {
      const int code = p.lcsr[j].x;
      const size_t ol = lidx(p, k, code >> 1, t);
      s += (code & 1) ? p.V2[cur][ol] : p.V1[cur][ol];
    }
    const float m = s / p.cnt_th[n];
    for (int j = l0; j < l1; ++j) {
      const int code = p.lcsr[j].x;
      const size_t ol = lidx(p, k, code >> 1, t);
      if (code & 1) p.V2[cur][ol] -= m; else p.V1[cur][ol] -= m;
    }
  }
}

// lines to caller numbering; v = sv (V + theta - theta_bar) unless fresh
__global__ void export_lines_kernel(Params p, int cur, float *pl, float *a1, float *a2, float *v1,
                                    float *v2) {
  const DevScalars sc = *p.sc;
  const float sv = (float)sc.sv;
  const int T = p.T, L = p.L;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)p.Kp * L * T;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / ((long long)L * T));
    const long long rem = i - (long long)k * L * T;
    const int l = (int)(rem / T), t = (int)(rem % T);
    const size_t dst = ((size_t)k * L + p.line_perm[l]) * T + t, li = lidx(p, k, l, t);
    float p2, th1, th2;
    line_terminals(p, cur, k, l, li, p2, th1, th2);
    if (v1 || v2) {
      float x = p.V1[cur][li], y = p.V2[cur][li];
      if (!sc.v_fresh) {
        x += th1 - p.THBAR[cur][nidx(p, k, p.line_n1[l], t)];
        y += th2 - p.THBAR[cur][nidx(p, k, p.line_n2[l], t)];
      }
      if (v1) v1[dst] = sv * x;
      if (v2) v2[dst] = sv * y;
    }
    if (p.alpha != 1.f && !sc.v_fresh) {
      // over-relaxed: the buffers hold P = alpha p + (1 - alpha) P_prev
      float q2, q1a, q2a;
      line_terminals(p, cur ^ 1, k, l, li, q2, q1a, q2a);
      p2 = actual(p.alpha, p2, q2);
      th1 = actual(p.alpha, th1, q1a);
      th2 = actual(p.alpha, th2, q2a);
    }
    if (pl) pl[dst] = p2;
    if (a1) a1[dst] = th1;
    if (a2) a2[dst] = th2;
  }
}

// nodes to caller numbering: u (pending rescale applied), theta_bar, and the
// prices -rho_p sum_k u_k
__global__ void export_nodes_kernel(Params p, int cur, float *u, float *theta, float *price) {
  const DevScalars sc = *p.sc;
  const int T = p.T, N = p.N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)N * T;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / T), t = (int)(i % T);
    const size_t ext = (size_t)p.node_perm[n] * T + t;
    double s = 0.0;
    for (int k = 0; k < p.Kp; ++k) {
      const size_t o = nidx(p, k, n, t);
      const float uu = p.U[cur][o];
      if (u) u[(size_t)k * N * T + ext] = (float)(sc.su * uu);
      if (theta)
        theta[(size_t)k * N * T + ext] = (p.alpha != 1.f && !sc.v_fresh)
                                             ? actual(p.alpha, p.THBAR[cur][o], p.THBAR[cur ^ 1][o])
                                             : p.THBAR[cur][o];
      s += uu;
    }
    if (price) price[ext] = (float)(-sc.rho_p * sc.su * s);
  }
}

// device powers in caller order: the actual iterate (relaxed state undone)
__global__ void export_pdev_kernel(Params p, float *out) {
  const DevScalars sc = *p.sc;
  const bool rx = p.alpha != 1.f && !sc.v_fresh;
  const float c = (1.f - p.alpha) / p.alpha;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)p.S * p.T;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = rx ? fmaf(c, p.DPD[i], p.PD[i]) : p.PD[i];
}

__global__ void begin_kernel(DevScalars *sc, long long n, int clear_stop) {
  if (clear_stop) {
    sc->stop = 0;
    if (sc->stalled) {   // a new call after a stall restarts the stall window
      sc->stalled = 0;
      sc->stall_ref = HUGE_VAL;
      sc->stall_it = sc->it;
    }
  }
  sc->it_last = sc->it + n;
}

__global__ void begin_batch_kernel(const Params *ps, int n_inst, long long n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_inst) ps[i].sc->it_last = ps[i].sc->it + n;
}

__global__ void set_rho_kernel(DevScalars *sc, double rho) {
  DevScalars s = *sc;
  s.su *= s.rho_p / rho;
  s.sv *= s.rho_th / rho;
  s.rho_p = rho;
  s.rho_th = rho;
  *sc = s;
}

static size_t inner_smem(int T) { return (size_t)WARPS * warp_smem_floats(T) * sizeof(float); }

}  // namespace opfk

using namespace opfk;

// blocks of a grid-stride kernel: resident CTAs per SM times the SM count
template <class F>
static int resident_grid(F fn, size_t smem) {
  int dev = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, BLOCK, smem) != cudaSuccess || nb < 1) return -1;
  return nb * sms;
}

int opfk_plan(const Params &p, IterPlan *plan) {
  const bool v4 = (p.T % 4 == 0), v2 = (p.T % 2 == 0);
  // the inner ADMM in registers up to REG_T steps, else in shared memory
  const int ic = inner_chunk(p.T);
  const size_t ism = ic ? 0 : inner_smem(p.T);
  if (ism > 48 * 1024 &&
      cudaFuncSetAttribute(inner_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism) != cudaSuccess)
    return -1;
  const bool vn = (p.T % NODE_VW == 0);
  const int gn = vn ? resident_grid(node_kernel<NODE_VW, false>, 0) : resident_grid(node_kernel<1, false>, 0);
  const int gl = vn ? resident_grid(node_kernel_lean<0>, 0) : 0;
  const int gx = v4 ? resident_grid(xs_kernel<4>, 0) : resident_grid(xs_kernel<1>, 0);
  const int gd = v2 ? resident_grid(dsum_kernel<2>, 0) : resident_grid(dsum_kernel<1>, 0);
  if (gn < 1 || gx < 1 || gd < 1) return -1;
  // contingency slabs: the node sums of slab s run beside the line proxes of
  // slab s + 1, so the latency-bound node pass overlaps the bandwidth-bound
  // line pass; a few slabs keep the launch count low
  int ns = std::min(N_SLABS, p.Kp);
  int G = (p.Kp + ns - 1) / ns;
  ns = (p.Kp + G - 1) / G;
  plan->n_slabs = ns;
  plan->slab_k = G;
  const long long tvl = p.T / (v4 ? 4 : 1), tvn = p.T / (vn ? NODE_VW : 1);
  const long long nl = (long long)G * p.L * tvl, nn = (long long)G * p.N * tvn;
  const long long nx = (long long)p.n_dnode * (p.T / (v4 ? 4 : 1));
  const int n_inner = p.n_stor + p.n_ramp + p.n_hvdc;
  plan->line_grid = (int)((nl + (long long)BLOCK * LINE_IPT - 1) / ((long long)BLOCK * LINE_IPT));
  plan->node_grid = (int)std::min<long long>(gn, (nn + BLOCK - 1) / BLOCK);
  plan->lean_grid = vn ? (int)std::min<long long>(gl, (nn + BLOCK - 1) / BLOCK) : 0;
  plan->xs_grid = (int)std::min<long long>(gx, (nx + BLOCK - 1) / BLOCK);
  plan->inner_grid = (n_inner + WARPS - 1) / WARPS;
  {
    // The inner-ADMM kernel is latency-bound (one warp per device through its
    // ten Appendix D iterations) and runs beside the bandwidth-bound line
    // kernel, whose CTAs it displaces.  When the line pass is long enough to
    // hide it, fewer CTAs walking the devices in several rounds leave the
    // line kernel more of the GPU.  The estimates: the line pass moves about
    // 32 bytes per (line, contingency, step) at 6.5 TB/s; a round of devices
    // takes about 0.13 T microseconds from registers, 0.45 T in shared memory.
    // Registers: the fewest CTAs whose rounds fit in half the line pass (10k
    // buses, T = 96, K = 50, 3,000 devices, in ms per iteration: 375 CTAs
    // 0.706, 76 CTAs 0.706, 38 0.698, 25 0.696, 19 0.704, 12 0.851).  Shared
    // memory: one CTA on every other SM while its rounds fit in 70 % of it
    // (0.741 -> 0.706 at the same size).
    const double line_us = (double)p.Kp * p.L * p.T * 32.0 / 6.5e6;
    plan->dsum_lean = 0;
    if (ic) {
      const int max_rounds = (int)std::floor(0.5 * line_us / (0.13 * p.T));
      if (max_rounds >= 2) plan->inner_grid = (plan->inner_grid + max_rounds - 1) / max_rounds;
      // a line pass too short to hide the device chain (xs, inner, dsum):
      // shorten the chain by summing device powers in the node passes that
      // form no residuals (2k buses, T = 24: 35.5 -> 34.0 us per iteration;
      // at 10k, where the chain is hidden, the extra loads of the node pass
      // cost more than dsum: 0.697 -> 0.701 ms)
      else plan->dsum_lean = 1;
    } else {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms >= 2) {
        const int half = sms / 2;
        if (plan->inner_grid > half) {
          const double rounds = std::ceil((double)plan->inner_grid / half);
          if (rounds * 0.45 * p.T <= 0.7 * line_us) plan->inner_grid = half;
        }
      }
    }
  }
  const long long nd = (long long)p.N * (p.T / (v2 ? 2 : 1));
  plan->dsum_grid = (int)std::min<long long>(gd, (nd + BLOCK - 1) / BLOCK);
  plan->inner_smem = ism;
  plan->inner_c = ic;
  return 0;
}

static int aux_grid(long long work);

static int iteration_enqueue(const Params &p, const IterPlan &plan, void *main_stream, void *aux_stream,
                             void *ev_fork, void *ev_join, bool slice) {
  cudaStream_t sm = (cudaStream_t)main_stream, sa = (cudaStream_t)aux_stream;
  const bool v4 = (p.T % 4 == 0), v2 = (p.T % 2 == 0);
  // The line proxes of slab s (aux stream) read only the previous iterate;
  // the node sums of slab s (main stream) follow them and the device
  // kernels, and run beside the line proxes of slab s + 1.
  if (cudaEventRecord((cudaEvent_t)ev_fork, sm) != cudaSuccess) return -1;
  if (cudaStreamWaitEvent(sa, (cudaEvent_t)ev_fork, 0) != cudaSuccess) return -1;
  if (plan.xs_grid > 0) {
    if (v4) xs_kernel<4><<<plan.xs_grid, BLOCK, 0, sm>>>(p);
    else xs_kernel<1><<<plan.xs_grid, BLOCK, 0, sm>>>(p);
  }
  if (plan.inner_grid > 0) {
    switch (plan.inner_c) {
      case 1: inner_kernel<1><<<plan.inner_grid, BLOCK, 0, sm>>>(p); break;
      case 2: inner_kernel<2><<<plan.inner_grid, BLOCK, 0, sm>>>(p); break;
      case 3: inner_kernel<3><<<plan.inner_grid, BLOCK, 0, sm>>>(p); break;
      case 4: inner_kernel<4><<<plan.inner_grid, BLOCK, 0, sm>>>(p); break;
      default: inner_kernel<0><<<plan.inner_grid, BLOCK, plan.inner_smem, sm>>>(p); break;
    }
  }
  if (v2) dsum_kernel<2><<<plan.dsum_grid, BLOCK, 0, sm>>>(p);
  else dsum_kernel<1><<<plan.dsum_grid, BLOCK, 0, sm>>>(p);
  for (int s = 0; s < plan.n_slabs; ++s) {
    const int k0 = s * plan.slab_k, k1 = std::min(p.Kp, k0 + plan.slab_k);
    if (plan.line_grid > 0 && p.L > 0) {
      const int lg = (int)(((long long)(k1 - k0) * p.L * (p.T / (v4 ? 4 : 1)) + (long long)BLOCK * LINE_IPT - 1) /
                           ((long long)BLOCK * LINE_IPT));
      if (v4) line_kernel<4><<<lg, BLOCK, 0, sa>>>(p, k0, k1);
      else line_kernel<1><<<lg, BLOCK, 0, sa>>>(p, k0, k1);
      if (cudaEventRecord((cudaEvent_t)ev_join, sa) != cudaSuccess) return -1;
      if (cudaStreamWaitEvent(sm, (cudaEvent_t)ev_join, 0) != cudaSuccess) return -1;
    }
    const bool vn = p.T % NODE_VW == 0, rx = p.alpha != 1.f;
    if (vn && !rx) {
      // one of the two returns at once: the general pass forms residuals,
      // the lean one runs the iterations that need none
      node_kernel<NODE_VW, false><<<plan.node_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
      if (p.dsum_lean) node_kernel_lean<1><<<plan.lean_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
      else node_kernel_lean<0><<<plan.lean_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
    }
    else if (!rx) node_kernel<1, false><<<plan.node_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
    else if (vn) node_kernel<NODE_VW, true><<<plan.node_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
    else node_kernel<1, true><<<plan.node_grid, BLOCK, 0, sm>>>(p, k0, k1, s == 0);
  }
  if (slice) slice_sums_kernel<<<aux_grid((long long)p.n_dnode * p.T), BLOCK, 0, sm>>>(p, 0);
  else decide_kernel<<<1, BLOCK, 0, sm>>>(p, plan.node_grid);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_iteration_enqueue(const Params &p, const IterPlan &plan, void *main_stream, void *aux_stream,
                           void *ev_fork, void *ev_join) {
  return iteration_enqueue(p, plan, main_stream, aux_stream, ev_fork, ev_join, false);
}

int opfk_slice_local_enqueue(const Params &p, const IterPlan &plan, void *main_stream, void *aux_stream,
                             void *ev_fork, void *ev_join) {
  return iteration_enqueue(p, plan, main_stream, aux_stream, ev_fork, ev_join, true);
}

int opfk_slice_finish_enqueue(const Params &p, void *stream) {
  decide_kernel<<<1, BLOCK, 0, (cudaStream_t)stream>>>(p, p.node_grid);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_slice_prime_launch(const Params &p, void *stream) {
  slice_sums_kernel<<<aux_grid((long long)p.n_dnode * p.T), BLOCK, 0, (cudaStream_t)stream>>>(p, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_batch_plan(const Params *hp, const IterPlan *plans, int n, const BatchLayout &lay, int *sched_out,
                    long long sched_cap, long long *sched_len, BatchPlan *bp) {
  long long len = 0;
  size_t ism = 0;
  int ic_max = 0;
  auto put = [&](int inst, long long b, long long blocks) -> bool {
    if (sched_out) {
      if (len >= sched_cap) return false;
      int *e = sched_out + 4 * len;
      e[0] = inst;
      e[1] = (int)b;
      e[2] = (int)blocks;
      e[3] = 0;
    }
    ++len;
    return true;
  };
  const int div = std::max(1, lay.div);
  std::vector<long long> nb(n);
  for (int kind = 0; kind < BK_COUNT; ++kind) {
    bp->offset[kind] = (int)len;
    long long most = 0;
    for (int j = 0; j < n; ++j) {
      const int i = lay.order ? lay.order[j] : j;
      const Params &p = hp[i];
      const bool v4 = (p.T % 4 == 0), v2 = (p.T % 2 == 0), vn = (p.T % NODE_VW == 0);
      const long long tv4 = p.T / (v4 ? 4 : 1), tv2 = p.T / (v2 ? 2 : 1);
      const int n_inner = p.n_stor + p.n_ramp + p.n_hvdc;
      long long blocks = 0;
      switch (kind) {
        case BK_XS4: case BK_XS1:
          if ((kind == BK_XS4) == v4) blocks = ((long long)p.n_dnode * tv4 + BLOCK - 1) / BLOCK;
          break;
        case BK_INNER:
          blocks = (n_inner + WARPS - 1) / WARPS;
          if (blocks) {
            const int ic = inner_chunk(p.T);
            if (ic) ic_max = std::max(ic_max, ic);
            else ism = std::max(ism, inner_smem(p.T));   // the shared-memory path
          }
          break;
        case BK_DSUM2: case BK_DSUM1:
          if ((kind == BK_DSUM2) == v2) blocks = ((long long)p.N * tv2 + BLOCK - 1) / BLOCK;
          break;
        case BK_LINE4: case BK_LINE1:
          if ((kind == BK_LINE4) == v4 && p.L > 0)
            blocks = ((long long)p.Kp * p.L * tv4 + (long long)BLOCK * LINE_IPT - 1) / ((long long)BLOCK * LINE_IPT);
          break;
        case BK_NODE4: case BK_NODE1:
          if ((kind == BK_NODE4) == vn) blocks = plans[i].node_grid;
          break;
        case BK_DECIDE:
          blocks = 1;
          break;
      }
      // the grid-stride phases take any block count: `div` puts more work in
      // each CTA (for the node phase the caller sets the instance's partial-sum
      // count to the same number, batch_node_blocks)
      if (blocks > 0 && (kind == BK_XS4 || kind == BK_XS1 || kind == BK_INNER || kind == BK_DSUM2 ||
                         kind == BK_DSUM1 || kind == BK_NODE4 || kind == BK_NODE1))
        blocks = (blocks + div - 1) / div;
      nb[j] = blocks;
      most = std::max(most, blocks);
    }
    // instances in `order`, each instance's CTAs together or dealt round-robin
    if (lay.interleave) {
      for (long long r = 0; r < most; ++r)
        for (int j = 0; j < n; ++j)
          if (r < nb[j] && !put(lay.order ? lay.order[j] : j, r, nb[j])) return -1;
    } else {
      for (int j = 0; j < n; ++j)
        for (long long r = 0; r < nb[j]; ++r)
          if (!put(lay.order ? lay.order[j] : j, r, nb[j])) return -1;
    }
    bp->count[kind] = (int)(len - bp->offset[kind]);
  }
  static_assert(NODE_VW == 4, "the batch node kernels are instantiated for widths 4 and 1");
  bp->inner_c = ic_max;
  bp->inner_smem = ism;
  bp->relax = (n > 0 && hp[0].alpha != 1.f) ? 1 : 0;
  for (int i = 0; i < n; ++i)
    if ((hp[i].alpha != 1.f) != (bp->relax != 0)) return -2;   // one node kernel for every instance
  if (ism > 48 * 1024) {
    const int a = (int)ism;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(inner_kernel_b<0>, at, a) != cudaSuccess ||
        cudaFuncSetAttribute(inner_kernel_b<1>, at, a) != cudaSuccess ||
        cudaFuncSetAttribute(inner_kernel_b<2>, at, a) != cudaSuccess ||
        cudaFuncSetAttribute(inner_kernel_b<3>, at, a) != cudaSuccess ||
        cudaFuncSetAttribute(inner_kernel_b<4>, at, a) != cudaSuccess)
      return -1;
  }
  *sched_len = len;
  return 0;
}

int opfk_batch_node_blocks(const IterPlan &plan, int div) {
  const int d = div > 1 ? div : 1;
  return (plan.node_grid + d - 1) / d;
}

int opfk_batch_enqueue(const Params *d_params, const int *d_sched, const BatchPlan &bp, void *main_stream,
                       void *aux_stream, void *ev_fork, void *ev_join) {
  cudaStream_t sm = (cudaStream_t)main_stream, sa = (cudaStream_t)aux_stream;
  const int4 *sched = reinterpret_cast<const int4 *>(d_sched);
  auto at = [&](int kind) { return sched + bp.offset[kind]; };
  if (cudaEventRecord((cudaEvent_t)ev_fork, sm) != cudaSuccess) return -1;
  if (cudaStreamWaitEvent(sa, (cudaEvent_t)ev_fork, 0) != cudaSuccess) return -1;
  if (bp.count[BK_LINE4]) line_kernel_b<4><<<bp.count[BK_LINE4], BLOCK, 0, sa>>>(d_params, at(BK_LINE4));
  if (bp.count[BK_LINE1]) line_kernel_b<1><<<bp.count[BK_LINE1], BLOCK, 0, sa>>>(d_params, at(BK_LINE1));
  if (cudaEventRecord((cudaEvent_t)ev_join, sa) != cudaSuccess) return -1;
  if (bp.count[BK_XS4]) xs_kernel_b<4><<<bp.count[BK_XS4], BLOCK, 0, sm>>>(d_params, at(BK_XS4));
  if (bp.count[BK_XS1]) xs_kernel_b<1><<<bp.count[BK_XS1], BLOCK, 0, sm>>>(d_params, at(BK_XS1));
  if (bp.count[BK_INNER]) {
    const int4 *si = at(BK_INNER);
    const int nb = bp.count[BK_INNER];
    switch (bp.inner_c) {
      case 1: inner_kernel_b<1><<<nb, BLOCK, bp.inner_smem, sm>>>(d_params, si); break;
      case 2: inner_kernel_b<2><<<nb, BLOCK, bp.inner_smem, sm>>>(d_params, si); break;
      case 3: inner_kernel_b<3><<<nb, BLOCK, bp.inner_smem, sm>>>(d_params, si); break;
      case 4: inner_kernel_b<4><<<nb, BLOCK, bp.inner_smem, sm>>>(d_params, si); break;
      default: inner_kernel_b<0><<<nb, BLOCK, bp.inner_smem, sm>>>(d_params, si); break;
    }
  }
  if (bp.count[BK_DSUM2]) dsum_kernel_b<2><<<bp.count[BK_DSUM2], BLOCK, 0, sm>>>(d_params, at(BK_DSUM2));
  if (bp.count[BK_DSUM1]) dsum_kernel_b<1><<<bp.count[BK_DSUM1], BLOCK, 0, sm>>>(d_params, at(BK_DSUM1));
  if (cudaStreamWaitEvent(sm, (cudaEvent_t)ev_join, 0) != cudaSuccess) return -1;
  if (!bp.relax) {
    if (bp.count[BK_NODE4]) node_kernel_b<4, false><<<bp.count[BK_NODE4], BLOCK, 0, sm>>>(d_params, at(BK_NODE4));
    if (bp.count[BK_NODE1]) node_kernel_b<1, false><<<bp.count[BK_NODE1], BLOCK, 0, sm>>>(d_params, at(BK_NODE1));
  } else {
    if (bp.count[BK_NODE4]) node_kernel_b<4, true><<<bp.count[BK_NODE4], BLOCK, 0, sm>>>(d_params, at(BK_NODE4));
    if (bp.count[BK_NODE1]) node_kernel_b<1, true><<<bp.count[BK_NODE1], BLOCK, 0, sm>>>(d_params, at(BK_NODE1));
  }
  if (bp.count[BK_DECIDE]) decide_kernel_b<<<bp.count[BK_DECIDE], BLOCK, 0, sm>>>(d_params, at(BK_DECIDE));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

static int aux_grid(long long work) {
  long long g = (work + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

int opfk_import_launch(const Params &p, int cur, const float *pl, const float *a1, const float *a2,
                       const float *v1, const float *v2, const float *u, void *stream) {
  const long long work = (long long)p.Kp * (p.L + p.N) * p.T;
  import_kernel<<<aux_grid(work), 256, 0, (cudaStream_t)stream>>>(p, cur, pl, a1, a2, v1, v2, u);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_start_from_nodes_launch(const Params &p, int cur, const float *rows, int stride, float price_scale,
                                 float u_scale, void *stream) {
  start_from_nodes_kernel<<<aux_grid((long long)p.Kp * (p.L + p.N) * p.T), 256, 0, (cudaStream_t)stream>>>(
      p, cur, rows, stride, price_scale, u_scale);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_node_average_launch(const Params &p, int cur, void *stream) {
  node_average_kernel<<<aux_grid((long long)p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p, cur);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_project_v_launch(const Params &p, int cur, void *stream) {
  project_v_kernel<<<aux_grid((long long)p.Kp * p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p, cur);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_export_lines_launch(const Params &p, int cur, float *pl, float *a1, float *a2, float *v1,
                             float *v2, void *stream) {
  export_lines_kernel<<<aux_grid((long long)p.Kp * p.L * p.T), 256, 0, (cudaStream_t)stream>>>(
      p, cur, pl, a1, a2, v1, v2);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_begin_launch(DevScalars *sc, long long n, int clear_stop, void *stream) {
  begin_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(sc, n, clear_stop);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_begin_batch_launch(const Params *d_params, int n_inst, long long n, void *stream) {
  begin_batch_kernel<<<(n_inst + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, n_inst, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_export_pdev_launch(const Params &p, float *out, void *stream) {
  export_pdev_kernel<<<aux_grid((long long)p.S * p.T), 256, 0, (cudaStream_t)stream>>>(p, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_export_nodes_launch(const Params &p, int cur, float *u, float *theta, float *price,
                             void *stream) {
  export_nodes_kernel<<<aux_grid((long long)p.N * p.T), 256, 0, (cudaStream_t)stream>>>(p, cur, u, theta,
                                                                                         price);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opfk_set_rho_launch(DevScalars *sc, double rho, void *stream) {
  set_rho_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(sc, rho);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
