// Gradients of the system cost after K unrolled iterations (include/opf_diff.h).
//
// A self-contained differentiable path in the caller's numbering: the state
// (p, theta1, theta2, v1, v2 per line and contingency; device power; u, and
// the node averages pbar, theta_bar per node and contingency; the inner-ADMM
// duals beta, lambda of ramp-limited generators and batteries) is kept in
// plain arrays, and every step of the iteration has a forward kernel and an
// adjoint kernel.  Forward states are stored every `checkpoint_every`
// iterations and recomputed segment by segment during the reverse pass.
// Every adjoint item writes only its own entries (sums over a node's
// terminals are CSR gathers, an inner device is one CTA), so the gradients
// are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "opf_diff.h"
#include "opf_internal.h"

namespace {

constexpr int TB = 256;       // threads per CTA of the element-wise kernels (eight per SM: they wait
                              // on gathers, so they are held to 32 registers for the most warps)
constexpr int VW4_CTAS = 4;   // ... the line and node kernels on four steps per thread: more registers
constexpr int TBI = 128;      // threads per CTA of the inner-ADMM kernels (one CTA per device)
constexpr int N_INNER = 10;   // Appendix D iterations per prox evaluation (Section 4.5)

// one inner-ADMM device: its index among all devices, its constraint shape,
// and offsets of its inverse system matrix, right-hand side rows and linear cost
struct IDev {
  int dev, shape, minv, h, q, bat, piv, pad1;  // bat: battery index, -1 for a generator; piv: see DP::piv
};

// constraint rows A z <= h (eq: = h) of one device kind, in CSR and CSC form
// (nnz nonzeros)
struct Shape {
  int n, m, rp, ci, tp, ti, eq, nnz;
};

struct DP {
  int N, L, T, Kp, G, D, B, H, S;       // H HVDC links, terminals H0 + 2h and H0 + 2h + 1 (H0 = G + D + B)
  float rp, rt, rd;                    // rho_p, rho_theta, (K+1) rho_p (= omega of the inner ADMM)
  const int *n1, *n2;                  // line ends (terminal 1 at n1 carries -p)
  const float *b;                      // susceptance [L]
  const int *out;                      // [Kp] outaged line, -1 = none
  const int *lptr, *lcode;             // node -> line terminal codes 2 l + end (end 1: terminal 2)
  const int *dptr, *didx;              // node -> devices
  const float *cnt, *cth;              // terminals at a node: all, line (0: none)
  // the reverse pass's factors: 1 / cnt, 1 / cth (0 for none) [N]; per line
  // 1 / (2b), rho_p / den, rho_theta / (2b den) [3][L]
  const float *icnt, *icth, *lfac;
  const int *dnode;                    // device node [S]
  const int *kind;                     // [S] 0: closed-form prox, 1: inner ADMM, 2: HVDC terminal
  const float *hvdc_u;                 // [H]
  const float *ga, *gb, *gpmin;        // generators: a, b [G]; pmin [G][T]
  const float *voll;                   // loads [D], < 0: fixed
  const float *load_p, *gpmax, *lu;    // data: [D][T], [G][T], [L]
  // inner ADMM (Appendix D)
  int n_inner, Mtot;                   // devices, rows over all devices
  int n_inode;                         // nodes with an inner-ADMM device: inode [n_inode], hasin [N]
  const int *inode;
  const unsigned char *hasin;
  const IDev *idev;
  const Shape *shape;
  const int *arp, *aci, *atp, *ati;
  const float *acv, *atv, *minv, *RH, *Q, *scost;   // RH: right-hand sides of the inner rows
  const unsigned char *aeq;
  // the register path of the inner ADMM (horizons up to DREG_T): chunk of
  // steps per lane (0: the shared-memory path), each device's factor at
  // IDev::piv -- a ramp generator its pivots q [T] and a = 2 omega / q [T],
  // a battery eight constants (H^-1: i00 i01 i11, g = H^-1 f: gc gd), then
  // q [T+1] and a = gam / q [T+1] -- and the batteries' efficiencies
  int reg_c;
  const float *piv, *beff;
};

struct St {
  float *P, *TH1, *TH2, *V1, *V2, *PD, *U, *PB, *TBR, *INS;  // INS: beta [Mtot] then lambda [Mtot]
};

struct Adj {
  float *LP, *LT1, *LT2, *LV1, *LV2, *LPD, *LU, *LINS;
};

__device__ __forceinline__ size_t li(const DP &p, int k, int l, int t) { return ((size_t)k * p.L + l) * p.T + t; }
__device__ __forceinline__ size_t ni(const DP &p, int k, int n, int t) { return ((size_t)k * p.N + n) * p.T + t; }

// item loops with 32-bit indices: opf_diff_create checks that every item
// count stays below 2^31 (64-bit divisions per item cost more than the work)
#define GRID_STRIDE(i, n) \
  for (unsigned i = blockIdx.x * TB + threadIdx.x, n_##i = (unsigned)(n); i < n_##i; i += gridDim.x * TB)

// The device kernels give each device step (d, t) a group of KL lanes, which
// split its sums over the K+1 contingencies: lane j takes k = j, j + KL, ...,
// and the partial sums meet in a butterfly whose pattern is fixed (so the
// result is the same wherever it is formed; floating-point addition is
// commutative, so every lane ends with the same total).  Without the split a
// device kernel ran about 200 CTAs of threads each walking 21 contingencies
// one load after another.  The loop trip count is the same for the lanes of
// a group.
constexpr int KL = 8;
#define GROUP_STRIDE(i, n)                                                                   \
  for (unsigned i = (blockIdx.x * TB + threadIdx.x) / KL, n_##i = (unsigned)(n); i < n_##i; \
       i += gridDim.x * (TB / KL))
// the same loops over blocks bid of nb (a kernel whose blocks take two roles)
#define GRID_STRIDE_B(i, n, bid, nb) \
  for (unsigned i = (bid) * TB + threadIdx.x, n_##i = (unsigned)(n); i < n_##i; i += (nb) * TB)
#define GROUP_STRIDE_B(i, n, bid, nb)                                                   \
  for (unsigned i = ((bid) * TB + threadIdx.x) / KL, n_##i = (unsigned)(n); i < n_##i; \
       i += (nb) * (TB / KL))

__device__ __forceinline__ unsigned group_mask() { return 0xFFu << ((threadIdx.x & 31) & ~(KL - 1)); }

// sum over the contingencies of V (and W, when not NULL) at node n, step t,
// split over the group's lanes (lane j = threadIdx.x % KL)
__device__ __forceinline__ float ksum(const DP &p, const float *V, const float *W, int n, int t) {
  const int j = threadIdx.x & (KL - 1);
  float s = 0.f;
  if (W) {
#pragma unroll 3
    for (int k = j; k < p.Kp; k += KL) s += V[ni(p, k, n, t)] + W[ni(p, k, n, t)];
  } else {
#pragma unroll 3
    for (int k = j; k < p.Kp; k += KL) s += V[ni(p, k, n, t)];
  }
  const unsigned gm = group_mask();
#pragma unroll
  for (int o = KL / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gm, s, o);
  return s;
}

// ---------------------------------------------------------------------------
// forward (Section 3.2)
// ---------------------------------------------------------------------------

// The line and node kernels take VW consecutive time steps per thread: 4
// when T is a multiple of 4 (then every row offset is a multiple of 4 floats
// and every array starts on a 16-byte boundary, so rows move as 128-bit
// loads and stores and an item's index arithmetic is shared by its steps),
// else 1.  Each step's arithmetic is the same whatever VW.
template <int VW>
struct Vf {
  float x[VW];
};
template <int VW>
__device__ __forceinline__ Vf<VW> ldv(const float *q) {
  Vf<VW> r;
  if constexpr (VW == 4) {
    const float4 f = *reinterpret_cast<const float4 *>(q);
    r.x[0] = f.x;
    r.x[1] = f.y;
    r.x[2] = f.z;
    r.x[3] = f.w;
  } else {
    r.x[0] = *q;
  }
  return r;
}
template <int VW>
__device__ __forceinline__ void stv(float *q, const Vf<VW> &v) {
  if constexpr (VW == 4) *reinterpret_cast<float4 *>(q) = make_float4(v.x[0], v.x[1], v.x[2], v.x[3]);
  else *q = v.x[0];
}
template <int VW>
struct Vb {
  unsigned char x[VW];
};
template <int VW>
__device__ __forceinline__ Vb<VW> ldb(const unsigned char *q) {
  Vb<VW> r;
  if constexpr (VW == 4) {
    const uchar4 c = *reinterpret_cast<const uchar4 *>(q);
    r.x[0] = c.x;
    r.x[1] = c.y;
    r.x[2] = c.z;
    r.x[3] = c.w;
  } else {
    r.x[0] = *q;
  }
  return r;
}
template <int VW>
__device__ __forceinline__ void stb(unsigned char *q, const Vb<VW> &v) {
  if constexpr (VW == 4) *reinterpret_cast<uchar4 *>(q) = make_uchar4(v.x[0], v.x[1], v.x[2], v.x[3]);
  else *q = v.x[0];
}

// item i of a [Kp][M][T / VW] field (M lines or nodes): its row (k, m), its
// first step t0 and its offset in the [Kp][M][T] arrays
struct Item {
  int k, m, t0;
  size_t o;
};
template <int VW>
__device__ __forceinline__ Item item_of(unsigned i, int M, int T) {
  const unsigned TV = (unsigned)(T / VW), q = i / TV;
  Item r;
  r.t0 = (int)(i - q * TV) * VW;
  r.m = (int)(q % (unsigned)M);
  r.k = (int)(q / (unsigned)M);
  r.o = (size_t)i * VW;
  return r;
}

// node averages (Eq. average-op) of the terminal values of the new state nx,
// and the price updates u' = u + pbar', v' = v + theta' - theta_bar' (step
// 3) from the old state s
template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) fwd_avg(DP p, St s, St nx) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.N, p.T);
    const int n = it.m, k = it.k, t0 = it.t0;
    float sp[VW], st[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) sp[e] = st[e] = 0.f;
    for (int j = p.dptr[n]; j < p.dptr[n + 1]; ++j) {
      const Vf<VW> v = ldv<VW>(nx.PD + (size_t)p.didx[j] * p.T + t0);
#pragma unroll
      for (int e = 0; e < VW; ++e) sp[e] += v.x[e];
    }
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j];
      const size_t ol = li(p, k, c >> 1, t0);
      const Vf<VW> v = ldv<VW>(nx.P + ol), th = ldv<VW>(((c & 1) ? nx.TH2 : nx.TH1) + ol);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        sp[e] += (c & 1) ? v.x[e] : -v.x[e];
        st[e] += th.x[e];
      }
    }
    const Vf<VW> u = ldv<VW>(s.U + it.o);
    Vf<VW> pb, tbr, un;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      pb.x[e] = sp[e] / p.cnt[n];
      tbr.x[e] = p.cth[n] > 0.f ? st[e] / p.cth[n] : 0.f;
      un.x[e] = u.x[e] + pb.x[e];
    }
    stv<VW>(nx.PB + it.o, pb);
    stv<VW>(nx.TBR + it.o, tbr);
    stv<VW>(nx.U + it.o, un);
    // v' = v + theta' - theta_bar' of the node's line terminals (each
    // terminal belongs to one node, so every v entry is written once)
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j];
      const size_t ol = li(p, k, c >> 1, t0);
      float *V = (c & 1) ? nx.V2 : nx.V1;
      const Vf<VW> v = ldv<VW>(((c & 1) ? s.V2 : s.V1) + ol), th = ldv<VW>(((c & 1) ? nx.TH2 : nx.TH1) + ol);
      Vf<VW> w;
#pragma unroll
      for (int e = 0; e < VW; ++e) w.x[e] = v.x[e] + th.x[e] - tbr.x[e];
      stv<VW>(V + ol, w);
    }
  }
}

struct LineIn {
  float x1, x2, y1, y2;
};

__device__ __forceinline__ LineIn line_inputs(const DP &p, const St &s, int k, int l, int t) {
  const int a = p.n1[l], c = p.n2[l];
  const size_t o = li(p, k, l, t), o1 = ni(p, k, a, t), o2 = ni(p, k, c, t);
  LineIn r;
  r.x1 = -s.P[o] - s.PB[o1] - s.U[o1];        // p~ - u at terminal 1
  r.x2 = s.P[o] - s.PB[o2] - s.U[o2];
  r.y1 = s.TBR[o1] - s.V1[o];                  // theta_bar - v
  r.y2 = s.TBR[o2] - s.V2[o];
  return r;
}

// The prox inputs that decide a clip, each rounding written out, so that the
// reverse pass's recomputation (without a record) takes the forward's
// decisions whatever the compiler contracts elsewhere: the line prox's
// denominator 2 rho_p + rho_theta / (2 b^2) and unclipped flow (Section 4.2),
// a generator's and a curtailable load's unclipped power (Section 4.1)
__device__ __forceinline__ float line_den(const DP &p, float b, float tb) {
  return __fadd_rn(__fmul_rn(2.f, p.rp), p.rt / (tb * b));
}
__device__ __forceinline__ float line_z(const DP &p, const LineIn &in, float tb, float den) {
  return __fadd_rn(__fmul_rn(p.rp, in.x2 - in.x1), __fmul_rn(p.rt, in.y1 - in.y2) / tb) / den;
}
__device__ __forceinline__ float gen_den(const DP &p, int d) { return __fadd_rn(__fmul_rn(2.f, p.ga[d]), p.rd); }
__device__ __forceinline__ float gen_z(const DP &p, int d, float X) {
  return __fsub_rn(__fmul_rn(p.rd, X), p.gb[d]) / gen_den(p, d);
}
__device__ __forceinline__ float load_z(const DP &p, int e, float X) {
  return __fsub_rn(__fmul_rn(p.rd, X), p.voll[e]) / p.rd;
}

// where an unclipped value z lies against [lo, hi]: 0 inside, 1 above, 2
// below, 3 unordered (not a number); the reverse pass reads it from the
// forward's record
enum { CLIP_IN = 0, CLIP_HI = 1, CLIP_LO = 2, CLIP_NAN = 3 };
__device__ __forceinline__ unsigned char clip_code(float z, float lo, float hi) {
  return (z >= lo && z <= hi) ? CLIP_IN : z > hi ? CLIP_HI : z < lo ? CLIP_LO : CLIP_NAN;
}

// step 1: line prox (Section 4.2); outaged lines decouple.  lmask (optional):
// the iteration's record of where each line's unclipped flow lay
template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) fwd_line(DP p, St s, St nx, unsigned char *lmask) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.L, p.T);
    const int l = it.m, k = it.k;
    const size_t o = it.o, o1 = ni(p, k, p.n1[l], it.t0), o2 = ni(p, k, p.n2[l], it.t0);
    const Vf<VW> P = ldv<VW>(s.P + o), PB1 = ldv<VW>(s.PB + o1), U1 = ldv<VW>(s.U + o1);
    const Vf<VW> PB2 = ldv<VW>(s.PB + o2), U2 = ldv<VW>(s.U + o2), TB1 = ldv<VW>(s.TBR + o1);
    const Vf<VW> TB2 = ldv<VW>(s.TBR + o2), V1 = ldv<VW>(s.V1 + o), V2 = ldv<VW>(s.V2 + o);
    Vf<VW> np, t1, t2;
    if (p.out[k] != l) {
      const float b = p.b[l], tb = 2.f * b, u = p.lu[l], den = line_den(p, b, tb);
      Vb<VW> code;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        // the prox inputs as line_inputs forms them
        const LineIn in{-P.x[e] - PB1.x[e] - U1.x[e], P.x[e] - PB2.x[e] - U2.x[e], TB1.x[e] - V1.x[e],
                        TB2.x[e] - V2.x[e]};
        const float z = line_z(p, in, tb, den);
        code.x[e] = clip_code(z, -u, u);
        const float p2 = fminf(fmaxf(z, -u), u);
        const float mid = 0.5f * (in.y1 + in.y2);
        np.x[e] = p2;
        t1.x[e] = mid + p2 / tb;
        t2.x[e] = mid - p2 / tb;
      }
      if (lmask) stb<VW>(lmask + o, code);
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        np.x[e] = 0.f;
        t1.x[e] = TB1.x[e] - V1.x[e];
        t2.x[e] = TB2.x[e] - V2.x[e];
      }
    }
    stv<VW>(nx.P + o, np);
    stv<VW>(nx.TH1 + o, t1);
    stv<VW>(nx.TH2 + o, t2);
  }
}

// a device's prox input X = p_d - avg_k(pbar + u) (every lane of the group)
__device__ __forceinline__ float dev_x(const DP &p, const St &s, int d, int t) {
  return s.PD[(size_t)d * p.T + t] - ksum(p, s.PB, s.U, p.dnode[d], t) / (float)p.Kp;
}

// the HVDC partner of terminal d (its index), or -1
__device__ __forceinline__ int hvdc_partner(const DP &p, int d) {
  if (p.kind[d] != 2) return -1;
  const int e = d - (p.G + p.D + p.B);
  return (e & 1) ? d - 1 : d + 1;
}

// step 2: devices shared by all contingencies, weight (K+1) rho_p; the
// inner-ADMM devices only record their input X here.  An HVDC terminal
// evaluates its link's prox p2 = clip((x2 - x1)/2, -u, u), p1 = -p2.
// dmask (optional): the iteration's record of where each closed-form
// device's unclipped power lay
__global__ void __launch_bounds__(TB, 8) fwd_dev(DP p, St s, St nx, float *XD, unsigned char *dmask) {
  GROUP_STRIDE(i, (long long)p.S * p.T) {
    const int d = (int)(i / (unsigned)p.T), t = (int)(i - (unsigned)d * (unsigned)p.T), d2 = hvdc_partner(p, d);
    const float X = dev_x(p, s, d, t), Xo = d2 < 0 ? 0.f : dev_x(p, s, d2, t);
    if (threadIdx.x & (KL - 1)) continue;   // the group's first lane writes
    if (p.kind[d] == 1) {
      XD[i] = X;
      continue;
    }
    if (p.kind[d] == 2) {
      const int e = d - (p.G + p.D + p.B), h = e >> 1;
      const float x1 = (e & 1) ? Xo : X, x2 = (e & 1) ? X : Xo;
      const float z = 0.5f * (x2 - x1), u = p.hvdc_u[h];
      if (dmask) dmask[i] = clip_code(z, -u, u);
      const float f = fminf(fmaxf(z, -u), u);
      nx.PD[i] = (e & 1) ? f : -f;
      continue;
    }
    float r;
    if (d < p.G) {
      const float z = gen_z(p, d, X);
      if (dmask) dmask[i] = clip_code(z, p.gpmin[i], p.gpmax[i]);
      r = fminf(fmaxf(z, p.gpmin[i]), p.gpmax[i]);
    } else {
      const int e = d - p.G;
      const size_t o = (size_t)e * p.T + t;
      if (p.voll[e] < 0.f) {
        r = -p.load_p[o];
      } else {
        const float z = load_z(p, e, X);
        if (dmask) dmask[i] = clip_code(z, -p.load_p[o], 0.f);
        r = fminf(fmaxf(z, -p.load_p[o]), 0.f);
      }
    }
    nx.PD[i] = r;
  }
}

// One device's inner problem as the kernels read it: constraint rows in CSR
// (row pointers relative to the shape's nonzeros) and CSC form, the inverse
// system matrix, right-hand sides and linear cost.  stage_view copies them
// into shared memory, where the ten inner iterations re-read them, instead of
// chasing the same global pointers every iteration.
struct View {
  int n, m;
  const int *arp, *aci, *atp, *ati;
  const float *acv, *atv, *Mi, *h, *q;
  const unsigned char *eq;
};

// What the kernels copy into shared memory: 0 nothing (long horizons), 1 the
// constraint structure, right-hand sides and cost, 2 also the inverse.
// view_words: the 4-byte words that takes.
__host__ __device__ inline size_t view_words(int n, int m, int nnz, int level) {
  if (level <= 0) return 0;
  return (size_t)(m + 1) + (n + 1) + 2 * (size_t)nnz     // arp, atp, aci, ati
         + 2 * (size_t)nnz + m + n                         // acv, atv, h, q
         + ((size_t)m + 3) / 4                             // eq bytes
         + (level >= 2 ? (size_t)n * n : 0);
}

__device__ View stage_view(const DP &p, const Shape &sh, const IDev &di, float *sm, int level) {
  const int n = sh.n, m = sh.m, nnz = sh.nnz, tid = threadIdx.x, nt = blockDim.x;
  if (level <= 0) {
    View g;
    g.n = n;
    g.m = m;
    g.arp = p.arp + sh.rp;
    g.atp = p.atp + sh.tp;
    g.aci = p.aci + sh.ci;
    g.acv = p.acv + sh.ci;
    g.ati = p.ati + sh.ti;
    g.atv = p.atv + sh.ti;
    g.h = p.RH + di.h;
    g.q = p.Q + di.q;
    g.eq = p.aeq + sh.eq;
    g.Mi = p.minv + di.minv;
    return g;
  }
  const bool with_minv = level >= 2;
  int *arp = reinterpret_cast<int *>(sm), *atp = arp + m + 1, *aci = atp + n + 1, *ati = aci + nnz;
  float *acv = reinterpret_cast<float *>(ati + nnz), *atv = acv + nnz, *h = atv + nnz, *q = h + m;
  unsigned char *eq = reinterpret_cast<unsigned char *>(q + n);
  float *Mi = q + n + (m + 3) / 4;
  for (int i = tid; i <= m; i += nt) arp[i] = p.arp[sh.rp + i];
  for (int i = tid; i <= n; i += nt) atp[i] = p.atp[sh.tp + i];
  for (int i = tid; i < nnz; i += nt) {
    aci[i] = p.aci[sh.ci + i];
    acv[i] = p.acv[sh.ci + i];
    ati[i] = p.ati[sh.ti + i];
    atv[i] = p.atv[sh.ti + i];
  }
  for (int i = tid; i < m; i += nt) {
    h[i] = p.RH[di.h + i];
    eq[i] = p.aeq[sh.eq + i];
  }
  for (int i = tid; i < n; i += nt) q[i] = p.Q[di.q + i];
  const float *mg = p.minv + di.minv;
  if (with_minv)
    for (int i = tid; i < n * n; i += nt) Mi[i] = mg[i];
  __syncthreads();
  View v;
  v.n = n;
  v.m = m;
  v.arp = arp;
  v.atp = atp;
  v.aci = aci;
  v.ati = ati;
  v.acv = acv;
  v.atv = atv;
  v.h = h;
  v.q = q;
  v.eq = eq;
  v.Mi = with_minv ? Mi : mg;
  return v;
}

// N_INNER iterations of the Appendix D ADMM for the device of this CTA:
//   z = M^-1 (rho' E_p' x - q + omega A'(h + beta - lambda)),
//   alpha = A z - h, beta = min(alpha + lambda, 0) (0 on equality rows),
//   lambda = alpha + lambda - beta;
// mask (optional) records the rows where beta took alpha + lambda
__device__ void inner_forward(const DP &p, const View &v, const float *x, float *beta, float *lam,
                              float *w, float *r, float *z, unsigned char *mask) {
  const int n = v.n, m = v.m, T = p.T;
  const float rho = p.rd, om = p.rd;
  for (int it = 0; it < N_INNER; ++it) {
    for (int row = threadIdx.x; row < m; row += blockDim.x) w[row] = v.h[row] + beta[row] - lam[row];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      float acc = 0.f;
      for (int e = v.atp[j]; e < v.atp[j + 1]; ++e) acc += v.atv[e] * w[v.ati[e]];
      r[j] = -v.q[j] + om * acc + (j < T ? rho * x[j] : 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {     // M^-1 is symmetric: read its columns coalesced
      float acc = 0.f;
      for (int j = 0; j < n; ++j) acc += v.Mi[(size_t)j * n + i] * r[j];
      z[i] = acc;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < m; row += blockDim.x) {
      float al = -v.h[row];
      for (int e = v.arp[row]; e < v.arp[row + 1]; ++e) al += v.acv[e] * z[v.aci[e]];
      const float s = al + lam[row];
      const bool eq = v.eq[row] != 0;
      const float bt = eq ? 0.f : fminf(s, 0.f);
      if (mask) mask[it * m + row] = (!eq && s <= 0.f);
      beta[row] = bt;
      lam[row] = s - bt;
    }
    __syncthreads();
  }
}

// step 2 for the inner-ADMM devices: one CTA per device
// gmask: when not NULL, the iteration's record of which rows clipped
// (device blocks of N_INNER x m bytes at N_INNER x its first row)
__global__ void __launch_bounds__(TBI) fwd_inner(DP p, St s, St nx, const float *XD, float *DEL, int level,
                                                 unsigned char *gmask) {
  extern __shared__ float sm[];
  const IDev di = p.idev[blockIdx.x];
  const Shape sh = p.shape[di.shape];
  const int n = sh.n, m = sh.m, T = p.T;
  float *x = sm, *r = x + T, *z = r + n, *w = z + n, *beta = w + m, *lam = beta + m;
  const View v = stage_view(p, sh, di, lam + m, level);
  for (int t = threadIdx.x; t < T; t += blockDim.x) x[t] = XD[(size_t)di.dev * T + t];
  for (int row = threadIdx.x; row < m; row += blockDim.x) {
    beta[row] = s.INS[di.h + row];
    lam[row] = s.INS[p.Mtot + di.h + row];
  }
  __syncthreads();
  inner_forward(p, v, x, beta, lam, w, r, z, gmask ? gmask + (size_t)N_INNER * di.h : nullptr);
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    nx.PD[(size_t)di.dev * T + t] = z[t];
    if (di.bat >= 0) DEL[(size_t)di.bat * T + t] = z[2 * T + t];   // discharge, for the cost
  }
  for (int row = threadIdx.x; row < m; row += blockDim.x) {
    nx.INS[di.h + row] = beta[row];
    nx.INS[p.Mtot + di.h + row] = lam[row];
  }
}

// ---------------------------------------------------------------------------
// reverse pass of one iteration: the adjoint of state i in `a` becomes the
// adjoint of state i-1; s is state i-1
// ---------------------------------------------------------------------------

// The reverse pass of iteration i runs in two halves.  The first: the
// adjoints of the new node averages, the line prox and the device proxes
// transposed (bwd_node1, bwd_line1, bwd_dev), then the inner ADMM.  The
// second: gathers at the nodes (bwd_node2, on a second stream beside the
// inner ADMM, which it does not touch, complete at the nodes without an
// inner-ADMM device; bwd_node3 after it for the others) and their scatter back to the line and device
// values (bwd_scatter, one launch for both).  bwd_node2 and bwd_scatter also
// run iteration i-1's first-half step on the same item when `nxt` is set, so
// a reverse iteration takes four launches instead of seven; the arithmetic is
// the same device functions either way, so the results are the same bit for
// bit.  The adjoint of the new pbar' through u' = u + pbar' is u's adjoint
// itself: the kernels read it from a.LU (as `A`) before bwd_node2 (or
// bwd_node3, at the nodes with an inner-ADMM device) adds the increment.

// B = d/d theta_bar' through v' = v + theta' - theta_bar' at node item
// (k, n, t0 ..): minus the v adjoints of the node's line terminals
template <int VW>
__device__ __forceinline__ Vf<VW> node_b(const DP &p, const Adj &a, int k, int n, int t0) {
  Vf<VW> s;
#pragma unroll
  for (int e = 0; e < VW; ++e) s.x[e] = 0.f;
  for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
    const int c = p.lcode[j];
    const Vf<VW> v = ldv<VW>(((c & 1) ? a.LV2 : a.LV1) + li(p, k, c >> 1, t0));
#pragma unroll
    for (int e = 0; e < VW; ++e) s.x[e] += v.x[e];
  }
#pragma unroll
  for (int e = 0; e < VW; ++e) s.x[e] = -s.x[e];
  return s;
}

template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) bwd_node1(DP p, Adj a, float *B) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.N, p.T);
    stv<VW>(B + it.o, node_b<VW>(p, a, it.k, it.m, it.t0));
  }
}

// the line prox backwards at item `it` (line it.m, contingency it.k, steps
// it.t0 ..), given the adjoints of the step's outputs p, theta_1, theta_2
// (lp0, lt10, lt20) and A at the two ends (A1, A2); X2, Y1, Y2 receive
// d/d(x2, y1, y2) for the node gathers (d/d x1 = -d/d x2).  lmask
// (optional): the forward's record of the iteration's line clips, else the
// unclipped flow is recomputed from the step's input state s
template <int VW>
__device__ __forceinline__ void line_back(const DP &p, const St &s, const Adj &a, const Vf<VW> &A1,
                                          const Vf<VW> &A2, const float *B, float *X2, float *Y1, float *Y2,
                                          float *GU, const unsigned char *lmask, const Item &it, const Vf<VW> &lp0,
                                          const Vf<VW> &lt10, const Vf<VW> &lt20) {
  const int l = it.m, k = it.k, n1 = p.n1[l], n2 = p.n2[l];
  const size_t o = it.o, o1 = ni(p, k, n1, it.t0), o2 = ni(p, k, n2, it.t0);
  const float ic1 = p.icnt[n1], ic2 = p.icnt[n2], ih1 = p.icth[n1], ih2 = p.icth[n2];
  const Vf<VW> B1 = ldv<VW>(B + o1), B2 = ldv<VW>(B + o2), LV1 = ldv<VW>(a.LV1 + o), LV2 = ldv<VW>(a.LV2 + o);
  const bool act = p.out[k] != l;
  Vb<VW> code;
  if (act && lmask) code = ldb<VW>(lmask + o);
  Vf<VW> x2, y1, y2, lpn, v1, v2;
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    const float lp = fmaf(A2.x[e], ic2, fmaf(-A1.x[e], ic1, lp0.x[e]));
    const float lt1 = fmaf(B1.x[e], ih1, __fadd_rn(lt10.x[e], LV1.x[e]));
    const float lt2 = fmaf(B2.x[e], ih2, __fadd_rn(lt20.x[e], LV2.x[e]));
    float lx1 = 0.f, lx2 = 0.f, ly1, ly2;
    if (act) {
      const float b = p.b[l], tb = 2.f * b, u = p.lu[l];
      const unsigned char cd =
          lmask ? code.x[e] : clip_code(line_z(p, line_inputs(p, s, k, l, it.t0 + e), tb, line_den(p, b, tb)), -u, u);
      const float lpt = fmaf(lt1 - lt2, p.lfac[l], lp);     // theta_{1,2} = mid +- p / (2b)
      const float half = __fmul_rn(0.5f, lt1 + lt2);
      ly1 = ly2 = half;
      if (cd == CLIP_IN) {
        lx2 = __fmul_rn(lpt, p.lfac[p.L + l]);
        lx1 = -lx2;
        const float w = __fmul_rn(lpt, p.lfac[2 * p.L + l]);
        ly1 = __fadd_rn(half, w);
        ly2 = __fsub_rn(half, w);
      } else {
        GU[o + e] += cd == CLIP_HI ? lpt : -lpt;
      }
    } else {
      ly1 = lt1;
      ly2 = lt2;
    }
    x2.x[e] = lx2;
    y1.x[e] = ly1;
    y2.x[e] = ly2;
    lpn.x[e] = lx2 - lx1;                // x1 = -p - ..., x2 = p - ...
    v1.x[e] = LV1.x[e] - ly1;            // v enters y = theta_bar - v, and v' = v + ...
    v2.x[e] = LV2.x[e] - ly2;
  }
  stv<VW>(X2 + o, x2);
  stv<VW>(Y1 + o, y1);
  stv<VW>(Y2 + o, y2);
  stv<VW>(a.LP + o, lpn);
  stv<VW>(a.LV1 + o, v1);
  stv<VW>(a.LV2 + o, v2);
}

template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) bwd_line1(DP p, St s, Adj a, const float *A, const float *B, float *X2,
                                                   float *Y1, float *Y2, float *GU, const unsigned char *lmask) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.L, p.T);
    const size_t o1 = ni(p, it.k, p.n1[it.m], it.t0), o2 = ni(p, it.k, p.n2[it.m], it.t0);
    line_back<VW>(p, s, a, ldv<VW>(A + o1), ldv<VW>(A + o2), B, X2, Y1, Y2, GU, lmask, it, ldv<VW>(a.LP + it.o),
                  ldv<VW>(a.LT1 + it.o), ldv<VW>(a.LT2 + it.o));
  }
}


// the closed-form device proxes backwards at item i = (d, t), given the
// adjoint of the device's new power (lpd) and, for an HVDC terminal, its
// partner's (lpd_o); LX = d/dX per device.  An inner-ADMM device records
// the adjoint of its output for bwd_inner (and, without a record, X).
// dmask (optional): the forward's record of the iteration's device clips
// (the inner-ADMM devices then need no X either: their clipped rows are
// recorded too); else the caller passes X (and the HVDC partner's, Xo)
// recomputed from the step's input state.  One lane per device step.
__device__ __forceinline__ void dev_back(const DP &p, float *LX, float *GL, float *GP, float *XD, float *LPDT,
                                         const unsigned char *dmask, unsigned i, int d, int t, float lpd, float lpd_o,
                                         float X, float Xo) {
  if (p.kind[d] == 1) {
    if (!dmask) XD[i] = X;
    LPDT[i] = lpd;
    return;
  }
  if (p.kind[d] == 2) {                  // HVDC: both terminals' adjoints meet in d/d p2
    const int e = d - (p.G + p.D + p.B), h = e >> 1;
    const float l1 = (e & 1) ? lpd_o : lpd, l2 = (e & 1) ? lpd : lpd_o;
    const float u = p.hvdc_u[h];
    unsigned char code;
    if (dmask) {
      code = dmask[i];
    } else {
      const float x1 = (e & 1) ? Xo : X, x2 = (e & 1) ? X : Xo;
      code = clip_code(0.5f * (x2 - x1), -u, u);
    }
    const float lz = code == CLIP_IN ? 0.5f * (l2 - l1) : 0.f;
    LX[i] = (e & 1) ? lz : -lz;
    return;
  }
  float lx = 0.f;
  if (d < p.G) {
    const unsigned char code = dmask ? dmask[i] : clip_code(gen_z(p, d, X), p.gpmin[i], p.gpmax[i]);
    if (code == CLIP_IN) lx = lpd * p.rd / gen_den(p, d);
    else if (code == CLIP_HI) GP[i] += lpd;
  } else {
    const int e = d - p.G;
    const size_t o = (size_t)e * p.T + t;
    if (p.voll[e] < 0.f) {
      GL[o] -= lpd;                      // p = -P
    } else {
      const unsigned char code = dmask ? dmask[i] : clip_code(load_z(p, e, X), -p.load_p[o], 0.f);
      if (code == CLIP_IN) lx = lpd;
      else if (code == CLIP_LO) GL[o] -= lpd;
    }
  }
  LX[i] = lx;
}

// The reverse device kernels on VW steps per lane group: ksum and dev_x for
// steps t0 .. t0 + VW - 1, each step summed in the same order as the
// one-step forms (so the results are the same step by step), and
// add_node_kv: lpd + the sum over contingencies of V at device d's node
// divided by the node's terminal count (the k-average's adjoint)
template <int VW>
__device__ __forceinline__ Vf<VW> ksumv(const DP &p, const float *V, const float *W, int n, int t0) {
  const int j = threadIdx.x & (KL - 1);
  Vf<VW> s;
#pragma unroll
  for (int e = 0; e < VW; ++e) s.x[e] = 0.f;
#pragma unroll 3
  for (int k = j; k < p.Kp; k += KL) {
    const Vf<VW> v = ldv<VW>(V + ni(p, k, n, t0));
    if (W) {
      const Vf<VW> w = ldv<VW>(W + ni(p, k, n, t0));
#pragma unroll
      for (int e = 0; e < VW; ++e) s.x[e] += v.x[e] + w.x[e];
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) s.x[e] += v.x[e];
    }
  }
  const unsigned gm = group_mask();
#pragma unroll
  for (int o = KL / 2; o > 0; o >>= 1)
#pragma unroll
    for (int e = 0; e < VW; ++e) s.x[e] += __shfl_xor_sync(gm, s.x[e], o);
  return s;
}
template <int VW>
__device__ __forceinline__ Vf<VW> dev_xv(const DP &p, const St &s, int d, int t0) {
  const Vf<VW> pd = ldv<VW>(s.PD + (size_t)d * p.T + t0), k = ksumv<VW>(p, s.PB, s.U, p.dnode[d], t0);
  Vf<VW> r;
#pragma unroll
  for (int e = 0; e < VW; ++e) r.x[e] = pd.x[e] - k.x[e] / (float)p.Kp;
  return r;
}
template <int VW>
__device__ __forceinline__ Vf<VW> add_node_kv(const DP &p, const float *V, int d, int t0, const Vf<VW> &lpd) {
  const int n = p.dnode[d];
  const Vf<VW> k = ksumv<VW>(p, V, nullptr, n, t0);
  Vf<VW> r;
#pragma unroll
  for (int e = 0; e < VW; ++e) r.x[e] = fmaf(k.x[e], p.icnt[n], lpd.x[e]);
  return r;
}

// device item i of a [S][T / VW] field: device d, first step t0, offset
// d T + t0 = i VW
template <int VW>
__device__ __forceinline__ void dev_item(unsigned i, int T, int &d, int &t0) {
  const unsigned TV = (unsigned)(T / VW);
  d = (int)(i / TV);
  t0 = (int)(i - (unsigned)d * TV) * VW;
}

template <int VW>
__global__ void bwd_dev(DP p, St s, Adj a, const float *A, float *LX, float *GL, float *GP, float *XD, float *LPDT,
                        const unsigned char *dmask) {
  GROUP_STRIDE(i, (long long)p.S * (p.T / VW)) {
    int d, t0;
    dev_item<VW>(i, p.T, d, t0);
    const int d2 = hvdc_partner(p, d);
    const size_t o = (size_t)i * VW, o2 = (size_t)d2 * p.T + t0;
    const Vf<VW> lpd = add_node_kv<VW>(p, A, d, t0, ldv<VW>(a.LPD + o));
    Vf<VW> lpd_o{}, X{}, Xo{};
    if (d2 >= 0) lpd_o = add_node_kv<VW>(p, A, d2, t0, ldv<VW>(a.LPD + o2));
    if (!dmask) X = dev_xv<VW>(p, s, d, t0);
    if (!dmask && d2 >= 0) Xo = dev_xv<VW>(p, s, d2, t0);
    if (!(threadIdx.x & (KL - 1)))
#pragma unroll
      for (int e = 0; e < VW; ++e)
        dev_back(p, LX, GL, GP, XD, LPDT, dmask, (unsigned)(o + e), d, t0 + e, lpd.x[e], lpd_o.x[e], X.x[e], Xo.x[e]);
  }
}

// the inner ADMM backwards, one CTA per device: which rows clipped in each
// of the N_INNER iterations comes from the forward pass's record (gmask) or,
// without one, from recomputing the iterations from state i-1; then walk
// them in reverse.  Per iteration, with s = alpha + lambda:
//   d s = d lambda' + [clipped] (d beta' - d lambda'),
//   d z = A' d s (+ the output's adjoint on the last iteration), d h -= d s,
//   d r = M^-1 d z, d x += rho' (d r)_p, w = omega A d r:
//   d h += w, d beta = w, d lambda = d s - w.
// `last`: the iteration whose battery discharge enters the cost.
__global__ void __launch_bounds__(TBI) bwd_inner(DP p, St s, Adj a, const float *XD, const float *LPDT, float *LX,
                                                 float *HB, int last, int level, const unsigned char *gmask) {
  extern __shared__ float sm[];
  const IDev di = p.idev[blockIdx.x];
  const Shape sh = p.shape[di.shape];
  const int n = sh.n, m = sh.m, T = p.T;
  const float rho = p.rd, om = p.rd;
  float *x = sm, *r = x + T, *z = r + n, *w = z + n, *beta = w + m, *lam = beta + m;
  float *zt = lam + m, *rb = zt + n, *sb = rb + n, *bb = sb + m, *lb = bb + m, *hb = lb + m, *xb = hb + m;
  const View v = stage_view(p, sh, di, xb + T, level);
  const unsigned char *mask = reinterpret_cast<unsigned char *>(xb + T + view_words(n, m, sh.nnz, level));
  for (int t = threadIdx.x; t < T; t += blockDim.x) xb[t] = 0.f;
  if (gmask) {
    // recorded by the forward pass
    mask = gmask + (size_t)N_INNER * di.h;
  } else {
    unsigned char *msh = reinterpret_cast<unsigned char *>(xb + T + view_words(n, m, sh.nnz, level));
    for (int t = threadIdx.x; t < T; t += blockDim.x) x[t] = XD[(size_t)di.dev * T + t];
    for (int row = threadIdx.x; row < m; row += blockDim.x) {
      beta[row] = s.INS[di.h + row];
      lam[row] = s.INS[p.Mtot + di.h + row];
    }
    __syncthreads();
    inner_forward(p, v, x, beta, lam, w, r, z, msh);
  }
  for (int row = threadIdx.x; row < m; row += blockDim.x) {
    bb[row] = a.LINS[di.h + row];
    lb[row] = a.LINS[p.Mtot + di.h + row];
    hb[row] = 0.f;
  }
  __syncthreads();
  const float *Mi = v.Mi;
  const float dcost = (last && di.bat >= 0) ? p.scost[di.bat] : 0.f;
  for (int it = N_INNER - 1; it >= 0; --it) {
    for (int row = threadIdx.x; row < m; row += blockDim.x) {
      const float sv = lb[row] + (mask[it * m + row] ? bb[row] - lb[row] : 0.f);
      sb[row] = sv;
      hb[row] -= sv;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      float acc = 0.f;
      for (int e = v.atp[j]; e < v.atp[j + 1]; ++e) acc += v.atv[e] * sb[v.ati[e]];
      if (it == N_INNER - 1) {           // the output: p = z_p, and the discharge z_delta in the cost
        if (j < T) acc += LPDT[(size_t)di.dev * T + j];
        else if (j >= 2 * T && j < 3 * T) acc += dcost;
      }
      zt[j] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float acc = 0.f;
      for (int j = 0; j < n; ++j) acc += Mi[(size_t)j * n + i] * zt[j];
      rb[i] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) xb[t] += rho * rb[t];
    for (int row = threadIdx.x; row < m; row += blockDim.x) {
      float acc = 0.f;
      for (int e = v.arp[row]; e < v.arp[row + 1]; ++e) acc += v.acv[e] * rb[v.aci[e]];
      const float wv = om * acc;
      hb[row] += wv;
      bb[row] = wv;
      lb[row] = sb[row] - wv;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < T; t += blockDim.x) LX[(size_t)di.dev * T + t] = xb[t];
  for (int row = threadIdx.x; row < m; row += blockDim.x) {
    a.LINS[di.h + row] = bb[row];
    a.LINS[p.Mtot + di.h + row] = lb[row];
    HB[di.h + row] += hb[row];
  }
}

// ---------------------------------------------------------------------------
// The inner ADMM from registers (horizons up to DREG_T steps), one warp per
// device: lane l holds elements l C .. l C + C - 1 of each vector (steps t of
// p, c and delta, states of charge s_t), and the solves of M z = r use the
// structure of M = diag(qd) + omega A'A instead of its inverse: a ramp
// generator's M is tridiagonal; a battery's reduces, after eliminating p and
// then (c, delta) step by step (2 x 2 blocks H), to a tridiagonal system in
// s.  The same solve serves the forward iterations and the reverse pass (M is
// symmetric).  Every operation is written with its rounding, so the forward
// pass and a recomputation in the reverse pass repeat each other bit for bit.
// ---------------------------------------------------------------------------
constexpr int DREG_T = 127;
constexpr unsigned FULLM = 0xffffffffu;
constexpr int RWARPS = TB / 32;   // devices per CTA of the register kernels

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// x := M^-1 x for a tridiagonal M with pivots q and a = -off / q (element i
// = lane C + j, valid while i < n): first-order recurrences composed over
// each lane's chunk, then across the warp by shuffle scans
template <int C>
__device__ __forceinline__ void tri_solve_r(const float (&q)[C], const float (&a)[C], float (&x)[C], int n,
                                            int lane) {
  const int i0 = lane * C;
  float r[C];
  float Ac = 1.f, Bc = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    r[j] = 0.f;
    if (i0 + j < n) {
      r[j] = rdiv(x[j], q[j]);
      const float Ai = (i0 + j == 0) ? 0.f : a[j];
      Bc = rfma(Ai, Bc, r[j]);
      Ac = rmul(Ai, Ac);
    }
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_up_sync(FULLM, Ac, d), Bp = __shfl_up_sync(FULLM, Bc, d);
    if (lane >= d) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float prev = __shfl_up_sync(FULLM, Bc, 1);
  if (lane == 0) prev = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (i0 + j < n) {
      const float Ai = (i0 + j == 0) ? 0.f : a[j];
      prev = rfma(Ai, prev, r[j]);
      x[j] = prev;
    }
  }
  Ac = 1.f;
  Bc = 0.f;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    if (i0 + j < n) {
      const float Ci = (i0 + j == n - 1) ? 0.f : a[j];
      Bc = rfma(Ci, Bc, x[j]);
      Ac = rmul(Ci, Ac);
    }
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Ap = __shfl_down_sync(FULLM, Ac, d), Bp = __shfl_down_sync(FULLM, Bc, d);
    if (lane + d < 32) {
      Bc = rfma(Ac, Bp, Bc);
      Ac = rmul(Ac, Ap);
    }
  }
  float nxt = __shfl_down_sync(FULLM, Bc, 1);
  if (lane == 31) nxt = 0.f;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    if (i0 + j < n) {
      const float Ci = (i0 + j == n - 1) ? 0.f : a[j];
      nxt = rfma(Ci, nxt, x[j]);
      x[j] = nxt;
    }
  }
}

// The register path records which rows clipped as one 64-bit word per lane
// and inner iteration (bit g C + j: row group g, element j of the lane's
// chunk), [device][inner iteration][lane]: coalesced stores and loads.
constexpr size_t RREC_WORDS = (size_t)N_INNER * 32;   // words per device and outer iteration

// bytes of one outer iteration's record of the inner ADMM: the register
// path's words, or the shared-memory path's byte per row and inner iteration
// (a multiple of 16 bytes: the line record that follows it is read 4 bytes
// at a time)
__host__ __device__ inline size_t inner_record_bytes(const DP &p) {
  const size_t b = p.reg_c ? (size_t)p.n_inner * RREC_WORDS * sizeof(unsigned long long) : (size_t)N_INNER * p.Mtot;
  return (b + 15) & ~size_t(15);
}

// one inequality row of the inner ADMM: s = alpha + lambda, beta = min(s, 0),
// lambda = s - beta; bit b of the record says whether beta took s
__device__ __forceinline__ void ineq_r(float al, float &lam, float &bet, unsigned long long &bits, int b) {
  const float sv = radd(al, lam);
  const float bt = fminf(sv, 0.f);
  if (sv <= 0.f) bits |= 1ull << b;
  bet = bt;
  lam = rsub(sv, bt);
}

// the adjoint of that row: d s = d lambda' + [clipped] (d beta' - d lambda')
__device__ __forceinline__ float sbar_r(unsigned long long bits, int b, float bb, float lb) {
  return ((bits >> b) & 1ull) ? radd(lb, rsub(bb, lb)) : lb;
}

// A battery's constants: omega eta, H^-1 and g = H^-1 f with f = (-omega eta,
// omega) the coupling of (c_t, delta_t) to s_{t+1} - s_t
struct StorK {
  float rho, om, eta, rpo, i00, i01, i11, gc, gd;
};

// z := M^-1 z for a battery, z = (p, c, delta) at steps t < T, s at j <= T
// (element e = lane C + j holds step e and state of charge e)
template <int C>
__device__ __forceinline__ void stor_solve_r(const StorK &k, const float (&qv)[C], const float (&av)[C],
                                             float (&zp)[C], float (&zc)[C], float (&zd)[C], float (&zs)[C], int T,
                                             int lane) {
  const int t0 = lane * C;
  const float fc = -rmul(k.om, k.eta), fd = k.om;
  float u[C], yc[C], yd[C], fy[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    u[j] = yc[j] = yd[j] = fy[j] = 0.f;
    if (t0 + j < T) {
      u[j] = rdiv(zp[j], k.rpo);                          // p = u - omega (c - delta) / (rho + omega)
      const float rc = rsub(zc[j], rmul(k.om, u[j])), rd = radd(zd[j], rmul(k.om, u[j]));
      yc[j] = rfma(k.i00, rc, rmul(k.i01, rd));             // y = H^-1 r'
      yd[j] = rfma(k.i01, rc, rmul(k.i11, rd));
      fy[j] = rfma(fc, yc[j], rmul(fd, yd[j]));
    }
  }
  const float fyp = __shfl_up_sync(FULLM, fy[C - 1], 1);
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int e = t0 + j;
    if (e <= T) {
      float r = zs[j];
      if (e <= T - 1) r = radd(r, fy[j]);
      if (e >= 1) r = rsub(r, (j == 0) ? fyp : fy[j - 1]);
      zs[j] = r;
    }
  }
  tri_solve_r<C>(qv, av, zs, T + 1, lane);
  const float sn = __shfl_down_sync(FULLM, zs[0], 1);
#pragma unroll
  for (int j = 0; j < C; ++j) {
    if (t0 + j < T) {
      const float dsv = rsub((j == C - 1) ? sn : zs[j + 1], zs[j]);
      const float c = rsub(yc[j], rmul(k.gc, dsv)), dl = rsub(yd[j], rmul(k.gd, dsv));
      zc[j] = c;
      zd[j] = dl;
      zp[j] = rsub(u[j], rdiv(rmul(k.om, rsub(c, dl)), k.rpo));
    }
  }
}

// N_INNER forward iterations of a ramp generator from registers.  Rows (offset
// in the device's block): UP p_t <= pmax_t (t), LO -p_t <= -pmin_t (T + t),
// RU p_{t+1} - p_t <= R (2T + t), RD p_t - p_{t+1} <= R (3T - 1 + t).  mask:
// the device's record block (N_INNER x m bytes) or NULL
template <int C>
__device__ void ramp_fwd_r(int T, int lane, float rho, float om, float qlin, const float (&x)[C],
                           const float (&qv)[C], const float (&av)[C], const float (&hU)[C], const float (&hL)[C],
                           const float (&hRU)[C], const float (&hRD)[C], float (&bU)[C], float (&lU)[C],
                           float (&bL)[C], float (&lL)[C], float (&bRU)[C], float (&lRU)[C], float (&bRD)[C],
                           float (&lRD)[C], float (&z)[C], unsigned long long *rec) {
  const int t0 = lane * C;
  for (int it = 0; it < N_INNER; ++it) {
    unsigned long long bits = 0;
    float wRU[C], wRD[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      wRU[j] = rsub(radd(hRU[j], bRU[j]), lRU[j]);
      wRD[j] = rsub(radd(hRD[j], bRD[j]), lRD[j]);
    }
    const float pRU = __shfl_up_sync(FULLM, wRU[C - 1], 1), pRD = __shfl_up_sync(FULLM, wRD[C - 1], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      z[j] = 0.f;
      if (t < T) {
        float acc = rsub(rsub(radd(hU[j], bU[j]), lU[j]), rsub(radd(hL[j], bL[j]), lL[j]));   // A'w, w = h + beta - lambda
        if (t >= 1) acc = radd(acc, rsub(j ? wRU[j - 1] : pRU, j ? wRD[j - 1] : pRD));
        if (t <= T - 2) acc = rsub(acc, rsub(wRU[j], wRD[j]));
        z[j] = rfma(rho, x[j], rfma(om, acc, -qlin));                                           // r
      }
    }
    tri_solve_r<C>(qv, av, z, T, lane);
    const float zn = __shfl_down_sync(FULLM, z[0], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      if (t < T) {
        ineq_r(rsub(z[j], hU[j]), lU[j], bU[j], bits, j);
        ineq_r(rsub(-z[j], hL[j]), lL[j], bL[j], bits, C + j);
        if (t < T - 1) {
          const float znx = (j == C - 1) ? zn : z[j + 1];
          ineq_r(rsub(rsub(znx, z[j]), hRU[j]), lRU[j], bRU[j], bits, 2 * C + j);
          ineq_r(rsub(rsub(z[j], znx), hRD[j]), lRD[j], bRD[j], bits, 3 * C + j);
        }
      }
    }
    if (rec) rec[(size_t)it * 32 + lane] = bits;
  }
}

// A battery's rows (offset in the device's block): E1 p + c - delta = 0 (t),
// E2 s_{t+1} - s_t - eta c + delta = 0 (T + t), E3 s_0 = 0 (2T), s_T = 0
// (2T + 1), CU c <= P (2T + 2 + t), CL -c <= 0 (3T + 2 + t), DU delta <= P
// (4T + 2 + t), DL -delta <= 0 (5T + 2 + t), SU s <= E (6T + 2 + j), SL -s <=
// 0 (7T + 3 + j).  Per element its rows' values; E3's on the lanes that hold
// s_0 and s_T.
enum { SE1 = 0, SE2, SCU, SCL, SDU, SDL, SSU, SSL, SGROUPS };
template <int C>
struct StorRows {
  float v[SGROUPS][C];   // per group (SE1 .. SSL) and element
  float E3a, E3b;
};
// offset of group g's row for element e in the battery's block
__device__ __forceinline__ int srow(int g, int e, int T) { return g * T + (g >= SCU ? 2 : 0) + (g == SSL ? 1 : 0) + e; }
// whether element e has a row in group g (steps for SE1 .. SDL, states of charge for SSU, SSL)
__device__ __forceinline__ bool shas(int g, int e, int T) { return g < SSU ? e < T : e <= T; }

template <int C>
__device__ void stor_fwd_r(int T, int lane, const StorK &k, float cost, float Pm, float Em, const float (&x)[C],
                           const float (&qv)[C], const float (&av)[C], StorRows<C> &lam, StorRows<C> &bet,
                           float (&zp)[C], float (&zd)[C], unsigned long long *rec) {
  const int t0 = lane * C;
  for (int it = 0; it < N_INNER; ++it) {
    unsigned long long bits = 0;
    // w = h + beta - lambda (beta = 0 and h = 0 on the equality rows)
    float wE2[C];
#pragma unroll
    for (int j = 0; j < C; ++j) wE2[j] = -lam.v[SE2][j];
    const float pE2 = __shfl_up_sync(FULLM, wE2[C - 1], 1);
    float zc[C], zs[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      zp[j] = zc[j] = zd[j] = zs[j] = 0.f;
      if (e < T) {
        const float wE1 = -lam.v[SE1][j];
        const float wCU = rsub(radd(Pm, bet.v[SCU][j]), lam.v[SCU][j]), wCL = rsub(bet.v[SCL][j], lam.v[SCL][j]);
        const float wDU = rsub(radd(Pm, bet.v[SDU][j]), lam.v[SDU][j]), wDL = rsub(bet.v[SDL][j], lam.v[SDL][j]);
        zp[j] = rfma(k.rho, x[j], rmul(k.om, wE1));
        zc[j] = rmul(k.om, rsub(radd(rfma(-k.eta, wE2[j], wE1), wCU), wCL));
        zd[j] = rsub(rmul(k.om, rsub(radd(radd(-wE1, wE2[j]), wDU), wDL)), cost);
      }
      if (e <= T) {
        float as = rsub(rsub(radd(Em, bet.v[SSU][j]), lam.v[SSU][j]), rsub(bet.v[SSL][j], lam.v[SSL][j]));
        if (e >= 1) as = radd(as, (j == 0) ? pE2 : wE2[j - 1]);
        if (e <= T - 1) as = rsub(as, wE2[j]);
        if (e == 0) as = rsub(as, lam.E3a);
        if (e == T) as = rsub(as, lam.E3b);
        zs[j] = rmul(k.om, as);
      }
    }
    stor_solve_r<C>(k, qv, av, zp, zc, zd, zs, T, lane);
    const float sn = __shfl_down_sync(FULLM, zs[0], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      if (e < T) {
        const float snx = (j == C - 1) ? sn : zs[j + 1];
        lam.v[SE1][j] = radd(rsub(radd(zp[j], zc[j]), zd[j]), lam.v[SE1][j]);                          // equality rows
        lam.v[SE2][j] = radd(radd(rfma(-k.eta, zc[j], rsub(snx, zs[j])), zd[j]), lam.v[SE2][j]);
        ineq_r(rsub(zc[j], Pm), lam.v[SCU][j], bet.v[SCU][j], bits, SCU * C + j);
        ineq_r(-zc[j], lam.v[SCL][j], bet.v[SCL][j], bits, SCL * C + j);
        ineq_r(rsub(zd[j], Pm), lam.v[SDU][j], bet.v[SDU][j], bits, SDU * C + j);
        ineq_r(-zd[j], lam.v[SDL][j], bet.v[SDL][j], bits, SDL * C + j);
      }
      if (e <= T) {
        if (e == 0) lam.E3a = radd(zs[j], lam.E3a);
        if (e == T) lam.E3b = radd(zs[j], lam.E3b);
        ineq_r(rsub(zs[j], Em), lam.v[SSU][j], bet.v[SSU][j], bits, SSU * C + j);
        ineq_r(-zs[j], lam.v[SSL][j], bet.v[SSL][j], bits, SSL * C + j);
      }
    }
    if (rec) rec[(size_t)it * 32 + lane] = bits;   // equality rows never clip: their bits stay 0
  }
}

// the device's data from the parameters and state i-1 (x: its X)
struct RDev {
  int dev, h, bat, piv;
};

template <int C>
__device__ void ramp_load(const DP &p, const St &s, const RDev &dv, int T, int lane, float (&x)[C], float (&qv)[C],
                          float (&av)[C], float (&hU)[C], float (&hL)[C], float (&hRU)[C], float (&hRD)[C],
                          float (&bU)[C], float (&lU)[C], float (&bL)[C], float (&lL)[C], float (&bRU)[C],
                          float (&lRU)[C], float (&bRD)[C], float (&lRD)[C], const float *XD) {
  const int t0 = lane * C;
  const float *B = s.INS + dv.h, *Lm = s.INS + p.Mtot + dv.h, *Hh = p.RH + dv.h;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int t = t0 + j;
    const bool in = t < T, rr = t < T - 1;
    x[j] = (in && XD) ? XD[(size_t)dv.dev * T + t] : 0.f;
    qv[j] = in ? p.piv[dv.piv + t] : 1.f;
    av[j] = in ? p.piv[dv.piv + T + t] : 0.f;
    hU[j] = in ? Hh[t] : 0.f;
    hL[j] = in ? Hh[T + t] : 0.f;
    bU[j] = in ? B[t] : 0.f;
    lU[j] = in ? Lm[t] : 0.f;
    bL[j] = in ? B[T + t] : 0.f;
    lL[j] = in ? Lm[T + t] : 0.f;
    hRU[j] = rr ? Hh[2 * T + t] : 0.f;
    hRD[j] = rr ? Hh[3 * T - 1 + t] : 0.f;
    bRU[j] = rr ? B[2 * T + t] : 0.f;
    lRU[j] = rr ? Lm[2 * T + t] : 0.f;
    bRD[j] = rr ? B[3 * T - 1 + t] : 0.f;
    lRD[j] = rr ? Lm[3 * T - 1 + t] : 0.f;
  }
}

template <int C>
__device__ void stor_load(const DP &p, const St &s, const RDev &dv, int T, int lane, StorK &k, float &cost,
                          float &Pm, float &Em, float (&x)[C], float (&qv)[C], float (&av)[C], StorRows<C> &lam,
                          StorRows<C> &bet, const float *XD) {
  const int t0 = lane * C;
  const float *B = s.INS + dv.h, *Lm = s.INS + p.Mtot + dv.h, *Hh = p.RH + dv.h;
  const float *kc = p.piv + dv.piv;
  k.rho = p.rd;
  k.om = p.rd;
  k.eta = p.beff[dv.bat];
  k.rpo = radd(k.rho, k.om);
  k.i00 = kc[0];
  k.i01 = kc[1];
  k.i11 = kc[2];
  k.gc = kc[3];
  k.gd = kc[4];
  cost = p.scost[dv.bat];
  Pm = Hh[2 * T + 2];      // the CU rows' right-hand side
  Em = Hh[6 * T + 2];      // the SU rows'
  lam.E3a = Lm[2 * T];
  lam.E3b = Lm[2 * T + 1];
  bet.E3a = bet.E3b = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int e = t0 + j;
    const bool st = e < T, ss = e <= T;
    x[j] = (st && XD) ? XD[(size_t)dv.dev * T + e] : 0.f;
    qv[j] = ss ? kc[8 + e] : 1.f;
    av[j] = ss ? kc[8 + (T + 1) + e] : 0.f;
    lam.v[SE1][j] = st ? Lm[e] : 0.f;
    lam.v[SE2][j] = st ? Lm[T + e] : 0.f;
    lam.v[SCU][j] = st ? Lm[2 * T + 2 + e] : 0.f;
    lam.v[SCL][j] = st ? Lm[3 * T + 2 + e] : 0.f;
    lam.v[SDU][j] = st ? Lm[4 * T + 2 + e] : 0.f;
    lam.v[SDL][j] = st ? Lm[5 * T + 2 + e] : 0.f;
    lam.v[SSU][j] = ss ? Lm[6 * T + 2 + e] : 0.f;
    lam.v[SSL][j] = ss ? Lm[7 * T + 3 + e] : 0.f;
    bet.v[SE1][j] = bet.v[SE2][j] = 0.f;
    bet.v[SCU][j] = st ? B[2 * T + 2 + e] : 0.f;
    bet.v[SCL][j] = st ? B[3 * T + 2 + e] : 0.f;
    bet.v[SDU][j] = st ? B[4 * T + 2 + e] : 0.f;
    bet.v[SDL][j] = st ? B[5 * T + 2 + e] : 0.f;
    bet.v[SSU][j] = ss ? B[6 * T + 2 + e] : 0.f;
    bet.v[SSL][j] = ss ? B[7 * T + 3 + e] : 0.f;
  }
}

__device__ __forceinline__ RDev rdev(const DP &p, int w) {
  const IDev di = p.idev[w];
  return RDev{di.dev, di.h, di.bat, di.piv};
}

// step 2 for the inner-ADMM devices from registers, one warp per device
template <int C>
__global__ void __launch_bounds__(TB, 1) fwd_inner_r(DP p, St s, St nx, const float *XD, float *DEL,
                                                     unsigned long long *grec) {
  const int lane = threadIdx.x & 31, w = blockIdx.x * RWARPS + (threadIdx.x >> 5), T = p.T, t0 = lane * C;
  if (w >= p.n_inner) return;
  const RDev dv = rdev(p, w);
  unsigned long long *mask = grec ? grec + (size_t)w * RREC_WORDS : nullptr;
  float *Bo = nx.INS + dv.h, *Lo = nx.INS + p.Mtot + dv.h;
  float x[C], qv[C], av[C];
  if (dv.bat < 0) {
    float hU[C], hL[C], hRU[C], hRD[C], bU[C], lU[C], bL[C], lL[C], bRU[C], lRU[C], bRD[C], lRD[C], z[C];
    ramp_load<C>(p, s, dv, T, lane, x, qv, av, hU, hL, hRU, hRD, bU, lU, bL, lL, bRU, lRU, bRD, lRD, XD);
    ramp_fwd_r<C>(T, lane, p.rd, p.rd, p.gb[dv.dev], x, qv, av, hU, hL, hRU, hRD, bU, lU, bL, lL, bRU, lRU, bRD,
                  lRD, z, mask);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      if (t < T) {
        nx.PD[(size_t)dv.dev * T + t] = z[j];
        Bo[t] = bU[j];
        Lo[t] = lU[j];
        Bo[T + t] = bL[j];
        Lo[T + t] = lL[j];
      }
      if (t < T - 1) {
        Bo[2 * T + t] = bRU[j];
        Lo[2 * T + t] = lRU[j];
        Bo[3 * T - 1 + t] = bRD[j];
        Lo[3 * T - 1 + t] = lRD[j];
      }
    }
  } else {
    StorK k;
    float cost, Pm, Em, zp[C], zd[C];
    StorRows<C> lam, bet;
    stor_load<C>(p, s, dv, T, lane, k, cost, Pm, Em, x, qv, av, lam, bet, XD);
    stor_fwd_r<C>(T, lane, k, cost, Pm, Em, x, qv, av, lam, bet, zp, zd, mask);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      if (e < T) {
        nx.PD[(size_t)dv.dev * T + e] = zp[j];
        DEL[(size_t)dv.bat * T + e] = zd[j];   // discharge, for the cost
        Bo[e] = 0.f;
        Lo[e] = lam.v[SE1][j];
        Bo[T + e] = 0.f;
        Lo[T + e] = lam.v[SE2][j];
        Bo[2 * T + 2 + e] = bet.v[SCU][j];
        Lo[2 * T + 2 + e] = lam.v[SCU][j];
        Bo[3 * T + 2 + e] = bet.v[SCL][j];
        Lo[3 * T + 2 + e] = lam.v[SCL][j];
        Bo[4 * T + 2 + e] = bet.v[SDU][j];
        Lo[4 * T + 2 + e] = lam.v[SDU][j];
        Bo[5 * T + 2 + e] = bet.v[SDL][j];
        Lo[5 * T + 2 + e] = lam.v[SDL][j];
      }
      if (e <= T) {
        Bo[6 * T + 2 + e] = bet.v[SSU][j];
        Lo[6 * T + 2 + e] = lam.v[SSU][j];
        Bo[7 * T + 3 + e] = bet.v[SSL][j];
        Lo[7 * T + 3 + e] = lam.v[SSL][j];
      }
      if (e == 0) {
        Bo[2 * T] = 0.f;
        Lo[2 * T] = lam.E3a;
      }
      if (e == T) {
        Bo[2 * T + 1] = 0.f;
        Lo[2 * T + 1] = lam.E3b;
      }
    }
  }
}

// The inner ADMM backwards from registers, one warp per device: which rows
// clipped comes from the forward's record (gmask) or, without one, from the
// forward iterations run again here into `scratch` (one iteration's record);
// then the N_INNER iterations in reverse, as bwd_inner describes.
template <int C>
__global__ void __launch_bounds__(TB, 1) bwd_inner_r(DP p, St s, Adj a, const float *XD, const float *LPDT,
                                                     float *LX, float *HB, int last, const unsigned long long *grec,
                                                     unsigned long long *scratch) {
  const int lane = threadIdx.x & 31, w = blockIdx.x * RWARPS + (threadIdx.x >> 5), T = p.T, t0 = lane * C;
  if (w >= p.n_inner) return;
  const RDev dv = rdev(p, w);
  const float rho = p.rd, om = p.rd;
  float *BB = a.LINS + dv.h, *LB = a.LINS + p.Mtot + dv.h, *HBd = HB + dv.h;
  float x[C], qv[C], av[C], xb[C];
#pragma unroll
  for (int j = 0; j < C; ++j) xb[j] = 0.f;
  if (dv.bat < 0) {
    float hU[C], hL[C], hRU[C], hRD[C], bU[C], lU[C], bL[C], lL[C], bRU[C], lRU[C], bRD[C], lRD[C];
    // X (and the state) only to run the forward iterations again
    ramp_load<C>(p, s, dv, T, lane, x, qv, av, hU, hL, hRU, hRD, bU, lU, bL, lL, bRU, lRU, bRD, lRD,
                 grec ? nullptr : XD);
    const unsigned long long *mask = (grec ? grec : scratch) + (size_t)w * RREC_WORDS;
    if (!grec) {
      float z[C];
      ramp_fwd_r<C>(T, lane, rho, om, p.gb[dv.dev], x, qv, av, hU, hL, hRU, hRD, bU, lU, bL, lL, bRU, lRU, bRD,
                    lRD, z, scratch + (size_t)w * RREC_WORDS);
    }
    // adjoints of (beta, lambda) per row, and of the right-hand sides
    float ab[4][C], al[4][C], ah[4][C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      const bool in = t < T, rr = t < T - 1;
      const int rows[4] = {t, T + t, 2 * T + t, 3 * T - 1 + t};
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const bool ok = g < 2 ? in : rr;
        ab[g][j] = ok ? BB[rows[g]] : 0.f;
        al[g][j] = ok ? LB[rows[g]] : 0.f;
        ah[g][j] = 0.f;
      }
    }
    unsigned long long mnext = mask[(size_t)(N_INNER - 1) * 32 + lane];
    for (int it = N_INNER - 1; it >= 0; --it) {
      const unsigned long long mk = mnext;
      if (it > 0) mnext = mask[(size_t)(it - 1) * 32 + lane];   // in flight during this iteration
      float sv[4][C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int t = t0 + j;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const bool ok = g < 2 ? t < T : t < T - 1;
          sv[g][j] = ok ? sbar_r(mk, g * C + j, ab[g][j], al[g][j]) : 0.f;
          ah[g][j] = rsub(ah[g][j], sv[g][j]);
        }
      }
      const float pRU = __shfl_up_sync(FULLM, sv[2][C - 1], 1), pRD = __shfl_up_sync(FULLM, sv[3][C - 1], 1);
      float rb[C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int t = t0 + j;
        rb[j] = 0.f;
        if (t < T) {
          float acc = rsub(sv[0][j], sv[1][j]);   // A' d s
          if (t >= 1) acc = radd(acc, rsub(j ? sv[2][j - 1] : pRU, j ? sv[3][j - 1] : pRD));
          if (t <= T - 2) acc = rsub(acc, rsub(sv[2][j], sv[3][j]));
          if (it == N_INNER - 1) acc = radd(acc, LPDT[(size_t)dv.dev * T + t]);   // the output p = z_p
          rb[j] = acc;
        }
      }
      tri_solve_r<C>(qv, av, rb, T, lane);
      const float rn = __shfl_down_sync(FULLM, rb[0], 1);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int t = t0 + j;
        if (t < T) {
          xb[j] = rfma(rho, rb[j], xb[j]);
          const float rnx = (j == C - 1) ? rn : rb[j + 1];
          float wv[4] = {rmul(om, rb[j]), -rmul(om, rb[j]), 0.f, 0.f};
          if (t < T - 1) {
            wv[2] = rmul(om, rsub(rnx, rb[j]));
            wv[3] = rmul(om, rsub(rb[j], rnx));
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            ah[g][j] = radd(ah[g][j], wv[g]);
            ab[g][j] = wv[g];
            al[g][j] = rsub(sv[g][j], wv[g]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int t = t0 + j;
      if (t < T) LX[(size_t)dv.dev * T + t] = xb[j];
      const int rows[4] = {t, T + t, 2 * T + t, 3 * T - 1 + t};
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (g < 2 ? t < T : t < T - 1) {
          BB[rows[g]] = ab[g][j];
          LB[rows[g]] = al[g][j];
          HBd[rows[g]] += ah[g][j];
        }
      }
    }
  } else {
    StorK k;
    float cost, Pm, Em;
    StorRows<C> lam, bet;
    stor_load<C>(p, s, dv, T, lane, k, cost, Pm, Em, x, qv, av, lam, bet, grec ? nullptr : XD);
    const unsigned long long *mask = (grec ? grec : scratch) + (size_t)w * RREC_WORDS;
    if (!grec) {
      float zp[C], zd[C];
      stor_fwd_r<C>(T, lane, k, cost, Pm, Em, x, qv, av, lam, bet, zp, zd, scratch + (size_t)w * RREC_WORDS);
    }
    const float dcost = last ? cost : 0.f;
    // per row group: adjoints of beta (ab), lambda (al), the right-hand side (ah)
    StorRows<C> ab, al, ah;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
#pragma unroll
      for (int g = 0; g < SGROUPS; ++g) {
        const bool ok = shas(g, e, T);
        ab.v[g][j] = ok ? BB[srow(g, e, T)] : 0.f;
        al.v[g][j] = ok ? LB[srow(g, e, T)] : 0.f;
        ah.v[g][j] = 0.f;
      }
    }
    ab.E3a = BB[2 * T];
    ab.E3b = BB[2 * T + 1];
    al.E3a = LB[2 * T];
    al.E3b = LB[2 * T + 1];
    ah.E3a = ah.E3b = 0.f;
    unsigned long long mnext = mask[(size_t)(N_INNER - 1) * 32 + lane];
    for (int it = N_INNER - 1; it >= 0; --it) {
      const unsigned long long mk = mnext;
      if (it > 0) mnext = mask[(size_t)(it - 1) * 32 + lane];   // in flight during this iteration
      StorRows<C> sv;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int e = t0 + j;
#pragma unroll
        for (int g = 0; g < SGROUPS; ++g) {
          sv.v[g][j] = shas(g, e, T) ? sbar_r(mk, g * C + j, ab.v[g][j], al.v[g][j]) : 0.f;
          ah.v[g][j] = rsub(ah.v[g][j], sv.v[g][j]);
        }
      }
      sv.E3a = al.E3a;   // equality rows never clip
      sv.E3b = al.E3b;
      ah.E3a = rsub(ah.E3a, sv.E3a);
      ah.E3b = rsub(ah.E3b, sv.E3b);
      const float pE2 = __shfl_up_sync(FULLM, sv.v[SE2][C - 1], 1);
      float zp[C], zc[C], zd[C], zs[C];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int e = t0 + j;
        zp[j] = zc[j] = zd[j] = zs[j] = 0.f;
        if (e < T) {   // A' d s, and the outputs' adjoints on the last inner iterate
          zp[j] = sv.v[SE1][j];
          zc[j] = rsub(radd(rfma(-k.eta, sv.v[SE2][j], sv.v[SE1][j]), sv.v[SCU][j]), sv.v[SCL][j]);
          zd[j] = rsub(radd(radd(-sv.v[SE1][j], sv.v[SE2][j]), sv.v[SDU][j]), sv.v[SDL][j]);
          if (it == N_INNER - 1) {
            zp[j] = radd(zp[j], LPDT[(size_t)dv.dev * T + e]);
            zd[j] = radd(zd[j], dcost);
          }
        }
        if (e <= T) {
          float as = rsub(sv.v[SSU][j], sv.v[SSL][j]);
          if (e >= 1) as = radd(as, (j == 0) ? pE2 : sv.v[SE2][j - 1]);
          if (e <= T - 1) as = rsub(as, sv.v[SE2][j]);
          if (e == 0) as = radd(as, sv.E3a);
          if (e == T) as = radd(as, sv.E3b);
          zs[j] = as;
        }
      }
      stor_solve_r<C>(k, qv, av, zp, zc, zd, zs, T, lane);
      const float sn = __shfl_down_sync(FULLM, zs[0], 1);
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int e = t0 + j;
        float wv[SGROUPS];
#pragma unroll
        for (int g = 0; g < SGROUPS; ++g) wv[g] = 0.f;
        if (e < T) {
          xb[j] = rfma(rho, zp[j], xb[j]);
          const float snx = (j == C - 1) ? sn : zs[j + 1];
          wv[0] = rmul(om, rsub(radd(zp[j], zc[j]), zd[j]));
          wv[1] = rmul(om, radd(rfma(-k.eta, zc[j], rsub(snx, zs[j])), zd[j]));
          wv[2] = rmul(om, zc[j]);
          wv[3] = -rmul(om, zc[j]);
          wv[4] = rmul(om, zd[j]);
          wv[5] = -rmul(om, zd[j]);
        }
        if (e <= T) {
          wv[6] = rmul(om, zs[j]);
          wv[7] = -rmul(om, zs[j]);
        }
#pragma unroll
        for (int g = 0; g < SGROUPS; ++g) {
          if (shas(g, e, T)) {
            ah.v[g][j] = radd(ah.v[g][j], wv[g]);
            ab.v[g][j] = wv[g];
            al.v[g][j] = rsub(sv.v[g][j], wv[g]);
          }
        }
        if (e == 0) {
          const float w3 = rmul(om, zs[j]);
          ah.E3a = radd(ah.E3a, w3);
          ab.E3a = w3;
          al.E3a = rsub(sv.E3a, w3);
        }
        if (e == T) {
          const float w3 = rmul(om, zs[j]);
          ah.E3b = radd(ah.E3b, w3);
          ab.E3b = w3;
          al.E3b = rsub(sv.E3b, w3);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int e = t0 + j;
      if (e < T) LX[(size_t)dv.dev * T + e] = xb[j];
#pragma unroll
      for (int g = 0; g < SGROUPS; ++g) {
        if (shas(g, e, T)) {
          BB[srow(g, e, T)] = ab.v[g][j];
          LB[srow(g, e, T)] = al.v[g][j];
          HBd[srow(g, e, T)] += ah.v[g][j];
        }
      }
      if (e == 0) {
        BB[2 * T] = ab.E3a;
        LB[2 * T] = al.E3a;
        HBd[2 * T] += ah.E3a;
      }
      if (e == T) {
        BB[2 * T + 1] = ab.E3b;
        LB[2 * T + 1] = al.E3b;
        HBd[2 * T + 1] += ah.E3b;
      }
    }
  }
}

// C = d/d pbar (old) = -sx - avg_k(the node's devices' d/dX) (x = ... -
// pbar - u, X = ... - avg_k(pbar + u)), which is also u's adjoint's
// increment: the line terms sx and the device terms, sd = the sum of the
// node's devices' d/dX at steps t0 ..
template <int VW>
__device__ __forceinline__ void node_sd(const DP &p, const float *LX, int n, int t0, float (&sd)[VW]) {
#pragma unroll
  for (int e = 0; e < VW; ++e) sd[e] = 0.f;
  for (int j = p.dptr[n]; j < p.dptr[n + 1]; ++j) {
    const Vf<VW> v = ldv<VW>(LX + (size_t)p.didx[j] * p.T + t0);
#pragma unroll
    for (int e = 0; e < VW; ++e) sd[e] += v.x[e];
  }
}

// gathers at the nodes: D = d/d theta_bar (old), and C, complete (with u's
// adjoint's increment) at a node without an inner-ADMM device, else its line
// terms -sx, completed by bwd_node3 once the inner ADMM is done.  nxt: also
// iteration i-1's B (bwd_node1: the v adjoints are final after bwd_line1 of
// iteration i).  It reads nothing the inner ADMM writes (LX only of the
// other devices), and runs beside it.
template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) bwd_node2(DP p, Adj a, const float *X2, const float *Y1,
                                                                       const float *Y2, const float *LX, float *C,
                                                                       float *Dt, float *B, int nxt) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.N, p.T);
    const int n = it.m;
    float sx[VW], sy[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) sx[e] = sy[e] = 0.f;
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j];
      const size_t o = li(p, it.k, c >> 1, it.t0);
      const Vf<VW> x = ldv<VW>(X2 + o), y = ldv<VW>(((c & 1) ? Y2 : Y1) + o);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        sx[e] += (c & 1) ? x.x[e] : -x.x[e];
        sy[e] += y.x[e];
      }
    }
    Vf<VW> cv, dv;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      cv.x[e] = -sx[e];
      dv.x[e] = sy[e];                   // y = theta_bar - v
    }
    if (!p.hasin[n]) {
      float sd[VW];
      node_sd<VW>(p, LX, n, it.t0, sd);
      const Vf<VW> u = ldv<VW>(a.LU + it.o);
      Vf<VW> un;
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        cv.x[e] = cv.x[e] - sd[e] / (float)p.Kp;
        un.x[e] = u.x[e] + cv.x[e];
      }
      stv<VW>(a.LU + it.o, un);
    }
    stv<VW>(C + it.o, cv);
    stv<VW>(Dt + it.o, dv);
    if (nxt) stv<VW>(B + it.o, node_b<VW>(p, a, it.k, n, it.t0));
  }
}

// ... and at the nodes with an inner-ADMM device, once it is done (items
// (k, m, t0 ..) of the nodes inode[m])
template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) bwd_node3(DP p, Adj a, const float *LX, float *C) {
  GRID_STRIDE(i, (long long)p.Kp * p.n_inode * (p.T / VW)) {
    const Item it = item_of<VW>(i, p.n_inode, p.T);
    const int n = p.inode[it.m];
    const size_t o = ni(p, it.k, n, it.t0);
    float sd[VW];
    node_sd<VW>(p, LX, n, it.t0, sd);
    const Vf<VW> c0 = ldv<VW>(C + o), u = ldv<VW>(a.LU + o);
    Vf<VW> cv, un;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      cv.x[e] = c0.x[e] - sd[e] / (float)p.Kp;
      un.x[e] = u.x[e] + cv.x[e];
    }
    stv<VW>(C + o, cv);
    stv<VW>(a.LU + o, un);
  }
}

// The scatters of one reverse iteration, as one launch whose first
// dev_blocks blocks take the device items and the rest the line items (their
// writes are disjoint; the device items, fewer and waiting longer on their
// sums, start first).
struct Scatter {
  const float *C, *Dt, *A, *B, *LX;   // node gathers, u's adjoint, B of iteration i-1, this iteration's d/dX
  float *X2, *Y1, *Y2, *GU;           // iteration i-1's line terms
  float *LXn, *GL, *GP, *XD, *LPDT;   // iteration i-1's device terms
  const unsigned char *lmask, *dmask; // iteration i-1's record (or NULL)
};

// the old node averages back onto the old line values; nxt: then iteration
// i-1's line prox backwards on the same item (bwd_line1), from state s and
// record lmask of that iteration
template <int VW>
__device__ __forceinline__ void line2_part(const DP &p, const St &s, const Adj &a, const Scatter &g, int nxt,
                                           unsigned bid, unsigned nb) {
  GRID_STRIDE_B(i, (long long)p.Kp * p.L * (p.T / VW), bid, nb) {
    const Item it = item_of<VW>(i, p.L, p.T);
    const int n1 = p.n1[it.m], n2 = p.n2[it.m];
    const size_t o1 = ni(p, it.k, n1, it.t0), o2 = ni(p, it.k, n2, it.t0);
    const float ic1 = p.icnt[n1], ic2 = p.icnt[n2], ih1 = p.icth[n1], ih2 = p.icth[n2];
    const Vf<VW> C1 = ldv<VW>(g.C + o1), C2 = ldv<VW>(g.C + o2), D1 = ldv<VW>(g.Dt + o1), D2 = ldv<VW>(g.Dt + o2);
    const Vf<VW> lp0 = ldv<VW>(a.LP + it.o);
    Vf<VW> lp, lt1, lt2;
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      lp.x[e] = __fadd_rn(lp0.x[e], fmaf(C2.x[e], ic2, -__fmul_rn(C1.x[e], ic1)));
      lt1.x[e] = __fmul_rn(D1.x[e], ih1);
      lt2.x[e] = __fmul_rn(D2.x[e], ih2);
    }
    if (nxt) {
      line_back<VW>(p, s, a, ldv<VW>(g.A + o1), ldv<VW>(g.A + o2), g.B, g.X2, g.Y1, g.Y2, g.GU, g.lmask, it, lp,
                    lt1, lt2);
    } else {
      stv<VW>(a.LP + it.o, lp);
      stv<VW>(a.LT1 + it.o, lt1);
      stv<VW>(a.LT2 + it.o, lt2);
    }
  }
}

// ... and onto the old device powers (LX: this iteration's d/dX); nxt: then
// iteration i-1's device proxes backwards on the same item (bwd_dev), into
// LXn, from state s and record dmask of that iteration.  An HVDC terminal
// recomputes its partner's adjoint from the same inputs.
template <int VW>
__device__ __forceinline__ void dev2_part(const DP &p, const St &s, const Adj &a, const Scatter &g, int nxt,
                                          unsigned bid, unsigned nb) {
  GROUP_STRIDE_B(i, (long long)p.S * (p.T / VW), bid, nb) {
    int d, t0;
    dev_item<VW>(i, p.T, d, t0);
    const size_t o = (size_t)i * VW;
    const bool lead = !(threadIdx.x & (KL - 1));
    const Vf<VW> lpd = add_node_kv<VW>(p, g.C, d, t0, ldv<VW>(g.LX + o));
    if (lead) stv<VW>(a.LPD + o, lpd);
    if (nxt) {
      const int d2 = hvdc_partner(p, d);
      const size_t o2 = (size_t)d2 * p.T + t0;
      Vf<VW> lpd_o{}, X{}, Xo{};
      if (d2 >= 0) lpd_o = add_node_kv<VW>(p, g.A, d2, t0, add_node_kv<VW>(p, g.C, d2, t0, ldv<VW>(g.LX + o2)));
      const Vf<VW> lpdn = add_node_kv<VW>(p, g.A, d, t0, lpd);
      if (!g.dmask) X = dev_xv<VW>(p, s, d, t0);
      if (!g.dmask && d2 >= 0) Xo = dev_xv<VW>(p, s, d2, t0);
      if (lead)
#pragma unroll
        for (int e = 0; e < VW; ++e)
          dev_back(p, g.LXn, g.GL, g.GP, g.XD, g.LPDT, g.dmask, (unsigned)(o + e), d, t0 + e, lpdn.x[e], lpd_o.x[e],
                   X.x[e], Xo.x[e]);
    }
  }
}

template <int VW>
__global__ void __launch_bounds__(TB, VW == 4 ? VW4_CTAS : 8) bwd_scatter(DP p, St s, Adj a, Scatter g, int nxt, int dev_blocks) {
  if ((int)blockIdx.x < dev_blocks) dev2_part<VW>(p, s, a, g, nxt, blockIdx.x, dev_blocks);
  else line2_part<VW>(p, s, a, g, nxt, blockIdx.x - dev_blocks, gridDim.x - dev_blocks);
}

// d f / d p_d at the last iterate, and f's direct dependence on P (the
// battery discharge term enters through bwd_inner's `last`)
__global__ void bwd_init(DP p, St s, Adj a, float *GL) {
  GRID_STRIDE(i, (long long)p.S * p.T) {
    const int d = (int)(i / (unsigned)p.T), t = (int)(i - (unsigned)d * (unsigned)p.T);
    if (d < p.G) {
      a.LPD[i] = 2.f * p.ga[d] * s.PD[i] + p.gb[d];
    } else if (d < p.G + p.D) {
      const int e = d - p.G;
      a.LPD[i] = p.voll[e] < 0.f ? 0.f : p.voll[e];
      if (p.voll[e] >= 0.f) GL[(size_t)e * p.T + t] = p.voll[e];
    } else {
      a.LPD[i] = 0.f;
    }
  }
}

// the capacity rows of every ramp-limited generator (its first T inner rows,
// p_t <= pmax_t) from the capacity data of this call
__global__ void set_ramp_rhs(DP p, float *RH) {
  GRID_STRIDE(i, (long long)p.n_inner * p.T) {
    const int r = (int)(i / (unsigned)p.T), t = (int)(i - (unsigned)r * (unsigned)p.T);
    const IDev di = p.idev[r];
    if (di.bat < 0) RH[di.h + t] = p.gpmax[(size_t)di.dev * p.T + t];
  }
}

// d f / d u_l: the limit is the same in every contingency and step, so the
// per-(k, l, t) adjoints are summed (FP64, fixed order); and a ramp
// generator's capacity gradient gains the adjoint of its capacity rows
__global__ void finish_line_grad(DP p, const float *GU, float *out) {
  GRID_STRIDE(l, (long long)p.L) {
    double s = 0.0;
    for (int k = 0; k < p.Kp; ++k)
      for (int t = 0; t < p.T; ++t) s += GU[((size_t)k * p.L + l) * p.T + t];
    out[l] = (float)s;
  }
}

__global__ void finish_cap_grad(DP p, const float *HB, float *GP) {
  GRID_STRIDE(i, (long long)p.n_inner * p.T) {
    const int r = (int)(i / (unsigned)p.T), t = (int)(i - (unsigned)r * (unsigned)p.T);
    const IDev di = p.idev[r];
    if (di.bat < 0) GP[(size_t)di.dev * p.T + t] += HB[di.h + t];
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + TB - 1) / TB, 8192)); }

size_t fwd_inner_smem(int T, int n, int m, int nnz, int level) {
  return (size_t)(T + 2 * n + 3 * m + view_words(n, m, nnz, level)) * sizeof(float);
}
size_t bwd_inner_smem(int T, int n, int m, int nnz, int level) {
  return (size_t)(2 * T + 4 * n + 7 * m + view_words(n, m, nnz, level)) * sizeof(float) + (size_t)N_INNER * m;
}

}  // namespace

struct opf_diff {
  int N = 0, L = 0, T = 0, Kp = 0, G = 0, D = 0, B = 0, H = 0, S = 0, ckpt = 1;
  cudaStream_t stream = nullptr;
  // the reverse pass runs the node gathers of the line terms here, beside
  // the inner ADMM on `stream` (created by the first gradient call)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  DP p{};
  std::vector<float> ga, gb, voll, load_p, gpmax, lu, scost;  // host copies (cost and defaults)
  std::vector<double> gpmin, ramp, sP, sdur;                 // right-hand sides of the inner rows
  std::vector<int> ramp_gens;                                // generator of each ramp device
  std::vector<IDev> idev;
  int Mtot = 0;
  size_t smem_fwd = 0, smem_bwd = 0;
  int stage = 0;         // what the inner kernels copy into shared memory (view_words)
  float *RH = nullptr;                                       // device copy of the right-hand sides
  std::vector<void *> allocs;
  size_t state_floats = 0;
  // per-call buffers, kept between calls and grown when a call needs more:
  // checkpoints, one segment of states, the adjoint, work arrays, the
  // per-line limit gradient and the host staging of the cost's inputs
  float *ck = nullptr, *seg = nullptr, *adj = nullptr, *work = nullptr, *gline = nullptr;
  size_t ck_cap = 0, seg_cap = 0;
  // which inner-ADMM rows clipped, per iteration of the forward pass
  // ([K][N_INNER rows of every device], one byte each), for the reverse pass
  float *masks = nullptr;
  size_t masks_cap = 0;
  size_t record_limit = size_t(4) << 30;   // opf_diff_set_record_limit
  unsigned char *mask1 = nullptr;           // one iteration's inner record, for a reverse pass without one
};

namespace {

opf_status dfail(opf_status s, const char *m) { return (opf_status)opf_record_error((int)s, m); }

#define DCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return dfail(OPF_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t dalloc(std::vector<void *> &list, T **p, size_t n) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) list.push_back(*p);
  return e;
}

template <class T>
cudaError_t up(std::vector<void *> &list, const T **dst, const std::vector<T> &v) {
  T *d = nullptr;
  cudaError_t e = dalloc(list, &d, v.size());
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  *dst = d;
  return e;
}

// constraint rows of one device kind, as (row, column, value) lists
struct Rows {
  int n = 0, m = 0;
  std::vector<std::vector<std::pair<int, double>>> row;
  std::vector<unsigned char> eq;
  void add(std::vector<std::pair<int, double>> r, bool is_eq) {
    row.push_back(std::move(r));
    eq.push_back(is_eq ? 1 : 0);
    m = (int)row.size();
  }
};

// generator with box and ramp limits (Section 2.1), variables p_0..p_{T-1}:
// p_t <= pmax_t, -p_t <= -pmin_t, p_{t+1} - p_t <= R, p_t - p_{t+1} <= R
Rows ramp_shape(int T) {
  Rows r;
  r.n = T;
  for (int t = 0; t < T; ++t) r.add({{t, 1.0}}, false);
  for (int t = 0; t < T; ++t) r.add({{t, -1.0}}, false);
  for (int t = 0; t + 1 < T; ++t) r.add({{t + 1, 1.0}, {t, -1.0}}, false);
  for (int t = 0; t + 1 < T; ++t) r.add({{t, 1.0}, {t + 1, -1.0}}, false);
  return r;
}

void ramp_rhs(int T, const double *pmin, const double *pmax, double R, float *h) {
  int o = 0;
  for (int t = 0; t < T; ++t) h[o++] = (float)pmax[t];
  for (int t = 0; t < T; ++t) h[o++] = (float)(-pmin[t]);
  for (int i = 0; i < 2 * (T - 1); ++i) h[o++] = (float)R;
}

// battery (Section 2.1), variables (p, c, delta, s) with s of length T + 1:
// p + c - delta = 0, s_{t+1} - s_t - eff c_t + delta_t = 0, s_0 = s_T = 0,
// 0 <= c <= P, 0 <= delta <= P, 0 <= s <= dur P
Rows storage_shape(int T, double eff) {
  Rows r;
  r.n = 4 * T + 1;
  const int c0 = T, d0 = 2 * T, s0 = 3 * T;
  for (int t = 0; t < T; ++t) r.add({{t, 1.0}, {c0 + t, 1.0}, {d0 + t, -1.0}}, true);
  for (int t = 0; t < T; ++t) r.add({{s0 + t + 1, 1.0}, {s0 + t, -1.0}, {c0 + t, -eff}, {d0 + t, 1.0}}, true);
  r.add({{s0, 1.0}}, true);
  r.add({{s0 + T, 1.0}}, true);
  for (int t = 0; t < T; ++t) r.add({{c0 + t, 1.0}}, false);
  for (int t = 0; t < T; ++t) r.add({{c0 + t, -1.0}}, false);
  for (int t = 0; t < T; ++t) r.add({{d0 + t, 1.0}}, false);
  for (int t = 0; t < T; ++t) r.add({{d0 + t, -1.0}}, false);
  for (int t = 0; t <= T; ++t) r.add({{s0 + t, 1.0}}, false);
  for (int t = 0; t <= T; ++t) r.add({{s0 + t, -1.0}}, false);
  return r;
}

void storage_rhs(int T, double P, double dur, float *h) {
  int o = 0;
  for (int i = 0; i < 2 * T + 2; ++i) h[o++] = 0.f;
  for (int t = 0; t < T; ++t) h[o++] = (float)P;
  for (int t = 0; t < T; ++t) h[o++] = 0.f;
  for (int t = 0; t < T; ++t) h[o++] = (float)P;
  for (int t = 0; t < T; ++t) h[o++] = 0.f;
  for (int t = 0; t <= T; ++t) h[o++] = (float)(dur * P);
  for (int t = 0; t <= T; ++t) h[o++] = 0.f;
}

// inverse of the symmetric positive definite M = diag(qd) + omega A'A (FP64
// Cholesky, then one solve per unit vector), stored as FP32
bool spd_inverse(const Rows &r, const std::vector<double> &qd, double omega, std::vector<float> &out) {
  const int n = r.n;
  std::vector<double> M((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) M[(size_t)i * n + i] = qd[i];
  for (const auto &row : r.row)
    for (const auto &a : row)
      for (const auto &b : row) M[(size_t)a.first * n + b.first] += omega * a.second * b.second;
  for (int j = 0; j < n; ++j) {                      // M = C C', C lower, in place
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    M[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      M[(size_t)i * n + j] = v / d;
    }
  }
  const size_t base = out.size();
  out.resize(base + (size_t)n * n);
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {                    // C y = e_c
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= M[(size_t)i * n + k] * y[k];
      y[i] = v / M[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {               // C' x = y
      double v = y[i];
      for (int k = i + 1; k < n; ++k) v -= M[(size_t)k * n + i] * y[k];
      y[i] = v / M[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) out[base + (size_t)c * n + i] = (float)y[i];
  }
  return true;
}

// Thomas pivots of a tridiagonal matrix with diagonal d_end at both ends,
// d_mid inside and off-diagonal off (FP64, stored as FP32), then the solve's
// coefficients a = -off / q
void tri_pivots(int n, double d_end, double d_mid, double off, std::vector<float> &out) {
  std::vector<double> q(n);
  for (int i = 0; i < n; ++i) {
    const double d = (i == 0 || i == n - 1) ? d_end : d_mid;
    q[i] = i == 0 ? d : d - off * off / q[i - 1];
  }
  for (int i = 0; i < n; ++i) out.push_back((float)q[i]);
  for (int i = 0; i < n; ++i) out.push_back((float)(-off / q[i]));
}

// A battery's factor for the register path (omega = rho' = rd): with p
// eliminated, the 2 x 2 block H of (c_t, delta_t) and its inverse, the
// coupling f = (-omega eta, omega) of (c_t, delta_t) to s_{t+1} - s_t and
// g = H^-1 f, and the tridiagonal system of s whose neighbours couple with
// gam = omega - f'g: eight constants (i00 i01 i11 gc gd, three unused), then
// the pivots and coefficients of the s system
void stor_factor(int T, double rd, double eta, std::vector<float> &out) {
  const double rho = rd, om = rd;
  const double kap = rho * om / (rho + om);
  const double h00 = kap + 2.0 * om + om * eta * eta, h01 = -kap - om * eta, h11 = kap + 3.0 * om;
  const double det = h00 * h11 - h01 * h01;
  const double i00 = h11 / det, i01 = -h01 / det, i11 = h00 / det;
  const double fc = -om * eta, fd = om;
  const double gc = i00 * fc + i01 * fd, gd = i01 * fc + i11 * fd;
  const double gam = om - (fc * gc + fd * gd);
  for (double v : {i00, i01, i11, gc, gd, 0.0, 0.0, 0.0}) out.push_back((float)v);
  tri_pivots(T + 1, 3.0 * om + gam, 2.0 * om + 2.0 * gam, -gam, out);
}

St carve_state(const opf_diff *d, float *base) {
  const size_t KLT = (size_t)d->Kp * d->L * d->T, KNT = (size_t)d->Kp * d->N * d->T, ST = (size_t)d->S * d->T;
  St s;
  float *c = base;
  s.P = c; c += KLT;
  s.TH1 = c; c += KLT;
  s.TH2 = c; c += KLT;
  s.V1 = c; c += KLT;
  s.V2 = c; c += KLT;
  s.PD = c; c += ST;
  s.U = c; c += KNT;
  s.PB = c; c += KNT;
  s.TBR = c; c += KNT;
  s.INS = c;
  return s;
}

// mask (optional): the iteration's record for the reverse pass -- the
// clipped inner rows, then a byte per line item, then one per device step
void forward_step(const opf_diff *d, const St &s, const St &nx, float *XD, float *DEL,
                  unsigned char *mask = nullptr) {
  const DP &p = d->p;
  const long long nl = (long long)p.Kp * p.L * p.T, nn = (long long)p.Kp * p.N * p.T, ns = (long long)p.S * p.T;
  unsigned char *lmask = mask ? mask + inner_record_bytes(p) : nullptr;
  unsigned char *dmask = mask ? lmask + nl : nullptr;
  unsigned long long *rrec = reinterpret_cast<unsigned long long *>(mask);
  const bool v4 = p.T % 4 == 0;   // four steps per thread in the line and node kernels
  if (v4) fwd_line<4><<<grid_for(nl / 4), TB, 0, d->stream>>>(p, s, nx, lmask);
  else fwd_line<1><<<grid_for(nl), TB, 0, d->stream>>>(p, s, nx, lmask);
  fwd_dev<<<grid_for(ns * KL), TB, 0, d->stream>>>(p, s, nx, XD, dmask);
  if (p.n_inner) {
    const int g = (p.n_inner + RWARPS - 1) / RWARPS;
    switch (p.reg_c) {
      case 1: fwd_inner_r<1><<<g, TB, 0, d->stream>>>(p, s, nx, XD, DEL, rrec); break;
      case 2: fwd_inner_r<2><<<g, TB, 0, d->stream>>>(p, s, nx, XD, DEL, rrec); break;
      case 3: fwd_inner_r<3><<<g, TB, 0, d->stream>>>(p, s, nx, XD, DEL, rrec); break;
      case 4: fwd_inner_r<4><<<g, TB, 0, d->stream>>>(p, s, nx, XD, DEL, rrec); break;
      default: fwd_inner<<<p.n_inner, TBI, d->smem_fwd, d->stream>>>(p, s, nx, XD, DEL, d->stage, mask); break;
    }
  }
  if (v4) fwd_avg<4><<<grid_for(nn / 4), TB, 0, d->stream>>>(p, s, nx);
  else fwd_avg<1><<<grid_for(nn), TB, 0, d->stream>>>(p, s, nx);
}

}  // namespace

extern "C" {

opf_status opf_diff_create(const opf_network *net, int32_t T, const opf_contingencies *ctg, double rho_p,
                           double rho_theta, int32_t checkpoint_every, void *cuda_stream, opf_diff **out) {
  if (!out) return dfail(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!net || T < 1) return dfail(OPF_EINVAL, "NULL network or horizon < 1");
  if (!(rho_p > 0) || !(rho_theta > 0) || checkpoint_every < 1)
    return dfail(OPF_EINVAL, "diff: penalties must be > 0 and checkpoint_every >= 1");
  const int N = net->n_nodes, L = net->n_lines, G = net->n_gens, D = net->n_loads, B = net->n_stor;
  const int H = net->n_hvdc;
  if (N < 1 || L < 0 || G < 0 || D < 0 || B < 0 || H < 0) return dfail(OPF_EINVAL, "diff: bad sizes");
  for (int h = 0; h < H; ++h)
    if (net->hvdc_from[h] == net->hvdc_to[h] || !(net->hvdc_u[h] >= 0))
      return dfail(OPF_EINVAL, "diff: bad HVDC link");
  const int K = ctg ? ctg->K : 0;
  if (K < 0) return dfail(OPF_EINVAL, "diff: K must be >= 0");
  if ((double)(K + 1) * std::max(L, N) * T >= 2147483647.0 || (double)(G + D + B + 2 * H) * T >= 2147483647.0)
    return dfail(OPF_EINVAL, "diff: (K+1) * max(lines, nodes) * T and devices * T must stay below 2^31");
  for (int l = 0; l < L; ++l) {
    const int a = net->line_from[l], c = net->line_to[l];
    if (a < 0 || a >= N || c < 0 || c >= N || a == c || !(net->line_b[l] > 0))
      return dfail(OPF_EINVAL, "diff: bad line");
  }
  for (int k = 0; k < K; ++k)
    if (ctg->outaged_line[k] < -1 || ctg->outaged_line[k] >= L)
      return dfail(OPF_EINVAL, "diff: outaged line id out of range");
  for (int b = 0; b < B; ++b)
    if (!(net->stor_P[b] >= 0) || !(net->stor_dur[b] >= 0) || !(net->stor_eff[b] > 0 && net->stor_eff[b] <= 1))
      return dfail(OPF_EINVAL, "diff: bad battery data");
  auto *d = new (std::nothrow) opf_diff();
  if (!d) return dfail(OPF_ENOMEM, "host allocation failed");
  d->N = N;
  d->L = L;
  d->T = T;
  d->Kp = K + 1;
  d->G = G;
  d->D = D;
  d->B = B;
  d->H = H;
  d->S = G + D + B + 2 * H;
  d->ckpt = checkpoint_every;
  d->stream = (cudaStream_t)cuda_stream;
  // incidence by node (caller's numbering)
  std::vector<int> lptr(N + 1, 0), lcode(2 * (size_t)L), dptr(N + 1, 0), didx(d->S), dnode(d->S), kind(d->S, 0);
  std::vector<float> cnt(N, 0.f), cth(N, 0.f);
  for (int l = 0; l < L; ++l) {
    ++lptr[net->line_from[l] + 1];
    ++lptr[net->line_to[l] + 1];
  }
  for (int g = 0; g < G; ++g) dnode[g] = net->gen_node[g];
  for (int e = 0; e < D; ++e) dnode[G + e] = net->load_node[e];
  for (int b = 0; b < B; ++b) dnode[G + D + b] = net->stor_node[b];
  for (int h = 0; h < H; ++h) {
    dnode[G + D + B + 2 * h] = net->hvdc_from[h];
    dnode[G + D + B + 2 * h + 1] = net->hvdc_to[h];
    kind[G + D + B + 2 * h] = kind[G + D + B + 2 * h + 1] = 2;
  }
  for (int s = 0; s < d->S; ++s) {
    if (dnode[s] < 0 || dnode[s] >= N) {
      delete d;
      return dfail(OPF_EINVAL, "diff: device node id out of range");
    }
    ++dptr[dnode[s] + 1];
  }
  for (int n = 0; n < N; ++n) {
    lptr[n + 1] += lptr[n];
    dptr[n + 1] += dptr[n];
  }
  {
    std::vector<int> f(lptr.begin(), lptr.end() - 1), g(dptr.begin(), dptr.end() - 1);
    for (int l = 0; l < L; ++l) {
      lcode[f[net->line_from[l]]++] = 2 * l;
      lcode[f[net->line_to[l]]++] = 2 * l + 1;
    }
    for (int s = 0; s < d->S; ++s) didx[g[dnode[s]]++] = s;
  }
  for (int n = 0; n < N; ++n) {
    cth[n] = (float)(lptr[n + 1] - lptr[n]);
    cnt[n] = cth[n] + (float)(dptr[n + 1] - dptr[n]);
    if (cnt[n] == 0.f) {
      delete d;
      return dfail(OPF_EINVAL, "diff: a node has no terminal");
    }
  }
  std::vector<int> n1(net->line_from, net->line_from + L), n2(net->line_to, net->line_to + L);
  std::vector<float> b(L), gpmin((size_t)G * T);
  std::vector<int> outl(d->Kp, -1);
  for (int l = 0; l < L; ++l) b[l] = (float)net->line_b[l];
  for (int k = 0; k < K; ++k) outl[k + 1] = ctg->outaged_line[k];
  d->ga.resize(G);
  d->gb.resize(G);
  d->voll.resize(D);
  for (int g = 0; g < G; ++g) {
    d->ga[g] = (float)net->gen_a[g];
    d->gb[g] = (float)net->gen_b[g];
  }
  for (size_t i = 0; i < (size_t)G * T; ++i) gpmin[i] = (float)net->gen_pmin[i];
  for (int e = 0; e < D; ++e) d->voll[e] = (float)net->load_voll[e];
  d->load_p.assign((size_t)D * T, 0.f);
  d->gpmax.assign((size_t)G * T, 0.f);
  d->lu.assign(L, 0.f);
  for (size_t i = 0; i < (size_t)D * T; ++i) d->load_p[i] = (float)net->load_p[i];
  for (size_t i = 0; i < (size_t)G * T; ++i) d->gpmax[i] = (float)net->gen_pmax[i];
  for (int l = 0; l < L; ++l) d->lu[l] = (float)net->line_u[l];
  d->gpmin.assign(net->gen_pmin, net->gen_pmin + (size_t)G * T);
  // inner-ADMM devices (Appendix D): ramp-limited generators (T > 1), batteries
  const double rd = (double)d->Kp * rho_p;
  std::vector<Shape> shapes;
  std::vector<int> arp, aci, atp, ati;
  std::vector<float> acv, atv, minv, qv;
  std::vector<unsigned char> aeq;
  auto add_shape = [&](const Rows &r) {
    Shape s{};
    s.n = r.n;
    s.m = r.m;
    s.rp = (int)arp.size();
    s.ci = (int)aci.size();
    s.tp = (int)atp.size();
    s.ti = (int)ati.size();
    s.eq = (int)aeq.size();
    arp.push_back(0);
    std::vector<std::vector<std::pair<int, double>>> cols(r.n);
    for (int i = 0; i < r.m; ++i) {
      for (const auto &a : r.row[i]) {
        aci.push_back(a.first);
        acv.push_back((float)a.second);
        cols[a.first].push_back({i, a.second});
      }
      arp.push_back((int)(aci.size() - s.ci));
    }
    atp.push_back(0);
    for (int j = 0; j < r.n; ++j) {
      for (const auto &a : cols[j]) {
        ati.push_back(a.first);
        atv.push_back((float)a.second);
      }
      atp.push_back((int)(ati.size() - s.ti));
    }
    aeq.insert(aeq.end(), r.eq.begin(), r.eq.end());
    s.nnz = (int)(aci.size() - s.ci);
    shapes.push_back(s);
    return (int)shapes.size() - 1;
  };
  std::vector<float> piv;   // the register path's factors (DP::piv)
  bool ok = true;
  int hoff = 0;
  if (T > 1 && net->gen_ramp) {
    const Rows rr = ramp_shape(T);
    int sh = -1;
    for (int g = 0; g < G && ok; ++g) {
      if (!(net->gen_ramp[g] >= 0)) continue;
      if (sh < 0) sh = add_shape(rr);
      IDev di{};
      di.dev = g;
      di.shape = sh;
      di.minv = (int)minv.size();
      di.h = hoff;
      di.q = (int)qv.size();
      di.bat = -1;
      std::vector<double> qd(T, 2.0 * net->gen_a[g] + rd);   // 2 a + rho' on every step (all are power)
      ok = spd_inverse(rr, qd, rd, minv);
      // the register path's factor: M = (qd + 2 omega) I + 2 omega D'D
      di.piv = (int)piv.size();
      tri_pivots(T, qd[0] + 4.0 * rd, qd[0] + 6.0 * rd, -2.0 * rd, piv);
      for (int t = 0; t < T; ++t) qv.push_back((float)net->gen_b[g]);
      hoff += rr.m;
      kind[g] = 1;
      d->ramp_gens.push_back(g);
      d->ramp.push_back(net->gen_ramp[g]);
      d->idev.push_back(di);
    }
  }
  if (B > 0 && ok) {
    std::map<double, std::pair<int, int>> by_eff;   // eff -> (shape, minv offset)
    for (int bt = 0; bt < B && ok; ++bt) {
      const double eff = net->stor_eff[bt];
      auto it = by_eff.find(eff);
      const Rows rs = storage_shape(T, eff);
      if (it == by_eff.end()) {
        const int sh = add_shape(rs);
        const int mo = (int)minv.size();
        std::vector<double> qd(rs.n, 0.0);
        for (int t = 0; t < T; ++t) qd[t] = rd;       // rho' on the power entries
        ok = spd_inverse(rs, qd, rd, minv);
        it = by_eff.emplace(eff, std::make_pair(sh, mo)).first;
      }
      IDev di{};
      di.piv = (int)piv.size();
      stor_factor(T, rd, eff, piv);
      di.dev = G + D + bt;
      di.shape = it->second.first;
      di.minv = it->second.second;
      di.h = hoff;
      di.q = (int)qv.size();
      di.bat = bt;
      for (int j = 0; j < rs.n; ++j) qv.push_back((j >= 2 * T && j < 3 * T) ? (float)net->stor_cost[bt] : 0.f);
      hoff += rs.m;
      kind[G + D + bt] = 1;
      d->idev.push_back(di);
    }
  }
  if (!ok) {
    delete d;
    return dfail(OPF_EINVAL, "diff: an inner-ADMM system matrix is not positive definite");
  }
  d->Mtot = hoff;
  d->sP.assign(net->stor_P, net->stor_P + B);
  d->sdur.assign(net->stor_dur, net->stor_dur + B);
  d->scost.resize(B);
  for (int bt = 0; bt < B; ++bt) d->scost[bt] = (float)net->stor_cost[bt];
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the inverse joins the staged structure while the reverse kernel's shared
  // memory stays within 100 KB (two CTAs per SM); the structure alone while
  // it fits; longer horizons read both from global memory
  {
    size_t with2 = 0, with1 = 0;
    for (const Shape &s : shapes) {
      with2 = std::max(with2, bwd_inner_smem(T, s.n, s.m, s.nnz, 2));
      with1 = std::max(with1, std::max(bwd_inner_smem(T, s.n, s.m, s.nnz, 1), fwd_inner_smem(T, s.n, s.m, s.nnz, 1)));
    }
    d->stage = with2 <= 100 * 1024 ? 2 : (e == cudaSuccess && with1 <= (size_t)smem_max ? 1 : 0);
  }
  for (const Shape &s : shapes) {
    d->smem_fwd = std::max(d->smem_fwd, fwd_inner_smem(T, s.n, s.m, s.nnz, d->stage));
    d->smem_bwd = std::max(d->smem_bwd, bwd_inner_smem(T, s.n, s.m, s.nnz, d->stage));
  }
  if (e == cudaSuccess && (d->smem_bwd > (size_t)smem_max || d->smem_fwd > (size_t)smem_max)) {
    delete d;
    return dfail(OPF_EINVAL, "diff: the horizon is too long for one inner-ADMM device per CTA");
  }
  if (e == cudaSuccess && d->smem_fwd)
    e = cudaFuncSetAttribute(fwd_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem_fwd);
  if (e == cudaSuccess && d->smem_bwd)
    e = cudaFuncSetAttribute(bwd_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem_bwd);
  DP &p = d->p;
  p.N = N;
  p.L = L;
  p.T = T;
  p.Kp = d->Kp;
  p.G = G;
  p.D = D;
  p.B = B;
  p.H = H;
  p.S = d->S;
  p.rp = (float)rho_p;
  p.rt = (float)rho_theta;
  p.rd = (float)rd;
  p.n_inner = (int)d->idev.size();
  p.Mtot = d->Mtot;
  auto U = [&](auto **dst, const auto &v) {
    if (e == cudaSuccess) e = up(d->allocs, dst, v);
  };
  U(&p.n1, n1);
  U(&p.n2, n2);
  U(&p.b, b);
  U(&p.out, outl);
  U(&p.lptr, lptr);
  U(&p.lcode, lcode);
  U(&p.dptr, dptr);
  U(&p.didx, didx);
  U(&p.cnt, cnt);
  U(&p.cth, cth);
  {
    std::vector<float> ic(N), ih(N), lf(3 * (size_t)L);
    for (int n = 0; n < N; ++n) {
      ic[n] = (float)(1.0 / cnt[n]);
      ih[n] = cth[n] > 0.f ? (float)(1.0 / cth[n]) : 0.f;
    }
    for (int l = 0; l < L; ++l) {
      const double bl = b[l], tb = 2.0 * bl, den = 2.0 * rho_p + rho_theta / (tb * bl);
      lf[l] = (float)(1.0 / tb);
      lf[L + l] = (float)(rho_p / den);
      lf[2 * (size_t)L + l] = (float)(rho_theta / (tb * den));
    }
    U(&p.icnt, ic);
    U(&p.icth, ih);
    U(&p.lfac, lf);
  }
  U(&p.dnode, dnode);
  U(&p.kind, kind);
  {
    std::vector<unsigned char> hasin(N, 0);
    for (int s2 = 0; s2 < d->S; ++s2)
      if (kind[s2] == 1) hasin[dnode[s2]] = 1;
    std::vector<int> inode;
    for (int n = 0; n < N; ++n)
      if (hasin[n]) inode.push_back(n);
    p.n_inode = (int)inode.size();
    U(&p.hasin, hasin);
    U(&p.inode, inode);
  }
  U(&p.ga, d->ga);
  U(&p.gb, d->gb);
  U(&p.gpmin, gpmin);
  U(&p.voll, d->voll);
  U(&p.idev, d->idev);
  U(&p.shape, shapes);
  U(&p.arp, arp);
  U(&p.aci, aci);
  U(&p.acv, acv);
  U(&p.atp, atp);
  U(&p.ati, ati);
  U(&p.atv, atv);
  U(&p.aeq, aeq);
  U(&p.minv, minv);
  U(&p.Q, qv);
  U(&p.piv, piv);
  {
    std::vector<float> be(B);
    for (int bt = 0; bt < B; ++bt) be[bt] = (float)net->stor_eff[bt];
    U(&p.beff, be);
  }
  p.reg_c = T <= DREG_T ? (T + 32) / 32 : 0;   // chunk of T + 1 elements over 32 lanes
  U(&p.scost, d->scost);
  std::vector<float> hu(H);
  for (int h = 0; h < H; ++h) hu[h] = (float)net->hvdc_u[h];
  U(&p.hvdc_u, hu);
  // data arrays, rewritten by every call
  U(&p.load_p, d->load_p);
  U(&p.gpmax, d->gpmax);
  U(&p.lu, d->lu);
  if (e == cudaSuccess) e = dalloc(d->allocs, &d->RH, (size_t)d->Mtot);
  p.RH = d->RH;
  if (e == cudaSuccess) e = dalloc(d->allocs, &d->mask1, inner_record_bytes(p));
  if (e == cudaSuccess && d->Mtot) {
    // right-hand sides of the inner rows; a call rewrites the capacity rows
    // of the ramp-limited generators from its capacity data (set_ramp_rhs)
    std::vector<float> Hh((size_t)d->Mtot);
    for (size_t r = 0; r < d->ramp_gens.size(); ++r) {
      const int g = d->ramp_gens[r];
      std::vector<double> pmd(net->gen_pmax + (size_t)g * T, net->gen_pmax + (size_t)(g + 1) * T);
      ramp_rhs(T, d->gpmin.data() + (size_t)g * T, pmd.data(), d->ramp[r], Hh.data() + d->idev[r].h);
    }
    for (int bt = 0; bt < B; ++bt)
      storage_rhs(T, d->sP[bt], d->sdur[bt], Hh.data() + d->idev[d->ramp_gens.size() + bt].h);
    e = cudaMemcpy(d->RH, Hh.data(), Hh.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    for (void *q : d->allocs) cudaFree(q);
    delete d;
    return dfail(OPF_ECUDA, cudaGetErrorString(e));
  }
  // padded to 64 floats, so that every state in a buffer of states starts on
  // a 256-byte boundary (the line and node kernels move 16-byte rows)
  d->state_floats = (5 * (size_t)d->Kp * L * T + (size_t)d->S * T + 3 * (size_t)d->Kp * N * T + 2 * (size_t)d->Mtot +
                     63) & ~size_t(63);
  *out = d;
  return OPF_OK;
}

}  // extern "C"

namespace {

// grow one of the kept buffers to n floats (contents not kept)
cudaError_t ensure(float **buf, size_t *cap, size_t n) {
  if (*buf && *cap >= n) return cudaSuccess;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(buf), std::max<size_t>(n, 1) * sizeof(float));
  if (e == cudaSuccess) *cap = n;
  return e;
}

opf_status cost_grad(opf_diff *d, int32_t K, int on_device, const float *load_p, const float *gen_pmax,
                     const float *line_u, double *cost, float *g_load, float *g_pmax, float *g_u) {
  if (!d) return dfail(OPF_EINVAL, "diff is NULL");
  if (K < 1) return dfail(OPF_EINVAL, "diff: K must be >= 1");
  const DP &p = d->p;
  const int T = d->T;
  const size_t DT = (size_t)d->D * T, GT = (size_t)d->G * T, L = d->L, BT = (size_t)d->B * T;
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // this call's data (NULL: the network's own, kept on the host)
  if (load_p) DCK(cudaMemcpyAsync(const_cast<float *>(p.load_p), load_p, DT * 4, in_kind, d->stream));
  else DCK(cudaMemcpyAsync(const_cast<float *>(p.load_p), d->load_p.data(), DT * 4, cudaMemcpyHostToDevice, d->stream));
  if (gen_pmax) DCK(cudaMemcpyAsync(const_cast<float *>(p.gpmax), gen_pmax, GT * 4, in_kind, d->stream));
  else DCK(cudaMemcpyAsync(const_cast<float *>(p.gpmax), d->gpmax.data(), GT * 4, cudaMemcpyHostToDevice, d->stream));
  if (line_u) DCK(cudaMemcpyAsync(const_cast<float *>(p.lu), line_u, L * 4, in_kind, d->stream));
  else DCK(cudaMemcpyAsync(const_cast<float *>(p.lu), d->lu.data(), L * 4, cudaMemcpyHostToDevice, d->stream));
  // the capacity rows of the ramp-limited generators' inner problems
  if (p.n_inner) set_ramp_rhs<<<grid_for((long long)p.n_inner * T), TB, 0, d->stream>>>(p, d->RH);
  // states: checkpoints 0, C, 2C, ... and room for a segment's C - 1
  // recomputed states (at least the forward pass's two alternating ones)
  const int C = std::min(d->ckpt, K);
  const int n_ck = K / C + 1;
  const size_t SF = d->state_floats;
  const size_t KLT = (size_t)d->Kp * d->L * T, KNT = (size_t)d->Kp * d->N * T, ST = (size_t)d->S * T;
  const size_t MT = (size_t)d->Mtot;
  const size_t adj_floats = 5 * KLT + ST + KNT + 2 * MT;
  const size_t work_floats = 4 * KLT + 3 * KNT + 4 * ST + DT + GT + MT + BT;
  const bool grads = g_load || g_pmax || g_u;
  size_t adj_cap = d->adj ? adj_floats : 0, work_cap = d->work ? work_floats : 0, gl_cap = d->gline ? L : 0;
  // the forward pass records which inner rows clipped and where each line's
  // and closed-form device's unclipped value lay, so that the reverse pass
  // need not run each iteration's inner ADMM again nor recompute the prox
  // inputs, nor the states (while the record stays within the context's limit)
  const size_t mask_iter = (inner_record_bytes(p) + KLT + ST + 255) & ~size_t(255);
  const bool rec = grads && (size_t)K * mask_iter <= d->record_limit;
  cudaError_t e = ensure(&d->ck, &d->ck_cap, (size_t)n_ck * SF);
  if (e == cudaSuccess) e = ensure(&d->seg, &d->seg_cap, (size_t)(grads && !rec ? std::max(C, 2) : 2) * SF);
  if (e == cudaSuccess) e = ensure(&d->adj, &adj_cap, adj_floats);
  if (e == cudaSuccess) e = ensure(&d->work, &work_cap, work_floats);
  if (e == cudaSuccess) e = ensure(&d->gline, &gl_cap, L);
  if (e == cudaSuccess && rec) e = ensure(&d->masks, &d->masks_cap, ((size_t)K * mask_iter + 3) / 4);
  if (e != cudaSuccess)
    return dfail(e == cudaErrorMemoryAllocation ? OPF_ENOMEM : OPF_ECUDA, "diff: device allocation failed");
  unsigned char *masks = rec ? reinterpret_cast<unsigned char *>(d->masks) : nullptr;
  auto mask_of = [&](int i) { return masks ? masks + (size_t)(i - 1) * mask_iter : nullptr; };   // iteration i
  float *ck = d->ck, *seg = d->seg, *adj = d->adj, *work = d->work;
  float *X2 = work, *Y1 = X2 + KLT, *Y2 = Y1 + KLT, *GU = Y2 + KLT;
  float *Bn = GU + KLT, *Cn = Bn + KNT, *Dn = Cn + KNT, *LX0 = Dn + KNT, *LX1 = LX0 + ST, *XD = LX1 + ST;
  float *LPDT = XD + ST, *GL = LPDT + ST, *GP = GL + DT, *HB = GP + GT, *DEL = HB + MT;
  auto ckst = [&](int j) { return carve_state(d, ck + (size_t)j * SF); };
  auto sgst = [&](int j) { return carve_state(d, seg + (size_t)j * SF); };
  // forward, keeping checkpoints
  e = cudaMemsetAsync(ck, 0, SF * 4, d->stream);
  St cur = ckst(0);
  float *scratch = seg;  // two alternating states in the segment buffer
  for (int i = 1; e == cudaSuccess && i <= K; ++i) {
    St nx = (i % C == 0) ? ckst(i / C) : carve_state(d, scratch + (size_t)(i & 1) * SF);
    forward_step(d, cur, nx, XD, DEL, mask_of(i));
    cur = nx;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  std::vector<float> pd(ST), del(BT), lp(DT);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pd.data(), cur.PD, ST * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess && BT) e = cudaMemcpyAsync(del.data(), DEL, BT * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess && DT) e = cudaMemcpyAsync(lp.data(), p.load_p, DT * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) return dfail(OPF_ECUDA, cudaGetErrorString(e));
  if (cost) {
    double f = 0.0;
    for (int g = 0; g < d->G; ++g)
      for (int t = 0; t < T; ++t) {
        const double x = pd[(size_t)g * T + t];
        f += d->ga[g] * x * x + d->gb[g] * x;
      }
    for (int k = 0; k < d->D; ++k) {
      if (d->voll[k] < 0) continue;
      for (int t = 0; t < T; ++t)
        f += (double)d->voll[k] * ((double)pd[(size_t)(d->G + k) * T + t] + lp[(size_t)k * T + t]);
    }
    for (int bt = 0; bt < d->B; ++bt)
      for (int t = 0; t < T; ++t) f += (double)d->scost[bt] * del[(size_t)bt * T + t];
    *cost = f;
  }
  if (!grads) return OPF_OK;
  {
    cudaError_t ce = cudaSuccess;
    if (!d->aux) ce = cudaStreamCreateWithFlags(&d->aux, cudaStreamNonBlocking);
    if (ce == cudaSuccess && !d->ev_fork) ce = cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess && !d->ev_join) ce = cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming);
    if (ce != cudaSuccess) return dfail(OPF_ECUDA, cudaGetErrorString(ce));
  }
  // reverse pass
  Adj a;
  a.LP = adj;
  a.LT1 = a.LP + KLT;
  a.LT2 = a.LT1 + KLT;
  a.LV1 = a.LT2 + KLT;
  a.LV2 = a.LV1 + KLT;
  a.LPD = a.LV2 + KLT;
  a.LU = a.LPD + ST;
  a.LINS = a.LU + KNT;
  e = cudaMemsetAsync(adj, 0, adj_floats * 4, d->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(GU, 0, KLT * 4, d->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(GL, 0, (DT + GT + MT) * 4, d->stream);
  if (e == cudaSuccess) bwd_init<<<grid_for((long long)ST), TB, 0, d->stream>>>(p, cur, a, GL);
  const long long nl = (long long)KLT, nn = (long long)KNT, ns = (long long)ST;
  // d/d pbar' is u's adjoint itself (u' = u + pbar'), read before bwd_node2 or
  // bwd_node3 adds the iteration's increment to it
  const float *A = a.LU;
  const bool v4 = T % 4 == 0;   // four steps per thread in the line and node kernels
  bool primed = false;   // iteration i's first half already ran, fused into iteration i+1's second half
  for (int hi = K; e == cudaSuccess && hi > 0;) {
    // segment (lo, hi]: states lo + 1 .. hi - 1 recomputed from checkpoint lo
    // (read in place).  With the record the reverse pass reads no state (the
    // clips, and the inner rows that clipped, are all it needs), so nothing
    // is recomputed and every kernel is handed checkpoint lo, unread.
    const int lo = ((hi - 1) / C) * C;
    auto state = [&](int j) { return (j == lo || masks) ? ckst(lo / C) : sgst(j - lo); };   // state j, lo <= j < hi
    for (int i = lo + 1; e == cudaSuccess && !masks && i < hi; ++i)
      forward_step(d, state(i - 1), sgst(i - lo), XD, DEL);
    for (int i = hi; e == cudaSuccess && i > lo; --i) {
      const St s = state(i - 1);
      unsigned char *mi = mask_of(i);
      float *LX = (i & 1) ? LX1 : LX0, *LXn = (i & 1) ? LX0 : LX1;   // d/dX of iterations i and i - 1
      if (!primed) {
        const unsigned char *lmask = mi ? mi + inner_record_bytes(p) : nullptr, *dmask = mi ? lmask + KLT : nullptr;
        if (v4) {
          bwd_node1<4><<<grid_for(nn / 4), TB, 0, d->stream>>>(p, a, Bn);
          bwd_line1<4><<<grid_for(nl / 4), TB, 0, d->stream>>>(p, s, a, A, Bn, X2, Y1, Y2, GU, lmask);
        } else {
          bwd_node1<1><<<grid_for(nn), TB, 0, d->stream>>>(p, a, Bn);
          bwd_line1<1><<<grid_for(nl), TB, 0, d->stream>>>(p, s, a, A, Bn, X2, Y1, Y2, GU, lmask);
        }
        if (v4) bwd_dev<4><<<grid_for(ns / 4 * KL), TB, 0, d->stream>>>(p, s, a, A, LX, GL, GP, XD, LPDT, dmask);
        else bwd_dev<1><<<grid_for(ns * KL), TB, 0, d->stream>>>(p, s, a, A, LX, GL, GP, XD, LPDT, dmask);
      }
      // iteration i - 1's first half joins this second half when what it
      // reads is at hand: its record, or its input state i - 2 in this segment
      unsigned char *mp = i > 1 ? mask_of(i - 1) : nullptr;
      const int nxt = i > 1 && (mp || i - 2 >= lo) ? 1 : 0;
      // the node gathers beside the inner ADMM (at the nodes with its devices,
      // only the line terms; bwd_node3 adds the device terms after it)
      if (e == cudaSuccess) e = cudaEventRecord(d->ev_fork, d->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(d->aux, d->ev_fork, 0);
      if (e != cudaSuccess) break;
      if (v4) bwd_node2<4><<<grid_for(nn / 4), TB, 0, d->aux>>>(p, a, X2, Y1, Y2, LX, Cn, Dn, Bn, nxt);
      else bwd_node2<1><<<grid_for(nn), TB, 0, d->aux>>>(p, a, X2, Y1, Y2, LX, Cn, Dn, Bn, nxt);
      e = cudaEventRecord(d->ev_join, d->aux);
      if (p.n_inner) {
        const int g = (p.n_inner + RWARPS - 1) / RWARPS, lst = i == K ? 1 : 0;
        unsigned long long *m1 = reinterpret_cast<unsigned long long *>(d->mask1);
        const unsigned long long *rr = reinterpret_cast<const unsigned long long *>(mi);
        switch (p.reg_c) {
          case 1: bwd_inner_r<1><<<g, TB, 0, d->stream>>>(p, s, a, XD, LPDT, LX, HB, lst, rr, m1); break;
          case 2: bwd_inner_r<2><<<g, TB, 0, d->stream>>>(p, s, a, XD, LPDT, LX, HB, lst, rr, m1); break;
          case 3: bwd_inner_r<3><<<g, TB, 0, d->stream>>>(p, s, a, XD, LPDT, LX, HB, lst, rr, m1); break;
          case 4: bwd_inner_r<4><<<g, TB, 0, d->stream>>>(p, s, a, XD, LPDT, LX, HB, lst, rr, m1); break;
          default:
            bwd_inner<<<p.n_inner, TBI, d->smem_bwd, d->stream>>>(p, s, a, XD, LPDT, LX, HB, lst, d->stage, mi);
            break;
        }
      }
      if (e == cudaSuccess) e = cudaStreamWaitEvent(d->stream, d->ev_join, 0);
      if (e != cudaSuccess) break;
      const St sp = nxt && i - 2 >= lo ? state(i - 2) : s;   // read only without a record
      const unsigned char *lmp = mp ? mp + inner_record_bytes(p) : nullptr, *dmp = mp ? lmp + KLT : nullptr;
      const long long ni3 = (long long)p.Kp * p.n_inode * T;   // items of the nodes with inner-ADMM devices
      if (ni3 && v4) bwd_node3<4><<<grid_for(ni3 / 4), TB, 0, d->stream>>>(p, a, LX, Cn);
      else if (ni3) bwd_node3<1><<<grid_for(ni3), TB, 0, d->stream>>>(p, a, LX, Cn);
      {
        const Scatter g{Cn, Dn, A, Bn, LX, X2, Y1, Y2, GU, LXn, GL, GP, XD, LPDT, lmp, dmp};
        const int db = grid_for(ns / (v4 ? 4 : 1) * KL);
        if (v4) bwd_scatter<4><<<db + grid_for(nl / 4), TB, 0, d->stream>>>(p, sp, a, g, nxt, db);
        else bwd_scatter<1><<<db + grid_for(nl), TB, 0, d->stream>>>(p, sp, a, g, nxt, db);
      }
      primed = nxt != 0;
    }
    hi = lo;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && g_pmax && p.n_inner)
    finish_cap_grad<<<grid_for((long long)p.n_inner * T), TB, 0, d->stream>>>(p, HB, GP);
  if (e == cudaSuccess && g_u) finish_line_grad<<<grid_for((long long)L), TB, 0, d->stream>>>(p, GU, d->gline);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && g_load) e = cudaMemcpyAsync(g_load, GL, DT * 4, out_kind, d->stream);
  if (e == cudaSuccess && g_pmax) e = cudaMemcpyAsync(g_pmax, GP, GT * 4, out_kind, d->stream);
  if (e == cudaSuccess && g_u) e = cudaMemcpyAsync(g_u, d->gline, L * 4, out_kind, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    // a failed fork or join may leave work queued on the second stream
    cudaStreamSynchronize(d->stream);
    cudaStreamSynchronize(d->aux);
    return dfail(OPF_ECUDA, cudaGetErrorString(e));
  }
  return OPF_OK;
}

}  // namespace

extern "C" {

opf_status opf_diff_cost_grad(opf_diff *d, int32_t K, const float *load_p, const float *gen_pmax,
                              const float *line_u, double *cost, float *g_load, float *g_pmax, float *g_u) {
  return cost_grad(d, K, 0, load_p, gen_pmax, line_u, cost, g_load, g_pmax, g_u);
}

opf_status opf_diff_cost_grad_on(opf_diff *d, int32_t K, int32_t on_device, const float *load_p,
                                 const float *gen_pmax, const float *line_u, double *cost, float *g_load,
                                 float *g_pmax, float *g_u) {
  return cost_grad(d, K, on_device ? 1 : 0, load_p, gen_pmax, line_u, cost, g_load, g_pmax, g_u);
}

opf_status opf_diff_set_record_limit(opf_diff *d, int64_t bytes) {
  if (!d) return dfail(OPF_EINVAL, "diff is NULL");
  if (bytes < 0) return dfail(OPF_EINVAL, "diff: the record limit must be >= 0");
  d->record_limit = (size_t)bytes;
  return OPF_OK;
}

void opf_diff_destroy(opf_diff *d) {
  if (!d) return;
  cudaStreamSynchronize(d->stream);
  if (d->aux) cudaStreamSynchronize(d->aux);
  if (d->ev_fork) cudaEventDestroy(d->ev_fork);
  if (d->ev_join) cudaEventDestroy(d->ev_join);
  if (d->aux) cudaStreamDestroy(d->aux);
  for (void *q : d->allocs) cudaFree(q);
  for (float *q : {d->ck, d->seg, d->adj, d->work, d->gline, d->masks})
    if (q) cudaFree(q);
  delete d;
}

}  // extern "C"
