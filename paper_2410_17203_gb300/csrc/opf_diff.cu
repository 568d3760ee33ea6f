// Gradients of the system cost after K unrolled iterations (include/opf_diff.h).
//
// A self-contained differentiable path in the caller's numbering: the state
// (p, theta1, theta2, v1, v2 per line and contingency; device power; u, and
// the node averages pbar, theta_bar per node and contingency) is kept in
// plain arrays, and every step of the iteration has a forward kernel and an
// adjoint kernel.  Forward states are stored every `checkpoint_every`
// iterations and recomputed segment by segment during the reverse pass.
// Every adjoint item writes only its own entries (sums over a node's
// terminals are CSR gathers), so the gradients are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "opf_diff.h"
#include "opf_internal.h"

namespace {

constexpr int TB = 256;

struct DP {
  int N, L, T, Kp, G, D, S;
  float rp, rt, rd;                    // rho_p, rho_theta, (K+1) rho_p
  const int *n1, *n2;                  // line ends (terminal 1 at n1 carries -p)
  const float *b;                      // susceptance [L]
  const int *out;                      // [Kp] outaged line, -1 = none
  const int *lptr, *lcode;             // node -> line terminal codes 2 l + end (end 1: terminal 2)
  const int *dptr, *didx;              // node -> devices
  const float *cnt, *cth;              // terminals at a node: all, line (0: none)
  const int *dnode;                    // device node [S]
  const float *ga, *gb, *gpmin;        // generators: a, b [G]; pmin [G][T]
  const float *voll;                   // loads [D], < 0: fixed
  const float *load_p, *gpmax, *lu;    // data: [D][T], [G][T], [L]
};

struct St {
  float *P, *TH1, *TH2, *V1, *V2, *PD, *U, *PB, *TBR;
};

struct Adj {
  float *LP, *LT1, *LT2, *LV1, *LV2, *LPD, *LU;
};

__device__ __forceinline__ size_t li(const DP &p, int k, int l, int t) { return ((size_t)k * p.L + l) * p.T + t; }
__device__ __forceinline__ size_t ni(const DP &p, int k, int n, int t) { return ((size_t)k * p.N + n) * p.T + t; }

#define GRID_STRIDE(i, n) for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < (n); i += (long long)gridDim.x * TB)

// ---------------------------------------------------------------------------
// forward (Section 3.2)
// ---------------------------------------------------------------------------

// node averages (Eq. average-op) of the terminal values of a state
__global__ void fwd_avg(DP p, St s) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * p.T) {
    const int t = (int)(i % p.T), n = (int)((i / p.T) % p.N), k = (int)(i / ((long long)p.T * p.N));
    float sp = 0.f, st = 0.f;
    for (int j = p.dptr[n]; j < p.dptr[n + 1]; ++j) sp += s.PD[(size_t)p.didx[j] * p.T + t];
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j], l = c >> 1;
      const float v = s.P[li(p, k, l, t)];
      sp += (c & 1) ? v : -v;
      st += (c & 1) ? s.TH2[li(p, k, l, t)] : s.TH1[li(p, k, l, t)];
    }
    s.PB[i] = sp / p.cnt[n];
    s.TBR[i] = p.cth[n] > 0.f ? st / p.cth[n] : 0.f;
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

// step 1: line prox (Section 4.2); outaged lines decouple
__global__ void fwd_line(DP p, St s, St nx) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * p.T) {
    const int t = (int)(i % p.T), l = (int)((i / p.T) % p.L), k = (int)(i / ((long long)p.T * p.L));
    const LineIn in = line_inputs(p, s, k, l, t);
    if (p.out[k] != l) {
      const float b = p.b[l], tb = 2.f * b, u = p.lu[l];
      const float den = 2.f * p.rp + p.rt / (tb * b);
      const float z = (p.rp * (in.x2 - in.x1) + p.rt * (in.y1 - in.y2) / tb) / den;
      const float p2 = fminf(fmaxf(z, -u), u);
      const float mid = 0.5f * (in.y1 + in.y2);
      nx.P[i] = p2;
      nx.TH1[i] = mid + p2 / tb;
      nx.TH2[i] = mid - p2 / tb;
    } else {
      nx.P[i] = 0.f;
      nx.TH1[i] = in.y1;
      nx.TH2[i] = in.y2;
    }
  }
}

__device__ __forceinline__ float dev_x(const DP &p, const St &s, int d, int t) {
  const int n = p.dnode[d];
  float sum = 0.f;
  for (int k = 0; k < p.Kp; ++k) sum += s.PB[ni(p, k, n, t)] + s.U[ni(p, k, n, t)];
  return s.PD[(size_t)d * p.T + t] - sum / (float)p.Kp;   // p_d - avg_k(pbar + u)
}

// step 2: devices shared by all contingencies, weight (K+1) rho_p
__global__ void fwd_dev(DP p, St s, St nx) {
  GRID_STRIDE(i, (long long)p.S * p.T) {
    const int t = (int)(i % p.T), d = (int)(i / p.T);
    const float X = dev_x(p, s, d, t);
    float r;
    if (d < p.G) {
      const float z = (p.rd * X - p.gb[d]) / (2.f * p.ga[d] + p.rd);
      r = fminf(fmaxf(z, p.gpmin[i]), p.gpmax[i]);
    } else {
      const int e = d - p.G;
      const size_t o = (size_t)e * p.T + t;
      if (p.voll[e] < 0.f) r = -p.load_p[o];
      else r = fminf(fmaxf((p.rd * X - p.voll[e]) / p.rd, -p.load_p[o]), 0.f);
    }
    nx.PD[i] = r;
  }
}

// step 3: u += pbar, v += theta - theta_bar (after fwd_avg of the new state)
__global__ void fwd_upd_nodes(DP p, St s, St nx) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * p.T) nx.U[i] = s.U[i] + nx.PB[i];
}

__global__ void fwd_upd_lines(DP p, St s, St nx) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * p.T) {
    const int t = (int)(i % p.T), l = (int)((i / p.T) % p.L), k = (int)(i / ((long long)p.T * p.L));
    nx.V1[i] = s.V1[i] + nx.TH1[i] - nx.TBR[ni(p, k, p.n1[l], t)];
    nx.V2[i] = s.V2[i] + nx.TH2[i] - nx.TBR[ni(p, k, p.n2[l], t)];
  }
}

// ---------------------------------------------------------------------------
// reverse pass of one iteration: the adjoint of state i in `a` becomes the
// adjoint of state i-1; s is state i-1
// ---------------------------------------------------------------------------

// adjoints of the new node averages through u' = u + pbar' and
// v' = v + theta' - theta_bar': A = d/d pbar', B = d/d theta_bar'
__global__ void bwd_node1(DP p, Adj a, float *A, float *B) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * p.T) {
    const int t = (int)(i % p.T), n = (int)((i / p.T) % p.N), k = (int)(i / ((long long)p.T * p.N));
    float s = 0.f;
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j];
      s += (c & 1) ? a.LV2[li(p, k, c >> 1, t)] : a.LV1[li(p, k, c >> 1, t)];
    }
    A[i] = a.LU[i];
    B[i] = -s;
  }
}

// the line prox backwards; X1.. hold d/d(x1, x2, y1, y2) for the node gathers
__global__ void bwd_line1(DP p, St s, Adj a, const float *A, const float *B, float *X1, float *X2, float *Y1,
                          float *Y2, float *GU) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * p.T) {
    const int t = (int)(i % p.T), l = (int)((i / p.T) % p.L), k = (int)(i / ((long long)p.T * p.L));
    const int n1 = p.n1[l], n2 = p.n2[l];
    const size_t o1 = ni(p, k, n1, t), o2 = ni(p, k, n2, t);
    const float lp = a.LP[i] - A[o1] / p.cnt[n1] + A[o2] / p.cnt[n2];
    const float lt1 = a.LT1[i] + a.LV1[i] + (p.cth[n1] > 0.f ? B[o1] / p.cth[n1] : 0.f);
    const float lt2 = a.LT2[i] + a.LV2[i] + (p.cth[n2] > 0.f ? B[o2] / p.cth[n2] : 0.f);
    float lx1 = 0.f, lx2 = 0.f, ly1, ly2;
    if (p.out[k] != l) {
      const LineIn in = line_inputs(p, s, k, l, t);
      const float b = p.b[l], tb = 2.f * b, u = p.lu[l];
      const float den = 2.f * p.rp + p.rt / (tb * b);
      const float z = (p.rp * (in.x2 - in.x1) + p.rt * (in.y1 - in.y2) / tb) / den;
      const float lpt = lp + (lt1 - lt2) / tb;     // theta_{1,2} = mid +- p / (2b)
      ly1 = ly2 = 0.5f * (lt1 + lt2);
      if (z >= -u && z <= u) {
        lx2 = p.rp * lpt / den;
        lx1 = -lx2;
        const float w = p.rt * lpt / (tb * den);
        ly1 += w;
        ly2 -= w;
      } else {
        GU[i] += z > u ? lpt : -lpt;
      }
    } else {
      ly1 = lt1;
      ly2 = lt2;
    }
    X1[i] = lx1;
    X2[i] = lx2;
    Y1[i] = ly1;
    Y2[i] = ly2;
    a.LP[i] = lx2 - lx1;                 // x1 = -p - ..., x2 = p - ...
    a.LV1[i] -= ly1;                     // v enters y = theta_bar - v, and v' = v + ...
    a.LV2[i] -= ly2;
  }
}

// the device proxes backwards; LX = d/dX per device
__global__ void bwd_dev(DP p, St s, Adj a, const float *A, float *LX, float *GL, float *GP) {
  GRID_STRIDE(i, (long long)p.S * p.T) {
    const int t = (int)(i % p.T), d = (int)(i / p.T), n = p.dnode[d];
    float lpd = a.LPD[i];
    for (int k = 0; k < p.Kp; ++k) lpd += A[ni(p, k, n, t)] / p.cnt[n];
    const float X = dev_x(p, s, d, t);
    float lx = 0.f;
    if (d < p.G) {
      const float den = 2.f * p.ga[d] + p.rd;
      const float z = (p.rd * X - p.gb[d]) / den;
      if (z >= p.gpmin[i] && z <= p.gpmax[i]) lx = lpd * p.rd / den;
      else if (z > p.gpmax[i]) GP[i] += lpd;
    } else {
      const int e = d - p.G;
      const size_t o = (size_t)e * p.T + t;
      if (p.voll[e] < 0.f) {
        GL[o] -= lpd;                    // p = -P
      } else {
        const float z = (p.rd * X - p.voll[e]) / p.rd;
        if (z >= -p.load_p[o] && z <= 0.f) lx = lpd;
        else if (z < -p.load_p[o]) GL[o] -= lpd;
      }
    }
    LX[i] = lx;
  }
}

// gathers at the nodes: C = d/d pbar (old), D = d/d theta_bar (old); u's adjoint
__global__ void bwd_node2(DP p, Adj a, const float *X1, const float *X2, const float *Y1, const float *Y2,
                          const float *LX, float *C, float *Dt) {
  GRID_STRIDE(i, (long long)p.Kp * p.N * p.T) {
    const int t = (int)(i % p.T), n = (int)((i / p.T) % p.N), k = (int)(i / ((long long)p.T * p.N));
    float sx = 0.f, sy = 0.f, sd = 0.f;
    for (int j = p.lptr[n]; j < p.lptr[n + 1]; ++j) {
      const int c = p.lcode[j];
      const size_t o = li(p, k, c >> 1, t);
      sx += (c & 1) ? X2[o] : X1[o];
      sy += (c & 1) ? Y2[o] : Y1[o];
    }
    for (int j = p.dptr[n]; j < p.dptr[n + 1]; ++j) sd += LX[(size_t)p.didx[j] * p.T + t];
    sd /= (float)p.Kp;
    C[i] = -sx - sd;                     // x = ... - pbar - u, X = ... - avg_k(pbar + u)
    a.LU[i] += -sx - sd;
    Dt[i] = sy;                          // y = theta_bar - v
  }
}

// the old node averages back onto the old line values and device powers
__global__ void bwd_line2(DP p, Adj a, const float *C, const float *Dt) {
  GRID_STRIDE(i, (long long)p.Kp * p.L * p.T) {
    const int t = (int)(i % p.T), l = (int)((i / p.T) % p.L), k = (int)(i / ((long long)p.T * p.L));
    const int n1 = p.n1[l], n2 = p.n2[l];
    const size_t o1 = ni(p, k, n1, t), o2 = ni(p, k, n2, t);
    a.LP[i] += -C[o1] / p.cnt[n1] + C[o2] / p.cnt[n2];
    a.LT1[i] = p.cth[n1] > 0.f ? Dt[o1] / p.cth[n1] : 0.f;
    a.LT2[i] = p.cth[n2] > 0.f ? Dt[o2] / p.cth[n2] : 0.f;
  }
}

__global__ void bwd_dev2(DP p, Adj a, const float *LX, const float *C) {
  GRID_STRIDE(i, (long long)p.S * p.T) {
    const int t = (int)(i % p.T), d = (int)(i / p.T), n = p.dnode[d];
    float s = LX[i];
    for (int k = 0; k < p.Kp; ++k) s += C[ni(p, k, n, t)] / p.cnt[n];
    a.LPD[i] = s;
  }
}

// d f / d p_d at the last iterate, and f's direct dependence on P
__global__ void bwd_init(DP p, St s, Adj a, float *GL) {
  GRID_STRIDE(i, (long long)p.S * p.T) {
    const int t = (int)(i % p.T), d = (int)(i / p.T);
    if (d < p.G) {
      a.LPD[i] = 2.f * p.ga[d] * s.PD[i] + p.gb[d];
    } else {
      const int e = d - p.G;
      a.LPD[i] = p.voll[e] < 0.f ? 0.f : p.voll[e];
      if (p.voll[e] >= 0.f) GL[(size_t)e * p.T + t] = p.voll[e];
    }
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + TB - 1) / TB, 8192)); }

}  // namespace

struct opf_diff {
  int N = 0, L = 0, T = 0, Kp = 0, G = 0, D = 0, S = 0, ckpt = 1;
  cudaStream_t stream = nullptr;
  DP p{};
  std::vector<float> ga, gb, voll, load_p, gpmax, lu;  // host copies (cost and defaults)
  std::vector<void *> allocs;
  size_t state_floats = 0;
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
  s.TBR = c;
  return s;
}

void forward_step(const opf_diff *d, const St &s, const St &nx) {
  const DP &p = d->p;
  const long long nl = (long long)p.Kp * p.L * p.T, nn = (long long)p.Kp * p.N * p.T, ns = (long long)p.S * p.T;
  fwd_line<<<grid_for(nl), TB, 0, d->stream>>>(p, s, nx);
  fwd_dev<<<grid_for(ns), TB, 0, d->stream>>>(p, s, nx);
  fwd_avg<<<grid_for(nn), TB, 0, d->stream>>>(p, nx);
  fwd_upd_nodes<<<grid_for(nn), TB, 0, d->stream>>>(p, s, nx);
  fwd_upd_lines<<<grid_for(nl), TB, 0, d->stream>>>(p, s, nx);
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
  const int N = net->n_nodes, L = net->n_lines, G = net->n_gens, D = net->n_loads;
  if (N < 1 || L < 0 || G < 0 || D < 0) return dfail(OPF_EINVAL, "diff: bad sizes");
  if (net->n_stor > 0) return dfail(OPF_EINVAL, "diff: batteries are not covered (closed-form devices only)");
  for (int g = 0; g < G; ++g)
    if (net->gen_ramp && net->gen_ramp[g] >= 0 && T > 1)
      return dfail(OPF_EINVAL, "diff: ramp-limited generators are not covered (closed-form devices only)");
  const int K = ctg ? ctg->K : 0;
  for (int l = 0; l < L; ++l) {
    const int a = net->line_from[l], c = net->line_to[l];
    if (a < 0 || a >= N || c < 0 || c >= N || a == c || !(net->line_b[l] > 0))
      return dfail(OPF_EINVAL, "diff: bad line");
  }
  for (int k = 0; k < K; ++k)
    if (ctg->outaged_line[k] < -1 || ctg->outaged_line[k] >= L)
      return dfail(OPF_EINVAL, "diff: outaged line id out of range");
  auto *d = new (std::nothrow) opf_diff();
  if (!d) return dfail(OPF_ENOMEM, "host allocation failed");
  d->N = N;
  d->L = L;
  d->T = T;
  d->Kp = K + 1;
  d->G = G;
  d->D = D;
  d->S = G + D;
  d->ckpt = checkpoint_every;
  d->stream = (cudaStream_t)cuda_stream;
  // incidence by node (caller's numbering)
  std::vector<int> lptr(N + 1, 0), lcode(2 * (size_t)L), dptr(N + 1, 0), didx(d->S), dnode(d->S);
  std::vector<float> cnt(N, 0.f), cth(N, 0.f);
  for (int l = 0; l < L; ++l) {
    ++lptr[net->line_from[l] + 1];
    ++lptr[net->line_to[l] + 1];
  }
  for (int g = 0; g < G; ++g) dnode[g] = net->gen_node[g];
  for (int e = 0; e < D; ++e) dnode[G + e] = net->load_node[e];
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
  DP &p = d->p;
  p.N = N;
  p.L = L;
  p.T = T;
  p.Kp = d->Kp;
  p.G = G;
  p.D = D;
  p.S = d->S;
  p.rp = (float)rho_p;
  p.rt = (float)rho_theta;
  p.rd = (float)(d->Kp * rho_p);
  cudaError_t e = cudaSuccess;
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
  U(&p.dnode, dnode);
  U(&p.ga, d->ga);
  U(&p.gb, d->gb);
  U(&p.gpmin, gpmin);
  U(&p.voll, d->voll);
  // data arrays, rewritten by every call
  U(&p.load_p, d->load_p);
  U(&p.gpmax, d->gpmax);
  U(&p.lu, d->lu);
  if (e != cudaSuccess) {
    for (void *q : d->allocs) cudaFree(q);
    delete d;
    return dfail(OPF_ECUDA, cudaGetErrorString(e));
  }
  d->state_floats = 5 * (size_t)d->Kp * L * T + (size_t)d->S * T + 3 * (size_t)d->Kp * N * T;
  *out = d;
  return OPF_OK;
}

opf_status opf_diff_cost_grad(opf_diff *d, int32_t K, const float *load_p, const float *gen_pmax,
                              const float *line_u, double *cost, float *g_load, float *g_pmax, float *g_u) {
  if (!d) return dfail(OPF_EINVAL, "diff is NULL");
  if (K < 1) return dfail(OPF_EINVAL, "diff: K must be >= 1");
  const DP &p = d->p;
  const size_t DT = (size_t)d->D * d->T, GT = (size_t)d->G * d->T, L = d->L;
  std::vector<float> lp(load_p ? load_p : d->load_p.data(), (load_p ? load_p : d->load_p.data()) + DT);
  DCK(cudaMemcpyAsync(const_cast<float *>(p.load_p), lp.data(), DT * 4, cudaMemcpyHostToDevice, d->stream));
  DCK(cudaMemcpyAsync(const_cast<float *>(p.gpmax), gen_pmax ? gen_pmax : d->gpmax.data(), GT * 4,
                      cudaMemcpyHostToDevice, d->stream));
  DCK(cudaMemcpyAsync(const_cast<float *>(p.lu), line_u ? line_u : d->lu.data(), L * 4, cudaMemcpyHostToDevice,
                      d->stream));
  // states: checkpoints 0, C, 2C, ... and one segment of C + 1 states
  const int C = std::min(d->ckpt, K);
  const int n_ck = K / C + 1;
  const size_t SF = d->state_floats;
  std::vector<void *> tmp;
  auto release = [&]() {
    for (void *q : tmp) cudaFree(q);
  };
  float *ck = nullptr, *seg = nullptr, *adj = nullptr, *work = nullptr;
  const size_t KLT = (size_t)d->Kp * d->L * d->T, KNT = (size_t)d->Kp * d->N * d->T, ST = (size_t)d->S * d->T;
  cudaError_t e = dalloc(tmp, &ck, (size_t)n_ck * SF);
  if (e == cudaSuccess) e = dalloc(tmp, &seg, (size_t)(C + 1) * SF);
  if (e == cudaSuccess) e = dalloc(tmp, &adj, 5 * KLT + ST + KNT);
  if (e == cudaSuccess) e = dalloc(tmp, &work, 5 * KLT + 4 * KNT + ST + DT + GT);
  if (e != cudaSuccess) {
    release();
    return dfail(e == cudaErrorMemoryAllocation ? OPF_ENOMEM : OPF_ECUDA, "diff: device allocation failed");
  }
  auto ckst = [&](int j) { return carve_state(d, ck + (size_t)j * SF); };
  auto sgst = [&](int j) { return carve_state(d, seg + (size_t)j * SF); };
  // forward, keeping checkpoints
  e = cudaMemsetAsync(ck, 0, SF * 4, d->stream);
  St cur = ckst(0);
  float *scratch = seg;  // two alternating states in the segment buffer
  for (int i = 1; e == cudaSuccess && i <= K; ++i) {
    St nx = (i % C == 0) ? ckst(i / C) : carve_state(d, scratch + (size_t)(i & 1) * SF);
    forward_step(d, cur, nx);
    cur = nx;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  std::vector<float> pd(ST);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pd.data(), cur.PD, ST * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    release();
    return dfail(OPF_ECUDA, cudaGetErrorString(e));
  }
  if (cost) {
    double f = 0.0;
    for (int g = 0; g < d->G; ++g)
      for (int t = 0; t < d->T; ++t) {
        const double x = pd[(size_t)g * d->T + t];
        f += d->ga[g] * x * x + d->gb[g] * x;
      }
    for (int k = 0; k < d->D; ++k) {
      if (d->voll[k] < 0) continue;
      for (int t = 0; t < d->T; ++t)
        f += (double)d->voll[k] * ((double)pd[(size_t)(d->G + k) * d->T + t] + lp[(size_t)k * d->T + t]);
    }
    *cost = f;
  }
  if (!g_load && !g_pmax && !g_u) {
    release();
    return OPF_OK;
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
  float *X1 = work, *X2 = X1 + KLT, *Y1 = X2 + KLT, *Y2 = Y1 + KLT, *GU = Y2 + KLT;
  float *A = GU + KLT, *B = A + KNT, *Cn = B + KNT, *Dn = Cn + KNT, *LX = Dn + KNT, *GL = LX + ST, *GP = GL + DT;
  e = cudaMemsetAsync(adj, 0, (5 * KLT + ST + KNT) * 4, d->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(GU, 0, KLT * 4, d->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(GL, 0, (DT + GT) * 4, d->stream);
  if (e == cudaSuccess) bwd_init<<<grid_for((long long)ST), TB, 0, d->stream>>>(p, cur, a, GL);
  const long long nl = (long long)KLT, nn = (long long)KNT, ns = (long long)ST;
  for (int hi = K; e == cudaSuccess && hi > 0;) {
    // segment (lo, hi]: recompute states lo .. hi - 1 from checkpoint lo
    const int lo = ((hi - 1) / C) * C;
    e = cudaMemcpyAsync(seg, ck + (size_t)(lo / C) * SF, SF * 4, cudaMemcpyDeviceToDevice, d->stream);
    for (int i = lo + 1; e == cudaSuccess && i < hi; ++i) forward_step(d, sgst(i - 1 - lo), sgst(i - lo));
    for (int i = hi; e == cudaSuccess && i > lo; --i) {
      const St s = sgst(i - 1 - lo);   // state i - 1
      bwd_node1<<<grid_for(nn), TB, 0, d->stream>>>(p, a, A, B);
      bwd_line1<<<grid_for(nl), TB, 0, d->stream>>>(p, s, a, A, B, X1, X2, Y1, Y2, GU);
      bwd_dev<<<grid_for(ns), TB, 0, d->stream>>>(p, s, a, A, LX, GL, GP);
      bwd_node2<<<grid_for(nn), TB, 0, d->stream>>>(p, a, X1, X2, Y1, Y2, LX, Cn, Dn);
      bwd_line2<<<grid_for(nl), TB, 0, d->stream>>>(p, a, Cn, Dn);
      bwd_dev2<<<grid_for(ns), TB, 0, d->stream>>>(p, a, LX, Cn);
    }
    hi = lo;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  std::vector<float> gu(KLT);
  if (e == cudaSuccess && g_load) e = cudaMemcpyAsync(g_load, GL, DT * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess && g_pmax) e = cudaMemcpyAsync(g_pmax, GP, GT * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess && g_u) e = cudaMemcpyAsync(gu.data(), GU, KLT * 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  release();
  if (e != cudaSuccess) return dfail(OPF_ECUDA, cudaGetErrorString(e));
  if (g_u) {
    // d f / d u_l: the limit is the same in every contingency and step
    for (int l = 0; l < d->L; ++l) {
      double s = 0.0;
      for (int k = 0; k < d->Kp; ++k)
        for (int t = 0; t < d->T; ++t) s += gu[((size_t)k * d->L + l) * d->T + t];
      g_u[l] = (float)s;
    }
  }
  return OPF_OK;
}

void opf_diff_destroy(opf_diff *d) {
  if (!d) return;
  cudaStreamSynchronize(d->stream);
  for (void *q : d->allocs) cudaFree(q);
  delete d;
}

}  // extern "C"
