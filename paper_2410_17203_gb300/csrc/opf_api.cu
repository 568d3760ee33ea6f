// Host side of the C ABI declared in include/opf.h: input validation, the
// CSR-by-node incidence (Section 4.3 scatter/gather as node-ordered lists),
// device memory (one arena per context) and the entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <thread>
#include <string>
#include <vector>

#include "opf.h"
#include "opf_internal.h"

using opfk::DevScalars;
using opfk::Params;

namespace {

// message of the last failing call on this thread; a fixed buffer, so that
// reporting an error allocates nothing
thread_local char g_err[512];

opf_status fail(opf_status s, const char *msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  // the failure is returned here; clear the runtime's (non-sticky) last error
  // so that a later call's launch check does not report it a second time
  if (s == OPF_ECUDA || s == OPF_ENOMEM) (void)cudaGetLastError();
  return s;
}

opf_status fail(opf_status s, const std::string &msg) { return fail(s, msg.c_str()); }

}  // namespace

int opf_record_error(int s, const char *msg) { return (int)fail((opf_status)s, msg); }

namespace {

opf_status cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? OPF_ENOMEM : OPF_ECUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int kMaxT = 2048;
constexpr int kMaxHistory = 1 << 20;  // rows of residual history a context may keep
constexpr int kGraphIters = 16;  // iterations in the larger of the two iteration graphs

// bump allocator over one cudaMalloc
struct Arena {
  size_t off = 0;
  char *base = nullptr;
  template <class T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

}  // namespace

struct opf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  opf_options opt{};
  int N = 0, L = 0, T = 0, K = 0, Kp = 0, S = 0, G = 0, D = 0, B = 0, H = 0;
  // contingency slice: Kp local contingencies k_base .. k_base + Kp - 1 of
  // Kp_glob (= Kp for a whole context)
  int k_base = 0, Kp_glob = 0;
  bool slice = false;
  cudaGraphExec_t g_local = nullptr;   // a slice's local half of one iteration
  int n_closed = 0, n_dnode = 0, n_ramp = 0, n_stor = 0;
  size_t n_tcode = 0;  // padded terminal-code list length
  float *price_scratch = nullptr;  // this device's fixed price staging array
  opfk::IterPlan plan{};
  // iteration streams (main: devices, node sums, decisions; aux: line proxes),
  // the events that fork and join them, and the events that order them after
  // and before the caller's stream
  cudaStream_t s_main = nullptr, s_aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_in = nullptr, ev_out = nullptr, ev_sync = nullptr;
  // CUDA graphs of 1 and kGraphIters iterations, built on first use
  cudaGraphExec_t g_one = nullptr, g_many = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  Params P{};
  size_t state_bytes = 0;     // leading part of the arena zeroed by opf_reset
  // host copies used for the objective and the inner-state layout
  std::vector<double> gen_a, gen_b, load_voll, load_p, stor_cost;
  std::vector<int> ramp_gen;  // generator index of each ramp device
  double tol = 0.0;
  int host_status = 0;        // sticky status seen by the host
};

extern "C" {

void opf_default_options(opf_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rho_p = 1.0;
  o->rho_theta = 1.0;
  o->eps = 1e-4;
  o->mu = 2.0;
  o->gamma = 1.1;
  o->alpha = 1.0;
  o->adapt_every = 10;
  o->inner_iters = 10;
  o->check_every = 10;
  o->stall_window = 0;
  o->sync_timeout_ms = 0;
  o->cuda_stream = nullptr;
  o->adapt_until = 0;
  o->history_len = 4096;
}

const char *opf_status_str(opf_status s) {
  switch (s) {
    case OPF_OK: return "ok";
    case OPF_EINVAL: return "invalid argument";
    case OPF_ENOMEM: return "out of memory";
    case OPF_ECUDA: return "CUDA error";
    case OPF_ETIMEOUT: return "GPU work still running at the synchronization timeout";
    case OPF_ENONFINITE: return "non-finite residual";
    case OPF_ESTATE: return "call does not apply to the context in its state";
    case OPF_ESTALLED: return "residuals stopped falling at fixed penalties";
  }
  return "unknown status";
}

const char *opf_last_error(void) { return g_err; }

int32_t opf_abi_version(void) { return OPF_ABI_VERSION; }

}  // extern "C"

namespace {

bool finite_all(const double *a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

opf_status validate(const opf_network *net, int T, const opf_contingencies *ctg,
                    const opf_options &o) {
  if (!net) return fail(OPF_EINVAL, "network is NULL");
  if (T < 1 || T > kMaxT) return fail(OPF_EINVAL, "horizon T must be in [1, 2048]");
  if (net->n_nodes < 1) return fail(OPF_EINVAL, "n_nodes must be >= 1");
  if (net->n_lines < 0 || net->n_gens < 0 || net->n_loads < 0 || net->n_stor < 0 || net->n_hvdc < 0)
    return fail(OPF_EINVAL, "negative device count");
  const int N = net->n_nodes;
  auto bad_nodes = [N](const int32_t *a, int n) {
    for (int i = 0; i < n; ++i)
      if (a[i] < 0 || a[i] >= N) return true;
    return false;
  };
  const size_t nT = (size_t)T;
  if (net->n_lines) {
    if (!net->line_from || !net->line_to || !net->line_b || !net->line_u)
      return fail(OPF_EINVAL, "line arrays missing");
    if (bad_nodes(net->line_from, net->n_lines) || bad_nodes(net->line_to, net->n_lines))
      return fail(OPF_EINVAL, "line node id out of range");
    for (int l = 0; l < net->n_lines; ++l) {
      if (net->line_from[l] == net->line_to[l]) return fail(OPF_EINVAL, "line connects a node to itself");
      if (!(net->line_b[l] > 0.0) || !std::isfinite(net->line_b[l]))
        return fail(OPF_EINVAL, "line susceptance must be finite and > 0");
      if (!(net->line_u[l] >= 0.0) || !std::isfinite(net->line_u[l]))
        return fail(OPF_EINVAL, "line limit must be finite and >= 0");
    }
  }
  if (net->n_gens) {
    if (!net->gen_node || !net->gen_a || !net->gen_b || !net->gen_pmin || !net->gen_pmax || !net->gen_ramp)
      return fail(OPF_EINVAL, "generator arrays missing");
    if (bad_nodes(net->gen_node, net->n_gens)) return fail(OPF_EINVAL, "generator node id out of range");
    if (!finite_all(net->gen_a, net->n_gens) || !finite_all(net->gen_b, net->n_gens) ||
        !finite_all(net->gen_ramp, net->n_gens) || !finite_all(net->gen_pmin, net->n_gens * nT) ||
        !finite_all(net->gen_pmax, net->n_gens * nT))
      return fail(OPF_EINVAL, "non-finite generator data");
    for (int g = 0; g < net->n_gens; ++g) {
      if (net->gen_a[g] < 0) return fail(OPF_EINVAL, "generator quadratic cost must be >= 0");
      for (int t = 0; t < T; ++t)
        if (net->gen_pmin[g * nT + t] > net->gen_pmax[g * nT + t])
          return fail(OPF_EINVAL, "generator pmin > pmax");
    }
  }
  if (net->n_loads) {
    if (!net->load_node || !net->load_p || !net->load_voll) return fail(OPF_EINVAL, "load arrays missing");
    if (bad_nodes(net->load_node, net->n_loads)) return fail(OPF_EINVAL, "load node id out of range");
    if (!finite_all(net->load_p, net->n_loads * nT) || !finite_all(net->load_voll, net->n_loads))
      return fail(OPF_EINVAL, "non-finite load data");
  }
  if (net->n_stor) {
    if (!net->stor_node || !net->stor_P || !net->stor_dur || !net->stor_eff || !net->stor_cost)
      return fail(OPF_EINVAL, "battery arrays missing");
    if (bad_nodes(net->stor_node, net->n_stor)) return fail(OPF_EINVAL, "battery node id out of range");
    for (int b = 0; b < net->n_stor; ++b) {
      if (!(net->stor_P[b] >= 0) || !(net->stor_dur[b] >= 0) || !(net->stor_eff[b] > 0) ||
          !(net->stor_eff[b] <= 1) || !(net->stor_cost[b] >= 0) || !std::isfinite(net->stor_P[b]) ||
          !std::isfinite(net->stor_dur[b]) || !std::isfinite(net->stor_cost[b]))
        return fail(OPF_EINVAL, "battery data out of range");
    }
  }
  if (net->n_hvdc) {
    if (!net->hvdc_from || !net->hvdc_to || !net->hvdc_u) return fail(OPF_EINVAL, "HVDC arrays missing");
    if (bad_nodes(net->hvdc_from, net->n_hvdc) || bad_nodes(net->hvdc_to, net->n_hvdc))
      return fail(OPF_EINVAL, "HVDC node id out of range");
    for (int h = 0; h < net->n_hvdc; ++h) {
      if (net->hvdc_from[h] == net->hvdc_to[h]) return fail(OPF_EINVAL, "HVDC link connects a node to itself");
      if (!(net->hvdc_u[h] >= 0.0) || !std::isfinite(net->hvdc_u[h]))
        return fail(OPF_EINVAL, "HVDC limit must be finite and >= 0");
    }
  }
  if (ctg && ctg->K < 0) return fail(OPF_EINVAL, "K must be >= 0");
  {
    // item indices of the iteration kernel are 32-bit
    const double kp = 1.0 + (ctg ? ctg->K : 0);
    if (kp * std::max(net->n_lines, net->n_nodes) * T >= 2147483647.0)
      return fail(OPF_EINVAL, "(K+1) * max(lines, nodes) * T must stay below 2^31");
  }
  if (ctg && ctg->K > 0) {
    if (!ctg->outaged_line) return fail(OPF_EINVAL, "outaged_line is NULL");
    for (int k = 0; k < ctg->K; ++k)
      if (ctg->outaged_line[k] < -1 || ctg->outaged_line[k] >= net->n_lines)
        return fail(OPF_EINVAL, "outaged line index out of range");
  }
  if (!(o.rho_p > 0) || !(o.rho_theta > 0) || !std::isfinite(o.rho_p) || !std::isfinite(o.rho_theta))
    return fail(OPF_EINVAL, "penalties must be finite and > 0");
  if (!(o.alpha >= 1.0 && o.alpha < 2.0)) return fail(OPF_EINVAL, "over-relaxation alpha must be in [1, 2)");
  if (!(o.mu > 0) || !(o.gamma >= 1) || o.inner_iters < 1 || o.adapt_every < 0 || o.check_every < 0 ||
      !std::isfinite(o.eps))
    return fail(OPF_EINVAL, "invalid options");
  if (o.stall_window < 0 || o.adapt_until < 0 || o.history_len < 0 || o.history_len > kMaxHistory)
    return fail(OPF_EINVAL, "stall_window, adapt_until must be >= 0 and history_len in [0, 2^20]");
  return OPF_OK;
}

// Reverse Cuthill-McKee order of the node graph (lines as edges): order[new]
// = old.  Neighbours of a node end up with nearby numbers, so the two ends of
// a line are processed close together and its second read hits L2.
std::vector<int> rcm_order(int N, const std::vector<int> &ptr, const std::vector<int> &adj) {
  std::vector<int> deg(N), order, bydeg(N);
  order.reserve(N);
  for (int n = 0; n < N; ++n) deg[n] = ptr[n + 1] - ptr[n];
  for (int n = 0; n < N; ++n) bydeg[n] = n;
  std::stable_sort(bydeg.begin(), bydeg.end(), [&](int a, int b) { return deg[a] < deg[b]; });
  std::vector<char> seen(N, 0);
  std::vector<int> nb;
  for (int s : bydeg) {
    if (seen[s]) continue;
    seen[s] = 1;
    size_t head = order.size();
    order.push_back(s);
    while (head < order.size()) {
      const int v = order[head++];
      nb.clear();
      for (int j = ptr[v]; j < ptr[v + 1]; ++j)
        if (!seen[adj[j]]) {
          seen[adj[j]] = 1;
          nb.push_back(adj[j]);
        }
      std::stable_sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] < deg[b]; });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// doubles in a slice's exchange buffer: sum_k (pbar + u) and sum_k u at the
// nodes with devices, then the residual partial sums
size_t slice_exchange_len(const opf_ctx *c) { return (size_t)2 * c->n_dnode * c->T + opfk::NSLOT; }

// The arena layout; called once with a null base to size it.
void carve(opf_ctx *c, Arena &a) {
  Params &p = c->P;
  const size_t KLT = (size_t)c->Kp * c->L * c->T, KNT = (size_t)c->Kp * c->N * c->T;
  const size_t ST = (size_t)c->S * c->T;
  const int T = c->T, Tp = c->T + 1;
  // state first (zeroed on reset)
  for (int b = 0; b < 2; ++b) {
    p.P[b] = a.take<float>(KLT);
    p.MID[b] = a.take<float>(KLT);
    p.V1[b] = a.take<float>(KLT);
    p.V2[b] = a.take<float>(KLT);
    p.U[b] = a.take<float>(KNT);
    p.PU[b] = a.take<float>(KNT);
    p.THBAR[b] = a.take<float>(KNT);
  }
  p.PD = a.take<float>(ST);
  p.DPD = a.take<float>(ST);
  p.ramp_lam = a.take<float>((size_t)c->n_ramp * opfk::RG_N * T);
  p.ramp_beta = a.take<float>((size_t)c->n_ramp * opfk::RG_N * T);
  p.ramp_q = a.take<float>((size_t)c->n_ramp * T);
  p.ramp_rho = a.take<float>(c->n_ramp);
  p.stor_lam = a.take<float>((size_t)c->n_stor * opfk::SG_N * Tp);
  p.stor_beta = a.take<float>((size_t)c->n_stor * opfk::SG_N * Tp);
  p.stor_q = a.take<float>((size_t)c->n_stor * Tp);
  p.stor_rho = a.take<float>(c->n_stor);
  p.stor_delta = a.take<float>((size_t)c->n_stor * T);
  // residual history: part of the mutable state that a batch autotune saves
  // and restores
  p.hist = a.take<double>((size_t)c->opt.history_len * opfk::HIST_COLS);
  c->state_bytes = a.off;
  p.sc = a.take<DevScalars>(1);
  // parameters
  p.line_n1 = a.take<int>(c->L);
  p.line_n2 = a.take<int>(c->L);
  p.line_b = a.take<float>(c->L);
  p.line_u = a.take<float>(c->L);
  p.out_line = a.take<int>(c->Kp);
  p.lcsr_ptr = a.take<int>(c->N + 1);
  p.lcsr = a.take<int2>(2 * (size_t)c->L);
  p.dcsr_ptr = a.take<int>(c->N + 1);
  p.dcsr_idx = a.take<int>(c->S);
  p.cnt_p = a.take<float>(c->N);
  p.cnt_th = a.take<float>(c->N);
  p.rcnt_p = a.take<float>(c->N);
  p.rcnt_th = a.take<float>(c->N);
  p.nrec = a.take<int4>(3 * (size_t)c->N);
  p.tcode = a.take<int>(c->n_tcode);
  p.dev_node = a.take<int>(c->S);
  p.dev_type = a.take<int>(c->S);
  p.dnode_ids = a.take<int>(c->n_dnode);
  p.dnode_ptr = a.take<int>(c->n_dnode + 1);
  p.dnode_dev = a.take<int>(c->n_closed);
  p.dnode_keep = a.take<int>(c->n_dnode);
  p.dev_a = a.take<float>(c->S);
  p.dev_b = a.take<float>(c->S);
  p.dev_lo = a.take<float>(ST);
  p.dev_hi = a.take<float>(ST);
  p.ramp_ids = a.take<int>(c->n_ramp);
  p.ramp_R = a.take<float>(c->n_ramp);
  p.stor_ids = a.take<int>(c->n_stor);
  p.stor_eff = a.take<float>(c->n_stor);
  p.stor_P = a.take<float>(c->n_stor);
  p.stor_dur = a.take<float>(c->n_stor);
  p.stor_cost = a.take<float>(c->n_stor);
  p.hvdc_u = a.take<float>(c->H);
  p.node_perm = a.take<int>(c->N);
  p.line_perm = a.take<int>(c->L);
  // scratch
  p.XS = a.take<float>((size_t)c->N * T);
  p.DSP = a.take<float>((size_t)c->N * T);
  p.DSM = a.take<float>((size_t)c->N * T);
  p.DSQ = a.take<float>((size_t)c->N * T);
  p.partials = a.take<double>((size_t)c->plan.node_grid * opfk::NSLOT);
  p.xsum = c->slice ? a.take<double>(slice_exchange_len(c)) : nullptr;
}

opf_status init_scalars(opf_ctx *c) {
  DevScalars sc{};
  sc.rho_p = c->opt.rho_p;
  sc.rho_th = c->opt.rho_theta;
  sc.su = 1.0;
  sc.sv = 1.0;
  sc.v_fresh = 1;
  sc.stall_ref = HUGE_VAL;
  CK(cudaMemcpyAsync(c->P.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return OPF_OK;
}

// Wait until the work queued on the caller's stream (which includes the
// iterations, joined back into it) is done: without limit, or for at most
// sync_timeout_ms, after which OPF_ETIMEOUT reports work still running.
opf_status wait_stream(opf_ctx *c) {
  if (c->opt.sync_timeout_ms <= 0) {
    CK(cudaStreamSynchronize(c->stream));
    return OPF_OK;
  }
  CK(cudaEventRecord(c->ev_sync, c->stream));
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(c->ev_sync);
    if (e == cudaSuccess) return OPF_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
    if (ms.count() >= c->opt.sync_timeout_ms) return fail(OPF_ETIMEOUT, "GPU work still running at sync_timeout_ms");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

opf_status read_scalars(opf_ctx *c, DevScalars *sc) {
  opf_status s = wait_stream(c);
  if (s != OPF_OK) return s;
  CK(cudaMemcpy(sc, c->P.sc, sizeof(*sc), cudaMemcpyDeviceToHost));
  if (sc->status) c->host_status = sc->status;
  return OPF_OK;
}

// The iteration as a CUDA graph of `iters` iterations, captured from the two
// iteration streams.
opf_status build_graph(opf_ctx *c, int iters, cudaGraphExec_t *out, bool slice_local = false) {
  CK(cudaStreamBeginCapture(c->s_main, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < iters; ++i) {
    const int r = slice_local ? opfk_slice_local_enqueue(c->P, c->plan, c->s_main, c->s_aux, c->ev_fork, c->ev_join)
                              : opfk_iteration_enqueue(c->P, c->plan, c->s_main, c->s_aux, c->ev_fork, c->ev_join);
    if (r != 0) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c->s_main, &g);
      if (g) cudaGraphDestroy(g);
      return fail(OPF_ECUDA, "iteration enqueue failed during graph capture");
    }
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamEndCapture(c->s_main, &g));
  // keep the stream priorities of the captured kernels (device work ahead of
  // the line CTAs it runs beside)
  const cudaError_t e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return OPF_OK;
}

void release_cuda(opf_ctx *c) {
  if (c->g_local) cudaGraphExecDestroy(c->g_local);
  if (c->g_one) cudaGraphExecDestroy(c->g_one);
  if (c->g_many) cudaGraphExecDestroy(c->g_many);
  for (cudaEvent_t ev : {c->ev_fork, c->ev_join, c->ev_in, c->ev_out, c->ev_sync})
    if (ev) cudaEventDestroy(ev);
  if (c->s_main) cudaStreamDestroy(c->s_main);
  if (c->s_aux) cudaStreamDestroy(c->s_aux);
  if (c->arena) cudaFree(c->arena);
}

// device scratch for exports to host memory (not on the iteration path)
struct DevTmp {
  float *p = nullptr;
  ~DevTmp() {
    if (p) cudaFree(p);
  }
};

// Fixed staging array of opf_price_noalloc: a module-scope device variable,
// so it exists once per device the library runs on and is never allocated.
static __device__ __align__(256) float g_price_scratch[OPF_PRICE_SCRATCH_FLOATS];

// Its address on the current device.  In host code the variable's name is a
// host-side stand-in, never a device address, so the address is looked up
// with cudaGetSymbolAddress -- by every opf_create, with the context's device
// current, and kept in the context: a price call then makes no symbol lookup,
// and no address outlives the CUDA context it was resolved in (a cache keyed
// by device alone would go stale after cudaDeviceReset).
opf_status resolve_price_scratch(float **out) {
  void *a = nullptr;
  CK(cudaGetSymbolAddress(&a, g_price_scratch));
  *out = static_cast<float *>(a);
  return OPF_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// a context over contingencies k_begin .. k_end - 1 (all of them: 0 .. K + 1)
opf_status create_impl(const opf_network *net, int32_t T, const opf_contingencies *ctg, int k_begin, int k_end,
                       bool slice, const opf_options *opt_in, opf_ctx **out) {
  if (!out) return fail(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  opf_options opt;
  opf_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.sync_timeout_ms < 0) opt.sync_timeout_ms = 0;
  opf_status st = validate(net, T, ctg, opt);
  if (st != OPF_OK) return st;

  auto *c = new (std::nothrow) opf_ctx();
  if (!c) return fail(OPF_ENOMEM, "host allocation failed");
  c->opt = opt;
  c->stream = (cudaStream_t)opt.cuda_stream;
  c->N = net->n_nodes;
  c->L = net->n_lines;
  c->T = T;
  c->K = ctg ? ctg->K : 0;
  c->Kp_glob = c->K + 1;
  if (k_begin < 0 || k_end > c->Kp_glob || k_begin >= k_end) {
    delete c;
    return fail(OPF_EINVAL, "contingency range [k_begin, k_end) must lie in [0, K + 1) and be non-empty");
  }
  c->k_base = k_begin;
  c->Kp = k_end - k_begin;
  c->slice = slice;
  c->G = net->n_gens;
  c->D = net->n_loads;
  c->B = net->n_stor;
  c->H = net->n_hvdc;
  c->S = c->G + c->D + c->B + 2 * c->H;
  const int N = c->N, L = c->L, S = c->S, G = c->G, D = c->D;
  const size_t nT = (size_t)T;

  // every node needs a terminal
  std::vector<int> dev_node(S);
  for (int g = 0; g < G; ++g) dev_node[g] = net->gen_node[g];
  for (int d = 0; d < D; ++d) dev_node[G + d] = net->load_node[d];
  for (int b = 0; b < c->B; ++b) dev_node[G + D + b] = net->stor_node[b];
  for (int h = 0; h < c->H; ++h) {
    dev_node[G + D + c->B + 2 * h] = net->hvdc_from[h];
    dev_node[G + D + c->B + 2 * h + 1] = net->hvdc_to[h];
  }
  std::vector<int> lcnt(N, 0), dcnt(N, 0);
  for (int l = 0; l < L; ++l) {
    lcnt[net->line_from[l]]++;
    lcnt[net->line_to[l]]++;
  }
  for (int d = 0; d < S; ++d) dcnt[dev_node[d]]++;
  for (int n = 0; n < N; ++n)
    if (lcnt[n] + dcnt[n] == 0) {
      delete c;
      return fail(OPF_EINVAL, "node " + std::to_string(n) + " has no terminal");
    }

  // node renumbering (RCM) and line order (by owner = lower internal end)
  std::vector<int> aptr(N + 1, 0), adj(2 * (size_t)L);
  for (int n = 0; n < N; ++n) aptr[n + 1] = aptr[n] + lcnt[n];
  {
    std::vector<int> fill(aptr.begin(), aptr.end() - 1);
    for (int l = 0; l < L; ++l) {
      adj[fill[net->line_from[l]]++] = net->line_to[l];
      adj[fill[net->line_to[l]]++] = net->line_from[l];
    }
  }
  std::vector<int> node_perm = rcm_order(N, aptr, adj), node_inv(N);
  for (int i = 0; i < N; ++i) node_inv[node_perm[i]] = i;
  std::vector<int> line_perm(L), line_inv(L);
  for (int l = 0; l < L; ++l) line_perm[l] = l;
  auto key = [&](int l) {
    const int a = node_inv[net->line_from[l]], b = node_inv[net->line_to[l]];
    return std::make_pair(std::min(a, b), std::max(a, b));
  };
  std::stable_sort(line_perm.begin(), line_perm.end(), [&](int x, int y) { return key(x) < key(y); });
  for (int i = 0; i < L; ++i) line_inv[line_perm[i]] = i;

  // CSR by internal node: incident lines (2*l + end, other node) and devices
  std::vector<int> lptr(N + 1, 0), dptr(N + 1, 0);
  for (int n = 0; n < N; ++n) {
    lptr[n + 1] = lptr[n] + lcnt[node_perm[n]];
    dptr[n + 1] = dptr[n] + dcnt[node_perm[n]];
  }
  std::vector<int2> lcsr(2 * (size_t)L);
  std::vector<int> didx(S), n1(L), n2(L);
  {
    std::vector<int> lp(lptr.begin(), lptr.end() - 1), dp(dptr.begin(), dptr.end() - 1);
    for (int li = 0; li < L; ++li) {
      const int l = line_perm[li];
      const int a = node_inv[net->line_from[l]], b = node_inv[net->line_to[l]];
      n1[li] = a;
      n2[li] = b;
      lcsr[lp[a]++] = make_int2(2 * li, b);       // terminal 1 at a
      lcsr[lp[b]++] = make_int2(2 * li + 1, a);   // terminal 2 at b
    }
    for (int d = 0; d < S; ++d) didx[dp[node_inv[dev_node[d]]]++] = d;
  }
  std::vector<float> cnt_p(N), cnt_th(N), rcnt_p(N), rcnt_th(N);
  std::vector<int> dev_node_int(S);
  for (int n = 0; n < N; ++n) {
    cnt_p[n] = (float)(lcnt[node_perm[n]] + dcnt[node_perm[n]]);
    cnt_th[n] = (float)lcnt[node_perm[n]];
    rcnt_p[n] = (float)(1.0 / cnt_p[n]);
    rcnt_th[n] = cnt_th[n] > 0 ? (float)(1.0 / cnt_th[n]) : 0.f;
  }
  for (int d = 0; d < S; ++d) dev_node_int[d] = node_inv[dev_node[d]];

  // device classes and closed-form parameters
  std::vector<float> dev_a(S, 0.f), dev_b(S, 0.f), lo(S * nT, 0.f), hi(S * nT, 0.f);
  std::vector<int> dev_type(S, 0), ramp, stor;
  std::vector<float> rampR;
  for (int g = 0; g < G; ++g) {
    dev_a[g] = (float)net->gen_a[g];
    dev_b[g] = (float)net->gen_b[g];
    for (size_t t = 0; t < nT; ++t) {
      lo[g * nT + t] = (float)net->gen_pmin[g * nT + t];
      hi[g * nT + t] = (float)net->gen_pmax[g * nT + t];
    }
    if (net->gen_ramp[g] >= 0 && T > 1) {
      ramp.push_back(g);
      rampR.push_back((float)net->gen_ramp[g]);
      dev_type[g] = 1;
    }
  }
  for (int d = 0; d < D; ++d) {
    const bool fixed = net->load_voll[d] < 0;
    dev_b[G + d] = fixed ? 0.f : (float)net->load_voll[d];
    for (size_t t = 0; t < nT; ++t) {
      const float P = (float)net->load_p[d * nT + t];
      lo[(G + d) * nT + t] = -P;
      hi[(G + d) * nT + t] = fixed ? -P : 0.f;
    }
  }
  std::vector<float> seff, sP, sdur, scost;
  for (int b = 0; b < c->B; ++b) {
    stor.push_back(G + D + b);
    dev_type[G + D + b] = 1;
    seff.push_back((float)net->stor_eff[b]);
    sP.push_back((float)net->stor_P[b]);
    sdur.push_back((float)net->stor_dur[b]);
    scost.push_back((float)net->stor_cost[b]);
  }
  // HVDC terminals: evaluated by the inner kernel, which needs both ends' averages
  std::vector<float> hvdc_u(c->H);
  for (int h = 0; h < c->H; ++h) {
    dev_type[G + D + c->B + 2 * h] = dev_type[G + D + c->B + 2 * h + 1] = 2;
    hvdc_u[h] = (float)net->hvdc_u[h];
  }
  // nodes with devices (avg_k(pbar + u) is formed once per node), their
  // closed-form devices, and whether inner-ADMM devices need the average
  std::vector<int> dnode_ids, dnode_ptr(1, 0), dnode_dev, dnode_keep;
  for (int n = 0; n < N; ++n) {
    if (dptr[n + 1] == dptr[n]) continue;
    int keep = 0;
    for (int j = dptr[n]; j < dptr[n + 1]; ++j) {
      if (dev_type[didx[j]] == 0) dnode_dev.push_back(didx[j]);
      else keep = 1;
    }
    dnode_ids.push_back(n);
    dnode_ptr.push_back((int)dnode_dev.size());
    dnode_keep.push_back(keep);
  }
  c->n_closed = (int)dnode_dev.size();
  c->n_dnode = (int)dnode_ids.size();
  c->n_ramp = (int)ramp.size();
  c->n_stor = (int)stor.size();

  // host copies for the objective
  c->gen_a.assign(net->gen_a, net->gen_a + G);
  c->gen_b.assign(net->gen_b, net->gen_b + G);
  c->load_voll.assign(net->load_voll, net->load_voll + D);
  c->load_p.assign(net->load_p, net->load_p + D * nT);
  c->stor_cost.assign(net->stor_cost, net->stor_cost + c->B);

  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice");
  }
  {
    const opf_status ps = resolve_price_scratch(&c->price_scratch);
    if (ps != OPF_OK) {
      delete c;
      return ps;
    }
  }
  {
    // launch configuration (the node kernel's grid sizes the partial sums)
    Params q{};
    q.N = N;
    q.L = L;
    q.T = T;
    q.Kp = c->Kp;
    q.n_dnode = c->n_dnode;
    q.n_ramp = c->n_ramp;
    q.n_stor = c->n_stor;
    q.n_hvdc = c->H;
    q.S = S;
    if (opfk_plan(q, &c->plan) != 0) {
      delete c;
      return fail(OPF_ECUDA, "occupancy query for the iteration kernels failed");
    }
  }
  // line-terminal codes beyond the first four of each node, padded to a
  // multiple of 4 (the first four sit in the node record)
  std::vector<int> tcode, tptr(N + 1, 0);
  for (int n = 0; n < N; ++n) {
    for (int j = lptr[n] + 4; j < lptr[n + 1]; ++j) tcode.push_back(lcsr[j].x);
    while (tcode.size() % 4) tcode.push_back(-1);
    tptr[n + 1] = (int)tcode.size();
  }
  c->n_tcode = std::max<size_t>(tcode.size(), 4);
  Arena a;
  carve(c, a);
  c->arena_bytes = a.off + 256;
  e = cudaMalloc(&c->arena, c->arena_bytes);
  if (e != cudaSuccess) {
    opf_status s = cuda_fail(e, "cudaMalloc(arena)");
    delete c;
    return s;
  }
  a = Arena();
  a.base = c->arena;
  carve(c, a);
  {
    // iteration streams: devices and node sums at the higher priority so that
    // their CTAs are scheduled ahead of the concurrent line CTAs
    int lo = 0, hi = 0;
    cudaError_t ce = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&c->s_main, cudaStreamNonBlocking, hi);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&c->s_aux, cudaStreamNonBlocking, lo);
    for (cudaEvent_t *ev : {&c->ev_fork, &c->ev_join, &c->ev_in, &c->ev_out, &c->ev_sync})
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      opf_status es = cuda_fail(ce, "stream / event creation");
      release_cuda(c);
      delete c;
      return es;
    }
  }

  Params &p = c->P;
  p.N = N;
  p.L = L;
  p.T = T;
  p.Kp = c->Kp;
  p.S = S;
  p.n_dnode = c->n_dnode;
  p.n_ramp = c->n_ramp;
  p.n_stor = c->n_stor;
  p.n_hvdc = c->H;
  p.hvdc0 = G + D + c->B;
  p.node_grid = c->plan.node_grid;
  p.dsum_lean = c->plan.dsum_lean;
  p.eps = opt.eps;
  p.mu = opt.mu;
  p.gamma = opt.gamma;
  p.alpha = (float)opt.alpha;
  p.adapt_every = opt.adapt_every;
  p.check_every = opt.check_every;
  p.inner_iters = opt.inner_iters;
  p.Kp_glob = c->Kp_glob;
  p.k_base = c->k_base;
  p.slice = c->slice ? 1 : 0;
  p.stall_window = opt.stall_window;
  p.adapt_until = opt.adapt_until;
  p.hist_cap = opt.history_len;
  c->tol = opt.eps * std::sqrt(2.0 * (2.0 * L + S) * T * c->Kp_glob);
  p.tol = c->tol;

  std::vector<int> outl(c->Kp, -1);
  std::vector<float> lb(L), lu(L);
  for (int li = 0; li < L; ++li) {
    lb[li] = (float)net->line_b[line_perm[li]];
    lu[li] = (float)net->line_u[line_perm[li]];
  }
  for (int j = 0; j < c->Kp; ++j) {
    const int k = c->k_base + j;   // global contingency; 0 is the base case
    if (k >= 1) outl[j] = ctg->outaged_line[k - 1] >= 0 ? line_inv[ctg->outaged_line[k - 1]] : -1;
  }

  opf_status s = OPF_OK;
  auto up = [&](const void *dst, const auto &v) {
    if (s != OPF_OK || v.empty()) return;
    cudaError_t ee = cudaMemcpyAsync(const_cast<void *>(dst), v.data(), v.size() * sizeof(v[0]),
                                     cudaMemcpyHostToDevice, c->stream);
    if (ee != cudaSuccess) s = cuda_fail(ee, "cudaMemcpyAsync(parameters)");
  };
  e = cudaMemsetAsync(c->arena, 0, c->arena_bytes, c->stream);
  if (e != cudaSuccess) s = cuda_fail(e, "cudaMemsetAsync(arena)");
  up(p.line_n1, n1);
  up(p.line_n2, n2);
  up(p.line_b, lb);
  up(p.line_u, lu);
  up(p.out_line, outl);
  up(p.lcsr_ptr, lptr);
  up(p.lcsr, lcsr);
  up(p.dcsr_ptr, dptr);
  up(p.dcsr_idx, didx);
  up(p.cnt_p, cnt_p);
  up(p.cnt_th, cnt_th);
  up(p.rcnt_p, rcnt_p);
  up(p.rcnt_th, rcnt_th);
  {
    std::vector<int4> rec(3 * (size_t)N);
    auto fbits = [](float f) {
      int i;
      std::memcpy(&i, &f, sizeof(i));
      return i;
    };
    for (int n = 0; n < N; ++n) {
      int code[4] = {-1, -1, -1, -1};
      for (int j = lptr[n], q = 0; j < lptr[n + 1] && q < 4; ++j, ++q) code[q] = lcsr[j].x;
      rec[3 * n] = make_int4(fbits(cnt_p[n]), fbits(cnt_th[n]), fbits(rcnt_p[n]), fbits(rcnt_th[n]));
      rec[3 * n + 1] = make_int4(code[0], code[1], code[2], code[3]);
      rec[3 * n + 2] = make_int4(tptr[n], tptr[n + 1], dptr[n + 1] - dptr[n], dptr[n]);
    }
    up(p.nrec, rec);
  }
  up(p.tcode, tcode);
  up(p.dev_node, dev_node_int);
  up(p.dev_type, dev_type);
  up(p.dnode_ids, dnode_ids);
  up(p.dnode_ptr, dnode_ptr);
  up(p.dnode_dev, dnode_dev);
  up(p.dnode_keep, dnode_keep);
  up(p.dev_a, dev_a);
  up(p.dev_b, dev_b);
  up(p.dev_lo, lo);
  up(p.dev_hi, hi);
  up(p.ramp_ids, ramp);
  up(p.ramp_R, rampR);
  up(p.stor_ids, stor);
  up(p.stor_eff, seff);
  up(p.stor_P, sP);
  up(p.stor_dur, sdur);
  up(p.stor_cost, scost);
  up(p.hvdc_u, hvdc_u);
  up(p.node_perm, node_perm);
  up(p.line_perm, line_perm);
  if (s == OPF_OK) s = init_scalars(c);
  if (s != OPF_OK) {
    release_cuda(c);
    delete c;
    return s;
  }
  *out = c;
  return OPF_OK;
}

}  // namespace

extern "C" {

opf_status opf_create(const opf_network *net, int32_t T, const opf_contingencies *ctg,
                      const opf_options *opt, opf_ctx **out) {
  return create_impl(net, T, ctg, 0, 1 + (ctg ? std::max<int>(ctg->K, 0) : 0), false, opt, out);
}

opf_status opf_create_slice(const opf_network *net, int32_t T, const opf_contingencies *ctg, int32_t k_begin,
                            int32_t k_end, const opf_options *opt, opf_ctx **out) {
  if (opt && opt->alpha != 1.0) {
    if (out) *out = nullptr;
    return fail(OPF_EINVAL, "contingency slices run plain message passing (alpha = 1)");
  }
  return create_impl(net, T, ctg, k_begin, k_end, true, opt, out);
}

void opf_destroy(opf_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->s_main) cudaStreamSynchronize(c->s_main);
  release_cuda(c);
  delete c;
}

opf_status opf_iterate(opf_ctx *c, int32_t n_iters, double rho) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  if (c->slice) return fail(OPF_ESTATE, "a contingency slice iterates through opf_slice_local / opf_slice_finish");
  if (n_iters < 0) return fail(OPF_EINVAL, "n_iters must be >= 0");
  if (rho > 0 && !std::isfinite(rho)) return fail(OPF_EINVAL, "rho must be finite");
  if (n_iters > 0 && !c->g_one) {
    opf_status gs = build_graph(c, 1, &c->g_one);
    if (gs == OPF_OK) gs = build_graph(c, kGraphIters, &c->g_many);
    if (gs != OPF_OK) return gs;
  }
  // after the caller's earlier work on its stream ...
  CK(cudaEventRecord(c->ev_in, c->stream));
  CK(cudaStreamWaitEvent(c->s_main, c->ev_in, 0));
  if (rho > 0 && opfk_set_rho_launch(c->P.sc, rho, c->s_main) != 0) return fail(OPF_ECUDA, "set_rho launch failed");
  if (n_iters > 0) {
    if (opfk_begin_launch(c->P.sc, n_iters, 1, c->s_main) != 0) return fail(OPF_ECUDA, "begin launch failed");
    for (int i = 0; i < n_iters / kGraphIters; ++i) CK(cudaGraphLaunch(c->g_many, c->s_main));
    for (int i = 0; i < n_iters % kGraphIters; ++i) CK(cudaGraphLaunch(c->g_one, c->s_main));
  }
  // ... and before its later work
  CK(cudaEventRecord(c->ev_out, c->s_main));
  CK(cudaStreamWaitEvent(c->stream, c->ev_out, 0));
  return OPF_OK;
}

opf_status opf_slice_exchange(opf_ctx *c, double **buf, int64_t *n) {
  if (!c || !buf || !n) return fail(OPF_EINVAL, "NULL argument");
  if (!c->slice) return fail(OPF_ESTATE, "not a contingency slice (opf_create_slice)");
  *buf = c->P.xsum;
  *n = (int64_t)slice_exchange_len(c);
  return OPF_OK;
}

// order the context's streams after the caller's stream, and back
static opf_status slice_in(opf_ctx *c) {
  CK(cudaEventRecord(c->ev_in, c->stream));
  CK(cudaStreamWaitEvent(c->s_main, c->ev_in, 0));
  return OPF_OK;
}

static opf_status slice_out(opf_ctx *c) {
  CK(cudaEventRecord(c->ev_out, c->s_main));
  CK(cudaStreamWaitEvent(c->stream, c->ev_out, 0));
  return OPF_OK;
}

opf_status opf_slice_prime(opf_ctx *c) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  if (!c->slice) return fail(OPF_ESTATE, "not a contingency slice (opf_create_slice)");
  opf_status s = slice_in(c);
  if (s != OPF_OK) return s;
  if (opfk_slice_prime_launch(c->P, c->s_main) != 0) return fail(OPF_ECUDA, "slice prime launch failed");
  return slice_out(c);
}

opf_status opf_slice_begin(opf_ctx *c, int32_t n_iters, double rho) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  if (!c->slice) return fail(OPF_ESTATE, "not a contingency slice (opf_create_slice)");
  if (n_iters < 0) return fail(OPF_EINVAL, "n_iters must be >= 0");
  if (rho > 0 && !std::isfinite(rho)) return fail(OPF_EINVAL, "rho must be finite");
  opf_status s = slice_in(c);
  if (s != OPF_OK) return s;
  if (rho > 0 && opfk_set_rho_launch(c->P.sc, rho, c->s_main) != 0) return fail(OPF_ECUDA, "set_rho launch failed");
  if (opfk_begin_launch(c->P.sc, n_iters, 1, c->s_main) != 0) return fail(OPF_ECUDA, "begin launch failed");
  return slice_out(c);
}

opf_status opf_slice_local(opf_ctx *c) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  if (!c->slice) return fail(OPF_ESTATE, "not a contingency slice (opf_create_slice)");
  if (!c->g_local) {
    opf_status gs = build_graph(c, 1, &c->g_local, true);
    if (gs != OPF_OK) return gs;
  }
  opf_status s = slice_in(c);
  if (s != OPF_OK) return s;
  CK(cudaGraphLaunch(c->g_local, c->s_main));
  return slice_out(c);
}

opf_status opf_slice_finish(opf_ctx *c) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  if (!c->slice) return fail(OPF_ESTATE, "not a contingency slice (opf_create_slice)");
  opf_status s = slice_in(c);
  if (s != OPF_OK) return s;
  if (opfk_slice_finish_enqueue(c->P, c->s_main) != 0) return fail(OPF_ECUDA, "slice decision launch failed");
  return slice_out(c);
}

opf_status opf_residuals(opf_ctx *c, double out[6]) {
  if (!c || !out) return fail(OPF_EINVAL, "NULL argument");
  DevScalars sc;
  opf_status s = read_scalars(c, &sc);
  if (s != OPF_OK) return s;
  for (int j = 0; j < 6; ++j) out[j] = sc.res[j];
  if (sc.status) return (opf_status)sc.status;
  return sc.stalled ? OPF_ESTALLED : OPF_OK;
}

opf_status opf_get_info(opf_ctx *c, opf_info *info) {
  if (!c || !info) return fail(OPF_EINVAL, "NULL argument");
  DevScalars sc;
  opf_status s = read_scalars(c, &sc);
  if (s != OPF_OK) return s;
  std::memset(info, 0, sizeof(*info));
  info->iterations = sc.it;
  info->converged = sc.converged;
  info->status = c->host_status;
  info->rho_p = sc.rho_p;
  info->rho_theta = sc.rho_th;
  info->tolerance = c->tol;
  {
    const opfk::IterPlan &pl = c->plan;
    info->kernels_per_iteration = (pl.xs_grid > 0) + (pl.inner_grid > 0) + 1 +
                                  pl.n_slabs * ((pl.line_grid > 0 && c->L > 0) + 1 +
                                                (pl.lean_grid > 0 && c->opt.alpha == 1.0)) + 1;
  }
  info->N = c->N;
  info->L = c->L;
  info->S = c->S;
  info->T = c->T;
  info->K = c->K;
  info->J = 2 * c->L + c->S;
  info->n_ramp = c->n_ramp;
  info->n_stor = c->n_stor;
  info->inner_len = (int64_t)c->n_ramp * 2 * (4 * (int64_t)c->T - 2) +
                    (int64_t)c->n_stor * 2 * (8 * (int64_t)c->T + 4);
  info->device_bytes = (int64_t)c->arena_bytes;
  info->stalled = sc.stalled;
  info->frozen_at = sc.frozen_at;
  info->history_rows = sc.hist_n;
  info->k_begin = c->k_base;
  info->k_count = c->Kp;
  return OPF_OK;
}

opf_status opf_history(opf_ctx *c, int32_t max_rows, double *rows, int32_t *n_rows) {
  if (!c || !n_rows || (max_rows > 0 && !rows)) return fail(OPF_EINVAL, "NULL argument");
  if (max_rows < 0) return fail(OPF_EINVAL, "max_rows must be >= 0");
  DevScalars sc;
  opf_status s = read_scalars(c, &sc);
  if (s != OPF_OK) return s;
  const long long cap = c->opt.history_len;
  const long long n = std::min<long long>(std::min<long long>(sc.hist_n, cap), max_rows);
  *n_rows = (int32_t)n;
  if (n == 0) return OPF_OK;
  // rows hist_n - n .. hist_n - 1, oldest first, in at most two pieces of the ring
  const size_t row_bytes = opfk::HIST_COLS * sizeof(double);
  const long long first = (sc.hist_n - n) % cap;
  const long long n1 = std::min(n, cap - first);
  CK(cudaMemcpyAsync(rows, c->P.hist + first * opfk::HIST_COLS, n1 * row_bytes, cudaMemcpyDeviceToHost,
                     c->stream));
  if (n > n1)
    CK(cudaMemcpyAsync(rows + n1 * opfk::HIST_COLS, c->P.hist, (n - n1) * row_bytes, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return OPF_OK;
}

}  // extern "C"

namespace {

// canonical inner-state entry -> (device array, index)
struct InnerEntry {
  int arr;     // 0 ramp_lam, 1 ramp_beta, 2 stor_lam, 3 stor_beta, -1 always zero
  size_t idx;
};

std::vector<InnerEntry> inner_layout(const opf_ctx *c) {
  const int T = c->T, Tp = T + 1;
  std::vector<InnerEntry> v;
  for (int r = 0; r < c->n_ramp; ++r) {
    const size_t base = (size_t)r * opfk::RG_N * T;
    std::vector<size_t> rows;
    for (int t = 0; t < T; ++t) rows.push_back(base + opfk::RG_UP * T + t);
    for (int t = 0; t < T; ++t) rows.push_back(base + opfk::RG_LO * T + t);
    for (int t = 0; t < T - 1; ++t) rows.push_back(base + opfk::RG_RU * T + t);
    for (int t = 0; t < T - 1; ++t) rows.push_back(base + opfk::RG_RD * T + t);
    for (size_t x : rows) v.push_back({0, x});
    for (size_t x : rows) v.push_back({1, x});
  }
  for (int b = 0; b < c->n_stor; ++b) {
    const size_t base = (size_t)b * opfk::SG_N * Tp;
    std::vector<std::pair<size_t, bool>> rows;  // (device index, equality row)
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_E1 * Tp + t, true});
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_E2 * Tp + t, true});
    rows.push_back({base + opfk::SG_E3 * Tp + 0, true});
    rows.push_back({base + opfk::SG_E3 * Tp + 1, true});
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_CU * Tp + t, false});
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_CL * Tp + t, false});
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_DU * Tp + t, false});
    for (int t = 0; t < T; ++t) rows.push_back({base + opfk::SG_DL * Tp + t, false});
    for (int t = 0; t < Tp; ++t) rows.push_back({base + opfk::SG_SU * Tp + t, false});
    for (int t = 0; t < Tp; ++t) rows.push_back({base + opfk::SG_SL * Tp + t, false});
    for (auto &x : rows) v.push_back({2, x.first});
    for (auto &x : rows) v.push_back({x.second ? -1 : 3, x.first});
  }
  return v;
}

// Destination for an export: the caller's device buffer, or a device staging
// area that is copied to the caller's host buffer afterwards.
float *stage(float *user, int on_device, float *tmp) { return user ? (on_device ? user : tmp) : nullptr; }

opf_status alloc_tmp(DevTmp &t, size_t n) {
  if (n == 0) return OPF_OK;
  CK(cudaMalloc(&t.p, n * sizeof(float)));
  return OPF_OK;
}

}  // namespace

extern "C" {

opf_status opf_solution(opf_ctx *c, int32_t on_device, double *objective, float *p_dev, float *p_line,
                        float *theta_node, float *price) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  DevScalars sc;
  opf_status s;
  if ((s = read_scalars(c, &sc)) != OPF_OK) return s;
  const int cur = (int)(sc.it & 1);
  const size_t T = c->T, KLT = (size_t)c->Kp * c->L * T, KNT = (size_t)c->Kp * c->N * T, NT = (size_t)c->N * T;
  const size_t ST = (size_t)c->S * T;
  const bool relax = c->opt.alpha != 1.0;
  DevTmp tmp;
  if ((!on_device && (p_line || theta_node || price)) || (relax && (p_dev || objective))) {
    if ((s = alloc_tmp(tmp, (p_line ? KLT : 0) + (theta_node ? KNT : 0) + (price ? NT : 0) + ST)) != OPF_OK)
      return s;
  }
  float *tl = tmp.p, *tt = tmp.p ? tmp.p + (p_line ? KLT : 0) : nullptr;
  float *tp = tt ? tt + (theta_node ? KNT : 0) : nullptr;
  // device powers: PD itself, or the actual iterate rebuilt from the relaxed state
  const float *pd_src = c->P.PD;
  if (relax && (p_dev || objective)) {
    float *td = tmp.p + (p_line ? KLT : 0) + (theta_node ? KNT : 0) + (price ? NT : 0);
    if (opfk_export_pdev_launch(c->P, td, c->stream) != 0) return fail(OPF_ECUDA, "export launch failed");
    pd_src = td;
  }
  if (p_dev)
    CK(cudaMemcpyAsync(p_dev, pd_src, ST * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (p_line && opfk_export_lines_launch(c->P, cur, stage(p_line, on_device, tl), nullptr, nullptr,
                                         nullptr, nullptr, c->stream) != 0)
    return fail(OPF_ECUDA, "export launch failed");
  if ((theta_node || price) &&
      opfk_export_nodes_launch(c->P, cur, nullptr, stage(theta_node, on_device, tt),
                               stage(price, on_device, tp), c->stream) != 0)
    return fail(OPF_ECUDA, "export launch failed");
  if (!on_device) {
    if (p_line) CK(cudaMemcpyAsync(p_line, tl, KLT * 4, cudaMemcpyDeviceToHost, c->stream));
    if (theta_node) CK(cudaMemcpyAsync(theta_node, tt, KNT * 4, cudaMemcpyDeviceToHost, c->stream));
    if (price) CK(cudaMemcpyAsync(price, tp, NT * 4, cudaMemcpyDeviceToHost, c->stream));
  }
  if (objective) {
    std::vector<float> pd((size_t)c->S * T), dl((size_t)c->n_stor * T);
    CK(cudaMemcpyAsync(pd.data(), pd_src, pd.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (!dl.empty())
      CK(cudaMemcpyAsync(dl.data(), c->P.stor_delta, dl.size() * sizeof(float), cudaMemcpyDeviceToHost,
                         c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double f = 0.0;
    for (int g = 0; g < c->G; ++g)
      for (size_t t = 0; t < T; ++t) {
        const double x = pd[g * T + t];
        f += c->gen_a[g] * x * x + c->gen_b[g] * x;
      }
    for (int d = 0; d < c->D; ++d) {
      if (c->load_voll[d] < 0) continue;
      for (size_t t = 0; t < T; ++t)
        f += c->load_voll[d] * ((double)pd[(c->G + d) * T + t] + c->load_p[d * T + t]);
    }
    for (int b = 0; b < c->n_stor; ++b)
      for (size_t t = 0; t < T; ++t) f += c->stor_cost[b] * (double)dl[b * T + t];
    *objective = f;
  }
  CK(cudaStreamSynchronize(c->stream));
  return (opf_status)sc.status;
}

}  // extern "C"

struct opf_batch {
  std::vector<opf_ctx *> ctx;
  int device = 0;
  // the batch kernels run on these two streams (main: devices, node sums,
  // decisions; aux: line proxes); every instance's parameters and the CTA
  // schedules of the batch kernels live in device memory
  cudaStream_t stream = nullptr, s_aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
  opfk::Params *d_params = nullptr;
  int *d_sched = nullptr;
  opfk::BatchPlan plan{};
  long long sched_cap = 0;    // schedule entries d_sched holds (the longest layout)
  cudaGraphExec_t g_one = nullptr, g_many = nullptr;
  // the layout in force (opf_batch_autotune) and how many instances it
  // schedules (all, or those still running after opf_batch_compact)
  std::vector<int> lay_order;  // instance order; empty: as given
  int lay_interleave = 0, lay_div = 1;
  int n_sched = 0;
};

namespace {

void release_batch(opf_batch *b) {
  if (b->g_one) cudaGraphExecDestroy(b->g_one);
  if (b->g_many) cudaGraphExecDestroy(b->g_many);
  for (cudaEvent_t e : {b->ev_fork, b->ev_join, b->ev_done})
    if (e) cudaEventDestroy(e);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->s_aux) cudaStreamDestroy(b->s_aux);
  if (b->d_params) cudaFree(b->d_params);
  if (b->d_sched) cudaFree(b->d_sched);
}

// `iters` iterations of every instance as one graph: per iteration one
// launch per batch kernel (and width), whatever the number of instances.
opf_status build_batch_graph(opf_batch *b, int iters, cudaGraphExec_t *out) {
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  bool ok = true;
  for (int it = 0; ok && it < iters; ++it)
    ok = opfk_batch_enqueue(b->d_params, b->d_sched, b->plan, b->stream, b->s_aux, b->ev_fork, b->ev_join) == 0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (!ok || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ok ? cuda_fail(e, "cudaStreamEndCapture(batch)") : fail(OPF_ECUDA, "batch graph capture failed");
  }
  const cudaError_t ei = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate(batch)");
  return OPF_OK;
}

// Build the schedule of the n_sched instances that `lay` lists (lay.order;
// NULL: every instance as given) into d_sched and drop the graphs of the
// previous one (rebuilt on the next iteration).  Waits for the batch stream.
opf_status schedule_batch(opf_batch *b, int n_sched, const opfk::BatchLayout &lay) {
  const int n = (int)b->ctx.size();
  std::vector<Params> hp(n);
  std::vector<opfk::IterPlan> plans(n);
  for (int i = 0; i < n; ++i) {
    hp[i] = b->ctx[i]->P;
    plans[i] = b->ctx[i]->plan;
  }
  long long len = 0;
  opfk::BatchPlan bp{};
  if (opfk_batch_plan(hp.data(), plans.data(), n_sched, lay, nullptr, 0, &len, &bp) != 0 || len > b->sched_cap)
    return fail(OPF_ECUDA, "batch schedule");
  std::vector<int> sched(4 * (size_t)std::max(len, 1LL));
  if (opfk_batch_plan(hp.data(), plans.data(), n_sched, lay, sched.data(), len, &len, &bp) != 0)
    return fail(OPF_ECUDA, "batch schedule");
  CK(cudaStreamSynchronize(b->stream));
  if (b->g_one) cudaGraphExecDestroy(b->g_one);
  if (b->g_many) cudaGraphExecDestroy(b->g_many);
  b->g_one = b->g_many = nullptr;
  CK(cudaMemcpy(b->d_sched, sched.data(), sched.size() * sizeof(int), cudaMemcpyHostToDevice));
  // the node phase's CTA count sizes each instance's partial sums
  for (int i = 0; i < n; ++i) hp[i].node_grid = opfk_batch_node_blocks(plans[i], lay.div);
  CK(cudaMemcpy(b->d_params, hp.data(), n * sizeof(Params), cudaMemcpyHostToDevice));
  b->plan = bp;
  b->n_sched = n_sched;
  return OPF_OK;
}

// Apply layout `lay` to every instance and keep it for opf_batch_compact.
opf_status set_batch_layout(opf_batch *b, const opfk::BatchLayout &lay) {
  const int n = (int)b->ctx.size();
  if (lay.order) b->lay_order.assign(lay.order, lay.order + n);
  else b->lay_order.clear();
  b->lay_interleave = lay.interleave;
  b->lay_div = lay.div;
  return schedule_batch(b, n, lay);
}

opf_status ensure_batch_graphs(opf_batch *b) {
  if (b->g_one) return OPF_OK;
  opf_status gs = build_batch_graph(b, 1, &b->g_one);
  if (gs == OPF_OK) gs = build_batch_graph(b, kGraphIters, &b->g_many);
  return gs;
}

void launch_batch_steps(opf_batch *b, int n_iters, cudaError_t *e) {
  for (int i = 0; *e == cudaSuccess && i < n_iters / kGraphIters; ++i) *e = cudaGraphLaunch(b->g_many, b->stream);
  for (int i = 0; *e == cudaSuccess && i < n_iters % kGraphIters; ++i) *e = cudaGraphLaunch(b->g_one, b->stream);
}

// bytes of an instance's mutable state: the iterate, the inner-ADMM state and
// the device scalars lead its arena
size_t mutable_bytes(const opf_ctx *c) {
  return (size_t)(reinterpret_cast<const char *>(c->P.sc + 1) - c->arena);
}

}  // namespace

extern "C" {

opf_status opf_batch_create(opf_ctx *const *ctxs, int32_t n, opf_batch **out) {
  if (!out) return fail(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return fail(OPF_EINVAL, "a batch needs at least one context");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(OPF_EINVAL, "NULL context in batch");
    if (ctxs[i]->device != dev) return fail(OPF_EINVAL, "batch contexts must be on the current device");
    if (ctxs[i]->slice) return fail(OPF_EINVAL, "a contingency slice cannot join a batch");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(OPF_EINVAL, "a context appears twice in the batch");
  }
  auto *b = new (std::nothrow) opf_batch();
  if (!b) return fail(OPF_ENOMEM, "host allocation failed");
  b->ctx.assign(ctxs, ctxs + n);
  b->device = dev;
  std::vector<Params> hp(n);
  std::vector<opfk::IterPlan> plans(n);
  for (int i = 0; i < n; ++i) {
    hp[i] = ctxs[i]->P;
    plans[i] = ctxs[i]->plan;
  }
  long long len = 0;
  opf_status st = OPF_OK;
  const opfk::BatchLayout lay{nullptr, 0, 1};   // as given, contiguous: the longest schedule
  const int pr = opfk_batch_plan(hp.data(), plans.data(), n, lay, nullptr, 0, &len, &b->plan);
  if (pr == -2) st = fail(OPF_EINVAL, "a batch cannot mix over-relaxed (alpha != 1) and plain instances");
  else if (pr != 0) st = fail(OPF_ECUDA, "batch schedule");
  std::vector<int> sched(4 * (size_t)std::max(len, 1LL));
  if (st == OPF_OK && opfk_batch_plan(hp.data(), plans.data(), n, lay, sched.data(), len, &len, &b->plan) != 0)
    st = fail(OPF_ECUDA, "batch schedule");
  b->sched_cap = len;
  b->n_sched = n;
  int lo = 0, hi = 0;
  cudaError_t e = st == OPF_OK ? cudaDeviceGetStreamPriorityRange(&lo, &hi) : cudaSuccess;
  if (st == OPF_OK) {
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->s_aux, cudaStreamNonBlocking, lo);
    for (cudaEvent_t *ev : {&b->ev_fork, &b->ev_join, &b->ev_done})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_params, n * sizeof(Params));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sched, sched.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_params, hp.data(), n * sizeof(Params), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sched, sched.data(), sched.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "batch set-up");
  }
  if (st != OPF_OK) {
    release_batch(b);
    delete b;
    return st;
  }
  *out = b;
  return OPF_OK;
}

opf_status opf_batch_iterate(opf_batch *b, int32_t n_iters) {
  if (!b) return fail(OPF_EINVAL, "batch is NULL");
  if (n_iters < 0) return fail(OPF_EINVAL, "n_iters must be >= 0");
  // nothing to do with no iterations, or when opf_batch_compact found every
  // instance stopped (a stopped instance does not move)
  if (n_iters == 0 || b->n_sched == 0) return OPF_OK;
  const opf_status gs = ensure_batch_graphs(b);
  if (gs != OPF_OK) return gs;
  // after each instance's queued work ...
  for (opf_ctx *c : b->ctx) {
    CK(cudaEventRecord(c->ev_in, c->stream));
    CK(cudaStreamWaitEvent(b->stream, c->ev_in, 0));
  }
  if (opfk_begin_batch_launch(b->d_params, (int)b->ctx.size(), n_iters, b->stream) != 0)
    return fail(OPF_ECUDA, "begin launch failed");
  cudaError_t le = cudaSuccess;
  launch_batch_steps(b, n_iters, &le);
  if (le != cudaSuccess) return cuda_fail(le, "cudaGraphLaunch(batch)");
  // ... and before its later work
  CK(cudaEventRecord(b->ev_done, b->stream));
  for (opf_ctx *c : b->ctx) CK(cudaStreamWaitEvent(c->stream, b->ev_done, 0));
  return OPF_OK;
}

opf_status opf_batch_autotune(opf_batch *b, int32_t steps, int32_t *choice, double *ms_each) {
  if (!b) return fail(OPF_EINVAL, "batch is NULL");
  if (steps < 1) return fail(OPF_EINVAL, "steps must be >= 1");
  const int n = (int)b->ctx.size();
  // instances by decreasing work (line and node items), for longest-first layouts
  std::vector<int> lpt(n);
  for (int i = 0; i < n; ++i) lpt[i] = i;
  auto work = [&](int i) {
    const opf_ctx *c = b->ctx[i];
    return (double)c->Kp * c->T * ((double)c->L + c->N);
  };
  std::stable_sort(lpt.begin(), lpt.end(), [&](int x, int y) { return work(x) > work(y); });
  const opfk::BatchLayout cands[OPF_BATCH_LAYOUTS] = {
      {nullptr, 0, 1}, {lpt.data(), 0, 1}, {lpt.data(), 1, 1},
      {nullptr, 0, 4}, {lpt.data(), 0, 4}, {lpt.data(), 1, 4}};
  // save every instance's mutable state after its queued work
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + mutable_bytes(b->ctx[i]);
  char *snap = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaMalloc(&snap, std::max<size_t>(off[n], 1));
  if (e != cudaSuccess) return cuda_fail(e, "autotune snapshot");
  auto copy_all = [&](bool save) {
    for (int i = 0; e == cudaSuccess && i < n; ++i) {
      char *a = b->ctx[i]->arena, *s = snap + off[i];
      e = cudaMemcpyAsync(save ? s : a, save ? a : s, off[i + 1] - off[i], cudaMemcpyDeviceToDevice, b->stream);
    }
  };
  for (opf_ctx *c : b->ctx) {
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c->ev_in, 0);
  }
  copy_all(true);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  opf_status st = e == cudaSuccess ? OPF_OK : cuda_fail(e, "autotune set-up");
  int best = -1;
  float best_ms = 0.f;
  double times[OPF_BATCH_LAYOUTS] = {0};
  for (int ci = 0; st == OPF_OK && ci < OPF_BATCH_LAYOUTS; ++ci) {
    st = set_batch_layout(b, cands[ci]);
    if (st == OPF_OK) st = ensure_batch_graphs(b);
    if (st != OPF_OK) break;
    copy_all(false);
    launch_batch_steps(b, 1, &e);                    // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
    launch_batch_steps(b, steps, &e);
    if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune timing");
      break;
    }
    times[ci] = (double)ms / steps;
    if (best < 0 || ms < best_ms) {
      best = ci;
      best_ms = ms;
    }
  }
  if (st == OPF_OK) st = set_batch_layout(b, cands[best]);
  if (st == OPF_OK) {
    copy_all(false);                                 // the instances as they were
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_done, b->stream);
    for (opf_ctx *c : b->ctx)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, b->ev_done, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "autotune restore");
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaStreamSynchronize(b->stream);
  cudaFree(snap);
  if (st != OPF_OK) return st;
  if (choice) *choice = best;
  if (ms_each) std::copy(times, times + OPF_BATCH_LAYOUTS, ms_each);
  return OPF_OK;
}

opf_status opf_batch_converged(opf_batch *b, int32_t *n_converged) {
  if (!b || !n_converged) return fail(OPF_EINVAL, "NULL argument");
  int32_t n = 0;
  for (opf_ctx *c : b->ctx) {
    DevScalars sc;
    const opf_status s = read_scalars(c, &sc);
    if (s != OPF_OK) return s;
    n += sc.converged ? 1 : 0;
  }
  *n_converged = n;
  return OPF_OK;
}

opf_status opf_batch_stopped(opf_batch *b, int32_t *n_converged, int32_t *n_stalled, int32_t *n_error) {
  if (!b) return fail(OPF_EINVAL, "NULL argument");
  int32_t nc = 0, ns = 0, ne = 0;
  for (opf_ctx *c : b->ctx) {
    DevScalars sc;
    const opf_status s = read_scalars(c, &sc);
    if (s != OPF_OK) return s;
    nc += sc.converged ? 1 : 0;
    ns += sc.stalled ? 1 : 0;
    ne += sc.status ? 1 : 0;
  }
  if (n_converged) *n_converged = nc;
  if (n_stalled) *n_stalled = ns;
  if (n_error) *n_error = ne;
  return OPF_OK;
}

opf_status opf_batch_compact(opf_batch *b, int32_t *n_scheduled) {
  if (!b) return fail(OPF_EINVAL, "batch is NULL");
  // which instances still run, after the work queued so far
  CK(cudaStreamSynchronize(b->stream));
  const int n = (int)b->ctx.size();
  std::vector<char> run(n, 0);
  for (int i = 0; i < n; ++i) {
    DevScalars sc;
    CK(cudaMemcpy(&sc, b->ctx[i]->P.sc, sizeof(sc), cudaMemcpyDeviceToHost));
    if (sc.status) b->ctx[i]->host_status = sc.status;
    run[i] = (sc.stop == 0 && sc.status == 0) ? 1 : 0;
  }
  // the layout in force, restricted to them (the same order and CTA split)
  std::vector<int> order;
  for (int j = 0; j < n; ++j) {
    const int i = b->lay_order.empty() ? j : b->lay_order[j];
    if (run[i]) order.push_back(i);
  }
  if ((int)order.size() != b->n_sched) {
    const opfk::BatchLayout lay{order.data(), b->lay_interleave, b->lay_div};
    const opf_status st = schedule_batch(b, (int)order.size(), lay);
    if (st != OPF_OK) return st;
  }
  if (n_scheduled) *n_scheduled = (int32_t)order.size();
  return OPF_OK;
}

void opf_batch_destroy(opf_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  release_batch(b);
  delete b;
}

opf_status opf_price_noalloc(opf_ctx *c, float *price) {
  if (!c || !price) return fail(OPF_EINVAL, "NULL argument");
  const size_t NT = (size_t)c->N * c->T;
  if (NT > (size_t)OPF_PRICE_SCRATCH_FLOATS)
    return fail(OPF_EINVAL, "N * T exceeds OPF_PRICE_SCRATCH_FLOATS");
  if (!c->price_scratch) return fail(OPF_ESTATE, "price scratch not resolved");
  DevScalars sc;
  opf_status s;
  if ((s = read_scalars(c, &sc)) != OPF_OK) return s;
  // every element of [0, N*T) is written by the export before the copy reads it
  if (opfk_export_nodes_launch(c->P, (int)(sc.it & 1), nullptr, nullptr, c->price_scratch, c->stream) != 0)
    return fail(OPF_ECUDA, "export launch failed");
  CK(cudaMemcpyAsync(price, c->price_scratch, NT * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return (opf_status)sc.status;
}

opf_status opf_get_state(opf_ctx *c, int32_t on_device, const opf_state *dst) {
  if (!c || !dst) return fail(OPF_EINVAL, "NULL argument");
  DevScalars sc;
  opf_status s;
  if ((s = read_scalars(c, &sc)) != OPF_OK) return s;
  const int cur = (int)(sc.it & 1);
  const size_t KLT = (size_t)c->Kp * c->L * c->T, KNT = (size_t)c->Kp * c->N * c->T;
  const size_t ST = (size_t)c->S * c->T;
  const bool relax = c->opt.alpha != 1.0;
  float *lines[5] = {dst->p_line, dst->th1, dst->th2, dst->v1, dst->v2};
  DevTmp tmp;
  if (!on_device || (relax && dst->p_dev)) {
    size_t n = (dst->u ? KNT : 0) + ST;
    for (float *x : lines) n += x ? KLT : 0;
    if ((s = alloc_tmp(tmp, n)) != OPF_OK) return s;
  }
  if (dst->p_dev) {
    const float *pd_src = c->P.PD;
    if (relax) {
      float *td = tmp.p;   // the first ST floats of the staging area
      if (opfk_export_pdev_launch(c->P, td, c->stream) != 0) return fail(OPF_ECUDA, "export launch failed");
      pd_src = td;
    }
    CK(cudaMemcpyAsync(dst->p_dev, pd_src, ST * sizeof(float),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  float *stg[5];
  float *cursor = tmp.p ? tmp.p + ST : nullptr;
  for (int j = 0; j < 5; ++j) {
    stg[j] = lines[j] ? (on_device ? lines[j] : cursor) : nullptr;
    if (lines[j] && !on_device) cursor += KLT;
  }
  float *ustg = dst->u ? (on_device ? dst->u : cursor) : nullptr;
  if (lines[0] || lines[1] || lines[2] || lines[3] || lines[4]) {
    if (opfk_export_lines_launch(c->P, cur, stg[0], stg[1], stg[2], stg[3], stg[4], c->stream) != 0)
      return fail(OPF_ECUDA, "export launch failed");
  }
  if (ustg && opfk_export_nodes_launch(c->P, cur, ustg, nullptr, nullptr, c->stream) != 0)
    return fail(OPF_ECUDA, "export launch failed");
  if (!on_device) {
    for (int j = 0; j < 5; ++j)
      if (lines[j]) CK(cudaMemcpyAsync(lines[j], stg[j], KLT * 4, cudaMemcpyDeviceToHost, c->stream));
    if (dst->u) CK(cudaMemcpyAsync(dst->u, ustg, KNT * 4, cudaMemcpyDeviceToHost, c->stream));
  }
  if (dst->inner) {
    auto lay = inner_layout(c);
    const size_t nr = (size_t)c->n_ramp * opfk::RG_N * c->T, ns = (size_t)c->n_stor * opfk::SG_N * (c->T + 1);
    std::vector<float> rl(nr), rb(nr), sl(ns), sb(ns);
    if (nr) {
      CK(cudaMemcpyAsync(rl.data(), c->P.ramp_lam, nr * 4, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(rb.data(), c->P.ramp_beta, nr * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    if (ns) {
      CK(cudaMemcpyAsync(sl.data(), c->P.stor_lam, ns * 4, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(sb.data(), c->P.stor_beta, ns * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    std::vector<float> flat(lay.size());
    for (size_t i = 0; i < lay.size(); ++i) {
      const auto &e = lay[i];
      flat[i] = e.arr == 0 ? rl[e.idx] : e.arr == 1 ? rb[e.idx] : e.arr == 2 ? sl[e.idx] : e.arr == 3 ? sb[e.idx] : 0.f;
    }
    if (on_device) {
      CK(cudaMemcpyAsync(dst->inner, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    } else {
      std::memcpy(dst->inner, flat.data(), flat.size() * 4);
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return OPF_OK;
}

opf_status opf_set_state(opf_ctx *c, int32_t on_device, const opf_state *src) {
  if (!c || !src) return fail(OPF_EINVAL, "NULL argument");
  const size_t KLT = (size_t)c->Kp * c->L * c->T, KNT = (size_t)c->Kp * c->N * c->T;
  const size_t ST = (size_t)c->S * c->T;
  DevScalars sc;
  opf_status s;
  if ((s = read_scalars(c, &sc)) != OPF_OK) return s;
  const int cur = (int)(sc.it & 1);
  const float *lines[5] = {src->p_line, src->th1, src->th2, src->v1, src->v2};
  const float *dsrc[5], *usrc = src->u;
  DevTmp tmp;
  if (!on_device) {
    size_t n = src->u ? KNT : 0;
    for (const float *x : lines) n += x ? KLT : 0;
    if ((s = alloc_tmp(tmp, n)) != OPF_OK) return s;
    float *cursor = tmp.p;
    for (int j = 0; j < 5; ++j) {
      dsrc[j] = nullptr;
      if (lines[j]) {
        CK(cudaMemcpyAsync(cursor, lines[j], KLT * 4, cudaMemcpyHostToDevice, c->stream));
        dsrc[j] = cursor;
        cursor += KLT;
      }
    }
    if (src->u) {
      CK(cudaMemcpyAsync(cursor, src->u, KNT * 4, cudaMemcpyHostToDevice, c->stream));
      usrc = cursor;
    }
  } else {
    for (int j = 0; j < 5; ++j) dsrc[j] = lines[j];
  }
  if (opfk_import_launch(c->P, cur, dsrc[0], dsrc[1], dsrc[2], dsrc[3], dsrc[4], usrc, c->stream) != 0)
    return fail(OPF_ECUDA, "import launch failed");
  if (src->p_dev)
    CK(cudaMemcpyAsync(c->P.PD, src->p_dev, ST * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
  else
    CK(cudaMemsetAsync(c->P.PD, 0, ST * 4, c->stream));
  // inner duals: scaled for the current penalty; factors rebuilt on first use
  const float rho_dev = (float)(c->Kp_glob * sc.rho_p);
  const size_t nr = (size_t)c->n_ramp * opfk::RG_N * c->T, ns = (size_t)c->n_stor * opfk::SG_N * (c->T + 1);
  std::vector<float> rl(nr, 0.f), rb(nr, 0.f), sl(ns, 0.f), sb(ns, 0.f);
  if (src->inner) {
    auto lay = inner_layout(c);
    std::vector<float> flat(lay.size());
    if (on_device) {
      CK(cudaMemcpy(flat.data(), src->inner, flat.size() * 4, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(flat.data(), src->inner, flat.size() * 4);
    }
    for (size_t i = 0; i < lay.size(); ++i) {
      const auto &e = lay[i];
      if (e.arr == 0) rl[e.idx] = flat[i];
      else if (e.arr == 1) rb[e.idx] = flat[i];
      else if (e.arr == 2) sl[e.idx] = flat[i];
      else if (e.arr == 3) sb[e.idx] = flat[i];
    }
  }
  std::vector<float> rr(c->n_ramp, src->inner ? -rho_dev : 0.f), sr(c->n_stor, src->inner ? -rho_dev : 0.f);
  if (nr) {
    CK(cudaMemcpyAsync(c->P.ramp_lam, rl.data(), nr * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.ramp_beta, rb.data(), nr * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.ramp_rho, rr.data(), rr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  }
  if (ns) {
    CK(cudaMemcpyAsync(c->P.stor_lam, sl.data(), ns * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.stor_beta, sb.data(), ns * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.stor_rho, sr.data(), sr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  }
  if (opfk_project_v_launch(c->P, cur, c->stream) != 0) return fail(OPF_ECUDA, "project_v launch failed");
  if (opfk_node_average_launch(c->P, cur, c->stream) != 0) return fail(OPF_ECUDA, "node_average launch failed");
  sc.su = 1.0;
  sc.sv = 1.0;
  sc.v_fresh = 1;
  sc.status = 0;
  sc.converged = 0;
  // a warm start restarts the stall rule with adapting penalties
  sc.stalled = 0;
  sc.frozen_at = 0;
  sc.stall_ref = HUGE_VAL;
  sc.stall_it = sc.it;
  CK(cudaMemcpyAsync(c->P.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->host_status = 0;
  return OPF_OK;
}

opf_status opf_set_state_from_nodes(opf_ctx *c, int32_t on_device, const float *rows, int32_t stride,
                                    double price_scale) {
  if (!c || !rows) return fail(OPF_EINVAL, "NULL argument");
  if (stride < 2) return fail(OPF_EINVAL, "stride must be >= 2 (price, angle)");
  if (!(price_scale > 0) || !std::isfinite(price_scale)) return fail(OPF_EINVAL, "price_scale must be finite and > 0");
  DevScalars sc;
  opf_status s;
  if ((s = read_scalars(c, &sc)) != OPF_OK) return s;
  const int cur = (int)(sc.it & 1);
  const size_t n_rows = (size_t)c->T * c->N * stride;
  DevTmp tmp;
  const float *src = rows;
  if (!on_device) {
    if ((s = alloc_tmp(tmp, n_rows)) != OPF_OK) return s;
    CK(cudaMemcpyAsync(tmp.p, rows, n_rows * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    src = tmp.p;
  }
  // u = -price / (rho_p (K+1)) at the penalty in force
  const float u_scale = (float)(1.0 / (sc.rho_p * c->Kp_glob));
  if (opfk_start_from_nodes_launch(c->P, cur, src, stride, (float)price_scale, u_scale, c->stream) != 0)
    return fail(OPF_ECUDA, "start launch failed");
  // device powers and the inner duals from zero (factors rebuilt on first use)
  const size_t ST = (size_t)c->S * c->T;
  const size_t nr = (size_t)c->n_ramp * opfk::RG_N * c->T, ns = (size_t)c->n_stor * opfk::SG_N * (c->T + 1);
  CK(cudaMemsetAsync(c->P.PD, 0, ST * 4, c->stream));
  if (nr) {
    CK(cudaMemsetAsync(c->P.ramp_lam, 0, nr * 4, c->stream));
    CK(cudaMemsetAsync(c->P.ramp_beta, 0, nr * 4, c->stream));
    CK(cudaMemsetAsync(c->P.ramp_rho, 0, c->n_ramp * 4, c->stream));
  }
  if (ns) {
    CK(cudaMemsetAsync(c->P.stor_lam, 0, ns * 4, c->stream));
    CK(cudaMemsetAsync(c->P.stor_beta, 0, ns * 4, c->stream));
    CK(cudaMemsetAsync(c->P.stor_rho, 0, c->n_stor * 4, c->stream));
  }
  if (opfk_node_average_launch(c->P, cur, c->stream) != 0) return fail(OPF_ECUDA, "node_average launch failed");
  sc.su = 1.0;
  sc.sv = 1.0;
  sc.v_fresh = 1;
  sc.status = 0;
  sc.converged = 0;
  sc.stalled = 0;
  sc.frozen_at = 0;
  sc.stall_ref = HUGE_VAL;
  sc.stall_it = sc.it;
  CK(cudaMemcpyAsync(c->P.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->host_status = 0;
  return OPF_OK;
}

opf_status opf_reset(opf_ctx *c) {
  if (!c) return fail(OPF_EINVAL, "ctx is NULL");
  CK(cudaMemsetAsync(c->arena, 0, c->state_bytes, c->stream));
  c->host_status = 0;
  return init_scalars(c);
}

}  // extern "C"
