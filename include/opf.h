/*
 * opf.h -- C ABI of the GB300 proximal message passing solver for
 * contingency-constrained DC optimal power flow.
 *
 * The solver runs the message-passing form of ADMM (Section 3.2): per
 * iteration, the prox of every line in every contingency (step 1), the prox
 * of every generator, load and battery shared by all contingencies (step 2),
 * the node averages and the scaled price updates (step 3), then the primal and
 * dual residuals of Section 3.3, the stopping test of Eq. (converge) and the
 * adaptive penalty of Section 3.5.  Ramp-limited generators and batteries use
 * the inner ADMM of Appendix D for their prox.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an opf_status and never aborts the process.
 *   - Input arrays are read during the call only; the library copies them.
 *   - Output buffers are owned by the caller.  Where a function takes an
 *     `on_device` flag, 0 means host pointers and 1 means device pointers of
 *     the current CUDA device.
 *   - Arrays are row-major; the time step t is always the innermost index.
 *     K is the number of contingencies, Kp = K + 1 (contingency 0 is the base
 *     case), L lines, N nodes, S = n_gens + n_loads + n_stor + 2 n_hvdc
 *     device terminals with one schedule for all contingencies, ordered
 *     generators, loads, batteries, then terminal 1 and terminal 2 of each
 *     HVDC link.
 *   - Power p > 0 flows from a device into its node (Section 2).  A line's
 *     power is reported at its second terminal (the `to` node); its first
 *     terminal carries -p.
 *   - All GPU work is enqueued on the stream given in opf_options; functions
 *     that return data synchronize that stream.
 *   - A context lives on the device that is current when it is created;
 *     calls on it are made with that device current.
 */
#ifndef OPF_H_
#define OPF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OPF_ABI_VERSION 5

typedef struct opf_ctx opf_ctx; /* opaque, created by opf_create, freed by opf_destroy */

typedef enum {
  OPF_OK = 0,
  OPF_EINVAL = 1,     /* bad argument or inconsistent network data */
  OPF_ENOMEM = 2,     /* a host or device allocation failed */
  OPF_ECUDA = 3,      /* a CUDA runtime call failed (message in opf_last_error) */
  OPF_ETIMEOUT = 4,   /* a synchronizing call gave up waiting for the context's
                         queued GPU work after opf_options.sync_timeout_ms; the
                         work continues and a later call can wait again */
  OPF_ENONFINITE = 5, /* a residual became NaN or infinite; iteration stopped */
  OPF_ESTATE = 6,     /* the call does not apply to the context in its state */
  OPF_ESTALLED = 7    /* the residuals stopped falling at fixed penalties
                         (opf_options.stall_window); iteration stopped, and the
                         next opf_iterate call continues */
} opf_status;

/*
 * Network data (Section 2.1 device models, Section 2.3 contingencies).
 * Node ids are 0-based.  Every node needs at least one terminal.
 */
typedef struct {
  int32_t n_nodes;

  /* AC lines under the DC approximation: I{p1 + p2 = 0} + I{|p2| <= u}
   * + I{p2 = b (theta1 - theta2)}.  Terminal 1 sits at line_from, terminal 2
   * at line_to.  b > 0, u >= 0. */
  int32_t n_lines;
  const int32_t *line_from, *line_to;
  const double *line_b, *line_u;

  /* Generators: a p^2 + b p + I{pmin_t <= p_t <= pmax_t}; gen_pmin/gen_pmax
   * are [n_gens][T].  gen_ramp[g] >= 0 adds |p_{t+1} - p_t| <= ramp (for T > 1);
   * a negative value means no ramp limit. */
  int32_t n_gens;
  const int32_t *gen_node;
  const double *gen_a, *gen_b, *gen_pmin, *gen_pmax, *gen_ramp;

  /* Loads: load_p [n_loads][T] is the consumption (>= 0).  load_voll < 0 makes
   * the load fixed (p = -load_p); otherwise the load is curtailable on
   * [-load_p, 0] at cost voll * (p + load_p). */
  int32_t n_loads;
  const int32_t *load_node;
  const double *load_p, *load_voll;

  /* Batteries (Section 2.1): power limit P, duration dur (energy limit
   * dur * P), charge efficiency eff in (0, 1], discharge cost cost >= 0;
   * empty at the start and at the end of the horizon. */
  int32_t n_stor;
  const int32_t *stor_node;
  const double *stor_P, *stor_dur, *stor_eff, *stor_cost;

  /* HVDC links (Section 2.1, other devices): I{p1 + p2 = 0} + I{|p2| <= u},
   * no angle relation.  Terminal 1 sits at hvdc_from, terminal 2 at hvdc_to
   * (distinct nodes), hvdc_u >= 0.  Only AC lines change per contingency
   * (Section 2.3), so a link keeps one schedule for every contingency; its
   * prox is p2 = clip((x2 - x1) / 2, -u, u). */
  int32_t n_hvdc;
  const int32_t *hvdc_from, *hvdc_to;
  const double *hvdc_u;
} opf_network;

/* Contingencies k = 1..K: in contingency k the line outaged_line[k-1] has
 * u = b = 0 (Section 2.3, N-1 example); -1 keeps the base-case parameters. */
typedef struct {
  int32_t K;
  const int32_t *outaged_line;
} opf_contingencies;

/* Algorithm options.  opf_default_options fills the paper's defaults
 * (Section 5.2): rho_p = rho_theta = 1, mu = 2, gamma = 1.1, alpha = 1, adapt every 10
 * iterations, 10 inner iterations (Section 4.5), eps = 1e-4 tested every 10;
 * no limit on the adaptation and no stall rule; a residual history of 4096
 * rows.
 *
 * The penalty limit and the stall rule are not in the paper, which adapts the
 * penalties for the whole run (Section 3.5).  The residual balancing rule it
 * takes from Boyd et al. (2011, Section 3.4.1) keeps ADMM's convergence
 * guarantee only when the penalties stop changing after finitely many
 * iterations; applied for ever it can cycle (the residuals approach the
 * tolerance, then grow again).
 *   adapt_until   the last iteration that may adapt the penalties (0 = no limit).
 *   stall_window  at every stopping test that fails, let m = max(||r_primal||,
 *                 ||r_dual||).  When m falls below 0.99 times its best value
 *                 so far, that value and its iteration are kept.  When it has
 *                 not done so for stall_window iterations: while the penalties
 *                 still adapt, they are fixed from that iteration on and the
 *                 window restarts; with fixed penalties the call stops and
 *                 reports OPF_ESTALLED.  An infeasible problem stalls (its
 *                 primal residual stays bounded away from zero); so can a
 *                 feasible one that converges very slowly, and the window
 *                 sets how long to wait for a 1 % gain.  0 = off. */
typedef struct {
  double rho_p, rho_theta;  /* initial penalties (> 0) */
  double eps;               /* Eq. (converge) tolerance; <= 0 disables stopping */
  double mu, gamma;         /* adaptive penalty: threshold and factor (Section 3.5) */
  double alpha;             /* over-relaxation in [1, 2) (Section 3.6); 1 = message passing.
                               With alpha != 1 the copies and prices take
                               alpha p + (1 - alpha) z; exported schedules are the
                               actual iterate, and a state import restarts the
                               copies at z = p~, xi = theta_bar */
  int32_t adapt_every;      /* penalty update cadence; 0 disables adaptation */
  int32_t inner_iters;      /* Appendix D iterations per iterative prox (>= 1) */
  int32_t check_every;      /* stopping test cadence; 0 disables stopping */
  int32_t stall_window;     /* stall rule window in iterations (above); 0 = off */
  int64_t sync_timeout_ms;  /* longest wait of a synchronizing call for the
                               context's GPU work (OPF_ETIMEOUT after it); 0 = no limit */
  void *cuda_stream;        /* cudaStream_t to enqueue on; NULL = default stream */
  int64_t adapt_until;      /* last iteration that may adapt the penalties; 0 = no limit */
  int32_t history_len;      /* rows of residual history kept on the device (opf_history); 0 = none */
  int32_t reserved0;
} opf_options;

/* Solver state, the iterate s = (p, theta, u, v) of Section 4.4 plus the
 * inner ADMM duals.  Each pointer may be NULL to skip that array.
 *   p_line, th1, th2, v1, v2: [Kp][L][T]  line terminal-2 power, terminal
 *                                          angles and phase duals
 *   p_dev:  [S][T]                         device terminal power (one schedule)
 *   u:      [Kp][N][T]                     scaled power-balance duals (per node)
 *   inner:  [inner_len]                    inner ADMM (lambda, beta) of the
 *           iterative proxes, layout documented at opf_get_info. */
typedef struct {
  float *p_line, *th1, *th2, *v1, *v2;
  float *p_dev;
  float *u;
  float *inner;
} opf_state;

typedef struct {
  int64_t iterations;       /* iterations run since create / reset */
  int32_t converged;        /* 1 once Eq. (converge) held at a test */
  int32_t status;           /* sticky device status (an opf_status value) */
  double rho_p, rho_theta;  /* current penalties */
  double tolerance;         /* eps * sqrt(2 J T Kp) */
  int32_t N, L, S, T, K, J; /* sizes; J = 2L + S terminals */
  int32_t n_ramp, n_stor;   /* devices using the inner ADMM */
  /* inner_len = n_ramp * 2 * (4T - 2) + n_stor * 2 * (8T + 4).  Layout: for
   * each ramp-limited generator in generator order, lambda then beta over the
   * rows [p <= pmax (T), -p <= -pmin (T), ramp up (T-1), ramp down (T-1)];
   * then for each battery, lambda then beta over the rows [p + c - delta = 0
   * (T), soc dynamics (T), s_1 = 0, s_{T+1} = 0, c <= P (T), -c <= 0 (T),
   * delta <= P (T), -delta <= 0 (T), s <= dur P (T+1), -s <= 0 (T+1)]. */
  int64_t inner_len;
  int64_t device_bytes;     /* device memory held by the context */
  int32_t kernels_per_iteration; /* kernel launches one iteration makes */
  int32_t stalled;          /* 1 when the last call stopped at a stall (OPF_ESTALLED) */
  int64_t frozen_at;        /* iteration at which the stall rule fixed the penalties; 0 = never */
  int64_t history_rows;     /* residual-history rows written since create / reset */
  int32_t k_begin, k_count; /* contingencies held: k_begin .. k_begin + k_count - 1 (all
                               K + 1 of them unless the context is a slice) */
} opf_info;

/* Fill `opt` with the defaults listed above. */
void opf_default_options(opf_options *opt);

/* Validate the network, build the node-ordered incidence (CSR by node), upload
 * parameters and allocate the device state, zero-initialised (Section 3.4).
 * `opt` may be NULL for the defaults.  On success *out owns the context. */
opf_status opf_create(const opf_network *net, int32_t horizon_T,
                      const opf_contingencies *ctg, const opf_options *opt,
                      opf_ctx **out);

/* Enqueue n_iters message-passing iterations (Section 3.2).  Each iteration
 * is seven kernels (device averages and closed-form devices, inner-ADMM
 * devices, device sums, line proxes on a second stream, the node sums -- a
 * general pass on iterations that form residuals and a lean pass on the
 * others, each returning at once on the other's iterations -- and the
 * decisions), replayed from CUDA graphs of 1 and 16 iterations after a
 * one-thread kernel that records the call's last iteration.  Residuals
 * (Section 3.3) are formed on stopping-test iterations (every check_every),
 * adaptation iterations (every adapt_every) and the call's last iteration;
 * a non-finite value is reported (OPF_ENONFINITE) at the first of these
 * after it appears.  rho > 0 first sets rho_p = rho_theta = rho, rescaling
 * the scaled duals (Section 3.5); rho <= 0 keeps the current (possibly
 * adapted) penalties.  After a passed stopping test, a stall
 * (opf_options.stall_window) or an error the remaining iterations of the
 * call return at once; a call after a stall restarts the stall window, a
 * call after an error does nothing.  Asynchronous: the call
 * only enqueues on the context's streams, ordered after the caller's stream
 * and before its later work; device errors surface at the next
 * synchronizing call. */
opf_status opf_iterate(opf_ctx *ctx, int32_t n_iters, double rho);

/* Contingency slices: the iteration on several GPUs (one process each),
 * each holding a block of the contingencies.  The contingencies are coupled
 * only by the sums over k that feed the devices shared by all of them
 * (Section 3.2 step 2) and by the residual norms (Section 3.3), so a slice
 * keeps the lines, node arrays and phase duals of its own contingencies and
 * a replica of the shared devices, and the slices exchange one buffer per
 * iteration, which the caller sums over all slices (an all-reduce).
 *
 * opf_create_slice is opf_create for contingencies k_begin .. k_end - 1 of
 * 0 .. K (0 is the base case; the blocks of the slices must partition
 * 0 .. K).  Every slice gets the whole network and contingency list, the
 * same options (plain message passing, alpha = 1) and its own device.
 * Per iteration, on every slice, in this order:
 *   opf_slice_local   the devices (from the exchanged sums), this slice's
 *                     line proxes and node sums, then its share of the sums
 *                     written into the exchange buffer;
 *   (the caller)      sums the exchange buffers of all slices, in place, on
 *                     the stream of opf_options.cuda_stream;
 *   opf_slice_finish  the residuals, stopping test and adaptive penalty from
 *                     the summed buffer (the same decisions on every slice).
 * Before the first iteration after create, reset or a state import, call
 * opf_slice_prime and exchange once: it writes this slice's share of the
 * sums of its current state.  opf_slice_begin(n, rho) starts a call of n
 * iterations as opf_iterate does (the residuals are formed at its last
 * iteration; rho > 0 sets the penalties) and must precede them.  After a
 * stop (converged, stalled, error) the local half contributes the sums of
 * the unchanged state, so the exchange stays consistent.
 * opf_slice_exchange returns the library-owned device buffer (n doubles:
 * sum_k (pbar + u) and sum_k u at the nodes with devices, then the residual
 * partial sums) for the caller's all-reduce.  Exports of a slice hold its own
 * contingencies (K + 1 replaced by k_end - k_begin); opf_solution's price is
 * this slice's part of -rho_p sum_k u_k (sum it over the slices).  A slice
 * cannot be iterated by opf_iterate (OPF_ESTATE) or join a batch. */
opf_status opf_create_slice(const opf_network *net, int32_t horizon_T, const opf_contingencies *ctg,
                            int32_t k_begin, int32_t k_end, const opf_options *opt, opf_ctx **out);
opf_status opf_slice_exchange(opf_ctx *ctx, double **buffer, int64_t *n_doubles);
opf_status opf_slice_prime(opf_ctx *ctx);
opf_status opf_slice_begin(opf_ctx *ctx, int32_t n_iters, double rho);
opf_status opf_slice_local(opf_ctx *ctx);
opf_status opf_slice_finish(opf_ctx *ctx);

/* Residuals of the last iteration run (Section 3.3), FP64:
 * out[0] = ||r_primal||, out[1] = ||r_dual||, out[2] = primal power part,
 * out[3] = primal phase part, out[4] = dual power part, out[5] = dual phase part.
 * Synchronizes; returns the sticky device status, else OPF_ESTALLED when the
 * last call stopped at a stall, else OPF_OK. */
opf_status opf_residuals(opf_ctx *ctx, double out[6]);

/* Solution at the current iterate.  Any pointer may be NULL.
 *   objective   host double: sum of device costs (line costs are indicators)
 *   p_dev       [S][T]      device power
 *   p_line      [Kp][L][T]  line terminal-2 power
 *   theta_node  [Kp][N][T]  node angles theta_bar
 *   price       [N][T]      nodal prices -rho_p * sum_k u_k
 * Synchronizes. */
opf_status opf_solution(opf_ctx *ctx, int32_t on_device, double *objective, float *p_dev,
                        float *p_line, float *theta_node, float *price);

/* Residual history (Section 3.3), one row per iteration that formed its
 * residuals: the stopping-test iterations (every check_every), the adaptation
 * iterations (every adapt_every) and the last iteration of every call.  The
 * decision kernel writes each row into a ring of opf_options.history_len rows
 * on the device, so a convergence trace needs no host round trip.  Row layout
 * (OPF_HISTORY_COLS doubles):
 *   [0] iteration (1-based count after it)  [1] ||r_primal||  [2] ||r_dual||
 *   [3..6] primal power, primal phase, dual power, dual phase parts
 *   [7] rho_p, [8] rho_theta in force during the iteration
 *   [9] flags: 1 converged, 2 penalties changed after it, 4 the stall rule fixed
 *       the penalties, 8 stalled (OPF_ESTALLED), 16 non-finite
 * rows [max_rows][OPF_HISTORY_COLS] host, caller-owned, receives the most
 * recent min(max_rows, history_len, rows written) rows, oldest first;
 * *n_rows their count.  Synchronizes. */
#define OPF_HISTORY_COLS 10
opf_status opf_history(opf_ctx *ctx, int32_t max_rows, double *rows, int32_t *n_rows);

/* Nodal prices without any allocation: the same export as opf_solution's
 * `price`, staged through a fixed device array instead of a per-call device
 * buffer.  The paper has no counterpart; this is a serving convenience for
 * callers that must not allocate once set up.
 *   price   host float [N][T] (caller's node numbering), -rho_p * sum_k u_k
 * Scratch: one file-scope device array of OPF_PRICE_SCRATCH_FLOATS floats
 * (4 MiB) per device.  N * T above that returns OPF_EINVAL before any device
 * work.  opf_create looks up the array's device address (with the context's
 * device current) and keeps it in the context, so the call makes no symbol
 * lookup; the call itself makes no cudaMalloc / cudaFree or allocating
 * library call, on the device or the host.  Every staged element is written
 * before it is read, so nothing needs clearing between calls.  The array is
 * shared by all contexts of a device: calls that overlap in time (from
 * several threads, or on different streams) race on it and must be
 * serialized by the caller.  The call waits for the context's queued work
 * and synchronizes its stream, so it must not be made while that stream is
 * being captured into a CUDA graph. */
#define OPF_PRICE_SCRATCH_FLOATS (1 << 20)
opf_status opf_price_noalloc(opf_ctx *ctx, float *price);

/* Batched iteration of independent instances (the batch solver of the
 * expansion-planning application, Section 5.6).  A batch groups existing
 * contexts of the current device (the caller keeps owning them; each keeps
 * its own state, options and stream).  One batch step launches each phase
 * kernel once for all instances: every CTA finds its instance in a schedule
 * built at opf_batch_create, so the launch count does not grow with the
 * number of instances; steps are replayed from CUDA graphs of 1 and 16
 * iterations.  Iterates equal those of opf_iterate on each context.
 * opf_batch_iterate enqueues n_iters iterations of every instance after the
 * work already queued on each instance's stream, and orders each stream
 * after it.  Unlike opf_iterate it does not restart an instance that has
 * stopped (passed stopping test, stall or error): such an instance's CTAs
 * return at once, so a batch can be iterated until every instance has
 * stopped (opf_batch_stopped).
 * opf_batch_converged counts the converged instances (synchronizes).  The
 * contexts must outlive the batch; opf_batch_create allocates the device
 * copies of the instances' parameters and the schedule.  The instances of a
 * batch all run plain (alpha = 1) or all over-relaxed (OPF_EINVAL otherwise). */
typedef struct opf_batch opf_batch;
opf_status opf_batch_create(opf_ctx *const *ctxs, int32_t n, opf_batch **out);
opf_status opf_batch_iterate(opf_batch *batch, int32_t n_iters);
opf_status opf_batch_converged(opf_batch *batch, int32_t *n_converged);
/* Stopped instances of a batch: converged, stalled (OPF_ESTALLED) and holding
 * an error status; each pointer may be NULL.  Synchronizes. */
opf_status opf_batch_stopped(opf_batch *batch, int32_t *n_converged, int32_t *n_stalled, int32_t *n_error);
void opf_batch_destroy(opf_batch *batch);

/* Pick the batch's CTA-to-instance schedule by timing.  Candidate layouts
 * (index: instance order, CTAs per phase, CTAs of the grid-stride phases):
 *   0 as given, contiguous, 1x   1 longest first, contiguous, 1x
 *   2 longest first, round-robin, 1x   3 as given, contiguous, 1/4
 *   4 longest first, contiguous, 1/4   5 longest first, round-robin, 1/4
 * ("longest first" orders instances by (K+1) T (L + N); "round-robin" deals
 * one CTA per instance in turn; "1/4" gives the device-sum, inner-ADMM,
 * device-average and node-sum phases a quarter of the CTAs, each doing four
 * times the work; deeper divisors tuned on the first iterations lose on the
 * tail, when the largest instances run alone).  Every candidate runs
 * `steps` >= 1 batch iterations (after one warm-up) from the instances'
 * current state, which is saved before and restored after, so the call
 * leaves every iterate unchanged; the fastest layout is kept for later
 * opf_batch_iterate calls.  The layout changes which CTA computes what, not
 * the arithmetic of an iterate; only the split of the residual norms'
 * partial sums over CTAs moves (their last bits).  choice and
 * ms_each [OPF_BATCH_LAYOUTS] (each may be NULL) receive the chosen index
 * and every layout's milliseconds per batch iteration.  Synchronizes;
 * allocates a temporary copy of the instances' states. */
#define OPF_BATCH_LAYOUTS 6
opf_status opf_batch_autotune(opf_batch *batch, int32_t steps, int32_t *choice, double *ms_each);

/* Drop the batch's stopped instances (converged, stalled, error) from its
 * schedule, so that later steps launch CTAs for the running ones only (a
 * batch's last steps often run one or two instances while the stopped ones'
 * CTAs would still be scheduled).  The layout in force keeps its order and
 * CTA split, restricted to the running instances, so iterates do not change,
 * not even the residuals' last bits; counts and queries still cover every
 * instance, and an instance once dropped is not iterated again by this batch.
 * n_scheduled (may be NULL) receives the number of instances still
 * scheduled; with none, opf_batch_iterate does nothing.  Synchronizes; a
 * later opf_batch_autotune schedules every instance again. */
opf_status opf_batch_compact(opf_batch *batch, int32_t *n_scheduled);

/* Export / import the full state (warm start, checkpoint and resume,
 * Section 3.4).  Import recomputes the node averages from p and theta and
 * projects v onto v_bar = 0 per node (Appendix C); it clears a sticky
 * OPF_ETIMEOUT / OPF_ESTATE and restarts the stall rule with adapting
 * penalties.  Arrays left NULL on import are zeroed. */
opf_status opf_get_state(opf_ctx *ctx, int32_t on_device, const opf_state *dst);
opf_status opf_set_state(opf_ctx *ctx, int32_t on_device, const opf_state *src);

/* Starting state from nodal prices and node angles -- the learned warm
 * start's network output (include/opf_wsnet.h) or any other estimate; the
 * paper's warm start (Section 3.4) imports a whole previous state through
 * opf_set_state instead.  rows [T][N][stride] floats in the caller's node
 * numbering (host, or device when on_device): rows[(t N + n) stride] is the
 * price of node n at step t divided by price_scale, rows[(t N + n) stride + 1]
 * its angle; other columns are ignored (stride >= 2).  The state: u_k =
 * -price / (rho_p (K+1)) in every contingency at the context's current
 * rho_p (the prices are -rho_p sum_k u_k, opf_solution), every line terminal
 * at its node's angle, line power b (theta1 - theta2) clipped to the limit
 * (0 on the outaged line of a contingency), v = 0, device powers and inner
 * duals 0; the node averages are formed from it.  Like opf_set_state it
 * clears a sticky OPF_ETIMEOUT / OPF_ESTATE and restarts the stall rule.
 * With host rows the call stages them through a temporary device buffer.
 * Synchronizes. */
opf_status opf_set_state_from_nodes(opf_ctx *ctx, int32_t on_device, const float *rows, int32_t stride,
                                    double price_scale);

/* Zero the state (cold start); restore the initial penalties, the counters,
 * the stall rule and the residual history. */
opf_status opf_reset(opf_ctx *ctx);

opf_status opf_get_info(opf_ctx *ctx, opf_info *info);

/* Free all resources; NULL is ignored. */
void opf_destroy(opf_ctx *ctx);

const char *opf_status_str(opf_status s);

/* Message of the last failing call on this thread ("" if none). */
const char *opf_last_error(void);

int32_t opf_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OPF_H_ */
