// Internal layout shared by the host side (opf_api.cu) and the kernels
// (opf_kernels.cu).  Not part of the public ABI.
//
// Numbering: nodes are renumbered by reverse Cuthill-McKee and lines sorted by
// their lower-numbered end (the line's "owner"), so that the two ends of a
// line are processed close together in time; the C ABI converts to and from
// the caller's numbering on import and export.  Devices keep the caller's
// order (generators, loads, batteries).
//
// Device memory layout (structure of arrays, time innermost so that every row
// of T floats is one contiguous, 16-byte aligned segment when T % 4 == 0):
//   lines   P, MID, V1, V2                  2 x [L][Kp][T] float (double buffer)
//   nodes   U, PU = pbar + u, THBAR         2 x [N][Kp][T] float (double buffer)
// (line- and node-major: the K+1 contingency rows of one line or node are
// one contiguous run, so the node sums gather long runs per terminal)
//   devices PD, DPD                         [S][T]         float
//   inner ADMM state of ramp generators     lam, beta [n_ramp][4][T],  q [n_ramp][T]
//   inner ADMM state of batteries           lam, beta [n_stor][9][T+1], q [n_stor][T+1]
// Buffer (it & 1) holds the state after `it` iterations; an iteration reads
// the old buffers and writes the other ones, because both ends of a line
// evaluate its prox from the old line and node values.
// V1/V2 hold the phase duals one step behind: the update v += theta - theta_bar
// of iteration i is folded into the line pass of iteration i+1, which already
// reads theta and theta_bar (so v is read and written once per iteration).
#ifndef OPF_INTERNAL_H_
#define OPF_INTERNAL_H_

#include <stddef.h>
#include <stdint.h>

namespace opfk {

// threads per CTA of the iteration kernels
constexpr int BLOCK = 256;

// residual partial-sum slots.  SL_NF counts non-finite node values: the prox
// clamps (fminf/fmaxf) would otherwise turn a NaN input into a finite bound.
enum { SL_PP = 0, SL_PT = 1, SL_DP = 2, SL_DT = 3, SL_NF = 4, NSLOT = 5 };

// Scalars that persist on the device between launches.
struct DevScalars {
  double rho_p, rho_th;  // penalties in force for the next iteration
  double su, sv;         // pending rescale of u and v (1 = none), applied on next read
  double res[6];         // residuals of the last iteration
  long long it;          // iterations run
  int converged;
  int status;            // sticky opf_status from the device (0 = ok)
  int v_fresh;           // 1: V1/V2 already hold the current v (after import / reset)
  int stop;              // set by the decision kernel (passed stopping test, error);
                         // cleared at the start of every opf_iterate call
  long long it_last;     // the last iteration of the current call: residuals are formed
                         // there and at stopping-test and adaptation iterations only
  // stall rule (opf_options.stall_window): best max(||r_primal||, ||r_dual||)
  // at a stopping test and its iteration; the iteration at which the rule
  // fixed the penalties (0 = they still adapt); 1 after a stall at fixed
  // penalties (stops the call; the next opf_iterate restarts the window)
  double stall_ref;
  long long stall_it;
  long long frozen_at;
  int stalled;
  int pad0;
  long long hist_n;      // residual-history rows written (ring of Params::hist_cap rows)
};

// Battery group offsets inside lam/beta rows of stride Tp = T + 1.
enum { SG_E1 = 0, SG_E2 = 1, SG_E3 = 2, SG_CU = 3, SG_CL = 4, SG_DU = 5, SG_DL = 6,
       SG_SU = 7, SG_SL = 8, SG_N = 9 };
// Ramp-generator groups, stride T.
enum { RG_UP = 0, RG_LO = 1, RG_RU = 2, RG_RD = 3, RG_N = 4 };

struct Params {
  int N, L, T, Kp, S;
  int n_dnode, n_ramp, n_stor;
  int n_hvdc, hvdc0;                     // HVDC links; device id of the first link's terminal 1
  // lines (internal numbering)
  const int *line_n1, *line_n2;  // internal node of terminal 1 (from) and terminal 2 (to)
  const float *line_b, *line_u;
  const int *out_line;  // [Kp], internal index of the outaged line, -1 = none
  // double-buffered line state: terminal-2 power p, the mean terminal angle
  // mid (theta_{1,2} = mid +- p / (2b), the line prox keeps theta1 - theta2 =
  // p / b; the outaged line of a contingency has p = 0 and stores its half
  // angle difference in p's place), and the phase duals
  float *P[2], *MID[2], *V1[2], *V2[2];
  // nodes (internal numbering), double-buffered
  float *U[2], *PU[2], *THBAR[2];   // PU = pbar + u (unscaled): what the proxes read
  // incident lines of each node: x = 2*l + end (end 1: the node is terminal 2), y = other node
  const int *lcsr_ptr;
  const int2 *lcsr;
  const int *dcsr_ptr, *dcsr_idx;  // devices of each node
  const float *cnt_p, *cnt_th;     // terminals per node: all (power), line terminals (phase)
  const float *rcnt_p, *rcnt_th;   // their reciprocals (0 for a node without line terminals)
  // per node, 3 int4: (cnt_p, cnt_th, rcnt_p, rcnt_th as float bits), the first
  // four line-terminal codes 2*l + end (-1 = none), (tcode begin, end of the
  // rest, device count, first of the node's entries in dcsr_idx)
  const int4 *nrec;
  const int *tcode;                // line-terminal codes beyond the first four per node,
                                   // each node's list padded to a multiple of 4 with -1
  // per node and time step, over the node's devices (the same in every
  // contingency): sum of p_d, and the Welford mean and sum of squared
  // deviations of the change of p_d in this iteration
  float *DSP, *DSM, *DSQ;          // [N][T]
  // devices: type 0 = closed-form prox clip((rho X - b)/(2a + rho), lo, hi), 1 = inner ADMM
  float *PD, *DPD;
  const int *dev_node, *dev_type;
  // nodes with devices; per node its closed-form devices and whether it has
  // inner-ADMM devices, whose input avg_k(pbar + u) is then kept in XS
  const int *dnode_ids, *dnode_ptr, *dnode_dev, *dnode_keep;
  float *XS;  // [N][T], avg_k(pbar + u) of the previous iterate at kept nodes
  const float *dev_a, *dev_b;
  const float *dev_lo, *dev_hi;  // [S][T]
  // ramp-limited generators
  const int *ramp_ids;
  const float *ramp_R;
  float *ramp_lam, *ramp_beta, *ramp_q, *ramp_rho;
  // batteries
  const int *stor_ids;
  const float *stor_eff, *stor_P, *stor_dur, *stor_cost;
  const float *hvdc_u;                   // [n_hvdc]; link h has terminals hvdc0 + 2h, hvdc0 + 2h + 1
  float alpha;                           // over-relaxation (Section 3.6); 1 = plain message passing
  float *stor_lam, *stor_beta, *stor_q, *stor_rho, *stor_delta;  // delta [n_stor][T]
  // numbering maps (internal -> caller) for import / export
  const int *node_perm, *line_perm;
  // scratch
  double *partials;  // [node_grid][NSLOT] per-CTA residual partial sums of the node kernel
  int node_grid;     // CTAs of the node kernel (partial-sum slots)
  int dsum_lean;     // IterPlan::dsum_lean
  DevScalars *sc;
  // options
  double eps, mu, gamma, tol;
  int adapt_every, check_every, inner_iters;
  int stall_window;     // 0 = no stall rule
  long long adapt_until;  // last iteration that may adapt (0 = no limit)
  double *hist;         // residual history ring [hist_cap][HIST_COLS]
  int hist_cap;
  // contingency slice (opf_create_slice): this context holds contingencies
  // k_base .. k_base + Kp - 1 of Kp_glob; the sums over k that couple them
  // (Section 3.2 step 2) and the residual sums (Section 3.3) go through the
  // exchange buffer xsum, which the caller sums over the slices:
  //   [n_dnode][T] sum_k (pbar + u) at the nodes with devices,
  //   [n_dnode][T] sum_k u there (on adaptation iterations; else 0),
  //   [NSLOT] residual partial sums
  int Kp_glob;          // K + 1 of the whole problem (= Kp without slices)
  int k_base;
  int slice;            // 1: a slice context
  double *xsum;
};

// columns of a residual-history row (include/opf.h, opf_history)
constexpr int HIST_COLS = 10;
enum { HF_CONVERGED = 1, HF_ADAPTED = 2, HF_FROZEN = 4, HF_STALLED = 8, HF_NONFINITE = 16 };

// offsets of element (contingency k, line l / node n, step t)
__host__ __device__ __forceinline__ size_t lidx(const Params &p, int k, int l, int t) {
  return ((size_t)l * p.Kp + k) * p.T + t;
}
__host__ __device__ __forceinline__ size_t nidx(const Params &p, int k, int n, int t) {
  return ((size_t)n * p.Kp + k) * p.T + t;
}

// Launch configuration of one iteration's kernels.
struct IterPlan {
  int line_grid, node_grid, xs_grid, inner_grid, dsum_grid;  // 0: the kernel has no work
  int lean_grid;   // residual-free node pass (T % 4 == 0 and plain ADMM only)
  int n_slabs, slab_k;  // contingency slabs of the line / node kernels, slab_k contingencies each
  size_t inner_smem;
  int inner_c;     // register chunk of the inner-ADMM kernel (0: shared-memory path)
  int dsum_lean;   // 1: the passes without residuals sum device powers themselves (dsum only where
                   // residuals are formed); for instances whose device chain the line pass cannot hide
};

// A batch of instances: the CTA schedules of each batch kernel, concatenated
// in one array of (instance, block within the instance, blocks of the
// instance, 0), in the order of BatchKernel.
enum BatchKernel { BK_XS4, BK_XS1, BK_INNER, BK_DSUM2, BK_DSUM1, BK_LINE4, BK_LINE1, BK_NODE4, BK_NODE1,
                   BK_DECIDE, BK_COUNT };
struct BatchPlan {
  int count[BK_COUNT];
  int offset[BK_COUNT];
  size_t inner_smem;
  int inner_c;  // register chunk of the batch's inner-ADMM kernel (0: shared-memory path)
  int relax;   // the instances run over-relaxed (alpha != 1): the node kernels that carry it
};
// How a batch schedule lays out CTAs: instances in `order` (NULL: as given),
// each instance's CTAs of a phase contiguous or dealt round-robin across
// instances, and `div` times fewer CTAs for the grid-stride phases (xs,
// inner, dsum), each doing proportionally more work.
struct BatchLayout {
  const int *order;
  int interleave;
  int div;
};

}  // namespace opfk

// Launch wrappers implemented in opf_kernels.cu (host callable).
extern "C++" {
// Record the message returned by opf_last_error (opf_api.cu) and pass s on.
int opf_record_error(int s, const char *msg);
// Grids of the iteration kernels for this problem on the current device.
int opfk_plan(const opfk::Params &p, opfk::IterPlan *plan);
// Start a call of n iterations: the residuals are formed at its last one;
// clear_stop restarts a context that stopped (opf_iterate, not batches).
int opfk_begin_launch(opfk::DevScalars *sc, long long n, int clear_stop, void *stream);
int opfk_begin_batch_launch(const opfk::Params *d_params, int n_inst, long long n, void *stream);
// Enqueue one iteration: xs, inner, dsum, the node kernels and decide on
// main_stream, the line kernels on aux_stream (forked after the previous
// iteration; each slab joined before its node kernel).  Works under stream
// capture.
int opfk_iteration_enqueue(const opfk::Params &p, const opfk::IterPlan &plan, void *main_stream,
                           void *aux_stream, void *ev_fork, void *ev_join);
// Schedules of the batch kernels for n instances (host parameter copies and
// their plans): fills sched (4 ints per CTA, BatchPlan order) and the plan.
int opfk_batch_plan(const opfk::Params *hp, const opfk::IterPlan *plans, int n, const opfk::BatchLayout &lay,
                    int *sched_out, long long sched_cap, long long *sched_len, opfk::BatchPlan *bp);
// Node CTAs (and partial sums) of an instance under a layout's `div`: the
// batch's copy of the instance's Params must carry it as node_grid.
int opfk_batch_node_blocks(const opfk::IterPlan &plan, int div);
// Enqueue one iteration of every instance: d_params [n] and d_sched on the
// device; the same stream and event roles as opfk_iteration_enqueue.
int opfk_batch_enqueue(const opfk::Params *d_params, const int *d_sched, const opfk::BatchPlan &bp,
                       void *main_stream, void *aux_stream, void *ev_fork, void *ev_join);
// State import / export between internal and caller numbering; `cur` selects
// the node buffer holding the current state.
int opfk_import_launch(const opfk::Params &p, int cur, const float *p_line, const float *th1,
                       const float *th2, const float *v1, const float *v2, const float *u,
                       void *stream);
int opfk_node_average_launch(const opfk::Params &p, int cur, void *stream);
// Starting state from node rows [T][N][stride] (price / price_scale, angle),
// caller numbering; u = -price * u_scale
int opfk_start_from_nodes_launch(const opfk::Params &p, int cur, const float *rows, int stride,
                                 float price_scale, float u_scale, void *stream);
int opfk_project_v_launch(const opfk::Params &p, int cur, void *stream);
int opfk_export_lines_launch(const opfk::Params &p, int cur, float *p_line, float *th1, float *th2,
                             float *v1, float *v2, void *stream);
// Device powers [S][T] (caller order = internal order) of the actual iterate.
int opfk_export_pdev_launch(const opfk::Params &p, float *out, void *stream);
int opfk_export_nodes_launch(const opfk::Params &p, int cur, float *u, float *theta_node,
                             float *price, void *stream);
int opfk_set_rho_launch(opfk::DevScalars *sc, double rho, void *stream);
// Contingency slices: the local half of one iteration (devices from the
// exchanged sums, line proxes, node sums, then this slice's sums into the
// exchange buffer) and the decisions from the exchanged sums; `prime`
// writes the sums of the current state (before the first iteration).
int opfk_slice_local_enqueue(const opfk::Params &p, const opfk::IterPlan &plan, void *main_stream,
                             void *aux_stream, void *ev_fork, void *ev_join);
int opfk_slice_finish_enqueue(const opfk::Params &p, void *stream);
int opfk_slice_prime_launch(const opfk::Params &p, void *stream);
}

#endif  // OPF_INTERNAL_H_
