// Internal layout shared by the host side (opf_api.cu) and the kernels
// (opf_kernels.cu).  Not part of the public ABI.
//
// Device memory layout (structure of arrays, time innermost so that every
// row of T floats is one contiguous, 16-byte aligned segment when T % 4 == 0):
//   lines   P, TH1, TH2, V1, V2, DP       [Kp][L][T]   float
//   nodes   U, PBAR, THBAR                [Kp][N][T]   float
//           SPBAR, SU (sums over k)       [N][T]       float
//   devices PD                            [S][T]       float
//   inner ADMM state of ramp generators   lam, beta [n_ramp][4][T],  m [n_ramp][T]
//   inner ADMM state of batteries         lam, beta [n_stor][9][T+1], m [n_stor][T+1]
// V1/V2 hold the phase duals one step behind: the update v += theta - theta_bar
// of iteration i is folded into the line pass of iteration i+1, which already
// reads theta and theta_bar (so v is read and written once per iteration).
#ifndef OPF_INTERNAL_H_
#define OPF_INTERNAL_H_

#include <stdint.h>

namespace opfk {

// residual partial-sum slots (FP64)
// SL_NF counts non-finite node duals: the prox clamps (fminf/fmaxf) would
// otherwise turn a NaN input into a finite bound.
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
  int dual_valid;        // 1: res[1], res[4], res[5] belong to the last iteration
};

// Battery group offsets inside lam/beta rows of stride Tp = T + 1.
enum { SG_E1 = 0, SG_E2 = 1, SG_E3 = 2, SG_CU = 3, SG_CL = 4, SG_DU = 5, SG_DL = 6,
       SG_SU = 7, SG_SL = 8, SG_N = 9 };
// Ramp-generator groups, stride T.
enum { RG_UP = 0, RG_LO = 1, RG_RU = 2, RG_RD = 3, RG_N = 4 };

struct Params {
  int N, L, T, Kp, S;
  int n_closed, n_ramp, n_stor;
  // lines
  const int *line_n1, *line_n2;
  const float *line_b, *line_u;
  const int *out_line;  // [Kp], -1 = no outage (k = 0 always -1)
  float *P, *TH1, *TH2, *V1, *V2;
  float *DP;   // [Kp][L][T] line power change of the iteration (written on residual iterations)
  // nodes
  float *U, *PBAR, *THBAR, *SPBAR, *SU;
  const int *lcsr_ptr, *lcsr_idx;  // line terminals of each node: 2*l + end (end 1 = terminal 2)
  const int *dcsr_ptr, *dcsr_idx;  // devices of each node
  const float *cnt_p, *cnt_th;  // terminals per node: all (power), line terminals (phase)
  // devices (closed-form prox: clip((rho X - b)/(2a + rho), lo, hi))
  float *PD;
  float *DPD;  // [S][T] device power change (residual iterations)
  const int *dev_node;
  const float *dev_a, *dev_b;
  const float *dev_lo, *dev_hi;  // [S][T]
  const int *closed_ids;
  // ramp-limited generators
  const int *ramp_ids;
  const float *ramp_R;
  float *ramp_lam, *ramp_beta, *ramp_m, *ramp_rho;
  // batteries
  const int *stor_ids;
  const float *stor_eff, *stor_P, *stor_dur, *stor_cost;
  float *stor_lam, *stor_beta, *stor_m, *stor_rho, *stor_delta;  // delta [n_stor][T]
  // scratch
  double *partials;        // [2][grid][NSLOT]
  unsigned *bar_count, *bar_gen;
  int *err;
  DevScalars *sc;
  // options
  double eps, mu, gamma, tol;
  int adapt_every, check_every, inner_iters;
  long long barrier_budget;
  int n_iters;
};

}  // namespace opfk

// Launch wrappers implemented in opf_kernels.cu (host callable).
extern "C++" {
int opfk_iteration_launch(const opfk::Params &p, void *stream, int *grid_used, char *msg, int msglen);
int opfk_max_grid(int T, int *grid);
int opfk_node_average_launch(const opfk::Params &p, void *stream);
int opfk_export_v_launch(const opfk::Params &p, float *v1, float *v2, void *stream);
int opfk_price_launch(const opfk::Params &p, float *price, void *stream);
int opfk_project_v_launch(const opfk::Params &p, void *stream);
int opfk_export_u_launch(const opfk::Params &p, float *u, void *stream);
int opfk_set_rho_launch(opfk::DevScalars *sc, double rho, void *stream);
}

#endif  // OPF_INTERNAL_H_
