/*
 * opf_diff.h -- gradients of the system cost after K unrolled iterations.
 *
 * Section 4.4 writes K message-passing iterations as a composition of
 * almost-everywhere differentiable steps; Section 5.5 differentiates the
 * system cost f(p^K) with respect to problem data.  This entry point runs K
 * iterations of Section 3.2 from the zero state with fixed penalties (no
 * adaptation: the adaptive rule is a discrete decision) and returns
 *
 *     f(p^K) = sum_gen (a p^2 + b p) + sum_curtailable voll (p + P)
 *
 * and its gradient with respect to the load power P [D][T], the generator
 * capacity pmax [G][T] and the line limits u [L], by a hand-written reverse
 * pass over the iterations (adjoint kernels of the line prox, the device
 * proxes, the node averages and the price updates).  The forward states are
 * kept every `checkpoint_every` iterations and recomputed in between.
 *
 * Scope: devices with a closed-form prox -- generators without ramp limits
 * (or T = 1), fixed and curtailable loads; networks with batteries or
 * ramp-limited generators are rejected with OPF_EINVAL.  Clipping follows
 * torch.clamp: the clipped value passes its gradient where lo <= x <= hi, a
 * bound receives it where x leaves the interval on its side.
 *
 * Arrays are in the caller's numbering and layout (opf.h); host pointers.
 * The computation runs in FP32 on the device; the cost is summed in FP64.
 */
#ifndef OPF_DIFF_H_
#define OPF_DIFF_H_

#include <stdint.h>

#include "opf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opf_diff opf_diff; /* opaque */

/* Copy the network (as opf_create) for differentiation with penalties
 * rho_p, rho_theta > 0; checkpoint_every >= 1. */
opf_status opf_diff_create(const opf_network *net, int32_t horizon_T, const opf_contingencies *ctg,
                           double rho_p, double rho_theta, int32_t checkpoint_every,
                           void *cuda_stream, opf_diff **out);

/* Run K >= 1 iterations from zero with the given data (NULL: the network's
 * own load_p [D][T], gen_pmax [G][T], line_u [L]) and return the cost and
 * its gradients (each output may be NULL).  Synchronizes. */
opf_status opf_diff_cost_grad(opf_diff *d, int32_t K, const float *load_p, const float *gen_pmax,
                              const float *line_u, double *cost, float *grad_load_p,
                              float *grad_gen_pmax, float *grad_line_u);

void opf_diff_destroy(opf_diff *d);

#ifdef __cplusplus
}
#endif

#endif /* OPF_DIFF_H_ */
