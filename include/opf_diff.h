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
 *              + sum_batteries cost . delta
 *
 * and its gradient with respect to the load power P [D][T], the generator
 * capacity pmax [G][T] and the line limits u [L], by a hand-written reverse
 * pass over the iterations (adjoint kernels of the line prox, the device
 * proxes, the node averages and the price updates).  The forward pass keeps
 * a record of its clipping decisions (opf_diff_set_record_limit); the reverse
 * pass then reads no state.  Without the record the forward states are kept
 * every `checkpoint_every` iterations and recomputed in between.  A call
 * uses the context's stream and a second stream of its own, created by the
 * first gradient call; it returns after both are done.
 *
 * Every device type is covered.  Ramp-limited generators (T > 1) and
 * batteries take their prox from 10 iterations of the Appendix D inner ADMM
 * (omega = (K+1) rho_p, duals beta and lambda carried across outer
 * iterations from zero), differentiated through those iterations; delta is
 * a battery's discharge in the last inner iterate, and a ramp generator's
 * capacity enters through the right-hand side of its p_t <= pmax_t rows.
 * Clipping follows torch.clamp: the clipped value passes its gradient where
 * lo <= x <= hi, a bound receives it where x leaves the interval on its
 * side; the inner projection min(alpha + lambda, 0) is a clamp with upper
 * bound 0.
 *
 * Arrays are in the caller's numbering and layout (opf.h); host pointers
 * (opf_diff_cost_grad_on also takes device pointers).  A context lives on
 * the device current at opf_diff_create; calls on it are made with that
 * device current.  The computation runs
 * in FP32 on the device; the cost is summed in FP64, and so is the line-limit
 * gradient over contingencies and steps.
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
 * rho_p, rho_theta > 0; checkpoint_every >= 1.  OPF_EINVAL for invalid data
 * or a horizon whose inner-ADMM working set does not fit one CTA's shared
 * memory (about T = 600). */
opf_status opf_diff_create(const opf_network *net, int32_t horizon_T, const opf_contingencies *ctg,
                           double rho_p, double rho_theta, int32_t checkpoint_every,
                           void *cuda_stream, opf_diff **out);

/* Run K >= 1 iterations from zero with the given data (NULL: the network's
 * own load_p [D][T], gen_pmax [G][T], line_u [L]) and return the cost and
 * its gradients (each output may be NULL).  Synchronizes. */
opf_status opf_diff_cost_grad(opf_diff *d, int32_t K, const float *load_p, const float *gen_pmax,
                              const float *line_u, double *cost, float *grad_load_p,
                              float *grad_gen_pmax, float *grad_line_u);

/* The same with every array on the device when on_device != 0 (device
 * pointers of the context's device; the cost stays a host double), or on the
 * host when 0.  The buffers a call needs (checkpoints, one segment of states,
 * adjoints) are kept by the context and reused by later calls. */
opf_status opf_diff_cost_grad_on(opf_diff *d, int32_t K, int32_t on_device, const float *load_p,
                                 const float *gen_pmax, const float *line_u, double *cost, float *grad_load_p,
                                 float *grad_gen_pmax, float *grad_line_u);

/* The most device memory (bytes) a gradient call may keep for its record of
 * the forward pass: per iteration, which inner-ADMM rows clipped (one byte
 * per row and inner iteration) and where each line's and closed-form
 * device's unclipped value lay (one byte per line item and device step).
 * With the record the reverse pass runs no inner iteration, recomputes no
 * prox input and no state; a call whose record would exceed the limit (and
 * every call after a limit of 0) recomputes them from the checkpointed
 * states instead, with the same result bit for bit.  Default 4 GiB.
 * OPF_EINVAL for d NULL or bytes < 0. */
opf_status opf_diff_set_record_limit(opf_diff *d, int64_t bytes);

void opf_diff_destroy(opf_diff *d);

#ifdef __cplusplus
}
#endif

#endif /* OPF_DIFF_H_ */
