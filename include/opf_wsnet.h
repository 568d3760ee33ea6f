/*
 * opf_wsnet.h -- C ABI of the learned warm-start network.
 *
 * The paper has no counterpart: its warm start (Section 3.4) reuses a
 * previous solution.  This network proposes initial nodal prices and node
 * angles for the message-passing iteration from node features; the
 * iteration then runs unchanged to the same tolerance, so its own stopping
 * test still certifies the answer.
 *
 * Model (rows r = t * N + n, the same weights at every time step t):
 *   H0 = relu(X W0 + b0)                       X  [R][F],  W0 [F][64]
 *   H' = relu(H Ws + (A H) Wn + b)  x 3        Ws, Wn [64][64]
 *   Y  = H3 Wo + bo                            Wo [64][2], Y [R][2]
 * where (A H)[t, n] = sum over the lines l at n of w_{l,n} H[t, other end],
 * w_{l,n} = b_l / (sum of b over the lines at n); 0 for a node without lines.
 * Loss: mean over rows of sum_o scale[o] (Y[r][o] - Y*[r][o])^2.
 *
 * Parameters are one FP32 vector in the order W0, b0, (Ws, Wn, b) x 3, Wo,
 * bo, matrices row-major [in][out]: 64 F + 64 + 3 (2 * 4096 + 64) + 128 + 2
 * values.  The kernels use the matrices rounded to bfloat16 (round to nearest
 * even) and accumulate in FP32; gradients treat the rounding as the identity.
 * Training uses Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 vector.
 *
 * All GPU work is enqueued on the stream given at creation; functions that
 * return host data synchronize it.  Device pointers are of the current device.
 */
#ifndef OPF_WSNET_H_
#define OPF_WSNET_H_

#include <stdint.h>

#include "opf.h"

#ifdef __cplusplus
extern "C" {
#endif

#define OPF_WSNET_HIDDEN 64
#define OPF_WSNET_OUT 2

typedef struct opf_wsnet opf_wsnet; /* opaque */

/* Number of parameters for F input features. */
int64_t opf_wsnet_param_count(int32_t n_features);

/* Build the network for one bus graph and horizon T (R = T * n_nodes rows).
 * Lines are node pairs with susceptance line_b > 0 (host arrays, copied).
 * params: NULL for He-uniform weights from `seed` and zero biases, else
 * opf_wsnet_param_count(n_features) FP32 host values.  Allocates the
 * parameters, Adam state and activations of R rows on the device. */
opf_status opf_wsnet_create(int32_t n_nodes, int32_t n_lines, const int32_t *line_from,
                            const int32_t *line_to, const double *line_b, int32_t T,
                            int32_t n_features, const float *params, uint64_t seed,
                            void *cuda_stream, opf_wsnet **out);

/* Copy the FP32 parameter vector to / from host memory. */
opf_status opf_wsnet_get_params(opf_wsnet *net, float *params);
opf_status opf_wsnet_set_params(opf_wsnet *net, const float *params);

/* Y [R][2] from X [R][F] (device pointers).  Asynchronous. */
opf_status opf_wsnet_forward(opf_wsnet *net, const float *x, float *y);

/* Loss and its gradient with respect to the parameter vector (host outputs;
 * either may be NULL) for inputs X and targets Y* [R][2] on the device,
 * without changing the parameters.  Synchronizes. */
opf_status opf_wsnet_gradient(opf_wsnet *net, const float *x, const float *y_target,
                              const float scale[2], double *loss, float *grad);

/* One Adam step with learning rate lr on the loss of (X, Y*); *loss (may be
 * NULL) receives the loss before the step and then synchronizes. */
opf_status opf_wsnet_train_step(opf_wsnet *net, const float *x, const float *y_target,
                                const float scale[2], float lr, double *loss);

void opf_wsnet_destroy(opf_wsnet *net);

#ifdef __cplusplus
}
#endif

#endif /* OPF_WSNET_H_ */
