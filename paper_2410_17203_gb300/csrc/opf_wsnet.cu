// Learned warm-start network (include/opf_wsnet.h): forward pass, backward
// pass and Adam for a three-layer message-passing network over the bus graph.
// The paper has no counterpart; the network only proposes a starting point
// for the message-passing iteration.
//
// Layout: activations are row-major [R][64] with rows r = t * N + n.  The
// layers are small dense contractions (64 x 64) over many rows, so each
// linear kernel stages the bfloat16 weights of a layer in shared memory as
// FP32 and a tile of 32 input rows, and every thread accumulates eight
// outputs in FP32.  Weight gradients are reduced per CTA over fixed row
// ranges and then across CTAs in a fixed order, so results are
// deterministic.  The neighbour average and its adjoint are CSR gathers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "opf_internal.h"
#include "opf_wsnet.h"

namespace {

constexpr int HID = OPF_WSNET_HIDDEN;
constexpr int NOUT = OPF_WSNET_OUT;
constexpr int NMP = 3;         // message-passing layers
constexpr int TB = 256;        // threads per CTA
constexpr int ROWS = 32;       // rows per CTA in the linear kernels
constexpr int GRAD_ROWS = 256; // rows per CTA in the weight-gradient partial sums

// ---------------------------------------------------------------------------
// out[r][j] = act(sum_k a[r][k] W(k, j) + sum_k a2[r][k] W2(k, j) + bias[j]
//                 + (accum ? out[r][j] : 0)),  W(k, j) = W[k * J + j], or
// W[j * K + k] with TRANS (the product with W transposed, for the backward
// pass).  `pre` (optional) receives the value before the activation.
// ---------------------------------------------------------------------------
template <bool TRANS>
__global__ void __launch_bounds__(TB) linear_kernel(const float *__restrict__ a, const __nv_bfloat16 *__restrict__ W,
                                                    const float *__restrict__ a2,
                                                    const __nv_bfloat16 *__restrict__ W2,
                                                    const float *__restrict__ bias, float *out, float *pre,
                                                    int R, int K, int J, int relu, int accum) {
  __shared__ float ws[HID * HID], ws2[HID * HID];
  __shared__ float at[ROWS * HID], at2[ROWS * HID];
  const int r0 = blockIdx.x * ROWS;
  for (int i = threadIdx.x; i < K * J; i += TB) {
    const int k = i / J, j = i - k * J;
    const int src = TRANS ? j * K + k : k * J + j;
    ws[i] = __bfloat162float(W[src]);
    if (W2) ws2[i] = __bfloat162float(W2[src]);
  }
  for (int i = threadIdx.x; i < ROWS * K; i += TB) {
    const int rr = i / K, k = i - rr * K;
    const int r = r0 + rr;
    at[i] = r < R ? a[(size_t)r * K + k] : 0.f;
    if (a2) at2[i] = r < R ? a2[(size_t)r * K + k] : 0.f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ROWS * J; o += TB) {
    const int rr = o / J, j = o - rr * J;
    const int r = r0 + rr;
    if (r >= R) continue;
    float s = 0.f;
    for (int k = 0; k < K; ++k) s = fmaf(at[rr * K + k], ws[k * J + j], s);
    if (a2)
      for (int k = 0; k < K; ++k) s = fmaf(at2[rr * K + k], ws2[k * J + j], s);
    if (bias) s += bias[j];
    const size_t oi = (size_t)r * J + j;
    if (accum) s += out[oi];
    if (pre) pre[oi] = s;
    out[oi] = relu ? fmaxf(s, 0.f) : s;
  }
}

// The same for J = 64 outputs, register-tiled: a CTA computes TROWS rows x
// 64 columns, each thread 8 rows x 4 columns in registers (32 products per
// 12 shared-memory reads), with the layer's weights staged once per TROWS
// rows (the kernel above re-stages them for every 32 rows and runs one
// dependent chain of K products per output).  Shared memory: the weights
// [K][64] (twice with a2) and the row tiles [TROWS][K + 1] (the padding
// spreads a column's rows over the banks).
constexpr int TROWS = 128;

__host__ __device__ inline size_t linear64_smem(int K, bool two) {
  return ((size_t)(two ? 2 : 1) * (K * HID + TROWS * (K + 1))) * sizeof(float);
}

template <bool TRANS>
__global__ void __launch_bounds__(TB) linear64_kernel(const float *__restrict__ a, const __nv_bfloat16 *__restrict__ W,
                                                      const float *__restrict__ a2,
                                                      const __nv_bfloat16 *__restrict__ W2,
                                                      const float *__restrict__ bias, float *out, float *pre, int R,
                                                      int K, int relu, int accum) {
  extern __shared__ float sm64[];
  const int KP = K + 1;
  float *ws = sm64, *at = ws + K * HID;
  float *ws2 = at + TROWS * KP, *at2 = ws2 + K * HID;
  const int r0 = blockIdx.x * TROWS;
  for (int i = threadIdx.x; i < K * HID; i += TB) {
    const int k = i / HID, j = i - k * HID;
    const int src = TRANS ? j * K + k : k * HID + j;
    ws[i] = __bfloat162float(W[src]);
    if (a2) ws2[i] = __bfloat162float(W2[src]);
  }
  for (int i = threadIdx.x; i < TROWS * K; i += TB) {
    const int rr = i / K, k = i - rr * K;
    const int r = r0 + rr;
    at[rr * KP + k] = r < R ? a[(size_t)r * K + k] : 0.f;
    if (a2) at2[rr * KP + k] = r < R ? a2[(size_t)r * K + k] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // columns 4 tx .. 4 tx + 3, rows 8 ty .. 8 ty + 7
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  for (int pass = 0; pass < (a2 ? 2 : 1); ++pass) {
    const float *A = pass ? at2 : at, *Ws = pass ? ws2 : ws;
    for (int k = 0; k < K; ++k) {
      const float4 w4 = *reinterpret_cast<const float4 *>(Ws + k * HID + 4 * tx);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float av = A[(8 * ty + i) * KP + k];
        acc[i][0] = fmaf(av, w4.x, acc[i][0]);
        acc[i][1] = fmaf(av, w4.y, acc[i][1]);
        acc[i][2] = fmaf(av, w4.z, acc[i][2]);
        acc[i][3] = fmaf(av, w4.w, acc[i][3]);
      }
    }
  }
  float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (bias) b4 = *reinterpret_cast<const float4 *>(bias + 4 * tx);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + 8 * ty + i;
    if (r >= R) break;
    const size_t oi = (size_t)r * HID + 4 * tx;
    float4 v = make_float4(acc[i][0] + b4.x, acc[i][1] + b4.y, acc[i][2] + b4.z, acc[i][3] + b4.w);
    if (accum) {
      const float4 o = *reinterpret_cast<const float4 *>(out + oi);
      v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    if (pre) *reinterpret_cast<float4 *>(pre + oi) = v;
    if (relu) {
      v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
    }
    *reinterpret_cast<float4 *>(out + oi) = v;
  }
}

// out[t, n][c] = sum_{j in ptr[n]..ptr[n+1]} w[j] in[t, nbr[j]][c]
__global__ void __launch_bounds__(TB) agg_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                 const int *__restrict__ ptr, const int *__restrict__ nbr,
                                                 const float *__restrict__ w, int N, int R) {
  const size_t total = (size_t)R * HID;
  for (size_t i = (size_t)blockIdx.x * TB + threadIdx.x; i < total; i += (size_t)gridDim.x * TB) {
    const int r = (int)(i / HID), c = (int)(i - (size_t)r * HID);
    const int t = r / N, n = r - t * N;
    float s = 0.f;
    for (int j = ptr[n]; j < ptr[n + 1]; ++j) s = fmaf(w[j], in[((size_t)t * N + nbr[j]) * HID + c], s);
    out[i] = s;
  }
}

// g *= (z > 0)
__global__ void __launch_bounds__(TB) relu_bwd_kernel(float *g, const float *__restrict__ z, size_t n) {
  for (size_t i = (size_t)blockIdx.x * TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB)
    if (!(z[i] > 0.f)) g[i] = 0.f;
}

// part[cta][k][j] = sum over the CTA's rows of a[r][k] g[r][j] (a == NULL:
// a = 1, K = 1, the bias gradient)
__global__ void __launch_bounds__(TB) wgrad_part_kernel(const float *__restrict__ a, const float *__restrict__ g,
                                                        float *__restrict__ part, int R, int K, int J) {
  __shared__ float at[ROWS * HID], gt[ROWS * HID];
  const int r0 = blockIdx.x * GRAD_ROWS, r1 = min(R, r0 + GRAD_ROWS);
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int rb = r0; rb < r1; rb += ROWS) {
    const int nr = min(ROWS, r1 - rb);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * K; i += TB) {
      const int rr = i / K, k = i - rr * K;
      at[i] = rr < nr ? (a ? a[(size_t)(rb + rr) * K + k] : 1.f) : 0.f;
    }
    for (int i = threadIdx.x; i < ROWS * J; i += TB) {
      const int rr = i / J, j = i - rr * J;
      gt[i] = rr < nr ? g[(size_t)(rb + rr) * J + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int o = threadIdx.x + q * TB;
      if (o < K * J) {
        const int k = o / J, j = o - k * J;
        float s = acc[q];
        for (int rr = 0; rr < nr; ++rr) s = fmaf(at[rr * K + k], gt[rr * J + j], s);
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int o = threadIdx.x + q * TB;
    if (o < K * J) part[(size_t)blockIdx.x * K * J + o] = acc[q];
  }
}

// The same for J = 64 and K <= 64, register-tiled: thread (ty, tx) keeps the
// 4 x 4 block k = 4 ty .., j = 4 tx .. of the partial sums (16 products per 8
// shared-memory reads); every output still sums the CTA's rows in order, so
// the partial sums equal the kernel above's.
__global__ void __launch_bounds__(TB) wgrad64_part_kernel(const float *__restrict__ a, const float *__restrict__ g,
                                                          float *__restrict__ part, int R, int K) {
  __shared__ __align__(16) float at[ROWS * HID], gt[ROWS * HID];
  const int r0 = blockIdx.x * GRAD_ROWS, r1 = min(R, r0 + GRAD_ROWS);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  for (int rb = r0; rb < r1; rb += ROWS) {
    const int nr = min(ROWS, r1 - rb);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * HID; i += TB) {
      const int rr = i / HID, k = i - rr * HID;
      at[i] = (rr < nr && k < K) ? a[(size_t)(rb + rr) * K + k] : 0.f;
      gt[i] = rr < nr ? g[(size_t)(rb + rr) * HID + k] : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
      const float4 a4 = *reinterpret_cast<const float4 *>(at + rr * HID + 4 * ty);
      const float4 g4 = *reinterpret_cast<const float4 *>(gt + rr * HID + 4 * tx);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(av[i], gv[c], acc[i][c]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = 4 * ty + i;
    if (k < K)
      *reinterpret_cast<float4 *>(part + (size_t)blockIdx.x * K * HID + (size_t)k * HID + 4 * tx) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

// grad[o] = sum over CTAs c (in order) of part[c][o]
__global__ void __launch_bounds__(TB) wgrad_sum_kernel(const float *__restrict__ part, float *__restrict__ grad,
                                                       int n_part, int KJ) {
  const int o = blockIdx.x * TB + threadIdx.x;
  if (o >= KJ) return;
  float s = 0.f;
  for (int c = 0; c < n_part; ++c) s += part[(size_t)c * KJ + o];
  grad[o] = s;
}

// dY = 2 scale (Y - Y*) / R; per-CTA partial loss sums (FP64)
__global__ void __launch_bounds__(TB) loss_kernel(const float *__restrict__ y, const float *__restrict__ yt,
                                                  float *__restrict__ dy, double *__restrict__ lpart, int R,
                                                  float c0, float c1) {
  __shared__ double red[TB];
  double s = 0.0;
  const size_t n = (size_t)R * NOUT;
  for (size_t i = (size_t)blockIdx.x * TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    const float c = (i & 1) ? c1 : c0;
    const float d = y[i] - yt[i];
    dy[i] = 2.f * c * d / (float)R;
    s += (double)c * d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = TB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// Adam on the FP32 parameters, then their bfloat16 copy
__global__ void __launch_bounds__(TB) adam_kernel(float *p, const float *__restrict__ g, float *m, float *v,
                                                  __nv_bfloat16 *pb, long long n, float lr, float bc1, float bc2) {
  for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < n; i += (long long)gridDim.x * TB) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void __launch_bounds__(TB) to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *pb, long long n) {
  for (long long i = (long long)blockIdx.x * TB + threadIdx.x; i < n; i += (long long)gridDim.x * TB)
    pb[i] = __float2bfloat16_rn(p[i]);
}

int grid_for(size_t work) { return (int)std::min<size_t>((work + TB - 1) / TB, 4096); }

}  // namespace

struct opf_wsnet {
  int N = 0, T = 0, F = 0, R = 0;
  cudaStream_t stream = nullptr;
  long long C = 0;  // parameters
  long long oW0 = 0, ob0 = 0, oWs[NMP] = {}, oWn[NMP] = {}, ob[NMP] = {}, oWo = 0, obo = 0;
  int step = 0;
  // device memory
  int *ptr = nullptr, *nbr = nullptr;
  float *wA = nullptr, *wAT = nullptr;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  __nv_bfloat16 *Pb = nullptr;
  float *Z0 = nullptr, *H0 = nullptr, *M[NMP] = {}, *Z[NMP] = {}, *H[NMP] = {}, *Y = nullptr;
  float *dY = nullptr, *dA = nullptr, *dB = nullptr, *dC = nullptr, *part = nullptr;
  double *lpart = nullptr;
  int n_lpart = 0, n_gpart = 0;
  std::vector<void *> allocs;
};

namespace {

opf_status wfail(opf_status s, const char *msg) { return (opf_status)opf_record_error((int)s, msg); }

#define WCK(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return wfail(OPF_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t walloc(opf_wsnet *w, T **p, size_t n) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) w->allocs.push_back(*p);
  return e;
}

void wfree(opf_wsnet *w) {
  for (void *p : w->allocs) cudaFree(p);
  w->allocs.clear();
}

// He-uniform weights from a counter-based generator (splitmix64), zero biases
void he_init(std::vector<float> &p, const opf_wsnet *w, uint64_t seed) {
  uint64_t x = seed;
  auto next = [&]() {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  std::fill(p.begin(), p.end(), 0.f);
  auto fill = [&](long long off, int fan_in, long long n) {
    const double lim = std::sqrt(6.0 / fan_in);
    for (long long i = 0; i < n; ++i) p[off + i] = (float)((2.0 * next() - 1.0) * lim);
  };
  fill(w->oW0, w->F, (long long)w->F * HID);
  for (int l = 0; l < NMP; ++l) {
    fill(w->oWs[l], HID, HID * HID);
    fill(w->oWn[l], HID, HID * HID);
  }
  fill(w->oWo, HID, HID * NOUT);
}

void launch_linear(const opf_wsnet *w, bool trans, const float *a, long long oW, const float *a2, long long oW2,
                   const float *bias, float *out, float *pre, int K, int J, bool relu, bool accum) {
  const __nv_bfloat16 *W = w->Pb + oW, *W2 = a2 ? w->Pb + oW2 : nullptr;
  if (J == HID) {
    const int g = (w->R + TROWS - 1) / TROWS;
    const size_t sm = linear64_smem(K, a2 != nullptr);
    if (trans)
      linear64_kernel<true><<<g, TB, sm, w->stream>>>(a, W, a2, W2, bias, out, pre, w->R, K, relu, accum);
    else
      linear64_kernel<false><<<g, TB, sm, w->stream>>>(a, W, a2, W2, bias, out, pre, w->R, K, relu, accum);
    return;
  }
  const int grid = (w->R + ROWS - 1) / ROWS;
  if (trans)
    linear_kernel<true><<<grid, TB, 0, w->stream>>>(a, W, a2, W2, bias, out, pre, w->R, K, J, relu, accum);
  else
    linear_kernel<false><<<grid, TB, 0, w->stream>>>(a, W, a2, W2, bias, out, pre, w->R, K, J, relu, accum);
}

void launch_wgrad(opf_wsnet *w, const float *a, const float *g, int K, int J, long long off) {
  if (a && J == HID)
    wgrad64_part_kernel<<<w->n_gpart, TB, 0, w->stream>>>(a, g, w->part, w->R, K);
  else
    wgrad_part_kernel<<<w->n_gpart, TB, 0, w->stream>>>(a, g, w->part, w->R, K, J);
  wgrad_sum_kernel<<<(K * J + TB - 1) / TB, TB, 0, w->stream>>>(w->part, w->G + off, w->n_gpart, K * J);
}

void forward(opf_wsnet *w, const float *x) {
  const int R = w->R;
  launch_linear(w, false, x, w->oW0, nullptr, 0, w->P + w->ob0, w->H0, w->Z0, w->F, HID, true, false);
  const float *h = w->H0;
  for (int l = 0; l < NMP; ++l) {
    agg_kernel<<<grid_for((size_t)R * HID), TB, 0, w->stream>>>(h, w->M[l], w->ptr, w->nbr, w->wA, w->N, R);
    launch_linear(w, false, h, w->oWs[l], w->M[l], w->oWn[l], w->P + w->ob[l], w->H[l], w->Z[l], HID, HID, true,
                  false);
    h = w->H[l];
  }
  launch_linear(w, false, h, w->oWo, nullptr, 0, w->P + w->obo, w->Y, nullptr, HID, NOUT, false, false);
}

// loss partials and the gradient in w->G
void backward(opf_wsnet *w, const float *x, const float *yt, const float scale[2]) {
  const int R = w->R;
  const size_t RH = (size_t)R * HID;
  loss_kernel<<<w->n_lpart, TB, 0, w->stream>>>(w->Y, yt, w->dY, w->lpart, R, scale[0], scale[1]);
  launch_wgrad(w, w->H[NMP - 1], w->dY, HID, NOUT, w->oWo);
  launch_wgrad(w, nullptr, w->dY, 1, NOUT, w->obo);
  // dH = dY Wo^T
  float *dH = w->dA, *dM = w->dB, *tmp = w->dC;
  launch_linear(w, true, w->dY, w->oWo, nullptr, 0, nullptr, dH, nullptr, NOUT, HID, false, false);
  for (int l = NMP - 1; l >= 0; --l) {
    relu_bwd_kernel<<<grid_for(RH), TB, 0, w->stream>>>(dH, w->Z[l], RH);   // dZ, in place
    const float *hin = l == 0 ? w->H0 : w->H[l - 1];
    launch_wgrad(w, hin, dH, HID, HID, w->oWs[l]);
    launch_wgrad(w, w->M[l], dH, HID, HID, w->oWn[l]);
    launch_wgrad(w, nullptr, dH, 1, HID, w->ob[l]);
    // dM = dZ Wn^T; dH_in = A^T dM + dZ Ws^T
    launch_linear(w, true, dH, w->oWn[l], nullptr, 0, nullptr, dM, nullptr, HID, HID, false, false);
    agg_kernel<<<grid_for(RH), TB, 0, w->stream>>>(dM, tmp, w->ptr, w->nbr, w->wAT, w->N, R);
    launch_linear(w, true, dH, w->oWs[l], nullptr, 0, nullptr, tmp, nullptr, HID, HID, false, true);
    std::swap(dH, tmp);
  }
  relu_bwd_kernel<<<grid_for(RH), TB, 0, w->stream>>>(dH, w->Z0, RH);
  launch_wgrad(w, x, dH, w->F, HID, w->oW0);
  launch_wgrad(w, nullptr, dH, 1, HID, w->ob0);
}

opf_status read_loss(opf_wsnet *w, double *loss) {
  std::vector<double> lp(w->n_lpart);
  WCK(cudaMemcpyAsync(lp.data(), w->lpart, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, w->stream));
  WCK(cudaStreamSynchronize(w->stream));
  double s = 0.0;
  for (double x : lp) s += x;
  *loss = s / w->R;
  return OPF_OK;
}

}  // namespace

extern "C" {

int64_t opf_wsnet_param_count(int32_t F) {
  return (int64_t)F * HID + HID + NMP * (2 * HID * HID + HID) + HID * NOUT + NOUT;
}

opf_status opf_wsnet_create(int32_t n_nodes, int32_t n_lines, const int32_t *line_from, const int32_t *line_to,
                            const double *line_b, int32_t T, int32_t F, const float *params, uint64_t seed,
                            void *cuda_stream, opf_wsnet **out) {
  if (!out) return wfail(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_nodes < 1 || n_lines < 0 || T < 1 || F < 1 || F > HID)
    return wfail(OPF_EINVAL, "wsnet: need n_nodes >= 1, n_lines >= 0, T >= 1, 1 <= n_features <= 64");
  if ((long long)n_nodes * T * HID >= (1LL << 31)) return wfail(OPF_EINVAL, "wsnet: too many rows");
  if (n_lines > 0 && (!line_from || !line_to || !line_b)) return wfail(OPF_EINVAL, "wsnet: NULL line array");
  std::vector<double> bsum(n_nodes, 0.0);
  for (int l = 0; l < n_lines; ++l) {
    const int f = line_from[l], t = line_to[l];
    if (f < 0 || f >= n_nodes || t < 0 || t >= n_nodes || f == t || !(line_b[l] > 0) || !std::isfinite(line_b[l]))
      return wfail(OPF_EINVAL, "wsnet: bad line (node id, self loop or susceptance)");
    bsum[f] += line_b[l];
    bsum[t] += line_b[l];
  }
  // neighbour lists by node: weight of A (this end) and of A^T (other end)
  std::vector<int> ptr(n_nodes + 1, 0), nbr(2 * (size_t)n_lines);
  std::vector<float> wa(2 * (size_t)n_lines), wat(2 * (size_t)n_lines);
  for (int l = 0; l < n_lines; ++l) {
    ++ptr[line_from[l] + 1];
    ++ptr[line_to[l] + 1];
  }
  for (int n = 0; n < n_nodes; ++n) ptr[n + 1] += ptr[n];
  std::vector<int> fillp(ptr.begin(), ptr.end() - 1);
  for (int l = 0; l < n_lines; ++l) {
    const int f = line_from[l], t = line_to[l];
    const double wf = line_b[l] / bsum[f], wt = line_b[l] / bsum[t];
    int j = fillp[f]++;
    nbr[j] = t;
    wa[j] = (float)wf;
    wat[j] = (float)wt;
    j = fillp[t]++;
    nbr[j] = f;
    wa[j] = (float)wt;
    wat[j] = (float)wf;
  }
  auto *w = new (std::nothrow) opf_wsnet();
  if (!w) return wfail(OPF_ENOMEM, "host allocation failed");
  w->N = n_nodes;
  w->T = T;
  w->F = F;
  w->R = n_nodes * T;
  w->stream = (cudaStream_t)cuda_stream;
  w->C = opf_wsnet_param_count(F);
  long long o = 0;
  w->oW0 = o; o += (long long)F * HID;
  w->ob0 = o; o += HID;
  for (int l = 0; l < NMP; ++l) {
    w->oWs[l] = o; o += HID * HID;
    w->oWn[l] = o; o += HID * HID;
    w->ob[l] = o; o += HID;
  }
  w->oWo = o; o += HID * NOUT;
  w->obo = o; o += NOUT;
  w->n_lpart = 256;
  w->n_gpart = (w->R + GRAD_ROWS - 1) / GRAD_ROWS;
  const size_t RH = (size_t)w->R * HID;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto **p, size_t n) {
    if (e == cudaSuccess) e = walloc(w, p, n);
  };
  A(&w->ptr, n_nodes + 1);
  A(&w->nbr, nbr.size());
  A(&w->wA, wa.size());
  A(&w->wAT, wat.size());
  A(&w->P, w->C);
  A(&w->G, w->C);
  A(&w->Mo, w->C);
  A(&w->Vo, w->C);
  A(&w->Pb, w->C);
  A(&w->Z0, RH);
  A(&w->H0, RH);
  for (int l = 0; l < NMP; ++l) {
    A(&w->M[l], RH);
    A(&w->Z[l], RH);
    A(&w->H[l], RH);
  }
  A(&w->Y, (size_t)w->R * NOUT);
  A(&w->dY, (size_t)w->R * NOUT);
  A(&w->dA, RH);
  A(&w->dB, RH);
  A(&w->dC, RH);
  A(&w->part, (size_t)w->n_gpart * HID * HID);
  A(&w->lpart, w->n_lpart);
  // the register-tiled layers use up to 97 KB of shared memory per CTA
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(linear64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)linear64_smem(HID, true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(linear64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)linear64_smem(HID, true));
  std::vector<float> p0(w->C);
  if (params) std::memcpy(p0.data(), params, w->C * sizeof(float));
  else he_init(p0, w, seed);
  if (e == cudaSuccess) e = cudaMemcpy(w->ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_lines > 0) {
    e = cudaMemcpy(w->nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->wA, wa.data(), wa.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->wAT, wat.data(), wat.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(w->P, p0.data(), w->C * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(w->Mo, 0, w->C * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(w->Vo, 0, w->C * sizeof(float));
  if (e == cudaSuccess) {
    to_bf16_kernel<<<grid_for(w->C), TB>>>(w->P, w->Pb, w->C);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    const opf_status s = e == cudaErrorMemoryAllocation ? wfail(OPF_ENOMEM, "wsnet: device allocation failed")
                                                        : wfail(OPF_ECUDA, cudaGetErrorString(e));
    wfree(w);
    delete w;
    return s;
  }
  *out = w;
  return OPF_OK;
}

opf_status opf_wsnet_get_params(opf_wsnet *w, float *params) {
  if (!w || !params) return wfail(OPF_EINVAL, "NULL argument");
  WCK(cudaMemcpyAsync(params, w->P, w->C * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
  WCK(cudaStreamSynchronize(w->stream));
  return OPF_OK;
}

opf_status opf_wsnet_set_params(opf_wsnet *w, const float *params) {
  if (!w || !params) return wfail(OPF_EINVAL, "NULL argument");
  WCK(cudaMemcpyAsync(w->P, params, w->C * sizeof(float), cudaMemcpyHostToDevice, w->stream));
  to_bf16_kernel<<<grid_for(w->C), TB, 0, w->stream>>>(w->P, w->Pb, w->C);
  WCK(cudaGetLastError());
  WCK(cudaStreamSynchronize(w->stream));
  return OPF_OK;
}

opf_status opf_wsnet_forward(opf_wsnet *w, const float *x, float *y) {
  if (!w || !x || !y) return wfail(OPF_EINVAL, "NULL argument");
  forward(w, x);
  WCK(cudaMemcpyAsync(y, w->Y, (size_t)w->R * NOUT * sizeof(float), cudaMemcpyDeviceToDevice, w->stream));
  WCK(cudaGetLastError());
  return OPF_OK;
}

opf_status opf_wsnet_gradient(opf_wsnet *w, const float *x, const float *yt, const float scale[2], double *loss,
                              float *grad) {
  if (!w || !x || !yt || !scale) return wfail(OPF_EINVAL, "NULL argument");
  forward(w, x);
  backward(w, x, yt, scale);
  WCK(cudaGetLastError());
  if (grad) WCK(cudaMemcpyAsync(grad, w->G, w->C * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
  if (loss) return read_loss(w, loss);
  WCK(cudaStreamSynchronize(w->stream));
  return OPF_OK;
}

opf_status opf_wsnet_train_step(opf_wsnet *w, const float *x, const float *yt, const float scale[2], float lr,
                                double *loss) {
  if (!w || !x || !yt || !scale) return wfail(OPF_EINVAL, "NULL argument");
  if (!(lr > 0.f) || !std::isfinite(lr)) return wfail(OPF_EINVAL, "wsnet: learning rate must be > 0");
  forward(w, x);
  backward(w, x, yt, scale);
  ++w->step;
  const float bc1 = 1.f - std::pow(0.9f, (float)w->step), bc2 = 1.f - std::pow(0.999f, (float)w->step);
  adam_kernel<<<grid_for(w->C), TB, 0, w->stream>>>(w->P, w->G, w->Mo, w->Vo, w->Pb, w->C, lr, bc1, bc2);
  WCK(cudaGetLastError());
  if (loss) return read_loss(w, loss);
  return OPF_OK;
}

void opf_wsnet_destroy(opf_wsnet *w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  wfree(w);
  delete w;
}

}  // extern "C"
