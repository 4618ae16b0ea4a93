// optim.cu -- the optimisation loop around the forward map (paper Sec. III-C: Adam, at most
// 2000 epochs, learning rate 1e-13 for capacitances of order 1e-12 F; Sec. V-B: clipping to
// a tuning range, or a bounded tanh projection, to keep capacitances realisable).
//
// One Adam step (Kingma and Ba; the update order of torch.optim.Adam without weight decay):
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   theta <- theta - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// on theta = C (no projection, or clipping of C to [c_min, c_max] after the step) or on an
// unconstrained u with C = c_mid + c_half tanh(u) (tanh projection: g_u = g_C c_half (1 -
// tanh(u)^2)). The step counter t lives in device memory so that a captured CUDA graph of
// an epoch can be replayed: the update reads it, a one-thread kernel advances it.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mts {

__global__ void adam_kernel(int64_t n, mts_adam o, double* __restrict__ C, double* __restrict__ u,
                            const double* __restrict__ g, double* __restrict__ m,
                            double* __restrict__ v, const int64_t* __restrict__ step,
                            const double* __restrict__ loss, int64_t n_loss,
                            double* __restrict__ history, int64_t history_len) {
  const int64_t t = step[0] + 1;
  const double bc1 = 1.0 - pow(o.beta1, (double)t);
  const double bc2 = 1.0 - pow(o.beta2, (double)t);
  const double c_mid = 0.5 * (o.c_max + o.c_min), c_half = 0.5 * (o.c_max - o.c_min);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double gi = g[i];
    double th = o.projection == MTS_PROJ_TANH ? u[i] : C[i];
    double th_t = 0.0;
    if (o.projection == MTS_PROJ_TANH) {
      th_t = tanh(th);
      gi = gi * c_half * (1.0 - th_t * th_t);
    }
    const double mi = o.beta1 * m[i] + (1.0 - o.beta1) * gi;
    const double vi = o.beta2 * v[i] + (1.0 - o.beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const double denom = sqrt(vi) / sqrt(bc2) + o.eps;
    th = th - (o.lr / bc1) * (mi / denom);
    if (o.projection == MTS_PROJ_TANH) {
      u[i] = th;
      C[i] = c_mid + c_half * tanh(th);
    } else if (o.projection == MTS_PROJ_CLIP) {
      C[i] = fmin(fmax(th, o.c_min), o.c_max);
    } else {
      C[i] = th;
    }
  }
  // the objective of the configuration this step was computed from, kept per epoch
  if (history != nullptr && t <= history_len)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_loss;
         i += (int64_t)gridDim.x * blockDim.x)
      history[(t - 1) * n_loss + i] = loss[i];
}

__global__ void advance_step_kernel(int64_t* step) { step[0] += 1; }

cudaError_t launch_adam(int64_t n, const mts_adam& o, double* C, double* u, const double* g,
                        double* m, double* v, int64_t* step, const double* loss, int64_t n_loss,
                        double* history, int64_t history_len, cudaStream_t st) {
  const int64_t work = n > n_loss ? n : n_loss;
  const int64_t blocks = work > 0 ? (work + 255) / 256 : 1;
  adam_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(
      n, o, C, u, g, m, v, step, loss, n_loss, history, history_len);
  advance_step_kernel<<<1, 1, 0, st>>>(step);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace mts
