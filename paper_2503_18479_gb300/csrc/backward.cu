// backward.cu -- pieces of the adjoint path (paper Eq. 8-10 through d(A^-1) = -A^-1 dA A^-1)
// for a field cotangent grad_B = dL/dRe B + j dL/dIm B:
//   field_adjoint_kernel  u[b][f][k] = sum_p H[p][k] conj(grad_B[b][f][p])   (u = H^T conj(gB))
//   grad_combine_kernel   grad_C = grad_loss * dloss/dC + (field term)
//   count_bad_kernel      number of systems with a nonzero status word
// The solve kernels (solve.cu) then compute mu = A^-1 u and Im(mu_k I_k)/(w C_k^2).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mts {

constexpr int kFaSys = 8;     // systems per CTA (share the H reads)
constexpr int kFaChunk = 128; // points per staged chunk

// CTA = 128 threads (one per port k of the CTA's 128-port slice, blockIdx.z), kFaSys
// configurations of one frequency g. Inner sums over a chunk of points in the working
// precision, outer sums in FP64.
template <typename HT, typename GT>
__global__ void __launch_bounds__(128) field_adjoint_kernel(FieldAdjArgs a) {
  __shared__ GT sg[kFaSys][kFaChunk];
  const int g = blockIdx.x;
  const int64_t b0 = (int64_t)blockIdx.y * kFaSys;
  const int s = a.t.freq_struct[g];
  const int f = g - a.freq_off[s];
  const int N = a.port_off[s + 1] - a.port_off[s];
  if ((int)blockIdx.z * 128 >= N) return;  // slice beyond this structure's ports (CTA-uniform)
  const int64_t P = a.point_off[s + 1] - a.point_off[s];
  const int k = (int)blockIdx.z * 128 + threadIdx.x;
  const HT* H = static_cast<const HT*>(a.H) + a.t.pn_off[s];
  const GT* gB = static_cast<const GT*>(a.grad_B);
  double accx[kFaSys], accy[kFaSys];
#pragma unroll
  for (int i = 0; i < kFaSys; ++i) accx[i] = accy[i] = 0.0;
  for (int64_t p0 = 0; p0 < P; p0 += kFaChunk) {
    __syncthreads();
    for (int e = threadIdx.x; e < kFaSys * kFaChunk; e += blockDim.x) {
      int i = e / kFaChunk, q = e % kFaChunk;
      int64_t b = b0 + i;
      GT v;
      v.x = 0;
      v.y = 0;
      if (b < a.n_cfg && p0 + q < P) v = gB[b * a.sumFP + a.t.fp_off[s] + (int64_t)f * P + p0 + q];
      sg[i][q] = v;
    }
    __syncthreads();
    if (k < N) {
      HT cx[kFaSys], cy[kFaSys];
#pragma unroll
      for (int i = 0; i < kFaSys; ++i) cx[i] = cy[i] = 0;
      int qn = (int)min((int64_t)kFaChunk, P - p0);
      for (int q = 0; q < qn; ++q) {
        HT h = H[(p0 + q) * N + k];
#pragma unroll
        for (int i = 0; i < kFaSys; ++i) {
          cx[i] += h * sg[i][q].x;
          cy[i] -= h * sg[i][q].y;  // conj
        }
      }
#pragma unroll
      for (int i = 0; i < kFaSys; ++i) {
        accx[i] += (double)cx[i];
        accy[i] += (double)cy[i];
      }
    }
  }
  if (k < N) {
#pragma unroll
    for (int i = 0; i < kFaSys; ++i) {
      int64_t b = b0 + i;
      if (b < a.n_cfg) {
        double* up = a.u + 2 * (b * a.sumFN + a.t.fn_off[s] + (int64_t)f * N + k);
        up[0] = accx[i];
        up[1] = accy[i];
      }
    }
  }
}

cudaError_t launch_field_adjoint_rhs(const FieldAdjArgs& a, mts_precision prec, int max_ports,
                                     cudaStream_t st) {
  if (max_ports > kMaxPorts) return cudaErrorNotSupported;
  dim3 grid((unsigned)a.n_freq, (unsigned)((a.n_cfg + kFaSys - 1) / kFaSys),
            (unsigned)((max_ports + 127) / 128));
  if (prec == MTS_FP64)
    field_adjoint_kernel<double, double2><<<grid, 128, 0, st>>>(a);
  else
    field_adjoint_kernel<float, float2><<<grid, 128, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

__global__ void grad_combine_kernel(int64_t n_cfg, int n_struct, int n_ports,
                                    const int32_t* __restrict__ port_off,
                                    const double* __restrict__ grad_loss,
                                    const double* __restrict__ dldc,
                                    const double* __restrict__ gfield, double* __restrict__ grad_C) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cfg * n_ports) return;
  int64_t b = i / n_ports;
  int port = (int)(i - b * n_ports);
  double v = 0.0;
  if (grad_loss) {
    int s = find_struct_i32(port_off, n_struct, port);
    v = grad_loss[b * n_struct + s] * dldc[i];
  }
  if (gfield) v += gfield[i];
  grad_C[i] = v;
}

cudaError_t launch_grad_combine(int64_t n_cfg, int n_struct, int n_ports,
                                const int32_t* port_off, const double* grad_loss,
                                const double* dldc, const double* gfield, double* grad_C,
                                cudaStream_t st) {
  int64_t n = n_cfg * n_ports;
  if (n == 0) return cudaSuccess;
  grad_combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_cfg, n_struct, n_ports,
                                                                   port_off, grad_loss, dldc,
                                                                   gfield, grad_C);
  note_launch();
  return cudaGetLastError();
}

__global__ void count_bad_kernel(const int32_t* __restrict__ status, int64_t n, int32_t* out) {
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += status[i] != 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// dloss/dR_k = sum_f -Re(mu_k I_k), dloss/dL_k = sum_f w Im(mu_k I_k) (dA/dR_k = e_k e_k^T,
// dA/dM_kk = j w e_k e_k^T in d(A^-1) = -A^-1 dA A^-1, Eq. 8-9), divided by F_s L_s like the
// objective and weighted by the loss cotangent of the port's structure.
__global__ void param_grad_kernel(int64_t n_cfg, int n_struct, int n_ports,
                                  const int32_t* __restrict__ port_off,
                                  const int32_t* __restrict__ freq_off,
                                  const int32_t* __restrict__ loss_off, DevTables t, int64_t sumFN,
                                  const double* __restrict__ omega, const double* __restrict__ I,
                                  const double* __restrict__ mu, const double* __restrict__ grad_loss,
                                  double* __restrict__ grad_R, double* __restrict__ grad_L) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cfg * n_ports) return;
  const int64_t b = i / n_ports;
  const int port = (int)(i - b * n_ports);
  const int s = find_struct_i32(port_off, n_struct, port);
  const int N = port_off[s + 1] - port_off[s], k = port - port_off[s];
  const int F = freq_off[s + 1] - freq_off[s];
  const int L = loss_off[s + 1] - loss_off[s];
  double gr = 0.0, gl = 0.0;
  for (int f = 0; f < F; ++f) {
    const int64_t o = 2 * (b * sumFN + t.fn_off[s] + (int64_t)f * N + k);
    const double px = mu[o] * I[o] - mu[o + 1] * I[o + 1];  // Re(mu I)
    const double py = mu[o] * I[o + 1] + mu[o + 1] * I[o];  // Im(mu I)
    gr -= px;
    gl += omega[freq_off[s] + f] * py;
  }
  double scale = (F * L > 0) ? 1.0 / ((double)F * L) : 0.0;
  if (grad_loss) scale *= grad_loss[b * n_struct + s];
  if (grad_R) grad_R[i] = gr * scale;
  if (grad_L) grad_L[i] = gl * scale;
}

cudaError_t launch_param_grad(int64_t n_cfg, int n_struct, int n_ports, const int32_t* port_off,
                              const int32_t* freq_off, const int32_t* loss_off, DevTables t,
                              int64_t sumFN, const double* omega, const double* I,
                              const double* mu, const double* grad_loss, double* grad_R,
                              double* grad_L, cudaStream_t st) {
  const int64_t n = n_cfg * n_ports;
  if (n == 0) return cudaSuccess;
  param_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      n_cfg, n_struct, n_ports, port_off, freq_off, loss_off, t, sumFN, omega, I, mu, grad_loss,
      grad_R, grad_L);
  note_launch();
  return cudaGetLastError();
}

// dloss/dw_g with the drive held fixed (dA/dw = j M + diag(j/(w^2 C))):
//   Im(mu^T M I) + sum_k Im(mu_k I_k)/(w^2 C_k), divided by F_s L_s, times the loss cotangent.
// One warp per system (b, g); FP64 (an N^2 product per system).
__global__ void omega_grad_kernel(int64_t n_cfg, int n_freq, int n_struct, int n_ports,
                                  const int32_t* __restrict__ port_off,
                                  const int32_t* __restrict__ freq_off,
                                  const int32_t* __restrict__ loss_off, DevTables t,
                                  int64_t sumFN, const double* __restrict__ omega,
                                  const double* __restrict__ C, const double* __restrict__ M64,
                                  const double* __restrict__ I, const double* __restrict__ mu,
                                  const double* __restrict__ grad_loss,
                                  double* __restrict__ grad_w) {
  const int64_t sys = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (sys >= n_cfg * n_freq) return;  // warp-uniform
  const int64_t b = sys / n_freq;
  const int g = (int)(sys - b * n_freq);
  const int s = t.freq_struct[g];
  const int k0 = port_off[s], N = port_off[s + 1] - k0;
  const int F = freq_off[s + 1] - freq_off[s], f = g - freq_off[s];
  const int L = loss_off[s + 1] - loss_off[s];
  const double w = omega[g];
  const double* Ms = M64 + t.nn_off[s];
  const int64_t o = 2 * (b * sumFN + t.fn_off[s] + (int64_t)f * N);
  double im_muMI = 0.0, diag = 0.0;
  for (int k = lane; k < N; k += 32) {
    double tx = 0.0, ty = 0.0;  // (M I)_k
    for (int l = 0; l < N; ++l) {
      const double m = Ms[(int64_t)k * N + l];
      tx = fma(m, I[o + 2 * l], tx);
      ty = fma(m, I[o + 2 * l + 1], ty);
    }
    const double ux = mu[o + 2 * k], uy = mu[o + 2 * k + 1];
    im_muMI += ux * ty + uy * tx;
    const double ck = C[b * n_ports + k0 + k];
    diag += (ux * I[o + 2 * k + 1] + uy * I[o + 2 * k]) / (w * w * ck);
  }
  double v = im_muMI + diag;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) {
    double scale = (F * L > 0) ? 1.0 / ((double)F * L) : 0.0;
    if (grad_loss) scale *= grad_loss[b * n_struct + s];
    grad_w[b * n_freq + g] = v * scale;
  }
}

// cotangent of the drive (dL/dRe V + j dL/dIm V) = conj(mu) / (F_s L_s) times the loss cotangent
__global__ void drive_grad_kernel(int64_t n_cfg, int n_struct, const int32_t* __restrict__ freq_off,
                                  const int32_t* __restrict__ loss_off, DevTables t, int64_t sumFN,
                                  const double* __restrict__ mu, const double* __restrict__ grad_loss,
                                  double* __restrict__ grad_V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cfg * sumFN) return;
  const int64_t b = i / sumFN, e = i - b * sumFN;
  const int s = find_struct_i64(t.fn_off, n_struct, e);
  const int F = freq_off[s + 1] - freq_off[s], L = loss_off[s + 1] - loss_off[s];
  double scale = (F * L > 0) ? 1.0 / ((double)F * L) : 0.0;
  if (grad_loss) scale *= grad_loss[b * n_struct + s];
  grad_V[2 * i] = mu[2 * i] * scale;
  grad_V[2 * i + 1] = -mu[2 * i + 1] * scale;
}

cudaError_t launch_omega_v_grad(int64_t n_cfg, int n_freq, int n_struct, int n_ports,
                                const int32_t* port_off, const int32_t* freq_off,
                                const int32_t* loss_off, DevTables t, int64_t sumFN,
                                const double* omega, const double* C, const double* M64,
                                const double* I, const double* mu, const double* grad_loss,
                                double* grad_w, double* grad_V, cudaStream_t st) {
  if (grad_w && n_cfg * n_freq > 0) {
    const int64_t threads = n_cfg * n_freq * 32;
    omega_grad_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        n_cfg, n_freq, n_struct, n_ports, port_off, freq_off, loss_off, t, sumFN, omega, C, M64,
        I, mu, grad_loss, grad_w);
    note_launch();
  }
  if (grad_V && n_cfg * sumFN > 0) {
    const int64_t n = n_cfg * sumFN;
    drive_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_cfg, n_struct, freq_off,
                                                                  loss_off, t, sumFN, mu,
                                                                  grad_loss, grad_V);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_count_bad(const int32_t* status, int64_t n, int32_t* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(int32_t), st);
  if (n > 0) {
    count_bad_kernel<<<64, 256, 0, st>>>(status, n, out);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace mts
