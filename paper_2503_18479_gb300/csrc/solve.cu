// solve.cu -- (b) port solve, (d) objective and (adj) adjoint gradient, one system
// (configuration b, frequency g) per group of NM threads, thread r holding row r.
//
//   A = diag(R) + j w M + diag(1/(j w C_b))    (paper Eq. 2 and Eq. 11; Eq. 6 is the same
//   A I = V                                    linear network solve in scattering form)
//   b_l = sum_k H[l][k] I_k at the loss points (Eq. 7)
//   loss = sum_l e(b_l, t_l)                   (Eq. 1; e = (|b| - t)^2 or |b - t|^2)
//   u = H_loss^T conj(G),  A mu = u            (A^T = A: the same factors serve)
//   dloss/dC_k += Im(mu_k I_k)/(w C_k^2)       (from d(A^-1) = -A^-1 dA A^-1, Eq. 8-9)
//
// LU with partial pivoting is done without moving rows: at step k the largest |a_rk| among
// rows not yet chosen is the pivot; chosen rows keep U in place and the others keep their
// multipliers in column k. This file holds the FP64 variant (MTS_FP64, rows in shared
// memory) and the dispatch; the mixed-precision variant is in solve_mixed.cu.
// Padding rows r >= N (when N < NM) are identity rows with zero right-hand side.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "solve_common.cuh"

namespace mts {

// ---------------------------------------------------------------------------------------
// FP64 kernel: G groups of NM threads per CTA, rows in dynamic shared memory.
// ---------------------------------------------------------------------------------------
template <int NM>
struct Fp64Smem {
  static constexpr int P = NM + 1;  // row pitch (complex) to spread banks
  static constexpr size_t per_group =
      sizeof(cd) * (size_t)NM * P + sizeof(cd) * NM /* rhs */ + sizeof(cd) * NM /* xs */ +
      sizeof(cd) * NM /* G */ + sizeof(double) * 32 /* red */ + sizeof(int) * 32;
};

template <int NM>
__global__ void __launch_bounds__(NM >= 128 ? NM : 128) solve_fp64_kernel(SolveArgs a, int64_t n_sys) {
  constexpr int CT = NM >= 128 ? NM : 128;
  constexpr int G = CT / NM;
  constexpr int P = Fp64Smem<NM>::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = threadIdx.x / NM, r = threadIdx.x % NM;
  unsigned char* base = smem_raw + grp * Fp64Smem<NM>::per_group;
  cd* A = reinterpret_cast<cd*>(base);
  cd* rhs = A + NM * P;
  cd* xs = rhs + NM;
  cd* Gs = xs + NM;
  double* red = reinterpret_cast<double*>(Gs + NM);
  int* redi = reinterpret_cast<int*>(red + 32);

  const int64_t li = (int64_t)blockIdx.x * G + grp;
  const bool in_range = li < n_sys;
  const int64_t sys = in_range ? launch_sys(a, li) : 0;
  SysInfo si = sys_info(a, sys);
  const bool valid = in_range && si.N <= NM;  // larger systems: solve_large.cu
  if (!valid) si.N = 0;
  const int N = si.N;
  const double w = si.w;
  const bool real_row = r < N;
  double Cr = real_row ? a.C[si.b * a.n_ports + si.k0 + r] : 1.0;
  const double* Ms = a.M64 + a.t.nn_off[si.s];
  // assemble row r (Eq. 2, 11): A_rj = j w M_rj, A_rr += R_r + 1/(j w C_r)
  for (int j = 0; j < NM; ++j) {
    cd v = {0.0, 0.0};
    if (real_row && j < N) v.y = w * Ms[r * N + j];
    A[r * P + j] = v;
  }
  if (real_row) {
    A[r * P + r].x += a.R[si.k0 + r];
    A[r * P + r].y += -1.0 / (w * Cr);
  } else {
    A[r * P + r].x = 1.0;
  }
  const bool bwd = a.rhs_in != nullptr;
  const int64_t ioff = si.b * a.sumFN + a.t.fn_off[si.s] + (int64_t)si.f * N;
  cd v0 = {0.0, 0.0};
  if (real_row && !bwd) {
    const double* Vp = a.V + 2 * (a.t.fn_off[si.s] + (int64_t)si.f * N + r);
    v0 = {Vp[0], Vp[1]};
  }
  rhs[r] = v0;
  __syncthreads();

  // ---- LU with partial pivoting (rows stay in place) ----
  int pivstep = NM;  // step at which this row became the pivot
  for (int k = 0; k < NM; ++k) {
    double key = (pivstep < NM) ? -1.0 : cabs2(A[r * P + k]);
    if (!(key >= -1.0)) key = 0.0;  // NaN: still a candidate, never below a chosen row
    int idx = r;
    if (NM <= 32) {
      argmax_shfl_d(key, idx, NM);
    } else {
      argmax_shfl_d(key, idx, 32);
      if ((r & 31) == 0) {
        red[r >> 5] = key;
        redi[r >> 5] = idx;
      }
      __syncthreads();
      key = red[0];
      idx = redi[0];
      for (int q = 1; q < NM / 32; ++q)
        if (red[q] > key || (red[q] == key && redi[q] < idx)) {
          key = red[q];
          idx = redi[q];
        }
    }
    const int p = idx;
    if (r == p) pivstep = k;
    __syncthreads();
    if (pivstep > k) {
      cd l = cdiv(A[r * P + k], A[p * P + k]);
      A[r * P + k] = l;
      for (int j = k + 1; j < NM; ++j) A[r * P + j] = csub(A[r * P + j], cmul(l, A[p * P + j]));
    }
    __syncthreads();
  }

  // triangular solves on rhs (forward with the multipliers, then back with U)
  auto solve_inplace = [&](cd myrhs) -> cd {
    // forward: L y = P b
    for (int k = 0; k < NM; ++k) {
      if (pivstep == k) xs[k] = myrhs;
      __syncthreads();
      if (pivstep > k) myrhs = csub(myrhs, cmul(A[r * P + k], xs[k]));
      __syncthreads();
    }
    // back: U x = y
    for (int k = NM - 1; k >= 0; --k) {
      if (pivstep == k) xs[k] = cdiv(myrhs, A[r * P + k]);
      __syncthreads();
      if (pivstep < k) myrhs = csub(myrhs, cmul(A[r * P + k], xs[k]));
    }
    __syncthreads();
    return xs[r];
  };

  cd x = {0.0, 0.0};
  if (!bwd) {
    x = solve_inplace(rhs[r]);
  } else if (real_row) {
    const double* Ip = a.I + 2 * (ioff + r);
    x = {Ip[0], Ip[1]};
  }
  if (valid && real_row && !bwd) {
    double* Ip = a.I + 2 * (ioff + r);
    Ip[0] = x.x;
    Ip[1] = x.y;
    if (a.I_out) {
      a.I_out[2 * (ioff + r)] = x.x;
      a.I_out[2 * (ioff + r) + 1] = x.y;
    }
  }
  bool bad = !(isfinite(x.x) && isfinite(x.y)) && real_row;
  __syncthreads();
  xs[r] = x;  // currents visible to the whole group
  __syncthreads();

  // ---- objective and adjoint right-hand side ----
  bool do_adj = bwd || a.target != nullptr;
  cd u = {0.0, 0.0};
  double lsum = 0.0;
  if (!bwd && a.target != nullptr) {
    const int L0 = a.loss_off[si.s], L = a.loss_off[si.s + 1] - L0;
    const double* Hl = a.Hl64 + a.t.ln_off[si.s];
    const int tw = a.loss_mode == 0 ? 1 : 2;
    const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                       (a.t.fl_off[si.s] + (int64_t)si.f * L) * tw;
    const int64_t wo = a.t.fl_off[si.s] + (int64_t)si.f * L;  // weight / offset base
    for (int c0 = 0; c0 < a.max_loss; c0 += NM) {
      int l = c0 + r;
      cd Gl = {0.0, 0.0};
      if (l < L) {
        cd bl = {0.0, 0.0};
        for (int k = 0; k < N; ++k) {
          double h = Hl[(int64_t)l * N + k];
          bl.x += h * xs[k].x;
          bl.y += h * xs[k].y;
        }
        double wl = 1.0;
        if (a.loss_offset) {
          bl.x += a.loss_offset[2 * (wo + l)];
          bl.y += a.loss_offset[2 * (wo + l) + 1];
        }
        if (a.loss_weight) {
          wl = a.loss_weight[wo + l];
          bl.x *= wl;
          bl.y *= wl;
        }
        lsum += point_loss(a.loss_mode, bl, tb + (int64_t)l * tw, &Gl);
        Gl.x *= wl;
        Gl.y *= wl;
      }
      Gs[r] = Gl;
      __syncthreads();
      if (real_row) {
        int lc = max(0, min(NM, L - c0));
        for (int q = 0; q < lc; ++q) {
          double h = Hl[(int64_t)(c0 + q) * N + r];
          u.x += h * Gs[q].x;
          u.y -= h * Gs[q].y;  // conj(G)
        }
      }
      __syncthreads();
    }
  } else if (bwd && real_row) {
    const double* up = a.rhs_in + 2 * (ioff + r);
    u = {up[0], up[1]};
  }
  // group sum of the objective
  if (!bwd && a.target != nullptr) {
    double v = lsum;
    if constexpr (NM <= 32) {
      for (int off = NM >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, NM);
      if (r == 0 && valid) a.loss_part[sys] = v;
    } else {
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      __syncthreads();
      if ((r & 31) == 0) red[r >> 5] = v;
      __syncthreads();
      if (r == 0) {
        double tot = 0.0;
        for (int q = 0; q < NM / 32; ++q) tot += red[q];
        if (valid) a.loss_part[sys] = tot;
      }
    }
  }
  if (do_adj) {
    cd mu = solve_inplace(u);
    if (valid && real_row) {
      double g = (mu.x * x.y + mu.y * x.x) / (w * Cr * Cr);  // Im(mu x)/(w C^2)
      a.grad_part[ioff + r] = g;
      if (!bwd && a.mu_out) {
        a.mu_out[2 * (ioff + r)] = mu.x;
        a.mu_out[2 * (ioff + r) + 1] = mu.y;
      }
    }
  }
  // status
  // non-finite flag of this group's system only (a CTA holds G systems)
  __syncthreads();
  if (r == 0) redi[0] = 0;
  __syncthreads();
  if (bad) redi[0] = 1;
  __syncthreads();
  if (valid && r == 0 && !bwd) a.status[sys] = redi[0] ? 2 : 0;
}

// ---------------------------------------------------------------------------------------
// reduction over frequencies: loss[b][s], dldc[b][port]
// ---------------------------------------------------------------------------------------
__global__ void reduce_kernel(ReduceArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nport_items = a.n_cfg * a.n_ports;
  if (i < nport_items) {
    int64_t b = i / a.n_ports;
    int port = (int)(i - b * a.n_ports);
    int s = find_struct_i32(a.port_off, a.n_struct, port);
    int N = a.port_off[s + 1] - a.port_off[s];
    int k = port - a.port_off[s];
    int F = a.freq_off[s + 1] - a.freq_off[s];
    int L = a.loss_off ? a.loss_off[s + 1] - a.loss_off[s] : 0;
    double acc = 0.0;
    const double* gp = a.grad_part + b * a.sumFN + a.t.fn_off[s] + k;
    for (int f = 0; f < F; ++f) acc += gp[(int64_t)f * N];
    if (a.normalise) acc = (F * L > 0) ? acc / ((double)F * L) : 0.0;
    a.dldc[i] = acc;
  }
  int64_t j = i - nport_items;
  if (j >= 0 && j < a.n_cfg * a.n_struct && a.normalise) {
    int64_t b = j / a.n_struct;
    int s = (int)(j - b * a.n_struct);
    int F = a.freq_off[s + 1] - a.freq_off[s];
    int L = a.loss_off ? a.loss_off[s + 1] - a.loss_off[s] : 0;
    double acc = 0.0;
    const double* lp = a.loss_part + b * a.n_freq + a.freq_off[s];
    for (int f = 0; f < F; ++f) acc += lp[f];
    acc = (F * L > 0) ? acc / ((double)F * L) : 0.0;
    a.lossv[j] = acc;
    if (a.loss_out) a.loss_out[j] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
template <int NM>
static cudaError_t launch_fp64(const SolveArgs& a, int64_t n_sys, cudaStream_t st) {
  constexpr int CT = NM >= 128 ? NM : 128;
  constexpr int G = CT / NM;
  size_t smem = Fp64Smem<NM>::per_group * G;
  cudaError_t e = cudaFuncSetAttribute(solve_fp64_kernel<NM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)((n_sys + G - 1) / G);
  solve_fp64_kernel<NM><<<grid, CT, smem, st>>>(a, n_sys);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const SolveArgs& a, int64_t n_sys, int max_ports, cudaStream_t st);

// One launch per port class present (classes 0..3: the register-resident kernel with
// 8/16/32/64 threads per system; class 4: the blocked large-system kernel). A problem of one
// structure is a single class and launches over all systems without the frequency list.
cudaError_t launch_solve(const SolveArgs& a0, mts_precision prec, const ProblemSums& ps,
                         cudaStream_t st) {
  if (a0.n_cfg * a0.n_freq == 0) return cudaSuccess;
  if (ps.max_ports > kMaxPorts) return cudaErrorNotSupported;
  const bool one = a0.n_struct == 1;
  int64_t off = 0;
  for (int c = 0; c < kNumPortClasses; ++c) {
    const int64_t cnt = ps.cls_count[c];
    if (cnt == 0) continue;
    SolveArgs a = a0;
    a.glist = one ? nullptr : a0.t.cls_freq + off;
    a.gcount = cnt;
    off += cnt;
    const int64_t n_sys = a.n_cfg * cnt;
    cudaError_t e;
    // the register classes run in their own width, or one wider (reg_widen bit c)
    const int cw = (c < 3 && ((a.reg_widen >> c) & 1)) ? c + 1 : c;
    if (c == 4) {
      e = launch_solve_large(a, prec, n_sys, kRegMaxPorts, ps.cls_max_ports[c], a.lu, st);
    } else if (prec == MTS_FP64) {
      e = cw == 0 ? launch_fp64<8>(a, n_sys, st)
        : cw == 1 ? launch_fp64<16>(a, n_sys, st)
        : cw == 2 ? launch_fp64<32>(a, n_sys, st)
                  : launch_fp64<64>(a, n_sys, st);
    } else {
      e = launch_solve_mixed(a, n_sys, cw == c ? ps.cls_max_ports[c] : (8 << cw), st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  int64_t n = a.n_cfg * a.n_ports + a.n_cfg * a.n_struct;
  if (n == 0) return cudaSuccess;
  reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mts
