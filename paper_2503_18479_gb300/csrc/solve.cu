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
// multipliers in column k. Two variants:
//   solve_fp64_kernel   FP64 everywhere, rows in shared memory (MTS_FP64)
//   solve_mixed_kernel  FP32 complex rows in registers (step loop fully unrolled), then
//                       iterative refinement with residuals V - A x evaluated in
//                       double-float arithmetic on the FP32 pipe (M = hi + lo, x = hi + lo,
//                       error-free products and sums); the FP32 factors give the
//                       corrections (MTS_MIXED, MTS_BF16)
// Padding rows r >= N (when N < NM) are identity rows with zero right-hand side.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mts {

// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------
struct cd {
  double x, y;
};
__device__ inline cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ inline cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ inline cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ inline cd cdiv(cd a, cd b) {
  double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ inline double cabs2(cd a) { return a.x * a.x + a.y * a.y; }

// Objective term of one loss point and its cotangent G = de/dRe b + j de/dIm b.
__device__ inline double point_loss(int mode, cd b, const double* t, cd* G) {
  if (mode == 0) {
    double a = sqrt(b.x * b.x + b.y * b.y);
    double r = a - t[0];
    if (a > 0.0) {
      G->x = 2.0 * r * b.x / a;
      G->y = 2.0 * r * b.y / a;
    } else {
      G->x = 0.0;
      G->y = 0.0;
    }
    return r * r;
  }
  cd e = {b.x - t[0], b.y - t[1]};
  G->x = 2.0 * e.x;
  G->y = 2.0 * e.y;
  return e.x * e.x + e.y * e.y;
}

// arg-max of (key, idx) over aligned groups of `width` lanes (width a power of 2 <= 32);
// ties go to the smaller index.
__device__ inline void argmax_shfl(float& key, int& idx, int width) {
  for (int off = width >> 1; off > 0; off >>= 1) {
    float k2 = __shfl_xor_sync(0xffffffffu, key, off, width);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, off, width);
    if (k2 > key || (k2 == key && i2 < idx)) {
      key = k2;
      idx = i2;
    }
  }
}
__device__ inline void argmax_shfl_d(double& key, int& idx, int width) {
  for (int off = width >> 1; off > 0; off >>= 1) {
    double k2 = __shfl_xor_sync(0xffffffffu, key, off, width);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, off, width);
    if (k2 > key || (k2 == key && i2 < idx)) {
      key = k2;
      idx = i2;
    }
  }
}

// Locate system `sys` (= b * n_freq + g).
struct SysInfo {
  int64_t b;
  int g, s, f, N, k0;
  double w;
};
__device__ inline SysInfo sys_info(const SolveArgs& a, int64_t sys) {
  SysInfo si;
  si.b = sys / a.n_freq;
  si.g = (int)(sys - si.b * a.n_freq);
  si.s = a.t.freq_struct[si.g];
  si.f = si.g - a.freq_off[si.s];
  si.k0 = a.port_off[si.s];
  si.N = a.port_off[si.s + 1] - si.k0;
  si.w = a.omega[si.g];
  return si;
}

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

  int64_t sys = (int64_t)blockIdx.x * G + grp;
  const bool valid = sys < n_sys;
  SysInfo si = sys_info(a, valid ? sys : 0);
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
        lsum += point_loss(a.loss_mode, bl, tb + (int64_t)l * tw, &Gl);
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
    }
  }
  // status
  int nb = __syncthreads_or(bad ? 1 : 0);
  if (valid && r == 0 && !bwd) a.status[sys] = nb ? 2 : 0;
}

// ---------------------------------------------------------------------------------------
// Mixed kernel: FP32 factors in registers, double-float residuals.
// ---------------------------------------------------------------------------------------
struct df {
  float hi, lo;
};
// error-free product and sum on the FP32 pipe
__device__ inline void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float t = sh + p;
  float z = t - sh;
  float err = (sh - (t - z)) + (p - z);
  sh = t;
  sl += err + e;
}

template <int NM>
struct MixedSmem {
  float2 prow[2][NM];   // pivot row (double-buffered by step parity)
  float2 ys[NM];        // forward-substitution values
  float2 xs[NM];        // back-substitution values
  float4 xhl[NM];       // x split for residuals: (re_hi, re_lo, im_hi, im_lo)
  double2 x64[NM];      // FP64 iterate
  float2 Gs[NM];        // loss cotangents (FP32)
  float cand_key[2][2];
  int cand_idx[2][2];
  double red[4];
};

template <int NM>
__device__ inline void group_sync() {
  if constexpr (NM <= 32) __syncwarp();
  else __syncthreads();
}

template <int NM>
__device__ inline float group_max(float v, MixedSmem<NM>& sm, int r) {
  if constexpr (NM <= 32) {
    for (int off = NM >> 1; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off, NM));
    return v;
  } else {
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((r & 31) == 0) sm.red[r >> 5] = v;
    __syncthreads();
    float m = (float)sm.red[0];
    for (int q = 1; q < NM / 32; ++q) m = fmaxf(m, (float)sm.red[q]);
    return m;
  }
}

template <int NM>
__device__ inline double group_sum(double v, MixedSmem<NM>& sm, int r) {
  if constexpr (NM <= 32) {
    for (int off = NM >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, NM);
    return v;
  } else {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((r & 31) == 0) sm.red[r >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < NM / 32; ++q) s += sm.red[q];
    return s;
  }
}

template <int NM>
__global__ void __launch_bounds__(NM >= 64 ? NM : 128) solve_mixed_kernel(SolveArgs a, int64_t n_sys) {
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  __shared__ MixedSmem<NM> smem_all[G];
  const int grp = threadIdx.x / NM, r = threadIdx.x % NM;
  MixedSmem<NM>& sm = smem_all[grp];

  int64_t sys = (int64_t)blockIdx.x * G + grp;
  const bool valid = sys < n_sys;
  SysInfo si = sys_info(a, valid ? sys : 0);
  const int N = si.N;
  const double w = si.w;
  const bool real_row = r < N;
  const bool bwd = a.rhs_in != nullptr;
  const double Cr = real_row ? a.C[si.b * a.n_ports + si.k0 + r] : 1.0;
  // diagonal load D_r = R_r + 1/(j w C_r) (FP64), zero for padding rows
  cd Dr = {0.0, 0.0};
  if (real_row) Dr = {a.R[si.k0 + r], -1.0 / (w * Cr)};
  const int64_t mo = a.t.nn_off[si.s];
  const float* Mhi = a.M32hi + mo;
  const float* Mlo = a.M32lo + mo;
  const double* M64 = a.M64 + mo;

  // ---- row r of A in FP32 registers ----
  float2 row[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    float m = (real_row && j < N) ? (float)(w * M64[(int64_t)j * N + r]) : 0.0f;  // M symmetric
    row[j] = make_float2(0.0f, m);
    if (j == r) {
      if (real_row) {
        double dre = Dr.x, dim = w * M64[(int64_t)r * N + r] + Dr.y;
        row[j] = make_float2((float)dre, (float)dim);
      } else {
        row[j] = make_float2(1.0f, 0.0f);
      }
    }
  }

  // ---- LU with partial pivoting, rows in place ----
  int pivstep = NM;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    float key = (pivstep < NM) ? -1.0f : row[k].x * row[k].x + row[k].y * row[k].y;
    int idx = r;
    int p;
    if constexpr (NM <= 32) {
      argmax_shfl(key, idx, NM);
      p = idx;
    } else {
      argmax_shfl(key, idx, 32);
      if ((r & 31) == 0) {
        sm.cand_key[k & 1][r >> 5] = key;
        sm.cand_idx[k & 1][r >> 5] = idx;
      }
      __syncthreads();
      float k0 = sm.cand_key[k & 1][0], k1 = sm.cand_key[k & 1][1];
      int i0 = sm.cand_idx[k & 1][0], i1 = sm.cand_idx[k & 1][1];
      p = (k1 > k0 || (k1 == k0 && i1 < i0)) ? i1 : i0;
    }
    if (r == p) {
      pivstep = k;
#pragma unroll
      for (int j = k; j < NM; ++j) sm.prow[k & 1][j] = row[j];
    }
    group_sync<NM>();
    if (pivstep > k) {
      float2 pv = sm.prow[k & 1][k];
      float inv = 1.0f / (pv.x * pv.x + pv.y * pv.y);
      float2 l;
      l.x = (row[k].x * pv.x + row[k].y * pv.y) * inv;
      l.y = (row[k].y * pv.x - row[k].x * pv.y) * inv;
      row[k] = l;
#pragma unroll
      for (int j = k + 1; j < NM; ++j) {
        float2 u = sm.prow[k & 1][j];
        row[j].x = fmaf(-l.x, u.x, fmaf(l.y, u.y, row[j].x));
        row[j].y = fmaf(-l.x, u.y, fmaf(-l.y, u.x, row[j].y));
      }
    }
  }

  // FP32 solve with the in-register factors: returns x_r (the r-th unknown)
  auto lu_solve = [&](float2 b) -> float2 {
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      if (pivstep == k) sm.ys[k] = b;
      group_sync<NM>();
      if (pivstep > k) {
        float2 y = sm.ys[k];
        b.x = fmaf(-row[k].x, y.x, fmaf(row[k].y, y.y, b.x));
        b.y = fmaf(-row[k].x, y.y, fmaf(-row[k].y, y.x, b.y));
      }
    }
#pragma unroll
    for (int k = NM - 1; k >= 0; --k) {
      if (pivstep == k) {
        float2 d = row[k];
        float inv = 1.0f / (d.x * d.x + d.y * d.y);
        sm.xs[k] = make_float2((b.x * d.x + b.y * d.y) * inv, (b.y * d.x - b.x * d.y) * inv);
      }
      group_sync<NM>();
      if (pivstep < k) {
        float2 x = sm.xs[k];
        b.x = fmaf(-row[k].x, x.x, fmaf(row[k].y, x.y, b.x));
        b.y = fmaf(-row[k].x, x.y, fmaf(-row[k].y, x.x, b.y));
      }
    }
    float2 out = sm.xs[r];
    group_sync<NM>();
    return out;
  };

  // publish the FP64 iterate of this thread's unknown (and its double-float split)
  auto publish = [&](cd x) {
    sm.x64[r] = make_double2(x.x, x.y);
    float rh = (float)x.x, ih = (float)x.y;
    sm.xhl[r] = make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
    group_sync<NM>();
  };

  // residual of row r: rhs_r - sum_j A_rj x_j, with sum_j M_rj x_j in double-float
  auto residual = [&](cd rhs) -> cd {
    if (!real_row) {
      double2 xr = sm.x64[r];
      return {rhs.x - xr.x, rhs.y - xr.y};  // identity row
    }
    float srh = 0.f, srl = 0.f, sih = 0.f, sil = 0.f;
    for (int j = 0; j < N; ++j) {
      float mh = Mhi[(int64_t)j * N + r], ml = Mlo[(int64_t)j * N + r];
      float4 xj = sm.xhl[j];
      df_mac(srh, srl, mh, ml, xj.x, xj.y);
      df_mac(sih, sil, mh, ml, xj.z, xj.w);
    }
    double Sr = (double)srh + (double)srl, Si = (double)sih + (double)sil;
    double2 xr = sm.x64[r];
    // A_rr part that is not j w M: D_r x_r
    double ax = Dr.x * xr.x - Dr.y * xr.y;
    double ay = Dr.x * xr.y + Dr.y * xr.x;
    // j w S = (-w Si, w Sr)
    return {rhs.x - ax + w * Si, rhs.y - ay - w * Sr};
  };

  const double tol = a.tol;
  const int max_it = a.max_refine;
  // Solve A x = rhs64 with refinement; returns x_r. Stops when the correction is below
  // tol * |x| (converged) or stops contracting (the residual's precision is reached:
  // attainable relative accuracy ~ cond(A) * 2^-45 with double-float residuals).
  auto solve_refined = [&](cd rhs64, bool& conv) -> cd {
    float2 x32 = lu_solve(make_float2((float)rhs64.x, (float)rhs64.y));
    cd x = {(double)x32.x, (double)x32.y};
    conv = max_it == 0;
    float dprev = INFINITY;
    for (int it = 0; it < max_it; ++it) {
      publish(x);
      cd res = residual(rhs64);
      float2 d = lu_solve(make_float2((float)res.x, (float)res.y));
      x.x += (double)d.x;
      x.y += (double)d.y;
      float dm = group_max<NM>(fabsf(d.x) + fabsf(d.y), sm, r);
      float xm = group_max<NM>((float)(fabs(x.x) + fabs(x.y)), sm, r);
      conv = dm <= (float)tol * xm;
      bool stop = conv || !(dm <= 0.5f * dprev);  // converged, stalled or non-finite
      dprev = dm;
      if constexpr (NM <= 32) {
        if (__all_sync(0xffffffffu, stop)) break;
      } else {
        if (stop) break;
      }
    }
    return x;
  };

  const int64_t ioff = si.b * a.sumFN + a.t.fn_off[si.s] + (int64_t)si.f * N;
  bool conv_i = true, conv_m = true;
  cd x = {0.0, 0.0};
  if (!bwd) {
    cd v0 = {0.0, 0.0};
    if (real_row) {
      const double* Vp = a.V + 2 * (a.t.fn_off[si.s] + (int64_t)si.f * N + r);
      v0 = {Vp[0], Vp[1]};
    }
    x = solve_refined(v0, conv_i);
    if (valid && real_row) {
      double* Ip = a.I + 2 * (ioff + r);
      Ip[0] = x.x;
      Ip[1] = x.y;
      if (a.I_out) {
        a.I_out[2 * (ioff + r)] = x.x;
        a.I_out[2 * (ioff + r) + 1] = x.y;
      }
    }
    // tensor-core operand pieces of I: rows 2 (b F_s + f) + {0: re, 1: im}, column k
    if (valid && a.Bop != nullptr) {
      const int F = a.freq_off[si.s + 1] - a.freq_off[si.s];
      const int nkc = (N + kChunkK - 1) / kChunkK;
      const int64_t ntile = (2 * a.n_cfg * F + kTileN - 1) / kTileN;
      char* base = reinterpret_cast<char*>(a.Bop + a.bop_off[si.s]);
      const size_t tile_bytes = (size_t)kTileN * kChunkK * 2;
      // thread r owns column r; columns N .. K_pad-1 of the operand are zero
      for (int kg = r; kg < nkc * kChunkK; kg += NM) {
        const bool own = (kg == r) && real_row;
        const double vx = own ? x.x : 0.0, vy = own ? x.y : 0.0;
        const int kc = kg / kChunkK, kk = kg % kChunkK;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          int64_t n = 2 * (si.b * F + si.f) + c;
          int64_t tile = n / kTileN;
          uint32_t rr = (uint32_t)(n % kTileN);
          double remd = c == 0 ? vx : vy;
          for (int q = 0; q < a.npieces; ++q) {
            __nv_bfloat16 h = __float2bfloat16_rn((float)remd);
            remd -= (double)__bfloat162float(h);
            size_t off = ((size_t)(q * ntile + tile) * nkc + kc) * tile_bytes + swz128(rr, kk);
            *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
          }
        }
      }
    }
  } else if (real_row) {
    const double* Ip = a.I + 2 * (ioff + r);
    x = {Ip[0], Ip[1]};
  }
  bool bad = real_row && !(isfinite(x.x) && isfinite(x.y));

  const bool has_obj = !bwd && a.target != nullptr;
  if (has_obj || bwd) {
    cd u = {0.0, 0.0};
    if (has_obj) {
      publish(x);
      const int L0 = a.loss_off[si.s], L = a.loss_off[si.s + 1] - L0;
      const float* Hl = a.Hl32 + a.t.ln_off[si.s];
      const int tw = a.loss_mode == 0 ? 1 : 2;
      const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                         (a.t.fl_off[si.s] + (int64_t)si.f * L) * tw;
      double lsum = 0.0;
      for (int c0 = 0; c0 < a.max_loss; c0 += NM) {
        int l = c0 + r;
        cd Gl = {0.0, 0.0};
        if (l < L) {
          double bx = 0.0, by = 0.0;
          for (int k = 0; k < N; ++k) {
            double h = (double)Hl[(int64_t)l * N + k];
            double2 xk = sm.x64[k];
            bx += h * xk.x;
            by += h * xk.y;
          }
          lsum += point_loss(a.loss_mode, cd{bx, by}, tb + (int64_t)l * tw, &Gl);
        }
        sm.Gs[r] = make_float2((float)Gl.x, (float)Gl.y);
        group_sync<NM>();
        if (real_row) {
          int lc = max(0, min(NM, L - c0));
          for (int q = 0; q < lc; ++q) {
            double h = (double)Hl[(int64_t)(c0 + q) * N + r];
            float2 g = sm.Gs[q];
            u.x += h * (double)g.x;
            u.y -= h * (double)g.y;
          }
        }
        group_sync<NM>();
      }
      double tot = group_sum<NM>(lsum, sm, r);
      if (valid && r == 0) a.loss_part[sys] = tot;
    } else if (real_row) {
      const double* up = a.rhs_in + 2 * (ioff + r);
      u = {up[0], up[1]};
    }
    cd mu = solve_refined(u, conv_m);
    if (valid && real_row) {
      a.grad_part[ioff + r] = (mu.x * x.y + mu.y * x.x) / (w * Cr * Cr);
    }
    bad = bad || (real_row && !(isfinite(mu.x) && isfinite(mu.y)));
  }
  // group status: 2 non-finite, 1 refinement did not converge
  float fb = group_max<NM>(bad ? 2.0f : ((conv_i && conv_m) ? 0.0f : 1.0f), sm, r);
  if (valid && r == 0 && !bwd) a.status[sys] = (int)fb;
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

template <int NM>
static cudaError_t launch_mixed(const SolveArgs& a, int64_t n_sys, cudaStream_t st) {
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  unsigned grid = (unsigned)((n_sys + G - 1) / G);
  solve_mixed_kernel<NM><<<grid, CT, 0, st>>>(a, n_sys);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve(const SolveArgs& a, mts_precision prec, int max_ports, cudaStream_t st) {
  int64_t n_sys = a.n_cfg * a.n_freq;
  if (n_sys == 0) return cudaSuccess;
  if (prec == MTS_FP64) {
    if (max_ports <= 8) return launch_fp64<8>(a, n_sys, st);
    if (max_ports <= 16) return launch_fp64<16>(a, n_sys, st);
    if (max_ports <= 32) return launch_fp64<32>(a, n_sys, st);
    if (max_ports <= 64) return launch_fp64<64>(a, n_sys, st);
    return cudaErrorNotSupported;
  }
  if (max_ports <= 8) return launch_mixed<8>(a, n_sys, st);
  if (max_ports <= 16) return launch_mixed<16>(a, n_sys, st);
  if (max_ports <= 32) return launch_mixed<32>(a, n_sys, st);
  if (max_ports <= 64) return launch_mixed<64>(a, n_sys, st);
  return cudaErrorNotSupported;
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  int64_t n = a.n_cfg * a.n_ports + a.n_cfg * a.n_struct;
  if (n == 0) return cudaSuccess;
  reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace mts
