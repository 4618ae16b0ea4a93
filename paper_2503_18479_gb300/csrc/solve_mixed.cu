// solve_mixed.cu -- (b) port solve, (d) objective and (adj) adjoint for MTS_MIXED and
// MTS_BF16: FP32 complex LU with partial pivoting, iterative refinement with residuals in
// double-float (FP32-pair) arithmetic, one system per group of NM threads (thread r owns
// row r of A = diag(R) + j w M + diag(1/(j w C)); paper Eq. 2, 6, 11).
//
// Register layout: row r lives in NB = NM/8 blocks of 8 complex values, blk[b][j] for
// column 8b + j. Rows are never moved; the pivot of step k is the row with the largest
// |a_rk| among rows not chosen yet, and its step is recorded in `pivstep`.
//
// LU in panels of 8 columns: the 8 steps of a panel are unrolled with static register
// indices; the panel loop is a runtime loop, and after each panel the blocks rotate by one
// (blk[b] <- blk[b+1], the finished panel to the end), so the active panel is always
// blk[0] and the code stays one panel long. NB rotations restore the original order.
//
// Triangular solves in 8x8 blocks (pivot order): the diagonal blocks of L and U are
// inverted once (W = L_bb^-1, V = U_bb^-1, all blocks in parallel, 8 group barriers), and
// the off-diagonal factor rows are premultiplied in place (l~ = l W, u~ = u V). A forward
// block step is then y_b = W_b c_b for the block's pivot rows and c_r -= l~_r c_b for later
// rows, both from the raw c_b values; the backward step likewise with V and u~. A solve is
// 2 NB + 2 group barriers instead of 2 NM + 1.
//
// Objective and adjoint as in solve.cu: b_l = H_loss I, loss = sum e(b_l, t_l),
// u = H_loss^T conj(G), A mu = u (A^T = A), dloss/dC_k = Im(mu_k I_k)/(w C_k^2) (Eq. 8-9).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "solve_common.cuh"

namespace mts {

template <int NM>
struct SmemV2 {
  static constexpr int NB = NM / 8;
  static constexpr int NW = NM > 32 ? NM / 32 : 1;  // candidate buffers (warps per group)
  float2 prow[2][NW][NM];  // pivot-row candidates, [step parity][warp][rotated column]
  float ckey[2][NW];
  int cidx[2][NW];
  float2 Wb[NB][8][8];     // inverses of the diagonal blocks of L (unit lower)
  float2 Vb[NB][8][8];     // and of U (upper)
  float2 bp[2][8];
  float2 bq[2][8];
  float2 xs[NM];
  float4 xhl[NM];
  double2 x64[NM];
  float2 Gs[NM];
  double red[NW];
  float redf[NW];
};

template <int NM>
__device__ inline void gsync() {
  if constexpr (NM <= 32) __syncwarp();
  else __syncthreads();
}

template <int NM>
__device__ inline float gmax(float v, SmemV2<NM>& sm, int r) {
  if constexpr (NM <= 32) {
    for (int off = NM >> 1; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off, NM));
    return v;
  } else {
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((r & 31) == 0) sm.redf[r >> 5] = v;
    __syncthreads();
    float m = sm.redf[0];
#pragma unroll
    for (int q = 1; q < SmemV2<NM>::NW; ++q) m = fmaxf(m, sm.redf[q]);
    return m;
  }
}

template <int NM>
__device__ inline double gsum(double v, SmemV2<NM>& sm, int r) {
  if constexpr (NM <= 32) {
    for (int off = NM >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, NM);
    return v;
  } else {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((r & 31) == 0) sm.red[r >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < SmemV2<NM>::NW; ++q) s += sm.red[q];
    return s;
  }
}

// c -= a * b (complex, FP32)
__device__ inline void cms(float2& c, float2 a, float2 b) {
  c.x = fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x));
  c.y = fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y));
}
// c += a * b
__device__ inline void cma(float2& c, float2 a, float2 b) {
  c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
  c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
}
__device__ inline float2 crecip(float2 a) {
  float inv = 1.0f / (a.x * a.x + a.y * a.y);
  return make_float2(a.x * inv, -a.y * inv);
}
__device__ inline float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int NM>
__global__ void __launch_bounds__(NM >= 64 ? NM : 128) solve_mixed_v2(SolveArgs a, int64_t n_sys) {
  constexpr int NB = NM / 8;
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  __shared__ SmemV2<NM> smem_all[G];
  const int grp = threadIdx.x / NM, r = threadIdx.x % NM;
  SmemV2<NM>& sm = smem_all[grp];

  const int64_t sys = (int64_t)blockIdx.x * G + grp;
  const bool valid = sys < n_sys;
  SysInfo si = sys_info(a, valid ? sys : 0);
  const int N = si.N;
  const double w = si.w;
  const bool real_row = r < N;
  const bool bwd = a.rhs_in != nullptr;
  const double Cr = real_row ? a.C[si.b * a.n_ports + si.k0 + r] : 1.0;
  cd Dr = {0.0, 0.0};
  if (real_row) Dr = {a.R[si.k0 + r], -1.0 / (w * Cr)};
  const int64_t mo = a.t.nn_off[si.s];
  const float* Mhi = a.M32hi + mo;
  const float* Mlo = a.M32lo + mo;
  const double* M64 = a.M64 + mo;

  // ---- row r of A (FP32), identity rows for padding ----
  float2 blk[NB][8];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * b + j;
      float m = (real_row && c < N) ? (float)(w * M64[(int64_t)c * N + r]) : 0.0f;
      blk[b][j] = make_float2(0.0f, m);
      if (c == r) {
        if (real_row)
          blk[b][j] = make_float2((float)Dr.x, (float)(w * M64[(int64_t)r * N + r] + Dr.y));
        else
          blk[b][j] = make_float2(1.0f, 0.0f);
      }
    }

  // ---- LU with partial pivoting, panels of 8 columns ----
  int pivstep = NM;
#pragma unroll 1
  for (int kb = 0; kb < NB; ++kb) {
    const int nact = NB - kb;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = 8 * kb + kk;
      const int par = kk & 1;
      float key = (pivstep < NM) ? -1.0f : blk[0][kk].x * blk[0][kk].x + blk[0][kk].y * blk[0][kk].y;
      int idx = r;
      int p, src;
      if constexpr (NM <= 32) {
        argmax_shfl(key, idx, NM);
        p = idx;
        src = 0;
        if (r == p) {
#pragma unroll
          for (int j = kk; j < 8; ++j) sm.prow[par][0][j] = blk[0][j];
#pragma unroll
          for (int b = 1; b < NB; ++b)
            if (b < nact)
#pragma unroll
              for (int j = 0; j < 8; ++j) sm.prow[par][0][8 * b + j] = blk[b][j];
        }
        __syncwarp();
      } else {
        argmax_shfl(key, idx, 32);
        const int wv = r >> 5;
        if (r == idx) {  // this warp's candidate publishes its row speculatively
          sm.ckey[par][wv] = key;
          sm.cidx[par][wv] = idx;
#pragma unroll
          for (int j = kk; j < 8; ++j) sm.prow[par][wv][j] = blk[0][j];
#pragma unroll
          for (int b = 1; b < NB; ++b)
            if (b < nact)
#pragma unroll
              for (int j = 0; j < 8; ++j) sm.prow[par][wv][8 * b + j] = blk[b][j];
        }
        __syncthreads();
        src = 0;
        float kbest = sm.ckey[par][0];
        int ibest = sm.cidx[par][0];
#pragma unroll
        for (int q = 1; q < SmemV2<NM>::NW; ++q) {
          float kq = sm.ckey[par][q];
          int iq = sm.cidx[par][q];
          if (kq > kbest || (kq == kbest && iq < ibest)) {
            kbest = kq;
            ibest = iq;
            src = q;
          }
        }
        p = ibest;
      }
      if (r == p) pivstep = k;
      if (pivstep > k) {
        const float2* pr = sm.prow[par][src];
        float2 l = cmulf(blk[0][kk], crecip(pr[kk]));
        blk[0][kk] = l;
#pragma unroll
        for (int j = kk + 1; j < 8; ++j) cms(blk[0][j], l, pr[j]);
#pragma unroll
        for (int b = 1; b < NB; ++b)
          if (b < nact)
#pragma unroll
            for (int j = 0; j < 8; ++j) cms(blk[b][j], l, pr[8 * b + j]);
      }
    }
    // rotate: the finished panel goes to the end
    if constexpr (NB > 1) {
      float2 t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t[j] = blk[0][j];
#pragma unroll
      for (int b = 0; b < NB - 1; ++b)
#pragma unroll
        for (int j = 0; j < 8; ++j) blk[b][j] = blk[b + 1][j];
#pragma unroll
      for (int j = 0; j < 8; ++j) blk[NB - 1][j] = t[j];
    }
  }

  // ---- inverses of the 8x8 diagonal blocks (pivot order), all blocks at once ----
  const int Mb = pivstep >> 3, ii = pivstep & 7;
  float2 dg[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) dg[j] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b == Mb)
#pragma unroll
      for (int j = 0; j < 8; ++j) dg[j] = blk[b][j];
  float2 wrow[8], vrow[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    wrow[j] = make_float2(0.0f, 0.0f);
    vrow[j] = make_float2(0.0f, 0.0f);
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (ii == s) {  // W_s = e_s - sum_{m<s} L[s][m] W_m
#pragma unroll
      for (int j = 0; j < s; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = j; m < s; ++m) cma(acc, dg[m], sm.Wb[Mb][m][j]);
        wrow[j] = make_float2(-acc.x, -acc.y);
      }
      wrow[s] = make_float2(1.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < 8; ++j) sm.Wb[Mb][s][j] = wrow[j];
    }
    constexpr int dummy = 0;
    (void)dummy;
    if (ii == 7 - s) {  // V_i = (e_i - sum_{m>i} U[i][m] V_m) / U[i][i], i = 7 - s
      const int i = 7 - s;
      float2 dinv = crecip(dg[i]);
      vrow[i] = dinv;
#pragma unroll
      for (int j = i + 1; j < 8; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = i + 1; m <= j; ++m) cma(acc, dg[m], sm.Vb[Mb][m][j]);
        float2 v = cmulf(acc, dinv);
        vrow[j] = make_float2(-v.x, -v.y);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) sm.Vb[Mb][i][j] = vrow[j];
    }
    gsync<NM>();
  }
  // diagonal block <- W (strictly lower) and V (upper); off-diagonal blocks premultiplied
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (b == Mb) {
#pragma unroll
      for (int j = 0; j < 8; ++j) blk[b][j] = (j < ii) ? wrow[j] : vrow[j];
    } else if (b < Mb) {  // multipliers: l~ = l W_b, W_b[m][j] = 0 for j > m
      float2 nv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float2 acc = blk[b][j];  // W_b[j][j] = 1
#pragma unroll
        for (int m = j + 1; m < 8; ++m) cma(acc, blk[b][m], sm.Wb[b][m][j]);
        nv[j] = acc;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) blk[b][j] = nv[j];
    } else {  // U entries: u~ = u V_b, V_b[m][j] = 0 for j < m
      float2 nv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m <= j; ++m) cma(acc, blk[b][m], sm.Vb[b][m][j]);
        nv[j] = acc;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) blk[b][j] = nv[j];
    }
  }

  // ---- block triangular solve: returns the unknown x_r for right-hand side entry rhs ----
  auto lu_solve = [&](float2 rhs) -> float2 {
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) {
      if (Mb == kb) sm.bp[kb & 1][ii] = rhs;
      gsync<NM>();
      if (Mb == kb) {
        float2 y = rhs;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < ii) cma(y, blk[kb][j], sm.bp[kb & 1][j]);
        rhs = y;
      } else if (Mb > kb) {
#pragma unroll
        for (int j = 0; j < 8; ++j) cms(rhs, blk[kb][j], sm.bp[kb & 1][j]);
      }
    }
#pragma unroll
    for (int kb = NB - 1; kb >= 0; --kb) {
      if (Mb == kb) sm.bq[kb & 1][ii] = rhs;
      gsync<NM>();
      if (Mb == kb) {
        float2 x = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j >= ii) cma(x, blk[kb][j], sm.bq[kb & 1][j]);
        rhs = x;
      } else if (Mb < kb) {
#pragma unroll
        for (int j = 0; j < 8; ++j) cms(rhs, blk[kb][j], sm.bq[kb & 1][j]);
      }
    }
    sm.xs[pivstep] = rhs;
    gsync<NM>();
    float2 out = sm.xs[r];
    gsync<NM>();
    return out;
  };

  // publish the FP64 iterate of this thread's unknown and its double-float split
  auto publish = [&](cd x) {
    sm.x64[r] = make_double2(x.x, x.y);
    float rh = (float)x.x, ih = (float)x.y;
    sm.xhl[r] = make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
    gsync<NM>();
  };

  // residual of row r: rhs_r - sum_j A_rj x_j, sum_j M_rj x_j in double-float
  auto residual = [&](cd rhs) -> cd {
    if (!real_row) {
      double2 xr = sm.x64[r];
      return {rhs.x - xr.x, rhs.y - xr.y};
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
    double ax = Dr.x * xr.x - Dr.y * xr.y;
    double ay = Dr.x * xr.y + Dr.y * xr.x;
    return {rhs.x - ax + w * Si, rhs.y - ay - w * Sr};
  };

  const double tol = a.tol;
  const int max_it = a.max_refine;
  // Refined solve. The error of x_k is estimated as |d_k|^2 / |d_{k-1}| (geometric
  // contraction; d_0 = x_0); converged when that is <= tol |x|. Stops on convergence or when
  // the correction no longer halves (residual precision reached).
  auto solve_refined = [&](cd rhs64, bool& conv) -> cd {
    float2 x32 = lu_solve(make_float2((float)rhs64.x, (float)rhs64.y));
    cd x = {(double)x32.x, (double)x32.y};
    float dprev = gmax<NM>(fabsf(x32.x) + fabsf(x32.y), sm, r);
    conv = max_it == 0;
    for (int it = 0; it < max_it; ++it) {
      publish(x);
      cd res = residual(rhs64);
      float2 d = lu_solve(make_float2((float)res.x, (float)res.y));
      x.x += (double)d.x;
      x.y += (double)d.y;
      float dm = gmax<NM>(fabsf(d.x) + fabsf(d.y), sm, r);
      float xm = gmax<NM>((float)(fabs(x.x) + fabs(x.y)), sm, r);
      float est = dm * fminf(1.0f, dm / fmaxf(dprev, 1e-30f));
      conv = est <= (float)tol * xm;
      bool stop = conv || !(dm <= 0.5f * dprev);
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
    if (valid && a.Bop != nullptr) {
      // tensor-core operand pieces of I: rows 2 (b F_s + f) + {0: re, 1: im}; thread r owns
      // column r, columns N .. K_pad-1 are zero
      const int F = a.freq_off[si.s + 1] - a.freq_off[si.s];
      const int nkc = (N + kChunkK - 1) / kChunkK;
      const int64_t ntile = (2 * a.n_cfg * F + kTileN - 1) / kTileN;
      char* base = reinterpret_cast<char*>(a.Bop + a.bop_off[si.s]);
      const size_t tile_bytes = (size_t)kTileN * kChunkK * 2;
      for (int kg = r; kg < nkc * kChunkK; kg += NM) {
        const bool own = (kg == r) && real_row;
        const int kc = kg / kChunkK, kk = kg % kChunkK;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int64_t n = 2 * (si.b * F + si.f) + c;
          const int64_t tile = n / kTileN;
          const uint32_t rr = (uint32_t)(n % kTileN);
          double remd = own ? (c == 0 ? x.x : x.y) : 0.0;
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
      const int L = a.loss_off[si.s + 1] - a.loss_off[si.s];
      const float* Hl = a.Hl32 + a.t.ln_off[si.s];
      const int tw = a.loss_mode == 0 ? 1 : 2;
      const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                         (a.t.fl_off[si.s] + (int64_t)si.f * L) * tw;
      double lsum = 0.0;
      for (int c0 = 0; c0 < a.max_loss; c0 += NM) {
        const int l = c0 + r;
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
        gsync<NM>();
        if (real_row) {
          const int lc = max(0, min(NM, L - c0));
          for (int q = 0; q < lc; ++q) {
            double h = (double)Hl[(int64_t)(c0 + q) * N + r];
            float2 g = sm.Gs[q];
            u.x += h * (double)g.x;
            u.y -= h * (double)g.y;
          }
        }
        gsync<NM>();
      }
      double tot = gsum<NM>(lsum, sm, r);
      if (valid && r == 0) a.loss_part[sys] = tot;
    } else if (real_row) {
      const double* up = a.rhs_in + 2 * (ioff + r);
      u = {up[0], up[1]};
    }
    cd mu = solve_refined(u, conv_m);
    if (valid && real_row) a.grad_part[ioff + r] = (mu.x * x.y + mu.y * x.x) / (w * Cr * Cr);
    bad = bad || (real_row && !(isfinite(mu.x) && isfinite(mu.y)));
  }
  float fb = gmax<NM>(bad ? 2.0f : ((conv_i && conv_m) ? 0.0f : 1.0f), sm, r);
  if (valid && r == 0 && !bwd) a.status[sys] = (int)fb;
}

template <int NM>
static cudaError_t launch_v2(const SolveArgs& a, int64_t n_sys, cudaStream_t st) {
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  unsigned grid = (unsigned)((n_sys + G - 1) / G);
  solve_mixed_v2<NM><<<grid, CT, 0, st>>>(a, n_sys);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const SolveArgs& a, int64_t n_sys, int max_ports, cudaStream_t st) {
  if (max_ports <= 8) return launch_v2<8>(a, n_sys, st);
  if (max_ports <= 16) return launch_v2<16>(a, n_sys, st);
  if (max_ports <= 32) return launch_v2<32>(a, n_sys, st);
  if (max_ports <= 64) return launch_v2<64>(a, n_sys, st);
  return cudaErrorNotSupported;
}

}  // namespace mts
