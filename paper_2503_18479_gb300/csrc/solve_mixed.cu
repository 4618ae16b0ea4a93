// solve_mixed.cu -- (b) port solve, (d) objective and (adj) adjoint for MTS_MIXED and
// MTS_BF16: FP32 complex LU with partial pivoting, iterative refinement with residuals in
// double-float (FP32-pair) arithmetic, one system per group of NM threads (thread r owns
// row r of A = diag(R) + j w M + diag(1/(j w C)); paper Eq. 2, 6, 11).
//
// Register layout: row r lives in NB = NM/8 blocks of 8 columns; each block keeps the real
// parts of its columns in 4 packed 64-bit pairs (columns 2m, 2m+1) and the imaginary parts
// in another 4, so that the row update runs on the packed FP32x2 pipe over adjacent
// columns (re' = re - l.x ux + l.y uy, im' = im - l.x uy - l.y ux: four fma.rn.f32x2 per
// column pair) and the pivot row is published with 128-bit stores. Rows are never moved;
// the pivot of step k is the row with the largest |a_rk| among rows not chosen yet (one
// redux.sync.max per warp on the magnitude with the row index in the low bits), and its
// step is recorded in `pivstep`.
//
// LU in panels of 8 columns: the 8 steps of a panel are unrolled with static register
// indices; the panel loop is a runtime loop, and after each panel the blocks rotate by one
// (block b <- block b+1, the finished panel to the end), so the active panel is always
// block 0 and the code stays one panel long. NB rotations restore the original order.
//
// Triangular solves in 8x8 blocks (pivot order): the diagonal blocks of L and U are
// inverted once (W = L_bb^-1, V = U_bb^-1, all blocks in parallel, 8 group barriers), and
// the off-diagonal factor rows are premultiplied and negated in place (-l W, -u V). A forward
// block step is then y_b = W_b c_b for the block's pivot rows and c_r += (-l~_r) c_b for
// later rows, both from the raw c_b values, with one barrier; the backward step likewise
// with V and -u~. The block steps are branch-free (predicated), so a warp never runs both
// sides of a row-role test.
//
// Refinement: x_0 = LU \ rhs; the first residual r_1 = rhs - A x_0 is evaluated in
// double-float arithmetic (M = hi + lo, x = hi + lo, error-free products and sums on the
// FP32x2 pipe); later residuals are updated incrementally, r_{k+1} = r_k - A d_k, in FP32,
// since d_k is already small. One solve call site serves every right-hand side.
//
// Objective and adjoint (Eq. 1, 7-9): b_l = H_loss I, loss = sum e(b_l, t_l),
// u = H_loss^T conj(G), A mu = u (A^T = A), dloss/dC_k = Im(mu_k I_k)/(w C_k^2).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "solve_common.cuh"

namespace mts {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 up(u64 v) {
  float2 r;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 fadd2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

template <int NM>
struct SmemV3 {
  static constexpr int NB = NM / 8;
  static constexpr int NW = NM > 32 ? NM / 32 : 1;  // candidate buffers (warps per group)
  float prow_re[2][NW][NM];    // pivot-row candidates, real parts, [parity][warp][col]
  float prow_im[2][NW][NM];    // imaginary parts
  float2 Wb[NB][8][8];         // inverses of the diagonal blocks of L (unit lower)
  float2 Vb[NB][8][8];         // and of U (upper)
  ulonglong2 xhl[NM];          // x split: ((re_hi, im_hi), (re_lo, im_lo))
  double2 x64[NM];
  float2 Gs[NM];               // conj(G) of a chunk of loss points
  float2 bp[2][8];
  float2 bq[2][8];
  float2 xs[NM];
  double red[NW];
  float redf[NW];
  float ckey[2][NW];
  int cidx[2][NW];
  unsigned ukey[2][NW];
};

template <int NM>
__device__ __forceinline__ void gsync() {
  if constexpr (NM <= 32) __syncwarp();
  else __syncthreads();
}

template <int NM>
__device__ inline float gmax(float v, SmemV3<NM>& sm, int r) {
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
    for (int q = 1; q < SmemV3<NM>::NW; ++q) m = fmaxf(m, sm.redf[q]);
    return m;
  }
}

template <int NM>
__device__ inline double gsum(double v, SmemV3<NM>& sm, int r) {
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
    for (int q = 0; q < SmemV3<NM>::NW; ++q) s += sm.red[q];
    return s;
  }
}

// c += a * b (complex, FP32)
__device__ __forceinline__ void cma(float2& c, float2 a, float2 b) {
  c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
  c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
}
__device__ __forceinline__ float2 crecip(float2 a) {
  // hardware approximate reciprocal (one instruction, <= 1 ulp): the factors are FP32 and
  // refinement on double-float residuals removes their rounding; it shortens the per-step
  // pivot chain of the LU
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(a.x * a.x + a.y * a.y));
  return make_float2(a.x * inv, -a.y * inv);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Objective term of one loss point in FP32 and its cotangent G = de/dRe b + j de/dIm b
// (targets are read as FP64 and rounded).
__device__ __forceinline__ float point_loss_f(int mode, float2 b, const double* t, float* gx, float* gy) {
  if (mode == 0) {
    const float a = sqrtf(b.x * b.x + b.y * b.y);
    const float r = a - (float)t[0];
    const float s = a > 0.0f ? 2.0f * r / a : 0.0f;
    *gx = s * b.x;
    *gy = s * b.y;
    return r * r;
  }
  const float ex = b.x - (float)t[0], ey = b.y - (float)t[1];
  *gx = 2.0f * ex;
  *gy = 2.0f * ey;
  return ex * ex + ey * ey;
}

// column j (a compile-time constant after unrolling) of a block stored as 4 real pairs and
// 4 imaginary pairs
__device__ __forceinline__ float2 elem(const u64* re4, const u64* im4, int j) {
  const float2 r = up(re4[j >> 1]), i = up(im4[j >> 1]);
  return (j & 1) ? make_float2(r.y, i.y) : make_float2(r.x, i.x);
}
__device__ __forceinline__ void set_elem(u64* re4, u64* im4, int j, float2 v) {
  const float2 r = up(re4[j >> 1]), i = up(im4[j >> 1]);
  if (j & 1) {
    re4[j >> 1] = pk(r.x, v.x);
    im4[j >> 1] = pk(i.x, v.y);
  } else {
    re4[j >> 1] = pk(v.x, r.y);
    im4[j >> 1] = pk(v.y, i.y);
  }
}

template <int NM>
__global__ void __launch_bounds__(NM >= 64 ? NM : 128, NM >= 64 ? 5 : 1) solve_mixed_v3(SolveArgs a, int64_t n_sys) {
  constexpr int NB = NM / 8;
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int grp = threadIdx.x / NM, r = threadIdx.x % NM;
  SmemV3<NM>& sm = reinterpret_cast<SmemV3<NM>*>(dsm)[grp];

  const int64_t li = (int64_t)blockIdx.x * G + grp;
  const bool in_range = li < n_sys;
  const int64_t sys = in_range ? launch_sys(a, li) : 0;
  SysInfo si = sys_info(a, sys);
  const bool valid = in_range && si.N <= NM;  // larger systems: solve_large.cu
  if (!valid) si.N = 0;
  const int N = si.N;
  const double w = si.w;
  const float w32 = (float)w;
  const bool real_row = r < N;
  const bool bwd = a.rhs_in != nullptr;
  const double Cr = real_row ? a.C[si.b * a.n_ports + si.k0 + r] : 1.0;
  cd Dr = {0.0, 0.0};
  if (real_row) Dr = {a.R[si.k0 + r], -1.0 / (w * Cr)};
  // M = hi + lo of this structure, read through L1 (shared by every system of the structure)
  const int64_t mo = a.t.nn_off[si.s];
  const float* __restrict__ Mh = a.M32hi + mo;
  const float* __restrict__ Ml = a.M32lo + mo;

  // ---- row r of A (FP32), identity rows for padding ----
  // The diagonal entry needs FP64 (w (M_rr hi + lo) + Im D_r, then rounded): it is computed
  // once per thread here, not inside the unrolled column loop, where each column's branch
  // would run its FP64 instructions for the one lane with c == r (this part's FP64 rate is
  // 1/62 of FP32).
  float dre = 1.0f, dim = 0.0f;
  if (real_row) {
    dre = (float)Dr.x;
    dim = (float)(w * ((double)__ldg(Mh + r * N + r) + (double)__ldg(Ml + r * N + r)) + Dr.y);
  }
  u64 ReP[NB][4], ImP[NB][4];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float re2[2], im2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 8 * b + 2 * m + h;
        const float mm = (real_row && c < N) ? w32 * __ldg(Mh + c * N + r) : 0.0f;  // M symmetric
        re2[h] = (c == r) ? dre : 0.0f;
        im2[h] = (c == r) ? dim : mm;
      }
      ReP[b][m] = pk(re2[0], re2[1]);
      ImP[b][m] = pk(im2[0], im2[1]);
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
      const float2 cur = elem(ReP[0], ImP[0], kk);
      int p, src = 0;
      if constexpr (NM >= 32) {
        // magnitude bits with the row index in the low 6 bits (ties -> smaller row)
        const float mag = cur.x * cur.x + cur.y * cur.y;
        const unsigned key = (pivstep < NM) ? 0u : ((__float_as_uint(mag) & ~63u) | (unsigned)(63 - r));
        unsigned wmax;
        asm volatile("redux.sync.max.u32 %0, %1, 0xffffffff;" : "=r"(wmax) : "r"(key));
        const int cand = 63 - (int)(wmax & 63u);
        const int wv = r >> 5;
        if constexpr (NM == 32) {
          p = cand;
        } else {
          if ((r & 31) == 0) sm.ukey[par][wv] = wmax;
          if (r == cand) {  // this warp's candidate publishes its row speculatively
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              if (b >= nact) break;  // finished panels sit at the end: skip them by a jump
              {
                ulonglong2* dr = reinterpret_cast<ulonglong2*>(&sm.prow_re[par][wv][8 * b]);
                ulonglong2* di = reinterpret_cast<ulonglong2*>(&sm.prow_im[par][wv][8 * b]);
                dr[0] = make_ulonglong2(ReP[b][0], ReP[b][1]);
                dr[1] = make_ulonglong2(ReP[b][2], ReP[b][3]);
                di[0] = make_ulonglong2(ImP[b][0], ImP[b][1]);
                di[1] = make_ulonglong2(ImP[b][2], ImP[b][3]);
              }
            }
          }
          __syncthreads();
          unsigned best = sm.ukey[par][0];
#pragma unroll
          for (int q = 1; q < SmemV3<NM>::NW; ++q) {
            const unsigned uq = sm.ukey[par][q];
            if (uq > best) {
              best = uq;
              src = q;
            }
          }
          p = 63 - (int)(best & 63u);
        }
      } else {
        float key = (pivstep < NM) ? -1.0f : cur.x * cur.x + cur.y * cur.y;
        int idx = r;
        argmax_shfl(key, idx, NM);
        p = idx;
      }
      if constexpr (NM <= 32) {
        if (r == p) {
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (b < nact) {
              ulonglong2* dr = reinterpret_cast<ulonglong2*>(&sm.prow_re[par][0][8 * b]);
              ulonglong2* di = reinterpret_cast<ulonglong2*>(&sm.prow_im[par][0][8 * b]);
              dr[0] = make_ulonglong2(ReP[b][0], ReP[b][1]);
              dr[1] = make_ulonglong2(ReP[b][2], ReP[b][3]);
              di[0] = make_ulonglong2(ImP[b][0], ImP[b][1]);
              di[1] = make_ulonglong2(ImP[b][2], ImP[b][3]);
            }
        }
        __syncwarp();
      }
      if (r == p) pivstep = k;
      if (pivstep > k) {
        const float* ur = sm.prow_re[par][src];
        const float* ui = sm.prow_im[par][src];
        const float2 l = cmulf(cur, crecip(make_float2(ur[kk], ui[kk])));
        const u64 NLx = pk(-l.x, -l.x), Ly = pk(l.y, l.y), NLy = pk(-l.y, -l.y);
        const u64* urp = reinterpret_cast<const u64*>(ur);
        const u64* uip = reinterpret_cast<const u64*>(ui);
#pragma unroll
        for (int m = (kk + 1) / 2; m < 4; ++m) {  // panel pairs right of column kk
          const u64 UX = urp[m], UY = uip[m];
          ReP[0][m] = ffma2(Ly, UY, ffma2(NLx, UX, ReP[0][m]));
          ImP[0][m] = ffma2(NLy, UX, ffma2(NLx, UY, ImP[0][m]));
        }
        set_elem(ReP[0], ImP[0], kk, l);
#pragma unroll
        for (int b = 1; b < NB; ++b) {
          if (b >= nact) break;  // finished panels sit at the end: skip them by a jump
          {
            const ulonglong2 x0 = reinterpret_cast<const ulonglong2*>(ur)[2 * b];
            const ulonglong2 x1 = reinterpret_cast<const ulonglong2*>(ur)[2 * b + 1];
            const ulonglong2 y0 = reinterpret_cast<const ulonglong2*>(ui)[2 * b];
            const ulonglong2 y1 = reinterpret_cast<const ulonglong2*>(ui)[2 * b + 1];
            const u64 UX[4] = {x0.x, x0.y, x1.x, x1.y}, UY[4] = {y0.x, y0.y, y1.x, y1.y};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              ReP[b][m] = ffma2(Ly, UY[m], ffma2(NLx, UX[m], ReP[b][m]));
              ImP[b][m] = ffma2(NLy, UX[m], ffma2(NLx, UY[m], ImP[b][m]));
            }
          }
        }
      }
    }
    if constexpr (NB > 1) {  // rotate: the finished panel goes to the end
      u64 tr[4], ti[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        tr[m] = ReP[0][m];
        ti[m] = ImP[0][m];
      }
#pragma unroll
      for (int b = 0; b < NB - 1; ++b)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          ReP[b][m] = ReP[b + 1][m];
          ImP[b][m] = ImP[b + 1][m];
        }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        ReP[NB - 1][m] = tr[m];
        ImP[NB - 1][m] = ti[m];
      }
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
      for (int j = 0; j < 8; ++j) dg[j] = elem(ReP[b], ImP[b], j);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (ii == s) {  // W_s = e_s - sum_{m<s} L[s][m] W_m
#pragma unroll
      for (int j = 0; j < s; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = j; m < s; ++m) cma(acc, dg[m], sm.Wb[Mb][m][j]);
        sm.Wb[Mb][s][j] = make_float2(-acc.x, -acc.y);
      }
      sm.Wb[Mb][s][s] = make_float2(1.0f, 0.0f);
#pragma unroll
      for (int j = s + 1; j < 8; ++j) sm.Wb[Mb][s][j] = make_float2(0.0f, 0.0f);
    }
    if (ii == 7 - s) {  // V_i = (e_i - sum_{m>i} U[i][m] V_m) / U[i][i], i = 7 - s
      const int i = 7 - s;
      const float2 dinv = crecip(dg[i]);
#pragma unroll
      for (int j = 0; j < i; ++j) sm.Vb[Mb][i][j] = make_float2(0.0f, 0.0f);
      sm.Vb[Mb][i][i] = dinv;
#pragma unroll
      for (int j = i + 1; j < 8; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = i + 1; m <= j; ++m) cma(acc, dg[m], sm.Vb[Mb][m][j]);
        const float2 v = cmulf(acc, dinv);
        sm.Vb[Mb][i][j] = make_float2(-v.x, -v.y);
      }
    }
    gsync<NM>();
  }
  // diagonal block <- W (strictly lower) and V (upper); off-diagonal blocks premultiplied
  // and negated in place: -(l W_b) for multipliers (columns in increasing order: entry j
  // reads columns >= j only), -(u V_b) for U entries (decreasing order: reads <= j only)
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (b == Mb) {
#pragma unroll
      for (int j = 0; j < 8; ++j) set_elem(ReP[b], ImP[b], j, (j < ii) ? sm.Wb[b][ii][j] : sm.Vb[b][ii][j]);
    } else if (b < Mb) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float2 acc = elem(ReP[b], ImP[b], j);  // W_b[j][j] = 1
#pragma unroll
        for (int m = j + 1; m < 8; ++m) cma(acc, elem(ReP[b], ImP[b], m), sm.Wb[b][m][j]);
        set_elem(ReP[b], ImP[b], j, make_float2(-acc.x, -acc.y));
      }
    } else {
#pragma unroll
      for (int j = 7; j >= 0; --j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m <= j; ++m) cma(acc, elem(ReP[b], ImP[b], m), sm.Vb[b][m][j]);
        set_elem(ReP[b], ImP[b], j, make_float2(-acc.x, -acc.y));
      }
    }
  }

  // ---- block triangular solve (branch-free): returns the unknown x_r ----
  auto lu_solve = [&](float2 rhs) -> float2 {
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) {
      if (Mb == kb) sm.bp[kb & 1][ii] = rhs;
      gsync<NM>();
      const bool piv = Mb == kb, later = Mb > kb;
      float2 acc1 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        // the mask is applied to the freshly loaded value, so that no masked copy of the
        // (loop-invariant) coefficients is kept in registers
        const bool use = later || (piv && j < ii);
        const float2 v = sm.bp[kb & 1][j];
        cma((j & 1) ? acc1 : rhs, elem(ReP[kb], ImP[kb], j), use ? v : make_float2(0.0f, 0.0f));
      }
      rhs.x += acc1.x;
      rhs.y += acc1.y;
    }
#pragma unroll
    for (int kb = NB - 1; kb >= 0; --kb) {
      if (Mb == kb) sm.bq[kb & 1][ii] = rhs;
      gsync<NM>();
      const bool piv = Mb == kb, earlier = Mb < kb;
      float2 acc = piv ? make_float2(0.0f, 0.0f) : rhs;
      float2 acc1 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bool use = earlier || (piv && j >= ii);
        const float2 v = sm.bq[kb & 1][j];
        cma((j & 1) ? acc1 : acc, elem(ReP[kb], ImP[kb], j), use ? v : make_float2(0.0f, 0.0f));
      }
      rhs = make_float2(acc.x + acc1.x, acc.y + acc1.y);
    }
    sm.xs[pivstep] = rhs;
    gsync<NM>();
    const float2 out = sm.xs[r];
    gsync<NM>();
    return out;
  };

  // publish the FP64 iterate of this thread's unknown and its double-float split
  auto publish = [&](cd x) {
    sm.x64[r] = make_double2(x.x, x.y);
    const float rh = (float)x.x, ih = (float)x.y;
    sm.xhl[r] = make_ulonglong2(pk(rh, ih), pk((float)(x.x - (double)rh), (float)(x.y - (double)ih)));
    gsync<NM>();
  };

  // accurate residual of row r: rhs_r - sum_j A_rj x_j, sum_j M_rj x_j in double-float
  auto residual = [&](cd rhs) -> cd {
    const double2 xr = sm.x64[r];
    if (!real_row) return {rhs.x - xr.x, rhs.y - xr.y};
    u64 S[2] = {0ull, 0ull}, Lo[2] = {0ull, 0ull};  // (re, im) high and low parts, 2 chains
    const u64 neg1 = pk(-1.0f, -1.0f);
    for (int j0 = 0; j0 < N; j0 += 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = j0 + h;
        if (j < N) {
          const float2 m = make_float2(__ldg(Mh + j * N + r), __ldg(Ml + j * N + r));
          const ulonglong2 xj = sm.xhl[j];
          const u64 A = pk(m.x, m.x), Al = pk(m.y, m.y);
          const u64 p = fmul2(A, xj.x);
          u64 e = ffma2(A, xj.x, fmul2(p, neg1));
          e = ffma2(A, xj.y, e);
          e = ffma2(Al, xj.x, e);
          const u64 t = fadd2(S[h], p);
          const u64 z = fsub2(t, S[h]);
          const u64 err = fadd2(fsub2(S[h], fsub2(t, z)), fsub2(p, z));
          S[h] = t;
          Lo[h] = fadd2(Lo[h], fadd2(err, e));
        }
      }
    }
    const float2 s0 = up(S[0]), s1 = up(S[1]), l0 = up(Lo[0]), l1 = up(Lo[1]);
    const double Sr = ((double)s0.x + (double)l0.x) + ((double)s1.x + (double)l1.x);
    const double Si = ((double)s0.y + (double)l0.y) + ((double)s1.y + (double)l1.y);
    const double ax = Dr.x * xr.x - Dr.y * xr.y;
    const double ay = Dr.x * xr.y + Dr.y * xr.x;
    return {rhs.x - ax + w * Si, rhs.y - ay - w * Sr};
  };

  // r -= A d for the correction d just solved (in sm.xs), FP32
  auto residual_update = [&](cd res, float2 dr) -> cd {
    if (!real_row) return {res.x - dr.x, res.y - dr.y};
    u64 S0 = 0ull, S1 = 0ull;
    int j = 0;
    for (; j + 1 < N; j += 2) {
      const float m0 = __ldg(Mh + j * N + r), m1 = __ldg(Mh + (j + 1) * N + r);
      const float2 d0 = sm.xs[j], d1 = sm.xs[j + 1];
      S0 = ffma2(pk(m0, m0), pk(d0.x, d0.y), S0);
      S1 = ffma2(pk(m1, m1), pk(d1.x, d1.y), S1);
    }
    if (j < N) {
      const float m0 = __ldg(Mh + j * N + r);
      const float2 d0 = sm.xs[j];
      S0 = ffma2(pk(m0, m0), pk(d0.x, d0.y), S0);
    }
    const float2 s = make_float2(up(S0).x + up(S1).x, up(S0).y + up(S1).y);
    const float dx = (float)Dr.x, dy = (float)Dr.y;
    const float adx = dx * dr.x - dy * dr.y - w32 * s.y;
    const float ady = dx * dr.y + dy * dr.x + w32 * s.x;
    return {res.x - (double)adx, res.y - (double)ady};
  };

  const float tol = (float)a.tol;
  const int max_it = a.max_refine;
  const int64_t ioff = si.b * a.sumFN + a.t.fn_off[si.s] + (int64_t)si.f * N;
  const bool has_obj = !bwd && a.target != nullptr;
  cd x = {0.0, 0.0};
  if (bwd && real_row) {
    const double* Ip = a.I + 2 * (ioff + r);
    x = {Ip[0], Ip[1]};
  }
  cd u = {0.0, 0.0};
  if (bwd && real_row) {
    const double* up_ = a.rhs_in + 2 * (ioff + r);
    u = {up_[0], up_[1]};
  }
  bool conv_all = true;
  bool bad = false;
  const int ph0 = bwd ? 1 : 0, ph1 = (bwd || has_obj) ? 2 : 1;
#pragma unroll 1
  for (int ph = ph0; ph < ph1; ++ph) {
    cd rhs64 = {0.0, 0.0};
    if (ph == 0) {
      if (real_row) {
        const double* Vp = a.V + 2 * (a.t.fn_off[si.s] + (int64_t)si.f * N + r);
        rhs64 = {Vp[0], Vp[1]};
      }
    } else {
      rhs64 = u;
    }
    cd xk = {0.0, 0.0};
    cd res = rhs64;
    float dprev = 0.0f;
    bool conv = max_it == 0;
#pragma unroll 1
    for (int it = 0;; ++it) {
      const float2 d = lu_solve(make_float2((float)res.x, (float)res.y));
      xk.x += (double)d.x;
      xk.y += (double)d.y;
      const float dm = gmax<NM>(fabsf(d.x) + fabsf(d.y), sm, r);
      bool stop = it >= max_it;
      if (it > 0) {
        const float xm = gmax<NM>((float)(fabs(xk.x) + fabs(xk.y)), sm, r);
        const float est = dm * fminf(1.0f, dm / fmaxf(dprev, 1e-30f));
        conv = conv || (est <= tol * xm);
        stop = stop || conv || !(dm <= 0.5f * dprev);
      }
      dprev = dm;
      if constexpr (NM <= 32) {
        if (__all_sync(0xffffffffu, stop)) break;
      } else {
        if (stop) break;
      }
      if (it == 0) {
        publish(xk);
        res = residual(rhs64);
      } else {
        res = residual_update(res, d);
      }
    }
    conv_all = conv_all && conv;
    bad = bad || (real_row && !(isfinite(xk.x) && isfinite(xk.y)));
    if (ph == 0) {
      x = xk;
      if (valid && real_row) {
        double* Ip = a.I + 2 * (ioff + r);
        Ip[0] = x.x;
        Ip[1] = x.y;
        if (a.I_out) {
          a.I_out[2 * (ioff + r)] = x.x;
          a.I_out[2 * (ioff + r) + 1] = x.y;
        }
      }
      if (valid && a.Bop != nullptr && a.bop_off[si.s + 1] > a.bop_off[si.s]) {
        // tensor-core operand pieces of I: rows 2 (b F_s + f) + {0: re, 1: im}; thread r
        // owns column r, columns N .. K_pad-1 are zero
        const int F = a.freq_off[si.s + 1] - a.freq_off[si.s];
        const int nkc = (N + kChunkK - 1) / kChunkK;
        const int64_t ntile = (2 * a.n_cfg * F + kTileN - 1) / kTileN;
        char* base = reinterpret_cast<char*>(a.Bop + a.bop_off[si.s]);
        const size_t tile_bytes = (size_t)kTileN * kChunkK * 2;
        for (int kg = r; kg < nkc * kChunkK; kg += NM) {
          const bool own = (kg == r) && real_row;
          const int kc = kg / kChunkK, kc_k = kg % kChunkK;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int64_t n = 2 * (si.b * F + si.f) + c;
            const int64_t tile = n / kTileN;
            const uint32_t rr = (uint32_t)(n % kTileN);
            // x = xh + xl (FP32 pair); pieces p_q = bf16(rem), rem -= p_q in FP32 (exact
            // apart from the final rounding of rem + xl, 2^-32 relative)
            const double xv = own ? (c == 0 ? x.x : x.y) : 0.0;
            const float xh = (float)xv, xl = (float)(xv - (double)xh);
            float rem = xh;
            for (int q = 0; q < a.npieces; ++q) {
              const __nv_bfloat16 h = __float2bfloat16_rn(rem);
              rem = rem - __bfloat162float(h);
              if (q == 0) rem += xl;
              size_t off = ((size_t)(q * ntile + tile) * nkc + kc) * tile_bytes + swz128(rr, kc_k);
              *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
            }
          }
        }
      }
      if (has_obj) {
        // objective at the loss points (FP32 sums of FP32 H rows, FP64 per-point terms)
        publish(x);
        const int L = a.loss_off[si.s + 1] - a.loss_off[si.s];
        const float* Hl = a.Hl32 + a.t.ln_off[si.s];
        const float* HlT = a.HlT32 + a.t.ln_off[si.s];  // [k][l]: lanes l read consecutively
        const int tw = a.loss_mode == 0 ? 1 : 2;
        const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                           (a.t.fl_off[si.s] + (int64_t)si.f * L) * tw;
        const int64_t wo = a.t.fl_off[si.s] + (int64_t)si.f * L;  // weight / offset base
        double lsum = 0.0;
        u64 U = 0ull;
        for (int c0 = 0; c0 < a.max_loss; c0 += NM) {
          const int l = c0 + r;
          cd Gl = {0.0, 0.0};
          if (l < L) {
            u64 b0 = 0ull, b1 = 0ull;
            int k = 0;
            for (; k + 1 < N; k += 2) {
              const float h0 = HlT[(int64_t)k * L + l], h1 = HlT[(int64_t)(k + 1) * L + l];
              b0 = ffma2(pk(h0, h0), sm.xhl[k].x, b0);
              b1 = ffma2(pk(h1, h1), sm.xhl[k + 1].x, b1);
            }
            if (k < N) {
              const float h0 = HlT[(int64_t)k * L + l];
              b0 = ffma2(pk(h0, h0), sm.xhl[k].x, b0);
            }
            float2 bl = make_float2(up(b0).x + up(b1).x, up(b0).y + up(b1).y);
            float wl = 1.0f;
            if (a.loss_offset) {
              bl.x += (float)a.loss_offset[2 * (wo + l)];
              bl.y += (float)a.loss_offset[2 * (wo + l) + 1];
            }
            if (a.loss_weight) {
              wl = (float)a.loss_weight[wo + l];
              bl.x *= wl;
              bl.y *= wl;
            }
            float gx, gy;
            lsum += (double)point_loss_f(a.loss_mode, bl, tb + (int64_t)l * tw, &gx, &gy);
            Gl = {(double)(gx * wl), (double)(gy * wl)};
          }
          sm.Gs[r] = make_float2((float)Gl.x, -(float)Gl.y);  // conj(G)
          gsync<NM>();
          if (real_row) {
            const int lc = max(0, min(NM, L - c0));
            for (int q = 0; q < lc; ++q) {
              const float h = Hl[(int64_t)(c0 + q) * N + r];
              const float2 g = sm.Gs[q];
              U = ffma2(pk(h, h), pk(g.x, g.y), U);
            }
          }
          gsync<NM>();
        }
        const double tot = gsum<NM>(lsum, sm, r);
        if (valid && r == 0) a.loss_part[sys] = tot;
        const float2 uf = up(U);
        u = {(double)uf.x, (double)uf.y};
      }
    } else {
      const cd mu = xk;
      // Im(mu x)/(w C^2) = Im(mu x) w (1/(w C))^2, without a second division
      if (valid && real_row) {
        a.grad_part[ioff + r] = (mu.x * x.y + mu.y * x.x) * w * (Dr.y * Dr.y);
        if (!bwd && a.mu_out) {
          a.mu_out[2 * (ioff + r)] = mu.x;
          a.mu_out[2 * (ioff + r) + 1] = mu.y;
        }
      }
    }
  }
  const float fb = gmax<NM>(bad ? 2.0f : (conv_all ? 0.0f : 1.0f), sm, r);
  if (valid && r == 0 && !bwd) a.status[sys] = (int)fb;
}

template <int NM>
static cudaError_t launch_v3(const SolveArgs& a, int64_t n_sys, cudaStream_t st) {
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  const size_t smem = sizeof(SmemV3<NM>) * G;
  cudaError_t e = cudaFuncSetAttribute(solve_mixed_v3<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n_sys + G - 1) / G);
  solve_mixed_v3<NM><<<grid, CT, smem, st>>>(a, n_sys);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const SolveArgs& a, int64_t n_sys, int max_ports, cudaStream_t st) {
  if (max_ports <= 8) return launch_v3<8>(a, n_sys, st);
  if (max_ports <= 16) return launch_v3<16>(a, n_sys, st);
  if (max_ports <= 32) return launch_v3<32>(a, n_sys, st);
  if (max_ports <= 64) return launch_v3<64>(a, n_sys, st);
  return cudaErrorNotSupported;
}

}  // namespace mts
