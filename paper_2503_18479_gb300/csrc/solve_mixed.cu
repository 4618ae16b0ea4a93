// solve_mixed.cu -- (b) port solve, (d) objective and (adj) adjoint for MTS_MIXED and
// MTS_BF16: FP32 complex LU with partial pivoting, iterative refinement with residuals in
// double-float (FP32-pair) arithmetic, one system per group of NM threads (thread r owns
// row r of A = diag(R) + j w M + diag(1/(j w C)); paper Eq. 2, 6, 11).
//
// Register layout: row r lives in NB = NM/8 blocks of 8 columns; each block keeps the real
// parts of its columns in 4 packed 64-bit pairs (columns 2m, 2m+1) and the imaginary parts
// in another 4, so that updates run on the packed FP32x2 pipe over adjacent columns
// (re' = re + n.x ux - n.y uy, im' = im + n.x uy + n.y ux: four fma.rn.f32x2 per column
// pair). Rows are never moved: the pivot of step k is the row with the largest |a_rk|
// among rows not chosen yet (one redux.sync.max per warp on the magnitude with the row
// index in the low bits), and the step at which a row was chosen is its `pivstep`.
//
// LU in panels of 8 columns with delayed updates. The active panel is always register
// block 0 (after each panel the blocks rotate by one; NB rotations restore the order).
// Inside a panel the 8 pivot steps update block 0 only (rank-1 on 8 columns), so a step
// publishes 8 columns of its pivot row. At the panel end, with L_bb and U_bb the panel's
// unit-lower and upper diagonal blocks in pivot order:
//   W_b = L_bb^-1 and V_b = U_bb^-1 (one column per thread, 16 threads);
//   every row solves lt L_bb = l for its panel multipliers l (rows chosen in this panel
//     use their multipliers left of their own pivot, rows chosen earlier use none), so
//     lt = l W_b;
//   the panel's pivot rows publish their trailing columns as they were before the panel,
//     and every row adds -lt times them: unchosen rows get A_22 - L_21 U_12, and the pivot
//     rows get U_12 = W_b A_12 itself (their lt is e_ii - W_b[ii]);
//   block 0 keeps -lt (unchosen rows: the block-L multipliers L_rb W_b of the forward
//     sweep), V_b's row ii (the panel's pivot row ii), or its U entries (earlier rows).
//
// Solves with P A = L U in blocks of 8 (pivot order), L = Lt D, D = diag(L_bb):
//   forward: yt_b = c_b - sum_{a<b} (L_ba W_a) yt_a, one barrier per block: the block's
//     pivot rows publish their value, every row adds its block-b coefficients times it
//     (rows past their own block add garbage to a value they no longer use);
//   z_b = W_b yt_b for all blocks at once;
//   backward: x_b = V_b (z_b - sum_{c>b} U_bc x_c), two barriers per block (publish the
//     block's partial values, the pivot rows apply their V row, publish x_b, earlier rows
//     subtract U_rb x_b).
// No step masks a coefficient: each row's block b holds exactly what its role in block b
// needs.
//
// Refinement: x_0 = LU \ rhs; the first residual r_1 = rhs - A x_0 is evaluated in
// double-float arithmetic (M = hi + lo, x_0 in FP32, error-free products and sums on the
// FP32x2 pipe); later residuals are updated incrementally, r_{k+1} = r_k - A d_k, in FP32.
// The stop test uses max|d_k| (folded into the permutation barrier of each solve).
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
struct SmemV4 {
  static constexpr int NB = NM / 8;
  static constexpr int NW = NM > 32 ? NM / 32 : 1;      // warps per group
  static constexpr int NT = NM > 8 ? NM - 8 : 8;        // trailing columns of the first panel
  __align__(16) float prow[2][NW][16];   // in-panel pivot-row candidates: block 0, re then im
  __align__(16) float dre[8][8];         // the panel's pivot rows (pivot order): L_bb below
  __align__(16) float dim[8][8];         // the diagonal, U_bb on and above it
  __align__(16) float vre[8][8];         // V_b = U_bb^-1 of the current panel
  __align__(16) float vim[8][8];
  __align__(16) float wre[NB][8][8];     // W_b = L_bb^-1 of every block
  __align__(16) float wim[NB][8][8];
  __align__(16) float tre[8][NT];        // trailing columns of the panel's pivot rows
  __align__(16) float tim[8][NT];
  __align__(16) float sre[2][8];         // block values published in the sweeps
  __align__(16) float sim[2][8];
  __align__(16) float yre[NM];           // forward-sweep values by pivot position
  __align__(16) float yim[NM];
  __align__(16) float2 xc[NM];           // unknowns by column (FP32), permutation buffer
  __align__(16) float2 Gs[NM];           // conj(G) of a chunk of loss points
  double red[NW];
  float redf[NW];
  unsigned ukey[2][NW];
  unsigned umax[NW];
};

template <int NM>
__device__ __forceinline__ void gsync() {
  if constexpr (NM <= 32) __syncwarp();
  else __syncthreads();
}

template <int NM>
__device__ inline float gmax(float v, SmemV4<NM>& sm, int r) {
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
    for (int q = 1; q < SmemV4<NM>::NW; ++q) m = fmaxf(m, sm.redf[q]);
    return m;
  }
}

template <int NM>
__device__ inline double gsum(double v, SmemV4<NM>& sm, int r) {
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
    for (int q = 0; q < SmemV4<NM>::NW; ++q) s += sm.red[q];
    return s;
  }
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
// c -= a * b (complex, FP32)
__device__ __forceinline__ void cms(float2& c, float2 a, float2 b) {
  c.x = fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x));
  c.y = fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y));
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

// sum_j a_j v_j over one register block (a: 4 re pairs, 4 im pairs) and 8 complex values
// stored as re[8], im[8] (16-byte aligned)
__device__ __forceinline__ float2 bdot(const u64* re4, const u64* im4, const float* vre, const float* vim) {
  const ulonglong2 r0 = reinterpret_cast<const ulonglong2*>(vre)[0];
  const ulonglong2 r1 = reinterpret_cast<const ulonglong2*>(vre)[1];
  const ulonglong2 i0 = reinterpret_cast<const ulonglong2*>(vim)[0];
  const ulonglong2 i1 = reinterpret_cast<const ulonglong2*>(vim)[1];
  const u64 VR[4] = {r0.x, r0.y, r1.x, r1.y}, VI[4] = {i0.x, i0.y, i1.x, i1.y};
  u64 A = 0ull, B = 0ull, C = 0ull, D = 0ull;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    A = ffma2(re4[m], VR[m], A);
    B = ffma2(im4[m], VI[m], B);
    C = ffma2(re4[m], VI[m], C);
    D = ffma2(im4[m], VR[m], D);
  }
  const float2 a = up(A), b = up(B), c = up(C), d = up(D);
  return make_float2((a.x + a.y) - (b.x + b.y), (c.x + c.y) + (d.x + d.y));
}

// KF: the problem keeps its factors (a separate instantiation, so that the common path
// carries none of the extra registers)
template <int NM, bool KF>
__global__ void __launch_bounds__(NM >= 64 ? NM : 128, NM >= 64 ? 6 : (NM == 32 ? 3 : 4))
solve_mixed_v4(SolveArgs a, int64_t n_sys) {
  constexpr int NB = NM / 8;
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int grp = threadIdx.x / NM, r = threadIdx.x % NM;
  SmemV4<NM>& sm = reinterpret_cast<SmemV4<NM>*>(dsm)[grp];

  const int64_t li = (int64_t)blockIdx.x * G + grp;
  const bool in_range = li < n_sys;
  const int64_t sys = in_range ? launch_sys(a, li) : 0;
  u64 ReP[NB][4], ImP[NB][4];
  int pivstep = NM;
  bool need_lu = true;
  if constexpr (NM == 64 && KF) {
    // ---- a backward solve of a problem that keeps its factors: load the forward's rows,
    // pivot steps and W blocks instead of factoring again (a pivot step out of range means
    // the block was never written: factor) ----
    if (a.rhs_in != nullptr && a.fac != nullptr) {
      const char* fb = static_cast<const char*>(a.fac) + (size_t)sys * kFacStride;
      const u64* fr = reinterpret_cast<const u64*>(fb);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          ReP[b][m] = fr[(size_t)(b * 4 + m) * NM + r];
          ImP[b][m] = fr[(size_t)(NB * 4 + b * 4 + m) * NM + r];
        }
      pivstep = reinterpret_cast<const int32_t*>(fb + kFacRows)[r];
      const float* fw = reinterpret_cast<const float*>(fb + kFacRows + kFacPiv);
      for (int i = r; i < NB * 64; i += NM) {
        (&sm.wre[0][0][0])[i] = fw[i];
        (&sm.wim[0][0][0])[i] = fw[NB * 64 + i];
      }
      need_lu = __syncthreads_or(!in_range || !((unsigned)pivstep < (unsigned)NM)) != 0;
    }
  }
  if (need_lu) {
  pivstep = NM;
  {
    // ---- row r of A (FP32), identity rows for padding. The per-system values used here are
    // derived again after the LU, so that none of them stays live across it. ----
    SysInfo si = sys_info(a, sys);
    const int N = (in_range && si.N <= NM) ? si.N : 0;
    const double w = si.w;
    const float w32 = (float)w;
    const bool real_row = r < N;
    const float* __restrict__ Mh = a.M32hi + a.t.nn_off[si.s];
    const float* __restrict__ Ml = a.M32lo + a.t.nn_off[si.s];
    // The diagonal entry needs FP64 (w (M_rr hi + lo) - 1/(w C_r), then rounded): it is
    // computed once per thread here, not inside the unrolled column loop, where each
    // column's branch would run its FP64 instructions for the one lane with c == r.
    float dre = 1.0f, dimv = 0.0f;
    if (real_row) {
      const double Cr = a.C[si.b * a.n_ports + si.k0 + r];
      dre = (float)a.R[si.k0 + r];
      dimv = (float)(w * ((double)__ldg(Mh + r * N + r) + (double)__ldg(Ml + r * N + r)) - 1.0 / (w * Cr));
    }
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
          im2[h] = (c == r) ? dimv : mm;
        }
        ReP[b][m] = pk(re2[0], re2[1]);
        ImP[b][m] = pk(im2[0], im2[1]);
      }
  }

  // ---- LU with partial pivoting, panels of 8 columns, delayed trailing updates ----
#pragma unroll 1
  for (int kb = 0; kb < NB; ++kb) {
    const int nact = NB - kb;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = 8 * kb + kk;
      const int par = kk & 1;
      const float2 cur = elem(ReP[0], ImP[0], kk);
      const bool unpiv = pivstep == NM;
      int p, src = 0;
      if constexpr (NM >= 32) {
        // magnitude bits, a "not chosen yet" bit and the row index in the low 7 bits
        // (ties -> smaller row); chosen rows have key 0
        const float mag = cur.x * cur.x + cur.y * cur.y;
        const unsigned key = unpiv ? ((__float_as_uint(mag) & ~127u) | 64u | (unsigned)(63 - r)) : 0u;
        unsigned wmax;
        asm volatile("redux.sync.max.u32 %0, %1, 0xffffffff;" : "=r"(wmax) : "r"(key));
        const int cand = 63 - (int)(wmax & 63u);
        if constexpr (NM == 32) {
          p = cand;
        } else {
          const int wv = r >> 5;
          if ((r & 31) == 0) sm.ukey[par][wv] = wmax;
          if (r == cand) {  // this warp's candidate publishes its panel block speculatively
            ulonglong2* d = reinterpret_cast<ulonglong2*>(sm.prow[par][wv]);
            d[0] = make_ulonglong2(ReP[0][0], ReP[0][1]);
            d[1] = make_ulonglong2(ReP[0][2], ReP[0][3]);
            d[2] = make_ulonglong2(ImP[0][0], ImP[0][1]);
            d[3] = make_ulonglong2(ImP[0][2], ImP[0][3]);
          }
          __syncthreads();
          unsigned best = sm.ukey[par][0];
#pragma unroll
          for (int q = 1; q < SmemV4<NM>::NW; ++q) {
            const unsigned uq = sm.ukey[par][q];
            if (uq > best) {
              best = uq;
              src = q;
            }
          }
          p = 63 - (int)(best & 63u);
        }
      } else {
        // chosen rows rank -1, the others by magnitude (a NaN magnitude ranks as 0, so
        // that the pick is always a row not chosen yet)
        float key = unpiv ? fmaxf(cur.x * cur.x + cur.y * cur.y, 0.0f) : -1.0f;
        int idx = r;
        argmax_shfl(key, idx, NM);
        p = idx;
      }
      if constexpr (NM <= 32) {
        if (r == p) {
          ulonglong2* d = reinterpret_cast<ulonglong2*>(sm.prow[par][0]);
          d[0] = make_ulonglong2(ReP[0][0], ReP[0][1]);
          d[1] = make_ulonglong2(ReP[0][2], ReP[0][3]);
          d[2] = make_ulonglong2(ImP[0][0], ImP[0][1]);
          d[3] = make_ulonglong2(ImP[0][2], ImP[0][3]);
        }
        __syncwarp();
      }
      if (r == p) {
        pivstep = k;
        // the pivot row of step kk (pivot order) for the panel's diagonal blocks
        ulonglong2* dr = reinterpret_cast<ulonglong2*>(sm.dre[kk]);
        ulonglong2* di = reinterpret_cast<ulonglong2*>(sm.dim[kk]);
        dr[0] = make_ulonglong2(ReP[0][0], ReP[0][1]);
        dr[1] = make_ulonglong2(ReP[0][2], ReP[0][3]);
        di[0] = make_ulonglong2(ImP[0][0], ImP[0][1]);
        di[1] = make_ulonglong2(ImP[0][2], ImP[0][3]);
      }
      if (pivstep > k) {  // rows not chosen yet: rank-1 update of the panel block
        const float* ur = sm.prow[par][src];
        const float2 l = cmulf(cur, crecip(make_float2(ur[kk], ur[8 + kk])));
        const u64 NLx = pk(-l.x, -l.x), Ly = pk(l.y, l.y), NLy = pk(-l.y, -l.y);
        const u64* urp = reinterpret_cast<const u64*>(ur);
        const u64* uip = reinterpret_cast<const u64*>(ur + 8);
#pragma unroll
        for (int m = (kk + 1) / 2; m < 4; ++m) {  // pairs right of column kk
          const u64 UX = urp[m], UY = uip[m];
          ReP[0][m] = ffma2(Ly, UY, ffma2(NLx, UX, ReP[0][m]));
          ImP[0][m] = ffma2(NLy, UX, ffma2(NLx, UY, ImP[0][m]));
        }
        set_elem(ReP[0], ImP[0], kk, l);
      }
    }

    // ---- panel end ----
    gsync<NM>();  // every step's pivot row recorded in dre/dim
    const bool fin = pivstep < 8 * kb;            // chosen in an earlier panel
    const bool pan = !fin && pivstep < 8 * kb + 8;  // chosen in this panel
    const int ii = pan ? pivstep - 8 * kb : 0;
    // V_b = U_bb^-1 (threads 0..7, column r) and W_b = L_bb^-1 (threads 32..39 for 64-row
    // groups, so that the two serial inversions run on different warps; threads 8..15 for
    // 16 and 32 rows; both by the 8 threads of an 8-thread group)
    if (r < 8) {
      const int c = r;
      float2 v[8];
#pragma unroll
      for (int i = 7; i >= 0; --i) {
        float2 acc = make_float2(i == c ? 1.0f : 0.0f, 0.0f);
#pragma unroll
        for (int m = i + 1; m < 8; ++m) cms(acc, make_float2(sm.dre[i][m], sm.dim[i][m]), v[m]);
        const float2 vi = cmulf(acc, crecip(make_float2(sm.dre[i][i], sm.dim[i][i])));
        v[i] = (i > c) ? make_float2(0.0f, 0.0f) : vi;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sm.vre[i][c] = v[i].x;
        sm.vim[i][c] = v[i].y;
      }
    }
    constexpr int WOFF = NM >= 64 ? 32 : 8;
    if ((NM == 8 && r < 8) || (NM > 8 && r >= WOFF && r < WOFF + 8)) {
      const int c = r & 7;
      float2 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float2 acc = make_float2(i == c ? 1.0f : 0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m < i; ++m) cms(acc, make_float2(sm.dre[i][m], sm.dim[i][m]), v[m]);
        v[i] = (i < c) ? make_float2(0.0f, 0.0f) : acc;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sm.wre[kb][i][c] = v[i].x;
        sm.wim[kb][i][c] = v[i].y;
      }
    }
    // lt L_bb = l (masked multipliers), from the last column to the first; block 0 then
    // holds n = -lt (rows chosen earlier keep their U entries and use n = 0)
    {
      float2 lt[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const bool use = !fin && (!pan || j < ii);
        lt[j] = use ? elem(ReP[0], ImP[0], j) : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int j = 6; j >= 0; --j)
#pragma unroll
        for (int m = j + 1; m < 8; ++m) cms(lt[j], lt[m], make_float2(sm.dre[m][j], sm.dim[m][j]));
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        ReP[0][m] = fin ? ReP[0][m] : pk(-lt[2 * m].x, -lt[2 * m + 1].x);
        ImP[0][m] = fin ? ImP[0][m] : pk(-lt[2 * m].y, -lt[2 * m + 1].y);
      }
    }
    gsync<NM>();  // V_b, W_b in place; dre/dim read by everyone
    if constexpr (NB > 1) {
      if (nact > 1) {
        // the panel's pivot rows publish their trailing blocks as they were before the panel
        if (pan) {
#pragma unroll
          for (int b = 1; b < NB; ++b) {
            if (b >= nact) break;
            ulonglong2* dr = reinterpret_cast<ulonglong2*>(&sm.tre[ii][8 * (b - 1)]);
            ulonglong2* di = reinterpret_cast<ulonglong2*>(&sm.tim[ii][8 * (b - 1)]);
            dr[0] = make_ulonglong2(ReP[b][0], ReP[b][1]);
            dr[1] = make_ulonglong2(ReP[b][2], ReP[b][3]);
            di[0] = make_ulonglong2(ImP[b][0], ImP[b][1]);
            di[1] = make_ulonglong2(ImP[b][2], ImP[b][3]);
          }
        }
        gsync<NM>();  // trailing blocks published
        // A_r,trail += n A_piv,trail (rows chosen earlier: n = 0)
#pragma unroll
        for (int b = 1; b < NB; ++b) {
          if (b >= nact) break;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float2 nj = fin ? make_float2(0.0f, 0.0f) : elem(ReP[0], ImP[0], j);
            const u64 NR = pk(nj.x, nj.x), NI = pk(nj.y, nj.y), NIn = pk(-nj.y, -nj.y);
            const ulonglong2 t0 = reinterpret_cast<const ulonglong2*>(&sm.tre[j][8 * (b - 1)])[0];
            const ulonglong2 t1 = reinterpret_cast<const ulonglong2*>(&sm.tre[j][8 * (b - 1)])[1];
            const ulonglong2 s0 = reinterpret_cast<const ulonglong2*>(&sm.tim[j][8 * (b - 1)])[0];
            const ulonglong2 s1 = reinterpret_cast<const ulonglong2*>(&sm.tim[j][8 * (b - 1)])[1];
            const u64 TR[4] = {t0.x, t0.y, t1.x, t1.y}, TI[4] = {s0.x, s0.y, s1.x, s1.y};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              ReP[b][m] = ffma2(NIn, TI[m], ffma2(NR, TR[m], ReP[b][m]));
              ImP[b][m] = ffma2(NI, TR[m], ffma2(NR, TI[m], ImP[b][m]));
            }
          }
        }
      }
    }
    // block 0 of this panel's pivot rows: V_b's row ii
    {
      const ulonglong2 v0 = reinterpret_cast<const ulonglong2*>(sm.vre[ii])[0];
      const ulonglong2 v1 = reinterpret_cast<const ulonglong2*>(sm.vre[ii])[1];
      const ulonglong2 u0 = reinterpret_cast<const ulonglong2*>(sm.vim[ii])[0];
      const ulonglong2 u1 = reinterpret_cast<const ulonglong2*>(sm.vim[ii])[1];
      const u64 VR[4] = {v0.x, v0.y, v1.x, v1.y}, VI[4] = {u0.x, u0.y, u1.x, u1.y};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        ReP[0][m] = pan ? VR[m] : ReP[0][m];
        ImP[0][m] = pan ? VI[m] : ImP[0][m];
      }
    }
    if constexpr (NB > 1) {
      // rotate: the finished panel goes to the end
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

  if constexpr (NM == 64 && KF) {
    // the factors of a problem that keeps them (forward only; rows coalesced per q)
    if (a.rhs_in == nullptr && a.fac != nullptr && in_range) {
      char* fb = static_cast<char*>(a.fac) + (size_t)sys * kFacStride;
      u64* fr = reinterpret_cast<u64*>(fb);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          fr[(size_t)(b * 4 + m) * NM + r] = ReP[b][m];
          fr[(size_t)(NB * 4 + b * 4 + m) * NM + r] = ImP[b][m];
        }
      reinterpret_cast<int32_t*>(fb + kFacRows)[r] = pivstep;
      float* fw = reinterpret_cast<float*>(fb + kFacRows + kFacPiv);
      for (int i = r; i < NB * 64; i += NM) {
        fw[i] = (&sm.wre[0][0][0])[i];
        fw[NB * 64 + i] = (&sm.wim[0][0][0])[i];
      }
    }
  }
  }  // need_lu

  const int Mb = pivstep >> 3, ii = pivstep & 7;

  // ---- the per-system values again (reloaded rather than kept through the LU) ----
  asm volatile("" ::: "memory");
  SysInfo si = sys_info(a, sys);
  const bool valid = in_range && si.N <= NM;  // larger systems: solve_large.cu
  if (!valid) si.N = 0;
  const int N = si.N;
  const double w = si.w;
  const float w32 = (float)w;
  const bool real_row = r < N;
  const bool bwd = a.rhs_in != nullptr;
  cd Dr = {0.0, 0.0};
  if (real_row) Dr = {a.R[si.k0 + r], -1.0 / (w * a.C[si.b * a.n_ports + si.k0 + r])};
  const int64_t mo = a.t.nn_off[si.s];
  const float* __restrict__ Mh = a.M32hi + mo;
  const float* __restrict__ Ml = a.M32lo + mo;

  // ---- solve A x = c with the blocked factors; returns the unknown of column pivstep ----
  auto lu_solve = [&](float2 c) -> float2 {
    float2 acc = c, yt = c;
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) {
      const int buf = kb & 1;
      if (Mb == kb) {
        sm.sre[buf][ii] = acc.x;
        sm.sim[buf][ii] = acc.y;
        yt = acc;
      }
      gsync<NM>();
      const float2 t = bdot(ReP[kb], ImP[kb], sm.sre[buf], sm.sim[buf]);
      acc.x += t.x;
      acc.y += t.y;
    }
    sm.yre[pivstep] = yt.x;
    sm.yim[pivstep] = yt.y;
    gsync<NM>();
    acc = bdot(reinterpret_cast<const u64*>(sm.wre[Mb][ii]), reinterpret_cast<const u64*>(sm.wim[Mb][ii]),
               &sm.yre[8 * Mb], &sm.yim[8 * Mb]);  // z = W yt (W rows via the same product)
    float2 x = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kb = NB - 1; kb >= 0; --kb) {
      if (Mb == kb) {
        sm.sre[0][ii] = acc.x;
        sm.sim[0][ii] = acc.y;
      }
      gsync<NM>();
      const float2 t = bdot(ReP[kb], ImP[kb], sm.sre[0], sm.sim[0]);
      if (Mb == kb) {
        x = t;
        sm.sre[1][ii] = t.x;
        sm.sim[1][ii] = t.y;
      }
      gsync<NM>();
      const float2 t2 = bdot(ReP[kb], ImP[kb], sm.sre[1], sm.sim[1]);
      acc.x -= t2.x;
      acc.y -= t2.y;
    }
    return x;
  };

  // solve, put the unknowns in column order (xc) and reduce max |re| + |im| over the
  // group in the same exchange
  auto solve_perm = [&](float2 c, float* dmax) -> float2 {
    const float2 x = lu_solve(c);
    sm.xc[pivstep] = x;
    float m = fabsf(x.x) + fabsf(x.y);
    if constexpr (NM >= 64) {
      unsigned u;
      asm volatile("redux.sync.max.u32 %0, %1, 0xffffffff;" : "=r"(u) : "r"(__float_as_uint(m)));
      if ((r & 31) == 0) sm.umax[r >> 5] = u;
      __syncthreads();
      unsigned best = sm.umax[0];
#pragma unroll
      for (int q = 1; q < SmemV4<NM>::NW; ++q) best = max(best, sm.umax[q]);
      m = __uint_as_float(best);
    } else {
      __syncwarp();
      for (int off = NM >> 1; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off, NM));
    }
    *dmax = m;
    return sm.xc[r];
  };

  // accurate residual of row r with the FP32 iterate in xc: rhs_r - sum_j A_rj x_j, the
  // sum over M_rj x_j in double-float (M = hi + lo exactly, x exact in FP32)
  auto residual = [&](cd rhs) -> cd {
    const float2 xr = sm.xc[r];
    if (!real_row) return {rhs.x - (double)xr.x, rhs.y - (double)xr.y};
    u64 S[2] = {0ull, 0ull}, Lo[2] = {0ull, 0ull};  // (re, im) high and low parts, 2 chains
    const u64 neg1 = pk(-1.0f, -1.0f);
    const u64* xv = reinterpret_cast<const u64*>(sm.xc);
    for (int j0 = 0; j0 < N; j0 += 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = j0 + h;
        if (j < N) {
          const float mh = __ldg(Mh + j * N + r), ml = __ldg(Ml + j * N + r);
          const u64 xj = xv[j];
          const u64 A = pk(mh, mh);
          const u64 pr = fmul2(A, xj);
          u64 e = ffma2(A, xj, fmul2(pr, neg1));
          e = ffma2(pk(ml, ml), xj, e);
          const u64 t = fadd2(S[h], pr);
          const u64 z = fsub2(t, S[h]);
          const u64 err = fadd2(fsub2(S[h], fsub2(t, z)), fsub2(pr, z));
          S[h] = t;
          Lo[h] = fadd2(Lo[h], fadd2(err, e));
        }
      }
    }
    const float2 s0 = up(S[0]), s1 = up(S[1]), l0 = up(Lo[0]), l1 = up(Lo[1]);
    const double Sr = ((double)s0.x + (double)l0.x) + ((double)s1.x + (double)l1.x);
    const double Si = ((double)s0.y + (double)l0.y) + ((double)s1.y + (double)l1.y);
    const double ax = Dr.x * (double)xr.x - Dr.y * (double)xr.y;
    const double ay = Dr.x * (double)xr.y + Dr.y * (double)xr.x;
    return {rhs.x - ax + w * Si, rhs.y - ay - w * Sr};
  };

  // r -= A d for the correction d in xc (FP32)
  auto residual_update = [&](cd res, float2 dr) -> cd {
    if (!real_row) return {res.x - dr.x, res.y - dr.y};
    u64 S0 = 0ull, S1 = 0ull;
    const u64* xv = reinterpret_cast<const u64*>(sm.xc);
    int j = 0;
    for (; j + 1 < N; j += 2) {
      const float m0 = __ldg(Mh + j * N + r), m1 = __ldg(Mh + (j + 1) * N + r);
      S0 = ffma2(pk(m0, m0), xv[j], S0);
      S1 = ffma2(pk(m1, m1), xv[j + 1], S1);
    }
    if (j < N) {
      const float m0 = __ldg(Mh + j * N + r);
      S0 = ffma2(pk(m0, m0), xv[j], S0);
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
    float dprev = 0.0f, xm0 = 0.0f;
    bool conv = max_it == 0;
#pragma unroll 1
    for (int it = 0;; ++it) {
      float dm;
      const float2 d = solve_perm(make_float2((float)res.x, (float)res.y), &dm);
      xk.x += (double)d.x;
      xk.y += (double)d.y;
      bool stop = it >= max_it;
      if (it == 0) {
        xm0 = dm;
      } else {
        const float est = dm * fminf(1.0f, dm / fmaxf(dprev, 1e-30f));
        conv = conv || (est <= tol * xm0);
        stop = stop || conv || !(dm <= 0.5f * dprev);
      }
      dprev = dm;
      if constexpr (NM <= 32) {
        if (__all_sync(0xffffffffu, stop)) break;
      } else {
        if (stop) break;
      }
      res = (it == 0) ? residual(rhs64) : residual_update(res, d);
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
        // objective at the loss points (FP32 sums of FP32 H rows, FP32 per-point terms)
        sm.xc[r] = make_float2((float)x.x, (float)x.y);
        gsync<NM>();
        const int L = a.loss_off[si.s + 1] - a.loss_off[si.s];
        const float* Hl = a.Hl32 + a.t.ln_off[si.s];
        const float* HlT = a.HlT32 + a.t.ln_off[si.s];  // [k][l]: lanes l read consecutively
        const int tw = a.loss_mode == 0 ? 1 : 2;
        const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                           (a.t.fl_off[si.s] + (int64_t)si.f * L) * tw;
        const int64_t wo = a.t.fl_off[si.s] + (int64_t)si.f * L;  // weight / offset base
        const u64* xv = reinterpret_cast<const u64*>(sm.xc);
        const u64* gv = reinterpret_cast<const u64*>(sm.Gs);
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
              b0 = ffma2(pk(h0, h0), xv[k], b0);
              b1 = ffma2(pk(h1, h1), xv[k + 1], b1);
            }
            if (k < N) {
              const float h0 = HlT[(int64_t)k * L + l];
              b0 = ffma2(pk(h0, h0), xv[k], b0);
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
              U = ffma2(pk(h, h), gv[q], U);
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

template <int NM, bool KF>
static cudaError_t launch_v4(const SolveArgs& a, int64_t n_sys, cudaStream_t st) {
  constexpr int CT = NM >= 64 ? NM : 128;
  constexpr int G = CT / NM;
  const size_t smem = sizeof(SmemV4<NM>) * G;
  cudaError_t e = cudaFuncSetAttribute(solve_mixed_v4<NM, KF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n_sys + G - 1) / G);
  solve_mixed_v4<NM, KF><<<grid, CT, smem, st>>>(a, n_sys);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const SolveArgs& a, int64_t n_sys, int max_ports, cudaStream_t st) {
  if (max_ports <= 8) return launch_v4<8, false>(a, n_sys, st);
  if (max_ports <= 16) return launch_v4<16, false>(a, n_sys, st);
  if (max_ports <= 32) return launch_v4<32, false>(a, n_sys, st);
  if (max_ports <= 64)
    return a.fac != nullptr ? launch_v4<64, true>(a, n_sys, st) : launch_v4<64, false>(a, n_sys, st);
  return cudaErrorNotSupported;
}

}  // namespace mts
