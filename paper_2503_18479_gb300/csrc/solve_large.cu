// solve_large.cu -- (b) port solve, (d) objective and (adj) adjoint for structures with more
// ports than the register-resident kernels hold (64 < N <= 1024).
//
// One system (configuration b, frequency g) per CTA of 128 (N <= 128), 256 (N <= 256) or 512
// threads. The matrix A = diag(R) + j w M + diag(1/(j w C)) (paper Eq. 2, 11) is assembled
// into the tape's factor scratch (global memory, L2-resident while in use; or shared memory,
// a schedule choice for FP32 classes of up to 128 ports) and factorised there by a blocked
// right-looking LU with partial pivoting, without moving rows (the pivot of column k is the
// largest |a_rk| among rows not chosen yet; chosen rows keep U in place, the others keep
// their multipliers):
//   panel   the NB columns [c0, c0+NB) of every row, staged column-major in shared memory,
//           factorised step by step (block arg-max per step, one barrier);
//   U12     the NB pivot rows of the panel over the trailing columns: a unit-lower
//           triangular solve against the panel's multipliers, a CW-column chunk at a time;
//   update  every row not chosen yet: A[r][j] -= sum_m L[r][m] U12[m][j]; FP32 register-
//           tiled (4 listed rows x 4 columns per thread), FP64 thread per column j with
//           U12[.][j] in registers.
// After the LU the NB x NB diagonal blocks are replaced by their inverses, and the
// triangular solves run block by block: warp 0 applies the block's inverse, then the other
// rows take the block's contribution (thread per row), with each step's entries copied a
// step ahead.
//
//   R = double: FP64 factors and one solve (MTS_FP64, NB = 8).
//   R = float : FP32 factors (NB = 16) and iterative refinement on residuals rhs - A x
//               taken in double-float on the FP32 pipe (M = hi + lo, x = hi + lo), stopped
//               by the same predictive estimate as the small systems. A, the pivot
//               magnitudes and the loss-point fields are FP32 too: this part's FP64 rate is
//               1/62 of FP32, and FP64 arithmetic there (an N^2 residual, per-step FP64
//               arg-max compares) outweighed the FP32 LU for N = 128.
// The objective at the loss points, the adjoint solve with the same matrix (A^T = A) and
// dloss/dC_k = Im(mu_k I_k)/(w C_k^2) (Eq. 8-9) are as in solve.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "solve_common.cuh"

namespace mts {

constexpr int kLargeMaxWarps = 16;  // CTAs of 128, 256 or 512 threads
// FP32 classes of up to this many ports keep the matrix in shared memory with CTAs of 256 or
// 512 threads (128 x 128 complex = 128 KB beside the 44 KB of panels and vectors): one CTA
// per SM, every access of the LU and the solves at shared-memory latency. With one system
// per SM instead of five, 14,206 systems of 128 ports took 32 ms against 17.5 ms in the
// scratch form, so the scratch form with 128 threads stays the default and the
// shared-resident one is a schedule choice that the autotuner times.
constexpr int kLargeSmemPorts = 128;

template <typename R>
struct Cx {
  R x, y;
};
template <typename R>
__device__ inline Cx<R> cx_div(Cx<R> a, Cx<R> b) {
  const R d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
// FP32 factors: a / b through the hardware approximate reciprocal of |b|^2 (<= 1 ulp; the
// rounding is removed by refinement), off the IEEE division's slow path
template <>
__device__ inline Cx<float> cx_div<float>(Cx<float> a, Cx<float> b) {
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(b.x * b.x + b.y * b.y));
  return {(a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv};
}
// v -= l * u
template <typename R>
__device__ inline void cx_fnma(Cx<R>& v, Cx<R> l, Cx<R> u) {
  v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
  v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
}

template <typename R>
struct LargeCfg;
template <>
struct LargeCfg<float> {
  static constexpr int NB = 16, CW = 128;
};
template <>
struct LargeCfg<double> {
  static constexpr int NB = 8, CW = 64;
};

struct BlockRed {
  double key[kLargeMaxWarps];  // block_max / block_sum
  int cnt;                     // rows in the active-row list of the trailing update
  // the pivot search's per-warp candidates, double-buffered by step parity (one barrier
  // per pivot step)
  double pkey[2][kLargeMaxWarps];
  float pkeyf[2][kLargeMaxWarps];
  int pidx[2][kLargeMaxWarps];
};

// Shared-memory carve-up for systems of up to n ports (host and device agree on it).
template <typename R>
struct LargeSmem {
  static constexpr int NB = LargeCfg<R>::NB, CW = LargeCfg<R>::CW;
  size_t pan, u12, wv, piv, ord, rhs, sv, xk, xc, red, pvec, amat, bytes;
  __host__ __device__ explicit LargeSmem(int n, bool sa = false) {
    const size_t cx = sizeof(Cx<R>);
    size_t o = 0;
    pan = o; o += cx * (size_t)NB * (n + 1);  // panel, column-major, pitch n + 1
    u12 = o; o += cx * (size_t)NB * CW;       // U12 chunk
    wv = o; o += cx * (size_t)n;              // triangular-solve vector (by row)
    piv = o; o += sizeof(int) * (size_t)n;    // step at which a row became the pivot
    ord = o; o += sizeof(int) * (size_t)n;    // pivot row of each step
    o = (o + 15) / 16 * 16;
    rhs = o; o += sizeof(cd) * (size_t)n;     // FP64 right-hand side / residual
    sv = o; o += sizeof(cd) * (size_t)n;      // FP64 saved right-hand side
    xk = o; o += sizeof(cd) * (size_t)n;      // FP64 iterate
    xc = o; o += sizeof(cd) * (size_t)n;      // FP64 currents I
    red = o; o += sizeof(BlockRed);
    o = (o + 15) / 16 * 16;
    pvec = o; o += cx * NB;                   // panel part of y or x
    o = (o + 15) / 16 * 16;
    amat = o;                                 // the matrix itself (shared-resident form)
    if (sa) o += cx * (size_t)n * n;
    bytes = o;
  }
};

// Pivot search across the CTA with one barrier: the warp winners go to buffer `buf` (step
// parity), so that a step's writes cannot overtake the previous step's reads; ties go to the
// smaller row. Every thread gets the row.
template <int W, typename K>
__device__ inline int pivot_argmax(K key, int idx, BlockRed* red, int buf) {
  if constexpr (sizeof(K) == 4) argmax_shfl(key, idx, 32);
  else argmax_shfl_d(key, idx, 32);
  if ((threadIdx.x & 31) == 0) {
    if constexpr (sizeof(K) == 4) red->pkeyf[buf][threadIdx.x >> 5] = key;
    else red->pkey[buf][threadIdx.x >> 5] = key;
    red->pidx[buf][threadIdx.x >> 5] = idx;
  }
  __syncthreads();
  K kb;
  if constexpr (sizeof(K) == 4) kb = red->pkeyf[buf][0];
  else kb = red->pkey[buf][0];
  int ib = red->pidx[buf][0];
#pragma unroll
  for (int q = 1; q < W; ++q) {
    K kq;
    if constexpr (sizeof(K) == 4) kq = red->pkeyf[buf][q];
    else kq = red->pkey[buf][q];
    const int iq = red->pidx[buf][q];
    if (kq > kb || (kq == kb && iq < ib)) {
      kb = kq;
      ib = iq;
    }
  }
  return ib;
}

// hi += a b exactly-split (FMA form of Dekker's TwoProd, Knuth's TwoSum) with the error in lo
__device__ inline void lg_df_acc(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  lo = __fadd_rn(lo, __fadd_rn(t, e));
  hi = s;
}

template <int W>
__device__ inline double block_max(double v, BlockRed* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red->key[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = red->key[0];
#pragma unroll
  for (int q = 1; q < W; ++q) m = fmax(m, red->key[q]);
  return m;
}

template <int W>
__device__ inline double block_sum(double v, BlockRed* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red->key[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < W; ++q) s += red->key[q];
  return s;
}

// T threads per CTA (one system): 128 for N <= 128, so that more systems share an SM, else 256.
// asynchronous copy of one matrix entry (8 or 16 bytes) from global to shared memory
template <typename R>
__device__ __forceinline__ void cp_async_elem(Cx<R>* dst, const Cx<R>* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(Cx<R>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// SA: the matrix lives in shared memory (FP32, up to kLargeSmemPorts ports) and goes to the
// factor scratch only as a copy for the backward; otherwise it stays in the scratch (L2).
template <typename R, int T, bool SA>
__global__ void __launch_bounds__(T, T == 128 ? 5 : (T == 256 ? 2 : 1)) solve_large_kernel(SolveArgs a, int64_t n_sys,
                                                                     int min_ports, int smem_n,
                                                                     Cx<R>* __restrict__ scratch) {
  constexpr int NB = LargeCfg<R>::NB, CW = LargeCfg<R>::CW;
  constexpr int W = T / 32;
  constexpr int RG = T / CW;  // row groups of the trailing update
  if ((int64_t)blockIdx.x >= n_sys) return;
  const int64_t sys = launch_sys(a, blockIdx.x);
  const SysInfo si = sys_info(a, sys);
  const int N = si.N;
  if (N <= min_ports) return;  // a register-resident kernel owns this system (CTA-uniform)

  extern __shared__ __align__(16) unsigned char dsm[];
  const LargeSmem<R> L(smem_n, SA);
  Cx<R>* pan = reinterpret_cast<Cx<R>*>(dsm + L.pan);
  Cx<R>* u12 = reinterpret_cast<Cx<R>*>(dsm + L.u12);
  Cx<R>* wv = reinterpret_cast<Cx<R>*>(dsm + L.wv);
  int* pivstep = reinterpret_cast<int*>(dsm + L.piv);
  int* order = reinterpret_cast<int*>(dsm + L.ord);
  cd* rhs = reinterpret_cast<cd*>(dsm + L.rhs);
  cd* sv = reinterpret_cast<cd*>(dsm + L.sv);
  cd* xk = reinterpret_cast<cd*>(dsm + L.xk);
  cd* xc = reinterpret_cast<cd*>(dsm + L.xc);
  BlockRed* red = reinterpret_cast<BlockRed*>(dsm + L.red);
  Cx<R>* pvec = reinterpret_cast<Cx<R>*>(dsm + L.pvec);
  // float2 hi / lo split of an FP64 vector for the double-float residual and the FP32
  // objective; they reuse the triangular-solve vector (n elements of at least 8 bytes) and
  // the U12 chunk (NB x CW >= n elements), both idle outside the LU and the solves
  float2* xh = reinterpret_cast<float2*>(dsm + L.wv);
  float2* xl = reinterpret_cast<float2*>(dsm + L.u12);
  constexpr bool kF = sizeof(R) == 4;  // FP32 factors: no FP64 on the per-element paths
  const int NP = N + 1;  // panel pitch

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double w = si.w;
  const bool bwd = a.rhs_in != nullptr;
  const double* __restrict__ M = a.M64 + a.t.nn_off[si.s];
  const double* __restrict__ Cb = a.C + si.b * a.n_ports + si.k0;
  const double* __restrict__ Rk = a.R + si.k0;
  const int F = a.freq_off[si.s + 1] - a.freq_off[si.s];
  Cx<R>* const Ag = scratch + si.b * a.lu_off[a.n_struct] + a.lu_off[si.s] + (int64_t)si.f * N * N;
  Cx<R>* const A = SA ? reinterpret_cast<Cx<R>*>(dsm + L.amat) : Ag;

  const int64_t ioff = si.b * a.sumFN + a.t.fn_off[si.s] + (int64_t)si.f * N;
  // A backward call reuses the factors and the pivot order the forward left in the tape
  // (the order is checked to be a permutation; otherwise A is assembled and factored again).
  bool need_lu = true;
  if (bwd && a.lu_order != nullptr) {
    for (int r = tid; r < N; r += T) pivstep[r] = N;
    __syncthreads();
    int bad = 0;
    for (int k = tid; k < N; k += T) {
      const int p = a.lu_order[ioff + k];
      if ((unsigned)p < (unsigned)N) {
        order[k] = p;
        pivstep[p] = k;
      } else {
        bad = 1;
      }
    }
    __syncthreads();
    for (int r = tid; r < N; r += T) bad |= pivstep[r] == N;
    need_lu = __syncthreads_or(bad) != 0;
  }
  if (need_lu) {
    // ---- assemble A (Eq. 2, 11), four independent loads of M in flight per thread ----
    const int NN = N * N;
    if constexpr (kF) {
      // off-diagonal (and the diagonal's placeholder) in FP32 from the FP32 part of M
      const float w32 = (float)w;
      const float* __restrict__ M32 = a.M32hi + a.t.nn_off[si.s];
      for (int e0 = 0; e0 < NN; e0 += 4 * T) {
        float mv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = e0 + q * T + tid;
          mv[q] = e < NN ? M32[e] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = e0 + q * T + tid;
          if (e < NN) A[e] = {(R)0, (R)(w32 * mv[q])};
        }
      }
      __syncthreads();
      // the diagonal once per row in FP64: R_r + j (w M_rr - 1/(w C_r))
      for (int r = tid; r < N; r += T)
        A[(int64_t)r * N + r] = {(R)Rk[r], (R)(w * M[(int64_t)r * N + r] - 1.0 / (w * Cb[r]))};
    } else
    for (int e0 = 0; e0 < NN; e0 += 4 * T) {
      double mv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + q * T + tid;
        mv[q] = e < NN ? M[e] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + q * T + tid;
        if (e < NN) {
          const int r = e / N, j = e - r * N;
          double im = w * mv[q], re = 0.0;
          if (j == r) {
            re = Rk[r];
            im -= 1.0 / (w * Cb[r]);
          }
          A[e] = {(R)re, (R)im};
        }
      }
    }
    for (int r = tid; r < N; r += T) pivstep[r] = N;
    __syncthreads();

    // ---- blocked LU with partial pivoting ----
    for (int c0 = 0; c0 < N; c0 += NB) {
      const int nb = min(NB, N - c0);
      // eight independent loads in flight per thread (the matrix may be in the scratch)
      for (int e0 = 0; e0 < N * NB; e0 += 8 * T) {
        Cx<R> v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = e0 + q * T + tid;
          const int r = e / NB, j = e - r * NB;
          v[q] = {0, 0};
          if (e < N * NB && j < nb && pivstep[r] == N) v[q] = A[(int64_t)r * N + c0 + j];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = e0 + q * T + tid;
          const int r = e / NB, j = e - r * NB;
          if (e < N * NB) pan[j * NP + r] = v[q];
        }
      }
      __syncthreads();
      // pivot steps with one barrier each: a thread reads and writes only its own rows of the
      // panel and their pivot steps, except the pivot row's entries, which its owner last
      // wrote before the barrier of this step's search
      for (int kk = 0; kk < nb; ++kk) {
        int p;
        if constexpr (kF) {
          float best = -1.0f;
          int bi = N;
          for (int r = tid; r < N; r += T)
            if (pivstep[r] == N) {
              const Cx<R> v = pan[kk * NP + r];
              float m = v.x * v.x + v.y * v.y;
              if (!(m >= 0.0f)) m = 0.0f;  // NaN: still a candidate, so a row is always chosen
              if (m > best) {
                best = m;
                bi = r;
              }
            }
          p = pivot_argmax<W>(best, bi, red, kk & 1);
        } else {
          double best = -1.0;
          int bi = N;
          for (int r = tid; r < N; r += T)
            if (pivstep[r] == N) {
              const Cx<R> v = pan[kk * NP + r];
              double m = (double)v.x * v.x + (double)v.y * v.y;
              if (!(m >= 0.0)) m = 0.0;  // NaN: still a candidate, so a row is always chosen
              if (m > best) {
                best = m;
                bi = r;
              }
            }
          p = pivot_argmax<W>(best, bi, red, kk & 1);
        }
        const Cx<R> piv = pan[kk * NP + p];
        for (int r = tid; r < N; r += T)
          if (pivstep[r] == N) {
            if (r == p) {
              pivstep[r] = c0 + kk;
            } else {
              const Cx<R> l = cx_div(pan[kk * NP + r], piv);
              pan[kk * NP + r] = l;
              for (int j = kk + 1; j < nb; ++j) cx_fnma(pan[j * NP + r], l, pan[j * NP + p]);
            }
          }
        if (tid == 0) order[c0 + kk] = p;
      }
      __syncthreads();  // every row's panel entries and pivot step in place
      // panel back to the matrix (rows chosen in this panel or later)
      for (int e = tid; e < N * NB; e += T) {
        const int r = e / NB, j = e - r * NB;
        if (j < nb && pivstep[r] >= c0) A[(int64_t)r * N + c0 + j] = pan[j * NP + r];
      }
      __syncthreads();
      // FP32: the rows still to be updated (not chosen as pivots yet), listed once per panel
      // in the triangular-solve vector (idle during the LU); warp-aggregated, so the order of
      // the list varies but every row's update is the same
      int nact = 0;
      int* alist = reinterpret_cast<int*>(wv);
      if constexpr (kF) {
        if (c0 + nb < N) {
          if (tid == 0) red->cnt = 0;
          __syncthreads();
          for (int rb = warp * 32; rb < N; rb += T) {
            const int r = rb + lane;
            const bool act = r < N && pivstep[r] == N;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&red->cnt, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (act) alist[base + __popc(bal & ((1u << lane) - 1u))] = r;
          }
          __syncthreads();
          nact = red->cnt;
        }
      }
      // trailing columns, CW at a time
      for (int j0 = c0 + nb; j0 < N; j0 += CW) {
        if (tid < CW) {
          const int j = j0 + tid;
          if (j < N) {  // columns past N skip the unrolled work as a whole
            // the nb entries of the pivot rows first (independent loads), then the unit
            // lower solve L_bb u = a in place
            Cx<R> uu[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
              uu[i] = {0, 0};
              if (i < nb) uu[i] = A[(int64_t)order[c0 + i] * N + j];
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
              if (i < nb) {
                const int pi = order[c0 + i];
#pragma unroll
                for (int m = 0; m < i; ++m) cx_fnma(uu[i], pan[m * NP + pi], uu[m]);
                A[(int64_t)pi * N + j] = uu[i];
              }
              u12[i * CW + tid] = uu[i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < NB; ++i) u12[i * CW + tid] = Cx<R>{0, 0};
          }
        }
        __syncthreads();
        if constexpr (kF) {
          // register-tiled update: a thread takes 4 listed rows x 4 columns (j0 + lane + 32 cc,
          // so that a warp's loads of one (row, cc) are 256 contiguous bytes: conflict-free in
          // shared memory, coalesced in the scratch),
          // the (re, im) pairs of a tile in packed registers; per panel column m, with the
          // multiplier l = (a, b) and the U12 entry u = (c, d):
          //   v -= l u  <=>  (v.re, v.im) += (b, b) (d, -c) + (-a, -a) (c, d)
          // two fma.rn.f32x2 per complex multiply-add, 8 shared loads per 16 of them
          const int jc = j0 + lane;  // the warp covers the chunk's 128 columns
          const int ntile = (nact + 3) >> 2;
          for (int t4 = warp; t4 < ntile; t4 += W) {
            int rw[4];
            bool okr[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              okr[rr] = 4 * t4 + rr < nact;
              rw[rr] = alist[okr[rr] ? 4 * t4 + rr : 0];
            }
            unsigned long long V[4][4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) {
                const int j = jc + 32 * cc;
                V[rr][cc] = (okr[rr] && j < N)
                                ? *reinterpret_cast<const unsigned long long*>(A + (int64_t)rw[rr] * N + j)
                                : 0ull;
              }
#pragma unroll 2
            for (int m = 0; m < NB; ++m) {
              unsigned long long LA[4], LB[4], P1[4], P2[4];
#pragma unroll
              for (int rr = 0; rr < 4; ++rr) {
                const Cx<R> l = pan[m * NP + rw[rr]];
                asm("mov.b64 %0, {%1,%1};" : "=l"(LA[rr]) : "f"(-l.x));
                asm("mov.b64 %0, {%1,%1};" : "=l"(LB[rr]) : "f"(l.y));
              }
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) {
                const Cx<R> u = u12[m * CW + lane + 32 * cc];
                asm("mov.b64 %0, {%1,%2};" : "=l"(P1[cc]) : "f"(u.x), "f"(u.y));
                asm("mov.b64 %0, {%1,%2};" : "=l"(P2[cc]) : "f"(u.y), "f"(-u.x));
              }
#pragma unroll
              for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                  // the order of cx_fnma (b d first): the same roundings as the per-column form
                  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(V[rr][cc]) : "l"(LB[rr]), "l"(P2[cc]));
                  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(V[rr][cc]) : "l"(LA[rr]), "l"(P1[cc]));
                }
            }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) {
                const int j = jc + 32 * cc;
                if (okr[rr] && j < N)
                  *reinterpret_cast<unsigned long long*>(A + (int64_t)rw[rr] * N + j) = V[rr][cc];
              }
          }
        } else {
          {
            const int col = tid % CW, rg = tid / CW;
            const int j = j0 + col;
            Cx<R> uu[NB];
  #pragma unroll
            for (int m = 0; m < NB; ++m) uu[m] = u12[m * CW + col];
            if (j < N) {
              constexpr int RF = 8;  // rows in flight: independent loads per thread
              int r = rg;
              for (; r + (RF - 1) * RG < N; r += RF * RG) {
                bool act[RF];
                Cx<R> v[RF];
  #pragma unroll
                for (int q = 0; q < RF; ++q) {
                  act[q] = pivstep[r + q * RG] == N;
                  v[q] = act[q] ? A[(int64_t)(r + q * RG) * N + j] : Cx<R>{0, 0};
                }
  #pragma unroll
                for (int q = 0; q < RF; ++q)
                  if (act[q]) {
  #pragma unroll
                    for (int m = 0; m < NB; ++m) cx_fnma(v[q], pan[m * NP + r + q * RG], uu[m]);
                    A[(int64_t)(r + q * RG) * N + j] = v[q];
                  }
              }
              for (; r < N; r += RG)
                if (pivstep[r] == N) {
                  Cx<R> v = A[(int64_t)r * N + j];
  #pragma unroll
                  for (int m = 0; m < NB; ++m) cx_fnma(v, pan[m * NP + r], uu[m]);
                  A[(int64_t)r * N + j] = v;
                }
            }
          }
        }
        __syncthreads();
      }
    }
    // ---- the diagonal blocks in place by their inverses: W_b = L_bb^-1 (unit lower, below
    // the diagonal) and V_b = U_bb^-1 (upper, diagonal included), so that the triangular
    // solves apply each block as one product instead of a 16-step substitution chain. A
    // warp stages its block (rows in pivot order) in the panel's shared memory, free after
    // the LU; lane c forms column c of both inverses. ----
    {
      Cx<R>* blk = pan + (int64_t)warp * NB * NB;  // [NB][NB], row i = pivot row order[c0 + i]
      const int wi_n = min(W, NP / NB);             // warps whose slice fits the panel region
      if (warp < wi_n) {
        for (int c0 = warp * NB; c0 < N; c0 += wi_n * NB) {
          const int nb = min(NB, N - c0);
          for (int e = lane; e < NB * NB; e += 32) {
            const int i = e / NB, m = e - i * NB;
            blk[e] = (i < nb && m < nb) ? A[(int64_t)order[c0 + i] * N + c0 + m] : Cx<R>{0, 0};
          }
          __syncwarp();
          if (lane < nb) {
            const int c = lane;
            Cx<R> w[NB], v[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {  // W column c: w_c = 1, w_i = -sum_{m<i} L_im w_m
              Cx<R> acc = {(R)(i == c ? 1 : 0), (R)0};
#pragma unroll
              for (int m = 0; m < i; ++m)
                if (m >= c) cx_fnma(acc, blk[i * NB + m], w[m]);
              w[i] = (i >= c && i < nb) ? acc : Cx<R>{0, 0};
            }
#pragma unroll
            for (int i = NB - 1; i >= 0; --i) {  // V column c: U v = e_c, rows c .. 0
              Cx<R> acc = {(R)(i == c ? 1 : 0), (R)0};
#pragma unroll
              for (int m = i + 1; m < NB; ++m)
                if (m <= c) cx_fnma(acc, blk[i * NB + m], v[m]);
              v[i] = (i <= c) ? cx_div(acc, blk[i * NB + i]) : Cx<R>{0, 0};
            }
#pragma unroll
            for (int i = 0; i < NB; ++i)
              if (i < nb) A[(int64_t)order[c0 + i] * N + c0 + c] = (i > c) ? w[i] : v[i];
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }
    if (!bwd && a.lu_order != nullptr)
      for (int k = tid; k < N; k += T) a.lu_order[ioff + k] = order[k];
  }  // need_lu
  if constexpr (SA) {
    // the factors between the forward and a backward that reuses them: 8-byte units (the
    // scratch base of a system is 8-byte aligned), eight loads in flight per thread
    using U8 = unsigned long long;
    const int NN = N * N;
    U8* sA = reinterpret_cast<U8*>(A);
    U8* gA = reinterpret_cast<U8*>(Ag);
    if (!need_lu || (!bwd && a.lu_order != nullptr)) {
      U8* dst = need_lu ? gA : sA;
      const U8* src = need_lu ? sA : gA;
      for (int e0 = 0; e0 < NN; e0 += 8 * T) {
        U8 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = e0 + q * T + tid;
          v[q] = e < NN ? src[e] : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = e0 + q * T + tid;
          if (e < NN) dst[e] = v[q];
        }
      }
      __syncthreads();
    }
  }

  // ---- solve A x = rhs (FP64 rhs in shared memory) into wv (by row) with the factors;
  // the unknown of column k ends in wv[order[k]]. With the factors in the scratch, each
  // step's entries are copied one step ahead (cp.async) into shared memory that is idle
  // during the solves: the blocks of the thread's rows that the row update needs (in the
  // panel region, element m of row r at m N + r) and warp 0's rows of the diagonal block (in
  // the U12 region), so that their latency overlaps the barrier and the diagonal block's
  // products. A thread reads only what it copied. ----
  Cx<R>* const stg = pan;  // [NB][N]
  Cx<R>* const dstg = u12;  // [NB][32]
  auto lu_solve = [&]() {
    for (int r = tid; r < N; r += T) wv[r] = {(R)rhs[r].x, (R)rhs[r].y};
    const int last = (N - 1) / NB * NB;
    // step (c0, forward or back): rows that take the step's update, and the diagonal rows
    auto fetch = [&](int c0, bool fwd) {
      if constexpr (!SA) {
        const int nb = min(NB, N - c0);
        for (int r = tid; r < N; r += T)
          if (fwd ? pivstep[r] >= c0 + nb : pivstep[r] < c0) {
#pragma unroll
            for (int m = 0; m < NB; ++m)
              if (m < nb) cp_async_elem(stg + m * N + r, A + (int64_t)r * N + c0 + m);
          }
        if (warp == 0 && lane < nb) {
          const int pi = order[c0 + lane];
#pragma unroll
          for (int m = 0; m < NB; ++m)  // W_b row (forward), V_b row (back)
            if (fwd ? m < lane : (m >= lane && m < nb))
              cp_async_elem(dstg + m * 32 + lane, A + (int64_t)pi * N + c0 + m);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
    };
    // entry m of the staged block of row r / of this lane's diagonal row (the matrix itself
    // when it is in shared memory)
    auto row_elem = [&](int r, int c0, int m) -> Cx<R> {
      if constexpr (SA) return A[(int64_t)r * N + c0 + m];
      else return stg[m * N + r];
    };
    auto diag_elem = [&](int c0, int pi, int m) -> Cx<R> {
      if constexpr (SA) return A[(int64_t)pi * N + c0 + m];
      else return dstg[m * 32 + lane];
    };
    fetch(0, true);
    __syncthreads();
    for (int c0 = 0; c0 < N; c0 += NB) {  // forward: L y = P rhs
      const int nb = min(NB, N - c0);
      if (warp == 0) {
        Cx<R> wi = {0, 0};
        int pi = 0;
        if (lane < nb) {
          pi = order[c0 + lane];
          wi = wv[pi];
        }
        if constexpr (!SA) asm volatile("cp.async.wait_all;" ::: "memory");
        // y_b = W_b w_b (unit diagonal): products of the block's original values
        const Cx<R> w0 = wi;
#pragma unroll
        for (int m = 0; m < NB; ++m) {
          const Cx<R> wm = {__shfl_sync(0xffffffffu, w0.x, m), __shfl_sync(0xffffffffu, w0.y, m)};
          if (lane > m && lane < nb) {  // wi += W_im w_m
            const Cx<R> l = diag_elem(c0, pi, m);
            wi.x = fma(l.x, wm.x, fma(-l.y, wm.y, wi.x));
            wi.y = fma(l.x, wm.y, fma(l.y, wm.x, wi.y));
          }
        }
        if (lane < NB) pvec[lane] = lane < nb ? wi : Cx<R>{0, 0};
        if (lane < nb) wv[pi] = wi;
      }
      __syncthreads();
      if constexpr (!SA) asm volatile("cp.async.wait_all;" ::: "memory");
      for (int r = tid; r < N; r += T)
        if (pivstep[r] >= c0 + nb) {
          Cx<R> v = wv[r];
#pragma unroll
          for (int m = 0; m < NB; ++m)
            if (m < nb) cx_fnma(v, row_elem(r, c0, m), pvec[m]);
          wv[r] = v;
        }
      if (c0 + NB < N) fetch(c0 + NB, true);
      else fetch(last, false);
      __syncthreads();
    }
    for (int c0 = last; c0 >= 0; c0 -= NB) {  // back: U x = y
      const int nb = min(NB, N - c0);
      if (warp == 0) {
        Cx<R> wi = {0, 0};
        int pi = 0;
        if (lane < nb) {
          pi = order[c0 + lane];
          wi = wv[pi];
        }
        if constexpr (!SA) asm volatile("cp.async.wait_all;" ::: "memory");
        // x_b = V_b y_b: products of the block's values
        const Cx<R> y0 = wi;
        wi = {0, 0};
#pragma unroll
        for (int m = 0; m < NB; ++m) {
          const Cx<R> ym = {__shfl_sync(0xffffffffu, y0.x, m), __shfl_sync(0xffffffffu, y0.y, m)};
          if (m >= lane && m < nb && lane < nb) {  // wi += V_im y_m
            const Cx<R> u = diag_elem(c0, pi, m);
            wi.x = fma(u.x, ym.x, fma(-u.y, ym.y, wi.x));
            wi.y = fma(u.x, ym.y, fma(u.y, ym.x, wi.y));
          }
        }
        if (lane < NB) pvec[lane] = lane < nb ? wi : Cx<R>{0, 0};
        if (lane < nb) wv[pi] = wi;
      }
      __syncthreads();
      if constexpr (!SA) asm volatile("cp.async.wait_all;" ::: "memory");
      for (int r = tid; r < N; r += T)
        if (pivstep[r] < c0) {
          Cx<R> v = wv[r];
#pragma unroll
          for (int m = 0; m < NB; ++m)
            if (m < nb) cx_fnma(v, row_elem(r, c0, m), pvec[m]);
          wv[r] = v;
        }
      if (c0 > 0) fetch(c0 - NB, false);
      __syncthreads();
    }
  };

  // refined solve of A x = rhs into xk (rhs is kept); returns whether it converged
  auto refined = [&]() -> bool {
    for (int r = tid; r < N; r += T) sv[r] = rhs[r];
    lu_solve();
    double xm = 0.0;
    for (int k = tid; k < N; k += T) {
      const Cx<R> v = wv[order[k]];
      xk[k] = {(double)v.x, (double)v.y};
      xm = fmax(xm, fabs((double)v.x) + fabs((double)v.y));
    }
    bool conv = true;
    if (sizeof(R) < 8) {
      double dprev = block_max<W>(xm, red);  // its barriers also publish xk
      conv = a.max_refine == 0;
      const float* __restrict__ Mh = a.M32hi + a.t.nn_off[si.s];
      const float* __restrict__ Ml = a.M32lo + a.t.nn_off[si.s];
      for (int it = 0; it < a.max_refine; ++it) {
        for (int k = tid; k < N; k += T) {  // x = hi + lo
          const float hx = (float)xk[k].x, hy = (float)xk[k].y;
          xh[k] = make_float2(hx, hy);
          xl[k] = make_float2((float)(xk[k].x - (double)hx), (float)(xk[k].y - (double)hy));
        }
        __syncthreads();
        for (int r = tid; r < N; r += T) {  // residual sv - A xk, M x in double-float
          float shx = 0.f, slx = 0.f, shy = 0.f, sly = 0.f;
#pragma unroll 4
          for (int j = 0; j < N; ++j) {
            const float mh = Mh[(int64_t)j * N + r], ml = Ml[(int64_t)j * N + r];  // column r
            const float2 ph = xh[j], pl = xl[j];
            lg_df_acc(shx, slx, mh, ph.x);
            lg_df_acc(shy, sly, mh, ph.y);
            slx = fmaf(mh, pl.x, fmaf(ml, ph.x, slx));
            sly = fmaf(mh, pl.y, fmaf(ml, ph.y, sly));
          }
          const double sx = (double)shx + (double)slx, sy = (double)shy + (double)sly;
          const double dx = Rk[r], dy = -1.0 / (w * Cb[r]);
          const double ax = dx * xk[r].x - dy * xk[r].y - w * sy;
          const double ay = dx * xk[r].y + dy * xk[r].x + w * sx;
          rhs[r] = {sv[r].x - ax, sv[r].y - ay};
        }
        __syncthreads();
        lu_solve();
        double dm = 0.0, xm2 = 0.0;
        for (int k = tid; k < N; k += T) {
          const Cx<R> d = wv[order[k]];
          xk[k].x += (double)d.x;
          xk[k].y += (double)d.y;
          dm = fmax(dm, fabs((double)d.x) + fabs((double)d.y));
          xm2 = fmax(xm2, fabs(xk[k].x) + fabs(xk[k].y));
        }
        dm = block_max<W>(dm, red);
        xm2 = block_max<W>(xm2, red);
        const double est = dm * fmin(1.0, dm / fmax(dprev, 1e-300));
        conv = conv || est <= a.tol * xm2;
        const bool stop = conv || !(dm <= 0.5 * dprev);
        dprev = dm;
        if (stop) break;
      }
      for (int r = tid; r < N; r += T) rhs[r] = sv[r];
    }
    __syncthreads();
    return conv;
  };

  bool conv_all = true;
  if (!bwd) {
    for (int r = tid; r < N; r += T) {
      const double* Vp = a.V + 2 * (a.t.fn_off[si.s] + (int64_t)si.f * N + r);
      rhs[r] = {Vp[0], Vp[1]};
    }
    __syncthreads();
    conv_all = refined();
    for (int r = tid; r < N; r += T) {
      xc[r] = xk[r];
      a.I[2 * (ioff + r)] = xk[r].x;
      a.I[2 * (ioff + r) + 1] = xk[r].y;
      if (a.I_out) {
        a.I_out[2 * (ioff + r)] = xk[r].x;
        a.I_out[2 * (ioff + r) + 1] = xk[r].y;
      }
    }
    if (a.Bop != nullptr && a.bop_off[si.s + 1] > a.bop_off[si.s]) {  // tensor-core structure
      // tensor-core operand pieces of I: rows 2 (b F_s + f) + {0: re, 1: im}, columns
      // N .. K_pad-1 zero; x = xh + xl, pieces bf16(rem), rem -= piece in FP32
      const int nkc = (N + kChunkK - 1) / kChunkK;
      const int64_t ntile = (2 * a.n_cfg * F + kTileN - 1) / kTileN;
      char* base = reinterpret_cast<char*>(a.Bop + a.bop_off[si.s]);
      const size_t tile_bytes = (size_t)kTileN * kChunkK * 2;
      for (int kg = tid; kg < nkc * kChunkK; kg += T) {
        const int kc = kg / kChunkK, kk = kg % kChunkK;
        for (int c = 0; c < 2; ++c) {
          const int64_t n = 2 * (si.b * F + si.f) + c;
          const int64_t tile = n / kTileN;
          const uint32_t rr = (uint32_t)(n % kTileN);
          const double xv = kg < N ? (c == 0 ? xk[kg].x : xk[kg].y) : 0.0;
          const float xh = (float)xv, xl = (float)(xv - (double)xh);
          float rem = xh;
          for (int q = 0; q < a.npieces; ++q) {
            const __nv_bfloat16 h = __float2bfloat16_rn(rem);
            rem = rem - __bfloat162float(h);
            if (q == 0) rem += xl;
            const size_t off = ((size_t)(q * ntile + tile) * nkc + kc) * tile_bytes + swz128(rr, kk);
            *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
          }
        }
      }
    }
  } else {
    for (int r = tid; r < N; r += T) xc[r] = {a.I[2 * (ioff + r)], a.I[2 * (ioff + r) + 1]};
  }
  __syncthreads();

  // ---- objective at the loss points and the adjoint right-hand side u = H_loss^T conj(G) ----
  const bool has_obj = !bwd && a.target != nullptr;
  if (has_obj || bwd) {
    if (has_obj) {
      const int Ls = a.loss_off[si.s + 1] - a.loss_off[si.s];
      const double* __restrict__ Hl = a.Hl64 + a.t.ln_off[si.s];
      const int tw = a.loss_mode == 0 ? 1 : 2;
      const double* tb = a.target + (a.target_per_cfg ? si.b * a.sumFL * tw : 0) +
                         (a.t.fl_off[si.s] + (int64_t)si.f * Ls) * tw;
      const int64_t wo = a.t.fl_off[si.s] + (int64_t)si.f * Ls;  // weight / offset base
      cd* Gs = reinterpret_cast<cd*>(dsm + L.pan);  // the panel is free after the LU
      float2* Gh = reinterpret_cast<float2*>(dsm + L.pan);  // conj(G) = hi + lo (FP32)
      float2* Glo = Gh + T;
      const float* __restrict__ Hl32 = a.Hl32 + a.t.ln_off[si.s];
      const float* __restrict__ HlT32 = a.HlT32 + a.t.ln_off[si.s];  // [k][l]
      double lsum = 0.0;
      for (int r = tid; r < N; r += T) rhs[r] = {0.0, 0.0};
      if constexpr (kF) {  // currents as hi + lo floats for the double-float sums below
        for (int k = tid; k < N; k += T) {
          const float hx = (float)xc[k].x, hy = (float)xc[k].y;
          xh[k] = make_float2(hx, hy);
          xl[k] = make_float2((float)(xc[k].x - (double)hx), (float)(xc[k].y - (double)hy));
        }
        __syncthreads();
      }
      for (int c0 = 0; c0 < Ls; c0 += T) {
        const int l = c0 + tid;
        cd Gl = {0.0, 0.0};
        if (l < Ls) {
          double bx = 0.0, by = 0.0;
          if constexpr (kF) {
            // FP32 rows (the basis is FP32), double-float sums: N terms with cancellation
            // (sum |H x| / |b| reaches ~100 at N = 1024) need more than FP32 accumulation
            float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll 4
            for (int k = 0; k < N; ++k) {
              const float h = HlT32[(int64_t)k * Ls + l];  // lanes l read consecutively
              lg_df_acc(hx, lx, h, xh[k].x);
              lg_df_acc(hy, ly, h, xh[k].y);
              lx = fmaf(h, xl[k].x, lx);
              ly = fmaf(h, xl[k].y, ly);
            }
            bx = (double)hx + (double)lx;
            by = (double)hy + (double)ly;
          } else {
#pragma unroll 8
            for (int k = 0; k < N; ++k) {
              const double h = Hl[(int64_t)l * N + k];
              bx = fma(h, xc[k].x, bx);
              by = fma(h, xc[k].y, by);
            }
          }
          double wl = 1.0;
          if (a.loss_offset) {
            bx += a.loss_offset[2 * (wo + l)];
            by += a.loss_offset[2 * (wo + l) + 1];
          }
          if (a.loss_weight) {
            wl = a.loss_weight[wo + l];
            bx *= wl;
            by *= wl;
          }
          lsum += point_loss(a.loss_mode, cd{bx, by}, tb + (int64_t)l * tw, &Gl);
          Gl.x *= wl;
          Gl.y *= wl;
        }
        if constexpr (kF) {  // conj(G)
          const float gx = (float)Gl.x, gy = (float)(-Gl.y);
          Gh[tid] = make_float2(gx, gy);
          Glo[tid] = make_float2((float)(Gl.x - (double)gx), (float)(-Gl.y - (double)gy));
        } else {
          Gs[tid] = {Gl.x, -Gl.y};
        }
        __syncthreads();
        const int lc = min(T, Ls - c0);
        for (int r = tid; r < N; r += T) {
          if constexpr (kF) {
            float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
#pragma unroll 4
            for (int q = 0; q < lc; ++q) {
              const float h = Hl32[(int64_t)(c0 + q) * N + r];
              lg_df_acc(hx, lx, h, Gh[q].x);
              lg_df_acc(hy, ly, h, Gh[q].y);
              lx = fmaf(h, Glo[q].x, lx);
              ly = fmaf(h, Glo[q].y, ly);
            }
            rhs[r] = {rhs[r].x + ((double)hx + (double)lx), rhs[r].y + ((double)hy + (double)ly)};
          } else {
            double ux = rhs[r].x, uy = rhs[r].y;
#pragma unroll 8
            for (int q = 0; q < lc; ++q) {
              const double h = Hl[(int64_t)(c0 + q) * N + r];
              ux = fma(h, Gs[q].x, ux);
              uy = fma(h, Gs[q].y, uy);
            }
            rhs[r] = {ux, uy};
          }
        }
        __syncthreads();
      }
      const double tot = block_sum<W>(lsum, red);
      if (tid == 0) a.loss_part[sys] = tot;
    } else {
      for (int r = tid; r < N; r += T)
        rhs[r] = {a.rhs_in[2 * (ioff + r)], a.rhs_in[2 * (ioff + r) + 1]};
    }
    __syncthreads();
    conv_all = refined() && conv_all;
    for (int r = tid; r < N; r += T) {
      const cd mu = xk[r], x = xc[r];
      a.grad_part[ioff + r] = (mu.x * x.y + mu.y * x.x) / (w * Cb[r] * Cb[r]);
      if (!bwd && a.mu_out) {
        a.mu_out[2 * (ioff + r)] = mu.x;
        a.mu_out[2 * (ioff + r) + 1] = mu.y;
      }
    }
  }
  double bad = 0.0;
  for (int r = tid; r < N; r += T)
    if (!(isfinite(xc[r].x) && isfinite(xc[r].y) && isfinite(xk[r].x) && isfinite(xk[r].y)))
      bad = 1.0;
  bad = block_max<W>(bad, red);
  if (tid == 0 && !bwd) a.status[sys] = bad > 0.0 ? 2 : (conv_all ? 0 : 1);
}

// CTA size for a class whose largest system has max_ports ports
static int large_threads(int max_ports) { return max_ports <= 128 ? 128 : (max_ports <= 256 ? 256 : 512); }

// the shared-resident form: FP32, a class of up to kLargeSmemPorts ports, 256 or 512 threads
static bool large_in_smem(mts_precision prec, int T, int max_ports) {
  return prec != MTS_FP64 && T >= 256 && max_ports <= kLargeSmemPorts;
}

size_t large_solve_smem(mts_precision prec, int max_ports) {
  if (prec == MTS_FP64) return LargeSmem<double>(max_ports).bytes;
  return LargeSmem<float>(max_ports, large_in_smem(prec, large_threads(max_ports), max_ports)).bytes;
}

template <typename R, int T, bool SA>
static cudaError_t launch_large(const SolveArgs& a, int64_t n_sys, int min_ports, int max_ports,
                                void* scratch, cudaStream_t st) {
  const size_t sm = LargeSmem<R>(max_ports, SA).bytes;
  cudaError_t e = cudaFuncSetAttribute(solve_large_kernel<R, T, SA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  solve_large_kernel<R, T, SA><<<(unsigned)n_sys, T, sm, st>>>(a, n_sys, min_ports, max_ports,
                                                               static_cast<Cx<R>*>(scratch));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_large(const SolveArgs& a, mts_precision prec, int64_t n_sys, int min_ports,
                               int max_ports, void* scratch, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  const int T = a.large_threads ? a.large_threads : large_threads(max_ports);
  if (prec == MTS_FP64)  // FP64 factors: at most 256 threads (the register budget of 512 is too small)
    return T == 128 ? launch_large<double, 128, false>(a, n_sys, min_ports, max_ports, scratch, st)
                    : launch_large<double, 256, false>(a, n_sys, min_ports, max_ports, scratch, st);
  const bool sa = large_in_smem(prec, T, max_ports);
  if (T == 128) return launch_large<float, 128, false>(a, n_sys, min_ports, max_ports, scratch, st);
  if (T == 256)
    return sa ? launch_large<float, 256, true>(a, n_sys, min_ports, max_ports, scratch, st)
              : launch_large<float, 256, false>(a, n_sys, min_ports, max_ports, scratch, st);
  return sa ? launch_large<float, 512, true>(a, n_sys, min_ports, max_ports, scratch, st)
            : launch_large<float, 512, false>(a, n_sys, min_ports, max_ports, scratch, st);
}

}  // namespace mts
