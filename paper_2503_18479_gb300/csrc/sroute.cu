// sroute.cu -- the scattering-parameter route (paper Sec. III and III-A, Eq. 3-7, Eq. 10):
// a structure given by its S-matrix S0 and per-port fields, a network tensor S_C built from
// a constant part and scattered variable entries, the wave ratio W = (1 - S11 S0)^-1 S12
// per configuration and frequency, the combined field Bcomb = field W, an objective at loss
// points, and the gradient with respect to the variable entries.
//
//   sr_solve_kernel    one CTA per system (configuration, frequency): assemble A and S12,
//                      LU with partial pivoting in shared memory (FP32, or FP64 for
//                      MTS_FP64), refinement on FP64 residuals, the objective partial, and
//                      the currents of the superposition
//   sr_adjoint_kernel  one CTA per system: the field derivative of the objective (and a
//                      field cotangent), Lambda = A^-H g_W with the stored factors and FP64
//                      refinement, and dL/dsvar (Eq. 10 in adjoint form)
//   superposition      the kernels of mts_superpose on an internal problem with one
//                      "structure" per frequency whose real basis is [Re field | Im field]
//                      and whose currents are [W_c ; j W_c] (2 n0 rows, one column per
//                      configuration and external port): field W = Re-part rows times W plus
//                      Im-part rows times j W
//
// Adjoint (dL = Re tr(g^H dX) for each complex X, torch's dL/dRe + j dL/dIm):
//   W = A^-1 S12, dW = A^-1 (dS12 - dA W), dA = -dS11 S0
//   Lambda = A^-H g_W,  g_S12 = Lambda,  g_S11 = Lambda (S0 W)^H,  S21 and S22: 0,
//   g_W = field^H g_B (the objective's g_B = 2 (|B| - t) B/|B| or 2 (B - t), over F n1 L).
// The factors P A = L U give A^H = U^H L^H P: forward substitution with U^H, backward with
// L^H, then the inverse row permutation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace mts {

constexpr int kSrMaxN0 = 96;
constexpr int kSrMaxN1 = 8;
constexpr int kSrMaxSvar = 1024;
constexpr int kSrThreads = 128;
constexpr int kSrWarps = kSrThreads / 32;
constexpr int kSrLossChunk = 64;  // loss points staged per pass of the adjoint kernel

// Scatter tables of the variable entries (host-built, copied into the route's basis by a
// kernel that takes them by value).
struct SrTables {
  int16_t row[kSrMaxSvar], col[kSrMaxSvar];  // every entry's position in S_C
  int16_t r_ptr[kSrMaxN0 + 1];               // S11 entries by row (CSR)
  int16_t r_col[kSrMaxSvar], r_var[kSrMaxSvar];
  int16_t c_ptr[kSrMaxN0 + 1];  // S11 entries by column (CSC)
  int16_t c_row[kSrMaxSvar], c_var[kSrMaxSvar];
  int16_t s12_row[kSrMaxSvar], s12_col[kSrMaxSvar], s12_var[kSrMaxSvar];  // S12 entries
  int32_t n11, n12;
};

template <typename LT>
struct SrT;
template <>
struct SrT<float> {
  using V = float2;
};
template <>
struct SrT<double> {
  using V = double2;
};

template <typename V>
__device__ inline V sr_mul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V>
__device__ inline V sr_mulc(V a, V b) {  // a conj(b)
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename V>
__device__ inline V sr_conj(V a) {
  a.y = -a.y;
  return a;
}
template <typename V>
__device__ inline V sr_recip(V a) {
  const auto d = a.x * a.x + a.y * a.y;
  V r;
  r.x = a.x / d;
  r.y = -a.y / d;
  return r;
}
// FP32 factors: the hardware approximate reciprocal (<= 1 ulp; refinement removes it)
template <>
__device__ inline float2 sr_recip<float2>(float2 a) {
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(a.x * a.x + a.y * a.y));
  return make_float2(a.x * inv, -a.y * inv);
}
template <typename V>
__device__ inline V sr_sub(V a, V b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename V>
__device__ inline V sr_add(V a, V b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename V>
__device__ inline V sr_from(double2 d) {
  V r;
  r.x = (decltype(r.x))d.x;
  r.y = (decltype(r.y))d.y;
  return r;
}
template <typename V>
__device__ inline double2 sr_to64(V v) {
  return make_double2((double)v.x, (double)v.y);
}

__device__ inline double sr_block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < kSrWarps; ++w) r = fmax(r, red[w]);
  return r;
}

// the same over FP32 values (convergence norms: a rough magnitude is all they need)
__device__ inline float sr_block_maxf(float v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  float r = (float)red[0];
  for (int w = 1; w < kSrWarps; ++w) r = fmaxf(r, (float)red[w]);
  return r;
}

// |re| + |im| of a complex FP64 value, as FP32 (one FP64 add)
__device__ inline float sr_mag1(double2 v) { return (float)(fabs(v.x) + fabs(v.y)); }

__device__ inline double sr_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < kSrWarps; ++w) r += red[w];
  return r;
}

// Double-float arithmetic on the FP32 pipe (this part's FP64 rate is 1/62 of FP32): a value
// is an unevaluated sum hi + lo of two floats. The product of two floats is split exactly by
// the FMA form of Dekker's TwoProd (p = a b, e = fma(a, b, -p)) and added to an accumulator
// with Knuth's TwoSum; the rounding-mode intrinsics keep the compiler from contracting these
// steps into fused operations.
__device__ inline void sr_df_acc(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  lo = __fadd_rn(lo, __fadd_rn(t, e));
  hi = s;
}

__device__ inline void sr_split(double2 v, float2& h, float2& l) {
  h = make_float2((float)v.x, (float)v.y);
  l = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
}

// sum_j M_j x_j (conj(M_j) x_j when CONJ) for complex M = Mh + Ml (element j at j*ms) and
// x = xh + xl (element j at j*xs): the hi x hi products exactly, the cross terms in FP32,
// all accumulated in double-float (about 2^-44 relative).
template <bool CONJ>
__device__ double2 sr_df_dot(const float2* __restrict__ Mh, const float2* __restrict__ Ml,
                             int ms, const float2* xh, const float2* xl, int xs, int n) {
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int j = 0; j < n; ++j) {
    float2 a = Mh[(int64_t)j * ms], c = Ml[(int64_t)j * ms];
    if (CONJ) {
      a.y = -a.y;
      c.y = -c.y;
    }
    const float2 p = xh[j * xs], q = xl[j * xs];
    sr_df_acc(rh, rl, a.x, p.x);
    sr_df_acc(rh, rl, -a.y, p.y);
    sr_df_acc(ih, il, a.x, p.y);
    sr_df_acc(ih, il, a.y, p.x);
    rl = fmaf(a.x, q.x, fmaf(-a.y, q.y, fmaf(c.x, p.x, fmaf(-c.y, p.y, rl))));
    il = fmaf(a.x, q.y, fmaf(a.y, q.x, fmaf(c.x, p.y, fmaf(c.y, p.x, il))));
  }
  return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

// LU with partial pivoting of the n x n matrix a (row-major, shared memory), in place:
// P a = L U, unit L below the diagonal. perm[i] = the original row now at row i. The pivot
// is the first row of largest |a_ik|^2 (a NaN candidate ranks as 0). Returns 1 on a zero
// (or non-finite) pivot.
template <typename LT>
__device__ int sr_factor(int n, typename SrT<LT>::V* a, int* perm, int* s_int) {
  using V = typename SrT<LT>::V;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += kSrThreads) perm[i] = i;
  __syncthreads();
  int bad = 0;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      LT best = (LT)-1;
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        const V v = a[i * n + k];
        LT m = v.x * v.x + v.y * v.y;
        if (!(m == m)) m = (LT)0;
        if (m > best) {
          best = m;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const LT ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_int[0] = bi;
        s_int[1] = !(best > (LT)0 && best < (LT)INFINITY);
        if (bi != k) {
          const int t = perm[k];
          perm[k] = perm[bi];
          perm[bi] = t;
        }
      }
    }
    __syncthreads();
    const int p = s_int[0];
    bad |= s_int[1];
    if (p != k)
      for (int j = tid; j < n; j += kSrThreads) {
        const V t = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = t;
      }
    __syncthreads();
    const V inv = sr_recip(a[k * n + k]);
    for (int i = k + 1 + tid; i < n; i += kSrThreads) a[i * n + k] = sr_mul(a[i * n + k], inv);
    __syncthreads();
    // trailing update: rows over warps, columns over lanes
    for (int i = k + 1 + warp; i < n; i += kSrWarps) {
      const V lik = a[i * n + k];
      for (int j = k + 1 + lane; j < n; j += 32) a[i * n + j] = sr_sub(a[i * n + j], sr_mul(lik, a[k * n + j]));
    }
    __syncthreads();
  }
  return bad;
}

// Triangular sweeps with the factors of sr_factor, one warp per right-hand-side column (n1
// columns, warps take columns w, w + 4, ...): lane l holds the unknowns of rows l, l + 32,
// l + 64 in registers; the unknown of step k is broadcast from its lane by a shuffle, so a
// sweep needs no CTA barrier (one at the end publishes x).
template <typename V>
__device__ inline V sr_bcast(V v, int src) {
  V r;
  r.x = __shfl_sync(0xffffffffu, v.x, src);
  r.y = __shfl_sync(0xffffffffu, v.y, src);
  return r;
}

// x <- U^-1 L^-1 x for the n1 columns of x ([n][n1]; x already row-permuted by P), n <= 96.
template <typename V>
__device__ void sr_solve_lu(int n, int n1, const V* a, V* x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < n1; c += kSrWarps) {
    V v[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int i = lane + 32 * s;
      v[s] = i < n ? x[i * n1 + c] : V{0, 0};
    }
    for (int k = 0; k + 1 < n; ++k) {  // L y = P b (unit diagonal)
      const int ks = k >> 5;
      const V mine = ks == 0 ? v[0] : (ks == 1 ? v[1] : v[2]);
      const V xk = sr_bcast(mine, k & 31);
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int i = lane + 32 * s;
        if (i > k && i < n) v[s] = sr_sub(v[s], sr_mul(a[i * n + k], xk));
      }
    }
    for (int k = n - 1; k >= 0; --k) {  // U x = y
      const int ks = k >> 5;
      if (lane == (k & 31)) {
        const V d = sr_recip(a[k * n + k]);
        if (ks == 0) v[0] = sr_mul(v[0], d);
        else if (ks == 1) v[1] = sr_mul(v[1], d);
        else v[2] = sr_mul(v[2], d);
      }
      const V mine = ks == 0 ? v[0] : (ks == 1 ? v[1] : v[2]);
      const V xk = sr_bcast(mine, k & 31);
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int i = lane + 32 * s;
        if (i < k) v[s] = sr_sub(v[s], sr_mul(a[i * n + k], xk));
      }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int i = lane + 32 * s;
      if (i < n) x[i * n1 + c] = v[s];
    }
  }
  __syncthreads();
}

// With P A = L U, A^H = U^H L^H P, so A^H z = g is z = P^T (L^H)^-1 (U^H)^-1 g; this applies
// (L^H)^-1 (U^H)^-1 and the caller applies P^T (z[perm[i]] = x[i]).
template <typename V>
__device__ void sr_solve_lu_h(int n, int n1, const V* a, V* x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < n1; c += kSrWarps) {
    V v[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int i = lane + 32 * s;
      v[s] = i < n ? x[i * n1 + c] : V{0, 0};
    }
    for (int k = 0; k < n; ++k) {  // U^H t = g: row i of U^H is conj(column i of U)
      const int ks = k >> 5;
      if (lane == (k & 31)) {
        const V d = sr_recip(sr_conj(a[k * n + k]));
        if (ks == 0) v[0] = sr_mul(v[0], d);
        else if (ks == 1) v[1] = sr_mul(v[1], d);
        else v[2] = sr_mul(v[2], d);
      }
      const V mine = ks == 0 ? v[0] : (ks == 1 ? v[1] : v[2]);
      const V xk = sr_bcast(mine, k & 31);
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int i = lane + 32 * s;
        if (i > k && i < n) v[s] = sr_sub(v[s], sr_mul(sr_conj(a[k * n + i]), xk));
      }
    }
    for (int k = n - 1; k > 0; --k) {  // L^H s = t (unit diagonal)
      const int ks = k >> 5;
      const V mine = ks == 0 ? v[0] : (ks == 1 ? v[1] : v[2]);
      const V xk = sr_bcast(mine, k & 31);
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int i = lane + 32 * s;
        if (i < k) v[s] = sr_sub(v[s], sr_mul(sr_conj(a[k * n + i]), xk));
      }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int i = lane + 32 * s;
      if (i < n) x[i * n1 + c] = v[s];
    }
  }
  __syncthreads();
}

// objective term of one point and its field derivative (mode 0: (|b| - t)^2,
// G = 2 (|b| - t) b/|b|, 0 at b = 0; mode 1: |b - t|^2, G = 2 (b - t))
// Objective term alone (forward): the same FP64 arithmetic as sr_point_loss's value.
__device__ inline double sr_point_value(int mode, double2 b, const double* t) {
  if (mode == 0) {
    const double r = hypot(b.x, b.y) - t[0];
    return r * r;
  }
  const double ex = b.x - t[0], ey = b.y - t[1];
  return ex * ex + ey * ey;
}

// Cotangent G of the term in FP32 (adjoint with FP32 factors, where the loss-point field it
// differentiates is itself an FP32 sum), as the impedance route's FP32 kernels take it.
__device__ inline double2 sr_point_grad_f(int mode, double2 b, const double* t) {
  const float bx = (float)b.x, by = (float)b.y;
  if (mode == 0) {
    const float m = sqrtf(bx * bx + by * by);
    const float s = m > 0.0f ? 2.0f * (m - (float)t[0]) / m : 0.0f;
    return make_double2((double)(s * bx), (double)(s * by));
  }
  return make_double2(2.0 * (double)(bx - (float)t[0]), 2.0 * (double)(by - (float)t[1]));
}

__device__ inline double sr_point_loss(int mode, double2 b, const double* t, double2* G) {
  if (mode == 0) {
    const double m = hypot(b.x, b.y);
    const double r = m - t[0];
    if (m > 0.0) *G = make_double2(2.0 * r * b.x / m, 2.0 * r * b.y / m);
    else *G = make_double2(0.0, 0.0);
    return r * r;
  }
  const double ex = b.x - t[0], ey = b.y - t[1];
  *G = make_double2(2.0 * ex, 2.0 * ey);
  return ex * ex + ey * ey;
}

struct SrArgs {
  int n0, n1, F, nS, L, loss_mode, max_refine;
  int64_t n_cfg, P, sumFNv;
  double tol;
  const double2* S0;        // [F][n0][n0]
  const double2* T;         // [F][n0][n0] = S_C,const11 S0
  const int32_t* tflag;     // [0] != 0: S_C,const11 is nonzero
  const double2* sc_const;  // [F][n][n] or nullptr
  const double2* svar;      // [n_cfg][F][nS]
  const double2* field;     // [F][P][n0]
  const int64_t* loss_idx;
  const double* target;  // [F][n1][L] (x1 or x2)
  const double* loss_weight;   // [F][n1][L] or nullptr
  const double2* loss_offset;  // [F][n1][L] or nullptr
  const SrTables* tabs;
  // FP32 factors only: S0 and T as hi/lo float pairs, loss-point rows of the field in FP32
  const float2 *S0h, *S0l, *Th, *Tl, *fl32;
  double2* W;        // tape [n_cfg F][n0][n1]
  double2* W_out;    // optional copy
  void* lu;          // tape [n_cfg F][n0][n0] (float2 or double2)
  int32_t* perm;     // tape [n_cfg F][n0]
  double* Iv;        // tape currents of the superposition [n_cfg n1][F][2 n0] complex
  double* loss_part; // tape [n_cfg F]
  int32_t* status;   // tape [n_cfg F]
  // adjoint
  const double* grad_loss;  // [n_cfg] or nullptr
  const double2* u;         // field cotangent term [n_cfg n1][F][2 n0] or nullptr
  double2* grad_svar;       // [n_cfg][F][nS]
  double norm;              // F n1 L
};

__host__ __device__ inline size_t sr_al16(size_t x) { return (x + 15) / 16 * 16; }

// Shared-memory carve of the forward kernel (bytes), LT = float or double.
template <typename LT>
__host__ __device__ inline size_t sr_solve_smem(int n, int n1, int nS, size_t* o) {
  const size_t v = sizeof(typename SrT<LT>::V);
  size_t off = 0;
  o[0] = off; off = sr_al16(off + v * n * n);        // lu
  o[1] = off; off = sr_al16(off + 16 * n * n1);      // rhs
  o[2] = off; off = sr_al16(off + 16 * n * n1);      // w
  o[3] = off; off = sr_al16(off + 16 * n * n1);      // r
  o[4] = off; off = sr_al16(off + 16 * n * n1);      // sw
  o[5] = off; off = sr_al16(off + v * n * n1);       // x
  o[6] = off; off = sr_al16(off + 16 * (size_t)nS);  // sv
  o[7] = off; off = sr_al16(off + 4 * n);            // perm
  o[8] = off; off = sr_al16(off + 8 * 32 + 16);      // reduction scratch, ints
  const size_t fs = v == 8 ? 8 * (size_t)n * n1 : 0;  // hi/lo split of w (FP32 factors)
  o[9] = off; off = sr_al16(off + fs);
  o[10] = off; off = sr_al16(off + fs);
  return off;
}

template <typename LT>
__global__ void __launch_bounds__(kSrThreads) sr_solve_kernel(SrArgs a) {
  using V = typename SrT<LT>::V;
  extern __shared__ __align__(16) unsigned char sm_sr[];
  const int n = a.n0, n1 = a.n1, nn1 = n * n1, ntot = a.n0 + a.n1;
  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t b = g / a.F;
  const int f = (int)(g - b * a.F);
  constexpr bool kDF = sizeof(V) == 8;  // FP32 factors: double-float residuals
  size_t o[11];
  sr_solve_smem<LT>(n, n1, a.nS, o);
  float2* wh = reinterpret_cast<float2*>(sm_sr + o[9]);
  float2* wlo = reinterpret_cast<float2*>(sm_sr + o[10]);
  const int64_t fo = (int64_t)f * n * n;
  V* lu = reinterpret_cast<V*>(sm_sr + o[0]);
  double2* rhs = reinterpret_cast<double2*>(sm_sr + o[1]);
  double2* w = reinterpret_cast<double2*>(sm_sr + o[2]);
  double2* r = reinterpret_cast<double2*>(sm_sr + o[3]);
  double2* sw = reinterpret_cast<double2*>(sm_sr + o[4]);
  V* x = reinterpret_cast<V*>(sm_sr + o[5]);
  double2* sv = reinterpret_cast<double2*>(sm_sr + o[6]);
  int* perm = reinterpret_cast<int*>(sm_sr + o[7]);
  double* red = reinterpret_cast<double*>(sm_sr + o[8]);
  int* sint = reinterpret_cast<int*>(red + 32);
  const SrTables& tb = *a.tabs;
  const double2* S0f = a.S0 + (int64_t)f * n * n;
  const double2* Tf = a.T + (int64_t)f * n * n;
  const bool tnz = a.sc_const != nullptr && a.tflag[0] != 0;

  for (int i = tid; i < a.nS; i += kSrThreads) sv[i] = a.svar[g * a.nS + i];
  for (int e = tid; e < nn1; e += kSrThreads) {
    const int i = e / n1, c = e % n1;
    rhs[e] = a.sc_const ? a.sc_const[((int64_t)f * ntot + i) * ntot + n + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int q = tid; q < tb.n12; q += kSrThreads) {  // distinct positions
    const int e = tb.s12_row[q] * n1 + tb.s12_col[q];
    rhs[e] = sr_add(rhs[e], sv[tb.s12_var[q]]);
  }
  // A = 1 - S_C,const11 S0 - sum over S11 entries v e_r S0[c, :]
  const int lane = tid & 31, warp = tid >> 5;
  for (int i = warp; i < n; i += kSrWarps)
  for (int j = lane; j < n; j += 32) {
    const int e = i * n + j;
    if constexpr (kDF) {  // the factors are FP32: assemble A in FP32
      float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
      if (tnz) v = sr_sub(v, a.Th[fo + e]);
      for (int q = tb.r_ptr[i]; q < tb.r_ptr[i + 1]; ++q) {
        const double2 s = sv[tb.r_var[q]];
        v = sr_sub(v, sr_mul(make_float2((float)s.x, (float)s.y), a.S0h[fo + tb.r_col[q] * n + j]));
      }
      lu[e] = sr_from<V>(make_double2(v.x, v.y));
    } else {
      double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
      if (tnz) v = sr_sub(v, Tf[e]);
      for (int q = tb.r_ptr[i]; q < tb.r_ptr[i + 1]; ++q)
        v = sr_sub(v, sr_mul(sv[tb.r_var[q]], S0f[tb.r_col[q] * n + j]));
      lu[e] = sr_from<V>(v);
    }
  }
  __syncthreads();
  const int singular = sr_factor<LT>(n, lu, perm, sint);

  // first solve
  for (int e = tid; e < nn1; e += kSrThreads) x[e] = sr_from<V>(rhs[perm[e / n1] * n1 + e % n1]);
  __syncthreads();
  sr_solve_lu(n, n1, lu, x);
  float loc = 0.0f;
  for (int e = tid; e < nn1; e += kSrThreads) {
    w[e] = sr_to64(x[e]);
    loc = fmaxf(loc, sr_mag1(w[e]));
  }
  float dprev = sr_block_maxf(loc, red);
  int converged = a.max_refine == 0;
  for (int it = 0; it < a.max_refine; ++it) {
    // residual in FP64 (double-float for FP32 factors): r = S12 - A w,
    // A w = w - T w - sum_q v_q e_row (S0 w)[col]
    if constexpr (kDF) {
      for (int e = tid; e < nn1; e += kSrThreads) sr_split(w[e], wh[e], wlo[e]);
      __syncthreads();
      for (int e = tid; e < nn1; e += kSrThreads) {
        const int i = e / n1, c = e % n1;
        sw[e] = sr_df_dot<false>(a.S0h + fo + i * n, a.S0l + fo + i * n, 1, wh + c, wlo + c, n1, n);
        if (tnz) r[e] = sr_df_dot<false>(a.Th + fo + i * n, a.Tl + fo + i * n, 1, wh + c, wlo + c, n1, n);
      }
    } else {
      for (int e = tid; e < nn1; e += kSrThreads) {
        const int i = e / n1, c = e % n1;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < n; ++j) acc = sr_add(acc, sr_mul(S0f[i * n + j], w[j * n1 + c]));
        sw[e] = acc;
      }
    }
    __syncthreads();
    for (int e = tid; e < nn1; e += kSrThreads) {
      const int i = e / n1, c = e % n1;
      double2 aw = w[e];
      if (tnz) {
        if constexpr (kDF) {
          aw = sr_sub(aw, r[e]);
        } else {
          for (int j = 0; j < n; ++j) aw = sr_sub(aw, sr_mul(Tf[i * n + j], w[j * n1 + c]));
        }
      }
      for (int q = tb.r_ptr[i]; q < tb.r_ptr[i + 1]; ++q)
        aw = sr_sub(aw, sr_mul(sv[tb.r_var[q]], sw[tb.r_col[q] * n1 + c]));
      r[e] = sr_sub(rhs[e], aw);
    }
    __syncthreads();
    for (int e = tid; e < nn1; e += kSrThreads) x[e] = sr_from<V>(r[perm[e / n1] * n1 + e % n1]);
    __syncthreads();
    sr_solve_lu(n, n1, lu, x);
    float dl = 0.0f, wl = 0.0f;
    for (int e = tid; e < nn1; e += kSrThreads) {
      const double2 d = sr_to64(x[e]);
      w[e] = sr_add(w[e], d);
      dl = fmaxf(dl, sr_mag1(d));
      wl = fmaxf(wl, sr_mag1(w[e]));
    }
    const float dn = sr_block_maxf(dl, red);
    const float wn = sr_block_maxf(wl, red);
    const double est = dn == 0.0f ? 0.0 : (double)dn * dn / dprev / wn;
    if (est <= a.tol) {
      converged = 1;
      break;
    }
    if (!(dn <= 0.5 * dprev)) break;  // no longer halving (or non-finite)
    dprev = dn;
  }
  double nf = 0.0;
  for (int e = tid; e < nn1; e += kSrThreads) nf += (isfinite(w[e].x) && isfinite(w[e].y)) ? 0.0 : 1.0;
  const bool finite = sr_block_max(nf, red) == 0.0;

  // outputs: wave ratios, factors, currents of the superposition
  for (int e = tid; e < nn1; e += kSrThreads) {
    a.W[g * nn1 + e] = w[e];
    if (a.W_out) a.W_out[g * nn1 + e] = w[e];
    const int k = e / n1, c = e % n1;
    const int64_t base = (b * n1 + c) * a.sumFNv + (int64_t)f * 2 * n;
    a.Iv[2 * (base + k)] = w[e].x;
    a.Iv[2 * (base + k) + 1] = w[e].y;
    a.Iv[2 * (base + n + k)] = -w[e].y;  // j w
    a.Iv[2 * (base + n + k) + 1] = w[e].x;
  }
  V* luo = static_cast<V*>(a.lu) + g * n * n;
  for (int e = tid; e < n * n; e += kSrThreads) luo[e] = lu[e];
  for (int i = tid; i < n; i += kSrThreads) a.perm[g * n + i] = perm[i];

  // objective partial at the loss points (FP32 rows and sums for FP32 factors, as in the
  // register-resident solve of the impedance route)
  if (a.target != nullptr) {
    const int tw = a.loss_mode == 0 ? 1 : 2;
    double acc = 0.0;
    if constexpr (kDF) {
      for (int e = tid; e < nn1; e += kSrThreads) wh[e] = make_float2((float)w[e].x, (float)w[e].y);
      __syncthreads();
    }
    for (int e = tid; e < n1 * a.L; e += kSrThreads) {
      const int c = e / a.L, l = e % a.L;
      double2 bl = make_double2(0.0, 0.0);
      if constexpr (kDF) {
        const float2* fr = a.fl32 + ((int64_t)f * a.L + l) * n;
        float2 b32 = make_float2(0.f, 0.f);
        for (int k = 0; k < n; ++k) b32 = sr_add(b32, sr_mul(fr[k], wh[k * n1 + c]));
        bl = make_double2(b32.x, b32.y);
      } else {
        const double2* fr = a.field + ((int64_t)f * a.P + a.loss_idx[l]) * n;
        for (int k = 0; k < n; ++k) bl = sr_add(bl, sr_mul(fr[k], w[k * n1 + c]));
      }
      const int64_t ti = ((int64_t)f * n1 + c) * a.L + l;
      if (a.loss_offset) bl = sr_add(bl, a.loss_offset[ti]);
      if (a.loss_weight) {
        bl.x *= a.loss_weight[ti];
        bl.y *= a.loss_weight[ti];
      }
      acc += sr_point_value(a.loss_mode, bl, a.target + ti * tw);
    }
    acc = sr_block_sum(acc, red);
    if (tid == 0) a.loss_part[g] = acc;
  }
  if (tid == 0) a.status[g] = (singular || !finite) ? 2 : (converged ? 0 : 1);
}

// Shared-memory carve of the adjoint kernel.
template <typename LT>
__host__ __device__ inline size_t sr_adj_smem(int n, int n1, int nS, size_t* o) {
  const size_t v = sizeof(typename SrT<LT>::V);
  size_t off = 0;
  size_t rsz = 16 * (size_t)n * n1;
  const size_t gsz = 16 * (size_t)n1 * kSrLossChunk;
  if (gsz > rsz) rsz = gsz;
  o[0] = off; off = sr_al16(off + v * n * n);    // lu
  o[1] = off; off = sr_al16(off + 16 * n * n1);  // lam
  o[2] = off; off = sr_al16(off + 16 * n * n1);  // gw (right-hand side)
  o[3] = off; off = sr_al16(off + rsz);          // r (also the staged G of a loss chunk)
  o[4] = off; off = sr_al16(off + 16 * n * n1);  // y (also S0 W at the end)
  // x: for FP64 factors it shares r's storage (x[e] is converted from r[e] in place)
  o[5] = v == 16 ? o[3] : off;
  if (v != 16) off = sr_al16(off + v * n * n1);
  o[6] = off; off = sr_al16(off + 16 * n * n1);  // w
  o[7] = off; off = sr_al16(off + 16 * (size_t)nS);
  o[8] = off; off = sr_al16(off + 4 * n);
  o[9] = off; off = sr_al16(off + 8 * 32 + 16);
  const size_t fs = v == 8 ? 8 * (size_t)n * n1 : 0;  // two hi/lo splits (FP32 factors)
  for (int q = 10; q < 14; ++q) {
    o[q] = off;
    off = sr_al16(off + fs);
  }
  return off;
}

template <typename LT>
__global__ void __launch_bounds__(kSrThreads) sr_adjoint_kernel(SrArgs a) {
  using V = typename SrT<LT>::V;
  extern __shared__ __align__(16) unsigned char sm_sa[];
  const int n = a.n0, n1 = a.n1, nn1 = n * n1;
  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t b = g / a.F;
  const int f = (int)(g - b * a.F);
  constexpr bool kDF = sizeof(V) == 8;  // FP32 factors: double-float residuals
  size_t o[14];
  sr_adj_smem<LT>(n, n1, a.nS, o);
  float2* ah = reinterpret_cast<float2*>(sm_sa + o[10]);
  float2* al = reinterpret_cast<float2*>(sm_sa + o[11]);
  float2* bh = reinterpret_cast<float2*>(sm_sa + o[12]);
  float2* bl2 = reinterpret_cast<float2*>(sm_sa + o[13]);
  const int64_t fo = (int64_t)f * n * n;
  V* lu = reinterpret_cast<V*>(sm_sa + o[0]);
  double2* lam = reinterpret_cast<double2*>(sm_sa + o[1]);
  double2* gw = reinterpret_cast<double2*>(sm_sa + o[2]);
  double2* r = reinterpret_cast<double2*>(sm_sa + o[3]);
  double2* y = reinterpret_cast<double2*>(sm_sa + o[4]);
  V* x = reinterpret_cast<V*>(sm_sa + o[5]);
  double2* w = reinterpret_cast<double2*>(sm_sa + o[6]);
  double2* sv = reinterpret_cast<double2*>(sm_sa + o[7]);
  int* perm = reinterpret_cast<int*>(sm_sa + o[8]);
  double* red = reinterpret_cast<double*>(sm_sa + o[9]);
  const SrTables& tb = *a.tabs;
  const double2* S0f = a.S0 + (int64_t)f * n * n;
  const double2* Tf = a.T + (int64_t)f * n * n;
  const bool tnz = a.sc_const != nullptr && a.tflag[0] != 0;

  const V* lui = static_cast<const V*>(a.lu) + g * n * n;
  for (int e = tid; e < n * n; e += kSrThreads) lu[e] = lui[e];
  for (int i = tid; i < n; i += kSrThreads) perm[i] = a.perm[g * n + i];
  for (int i = tid; i < a.nS; i += kSrThreads) sv[i] = a.svar[g * a.nS + i];
  for (int e = tid; e < nn1; e += kSrThreads) {
    w[e] = a.W[g * nn1 + e];
    gw[e] = make_double2(0.0, 0.0);
    if constexpr (kDF) sr_split(w[e], bh[e], bl2[e]);  // w split, kept to the end
  }
  __syncthreads();

  // g_W = field^H g_B at the loss points (objective) ...
  if (a.grad_loss != nullptr && a.target != nullptr && a.L > 0) {
    const double gl = a.grad_loss[b] / a.norm;
    const int tw = a.loss_mode == 0 ? 1 : 2;
    double2* Gs = r;  // [n1][chunk]
    for (int l0 = 0; l0 < a.L; l0 += kSrLossChunk) {
      const int lc = min(kSrLossChunk, a.L - l0);
      for (int e = tid; e < n1 * lc; e += kSrThreads) {
        const int c = e / lc, l = l0 + e % lc;
        double2 bl = make_double2(0.0, 0.0);
        if constexpr (kDF) {
          const float2* fr = a.fl32 + ((int64_t)f * a.L + l) * n;
          float2 b32 = make_float2(0.f, 0.f);
          for (int k = 0; k < n; ++k) b32 = sr_add(b32, sr_mul(fr[k], bh[k * n1 + c]));
          bl = make_double2(b32.x, b32.y);
        } else {
          const double2* fr = a.field + ((int64_t)f * a.P + a.loss_idx[l]) * n;
          for (int k = 0; k < n; ++k) bl = sr_add(bl, sr_mul(fr[k], w[k * n1 + c]));
        }
        const int64_t ti = ((int64_t)f * n1 + c) * a.L + l;
        double wl = 1.0;
        if (a.loss_offset) bl = sr_add(bl, a.loss_offset[ti]);
        if (a.loss_weight) {
          wl = a.loss_weight[ti];
          bl.x *= wl;
          bl.y *= wl;
        }
        double2 G;
        if constexpr (kDF) G = sr_point_grad_f(a.loss_mode, bl, a.target + ti * tw);
        else sr_point_loss(a.loss_mode, bl, a.target + ti * tw, &G);
        Gs[c * kSrLossChunk + (e % lc)] = make_double2(G.x * gl * wl, G.y * gl * wl);
      }
      __syncthreads();
      for (int e = tid; e < nn1; e += kSrThreads) {
        const int k = e / n1, c = e % n1;
        double2 acc = gw[e];
        if constexpr (kDF) {
          float2 a32 = make_float2(0.f, 0.f);
          for (int q = 0; q < lc; ++q) {
            const double2 gq = Gs[c * kSrLossChunk + q];
            a32 = sr_add(a32, sr_mul(sr_conj(a.fl32[((int64_t)f * a.L + l0 + q) * n + k]),
                                     make_float2((float)gq.x, (float)gq.y)));
          }
          acc = sr_add(acc, make_double2(a32.x, a32.y));
        } else {
          for (int q = 0; q < lc; ++q) {
            const double2 fv = a.field[((int64_t)f * a.P + a.loss_idx[l0 + q]) * n + k];
            acc = sr_add(acc, sr_mul(sr_conj(fv), Gs[c * kSrLossChunk + q]));
          }
        }
        gw[e] = acc;
      }
      __syncthreads();
    }
  }
  // ... plus the field cotangent: u = [Re field | Im field]^T conj(grad_B) per column, and
  // g_W = conj(u_re) - j conj(u_im)
  if (a.u != nullptr) {
    for (int e = tid; e < nn1; e += kSrThreads) {
      const int k = e / n1, c = e % n1;
      const int64_t base = (b * n1 + c) * a.sumFNv + (int64_t)f * 2 * n;
      const double2 ut = a.u[base + k], ub = a.u[base + n + k];
      gw[e] = sr_add(gw[e], make_double2(ut.x - ub.y, -ut.y - ub.x));
    }
  }
  __syncthreads();

  // Lambda = A^-H g_W
  for (int e = tid; e < nn1; e += kSrThreads) x[e] = sr_from<V>(gw[e]);
  __syncthreads();
  sr_solve_lu_h(n, n1, lu, x);
  float loc = 0.0f;
  for (int e = tid; e < nn1; e += kSrThreads) {
    const int i = e / n1, c = e % n1;
    const double2 v = sr_to64(x[e]);
    lam[perm[i] * n1 + c] = v;
    loc = fmaxf(loc, sr_mag1(v));
  }
  float dprev = sr_block_maxf(loc, red);
  int converged = a.max_refine == 0;
  for (int it = 0; it < a.max_refine; ++it) {
    // r = g_W - A^H lam,  A^H lam = lam - T^H lam - S0^H y,  y = sum_q conj(v_q) e_col lam[row]
    for (int e = tid; e < nn1; e += kSrThreads) {
      const int j = e / n1, c = e % n1;
      double2 acc = make_double2(0.0, 0.0);
      for (int q = tb.c_ptr[j]; q < tb.c_ptr[j + 1]; ++q)
        acc = sr_add(acc, sr_mul(sr_conj(sv[tb.c_var[q]]), lam[tb.c_row[q] * n1 + c]));
      y[e] = acc;
      if constexpr (kDF) {
        sr_split(acc, ah[e], al[e]);
        if (tnz) sr_split(lam[e], bh[e], bl2[e]);  // lam split (w's split is redone below)
      }
    }
    __syncthreads();
    for (int e = tid; e < nn1; e += kSrThreads) {
      const int i = e / n1, c = e % n1;
      double2 acc = lam[e];
      if constexpr (kDF) {
        // column i of S0 (and T): conj(S0[j][i]) at j n + i
        acc = sr_sub(acc, sr_df_dot<true>(a.S0h + fo + i, a.S0l + fo + i, n, ah + c, al + c, n1, n));
        if (tnz)
          acc = sr_sub(acc, sr_df_dot<true>(a.Th + fo + i, a.Tl + fo + i, n, bh + c, bl2 + c, n1, n));
      } else {
        for (int j = 0; j < n; ++j) {
          acc = sr_sub(acc, sr_mul(sr_conj(S0f[j * n + i]), y[j * n1 + c]));
          if (tnz) acc = sr_sub(acc, sr_mul(sr_conj(Tf[j * n + i]), lam[j * n1 + c]));
        }
      }
      r[e] = sr_sub(gw[e], acc);
    }
    __syncthreads();
    for (int e = tid; e < nn1; e += kSrThreads) x[e] = sr_from<V>(r[e]);
    __syncthreads();
    sr_solve_lu_h(n, n1, lu, x);
    float dl = 0.0f, ll = 0.0f;
    for (int e = tid; e < nn1; e += kSrThreads) {
      const int i = e / n1, c = e % n1;
      const double2 d = sr_to64(x[e]);
      const int t = perm[i] * n1 + c;
      lam[t] = sr_add(lam[t], d);
      dl = fmaxf(dl, sr_mag1(d));
    }
    __syncthreads();
    for (int e = tid; e < nn1; e += kSrThreads) ll = fmaxf(ll, sr_mag1(lam[e]));
    const float dn = sr_block_maxf(dl, red);
    const float ln = sr_block_maxf(ll, red);
    const double est = dn == 0.0f ? 0.0 : (double)dn * dn / dprev / ln;
    if (est <= a.tol) {
      converged = 1;
      break;
    }
    if (!(dn <= 0.5 * dprev)) break;
    dprev = dn;
  }

  // gradient: S11 entry (r, c): sum_col lam[r][col] conj((S0 W)[c][col]); S12 entry (r, c):
  // lam[r][c - n0]; S21, S22: 0
  double2* sw = y;
  if constexpr (kDF) {
    for (int e = tid; e < nn1; e += kSrThreads) sr_split(w[e], bh[e], bl2[e]);
    __syncthreads();
  }
  for (int e = tid; e < nn1; e += kSrThreads) {
    const int i = e / n1, c = e % n1;
    if constexpr (kDF) {
      sw[e] = sr_df_dot<false>(a.S0h + fo + i * n, a.S0l + fo + i * n, 1, bh + c, bl2 + c, n1, n);
    } else {
      double2 acc = make_double2(0.0, 0.0);
      for (int j = 0; j < n; ++j) acc = sr_add(acc, sr_mul(S0f[i * n + j], w[j * n1 + c]));
      sw[e] = acc;
    }
  }
  __syncthreads();
  for (int q = tid; q < a.nS; q += kSrThreads) {
    const int rr = tb.row[q], cc = tb.col[q];
    double2 gv = make_double2(0.0, 0.0);
    if (rr < n) {
      if (cc < n) {
        for (int c = 0; c < n1; ++c) gv = sr_add(gv, sr_mulc(lam[rr * n1 + c], sw[cc * n1 + c]));
      } else {
        gv = lam[rr * n1 + (cc - n)];
      }
    }
    a.grad_svar[g * a.nS + q] = gv;
  }
  if (tid == 0 && !converged) atomicOr(&a.status[g], 4);
}

// currents of the superposition -> bf16 pieces of the tensor-core B operand (rows 2 cfg + c
// of each per-frequency structure, as the solve kernels of mts_solve write them)
__global__ void sr_pack_kernel(int F, int64_t n_cfg_v, int Kv, int npieces, int64_t sumFNv,
                               const int64_t* __restrict__ bop_off, const double* __restrict__ I,
                               __nv_bfloat16* __restrict__ Bop) {
  const int s = blockIdx.y;
  const int nkc = (Kv + kChunkK - 1) / kChunkK, Kpad = nkc * kChunkK;
  const int64_t ntile = (2 * n_cfg_v + kTileN - 1) / kTileN;
  const size_t tile_bytes = (size_t)kTileN * kChunkK * 2;
  char* base = reinterpret_cast<char*>(Bop + bop_off[s]);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_cfg_v * Kpad;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nsys = idx / Kpad;
    const int kg = (int)(idx % Kpad), kc = kg / kChunkK, kk = kg % kChunkK;
    for (int c = 0; c < 2; ++c) {
      const int64_t row = 2 * nsys + c;
      const int64_t tile = row / kTileN;
      const uint32_t rr = (uint32_t)(row % kTileN);
      const double xv = kg < Kv ? I[2 * (nsys * sumFNv + (int64_t)s * Kv + kg) + c] : 0.0;
      const float xh = (float)xv, xl = (float)(xv - (double)xh);
      float rem = xh;
      for (int q = 0; q < npieces; ++q) {
        const __nv_bfloat16 h = __float2bfloat16_rn(rem);
        rem = rem - __bfloat162float(h);
        if (q == 0) rem += xl;
        const size_t off = ((size_t)(q * ntile + tile) * nkc + kc) * tile_bytes + swz128(rr, kk);
        *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
      }
    }
  }
}

__global__ void sr_voff_kernel(int F, int Kv, int64_t P, int32_t* port, int64_t* point,
                               int32_t* freq) {
  for (int i = threadIdx.x; i <= F; i += blockDim.x) {
    port[i] = i * Kv;
    point[i] = (int64_t)i * P;
    freq[i] = i;
  }
}

template <typename HT>
__global__ void sr_field_kernel(int F, int64_t P, int n0, const double2* __restrict__ field,
                                const int64_t* __restrict__ pn_off, HT* __restrict__ H) {
  const int64_t total = (int64_t)F * P * n0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % n0);
    const int64_t fp = i / n0;
    const int f = (int)(fp / P);
    const int64_t p = fp - (int64_t)f * P;
    const double2 v = field[i];
    HT* row = H + pn_off[f] + p * 2 * n0;
    row[k] = (HT)v.x;
    row[n0 + k] = (HT)v.y;
  }
}

// T[f] = S_C,const11[f] S0[f]; flag[0] = 1 if S_C,const11 has a nonzero entry
__global__ void sr_const_kernel(int n0, int n1, const double2* __restrict__ S0,
                                const double2* __restrict__ sc, double2* __restrict__ T,
                                int32_t* flag) {
  const int i = blockIdx.x, f = blockIdx.y, n = n0 + n1;
  const double2* Sc = sc + (int64_t)f * n * n + (int64_t)i * n;
  const double2* S0f = S0 + (int64_t)f * n0 * n0;
  for (int j = threadIdx.x; j < n0; j += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < n0; ++k) acc = sr_add(acc, sr_mul(Sc[k], S0f[k * n0 + j]));
    T[((int64_t)f * n0 + i) * n0 + j] = acc;
    if (Sc[j].x != 0.0 || Sc[j].y != 0.0) atomicOr(flag, 1);
  }
}

// hi/lo float pairs of a complex FP64 array (double-float operands of the residuals)
__global__ void sr_split_kernel(int64_t n, const double2* __restrict__ src, float2* __restrict__ hi,
                                float2* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sr_split(src[i], hi[i], lo[i]);
}

// the field's rows at the loss points in FP32, [F][L][n0]
__global__ void sr_lossrows_kernel(int F, int64_t P, int L, int n0, const double2* __restrict__ field,
                                   const int64_t* __restrict__ loss_idx, float2* __restrict__ out) {
  const int64_t total = (int64_t)F * L * n0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % n0);
    const int64_t fl = i / n0;
    const int f = (int)(fl / L), l = (int)(fl % L);
    const double2 v = field[((int64_t)f * P + loss_idx[l]) * n0 + k];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void sr_tables_kernel(SrTables t, SrTables* out) {
  const int32_t* src = reinterpret_cast<const int32_t*>(&t);
  int32_t* dst = reinterpret_cast<int32_t*>(out);
  for (int i = threadIdx.x; i < (int)(sizeof(SrTables) / 4); i += blockDim.x) dst[i] = src[i];
}

__global__ void sr_loss_kernel(int64_t n_cfg, int F, double norm, const double* __restrict__ part,
                               double* __restrict__ loss) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_cfg) return;
  double s = 0.0;
  for (int f = 0; f < F; ++f) s += part[b * F + f];
  loss[b] = norm > 0.0 ? s / norm : 0.0;
}

// Eq. 2-3 for series RC loads, and the vector-Jacobian product
__device__ inline double2 sr_rc_gamma(double R, double C, double w, double Z0, double2* dgdz) {
  const double2 Z = make_double2(R, -1.0 / (w * C));
  const double2 num = make_double2(Z.x - Z0, Z.y), den = make_double2(Z.x + Z0, Z.y);
  const double2 iden = sr_recip(den);
  if (dgdz) *dgdz = sr_mul(make_double2(2.0 * Z0, 0.0), sr_mul(iden, iden));
  return sr_mul(num, iden);
}

__global__ void sr_rc_kernel(int64_t n_cfg, int F, int nL, const double* __restrict__ omega,
                             const double* __restrict__ R, const double* __restrict__ C, double Z0,
                             int stride, int off, double2* __restrict__ svar) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cfg * F * nL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % nL);
    const int64_t bf = i / nL;
    const int f = (int)(bf % F);
    const int64_t b = bf / F;
    const double r = R ? R[b * nL + k] : 0.0;
    svar[bf * stride + off + k] = sr_rc_gamma(r, C[b * nL + k], omega[f], Z0, nullptr);
  }
}

__global__ void sr_rc_vjp_kernel(int64_t n_cfg, int F, int nL, const double* __restrict__ omega,
                                 const double* __restrict__ R, const double* __restrict__ C,
                                 double Z0, int stride, int off, const double2* __restrict__ gs,
                                 double* __restrict__ gR, double* __restrict__ gC) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cfg * nL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % nL);
    const int64_t b = i / nL;
    const double r = R ? R[i] : 0.0, c = C[i];
    double sc = 0.0, sr = 0.0;
    for (int f = 0; f < F; ++f) {
      const double w = omega[f];
      double2 dgdz;
      sr_rc_gamma(r, c, w, Z0, &dgdz);
      const double2 gv = gs[(b * F + f) * stride + off + k];
      // dGamma/dC = dGamma/dZ * j/(w C^2); Re(conj(g) x) = g.x x.x + g.y x.y
      const double2 dc = sr_mul(dgdz, make_double2(0.0, 1.0 / (w * c * c)));
      sc += gv.x * dc.x + gv.y * dc.y;
      sr += gv.x * dgdz.x + gv.y * dgdz.y;
    }
    if (gC) gC[i] = sc;
    if (gR) gR[i] = sr;
  }
}

// ---------------------------------------------------------------------------------------
// host side: layouts, the internal per-frequency problem, launch sequences
// ---------------------------------------------------------------------------------------
struct SrBasisLayout {
  size_t vport, vpoint, vfreq, vbasis, T, tflag, tabs, S0h, S0l, Th, Tl, fl32, total;
  BasisLayout vb;
};

struct SrTapeLayout {
  size_t I, mu, Bop, plan, err, W, lu, perm, loss_part, status, total;
};

// The superposition's view of the route: one structure per frequency, 2 n0 real basis
// columns, the (configuration, external port) pairs as its configurations.
struct SrVirtual {
  std::vector<int32_t> port, freq;
  std::vector<int64_t> point;
  mts_problem pb;
  explicit SrVirtual(const mts_sparams* sp) {
    const int F = sp->n_freq, Kv = 2 * sp->n0;
    port.resize(F + 1);
    freq.resize(F + 1);
    point.resize(F + 1);
    for (int i = 0; i <= F; ++i) {
      port[i] = i * Kv;
      freq[i] = i;
      point[i] = (int64_t)i * sp->n_points;
    }
    std::memset(&pb, 0, sizeof(pb));
    pb.n_struct = F;
    pb.n_ports = F * Kv;
    pb.n_freq = F;
    pb.n_points = (int64_t)F * sp->n_points;
    pb.wire_radius = 1.0;
    pb.h_port_off = port.data();
    pb.h_point_off = point.data();
    pb.h_freq_off = freq.data();
  }
  void bind(const char* sbasis, const SrBasisLayout& L) {
    pb.port_off = reinterpret_cast<const int32_t*>(sbasis + L.vport);
    pb.point_off = reinterpret_cast<const int64_t*>(sbasis + L.vpoint);
    pb.freq_off = reinterpret_cast<const int32_t*>(sbasis + L.vfreq);
  }
};

static SrBasisLayout sr_basis_layout(const mts_sparams* sp, mts_precision prec, const SrVirtual& v) {
  SrBasisLayout L;
  const size_t F = (size_t)sp->n_freq, n0 = (size_t)sp->n0;
  size_t o = 0;
  L.vport = o; o += align256(4 * (F + 1));
  L.vpoint = o; o += align256(8 * (F + 1));
  L.vfreq = o; o += align256(4 * (F + 1));
  L.vb = basis_layout(&v.pb, prec);
  L.vbasis = o; o += align256(L.vb.total);
  L.T = o; o += align256(16 * F * n0 * n0);
  L.tflag = o; o += 256;
  L.tabs = o; o += align256(sizeof(SrTables));
  L.S0h = o; o += align256(8 * F * n0 * n0);
  L.S0l = o; o += align256(8 * F * n0 * n0);
  L.Th = o; o += align256(8 * F * n0 * n0);
  L.Tl = o; o += align256(8 * F * n0 * n0);
  L.fl32 = o; o += align256(8 * F * (size_t)sp->n_loss * n0);
  L.total = o;
  return L;
}

static SrTapeLayout sr_tape_layout(const mts_sparams* sp, int64_t n_cfg, mts_precision prec,
                                   const SrVirtual& v) {
  SrTapeLayout L;
  const size_t F = (size_t)sp->n_freq, n0 = (size_t)sp->n0, n1 = (size_t)sp->n1;
  const size_t nc = (size_t)n_cfg;
  size_t o = 0;
  L.I = o; o += align256(16 * nc * n1 * F * 2 * n0);
  L.mu = o; o += align256(16 * nc * n1 * F * 2 * n0);
  L.Bop = o; o += align256(2 * (size_t)bop_elems(&v.pb, n_cfg * (int64_t)n1, n_pieces(prec), nullptr));
  L.plan = o; o += plan_layout(sp->n_freq).bytes;
  L.err = o; o += 256;
  L.W = o; o += align256(16 * nc * F * n0 * n1);
  L.lu = o; o += align256((prec == MTS_FP64 ? 16 : 8) * nc * F * n0 * n0);
  L.perm = o; o += align256(4 * nc * F * n0);
  L.loss_part = o; o += align256(8 * nc * F);
  L.status = o; o += align256(4 * nc * F);
  L.total = o;
  return L;
}

static mts_status sr_validate(const mts_sparams* sp) {
  if (!sp) return MTS_EINVAL;
  if (sp->n0 < 1 || sp->n1 < 1 || sp->n_freq < 1 || sp->n_points < 0 || sp->n_svar < 1 ||
      sp->n_loss < 0)
    return MTS_EINVAL;
  if (sp->n0 > kSrMaxN0 || sp->n1 > kSrMaxN1 || sp->n_svar > kSrMaxSvar) return MTS_EUNSUPPORTED;
  if (!sp->h_svar_row || !sp->h_svar_col || !sp->S0) return MTS_EINVAL;
  if (sp->n_points > 0 && !sp->field) return MTS_EINVAL;
  if (sp->n_loss > 0 && (!sp->loss_idx || sp->n_points == 0)) return MTS_EINVAL;
  const int n = sp->n0 + sp->n1;
  std::vector<char> seen((size_t)n * n, 0);
  for (int i = 0; i < sp->n_svar; ++i) {
    const int r = sp->h_svar_row[i], c = sp->h_svar_col[i];
    if (r < 0 || r >= n || c < 0 || c >= n) return MTS_EINVAL;
    if (seen[(size_t)r * n + c]) return MTS_EINVAL;
    seen[(size_t)r * n + c] = 1;
  }
  return MTS_OK;
}

static mts_status sr_validate_prec(mts_precision prec) {
  return (prec == MTS_FP64 || prec == MTS_MIXED || prec == MTS_BF16) ? MTS_OK : MTS_EINVAL;
}

static bool sr_aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

static mts_status sr_validate_eval(const mts_sparams* sp, const mts_sroute_eval* ev) {
  if (!ev || ev->n_cfg < 0) return MTS_EINVAL;
  if (ev->n_cfg > 0 && !ev->svar) return MTS_EINVAL;
  if (ev->loss_mode != MTS_LOSS_ABS && ev->loss_mode != MTS_LOSS_COMPLEX) return MTS_EINVAL;
  if (!(ev->refine_tol >= 0.0) || !std::isfinite(ev->refine_tol) || ev->max_refine < 0)
    return MTS_EINVAL;
  if (ev->n_cfg * (int64_t)sp->n_freq > 0x7fffffffLL) return MTS_EUNSUPPORTED;  // grid x
  return MTS_OK;
}

static SrTables sr_build_tables(const mts_sparams* sp) {
  SrTables t;
  std::memset(&t, 0, sizeof(t));
  const int n0 = sp->n0;
  std::vector<int> cnt_r(n0 + 1, 0), cnt_c(n0 + 1, 0);
  for (int i = 0; i < sp->n_svar; ++i) {
    const int r = sp->h_svar_row[i], c = sp->h_svar_col[i];
    t.row[i] = (int16_t)r;
    t.col[i] = (int16_t)c;
    if (r < n0 && c < n0) {
      ++cnt_r[r + 1];
      ++cnt_c[c + 1];
    } else if (r < n0) {
      t.s12_row[t.n12] = (int16_t)r;
      t.s12_col[t.n12] = (int16_t)(c - n0);
      t.s12_var[t.n12] = (int16_t)i;
      ++t.n12;
    }
  }
  for (int i = 0; i < n0; ++i) {
    cnt_r[i + 1] += cnt_r[i];
    cnt_c[i + 1] += cnt_c[i];
  }
  for (int i = 0; i <= n0; ++i) {
    t.r_ptr[i] = (int16_t)cnt_r[i];
    t.c_ptr[i] = (int16_t)cnt_c[i];
  }
  std::vector<int> fr(cnt_r.begin(), cnt_r.end()), fc(cnt_c.begin(), cnt_c.end());
  for (int i = 0; i < sp->n_svar; ++i) {
    const int r = sp->h_svar_row[i], c = sp->h_svar_col[i];
    if (r < n0 && c < n0) {
      const int qr = fr[r]++, qc = fc[c]++;
      t.r_col[qr] = (int16_t)c;
      t.r_var[qr] = (int16_t)i;
      t.c_row[qc] = (int16_t)r;
      t.c_var[qc] = (int16_t)i;
      ++t.n11;
    }
  }
  return t;
}

static mts_status sr_cuda(cudaError_t e) { return e == cudaSuccess ? MTS_OK : MTS_ECUDA; }

constexpr size_t kSrMaxSmem = 227 * 1024;  // opt-in shared memory per CTA

template <typename LT>
static cudaError_t sr_launch_solve(const SrArgs& a, int64_t n_sys, cudaStream_t st) {
  size_t o[11];
  const size_t sm = sr_solve_smem<LT>(a.n0, a.n1, a.nS, o);
  if (sm > kSrMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(sr_solve_kernel<LT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  sr_solve_kernel<LT><<<(unsigned)n_sys, kSrThreads, sm, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <typename LT>
static cudaError_t sr_launch_adjoint(const SrArgs& a, int64_t n_sys, cudaStream_t st) {
  size_t o[14];
  const size_t sm = sr_adj_smem<LT>(a.n0, a.n1, a.nS, o);
  if (sm > kSrMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(sr_adjoint_kernel<LT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  sr_adjoint_kernel<LT><<<(unsigned)n_sys, kSrThreads, sm, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

static SrArgs sr_args(const mts_sparams* sp, mts_precision prec, const char* SB,
                      const SrBasisLayout& BL, const mts_sroute_eval* ev, char* T,
                      const SrTapeLayout& TL) {
  SrArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n0 = sp->n0;
  a.n1 = sp->n1;
  a.F = sp->n_freq;
  a.nS = sp->n_svar;
  a.L = sp->n_loss;
  a.loss_mode = ev->loss_mode;
  a.max_refine = ev->max_refine > 0 ? ev->max_refine : 8;
  a.tol = ev->refine_tol > 0.0 ? ev->refine_tol : 1e-8;
  a.n_cfg = ev->n_cfg;
  a.P = sp->n_points;
  a.sumFNv = (int64_t)sp->n_freq * 2 * sp->n0;
  a.S0 = reinterpret_cast<const double2*>(sp->S0);
  a.T = reinterpret_cast<const double2*>(SB + BL.T);
  a.tflag = reinterpret_cast<const int32_t*>(SB + BL.tflag);
  a.sc_const = reinterpret_cast<const double2*>(sp->sc_const);
  a.svar = reinterpret_cast<const double2*>(ev->svar);
  a.field = reinterpret_cast<const double2*>(sp->field);
  a.loss_idx = sp->loss_idx;
  a.target = sp->n_loss > 0 ? ev->target : nullptr;
  a.loss_weight = ev->loss_weight;
  a.loss_offset = reinterpret_cast<const double2*>(ev->loss_offset);
  a.tabs = reinterpret_cast<const SrTables*>(SB + BL.tabs);
  a.S0h = reinterpret_cast<const float2*>(SB + BL.S0h);
  a.S0l = reinterpret_cast<const float2*>(SB + BL.S0l);
  a.Th = reinterpret_cast<const float2*>(SB + BL.Th);
  a.Tl = reinterpret_cast<const float2*>(SB + BL.Tl);
  a.fl32 = reinterpret_cast<const float2*>(SB + BL.fl32);
  a.W = reinterpret_cast<double2*>(T + TL.W);
  a.lu = T + TL.lu;
  a.perm = reinterpret_cast<int32_t*>(T + TL.perm);
  a.Iv = reinterpret_cast<double*>(T + TL.I);
  a.loss_part = reinterpret_cast<double*>(T + TL.loss_part);
  a.status = reinterpret_cast<int32_t*>(T + TL.status);
  a.norm = (double)sp->n_freq * sp->n1 * sp->n_loss;
  return a;
}

}  // namespace mts

using namespace mts;

extern "C" {

size_t mts_sroute_basis_bytes(const mts_sparams* sp, mts_precision prec) {
  if (sr_validate(sp) != MTS_OK || sr_validate_prec(prec) != MTS_OK) return 0;
  SrVirtual v(sp);
  return sr_basis_layout(sp, prec, v).total;
}

mts_status mts_sroute_build(const mts_sparams* sp, mts_precision prec, void* sbasis,
                            size_t sbasis_bytes, mts_stream stream) {
  mts_status s = sr_validate(sp);
  if (s != MTS_OK) return s;
  if (sr_validate_prec(prec) != MTS_OK || !sbasis || !sr_aligned(sbasis)) return MTS_EINVAL;
  SrVirtual v(sp);
  const SrBasisLayout L = sr_basis_layout(sp, prec, v);
  if (sbasis_bytes < L.total) return MTS_EWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* SB = static_cast<char*>(sbasis);
  v.bind(SB, L);
  const int F = sp->n_freq, n0 = sp->n0;
  sr_voff_kernel<<<1, 256, 0, st>>>(F, 2 * n0, sp->n_points, (int32_t*)(SB + L.vport),
                                    (int64_t*)(SB + L.vpoint), (int32_t*)(SB + L.vfreq));
  note_launch();
  void* vb = SB + L.vbasis;
  cudaError_t e = launch_basis_tables(&v.pb, prec, vb, L.vb, st);
  if (e != cudaSuccess) return MTS_ECUDA;
  if (sp->n_points > 0) {
    DevTables t = dev_tables(vb, L.vb, F, F);
    const int64_t total = (int64_t)F * sp->n_points * n0;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 65536 ? (total + 255) / 256 : 65536);
    if (prec == MTS_FP64)
      sr_field_kernel<double><<<blocks, 256, 0, st>>>(
          F, sp->n_points, n0, reinterpret_cast<const double2*>(sp->field), t.pn_off,
          reinterpret_cast<double*>(static_cast<char*>(vb) + L.vb.H));
    else
      sr_field_kernel<float><<<blocks, 256, 0, st>>>(
          F, sp->n_points, n0, reinterpret_cast<const double2*>(sp->field), t.pn_off,
          reinterpret_cast<float*>(static_cast<char*>(vb) + L.vb.H));
    note_launch();
    e = launch_pack_a(&v.pb, prec, vb, L.vb, st);
    if (e != cudaSuccess) return MTS_ECUDA;
  }
  cudaMemsetAsync(SB + L.tflag, 0, 16, st);
  if (sp->sc_const) {
    sr_const_kernel<<<dim3(n0, F), 128, 0, st>>>(n0, sp->n1, reinterpret_cast<const double2*>(sp->S0),
                                                 reinterpret_cast<const double2*>(sp->sc_const),
                                                 reinterpret_cast<double2*>(SB + L.T),
                                                 reinterpret_cast<int32_t*>(SB + L.tflag));
    note_launch();
  }
  sr_tables_kernel<<<1, 256, 0, st>>>(sr_build_tables(sp), reinterpret_cast<SrTables*>(SB + L.tabs));
  note_launch();
  // double-float operands and FP32 loss rows of the FP32-factor kernels
  const int64_t nsq = (int64_t)F * n0 * n0;
  const unsigned sb = (unsigned)((nsq + 255) / 256 < 4096 ? (nsq + 255) / 256 : 4096);
  sr_split_kernel<<<sb, 256, 0, st>>>(nsq, reinterpret_cast<const double2*>(sp->S0),
                                      reinterpret_cast<float2*>(SB + L.S0h),
                                      reinterpret_cast<float2*>(SB + L.S0l));
  note_launch();
  if (sp->sc_const) {
    sr_split_kernel<<<sb, 256, 0, st>>>(nsq, reinterpret_cast<const double2*>(SB + L.T),
                                        reinterpret_cast<float2*>(SB + L.Th),
                                        reinterpret_cast<float2*>(SB + L.Tl));
    note_launch();
  }
  if (sp->n_loss > 0) {
    const int64_t nl = (int64_t)F * sp->n_loss * n0;
    sr_lossrows_kernel<<<(unsigned)((nl + 255) / 256 < 4096 ? (nl + 255) / 256 : 4096), 256, 0, st>>>(
        F, sp->n_points, sp->n_loss, n0, reinterpret_cast<const double2*>(sp->field), sp->loss_idx,
        reinterpret_cast<float2*>(SB + L.fl32));
    note_launch();
  }
  return sr_cuda(cudaGetLastError());
}

size_t mts_sroute_tape_bytes(const mts_sparams* sp, int64_t n_cfg, mts_precision prec) {
  if (sr_validate(sp) != MTS_OK || sr_validate_prec(prec) != MTS_OK || n_cfg < 0) return 0;
  SrVirtual v(sp);
  return sr_tape_layout(sp, n_cfg, prec, v).total;
}

mts_status mts_sroute_forward(const mts_sparams* sp, mts_precision prec, const void* sbasis,
                              const mts_sroute_eval* ev, void* B_out, double* W_out,
                              double* loss_out, void* tape, size_t tape_bytes,
                              mts_stream stream) {
  mts_status s = sr_validate(sp);
  if (s != MTS_OK) return s;
  if (sr_validate_prec(prec) != MTS_OK || !sbasis || !tape) return MTS_EINVAL;
  s = sr_validate_eval(sp, ev);
  if (s != MTS_OK) return s;
  if (loss_out && !ev->target) return MTS_EINVAL;
  SrVirtual v(sp);
  const SrBasisLayout BL = sr_basis_layout(sp, prec, v);
  const SrTapeLayout TL = sr_tape_layout(sp, ev->n_cfg, prec, v);
  if (tape_bytes < TL.total) return MTS_EWORKSPACE;
  if (ev->n_cfg == 0) return MTS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const char* SB = static_cast<const char*>(sbasis);
  char* T = static_cast<char*>(tape);
  v.bind(SB, BL);
  const int64_t n_cfg_v = ev->n_cfg * sp->n1;
  const int npieces = n_pieces(prec);
  const PlanLayout pl = plan_layout(sp->n_freq);
  cudaError_t e = cudaMemsetAsync(T + TL.err, 0, 16, st);
  if (e == cudaSuccess)
    e = launch_plan(&v.pb, n_cfg_v, npieces, kSimtSys, reinterpret_cast<int64_t*>(T + TL.plan + pl.bop_off),
                    reinterpret_cast<int64_t*>(T + TL.plan + pl.unit_off),
                    reinterpret_cast<int64_t*>(T + TL.plan + pl.lu_off),
                    reinterpret_cast<int64_t*>(T + TL.plan + pl.simt_off), st);
  if (e != cudaSuccess) return MTS_ECUDA;
  SrArgs a = sr_args(sp, prec, SB, BL, ev, T, TL);
  a.W_out = reinterpret_cast<double2*>(W_out);
  const int64_t n_sys = ev->n_cfg * sp->n_freq;
  e = prec == MTS_FP64 ? sr_launch_solve<double>(a, n_sys, st) : sr_launch_solve<float>(a, n_sys, st);
  if (e != cudaSuccess) return MTS_ECUDA;
  if (B_out && sp->n_points > 0) {
    const int Kv = 2 * sp->n0;
    if (npieces > 0) {
      const int64_t work = n_cfg_v * round_up(Kv, kChunkK);
      const unsigned gx = (unsigned)((work + 255) / 256 < 1024 ? (work + 255) / 256 : 1024);
      sr_pack_kernel<<<dim3(gx, sp->n_freq), 256, 0, st>>>(
          sp->n_freq, n_cfg_v, Kv, npieces, a.sumFNv,
          reinterpret_cast<const int64_t*>(T + TL.plan + pl.bop_off),
          reinterpret_cast<const double*>(T + TL.I), reinterpret_cast<__nv_bfloat16*>(T + TL.Bop));
      note_launch();
    }
    e = superpose_core(&v.pb, prec, SB + BL.vbasis, n_cfg_v, kSimtSys,
                       reinterpret_cast<const double*>(T + TL.I),
                       reinterpret_cast<const __nv_bfloat16*>(T + TL.Bop), T + TL.plan,
                       reinterpret_cast<int32_t*>(T + TL.err), B_out, st);
    if (e != cudaSuccess) return MTS_ECUDA;
  }
  if (loss_out) {
    sr_loss_kernel<<<(unsigned)((ev->n_cfg + 255) / 256), 256, 0, st>>>(
        ev->n_cfg, sp->n_freq, a.norm, reinterpret_cast<const double*>(T + TL.loss_part), loss_out);
    note_launch();
  }
  return sr_cuda(cudaGetLastError());
}

mts_status mts_sroute_backward(const mts_sparams* sp, mts_precision prec, const void* sbasis,
                               const mts_sroute_eval* ev, void* tape, size_t tape_bytes,
                               const void* grad_B, const double* grad_loss, double* grad_svar,
                               mts_stream stream) {
  mts_status s = sr_validate(sp);
  if (s != MTS_OK) return s;
  if (sr_validate_prec(prec) != MTS_OK || !sbasis || !tape || !grad_svar) return MTS_EINVAL;
  s = sr_validate_eval(sp, ev);
  if (s != MTS_OK) return s;
  if (grad_loss && !ev->target) return MTS_EINVAL;
  SrVirtual v(sp);
  const SrBasisLayout BL = sr_basis_layout(sp, prec, v);
  const SrTapeLayout TL = sr_tape_layout(sp, ev->n_cfg, prec, v);
  if (tape_bytes < TL.total) return MTS_EWORKSPACE;
  if (ev->n_cfg == 0) return MTS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const char* SB = static_cast<const char*>(sbasis);
  char* T = static_cast<char*>(tape);
  v.bind(SB, BL);
  SrArgs a = sr_args(sp, prec, SB, BL, ev, T, TL);
  a.grad_loss = grad_loss;
  a.grad_svar = reinterpret_cast<double2*>(grad_svar);
  cudaError_t e = cudaSuccess;
  if (grad_B && sp->n_points > 0) {
    FieldAdjArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.n_struct = sp->n_freq;
    fa.n_freq = sp->n_freq;
    fa.n_ports = v.pb.n_ports;
    fa.port_off = v.pb.port_off;
    fa.freq_off = v.pb.freq_off;
    fa.point_off = v.pb.point_off;
    fa.t = dev_tables(SB + BL.vbasis, BL.vb, sp->n_freq, sp->n_freq);
    fa.n_cfg = ev->n_cfg * sp->n1;
    fa.sumFN = a.sumFNv;
    fa.sumFP = (int64_t)sp->n_freq * sp->n_points;
    fa.H = SB + BL.vbasis + BL.vb.H;
    fa.grad_B = grad_B;
    fa.u = reinterpret_cast<double*>(T + TL.mu);
    e = launch_field_adjoint_rhs(fa, prec, 2 * sp->n0, st);
    if (e != cudaSuccess) return MTS_ECUDA;
    a.u = reinterpret_cast<const double2*>(T + TL.mu);
  }
  const int64_t n_sys = ev->n_cfg * sp->n_freq;
  e = prec == MTS_FP64 ? sr_launch_adjoint<double>(a, n_sys, st) : sr_launch_adjoint<float>(a, n_sys, st);
  return sr_cuda(e);
}

mts_status mts_sroute_status(const mts_sparams* sp, int64_t n_cfg, mts_precision prec,
                             const void* tape, int64_t* n_bad, mts_stream stream) {
  mts_status s = sr_validate(sp);
  if (s != MTS_OK) return s;
  if (sr_validate_prec(prec) != MTS_OK || !tape || n_cfg < 0) return MTS_EINVAL;
  SrVirtual v(sp);
  const SrTapeLayout TL = sr_tape_layout(sp, n_cfg, prec, v);
  char* T = const_cast<char*>(static_cast<const char*>(tape));
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* words = reinterpret_cast<int32_t*>(T + TL.err);
  if (launch_count_bad(reinterpret_cast<const int32_t*>(T + TL.status), n_cfg * sp->n_freq,
                       words + 1, st) != cudaSuccess)
    return MTS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MTS_ECUDA;
  int32_t h[2] = {0, 0};
  if (cudaMemcpy(h, words, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return MTS_ECUDA;
  if (n_bad) *n_bad = h[1];
  if (h[0] != 0) return MTS_ECUDA;
  return h[1] ? MTS_ENOCONV : MTS_OK;
}

mts_status mts_rc_reflection(int64_t n_cfg, int32_t n_freq, int32_t n_loads, const double* omega,
                             const double* R, const double* C, double Z0, int32_t svar_stride,
                             int32_t svar_offset, double* svar, mts_stream stream) {
  if (n_cfg < 0 || n_freq < 0 || n_loads < 0 || svar_offset < 0 ||
      svar_offset + n_loads > svar_stride || !(Z0 > 0.0) || !std::isfinite(Z0))
    return MTS_EINVAL;
  const int64_t total = n_cfg * n_freq * n_loads;
  if (total == 0) return MTS_OK;
  if (!omega || !C || !svar) return MTS_EINVAL;
  const unsigned blocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  sr_rc_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n_cfg, n_freq, n_loads, omega, R, C, Z0,
                                                         svar_stride, svar_offset,
                                                         reinterpret_cast<double2*>(svar));
  note_launch();
  return sr_cuda(cudaGetLastError());
}

mts_status mts_rc_reflection_vjp(int64_t n_cfg, int32_t n_freq, int32_t n_loads,
                                 const double* omega, const double* R, const double* C, double Z0,
                                 int32_t svar_stride, int32_t svar_offset,
                                 const double* grad_svar, double* grad_R, double* grad_C,
                                 mts_stream stream) {
  if (n_cfg < 0 || n_freq < 0 || n_loads < 0 || svar_offset < 0 ||
      svar_offset + n_loads > svar_stride || !(Z0 > 0.0) || !std::isfinite(Z0))
    return MTS_EINVAL;
  const int64_t total = n_cfg * n_loads;
  if (total == 0 || (!grad_R && !grad_C)) return MTS_OK;
  if (!C || (n_freq > 0 && (!omega || !grad_svar))) return MTS_EINVAL;
  const unsigned blocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  sr_rc_vjp_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
      n_cfg, n_freq, n_loads, omega, R, C, Z0, svar_stride, svar_offset,
      reinterpret_cast<const double2*>(grad_svar), grad_R, grad_C);
  note_launch();
  return sr_cuda(cudaGetLastError());
}

}  // extern "C"
