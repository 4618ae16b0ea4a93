// basis.cu -- (a) of the method: the Biot-Savart field basis H[p][k] (Bz at point p per
// ampere in loop k; paper Sec. I-A: circuit model plus Biot-Savart law for structures
// small against the wavelength) and the inductance coupling M (Eq. 12-13: self L on the
// diagonal, mutual M off it; here from Neumann partial inductances of straight wires).
//
// Kernels
//   tables_kernel        per-structure prefix tables into the basis buffer
//   basis_fp64_kernel    H in FP64 (one thread per point and loop)
//   basis_fp32_kernel    H in FP32 with loop-local coordinates; the loop's segments are
//                        staged in shared memory once per CTA (128 points x 1 loop);
//                        terms of segments closer to the point than one segment length
//                        are evaluated in FP64
//   inductance_kernel    M in FP64, one CTA per loop pair, deterministic tree reduction
//   hloss_kernel         rows of H at the loss points (FP64 and FP32 copies)
//   msplit_kernel        M = hi + lo in FP32 pairs for double-float residuals
//   pack_a_kernel        bf16 pieces of H in the swizzled tensor-core operand image
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mts {

// ---------------------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------------------
__global__ void tables_kernel(int n_struct, int n_freq, const int32_t* __restrict__ port_off,
                              const int64_t* __restrict__ point_off,
                              const int32_t* __restrict__ freq_off,
                              const int32_t* __restrict__ loss_off, int npieces, int64_t* nn,
                              int64_t* pn, int64_t* pnr, int64_t* ln, int64_t* fn, int64_t* fp,
                              int64_t* fl, int64_t* aop, int64_t* ptile, int64_t* pair,
                              int32_t* freq_struct, int32_t* cls_freq) {
  __shared__ int cls_base[kNumPortClasses];
  __shared__ int wcnt[8][kNumPortClasses];
  if (threadIdx.x == 0) {
    int64_t a = 0, b = 0, br = 0, c = 0, d = 0, e = 0, f = 0, g = 0, h = 0, q = 0;
    for (int s = 0; s < n_struct; ++s) {
      nn[s] = a; pn[s] = b; pnr[s] = br; ln[s] = c; fn[s] = d; fp[s] = e; fl[s] = f; aop[s] = g;
      ptile[s] = h; pair[s] = q;
      int64_t N = port_off[s + 1] - port_off[s];
      int64_t P = point_off[s + 1] - point_off[s];
      int64_t F = freq_off[s + 1] - freq_off[s];
      int64_t L = loss_off ? (loss_off[s + 1] - loss_off[s]) : 0;
      a += N * N; b += round_up(P * N, kHAlign); br += P * N; c += L * N; d += F * N; e += F * P;
      f += F * L;
      g += (int64_t)npieces * ((P + kTileP - 1) / kTileP * kTileP) * ((N + kChunkK - 1) / kChunkK * kChunkK);
      h += (P + kTileP - 1) / kTileP;
      q += N * (N + 1) / 2;
    }
    nn[n_struct] = a; pn[n_struct] = b; pnr[n_struct] = br; ln[n_struct] = c; fn[n_struct] = d;
    fp[n_struct] = e;
    fl[n_struct] = f; aop[n_struct] = g; ptile[n_struct] = h; pair[n_struct] = q;
  }
  for (int gi = threadIdx.x; gi < n_freq; gi += blockDim.x) {
    int lo = 0, hi = n_struct;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (freq_off[mid] <= gi) lo = mid; else hi = mid;
    }
    freq_struct[gi] = lo;
  }
  // frequencies grouped by the port class of their structure, ascending within a class
  // (stable partition: class counts, then ballot prefix sums over chunks of 256)
  if (threadIdx.x < kNumPortClasses) cls_base[threadIdx.x] = 0;
  __syncthreads();
  for (int gi = threadIdx.x; gi < n_freq; gi += blockDim.x) {
    int s = freq_struct[gi];
    atomicAdd(&cls_base[port_class(port_off[s + 1] - port_off[s])], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0;
    for (int c = 0; c < kNumPortClasses; ++c) {
      int n = cls_base[c];
      cls_base[c] = o;
      o += n;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int g0 = 0; g0 < n_freq; g0 += blockDim.x) {
    const int gi = g0 + threadIdx.x;
    int c = -1;
    if (gi < n_freq) {
      int s = freq_struct[gi];
      c = port_class(port_off[s + 1] - port_off[s]);
    }
    unsigned mine = 0u;
    for (int cc = 0; cc < kNumPortClasses; ++cc) {
      unsigned bal = __ballot_sync(0xffffffffu, c == cc);
      if (lane == 0) wcnt[w][cc] = __popc(bal);
      if (c == cc) mine = __popc(bal & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (c >= 0) {
      int o = cls_base[c] + (int)mine;
      for (int q = 0; q < w; ++q) o += wcnt[q][c];
      cls_freq[o] = gi;
    }
    __syncthreads();
    if (threadIdx.x < kNumPortClasses) {
      int t = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += wcnt[q][threadIdx.x];
      cls_base[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Biot-Savart: field of a straight segment r1 -> r2 carrying 1 A at the origin-shifted
// point (R1 = r1 - p, R2 = r2 - p):
//   B = mu0/(4 pi) (R1 x R2) (|R1| + |R2|) / (|R1||R2| (|R1||R2| + R1.R2)),
// of which one component is taken per field point (comp 0 = z, the paper's Bz; 1 = x; 2 = y),
// with |R1||R2| + R1.R2 = |R1 x R2|^2 / (|R1||R2| - R1.R2) when R1.R2 < 0 (no cancellation
// beside the span). Inside the wire (rho < rw, foot on the span) a uniform current gives a
// field linear in rho: the thin-wire value is scaled by rho^2/rw^2.
// ---------------------------------------------------------------------------------------
constexpr double kMu0Over4Pi = 1e-7;  // mu0/(4 pi) with mu0 = 4 pi 1e-7 H/m
// status bit of a component code outside {0, 1, 2} (its basis rows are NaN)
constexpr int32_t kBadComponent = 1 << 30;

__device__ inline double seg_b_f64(double ax, double ay, double az, double bx, double by,
                                   double bz, double rw, int comp) {
  // (ax,ay,az) = R1, (bx,by,bz) = R2
  double cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
  double n1 = sqrt(ax * ax + ay * ay + az * az);
  double n2 = sqrt(bx * bx + by * by + bz * bz);
  double dot = ax * bx + ay * by + az * bz;
  double c2 = cx * cx + cy * cy + cz * cz;
  double dx = bx - ax, dy = by - ay, dz = bz - az;
  double dd = dx * dx + dy * dy + dz * dz;
  if (dd == 0.0) return 0.0;
  double t = -(ax * dx + ay * dy + az * dz) / dd;
  double rho2 = c2 / dd;
  double scale = 1.0;
  if (t >= 0.0 && t <= 1.0 && rho2 < rw * rw) {
    if (rho2 == 0.0) return 0.0;
    scale = rho2 / (rw * rw);
  }
  double f;
  if (dot >= 0.0) {
    double den = n1 * n2 * (n1 * n2 + dot);
    if (den == 0.0) return 0.0;
    f = (n1 + n2) / den;
  } else {
    if (c2 == 0.0) return 0.0;
    f = (n1 + n2) * (n1 * n2 - dot) / (n1 * n2 * c2);
  }
  const double cc = comp == 1 ? cx : (comp == 2 ? cy : cz);
  return kMu0Over4Pi * cc * f * scale;
}

__device__ inline float seg_b_f32(float ax, float ay, float az, float dx, float dy, float dz,
                                  float rw2, int comp) {
  float bx = ax + dx, by = ay + dy, bz = az + dz;
  float cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
  float q1 = ax * ax + ay * ay + az * az;
  float q2 = bx * bx + by * by + bz * bz;
  float n1 = sqrtf(q1), n2 = sqrtf(q2);
  float dot = ax * bx + ay * by + az * bz;
  float c2 = cx * cx + cy * cy + cz * cz;
  float dd = dx * dx + dy * dy + dz * dz;
  float t = -(ax * dx + ay * dy + az * dz);
  float rho2dd = c2;  // rho^2 * dd
  float scale = 1.0f;
  if (t >= 0.0f && t <= dd && rho2dd < rw2 * dd) {
    if (rho2dd == 0.0f) return 0.0f;
    scale = rho2dd / (rw2 * dd);
  }
  float n12 = n1 * n2;
  float f;
  if (dot >= 0.0f) {
    float den = n12 * (n12 + dot);
    if (den == 0.0f) return 0.0f;
    f = (n1 + n2) / den;
  } else {
    if (c2 == 0.0f) return 0.0f;
    f = (n1 + n2) * (n12 - dot) / (n12 * c2);
  }
  const float cc = comp == 1 ? cx : (comp == 2 ? cy : cz);
  return cc * f * scale;  // times mu0/(4 pi) by the caller
}

__global__ void basis_fp64_kernel(int n_struct, const int64_t* __restrict__ point_off,
                                  const int32_t* __restrict__ port_off,
                                  const int32_t* __restrict__ loop_vtx_off,
                                  const double* __restrict__ vx, const double* __restrict__ vy,
                                  const double* __restrict__ vz, const double* __restrict__ px,
                                  const double* __restrict__ py, const double* __restrict__ pz,
                                  const int8_t* __restrict__ pcomp, double rw, int64_t n_points,
                                  const int64_t* __restrict__ pn_off, double* __restrict__ H,
                                  int32_t* __restrict__ status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (p >= n_points) return;
  int s = find_struct_i64(point_off, n_struct, p);
  int N = port_off[s + 1] - port_off[s];
  if (k >= N) return;
  int loop = port_off[s] + k;
  int a = loop_vtx_off[loop], b = loop_vtx_off[loop + 1];
  double x = px[p], y = py[p], z = pz[p];
  const int comp = pcomp != nullptr ? pcomp[p] : 0;
  double acc = 0.0;
  for (int v = a; v < b; ++v) {
    int w = (v + 1 < b) ? v + 1 : a;
    acc += seg_b_f64(vx[v] - x, vy[v] - y, vz[v] - z, vx[w] - x, vy[w] - y, vz[w] - z, rw, comp);
  }
  if (comp < 0 || comp > 2) {
    atomicOr(status, kBadComponent);
    acc = __longlong_as_double(0x7ff8000000000000LL);
  }
  H[pn_off[s] + (p - point_off[s]) * N + k] = acc;
}

// FP32 basis: CTA = 128 points of one structure x one loop. The loop's segments are staged
// in shared memory in loop-local FP32 coordinates (relative to the loop's first vertex),
// in chunks of kSegChunk. Each thread accumulates with compensated (Kahan) summation.
constexpr int kSegChunk = 256;

__global__ void __launch_bounds__(128) basis_fp32_kernel(
    int n_struct, const int64_t* __restrict__ point_off, const int32_t* __restrict__ port_off,
    const int32_t* __restrict__ loop_vtx_off, const double* __restrict__ vx,
    const double* __restrict__ vy, const double* __restrict__ vz, const double* __restrict__ px,
    const double* __restrict__ py, const double* __restrict__ pz,
    const int8_t* __restrict__ pcomp, double rw, const int64_t* __restrict__ ptile_off,
    const int64_t* __restrict__ pn_off, float* __restrict__ H, int32_t* __restrict__ status) {
  __shared__ float s_seg[6][kSegChunk];  // ax, ay, az (start), dx, dy, dz
  __shared__ float s_len2[kSegChunk];
  int64_t tile = blockIdx.x;
  int k = blockIdx.y;
  int s = find_struct_i64(ptile_off, n_struct, tile);
  int N = port_off[s + 1] - port_off[s];
  if (k >= N) return;  // whole CTA
  int64_t P = point_off[s + 1] - point_off[s];
  int64_t lp = (tile - ptile_off[s]) * kTileP + threadIdx.x;
  bool valid = lp < P;
  int64_t p = point_off[s] + (valid ? lp : 0);
  int loop = port_off[s] + k;
  int a = loop_vtx_off[loop], b = loop_vtx_off[loop + 1];
  double ox = vx[a], oy = vy[a], oz = vz[a];
  double xd = px[p], yd = py[p], zd = pz[p];
  const int fc = pcomp != nullptr ? pcomp[p] : 0;  // field component
  float x = (float)(xd - ox), y = (float)(yd - oy), z = (float)(zd - oz);
  float rw2 = (float)(rw * rw);
  float acc = 0.0f, comp = 0.0f;
  double acc64 = 0.0;  // near-field terms
  int nseg = b - a;
  for (int c0 = 0; c0 < nseg; c0 += kSegChunk) {
    int cn = min(kSegChunk, nseg - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) {
      int v = a + c0 + i;
      int w = (v + 1 < b) ? v + 1 : a;
      float sx = (float)(vx[v] - ox), sy = (float)(vy[v] - oy), sz = (float)(vz[v] - oz);
      float dx = (float)(vx[w] - vx[v]), dy = (float)(vy[w] - vy[v]), dz = (float)(vz[w] - vz[v]);
      s_seg[0][i] = sx; s_seg[1][i] = sy; s_seg[2][i] = sz;
      s_seg[3][i] = dx; s_seg[4][i] = dy; s_seg[5][i] = dz;
      s_len2[i] = dx * dx + dy * dy + dz * dz;
    }
    __syncthreads();
    for (int i = 0; i < cn; ++i) {
      float ax = s_seg[0][i] - x, ay = s_seg[1][i] - y, az = s_seg[2][i] - z;
      float dx = s_seg[3][i], dy = s_seg[4][i], dz = s_seg[5][i];
      float len2 = s_len2[i];
      // distance^2 from the point to the segment (closest point on the span)
      float t = -(ax * dx + ay * dy + az * dz);
      float q1 = ax * ax + ay * ay + az * az;
      float dist2;
      if (t <= 0.0f) dist2 = q1;
      else if (t >= len2) {
        float bx = ax + dx, by = ay + dy, bz = az + dz;
        dist2 = bx * bx + by * by + bz * bz;
      } else {
        dist2 = q1 - t * t / len2;
      }
      if (dist2 < len2) {
        int v = a + c0 + i;
        int w = (v + 1 < b) ? v + 1 : a;
        acc64 += seg_b_f64(vx[v] - xd, vy[v] - yd, vz[v] - zd, vx[w] - xd, vy[w] - yd,
                           vz[w] - zd, rw, fc);
      } else {
        float term = seg_b_f32(ax, ay, az, dx, dy, dz, rw2, fc);
        float yk = term - comp;
        float tk = acc + yk;
        comp = (tk - acc) - yk;
        acc = tk;
      }
    }
  }
  if (valid) {
    double v = (double)acc * kMu0Over4Pi + acc64;
    if (fc < 0 || fc > 2) {
      atomicOr(status, kBadComponent);
      v = __longlong_as_double(0x7ff8000000000000LL);
    }
    H[pn_off[s] + lp * N + k] = (float)v;
  }
}

// ---------------------------------------------------------------------------------------
// Partial inductance of two straight filaments (Neumann integral), FP64.
//   perpendicular: 0;  parallel at offset d > 0, spans [a1,a2], [b1,b2] along the common
//   direction, sign s = +-1 for equal/opposite directions:
//     s mu0/(4 pi) [G(a2-b1) - G(a1-b1) - G(a2-b2) + G(a1-b2)],
//     G(u) = u asinh(u/d) - sqrt(u^2 + d^2);
//   collinear, non-overlapping: G replaced by its d -> 0 form |u| ln|u| - |u|;
//   a segment with itself: mu0 l/(2 pi) (ln(2l/rw) - 1).
//   oblique (neither parallel nor perpendicular) and not touching: the Neumann integral
//     mu0/(4 pi) (u1.u2) int int ds dt / |r1(s) - r2(t)| with the inner integral in closed
//     form (ln((R1 + l2 - t0)/(R0 - t0)), cancelling factors rewritten through rho^2) and the
//     outer one by a composite 16-point Gauss-Legendre rule on m = min(8, ceil(l1/d))
//     equal panels, d the smallest end-point-to-segment distance.
//   oblique and sharing an end point O (a corner of a non-rectilinear polygon), far end
//     points P, Q, lengths l = |OP|, m = |OQ|, R = |PQ|: two rays from O at angle e have
//     distance sqrt(s^2 + t^2 - 2 s t cos e), whose double integral is
//     F = 2 [l atanh(m / (l + R)) + m atanh(l / (m + R))]; M = mu0/(4 pi) (u1.u2) F.
// Returns 0, or 2 (overlapping collinear pair) with value 0.
// ---------------------------------------------------------------------------------------
struct GaussRule16 {
  double x[16], w[16];
};

// 16-point Gauss-Legendre rule on [-1, 1] (host): roots of P_16 by Newton's method with
// the three-term recurrence, weights 2 / ((1 - x^2) P_16'(x)^2).
static GaussRule16 gauss_legendre16() {
  GaussRule16 g;
  const int n = 16;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    g.x[i] = z;
    g.w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return g;
}

__device__ inline double inv_distance_line(double px, double py, double pz, double b0x,
                                           double b0y, double b0z, double ux, double uy,
                                           double uz, double l2) {
  const double w0x = px - b0x, w0y = py - b0y, w0z = pz - b0z;
  const double t0 = w0x * ux + w0y * uy + w0z * uz;
  const double R0 = sqrt(w0x * w0x + w0y * w0y + w0z * w0z);
  const double w1x = w0x - l2 * ux, w1y = w0y - l2 * uy, w1z = w0z - l2 * uz;
  const double R1 = sqrt(w1x * w1x + w1y * w1y + w1z * w1z);
  const double a = l2 - t0;
  if (t0 <= 0.0) return log((R1 + a) / (R0 - t0));
  if (a < 0.0) return log((R0 + t0) / (R1 - a));
  const double rho2 = R0 * R0 - t0 * t0;
  return log((R1 + a) * (R0 + t0) / rho2);
}

__device__ inline double point_segment_distance(double px, double py, double pz, double ax,
                                                double ay, double az, double bx, double by,
                                                double bz) {
  const double dx = bx - ax, dy = by - ay, dz = bz - az;
  const double wx = px - ax, wy = py - ay, wz = pz - az;
  const double dd = dx * dx + dy * dy + dz * dz;
  double t = dd > 0.0 ? (wx * dx + wy * dy + wz * dz) / dd : 0.0;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double ex = wx - t * dx, ey = wy - t * dy, ez = wz - t * dz;
  return sqrt(ex * ex + ey * ey + ez * ez);
}

__device__ double pair_quadrature(double s1x, double s1y, double s1z, double e1x, double e1y,
                                  double e1z, double s2x, double s2y, double s2z, double e2x,
                                  double e2y, double e2z, const GaussRule16& g) {
  const double d1x = e1x - s1x, d1y = e1y - s1y, d1z = e1z - s1z;
  const double d2x = e2x - s2x, d2y = e2y - s2y, d2z = e2z - s2z;
  const double l1 = sqrt(d1x * d1x + d1y * d1y + d1z * d1z);
  const double l2 = sqrt(d2x * d2x + d2y * d2y + d2z * d2z);
  const double ux = d2x / l2, uy = d2y / l2, uz = d2z / l2;
  const double cosang = (d1x * d2x + d1y * d2y + d1z * d2z) / (l1 * l2);
  double d = point_segment_distance(s1x, s1y, s1z, s2x, s2y, s2z, e2x, e2y, e2z);
  d = fmin(d, point_segment_distance(e1x, e1y, e1z, s2x, s2y, s2z, e2x, e2y, e2z));
  d = fmin(d, point_segment_distance(s2x, s2y, s2z, s1x, s1y, s1z, e1x, e1y, e1z));
  d = fmin(d, point_segment_distance(e2x, e2y, e2z, s1x, s1y, s1z, e1x, e1y, e1z));
  int m = 8;
  if (d > 0.0) {
    const double mm = ceil(l1 / d);
    m = mm < 1.0 ? 1 : (mm > 8.0 ? 8 : (int)mm);
  }
  double acc = 0.0;
  for (int q = 0; q < m; ++q)
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const double sp = (q + 0.5 * (g.x[i] + 1.0)) / m;
      acc += g.w[i] * inv_distance_line(s1x + sp * d1x, s1y + sp * d1y, s1z + sp * d1z, s2x,
                                        s2y, s2z, ux, uy, uz, l2);
    }
  return kMu0Over4Pi * cosang * 0.5 * (l1 / m) * acc;
}

__device__ inline double dist3(double ax, double ay, double az, double bx, double by, double bz) {
  return sqrt((ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz));
}

// Neumann integral of two filaments sharing the end point O (far end points P and Q),
// cosang the cosine between the two current directions.
__device__ inline double touching_pair(double ox, double oy, double oz, double px, double py,
                                       double pz, double qx, double qy, double qz,
                                       double cosang) {
  const double l = dist3(px, py, pz, ox, oy, oz), m = dist3(qx, qy, qz, ox, oy, oz);
  const double R = dist3(px, py, pz, qx, qy, qz);
  return kMu0Over4Pi * cosang * 2.0 * (l * atanh(m / (l + R)) + m * atanh(l / (m + R)));
}

__device__ inline double Gpar(double u, double d) { return u * asinh(u / d) - sqrt(u * u + d * d); }
__device__ inline double Gcol(double u) {
  double a = fabs(u);
  return a == 0.0 ? 0.0 : a * log(a) - a;
}

__device__ int pair_inductance(double s1x, double s1y, double s1z, double e1x, double e1y,
                               double e1z, double s2x, double s2y, double s2z, double e2x,
                               double e2y, double e2z, double rw, bool self, double* out,
                               const GaussRule16& g) {
  double d1x = e1x - s1x, d1y = e1y - s1y, d1z = e1z - s1z;
  double d2x = e2x - s2x, d2y = e2y - s2y, d2z = e2z - s2z;
  double l1 = sqrt(d1x * d1x + d1y * d1y + d1z * d1z);
  double l2 = sqrt(d2x * d2x + d2y * d2y + d2z * d2z);
  *out = 0.0;
  if (l1 == 0.0 || l2 == 0.0) return 0;
  if (self) {
    *out = 2.0 * kMu0Over4Pi * l1 * (log(2.0 * l1 / rw) - 1.0);
    return 0;
  }
  double dot = d1x * d2x + d1y * d2y + d1z * d2z;
  double cx = d1y * d2z - d1z * d2y, cy = d1z * d2x - d1x * d2z, cz = d1x * d2y - d1y * d2x;
  double cr = sqrt(cx * cx + cy * cy + cz * cz);
  double tol = 1e-12 * l1 * l2;
  if (fabs(dot) <= tol) return 0;
  if (cr > tol) {  // oblique
    const double e2 = 1e-24 * (l1 + l2) * (l1 + l2);
    const double c = dot / (l1 * l2);
    auto d2 = [](double ax, double ay, double az, double bx, double by, double bz) {
      return (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
    };
    if (d2(s1x, s1y, s1z, s2x, s2y, s2z) <= e2)
      *out = touching_pair(s1x, s1y, s1z, e1x, e1y, e1z, e2x, e2y, e2z, c);
    else if (d2(s1x, s1y, s1z, e2x, e2y, e2z) <= e2)
      *out = touching_pair(s1x, s1y, s1z, e1x, e1y, e1z, s2x, s2y, s2z, c);
    else if (d2(e1x, e1y, e1z, s2x, s2y, s2z) <= e2)
      *out = touching_pair(e1x, e1y, e1z, s1x, s1y, s1z, e2x, e2y, e2z, c);
    else if (d2(e1x, e1y, e1z, e2x, e2y, e2z) <= e2)
      *out = touching_pair(e1x, e1y, e1z, s1x, s1y, s1z, s2x, s2y, s2z, c);
    else
      *out = pair_quadrature(s1x, s1y, s1z, e1x, e1y, e1z, s2x, s2y, s2z, e2x, e2y, e2z, g);
    return 0;
  }
  double ux = d1x / l1, uy = d1y / l1, uz = d1z / l1;
  double wx = s2x - s1x, wy = s2y - s1y, wz = s2z - s1z;
  double bs = wx * ux + wy * uy + wz * uz;
  double be = (e2x - s1x) * ux + (e2y - s1y) * uy + (e2z - s1z) * uz;
  double qx = wx - bs * ux, qy = wy - bs * uy, qz = wz - bs * uz;
  double dist = sqrt(qx * qx + qy * qy + qz * qz);
  double b1 = fmin(bs, be), b2 = fmax(bs, be);
  double a1 = 0.0, a2 = l1;
  double v;
  if (dist <= 1e-12 * (l1 + l2)) {
    // spans that meet within rounding of their lengths are the touching case of G0
    const double ov = 1e-12 * (l1 + l2);
    if (b1 < a2 - ov && a1 < b2 - ov) return 2;
    v = Gcol(a2 - b1) - Gcol(a1 - b1) - Gcol(a2 - b2) + Gcol(a1 - b2);
  } else {
    v = Gpar(a2 - b1, dist) - Gpar(a1 - b1, dist) - Gpar(a2 - b2, dist) + Gpar(a1 - b2, dist);
  }
  *out = (dot > 0.0 ? 1.0 : -1.0) * kMu0Over4Pi * v;
  return 0;
}

constexpr int kIndThreads = 256;

__global__ void __launch_bounds__(kIndThreads) inductance_kernel(
    int n_struct, const int32_t* __restrict__ port_off, const int32_t* __restrict__ loop_vtx_off,
    const double* __restrict__ vx, const double* __restrict__ vy, const double* __restrict__ vz,
    const double* __restrict__ L_self, double rw, const int64_t* __restrict__ pair_off,
    const int64_t* __restrict__ nn_off, double* __restrict__ M, int32_t* status,
    GaussRule16 gauss) {
  __shared__ double red[kIndThreads];
  int64_t q = blockIdx.x;
  int s = find_struct_i64(pair_off, n_struct, q);
  int N = port_off[s + 1] - port_off[s];
  // loop pair (k, l), k <= l, from the triangular index t = q - pair_off[s]
  int64_t t = q - pair_off[s];
  int k = 0;
  while (t >= N - k) { t -= N - k; ++k; }
  int l = k + (int)t;
  int lk = port_off[s] + k, ll = port_off[s] + l;
  double acc = 0.0;
  int st = 0;
  if (k == l && L_self != nullptr) {
    acc = (threadIdx.x == 0) ? L_self[lk] : 0.0;
  } else {
    int ka = loop_vtx_off[lk], kb = loop_vtx_off[lk + 1];
    int la = loop_vtx_off[ll], lb = loop_vtx_off[ll + 1];
    int nk = kb - ka, nl = lb - la;
    int64_t npairs = (int64_t)nk * nl;
    for (int64_t e = threadIdx.x; e < npairs; e += blockDim.x) {
      int i = ka + (int)(e / nl), j = la + (int)(e % nl);
      int ie = (i + 1 < kb) ? i + 1 : ka;
      int je = (j + 1 < lb) ? j + 1 : la;
      double m;
      int r = pair_inductance(vx[i], vy[i], vz[i], vx[ie], vy[ie], vz[ie], vx[j], vy[j], vz[j],
                              vx[je], vy[je], vz[je], rw, (k == l && i == j), &m, gauss);
      if (r && !st) st = r;
      acc += m;
    }
  }
  if (st) atomicOr(status, 1 << st);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kIndThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* Ms = M + nn_off[s];
    Ms[k * N + l] = red[0];
    Ms[l * N + k] = red[0];
  }
}

// ---------------------------------------------------------------------------------------
// derived arrays
// ---------------------------------------------------------------------------------------
template <typename HT>
__global__ void hloss_kernel(int n_struct, int n_loss, const int32_t* __restrict__ loss_off,
                             const int64_t* __restrict__ loss_idx,
                             const int32_t* __restrict__ port_off,
                             const int64_t* __restrict__ point_off,
                             const int64_t* __restrict__ pn_off,
                             const int64_t* __restrict__ ln_off, const HT* __restrict__ H,
                             double* __restrict__ Hl64, float* __restrict__ Hl32,
                             float* __restrict__ HlT32) {
  int l = blockIdx.x;
  if (l >= n_loss) return;
  int s = find_struct_i32(loss_off, n_struct, l);
  int N = port_off[s + 1] - port_off[s];
  int64_t lp = loss_idx[l] - point_off[s];
  int ll = l - loss_off[s];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double h = (double)H[pn_off[s] + lp * N + k];
    Hl64[ln_off[s] + (int64_t)ll * N + k] = h;
    Hl32[ln_off[s] + (int64_t)ll * N + k] = (float)h;
    HlT32[ln_off[s] + (int64_t)k * (loss_off[s + 1] - loss_off[s]) + ll] = (float)h;
  }
}

__global__ void msplit_kernel(int64_t n, const double* __restrict__ M, float* __restrict__ hi,
                              float* __restrict__ lo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m = M[i];
  float h = (float)m;
  hi[i] = h;
  lo[i] = (float)(m - (double)h);
}

// bf16 pieces of H: x = x0 + x1 + x2 with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)
// (exact in FP32 arithmetic), written into the swizzled operand image; padding rows and K
// columns are zero.
__global__ void pack_a_kernel(int n_struct, const int64_t* __restrict__ ptile_off,
                              const int32_t* __restrict__ port_off,
                              const int64_t* __restrict__ point_off,
                              const int64_t* __restrict__ pn_off,
                              const int64_t* __restrict__ aop_off, const float* __restrict__ H,
                              int npieces, __nv_bfloat16* __restrict__ A) {
  int64_t tile = blockIdx.x;
  int s = find_struct_i64(ptile_off, n_struct, tile);
  int N = port_off[s + 1] - port_off[s];
  int64_t P = point_off[s + 1] - point_off[s];
  int nkc = (N + kChunkK - 1) / kChunkK;
  int64_t nptile = ptile_off[s + 1] - ptile_off[s];
  int64_t pt = tile - ptile_off[s];
  const float* Hs = H + pn_off[s];
  char* base = reinterpret_cast<char*>(A + aop_off[s]);
  for (int e = threadIdx.x; e < kTileP * nkc * kChunkK; e += blockDim.x) {
    int r = e / (nkc * kChunkK);
    int kg = e % (nkc * kChunkK);
    int kc = kg / kChunkK, kk = kg % kChunkK;
    int64_t p = pt * kTileP + r;
    float x = (p < P && kg < N) ? Hs[p * N + kg] : 0.0f;
    float rem = x;
    for (int q = 0; q < npieces; ++q) {
      __nv_bfloat16 h = __float2bfloat16_rn(rem);
      rem = rem - __bfloat162float(h);
      size_t tile_bytes = (size_t)kTileP * kChunkK * 2;
      size_t off = ((size_t)(q * nptile + pt) * nkc + kc) * tile_bytes + swz128(r, kk);
      *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
    }
  }
}

template <typename HT>
__global__ void export_h_kernel(int64_t n, int n_struct, const int64_t* __restrict__ pn_off,
                                const int64_t* __restrict__ pnr_off, const HT* __restrict__ H,
                                double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = find_struct_i64(pnr_off, n_struct, i);  // unpadded position -> structure
  out[i] = (double)H[pn_off[s] + (i - pnr_off[s])];
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_basis_tables(const mts_problem* pb, mts_precision prec, void* basis,
                                const BasisLayout& bl, cudaStream_t st) {
  char* B = static_cast<char*>(basis);
  TableLayout tl = table_layout(pb->n_struct, pb->n_freq);
  char* T = B + bl.tables;
  int npieces = n_pieces(prec);
  cudaMemsetAsync(B + bl.status, 0, 16, st);
  tables_kernel<<<1, 256, 0, st>>>(
      pb->n_struct, pb->n_freq, pb->port_off, pb->point_off, pb->freq_off, pb->loss_off, npieces,
      (int64_t*)(T + tl.nn_off), (int64_t*)(T + tl.pn_off), (int64_t*)(T + tl.pnr_off),
      (int64_t*)(T + tl.ln_off),
      (int64_t*)(T + tl.fn_off), (int64_t*)(T + tl.fp_off), (int64_t*)(T + tl.fl_off),
      (int64_t*)(T + tl.aop_off), (int64_t*)(T + tl.ptile_off), (int64_t*)(T + tl.pair_off),
      (int32_t*)(T + tl.freq_struct), (int32_t*)(T + tl.cls_freq));
  note_launch();
  return cudaGetLastError();
}

static int64_t point_tiles(const mts_problem* pb) {
  int64_t ntiles = 0;
  for (int s = 0; s < pb->n_struct; ++s)
    ntiles += (pb->h_point_off[s + 1] - pb->h_point_off[s] + kTileP - 1) / kTileP;
  return ntiles;
}

cudaError_t launch_pack_a(const mts_problem* pb, mts_precision prec, void* basis,
                          const BasisLayout& bl, cudaStream_t st) {
  const int npieces = n_pieces(prec);
  const int64_t ntiles = point_tiles(pb);
  if (npieces == 0 || ntiles == 0) return cudaSuccess;
  char* B = static_cast<char*>(basis);
  DevTables t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  pack_a_kernel<<<(unsigned)ntiles, 256, 0, st>>>(pb->n_struct, t.ptile_off, pb->port_off,
                                                  pb->point_off, t.pn_off, t.aop_off,
                                                  (const float*)(B + bl.H), npieces,
                                                  (__nv_bfloat16*)(B + bl.Aop));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_build_basis(const mts_problem* pb, mts_precision prec, void* basis,
                               const BasisLayout& bl, const ProblemSums& ps, cudaStream_t st) {
  char* B = static_cast<char*>(basis);
  cudaError_t e = launch_basis_tables(pb, prec, basis, bl, st);
  if (e != cudaSuccess) return e;
  DevTables t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  // host copies of the tile and pair counts
  int64_t ntiles = 0, npairs = 0;
  for (int s = 0; s < pb->n_struct; ++s) {
    int64_t P = pb->h_point_off[s + 1] - pb->h_point_off[s];
    int64_t N = pb->h_port_off[s + 1] - pb->h_port_off[s];
    ntiles += (P + kTileP - 1) / kTileP;
    npairs += N * (N + 1) / 2;
  }
  if (prec == MTS_FP64) {
    dim3 grid(nblk(pb->n_points, 128), ps.max_ports);
    basis_fp64_kernel<<<grid, 128, 0, st>>>(pb->n_struct, pb->point_off, pb->port_off,
                                            pb->loop_vtx_off, pb->vx, pb->vy, pb->vz, pb->px,
                                            pb->py, pb->pz, pb->pcomp, pb->wire_radius,
                                            pb->n_points, t.pn_off, (double*)(B + bl.H),
                                            (int32_t*)(B + bl.status));
  } else {
    dim3 grid((unsigned)ntiles, ps.max_ports);
    basis_fp32_kernel<<<grid, 128, 0, st>>>(pb->n_struct, pb->point_off, pb->port_off,
                                            pb->loop_vtx_off, pb->vx, pb->vy, pb->vz, pb->px,
                                            pb->py, pb->pz, pb->pcomp, pb->wire_radius,
                                            t.ptile_off, t.pn_off, (float*)(B + bl.H),
                                            (int32_t*)(B + bl.status));
  }
  note_launch();
  inductance_kernel<<<(unsigned)npairs, kIndThreads, 0, st>>>(
      pb->n_struct, pb->port_off, pb->loop_vtx_off, pb->vx, pb->vy, pb->vz, pb->L_self,
      pb->wire_radius, t.pair_off, t.nn_off, (double*)(B + bl.M64), (int32_t*)(B + bl.status),
      gauss_legendre16());
  note_launch();
  msplit_kernel<<<nblk(ps.sumNN, 256), 256, 0, st>>>(ps.sumNN, (const double*)(B + bl.M64),
                                                      (float*)(B + bl.M32hi),
                                                      (float*)(B + bl.M32lo));
  note_launch();
  if (pb->n_loss > 0) {
    if (prec == MTS_FP64)
      hloss_kernel<double><<<pb->n_loss, 128, 0, st>>>(
          pb->n_struct, pb->n_loss, pb->loss_off, pb->loss_idx, pb->port_off, pb->point_off,
          t.pn_off, t.ln_off, (const double*)(B + bl.H), (double*)(B + bl.Hloss64),
          (float*)(B + bl.Hloss32), (float*)(B + bl.HlossT32));
    else
      hloss_kernel<float><<<pb->n_loss, 128, 0, st>>>(
          pb->n_struct, pb->n_loss, pb->loss_off, pb->loss_idx, pb->port_off, pb->point_off,
          t.pn_off, t.ln_off, (const float*)(B + bl.H), (double*)(B + bl.Hloss64),
          (float*)(B + bl.Hloss32), (float*)(B + bl.HlossT32));
    note_launch();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pack_a(pb, prec, basis, bl, st);
}

cudaError_t launch_export_basis(const mts_problem* pb, mts_precision prec, const void* basis,
                                const BasisLayout& bl, const ProblemSums& ps, double* H_out,
                                double* M_out, cudaStream_t st) {
  const char* B = static_cast<const char*>(basis);
  if (H_out && ps.sumPNraw > 0) {
    DevTables t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
    if (prec == MTS_FP64)
      export_h_kernel<double><<<nblk(ps.sumPNraw, 256), 256, 0, st>>>(
          ps.sumPNraw, pb->n_struct, t.pn_off, t.pnr_off, (const double*)(B + bl.H), H_out);
    else
      export_h_kernel<float><<<nblk(ps.sumPNraw, 256), 256, 0, st>>>(
          ps.sumPNraw, pb->n_struct, t.pn_off, t.pnr_off, (const float*)(B + bl.H), H_out);
    note_launch();
  }
  if (M_out)
    cudaMemcpyAsync(M_out, B + bl.M64, sizeof(double) * ps.sumNN, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

}  // namespace mts
