// solve_common.cuh -- device helpers shared by the FP64 and mixed-precision solve kernels.
#pragma once
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

// System of launch index li: li itself, or configuration li / gcount at the frequency
// glist[li % gcount] of the launch's port class.
__device__ inline int64_t launch_sys(const SolveArgs& a, int64_t li) {
  if (a.glist == nullptr) return li;
  const int64_t b = li / a.gcount;
  return b * a.n_freq + a.glist[li - b * a.gcount];
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


// error-free product and sum on the FP32 pipe: (sh, sl) += (ah + al) * (bh + bl), dropping
// al * bl (2^-48 relative)
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

}  // namespace mts
