// superpose.cu -- (c) of the method: B = H I (paper Eq. 7), the field of every
// configuration and frequency as the superposition of the per-port basis fields.
//
//   plan_kernel          per-call tables: bases of the tensor-core operand of I, the
//                        prefix of GEMM work units and the bases of the LU factor scratch
//                        per structure
//   superpose_fp64_kernel  FP64 SIMT (MTS_FP64): CTA = 128 points x 64 systems
//   The tensor-core kernel for MTS_MIXED / MTS_BF16 lives in superpose_tc.cu.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mts {

__global__ void plan_kernel(int n_struct, int64_t n_cfg, const int32_t* __restrict__ port_off,
                            const int64_t* __restrict__ point_off,
                            const int32_t* __restrict__ freq_off, int npieces,
                            int64_t* bop_off, int64_t* unit_off, int64_t* lu_off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t a = 0, u = 0, f = 0;
  for (int s = 0; s < n_struct; ++s) {
    bop_off[s] = a;
    unit_off[s] = u;
    lu_off[s] = f;
    int64_t N = port_off[s + 1] - port_off[s];
    int64_t P = point_off[s + 1] - point_off[s];
    int64_t F = freq_off[s + 1] - freq_off[s];
    int64_t nn = (2 * n_cfg * F + kTileN - 1) / kTileN;
    int64_t np = (P + kTileP - 1) / kTileP;
    int64_t nkc = (N + kChunkK - 1) / kChunkK;
    a += (int64_t)npieces * nn * nkc * kTileN * kChunkK;
    u += np * nn;
    if (N > kRegMaxPorts) f += F * N * N;
  }
  bop_off[n_struct] = a;
  unit_off[n_struct] = u;
  lu_off[n_struct] = f;
}

cudaError_t launch_plan(const mts_problem* pb, int64_t n_cfg, int npieces, int64_t* bop_off,
                        int64_t* unit_off, int64_t* lu_off, cudaStream_t st) {
  plan_kernel<<<1, 32, 0, st>>>(pb->n_struct, n_cfg, pb->port_off, pb->point_off, pb->freq_off,
                                npieces, bop_off, unit_off, lu_off);
  note_launch();
  return cudaGetLastError();
}

// FP64 SIMT superposition. A unit is 128 points x 64 systems (the GEMM unit of 128 x 128
// real columns); 512 threads: point = t % 128, 16 systems per thread. I tile staged in
// shared memory in K chunks of 32 ports.
constexpr int kSupSys = 64;
constexpr int kSupK = 32;

__global__ void __launch_bounds__(512) superpose_fp64_kernel(SuperposeArgs a) {
  __shared__ double2 sI[kSupSys][kSupK + 1];
  int64_t unit = blockIdx.x;
  int s = find_struct_i64(a.unit_off, a.n_struct, unit);
  int N = a.port_off[s + 1] - a.port_off[s];
  int64_t P = a.point_off[s + 1] - a.point_off[s];
  int F = a.freq_off[s + 1] - a.freq_off[s];
  int64_t nsys = a.n_cfg * F;
  int64_t np = (P + kTileP - 1) / kTileP;
  int64_t lu = unit - a.unit_off[s];
  int64_t pt = lu % np, nt = lu / np;
  int t = threadIdx.x;
  int pl = t % kTileP, sg = t / kTileP;  // sg in 0..3
  int64_t p = pt * kTileP + pl;
  const double* H = static_cast<const double*>(a.H) + a.t.pn_off[s];
  double2 acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < N; k0 += kSupK) {
    __syncthreads();
    for (int e = t; e < kSupSys * kSupK; e += 512) {
      int ls = e / kSupK, kk = e % kSupK;
      int64_t sysl = nt * kSupSys + ls;  // local system index = b * F + f
      double2 v = make_double2(0.0, 0.0);
      if (sysl < nsys && k0 + kk < N) {
        int64_t b = sysl / F;
        int f = (int)(sysl - b * F);
        const double* Ip = a.I + 2 * (b * a.sumFN + a.t.fn_off[s] + (int64_t)f * N + k0 + kk);
        v = make_double2(Ip[0], Ip[1]);
      }
      sI[ls][kk] = v;
    }
    __syncthreads();
    int kn = min(kSupK, N - k0);
    if (p < P) {
      for (int kk = 0; kk < kn; ++kk) {
        double h = H[p * N + k0 + kk];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          double2 v = sI[sg * 16 + i][kk];
          acc[i].x = fma(h, v.x, acc[i].x);
          acc[i].y = fma(h, v.y, acc[i].y);
        }
      }
    }
  }
  if (p < P) {
    double2* out = static_cast<double2*>(a.B_out);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      int64_t sysl = nt * kSupSys + sg * 16 + i;
      if (sysl < nsys) {
        int64_t b = sysl / F;
        int f = (int)(sysl - b * F);
        out[b * a.sumFP + a.t.fp_off[s] + (int64_t)f * P + p] = acc[i];
      }
    }
  }
}

cudaError_t launch_superpose_tc(const SuperposeArgs& a, mts_precision prec, cudaStream_t st);

cudaError_t launch_superpose(const SuperposeArgs& a, mts_precision prec, cudaStream_t st) {
  if (a.total_units == 0) return cudaSuccess;
  if (prec == MTS_FP64) {
    superpose_fp64_kernel<<<(unsigned)a.total_units, 512, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
  }
  return launch_superpose_tc(a, prec, st);
}

}  // namespace mts
