// superpose.cu -- (c) of the method: B = H I (paper Eq. 7), the field of every
// configuration and frequency as the superposition of the per-port basis fields.
//
//   plan_kernel          per-call tables: bases of the tensor-core operand of I, the
//                        prefix of GEMM work units and the bases of the LU factor scratch
//                        per structure
//   superpose_simt_kernel  SIMT: MTS_FP64, and structures with at most 16 systems
//   The tensor-core kernel for MTS_MIXED / MTS_BF16 lives in superpose_tc.cu.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace mts {

// Per-structure work of the plan: B-operand elements, tensor-core units, LU scratch
// elements and SIMT units of structure s.
struct PlanWork {
  int64_t a, u, f, v;
};

__device__ inline PlanWork plan_work(int s, int64_t n_cfg, const int32_t* __restrict__ port_off,
                                     const int64_t* __restrict__ point_off,
                                     const int32_t* __restrict__ freq_off, int npieces,
                                     int64_t simt_max_sys) {
  const int64_t N = port_off[s + 1] - port_off[s];
  const int64_t P = point_off[s + 1] - point_off[s];
  const int64_t F = freq_off[s + 1] - freq_off[s];
  PlanWork w{0, 0, 0, 0};
  // the B operand exists for every structure (the schedule does not change memory)
  const int64_t nn = (2 * n_cfg * F + kTileN - 1) / kTileN;
  w.a = (int64_t)npieces * nn * ((N + kChunkK - 1) / kChunkK) * kTileN * kChunkK;
  if (use_tensor_path(npieces, n_cfg, F, simt_max_sys))
    w.u = (P + kTileP - 1) / kTileP * nn;
  else
    w.v = simt_point_groups(P) * ((n_cfg * F + kSimtSys - 1) / kSimtSys);
  if (N > kRegMaxPorts) w.f = F * N * N;
  return w;
}

// Exclusive prefix sums of the per-structure work, one CTA of kPlanThreads: thread t sums a
// contiguous run of structures, the runs' totals are scanned across the CTA (warp shuffles,
// then the warp totals), and each thread writes the offsets of its run. Entry n_struct holds
// the totals. Integer sums: the same values as a serial scan.
constexpr int kPlanThreads = 1024;

__device__ inline int64_t plan_warp_incl(int64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__global__ void __launch_bounds__(kPlanThreads) plan_kernel(
    int n_struct, int64_t n_cfg, const int32_t* __restrict__ port_off,
    const int64_t* __restrict__ point_off, const int32_t* __restrict__ freq_off, int npieces,
    int64_t simt_max_sys, int64_t* bop_off, int64_t* unit_off, int64_t* lu_off,
    int64_t* simt_off) {
  __shared__ int64_t wsum[4][kPlanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int per = (n_struct + kPlanThreads - 1) / kPlanThreads;
  const int s0 = min(n_struct, t * per), s1 = min(n_struct, s0 + per);
  int64_t run[4] = {0, 0, 0, 0};
  for (int s = s0; s < s1; ++s) {
    const PlanWork w = plan_work(s, n_cfg, port_off, point_off, freq_off, npieces, simt_max_sys);
    run[0] += w.a;
    run[1] += w.u;
    run[2] += w.f;
    run[3] += w.v;
  }
  int64_t excl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t inc = plan_warp_incl(run[q], lane);
    excl[q] = inc - run[q];
    if (lane == 31) wsum[q][wp] = inc;
  }
  __syncthreads();
  if (wp == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t v = wsum[q][lane];
      wsum[q][lane] = plan_warp_incl(v, lane) - v;  // exclusive over the warps
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) excl[q] += wsum[q][wp];
  for (int s = s0; s < s1; ++s) {
    bop_off[s] = excl[0];
    unit_off[s] = excl[1];
    lu_off[s] = excl[2];
    simt_off[s] = excl[3];
    const PlanWork w = plan_work(s, n_cfg, port_off, point_off, freq_off, npieces, simt_max_sys);
    excl[0] += w.a;
    excl[1] += w.u;
    excl[2] += w.f;
    excl[3] += w.v;
  }
  if (t == kPlanThreads - 1) {  // its run ends at n_struct (or is empty past it)
    bop_off[n_struct] = excl[0];
    unit_off[n_struct] = excl[1];
    lu_off[n_struct] = excl[2];
    simt_off[n_struct] = excl[3];
  }
}

cudaError_t launch_plan(const mts_problem* pb, int64_t n_cfg, int npieces, int64_t simt_max_sys,
                        int64_t* bop_off, int64_t* unit_off, int64_t* lu_off, int64_t* simt_off,
                        cudaStream_t st) {
  plan_kernel<<<1, kPlanThreads, 0, st>>>(pb->n_struct, n_cfg, pb->port_off, pb->point_off, pb->freq_off,
                                npieces, simt_max_sys, bop_off, unit_off, lu_off, simt_off);
  note_launch();
  return cudaGetLastError();
}

// SIMT superposition. A unit is 128 points x up to 16 systems of one structure; thread t owns
// point t of the tile and accumulates its systems in registers. FP32 with N a multiple of 4
// (every structure's block starts on a 128-byte boundary): the tile's rows of H arrive in
// shared memory by coalesced cp.async copies and each (re, im) pair takes one packed FMA;
// otherwise each thread reads its own row of H straight from global memory.
// The currents of the unit's systems are staged per K chunk in shared memory (k-major: the
// systems of one k are contiguous, read as broadcasts). Used for MTS_FP64 (T = double, FP64
// basis) and, in the other precisions, for structures with at most 16 systems (T = float,
// FP32 basis, FP32 accumulation), where tensor-core column tiles would be mostly padding and
// the work is a read of H.
template <typename T>
struct SimtCfg;
template <>
struct SimtCfg<float> {
  static constexpr int KC = 64;  // K chunk (registers of H per thread)
  static constexpr int VEC = 4;  // elements per 16-byte load
  using C2 = float2;
  using V = float4;
};
template <>
struct SimtCfg<double> {
  static constexpr int KC = 32;
  static constexpr int VEC = 2;
  using C2 = double2;
  using V = double2;
};

template <typename T>
__host__ __device__ constexpr size_t simt_smem_bytes() {
  return sizeof(T) * 2 * (size_t)SimtCfg<T>::KC * kSimtSys;
}

template <typename T, int SC, int KR>
__device__ inline void simt_accumulate(const T (&h)[KR], const T* __restrict__ sI, int kn,
                                       T (&ax)[kSimtSys], T (&ay)[kSimtSys]) {
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    if (k < kn) {
      const T* ik = sI + 2 * kSimtSys * k;
#pragma unroll
      for (int i = 0; i < SC; ++i) {
        ax[i] = fma(h[k], ik[2 * i], ax[i]);
        ay[i] = fma(h[k], ik[2 * i + 1], ay[i]);
      }
    }
  }
}

// FP32 path, N a multiple of 4: (re, im) of a system accumulate as one packed pair, so one
// fma.rn.f32x2 serves both; h comes from the unit's H tile in shared memory, four k at a time.
constexpr int kSimtHPitch = SimtCfg<float>::KC + 4;  // floats per staged H row (bank spread)

template <int SC>
__device__ inline void simt_accumulate_f2(const float* __restrict__ hr, const float* __restrict__ sI,
                                          int kn, unsigned long long (&acc)[kSimtSys]) {
#pragma unroll
  for (int k4 = 0; k4 < SimtCfg<float>::KC; k4 += 4) {
    if (k4 < kn) {  // kn is a multiple of 4
      const float4 h4 = *reinterpret_cast<const float4*>(hr + k4);
      const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        unsigned long long hh;
        asm("mov.b64 %0, {%1,%1};" : "=l"(hh) : "f"(hv[e]));
        const ulonglong2* ik = reinterpret_cast<const ulonglong2*>(sI + 2 * kSimtSys * (k4 + e));
#pragma unroll
        for (int i2 = 0; i2 < SC / 2; ++i2) {
          const ulonglong2 c = ik[i2];
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[2 * i2]) : "l"(hh), "l"(c.x));
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[2 * i2 + 1]) : "l"(hh), "l"(c.y));
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kSimtPts) superpose_simt_kernel(SuperposeArgs a) {
  constexpr int KC = SimtCfg<T>::KC, VEC = SimtCfg<T>::VEC;
  using C2 = typename SimtCfg<T>::C2;
  using V = typename SimtCfg<T>::V;
  extern __shared__ __align__(16) unsigned char sm_simt[];
  T* sI = reinterpret_cast<T*>(sm_simt);  // [KC][kSimtSys][re, im]
  // 2-D grid: y = structure, x = unit within it (no search); 1-D: search the unit prefix
  int s;
  int64_t unit;
  if (gridDim.y > 1) {
    s = blockIdx.y;
    unit = a.simt_off[s] + blockIdx.x;
    if (unit >= a.simt_off[s + 1]) return;  // CTA-uniform
  } else {
    unit = blockIdx.x;
    s = find_struct_i64(a.simt_off, a.n_struct, unit);
  }
  const int N = a.port_off[s + 1] - a.port_off[s];
  const int64_t P = a.point_off[s + 1] - a.point_off[s];
  const int F = a.freq_off[s + 1] - a.freq_off[s];
  const int64_t nsys = a.n_cfg * F;
  const int64_t np = (P + kSimtPts - 1) / kSimtPts;
  const int64_t npg = simt_point_groups(P);
  const int64_t lu = unit - a.simt_off[s];
  const int64_t pt0 = (lu % npg) * kSimtTiles, sys0 = (lu / npg) * kSimtSys;
  const int nsv = (int)min((int64_t)kSimtSys, nsys - sys0);
  const int t = threadIdx.x;
  const bool vec = (N % VEC) == 0;
  // offsets of the unit's systems in I and in B, one 64-bit division per system (not one per
  // staged current and per stored value)
  __shared__ int64_t s_ioff[kSimtSys], s_ooff[kSimtSys];
  const int64_t fpo = a.t.fp_off[s];
  if (t < kSimtSys) {
    int64_t io = 0, oo = 0;
    if (t < nsv) {
      const int64_t sl = sys0 + t, b = sl / F;
      const int f = (int)(sl - b * F);
      io = 2 * (b * a.sumFN + a.t.fn_off[s] + (int64_t)f * N);
      oo = b * a.sumFP + fpo + (int64_t)f * P;
    }
    s_ioff[t] = io;
    s_ooff[t] = oo;
  }
  __syncthreads();
  // the unit's point tiles in turn (CTA-uniform bounds)
  for (int64_t pt = pt0; pt < min(np, pt0 + kSimtTiles); ++pt) {
    const int64_t p = pt * kSimtPts + t;
    const bool live = p < P;
    const T* hrow = static_cast<const T*>(a.H) + a.t.pn_off[s] + (live ? p : 0) * N;
    // the currents of a single K chunk are staged once, for the unit's first tile
    const bool stage_I = pt == pt0 || N > KC;
    if constexpr (sizeof(T) == 4) {
      if (vec) {
        // The tile's 128 rows of H are one contiguous block: each K chunk of them is copied
        // into shared memory with cp.async (consecutive threads, consecutive 16-byte pieces
        // of a row; rows past P are zero-filled) while the chunk's currents are staged, and
        // each thread then reads its own padded row.
        float* sH = reinterpret_cast<float*>(sm_simt + simt_smem_bytes<float>());  // [128][HP]
        constexpr int HP = kSimtHPitch;
        unsigned long long acc[kSimtSys];
#pragma unroll
        for (int i = 0; i < kSimtSys; ++i) acc[i] = 0ull;
        const float* hblk = static_cast<const float*>(a.H) + a.t.pn_off[s] + pt * kSimtPts * (int64_t)N;
        const int rows = (int)min((int64_t)kSimtPts, P - pt * kSimtPts);
        for (int k0 = 0; k0 < N; k0 += KC) {
          const int kn = min(KC, N - k0);
          const int q4 = kn / 4;  // 16-byte pieces per row
          for (int e = t; e < kSimtPts * q4; e += kSimtPts) {
            const int r = e / q4, c = e - r * q4;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(sH + r * HP + 4 * c);
            const float* src = r < rows ? hblk + (int64_t)r * N + k0 + 4 * c : hblk;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                         "r"(r < rows ? 16u : 0u)
                         : "memory");
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (stage_I) {
            for (int e = t; e < kn * kSimtSys; e += kSimtPts) {
              const int k = e / kSimtSys, i = e - k * kSimtSys;
              float re = 0.0f, im = 0.0f;
              if (i < nsv) {
                const double* Ip = a.I + s_ioff[i] + 2 * (k0 + k);
                re = (float)Ip[0];
                im = (float)Ip[1];
              }
              sI[2 * (k * kSimtSys + i)] = re;
              sI[2 * (k * kSimtSys + i) + 1] = im;
            }
          }
          asm volatile("cp.async.wait_all;" ::: "memory");
          __syncthreads();
          const float* hr = sH + t * HP;
          if (nsv <= 4) simt_accumulate_f2<4>(hr, sI, kn, acc);
          else if (nsv <= 8) simt_accumulate_f2<8>(hr, sI, kn, acc);
          else simt_accumulate_f2<16>(hr, sI, kn, acc);
          __syncthreads();
        }
        if (live) {
          float2* out = static_cast<float2*>(a.B_out);
#pragma unroll
          for (int i = 0; i < kSimtSys; ++i)
            if (i < nsv) {
              float2 v;
              asm("mov.b64 {%0,%1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(acc[i]));
              out[s_ooff[i] + p] = v;
            }
        }
        continue;
      }
    }
    // FP64, or FP32 with N not a multiple of 4 (a short register chunk: this path is rare in
    // FP32 and should not set the kernel's register count)
    constexpr int KR = sizeof(T) == 4 ? 16 : KC;
    T ax[kSimtSys], ay[kSimtSys];
#pragma unroll
    for (int i = 0; i < kSimtSys; ++i) ax[i] = ay[i] = T(0);
    for (int k0 = 0; k0 < N; k0 += KR) {
      const int kn = min(KR, N - k0);
      T h[KR];
      if (vec) {  // kn is a multiple of VEC here
#pragma unroll
        for (int q = 0; q < KR / VEC; ++q) {
          V v;
          if (live && q * VEC < kn) {
            v = *reinterpret_cast<const V*>(hrow + k0 + q * VEC);
          } else {
            v = V{};
          }
          const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int e = 0; e < VEC; ++e) h[q * VEC + e] = pv[e];
        }
      } else {
#pragma unroll
        for (int k = 0; k < KR; ++k) h[k] = (live && k < kn) ? hrow[k0 + k] : T(0);
      }
      __syncthreads();
      for (int e = t; e < kn * kSimtSys; e += kSimtPts) {
        const int k = e / kSimtSys, i = e - k * kSimtSys;
        T re = T(0), im = T(0);
        if (i < nsv) {
          const double* Ip = a.I + s_ioff[i] + 2 * (k0 + k);
          re = (T)Ip[0];
          im = (T)Ip[1];
        }
        sI[2 * (k * kSimtSys + i)] = re;
        sI[2 * (k * kSimtSys + i) + 1] = im;
      }
      __syncthreads();
      if (nsv <= 4) simt_accumulate<T, 4, KR>(h, sI, kn, ax, ay);
      else if (nsv <= 8) simt_accumulate<T, 8, KR>(h, sI, kn, ax, ay);
      else simt_accumulate<T, 16, KR>(h, sI, kn, ax, ay);
    }
    if (live) {
      C2* out = static_cast<C2*>(a.B_out);
#pragma unroll
      for (int i = 0; i < kSimtSys; ++i)
        if (i < nsv) {
          C2 v;
          v.x = ax[i];
          v.y = ay[i];
          out[s_ooff[i] + p] = v;
        }
    }
  }
}

cudaError_t launch_superpose_tc(const SuperposeArgs& a, mts_precision prec, cudaStream_t st);

template <typename T>
static cudaError_t launch_simt(const SuperposeArgs& a, cudaStream_t st) {
  // FP32: the currents plus the staged H tile of the N % 4 == 0 path
  constexpr size_t sm = simt_smem_bytes<T>() +
                        (sizeof(T) == 4 ? sizeof(float) * (size_t)kSimtPts * kSimtHPitch : 0);
  cudaError_t e = cudaFuncSetAttribute(superpose_simt_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // one grid row per structure when the padding (units of the largest structure times the
  // structures) stays within twice the work and the structures fit the y dimension
  dim3 grid((unsigned)a.total_simt);
  if (a.n_struct > 1 && a.n_struct <= 65535 && a.max_simt * a.n_struct <= 2 * a.total_simt)
    grid = dim3((unsigned)a.max_simt, (unsigned)a.n_struct);
  superpose_simt_kernel<T><<<grid, kSimtPts, sm, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_superpose(const SuperposeArgs& a, mts_precision prec, cudaStream_t st) {
  if (a.total_units > 0) {
    cudaError_t e = launch_superpose_tc(a, prec, st);
    if (e != cudaSuccess) return e;
  }
  if (a.total_simt > 0)
    return prec == MTS_FP64 ? launch_simt<double>(a, st) : launch_simt<float>(a, st);
  return cudaSuccess;
}

}  // namespace mts
