// superpose_tc.cu -- (c) B = H I (paper Eq. 7) on the 5th-generation tensor cores.
//
// Real GEMM per structure: rows = field points p (A operand: H, bf16 pieces), columns =
// (configuration, frequency, re/im) (B operand: I, bf16 pieces), K = ports. With
// x = x0 + x1 + x2 (bf16 pieces, exact for FP32 data) the product keeps the six piece
// pairs of order >= 2^-16 (x0y0, x0y1, x1y0, x0y2, x1y1, x2y0) accumulated in FP32 in
// tensor memory: relative error ~2^-24 per product (MTS_MIXED). MTS_BF16 uses x0 y0 only.
// When K spans more than kSumMaxPlain 64-wide chunks (MTS_MIXED, more than 256 ports), each
// group of kSumChunks chunks goes to a fresh accumulator and the epilogue adds the group
// partials into a running double-float sum (hi + lo, Knuth's TwoSum) held in two more TMEM
// regions: the FP32 accumulator then grows only to the magnitude of one group's partial sum
// instead of the running sum over the whole K range (measured on the 1024-port array:
// 2.4e-6 relative error with one accumulator, 2e-7 with one per chunk).
//
// Persistent kernel, one CTA per SM, 192 threads:
//   warp 0      producer: cp.async.bulk copies of the pre-swizzled 16 KB operand tiles
//               (global images already in the 128-byte-swizzled K-major layout) into a
//               ring of shared-memory stages, completion via mbarrier transaction counts
//   warp 1      allocates 256 TMEM columns (two 128x128 FP32 accumulators); lane 0
//               issues tcgen05.mma (M=128, N=128, K=16, kind::f16 with bf16 inputs) and
//               tcgen05.commit to release stages and hand accumulators to the epilogue
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (warp w reads lanes 32*(w%4)..),
//               release of the accumulator, then streaming complex64 stores: lane = point,
//               so each warp store writes 32 consecutive points (256 contiguous bytes)
// Every mbarrier wait is bounded; on timeout the kernel records an error word, stops
// issuing work, waits (bounded) for its own copies, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace mts {

namespace tc {

constexpr int kThreads = 192;
constexpr uint32_t kTileBytes = kTileP * kChunkK * 2;  // 16 KB (also kTileN x 64 x 2)
constexpr uint32_t kTmemCols = 512;  // two 128-column accumulators + running sum hi, lo
constexpr uint32_t kHiCol = 256, kLoCol = 384;
constexpr int kSumChunks = 2;    // K chunks per accumulator when the running sum is used
constexpr int kSumMaxPlain = 4;  // up to this many K chunks, one FP32 accumulator (at most
                                 // 4 x 4 K-steps x 6 piece pairs = 96 FP32 roundings)

struct Unit {
  int s, N, F, nkc;
  int64_t P, pt, nt, nptile, nntile;
};

__device__ inline Unit unit_info(const SuperposeArgs& a, int64_t u) {
  Unit x;
  if (a.uni.on) {  // one structure: geometry from the arguments, no table loads
    x.s = 0;
    x.N = a.uni.N;
    x.F = a.uni.F;
    x.P = a.uni.P;
    x.nkc = a.uni.nkc;
    x.nptile = a.uni.nptile;
    x.nntile = a.uni.nntile;
    x.pt = u % x.nptile;
    x.nt = u / x.nptile;
    return x;
  }
  x.s = find_struct_i64(a.unit_off, a.n_struct, u);
  x.N = a.port_off[x.s + 1] - a.port_off[x.s];
  x.F = a.freq_off[x.s + 1] - a.freq_off[x.s];
  x.P = a.point_off[x.s + 1] - a.point_off[x.s];
  x.nkc = (x.N + kChunkK - 1) / kChunkK;
  x.nptile = (x.P + kTileP - 1) / kTileP;
  x.nntile = (2 * a.n_cfg * x.F + kTileN - 1) / kTileN;
  int64_t lu = u - a.unit_off[x.s];
  x.pt = lu % x.nptile;
  x.nt = lu / x.nptile;
  return x;
}

template <int NPIECE>
__global__ void __launch_bounds__(kThreads, 1) superpose_tc_kernel(SuperposeArgs a, int32_t* err) {
  constexpr int NSTAGE = NPIECE == 3 ? 2 : 4;
  constexpr uint32_t kStageBytes = 2u * NPIECE * kTileBytes;
  constexpr int NPAIR = NPIECE == 3 ? 6 : 1;
  // piece pairs (A piece, B piece), smallest products first
  constexpr int pa[6] = {2, 1, 0, 1, 0, 0};
  constexpr int pb[6] = {0, 1, 2, 0, 1, 0};

  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  // 1024-byte aligned operand area
  uintptr_t sbase = (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023);
  unsigned char* stages = reinterpret_cast<unsigned char*>(sbase);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + NSTAGE * kStageBytes);
  uint64_t* full = bars;                 // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;       // [NSTAGE]
  uint64_t* tfull = bars + 2 * NSTAGE;   // [2]
  uint64_t* tempty = tfull + 2;          // [2]
  uint64_t* mdone = tempty + 2;          // [1] all issued MMAs complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t u_begin = a.total_units * blockIdx.x / G;
  const int64_t u_end = a.total_units * (blockIdx.x + 1) / G;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t last_phase[NSTAGE];
      bool used[NSTAGE];
      // the B-operand tile (structure, column tile, K chunk) each stage holds: consecutive
      // units of a CTA usually share it (units advance along the point tiles first), and a
      // stage whose B image is already the one needed only refills its A pieces
      uint64_t bkey[NSTAGE];
      for (int i = 0; i < NSTAGE; ++i) {
        used[i] = false;
        last_phase[i] = 0;
        bkey[i] = ~0ull;
      }
      for (int64_t u = u_begin; u < u_end && ok; ++u) {
        Unit x = unit_info(a, u);
        const unsigned char* Ab =
            reinterpret_cast<const unsigned char*>(a.Aop + (a.uni.on ? 0 : a.t.aop_off[x.s]));
        const unsigned char* Bb =
            reinterpret_cast<const unsigned char*>(a.Bop + (a.uni.on ? 0 : a.bop_off[x.s]));
        for (int kc = 0; kc < x.nkc && ok; ++kc) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, 1)) {
            ok = false;
            break;
          }
          unsigned char* sA = stages + stage * kStageBytes;
          unsigned char* sB = sA + NPIECE * kTileBytes;
          const uint64_t key = ((uint64_t)x.s << 44) | ((uint64_t)x.nt << 12) | (uint64_t)kc;
          const bool needB = bkey[stage] != key;
          mbar_arrive_expect_tx(&full[stage], needB ? kStageBytes : NPIECE * kTileBytes);
          for (int q = 0; q < NPIECE; ++q) {
            const unsigned char* ga =
                Ab + ((size_t)(q * x.nptile + x.pt) * x.nkc + kc) * kTileBytes;
            bulk_g2s(sA + q * kTileBytes, ga, kTileBytes, &full[stage]);
            if (needB) {
              const unsigned char* gb =
                  Bb + ((size_t)(q * x.nntile + x.nt) * x.nkc + kc) * kTileBytes;
              bulk_g2s(sB + q * kTileBytes, gb, kTileBytes, &full[stage]);
            }
          }
          bkey[stage] = key;
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // no copy may still be in flight when the CTA exits
      for (int i = 0; i < NSTAGE; ++i)
        if (used[i]) mbar_wait(&full[i], last_phase[i], err, 5);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++u) {
        Unit x = unit_info(a, u);
        // K chunks per accumulator hand-off: all of them, or kSumChunks with the running sum
        const int group = (NPIECE == 3 && x.nkc > kSumMaxPlain) ? kSumChunks : x.nkc;
        for (int k0 = 0; k0 < x.nkc && ok; k0 += group) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1u, err, 2)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)acc * 128u;
          const int k1 = min(k0 + group, x.nkc);
          for (int kc = k0; kc < k1; ++kc) {
            if (!mbar_wait(&full[stage], phase, err, 3)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sA = smem_u32(stages + stage * kStageBytes);
            const uint32_t sB = sA + NPIECE * kTileBytes;
            // K-steps of 16 that hold data (the tail of the last chunk is zero in both
            // operands: its all-zero steps are not issued)
            const int ksteps = min(kChunkK / 16, (x.N - kc * kChunkK + 15) / 16);
#pragma unroll
            for (int pp = 0; pp < NPAIR; ++pp) {
              const int qa = NPIECE == 3 ? pa[pp] : 0, qb = NPIECE == 3 ? pb[pp] : 0;
              const uint64_t da = make_desc(sA + qa * kTileBytes);
              const uint64_t db = make_desc(sB + qb * kTileBytes);
#pragma unroll
              for (int kk = 0; kk < kChunkK / 16; ++kk) {
                // advance 16 elements (32 bytes) along K inside the swizzle atom
                if (kk < ksteps)
                  mma_bf16(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2),
                           (kc > k0 || pp > 0 || kk > 0) ? 1u : 0u);
              }
            }
            mma_commit(&empty[stage]);
            if (++stage == NSTAGE) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&tfull[acc]);
          if (++acc == 2) {
            acc = 0;
            aphase ^= 1u;
          }
        }
      }
      // every MMA issued by this thread has finished before TMEM is released
      mma_commit(mdone);
      mbar_wait(mdone, 0, err, 6);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    int acc = 0;
    uint32_t aphase = 0;
    float2* Bout = static_cast<float2*>(a.B_out);
    bool alive = true;
    for (int64_t u = u_begin; u < u_end && alive; ++u) {
      Unit x = unit_info(a, u);
      const int64_t p = x.pt * kTileP + quarter * 32 + lane;
      const int64_t nsys = a.n_cfg * x.F;
      const int64_t sys0 = x.nt * (kTileN / 2);
      const int64_t fpo = a.uni.on ? 0 : a.t.fp_off[x.s];
      if (NPIECE == 3 && x.nkc > kSumMaxPlain) {
        // one partial per group of kSumChunks K chunks, added into the running sum (hi, lo)
        const uint32_t lrow = (uint32_t)(quarter * 32) << 16;
        for (int kc = 0; kc < x.nkc; kc += kSumChunks) {
          int ok = (lane == 0) ? (int)mbar_wait(&tfull[acc], aphase, err, 4) : 1;
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) {
            alive = false;
            break;
          }
          mbar_wait(&tfull[acc], aphase, err, 4);
          tc_fence_after();
          const bool last = kc + kSumChunks >= x.nkc;
#pragma unroll 1
          for (int c = 0; c < 4; ++c) {
            float pv[32], hi[32], lo[32];
            tmem_ld32(tmem_base + lrow + (uint32_t)acc * 128u + c * 32, pv);
            if (kc > 0) {
              tmem_ld32(tmem_base + lrow + kHiCol + c * 32, hi);
              tmem_ld32(tmem_base + lrow + kLoCol + c * 32, lo);
            }
            tmem_wait_ld();
            if (kc == 0) {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                hi[i] = pv[i];
                lo[i] = 0.0f;
              }
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) two_sum_acc(hi[i], lo[i], pv[i]);
            }
            if (!last) {
              tmem_st32(tmem_base + lrow + kHiCol + c * 32, hi);
              tmem_st32(tmem_base + lrow + kLoCol + c * 32, lo);
            } else if (p < x.P) {
              // columns 32c .. 32c + 31: systems sys0 + 16c .. + 15
              int64_t sy = sys0 + 16 * c;
              int64_t b = sy / x.F;
              int f = (int)(sy - b * x.F);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                if (sy + i < nsys) {
                  float2* dst = Bout + (b * a.sumFP + fpo + (int64_t)f * x.P + p);
                  st_cs_f2(dst, __fadd_rn(hi[2 * i], lo[2 * i]), __fadd_rn(hi[2 * i + 1], lo[2 * i + 1]));
                }
                if (++f == x.F) {
                  f = 0;
                  ++b;
                }
              }
            }
          }
          tmem_wait_st();
          tc_fence_before();
          mbar_arrive(&tempty[acc]);
          if (++acc == 2) {
            acc = 0;
            aphase ^= 1u;
          }
        }
        continue;
      }
      // lane 0 does the bounded wait; the outcome is made warp-uniform before the
      // warp-collective tcgen05.ld
      int ok = (lane == 0) ? (int)mbar_wait(&tfull[acc], aphase, err, 4) : 1;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      mbar_wait(&tfull[acc], aphase, err, 4);  // already complete: acquire for every lane
      tc_fence_after();
      float v[128];
      const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * 128u;
#pragma unroll
      for (int c = 0; c < 4; ++c) tmem_ld32(taddr + c * 32, v + c * 32);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
      if (p < x.P) {
        if (x.F == 1 && sys0 + kTileN / 2 <= nsys) {
          // full tile, one frequency: system i of the tile is row sys0 + i of the output
          float2* dst = Bout + (sys0 * a.sumFP + fpo + p);
          const int64_t stride = a.sumFP;
#pragma unroll
          for (int i = 0; i < kTileN / 2; ++i) {
            st_cs_f2(dst, v[2 * i], v[2 * i + 1]);
            dst += stride;
          }
        } else {
          int64_t b = sys0 / x.F;
          int f = (int)(sys0 - b * x.F);
#pragma unroll
          for (int i = 0; i < kTileN / 2; ++i) {
            if (sys0 + i < nsys) {
              float2* dst = Bout + (b * a.sumFP + fpo + (int64_t)f * x.P + p);
              st_cs_f2(dst, v[2 * i], v[2 * i + 1]);
            }
            if (++f == x.F) {
              f = 0;
              ++b;
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

template <int NPIECE>
size_t smem_bytes() {
  constexpr int NSTAGE = NPIECE == 3 ? 2 : 4;
  return 1024 + (size_t)NSTAGE * 2 * NPIECE * kTileBytes + 8 * (2 * NSTAGE + 5) + 16;
}

}  // namespace tc

static int g_num_sms = 0;

cudaError_t launch_superpose_tc(const SuperposeArgs& a, mts_precision prec, cudaStream_t st) {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  int64_t grid = a.total_units < g_num_sms ? a.total_units : g_num_sms;
  int32_t* err = a.err;
  if (err == nullptr) return cudaErrorInvalidValue;
  if (prec == MTS_MIXED) {
    size_t sm = tc::smem_bytes<3>();
    cudaError_t e = cudaFuncSetAttribute(tc::superpose_tc_kernel<3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    tc::superpose_tc_kernel<3><<<(unsigned)grid, tc::kThreads, sm, st>>>(a, err);
  } else {
    size_t sm = tc::smem_bytes<1>();
    cudaError_t e = cudaFuncSetAttribute(tc::superpose_tc_kernel<1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    tc::superpose_tc_kernel<1><<<(unsigned)grid, tc::kThreads, sm, st>>>(a, err);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace mts
