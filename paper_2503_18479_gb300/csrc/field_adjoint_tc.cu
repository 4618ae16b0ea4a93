// field_adjoint_tc.cu -- the adjoint right-hand side of a full-field cotangent on the
// 5th-generation tensor cores (paper Eq. 8-10 through d(A^-1) = -A^-1 dA A^-1):
//   u[b][f][k] = sum_p H[p][k] conj(grad_B[b][f][p])
// for a problem with one structure on the tensor path (MTS_MIXED, MTS_BF16).
//
// Real GEMM: rows = (system i = b F + f, c) with c = 0 for Re grad_B and c = 1 for -Im grad_B,
// K = field points, columns = ports: D[2i + c][k] = sum_p G_c[i][p] H[p][k], so that
// u = D[2i][k] + j D[2i + 1][k]. The H operand is the basis image the superposition already
// keeps (bf16 pieces of H, [piece][point tile][port chunk][128 points x 64 ports] in the
// 128-byte-swizzled layout): read with points as K and ports as the contiguous dimension it
// is the MN-major B operand of this GEMM, so nothing is repacked. grad_B (complex64, the
// 2 n_cfg F x P operand that is read once) is split into bf16 pieces in shared memory by
// converter warps; the six piece pairs of order >= 2^-16 (MTS_MIXED) give FP32-accurate
// products, MTS_BF16 uses one pair.
//
// Work units: (64-system row tile) x (64-port chunk) x (K split). Persistent kernel, one CTA
// per SM, 480 threads:
//   warp 0      producer: cp.async.bulk of the H half-tiles (64 points x 64 ports per
//               piece) into a ring of stages, mbarrier transaction counts
//   warp 1      TMEM allocation (128 columns: two 64-column FP32 accumulators); lane 0
//               issues tcgen05.mma (M = 128, N = 64, K = 16, kind::f16, bf16 inputs, B
//               MN-major) and hands an accumulator to the epilogue every kDrain K steps
//   warps 2..5  converters: read 64 systems x 64 points of grad_B from the raw ring, write
//               the conj pieces in the K-major swizzled image, fence the async proxy, arrive
//   warp 14     raw producer: cp.async.bulk of each system's 64 points (512 bytes) into a
//               ring of raw grad_B stages (row pitch 528 bytes, so that the converters'
//               16-byte reads of eight consecutive rows fall in distinct banks); rows whose
//               address is not 16-byte aligned, and an odd last point, are read by the
//               converters from global memory instead
//   warps 6..13 epilogue: tcgen05.ld of the accumulator into FP64 running sums (one TMEM
//               lane = one row, 32 of the 64 columns per thread: two warps per lane
//               quarter), at the unit's end the FP32 partial of its K split to the tape
// fa_reduce_kernel then sums the K splits of each (system, port) in FP64 into u. Every
// mbarrier wait is bounded (2 s of %globaltimer; on timeout an error word, then drain and
// return).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace mts {
namespace fa {

using namespace tc;

constexpr int kThreads = 480;
constexpr int kEpiThreads = 256;  // warps 6..13
constexpr int kStepPts = 64;                            // points per K step
constexpr uint32_t kAPiece = 128u * kStepPts * 2u;      // 16 KB: 128 rows x 64 points
constexpr uint32_t kBPiece = (uint32_t)kStepPts * 64u * 2u;  // 8 KB: 64 points x 64 ports
constexpr uint32_t kTmemCols = 128;                     // two 64-column accumulators
constexpr int kDrain = 4;                               // K steps per accumulator hand-off
constexpr uint32_t kRawPitch = 528;                     // bytes per system row of a raw stage
constexpr uint32_t kRawStage = 64u * kRawPitch;          // 64 systems x 64 points of grad_B

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, A K-major, B MN-major,
// M = 128, N = 64.
constexpr uint32_t kIdescMN = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) |
                              ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ inline void mma_mn(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdescMN), "r"(accum)
      : "memory");
}

__device__ inline void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int NPIECE>
struct Cfg {
  static constexpr int NSTAGE = NPIECE == 3 ? 2 : 4;  // operand stages (pieces of both)
  static constexpr int RAW = NPIECE == 3 ? 2 : 3;     // raw grad_B stages
  static constexpr uint32_t kStage = (uint32_t)NPIECE * (kAPiece + kBPiece);
};

struct UnitPos {
  int64_t mt;
  int kc, ks, t0, t1;
};

__device__ inline UnitPos unit_pos(const FaTcArgs& a, int64_t u) {
  UnitPos q;
  q.ks = (int)(u % a.nsplit);
  const int64_t r = u / a.nsplit;
  q.kc = (int)(r % a.nkc);
  q.mt = r / a.nkc;
  q.t0 = (int)((int64_t)q.ks * a.nsteps / a.nsplit);
  q.t1 = (int)((int64_t)(q.ks + 1) * a.nsteps / a.nsplit);
  return q;
}

// 8 values -> one 16-byte chunk of bf16 (x0 piece) and the remainder
__device__ inline uint4 bf16_chunk(const float* x, float* rem) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 back = __bfloat1622float2(h);
    rem[2 * i] = x[2 * i] - back.x;
    rem[2 * i + 1] = x[2 * i + 1] - back.y;
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int NPIECE>
__global__ void __launch_bounds__(kThreads, 1) field_adjoint_tc_kernel(FaTcArgs a) {
  constexpr int NSTAGE = Cfg<NPIECE>::NSTAGE;
  constexpr int RAW = Cfg<NPIECE>::RAW;
  constexpr uint32_t kStage = Cfg<NPIECE>::kStage;
  constexpr int NPAIR = NPIECE == 3 ? 6 : 1;
  constexpr int pa[6] = {2, 1, 0, 1, 0, 0};  // piece pairs (A = grad_B, B = H), small first
  constexpr int pb[6] = {0, 1, 2, 0, 1, 0};

  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  uintptr_t sbase = (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023);
  unsigned char* stages = reinterpret_cast<unsigned char*>(sbase);  // [stage][A pieces, B pieces]
  unsigned char* raws = stages + NSTAGE * kStage;  // [RAW][64 rows, pitch kRawPitch]
  uint64_t* bars = reinterpret_cast<uint64_t*>(raws + RAW * kRawStage);
  uint64_t* bfull = bars;               // [NSTAGE] H copies landed
  uint64_t* afull = bars + NSTAGE;      // [NSTAGE] grad_B pieces written (128 arrivals)
  uint64_t* empty = bars + 2 * NSTAGE;  // [NSTAGE] MMAs of the stage done
  uint64_t* tfull = bars + 3 * NSTAGE;  // [2]
  uint64_t* tempty = tfull + 2;         // [2] (128 arrivals)
  uint64_t* mdone = tempty + 2;         // [1]
  uint64_t* rfull = mdone + 1;          // [RAW] raw copies landed
  uint64_t* rempty = rfull + RAW;       // [RAW] raw stage read (128 arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rempty + RAW);
  int32_t* err = a.err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t u_begin = a.units * blockIdx.x / G;
  const int64_t u_end = a.units * (blockIdx.x + 1) / G;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&afull[i], 128);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kEpiThreads);
    }
    mbar_init(mdone, 1);
    for (int i = 0; i < RAW; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], 128);
    }
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
    // ---------------- producer of the H operand ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t last_phase[NSTAGE];
      bool used[NSTAGE];
      for (int i = 0; i < NSTAGE; ++i) {
        used[i] = false;
        last_phase[i] = 0;
      }
      const unsigned char* Ab = reinterpret_cast<const unsigned char*>(a.Aop);
      for (int64_t u = u_begin; u < u_end && ok; ++u) {
        const UnitPos q = unit_pos(a, u);
        for (int t = q.t0; t < q.t1 && ok; ++t) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, err, 11)) {
            ok = false;
            break;
          }
          unsigned char* sB = stages + stage * kStage + NPIECE * kAPiece;
          mbar_arrive_expect_tx(&bfull[stage], NPIECE * kBPiece);
          for (int p = 0; p < NPIECE; ++p) {
            const unsigned char* g =
                Ab + ((size_t)(p * a.nptile + (t >> 1)) * a.nkc + q.kc) * (2 * kBPiece) +
                (size_t)(t & 1) * kBPiece;
            bulk_g2s(sB + p * kBPiece, g, kBPiece, &bfull[stage]);
          }
          used[stage] = true;
          last_phase[stage] = phase;
          if (++stage == NSTAGE) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      for (int i = 0; i < NSTAGE; ++i)
        if (used[i]) mbar_wait(&bfull[i], last_phase[i], err, 15);
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
        const UnitPos q = unit_pos(a, u);
        for (int g0 = q.t0; g0 < q.t1 && ok; g0 += kDrain) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1u, err, 12)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)acc * 64u;
          const int g1 = min(g0 + kDrain, q.t1);
          for (int t = g0; t < g1; ++t) {
            if (!mbar_wait(&afull[stage], phase, err, 13) || !mbar_wait(&bfull[stage], phase, err, 14)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sA = smem_u32(stages + stage * kStage);
            const uint32_t sB = sA + NPIECE * kAPiece;
#pragma unroll
            for (int pp = 0; pp < NPAIR; ++pp) {
              const int qa = NPIECE == 3 ? pa[pp] : 0, qb = NPIECE == 3 ? pb[pp] : 0;
              const uint64_t da = make_desc(sA + qa * kAPiece);
              const uint64_t db = make_desc(sB + qb * kBPiece);
#pragma unroll
              for (int kk = 0; kk < kStepPts / 16; ++kk) {
                // A (K-major): 16 points = 32 bytes along the row; B (MN-major): 16 point
                // rows = 2048 bytes
                mma_mn(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 128),
                       (t > g0 || pp > 0 || kk > 0) ? 1u : 0u);
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
      mma_commit(mdone);
      mbar_wait(mdone, 0, err, 16);
    }
  } else if (warp < 6) {
    // ---------------- converters: raw grad_B -> conj bf16 pieces ----------------
    const int tid = threadIdx.x - 64;        // 0..127
    const int il = tid & 63, h = tid >> 6;   // system of the tile, half of the 64 points
    const int cfirst = (il >> 2) & 1;        // component written first: eight consecutive
                                             // rows then cover all eight 16-byte slots
    int stage = 0, rs = 0;
    uint32_t phase = 0, rph = 0;
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok; ++u) {
      const UnitPos q = unit_pos(a, u);
      const int64_t sys = q.mt * 64 + il;
      const bool vs = sys < a.nsys;
      const int64_t b = vs ? sys / a.F : 0;
      const int64_t f = vs ? sys - b * a.F : 0;
      const float2* src = a.gB + b * a.sumFP + a.fpo + f * a.P;
      const bool bulk = vs && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0);
      for (int t = q.t0; t < q.t1; ++t) {
        if (!mbar_wait(&rfull[rs], rph, err, 19) || !mbar_wait(&empty[stage], phase ^ 1u, err, 17)) {
          ok = false;
          break;
        }
        const unsigned char* row = raws + rs * kRawStage + il * kRawPitch;
        unsigned char* sA = stages + stage * kStage;
        const int64_t p0 = (int64_t)t * kStepPts;
        const int np = (int)min((int64_t)kStepPts, a.P - p0);
        const int npe = bulk ? (np & ~1) : 0;  // points of this row in the raw stage
#pragma unroll 1
        for (int c8 = 0; c8 < 4; ++c8) {
          const int e0 = 32 * h + 8 * c8;
          float re[8], im[8];
          if (e0 + 8 <= npe) {
            const float4* s4 = reinterpret_cast<const float4*>(row + 8 * e0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 v = s4[i];
              re[2 * i] = v.x;
              im[2 * i] = -v.y;  // conj
              re[2 * i + 1] = v.z;
              im[2 * i + 1] = -v.w;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int p = e0 + e;
              float2 g = make_float2(0.0f, 0.0f);
              if (p < npe)
                g = reinterpret_cast<const float2*>(row)[p];
              else if (vs && p < np)
                g = __ldg(src + p0 + p);
              re[e] = g.x;
              im[e] = -g.y;
            }
          }
          const int j = 4 * h + c8;  // 16-byte chunk of the 128-byte row
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int c = cc ^ cfirst;
            const uint32_t R = 2u * il + c;
            const uint32_t off = R * 128u + ((((uint32_t)j ^ (R & 7u)) & 7u) << 4);
            float x[8], r1[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = c == 0 ? re[e] : im[e];
            *reinterpret_cast<uint4*>(sA + off) = bf16_chunk(x, r1);
            if (NPIECE == 3) {
              float r2[8], r3[8];
              *reinterpret_cast<uint4*>(sA + kAPiece + off) = bf16_chunk(r1, r2);
              *reinterpret_cast<uint4*>(sA + 2 * kAPiece + off) = bf16_chunk(r2, r3);
            }
          }
        }
        fence_async_smem();  // generic-proxy writes become visible to the tensor core
        mbar_arrive(&afull[stage]);
        mbar_arrive(&rempty[rs]);
        if (++stage == NSTAGE) {
          stage = 0;
          phase ^= 1u;
        }
        if (++rs == RAW) {
          rs = 0;
          rph ^= 1u;
        }
      }
    }
  } else if (warp == 14) {
    // ---------------- raw producer: 64 points of each system row per K step ----------------
    int rs = 0;
    uint32_t rph = 0;
    uint32_t last_phase[RAW];
    bool used[RAW];
    for (int i = 0; i < RAW; ++i) {
      used[i] = false;
      last_phase[i] = 0;
    }
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok; ++u) {
      const UnitPos q = unit_pos(a, u);
      const float2* src[2];
      bool bulk[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int64_t sys = q.mt * 64 + lane + 32 * hh;
        const bool vs = sys < a.nsys;
        const int64_t b = vs ? sys / a.F : 0;
        const int64_t f = vs ? sys - b * a.F : 0;
        src[hh] = a.gB + b * a.sumFP + a.fpo + f * a.P;
        bulk[hh] = vs && ((reinterpret_cast<uintptr_t>(src[hh]) & 15u) == 0);
      }
      const uint32_t nbulk = __popc(__ballot_sync(0xffffffffu, bulk[0])) +
                             __popc(__ballot_sync(0xffffffffu, bulk[1]));
      for (int t = q.t0; t < q.t1; ++t) {
        int okw = (lane == 0) ? (int)mbar_wait(&rempty[rs], rph ^ 1u, err, 20) : 1;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          ok = false;
          break;
        }
        const int64_t p0 = (int64_t)t * kStepPts;
        const int np = (int)min((int64_t)kStepPts, a.P - p0);
        const uint32_t bytes = 8u * (uint32_t)(np & ~1);  // a multiple of 16
        if (lane == 0) mbar_arrive_expect_tx(&rfull[rs], nbulk * bytes);
        __syncwarp();
        if (bytes > 0) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh)
            if (bulk[hh])
              bulk_g2s(raws + rs * kRawStage + (lane + 32 * hh) * kRawPitch, src[hh] + p0, bytes,
                       &rfull[rs]);
        }
        used[rs] = true;
        last_phase[rs] = rph;
        if (++rs == RAW) {
          rs = 0;
          rph ^= 1u;
        }
      }
    }
    if (lane == 0)  // own copies in flight land before the CTA ends
      for (int i = 0; i < RAW; ++i)
        if (used[i]) mbar_wait(&rfull[i], last_phase[i], err, 21);
  } else {
    // ------- epilogue: double-float (FP32 hi + lo) running sums, FP32 partial per K split -------
    // (FP32 TwoSum on the FP32 pipe: FP64 adds would run at 1/64 of its rate)
    const int quarter = warp & 3;        // TMEM lanes 32*quarter .. +31
    const int half = (warp - 6) >> 2;    // accumulator columns 32*half .. +31
    int acc = 0;
    uint32_t aphase = 0;
    bool alive = true;
    for (int64_t u = u_begin; u < u_end && alive; ++u) {
      const UnitPos q = unit_pos(a, u);
      float hi[32], lo[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.0f;
      for (int g0 = q.t0; g0 < q.t1; g0 += kDrain) {
        int ok = (lane == 0) ? (int)mbar_wait(&tfull[acc], aphase, err, 18) : 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          alive = false;
          break;
        }
        mbar_wait(&tfull[acc], aphase, err, 18);
        tc_fence_after();
        float v[32];
        tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * 64u + 32u * half, v);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        if (++acc == 2) {
          acc = 0;
          aphase ^= 1u;
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) two_sum_acc(hi[c], lo[c], v[c]);
      }
      if (!alive) break;
      const int64_t row = q.mt * 128 + quarter * 32 + lane;
      float* dst = a.part + ((int64_t)q.ks * a.npad + (int64_t)q.kc * 64 + 32 * half) * a.rows_pad + row;
#pragma unroll
      for (int c = 0; c < 32; ++c) dst[(int64_t)c * a.rows_pad] = hi[c] + lo[c];
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
  return 1024 + (size_t)Cfg<NPIECE>::NSTAGE * Cfg<NPIECE>::kStage +
         (size_t)Cfg<NPIECE>::RAW * kRawStage + 8 * (4 * Cfg<NPIECE>::NSTAGE + 5 + 2 * Cfg<NPIECE>::RAW) +
         16;
}

// u[b][fn + f N + k] = sum over K splits of the row pair (2i, 2i + 1), i = b F + f
__global__ void fa_reduce_kernel(FaTcArgs a, double* __restrict__ u, int64_t sumFN, int64_t fno) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.nsys * a.N) return;
  const int64_t i = e / a.N;
  const int k = (int)(e - i * a.N);
  double sr = 0.0, si = 0.0;
  for (int ks = 0; ks < a.nsplit; ++ks) {
    const float* p = a.part + ((int64_t)ks * a.npad + k) * a.rows_pad + 2 * i;
    sr += (double)p[0];
    si += (double)p[1];
  }
  const int64_t b = i / a.F, f = i - b * a.F;
  double* d = u + 2 * (b * sumFN + fno + f * a.N + k);
  d[0] = sr;
  d[1] = si;
}

}  // namespace fa

static int g_fa_sms = 0;

cudaError_t launch_field_adjoint_tc(FaTcArgs a, mts_precision prec, double* u, int64_t sumFN,
                                    int64_t fno, cudaStream_t st) {
  if (g_fa_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_fa_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_fa_sms <= 0) g_fa_sms = 1;
  }
  if (a.err == nullptr || a.part == nullptr) return cudaErrorInvalidValue;
  if (a.nsys > 0 && a.N > 0) {
    const int64_t grid = a.units < g_fa_sms ? a.units : g_fa_sms;
    if (prec == MTS_MIXED) {
      const size_t sm = fa::smem_bytes<3>();
      cudaError_t e = cudaFuncSetAttribute(fa::field_adjoint_tc_kernel<3>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      fa::field_adjoint_tc_kernel<3><<<(unsigned)grid, fa::kThreads, sm, st>>>(a);
    } else {
      const size_t sm = fa::smem_bytes<1>();
      cudaError_t e = cudaFuncSetAttribute(fa::field_adjoint_tc_kernel<1>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      fa::field_adjoint_tc_kernel<1><<<(unsigned)grid, fa::kThreads, sm, st>>>(a);
    }
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = a.nsys * a.N;
    fa::fa_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, u, sumFN, fno);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace mts
