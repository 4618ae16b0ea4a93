// field_adjoint_tc.cu -- the adjoint right-hand side of a full-field cotangent on the
// 5th-generation tensor cores (paper Eq. 8-10 through d(A^-1) = -A^-1 dA A^-1):
//   u[b][f][k] = sum_p H[p][k] conj(grad_B[b][f][p])
// for a problem with one structure on the tensor path (MTS_MIXED, MTS_BF16).
//
// Real GEMM: per tile of 64 systems i = b F + f, rows il (Re grad_B) and 64 + il (Im grad_B),
// K = field points, columns = ports: D[c 64 + il][k] = sum_p G_c[i][p] H[p][k], so that
// u = D[il][k] - j D[64 + il][k]. The H operand is the basis image the superposition already
// keeps (bf16 pieces of H, [piece][point tile][port chunk][128 points x 64 ports] in the
// 128-byte-swizzled layout): read with points as K and ports as the contiguous dimension it
// is the MN-major B operand of this GEMM, so nothing is repacked. grad_B (complex64, the
// 2 n_cfg F x P operand that is read once) is split into bf16 pieces by converter warps
// that write them straight into tensor memory, where the MMA reads its A operand; the six
// piece pairs of order >= 2^-16 (MTS_MIXED) give FP32-accurate products, MTS_BF16 uses one
// pair. With A in tensor memory, shared memory holds only the H stages and a deep ring of
// raw grad_B rows, so that enough bytes are in flight to stream grad_B at HBM speed.
//
// Work units: (64-system row tile) x (64-port chunk) x (K split). Persistent kernel, one CTA
// per SM, 576 threads:
//   warp 0       producer: cp.async.bulk of the H half-tiles (64 points x 64 ports per
//                piece) into a ring of stages, mbarrier transaction counts
//   warp 1       TMEM allocation (512 columns: two 64-column FP32 accumulators, then the A
//                stages, 32 columns per piece); lane 0 issues tcgen05.mma (M = 128, N = 64,
//                K = 16, kind::f16, bf16 inputs, A in TMEM, B MN-major in shared memory) and
//                hands an accumulator to the epilogue every kDrain K steps
//   warps 2..9   converters: copy grad_B rows into a ring of raw stages with cp.async (each
//                warp instruction reads 512 contiguous bytes of one row; row pitch 528 bytes
//                in shared memory so that the 16-byte reads below hit distinct banks), RAW - 1
//                K steps ahead; then thread = one A row (TMEM lane 32 (warp % 4) + lane: Re
//                of system lane quarters 0-1, Im quarters 2-3), 32 of the step's 64 points
//                (warps 2..5 the first half, 6..9 the second): bf16 pieces, tcgen05.st (the
//                conj's sign is applied in the K-split reduction)
//   warps 10..17 epilogue: tcgen05.ld of the accumulator into double-float (FP32 hi + lo)
//                running sums (one TMEM lane = one row, 32 of the 64 columns per thread: two
//                warps per lane quarter), at the unit's end the FP32 partial of its K split
//                to the tape
// (Bulk copies of 512 bytes per row streamed grad_B at 2.0 TB/s on a GB300, 1 KB copies at
// 3.9 TB/s, warp-coalesced 16-byte loads at 6.2 TB/s: the per-copy cost of the bulk engine
// bounds small row segments, so the rows go through cp.async.)
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

constexpr int kThreads = 576;
constexpr int kConvThreads = 256;  // warps 2..9
constexpr int kEpiThreads = 256;   // warps 10..17
constexpr int kStepPts = 64;                                 // points per K step
constexpr uint32_t kBPiece = (uint32_t)kStepPts * 64u * 2u;  // 8 KB: 64 points x 64 ports
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 64;       // per accumulator
constexpr uint32_t kAColBase = 128;     // first A column (after the two accumulators)
constexpr uint32_t kAPieceCols = 32;    // 64 bf16 points per row = 32 columns
constexpr int kDrain = 4;                                    // K steps per accumulator hand-off
constexpr uint32_t kRawPitch = 528;                          // bytes per system row of a raw stage
constexpr uint32_t kRawStage = 64u * kRawPitch;              // 64 systems x 64 points of grad_B

// Instruction descriptor: kind::f16, A = B = bf16, D = f32, A K-major, B MN-major,
// M = 128, N = 64.
constexpr uint32_t kIdescMN = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) |
                              ((64u >> 3) << 17) | ((128u >> 4) << 24);

// D (+)= A B with A in tensor memory (M = 128 lanes, K = 16 bf16 = 8 columns)
__device__ inline void mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(kIdescMN), "r"(accum)
      : "memory");
}

__device__ inline void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// TwoSum on two columns at once: (hi, lo) += v per lane of the packed FP32 pairs (the same
// roundings as the scalar form; add/sub.rn.f32x2 round each lane as add/sub.rn.f32)
__device__ inline void two_sum_acc2(unsigned long long& hi, unsigned long long& lo,
                                    unsigned long long v) {
  unsigned long long sm, bp, t1, t2, e;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(sm) : "l"(hi), "l"(v));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bp) : "l"(sm), "l"(hi));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1) : "l"(sm), "l"(bp));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1) : "l"(hi), "l"(t1));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2) : "l"(v), "l"(bp));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e) : "l"(t1), "l"(t2));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(lo) : "l"(lo), "l"(e));
  hi = sm;
}

// 2 n values -> n packed bf16 pairs (round to nearest), no remainder (the last piece)
template <int n>
__device__ inline void bf16_pack(const float* x, uint32_t* pk) {
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    pk[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
}

template <int NPIECE>
struct Cfg {
  static constexpr int NSTAGE = NPIECE == 3 ? 3 : 4;  // operand stages (A in TMEM, B in smem)
  static constexpr int RAW = NPIECE == 3 ? 4 : 5;     // raw grad_B stages
  static constexpr uint32_t kBStage = (uint32_t)NPIECE * kBPiece;
  static_assert(kAColBase + NSTAGE * NPIECE * kAPieceCols <= kTmemCols, "TMEM columns");
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

// 2 n values -> n packed bf16 pairs (round to nearest) and the remainders, in place. The
// pair's bf16 values are widened by bit operations and subtracted as one packed FP32 pair.
template <int n>
__device__ inline void bf16_split(float* x, uint32_t* pk) {
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);  // x[2i] in the low half
    unsigned long long xv, bv;
    asm("mov.b64 %0, {%1,%2};" : "=l"(xv) : "f"(x[2 * i]), "f"(x[2 * i + 1]));
    asm("mov.b64 %0, {%1,%2};" : "=l"(bv) : "r"(hb << 16), "r"(hb & 0xffff0000u));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(xv) : "l"(xv), "l"(bv));
    asm("mov.b64 {%0,%1}, %2;" : "=f"(x[2 * i]), "=f"(x[2 * i + 1]) : "l"(xv));
    pk[i] = hb;
  }
}

// 18 warps: five on some SM sub-partition, whose 16,384 registers then allow 96 per thread;
// the epilogue's running sums spill a little (they are touched once per kDrain K steps)
template <int NPIECE>
__global__ void __launch_bounds__(kThreads, 1) field_adjoint_tc_kernel(FaTcArgs a) {
  constexpr int NSTAGE = Cfg<NPIECE>::NSTAGE;
  constexpr int RAW = Cfg<NPIECE>::RAW;
  constexpr uint32_t kBStage = Cfg<NPIECE>::kBStage;
  constexpr int NPAIR = NPIECE == 3 ? 6 : 1;
  constexpr int pa[6] = {2, 1, 0, 1, 0, 0};  // piece pairs (A = grad_B, B = H), small first
  constexpr int pb[6] = {0, 1, 2, 0, 1, 0};

  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  uintptr_t sbase = (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023);
  unsigned char* bst = reinterpret_cast<unsigned char*>(sbase);  // [NSTAGE][NPIECE][64 x 64]
  unsigned char* raws = bst + NSTAGE * kBStage;                  // [RAW][64 rows, kRawPitch]
  uint64_t* bars = reinterpret_cast<uint64_t*>(raws + RAW * kRawStage);
  uint64_t* bfull = bars;               // [NSTAGE] H copies landed
  uint64_t* afull = bars + NSTAGE;      // [NSTAGE] grad_B pieces stored (kConvThreads arrivals)
  uint64_t* empty = bars + 2 * NSTAGE;  // [NSTAGE] MMAs of the stage done
  uint64_t* tfull = bars + 3 * NSTAGE;  // [2]
  uint64_t* tempty = tfull + 2;         // [2] (kEpiThreads arrivals)
  uint64_t* mdone = tempty + 2;         // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  int32_t* err = a.err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t u_begin = a.units * blockIdx.x / G;
  const int64_t u_end = a.units * (blockIdx.x + 1) / G;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&afull[i], kConvThreads);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kEpiThreads);
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
          if (!mbar_wait_sleep(&empty[stage], phase ^ 1u, err, 11)) {
            ok = false;
            break;
          }
          unsigned char* sB = bst + stage * kBStage;
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
          const uint32_t d_tmem = tmem_base + (uint32_t)acc * kAccCols;
          const int g1 = min(g0 + kDrain, q.t1);
          for (int t = g0; t < g1; ++t) {
            if (!mbar_wait(&afull[stage], phase, err, 13) || !mbar_wait(&bfull[stage], phase, err, 14)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t tA = tmem_base + kAColBase + (uint32_t)(stage * NPIECE) * kAPieceCols;
            const uint32_t sB = smem_u32(bst + stage * kBStage);
#pragma unroll
            for (int pp = 0; pp < NPAIR; ++pp) {
              const int qa = NPIECE == 3 ? pa[pp] : 0, qb = NPIECE == 3 ? pb[pp] : 0;
              const uint64_t db = make_desc(sB + qb * kBPiece);
#pragma unroll
              for (int kk = 0; kk < kStepPts / 16; ++kk) {
                // A: 16 points = 8 TMEM columns; B (MN-major): 16 point rows = 2048 bytes
                mma_ta(d_tmem, tA + (uint32_t)qa * kAPieceCols + (uint32_t)(kk * 8),
                       db + (uint64_t)(kk * 128), (t > g0 || pp > 0 || kk > 0) ? 1u : 0u);
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
  } else if (warp < 10) {
    // ---------------- converters: grad_B -> raw ring (cp.async) -> conj bf16 pieces in TMEM
    // Each converter warp copies 8 system rows of every K step (lane l: bytes 16 l .. 16 l + 15
    // of the row's 512, so one instruction reads 512 contiguous bytes), RAW - 1 steps ahead
    // of the step it converts; a named barrier over the 256 converter threads per step makes
    // the landed copies visible and frees the slot read one step earlier.
    const int ct = threadIdx.x - 64;       // 0..255
    const int cw = ct >> 5;                // copies rows 8 cw .. 8 cw + 7
    const int quarter = warp & 3;          // TMEM lane quarter this warp may access
    const int R = quarter * 32 + lane;     // A row = TMEM lane
    const int il = R & 63;                 // system of the tile
    const bool imag = R >= 64;             // rows 64.. hold Im grad_B (warp-uniform; the
                                           // reduce applies the conj's sign)
    const int hp = (warp - 2) >> 2;        // half of the step's 64 points
    const uint32_t trow = tmem_base + ((uint32_t)(quarter * 32) << 16) + kAColBase + 16u * hp;
    // prefetch cursor: (unit, step) RAW - 1 steps ahead, with the first copied row's (b, f)
    int64_t pu = u_begin;
    int pt = 0, pt1 = 0;
    const float2* rsrc[8];  // the warp's 8 rows of the cursor's unit (NULL past nsys)
    unsigned ralign = 0;    // bit j: row j starts on a 16-byte boundary
    auto cur_unit = [&]() {
      if (pu < u_end) {
        const UnitPos q = unit_pos(a, pu);
        pt = q.t0;
        pt1 = q.t1;
        const int64_t psys0 = q.mt * 64 + 8 * cw;
        int64_t bb = psys0 / a.F;
        int ff = (int)(psys0 - bb * a.F);
        ralign = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2* src = a.gB + bb * a.sumFP + a.fpo + (int64_t)ff * a.P;
          rsrc[j] = psys0 + j < a.nsys ? src : nullptr;
          if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) ralign |= 1u << j;
          if (++ff == a.F) {
            ff = 0;
            ++bb;
          }
        }
      }
    };
    auto issue = [&](int slot) {  // copies of the cursor's step into raw slot `slot`, one group
      if (pu < u_end) {
        const int64_t p0 = (int64_t)pt * kStepPts + 2 * lane;  // this lane's first point
        const int nvalid = (int)max((int64_t)0, min((int64_t)2, a.P - p0));
        const uint32_t dst0 = smem_u32(raws + slot * kRawStage + 8 * cw * kRawPitch + 16 * lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2* src = rsrc[j];
          const uint32_t dst = dst0 + (uint32_t)(j * kRawPitch);
          const int n = src ? nvalid : 0;
          const float2* sp = n > 0 ? src + p0 : a.gB;
          if ((ralign >> j) & 1u) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(sp),
                         "r"((uint32_t)(8 * n))
                         : "memory");
          } else {  // a row starting on an odd point: two 8-byte copies
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(sp),
                         "r"(n >= 1 ? 8u : 0u)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst + 8u),
                         "l"(n >= 2 ? sp + 1 : a.gB), "r"(n >= 2 ? 8u : 0u)
                         : "memory");
          }
        }
        if (++pt == pt1) {
          ++pu;
          cur_unit();
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    cur_unit();
    for (int i = 0; i < RAW - 1; ++i) issue(i);
    int stage = 0, rs = 0, ws = RAW - 1;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok; ++u) {
      const UnitPos q = unit_pos(a, u);
      const int64_t sys = q.mt * 64 + il;
      const bool vs = sys < a.nsys;
      for (int t = q.t0; t < q.t1; ++t) {
        asm volatile("cp.async.wait_group %0;" ::"n"(RAW - 2) : "memory");
        int okw = (lane == 0) ? (int)mbar_wait(&empty[stage], phase ^ 1u, err, 17) : 1;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        int fail;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.eq.s32 p, %1, 0;\n\t"
            "bar.red.or.pred q, 1, 256, p;\n\t"
            "selp.s32 %0, 1, 0, q;\n\t}"
            : "=r"(fail)
            : "r"(okw)
            : "memory");
        if (fail) {
          ok = false;
          break;
        }
        issue(ws);  // the slot every converter finished reading a step ago
        if (++ws == RAW) ws = 0;
        mbar_wait(&empty[stage], phase ^ 1u, err, 17);
        tc_fence_after();
        const unsigned char* row = raws + rs * kRawStage + il * kRawPitch;
        const int e0 = 32 * hp;
        float x[32];
        const float4* s4 = reinterpret_cast<const float4*>(row + 8 * e0);
        if (!vs) {
#pragma unroll
          for (int i = 0; i < 32; ++i) x[i] = 0.0f;
        } else if (imag) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float4 v = s4[i];
            x[2 * i] = v.y;
            x[2 * i + 1] = v.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float4 v = s4[i];
            x[2 * i] = v.x;
            x[2 * i + 1] = v.z;
          }
        }
        const uint32_t ta = trow + (uint32_t)(stage * NPIECE) * kAPieceCols;
        uint32_t pk[16];
        if (NPIECE == 3) {
          bf16_split<16>(x, pk);
          tmem_st16(ta, pk);
          bf16_split<16>(x, pk);
          tmem_st16(ta + kAPieceCols, pk);
          bf16_pack<16>(x, pk);
          tmem_st16(ta + 2 * kAPieceCols, pk);
        } else {
          bf16_pack<16>(x, pk);
          tmem_st16(ta, pk);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&afull[stage]);
        if (++stage == NSTAGE) {
          stage = 0;
          phase ^= 1u;
        }
        if (++rs == RAW) rs = 0;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the CTA
  } else {
    // ------- epilogue: double-float (FP32 hi + lo) running sums, FP32 partial per K split -------
    // (FP32 TwoSum on the FP32 pipe: FP64 adds would run at 1/64 of its rate)
    const int quarter = warp & 3;        // TMEM lanes 32*quarter .. +31
    const int half = (warp - 10) >> 2;   // accumulator columns 32*half .. +31
    int acc = 0;
    uint32_t aphase = 0;
    bool alive = true;
    for (int64_t u = u_begin; u < u_end && alive; ++u) {
      const UnitPos q = unit_pos(a, u);
      unsigned long long hi[16], lo[16];  // columns (2c, 2c + 1) as packed pairs
#pragma unroll
      for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0ull;
      for (int g0 = q.t0; g0 < q.t1; g0 += kDrain) {
        int ok = (lane == 0) ? (int)mbar_wait_sleep(&tfull[acc], aphase, err, 18) : 1;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          alive = false;
          break;
        }
        mbar_wait(&tfull[acc], aphase, err, 18);
        tc_fence_after();
        const uint32_t tcol = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)acc * kAccCols + 32u * half;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16];
          tmem_ld16(tcol + 16u * hh, v);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            unsigned long long vv;
            asm("mov.b64 %0, {%1,%2};" : "=l"(vv) : "f"(v[2 * c]), "f"(v[2 * c + 1]));
            two_sum_acc2(hi[8 * hh + c], lo[8 * hh + c], vv);
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        if (++acc == 2) {
          acc = 0;
          aphase ^= 1u;
        }
      }
      if (!alive) break;
      const int64_t row = q.mt * 128 + quarter * 32 + lane;
      float* dst = a.part + ((int64_t)q.ks * a.npad + (int64_t)q.kc * 64 + 32 * half) * a.rows_pad + row;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float h0, h1, l0, l1;
        asm("mov.b64 {%0,%1}, %2;" : "=f"(h0), "=f"(h1) : "l"(hi[c]));
        asm("mov.b64 {%0,%1}, %2;" : "=f"(l0), "=f"(l1) : "l"(lo[c]));
        dst[(int64_t)(2 * c) * a.rows_pad] = h0 + l0;
        dst[(int64_t)(2 * c + 1) * a.rows_pad] = h1 + l1;
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
  return 1024 + (size_t)Cfg<NPIECE>::NSTAGE * Cfg<NPIECE>::kBStage +
         (size_t)Cfg<NPIECE>::RAW * kRawStage +
         8 * (3 * Cfg<NPIECE>::NSTAGE + 5) + 16;
}

// u[b][fn + f N + k] = sum over K splits of the rows (il, 64 + il) of system i = b F + f's
// tile
__global__ void fa_reduce_kernel(FaTcArgs a, double* __restrict__ u, int64_t sumFN, int64_t fno) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.nsys * a.N) return;
  const int64_t i = e / a.N;
  const int k = (int)(e - i * a.N);
  double sr = 0.0, si = 0.0;
  const int64_t row = (i >> 6) * 128 + (i & 63);
  for (int ks = 0; ks < a.nsplit; ++ks) {
    const float* p = a.part + ((int64_t)ks * a.npad + k) * a.rows_pad + row;
    sr += (double)p[0];
    si -= (double)p[64];  // rows 64.. hold Im grad_B: conj
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
