// common.cuh -- internal definitions shared by the kernels and the C ABI layer.
//
// Buffer layouts (all offsets in bytes from the caller's 256-byte aligned buffer):
//
// Basis (built by mts_build_basis, read-only afterwards):
//   tables     int64 per-structure prefix tables (device copies, written by a kernel), the
//              structure of every frequency, and the frequencies grouped by port class
//   M64        FP64 [sum_s N_s^2]               inductance matrix blocks
//   H          FP64 (MTS_FP64) or FP32, structure s a [P_s][N_s] block starting at a
//              multiple of 32 elements: field basis, points x loops
//   Hloss64    FP64 [sum_s L_s N_s]             rows of H at the loss points
//   Hloss32    FP32 [sum_s L_s N_s]
//   HlossT32   FP32 [sum_s N_s L_s]              the same rows transposed (k-major), for
//                                                coalesced loads with one loss point per lane
//   M32hi/lo   FP32 [sum_s N_s^2]               M = hi + lo (double-float split)
//   Aop        bf16 tensor-core operand of H (MTS_MIXED: 3 pieces, MTS_BF16: 1),
//              per structure [piece][p_tile][k_chunk][128 rows x 64 k] in the
//              128-byte-swizzled K-major image of shared memory (see swz128)
//   status     int32 [4]
//
// Tape (written by mts_solve, read by mts_superpose and mts_backward):
//   I          FP64 complex [n_cfg][sum_s F_s N_s]
//   loss_part  FP64 [n_cfg][n_freq]             per-system objective sums
//   grad_part  FP64 [n_cfg][sum_s F_s N_s]      per-system dloss/dC terms
//   dldc       FP64 [n_cfg][n_ports]            reduced dloss/dC
//   lossv      FP64 [n_cfg][n_struct]           reduced objective
//   status     int32 [n_cfg][n_freq]            0 ok, 1 not converged, 2 non-finite
//   mu         FP64 complex [n_cfg][sum F N]    backward scratch (u = H^T conj(grad_B))
//   gfield     FP64 [n_cfg][n_ports]            field-cotangent part of the gradient
//   plan       int64 per-call tables (B-operand bases, GEMM and SIMT unit prefixes, factor
//              bases)
//   err        int32 [4]: [0] bounded-wait timeout code, [1] count of bad systems
//   Bop        bf16 tensor-core operand of I, per structure
//              [piece][n_tile][k_chunk][128 rows x 64 k], row = 2 (b F_s + f) + c
//   mu_loss    FP64 complex [n_cfg][sum F N]    adjoint solution of the objective
//   lu         complex FP32 (FP64 for MTS_FP64) [n_cfg][sum_{N_s > 64} F_s N_s^2]: LU
//              factors of the systems too large for the register-resident solve
//   fa_part    FP32 [kFaMaxSplit][N rounded to 64][128 ceil(n_cfg F / 64)]: K-split
//              partials of the tensor-core field adjoint (one-structure MTS_MIXED/MTS_BF16
//              problems; empty otherwise)
//   lu_ord     int32 [n_cfg][sum F N]: pivot order of each blocked LU (column k's pivot row),
//              written by the forward, read by a backward call that reuses the factors
//   fac        [n_cfg][n_freq] blocks of kFacStride bytes, only with keep_factors (MTS_MIXED,
//              MTS_BF16): the register solve's factors of each 33..64-port system
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/mts.h"

namespace mts {

constexpr int kTileP = 128;   // GEMM rows (points) per tile = TMEM lanes
constexpr int kTileN = 128;   // GEMM columns ((cfg, freq, re/im)) per tile
constexpr int kChunkK = 64;   // K elements per 128-byte swizzle atom (16-bit types)
constexpr int kMaxPorts = 1024;    // largest structure (ports) the library accepts
constexpr int kRegMaxPorts = 64;   // largest system the register-resident solve kernels hold

// Solve schedules by port count: classes 0..3 run the register-resident kernels with
// 8/16/32/64 threads per system, class 4 the blocked large-system kernel.
constexpr int kNumPortClasses = 5;
#ifdef __CUDACC__
__host__ __device__
#endif
inline int port_class(int64_t N) { return N <= 8 ? 0 : N <= 16 ? 1 : N <= 32 ? 2 : N <= 64 ? 3 : 4; }

// Superposition schedule of a structure: the tensor-core GEMM when its configurations x
// frequencies exceed the threshold (column tiles fill), else the SIMT kernel (H read once,
// no padded columns). MTS_FP64 (npieces == 0) always takes the SIMT kernel; a negative
// threshold puts every structure of the other precisions on the tensor cores.
constexpr int kSimtPts = 128;  // points per SIMT unit (one per thread)
constexpr int kSimtSys = 16;   // systems per SIMT unit, and the default threshold
#ifdef __CUDACC__
__host__ __device__
#endif
inline bool use_tensor_path(int npieces, int64_t n_cfg, int64_t F, int64_t simt_max_sys) {
  return npieces > 0 && (simt_max_sys < 0 || n_cfg * F > simt_max_sys);
}

// A SIMT unit is up to kSimtTiles consecutive tiles of kSimtPts points x kSimtSys systems
// of one structure, taken in turn by one CTA (the systems' offsets and, for N <= one K
// chunk, their staged currents serve every tile).
constexpr int kSimtTiles = 4;
#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t simt_point_groups(int64_t P) {
  return ((P + kSimtPts - 1) / kSimtPts + kSimtTiles - 1) / kSimtTiles;
}

// Each structure's H block starts at a multiple of 32 elements (128 bytes), so that its rows
// are 16-byte aligned whenever N_s is a multiple of 4 (vector loads in the SIMT kernel).
constexpr int64_t kHAlign = 32;

#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline size_t align256(size_t a) { return (a + 255) / 256 * 256; }

inline int n_pieces(mts_precision p) { return p == MTS_MIXED ? 3 : (p == MTS_BF16 ? 1 : 0); }

// Host-side summary of a problem (computed from the host offset tables).
struct ProblemSums {
  int n_struct = 0;
  int max_ports = 0;
  int min_ports = 0;
  int64_t sumLU = 0;  // sum over structures with N_s > kRegMaxPorts of F_s N_s^2 (factor scratch)
  int64_t cls_count[kNumPortClasses] = {0, 0, 0, 0, 0};  // frequencies per port class
  int cls_max_ports[kNumPortClasses] = {0, 0, 0, 0, 0};
  int64_t sumNN = 0, sumLN = 0, sumFN = 0, sumFP = 0, sumFL = 0;
  int64_t sumPN = 0;     // H elements with each structure's block padded to kHAlign
  int64_t sumPNraw = 0;  // sum_s P_s N_s (exported layout)
  int64_t sumAop = 0;  // bf16 elements per piece-set of the H operand (all pieces)
};

struct BasisLayout {
  size_t tables = 0, M64 = 0, H = 0, Hloss64 = 0, Hloss32 = 0, HlossT32 = 0, M32hi = 0, M32lo = 0, Aop = 0,
         status = 0, total = 0;
  int h_elem = 8;
};

// Device-side table block inside the basis (arrays of n_struct+1 int64 unless noted).
struct TableLayout {
  size_t nn_off, pn_off, pnr_off, ln_off, fn_off, fp_off, fl_off, aop_off, ptile_off, pair_off,
      freq_struct /* int32 [n_freq] */, cls_freq /* int32 [n_freq] */, bytes;
};

struct TapeLayout {
  size_t I = 0, loss_part = 0, grad_part = 0, dldc = 0, lossv = 0, status = 0, mu = 0,
         gfield = 0, plan = 0, err = 0, Bop = 0, lu = 0, mu_loss = 0, fa_part = 0, lu_ord = 0,
         fac = 0, total = 0;
};

// Per-call plan tables inside the tape (arrays of n_struct+1 int64).
struct PlanLayout {
  size_t bop_off, unit_off, lu_off, simt_off, bytes;
};

ProblemSums problem_sums(const mts_problem* pb, mts_precision prec);
TableLayout table_layout(int n_struct, int n_freq);
BasisLayout basis_layout(const mts_problem* pb, mts_precision prec);
PlanLayout plan_layout(int n_struct);
TapeLayout tape_layout(const mts_problem* pb, int64_t n_cfg, mts_precision prec);

// Device pointers of the basis tables.
struct DevTables {
  const int64_t* nn_off;
  const int64_t* pn_off;   // H block of structure s (padded to kHAlign)
  const int64_t* pnr_off;  // unpadded prefix of P_s N_s (exported layout)
  const int64_t* ln_off;
  const int64_t* fn_off;
  const int64_t* fp_off;
  const int64_t* fl_off;
  const int64_t* aop_off;
  const int64_t* ptile_off;  // prefix of ceil(P_s / 128): point tiles of the basis kernels
  const int64_t* pair_off;   // prefix of N_s (N_s + 1) / 2: loop pairs of the M kernel
  const int32_t* freq_struct;
  const int32_t* cls_freq;  // frequencies grouped by port class, ascending within a class
};

inline DevTables dev_tables(const void* basis, const BasisLayout& bl, int n_struct, int n_freq) {
  TableLayout tl = table_layout(n_struct, n_freq);
  const char* b = static_cast<const char*>(basis) + bl.tables;
  DevTables t;
  t.nn_off = reinterpret_cast<const int64_t*>(b + tl.nn_off);
  t.pn_off = reinterpret_cast<const int64_t*>(b + tl.pn_off);
  t.pnr_off = reinterpret_cast<const int64_t*>(b + tl.pnr_off);
  t.ln_off = reinterpret_cast<const int64_t*>(b + tl.ln_off);
  t.fn_off = reinterpret_cast<const int64_t*>(b + tl.fn_off);
  t.fp_off = reinterpret_cast<const int64_t*>(b + tl.fp_off);
  t.fl_off = reinterpret_cast<const int64_t*>(b + tl.fl_off);
  t.aop_off = reinterpret_cast<const int64_t*>(b + tl.aop_off);
  t.ptile_off = reinterpret_cast<const int64_t*>(b + tl.ptile_off);
  t.pair_off = reinterpret_cast<const int64_t*>(b + tl.pair_off);
  t.freq_struct = reinterpret_cast<const int32_t*>(b + tl.freq_struct);
  t.cls_freq = reinterpret_cast<const int32_t*>(b + tl.cls_freq);
  return t;
}

// Launch bookkeeping (count of kernels launched by this library).
void note_launch(int n = 1);

}  // namespace mts

// ------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------
#ifdef __CUDACC__
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mts {

// Byte offset of element (r, kk) of a 128-row x 64-column 16-bit tile in the K-major,
// 128-byte-swizzled shared-memory image used by the tensor-core descriptors: row r at
// r*128 bytes, its 16-byte chunk j = kk/8 stored at chunk position j ^ (r % 8).
__host__ __device__ inline uint32_t swz128(uint32_t r, uint32_t kk) {
  return r * 128u + ((((kk >> 3) ^ (r & 7u)) & 7u) << 4) + ((kk & 7u) << 1);
}

__device__ inline int find_struct_i32(const int32_t* off, int n, int64_t x) {
  int lo = 0, hi = n;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ inline int find_struct_i64(const int64_t* off, int n, int64_t x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace mts
#endif
