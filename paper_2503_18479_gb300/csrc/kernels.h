// kernels.h -- internal launcher interface between the C ABI layer and the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mts {

// Kept factors of one 33..64-port system of the register solve (keep_factors): row r's 64
// packed FP32 pairs [q][r] (u64, q < 32 real parts, q >= 32 imaginary parts, blocks rotated
// as the LU leaves them), each row's pivot step (int32 [64]), then W_b = L_bb^-1 of every
// panel (FP32 [8][8][8] real, then imaginary).
constexpr size_t kFacRows = 64 * 64 * 8, kFacPiv = 64 * 4, kFacW = 2 * 8 * 64 * 4;
constexpr size_t kFacStride = kFacRows + kFacPiv + kFacW;  // 37,120 bytes

// Everything the per-system solve kernels read and write.
struct SolveArgs {
  int n_struct, n_freq, n_ports;
  const int32_t* port_off;
  const int32_t* freq_off;
  const int32_t* loss_off;
  const double* R;
  DevTables t;
  const double* M64;
  const float* M32hi;
  const float* M32lo;
  const double* Hl64;
  const float* Hl32;
  const float* HlT32;  // Hl32 transposed per structure: [N_s][L_s]
  int64_t n_cfg;
  const double* C;
  const double* omega;
  const double* V;
  const double* target;
  int target_per_cfg;
  int loss_mode;
  const double* loss_weight;  // [sumFL] or nullptr
  const double* loss_offset;  // complex [sumFL] or nullptr
  double tol;
  int max_refine;
  int64_t sumFN, sumFL;
  double* I;          // tape
  double* I_out;      // optional copy
  double* loss_part;  // [n_cfg][n_freq]
  double* grad_part;  // [n_cfg][sumFN]
  int32_t* status;    // [n_cfg][n_freq]
  __nv_bfloat16* Bop;      // tensor-core operand of I (nullptr for FP64)
  const int64_t* bop_off;  // per-structure element base of Bop (plan table)
  const int64_t* lu_off;   // per-structure element base of the factor scratch (plan table;
                           // [n_struct] = elements per configuration)
  void* lu;                // factor scratch of the large-system kernel
  void* fac;               // register-solve factors of 33..64-port systems, kFacStride bytes
                           // per system (keep_factors), or NULL
  int32_t* lu_order;       // pivot order of each large system (forward writes; a backward
                           // call with rhs_in reuses it and the factors; NULL: refactor)
  double* mu_out;          // adjoint solution mu of the objective (forward with a target)
  // systems of one launch: all (glist == nullptr: system = launch index), or the
  // configurations x the gcount frequencies glist[0 .. gcount-1] of one port class
  const int32_t* glist;
  int64_t gcount;
  int large_threads;  // 0: the library's rule (solve_large.cu: large_threads)
  int reg_widen;      // bit c: register class c (N <= 8, 16, 32) in the next wider kernel
  int npieces;
  int max_loss;  // max loss points of one structure (uniform trip count for group loops)
  // backward (field cotangent) mode: solve A mu = rhs_in and write grad terms only
  const double* rhs_in;  // [n_cfg][sumFN] complex, or nullptr for the forward
};

struct ReduceArgs {
  int n_struct, n_freq, n_ports;
  const int32_t* port_off;
  const int32_t* freq_off;
  const int32_t* loss_off;
  DevTables t;
  int64_t n_cfg, sumFN;
  const double* loss_part;
  const double* grad_part;
  double* dldc;      // [n_cfg][n_ports]
  double* lossv;     // [n_cfg][n_struct]
  double* loss_out;  // optional
  int normalise;     // 1: divide by F_s L_s (objective), 0: plain sum over frequencies
};

cudaError_t launch_build_basis(const mts_problem* pb, mts_precision prec, void* basis,
                               const BasisLayout& bl, const ProblemSums& ps, cudaStream_t st);
// The two table/operand steps of launch_build_basis, reused for bases built from given fields.
cudaError_t launch_basis_tables(const mts_problem* pb, mts_precision prec, void* basis,
                                const BasisLayout& bl, cudaStream_t st);
cudaError_t launch_pack_a(const mts_problem* pb, mts_precision prec, void* basis,
                          const BasisLayout& bl, cudaStream_t st);
cudaError_t launch_export_basis(const mts_problem* pb, mts_precision prec, const void* basis,
                                const BasisLayout& bl, const ProblemSums& ps, double* H_out,
                                double* M_out, cudaStream_t st);

// Per-call plan tables in the tape (bases of the B operand, GEMM unit prefixes).
cudaError_t launch_plan(const mts_problem* pb, int64_t n_cfg, int npieces, int64_t simt_max_sys,
                        int64_t* bop_off, int64_t* unit_off, int64_t* lu_off, int64_t* simt_off,
                        cudaStream_t st);

// Solve of every system: the register-resident kernels for N <= kRegMaxPorts, the blocked
// large-system kernel (solve_large.cu) for the others.
cudaError_t launch_solve(const SolveArgs& a, mts_precision prec, const ProblemSums& ps,
                         cudaStream_t st);
size_t large_solve_smem(mts_precision prec, int max_ports);
cudaError_t launch_solve_large(const SolveArgs& a, mts_precision prec, int64_t n_sys,
                               int min_ports, int max_ports, void* scratch, cudaStream_t st);
cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st);

// Unit geometry of a single-structure problem, passed by value so that the persistent
// GEMM derives every tile's coordinates without table loads.
struct UniformUnits {
  int on;  // 1 when the problem has one structure
  int N, F, nkc;
  int64_t P, nptile, nntile;
};

struct SuperposeArgs {
  int n_struct, n_freq, n_ports;
  const int32_t* port_off;
  const int32_t* freq_off;
  const int64_t* point_off;
  DevTables t;
  int64_t n_cfg, sumFN, sumFP;
  int64_t total_units;      // GEMM work units (host-computed)
  const int64_t* unit_off;  // per-structure prefix of GEMM units (plan table)
  int64_t total_simt;       // SIMT work units (host-computed)
  int64_t max_simt;         // most SIMT units of one structure (2-D grid: x unit, y structure)
  const int64_t* simt_off;  // per-structure prefix of SIMT units (plan table)
  const void* H;            // FP64 (MTS_FP64) basis
  const double* I;          // tape currents
  const __nv_bfloat16* Aop;
  const __nv_bfloat16* Bop;
  const int64_t* bop_off;
  int npieces;
  void* B_out;
  int32_t* err;  // device error word (bounded-wait timeouts)
  UniformUnits uni;
};

cudaError_t launch_superpose(const SuperposeArgs& a, mts_precision prec, cudaStream_t st);

// Elements of the tensor-core B operand of a problem, and its GEMM / SIMT work units.
int64_t bop_elems(const mts_problem* pb, int64_t n_cfg, int npieces, int64_t* units,
                  int64_t* simt_units = nullptr, int64_t* max_simt = nullptr,
                  int64_t simt_max_sys = kSimtSys);

// B = H I of a problem for currents I (device complex [n_cfg][sum F N]) whose B operand and
// plan tables (launch_plan) are in place: the superposition step of mts_superpose.
cudaError_t superpose_core(const mts_problem* pb, mts_precision prec, const void* basis,
                           int64_t n_cfg, int64_t simt_thr, const double* I,
                           const __nv_bfloat16* Bop, const void* plan, int32_t* err, void* B_out,
                           cudaStream_t st);

struct FieldAdjArgs {
  int n_struct, n_freq, n_ports;
  const int32_t* port_off;
  const int32_t* freq_off;
  const int64_t* point_off;
  DevTables t;
  int64_t n_cfg, sumFN, sumFP;
  const void* H;       // FP64 or FP32 basis
  const void* grad_B;  // complex128 (FP64) or complex64
  double* u;           // out: [n_cfg][sumFN] complex, u = H^T conj(grad_B)
};

cudaError_t launch_field_adjoint_rhs(const FieldAdjArgs& a, mts_precision prec, int max_ports,
                                     cudaStream_t st);

// u = H^T conj(grad_B) on the tensor cores for a one-structure problem on the tensor path
// (field_adjoint_tc.cu): work units of 64 systems x 64 ports x one of nsplit K ranges, FP32
// partial per split in the tape (`part`, [nsplit][npad][rows_pad]), summed in FP64 into u.
constexpr int kFaMaxSplit = 16;
struct FaTcArgs {
  int64_t nsys;      // systems n_cfg F
  int64_t P;         // field points
  int64_t sumFP, fpo;  // row stride of grad_B and the structure's offset in a row
  int F, N, nkc, nsteps, nsplit;
  int64_t nptile;    // point tiles (128) of the basis operand image
  int64_t nmt;       // row tiles of 64 systems
  int64_t units;     // nmt * nkc * nsplit
  int64_t npad;      // ports rounded up to 64
  int64_t rows_pad;  // 128 * nmt
  const __nv_bfloat16* Aop;  // the structure's basis operand image (bf16 pieces of H)
  const float2* gB;          // grad_B, complex64 [n_cfg][sumFP]
  float* part;               // K-split partials (tape)
  int32_t* err;              // bounded-wait error word (tape)
};
size_t fa_part_bytes(const mts_problem* pb, int64_t n_cfg, mts_precision prec);
cudaError_t launch_field_adjoint_tc(FaTcArgs a, mts_precision prec, double* u, int64_t sumFN,
                                    int64_t fno, cudaStream_t st);

cudaError_t launch_grad_combine(int64_t n_cfg, int n_struct, int n_ports,
                                const int32_t* port_off, const double* grad_loss,
                                const double* dldc, const double* gfield, double* grad_C,
                                cudaStream_t st);

cudaError_t launch_count_bad(const int32_t* status, int64_t n, int32_t* out, cudaStream_t st);

// dloss/dw (drive fixed) and the drive cotangent from the stored adjoint solutions
cudaError_t launch_omega_v_grad(int64_t n_cfg, int n_freq, int n_struct, int n_ports,
                                const int32_t* port_off, const int32_t* freq_off,
                                const int32_t* loss_off, DevTables t, int64_t sumFN,
                                const double* omega, const double* C, const double* M64,
                                const double* I, const double* mu, const double* grad_loss,
                                double* grad_w, double* grad_V, cudaStream_t st);

// dloss/dR and dloss/dL (self inductances) from the stored adjoint solutions and currents
cudaError_t launch_param_grad(int64_t n_cfg, int n_struct, int n_ports, const int32_t* port_off,
                              const int32_t* freq_off, const int32_t* loss_off, DevTables t,
                              int64_t sumFN, const double* omega, const double* I,
                              const double* mu, const double* grad_loss, double* grad_R,
                              double* grad_L, cudaStream_t st);

cudaError_t launch_adam(int64_t n, const mts_adam& o, double* C, double* u, const double* g,
                        double* m, double* v, int64_t* step, const double* loss, int64_t n_loss,
                        double* history, int64_t history_len, cudaStream_t st);

}  // namespace mts
