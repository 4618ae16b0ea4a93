// abi.cu -- the extern "C" entry points declared in include/mts.h: argument validation,
// buffer layouts, and the launch sequence of each call. No device memory is allocated here.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace mts {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

ProblemSums problem_sums(const mts_problem* pb, mts_precision prec) {
  ProblemSums ps;
  ps.n_struct = pb->n_struct;
  int np = n_pieces(prec);
  for (int s = 0; s < pb->n_struct; ++s) {
    int64_t N = pb->h_port_off[s + 1] - pb->h_port_off[s];
    int64_t P = pb->h_point_off[s + 1] - pb->h_point_off[s];
    int64_t F = pb->h_freq_off[s + 1] - pb->h_freq_off[s];
    int64_t L = pb->h_loss_off ? pb->h_loss_off[s + 1] - pb->h_loss_off[s] : 0;
    if (N > ps.max_ports) ps.max_ports = (int)N;
    if (s == 0 || N < ps.min_ports) ps.min_ports = (int)N;
    if (N > kRegMaxPorts) ps.sumLU += F * N * N;
    const int c = port_class(N);
    ps.cls_count[c] += F;
    if (N > ps.cls_max_ports[c]) ps.cls_max_ports[c] = (int)N;
    ps.sumNN += N * N;
    ps.sumPN += round_up(P * N, kHAlign);
    ps.sumPNraw += P * N;
    ps.sumLN += L * N;
    ps.sumFN += F * N;
    ps.sumFP += F * P;
    ps.sumFL += F * L;
    ps.sumAop += (int64_t)np * round_up(P, kTileP) * round_up(N, kChunkK);
  }
  return ps;
}

TableLayout table_layout(int n_struct, int n_freq) {
  TableLayout t;
  size_t o = 0;
  size_t arr = align256(sizeof(int64_t) * (size_t)(n_struct + 1));
  t.nn_off = o; o += arr;
  t.pn_off = o; o += arr;
  t.pnr_off = o; o += arr;
  t.ln_off = o; o += arr;
  t.fn_off = o; o += arr;
  t.fp_off = o; o += arr;
  t.fl_off = o; o += arr;
  t.aop_off = o; o += arr;
  t.ptile_off = o; o += arr;
  t.pair_off = o; o += arr;
  t.freq_struct = o; o += align256(sizeof(int32_t) * (size_t)(n_freq > 0 ? n_freq : 1));
  t.cls_freq = o; o += align256(sizeof(int32_t) * (size_t)(n_freq > 0 ? n_freq : 1));
  t.bytes = o;
  return t;
}

BasisLayout basis_layout(const mts_problem* pb, mts_precision prec) {
  ProblemSums ps = problem_sums(pb, prec);
  BasisLayout b;
  b.h_elem = prec == MTS_FP64 ? 8 : 4;
  size_t o = 0;
  b.tables = o; o += table_layout(pb->n_struct, pb->n_freq).bytes;
  b.M64 = o; o += align256(sizeof(double) * ps.sumNN);
  b.H = o; o += align256((size_t)b.h_elem * ps.sumPN);
  b.Hloss64 = o; o += align256(sizeof(double) * ps.sumLN);
  b.Hloss32 = o; o += align256(sizeof(float) * ps.sumLN);
  b.HlossT32 = o; o += align256(sizeof(float) * ps.sumLN);
  b.M32hi = o; o += align256(sizeof(float) * ps.sumNN);
  b.M32lo = o; o += align256(sizeof(float) * ps.sumNN);
  b.Aop = o; o += align256(2 * (size_t)ps.sumAop);
  b.status = o; o += 256;
  b.total = o;
  return b;
}

PlanLayout plan_layout(int n_struct) {
  PlanLayout p;
  size_t arr = align256(sizeof(int64_t) * (size_t)(n_struct + 1));
  p.bop_off = 0;
  p.unit_off = arr;
  p.lu_off = 2 * arr;
  p.simt_off = 3 * arr;
  p.bytes = 4 * arr;
  return p;
}

// Elements of the tensor-core B operand, and the GEMM / SIMT work units of the superposition.
int64_t bop_elems(const mts_problem* pb, int64_t n_cfg, int npieces, int64_t* units,
                  int64_t* simt_units, int64_t* max_simt, int64_t simt_max_sys) {
  int64_t a = 0, u = 0, v = 0, vmax = 0;
  for (int s = 0; s < pb->n_struct; ++s) {
    int64_t N = pb->h_port_off[s + 1] - pb->h_port_off[s];
    int64_t P = pb->h_point_off[s + 1] - pb->h_point_off[s];
    int64_t F = pb->h_freq_off[s + 1] - pb->h_freq_off[s];
    // the B operand exists for every structure (the schedule does not change memory)
    const int64_t nn = (2 * n_cfg * F + kTileN - 1) / kTileN;
    a += (int64_t)npieces * nn * ((N + kChunkK - 1) / kChunkK) * kTileN * kChunkK;
    if (use_tensor_path(npieces, n_cfg, F, simt_max_sys)) {
      u += (P + kTileP - 1) / kTileP * nn;
    } else {
      const int64_t vs = simt_point_groups(P) * ((n_cfg * F + kSimtSys - 1) / kSimtSys);
      v += vs;
      if (vs > vmax) vmax = vs;
    }
  }
  if (units) *units = u;
  if (simt_units) *simt_units = v;
  if (max_simt) *max_simt = vmax;
  return a;
}

TapeLayout tape_layout(const mts_problem* pb, int64_t n_cfg, mts_precision prec) {
  ProblemSums ps = problem_sums(pb, prec);
  TapeLayout t;
  size_t o = 0;
  size_t nc = (size_t)n_cfg;
  t.I = o; o += align256(16 * nc * ps.sumFN);
  t.loss_part = o; o += align256(8 * nc * pb->n_freq);
  t.grad_part = o; o += align256(8 * nc * ps.sumFN);
  t.dldc = o; o += align256(8 * nc * pb->n_ports);
  t.lossv = o; o += align256(8 * nc * pb->n_struct);
  t.status = o; o += align256(4 * nc * pb->n_freq);
  t.mu = o; o += align256(16 * nc * ps.sumFN);
  t.gfield = o; o += align256(8 * nc * pb->n_ports);
  t.plan = o; o += plan_layout(pb->n_struct).bytes;
  t.err = o; o += 256;
  t.Bop = o; o += align256(2 * (size_t)bop_elems(pb, n_cfg, n_pieces(prec), nullptr));
  t.lu = o; o += align256((prec == MTS_FP64 ? 16 : 8) * nc * (size_t)ps.sumLU);
  t.mu_loss = o; o += align256(16 * nc * ps.sumFN);
  t.fa_part = o; o += align256(fa_part_bytes(pb, n_cfg, prec));
  t.lu_ord = o; o += align256(4 * nc * ps.sumFN);
  t.fac = o;
  if (pb->keep_factors && prec != MTS_FP64) o += align256(kFacStride * nc * (size_t)pb->n_freq);
  t.total = o;
  return t;
}

size_t fa_part_bytes(const mts_problem* pb, int64_t n_cfg, mts_precision prec) {
  if (pb->n_struct != 1 || prec == MTS_FP64 || n_cfg <= 0) return 0;
  const int64_t N = pb->h_port_off[1], F = pb->h_freq_off[1];
  const int64_t nmt = (n_cfg * F + 63) / 64;
  return sizeof(float) * (size_t)kFaMaxSplit * (size_t)round_up(N, 64) * (size_t)(128 * nmt);
}

// ---------------------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------------------
template <typename T>
static bool prefix_ok(const T* h, int n, int64_t total, int64_t min_each) {
  if (!h || h[0] != 0) return false;
  for (int s = 0; s < n; ++s)
    if (h[s + 1] - h[s] < min_each) return false;
  return h[n] == total;
}

static mts_status validate_problem(const mts_problem* pb) {
  if (!pb) return MTS_EINVAL;
  if (pb->n_struct < 1 || pb->n_ports < 1 || pb->n_vertices < 0 || pb->n_freq < 0 ||
      pb->n_points < 0 || pb->n_loss < 0)
    return MTS_EINVAL;
  if (!(pb->wire_radius > 0.0) || !std::isfinite(pb->wire_radius)) return MTS_EINVAL;
  if (!prefix_ok(pb->h_port_off, pb->n_struct, pb->n_ports, 1)) return MTS_EINVAL;
  if (!prefix_ok(pb->h_point_off, pb->n_struct, pb->n_points, 0)) return MTS_EINVAL;
  if (!prefix_ok(pb->h_freq_off, pb->n_struct, pb->n_freq, 0)) return MTS_EINVAL;
  if (pb->n_loss > 0 && !prefix_ok(pb->h_loss_off, pb->n_struct, pb->n_loss, 0)) return MTS_EINVAL;
  if (!pb->port_off || !pb->point_off || !pb->freq_off || !pb->loop_vtx_off || !pb->R)
    return MTS_EINVAL;
  if (pb->n_vertices > 0 && (!pb->vx || !pb->vy || !pb->vz)) return MTS_EINVAL;
  if (pb->n_points > 0 && (!pb->px || !pb->py || !pb->pz)) return MTS_EINVAL;
  if (pb->n_loss > 0 && (!pb->loss_off || !pb->loss_idx)) return MTS_EINVAL;
  for (int s = 0; s < pb->n_struct; ++s)
    if (pb->h_port_off[s + 1] - pb->h_port_off[s] > kMaxPorts) return MTS_EUNSUPPORTED;
  return MTS_OK;
}

static mts_status validate_prec(mts_precision prec) {
  return (prec == MTS_FP64 || prec == MTS_MIXED || prec == MTS_BF16) ? MTS_OK : MTS_EINVAL;
}

static int64_t simt_threshold(const mts_eval* ev) {
  return ev->simt_max_sys == 0 ? kSimtSys : ev->simt_max_sys;
}

static mts_status validate_eval(const mts_problem* pb, const mts_eval* ev) {
  if (!ev) return MTS_EINVAL;
  if (ev->large_threads != 0 && ev->large_threads != 128 && ev->large_threads != 256 &&
      ev->large_threads != 512)
    return MTS_EINVAL;
  if ((ev->reg_widen & ~7) != 0) return MTS_EINVAL;
  if (ev->n_cfg < 0) return MTS_EINVAL;
  if (ev->n_cfg > 0 && !ev->C) return MTS_EINVAL;
  if (pb->n_freq > 0 && (!ev->omega || !ev->V)) return MTS_EINVAL;
  if (ev->loss_mode != MTS_LOSS_ABS && ev->loss_mode != MTS_LOSS_COMPLEX) return MTS_EINVAL;
  if (ev->target && pb->n_loss <= 0) return MTS_EINVAL;
  if (!(ev->refine_tol >= 0.0) || ev->max_refine < 0) return MTS_EINVAL;
  return MTS_OK;
}

static bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

static mts_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MTS_OK : MTS_ECUDA; }

static int max_loss_points(const mts_problem* pb) {
  int m = 0;
  if (pb->n_loss > 0)
    for (int s = 0; s < pb->n_struct; ++s) {
      int L = pb->h_loss_off[s + 1] - pb->h_loss_off[s];
      if (L > m) m = L;
    }
  return m;
}

static SolveArgs solve_args(const mts_problem* pb, mts_precision prec, const void* basis,
                            const mts_eval* ev, void* tape, const ProblemSums& ps) {
  BasisLayout bl = basis_layout(pb, prec);
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  PlanLayout pl = plan_layout(pb->n_struct);
  const char* B = static_cast<const char*>(basis);
  char* T = static_cast<char*>(tape);
  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_struct = pb->n_struct;
  a.n_freq = pb->n_freq;
  a.n_ports = pb->n_ports;
  a.port_off = pb->port_off;
  a.freq_off = pb->freq_off;
  a.loss_off = pb->loss_off;
  a.R = pb->R;
  a.t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  a.M64 = reinterpret_cast<const double*>(B + bl.M64);
  a.M32hi = reinterpret_cast<const float*>(B + bl.M32hi);
  a.M32lo = reinterpret_cast<const float*>(B + bl.M32lo);
  a.Hl64 = reinterpret_cast<const double*>(B + bl.Hloss64);
  a.Hl32 = reinterpret_cast<const float*>(B + bl.Hloss32);
  a.HlT32 = reinterpret_cast<const float*>(B + bl.HlossT32);
  a.n_cfg = ev->n_cfg;
  a.C = ev->C;
  a.omega = ev->omega;
  a.V = ev->V;
  a.target = ev->target;
  a.target_per_cfg = ev->target_per_cfg;
  a.loss_mode = ev->loss_mode;
  a.loss_weight = ev->loss_weight;
  a.loss_offset = ev->loss_offset;
  a.tol = ev->refine_tol > 0.0 ? ev->refine_tol : 1e-8;
  a.max_refine = ev->max_refine > 0 ? ev->max_refine : 8;
  a.sumFN = ps.sumFN;
  a.sumFL = ps.sumFL;
  a.I = reinterpret_cast<double*>(T + tl.I);
  a.loss_part = reinterpret_cast<double*>(T + tl.loss_part);
  a.grad_part = reinterpret_cast<double*>(T + tl.grad_part);
  a.status = reinterpret_cast<int32_t*>(T + tl.status);
  a.npieces = n_pieces(prec);
  a.Bop = a.npieces ? reinterpret_cast<__nv_bfloat16*>(T + tl.Bop) : nullptr;
  a.bop_off = reinterpret_cast<const int64_t*>(T + tl.plan + pl.bop_off);
  a.lu_off = reinterpret_cast<const int64_t*>(T + tl.plan + pl.lu_off);
  a.lu = T + tl.lu;
  a.lu_order = reinterpret_cast<int32_t*>(T + tl.lu_ord);
  a.fac = (pb->keep_factors && prec != MTS_FP64) ? static_cast<void*>(T + tl.fac) : nullptr;
  a.mu_out = reinterpret_cast<double*>(T + tl.mu_loss);
  a.max_loss = max_loss_points(pb);
  a.large_threads = ev->large_threads;
  a.reg_widen = ev->reg_widen;
  a.rhs_in = nullptr;
  return a;
}

static ReduceArgs reduce_args(const mts_problem* pb, mts_precision prec, const void* basis,
                              const mts_eval* ev, void* tape, const ProblemSums& ps) {
  BasisLayout bl = basis_layout(pb, prec);
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  char* T = static_cast<char*>(tape);
  ReduceArgs r;
  std::memset(&r, 0, sizeof(r));
  r.n_struct = pb->n_struct;
  r.n_freq = pb->n_freq;
  r.n_ports = pb->n_ports;
  r.port_off = pb->port_off;
  r.freq_off = pb->freq_off;
  r.loss_off = pb->n_loss > 0 ? pb->loss_off : nullptr;
  r.t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  r.n_cfg = ev->n_cfg;
  r.sumFN = ps.sumFN;
  r.loss_part = reinterpret_cast<const double*>(T + tl.loss_part);
  r.grad_part = reinterpret_cast<const double*>(T + tl.grad_part);
  r.dldc = reinterpret_cast<double*>(T + tl.dldc);
  r.lossv = reinterpret_cast<double*>(T + tl.lossv);
  r.normalise = 1;
  return r;
}

cudaError_t superpose_core(const mts_problem* pb, mts_precision prec, const void* basis,
                           int64_t n_cfg, int64_t simt_thr, const double* I,
                           const __nv_bfloat16* Bop, const void* plan, int32_t* err, void* B_out,
                           cudaStream_t st) {
  BasisLayout bl = basis_layout(pb, prec);
  PlanLayout pl = plan_layout(pb->n_struct);
  ProblemSums ps = problem_sums(pb, prec);
  const char* B = static_cast<const char*>(basis);
  const char* Pl = static_cast<const char*>(plan);
  SuperposeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_struct = pb->n_struct;
  a.n_freq = pb->n_freq;
  a.n_ports = pb->n_ports;
  a.port_off = pb->port_off;
  a.freq_off = pb->freq_off;
  a.point_off = pb->point_off;
  a.t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  a.n_cfg = n_cfg;
  a.sumFN = ps.sumFN;
  a.sumFP = ps.sumFP;
  bop_elems(pb, n_cfg, n_pieces(prec), &a.total_units, &a.total_simt, &a.max_simt, simt_thr);
  a.unit_off = reinterpret_cast<const int64_t*>(Pl + pl.unit_off);
  a.simt_off = reinterpret_cast<const int64_t*>(Pl + pl.simt_off);
  a.H = B + bl.H;
  a.I = I;
  a.Aop = reinterpret_cast<const __nv_bfloat16*>(B + bl.Aop);
  a.Bop = Bop;
  a.bop_off = reinterpret_cast<const int64_t*>(Pl + pl.bop_off);
  a.npieces = n_pieces(prec);
  a.B_out = B_out;
  a.err = err;
  if (pb->n_struct == 1 && a.total_units > 0) {
    a.uni.on = 1;
    a.uni.N = pb->h_port_off[1];
    a.uni.F = pb->h_freq_off[1];
    a.uni.P = pb->h_point_off[1];
    a.uni.nkc = (a.uni.N + kChunkK - 1) / kChunkK;
    a.uni.nptile = (a.uni.P + kTileP - 1) / kTileP;
    a.uni.nntile = (2 * n_cfg * a.uni.F + kTileN - 1) / kTileN;
  }
  return launch_superpose(a, prec, st);
}

}  // namespace mts

using namespace mts;

extern "C" {

const char* mts_status_string(mts_status s) {
  switch (s) {
    case MTS_OK: return "MTS_OK";
    case MTS_EINVAL: return "MTS_EINVAL: invalid argument";
    case MTS_EWORKSPACE: return "MTS_EWORKSPACE: buffer smaller than the size query";
    case MTS_ECUDA: return "MTS_ECUDA: CUDA launch or runtime call failed";
    case MTS_ENOCONV: return "MTS_ENOCONV: a system missed the refinement tolerance";
    case MTS_EUNSUPPORTED: return "MTS_EUNSUPPORTED: geometry or size not handled";
  }
  return "unknown mts_status";
}

const char* mts_version(void) { return "mts 0.1.0 (sm_103a)"; }

uint64_t mts_launch_count(void) { return g_launches.load(); }

size_t mts_basis_bytes(const mts_problem* pb, mts_precision prec) {
  if (validate_problem(pb) != MTS_OK || validate_prec(prec) != MTS_OK) return 0;
  return basis_layout(pb, prec).total;
}

mts_status mts_build_basis(const mts_problem* pb, mts_precision prec, void* basis,
                           size_t basis_bytes, mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !basis || !aligned256(basis)) return MTS_EINVAL;
  BasisLayout bl = basis_layout(pb, prec);
  if (basis_bytes < bl.total) return MTS_EWORKSPACE;
  ProblemSums ps = problem_sums(pb, prec);
  return cuda_status(launch_build_basis(pb, prec, basis, bl, ps, (cudaStream_t)stream));
}

mts_status mts_basis_export(const mts_problem* pb, mts_precision prec, const void* basis,
                            double* H_out, double* M_out, mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !basis) return MTS_EINVAL;
  BasisLayout bl = basis_layout(pb, prec);
  ProblemSums ps = problem_sums(pb, prec);
  return cuda_status(
      launch_export_basis(pb, prec, basis, bl, ps, H_out, M_out, (cudaStream_t)stream));
}

mts_status mts_basis_status(const mts_problem* pb, mts_precision prec, const void* basis,
                            mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !basis) return MTS_EINVAL;
  BasisLayout bl = basis_layout(pb, prec);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MTS_ECUDA;
  int32_t w = 0;
  if (cudaMemcpy(&w, static_cast<const char*>(basis) + bl.status, sizeof(w),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return MTS_ECUDA;
  if (w & (1 << 30)) return MTS_EINVAL;  // a component code outside {0, 1, 2}
  return w ? MTS_EUNSUPPORTED : MTS_OK;
}

size_t mts_tape_bytes(const mts_problem* pb, int64_t n_cfg, mts_precision prec) {
  if (validate_problem(pb) != MTS_OK || validate_prec(prec) != MTS_OK || n_cfg < 0) return 0;
  return tape_layout(pb, n_cfg, prec).total;
}

static mts_status check_solve_args(const mts_problem* pb, mts_precision prec, const void* basis,
                                   const mts_eval* ev, void* tape, size_t tape_bytes) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !basis || !tape || !aligned256(tape)) return MTS_EINVAL;
  v = validate_eval(pb, ev);
  if (v != MTS_OK) return v;
  if (tape_bytes < tape_layout(pb, ev->n_cfg, prec).total) return MTS_EWORKSPACE;
  return MTS_OK;
}

mts_status mts_solve(const mts_problem* pb, mts_precision prec, const void* basis,
                     const mts_eval* ev, double* I_out, double* loss_out, void* tape,
                     size_t tape_bytes, mts_stream stream) {
  mts_status v = check_solve_args(pb, prec, basis, ev, tape, tape_bytes);
  if (v != MTS_OK) return v;
  if (loss_out && !ev->target) return MTS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ProblemSums ps = problem_sums(pb, prec);
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  PlanLayout pl = plan_layout(pb->n_struct);
  char* T = static_cast<char*>(tape);
  cudaError_t e = cudaMemsetAsync(T + tl.err, 0, 16, st);
  if (e == cudaSuccess)
    e = launch_plan(pb, ev->n_cfg, n_pieces(prec), simt_threshold(ev),
                    reinterpret_cast<int64_t*>(T + tl.plan + pl.bop_off),
                    reinterpret_cast<int64_t*>(T + tl.plan + pl.unit_off),
                    reinterpret_cast<int64_t*>(T + tl.plan + pl.lu_off),
                    reinterpret_cast<int64_t*>(T + tl.plan + pl.simt_off), st);
  if (e != cudaSuccess) return MTS_ECUDA;
  SolveArgs a = solve_args(pb, prec, basis, ev, tape, ps);
  a.I_out = I_out;
  e = launch_solve(a, prec, ps, st);
  if (e == cudaErrorNotSupported) return MTS_EUNSUPPORTED;
  if (e != cudaSuccess) return MTS_ECUDA;
  if (ev->target) {
    ReduceArgs r = reduce_args(pb, prec, basis, ev, tape, ps);
    r.loss_out = loss_out;
    e = launch_reduce(r, st);
    if (e != cudaSuccess) return MTS_ECUDA;
  }
  return MTS_OK;
}

mts_status mts_superpose(const mts_problem* pb, mts_precision prec, const void* basis,
                         const mts_eval* ev, const void* tape, void* B_out, mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !basis || !tape || !B_out) return MTS_EINVAL;
  v = validate_eval(pb, ev);
  if (v != MTS_OK) return v;
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  const char* T = static_cast<const char*>(tape);
  return cuda_status(superpose_core(
      pb, prec, basis, ev->n_cfg, simt_threshold(ev), reinterpret_cast<const double*>(T + tl.I),
      reinterpret_cast<const __nv_bfloat16*>(T + tl.Bop), T + tl.plan,
      reinterpret_cast<int32_t*>(const_cast<char*>(T) + tl.err), B_out, (cudaStream_t)stream));
}

mts_status mts_forward(const mts_problem* pb, mts_precision prec, const void* basis,
                       const mts_eval* ev, void* B_out, double* I_out, double* loss_out,
                       void* tape, size_t tape_bytes, mts_stream stream) {
  mts_status v = mts_solve(pb, prec, basis, ev, I_out, loss_out, tape, tape_bytes, stream);
  if (v != MTS_OK || !B_out) return v;
  return mts_superpose(pb, prec, basis, ev, tape, B_out, stream);
}

mts_status mts_backward(const mts_problem* pb, mts_precision prec, const void* basis,
                        const mts_eval* ev, void* tape, size_t tape_bytes, const void* grad_B,
                        const double* grad_loss, double* grad_C, mts_stream stream) {
  mts_status v = check_solve_args(pb, prec, basis, ev, tape, tape_bytes);
  if (v != MTS_OK) return v;
  if (!grad_C) return MTS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ProblemSums ps = problem_sums(pb, prec);
  BasisLayout bl = basis_layout(pb, prec);
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  char* T = static_cast<char*>(tape);
  const double* gfield = nullptr;
  cudaError_t e = cudaSuccess;
  if (grad_B) {
    FieldAdjArgs fa;
    std::memset(&fa, 0, sizeof(fa));
    fa.n_struct = pb->n_struct;
    fa.n_freq = pb->n_freq;
    fa.n_ports = pb->n_ports;
    fa.port_off = pb->port_off;
    fa.freq_off = pb->freq_off;
    fa.point_off = pb->point_off;
    fa.t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
    fa.n_cfg = ev->n_cfg;
    fa.sumFN = ps.sumFN;
    fa.sumFP = ps.sumFP;
    fa.H = static_cast<const char*>(basis) + bl.H;
    fa.grad_B = grad_B;
    fa.u = reinterpret_cast<double*>(T + tl.mu);
    const int64_t F0 = pb->h_freq_off[1];
    if (pb->n_struct == 1 && prec != MTS_FP64 && pb->n_points > 0 &&
        use_tensor_path(n_pieces(prec), ev->n_cfg, F0, simt_threshold(ev))) {
      // tensor cores: the basis operand image doubles as the MN-major H operand
      FaTcArgs t;
      std::memset(&t, 0, sizeof(t));
      t.F = (int)F0;
      t.N = pb->h_port_off[1];
      t.P = pb->h_point_off[1];
      t.nsys = ev->n_cfg * F0;
      t.sumFP = ps.sumFP;
      t.fpo = 0;
      t.nkc = (t.N + kChunkK - 1) / kChunkK;
      t.nptile = (t.P + kTileP - 1) / kTileP;
      t.nsteps = (int)((t.P + 63) / 64);
      t.nmt = (t.nsys + 63) / 64;
      t.npad = round_up(t.N, 64);
      t.rows_pad = 128 * t.nmt;
      static int sms = 0;
      if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
          sms = 1;
      }
      // K splits: about four work units per SM, at most kFaMaxSplit and one per K step
      int64_t ns = (4 * (int64_t)sms + t.nmt * t.nkc - 1) / (t.nmt * t.nkc);
      ns = ns < 1 ? 1 : (ns > kFaMaxSplit ? kFaMaxSplit : ns);
      if (ns > t.nsteps) ns = t.nsteps;
      t.nsplit = (int)ns;
      t.units = t.nmt * t.nkc * t.nsplit;
      t.Aop = reinterpret_cast<const __nv_bfloat16*>(static_cast<const char*>(basis) + bl.Aop);
      t.gB = static_cast<const float2*>(grad_B);
      t.part = reinterpret_cast<float*>(T + tl.fa_part);
      t.err = reinterpret_cast<int32_t*>(T + tl.err);
      e = launch_field_adjoint_tc(t, prec, fa.u, ps.sumFN, 0, st);
    } else {
      e = launch_field_adjoint_rhs(fa, prec, ps.max_ports, st);
    }
    if (e != cudaSuccess) return MTS_ECUDA;
    SolveArgs a = solve_args(pb, prec, basis, ev, tape, ps);
    a.rhs_in = reinterpret_cast<const double*>(T + tl.mu);
    a.Bop = nullptr;
    a.target = nullptr;
    e = launch_solve(a, prec, ps, st);
    if (e == cudaErrorNotSupported) return MTS_EUNSUPPORTED;
    if (e != cudaSuccess) return MTS_ECUDA;
    ReduceArgs r = reduce_args(pb, prec, basis, ev, tape, ps);
    r.normalise = 0;
    r.dldc = reinterpret_cast<double*>(T + tl.gfield);
    e = launch_reduce(r, st);
    if (e != cudaSuccess) return MTS_ECUDA;
    gfield = r.dldc;
  }
  e = launch_grad_combine(ev->n_cfg, pb->n_struct, pb->n_ports, pb->port_off, grad_loss,
                          reinterpret_cast<const double*>(T + tl.dldc), gfield, grad_C, st);
  return cuda_status(e);
}

mts_status mts_tape_status(const mts_problem* pb, int64_t n_cfg, mts_precision prec,
                           const void* tape, int64_t* n_bad, mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !tape || n_cfg < 0) return MTS_EINVAL;
  TapeLayout tl = tape_layout(pb, n_cfg, prec);
  char* T = const_cast<char*>(static_cast<const char*>(tape));
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* words = reinterpret_cast<int32_t*>(T + tl.err);
  if (launch_count_bad(reinterpret_cast<const int32_t*>(T + tl.status), n_cfg * pb->n_freq,
                       words + 1, st) != cudaSuccess)
    return MTS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MTS_ECUDA;
  int32_t h[2] = {0, 0};
  if (cudaMemcpy(h, words, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return MTS_ECUDA;
  if (n_bad) *n_bad = h[1];
  if (h[0] != 0) return MTS_ECUDA;  // a kernel gave up on a bounded wait
  return h[1] ? MTS_ENOCONV : MTS_OK;
}

mts_status mts_system_status(const mts_problem* pb, int64_t n_cfg, mts_precision prec,
                             const void* tape, int32_t* status_out, mts_stream stream) {
  mts_status v = validate_problem(pb);
  if (v != MTS_OK) return v;
  if (validate_prec(prec) != MTS_OK || !tape || !status_out || n_cfg < 0) return MTS_EINVAL;
  if (n_cfg == 0 || pb->n_freq == 0) return MTS_OK;
  TapeLayout tl = tape_layout(pb, n_cfg, prec);
  return cuda_status(cudaMemcpyAsync(status_out, static_cast<const char*>(tape) + tl.status,
                                     sizeof(int32_t) * (size_t)n_cfg * pb->n_freq,
                                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

mts_status mts_param_grad(const mts_problem* pb, mts_precision prec, const void* basis,
                          const mts_eval* ev, const void* tape, size_t tape_bytes,
                          const double* grad_loss, double* grad_R, double* grad_L,
                          double* grad_omega, double* grad_V, mts_stream stream) {
  mts_status v = check_solve_args(pb, prec, basis, ev, const_cast<void*>(tape), tape_bytes);
  if (v != MTS_OK) return v;
  if (!ev->target || (!grad_R && !grad_L && !grad_omega && !grad_V)) return MTS_EINVAL;
  BasisLayout bl = basis_layout(pb, prec);
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  ProblemSums ps = problem_sums(pb, prec);
  const char* T = static_cast<const char*>(tape);
  const char* Bz = static_cast<const char*>(basis);
  const DevTables t = dev_tables(basis, bl, pb->n_struct, pb->n_freq);
  const double* I = reinterpret_cast<const double*>(T + tl.I);
  const double* mu = reinterpret_cast<const double*>(T + tl.mu_loss);
  cudaError_t e = cudaSuccess;
  if (grad_R || grad_L)
    e = launch_param_grad(ev->n_cfg, pb->n_struct, pb->n_ports, pb->port_off, pb->freq_off,
                          pb->loss_off, t, ps.sumFN, ev->omega, I, mu, grad_loss, grad_R, grad_L,
                          (cudaStream_t)stream);
  if (e == cudaSuccess && (grad_omega || grad_V))
    e = launch_omega_v_grad(ev->n_cfg, pb->n_freq, pb->n_struct, pb->n_ports, pb->port_off,
                            pb->freq_off, pb->loss_off, t, ps.sumFN, ev->omega, ev->C,
                            reinterpret_cast<const double*>(Bz + bl.M64), I, mu, grad_loss,
                            grad_omega, grad_V, (cudaStream_t)stream);
  return cuda_status(e);
}

mts_status mts_adam_step(int64_t n, const mts_adam* opt, double* C, double* u,
                         const double* grad_C, double* m, double* v, int64_t* step,
                         const double* loss, int64_t n_loss, double* loss_history,
                         int64_t history_len, mts_stream stream) {
  if (n < 0 || !opt || n_loss < 0 || history_len < 0) return MTS_EINVAL;
  const mts_adam& o = *opt;
  if (!(std::isfinite(o.lr) && o.lr >= 0.0) || !(std::isfinite(o.eps) && o.eps >= 0.0))
    return MTS_EINVAL;
  if (!(o.beta1 >= 0.0 && o.beta1 < 1.0) || !(o.beta2 >= 0.0 && o.beta2 < 1.0)) return MTS_EINVAL;
  if (o.projection != MTS_PROJ_NONE && o.projection != MTS_PROJ_CLIP && o.projection != MTS_PROJ_TANH)
    return MTS_EINVAL;
  if (o.projection != MTS_PROJ_NONE && !(o.c_min < o.c_max && std::isfinite(o.c_min) && std::isfinite(o.c_max)))
    return MTS_EINVAL;
  if (!step || (n > 0 && (!C || !grad_C || !m || !v))) return MTS_EINVAL;
  if (n > 0 && o.projection == MTS_PROJ_TANH && !u) return MTS_EINVAL;
  if (loss_history && n_loss > 0 && !loss) return MTS_EINVAL;
  return cuda_status(launch_adam(n, o, C, u, grad_C, m, v, step, loss, loss_history ? n_loss : 0,
                                 loss_history, history_len, (cudaStream_t)stream));
}

}  // extern "C"
