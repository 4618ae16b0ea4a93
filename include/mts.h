/*
 * mts.h -- C ABI of the GB300 (sm_103a) library for the differentiable forward map
 * from tuning capacitances C to the normal field Bz of capacitively loaded loop arrays,
 * and for its adjoint gradient.
 *
 * Method (paper: "Differentiable Cosimulator for Electrically Reconfigurable Structures",
 * Mueller, Philipp, Guenther):
 *   (a) field basis  H[p][k] = Bz (or Bx, By: pcomp) at point p per ampere in loop k,
 *       from the Biot-Savart law over straight wire segments (Sec. I-A: circuit model plus Biot-Savart for
 *       structures small against the wavelength); coupling M[k][l] = self and mutual
 *       inductances (Eq. 12-13, here from Neumann partial inductances).
 *   (b) port solve   (diag(R) + j w M + diag(1/(j w C))) I = V per configuration and
 *       frequency (Eq. 2 and Eq. 11 give the loaded-loop impedance; Eq. 6 is the same
 *       linear network solve in scattering form).
 *   (c) superposition B = H I (Eq. 7).
 *   (d) objective    mean over frequencies and loss points of (|Bz| - t)^2 (Eq. 1; the
 *       paper optimises |Hz| at collocation points, Sec. IV-C), or of |Bz - t|^2.
 *   (adj) gradient   dloss/dC_k = sum_f Im(mu_k I_k)/(w C_k^2), mu = A^-1 H^T conj(G),
 *       from d(A^-1) = -A^-1 dA A^-1 (Eq. 8-9); A is complex symmetric so the stored
 *       factorisation serves the adjoint solve.
 *
 * Conventions
 *   - SI units; time dependence e^{+j w t} (Eq. 2, Eq. 11); mu0 = 4 pi 1e-7 H/m.
 *   - Complex arrays are interleaved (re, im) pairs of double (complex128) unless stated.
 *   - Every pointer marked "device" must point to device memory of the current CUDA
 *     device; "host" pointers to host memory. All buffers are caller-owned. The library
 *     allocates no device memory and never synchronises the stream, except the
 *     mts_*_status readers, which say so.
 *   - Every entry point validates its host-visible arguments before any launch and
 *     returns MTS_EINVAL (nothing launched) on a violation. Device-side table contents
 *     are trusted to match their host copies.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL means the legacy default
 *     stream). Results are valid after the stream reaches that point.
 *   - Thread safety: calls on different streams with disjoint output buffers may run
 *     concurrently; calls that write the same tape or basis buffer must be ordered.
 */
#ifndef MTS_H
#define MTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mts_stream; /* cudaStream_t */

typedef enum {
  MTS_OK = 0,
  MTS_EINVAL = 1,       /* invalid argument; nothing was launched */
  MTS_EWORKSPACE = 2,   /* basis or tape buffer smaller than the *_bytes query */
  MTS_ECUDA = 3,        /* a CUDA launch or runtime call failed */
  MTS_ENOCONV = 4,      /* (status readers) a system missed the refinement tolerance */
  MTS_EUNSUPPORTED = 5  /* geometry or size the kernels do not handle */
} mts_status;

typedef enum {
  /* FP64 everywhere: basis, FP64 LU with partial pivoting, FP64 superposition;
     B_out is complex128. Target error against the FP64 oracle <= 1e-10. */
  MTS_FP64 = 0,
  /* FP32 basis with FP64 near-field terms; FP32 complex LU with partial pivoting and
     iterative refinement on residuals taken in FP64-equivalent precision; superposition
     on the tensor cores with three-way bf16 operand splitting and FP32 accumulation;
     B_out is complex64. Target error <= 1e-6. */
  MTS_MIXED = 1,
  /* As MTS_MIXED but the superposition uses single bf16 operands (one tensor-core pass);
     B_out is complex64. Target error <= 1e-2 on B. */
  MTS_BF16 = 2
} mts_precision;

typedef enum {
  MTS_LOSS_ABS = 0,     /* (|Bz| - t)^2, t real: the paper's magnitude objective */
  MTS_LOSS_COMPLEX = 1  /* |Bz - t|^2, t complex (re, im) */
} mts_loss_mode;

/*
 * A batch of independent structures (n_struct >= 1). Structure s owns
 *   ports      port_off[s]  .. port_off[s+1]-1    (port k = loop k, closed by one capacitor)
 *   points     point_off[s] .. point_off[s+1]-1   (field points, metres)
 *   freqs      freq_off[s]  .. freq_off[s+1]-1    (angular frequencies in mts_eval.omega)
 *   loss pts   loss_off[s]  .. loss_off[s+1]-1    (entries of loss_idx; global point
 *                                                   indices inside structure s)
 * Loop k is the closed polyline of vertices loop_vtx_off[k] .. loop_vtx_off[k+1]-1, the
 * last joined back to the first; its orientation fixes the sign of its current. Each
 * structure is coupled only within itself. Inductances come from the Neumann integral over
 * segment pairs: in closed form for parallel and perpendicular pairs and for oblique
 * pairs that share an end point (the corners of a non-rectilinear polygon: two rays from
 * the corner, lengths l and m, far ends R apart, integrate to
 * 2 [l atanh(m/(l+R)) + m atanh(l/(m+R))] times mu0/(4 pi) and the direction cosine), by
 * quadrature (composite 16-point Gauss-Legendre, inner integral exact) for the other
 * oblique pairs. So polygonal loops of any shape get L and M from their geometry; L_self,
 * when given, overrides the diagonal.
 * Offset tables are given twice, identical: host copies (h_*) plan launches, device
 * copies are read by the kernels. Limits: 1 <= ports per structure <= 1024 (more give
 * MTS_EUNSUPPORTED from every entry point, before any launch). Systems of up to 64 ports
 * are solved in registers; larger ones by a blocked LU whose factors live in the tape.
 */
typedef struct mts_problem {
  int32_t n_struct;
  int32_t n_ports;     /* total over structures */
  int32_t n_vertices;  /* total */
  int32_t n_freq;      /* total frequencies, sum over structures */
  int64_t n_points;    /* total */
  int32_t n_loss;      /* total loss points (0: no objective possible) */
  double wire_radius;  /* metres, > 0 */
  const int32_t* h_port_off;   /* host   [n_struct+1] */
  const int64_t* h_point_off;  /* host   [n_struct+1] */
  const int32_t* h_freq_off;   /* host   [n_struct+1] */
  const int32_t* h_loss_off;   /* host   [n_struct+1] */
  const int32_t* port_off;     /* device [n_struct+1] */
  const int64_t* point_off;    /* device [n_struct+1] */
  const int32_t* freq_off;     /* device [n_struct+1] */
  const int32_t* loss_off;     /* device [n_struct+1] */
  const int32_t* loop_vtx_off; /* device [n_ports+1] */
  const double* vx;            /* device [n_vertices] */
  const double* vy;
  const double* vz;
  const double* px;            /* device [n_points] */
  const double* py;
  const double* pz;
  const int64_t* loss_idx;     /* device [n_loss] */
  const double* R;             /* device [n_ports], ohm, > 0 */
  const double* L_self;        /* device [n_ports] henry, or NULL (partial inductances) */
  const int8_t* pcomp;         /* device [n_points] field component per point: 0 = Bz (the
                                  paper's normal field), 1 = Bx, 2 = By; NULL = Bz everywhere.
                                  Another code makes that point's basis rows NaN and
                                  mts_basis_status report MTS_EINVAL. */
  int32_t keep_factors;        /* nonzero: the tape also holds the LU factors of the systems
                                  of 33..64 ports (37,120 bytes per configuration and
                                  frequency, MTS_MIXED / MTS_BF16), written by every solve
                                  and read by mts_backward's field-cotangent solve instead of
                                  factoring again. Larger systems always keep theirs. */
} mts_problem;

/*
 * Per-call inputs. Layouts, with FN = sum_s F_s N_s and FL = sum_s F_s L_s:
 *   C       device [n_cfg][n_ports]             farad, finite, nonzero (Eq. 1 leaves C
 *                                                unbounded, so negative C is accepted)
 *   omega   device [n_freq]                      rad/s, > 0
 *   V       device complex [FN]: structure s at sum_{s'<s} F_s' N_s', as [F_s][N_s] volt
 *   target  device, NULL = no objective; real [FL] (MTS_LOSS_ABS) or complex [FL]
 *           (MTS_LOSS_COMPLEX), structure s at sum_{s'<s} F_s' L_s' as [F_s][L_s];
 *           with target_per_cfg != 0 one such block per configuration ([n_cfg][...]).
 * refine_tol: a system has converged when the estimated relative error of its solution,
 *   |d_k|^2 / |d_(k-1)| / |x| for the last two refinement corrections (d_0 = x_0), is at most
 *   refine_tol (MTS_MIXED, MTS_BF16; 0 selects 1e-8). Refinement also stops early when the
 *   correction no longer halves (the residual precision, about cond(A) * 2^-45 relative,
 *   is reached); such a system is flagged if it missed refine_tol. max_refine: refinement
 *   steps per solve (0 selects 8).
 * Schedule (results agree to rounding whatever the choice; an autotuner may time them):
 *   simt_max_sys  superposition of a structure on the SIMT kernel when its configurations x
 *                 frequencies are at most this, else on the tensor cores (MTS_MIXED,
 *                 MTS_BF16); 0 selects 16, a negative value puts every structure on the
 *                 tensor cores. Memory does not depend on it.
 *   large_threads threads per system of the blocked solve for N > 64: 128, 256 or 512 (512
 *                 runs as 256 for MTS_FP64). With MTS_MIXED / MTS_BF16 and at most 128
 *                 ports in the class, 256 and 512 keep the matrix in shared memory (one
 *                 system per SM: faster per system, slower for a full machine) and 128
 *                 keeps it in the factor scratch of the tape. 0 selects 128 for N <= 128,
 *                 256 for N <= 256 and 512 above. Other values give MTS_EINVAL.
 *   reg_widen     bit c (c = 0, 1, 2 for the classes of N <= 8, 16, 32 ports) runs that
 *                 class in the register-resident kernel of the next wider mapping (16, 32 or
 *                 64 threads per system: a half warp, a warp, a two-warp CTA) instead of its
 *                 own (8, 16, 32); 0 keeps each class in its own. Other bits give
 *                 MTS_EINVAL. Memory does not depend on it.
 * Enhancement objective (Sec. IV-B: beta = |B_MTS| / |B_ref|, the field with the structure
 * over that of a reference run without it): with loss_weight w and loss_offset o (layout of
 * the target without its configuration blocks; either may be NULL) the objective term of a
 * loss point is evaluated on w (B + o) instead of B, and every gradient follows. With
 * w = 1/|B_ref|, o = the incident field and target = beta_target the objective is the mean of
 * (beta - beta_target)^2.
 */
typedef struct mts_eval {
  int64_t n_cfg;
  const double* C;
  const double* omega;
  const double* V;
  const double* target;
  int32_t target_per_cfg;
  int32_t loss_mode; /* mts_loss_mode */
  double refine_tol;
  int32_t max_refine;
  int32_t simt_max_sys;
  int32_t large_threads;
  const double* loss_weight; /* device [FL] real, or NULL (1) */
  const double* loss_offset; /* device complex [FL], or NULL (0) */
  int32_t reg_widen;
} mts_eval;

/* Human-readable name of a status code (static string). */
const char* mts_status_string(mts_status s);

/* Library version string (static). */
const char* mts_version(void);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t mts_launch_count(void);

/* ---------------------------------------------------------------------------------
 * (a) basis: H, M and derived tables, in a library-defined layout inside a caller
 * buffer of mts_basis_bytes(...) bytes (device, 256-byte aligned). Built once per
 * geometry and precision; read-only afterwards. Returns MTS_EWORKSPACE if
 * basis_bytes is too small.
 * --------------------------------------------------------------------------------- */
size_t mts_basis_bytes(const mts_problem* pb, mts_precision prec);
mts_status mts_build_basis(const mts_problem* pb, mts_precision prec, void* basis,
                           size_t basis_bytes, mts_stream stream);

/* Copy of the field basis as FP64 [P_s][N_s] blocks (structure s at sum P N), and of
 * the inductance matrix as FP64 [N_s][N_s] blocks (at sum N^2); either output may be
 * NULL. Device outputs. For testing and for callers that want the basis itself. */
mts_status mts_basis_export(const mts_problem* pb, mts_precision prec, const void* basis,
                            double* H_out, double* M_out, mts_stream stream);

/* Synchronises `stream`, then reports MTS_EINVAL if a component code in pcomp was not 0, 1
 * or 2, else MTS_EUNSUPPORTED if a segment pair needed for M could not be integrated (two
 * collinear segments overlapped by more than rounding). */
mts_status mts_basis_status(const mts_problem* pb, mts_precision prec, const void* basis,
                            mts_stream stream);

/* ---------------------------------------------------------------------------------
 * Tape: the per-call state written by the forward calls and read by mts_backward
 * (currents I, tensor-core operand copies of I, per-system objective and gradient
 * partials, per-system status, backward scratch, and the LU factors of systems with more
 * than 64 ports: 8 bytes (16 for MTS_FP64) per matrix element, per configuration and
 * frequency of such a structure). Device buffer of
 * mts_tape_bytes(...) bytes, 256-byte aligned.
 * --------------------------------------------------------------------------------- */
size_t mts_tape_bytes(const mts_problem* pb, int64_t n_cfg, mts_precision prec);

/* ---------------------------------------------------------------------------------
 * (b)+(d)+(adj) mts_solve: for every configuration b and frequency f of every
 * structure, assemble A = diag(R) + j w M + diag(1/(j w C_b)) (Eq. 2, 11), solve A I = V
 * (Eq. 6 in impedance form) with partial pivoting, and store I in the tape (and in
 * I_out, device complex [n_cfg][FN], if not NULL). If ev->target is not NULL it also
 * evaluates the objective at the loss points (Eq. 1) and the adjoint gradient
 * dloss/dC (Eq. 8-9) while the factors are resident; the loss is written to loss_out
 * (device [n_cfg][n_struct], may be NULL) and the gradient kept in the tape.
 * --------------------------------------------------------------------------------- */
mts_status mts_solve(const mts_problem* pb, mts_precision prec, const void* basis,
                     const mts_eval* ev, double* I_out, double* loss_out, void* tape,
                     size_t tape_bytes, mts_stream stream);

/* (c) mts_superpose: B = H I for the currents in the tape (Eq. 7). B_out is device
 * [n_cfg][sum_s F_s P_s] complex, structure s at sum_{s'<s} F_s' P_s' as [F_s][P_s]:
 * complex128 for MTS_FP64, complex64 (interleaved float re, im) otherwise. */
mts_status mts_superpose(const mts_problem* pb, mts_precision prec, const void* basis,
                         const mts_eval* ev, const void* tape, void* B_out,
                         mts_stream stream);

/* mts_forward = mts_solve followed by mts_superpose (B_out may be NULL: loss only). */
mts_status mts_forward(const mts_problem* pb, mts_precision prec, const void* basis,
                       const mts_eval* ev, void* B_out, double* I_out, double* loss_out,
                       void* tape, size_t tape_bytes, mts_stream stream);

/* (adj) mts_backward: grad_C (device [n_cfg][n_ports], overwritten) =
 *     grad_loss[b][s] * dloss_{b,s}/dC            (grad_loss device [n_cfg][n_struct];
 *                                                   needs a forward with a target)
 *   + dL/dC from a field cotangent grad_B         (device, same layout and element type
 *                                                   as B_out; torch convention
 *                                                   dL/dRe B + j dL/dIm B)
 * Either input may be NULL (both NULL gives zeros). `ev` must be the forward's. The
 * field-cotangent term re-solves A mu = H^T conj(grad_B) per system. For one-structure
 * MTS_MIXED / MTS_BF16 problems on the tensor-core superposition path, u = H^T conj(grad_B)
 * runs on the tensor cores with the split-bf16 basis operand (grad_B rounded to three bf16
 * pieces, FP32 partial sums over K ranges of points, the partials summed in FP64); otherwise
 * one FP32 sum per point block on the SIMT cores. */
mts_status mts_backward(const mts_problem* pb, mts_precision prec, const void* basis,
                        const mts_eval* ev, void* tape, size_t tape_bytes,
                        const void* grad_B, const double* grad_loss, double* grad_C,
                        mts_stream stream);

/* mts_param_grad: gradients of the objective with respect to the other parameters Fig. 2
 * of the paper names as optimisation variables (R, L, w) and to the drive, from the adjoint
 * solution mu the forward kept in the tape (d(A^-1) = -A^-1 dA A^-1, Eq. 8-9):
 *   grad_R[b][port]  = g sum_f -Re(mu_k I_k)            (dA/dR_k = e_k e_k^T)
 *   grad_L[b][port]  = g sum_f  w Im(mu_k I_k)          (L_k = M_kk, dA/dM_kk = j w e_k e_k^T)
 *   grad_omega[b][g] = g (Im(mu^T M I) + sum_k Im(mu_k I_k)/(w^2 C_k))  (V held fixed;
 *                      dA/dw = j M + diag(j/(w^2 C)))
 *   grad_V[b][FN]    = g conj(mu)                       (dL/dRe V + j dL/dIm V; complex)
 * with g = grad_loss[b][s] / (F_s L_s). Needs a preceding mts_solve / mts_forward on this
 * tape with ev->target (the objective's adjoint); covers the loss cotangent only (not a field
 * cotangent grad_B). grad_loss device [n_cfg][n_struct] or NULL (all ones); grad_R, grad_L
 * device [n_cfg][n_ports], grad_omega device [n_cfg][n_freq], grad_V device complex
 * [n_cfg][FN], each may be NULL (at least one given). grad_omega costs an N^2 FP64 product
 * per system. MTS_EINVAL if ev has no target or every output is NULL. */
mts_status mts_param_grad(const mts_problem* pb, mts_precision prec, const void* basis,
                          const mts_eval* ev, const void* tape, size_t tape_bytes,
                          const double* grad_loss, double* grad_R, double* grad_L,
                          double* grad_omega, double* grad_V, mts_stream stream);

/* Synchronises `stream` and summarises the per-system status of the last forward on
 * this tape: MTS_OK, or MTS_ENOCONV if any system missed the refinement tolerance or
 * met a non-finite value. If n_bad is not NULL it receives the number of such systems. */
mts_status mts_tape_status(const mts_problem* pb, int64_t n_cfg, mts_precision prec,
                           const void* tape, int64_t* n_bad, mts_stream stream);

/* Per-system status of the last forward on this tape, copied to status_out (device int32
 * [n_cfg][n_freq], the frequency index global as in mts_eval.omega): 0 converged, 1 missed
 * the refinement tolerance, 2 zero pivot or non-finite value (results written either way).
 * Enqueued on `stream`; no synchronisation. */
mts_status mts_system_status(const mts_problem* pb, int64_t n_cfg, mts_precision prec,
                             const void* tape, int32_t* status_out, mts_stream stream);

/* ---------------------------------------------------------------------------------
 * mts_solve_static: mts_solve without a tape, for callers that cannot allocate device
 * memory when they solve (a real-time loop that may not call the allocator, a plugin
 * whose host application owns every device allocation, a process with a fixed memory
 * budget). The paper has no counterpart; this is a deployment convenience.
 *
 * The per-call working state lives in one library-owned device array of
 * MTS_STATIC_SCRATCH_BYTES bytes, which every GPU that loads the library holds until the
 * process exits. The caller still passes the problem, the basis, the inputs (ev) and the
 * outputs, all as for mts_solve:
 *   I_out        device complex [n_cfg][FN] currents, or NULL
 *   loss_out     device [n_cfg][n_struct] objective, or NULL (needs ev->target)
 *   dloss_dC_out device [n_cfg][n_ports] dloss_{b,s}/dC of each port's own structure,
 *                or NULL (needs ev->target)
 * Returns MTS_EWORKSPACE, before any launch, when the work would need more than
 * MTS_STATIC_SCRATCH_BYTES (compare mts_tape_bytes(pb, n_cfg, prec)). Calls no device
 * allocator. Every call looks up the array's device address in the current context; the
 * first lookup in a context loads the library's device code, so make the first call on each
 * device before any stream capture. Returns MTS_OK once the work is enqueued: systems that
 * missed the refinement tolerance are reported by mts_solve_static_status, not here. Every
 * call on a device shares the one array, so calls whose GPU work overlaps in time (other
 * streams, other threads) race: order them on one stream. The array keeps the last call's contents; each
 * call clears what must start at zero and never reads a region it did not write.
 * --------------------------------------------------------------------------------- */
#define MTS_STATIC_SCRATCH_BYTES (32u << 20)
mts_status mts_solve_static(const mts_problem* pb, mts_precision prec, const void* basis,
                            const mts_eval* ev, double* I_out, double* loss_out,
                            double* dloss_dC_out, mts_stream stream);

/* Synchronises `stream` and summarises the per-system status words of the last
 * mts_solve_static call on this device, for the same (pb, n_cfg, prec): MTS_OK, MTS_ENOCONV
 * if any system missed the refinement tolerance or met a zero pivot or a non-finite value
 * (its results are written either way), or MTS_ECUDA. If n_bad is not NULL it receives the
 * number of such systems. Like mts_solve_static it allocates nothing: it counts the words in
 * the library's static array (the same reduction as mts_tape_status) and reads two words
 * back. MTS_EINVAL / MTS_EWORKSPACE for arguments mts_solve_static would reject. The paper
 * has no counterpart. */
mts_status mts_solve_static_status(const mts_problem* pb, int64_t n_cfg, mts_precision prec,
                                   int64_t* n_bad, mts_stream stream);

/* ---------------------------------------------------------------------------------
 * Optimisation loop (paper Sec. III-C: the capacitances are fitted by gradient descent with
 * Adam, at most 2000 epochs, learning rate 1e-13 for values of order 1e-12 F; Sec. V-B:
 * clipping to the tuning range, or a bounded tanh projection, keeps them realisable).
 *
 * mts_adam_step applies one Adam update (Kingma and Ba; the update order of PyTorch's Adam
 * without weight decay) to n parameters, with the step counter t in device memory so that
 * an epoch (mts_solve, mts_backward, mts_adam_step) can be captured once in a CUDA graph and
 * replayed:
 *   t  = *step + 1;  m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   th = th - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps);  *step = t
 * MTS_PROJ_NONE : th = C (device [n]), g = grad_C.
 * MTS_PROJ_CLIP : th = C, and C is clipped to [c_min, c_max] after the update.
 * MTS_PROJ_TANH : th = u (device [n], unconstrained), C = c_mid + c_half tanh(u) with
 *                 c_mid = (c_max + c_min)/2, c_half = (c_max - c_min)/2, and
 *                 g = grad_C c_half (1 - tanh(u)^2); C is rewritten from u after the update.
 * m, v: device [n] moment estimates (zero them before the first step); step: device int64
 * (zero before the first step). If loss_history is not NULL, the n_loss values of `loss`
 * (device; the objective the gradient came from) are copied to loss_history[(t-1) n_loss ..]
 * while t <= history_len. Returns MTS_EINVAL (nothing launched) for n < 0, a NULL buffer
 * the mode needs, lr or eps not finite and >= 0, betas outside [0, 1), or c_min >= c_max in
 * a bounded mode.
 * --------------------------------------------------------------------------------- */
typedef enum { MTS_PROJ_NONE = 0, MTS_PROJ_CLIP = 1, MTS_PROJ_TANH = 2 } mts_projection;

typedef struct mts_adam {
  double lr;      /* learning rate (the paper: 1e-13) */
  double beta1;   /* 0.9 */
  double beta2;   /* 0.999 */
  double eps;     /* 1e-8 */
  int32_t projection; /* mts_projection */
  double c_min, c_max; /* tuning range for MTS_PROJ_CLIP and MTS_PROJ_TANH, farad */
} mts_adam;

mts_status mts_adam_step(int64_t n, const mts_adam* opt, double* C, double* u,
                         const double* grad_C, double* m, double* v, int64_t* step,
                         const double* loss, int64_t n_loss, double* loss_history,
                         int64_t history_len, mts_stream stream);

/* =====================================================================================
 * Scattering-parameter route (paper Sec. III and III-A, Eq. 3-7, Eq. 10): the paper's own
 * pipeline, on a structure described by its S-matrix S0 and per-port fields exported from
 * any solver, with a network tensor S_C whose variable entries the caller computes (the
 * "user-defined preprocessing" of Sec. III-A, e.g. mts_rc_reflection below).
 *
 * With n = n0 + n1, per configuration b and frequency f:
 *   S_C   = S_C,const[f] + scatter(svar[b][f]) (entry i at row svar_row[i], column
 *           svar_col[i]; Sec. III-A steps 1-3)
 *   S11   = S_C[0:n0, 0:n0],  S12 = S_C[0:n0, n0:n]       (Fig. 1: S21, S22 do not reach
 *                                                           the structure's field)
 *   A     = 1 - S11 S0[f],    W = A^-1 S12                (Eq. 6: the wave ratio
 *                                                           V+res / V-exc, n0 x n1)
 *   Bcomb[b][c][f][p] = sum_k field[f][p][k] W[k][c]      (Eq. 7)
 * objective: mean over (f, c, loss point l) of (|Bcomb| - t)^2 or |Bcomb - t|^2, and its
 * gradient with respect to every svar entry (Eq. 10, evaluated in adjoint form: one solve
 * with A^H per system), in torch's convention dL/dRe + j dL/dIm.
 *
 * Solve: LU with partial pivoting of A in shared memory (FP32 for MTS_MIXED / MTS_BF16,
 * FP64 for MTS_FP64) with iterative refinement on FP64 residuals, stopping as for mts_eval's
 * refine_tol / max_refine. Superposition: the kernels of mts_superpose, with field[f] as the
 * real basis [Re field | Im field] of 2 n0 columns (complex field times complex W).
 * ===================================================================================== */
typedef struct mts_sparams {
  int32_t n0;        /* structure ports, 1 <= n0 <= 96 (more: MTS_EUNSUPPORTED) */
  int32_t n1;        /* external (excitation) ports, 1 <= n1 <= 8 (more: MTS_EUNSUPPORTED) */
  int32_t n_freq;    /* >= 1 */
  int64_t n_points;  /* >= 0 */
  int32_t n_svar;    /* variable S-parameters per (configuration, frequency), 1 .. 1024 */
  int32_t n_loss;    /* loss points, >= 0 */
  const int32_t* h_svar_row; /* host [n_svar]: row of S_C, 0 .. n-1 */
  const int32_t* h_svar_col; /* host [n_svar]: column of S_C, 0 .. n-1; (row, col) distinct */
  const double* S0;          /* device complex [n_freq][n0][n0] (Eq. 5: V-res = S0 V+res) */
  const double* field;       /* device complex [n_freq][n_points][n0]: one field component
                                at point p when port k receives a unit incident wave and the
                                other ports are matched (Eq. 7's B); NULL if n_points == 0 */
  const double* sc_const;    /* device complex [n_freq][n][n] S_C,const, or NULL (zero) */
  const int64_t* loss_idx;   /* device [n_loss] point indices (0 .. n_points-1, trusted) */
} mts_sparams;

/* Per-call inputs of the route.
 *   svar    device complex [n_cfg][n_freq][n_svar]
 *   target  device [n_freq][n1][n_loss], real (MTS_LOSS_ABS) or complex (MTS_LOSS_COMPLEX);
 *           NULL = no objective
 *   refine_tol, max_refine as in mts_eval (0 selects 1e-8 and 8).
 *   loss_weight device [n_freq][n1][n_loss] real, loss_offset device complex, same layout
 *           (either NULL): the objective term of a loss point is taken on w (Bcomb + o), as
 *           in mts_eval (the enhancement objective of Sec. IV-B with w = 1/|B_ref|). */
typedef struct mts_sroute_eval {
  int64_t n_cfg;
  const double* svar;
  const double* target;
  int32_t loss_mode; /* mts_loss_mode */
  double refine_tol;
  int32_t max_refine;
  const double* loss_weight;
  const double* loss_offset;
} mts_sroute_eval;

/* Basis of the route: the field as superposition operands, T[f] = S_C,const11 S0[f] (the
 * constant part of S11 S0), and the scatter tables of svar. Device buffer of
 * mts_sroute_basis_bytes(...) bytes, 256-byte aligned, written by mts_sroute_build (once per
 * S0, field and S_C,const; rebuild when any of them changes). */
size_t mts_sroute_basis_bytes(const mts_sparams* sp, mts_precision prec);
mts_status mts_sroute_build(const mts_sparams* sp, mts_precision prec, void* sbasis,
                            size_t sbasis_bytes, mts_stream stream);

/* Tape of the route (wave ratios, currents of the superposition, LU factors and pivots of
 * every system, objective partials, status): device buffer of mts_sroute_tape_bytes(...)
 * bytes, 256-byte aligned. */
size_t mts_sroute_tape_bytes(const mts_sparams* sp, int64_t n_cfg, mts_precision prec);

/* Eq. 3-7 for every configuration and frequency. Outputs (each may be NULL):
 *   B_out    device [n_cfg][n1][n_freq][n_points] complex (complex128 for MTS_FP64, else
 *            complex64): Bcomb
 *   W_out    device complex [n_cfg][n_freq][n0][n1]: the wave ratios
 *   loss_out device [n_cfg]: the objective (needs ev->target) */
mts_status mts_sroute_forward(const mts_sparams* sp, mts_precision prec, const void* sbasis,
                              const mts_sroute_eval* ev, void* B_out, double* W_out,
                              double* loss_out, void* tape, size_t tape_bytes,
                              mts_stream stream);

/* Eq. 10 in adjoint form: grad_svar (device complex [n_cfg][n_freq][n_svar], overwritten) =
 *     grad_loss[b] * dloss_b/dsvar          (grad_loss device [n_cfg], or NULL: no term;
 *                                             needs ev->target)
 *   + dL/dsvar of a field cotangent grad_B   (device, layout and type of B_out, or NULL)
 * `ev` must be the forward's (same svar). Entries in rows n0 .. n-1 (S21, S22) get 0. */
mts_status mts_sroute_backward(const mts_sparams* sp, mts_precision prec, const void* sbasis,
                               const mts_sroute_eval* ev, void* tape, size_t tape_bytes,
                               const void* grad_B, const double* grad_loss, double* grad_svar,
                               mts_stream stream);

/* Synchronises `stream` and summarises the per-system status of the last forward on this
 * tape: MTS_OK, or MTS_ENOCONV if a system missed the refinement tolerance, had a zero
 * pivot or met a non-finite value (n_bad, if not NULL, receives their number). */
mts_status mts_sroute_status(const mts_sparams* sp, int64_t n_cfg, mts_precision prec,
                             const void* tape, int64_t* n_bad, mts_stream stream);

/* Preprocessing for loads that are series RC circuits (Eq. 2: Z = R - j/(w C); Eq. 3:
 * Gamma = (Z - Z0)/(Z + Z0)): svar[b][f][svar_offset + k] = Gamma(R[b][k], C[b][k], w_f) for
 * k < n_loads, other entries untouched. R, C device [n_cfg][n_loads] (R may be NULL: 0 ohm),
 * omega device [n_freq], Z0 > 0 ohm, svar device complex [n_cfg][n_freq][svar_stride] with
 * svar_offset + n_loads <= svar_stride. */
mts_status mts_rc_reflection(int64_t n_cfg, int32_t n_freq, int32_t n_loads, const double* omega,
                             const double* R, const double* C, double Z0, int32_t svar_stride,
                             int32_t svar_offset, double* svar, mts_stream stream);

/* Its vector-Jacobian product: from grad_svar (device complex, the layout of svar above),
 *   grad_C[b][k] = sum_f Re(conj(g) dGamma/dC),  dGamma/dC = 2 Z0/(Z + Z0)^2 * j/(w C^2)
 *   grad_R[b][k] = sum_f Re(conj(g) dGamma/dR),  dGamma/dR = 2 Z0/(Z + Z0)^2
 * (overwritten; either may be NULL). */
mts_status mts_rc_reflection_vjp(int64_t n_cfg, int32_t n_freq, int32_t n_loads,
                                 const double* omega, const double* R, const double* C, double Z0,
                                 int32_t svar_stride, int32_t svar_offset,
                                 const double* grad_svar, double* grad_R, double* grad_C,
                                 mts_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* MTS_H */
