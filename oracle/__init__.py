"""FP64 CPU oracle for the capacitance -> Bz forward map and its gradient.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The CUDA product path neither imports this package nor
links ``liboracle.so``; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, ``double complex``, every function citing the
paper passage it follows). This module compiles it with gcc on first use (or when the source
is newer than the library) and wraps it for numpy arrays. Structures are handled one at a
time; the caller loops over the structures of a ragged batch.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MU0 = 4e-7 * np.pi


def build(force: bool = False) -> str:
    """Compile liboracle.so (OpenMP over configurations; no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ct.CDLL(_LIB)
            d, i32, i64, p = ct.c_double, ct.c_int32, ct.c_int64, ct.c_void_p
            lib.oracle_segment_bz.restype = d
            lib.oracle_segment_bz.argtypes = [d] * 10
            lib.oracle_basis.restype = None
            lib.oracle_basis.argtypes = [i32, p, p, p, p, i64, p, p, p, d, p]
            lib.oracle_basis_comp.restype = None
            lib.oracle_basis_comp.argtypes = [i32, p, p, p, p, i64, p, p, p, p, d, p]
            lib.oracle_segment_pair_inductance.restype = ct.c_int
            lib.oracle_segment_pair_inductance.argtypes = [p, p, p, p, d, ct.c_int, p]
            lib.oracle_inductance.restype = ct.c_int
            lib.oracle_inductance.argtypes = [i32, p, p, p, p, d, p, p]
            lib.oracle_assemble.restype = None
            lib.oracle_assemble.argtypes = [i32, p, p, d, p, p]
            lib.oracle_lu.restype = ct.c_int
            lib.oracle_lu.argtypes = [i32, p, p]
            lib.oracle_lu_solve.restype = None
            lib.oracle_lu_solve.argtypes = [i32, p, p, p]
            lib.oracle_solve_loaded.restype = ct.c_int
            lib.oracle_solve_loaded.argtypes = [i32, p, p, p, p]
            lib.oracle_forward.restype = ct.c_int
            lib.oracle_forward.argtypes = [i32, i64, p, p, p, i64, p, i32, p, p, i32, p, p, i32,
                                           i32, p, p, p]
            lib.oracle_forward_w.restype = ct.c_int
            lib.oracle_forward_w.argtypes = [i32, i64, p, p, p, i64, p, i32, p, p, i32, p, p, i32,
                                             i32, p, p, p, p, p]
            lib.oracle_gradient_adjoint_w.restype = ct.c_int
            lib.oracle_gradient_adjoint_w.argtypes = [i32, i64, p, p, p, i64, p, i32, p, p, i32,
                                                      p, p, i32, i32, p, p, p]
            lib.oracle_gradient_adjoint.restype = ct.c_int
            lib.oracle_gradient_adjoint.argtypes = [i32, i64, p, p, p, i64, p, i32, p, p, i32, p,
                                                    p, i32, i32, p]
            lib.oracle_gradient_field.restype = ct.c_int
            lib.oracle_gradient_field.argtypes = [i32, i64, p, p, p, i64, p, i32, p, p, p, p]
            lib.oracle_segment_pair_quadrature.restype = d
            lib.oracle_segment_pair_quadrature.argtypes = [p, p, p, p, ct.c_int]
            lib.oracle_gauss_legendre.restype = None
            lib.oracle_gauss_legendre.argtypes = [ct.c_int, p, p]
            lib.oracle_gradient_omega_v.restype = ct.c_int
            lib.oracle_gradient_omega_v.argtypes = [i32, p, p, p, i64, p, i32, p, p, i32, p, p,
                                                    i32, i32, p, p]
            lib.oracle_gradient_rl.restype = ct.c_int
            lib.oracle_gradient_rl.argtypes = [i32, p, p, p, i64, p, i32, p, p, i32, p, p, i32,
                                               i32, p, p]
            lib.oracle_dcurrents_dC.restype = ct.c_int
            lib.oracle_dcurrents_dC.argtypes = [i32, p, p, d, p, p, p]
            lib.oracle_sroute.restype = ct.c_int
            lib.oracle_sroute.argtypes = [i32, p, p, i32, d, d, d, p, p, p]
            sr = [i32, i32, i32, i64, i32, p, p, p, p, p, i64, p, i32, p, p, i32, p, p]
            lib.oracle_sroute_forward.restype = ct.c_int
            lib.oracle_sroute_forward.argtypes = sr + [p, p, p]
            lib.oracle_sroute_gradient.restype = ct.c_int
            lib.oracle_sroute_gradient.argtypes = sr + [p]
            lib.oracle_num_threads.restype = ct.c_int
            lib.oracle_num_threads.argtypes = []
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _ptr(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def segment_bz(r1, r2, p, wire_radius: float) -> float:
    """Bz of one straight segment r1 -> r2 carrying 1 A at point p (Biot-Savart)."""
    return float(_load().oracle_segment_bz(*map(float, r1), *map(float, r2), *map(float, p),
                                           float(wire_radius)))


def basis(loop_vtx_off, vx, vy, vz, px, py, pz, wire_radius: float, comp=None) -> np.ndarray:
    """H[p, k] = B component comp[p] (0: z, 1: x, 2: y; None: z) at point p per ampere in
    loop k."""
    off = _i32(loop_vtx_off)
    vx, vy, vz, px, py, pz = map(_f64, (vx, vy, vz, px, py, pz))
    n, P = len(off) - 1, len(px)
    H = np.zeros((P, n), dtype=np.float64)
    c = None if comp is None else np.ascontiguousarray(comp, dtype=np.int8)
    _load().oracle_basis_comp(n, _ptr(off), _ptr(vx), _ptr(vy), _ptr(vz), P, _ptr(px), _ptr(py),
                              _ptr(pz), _ptr(c), float(wire_radius), _ptr(H))
    return H


def segment_pair_inductance(a0, a1, b0, b1, wire_radius: float, same_segment: bool = False):
    """Partial mutual inductance of two straight filaments; returns (status, value)."""
    a0, a1, b0, b1 = map(_f64, (a0, a1, b0, b1))
    out = np.zeros(1)
    st = _load().oracle_segment_pair_inductance(_ptr(a0), _ptr(a1), _ptr(b0), _ptr(b1),
                                                float(wire_radius), int(same_segment), _ptr(out))
    return int(st), float(out[0])


def segment_pair_quadrature(a0, a1, b0, b1, order: int = 16):
    """Neumann integral of two straight filaments by Gauss-Legendre (inner integral exact)."""
    a0, a1, b0, b1 = map(_f64, (a0, a1, b0, b1))
    return float(_load().oracle_segment_pair_quadrature(_ptr(a0), _ptr(a1), _ptr(b0), _ptr(b1),
                                                         int(order)))


def gauss_legendre(n: int):
    """Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]."""
    x, w = np.zeros(n), np.zeros(n)
    _load().oracle_gauss_legendre(int(n), _ptr(x), _ptr(w))
    return x, w


def inductance(loop_vtx_off, vx, vy, vz, wire_radius: float, L_self=None):
    """Inductance matrix M (self on the diagonal); returns (status, M)."""
    off = _i32(loop_vtx_off)
    vx, vy, vz = map(_f64, (vx, vy, vz))
    n = len(off) - 1
    M = np.zeros((n, n), dtype=np.float64)
    ls = _f64(L_self) if L_self is not None else None
    st = _load().oracle_inductance(n, _ptr(off), _ptr(vx), _ptr(vy), _ptr(vz), float(wire_radius),
                                   _ptr(ls), _ptr(M))
    return int(st), M


def assemble(M, R, omega: float, C) -> np.ndarray:
    """A = diag(R) + j w M + diag(1/(j w C))."""
    M, R, C = _f64(M), _f64(R), _f64(C)
    n = len(R)
    A = np.zeros((n, n), dtype=np.complex128)
    _load().oracle_assemble(n, _ptr(M), _ptr(R), float(omega), _ptr(C), _ptr(A))
    return A


def lu(A):
    """Partial-pivoting LU; returns (status, LU, piv)."""
    A = _c128(A).copy()
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    st = _load().oracle_lu(n, _ptr(A), _ptr(piv))
    return int(st), A, piv


def lu_solve(LU, piv, b):
    LU, piv = _c128(LU), _i32(piv)
    x = _c128(b).copy()
    _load().oracle_lu_solve(LU.shape[0], _ptr(LU), _ptr(piv), _ptr(x))
    return x


def solve_loaded(Z, Zload, V):
    """(Z + diag(Zload)) I = V; returns (status, I)."""
    Z, Zload, V = _c128(Z), _c128(Zload), _c128(V)
    n = len(V)
    out = np.zeros(n, dtype=np.complex128)
    st = _load().oracle_solve_loaded(n, _ptr(Z), _ptr(Zload), _ptr(V), _ptr(out))
    return int(st), out


def _target_arr(target, mode):
    t = _f64(target.view(np.float64) if np.iscomplexobj(target) else target)
    return t


def forward(H, M, R, C, omega, V, loss_idx=None, target=None, mode: int = 0,
            target_per_cfg: bool = False, want_B: bool = True, want_loss: bool = True,
            weight=None, offset=None):
    """Forward map of one structure: returns dict with I [n_cfg,F,N], B [n_cfg,F,P], loss.
    weight [F, L] real and offset [F, L] complex (optional) turn the objective term of a loss
    point into that of weight * (B + offset) (the enhancement objective of Sec. IV-B)."""
    H, M, R, C, omega = _f64(H), _f64(M), _f64(R), _f64(np.atleast_2d(C)), _f64(np.atleast_1d(omega))
    V = _c128(np.atleast_2d(V))
    P, N = H.shape
    n_cfg, F = C.shape[0], len(omega)
    Iout = np.zeros((n_cfg, F, N), dtype=np.complex128)
    Bout = np.zeros((n_cfg, F, P), dtype=np.complex128) if want_B else None
    L = 0 if loss_idx is None else len(loss_idx)
    li = _i64(loss_idx if loss_idx is not None else np.zeros(0, np.int64))
    do_loss = want_loss and L > 0
    t = _target_arr(np.asarray(target), mode) if do_loss else np.zeros(1)
    loss = np.zeros(n_cfg) if do_loss else None
    w = None if weight is None else _f64(weight)
    o = None if offset is None else _c128(offset)
    bad = _load().oracle_forward_w(N, P, _ptr(H), _ptr(M), _ptr(R), n_cfg, _ptr(C), F,
                                   _ptr(omega), _ptr(V), L, _ptr(li), _ptr(t),
                                   int(target_per_cfg), int(mode), _ptr(w), _ptr(o), _ptr(Iout),
                                   _ptr(Bout), _ptr(loss))
    return {"I": Iout, "B": Bout, "loss": loss, "n_singular": int(bad)}


def gradient(H, M, R, C, omega, V, loss_idx, target, mode: int = 0, target_per_cfg: bool = False,
             weight=None, offset=None):
    """d loss / d C (adjoint form), shape [n_cfg, N]; weight/offset as in forward()."""
    H, M, R, C, omega = _f64(H), _f64(M), _f64(R), _f64(np.atleast_2d(C)), _f64(np.atleast_1d(omega))
    V = _c128(np.atleast_2d(V))
    P, N = H.shape
    n_cfg, F = C.shape[0], len(omega)
    li = _i64(loss_idx)
    t = _target_arr(np.asarray(target), mode)
    g = np.zeros((n_cfg, N))
    w = None if weight is None else _f64(weight)
    o = None if offset is None else _c128(offset)
    _load().oracle_gradient_adjoint_w(N, P, _ptr(H), _ptr(M), _ptr(R), n_cfg, _ptr(C), F,
                                      _ptr(omega), _ptr(V), len(li), _ptr(li), _ptr(t),
                                      int(target_per_cfg), int(mode), _ptr(w), _ptr(o), _ptr(g))
    return g


def gradient_rl(H, M, R, C, omega, V, loss_idx, target, mode: int = 0, target_per_cfg: bool = False):
    """(d loss / d R, d loss / d L) with L_k = M_kk the self inductances, shapes [n_cfg, N]."""
    H, M, R, C, omega = _f64(H), _f64(M), _f64(R), _f64(np.atleast_2d(C)), _f64(np.atleast_1d(omega))
    V = _c128(np.atleast_2d(V))
    P, N = H.shape
    n_cfg, F = C.shape[0], len(omega)
    li = _i64(loss_idx)
    t = _target_arr(np.asarray(target), mode)
    gR = np.zeros((n_cfg, N))
    gL = np.zeros((n_cfg, N))
    _load().oracle_gradient_rl(N, _ptr(H), _ptr(M), _ptr(R), n_cfg, _ptr(C), F, _ptr(omega),
                               _ptr(V), len(li), _ptr(li), _ptr(t), int(target_per_cfg), int(mode),
                               _ptr(gR), _ptr(gL))
    return gR, gL


def gradient_omega_v(H, M, R, C, omega, V, loss_idx, target, mode: int = 0,
                     target_per_cfg: bool = False):
    """(d loss / d omega with V fixed [n_cfg, F], d loss / d V cotangent [n_cfg, F, N])."""
    H, M, R, C, omega = _f64(H), _f64(M), _f64(R), _f64(np.atleast_2d(C)), _f64(np.atleast_1d(omega))
    V = _c128(np.atleast_2d(V))
    P, N = H.shape
    n_cfg, F = C.shape[0], len(omega)
    li = _i64(loss_idx)
    t = _target_arr(np.asarray(target), mode)
    gw = np.zeros((n_cfg, F))
    gV = np.zeros((n_cfg, F, N), np.complex128)
    _load().oracle_gradient_omega_v(N, _ptr(H), _ptr(M), _ptr(R), n_cfg, _ptr(C), F, _ptr(omega),
                                    _ptr(V), len(li), _ptr(li), _ptr(t), int(target_per_cfg),
                                    int(mode), _ptr(gw), _ptr(gV))
    return gw, gV


def gradient_field(H, M, R, C, omega, V, gB):
    """dL/dC for a field cotangent gB [n_cfg, F, P] (torch convention dL/dRe + j dL/dIm)."""
    H, M, R, C, omega = _f64(H), _f64(M), _f64(R), _f64(np.atleast_2d(C)), _f64(np.atleast_1d(omega))
    V, gB = _c128(np.atleast_2d(V)), _c128(gB)
    P, N = H.shape
    n_cfg, F = C.shape[0], len(omega)
    g = np.zeros((n_cfg, N))
    _load().oracle_gradient_field(N, P, _ptr(H), _ptr(M), _ptr(R), n_cfg, _ptr(C), F, _ptr(omega),
                                  _ptr(V), _ptr(gB), _ptr(g))
    return g


def dcurrents_dC(M, R, omega: float, C, V):
    """dI_i/dC_k as an array [k, i] (direct form, one solve per capacitor)."""
    M, R, C, V = _f64(M), _f64(R), _f64(C), _c128(V)
    n = len(R)
    out = np.zeros((n, n), dtype=np.complex128)
    st = _load().oracle_dcurrents_dC(n, _ptr(M), _ptr(R), float(omega), _ptr(C), _ptr(V), _ptr(out))
    return int(st), out


def sroute(Z, Zload, drive: int, Z0: float, P_in: float, omega: float, C=None, want_dI=False):
    """Scattering-parameter route (Eq. 3-7, Eq. 10); returns (status, I, dI or None)."""
    Z, Zload = _c128(Z), _c128(Zload)
    n = Z.shape[0]
    Cv = _f64(C if C is not None else np.ones(n))
    Iout = np.zeros(n, dtype=np.complex128)
    dI = np.zeros((n, n), dtype=np.complex128) if want_dI else None
    st = _load().oracle_sroute(n, _ptr(Z), _ptr(Zload), int(drive), float(Z0), float(P_in),
                               float(omega), _ptr(Cv), _ptr(Iout), _ptr(dI))
    return int(st), Iout, dI


def sroute_pipeline(S0, field, Sconst, rows, cols, svar, loss_idx=None, target=None,
                    mode: int = 0, want_B: bool = True, want_loss: bool = True, weight=None,
                    offset=None):
    """The S-parameter pipeline (Sec. III-A, Eq. 3-7) for a batch of variable S-parameters.
    S0 [F, n0, n0], field [F, P, n0], Sconst [F, n, n] (n = n0 + n1), svar [n_batch, F, nS],
    rows/cols [nS], target [F, n1, L] (real, or complex for mode 1).
    weight [F, n1, L] real / offset [F, n1, L] complex: objective on weight * (B + offset).
    Returns dict W [n_batch, F, n0, n1], B [n_batch, n1, F, P], loss [n_batch], n_singular."""
    S0, field, Sconst, svar = _c128(S0), _c128(field), _c128(Sconst), _c128(svar)
    F, n0 = S0.shape[0], S0.shape[1]
    n1 = Sconst.shape[1] - n0
    P = field.shape[1]
    n_batch, nS = svar.shape[0], svar.shape[2]
    li = _i64(loss_idx if loss_idx is not None else np.zeros(0, np.int64))
    L = len(li)
    do_loss = want_loss and L > 0
    t = _target_arr(np.asarray(target), mode) if do_loss else np.zeros(1)
    W = np.zeros((n_batch, F, n0, n1), dtype=np.complex128)
    B = np.zeros((n_batch, n1, F, P), dtype=np.complex128) if want_B else None
    loss = np.zeros(n_batch) if do_loss else None
    bad = _load().oracle_sroute_forward(n0, n1, F, P, nS, _ptr(_i32(rows)), _ptr(_i32(cols)),
                                        _ptr(S0), _ptr(field), _ptr(Sconst), n_batch, _ptr(svar),
                                        L, _ptr(li), _ptr(t), int(mode),
                                        _ptr(None if weight is None else _f64(weight)),
                                        _ptr(None if offset is None else _c128(offset)), _ptr(W),
                                        _ptr(B), _ptr(loss))
    return {"W": W, "B": B, "loss": loss, "n_singular": int(bad)}


def sroute_gradient(S0, field, Sconst, rows, cols, svar, loss_idx, target, mode: int = 0,
                    weight=None, offset=None):
    """d objective / d svar (Eq. 10, forward mode), torch's convention, [n_batch, F, nS]."""
    S0, field, Sconst, svar = _c128(S0), _c128(field), _c128(Sconst), _c128(svar)
    F, n0 = S0.shape[0], S0.shape[1]
    n1 = Sconst.shape[1] - n0
    P = field.shape[1]
    n_batch, nS = svar.shape[0], svar.shape[2]
    li = _i64(loss_idx)
    t = _target_arr(np.asarray(target), mode)
    g = np.zeros((n_batch, F, nS), dtype=np.complex128)
    bad = _load().oracle_sroute_gradient(n0, n1, F, P, nS, _ptr(_i32(rows)), _ptr(_i32(cols)),
                                         _ptr(S0), _ptr(field), _ptr(Sconst), n_batch,
                                         _ptr(svar), len(li), _ptr(li), _ptr(t), int(mode),
                                         _ptr(None if weight is None else _f64(weight)),
                                         _ptr(None if offset is None else _c128(offset)),
                                         _ptr(g))
    assert bad == 0, bad
    return g
