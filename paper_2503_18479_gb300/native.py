"""ctypes binding of libmts.so (include/mts.h): same names, argument marshalling only.

Device buffers are torch tensors (PyTorch supplies device memory and streams); every step
of the method runs in the library's CUDA kernels. If the library is missing this module
raises ImportError on use: there is no CPU path.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmts.so")

MTS_OK, MTS_EINVAL, MTS_EWORKSPACE, MTS_ECUDA, MTS_ENOCONV, MTS_EUNSUPPORTED = range(6)
MTS_FP64, MTS_MIXED, MTS_BF16 = 0, 1, 2
MTS_LOSS_ABS, MTS_LOSS_COMPLEX = 0, 1
PRECISIONS = {"fp64": MTS_FP64, "mixed": MTS_MIXED, "bf16": MTS_BF16}

# symbols declared in include/mts.h
EXPORTED = ["mts_status_string", "mts_version", "mts_launch_count", "mts_basis_bytes",
            "mts_build_basis", "mts_basis_export", "mts_basis_status", "mts_tape_bytes",
            "mts_solve", "mts_superpose", "mts_forward", "mts_backward", "mts_tape_status",
            "mts_solve_static", "mts_solve_static_status", "mts_adam_step", "mts_param_grad",
            "mts_sroute_basis_bytes", "mts_sroute_build", "mts_sroute_tape_bytes",
            "mts_sroute_forward", "mts_sroute_backward", "mts_sroute_status", "mts_rc_reflection",
            "mts_rc_reflection_vjp", "mts_system_status"]
MTS_PROJ_NONE, MTS_PROJ_CLIP, MTS_PROJ_TANH = 0, 1, 2
PROJECTIONS = {None: MTS_PROJ_NONE, "none": MTS_PROJ_NONE, "clip": MTS_PROJ_CLIP, "tanh": MTS_PROJ_TANH}


class MtsProblem(ct.Structure):
    _fields_ = [
        ("n_struct", ct.c_int32), ("n_ports", ct.c_int32), ("n_vertices", ct.c_int32),
        ("n_freq", ct.c_int32), ("n_points", ct.c_int64), ("n_loss", ct.c_int32),
        ("wire_radius", ct.c_double),
        ("h_port_off", ct.c_void_p), ("h_point_off", ct.c_void_p), ("h_freq_off", ct.c_void_p),
        ("h_loss_off", ct.c_void_p),
        ("port_off", ct.c_void_p), ("point_off", ct.c_void_p), ("freq_off", ct.c_void_p),
        ("loss_off", ct.c_void_p),
        ("loop_vtx_off", ct.c_void_p), ("vx", ct.c_void_p), ("vy", ct.c_void_p),
        ("vz", ct.c_void_p), ("px", ct.c_void_p), ("py", ct.c_void_p), ("pz", ct.c_void_p),
        ("loss_idx", ct.c_void_p), ("R", ct.c_void_p), ("L_self", ct.c_void_p),
        ("pcomp", ct.c_void_p), ("keep_factors", ct.c_int32),
    ]


class MtsEval(ct.Structure):
    _fields_ = [
        ("n_cfg", ct.c_int64), ("C", ct.c_void_p), ("omega", ct.c_void_p), ("V", ct.c_void_p),
        ("target", ct.c_void_p), ("target_per_cfg", ct.c_int32), ("loss_mode", ct.c_int32),
        ("refine_tol", ct.c_double), ("max_refine", ct.c_int32),
        ("simt_max_sys", ct.c_int32), ("large_threads", ct.c_int32),
        ("loss_weight", ct.c_void_p), ("loss_offset", ct.c_void_p), ("reg_widen", ct.c_int32),
    ]


class MtsAdam(ct.Structure):
    _fields_ = [("lr", ct.c_double), ("beta1", ct.c_double), ("beta2", ct.c_double),
                ("eps", ct.c_double), ("projection", ct.c_int32), ("c_min", ct.c_double),
                ("c_max", ct.c_double)]


class MtsSparams(ct.Structure):
    _fields_ = [
        ("n0", ct.c_int32), ("n1", ct.c_int32), ("n_freq", ct.c_int32), ("n_points", ct.c_int64),
        ("n_svar", ct.c_int32), ("n_loss", ct.c_int32), ("h_svar_row", ct.c_void_p),
        ("h_svar_col", ct.c_void_p), ("S0", ct.c_void_p), ("field", ct.c_void_p),
        ("sc_const", ct.c_void_p), ("loss_idx", ct.c_void_p),
    ]


class MtsSrouteEval(ct.Structure):
    _fields_ = [("n_cfg", ct.c_int64), ("svar", ct.c_void_p), ("target", ct.c_void_p),
                ("loss_mode", ct.c_int32), ("refine_tol", ct.c_double), ("max_refine", ct.c_int32),
                ("loss_weight", ct.c_void_p), ("loss_offset", ct.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libmts.so (raises ImportError if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -m paper_2503_18479_gb300.build_lib` (needs nvcc)")
            L = ct.CDLL(LIB_PATH)
            p, i32, i64, sz = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_size_t
            PP, PE = ct.POINTER(MtsProblem), ct.POINTER(MtsEval)
            L.mts_status_string.restype = ct.c_char_p
            L.mts_status_string.argtypes = [ct.c_int]
            L.mts_version.restype = ct.c_char_p
            L.mts_version.argtypes = []
            L.mts_launch_count.restype = ct.c_uint64
            L.mts_launch_count.argtypes = []
            L.mts_basis_bytes.restype = sz
            L.mts_basis_bytes.argtypes = [PP, ct.c_int]
            L.mts_build_basis.restype = ct.c_int
            L.mts_build_basis.argtypes = [PP, ct.c_int, p, sz, p]
            L.mts_basis_export.restype = ct.c_int
            L.mts_basis_export.argtypes = [PP, ct.c_int, p, p, p, p]
            L.mts_basis_status.restype = ct.c_int
            L.mts_basis_status.argtypes = [PP, ct.c_int, p, p]
            L.mts_tape_bytes.restype = sz
            L.mts_tape_bytes.argtypes = [PP, i64, ct.c_int]
            L.mts_solve.restype = ct.c_int
            L.mts_solve.argtypes = [PP, ct.c_int, p, PE, p, p, p, sz, p]
            L.mts_superpose.restype = ct.c_int
            L.mts_superpose.argtypes = [PP, ct.c_int, p, PE, p, p, p]
            L.mts_forward.restype = ct.c_int
            L.mts_forward.argtypes = [PP, ct.c_int, p, PE, p, p, p, p, sz, p]
            L.mts_backward.restype = ct.c_int
            L.mts_backward.argtypes = [PP, ct.c_int, p, PE, p, sz, p, p, p, p]
            L.mts_solve_static.restype = ct.c_int
            L.mts_solve_static.argtypes = [PP, ct.c_int, p, PE, p, p, p, p]
            L.mts_solve_static_status.restype = ct.c_int
            L.mts_solve_static_status.argtypes = [PP, i64, ct.c_int, ct.POINTER(ct.c_int64), p]
            L.mts_param_grad.restype = ct.c_int
            L.mts_param_grad.argtypes = [PP, ct.c_int, p, PE, p, sz, p, p, p, p, p, p]
            L.mts_adam_step.restype = ct.c_int
            L.mts_adam_step.argtypes = [i64, ct.POINTER(MtsAdam), p, p, p, p, p, p, p, i64, p, i64, p]
            PS, PSE = ct.POINTER(MtsSparams), ct.POINTER(MtsSrouteEval)
            d = ct.c_double
            L.mts_sroute_basis_bytes.restype = sz
            L.mts_sroute_basis_bytes.argtypes = [PS, ct.c_int]
            L.mts_sroute_build.restype = ct.c_int
            L.mts_sroute_build.argtypes = [PS, ct.c_int, p, sz, p]
            L.mts_sroute_tape_bytes.restype = sz
            L.mts_sroute_tape_bytes.argtypes = [PS, i64, ct.c_int]
            L.mts_sroute_forward.restype = ct.c_int
            L.mts_sroute_forward.argtypes = [PS, ct.c_int, p, PSE, p, p, p, p, sz, p]
            L.mts_sroute_backward.restype = ct.c_int
            L.mts_sroute_backward.argtypes = [PS, ct.c_int, p, PSE, p, sz, p, p, p, p]
            L.mts_sroute_status.restype = ct.c_int
            L.mts_sroute_status.argtypes = [PS, i64, ct.c_int, p, ct.POINTER(ct.c_int64), p]
            L.mts_rc_reflection.restype = ct.c_int
            L.mts_rc_reflection.argtypes = [i64, i32, i32, p, p, p, d, i32, i32, p, p]
            L.mts_rc_reflection_vjp.restype = ct.c_int
            L.mts_rc_reflection_vjp.argtypes = [i64, i32, i32, p, p, p, d, i32, i32, p, p, p, p]
            L.mts_system_status.restype = ct.c_int
            L.mts_system_status.argtypes = [PP, i64, ct.c_int, p, p, p]
            L.mts_tape_status.restype = ct.c_int
            L.mts_tape_status.argtypes = [PP, i64, ct.c_int, p, ct.POINTER(ct.c_int64), p]
            _lib = L
    return _lib


class MtsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {mts_status_string(code)}")
        self.code = code


def _check(code: int, where: str):
    if code != MTS_OK:
        raise MtsError(code, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream(stream) -> ct.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


# ---------------------------------------------------------------------------------------
# problem / eval holders (keep the tensors that the ctypes structs point to alive)
# ---------------------------------------------------------------------------------------
class Problem:
    """Device and host copies of a batch of structures (mts_problem)."""

    def __init__(self, flat: dict, wire_radius: float, device="cuda", keep_factors: bool = False):
        def dev(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)
        self.h_port_off = np.ascontiguousarray(flat["port_off"], np.int32)
        self.h_point_off = np.ascontiguousarray(flat["point_off"], np.int64)
        self.h_freq_off = np.ascontiguousarray(flat["freq_off"], np.int32)
        self.h_loss_off = np.ascontiguousarray(flat["loss_off"], np.int32)
        self.d = {
            "port_off": dev(flat["port_off"], np.int32), "point_off": dev(flat["point_off"], np.int64),
            "freq_off": dev(flat["freq_off"], np.int32), "loss_off": dev(flat["loss_off"], np.int32),
            "loop_vtx_off": dev(flat["loop_vtx_off"], np.int32),
            "vx": dev(flat["vx"], np.float64), "vy": dev(flat["vy"], np.float64),
            "vz": dev(flat["vz"], np.float64), "px": dev(flat["px"], np.float64),
            "py": dev(flat["py"], np.float64), "pz": dev(flat["pz"], np.float64),
            "loss_idx": dev(flat["loss_idx"], np.int64), "R": dev(flat["R"], np.float64),
        }
        if flat.get("L_self") is not None:
            self.d["L_self"] = dev(flat["L_self"], np.float64)
        if flat.get("pcomp") is not None:
            self.d["pcomp"] = dev(flat["pcomp"], np.int8)
        n_struct = len(self.h_port_off) - 1
        c = MtsProblem()
        c.n_struct = n_struct
        c.n_ports = int(self.h_port_off[-1])
        c.n_vertices = len(flat["vx"])
        c.n_freq = int(self.h_freq_off[-1])
        c.n_points = int(self.h_point_off[-1])
        c.n_loss = int(self.h_loss_off[-1])
        c.wire_radius = float(wire_radius)
        c.h_port_off = self.h_port_off.ctypes.data
        c.h_point_off = self.h_point_off.ctypes.data
        c.h_freq_off = self.h_freq_off.ctypes.data
        c.h_loss_off = self.h_loss_off.ctypes.data
        for k in ("port_off", "point_off", "freq_off", "loss_off", "loop_vtx_off", "vx", "vy",
                  "vz", "px", "py", "pz", "loss_idx", "R"):
            setattr(c, k, self.d[k].data_ptr() if self.d[k].numel() else None)
        c.L_self = self.d["L_self"].data_ptr() if "L_self" in self.d else None
        c.pcomp = self.d["pcomp"].data_ptr() if "pcomp" in self.d else None
        c.keep_factors = 1 if keep_factors else 0
        self.c = c
        self.n_struct = n_struct

    @property
    def ref(self):
        return ct.byref(self.c)


class Eval:
    """Per-call inputs (mts_eval): C [n_cfg, n_ports], omega, V (complex), target."""

    def __init__(self, C: torch.Tensor, omega: torch.Tensor, V: torch.Tensor,
                 target: Optional[torch.Tensor] = None, target_per_cfg: bool = False,
                 loss_mode: int = MTS_LOSS_ABS, refine_tol: float = 0.0, max_refine: int = 0,
                 simt_max_sys: int = 0, large_threads: int = 0,
                 loss_weight: Optional[torch.Tensor] = None,
                 loss_offset: Optional[torch.Tensor] = None, reg_widen: int = 0):
        self.C = C.contiguous()
        self.loss_weight = None if loss_weight is None else loss_weight.contiguous()
        self.loss_offset = None if loss_offset is None else loss_offset.contiguous()
        self.omega = omega.contiguous()
        self.V = V.contiguous()
        self.target = None if target is None else target.contiguous()
        e = MtsEval()
        e.n_cfg = self.C.shape[0]
        e.C = self.C.data_ptr()
        e.omega = self.omega.data_ptr()
        e.V = self.V.data_ptr()
        e.target = None if self.target is None else self.target.data_ptr()
        e.target_per_cfg = int(target_per_cfg)
        e.loss_mode = int(loss_mode)
        e.refine_tol = float(refine_tol)
        e.max_refine = int(max_refine)
        e.simt_max_sys = int(simt_max_sys)
        e.large_threads = int(large_threads)
        e.reg_widen = int(reg_widen)
        e.loss_weight = None if self.loss_weight is None else self.loss_weight.data_ptr()
        e.loss_offset = None if self.loss_offset is None else self.loss_offset.data_ptr()
        self.c = e

    @property
    def n_cfg(self) -> int:
        return int(self.c.n_cfg)

    @property
    def ref(self):
        return ct.byref(self.c)


# ---------------------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------------------
def mts_status_string(code: int) -> str:
    return lib().mts_status_string(int(code)).decode()


def mts_version() -> str:
    return lib().mts_version().decode()


def mts_launch_count() -> int:
    return int(lib().mts_launch_count())


def mts_basis_bytes(pb: Problem, prec) -> int:
    return int(lib().mts_basis_bytes(pb.ref, _prec(prec)))


def mts_build_basis(pb: Problem, prec, basis: torch.Tensor, stream=None):
    _check(lib().mts_build_basis(pb.ref, _prec(prec), _ptr(basis), basis.numel() * basis.element_size(),
                                 _stream(stream)), "mts_build_basis")


def mts_basis_export(pb: Problem, prec, basis: torch.Tensor, H_out=None, M_out=None, stream=None):
    _check(lib().mts_basis_export(pb.ref, _prec(prec), _ptr(basis), _ptr(H_out), _ptr(M_out),
                                  _stream(stream)), "mts_basis_export")


def mts_basis_status(pb: Problem, prec, basis: torch.Tensor, stream=None) -> int:
    return int(lib().mts_basis_status(pb.ref, _prec(prec), _ptr(basis), _stream(stream)))


def mts_tape_bytes(pb: Problem, n_cfg: int, prec) -> int:
    return int(lib().mts_tape_bytes(pb.ref, int(n_cfg), _prec(prec)))


def mts_solve(pb, prec, basis, ev: Eval, I_out=None, loss_out=None, tape=None, stream=None):
    _check(lib().mts_solve(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(I_out), _ptr(loss_out),
                           _ptr(tape), tape.numel() * tape.element_size(), _stream(stream)),
           "mts_solve")


def mts_superpose(pb, prec, basis, ev: Eval, tape, B_out, stream=None):
    _check(lib().mts_superpose(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(tape), _ptr(B_out),
                               _stream(stream)), "mts_superpose")


def mts_forward(pb, prec, basis, ev: Eval, B_out=None, I_out=None, loss_out=None, tape=None,
                stream=None):
    _check(lib().mts_forward(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(B_out), _ptr(I_out),
                             _ptr(loss_out), _ptr(tape), tape.numel() * tape.element_size(),
                             _stream(stream)), "mts_forward")


def mts_backward(pb, prec, basis, ev: Eval, tape, grad_B=None, grad_loss=None, grad_C=None,
                 stream=None):
    _check(lib().mts_backward(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(tape),
                              tape.numel() * tape.element_size(), _ptr(grad_B), _ptr(grad_loss),
                              _ptr(grad_C), _stream(stream)), "mts_backward")


def mts_tape_status(pb, n_cfg: int, prec, tape, stream=None):
    n_bad = ct.c_int64(0)
    code = lib().mts_tape_status(pb.ref, int(n_cfg), _prec(prec), _ptr(tape), ct.byref(n_bad),
                                 _stream(stream))
    return int(code), int(n_bad.value)


def mts_system_status(pb, n_cfg: int, prec, tape, status_out, stream=None):
    """Per-system status words [n_cfg, n_freq] (int32 device tensor) of the last forward."""
    _check(lib().mts_system_status(pb.ref, int(n_cfg), _prec(prec), _ptr(tape), _ptr(status_out),
                                   _stream(stream)), "mts_system_status")


def mts_solve_static(pb, prec, basis, ev: Eval, I_out=None, loss_out=None, dloss_dC_out=None,
                     stream=None):
    """mts_solve without a tape: the library's own fixed device scratch serves as working
    memory, for callers that cannot allocate device memory when they solve. Calls on one
    device share that scratch; keep them on one stream."""
    _check(lib().mts_solve_static(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(I_out),
                                  _ptr(loss_out), _ptr(dloss_dC_out), _stream(stream)),
           "mts_solve_static")


def mts_solve_static_status(pb, n_cfg: int, prec, stream=None):
    """(status code, number of flagged systems) of the last mts_solve_static call on this
    device for the same problem, batch size and precision (synchronises the stream)."""
    n_bad = ct.c_int64(0)
    code = lib().mts_solve_static_status(pb.ref, int(n_cfg), _prec(prec), ct.byref(n_bad),
                                         _stream(stream))
    return int(code), int(n_bad.value)


def alloc_bytes(nbytes: int, device="cuda") -> torch.Tensor:
    """A device byte buffer; torch's allocator returns 512-byte aligned blocks."""
    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


def mts_adam_step(n: int, opt: MtsAdam, C, u, grad_C, m, v, step, loss=None, loss_history=None,
                  stream=None):
    """One Adam update of n parameters (device tensors; step is a device int64 counter)."""
    n_loss = 0 if loss is None else loss.numel()
    hist_len = 0 if loss_history is None or n_loss == 0 else loss_history.numel() // n_loss
    _check(lib().mts_adam_step(int(n), ct.byref(opt), _ptr(C), _ptr(u), _ptr(grad_C), _ptr(m),
                               _ptr(v), _ptr(step), _ptr(loss), int(n_loss), _ptr(loss_history),
                               int(hist_len), _stream(stream)), "mts_adam_step")


def mts_param_grad(pb, prec, basis, ev: Eval, tape, grad_loss=None, grad_R=None, grad_L=None,
                   grad_omega=None, grad_V=None, stream=None):
    """dloss/dR, dloss/dL (self inductances), dloss/domega (drive fixed) and the drive
    cotangent after a forward with a target."""
    _check(lib().mts_param_grad(pb.ref, _prec(prec), _ptr(basis), ev.ref, _ptr(tape),
                                tape.numel() * tape.element_size(), _ptr(grad_loss),
                                _ptr(grad_R), _ptr(grad_L), _ptr(grad_omega), _ptr(grad_V),
                                _stream(stream)), "mts_param_grad")


# ---------------------------------------------------------------------------------------
# scattering-parameter route
# ---------------------------------------------------------------------------------------
class Sparams:
    """A structure in S-parameter form (mts_sparams): S0 [F, n0, n0], field [F, P, n0],
    S_C,const [F, n, n] (or None), the (row, col) of each variable entry, loss points."""

    def __init__(self, S0, field, rows, cols, n1: int, sc_const=None, loss_idx=None,
                 device="cuda"):
        def dev(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)

        def cdev(a):
            return torch.view_as_real(torch.from_numpy(np.ascontiguousarray(a, np.complex128))).contiguous().to(device)
        S0 = np.asarray(S0)
        field = np.asarray(field)
        self.F, self.n0 = S0.shape[0], S0.shape[1]
        self.P = field.shape[1]
        self.h_rows = np.ascontiguousarray(rows, np.int32)
        self.h_cols = np.ascontiguousarray(cols, np.int32)
        self.d = {"S0": cdev(S0), "field": cdev(field)}
        self.n1 = int(n1)
        if sc_const is not None:
            self.d["sc_const"] = cdev(sc_const)
        li = np.zeros(0, np.int64) if loss_idx is None else np.asarray(loss_idx, np.int64)
        self.d["loss_idx"] = dev(li, np.int64)
        self.L = len(li)
        self.nS = len(self.h_rows)
        c = MtsSparams()
        c.n0, c.n1, c.n_freq, c.n_points = self.n0, self.n1, self.F, self.P
        c.n_svar, c.n_loss = self.nS, self.L
        c.h_svar_row = self.h_rows.ctypes.data
        c.h_svar_col = self.h_cols.ctypes.data
        c.S0 = self.d["S0"].data_ptr()
        c.field = self.d["field"].data_ptr() if self.d["field"].numel() else None
        c.sc_const = self.d["sc_const"].data_ptr() if "sc_const" in self.d else None
        c.loss_idx = self.d["loss_idx"].data_ptr() if self.L else None
        self.c = c

    @property
    def ref(self):
        return ct.byref(self.c)


class SrouteEval:
    """Per-call inputs of the route (mts_sroute_eval): svar complex [n_cfg, F, nS] (as a
    float64 view [..., 2]), target [F, n1, L] (real, or [..., 2] complex) or None."""

    def __init__(self, svar: torch.Tensor, target: Optional[torch.Tensor] = None,
                 loss_mode: int = MTS_LOSS_ABS, refine_tol: float = 0.0, max_refine: int = 0,
                 loss_weight: Optional[torch.Tensor] = None,
                 loss_offset: Optional[torch.Tensor] = None):
        self.svar = svar.contiguous()
        self.loss_weight = None if loss_weight is None else loss_weight.contiguous()
        self.loss_offset = None if loss_offset is None else loss_offset.contiguous()
        self.target = None if target is None else target.contiguous()
        e = MtsSrouteEval()
        e.n_cfg = self.svar.shape[0]
        e.svar = self.svar.data_ptr() if self.svar.numel() else None
        e.target = None if self.target is None else self.target.data_ptr()
        e.loss_mode = int(loss_mode)
        e.refine_tol = float(refine_tol)
        e.max_refine = int(max_refine)
        e.loss_weight = None if self.loss_weight is None else self.loss_weight.data_ptr()
        e.loss_offset = None if self.loss_offset is None else self.loss_offset.data_ptr()
        self.c = e

    @property
    def n_cfg(self) -> int:
        return int(self.c.n_cfg)

    @property
    def ref(self):
        return ct.byref(self.c)


def _nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def mts_sroute_basis_bytes(sp: Sparams, prec) -> int:
    return int(lib().mts_sroute_basis_bytes(sp.ref, _prec(prec)))


def mts_sroute_build(sp: Sparams, prec, sbasis: torch.Tensor, stream=None):
    _check(lib().mts_sroute_build(sp.ref, _prec(prec), _ptr(sbasis), _nbytes(sbasis),
                                  _stream(stream)), "mts_sroute_build")


def mts_sroute_tape_bytes(sp: Sparams, n_cfg: int, prec) -> int:
    return int(lib().mts_sroute_tape_bytes(sp.ref, int(n_cfg), _prec(prec)))


def mts_sroute_forward(sp: Sparams, prec, sbasis, ev: SrouteEval, B_out=None, W_out=None,
                       loss_out=None, tape=None, stream=None):
    _check(lib().mts_sroute_forward(sp.ref, _prec(prec), _ptr(sbasis), ev.ref, _ptr(B_out),
                                    _ptr(W_out), _ptr(loss_out), _ptr(tape), _nbytes(tape),
                                    _stream(stream)), "mts_sroute_forward")


def mts_sroute_backward(sp: Sparams, prec, sbasis, ev: SrouteEval, tape, grad_B=None,
                        grad_loss=None, grad_svar=None, stream=None):
    _check(lib().mts_sroute_backward(sp.ref, _prec(prec), _ptr(sbasis), ev.ref, _ptr(tape),
                                     _nbytes(tape), _ptr(grad_B), _ptr(grad_loss),
                                     _ptr(grad_svar), _stream(stream)), "mts_sroute_backward")


def mts_sroute_status(sp: Sparams, n_cfg: int, prec, tape, stream=None):
    n_bad = ct.c_int64(0)
    code = lib().mts_sroute_status(sp.ref, int(n_cfg), _prec(prec), _ptr(tape), ct.byref(n_bad),
                                   _stream(stream))
    return int(code), int(n_bad.value)


def mts_rc_reflection(n_cfg: int, n_freq: int, n_loads: int, omega, R, C, Z0: float,
                      svar_stride: int, svar_offset: int, svar, stream=None):
    _check(lib().mts_rc_reflection(int(n_cfg), int(n_freq), int(n_loads), _ptr(omega), _ptr(R),
                                   _ptr(C), float(Z0), int(svar_stride), int(svar_offset),
                                   _ptr(svar), _stream(stream)), "mts_rc_reflection")


def mts_rc_reflection_vjp(n_cfg: int, n_freq: int, n_loads: int, omega, R, C, Z0: float,
                          svar_stride: int, svar_offset: int, grad_svar, grad_R=None, grad_C=None,
                          stream=None):
    _check(lib().mts_rc_reflection_vjp(int(n_cfg), int(n_freq), int(n_loads), _ptr(omega),
                                       _ptr(R), _ptr(C), float(Z0), int(svar_stride),
                                       int(svar_offset), _ptr(grad_svar), _ptr(grad_R),
                                       _ptr(grad_C), _stream(stream)), "mts_rc_reflection_vjp")
