"""The scattering-parameter route (paper Sec. III and III-A, Eq. 3-7, Eq. 10) as a torch
module over the library's kernels: a structure given by its S-matrix S0 and per-port fields
from any solver, a network tensor S_C = S_C,const + scatter(svar), the wave ratio
W = (1 - S11 S0)^-1 S12 (Eq. 6) and the combined field Bcomb = field W (Eq. 7), with an
objective at loss points and the gradient with respect to svar (Eq. 10, adjoint form).

`SRoute(svar)` returns (Bcomb [n_cfg, n1, F, P] complex, loss [n_cfg]) and differentiates
through `SRouteFunction`; `rc_reflection(R, C, omega, Z0)` is the series-RC preprocessing of
Eq. 2-3 (Gamma = (Z - Z0)/(Z + Z0), Z = R - j/(w C)) with its own backward. Every step runs
in libmts.so; there is no CPU path.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import native as nv


class SRoute:
    def __init__(self, S0, field, rows, cols, n1: int, sc_const=None, loss_idx=None,
                 target=None, loss_mode: int = nv.MTS_LOSS_ABS, precision: str = "mixed",
                 device="cuda", loss_weight=None, loss_offset=None):
        """loss_weight [F, n1, L] real and loss_offset [F, n1, L] complex (optional): the
        objective is taken on weight * (Bcomb + offset) at the loss points (the enhancement
        objective of Sec. IV-B with weight 1/|B_ref|)."""
        self.device = torch.device(device)
        self.prec = nv.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.sp = nv.Sparams(S0, field, rows, cols, n1, sc_const=sc_const, loss_idx=loss_idx,
                             device=self.device)
        self.F, self.n0, self.n1, self.P, self.nS = self.sp.F, self.sp.n0, self.sp.n1, self.sp.P, self.sp.nS
        self.sbasis = nv.alloc_bytes(nv.mts_sroute_basis_bytes(self.sp, self.prec), self.device)
        if self.sbasis.numel() <= 1:
            raise nv.MtsError(nv.MTS_EINVAL, "mts_sroute_basis_bytes")
        nv.mts_sroute_build(self.sp, self.prec, self.sbasis)
        self.loss_mode = int(loss_mode)
        self.target = None
        if target is not None:
            t = np.asarray(target)
            t = t.view(np.float64).reshape(t.shape + (2,)) if np.iscomplexobj(t) else t
            self.target = torch.from_numpy(np.ascontiguousarray(t, np.float64)).to(self.device)
        self.loss_weight = None if loss_weight is None else torch.from_numpy(
            np.ascontiguousarray(loss_weight, np.float64)).to(self.device)
        self.loss_offset = None if loss_offset is None else torch.view_as_real(torch.from_numpy(
            np.ascontiguousarray(loss_offset, np.complex128))).contiguous().to(self.device)

    @property
    def b_dtype(self):
        return torch.complex128 if self.prec == nv.MTS_FP64 else torch.complex64

    def make_eval(self, svar: torch.Tensor, refine_tol: float = 0.0, max_refine: int = 0):
        sv = svar.to(self.device, torch.complex128).contiguous()
        if sv.dim() != 3 or sv.shape[1:] != (self.F, self.nS):
            raise ValueError(f"svar must be [n_cfg, {self.F}, {self.nS}] complex")
        return nv.SrouteEval(torch.view_as_real(sv), self.target, self.loss_mode, refine_tol,
                             max_refine, self.loss_weight, self.loss_offset)

    def alloc_tape(self, n_cfg: int):
        return nv.alloc_bytes(nv.mts_sroute_tape_bytes(self.sp, n_cfg, self.prec), self.device)

    def forward(self, svar: torch.Tensor, want_B: bool = True, want_W: bool = False):
        ev = self.make_eval(svar)
        n = ev.n_cfg
        tape = self.alloc_tape(n)
        B = torch.empty((n, self.n1, self.F, self.P), dtype=self.b_dtype, device=self.device) if want_B else None
        W = torch.empty((n, self.F, self.n0, self.n1), dtype=torch.complex128, device=self.device) if want_W else None
        loss = torch.empty(n, dtype=torch.float64, device=self.device) if self.target is not None else None
        nv.mts_sroute_forward(self.sp, self.prec, self.sbasis, ev, B_out=B, W_out=W, loss_out=loss,
                              tape=tape)
        return {"B": B, "W": W, "loss": loss, "tape": tape, "ev": ev}

    def backward(self, out: dict, grad_B: Optional[torch.Tensor] = None,
                 grad_loss: Optional[torch.Tensor] = None) -> torch.Tensor:
        ev = out["ev"]
        g = torch.empty((ev.n_cfg, self.F, self.nS), dtype=torch.complex128, device=self.device)
        gB = None if grad_B is None else grad_B.to(self.b_dtype).contiguous()
        gl = None if grad_loss is None else grad_loss.to(torch.float64).contiguous()
        nv.mts_sroute_backward(self.sp, self.prec, self.sbasis, ev, out["tape"], grad_B=gB,
                               grad_loss=gl, grad_svar=g)
        return g

    def status(self, tape, n_cfg: int):
        return nv.mts_sroute_status(self.sp, n_cfg, self.prec, tape)

    def __call__(self, svar: torch.Tensor, want_B: bool = True):
        return SRouteFunction.apply(svar, self, want_B)


class SRouteFunction(torch.autograd.Function):
    """svar (complex128 [n_cfg, F, nS]) -> (Bcomb, loss); backward by mts_sroute_backward
    (torch's complex convention dL/dRe + j dL/dIm on both sides)."""

    @staticmethod
    def forward(ctx, svar, sr: SRoute, want_B: bool):
        out = sr.forward(svar.detach(), want_B=want_B)
        ctx.sr = sr
        ctx.out = out
        B = out["B"] if out["B"] is not None else torch.zeros(0, dtype=sr.b_dtype, device=sr.device)
        loss = out["loss"] if out["loss"] is not None else torch.zeros(0, dtype=torch.float64, device=sr.device)
        return B, loss

    @staticmethod
    def backward(ctx, gB, gl):
        sr, out = ctx.sr, ctx.out
        gB = gB if (out["B"] is not None and gB is not None and gB.numel()) else None
        gl = gl if (out["loss"] is not None and gl is not None and gl.numel()) else None
        g = sr.backward(out, grad_B=gB, grad_loss=gl)
        return g, None, None


class RCReflection(torch.autograd.Function):
    """Eq. 2-3 for series RC loads: Gamma[b, f, k] = (Z - Z0)/(Z + Z0), Z = R - j/(w_f C),
    R and C [n_cfg, n_loads] float64, omega [F]; backward by mts_rc_reflection_vjp."""

    @staticmethod
    def forward(ctx, R, C, omega, Z0: float):
        C = C.contiguous().to(torch.float64)
        R = None if R is None else R.contiguous().to(torch.float64)
        omega = omega.contiguous().to(torch.float64)
        n, nl = C.shape
        F = omega.numel()
        out = torch.empty((n, F, nl, 2), dtype=torch.float64, device=C.device)
        nv.mts_rc_reflection(n, F, nl, omega, R, C, Z0, nl, 0, out)
        ctx.save_for_backward(C, omega)
        ctx.R = R
        ctx.Z0 = Z0
        return torch.view_as_complex(out)

    @staticmethod
    def backward(ctx, g):
        C, omega = ctx.saved_tensors
        R = ctx.R
        n, nl = C.shape
        F = omega.numel()
        gs = torch.view_as_real(g.to(torch.complex128).contiguous()).contiguous()
        gC = torch.empty_like(C)
        gR = torch.empty_like(C) if (R is not None and ctx.needs_input_grad[0]) else None
        nv.mts_rc_reflection_vjp(n, F, nl, omega, R, C, ctx.Z0, nl, 0, gs, grad_R=gR, grad_C=gC)
        return gR, gC, None, None


def rc_reflection(R: Optional[torch.Tensor], C: torch.Tensor, omega: torch.Tensor, Z0: float = 50.0):
    return RCReflection.apply(R, C, omega, Z0)

