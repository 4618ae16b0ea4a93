"""Convenience layer over the C ABI: a Simulator that owns the device problem and basis,
and a torch.autograd.Function whose forward/backward are mts_forward/mts_backward.

Forward map (paper Eq. 1-2, 6-7, 11): C -> B = H I(C) with (diag(R) + j w M +
diag(1/(j w C))) I = V, plus the objective at the loss points. Backward (Eq. 8-10 via
d(A^-1) = -A^-1 dA A^-1): the adjoint gradient with respect to C.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import native as nv
from .workloads import Workload


class Simulator:
    def __init__(self, wl: Workload, precision="mixed", device="cuda", target=None,
                 target_per_cfg: Optional[bool] = None, refine_tol: float = 0.0,
                 max_refine: int = 0, loss_weight=None, loss_offset=None,
                 keep_factors: bool = False):
        """loss_weight [FL] real and loss_offset [FL] complex (optional): the objective is
        taken on weight * (B + offset) at the loss points -- the enhancement objective of
        Sec. IV-B with weight 1/|B_ref| and offset the incident field. keep_factors: the tape
        keeps the register solve's LU factors for a later field-cotangent backward."""
        self.wl = wl
        self.prec = nv._prec(precision)
        self.device = torch.device(device)
        flat = wl.flat()
        self.flat = flat
        self.pb = nv.Problem(flat, wl.wire_radius, device, keep_factors=keep_factors)
        self.basis = nv.alloc_bytes(nv.mts_basis_bytes(self.pb, self.prec), device)
        nv.mts_build_basis(self.pb, self.prec, self.basis)
        code = nv.mts_basis_status(self.pb, self.prec, self.basis)
        if code != nv.MTS_OK:
            raise nv.MtsError(code, "mts_build_basis (segment pairs)")
        self.omega = torch.from_numpy(flat["omega"]).to(self.device)
        self.V = torch.view_as_real(torch.from_numpy(flat["V"])).contiguous().to(self.device)
        t = wl.target if target is None else target
        self.target = None if t is None else torch.as_tensor(np.asarray(t, np.float64)).to(self.device)
        self.target_per_cfg = wl.target_per_cfg if target_per_cfg is None else target_per_cfg
        self.loss_mode = wl.loss_mode
        self.loss_weight = None if loss_weight is None else torch.as_tensor(
            np.asarray(loss_weight, np.float64)).to(self.device)
        self.loss_offset = None if loss_offset is None else torch.view_as_real(torch.as_tensor(
            np.asarray(loss_offset, np.complex128))).contiguous().to(self.device)
        self.refine_tol = refine_tol
        self.max_refine = max_refine
        self.n_struct = len(wl.structures)
        self.sumFP = int(sum(s.n_freq * s.n_points for s in wl.structures))
        self.sumFN = int(sum(s.n_freq * s.n_ports for s in wl.structures))
        self.n_ports = wl.n_ports
        self.b_dtype = torch.complex128 if self.prec == nv.MTS_FP64 else torch.complex64
        # launch schedule (mts_eval.simt_max_sys, large_threads, reg_widen); 0 = the library's rules,
        # set by tune.autotune
        self.tuning = {"simt_max_sys": 0, "large_threads": 0, "reg_widen": 0}

    # ------------------------------------------------------------------
    def make_eval(self, C: torch.Tensor, with_target: bool = True) -> nv.Eval:
        return nv.Eval(C, self.omega, self.V, self.target if with_target else None,
                       self.target_per_cfg, self.loss_mode, self.refine_tol, self.max_refine,
                       loss_weight=self.loss_weight, loss_offset=self.loss_offset, **self.tuning)

    def alloc_tape(self, n_cfg: int) -> torch.Tensor:
        return nv.alloc_bytes(nv.mts_tape_bytes(self.pb, n_cfg, self.prec), self.device)

    def forward(self, C: torch.Tensor, want_B: bool = True, want_I: bool = False,
                want_loss: bool = True, tape: Optional[torch.Tensor] = None, B_out=None,
                stream=None):
        C = C.to(self.device, torch.float64).contiguous()
        n_cfg = C.shape[0]
        has_t = want_loss and self.target is not None
        ev = self.make_eval(C, has_t)
        if tape is None:
            tape = self.alloc_tape(n_cfg)
        B = None
        if want_B:
            B = B_out if B_out is not None else torch.empty((n_cfg, self.sumFP), dtype=self.b_dtype,
                                                             device=self.device)
        I = torch.empty((n_cfg, self.sumFN), dtype=torch.complex128, device=self.device) if want_I else None
        loss = torch.empty((n_cfg, self.n_struct), dtype=torch.float64, device=self.device) if has_t else None
        nv.mts_forward(self.pb, self.prec, self.basis, ev, B, I, loss, tape, stream)
        return {"B": B, "I": I, "loss": loss, "tape": tape, "ev": ev}

    def backward(self, ev: nv.Eval, tape: torch.Tensor, grad_B=None, grad_loss=None, stream=None):
        grad_C = torch.empty((ev.n_cfg, self.n_ports), dtype=torch.float64, device=self.device)
        gB = None if grad_B is None else grad_B.to(self.b_dtype).contiguous()
        gl = None if grad_loss is None else grad_loss.to(torch.float64).contiguous()
        nv.mts_backward(self.pb, self.prec, self.basis, ev, tape, gB, gl, grad_C, stream)
        return grad_C

    def param_grad(self, ev: nv.Eval, tape: torch.Tensor, grad_loss=None, stream=None,
                   with_omega: bool = False):
        """(dloss/dR, dloss/dL) per configuration and port, [n_cfg, n_ports] each, after a
        forward with the objective (loss cotangent grad_loss [n_cfg, n_struct], default 1);
        with_omega adds dloss/domega [n_cfg, n_freq] (drive fixed) and the drive cotangent
        [n_cfg, sum F N] (complex128)."""
        gR = torch.empty((ev.n_cfg, self.n_ports), dtype=torch.float64, device=self.device)
        gL = torch.empty_like(gR)
        gw = gV = None
        if with_omega:
            gw = torch.empty((ev.n_cfg, int(self.omega.numel())), dtype=torch.float64, device=self.device)
            gV = torch.empty((ev.n_cfg, self.sumFN), dtype=torch.complex128, device=self.device)
        gl = None if grad_loss is None else grad_loss.to(torch.float64).contiguous()
        nv.mts_param_grad(self.pb, self.prec, self.basis, ev, tape, gl, gR, gL, gw, gV, stream)
        return (gR, gL, gw, gV) if with_omega else (gR, gL)

    def status(self, tape: torch.Tensor, n_cfg: int):
        return nv.mts_tape_status(self.pb, n_cfg, self.prec, tape)

    def export_basis(self):
        """FP64 copies of H (concatenated [P_s, N_s] blocks) and M ([N_s, N_s] blocks)."""
        sumPN = int(sum(s.n_points * s.n_ports for s in self.wl.structures))
        sumNN = int(sum(s.n_ports ** 2 for s in self.wl.structures))
        H = torch.empty(max(sumPN, 1), dtype=torch.float64, device=self.device)
        M = torch.empty(max(sumNN, 1), dtype=torch.float64, device=self.device)
        nv.mts_basis_export(self.pb, self.prec, self.basis, H, M)
        return H[:sumPN], M[:sumNN]

    def __call__(self, C: torch.Tensor, want_B: bool = True):
        return MtsFunction.apply(C, self, want_B)


class MtsFunction(torch.autograd.Function):
    """(B, loss) = f(C); backward calls mts_backward with the incoming cotangents."""

    @staticmethod
    def forward(ctx, C, sim: Simulator, want_B: bool = True):
        out = sim.forward(C.detach(), want_B=want_B, want_loss=True)
        ctx.sim = sim
        ctx.ev = out["ev"]
        ctx.tape = out["tape"]
        ctx.has_loss = out["loss"] is not None
        B = out["B"] if out["B"] is not None else torch.zeros(0, device=sim.device)
        loss = out["loss"] if out["loss"] is not None else torch.zeros(0, device=sim.device)
        return B, loss

    @staticmethod
    def backward(ctx, gB, gloss):
        sim = ctx.sim
        gB = gB if (gB is not None and gB.numel() > 0) else None
        gl = gloss if (ctx.has_loss and gloss is not None and gloss.numel() > 0) else None
        grad_C = sim.backward(ctx.ev, ctx.tape, grad_B=gB, grad_loss=gl)
        return grad_C, None, None
