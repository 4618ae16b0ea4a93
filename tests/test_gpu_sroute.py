"""Parity of the scattering-parameter route (Eq. 3-7, Eq. 10) on the GPU, through the C ABI,
with the FP64 oracle's pipeline (oracle.sroute_pipeline / sroute_gradient) on seeded inputs:
a general network (variable S11 diagonal and off-diagonal entries, S12, S21 and S22 entries,
a nonzero S_C,const) on several point tiles with a ragged tail and enough configurations for
the tensor-core superposition; the synthetic 8x8-plus-drive workload with series RC loads
(Eq. 2-3 on the GPU, gradient with respect to C through its vector-Jacobian product); a field
cotangent; the size limits; a system too ill-conditioned for FP32 factors is flagged.

Tolerances: MTS_FP64 1e-10; MTS_MIXED 1e-6 on Bcomb, W, the objective and dL/dsvar;
MTS_BF16 1e-2 on Bcomb."""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel
from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _general(seed=3, F=3, n0=20, n1=3, P=300, n_cfg=40, mode=0):
    rng = np.random.default_rng(seed)
    S0 = (rng.standard_normal((F, n0, n0)) + 1j * rng.standard_normal((F, n0, n0))) * (0.5 / np.sqrt(n0))
    field = (rng.standard_normal((F, P, n0)) + 1j * rng.standard_normal((F, P, n0))) * 1e-6
    n = n0 + n1
    sc = (rng.standard_normal((F, n, n)) + 1j * rng.standard_normal((F, n, n))) * (0.2 / np.sqrt(n))
    pos = [(i, i) for i in range(n0)] + [(0, 5), (7, 2), (3, n0), (9, n - 1), (n0, 4), (n - 1, n - 1)]
    rows = np.array([p[0] for p in pos], np.int32)
    cols = np.array([p[1] for p in pos], np.int32)
    svar = (rng.uniform(-0.8, 0.8, (n_cfg, F, len(pos))) + 1j * rng.uniform(-0.8, 0.8, (n_cfg, F, len(pos))))
    li = np.sort(rng.choice(P, size=17, replace=False)).astype(np.int64)
    if mode == 0:
        t = np.abs(rng.standard_normal((F, n1, len(li)))) * 1e-6
    else:
        t = rng.standard_normal((F, n1, len(li), 2)) * 1e-6
    return dict(S0=S0, field=field, sc=sc, rows=rows, cols=cols, svar=svar, li=li, t=t, n1=n1, mode=mode)


def _route(c, prec):
    from paper_2503_18479_gb300.sroute import SRoute
    t = c["t"]
    if c["mode"] == 1:
        t = t[..., 0] + 1j * t[..., 1]
    return SRoute(c["S0"], c["field"], c["rows"], c["cols"], c["n1"], sc_const=c["sc"],
                  loss_idx=c["li"], target=t, loss_mode=c["mode"], precision=prec)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "bf16"])
def test_general_network(prec, mode):
    c = _general(mode=mode)
    ref = oracle.sroute_pipeline(c["S0"], c["field"], c["sc"], c["rows"], c["cols"], c["svar"],
                                 c["li"], c["t"], mode=mode)
    gref = oracle.sroute_gradient(c["S0"], c["field"], c["sc"], c["rows"], c["cols"], c["svar"],
                                  c["li"], c["t"], mode=mode)
    sr = _route(c, prec)
    out = sr.forward(torch.from_numpy(c["svar"]), want_B=True, want_W=True)
    g = sr.backward(out, grad_loss=torch.ones(c["svar"].shape[0], dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert sr.status(out["tape"], c["svar"].shape[0]) == (0, 0)
    tol = TOL[prec]
    assert rel(out["B"].cpu().numpy(), ref["B"]) < tol, rel(out["B"].cpu().numpy(), ref["B"])
    if prec == "bf16":
        return
    assert rel(out["W"].cpu().numpy(), ref["W"]) < tol
    assert rel(out["loss"].cpu().numpy(), ref["loss"]) < tol
    gg = g.cpu().numpy()
    assert rel(gg, gref) < tol, rel(gg, gref)
    assert np.all(gg[:, :, c["rows"] >= c["S0"].shape[1]] == 0)


def test_field_cotangent():
    """dL/dsvar of a field cotangent grad_B: the oracle's objective gradient with every point a
    loss point, the complex objective and, per configuration, the target B - grad_B n/2 (so
    that its field derivative 2 (B - t)/n is grad_B)."""
    c = _general(seed=5, F=2, n0=12, n1=2, P=150, n_cfg=3, mode=1)
    rng = np.random.default_rng(9)
    gB = (rng.standard_normal((3, 2, 2, 150)) + 1j * rng.standard_normal((3, 2, 2, 150))) * 1e3
    for prec in ("fp64", "mixed"):
        sr = _route(c, prec)
        sv = torch.from_numpy(c["svar"])
        out = sr.forward(sv, want_B=True)
        g = sr.backward(out, grad_B=torch.from_numpy(gB).cuda()).cpu().numpy()
        allp = np.arange(150)
        F, n1 = 2, 2
        norm = F * n1 * 150
        for b in range(3):
            r0 = oracle.sroute_pipeline(c["S0"], c["field"], c["sc"], c["rows"], c["cols"],
                                        c["svar"][b:b + 1], want_loss=False)
            Bb = r0["B"][0]  # [n1, F, P]
            t = np.transpose(Bb - gB[b] * norm / 2, (1, 0, 2))  # [F, n1, P]
            tt = np.stack([t.real, t.imag], axis=-1)
            gr = oracle.sroute_gradient(c["S0"], c["field"], c["sc"], c["rows"], c["cols"],
                                        c["svar"][b:b + 1], allp, tt, mode=1)
            assert rel(g[b], gr[0]) < TOL[prec], (prec, b, rel(g[b], gr[0]))


def test_rc_loads_on_the_array_workload():
    """The synthetic 8x8-plus-drive workload (n0 = 65): Gamma from (R, C) on the GPU (Eq. 2-3),
    Bcomb and the objective against the oracle for a sample of configurations, and dL/dC
    through SRouteFunction and RCReflection (torch autograd) against the oracle's Eq. 10
    gradient chained through dGamma/dC."""
    from paper_2503_18479_gb300.sroute import SRoute, rc_reflection
    wl = W.sroute_array(n_cfg=64, grid=16, seed=2)
    sr = SRoute(wl.S0, wl.field, wl.rows, wl.cols, wl.n1, sc_const=wl.sc_const,
                loss_idx=wl.loss_idx, target=wl.target, precision="mixed")
    R = torch.from_numpy(wl.R).cuda()
    C = torch.from_numpy(wl.C).cuda().requires_grad_(True)
    om = torch.from_numpy(wl.omega).cuda()
    gam = rc_reflection(R, C, om, wl.Z0)
    B, loss = sr(gam)
    loss.sum().backward()
    w = wl.omega[None, :, None]
    Zl = wl.R[:, None, :] - 1j / (w * wl.C[:, None, :])
    svar = (Zl - wl.Z0) / (Zl + wl.Z0)  # Eq. 3
    assert rel(gam.detach().cpu().numpy(), svar) < 1e-14
    cfg = np.arange(0, 64, 9)
    ref = oracle.sroute_pipeline(wl.S0, wl.field, wl.sc_const, wl.rows, wl.cols, svar[cfg],
                                 wl.loss_idx, wl.target)
    assert rel(B.detach().cpu().numpy()[cfg], ref["B"]) < 1e-6
    assert rel(loss.detach().cpu().numpy()[cfg], ref["loss"]) < 1e-6
    g = oracle.sroute_gradient(wl.S0, wl.field, wl.sc_const, wl.rows, wl.cols, svar[cfg],
                               wl.loss_idx, wl.target)
    dgam = 2 * wl.Z0 / (Zl[cfg] + wl.Z0) ** 2 * (1j / (w * wl.C[cfg][:, None, :] ** 2))
    gC = np.real(np.conj(g) * dgam).sum(axis=1)
    assert rel(C.grad.cpu().numpy()[cfg], gC) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_size_limits(prec):
    """n0 = 96 and n1 = 8 (the largest shared-memory carve), and n0 = n1 = 1."""
    for n0, n1, P, n_cfg in ((96, 8, 40, 3), (1, 1, 5, 20)):
        rng = np.random.default_rng(n0)
        F = 1
        S0 = (rng.standard_normal((F, n0, n0)) + 1j * rng.standard_normal((F, n0, n0))) * (0.4 / np.sqrt(n0))
        field = rng.standard_normal((F, P, n0)) + 1j * rng.standard_normal((F, P, n0))
        n = n0 + n1
        sc = np.zeros((F, n, n), complex)
        sc[:, :n0, n0:] = rng.standard_normal((n0, n1))
        rows = np.arange(n0, dtype=np.int32)
        svar = rng.uniform(-0.9, 0.9, (n_cfg, F, n0)) + 1j * rng.uniform(-0.9, 0.9, (n_cfg, F, n0))
        li = np.arange(min(P, 4))
        t = np.ones((F, n1, len(li)))
        c = dict(S0=S0, field=field, sc=sc, rows=rows, cols=rows, svar=svar, li=li, t=t, n1=n1, mode=0)
        ref = oracle.sroute_pipeline(S0, field, sc, rows, rows, svar, li, t)
        gref = oracle.sroute_gradient(S0, field, sc, rows, rows, svar, li, t)
        sr = _route(c, prec)
        out = sr.forward(torch.from_numpy(svar), want_B=True)
        g = sr.backward(out, grad_loss=torch.ones(n_cfg, dtype=torch.float64, device="cuda"))
        assert rel(out["B"].cpu().numpy(), ref["B"]) < TOL[prec], (n0, rel(out["B"].cpu().numpy(), ref["B"]))
        assert rel(out["loss"].cpu().numpy(), ref["loss"]) < TOL[prec]
        assert rel(g.cpu().numpy(), gref) < TOL[prec], (n0, rel(g.cpu().numpy(), gref))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_enhancement_objective(prec):
    """The weighted, offset objective (Sec. IV-B) of the route against the oracle's."""
    from paper_2503_18479_gb300.sroute import SRoute
    c = _general(seed=11, mode=0)
    rng = np.random.default_rng(13)
    w = rng.uniform(0.5, 2.0, c["t"].shape) * 1e6
    o = (rng.standard_normal(c["t"].shape) + 1j * rng.standard_normal(c["t"].shape)) * 3e-7
    t = c["t"] * 1e6
    ref = oracle.sroute_pipeline(c["S0"], c["field"], c["sc"], c["rows"], c["cols"], c["svar"],
                                 c["li"], t, want_B=False, weight=w, offset=o)
    gref = oracle.sroute_gradient(c["S0"], c["field"], c["sc"], c["rows"], c["cols"], c["svar"],
                                  c["li"], t, weight=w, offset=o)
    sr = SRoute(c["S0"], c["field"], c["rows"], c["cols"], c["n1"], sc_const=c["sc"],
                loss_idx=c["li"], target=t, precision=prec, loss_weight=w, loss_offset=o)
    out = sr.forward(torch.from_numpy(c["svar"]), want_B=False)
    g = sr.backward(out, grad_loss=torch.ones(c["svar"].shape[0], dtype=torch.float64, device="cuda"))
    assert rel(out["loss"].cpu().numpy(), ref["loss"]) < TOL[prec]
    assert rel(g.cpu().numpy(), gref) < TOL[prec], rel(g.cpu().numpy(), gref)


@pytest.mark.parametrize("prec", ["mixed", "bf16"])
def test_unconverged_system_is_flagged(prec):
    """One S11 diagonal entry of one (configuration, frequency) moved to s*(1 + 1e-9), where
    A(s) = 1 - S11(s) S0 (a rank-one function of s) is singular at s*: condition number
    about 6e9, far beyond what FP32 factors can refine (rounding A to FP32 moves its smallest
    singular value by about 1e-7 of the norm, so successive corrections stay the same
    size). The status reader must count exactly that system; every other system keeps
    bit-identical W, Bcomb and objective."""
    from paper_2503_18479_gb300 import native as nv
    c = _general()
    S0, sc, rows, cols = c["S0"], c["sc"], c["rows"], c["cols"]
    n0 = S0.shape[1]
    b, f = 5, 0
    k0 = int(np.nonzero((rows == 0) & (cols == 0))[0][0])
    S = sc[f].copy()
    S[rows, cols] += c["svar"][b, f]
    A = np.eye(n0) - S[:n0, :n0] @ S0[f]
    e0 = np.zeros(n0)
    e0[0] = 1.0
    # A(s) = A - (s - s_old) e0 (e0^T S0) is singular where (s - s_old) e0^T S0 A^-1 e0 = 1
    s_star = c["svar"][b, f, k0] + 1.0 / ((e0 @ S0[f]) @ np.linalg.solve(A, e0))
    bad = c["svar"].copy()
    bad[b, f, k0] = s_star * (1.0 + 1e-9)
    sr = _route(c, prec)
    n_cfg = c["svar"].shape[0]
    ref = sr.forward(torch.from_numpy(c["svar"]), want_B=True, want_W=True)
    assert sr.status(ref["tape"], n_cfg) == (nv.MTS_OK, 0)
    out = sr.forward(torch.from_numpy(bad), want_B=True, want_W=True)
    assert sr.status(out["tape"], n_cfg) == (nv.MTS_ENOCONV, 1)
    keep = [i for i in range(n_cfg) if i != b]
    for key in ("B", "W", "loss"):
        assert torch.equal(out[key][keep], ref[key][keep]), key
    # the planted configuration's other frequencies are separate systems and still converge
    assert torch.equal(out["W"][b, 1:], ref["W"][b, 1:])
