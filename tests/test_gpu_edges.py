"""Edge cases of the batched path against the FP64 oracle: a structure without field points
and one without frequencies inside a batch, a one-port structure on the tensor-core path
(K = 1 padded to 64), per-configuration complex targets on a 128-port structure (the
large-system kernel in the complex-objective mode), and a problem whose only structure
takes the SIMT superposition; an invalid field-component code."""
import numpy as np
import pytest
import torch

from helpers import oracle_reference, rel, split_B, split_I, structure_basis
from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    build_lib.build()


def _struct(nx, ny, n_freq, grid, with_loss=True):
    loops = W.square_array(nx, ny, seg_per_side=2)
    omega = 2 * np.pi * np.linspace(60e6, 68e6, n_freq) if n_freq else np.zeros(0)
    if grid:
        hx, hy = (nx + 1) * 0.055 / 2, (ny + 1) * 0.055 / 2
        pts = W._concat_points(W.grid_plane(grid, hx, 0.02, half_span_y=hy),
                               W._cell_centre_points(nx, ny, 0.055, 0.04))
        li = np.arange(grid * grid, grid * grid + nx * ny) if with_loss else np.zeros(0, np.int64)
    else:
        pts = (np.zeros(0), np.zeros(0), np.zeros(0))
        li = np.zeros(0, np.int64)
    return W._structure_from(loops, pts, omega, 0.1, li)


def _check(wl, prec, tol_b, tol_l):
    from paper_2503_18479_gb300.simulator import Simulator
    bases = [structure_basis(wl, s) for s in range(len(wl.structures))]
    ref = oracle_reference(wl, bases=bases)
    sim = Simulator(wl, prec)
    C = torch.from_numpy(wl.C).cuda().requires_grad_(True)
    B, loss = sim(C)
    loss.sum().backward()
    Bs = split_B(wl, B.detach().cpu().numpy())
    lo = loss.detach().cpu().numpy()
    g = C.grad.cpu().numpy()
    po = wl.port_off()
    for s, st in enumerate(wl.structures):
        if st.n_points and st.n_freq:
            assert rel(Bs[s], ref[s]["B"]) < tol_b, (s, rel(Bs[s], ref[s]["B"]))
        if st.n_loss and st.n_freq:
            assert rel(lo[:, s], ref[s]["loss"]) < tol_l, s
            assert rel(g[:, po[s]:po[s + 1]], ref[s]["grad"]) < tol_l, s
        else:
            assert np.all(lo[:, s] == 0.0) and np.all(g[:, po[s]:po[s + 1]] == 0.0), s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_empty_points_and_frequencies_in_a_batch(prec):
    rng = np.random.Generator(np.random.PCG64(1))
    structs = [_struct(2, 2, 3, 6), _struct(3, 1, 2, 0), _struct(2, 1, 0, 5), _struct(1, 1, 4, 6)]
    n_cfg = 20
    C = rng.uniform(20e-12, 200e-12, (n_cfg, sum(s.n_ports for s in structs)))
    t = rng.standard_normal(sum(s.n_freq * s.n_loss for s in structs)) * 1e-6
    wl = W.Workload("edges", structs, C, 0.001, target=t)
    _check(wl, prec, 1e-10 if prec == "fp64" else 1e-6, 1e-10 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["mixed", "bf16"])
def test_one_port_structure_on_the_tensor_path(prec):
    """One loop, 40 configurations x 3 frequencies = 120 systems: the GEMM with K = 1."""
    rng = np.random.Generator(np.random.PCG64(2))
    st = _struct(1, 1, 3, 10)
    C = rng.uniform(20e-12, 200e-12, (40, 1))
    wl = W.Workload("one_port", [st], C, 0.001, target=rng.standard_normal(3) * 1e-6)
    _check(wl, prec, 1e-6 if prec == "mixed" else 1e-2, 1e-6)


def test_complex_targets_per_config_on_a_large_structure():
    from paper_2503_18479_gb300.simulator import Simulator
    rng = np.random.Generator(np.random.PCG64(3))
    st = _struct(16, 8, 2, 6)
    n_cfg = 3
    C = rng.uniform(20e-12, 200e-12, (n_cfg, 128))
    t = rng.standard_normal((n_cfg, 2, 128, 2)) * 1e-6
    wl = W.Workload("complex128", [st], C, 0.001, loss_mode=1, target=t.ravel(), target_per_cfg=True)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        ref = oracle_reference(wl, want_B=False, bases=[structure_basis(wl, 0)])
        sim = Simulator(wl, prec)
        Cg = torch.from_numpy(wl.C).cuda().requires_grad_(True)
        _, loss = sim(Cg, want_B=False)
        loss.sum().backward()
        assert rel(loss.detach().cpu().numpy()[:, 0], ref[0]["loss"]) < tol
        assert rel(Cg.grad.cpu().numpy(), ref[0]["grad"]) < tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_invalid_component_code_is_reported(prec):
    """A field-component code other than 0, 1, 2 makes the basis build report MTS_EINVAL."""
    import dataclasses
    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300.simulator import Simulator
    st = _struct(2, 2, 2, 6)
    pc = np.zeros(st.n_points, np.int8)
    pc[5] = 3
    wl = W.Workload("bad_component", [dataclasses.replace(st, pcomp=pc)], np.full((2, 4), 50e-12),
                    0.001, target=np.zeros(2 * st.n_loss))
    with pytest.raises(nv.MtsError) as e:
        Simulator(wl, prec)
    assert e.value.code == nv.MTS_EINVAL
