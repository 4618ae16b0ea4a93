"""The seeded synthetic workloads have the shapes, sizes and value ranges of the five
configurations they stand in for (the single loop, the 8x1 line, the 8x8 array the
benchmark times, the uneven batch and the 32x32 array), and the same seed gives the same
bytes. CPU only; the generators hold no arithmetic of the method."""
import numpy as np
import pytest

from paper_2503_18479_gb300 import workloads as W

PF, MHZ = 1e-12, 1e6


def _segments(st):
    return int(st.loop_vtx_off[-1])  # closed polylines: one segment per vertex


def _planes(st, n_grid):
    return sorted(set(np.round(st.pz[:n_grid], 6)))


def _capacitances(C):
    assert C.min() >= 20 * PF and C.max() <= 200 * PF
    # uniform over [20, 200] pF: mean 110 pF, standard deviation 180/sqrt(12) = 52 pF
    if C.size >= 1000:
        assert abs(C.mean() / PF - 110.0) < 3.0 and abs(C.std() / PF - 51.96) < 2.0


def test_single_loop():
    wl = W.single_loop(seed=0)
    (st,) = wl.structures
    assert st.n_ports == 1 and _segments(st) == 64
    r = np.hypot(st.vx, st.vy)
    assert np.allclose(r, 0.050) and wl.wire_radius == 0.001
    f = st.omega / (2 * np.pi) / MHZ
    assert len(f) == 101 and np.isclose(f[0], 60.0) and np.isclose(f[-1], 68.0)
    assert st.n_points == 32 * 32 and np.allclose(st.pz, 0.020)
    assert np.isclose(st.px.min(), -0.100) and np.isclose(st.px.max(), 0.100)
    assert len(st.loss_idx) == 4 and np.allclose(st.R, 0.1)
    assert wl.C.shape == (1, 1)
    _capacitances(wl.C)
    assert wl.target_rule == ("field_at_C", 100 * PF)


def test_line_8x1():
    wl = W.line_8x1(seed=0)
    (st,) = wl.structures
    assert st.n_ports == 8 and _segments(st) == 8 * 64
    f = st.omega / (2 * np.pi) / MHZ
    assert len(f) == 201 and np.isclose(f[0], 60.0) and np.isclose(f[-1], 68.0)
    assert st.n_points == 64 * 64 + 8 and _planes(st, 64 * 64) == [0.02]
    assert wl.C.shape == (1024, 8)
    _capacitances(wl.C)


def test_array_8x8_benchmark_workload():
    wl = W.array_8x8(seed=0)
    (st,) = wl.structures
    assert st.n_ports == 64 and _segments(st) == 64 * 64
    side = np.ptp(st.vx[st.loop_vtx_off[0]:st.loop_vtx_off[1]])
    assert np.isclose(side, 0.050)
    centre = [st.vx[st.loop_vtx_off[k]:st.loop_vtx_off[k + 1]].mean() for k in (0, 1)]
    assert np.isclose(abs(centre[1] - centre[0]), 0.055)  # pitch
    assert len(st.omega) == 1 and np.isclose(st.omega[0] / (2 * np.pi), 63.6 * MHZ)
    n_grid = 4 * 128 * 128
    assert st.n_points == n_grid + 64 == 65600
    assert _planes(st, n_grid) == [0.01, 0.02, 0.03, 0.04]
    assert np.isclose(st.px[:n_grid].min(), -0.250) and np.isclose(st.px[:n_grid].max(), 0.250)
    assert len(st.loss_idx) == 64 and np.allclose(st.pz[st.loss_idx], 0.040)
    assert wl.C.shape == (4096, 64)
    _capacitances(wl.C)
    assert wl.target.shape == (64,) and abs(wl.target.std() / 1e-6 - 1.0) < 0.35


def test_uneven_batch():
    wl = W.ragged(seed=0, n_struct=600)
    ports = np.array([st.n_ports for st in wl.structures])
    freqs = np.array([st.n_freq for st in wl.structures])
    assert set(ports) == {1, 8, 16, 32, 64, 128}
    assert freqs.min() == 1 and freqs.max() == 16
    assert all(st.n_points == 64 * 64 + st.n_ports for st in wl.structures)
    f = np.concatenate([st.omega for st in wl.structures]) / (2 * np.pi) / MHZ
    assert f.min() >= 60.0 and f.max() <= 68.0
    assert wl.C.shape == (1, ports.sum())
    _capacitances(wl.C)


def test_array_32x32():
    wl = W.array_32x32(seed=0)
    (st,) = wl.structures
    assert st.n_ports == 1024 and _segments(st) == 65536
    n_grid = 4 * 512 * 512
    assert st.n_points == n_grid + 1024 and n_grid == 1048576
    assert wl.C.shape == (256, 1024)
    _capacitances(wl.C)


@pytest.mark.parametrize("make", [lambda s: W.array_8x8(seed=s, n_cfg=64, grid=8),
                                  lambda s: W.ragged(seed=s, n_struct=20, grid=4),
                                  lambda s: W.sroute_array(seed=s, n_cfg=16, grid=8)])
def test_same_seed_same_bytes(make):
    a, b, c = make(0), make(0), make(1)
    assert np.array_equal(a.C, b.C) and not np.array_equal(a.C, c.C)
