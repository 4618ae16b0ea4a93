"""C ABI checks that need no GPU: the library builds, loads, exports every entry point that
include/mts.h declares, and its host-side validation and size queries behave as documented;
the binding's structs, prototypes and constants agree with the header as a C compiler reads
it. No call here reaches a CUDA launch."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2503_18479_gb300 import build_lib
from paper_2503_18479_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nv():
    build_lib.build()
    from paper_2503_18479_gb300 import native
    native.lib()
    return native


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mts_[a-z_]+)\s*\(", src)))


def test_header_declares_the_abi():
    syms = declared_symbols()
    for name in ("mts_build_basis", "mts_forward", "mts_backward", "mts_solve", "mts_superpose",
                 "mts_basis_bytes", "mts_tape_bytes", "mts_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(nv):
    L = nv.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert sorted(nv.EXPORTED) == declared_symbols()


def test_status_strings_and_version(nv):
    assert nv.mts_status_string(0) == "MTS_OK"
    for c in range(1, 6):
        assert nv.mts_status_string(c).startswith("MTS_E")
    assert "sm_103a" in nv.mts_version()
    assert nv.mts_launch_count() == 0  # nothing launched in this process


FAKE = 0x10000  # a non-null device address; the calls below never dereference it


def fake_problem(nv, wl, **over):
    flat = wl.flat()
    keep = {k: np.ascontiguousarray(flat[k]) for k in ("port_off", "point_off", "freq_off", "loss_off")}
    c = nv.MtsProblem()
    c.n_struct = len(wl.structures)
    c.n_ports = int(keep["port_off"][-1])
    c.n_vertices = len(flat["vx"])
    c.n_freq = int(keep["freq_off"][-1])
    c.n_points = int(keep["point_off"][-1])
    c.n_loss = int(keep["loss_off"][-1])
    c.wire_radius = wl.wire_radius
    c.h_port_off = keep["port_off"].ctypes.data
    c.h_point_off = keep["point_off"].ctypes.data
    c.h_freq_off = keep["freq_off"].ctypes.data
    c.h_loss_off = keep["loss_off"].ctypes.data
    for k in ("port_off", "point_off", "freq_off", "loss_off", "loop_vtx_off", "vx", "vy", "vz",
              "px", "py", "pz", "loss_idx", "R"):
        setattr(c, k, FAKE)
    c.L_self = None
    for k, v in over.items():
        setattr(c, k, v)
    return c, keep


def test_size_queries(nv):
    wl = W.array_8x8(n_cfg=4, grid=8, planes=(0.02,))
    c, keep = fake_problem(nv, wl)
    L = nv.lib()
    b64 = L.mts_basis_bytes(ct.byref(c), nv.MTS_FP64)
    bmx = L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED)
    P, N = wl.n_points, 64
    assert b64 >= 8 * P * N + 8 * N * N
    # mixed: FP32 H plus three bf16 pieces of the padded operand
    assert bmx >= 4 * P * N + 3 * 2 * ((P + 127) // 128 * 128) * 64
    t1 = L.mts_tape_bytes(ct.byref(c), 1, nv.MTS_MIXED)
    t2 = L.mts_tape_bytes(ct.byref(c), 4096, nv.MTS_MIXED)
    assert t2 > t1 > 0
    assert t2 >= 4096 * 64 * 16  # the currents alone
    assert L.mts_tape_bytes(ct.byref(c), -1, nv.MTS_MIXED) == 0
    assert L.mts_basis_bytes(ct.byref(c), 7) == 0


def test_validation_rejects_bad_problems(nv):
    L = nv.lib()
    wl = W.array_8x8(n_cfg=2, grid=8, planes=(0.02,))
    cases = [dict(n_struct=0), dict(wire_radius=0.0), dict(wire_radius=float("nan")),
             dict(n_ports=63), dict(port_off=None), dict(R=None), dict(loss_idx=None)]
    for over in cases:
        c, keep = fake_problem(nv, wl, **over)
        assert L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED) == 0, over
        code = L.mts_build_basis(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), 1 << 40, None)
        assert code == nv.MTS_EINVAL, over
    # too many ports in one structure
    big = W.ragged(n_struct=1, grid=4, max_freq=1, port_choices=(128,))
    c, keep = fake_problem(nv, big)
    assert L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED) > 0
    # non-monotonic host offsets
    wl2 = W.ragged(n_struct=3, grid=4, max_freq=2, port_choices=(8,))
    c, keep = fake_problem(nv, wl2)
    keep["port_off"][1], keep["port_off"][2] = keep["port_off"][2], keep["port_off"][1]
    assert L.mts_basis_bytes(ct.byref(c), nv.MTS_FP64) == 0


def test_workspace_and_alignment_checks(nv):
    L = nv.lib()
    wl = W.array_8x8(n_cfg=2, grid=8, planes=(0.02,))
    c, keep = fake_problem(nv, wl)
    need = L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED)
    assert L.mts_build_basis(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), need - 1, None) == nv.MTS_EWORKSPACE
    assert L.mts_build_basis(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE + 8), need, None) == nv.MTS_EINVAL
    assert L.mts_build_basis(ct.byref(c), nv.MTS_MIXED, None, need, None) == nv.MTS_EINVAL
    ev = nv.MtsEval()
    ev.n_cfg = 2
    ev.C = ev.omega = ev.V = FAKE
    ev.target = None
    ev.loss_mode = 0
    tneed = L.mts_tape_bytes(ct.byref(c), 2, nv.MTS_MIXED)
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                       ct.c_void_p(FAKE), tneed - 1, None)
    assert code == nv.MTS_EWORKSPACE
    ev.loss_mode = 5
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                       ct.c_void_p(FAKE), tneed, None)
    assert code == nv.MTS_EINVAL
    ev.loss_mode = 0
    ev.C = None
    code = L.mts_forward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                         None, ct.c_void_p(FAKE), tneed, None)
    assert code == nv.MTS_EINVAL
    # a loss output without a target
    ev.C = FAKE
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None,
                       ct.c_void_p(FAKE), ct.c_void_p(FAKE), tneed, None)
    assert code == nv.MTS_EINVAL
    assert L.mts_backward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev),
                          ct.c_void_p(FAKE), tneed, None, None, None, None) == nv.MTS_EINVAL
    assert nv.mts_launch_count() == 0


def test_static_solve_argument_checks(nv):
    """mts_solve_static and its status reader check their arguments before any CUDA call:
    no evaluation, an invalid precision, a loss gradient without a target, and a batch whose
    working state would not fit the static scratch."""
    L = nv.lib()
    wl = W.array_8x8(n_cfg=2, grid=8, planes=(0.02,))
    c, keep = fake_problem(nv, wl)
    ev = nv.MtsEval()
    ev.n_cfg = 2
    ev.C = ev.omega = ev.V = FAKE
    ev.target = None
    ev.loss_mode = 0
    basis = ct.c_void_p(FAKE)
    assert L.mts_solve_static(ct.byref(c), nv.MTS_MIXED, basis, None, None, None, None, None) == nv.MTS_EINVAL
    assert L.mts_solve_static(ct.byref(c), 7, basis, ct.byref(ev), None, None, None, None) == nv.MTS_EINVAL
    assert L.mts_solve_static(ct.byref(c), nv.MTS_MIXED, basis, ct.byref(ev), None, None,
                              ct.c_void_p(FAKE), None) == nv.MTS_EINVAL
    assert L.mts_solve_static(ct.byref(c), nv.MTS_MIXED, basis, ct.byref(ev), None,
                              ct.c_void_p(FAKE), None, None) == nv.MTS_EINVAL
    limit = 32 << 20
    n_big = 1
    while L.mts_tape_bytes(ct.byref(c), n_big, nv.MTS_MIXED) <= limit:
        n_big *= 2
    ev.n_cfg = n_big
    assert L.mts_solve_static(ct.byref(c), nv.MTS_MIXED, basis, ct.byref(ev), None, None, None,
                              None) == nv.MTS_EWORKSPACE
    nb = ct.c_int64(-1)
    assert L.mts_solve_static_status(ct.byref(c), n_big, nv.MTS_MIXED, ct.byref(nb), None) == nv.MTS_EWORKSPACE
    assert L.mts_solve_static_status(ct.byref(c), -1, nv.MTS_MIXED, ct.byref(nb), None) == nv.MTS_EINVAL
    assert L.mts_solve_static_status(ct.byref(c), 2, 9, ct.byref(nb), None) == nv.MTS_EINVAL
    assert nv.mts_launch_count() == 0


def _wide_workload(nx, ny, n_freq=1):
    loops = W.square_array(nx, ny, seg_per_side=1)
    pts = W.grid_plane(2, 0.1, 0.02)
    omega = 2 * np.pi * np.linspace(60e6, 68e6, n_freq)
    st = W._structure_from(loops, pts, omega, 0.1, np.arange(2))
    C = np.full((1, nx * ny), 50e-12)
    return W.Workload("wide", [st], C, 0.001, target=np.zeros(2 * n_freq))


def test_port_limit_is_reported(nv):
    """Up to 1024 ports per structure validate; 1025 ports give MTS_EUNSUPPORTED (before any
    launch) from every entry point that validates the problem."""
    L = nv.lib()
    c, keep = fake_problem(nv, _wide_workload(32, 32))
    assert L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED) > 0
    c, keep = fake_problem(nv, _wide_workload(41, 25))
    assert L.mts_basis_bytes(ct.byref(c), nv.MTS_MIXED) == 0
    ev = nv.MtsEval()
    ev.n_cfg = 1
    ev.C = ev.omega = ev.V = FAKE
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                       ct.c_void_p(FAKE), 1 << 40, None)
    assert code == nv.MTS_EUNSUPPORTED


def test_tape_holds_factors_of_large_systems(nv):
    """Structures with more than 64 ports keep their LU factors in the tape: complex FP32
    (8 bytes) per matrix element for MTS_MIXED, complex FP64 (16 bytes) for MTS_FP64, for
    every configuration and frequency; structures of up to 64 ports add nothing."""
    L = nv.lib()
    small, k1 = fake_problem(nv, _wide_workload(8, 8, n_freq=3))
    big, k2 = fake_problem(nv, _wide_workload(16, 8, n_freq=3))
    for prec, elem in ((nv.MTS_MIXED, 8), (nv.MTS_FP64, 16)):
        t1 = L.mts_tape_bytes(ct.byref(big), 5, prec) - L.mts_tape_bytes(ct.byref(big), 4, prec)
        t0 = L.mts_tape_bytes(ct.byref(small), 5, prec) - L.mts_tape_bytes(ct.byref(small), 4, prec)
        # per-configuration growth: the factor block plus the small per-port arrays
        assert t1 - elem * 3 * 128 * 128 > 0
        assert t1 - elem * 3 * 128 * 128 < 4 * t0 + 4096


def test_adam_step_validation(nv):
    """Invalid optimiser settings are rejected before any launch."""
    L = nv.lib()
    good = nv.MtsAdam(1e-13, 0.9, 0.999, 1e-8, nv.MTS_PROJ_NONE, 0.0, 0.0)
    fp = ct.c_void_p(FAKE)

    def call(opt, n=4, C=fp, u=None, step=fp):
        return L.mts_adam_step(n, ct.byref(opt), C, u, fp, fp, fp, step, None, 0, None, 0, None)

    for bad in (nv.MtsAdam(-1.0, 0.9, 0.999, 1e-8, 0, 0.0, 0.0),
                nv.MtsAdam(1e-13, 1.0, 0.999, 1e-8, 0, 0.0, 0.0),
                nv.MtsAdam(1e-13, 0.9, -0.1, 1e-8, 0, 0.0, 0.0),
                nv.MtsAdam(1e-13, 0.9, 0.999, float("nan"), 0, 0.0, 0.0),
                nv.MtsAdam(1e-13, 0.9, 0.999, 1e-8, nv.MTS_PROJ_CLIP, 2e-10, 1e-10),
                nv.MtsAdam(1e-13, 0.9, 0.999, 1e-8, 7, 0.0, 1.0)):
        assert call(bad) == nv.MTS_EINVAL
    assert call(good, n=-1) == nv.MTS_EINVAL
    assert call(good, step=None) == nv.MTS_EINVAL
    tanh = nv.MtsAdam(1e-13, 0.9, 0.999, 1e-8, nv.MTS_PROJ_TANH, 1e-11, 2e-10)
    assert call(tanh, u=None) == nv.MTS_EINVAL


def test_schedule_fields_are_validated(nv):
    """large_threads must be 0, 128, 256 or 512 and reg_widen a combination of bits 0..2; the
    schedule does not change the tape size."""
    L = nv.lib()
    wl = W.array_8x8(n_cfg=2, grid=4, planes=(0.02,))
    c, keep = fake_problem(nv, wl)
    ev = nv.MtsEval()
    ev.n_cfg = 2
    ev.C = ev.omega = ev.V = FAKE
    tneed = L.mts_tape_bytes(ct.byref(c), 2, nv.MTS_MIXED)
    ev.large_threads = 64
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                       ct.c_void_p(FAKE), tneed, None)
    assert code == nv.MTS_EINVAL
    ev.large_threads = 0
    ev.reg_widen = 8
    code = L.mts_solve(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                       ct.c_void_p(FAKE), tneed, None)
    assert code == nv.MTS_EINVAL


def fake_sparams(nv, n0=4, n1=1, F=2, P=10, rows=(0, 1, 2), cols=(0, 1, 2), n_loss=0):
    c = nv.MtsSparams()
    c.n0, c.n1, c.n_freq, c.n_points = n0, n1, F, P
    keep = (np.ascontiguousarray(rows, np.int32), np.ascontiguousarray(cols, np.int32))
    c.n_svar = len(keep[0])
    c.n_loss = n_loss
    c.h_svar_row = keep[0].ctypes.data
    c.h_svar_col = keep[1].ctypes.data
    c.S0 = FAKE
    c.field = FAKE
    c.loss_idx = FAKE if n_loss else None
    return c, keep


def test_sroute_validation(nv):
    """The scattering-parameter route's host checks: sizes, index ranges, duplicate entries,
    the n0 <= 96 / n1 <= 8 / n_svar <= 1024 limits, and the RC preprocessing's arguments."""
    L = nv.lib()
    c, keep = fake_sparams(nv)
    assert L.mts_sroute_basis_bytes(ct.byref(c), nv.MTS_MIXED) > 0
    t1 = L.mts_sroute_tape_bytes(ct.byref(c), 10, nv.MTS_MIXED)
    t2 = L.mts_sroute_tape_bytes(ct.byref(c), 20, nv.MTS_MIXED)
    assert 0 < t1 < t2
    assert L.mts_sroute_tape_bytes(ct.byref(c), 10, nv.MTS_FP64) > 0
    assert L.mts_sroute_tape_bytes(ct.byref(c), -1, nv.MTS_FP64) == 0
    bad = [dict(rows=(0, 0), cols=(1, 1)),        # duplicate position
           dict(rows=(0, 5), cols=(0, 0)),        # row outside n0 + n1
           dict(rows=(0,), cols=(-1,)),
           dict(n0=0), dict(n1=0), dict(F=0), dict(P=-1)]
    for kw in bad:
        cb, kb = fake_sparams(nv, **kw)
        assert L.mts_sroute_basis_bytes(ct.byref(cb), nv.MTS_MIXED) == 0, kw
        assert L.mts_sroute_build(ct.byref(cb), nv.MTS_MIXED, ct.c_void_p(FAKE), 1 << 30, None) == nv.MTS_EINVAL, kw
    for kw in (dict(n0=97), dict(n1=9), dict(rows=tuple(range(1025)), cols=tuple([0] * 1025))):
        if "rows" in kw:
            cb, kb = fake_sparams(nv, n0=96, n1=8, rows=[i % 104 for i in range(1025)],
                                  cols=[i // 104 for i in range(1025)])
        else:
            cb, kb = fake_sparams(nv, **kw)
        assert L.mts_sroute_build(ct.byref(cb), nv.MTS_MIXED, ct.c_void_p(FAKE), 1 << 30, None) == nv.MTS_EUNSUPPORTED, kw
    # loss points without field points, too small a basis buffer, unaligned buffer
    cb, kb = fake_sparams(nv, P=0, n_loss=2)
    assert L.mts_sroute_build(ct.byref(cb), nv.MTS_MIXED, ct.c_void_p(FAKE), 1 << 30, None) == nv.MTS_EINVAL
    need = L.mts_sroute_basis_bytes(ct.byref(c), nv.MTS_MIXED)
    assert L.mts_sroute_build(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), need - 1, None) == nv.MTS_EWORKSPACE
    assert L.mts_sroute_build(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE + 8), need, None) == nv.MTS_EINVAL
    # per-call inputs
    ev = nv.MtsSrouteEval()
    ev.n_cfg, ev.svar, ev.loss_mode = 4, FAKE, 2
    tb = L.mts_sroute_tape_bytes(ct.byref(c), 4, nv.MTS_MIXED)
    assert L.mts_sroute_forward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                                None, ct.c_void_p(FAKE), tb, None) == nv.MTS_EINVAL
    ev.loss_mode = 0
    assert L.mts_sroute_forward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                                ct.c_void_p(FAKE), ct.c_void_p(FAKE), tb, None) == nv.MTS_EINVAL  # loss, no target
    assert L.mts_sroute_forward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev), None, None,
                                None, ct.c_void_p(FAKE), tb - 1, None) == nv.MTS_EWORKSPACE
    assert L.mts_sroute_backward(ct.byref(c), nv.MTS_MIXED, ct.c_void_p(FAKE), ct.byref(ev),
                                 ct.c_void_p(FAKE), tb, None, None, None, None) == nv.MTS_EINVAL
    # RC preprocessing
    assert L.mts_rc_reflection(2, 1, 3, FAKE, None, FAKE, 0.0, 3, 0, FAKE, None) == nv.MTS_EINVAL
    assert L.mts_rc_reflection(2, 1, 3, FAKE, None, FAKE, 50.0, 2, 0, FAKE, None) == nv.MTS_EINVAL
    assert L.mts_rc_reflection_vjp(2, 1, 3, FAKE, None, FAKE, 50.0, 4, 2, FAKE, None, FAKE, None) == nv.MTS_EINVAL
    assert nv.mts_launch_count() == 0


def test_system_status_validation(nv):
    """mts_system_status checks its arguments before touching the device; zero
    configurations is a no-op."""
    L = nv.lib()
    wl = W.array_8x8(n_cfg=2, grid=8, planes=(0.02,))
    c, keep = fake_problem(nv, wl)
    assert L.mts_system_status(ct.byref(c), 2, nv.MTS_MIXED, None, ct.c_void_p(FAKE), None) == nv.MTS_EINVAL
    assert L.mts_system_status(ct.byref(c), 2, nv.MTS_MIXED, ct.c_void_p(FAKE), None, None) == nv.MTS_EINVAL
    assert L.mts_system_status(ct.byref(c), -1, nv.MTS_MIXED, ct.c_void_p(FAKE), ct.c_void_p(FAKE), None) == nv.MTS_EINVAL
    assert L.mts_system_status(ct.byref(c), 2, 7, ct.c_void_p(FAKE), ct.c_void_p(FAKE), None) == nv.MTS_EINVAL
    assert L.mts_system_status(ct.byref(c), 0, nv.MTS_MIXED, ct.c_void_p(FAKE), ct.c_void_p(FAKE), None) == nv.MTS_OK
    cb, kb = fake_problem(nv, wl, n_struct=0)
    assert L.mts_system_status(ct.byref(cb), 2, nv.MTS_MIXED, ct.c_void_p(FAKE), ct.c_void_p(FAKE), None) == nv.MTS_EINVAL
    assert nv.mts_launch_count() == 0


@pytest.mark.skipif(__import__("shutil").which("gcc") is None, reason="gcc compiles the probe")
def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C compiler
    gives the struct of the same name in include/mts.h (a field name missing from the header
    fails the compile): the argument blocks cross the boundary unchanged."""
    import subprocess
    from paper_2503_18479_gb300 import native
    structs = {"mts_problem": native.MtsProblem, "mts_eval": native.MtsEval,
               "mts_adam": native.MtsAdam, "mts_sparams": native.MtsSparams,
               "mts_sroute_eval": native.MtsSrouteEval}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mts.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ct.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def _header_prototypes():
    src = open(os.path.join(ROOT, "include", "mts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    protos = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(mts_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src):
        ps = [q.strip() for q in params.split(",")]
        protos[name] = (ret.strip(), [] if ps == ["void"] or ps == [""] else ps)
    return protos


def _c_kind(decl: str) -> str:
    """Argument class of a C declaration: ptr, i32, i64, u64 (size_t too) or f64."""
    t = decl.replace("const ", "").split()[0]
    if "*" in decl or t == "mts_stream":  # mts_stream is a pointer typedef
        return "ptr"
    return {"int32_t": "i32", "int": "i32", "mts_status": "i32", "mts_precision": "i32",
            "mts_loss_mode": "i32", "mts_projection": "i32", "int64_t": "i64", "uint64_t": "u64",
            "size_t": "u64", "double": "f64"}[t]


def _ct_kind(t) -> str:
    if t is ct.c_void_p or t is ct.c_char_p or isinstance(t, type(ct.POINTER(ct.c_int))):
        return "ptr"
    # ctypes aliases c_int32 to c_int and c_uint64 to c_size_t on LP64 platforms
    return {ct.c_int32: "i32", ct.c_int: "i32", ct.c_int64: "i64", ct.c_uint64: "u64",
            ct.c_size_t: "u64", ct.c_double: "f64"}[t]


def test_binding_prototypes_match_the_header(nv):
    """Every entry point the binding declares takes, in the header, the same number of
    arguments with the same classes (pointer, 32- or 64-bit integer, size_t, double) in the
    same order, and returns the same class."""
    L = nv.lib()
    protos = _header_prototypes()
    assert set(protos) == set(declared_symbols())
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        want = [_c_kind(q) for q in params]
        got = [_ct_kind(t) for t in (f.argtypes or [])]
        assert got == want, (name, got, want)
        rk = "ptr" if "*" in ret else _c_kind(ret.split()[-1])
        assert _ct_kind(f.restype) == rk, (name, f.restype, ret)


@pytest.mark.skipif(__import__("shutil").which("gcc") is None, reason="gcc compiles the probe")
def test_binding_constants_match_the_header(tmp_path):
    """Every MTS_* constant of the binding (status codes, precisions, loss modes, projections)
    has the value the header gives it."""
    import subprocess
    from paper_2503_18479_gb300 import native
    names = sorted(n for n in vars(native) if re.fullmatch(r"MTS_[A-Z0-9_]+", n)
                   and isinstance(getattr(native, n), int))
    assert names
    lines = ["#include <stdio.h>", '#include "mts.h"', "int main(void) {"]
    lines += [f'  printf("{n} %lld\\n", (long long)({n}));' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {l.split()[0]: int(l.split()[1]) for l in out if l.strip()}
    for n in names:
        assert got[n] == getattr(native, n), n
