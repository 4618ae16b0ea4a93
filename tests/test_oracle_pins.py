"""Pins of the FP64 oracle against facts fixed outside it (closed forms, textbook limits,
exact identities, brute force). Each test names what a plausible mistake in the oracle
(a dropped term, a wrong sign, a transposed operand) would break. CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_18479_gb300 import workloads as W

MU0 = 4e-7 * np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def _loop_arrays(loops):
    return W.loops_to_arrays(loops)


# ---------------------------------------------------------------- Biot-Savart basis
@pytest.mark.parametrize("n_seg", [3, 4, 8, 64])
@pytest.mark.parametrize("z", [0.002, 0.020, -0.035, 0.3])
def test_regular_polygon_on_axis_closed_form(n_seg, z):
    """On the axis of a regular N-gon each side is a finite wire of half-length
    h = a sin(pi/N) at distance rho = sqrt(d^2 + z^2), d = a cos(pi/N); its field is
    mu0 I/(4 pi rho) 2h/sqrt(h^2 + rho^2) with z-fraction d/rho. Wrong sign of a cross
    product or a dropped |R2| term breaks this at 1e-12."""
    a = 0.05
    off, vx, vy, vz = _loop_arrays([W.circular_loop(a, n_seg)])
    H = oracle.basis(off, vx, vy, vz, [0.0], [0.0], [z], 1e-3)
    h, d = a * np.sin(np.pi / n_seg), a * np.cos(np.pi / n_seg)
    want = n_seg * MU0 / (4 * np.pi) * 2 * h * d / ((d * d + z * z) * np.sqrt(h * h + d * d + z * z))
    assert abs(H[0, 0] - want) <= 1e-12 * abs(want)


def test_polygon_value_at_20mm():
    """64-gon, a = 50 mm, z = 20 mm: 1.00630e-5 T/A; the circle gives 1.00583e-5."""
    off, vx, vy, vz = _loop_arrays([W.circular_loop(0.05, 64)])
    H = oracle.basis(off, vx, vy, vz, [0.0], [0.0], [0.02], 1e-3)
    assert abs(H[0, 0] - 1.00630e-5) < 5e-10
    circ = MU0 * 0.05 ** 2 / (2 * (0.05 ** 2 + 0.02 ** 2) ** 1.5)
    assert abs(circ - 1.00583e-5) < 5e-10


def test_circle_limit_on_axis():
    """N -> infinity: mu0 a^2 / (2 (a^2 + z^2)^(3/2)); the polygon error is O(N^-2)."""
    a, z = 0.05, 0.02
    want = MU0 * a * a / (2 * (a * a + z * z) ** 1.5)
    errs = []
    for n in (256, 512, 4096):
        off, vx, vy, vz = _loop_arrays([W.circular_loop(a, n)])
        H = oracle.basis(off, vx, vy, vz, [0.0], [0.0], [z], 1e-3)
        errs.append(abs(H[0, 0] / want - 1))
    assert errs[2] < 2e-6
    assert 3.5 < errs[0] / errs[1] < 4.5  # second order in 1/N


@pytest.mark.parametrize("rho,zp", [(0.02, 0.01), (0.049, 0.003), (0.08, -0.02), (0.0, 0.05)])
def test_circle_off_axis_elliptic(rho, zp):
    """Off-axis field of a circular loop from complete elliptic integrals (scipy's K, E):
    Bz = mu0/(2 pi) [K + (a^2 - rho^2 - z^2)/((a - rho)^2 + z^2) E]/sqrt((a + rho)^2 + z^2),
    m = 4 a rho/((a + rho)^2 + z^2). Checks the basis away from the symmetry axis."""
    from scipy.special import ellipe, ellipk
    a = 0.05
    m = 4 * a * rho / ((a + rho) ** 2 + zp ** 2)
    want = MU0 / (2 * np.pi) / np.sqrt((a + rho) ** 2 + zp ** 2) * (
        ellipk(m) + (a * a - rho * rho - zp * zp) / ((a - rho) ** 2 + zp ** 2) * ellipe(m))
    off, vx, vy, vz = _loop_arrays([W.circular_loop(a, 8192)])
    for phi in (0.0, 0.3):
        H = oracle.basis(off, vx, vy, vz, [rho * np.cos(phi)], [rho * np.sin(phi)], [zp], 1e-4)
        assert abs(H[0, 0] / want - 1) < 2e-5


def test_infinite_wire_limit():
    """A long straight segment at distance rho: Bz -> mu0 I/(2 pi rho); sign by the right
    hand rule (current along +x, point at -y: field along -z... here point at +y)."""
    L = 1e3
    rho = 0.01
    v = oracle.segment_bz((-L, 0, 0), (L, 0, 0), (0.0, rho, 0.0), 1e-3)
    assert abs(v / (MU0 / (2 * np.pi * rho)) - 1) < 1e-9
    v2 = oracle.segment_bz((-L, 0, 0), (L, 0, 0), (0.0, -rho, 0.0), 1e-3)
    assert abs(v2 + v) < 1e-15


def test_inside_wire_uniform_current():
    """Inside a round wire (rho < r_w) a uniform current gives mu0 I rho/(2 pi r_w^2)."""
    L, rw = 1e3, 1e-3
    for rho in (0.2e-3, 0.7e-3):
        v = oracle.segment_bz((-L, 0, 0), (L, 0, 0), (0.0, rho, 0.0), rw)
        assert abs(v / (MU0 * rho / (2 * np.pi * rw * rw)) - 1) < 1e-9
    assert oracle.segment_bz((-L, 0, 0), (L, 0, 0), (0.0, 0.0, 0.0), rw) == 0.0


def test_segment_beside_span_is_stable():
    """Point beside the middle of a short segment (R1.R2 < 0): the rewritten denominator
    must agree with the closed form mu0 I/(4 pi rho) 2h/sqrt(h^2+rho^2)."""
    h, rho = 1e-3, 5e-3
    v = oracle.segment_bz((-h, 0, 0), (h, 0, 0), (0.0, rho, 0.0), 1e-4)
    want = MU0 / (4 * np.pi * rho) * 2 * h / np.sqrt(h * h + rho * rho)
    assert abs(v / want - 1) < 1e-13


def test_mirror_symmetry_and_far_dipole():
    """Planar loop at z = 0: Bz(x, y, -z) = Bz(x, y, z); on the axis far away
    Bz -> mu0 m/(2 pi z^3) with m = area x 1 A (error O((a/z)^2))."""
    off, vx, vy, vz = _loop_arrays([W.square_loop(0.05, 16)])
    pts = np.array([[0.01, -0.02, 0.03], [0.2, 0.1, 0.005]])
    Hp = oracle.basis(off, vx, vy, vz, pts[:, 0], pts[:, 1], pts[:, 2], 1e-3)
    Hm = oracle.basis(off, vx, vy, vz, pts[:, 0], pts[:, 1], -pts[:, 2], 1e-3)
    assert np.allclose(Hp, Hm, rtol=1e-14, atol=0)
    z = 2.0
    Hf = oracle.basis(off, vx, vy, vz, [0.0], [0.0], [z], 1e-3)
    dip = MU0 * 0.05 ** 2 / (2 * np.pi * z ** 3)
    assert abs(Hf[0, 0] / dip - 1) < 2e-3


def test_loop_orientation_sign():
    """A counter-clockwise loop (seen from +z) with positive current makes +z field inside."""
    off, vx, vy, vz = _loop_arrays([W.square_loop(0.05, 4)])
    H = oracle.basis(off, vx, vy, vz, [0.0], [0.0], [0.0], 1e-3)
    assert H[0, 0] > 0


# ---------------------------------------------------------------- inductance
def test_square_loop_inductance_grover():
    """Square loop of side a, thin round wire of radius r: L = (2 mu0 a/pi)(ln(a/r) - 0.774)
    (Grover's formula, no internal inductance). The exact partial-inductance constant is
    ln 2 - 2 - asinh 1 + sqrt 2 = -0.774013. Pins the self term, the opposite-side
    (antiparallel) sign and the factor mu0/(4 pi)."""
    for a, r in ((0.05, 1e-3), (0.028, 5e-4), (0.1, 2e-3)):
        off, vx, vy, vz = _loop_arrays([W.square_loop(a, 16)])
        st, M = oracle.inductance(off, vx, vy, vz, r)
        assert st == 0
        exact = 2 * MU0 * a / np.pi * (np.log(a / r) + np.log(2) - 2 - np.arcsinh(1) + np.sqrt(2))
        assert abs(M[0, 0] / exact - 1) < 1e-12
        grover = 2 * MU0 * a / np.pi * (np.log(a / r) - 0.774)
        assert abs(M[0, 0] / grover - 1) < 1e-4
    off, vx, vy, vz = _loop_arrays([W.square_loop(0.05, 16)])
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    assert abs(M[0, 0] - 125.52e-9) < 0.01e-9


def test_parallel_filaments_textbook():
    """Two equal parallel filaments, length l, distance d (textbook Neumann result):
    M = mu0 l/(2 pi) [asinh(l/d) - sqrt(1 + d^2/l^2) + d/l]; opposite currents flip the
    sign; a perpendicular pair gives 0."""
    l, d = 0.05, 0.013
    st, m = oracle.segment_pair_inductance((0, 0, 0), (l, 0, 0), (0, d, 0), (l, d, 0), 1e-3)
    want = MU0 * l / (2 * np.pi) * (np.arcsinh(l / d) - np.sqrt(1 + d * d / (l * l)) + d / l)
    assert st == 0 and abs(m / want - 1) < 1e-13
    st, m2 = oracle.segment_pair_inductance((0, 0, 0), (l, 0, 0), (l, d, 0), (0, d, 0), 1e-3)
    assert st == 0 and abs(m2 + m) < 1e-24
    st, m3 = oracle.segment_pair_inductance((0, 0, 0), (l, 0, 0), (0, d, 0), (0, d + l, 0), 1e-3)
    assert st == 0 and m3 == 0.0


@pytest.mark.parametrize("ends", ["end-start", "end-end", "start-start", "start-end"])
def test_touching_filaments_neumann(ends):
    """Oblique filaments that share an end point (a polygon corner): the oracle's closed form
    against the Neumann double integral mu0/(4 pi) int int dl1.dl2 / |r1 - r2| done by
    scipy's 2-D adaptive quadrature (the integrand's 1/r corner singularity is integrable),
    for every way the shared point can be an end of each segment, at acute and obtuse
    angles; a right-angle corner gives exactly 0."""
    integrate = pytest.importorskip("scipy.integrate")
    O = np.array([0.01, 0.004, 0.0])
    for P, Q in ((O + [0.02, 0.0, 0.0], O + [0.01, 0.015, 0.0]),
                 (O + [0.012, 0.003, 0.0], O + [-0.02, 0.01, 0.004])):
        a0, a1 = (P, O) if ends.startswith("end") else (O, P)
        b0, b1 = (O, Q) if ends.endswith("start") else (Q, O)
        d1, d2 = a1 - a0, b1 - b0
        f = lambda t, u: 1.0 / np.linalg.norm(a0 + u * d1 - (b0 + t * d2))
        v, _ = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-13, epsrel=1e-11)
        want = MU0 / (4 * np.pi) * float(d1 @ d2) * v
        st, m = oracle.segment_pair_inductance(a0, a1, b0, b1, 1e-3)
        assert st == 0 and abs(m / want - 1) < 1e-9, (m, want)
    st, m = oracle.segment_pair_inductance(O + [0.02, 0, 0], O, O, O + [0, 0.03, 0], 1e-3)
    assert st == 0 and m == 0.0


def test_polygon_self_inductance_circle_limit():
    """A regular n-gon's self inductance from its segments (self terms, collinear-free
    corners by the touching closed form, the rest by quadrature) tends to the circular
    loop's mu0 a (ln(8a/rw) - 2) (high-frequency form) as n grows: the gap shrinks as
    1/n^2, and the Richardson extrapolation of n = 128 and 256 lands within 2e-5."""
    a, rw = 0.05, 1e-4
    circle = MU0 * a * (np.log(8 * a / rw) - 2)
    Ls = []
    for n in (64, 128, 256):
        off, vx, vy, vz = _loop_arrays([W.circular_loop(a, n)])
        st, M = oracle.inductance(off, vx, vy, vz, rw)
        assert st == 0
        Ls.append(M[0, 0])
    gaps = [circle - L for L in Ls]
    assert all(g > 0 for g in gaps)
    assert 3.5 < gaps[0] / gaps[1] < 4.2 and 3.5 < gaps[1] / gaps[2] < 4.2
    assert abs((4 * Ls[2] - Ls[1]) / 3 / circle - 1) < 2e-5


def test_polygon_subdivision_invariance():
    """Splitting every side of a regular octagon (wire radius well below the pieces) into
    2, 3 or 4 collinear pieces leaves its self inductance unchanged: the touching corners,
    the collinear pieces and the oblique pairs across corners (quadrature) add up to the
    same Neumann integral."""
    a, rw = 0.05, 1e-4
    v = np.stack(W.circular_loop(a, 8), 1)
    Ls = []
    for sub in (1, 2, 3, 4):
        pts = [p + (q - p) * s / sub for p, q in zip(v, np.roll(v, -1, 0)) for s in range(sub)]
        P = np.array(pts)
        st, M = oracle.inductance(np.array([0, len(P)], np.int32), P[:, 0], P[:, 1], P[:, 2], rw)
        assert st == 0
        Ls.append(M[0, 0])
    assert max(abs(L / Ls[0] - 1) for L in Ls[1:]) < 1e-10, Ls


def test_collinear_filaments_textbook():
    """Collinear filaments of lengths a and b separated by a gap g (Neumann):
    M = mu0/(4 pi)[F(a+b+g) - F(a+g) - F(b+g) + F(g)], F(x) = x ln x."""
    F = lambda x: x * np.log(x) if x > 0 else 0.0
    for a, b, g in ((0.01, 0.02, 0.0), (0.01, 0.03, 0.005)):
        st, m = oracle.segment_pair_inductance((0, 0, 0), (a, 0, 0), (a + g, 0, 0), (a + g + b, 0, 0), 1e-3)
        want = MU0 / (4 * np.pi) * (F(a + b + g) - F(a + g) - F(b + g) + F(g))
        assert st == 0 and abs(m / want - 1) < 1e-12
    st, _ = oracle.segment_pair_inductance((0, 0, 0), (0.02, 0, 0), (0.01, 0, 0), (0.03, 0, 0), 1e-3)
    assert st == 2


def test_inductance_subdivision_invariance_and_symmetry():
    """Partial inductances add exactly under subdivision of a straight side, so 1, 2 and 16
    segments per side give the same self and mutual inductances; M is symmetric."""
    Ms = []
    for seg in (1, 2, 16):
        off, vx, vy, vz = _loop_arrays(W.square_array(3, 2, seg_per_side=seg))
        st, M = oracle.inductance(off, vx, vy, vz, 1e-3)
        assert st == 0
        assert np.allclose(M, M.T, rtol=1e-13, atol=0)
        Ms.append(M)
    assert _rel(Ms[1], Ms[0]) < 1e-13 and _rel(Ms[2], Ms[0]) < 1e-12
    assert np.all(np.diag(Ms[0]) > 0)
    # neighbours along x and y couple negatively (coplanar loops), stronger than diagonal ones
    assert Ms[0][0, 1] < 0 and Ms[0][0, 3] < 0 and abs(Ms[0][0, 1]) > abs(Ms[0][0, 4])


def test_mutual_inductance_equals_flux_of_basis():
    """Reciprocity between the two halves of the oracle: M_kl (Neumann double line
    integral) equals the flux of loop l's Biot-Savart field through the area of loop k
    (Stokes). 2-D Gauss-Legendre quadrature of the basis over loop k's square."""
    side, pitch = 0.05, 0.055
    loops = W.square_array(2, 2, seg_per_side=4)
    off, vx, vy, vz = _loop_arrays(loops)
    st, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    xg, wg = np.polynomial.legendre.leggauss(160)
    h = side / 2
    for k, l in ((0, 1), (0, 3), (2, 1)):
        cx = np.mean(vx[off[k]:off[k + 1]])
        cy = np.mean(vy[off[k]:off[k + 1]])
        X, Y = np.meshgrid(cx + h * xg, cy + h * xg)
        WW = np.outer(wg, wg) * h * h
        sub = np.array([off[l], off[l + 1]]) - off[l]
        Hl = oracle.basis(sub, vx[off[l]:off[l + 1]], vy[off[l]:off[l + 1]], vz[off[l]:off[l + 1]],
                          X.ravel(), Y.ravel(), np.zeros(X.size), 1e-3)
        flux = float(np.sum(Hl[:, 0] * WW.ravel()))
        assert abs(flux / M[k, l] - 1) < 1e-5, (k, l, flux, M[k, l])


def test_L_self_override():
    """Given L_self replaces the diagonal only."""
    off, vx, vy, vz = _loop_arrays(W.square_array(2, 1))
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    _, M2 = oracle.inductance(off, vx, vy, vz, 1e-3, L_self=[1e-7, 2e-7])
    assert M2[0, 0] == 1e-7 and M2[1, 1] == 2e-7 and M2[0, 1] == M[0, 1]


# ---------------------------------------------------------------- port solve
def _det(A):
    """Determinant by permutation expansion (brute force, N <= 4)."""
    n = A.shape[0]
    tot = 0j
    for perm in itertools.permutations(range(n)):
        sgn = 1
        for i in range(n):
            for j in range(i + 1, n):
                if perm[i] > perm[j]:
                    sgn = -sgn
        term = 1 + 0j
        for i in range(n):
            term *= A[i, perm[i]]
        tot += sgn * term
    return tot


def _small_problem(n, seed=3):
    rng = np.random.default_rng(seed)
    loops = W.square_array(n, 1)
    off, vx, vy, vz = _loop_arrays(loops)
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    R = np.full(n, 0.1)
    C = rng.uniform(20e-12, 200e-12, n)
    w = 2 * np.pi * 63.6e6
    V = W.drive_uniform_field(loops, np.array([w]))[0]
    return M, R, C, w, V


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_solve_matches_cramer(n):
    """Cramer's rule with brute-force determinants versus the LU solve."""
    M, R, C, w, V = _small_problem(n)
    A = oracle.assemble(M, R, w, C)
    st, Iv = oracle.solve_loaded(A, np.zeros(n), V)
    d = _det(A)
    for k in range(n):
        Ak = A.copy()
        Ak[:, k] = V
        assert abs(_det(Ak) / d - Iv[k]) <= 1e-12 * np.abs(Iv).max()


def test_assemble_entries():
    """A = diag(R) + j w M + diag(1/(j w C)) = R + j w L - j/(w C) on the diagonal (Eq. 11)."""
    M, R, C, w, V = _small_problem(3)
    A = oracle.assemble(M, R, w, C)
    for i in range(3):
        assert abs(A[i, i] - (R[i] + 1j * w * M[i, i] - 1j / (w * C[i]))) < 1e-12 * abs(A[i, i])
        for j in range(3):
            if i != j:
                assert A[i, j] == 1j * w * M[i, j]


def test_lu_pivoting_and_residual():
    """LU on a matrix whose (0,0) entry is 0 needs a row swap; P A = L U and the residual of
    a solve is at rounding level."""
    A = np.array([[0, 2, 1], [1, 1, 1], [3, 0, 2]], dtype=complex) + 1j * np.eye(3) * 0
    st, LU, piv = oracle.lu(A)
    assert st == 0 and piv[0] == 2
    n = 3
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert np.allclose(L @ U, PA, atol=1e-14)
    M, R, C, w, V = _small_problem(8)
    A = oracle.assemble(M, R, w, C)
    st, LU, piv = oracle.lu(A)
    x = oracle.lu_solve(LU, piv, V)
    assert np.linalg.norm(A @ x - V) <= 1e-13 * np.linalg.norm(A) * np.linalg.norm(x)


def test_passivity_and_linearity():
    """Re(I^H V) = sum R |I|^2 exactly (M real symmetric and 1/(jwC) imaginary carry no
    real power); the solution is linear in V."""
    M, R, C, w, V = _small_problem(8)
    A = oracle.assemble(M, R, w, C)
    _, I1 = oracle.solve_loaded(A, np.zeros(8), V)
    p_in = np.real(np.vdot(I1, V))
    assert abs(p_in - np.sum(R * np.abs(I1) ** 2)) < 1e-12 * p_in
    V2 = np.roll(V, 3) * (0.3 - 2j)
    _, I2 = oracle.solve_loaded(A, np.zeros(8), V2)
    _, I3 = oracle.solve_loaded(A, np.zeros(8), 2 * V + V2)
    assert _rel(I3, 2 * I1 + I2) < 1e-12


def test_single_loop_resonance():
    """Eq. 11, 13: at w0 = 1/sqrt(L C) the reactance cancels and I = V/R exactly; |I| peaks
    at f0 = 1/(2 pi sqrt(L C))."""
    L, R, C = 250.79e-9, 0.1, 24.97e-12
    w0 = 1 / np.sqrt(L * C)
    V = np.array([1e-3 + 0.5e-3j])
    _, Iv = oracle.solve_loaded(oracle.assemble(np.array([[L]]), [R], w0, [C]), [0], V)
    assert abs(Iv[0] - V[0] / R) < 1e-12 * abs(V[0] / R)
    ws = w0 * np.linspace(0.98, 1.02, 401)
    mags = [abs(oracle.solve_loaded(oracle.assemble(np.array([[L]]), [R], w, [C]), [0], V)[1][0]) for w in ws]
    assert abs(ws[int(np.argmax(mags))] / w0 - 1) < 1e-4


def test_resonance_golden_single_loop():
    """Resonant capacitances of the single-loop workload (Eq. 13 with M = 0) stored in
    tests/golden/resonance_single_loop.txt."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "resonance_single_loop.txt"))
            if l.strip() and not l.startswith("#")]
    L = W.circular_loop_inductance(0.05, 1e-3)
    assert abs(L - 250.79e-9) < 0.01e-9
    for f_mhz, c_pf in rows:
        w = 2 * np.pi * float(f_mhz) * 1e6
        cr = 1 / (w * w * L)
        assert abs(cr / 1e-12 - float(c_pf)) < 0.005
        # the oracle's solve sees zero reactance there: I = V/R
        _, Iv = oracle.solve_loaded(oracle.assemble(np.array([[L]]), [0.1], w, [cr]), [0], [1.0])
        assert abs(Iv[0] - 10.0) < 1e-9


def test_paper_0d_cell_resonance_plausible():
    """Sec. IV-A prints C_r = 8.39 pF at 123.5 MHz for a loop of 30 mm inner radius and 1 mm
    strip width (its L came from the full-wave model, with the phantom). Our thin-loop
    inductance for that loop (centre radius 30.5 mm, strip-equivalent wire radius w/4)
    lands within 10 % of it. A plausibility check, not a parity claim."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_values.txt"))
            if l.strip() and not l.startswith("#")]
    vals = {k: float(v) for k, v in rows}
    w = 2 * np.pi * vals["f0_mhz"] * 1e6
    L = W.circular_loop_inductance(0.0305, 0.25e-3)
    cr = 1 / (w * w * L)
    assert abs(cr / (vals["C_r_pf"] * 1e-12) - 1) < 0.10


def test_d4_symmetry_of_8x8():
    """Mirroring the 8x8 array in x maps loop (i, j) to (7 - i, j). Mirroring the
    capacitances the same way mirrors the currents and the field map."""
    wl = W.array_8x8(n_cfg=1, grid=8, planes=(0.02,))
    s = wl.structures[0]
    H = oracle.basis(s.loop_vtx_off, s.vx, s.vy, s.vz, s.px, s.py, s.pz, wl.wire_radius)
    _, M = oracle.inductance(s.loop_vtx_off, s.vx, s.vy, s.vz, wl.wire_radius)
    perm = np.array([j * 8 + (7 - i) for j in range(8) for i in range(8)])
    C = wl.C[0]
    out1 = oracle.forward(H, M, s.R, C[None], s.omega, s.V, want_loss=False)
    out2 = oracle.forward(H, M, s.R, C[perm][None], s.omega, s.V, want_loss=False)
    assert _rel(out2["I"][0, 0], out1["I"][0, 0][perm]) < 1e-12
    g = 8
    pm = np.array([iy * g + (g - 1 - ix) for iy in range(g) for ix in range(g)])
    assert _rel(out2["B"][0, 0, :g * g], out1["B"][0, 0, :g * g][pm]) < 1e-11


# ---------------------------------------------------------------- S-parameter route
def _drive_structure(n_cells=3, seed=5):
    """n_cells square loops plus a larger drive loop around them (a one-port excitation
    coil, like the paper's PEC drive loop in Sec. III-B)."""
    rng = np.random.default_rng(seed)
    loops = W.square_array(n_cells, 1, seg_per_side=4)
    loops.append(W.square_loop(0.2, 4, 0.0, 0.0, 0.03))
    off, vx, vy, vz = _loop_arrays(loops)
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    n = len(loops)
    w = 2 * np.pi * 63.6e6
    R = np.full(n, 0.1)
    C = rng.uniform(20e-12, 200e-12, n)
    Z = np.diag(R).astype(complex) + 1j * w * M
    return Z, C, w, n


def test_sroute_equals_zroute():
    """Eq. 3-7: terminating every loop port by 1/(jwC) through its reflection coefficient,
    driving the last port by a matched source sqrt(Z0 P), and reading the currents
    (1 - S0) V+/Z0 equals the impedance route with a Thevenin source E = 2 sqrt(Z0 P)
    behind Z0 on the drive port."""
    Z, C, w, n = _drive_structure()
    Z0, P = 50.0, 1.0
    Zl = 1 / (1j * w * C)
    st, I_s, _ = oracle.sroute(Z, Zl, n - 1, Z0, P, w)
    assert st == 0
    Zl_z = Zl.copy()
    Zl_z[n - 1] = Z0
    E = np.zeros(n, complex)
    E[n - 1] = 2 * np.sqrt(Z0 * P)
    _, I_z = oracle.solve_loaded(Z, Zl_z, E)
    assert _rel(I_s, I_z) < 1e-11


def test_eq10_derivative_equals_direct():
    """Eq. 10 (S-route derivative of the wave ratio) equals the impedance-route direct
    sensitivity dI/dC_k = -A^-1 e_k (j/(w C_k^2)) I_k (Eq. 9 in Z form)."""
    Z, C, w, n = _drive_structure()
    Z0, P = 50.0, 1.0
    Zl = 1 / (1j * w * C)
    st, I_s, dI_s = oracle.sroute(Z, Zl, n - 1, Z0, P, w, C=C, want_dI=True)
    # Z route: the drive port's load is Z0 (not a capacitor); the source is E
    Mfake = (Z - np.diag(np.diag(Z).real)) / (1j * w)
    R = np.diag(Z).real.copy()
    Cz = C.copy()
    # fold the drive port's Z0 into R and give it an "infinite" capacitor
    R[n - 1] += Z0
    Cz[n - 1] = 1e30
    E = np.zeros(n, complex)
    E[n - 1] = 2 * np.sqrt(Z0 * P)
    st2, dI_z = oracle.dcurrents_dC(Mfake.real, R, w, Cz, E)
    assert st2 == 0
    for k in range(n - 1):
        assert _rel(dI_s[k], dI_z[k]) < 1e-9


def _sroute_from_zroute(n_cells=3, seed=5, F=2, n_batch=3, Z0=50.0, P_in=1.0):
    """A loop structure written in the pipeline's terms (Sec. III, Eq. 3-7): ports at the
    cell capacitors and at the drive loop, S0 = (Z - Z0)(Z + Z0)^-1 per frequency, fields
    per unit incident wave at port k with the other ports matched, i.e. the Biot-Savart
    field of the currents (1 - S0) e_k / Z0, times sqrt(Z0 P) (Eq. 4's V-exc) so that the
    combined field is the physical one. The drive port sees a matched source through S_C12;
    each cell port is loaded by its capacitor, scattered into S_C11 as Gamma (Eq. 3)."""
    rng = np.random.default_rng(seed)
    loops = W.square_array(n_cells, 1, seg_per_side=4)
    loops.append(W.square_loop(0.2, 4, 0.0, 0.0, 0.03))
    off, vx, vy, vz = _loop_arrays(loops)
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    px, py, pz = W.grid_plane(5, 0.1, 0.02)
    H = oracle.basis(off, vx, vy, vz, px, py, pz, 1e-3)
    n0 = len(loops)
    omega = 2 * np.pi * np.linspace(62e6, 65e6, F)
    R = np.full(n0, 0.1)
    C = rng.uniform(20e-12, 200e-12, (n_batch, n0 - 1))
    S0 = np.zeros((F, n0, n0), complex)
    field = np.zeros((F, len(px), n0), complex)
    for f, w in enumerate(omega):
        Z = np.diag(R).astype(complex) + 1j * w * M
        S0[f] = np.linalg.solve((Z + Z0 * np.eye(n0)).T, (Z - Z0 * np.eye(n0)).T).T
        field[f] = H @ (np.eye(n0) - S0[f]) / Z0 * np.sqrt(Z0 * P_in)
    Sconst = np.zeros((F, n0 + 1, n0 + 1), complex)
    Sconst[:, n0 - 1, n0] = 1.0  # S_C12: the source's wave enters the drive port
    rows = np.arange(n0 - 1)
    Zl = 1 / (1j * omega[None, :, None] * C[:, None, :])  # [b, f, k]
    svar = (Zl - Z0) / (Zl + Z0)  # Eq. 3
    return dict(H=H, M=M, R=R, C=C, omega=omega, S0=S0, field=field, Sconst=Sconst,
                rows=rows, cols=rows, svar=svar, Z0=Z0, P_in=P_in, n0=n0)


def test_sroute_pipeline_equals_impedance_route():
    """The pipeline's combined field equals H I of the impedance route with the drive loop
    fed by a Thevenin source E = 2 sqrt(Z0 P) behind Z0 and the cells closed by their
    capacitors (the Z <-> S identity of Eq. 3-6 carried through Eq. 7)."""
    c = _sroute_from_zroute()
    out = oracle.sroute_pipeline(c["S0"], c["field"], c["Sconst"], c["rows"], c["cols"], c["svar"])
    assert out["n_singular"] == 0
    n0, Z0 = c["n0"], c["Z0"]
    for b in range(c["C"].shape[0]):
        for f, w in enumerate(c["omega"]):
            Z = np.diag(c["R"]).astype(complex) + 1j * w * c["M"]
            Zl = np.append(1 / (1j * w * c["C"][b]), Z0)
            E = np.zeros(n0, complex)
            E[-1] = 2 * np.sqrt(Z0 * c["P_in"])
            _, I = oracle.solve_loaded(Z, Zl, E)
            assert _rel(out["B"][b, 0, f], c["H"] @ I) < 1e-11


def test_sroute_one_port_closed_form():
    """n0 = n1 = 1: A = 1 - s11 s0 and W = s12 / (1 - s11 s0) (Eq. 6), B = field W (Eq. 7)."""
    rng = np.random.default_rng(3)
    F, P = 3, 4
    S0 = (rng.uniform(-0.6, 0.6, (F, 1, 1)) + 1j * rng.uniform(-0.6, 0.6, (F, 1, 1)))
    field = rng.standard_normal((F, P, 1)) + 1j * rng.standard_normal((F, P, 1))
    Sconst = np.zeros((F, 2, 2), complex)
    Sconst[:, 0, 1] = 0.7 - 0.2j
    svar = rng.uniform(-0.9, 0.9, (2, F, 1)) + 1j * rng.uniform(-0.9, 0.9, (2, F, 1))
    out = oracle.sroute_pipeline(S0, field, Sconst, [0], [0], svar)
    Wc = (0.7 - 0.2j) / (1 - svar[:, :, 0] * S0[None, :, 0, 0])
    assert _rel(out["W"][:, :, 0, 0], Wc) < 1e-14
    assert _rel(out["B"][:, 0], Wc[:, :, None] * field[None, :, :, 0]) < 1e-14


def test_sroute_two_ports_by_cramer():
    """A general 2 x 2 network (every S11 entry variable, two external ports): W from
    Cramer's rule on A = 1 - S11 S0."""
    rng = np.random.default_rng(4)
    F, P, n0, n1 = 1, 3, 2, 2
    S0 = (rng.standard_normal((F, n0, n0)) + 1j * rng.standard_normal((F, n0, n0))) * 0.4
    field = rng.standard_normal((F, P, n0)) + 1j * rng.standard_normal((F, P, n0))
    Sconst = (rng.standard_normal((F, 4, 4)) + 1j * rng.standard_normal((F, 4, 4))) * 0.3
    rows, cols = [0, 0, 1, 1, 2], [0, 1, 0, 1, 3]
    svar = (rng.standard_normal((1, F, 5)) + 1j * rng.standard_normal((1, F, 5))) * 0.3
    out = oracle.sroute_pipeline(S0, field, Sconst, rows, cols, svar)
    SC = Sconst[0].copy()
    for i, (r, q) in enumerate(zip(rows, cols)):
        SC[r, q] += svar[0, 0, i]
    A = np.eye(2) - SC[:2, :2] @ S0[0]
    det = A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
    for c in range(n1):
        b0, b1 = SC[0, 2 + c], SC[1, 2 + c]
        w0 = (b0 * A[1, 1] - A[0, 1] * b1) / det
        w1 = (A[0, 0] * b1 - b0 * A[1, 0]) / det
        assert _rel(out["W"][0, 0, :, c], [w0, w1]) < 1e-13
        assert _rel(out["B"][0, c, 0], field[0] @ np.array([w0, w1])) < 1e-13


def _sroute_random(mode, seed=7, F=2, n0=4, n1=2, P=9, n_batch=2):
    rng = np.random.default_rng(seed)
    S0 = (rng.standard_normal((F, n0, n0)) + 1j * rng.standard_normal((F, n0, n0))) * 0.25
    field = rng.standard_normal((F, P, n0)) + 1j * rng.standard_normal((F, P, n0))
    n = n0 + n1
    Sconst = (rng.standard_normal((F, n, n)) + 1j * rng.standard_normal((F, n, n))) * 0.2
    # S11 diagonal and off-diagonal, S12, S21 and S22 entries
    rows = np.array([0, 1, 2, 3, 1, 0, 2, 5, 4])
    cols = np.array([0, 1, 2, 3, 3, 4, 5, 1, 4])
    svar = (rng.standard_normal((n_batch, F, len(rows))) + 1j * rng.standard_normal((n_batch, F, len(rows)))) * 0.3
    li = np.array([0, 4, 7])
    if mode == 0:
        t = np.abs(rng.standard_normal((F, n1, len(li))))
    else:
        t = rng.standard_normal((F, n1, len(li), 2))
    return S0, field, Sconst, rows, cols, svar, li, t


@pytest.mark.parametrize("mode", [0, 1])
def test_sroute_gradient_central_differences(mode):
    """Eq. 10's gradient against central differences of the objective along the real and
    imaginary part of every variable S-parameter (torch's dL/dRe + j dL/dIm); S21 and S22
    entries do not reach the field and get exactly 0."""
    S0, field, Sconst, rows, cols, svar, li, t = _sroute_random(mode)
    g = oracle.sroute_gradient(S0, field, Sconst, rows, cols, svar, li, t, mode=mode)
    h = 1e-6
    fd = np.zeros_like(g)
    for idx in np.ndindex(*svar.shape):
        for unit in (1.0, 1j):
            sp, sm = svar.copy(), svar.copy()
            sp[idx] += h * unit
            sm[idx] -= h * unit
            lp = oracle.sroute_pipeline(S0, field, Sconst, rows, cols, sp, li, t, mode=mode, want_B=False)["loss"]
            lm = oracle.sroute_pipeline(S0, field, Sconst, rows, cols, sm, li, t, mode=mode, want_B=False)["loss"]
            d = (lp[idx[0]] - lm[idx[0]]) / (2 * h)
            fd[idx] += d * (1.0 if unit == 1.0 else 1j)
    assert _rel(g, fd) < 1e-7
    assert np.all(g[:, :, rows >= 4] == 0)


def test_sroute_enhancement_objective():
    """The weighted, offset objective of the pipeline: its value is the mean of
    (|w (B + o)| - t)^2 over (f, c, l) from the pipeline's own field, and its Eq. 10 gradient
    matches central differences."""
    S0, field, Sconst, rows, cols, svar, li, t = _sroute_random(0)
    rng = np.random.default_rng(12)
    w = rng.uniform(0.5, 2.0, t.shape)
    o = (rng.standard_normal(t.shape) + 1j * rng.standard_normal(t.shape)) * 0.3
    out = oracle.sroute_pipeline(S0, field, Sconst, rows, cols, svar, li, t, weight=w, offset=o)
    Bl = np.transpose(out["B"][:, :, :, li], (0, 2, 1, 3))  # [b, F, n1, L]
    want = ((np.abs(w[None] * (Bl + o[None])) - t[None]) ** 2).mean(axis=(1, 2, 3))
    assert _rel(out["loss"], want) < 1e-13
    g = oracle.sroute_gradient(S0, field, Sconst, rows, cols, svar, li, t, weight=w, offset=o)
    h = 1e-6
    fd = np.zeros_like(g)
    for idx in np.ndindex(*svar.shape):
        for unit in (1.0, 1j):
            sp, sm = svar.copy(), svar.copy()
            sp[idx] += h * unit
            sm[idx] -= h * unit
            kw = dict(want_B=False, weight=w, offset=o)
            d = (oracle.sroute_pipeline(S0, field, Sconst, rows, cols, sp, li, t, **kw)["loss"][idx[0]]
                 - oracle.sroute_pipeline(S0, field, Sconst, rows, cols, sm, li, t, **kw)["loss"][idx[0]]) / (2 * h)
            fd[idx] += d * unit
    assert _rel(g, fd) < 1e-7


def test_sroute_gradient_through_eq3_equals_impedance_adjoint():
    """Chaining Eq. 10 through Eq. 3 (dGamma/dC = 2 Z0 / (Zl + Z0)^2 * j/(w C^2)) gives the
    impedance route's adjoint dloss/dC on the same structure and objective."""
    c = _sroute_from_zroute(n_batch=2)
    F, n0, Z0 = len(c["omega"]), c["n0"], c["Z0"]
    li = np.array([2, 7, 12, 20])
    t = np.full((F, 1, len(li)), 2e-7)
    g = oracle.sroute_gradient(c["S0"], c["field"], c["Sconst"], c["rows"], c["cols"], c["svar"], li, t)
    w = c["omega"][None, :, None]
    Zl = 1 / (1j * w * c["C"][:, None, :])
    dgam = 2 * Z0 / (Zl + Z0) ** 2 * (1j / (w * c["C"][:, None, :] ** 2))
    gC = np.real(np.conj(g) * dgam).sum(axis=1)  # [b, n0 - 1]
    # impedance route: the drive loop's Z0 in R, an "infinite" capacitor, EMF 2 sqrt(Z0 P)
    R = c["R"].copy()
    R[-1] += Z0
    Cz = np.concatenate([c["C"], np.full((c["C"].shape[0], 1), 1e30)], axis=1)
    V = np.zeros((F, n0), complex)
    V[:, -1] = 2 * np.sqrt(Z0 * c["P_in"])
    gz = oracle.gradient(c["H"], c["M"], R, Cz, c["omega"], V, li, t[:, 0, :])
    out = oracle.sroute_pipeline(c["S0"], c["field"], c["Sconst"], c["rows"], c["cols"], c["svar"],
                                 li, t, want_B=False)
    lz = oracle.forward(c["H"], c["M"], R, Cz, c["omega"], V, li, t[:, 0, :], want_B=False)["loss"]
    assert _rel(out["loss"], lz) < 1e-10
    assert _rel(gC, gz[:, :-1]) < 1e-9


# ---------------------------------------------------------------- objective and gradient
def _grad_case(mode=0, n=6, F=3, n_cfg=2, seed=11):
    rng = np.random.default_rng(seed)
    loops = W.square_array(n // 2, 2, seg_per_side=4)
    off, vx, vy, vz = _loop_arrays(loops)
    px, py, pz = W.grid_plane(6, 0.1, 0.02)
    H = oracle.basis(off, vx, vy, vz, px, py, pz, 1e-3)
    _, M = oracle.inductance(off, vx, vy, vz, 1e-3)
    R = np.full(n, 0.1)
    C = rng.uniform(20e-12, 200e-12, (n_cfg, n))
    omega = 2 * np.pi * np.linspace(61e6, 66e6, F)
    V = W.drive_uniform_field(loops, omega)
    li = np.array([3, 10, 17, 29])
    if mode == 0:
        t = np.abs(rng.standard_normal((F, len(li)))) * 3e-7
    else:
        t = (rng.standard_normal((F, len(li), 2)) * 3e-7)
    return H, M, R, C, omega, V, li, t


def _beta_inputs(H, li, F, seed=21):
    rng = np.random.default_rng(seed)
    L = len(li)
    Bref = (rng.uniform(0.5, 1.5, (F, L)) * 3e-7) * np.exp(1j * rng.uniform(-np.pi, np.pi, (F, L)))
    Binc = (rng.standard_normal((F, L)) + 1j * rng.standard_normal((F, L))) * 2e-7
    beta_t = rng.uniform(0.5, 2.5, (F, L))
    return Bref, Binc, beta_t


def test_enhancement_objective_definition():
    """Sec. IV-B: the enhancement beta = |B + B_inc| / |B_ref| at each loss point; the
    weighted objective (weight 1/|B_ref|, offset B_inc, target beta_t) equals the mean of
    (beta - beta_t)^2 computed here from the oracle's own field B."""
    H, M, R, C, omega, V, li, _ = _grad_case(0)
    F = len(omega)
    Bref, Binc, bt = _beta_inputs(H, li, F)
    out = oracle.forward(H, M, R, C, omega, V, li, bt, weight=1 / np.abs(Bref), offset=Binc)
    B = out["B"][:, :, li]  # [n_cfg, F, L]
    beta = np.abs(B + Binc[None]) / np.abs(Bref)[None]
    want = ((beta - bt[None]) ** 2).mean(axis=(1, 2))
    assert _rel(out["loss"], want) < 1e-13
    # weight 1 and offset 0 reproduce the plain objective
    plain = oracle.forward(H, M, R, C, omega, V, li, bt * 1e-7)["loss"]
    same = oracle.forward(H, M, R, C, omega, V, li, bt * 1e-7, weight=np.ones((F, len(li))),
                          offset=np.zeros((F, len(li)), complex))["loss"]
    assert np.array_equal(plain, same)


@pytest.mark.parametrize("mode", [0, 1])
def test_enhancement_gradient_central_differences(mode):
    """The adjoint gradient of the weighted, offset objective against central differences."""
    H, M, R, C, omega, V, li, t = _grad_case(mode)
    F = len(omega)
    Bref, Binc, bt = _beta_inputs(H, li, F)
    w = 1 / np.abs(Bref)
    tt = bt if mode == 0 else np.stack([bt, -bt], axis=-1)
    g = oracle.gradient(H, M, R, C, omega, V, li, tt, mode=mode, weight=w, offset=Binc)

    def cd(h):
        fd = np.zeros_like(g)
        for k in range(C.shape[1]):
            Cp, Cm = C.copy(), C.copy()
            Cp[:, k] += h
            Cm[:, k] -= h
            kw = dict(mode=mode, want_B=False, weight=w, offset=Binc)
            fd[:, k] = (oracle.forward(H, M, R, Cp, omega, V, li, tt, **kw)["loss"]
                        - oracle.forward(H, M, R, Cm, omega, V, li, tt, **kw)["loss"]) / (2 * h)
        return fd
    f1, f2 = cd(1e-15), cd(0.5e-15)  # Richardson, as in test_gradient_central_differences
    assert _rel(g, (4 * f2 - f1) / 3) < 1e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_central_differences(mode):
    """Adjoint gradient versus central differences of the oracle loss, h = 1e-3 pF."""
    H, M, R, C, omega, V, li, t = _grad_case(mode)
    g = oracle.gradient(H, M, R, C, omega, V, li, t, mode=mode)
    def cd(h):
        fd = np.zeros_like(g)
        for k in range(C.shape[1]):
            Cp, Cm = C.copy(), C.copy()
            Cp[:, k] += h
            Cm[:, k] -= h
            lp = oracle.forward(H, M, R, Cp, omega, V, li, t, mode=mode, want_B=False)["loss"]
            lm = oracle.forward(H, M, R, Cm, omega, V, li, t, mode=mode, want_B=False)["loss"]
            fd[:, k] = (lp - lm) / (2 * h)
        return fd
    # Richardson extrapolation of central differences at h = 1e-3 pF and h/2 (O(h^4));
    # plain central differences carry O((h Q/C)^2) ~ 1e-5 near a resonance.
    f1, f2 = cd(1e-15), cd(0.5e-15)
    assert _rel(g, (4 * f2 - f1) / 3) < 1e-6


def test_gradient_adjoint_equals_direct():
    """The adjoint form equals the direct form built from dI/dC (one solve per capacitor)
    and the chain rule through |B| at the loss points."""
    H, M, R, C, omega, V, li, t = _grad_case(0, n_cfg=1)
    g = oracle.gradient(H, M, R, C, omega, V, li, t)
    out = oracle.forward(H, M, R, C, omega, V, li, t)
    F, L = len(omega), len(li)
    gd = np.zeros(C.shape[1])
    for f in range(F):
        _, dI = oracle.dcurrents_dC(M, R, omega[f], C[0], V[f])
        b = H[li] @ out["I"][0, f]
        dldb = 2 * (np.abs(b) - t[f]) / np.abs(b)  # d/d(b) of (|b|-t)^2 along b/|b|
        for k in range(C.shape[1]):
            db = H[li] @ dI[k]
            gd[k] += np.sum(dldb * np.real(np.conj(b) * db))
    gd /= F * L
    assert _rel(g[0], gd) < 1e-10


def test_single_loop_gradient_closed_form():
    """N = 1: I = V/(R + jwL + 1/(jwC)), dI/dC = -(I^2/V) j/(w C^2); with one loss point
    b = h I the loss (|b| - t)^2 has an exact derivative."""
    L, R, C, w, h, t = 250.79e-9, 0.1, 30e-12, 2 * np.pi * 63.6e6, 2e-5, 1e-7
    V = np.array([[-1j * w * 1e-6 * 7.8e-3]])
    H = np.array([[h]])
    I_ = V[0, 0] / (R + 1j * w * L + 1 / (1j * w * C))
    dI = -(I_ ** 2 / V[0, 0]) * 1j / (w * C * C)
    b, db = h * I_, h * dI
    want = 2 * (abs(b) - t) * np.real(np.conj(b) * db) / abs(b)
    g = oracle.gradient(H, np.array([[L]]), [R], [[C]], [w], V, [0], np.array([[t]]))
    assert abs(g[0, 0] / want - 1) < 1e-12


def test_loss_zero_at_own_field():
    """Targets equal to |B| at the same C give zero loss and zero gradient."""
    H, M, R, C, omega, V, li, _ = _grad_case(0, n_cfg=1)
    out = oracle.forward(H, M, R, C, omega, V, li, np.zeros((len(omega), len(li))))
    t = np.abs(out["B"][0][:, li])
    o2 = oracle.forward(H, M, R, C, omega, V, li, t)
    assert o2["loss"][0] < 1e-40
    g = oracle.gradient(H, M, R, C, omega, V, li, t)
    g_ref = oracle.gradient(H, M, R, C, omega, V, li, 0.5 * t)
    assert np.abs(g).max() < 1e-12 * np.abs(g_ref).max()


def test_gradient_field_cotangent_fd():
    """Field cotangent path: for L = Re(sum conj(gB) B), dL/dC by central differences."""
    H, M, R, C, omega, V, li, _ = _grad_case(0, n_cfg=2, F=2)
    gB = W.random_cotangent((2, 2, H.shape[0]), seed=4) * 1e5
    g = oracle.gradient_field(H, M, R, C, omega, V, gB)
    def cd(h):
        fd = np.zeros_like(g)
        for k in range(C.shape[1]):
            Cp, Cm = C.copy(), C.copy()
            Cp[:, k] += h
            Cm[:, k] -= h
            Bp = oracle.forward(H, M, R, Cp, omega, V, want_loss=False)["B"]
            Bm = oracle.forward(H, M, R, Cm, omega, V, want_loss=False)["B"]
            fd[:, k] = np.real(np.sum(np.conj(gB) * (Bp - Bm), axis=(1, 2))) / (2 * h)
        return fd
    f1, f2 = cd(1e-15), cd(0.5e-15)
    assert _rel(g, (4 * f2 - f1) / 3) < 1e-6


def test_forward_threads_do_not_change_bits():
    """Configurations are independent: the oracle gives the same bits for a batch and for
    each configuration alone."""
    H, M, R, C, omega, V, li, t = _grad_case(0, n_cfg=5)
    out = oracle.forward(H, M, R, C, omega, V, li, t)
    for b in range(5):
        o1 = oracle.forward(H, M, R, C[b:b + 1], omega, V, li, t)
        assert np.array_equal(o1["B"][0], out["B"][b]) and o1["loss"][0] == out["loss"][b]


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_rl_central_differences(mode):
    """dloss/dR_k and dloss/dL_k (L_k = M_kk) from the adjoint versus Richardson-extrapolated
    central differences of the oracle loss in R_k and M_kk."""
    H, M, R, C, omega, V, li, t = _grad_case(mode)
    gR, gL = oracle.gradient_rl(H, M, R, C, omega, V, li, t, mode=mode)
    N = C.shape[1]

    def cd_R(h):
        fd = np.zeros_like(gR)
        for k in range(N):
            Rp, Rm = np.array(R, float), np.array(R, float)
            Rp[k] += h
            Rm[k] -= h
            lp = oracle.forward(H, M, Rp, C, omega, V, li, t, mode=mode, want_B=False)["loss"]
            lm = oracle.forward(H, M, Rm, C, omega, V, li, t, mode=mode, want_B=False)["loss"]
            fd[:, k] = (lp - lm) / (2 * h)
        return fd

    def cd_L(h):
        fd = np.zeros_like(gL)
        for k in range(N):
            Mp, Mm = M.copy(), M.copy()
            Mp[k, k] += h
            Mm[k, k] -= h
            lp = oracle.forward(H, Mp, R, C, omega, V, li, t, mode=mode, want_B=False)["loss"]
            lm = oracle.forward(H, Mm, R, C, omega, V, li, t, mode=mode, want_B=False)["loss"]
            fd[:, k] = (lp - lm) / (2 * h)
        return fd

    r1, r2 = cd_R(1e-4), cd_R(0.5e-4)      # R ~ 0.1 ohm
    l1, l2 = cd_L(1e-12), cd_L(0.5e-12)    # L ~ 1e-7 H
    assert _rel(gR, (4 * r2 - r1) / 3) < 1e-6
    assert _rel(gL, (4 * l2 - l1) / 3) < 1e-6


def test_gradient_rl_single_loop_closed_form():
    """N = 1: dI/dR = -I^2/V and dI/dL = -j w I^2/V, chained through (|b| - t)^2, b = h I."""
    L, R, C, w, h, t = 250.79e-9, 0.1, 30e-12, 2 * np.pi * 63.6e6, 2e-5, 1e-7
    V = np.array([[-1j * w * 1e-6 * 7.8e-3]])
    I_ = V[0, 0] / (R + 1j * w * L + 1 / (1j * w * C))
    b = h * I_
    def d(db):
        return 2 * (abs(b) - t) * np.real(np.conj(b) * db) / abs(b)
    wantR = d(h * (-(I_ ** 2) / V[0, 0]))
    wantL = d(h * (-1j * w * I_ ** 2 / V[0, 0]))
    gR, gL = oracle.gradient_rl(np.array([[h]]), np.array([[L]]), [R], [[C]], [w], V, [0], np.array([[t]]))
    assert abs(gR[0, 0] / wantR - 1) < 1e-12
    assert abs(gL[0, 0] / wantL - 1) < 1e-12



# ---------------------------------------------------------------- oblique segment pairs
def test_gauss_legendre_rule():
    """The n-point rule integrates polynomials of degree 2n - 1 exactly and no higher."""
    for n in (1, 2, 5, 16, 32):
        x, w = oracle.gauss_legendre(n)
        for deg in range(0, 2 * n, 1):
            exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
            assert abs((w * x ** deg).sum() - exact) < 1e-13
        if n <= 5:  # the error term for x^(2n) is visible at low orders
            assert abs((w * x ** (2 * n)).sum() - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("d", [0.01, 0.03, 0.2])
@pytest.mark.parametrize("shift", [0.0, 0.02, -0.07])
def test_quadrature_matches_parallel_closed_form(d, shift):
    """For parallel filaments the quadrature reproduces the closed form (textbook G)."""
    l1, l2 = 0.05, 0.03
    a0, a1 = (0, 0, 0), (l1, 0, 0)
    b0, b1 = (shift, d, 0.004), (shift + l2, d, 0.004)
    st, exact = oracle.segment_pair_inductance(a0, a1, b0, b1, 1e-3)
    assert st == 0
    q = oracle.segment_pair_quadrature(a0, a1, b0, b1, 16)
    assert abs(q / exact - 1) < 1e-10
    # reversed second filament: sign flips
    assert abs(oracle.segment_pair_quadrature(a0, a1, b1, b0, 16) + q) < 1e-12 * abs(q)


def test_quadrature_symmetric_and_converged_for_skew_pairs():
    """A skew pair: M(a, b) = M(b, a) (outer and inner integrals swap roles), order 16 agrees
    with order 64, perpendicular directions give zero, and the pair the inductance routine
    now accepts equals the quadrature."""
    a0, a1 = np.array([0.0, 0.0, 0.0]), np.array([0.04, 0.01, 0.0])
    b0, b1 = np.array([0.01, 0.03, 0.005]), np.array([0.05, 0.02, 0.02])
    m_ab = oracle.segment_pair_quadrature(a0, a1, b0, b1, 16)
    m_ba = oracle.segment_pair_quadrature(b0, b1, a0, a1, 16)
    m64 = oracle.segment_pair_quadrature(a0, a1, b0, b1, 64)
    assert abs(m_ab / m_ba - 1) < 1e-12 and abs(m_ab / m64 - 1) < 1e-12
    st, m = oracle.segment_pair_inductance(a0, a1, b0, b1, 1e-3)
    assert st == 0 and m == m_ab
    assert oracle.segment_pair_quadrature(a0, a1, b0, b0 + np.array([0.0, 0.0, 0.03]), 16) == 0.0


def test_coaxial_circles_maxwell():
    """Mutual inductance of two coaxial circular loops (radii a, b, axial distance h) from
    polygons of n and 2n segments, Richardson-extrapolated in 1/n^2, against Maxwell's
    formula M = mu0 sqrt(ab) ((2/k - k) K(k) - (2/k) E(k)), k^2 = 4ab/((a+b)^2 + h^2)."""
    sp = pytest.importorskip("scipy.special")
    a, b, h = 0.05, 0.03, 0.02
    k2 = 4 * a * b / ((a + b) ** 2 + h * h)
    k = np.sqrt(k2)
    exact = MU0 * np.sqrt(a * b) * ((2 / k - k) * sp.ellipk(k2) - (2 / k) * sp.ellipe(k2))

    def polygon_pair(n):
        loops = [W.circular_loop(a, n), W.circular_loop(b, n, z=h)]
        off, vx, vy, vz = _loop_arrays(loops)
        st, M = oracle.inductance(off, vx, vy, vz, 1e-3, L_self=np.array([1.0, 1.0]))
        assert st == 0
        return M[0, 1]

    m1, m2 = polygon_pair(128), polygon_pair(256)
    assert abs(m2 / exact - 1) < 1e-3
    assert abs((4 * m2 - m1) / 3 / exact - 1) < 1e-6



@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_omega_and_drive_central_differences(mode):
    """dloss/dw_f (V held fixed) and the cotangent of V (dL/dRe V + j dL/dIm V) from the
    adjoint versus Richardson-extrapolated central differences of the oracle loss."""
    H, M, R, C, omega, V, li, t = _grad_case(mode)
    gw, gV = oracle.gradient_omega_v(H, M, R, C, omega, V, li, t, mode=mode)
    F, N = len(omega), C.shape[1]

    def loss(om, VV):
        return oracle.forward(H, M, R, C, om, VV, li, t, mode=mode, want_B=False)["loss"]

    def cd_w(h):
        fd = np.zeros_like(gw)
        for f in range(F):
            op, om = np.array(omega, float), np.array(omega, float)
            op[f] += h
            om[f] -= h
            fd[:, f] = (loss(op, V) - loss(om, V)) / (2 * h)
        return fd

    w1, w2 = cd_w(1e2), cd_w(0.5e2)  # w ~ 4e8 rad/s
    assert _rel(gw, (4 * w2 - w1) / 3) < 1e-6
    V = np.asarray(V)
    scale = np.abs(V).max()
    for f, k in ((0, 0), (F - 1, N - 1), (1, 3)):
        for part in (1.0, 1j):
            h = 1e-6 * scale
            Vp, Vm = V.copy(), V.copy()
            Vp[f, k] += part * h
            Vm[f, k] -= part * h
            fd = (loss(omega, Vp) - loss(omega, Vm)) / (2 * h)
            want = gV[:, f, k].real if part == 1.0 else gV[:, f, k].imag
            assert _rel(want, fd) < 1e-6


# ---------------------------------------------------------------- in-plane field components
@pytest.mark.parametrize("rho,zp", [(0.02, 0.01), (0.049, 0.003), (0.08, -0.02)])
def test_circle_radial_field_elliptic(rho, zp):
    """Radial field of a circular loop (complete elliptic integrals, scipy's K, E):
    B_rho = mu0 z / (2 pi rho sqrt((a+rho)^2+z^2)) [-K + (a^2+rho^2+z^2)/((a-rho)^2+z^2) E];
    at azimuth phi, Bx = B_rho cos(phi), By = B_rho sin(phi)."""
    from scipy.special import ellipe, ellipk
    a = 0.05
    m = 4 * a * rho / ((a + rho) ** 2 + zp ** 2)
    brho = MU0 * zp / (2 * np.pi * rho * np.sqrt((a + rho) ** 2 + zp ** 2)) * (
        -ellipk(m) + (a * a + rho * rho + zp * zp) / ((a - rho) ** 2 + zp ** 2) * ellipe(m))
    off, vx, vy, vz = _loop_arrays([W.circular_loop(a, 8192)])
    for phi in (0.0, 0.7):
        px, py = [rho * np.cos(phi)] * 2, [rho * np.sin(phi)] * 2
        H = oracle.basis(off, vx, vy, vz, px, py, [zp] * 2, 1e-4, comp=[1, 2])
        assert abs(H[0, 0] - brho * np.cos(phi)) < 2e-5 * abs(brho) + 1e-15
        assert abs(H[1, 0] - brho * np.sin(phi)) < 2e-5 * abs(brho) + 1e-15


def test_components_of_a_wire_and_on_axis():
    """A long straight side (current along +x) of a huge rectangle: at (0, 0, d) the field
    is -mu0 I/(2 pi d) along y (right-hand rule), with no x or z component; on the axis of
    a square loop the in-plane components vanish."""
    L, D, d = 1e3, 1e3, 0.01
    vx = np.array([-L, L, L, -L])
    vy = np.array([0.0, 0.0, D, D])
    vz = np.zeros(4)
    H = oracle.basis(np.array([0, 4], np.int32), vx, vy, vz, [0.0] * 3, [0.0] * 3, [d] * 3, 1e-3,
                     comp=[1, 2, 0])[:, 0]
    want = -MU0 / (2 * np.pi * d)
    assert abs(H[1] / want - 1) < 1e-4          # far sides contribute ~d/L
    assert abs(H[0]) < 1e-12 * abs(want) and abs(H[2]) < 1e-4 * abs(want)
    off, vx, vy, vz = _loop_arrays([W.square_loop(0.05, 16)])
    H = oracle.basis(off, vx, vy, vz, [0.0] * 2, [0.0] * 2, [0.02] * 2, 1e-3, comp=[1, 2])
    assert np.all(np.abs(H) < 1e-20)


def test_square_loop_quarter_turn_maps_components():
    """A square loop centred at the origin is invariant under a quarter turn about z, so
    B(R p) = R B(p): Bx(Rp) = -By(p), By(Rp) = Bx(p), Bz(Rp) = Bz(p)."""
    off, vx, vy, vz = _loop_arrays([W.square_loop(0.05, 16)])
    p = np.array([0.013, -0.021, 0.017])
    q = np.array([-p[1], p[0], p[2]])  # R p
    Hp = oracle.basis(off, vx, vy, vz, [p[0]] * 3, [p[1]] * 3, [p[2]] * 3, 1e-3, comp=[1, 2, 0])[:, 0]
    Hq = oracle.basis(off, vx, vy, vz, [q[0]] * 3, [q[1]] * 3, [q[2]] * 3, 1e-3, comp=[1, 2, 0])[:, 0]
    assert abs(Hq[0] + Hp[1]) < 1e-12 * np.abs(Hp).max()
    assert abs(Hq[1] - Hp[0]) < 1e-12 * np.abs(Hp).max()
    assert abs(Hq[2] - Hp[2]) < 1e-12 * np.abs(Hp).max()
