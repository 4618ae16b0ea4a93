"""The oracle's pins must catch plausible mistakes in the oracle itself. Each case plants one
mistake (a flipped sign, a dropped term, a transposed operand, a missing conjugate or factor)
in a copy of oracle/oracle.c under a temporary directory, builds that copy with gcc, and runs
the unchanged pin suite (tests/test_oracle_pins.py) against it in a subprocess: the suite
must fail. The control case plants nothing and must pass. The repository's oracle and the
CUDA path are not touched. CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# name: (text in oracle.c, replacement, occurrence to replace (0 = first), the mistake)
MUTANTS = {
    "control": (None, None, 0, "nothing planted"),
    "biot_savart_cross_sign": (
        "R1[0] * R2[1] - R1[1] * R2[0]}", "R1[1] * R2[0] - R1[0] * R2[1]}", 0,
        "z component of R1 x R2 with the wrong sign (Biot-Savart, Sec. I-A)"),
    "biot_savart_dropped_r2": (
        "f = (n1 + n2) / denom;", "f = n1 / denom;", 0,
        "|R2| dropped from the segment's field factor"),
    "component_xy_swapped": (
        "comp == 1 ? c[0] : (comp == 2 ? c[1] : c[2])", "comp == 1 ? c[1] : (comp == 2 ? c[0] : c[2])", 0,
        "Bx and By exchanged"),
    "neumann_g_sign": (
        "return u * asinh(u / d) - sqrt(u * u + d * d);", "return u * asinh(u / d) + sqrt(u * u + d * d);", 0,
        "sign of the square-root term of the parallel-filament Neumann integral (Eq. 12)"),
    "self_inductance_constant": (
        "(log(2.0 * l1 / rw) - 1.0)", "(log(2.0 * l1 / rw) - 0.75)", 0,
        "internal-inductance constant in a straight segment's self inductance"),
    "reactance_sign": (
        "A[i * n + i] += R[i] + 1.0 / (I * omega * C[i]);", "A[i * n + i] += R[i] - 1.0 / (I * omega * C[i]);", 0,
        "capacitor impedance +j/(wC) instead of 1/(jwC) (Eq. 2, 11)"),
    "lu_forward_transposed": (
        "for (int32_t j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];",
        "for (int32_t j = 0; j < i; ++j) b[i] -= LU[j * n + i] * b[j];", 0,
        "forward substitution reading the transposed factor"),
    "objective_mean_over_f_only": (
        "if (loss_out) loss_out[b] = (F * L > 0) ? acc / ((double)F * L) : 0.0;",
        "if (loss_out) loss_out[b] = (F * L > 0) ? acc / ((double)F) : 0.0;", 0,
        "objective averaged over frequencies but not loss points (Eq. 1)"),
    "objective_gradient_factor_two": (
        "*G = (a > 0.0) ? 2.0 * r * b / a : 0.0;", "*G = (a > 0.0) ? r * b / a : 0.0;", 0,
        "factor 2 of d(|b| - t)^2 dropped"),
    "enhancement_weight_not_in_cotangent": (
        "  *G *= w;\n", "  (void)w;\n", 0,
        "chain-rule factor of the enhancement weight 1/|B_ref| dropped (Sec. IV-B)"),
    "adjoint_no_conjugate_c": (
        "mu[k] += H[loss_idx[l] * N + k] * conj(G);", "mu[k] += H[loss_idx[l] * N + k] * G;", 0,
        "adjoint right-hand side without the conjugate (dloss/dC)"),
    "adjoint_no_conjugate_rl": (
        "mu[k] += H[loss_idx[l] * N + k] * conj(G);", "mu[k] += H[loss_idx[l] * N + k] * G;", 1,
        "adjoint right-hand side without the conjugate (dloss/dR, dloss/dL)"),
    "adjoint_no_conjugate_omega": (
        "mu[k] += H[loss_idx[l] * N + k] * conj(G);", "mu[k] += H[loss_idx[l] * N + k] * G;", 2,
        "adjoint right-hand side without the conjugate (dloss/dw, drive)"),
    "gradient_sign": (
        "grad_out[b * N + k] += cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);",
        "grad_out[b * N + k] -= cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);", 0,
        "dloss/dC with the wrong sign (Eq. 8-9)"),
    "sroute_operand_order": (
        "for (int32_t k = 0; k < n0; ++k) s += SC[i * n + k] * S0[k * n0 + j];",
        "for (int32_t k = 0; k < n0; ++k) s += S0[i * n0 + k] * SC[k * n + j];", 0,
        "1 - S0 S11 instead of 1 - S11 S0 (Eq. 6)"),
    "sroute_gradient_without_s0": (
        "if (cc < n0) col[r] = SW[cc * n1 + c];", "if (cc < n0) col[r] = W[cc * n1 + c];", 0,
        "S0 dropped from the Eq. 10 bracket"),
    "reflection_sign": (
        "(Zload[k] - Z0) / (Zload[k] + Z0); /* Eq. 3 */", "(Z0 - Zload[k]) / (Zload[k] + Z0); /* Eq. 3 */", 0,
        "reflection coefficient of a load with the wrong sign (Eq. 3)"),
    "reflection_derivative_factor": (
        "2.0 * Z0 / ((zl + Z0) * (zl + Z0))", "Z0 / ((zl + Z0) * (zl + Z0))", 0,
        "factor 2 of d Gamma / d Z dropped (Eq. 3 chain rule)"),
    "basis_polygon_open": (
        "int32_t w = (v + 1 < b) ? v + 1 : a;", "int32_t w = (v + 1 < b) ? v + 1 : v;", 0,
        "closing segment of a loop left out of its field"),
    "inductance_polygon_open": (
        "int32_t ie = (i + 1 < loop_vtx_off[k + 1]) ? i + 1 : loop_vtx_off[k];",
        "int32_t ie = (i + 1 < loop_vtx_off[k + 1]) ? i + 1 : i;", 0,
        "closing segment of a loop left out of its inductances"),
    "gauss_legendre_weight": (
        "w[i] = 2.0 / ((1.0 - z * z) * dp * dp);", "w[i] = 1.0 / ((1.0 - z * z) * dp * dp);", 0,
        "Gauss-Legendre weights off by a factor 2"),
    "oblique_direction_cosine_dropped": (
        "* cosang * 0.5 * (l1 / m) * acc", "* 0.5 * (l1 / m) * acc", 0,
        "u1.u2 dropped from the oblique Neumann integral"),
    "inner_integral_sign": (
        "return log((R1 + a) * (R0 + t0) / rho2);", "return log((R1 + a) * (R0 - t0) / rho2);", 0,
        "sign error in the rewritten inner integral of the oblique pair"),
    "dloss_dr_sign": (
        "gR[b * N + k] += -creal(mu[k] * x[k]);", "gR[b * N + k] += creal(mu[k] * x[k]);", 0,
        "dloss/dR with the wrong sign"),
    "dloss_dl_omega_dropped": (
        "gL[b * N + k] += omega[f] * cimag(mu[k] * x[k]);", "gL[b * N + k] += cimag(mu[k] * x[k]);", 0,
        "factor w of dA/dL dropped"),
    "dloss_domega_capacitor_term_dropped": (
        "gw[b * F + f] = (cimag(muMI) + diag) * nrm;", "gw[b * F + f] = cimag(muMI) * nrm;", 0,
        "capacitor term of dA/dw dropped"),
    "drive_cotangent_no_conjugate": (
        "gV[(b * F + f) * N + k] = conj(mu[k]) * nrm;", "gV[(b * F + f) * N + k] = mu[k] * nrm;", 0,
        "drive cotangent without the conjugate"),
    "enhancement_offset_sign": (
        "(offset ? b + offset[i] : b) * w", "(offset ? b - offset[i] : b) * w", 0,
        "incident field subtracted instead of added (Sec. IV-B)"),
    "drive_wave_amplitude": (
        "csqrt(Z0 * P_in)", "csqrt(P_in / Z0)", 0,
        "excitation wave sqrt(P / Z') instead of sqrt(Z' P) (Eq. 4)"),
    "touching_pair_factor_two": (
        "double F = 2.0 * (l * atanh(m / (l + R)) + m * atanh(l / (m + R)));",
        "double F = (l * atanh(m / (l + R)) + m * atanh(l / (m + R)));", 0,
        "factor 2 of the touching-filament Neumann integral dropped"),
    "touching_pair_far_end_swapped": (
        "*out = oracle_touching_pair(r1s, r1e, r2e, cosang);",
        "*out = oracle_touching_pair(r1s, r1e, r2s, cosang);", 0,
        "shared end point taken as a far end point of a touching pair"),
    "field_cotangent_gradient_sign": (
        "grad_out[b * N + k] += cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);",
        "grad_out[b * N + k] -= cimag(mu[k] * x[k]) / (omega[f] * Cb[k] * Cb[k]);", 1,
        "dloss/dC of a field cotangent with the wrong sign"),
}


def _plant(src: str, old, new, occurrence: int) -> str:
    if old is None:
        return src
    at = -1
    for _ in range(occurrence + 1):
        at = src.find(old, at + 1)
        assert at >= 0, f"mutation site not found (occurrence {occurrence}): {old!r}"
    return src[:at] + new + src[at + len(old):]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc builds the oracle")
@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_a_planted_mistake(name, tmp_path):
    old, new, occurrence, what = MUTANTS[name]
    src = open(os.path.join(ORACLE, "oracle.c")).read()
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    shutil.copy(os.path.join(ORACLE, "__init__.py"), pkg / "__init__.py")
    (pkg / "oracle.c").write_text(_plant(src, old, new, occurrence))
    # run from the temporary directory so that `import oracle` resolves to the copy; the
    # repository root stays importable for the workload generators
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider", "--rootdir", ROOT,
                        "-c", os.path.join(ROOT, "pytest.ini")],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    summary = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-2000:]
    # the copy builds its own library on import: proof that the suite ran against it
    assert (pkg / "liboracle.so").exists(), f"the pin suite did not load the copy:\n{summary}"
    if old is None:
        assert r.returncode == 0, f"the unmodified copy must pass the pins:\n{r.stdout[-3000:]}"
    else:
        assert r.returncode == 1 and " failed" in summary and "error" not in summary, (
            f"planted mistake not caught by the pins ({what}):\n{summary}")
