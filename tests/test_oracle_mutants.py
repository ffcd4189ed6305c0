"""Plants plausible mistakes in a copy of the oracle (CPU only) and checks that the pin suite
fails on every one of them: a dropped term, a wrong sign, a wrong index or a transposed operand
anywhere in the oracle must not survive the pins."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pfsm_oracle.c")

MUTANTS = {
    "fs_shift_sign": ("y[i] = acc - eps[k] * x[i];", "y[i] = acc + eps[k] * x[i];"),
    "fs_second_product_uses_x": ("for (int64_t j = 0; j < n; j++) acc += A[i * n + j] * y[j];",
                                 "for (int64_t j = 0; j < n; j++) acc += A[i * n + j] * x[j];"),
    "fs_update_sign": ("x[i] -= alpha[k] * z[i];", "x[i] += alpha[k] * z[i];"),
    "mgs_no_normalise": ("for (int64_t i = 0; i < n; i++) qk[i] /= r;", ";"),
    "householder_drops_term": ("-= v[i] * p[j] + p[i] * v[j];", "-= v[i] * p[j];"),
    "qr_offdiag_sign": ("e[k] = c * s * (dk1 - dk) + (c * c - s * s) * f;",
                        "e[k] = c * s * (dk1 - dk) + (c * c + s * s) * f;"),
    "qr_accumulate_sign": ("q[row * n + k + 1] = -s * qk + c * qk1;",
                           "q[row * n + k + 1] = s * qk + c * qk1;"),
    "sort_descending": ("while (j >= 0 && d[ord[j]] > d[t])", "while (j >= 0 && d[ord[j]] < d[t])"),
    "select_slice_position": ("int64_t col = k - s[b];", "int64_t col = k - k0[b];"),
    "window_no_left_halo": ("int64_t lo = (int64_t)k0[b] - h;", "int64_t lo = (int64_t)k0[b];"),
    "alpha_not_squared": ("double a = prm->alpha_theta / (dmax * dmax);",
                          "double a = prm->alpha_theta / dmax;"),
    "gershgorin_counts_diagonal": ("if (j != i) r += fabs(a);", "r += fabs(a);"),
    "rayleigh_residual_drops_lambda": ("double t = wv[i] - l * q[i];", "double t = wv[i] - q[i];"),
    "snap_up_before_down": (
        "if (dn >= 1 && prev[dn] - prev[dn - 1] >= cluster_tol) { k0[b] = dn; break; }\n"
        "            if (up <= n - 1 && prev[up] - prev[up - 1] >= cluster_tol) { k0[b] = up; break; }",
        "if (up <= n - 1 && prev[up] - prev[up - 1] >= cluster_tol) { k0[b] = up; break; }\n"
        "            if (dn >= 1 && prev[dn] - prev[dn - 1] >= cluster_tol) { k0[b] = dn; break; }"),
    "backward_gap_sign": ("g = (fabs(gap) >= tau) ? acc / gap : 0.0;",
                          "g = (fabs(gap) >= tau) ? -acc / gap : 0.0;"),
    "backward_transposed_operand": ("acc += V[r * n + i] * dV[r * n + j];",
                                    "acc += V[i * n + r] * dV[r * n + j];"),
    "sign_rule_dropped": ("flip = (yh < 0.0) ? -1.0 : 1.0;", "flip = 1.0;"),
    "jacobi_drops_dinv": ("Z[i * n + j] += R[i * n + j] / B[i * n + i];", "Z[i * n + j] += R[i * n + j];"),
    "jacobi_update_sign": ("Z[i * n + j] += R[i * n + j] / B[i * n + i];",
                           "Z[i * n + j] -= R[i * n + j] / B[i * n + i];"),
    "jacobi_transposed_product": ("for (int64_t k = 0; k < n; k++) acc += B[i * n + k] * Z[k * n + j];",
                                  "for (int64_t k = 0; k < n; k++) acc += B[k * n + i] * Z[j * n + k];"),
    "newton_schulz_sign": ("T[i * n + j] = 0.5 * (((i == j) ? 3.0 : 0.0) - P[i * n + j]);",
                           "T[i * n + j] = 0.5 * (((i == j) ? 3.0 : 0.0) + P[i * n + j]);"),
    "newton_schulz_no_rescale": ("for (int64_t i = 0; i < n * n; i++) S[i] = Q[i] * isc;",
                                 "for (int64_t i = 0; i < n * n; i++) S[i] = Q[i];"),
    "guard_l1_not_l2": ("if (j != i) s += A[i * n + j] * A[i * n + j];", "if (j != i) s += fabs(A[i * n + j]);"),
    "guard_counts_diagonal": ("if (j != i) s += A[i * n + j] * A[i * n + j];", "s += A[i * n + j] * A[i * n + j];"),
    "full_home_index_swapped": ("double flip, yh = Y[k * n + k];", "double flip, yh = Y[k * n + 0];"),
    "full_sign_rule_dropped": ("flip = (yh >= 0.0) ? 1.0 : -1.0;", "flip = 1.0;"),
    "adaptive_shift_sign": ("eps[k] += delta;", "eps[k] -= delta;"),
    "adaptive_no_y_correction": ("for (int64_t i = 0; i < n; i++) { yr[i] -= delta * xr[i]; yy += yr[i] * yr[i]; }",
                                 "for (int64_t i = 0; i < n; i++) { yy += yr[i] * yr[i]; }"),
    "adaptive_residual_unnormalised": ("r[k] = sqrt(yy / xx);", "r[k] = sqrt(yy);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, PFSM_ORACLE_LIB_OVERRIDE=str(lib), OMP_NUM_THREADS="4")
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert proc.returncode != 0, f"planted mistake {name} survived the pins:\n{proc.stdout[-2000:]}"
