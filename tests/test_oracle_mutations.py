"""Planted mistakes in a copy of the oracle source must fail at least one pin.

Each mutation is a plausible slip (a wrong sign, a dropped factor, a transposed
operand, the wrong operator or inner product).  The mutant is compiled from a
temporary copy on the CPU; the committed oracle is never modified.
"""

import os
import subprocess
import tempfile

import pytest

import oracle
from tbsynth import config_c1

from . import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "marnoldi_oracle.c")

MUTATIONS = {
    "mgs_sign": ("wv[r] -= c * ki[r];", "wv[r] += c * ki[r];"),
    "euclidean_inner_product": ("double c = dot(m, ski, wv);", "double c = dot(m, ki, wv);"),
    "k1_not_S_normalised": ("K[j] = 1.0 / sqrt(sjj);", "K[j] = 1.0;"),
    "krylov_of_S": ("bsr_apply(nbr, rp, ci, Hv, kn, u);", "bsr_apply(nbr, rp, ci, Sv, kn, u);"),
    "Sk_not_updated": ("skn1[r] = Sw[r] / beta;", "skn1[r] = wv[r] / beta;"),
    "hsub_no_half": ("double s = 0.5 * (A[i * ne + l] + A[l * ne + i]);",
                     "double s = (A[i * ne + l] + A[l * ne + i]);"),
    "t_transposed_V": ("ta += V[i * ne + a] * K[(int64_t)i * m + j];",
                       "ta += V[a * ne + i] * K[(int64_t)i * m + j];"),
    "weight_wrong_row": ("w[a] = sqrt(sjj) * V[0 * ne + a] * ta;", "w[a] = sqrt(sjj) * V[a] * V[a];"),
    "weight_no_sqrt_sjj": ("w[a] = sqrt(sjj) * V[0 * ne + a] * ta;", "w[a] = V[0 * ne + a] * ta;"),
    "Y_transposed_V": ("s += K[(int64_t)i * m + r] * V[i * ne + a];",
                       "s += K[(int64_t)i * m + r] * V[a * ne + i];"),
    "jacobi_rotation_sign": ("A[r * n + p] = c * arp - s * arq;", "A[r * n + p] = c * arp + s * arq;"),
    "fermi_wrong_branch": ("return e / (1.0 + e);", "return 1.0 / (1.0 + e);"),
    "energy_drops_eps": ("se += f2 * eps[i] * w[i];", "se += f2 * w[i];"),
    "bisect_direction": ("if (N < Ne) lo = mu; else hi = mu;", "if (N > Ne) lo = mu; else hi = mu;"),
    "density_no_spin": ("double f2 = 2.0 * oracle_fermi((eps[c * nu + a] - mu) / kT);",
                        "double f2 = oracle_fermi((eps[c * nu + a] - mu) / kT);"),
    "rhoE_no_eps": ("ye[a] = f2 * eps[c * nu + a] * t[c * nu + a];", "ye[a] = f2 * t[c * nu + a];"),
}


def _pins(c1):
    return [
        lambda: pins.test_fermi_against_tanh_and_limits(),
        lambda: pins.test_jacobi_matches_lapack(40, 1),
        lambda: pins.test_p1_nu1_closed_form(c1),
        lambda: pins.test_p1_p3_p5_rescaled_orbitals(),
        lambda: pins.test_p3_dense_limit(8, 0),
        lambda: pins.test_p4_galerkin_and_s_orthonormality(3),
        lambda: pins.test_p5_weights_sum_to_one(c1),
        lambda: pins.test_p6_p7_pattern_traces(c1),
        lambda: pins.test_p8_lanczos_gauss_quadrature(),
        lambda: pins.test_p9_power_basis_brute_force_50_digits(),
        lambda: pins.test_p10_bisection(c1),
    ]


@pytest.fixture(scope="module")
def c1_sys():
    return config_c1(seed=0)


def test_unmutated_copy_passes(c1_sys, tmp_path):
    lib = tmp_path / "orig.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), SRC, "-lm"])
    with oracle.use_library(str(lib)):
        for p in _pins(c1_sys):
            p()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, c1_sys, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mutant = tmp_path / f"{name}.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                           str(mutant), "-lm"])
    caught = []
    with oracle.use_library(str(lib)):
        for i, p in enumerate(_pins(c1_sys)):
            try:
                p()
            except (AssertionError, RuntimeError, ValueError, FloatingPointError, KeyError):
                caught.append(i)
                break
    assert caught, f"no pin caught the planted mistake {name}"
