"""Planted mistakes in the oracle must each fail at least one pin (CPU only).

Every mutant is a one-token change to a copy of oracle/ebv_oracle.c (a dropped
term, a wrong sign, a shifted or transposed index, a window one short), compiled with gcc into a
temporary library and run against the pins.
"""
import os

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "ebv_oracle.c")

MUTANTS = {
    "update_sign": ("a[IDX(i, j, lda)] -= lik * a[IDX(k, j, lda)];",
                    "a[IDX(i, j, lda)] += lik * a[IDX(k, j, lda)];"),
    "pivot_multiply": ("const double lik = a[IDX(i, k, lda)] / p;",
                       "const double lik = a[IDX(i, k, lda)] * p;"),
    "update_skips_last_col": ("for (int64_t j = k + 1; j < n; ++j) /* Eq. 6c",
                              "for (int64_t j = k + 1; j < n - 1; ++j) /* Eq. 6c"),
    "forward_drops_term": ("for (int64_t j = 0; j < i; ++j) s -= lu[IDX(i, j, lda)] * b[IDX(j, c, ldb)];",
                           "for (int64_t j = 1; j < i; ++j) s -= lu[IDX(i, j, lda)] * b[IDX(j, c, ldb)];"),
    "backward_transposed": ("for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(i, j, lda)] * b[IDX(j, c, ldb)];",
                            "for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(j, i, lda)] * b[IDX(j, c, ldb)];"),
    "backward_no_divide": ("b[IDX(i, c, ldb)] = s / lu[IDX(i, i, lda)];",
                           "b[IDX(i, c, ldb)] = s;"),
    "band_short_update": ("const int64_t jend = (k + ku < n - 1) ? k + ku : n - 1;",
                          "const int64_t jend = (k + ku - 1 < n - 1) ? k + ku - 1 : n - 1;"),
    "band_short_rows": ("const int64_t iend = (k + kl < n - 1) ? k + kl : n - 1;",
                        "const int64_t iend = (k + kl - 1 < n - 1) ? k + kl - 1 : n - 1;"),
    "band_forward_window": ("const int64_t j0 = (i - kl > 0) ? i - kl : 0;\n      for (int64_t j = j0; j < i; ++j) s -= AB(i, j)",
                            "const int64_t j0 = (i - kl + 1 > 0) ? i - kl + 1 : 0;\n      for (int64_t j = j0; j < i; ++j) s -= AB(i, j)"),
    "adjoint_untransposed_U": ("for (int64_t j = 0; j < i; ++j) s -= lu[IDX(j, i, lda)] * grad_b[IDX(j, c, ldx)];",
                               "for (int64_t j = 0; j < i; ++j) s -= lu[IDX(i, j, lda)] * grad_b[IDX(j, c, ldx)];"),
    "adjoint_untransposed_L": ("for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(j, i, lda)] * grad_b[IDX(j, c, ldx)];",
                               "for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(i, j, lda)] * grad_b[IDX(j, c, ldx)];"),
    "adjoint_grad_a_sign": ("grad_a[IDX(i, j, ldga)] = -s;", "grad_a[IDX(i, j, ldga)] = s;"),
    "adjoint_grad_a_transposed": ("s += grad_b[IDX(i, c, ldx)] * x[IDX(j, c, ldx)];",
                                  "s += grad_b[IDX(j, c, ldx)] * x[IDX(i, c, ldx)];"),
    "band_pivot_multiply": ("const double lik = AB(i, k) / p;", "const double lik = AB(i, k) * p;"),
    "band_update_sign": ("for (int64_t j = k + 1; j <= jend; ++j) AB(i, j) -= lik * AB(k, j);",
                         "for (int64_t j = k + 1; j <= jend; ++j) AB(i, j) += lik * AB(k, j);"),
    "band_update_transposed": ("for (int64_t j = k + 1; j <= jend; ++j) AB(i, j) -= lik * AB(k, j);",
                               "for (int64_t j = k + 1; j <= jend; ++j) AB(i, j) -= lik * AB(j, k);"),
    "band_info_off_by_one": ("if (info == 0 && (p == 0.0 || !isfinite(p))) info = k + 1;\n    const int64_t iend",
                             "if (info == 0 && (p == 0.0 || !isfinite(p))) info = k;\n    const int64_t iend"),
    "band_backward_window": ("const int64_t j1 = (i + ku < n - 1) ? i + ku : n - 1;\n      for (int64_t j = i + 1; j <= j1; ++j) s -= AB(i, j)",
                             "const int64_t j1 = (i + ku - 1 < n - 1) ? i + ku - 1 : n - 1;\n      for (int64_t j = i + 1; j <= j1; ++j) s -= AB(i, j)"),
    "band_backward_no_divide": ("b[IDX(i, c, ldb)] = s / AB(i, i);", "b[IDX(i, c, ldb)] = s;"),
    "band_residual_window": ("for (int64_t j = j0; j <= j1; ++j) {\n        const double aij",
                             "for (int64_t j = j0; j < j1; ++j) {\n        const double aij"),
    "band_residual_drops_product_error": ("comp += pe + se;\n      }\n      r[IDX(i, c, ldr)]",
                                          "comp += se;\n      }\n      r[IDX(i, c, ldr)]"),
    "residual_drops_product_error": ("comp += pe + se;\n      }\n      r[IDX(t, c, ldr)]",
                                     "comp += se;\n      }\n      r[IDX(t, c, ldr)]"),
    "inverse_gauss_sign": ("for (int64_t j = 0; j < n; ++j) x[IDX(i, j, ldx)] -= lik * x[IDX(k, j, ldx)];",
                           "for (int64_t j = 0; j < n; ++j) x[IDX(i, j, ldx)] += lik * x[IDX(k, j, ldx)];"),
    "inverse_scales_by_pivot": ("x[IDX(k, j, ldx)] /= lu[IDX(k, k, lda)];", "x[IDX(k, j, ldx)] *= lu[IDX(k, k, lda)];"),
    "inverse_upper_transposed": ("s -= (lu[IDX(k, q, lda)] / lu[IDX(k, k, lda)]) * x[IDX(q, j, ldx)];",
                                 "s -= (lu[IDX(q, k, lda)] / lu[IDX(k, k, lda)]) * x[IDX(q, j, ldx)];"),
    "inverse_short_upper_sweep": ("for (int64_t q = k + 1; q < n; ++q) s -=",
                                  "for (int64_t q = k + 1; q < n - 1; ++q) s -="),
    "inverse_wrong_gauss_order": ("for (int64_t k = 0; k < n; ++k) { /* M_k",
                                  "for (int64_t k = n - 1; k >= 0; --k) { /* M_k"),
    "info_off_by_one": ("if (info == 0 && (p == 0.0 || !isfinite(p))) info = k + 1;\n#ifdef _OPENMP\n#pragma omp parallel for schedule(static) if (n - k > 128)",
                        "if (info == 0 && (p == 0.0 || !isfinite(p))) info = k;\n#ifdef _OPENMP\n#pragma omp parallel for schedule(static) if (n - k > 128)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mut_src = tmp_path / "mutant.c"
    mut_src.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    import subprocess
    r = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                        str(mut_src), "-o", so, "-lm"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = oracle.load(so)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
