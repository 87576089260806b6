"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
flipped sign, a dropped term, a transposed index, a wrong mask value or
normaliser), compiles it, swaps it in, and checks that at least one pin of
tests/test_oracle.py, tests/test_oracle_trials.py or tests/test_oracle_bands.py
fails.  CPU only; the committed oracle is untouched.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle as pins
from tests import test_oracle_bands as band_pins
from tests import test_oracle_trials as trial_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "plv_oracle.c")

MUTATIONS = {
    "dft_sign": ("tws[m] = -sin(a);", "tws[m] = sin(a);"),
    "mask_two": ("return (k < T / 2) ? 2.0 : 0.0;",
                 "return (k < T / 2) ? 1.0 : 0.0;"),
    "inverse_scale": ("z_re[r * T + t] = sr / (double)T;",
                      "z_re[r * T + t] = sr;"),
    "inverse_dropped_term": ("sr += Xr[k] * c - Xi[k] * s;",
                             "sr += Xr[k] * c;"),
    "pair_transposed": ("double d = pi[t] - pj[t];",
                        "double d = pj[t] - pi[t];"),
    "mean_normaliser": ("double cr = sr / (double)T, ci = si / (double)T;",
                        "double cr = sr / (double)(T + 1), "
                        "ci = si / (double)(T + 1);"),
    "ciplv_denominator": ("double d = (1.0 - cr) * (1.0 + cr);",
                          "double d = (1.0 - cr);"),
    "zero_phase_kept": ("if (!(hi[t] && hj[t])) continue;", ""),
    # functions over trials
    "trial_normaliser": ("const double cr = sr / (double)E, ci = si / (double)E;",
                         "const double cr = sr / (double)T, ci = si / (double)T;"),
    "trial_index_swapped": ("const double d = atan2(z_im[qi], z_re[qi]) - atan2(z_im[qj], z_re[qj]);",
                            "const double d = atan2(z_im[qj], z_re[qj]) - atan2(z_im[qi], z_re[qi]);"),
    "bins_offset_dropped": ("const long k = (f0 + f) % T;", "const long k = f % T;"),
    "bins_sign": ("tws[m] = -sin(2.0 * M_PI * (double)m / (double)T);",
                  "tws[m] = sin(2.0 * M_PI * (double)m / (double)T);"),
    "coh_denominator": ("const double den = sqrt(pii * pjj);",
                        "const double den = sqrt(pii * pii);"),
    "band_mask_ignored": ("double h = hmask(k, T) * (band ? band[k] : 1.0);",
                          "double h = hmask(k, T);"),
    "coh_conjugate": ("si += x_im[qi] * x_re[qj] - x_re[qi] * x_im[qj];",
                      "si += x_im[qi] * x_re[qj] + x_re[qi] * x_im[qj];"),
    # the analytic mask and the inverse transform
    "nyquist_weight": ("if (k == T / 2) return 1.0;", "if (k == T / 2) return 2.0;"),
    "odd_last_bin_dropped": ("return (k <= (T - 1) / 2) ? 2.0 : 0.0;",
                             "return (k < (T - 1) / 2) ? 2.0 : 0.0;"),
    "inverse_twiddle_sign": ("double c = twc[idx], s = -tws[idx];",
                             "double c = twc[idx], s = tws[idx];"),
    "iplv_signed": ("*iplv = fabs(ci);", "*iplv = ci;"),
}

PIN_CALLS = [
    lambda: pins.test_analytic_matches_scipy_hilbert(64),
    lambda: pins.test_analytic_matches_scipy_hilbert(17),
    lambda: pins.test_analytic_on_bin_tone(64, 5),
    pins.test_analytic_dc_and_nyquist_map_to_themselves,
    pins.test_analytic_real_part_is_input,
    pins.test_pairwise_equals_reformulated_gram,
    pins.test_pairwise_equals_numpy_matmul_of_phasors,
    pins.test_lagged_tones_golden,
    pins.test_metrics_closed_forms,
    pins.test_zero_row_contributes_nothing,
    pins.test_rayleigh_null_mean,
    trial_pins.test_time_resolved_equals_reformulated_gram_per_sample,
    trial_pins.test_time_resolved_tones_closed_form,
    trial_pins.test_time_resolved_rayleigh_null,
    trial_pins.test_dft_bins_equals_numpy_fft,
    trial_pins.test_coherency_of_unit_phasors_is_plv_over_trials,
    trial_pins.test_coherency_closed_form_of_a_scaled_copy,
    trial_pins.test_coherency_invariances_and_bounds,
    band_pins.test_band_selects_one_on_bin_tone,
    band_pins.test_band_is_linear_in_the_mask,
]


def _build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"mut_{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    str(path), "-o", str(so), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(tmp_path, name):
    so = _build_mutant(tmp_path, name)
    good = oracle._load()
    mut = ctypes.CDLL(so)
    for f in ("oracle_analytic", "oracle_plv_pairwise_rows",
              "oracle_plv_pairwise", "oracle_gram_direct", "oracle_metrics",
              "oracle_plv_time_resolved", "oracle_dft_bins",
              "oracle_coherency_trials", "oracle_analytic_band", "oracle_set_threads",
              "oracle_max_threads"):
        getattr(mut, f).argtypes = getattr(good, f).argtypes
        getattr(mut, f).restype = getattr(good, f).restype
    failed = 0
    oracle._lib = mut
    try:
        for call in PIN_CALLS:
            try:
                call()
            except AssertionError:
                failed += 1
    finally:
        oracle._lib = good
    assert failed > 0, f"no pin caught mutation {name}"
