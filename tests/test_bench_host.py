"""Host-side helpers of bench.py on CPU: the per-metric error report against
the oracle, the seeded channel sample, the uneven-batch problem list and the
any-length transform length."""
import numpy as np

import bench


def test_oracle_errors_reports_max_mean_and_conditioned_ciplv():
    rng = np.random.default_rng(0)
    n = 6
    ref = {"plv": rng.random((n, n)), "iplv": rng.random((n, n)) * 0.1,
           "ciplv": rng.random((n, n))}
    ref["plv"][0, 1] = 1.0  # |C| = 1, Im ~ 0: 1 - Re^2 ~ 0, ill-conditioned
    ref["iplv"][0, 1] = 0.0
    got = {k: v.copy() for k, v in ref.items()}
    got["plv"][2, 3] += 3e-6
    got["ciplv"][0, 1] += 1e-3  # only on the ill-conditioned pair
    rep = bench.oracle_errors({"bf16x3": got}, ref, n, 100)
    e = rep["bf16x3"]
    assert abs(e["plv"]["max"] - 3e-6) < 1e-12
    assert abs(e["plv"]["mean"] - 3e-6 / n ** 2) < 1e-12
    assert e["iplv"]["max"] == 0.0
    assert abs(e["ciplv"]["max"] - 1e-3) < 1e-12
    # the conditioned ciPLV error leaves out the pair with sqrt(1 - Re^2) < 0.05
    assert e["ciplv_well_conditioned"]["max"] == 0.0
    assert rep["ciplv_well_conditioned_pairs"] == n * n - 1


def test_sample_channels_is_seeded_sorted_and_distinct():
    a = bench.sample_channels(4096, 1002, 384)
    b = bench.sample_channels(4096, 1002, 384)
    assert np.array_equal(a, b)
    assert len(np.unique(a)) == 384 and np.all(np.diff(a) > 0)
    assert a.min() >= 0 and a.max() < 4096
    assert len(bench.sample_channels(10, 1, 384)) == 10


def test_grouped_problems_shape_the_uneven_batch():
    specs = bench.grouped_problems(seed=1004, nsub=256)
    assert len(specs) == 256 * 5
    Ns = np.array([s[0] for s in specs])
    Ts = np.array([s[1] for s in specs])
    assert Ns.min() >= 68 and Ns.max() <= 2000
    assert Ts.min() >= 500 and Ts.max() <= 10000
    # the five bands of a subject share its N and T, with distinct seeds
    for sj in range(0, 256, 37):
        sub = specs[5 * sj:5 * sj + 5]
        assert len({(s[0], s[1]) for s in sub}) == 1
        assert [s[2] for s in sub] == bench.BANDS
        assert len({s[3] for s in sub}) == 5


def test_transform_length_of_the_any_length_engine():
    for T in (2, 3, 16, 17, 100, 500, 1000, 2400, 4097, 9999, 12288):
        M = bench._conv_M(T)
        assert M >= 2 * T - 1 and M >= 32
        odd = M
        while odd % 2 == 0:
            odd //= 2
        assert odd in (1, 3, 5)
        # no smaller length of the three forms fits
        for f in (1, 3, 5):
            p = 32
            while f * p < M:
                assert f * p < 2 * T - 1
                p *= 2
