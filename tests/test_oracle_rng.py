"""Pins for the oracle's random inputs (oracle/rng.py)."""
import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

from conftest import golden_rows
from oracle import rng


def test_philox_known_answers():
    for row in golden_rows("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        out = rng.philox4x32_10(*vals[:6])
        assert [int(o) for o in out] == vals[6:10]


def test_philox_vectorised_matches_scalar():
    c = np.arange(10, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15 & 0xFFFFFFFF)
    out = rng.philox4x32_10(c, c + np.uint64(1), c + np.uint64(2), c + np.uint64(3), 7, 11)
    for i in range(10):
        one = rng.philox4x32_10(int(c[i]), int(c[i]) + 1, int(c[i]) + 2, int(c[i]) + 3, 7, 11)
        assert [int(o[i]) for o in out] == [int(v) for v in one]


def test_uniform_map_exact_and_open_interval():
    u = rng.uniform_from_words(np.array([0, 0xFFFFFFFF, 0x80000000]), np.array([0, 0xFFFFFFFF, 0]))
    assert u[0] == 2.0 ** -53                      # M = 0
    assert u[1] == 1.0 - 2.0 ** -53                # M = 2^52 - 1
    assert u[2] == 0.5 + 2.0 ** -53                # M = 2^51
    assert np.all((u > 0.0) & (u < 1.0))


def test_log_series_within_two_ulp_of_libm():
    g = np.random.default_rng(5)
    x = np.concatenate([g.random(200000) * 0.5 + 1e-300, np.exp(-g.random(20000) * 37.0),
                        [2.0 ** -53, 0.5, 0.25, 1.0 - 2.0 ** -53, 0.075]])
    ref = np.log(x)
    got = rng.log_series(x)
    ulp = np.abs(got - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 2.0
    assert rng.log_series(np.array([1.0]))[0] == 0.0


def test_as241_inverse_of_normal_cdf():
    g = np.random.default_rng(6)
    u = np.concatenate([g.random(300000), [2.0 ** -53, 1e-12, 0.075, 0.5 - 2.0 ** -40, 0.5 + 2.0 ** -40,
                                           0.925, 1.0 - 2.0 ** -53, 1e-300]])
    z = rng.normal_from_uniform(u)
    # against an independent library inverse (relative) and the forward CDF (absolute in u)
    zr = sp.ndtri(u)
    assert np.max(np.abs(z - zr) / np.maximum(np.abs(zr), 1e-3)) < 5e-15
    back = np.where(u < 0.5, sp.ndtr(z), sp.ndtr(-z))
    uu = np.where(u < 0.5, u, 1.0 - u)
    # d(log u)/dz = -z near the tails, so the relative error in u grows like |z| dz
    assert np.all(np.abs(back - uu) / uu <= 4e-15 * (1.0 + z * z))
    # odd symmetry for pairs u, 1 - u that are both exact
    v = np.array([0.125, 0.375, 2.0 ** -10, 2.0 ** -40])
    assert np.array_equal(rng.normal_from_uniform(v), -rng.normal_from_uniform(1.0 - v))


def test_xi_counter_mapping_and_streams():
    a = rng.draw_xi(seed=0, level=2, first=5, count=4, K=6)
    b = rng.draw_xi(seed=0, level=2, first=0, count=9, K=6)
    assert np.array_equal(a, b[5:9])                 # counter = sample index
    c = rng.draw_xi(seed=0, level=3, first=5, count=4, K=6)
    d = rng.draw_xi(seed=1, level=2, first=5, count=4, K=6)
    assert not np.any(a == c) and not np.any(a == d)  # level and seed select streams
    # explicit word selection for sample k = 2^32 + 3, term j = 5 (odd -> words 2, 3)
    k, j, lev, seed = (1 << 32) + 3, 5, 1, (7 << 32) | 9
    w = rng.philox4x32_10(k & 0xFFFFFFFF, k >> 32, lev, j >> 1, seed & 0xFFFFFFFF, seed >> 32)
    u = rng.uniform_from_words(w[2], w[3])
    assert rng.draw_xi(seed, lev, k, 1, 6)[0, j] == rng.normal_from_uniform(np.atleast_1d(u))[0]


def test_xi_is_standard_normal():
    z = rng.draw_xi(seed=123, level=0, first=0, count=20000, K=16).ravel()
    N = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / N)
    assert st.kstest(z, "norm").pvalue > 1e-4
    # neighbouring terms and samples are uncorrelated
    zz = rng.draw_xi(seed=123, level=0, first=0, count=20000, K=16)
    r = np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]
    assert abs(r) < 5.0 / np.sqrt(20000)


@pytest.mark.parametrize("K", [1, 2, 7, 64])
def test_xi_shapes(K):
    assert rng.draw_xi(0, 0, 0, 3, K).shape == (3, K)
    assert rng.draw_xi(0, 0, 0, 0, K).shape == (0, K)
