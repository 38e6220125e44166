"""Pins of the oracle's random-number layer against published values and closed forms.

* Philox4x32-10 against the generator's published known-answer vectors (tests/golden).
* The uniform map against its definition (exact 24-bit dyadic values inside (0, 1)).
* The d = 2 Green-density radius against the CDF printed in the proof of Prop. 2.6 (i.1):
  F(t) = t^2 - t^2 ln t^2, and against its moments E R = 4/9, E R^2 = 1/4.
* The ball-term radius S = 1 - sqrt(U) against the CDF 2t - t^2 of the proof of Prop. 2.6 (ii).
* The Beta(2,2) importance-weighted form of Prop. 2.6 (i.1) against the exact sampler.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers(oracle_lib):
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = oracle_lib.philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_uniform_map_is_exact_and_open(oracle_lib):
    assert oracle_lib.u01(0) == 2.0 ** -24
    assert oracle_lib.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    for x in [1, 511, 512, 0x80000000, 0x12345678, 0xFFFFFE00]:
        u = oracle_lib.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # representable in FP32 and FP64 alike
        assert u == ((x >> 9) + 0.5) / 2 ** 23


def _F(t):
    return t * t - t * t * np.log(t * t)


def test_green_radius_inverts_the_cdf(oracle_lib):
    us = np.concatenate([np.linspace(1e-7, 1 - 1e-7, 2001), [2.0 ** -24, 1 - 2.0 ** -24, 0.5]])
    R = np.array([oracle_lib.green_radius_2d(u) for u in us])
    assert np.all((R > 0) & (R <= 1))
    assert np.max(np.abs(_F(R) - us)) < 1e-12
    assert np.all(np.diff(R[:2001]) > 0)          # F is increasing, so is its inverse


def test_green_radius_moments(oracle_lib):
    # E R = int_0^1 -4 r^2 ln r dr = 4/9 ; E R^2 = int_0^1 -4 r^3 ln r dr = 1/4  (density rho of Prop. 2.6)
    K = 20000
    u = (np.arange(K) + 0.5) / K
    R = np.array([oracle_lib.green_radius_2d(v) for v in u])
    assert abs(R.mean() - 4.0 / 9.0) < 2e-4
    assert abs((R * R).mean() - 0.25) < 2e-4


def _philox_uniforms(oracle_lib, count, seed=7):
    out = []
    for j in range(count // 4 + 1):
        w = oracle_lib.philox4x32_10([j, 0, 0, 0x77], [seed, 0])
        out.extend(oracle_lib.u01(int(v)) for v in w)
    return np.array(out[:count])


def test_green_radius_ks(oracle_lib):
    u = _philox_uniforms(oracle_lib, 20000)
    R = np.array([oracle_lib.green_radius_2d(v) for v in u])
    assert stats.kstest(R, _F).pvalue > 1e-3


def test_ball_radius_ks(oracle_lib):
    u = _philox_uniforms(oracle_lib, 20000, seed=11)
    S = 1.0 - np.sqrt(u)
    assert stats.kstest(S, lambda t: 2 * t - t * t).pvalue > 1e-3


def test_beta22_weighted_form_matches_exact_sampler(oracle_lib):
    # Prop. 2.6 (i.1): E psi(Y) = -(2/3) E[ ln R / (1-R) psi(R Z) ], R = median of 3 uniforms.
    rng = np.random.default_rng(3)
    K = 400000
    Rb = np.median(rng.random((K, 3)), axis=1)
    wgt = -(2.0 / 3.0) * np.log(Rb) / (1.0 - Rb)
    u = (np.arange(4000) + 0.5) / 4000
    Re = np.array([oracle_lib.green_radius_2d(v) for v in u])
    for psi in (lambda r: r, lambda r: r ** 2, lambda r: np.cos(3 * r)):
        a = np.mean(wgt * psi(Rb))
        se = np.std(wgt * psi(Rb)) / math.sqrt(K)
        b = np.mean(psi(Re))
        assert abs(a - b) < 4 * se + 1e-4
