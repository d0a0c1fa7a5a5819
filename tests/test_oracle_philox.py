"""Pins for the oracle's Philox4x32-10 and its column sampler (CPU only)."""
import json
import os

import numpy as np
from scipy import stats

import oracle as O
from oracle.philox import philox4x32_10, step_uniforms, words_to_uniform

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")


def test_philox_known_answers():
    for case in json.load(open(GOLD))["cases"]:
        ctr = [int(v, 16) for v in case["counter"]]
        key = [int(v, 16) for v in case["key"]]
        assert [hex(v) for v in philox4x32_10(ctr, key)] == [hex(int(v, 16)) for v in case["out"]]


def test_uniform_construction_bounds():
    assert words_to_uniform(0, 0) == 0.0
    top = words_to_uniform(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and top == (2 ** 53 - 1) / 2 ** 53


def test_step_uniforms_are_uniform():
    us = np.array([step_uniforms(7, 3, 2, t) for t in range(4000)]).ravel()
    assert stats.kstest(us, "uniform").pvalue > 1e-3


def test_invcdf_column_sampler_law():
    """Alg. 2 steps 8/10: P(j) = ||A_1(:,j)||^2 / ||A_1||_F^2 (chi-square on Philox draws)."""
    rng = np.random.default_rng(5)
    A1 = rng.standard_normal((30, 6)) * np.array([0.3, 1.0, 2.0, 0.5, 1.5, 1.0])
    norms2, cum = O.column_cumsum(A1)
    draws = 6000
    counts = np.zeros(6)
    for t in range(draws // 2):
        u0, u1 = step_uniforms(11, 0, 0, t)
        counts[O.invcdf_pick(cum, u0)] += 1
        counts[O.invcdf_pick(cum, u1)] += 1
    expect = draws * norms2 / norms2.sum()
    assert stats.chisquare(counts, expect).pvalue > 1e-3


def test_invcdf_edges():
    cum = np.array([1.0, 1.0, 3.0, 6.0])  # column 1 has zero weight
    assert O.invcdf_pick(cum, 0.0) == 0
    assert O.invcdf_pick(cum, 1.0 / 6.0) == 2  # cum[0] = 1 is not > 1, column 1 skipped
    assert O.invcdf_pick(cum, 0.999999) == 3
