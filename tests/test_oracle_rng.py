"""Pins for the oracle's random numbers and probability thresholds.

* Philox4x32-10 against the published known-answer vectors (golden file).
* Direction bits (top three bits of word 0) uniform over the 8 Moore moves.
* SIR thresholds T_inf[k] against the exact rational value of
  floor((1 - (1 - beta)^k) * 2^32) (within one unit: the table is built with
  double arithmetic), T_rec exactly floor(gamma * 2^32).
"""
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    with open(GOLD) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert [int(v) for v in oracle.philox4x32_10(ctr, key)] == out


def test_philox_counter_and_key_sensitivity():
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for j in range(4):
        c = [1, 2, 3, 4]
        c[j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(c, [5, 6]), base)
    for j in range(2):
        k = [5, 6]
        k[j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10([1, 2, 3, 4], k), base)


def test_direction_bits_uniform():
    counts = np.zeros(8, dtype=np.int64)
    for i in range(20000):
        u = oracle.philox4x32_10([i, 7, 0, 0], [11, 0])
        counts[int(u[0]) >> 29] += 1
    assert stats.chisquare(counts).pvalue > 1e-4


def _exact_threshold_of_power(beta, k):
    """floor((1 - (1-beta)^k) * 2^32) with beta the exact value of the double."""
    b = Fraction(beta)
    q = (1 - b) ** k
    v = (1 - q) * (1 << 32)
    fl = v.numerator // v.denominator
    return min(fl, (1 << 32) - 1)


@pytest.mark.parametrize("beta", [0.05, 0.01, 0.2, 0.5, 0.123456789, 0.9])
def test_infection_thresholds_match_exact_power(beta):
    t_inf, _ = oracle.sir_thresholds(beta, 0.0, 10_000_000)
    K = t_inf.size - 1
    assert t_inf[0] == 0
    assert np.all(np.diff(t_inf.astype(np.int64)) >= 0)
    # table ends where it saturates
    assert t_inf[K] == 0xFFFFFFFF
    ks = list(range(1, min(K, 60) + 1)) + list(range(max(61, K - 5), K + 1))
    for k in ks:
        assert abs(int(t_inf[k]) - _exact_threshold_of_power(beta, k)) <= 1, (beta, k)


def test_worked_threshold_values():
    # beta = 0.05: p_1 = 0.05 -> floor(0.05 * 2^32) = floor(214748364.8)
    t_inf, t_rec = oracle.sir_thresholds(0.05, 0.02, 100)
    assert int(t_inf[1]) == 214748364
    # gamma = 0.02 -> floor(85899345.92)
    assert t_rec == 85899345
    # p_2 = 1 - 0.95^2 = 0.0975 -> floor(418759311.36)
    assert int(t_inf[2]) == 418759311


@pytest.mark.parametrize("gamma", [0.0, 0.02, 0.005, 0.05, 0.3333, 1.0])
def test_recovery_threshold_exact(gamma):
    _, t_rec = oracle.sir_thresholds(0.1, gamma, 10)
    v = Fraction(gamma) * (1 << 32)
    assert t_rec == min(v.numerator // v.denominator, (1 << 32) - 1)


def test_threshold_degenerate_cases():
    t_inf, t_rec = oracle.sir_thresholds(0.0, 0.0, 1000)
    assert t_inf.tolist() == [0, 0] and t_rec == 0
    t_inf, t_rec = oracle.sir_thresholds(1.0, 1.0, 1000)
    assert t_inf.tolist() == [0, 0xFFFFFFFF] and t_rec == 0xFFFFFFFF
    # the table never exceeds the population size
    t_inf, _ = oracle.sir_thresholds(1e-6, 0.0, 50)
    assert t_inf.size == 51
    with pytest.raises(RuntimeError):
        oracle.sir_thresholds(-0.1, 0.0, 10)
    with pytest.raises(RuntimeError):
        oracle.sir_thresholds(0.1, 1.5, 10)
    with pytest.raises(RuntimeError):
        oracle.sir_thresholds(float("nan"), 0.1, 10)
