"""Pins of the oracle's continuous-space models (paper Sec. 5.1.2 as the paper
states them: box [0, w] x [0, h], float32 positions).

Random walk: every coordinate stays in the box (the paper's clamp invariant,
Sec. 5.1.3); away from the walls a step is U[-s, s) on each axis (KS test,
variance s^2/3, independent axes); at a wall the position clamps exactly;
initial positions are uniform over the box (chi-square).
SIR: S + I + R = N, the initial infected count, R never decreases; with p = 0
an infected agent recovers after exactly rec_steps steps; contact is
distance <= r with the boundary itself included; when every pair is in contact
the epidemic is the chain-binomial (Reed-Frost) model with deterministic
recovery, whose exact distribution (dynamic programming with the exact
threshold probabilities) matches the oracle's frequencies."""
from collections import Counter
from fractions import Fraction
from math import comb

import numpy as np
from scipy import stats

import oracle

TWO32 = 1 << 32


def test_walk_bounds_and_clamp():
    p = oracle.CPopulation("cwalk", 20_000, seed=3, w=30.0, h=20.0, s=2.5)
    for _ in range(40):
        p.step(1)
        assert p.x.min() >= 0.0 and p.x.max() <= 30.0 and p.y.min() >= 0.0 and p.y.max() <= 20.0
    # agents pinned at the walls hit them exactly: a clamped coordinate is 0 or w
    assert (p.x == 0.0).sum() > 0 and (p.x == 30.0).sum() > 0


def test_walk_step_is_uniform_away_from_walls():
    n, s = 200_000, 1.5
    p = oracle.CPopulation("cwalk", n, seed=9, rep=2, w=100.0, h=100.0, s=s)
    x0, y0 = p.x.copy(), p.y.copy()
    p.step(1)
    inner = (x0 > 2 * s) & (x0 < 100 - 2 * s) & (y0 > 2 * s) & (y0 < 100 - 2 * s)
    dx = (p.x - x0)[inner].astype(np.float64)
    dy = (p.y - y0)[inner].astype(np.float64)
    assert dx.min() >= -s and dx.max() < s + 1e-4
    assert stats.kstest(dx, stats.uniform(loc=-s, scale=2 * s).cdf).pvalue > 1e-3
    assert stats.kstest(dy, stats.uniform(loc=-s, scale=2 * s).cdf).pvalue > 1e-3
    assert abs(dx.var() - s * s / 3) < 0.01 * s * s
    assert abs(np.corrcoef(dx, dy)[0, 1]) < 0.01


def test_walk_clamp_exact():
    p = oracle.CPopulation("cwalk", 4, seed=1, w=10.0, h=10.0, s=100.0)
    p.step(1)
    # with s far larger than the box every step lands on a wall
    assert np.all(np.isin(p.x, [0.0, 10.0])) and np.all(np.isin(p.y, [0.0, 10.0]))


def test_initial_positions_uniform():
    p = oracle.CPopulation("cwalk", 100_000, seed=5, w=100.0, h=50.0)
    assert p.x.min() >= 0 and p.x.max() < 100 and p.y.min() >= 0 and p.y.max() < 50
    h, _, _ = np.histogram2d(p.x, p.y, bins=[10, 10], range=[[0, 100], [0, 50]])
    assert stats.chisquare(h.ravel()).pvalue > 1e-3


def _check_sir(p, n, n0):
    c = p.counts()
    assert np.all(c[:, :3].sum(axis=1) == n)
    assert np.all(np.diff(np.concatenate([[0], c[:, 2]])) >= 0)
    S_prev = np.concatenate([[n - n0], c[:-1, 0]])
    assert np.all(S_prev - c[:, 0] == c[:, 3])


def test_sir_invariants_paper_setting():
    n = 2000
    p = oracle.CPopulation("csir", n, seed=4, w=100.0, h=100.0, s=0.0, r=5.0, p=0.1, rec_steps=14, n0=5)
    assert int((p.state == 1).sum()) == 5
    p.step(50)
    _check_sir(p, n, 5)
    c = p.counts()
    assert c[-1, 2] > 0 and c[:, 3].sum() > 0
    assert np.all(p.days[p.state == 1] < 14)


def test_sir_recovery_after_exactly_rec_steps():
    n, rec = 50, 14
    p = oracle.CPopulation("csir", n, seed=8, p=0.0, rec_steps=rec, n0=7)
    p.step(20)
    I = p.counts()[:, 1]
    assert np.all(I[: rec - 1] == 7) and np.all(I[rec - 1:] == 0)
    assert np.all(p.counts()[rec - 1:, 2] == 7)


def test_contact_boundary_is_inclusive():
    # two agents on a line: 0 infected, 1 susceptible at distance exactly r, 2 just beyond
    p = oracle.CPopulation("csir", 3, seed=1, s=0.0, r=5.0, p=1.0, rec_steps=10, n0=1)
    p.x[:] = [10.0, 15.0, 10.0]
    p.y[:] = [10.0, 10.0, 15.000002]
    p.step(1)
    assert list(p.state) == [1, 1, 0]


def _reed_frost_deterministic(n, n0, t_inf, rec_steps, T):
    """(S, infected by age) distribution: everyone in contact, every infected
    agent recovers after rec_steps steps."""
    K = len(t_inf) - 1
    dist = {(n - n0, (0,) * (rec_steps - 1) + (n0,)): Fraction(1)}  # ages: oldest first
    for _ in range(T):
        nxt = Counter()
        for (s, ages), pr in dist.items():
            i = sum(ages)
            p_inf = Fraction(int(t_inf[min(i, K)]), TWO32) if i >= 1 else Fraction(0)
            for a in range(s + 1):
                pa = comb(s, a) * p_inf ** a * (1 - p_inf) ** (s - a)
                if pa:
                    nxt[(s - a, ages[1:] + (a,))] += pr * pa
        dist = nxt
    out = Counter()
    for (s, ages), pr in dist.items():
        out[(s, sum(ages))] += pr
    return out


def _chi2(exact, freq, reps):
    obs, exp, po, pe = [], [], 0, 0.0
    for k in freq:
        assert k in exact, k
    for k, pr in exact.items():
        e = float(pr) * reps
        if e < 5:
            po += freq.get(k, 0)
            pe += e
        else:
            obs.append(freq.get(k, 0))
            exp.append(e)
    if pe:
        obs.append(po)
        exp.append(pe)
    exp = np.array(exp)
    exp *= sum(obs) / exp.sum()
    return stats.chisquare(obs, exp).pvalue


def test_everyone_in_contact_is_reed_frost():
    n, n0, prob, T = 5, 1, 0.35, 3
    t_inf, _ = oracle.sir_thresholds(prob, 0.0, n)
    for rec in (1, 2):
        exact = _reed_frost_deterministic(n, n0, t_inf, rec, T)
        assert sum(exact.values()) == 1
        reps = 12_000
        freq = Counter()
        for rep in range(reps):
            # a 1 x 1 box with radius 2: every pair is in contact, moving or not
            p = oracle.CPopulation("csir", n, seed=31, rep=rep, w=1.0, h=1.0, s=0.3, r=2.0, p=prob, rec_steps=rec,
                                   n0=n0)
            p.step(T)
            c = p.counts()[-1]
            freq[(int(c[0]), int(c[1]))] += 1
        assert _chi2(exact, freq, reps) > 1e-4, rec


def test_sir_moves_equal_walk():
    a = oracle.CPopulation("csir", 3000, seed=6, s=1.0, p=0.2, n0=20)
    b = oracle.CPopulation("cwalk", 3000, seed=6, s=1.0)
    a.step(15)
    b.step(15)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)
