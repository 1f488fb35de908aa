"""Pins for the oracle's spatial SIR step (paper Sec. 5.1.2, re-cast with
same-cell contacts on the grid; invariants of Sec. 5.1.3).

* Invariants: S + I + R = N every step, R never decreases, the initial
  infected count equals the parameter, the count recurrences hold.
* Movement is the random walk's (states never influence moves).
* beta = 0: no infection, and I(t) ~ Binomial(n0, (1 - p_rec)^t).
* L = 1 (one cell): the chain-binomial (Reed-Frost) model with geometric
  recovery; the exact distribution of (S, I) after a few steps, computed by
  dynamic programming with the exact threshold probabilities, against oracle
  frequencies over many replicate keys.
* L = 2, N = 3: exact distribution of every agent's (cell, state) after two
  steps by enumeration (moves, then same-cell counts of start-of-step
  infected in the NEW cells, then infection / recovery), against the oracle.
* beta = gamma = 1 corner: newly infected agents do not recover in the step
  in which they were infected.
"""
import itertools
from collections import Counter
from fractions import Fraction

import numpy as np
from scipy import stats

import oracle

TWO32 = 1 << 32


def _check_invariants(p, n, n0):
    c = p.counts()
    S, I, R, new = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    assert np.all(S + I + R == n)
    assert np.all(np.diff(np.concatenate([[0], R])) >= 0)
    S_prev = np.concatenate([[n - n0], S[:-1]])
    assert np.all(S_prev - S == new)


def test_invariants_medium():
    n, n0 = 30_000, 30
    p = oracle.Population("sir", n, seed=2, L=224, beta=0.2, gamma=0.05, n0=n0)
    assert int((p.state == oracle.I).sum()) == n0
    assert int((p.state == oracle.S).sum()) == n - n0
    p.step(60)
    _check_invariants(p, n, n0)
    assert p.counts()[-1, 2] > 0 and p.counts()[:, 3].sum() > 0
    assert p.x.min() >= 0 and p.x.max() < 224 and p.y.min() >= 0 and p.y.max() < 224


def test_moves_equal_random_walk():
    a = oracle.Population("sir", 5000, seed=13, rep=4, L=50, beta=0.3, gamma=0.1, n0=50)
    b = oracle.Population("walk", 5000, seed=13, rep=4, L=50)
    a.step(25)
    b.step(25)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)


def test_no_transmission_binomial_recovery():
    n, T, gamma = 3000, 10, 0.1
    p = oracle.Population("sir", n, seed=21, L=5, beta=0.0, gamma=gamma, n0=n)
    p.step(T)
    _, t_rec = oracle.sir_thresholds(0.0, gamma, n)
    q = (1.0 - t_rec / TWO32) ** T
    I_T = p.counts()[-1, 1]
    assert abs(I_T - n * q) < 5 * np.sqrt(n * q * (1 - q))
    p2 = oracle.Population("sir", n, seed=22, L=5, beta=0.0, gamma=gamma, n0=10)
    p2.step(T)
    assert np.all(p2.counts()[:, 0] == n - 10)
    assert np.all(p2.counts()[:, 3] == 0)


def test_newly_infected_do_not_recover_same_step():
    p = oracle.Population("sir", 100, seed=1, L=1, beta=1.0, gamma=1.0, n0=1)
    p.step(1)
    assert p.counts()[-1].tolist() == [0, 99, 1, 99]
    p.step(1)
    assert p.counts()[-1].tolist() == [0, 0, 100, 0]


def _binom_pmf(n, k, p):
    from math import comb
    return comb(n, k) * p ** k * (1 - p) ** (n - k)


def _reed_frost_exact(n, n0, t_inf, t_rec, T):
    K = len(t_inf) - 1
    p_rec = Fraction(t_rec, TWO32)
    dist = {(n - n0, n0): Fraction(1)}
    for _ in range(T):
        nxt = Counter()
        for (s, i), pr in dist.items():
            p_inf = Fraction(int(t_inf[min(i, K)]), TWO32) if i >= 1 else Fraction(0)
            for a in range(s + 1):
                pa = _binom_pmf(s, a, p_inf)
                if pa == 0:
                    continue
                for b in range(i + 1):
                    pb = _binom_pmf(i, b, p_rec)
                    if pb == 0:
                        continue
                    nxt[(s - a, i + a - b)] += pr * pa * pb
        dist = nxt
    return dist


def _chi2_pooled(exact, freq, reps, min_expected=5.0):
    for k in freq:
        assert k in exact, "impossible outcome %r" % (k,)
    obs, exp, pool_o, pool_e = [], [], 0.0, 0.0
    for k, pr in exact.items():
        e = float(pr) * reps
        if e < min_expected:
            pool_o += freq.get(k, 0)
            pool_e += e
        else:
            obs.append(freq.get(k, 0))
            exp.append(e)
    if pool_e > 0:
        obs.append(pool_o)
        exp.append(pool_e)
    obs = np.array(obs, dtype=float)
    exp = np.array(exp)
    exp *= obs.sum() / exp.sum()
    return stats.chisquare(obs, exp).pvalue


def test_single_cell_reed_frost_exact():
    n, n0, beta, gamma, T = 5, 1, 0.3, 0.25, 3
    t_inf, t_rec = oracle.sir_thresholds(beta, gamma, n)
    exact = _reed_frost_exact(n, n0, t_inf, t_rec, T)
    assert sum(exact.values()) == 1
    reps = 20000
    freq = Counter()
    for rep in range(reps):
        p = oracle.Population("sir", n, seed=77, rep=rep, L=1, beta=beta, gamma=gamma, n0=n0)
        p.step(T)
        c = p.counts()[-1]
        freq[(int(c[0]), int(c[1]))] += 1
    assert _chi2_pooled(exact, freq, reps) > 1e-4


# moves on the 2 x 2 torus: flip both coordinates 4/8, only y 2/8, only x 2/8
_FLIPS = [((1, 1), Fraction(1, 2)), ((0, 1), Fraction(1, 4)), ((1, 0), Fraction(1, 4))]


def _two_by_two_exact(init, t_inf, t_rec, T):
    K = len(t_inf) - 1
    p_rec = Fraction(t_rec, TWO32)
    dist = {tuple(init): Fraction(1)}
    for _ in range(T):
        nxt = Counter()
        for conf, pr in dist.items():
            for moves in itertools.product(_FLIPS, repeat=len(conf)):
                pm = pr
                cells = []
                for (x, y, _s), ((fx, fy), pf) in zip(conf, moves):
                    cells.append((x ^ fx, y ^ fy))
                    pm *= pf
                k = Counter(c for c, (_x, _y, s) in zip(cells, conf) if s == oracle.I)
                # per agent: list of (new state, probability)
                opts = []
                for c, (_x, _y, s) in zip(cells, conf):
                    if s == oracle.S and k[c] >= 1:
                        pi = Fraction(int(t_inf[min(k[c], K)]), TWO32)
                        opts.append([(oracle.I, pi), (oracle.S, 1 - pi)])
                    elif s == oracle.I:
                        opts.append([(oracle.R, p_rec), (oracle.I, 1 - p_rec)])
                    else:
                        opts.append([(s, Fraction(1))])
                for outcome in itertools.product(*opts):
                    po = pm
                    new = []
                    for c, (s2, ps) in zip(cells, outcome):
                        po *= ps
                        new.append((c[0], c[1], s2))
                    if po:
                        nxt[tuple(new)] += po
        dist = nxt
    return dist


def test_two_by_two_grid_exact():
    beta, gamma, T = 0.6, 0.3, 2
    init = [(0, 0, oracle.I), (1, 0, oracle.S), (1, 1, oracle.S)]
    t_inf, t_rec = oracle.sir_thresholds(beta, gamma, 3)
    exact = _two_by_two_exact(init, t_inf, t_rec, T)
    assert sum(exact.values()) == 1
    reps = 30000
    freq = Counter()
    for rep in range(reps):
        p = oracle.Population("sir", 3, seed=31, rep=rep, L=2, beta=beta, gamma=gamma, n0=1)
        p.x[:] = [a[0] for a in init]
        p.y[:] = [a[1] for a in init]
        p.state[:] = [a[2] for a in init]
        p.step(T)
        freq[tuple((int(p.x[j]), int(p.y[j]), int(p.state[j])) for j in range(3))] += 1
    assert _chi2_pooled(exact, freq, reps) > 1e-4
