"""Pins for the oracle's wealth-transfer rule (paper Sec. 5.1.2, Listings 2-3).

* Invariants of Sec. 5.1.3 / 6.2: total wealth = N * w_init after every step;
  added: wealth never negative, donors = agents with positive wealth.
* Brute force: for tiny populations the exact one-step outcome distribution
  (every donor gives one unit to a uniformly chosen OTHER agent, on the
  start-of-step snapshot) is enumerated with the exact bucket probabilities of
  the high-word mapping and compared with oracle frequencies over many
  replicate keys.
* Special cases: N = 1 (nothing happens), N = 2 (deterministic exchange).
"""
import itertools
from collections import Counter
from fractions import Fraction

import numpy as np
from scipy import stats

import oracle


def test_conservation_and_donors_10k_agents():
    n = 10_000
    p = oracle.Population("wealth", n, seed=0)
    assert np.all(p.w == 1)
    for _ in range(100):
        donors = int((p.w > 0).sum())
        p.step(1)
        cnt = p.counts()[-1]
        assert cnt[0] == donors
        assert cnt[1] == n
        assert int(p.w.sum()) == n
        assert p.w.min() >= 0


def _bucket_probs(m):
    """P(high word of u*m == j) for u uniform on 32 bits, exactly."""
    two32 = 1 << 32
    edges = [-(-(j * two32) // m) for j in range(m + 1)]
    return [Fraction(edges[j + 1] - edges[j], two32) for j in range(m)]


def _exact_outcomes(w0):
    n = len(w0)
    probs = _bucket_probs(n - 1)
    donors = [i for i in range(n) if w0[i] > 0]
    dist = Counter()
    for choice in itertools.product(range(n - 1), repeat=len(donors)):
        w = list(w0)
        pr = Fraction(1)
        for i, rp in zip(donors, choice):
            r = rp + (1 if rp >= i else 0)
            w[i] -= 1
            w[r] += 1
            pr *= probs[rp]
        dist[tuple(w)] += pr
    return dist


def _oracle_outcomes(w0, reps, seed=5, step=0):
    freq = Counter()
    for rep in range(reps):
        p = oracle.Population("wealth", len(w0), seed=seed, rep=rep)
        p.w[:] = np.asarray(w0, dtype=np.int32)
        p.t = step
        p.step(1)
        freq[tuple(int(v) for v in p.w)] += 1
    return freq


def _chi2_match(exact, freq, reps):
    keys = sorted(set(exact) | set(freq))
    for k in keys:
        assert k in exact, "oracle produced an impossible outcome %r" % (k,)
    obs = np.array([freq.get(k, 0) for k in keys], dtype=float)
    exp = np.array([float(exact[k]) * reps for k in keys])
    return stats.chisquare(obs, exp).pvalue


def test_brute_force_three_agents_all_donors():
    w0 = (1, 1, 1)
    exact = _exact_outcomes(w0)
    assert sum(exact.values()) == 1
    reps = 12000
    assert _chi2_match(exact, _oracle_outcomes(w0, reps), reps) > 1e-4


def test_brute_force_four_agents_mixed():
    w0 = (2, 0, 1, 0)
    exact = _exact_outcomes(w0)
    reps = 15000
    assert _chi2_match(exact, _oracle_outcomes(w0, reps, seed=9, step=3), reps) > 1e-4


def test_snapshot_semantics_receiver_does_not_give():
    # agent 0 gives to 1 or 2; the receiver had no wealth at the snapshot
    freq = _oracle_outcomes((1, 0, 0), 400)
    assert set(freq) <= {(0, 1, 0), (0, 0, 1)}
    assert len(freq) == 2


def test_two_agents_exchange_and_never_self():
    for rep in range(200):
        p = oracle.Population("wealth", 2, seed=1, rep=rep)
        p.w[:] = [1, 0]
        p.step(1)
        assert p.w.tolist() == [0, 1]
        p.w[:] = [3, 5]
        p.step(1)
        assert p.w.tolist() == [3, 5]


def test_single_agent_noop():
    p = oracle.Population("wealth", 1, seed=0, w_init=7)
    p.step(5)
    assert p.w.tolist() == [7]
    assert p.counts()[:, 0].tolist() == [0] * 5


def test_empty_population():
    p = oracle.Population("wealth", 0, seed=0)
    p.step(3)
    assert p.counts().shape == (3, 4)
    assert np.all(p.counts() == 0)
