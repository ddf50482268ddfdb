"""Pins of the oracle's Metropolis variant of the k sampler (the paper's Sec. 2.3 names a
Metropolis procedure without its proposal; the reading is a symmetric random walk with
acceptance min(1, w(k')/w(k)) on the sampler's box).  The paper gives no numbers to
check against, so the chain is pinned by what the mathematics fixes:

- one update from a fixed state follows the Metropolis transition kernel, computed here
  by enumeration (chi-square over many independent chains);
- the target P(k) = w(k)/S is stationary: chains started from exact draws still have the
  exact marginals after many updates (chi-square);
- chains started far from equilibrium reach the same marginals;
- the counter layout: chains are independent of P and of each other's index.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _sys(Lx=8.0, Ly=10.0, Lz=24.0, alpha=0.6):
    return O.System(Lx=Lx, Ly=Ly, H=2.0, Lz=Lz, gamma_top=0.0, gamma_bot=0.0, alpha=alpha, M=0)


def _w(n, s):
    return (O.w1d(n[0], s.alpha, s.Lx) * O.w1d(n[1], s.alpha, s.Ly) * O.w1d(n[2], s.alpha, s.Lz))


def _chisq_p(obs, exp, min_expected=5.0):
    """Pearson chi-square p-value after pooling bins with small expectation."""
    obs, exp = np.asarray(obs, float), np.asarray(exp, float)
    order = np.argsort(exp)
    o_b, e_b, o_acc, e_acc = [], [], 0.0, 0.0
    for i in order:
        o_acc += obs[i]
        e_acc += exp[i]
        if e_acc >= min_expected:
            o_b.append(o_acc); e_b.append(e_acc); o_acc = e_acc = 0.0
    if e_acc > 0:
        o_b[-1] += o_acc; e_b[-1] += e_acc
    o_b, e_b = np.array(o_b), np.array(e_b)
    chi2 = float(np.sum((o_b - e_b) ** 2 / e_b))
    return stats.chi2.sf(chi2, len(o_b) - 1)


def test_proposal_half_width_rule():
    # s_d = max(1, ceil(alpha L / (pi sqrt 2))): about one standard deviation of the 1-D factor
    assert O.metropolis_halfwidth(0.6, 8.0) == 2
    assert O.metropolis_halfwidth(0.6, 10.0) == 2
    assert O.metropolis_halfwidth(0.6, 24.0) == 4
    assert O.metropolis_halfwidth(0.1, 1.0) == 1
    assert O.metropolis_halfwidth(1.0772173450159417, 200.0) == math.ceil(1.0772173450159417 * 200 / (math.pi * math.sqrt(2)))


@pytest.mark.parametrize("n0", [(1, 0, 0), (0, 2, -3), (-3, 1, 6)])
def test_one_update_follows_the_metropolis_kernel(n0):
    s = _sys()
    hw = [O.metropolis_halfwidth(s.alpha, L) for L in (s.Lx, s.Ly, s.Lz)]
    nd = [O.nmax(s.alpha, L) for L in (s.Lx, s.Ly, s.Lz)]
    C = 200000
    st, _ = O.metropolis(s, 7, 3, 1, np.tile(np.array(n0, np.int32), (C, 1)))
    # analytic kernel: uniform proposal on the offset box, acceptance min(1, w'/w)
    w0 = _w(n0, s)
    q = 1.0 / np.prod([2 * h + 1 for h in hw])
    probs = {}
    stay = 1.0
    for dx in range(-hw[0], hw[0] + 1):
        for dy in range(-hw[1], hw[1] + 1):
            for dz in range(-hw[2], hw[2] + 1):
                m = (n0[0] + dx, n0[1] + dy, n0[2] + dz)
                if m == tuple(n0):
                    continue
                inside = all(abs(m[d]) <= nd[d] for d in range(3)) and m != (0, 0, 0)
                a = min(1.0, _w(m, s) / w0) if inside else 0.0
                probs[m] = q * a
                stay -= q * a
    probs[tuple(n0)] = stay
    keys = list(probs)
    index = {k: i for i, k in enumerate(keys)}
    obs = np.zeros(len(keys))
    for row in map(tuple, st):
        obs[index[row]] += 1  # a move outside the proposal box would raise KeyError
    exp = np.array([probs[k] for k in keys]) * C
    assert _chisq_p(obs, exp) > 1e-4


def _exact_marginals(s):
    """Marginals of P(k) = w(k)/S over the box without k = 0."""
    Ls = (s.Lx, s.Ly, s.Lz)
    nd = [O.nmax(s.alpha, L) for L in Ls]
    w = [np.array([O.w1d(n, s.alpha, L) for n in range(-h, h + 1)]) for h, L in zip(nd, Ls)]
    Sd = [x.sum() for x in w]
    S = Sd[0] * Sd[1] * Sd[2] - 1.0
    out = []
    for d in range(3):
        others = Sd[(d + 1) % 3] * Sd[(d + 2) % 3]
        m = w[d] * others
        m[nd[d]] -= 1.0  # n_d = 0 excludes k = 0 once: w(0)=1 in every factor
        out.append((np.arange(-nd[d], nd[d] + 1), m / S))
    return out


def _marginal_pvalues(states, s):
    ps = []
    for d, (ns, p) in enumerate(_exact_marginals(s)):
        obs = np.array([(states[:, d] == n).sum() for n in ns])
        assert obs.sum() == states.shape[0]
        ps.append(_chisq_p(obs, p * states.shape[0]))
    return ps


def test_exact_draws_stay_exact_under_the_chain():
    """Stationarity of w(k)/S: 20000 chains started from exact draws keep the exact
    marginals after 30 updates."""
    s = _sys()
    P = 20000
    st = O.sample_k(s, 3, 0, P)
    assert min(_marginal_pvalues(st, s)) > 1e-4  # the exact sampler itself
    for step in range(1, 4):
        st, acc = O.metropolis(s, 3, step, 10, st)
    assert 0.2 < acc / (10 * P) < 0.9
    assert min(_marginal_pvalues(st, s)) > 1e-4


def test_cold_chains_converge_to_the_target():
    s = _sys(alpha=0.5)
    P = 20000
    st = np.tile(np.array([1, 0, 0], np.int32), (P, 1))
    for step in range(20):
        st, _ = O.metropolis(s, 11, step, 10, st)
    assert min(_marginal_pvalues(st, s)) > 1e-4


def test_chains_depend_only_on_their_own_counter():
    s = _sys()
    st0 = O.sample_k(s, 5, 0, 64)
    a, _ = O.metropolis(s, 5, 2, 4, st0)
    b, _ = O.metropolis(s, 5, 2, 4, st0[10:20])
    assert not np.array_equal(a[10:20], b)  # the chain index is part of the counter
    # the same chain index with the same start gives the same result whatever P is
    c, _ = O.metropolis(s, 5, 2, 4, st0[:20])
    assert np.array_equal(a[:20], c)
    # another step or seed moves differently
    d, _ = O.metropolis(s, 5, 3, 4, st0)
    e, _ = O.metropolis(s, 6, 2, 4, st0)
    assert not np.array_equal(a, d) and not np.array_equal(a, e)
