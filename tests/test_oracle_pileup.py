"""Pins of the oracle's pile-up merging (Sec. 2.2: with a pile-up block the
parametric path merges minimum-bias interactions with the hard-scatter event
before the detector response; the block's parameters are mean pile-up,
vertex-z and vertex-time widths and truncations, and hard-vertex smearing).

Each pin checks the oracle against something independent of its arithmetic:
scipy's Poisson CDF and truncated normal, the Philox words recomputed from the
counter contract, counting statistics, and the structure of the merged events.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2606_26089_b300 import synth

SEED = 7


def _pu(mean, smear=True, sigma_z=0.053, max_z=0.25, sigma_t=160e-12, max_t=800e-12):
    return oracle.PileUp(float(mean), sigma_z, max_z, sigma_t, max_t, int(smear), 0)


def _words(slot, event, purpose, attempt=0, seed=SEED):
    ctr = np.array([[slot, event, purpose, attempt]], np.uint32)
    return oracle.philox_n(ctr, [seed & 0xFFFFFFFF, seed >> 32])[0]


@pytest.mark.parametrize("mean", [0.0, 0.5, 3.0, 50.0, 170.0, 400.0])
def test_thresholds_follow_the_poisson_cdf(mean):
    T = oracle.poisson_thresholds(mean)
    assert T[-1] == 2**32 and np.all(np.diff(T.astype(np.float64)) >= 0)
    k = np.arange(T.shape[0] - 1)
    assert np.max(np.abs(T[:-1].astype(np.float64) / 2**32 - stats.poisson.cdf(k, mean)), initial=0.0) < 1e-9
    # the table ends at the first k whose upper tail P(N > k) is below 2^-32
    # (up to the rounding of the CDF summed in double)
    assert stats.poisson.sf(T.shape[0] - 1, mean) < 2.0**-32 * 1.01


def test_interaction_counts_follow_the_counter_contract():
    """N is the smallest k with w0 / 2^32 < P(N <= k), w0 = word 0 of Philox
    counter (0, event, 5, 0): recomputed with scipy's CDF."""
    mean = 50.0
    T = oracle.poisson_thresholds(mean)
    cdf = stats.poisson.cdf(np.arange(400), mean)
    for ev in range(300):
        n = oracle.pileup_draws(_pu(mean), T, 1000, SEED, ev)[0]
        w0 = int(_words(0, ev, 5)[0])
        assert n == int(np.searchsorted(cdf, w0 / 2**32, side="right"))


def test_pool_indices_follow_the_counter_contract_and_are_uniform():
    mean, n_pool = 40.0, 997
    T = oracle.poisson_thresholds(mean)
    idx_all = []
    for ev in range(200):
        n, idx, z, t, zhs, ths, m = oracle.pileup_draws(_pu(mean), T, n_pool, SEED, ev)
        for k in range(0, n, 7):
            assert idx[k] == (int(_words(k, ev, 6)[0]) * n_pool) >> 32
        idx_all.append(idx)
    idx_all = np.concatenate(idx_all)
    hist = np.bincount(idx_all * 10 // n_pool, minlength=10)
    assert stats.chisquare(hist).pvalue > 1e-4


def test_counts_have_poisson_mean_and_variance():
    mean = 50.0
    T = oracle.poisson_thresholds(mean)
    n = np.array([oracle.pileup_draws(_pu(mean), T, 10, SEED, ev)[0] for ev in range(4000)])
    assert abs(n.mean() - mean) < 5 * np.sqrt(mean / n.shape[0])
    assert abs(n.var() / mean - 1.0) < 0.1


def test_vertex_z_is_a_truncated_gaussian():
    sigma, zmax = 0.053, 0.10  # a tight truncation so that redraws happen
    T = oracle.poisson_thresholds(30.0)
    z = np.concatenate([oracle.pileup_draws(_pu(30.0, sigma_z=sigma, max_z=zmax), T, 10, SEED, ev)[2]
                        for ev in range(600)])
    assert np.all(np.abs(z) <= zmax)
    ref = stats.truncnorm(-zmax / sigma, zmax / sigma, loc=0.0, scale=sigma)
    assert stats.kstest(z, ref.cdf).pvalue > 1e-4
    # first attempt: sigma times the Box-Muller normal of words 1, 2 of counter (k, event, 6, 0)
    n, idx, zz, tt, zhs, ths, m = oracle.pileup_draws(_pu(30.0, sigma_z=sigma, max_z=1.0), T, 10, SEED, 3)
    w = _words(0, 3, 6)
    assert zz[0] == pytest.approx(sigma * oracle.normal(int(w[1]), int(w[2])), rel=1e-15)


def test_vertex_time_is_a_truncated_gaussian_of_its_own_counters():
    """t = sigma_t x the normal of words 1, 2 of counter (k, event, 7, a),
    redrawn until |t| <= max_t: independent of z (its own counters), and a
    truncated normal by a KS test against scipy's."""
    st, mt = 160e-12, 200e-12  # a tight truncation so that redraws happen
    T = oracle.poisson_thresholds(30.0)
    z_all, t_all = [], []
    for ev in range(600):
        n, idx, z, t, zhs, ths, m = oracle.pileup_draws(_pu(30.0, sigma_t=st, max_t=mt), T, 10, SEED, ev)
        z_all.append(z)
        t_all.append(t)
    z, t = np.concatenate(z_all), np.concatenate(t_all)
    assert np.all(np.abs(t) <= mt * (1 + 1e-7))
    ref = stats.truncnorm(-mt / st, mt / st, loc=0.0, scale=st)
    assert stats.kstest(t, ref.cdf).pvalue > 1e-4
    assert abs(stats.pearsonr(z, t)[0]) < 5 / np.sqrt(z.shape[0])
    n, idx, z, t, zhs, ths, m = oracle.pileup_draws(_pu(30.0, max_t=1.0), T, 10, SEED, 5)
    w = _words(2, 5, 7)
    assert t[2] == pytest.approx(160e-12 * oracle.normal(int(w[1]), int(w[2])), rel=1e-15)
    # the hard-scatter time comes from counter (0, event, 8, 0) when accepted at once
    w = _words(0, 5, 8)
    assert ths == pytest.approx(160e-12 * oracle.normal(int(w[1]), int(w[2])), rel=1e-15)


def test_hard_vertex_smearing_switch():
    T = oracle.poisson_thresholds(5.0)
    on = [oracle.pileup_draws(_pu(5.0, smear=True), T, 10, SEED, ev) for ev in range(400)]
    off = [oracle.pileup_draws(_pu(5.0, smear=False), T, 10, SEED, ev) for ev in range(400)]
    assert all(d[4] == 0.0 and d[5] == 0.0 for d in off)
    assert np.std([d[4] for d in on]) == pytest.approx(0.053, rel=0.15)
    assert np.std([d[5] for d in on]) == pytest.approx(160e-12, rel=0.15)


def test_merged_events_are_hard_then_interactions_in_order():
    pool = synth.make_minbias_pool(300)
    hard = synth.make_hard(12)
    m = oracle.pileup_merge(hard, pool, 20.0, 0.053, 0.25, True, SEED)
    for e in range(hard.n_events):
        n, idx, z, t, zhs, ths = m["draws"][e]
        a, b = int(m["offsets"][e]), int(m["offsets"][e + 1])
        ev = hard.event(e)
        nh = len(ev["pt"])
        assert np.array_equal(m["pt"][a:a + nh], ev["pt"]) and np.array_equal(m["pdg"][a:a + nh], ev["pdg"])
        assert np.all(m["vz"][a:a + nh] == zhs) and np.all(m["vt"][a:a + nh] == ths)
        pos = a + nh
        for k in range(n):
            pe = pool.event(int(idx[k]))
            np_ = len(pe["pt"])
            for key in ("pt", "eta", "phi", "mass", "pdg", "charge"):
                assert np.array_equal(m[key][pos:pos + np_], pe[key])
            assert np.all(m["vz"][pos:pos + np_] == z[k]) and np.all(m["vt"][pos:pos + np_] == t[k])
            pos += np_
        assert pos == b


def test_no_pileup_leaves_the_hard_events():
    pool = synth.make_minbias_pool(50)
    hard = synth.make_hard(8)
    m = oracle.pileup_merge(hard, pool, 0.0, 0.053, 0.25, False, SEED)
    assert np.array_equal(m["offsets"], hard.offsets)
    assert np.array_equal(m["pt"], hard.pt) and np.all(m["vz"] == 0.0) and np.all(m["vt"] == 0.0)


def test_merging_does_not_depend_on_batching():
    pool = synth.make_minbias_pool(100)
    hard = synth.make_hard(10)
    whole = oracle.pileup_merge(hard, pool, 15.0, 0.053, 0.25, True, SEED)
    part = oracle.pileup_merge(hard.slice_events(3, 8), pool, 15.0, 0.053, 0.25, True, SEED, event_base=3)
    a, b = int(whole["offsets"][3]), int(whole["offsets"][8])
    for key in ("pt", "eta", "pdg", "vz", "vt"):
        assert np.array_equal(part[key], whole[key][a:b])


def test_forced_truncation_decision():
    """The parity protocol's forced branch of a truncation decision: with the
    bound set to exactly |v| of interaction 0's first vertex-z draw, that
    decision (|v| <= bound, taken in float32) is marginal and accepts; forced
    the other way, the draw is rejected and the vertex z is the next accepted
    attempt's value (attempt words recomputed from Philox here).  A decision
    that is not marginal, or one that never occurs, refuses to be forced."""
    sigma = 0.053
    T = oracle.poisson_thresholds(30.0)
    ev = 0
    for ev in range(50):  # an event with at least one interaction
        if oracle.pileup_draws(_pu(30.0), T, 100, SEED, ev)[0] > 0:
            break
    w0 = _words(0, ev, 6, 0)
    v0 = sigma * oracle.normal(int(w0[1]), int(w0[2]))
    bound = abs(v0)
    pu = _pu(30.0, smear=False, sigma_z=sigma, max_z=bound)
    marg = []
    k, _, z, _, _, _, m = oracle.pileup_draws(pu, T, 100, SEED, ev, marginal_out=marg)
    assert k > 0 and z[0] == v0 and (6, 0, 0) in marg
    _, _, zf, _, _, _, _ = oracle.pileup_draws(pu, T, 100, SEED, ev, flips=[(6, 0, 0)])
    nxt = None
    for a in range(1, 1000):
        w = _words(0, ev, 6, a)
        v = sigma * oracle.normal(int(w[1]), int(w[2]))
        if abs(np.float32(v)) <= np.float32(bound):
            nxt = v
            break
    assert zf[0] == nxt and zf[0] != z[0]
    assert np.array_equal(zf[1:], z[1:])  # other interactions untouched
    with pytest.raises(ValueError):
        oracle.pileup_draws(pu, T, 100, SEED, ev, flips=[(6, 1, 0)])       # interaction 1's first z: not marginal
    with pytest.raises(ValueError):
        oracle.pileup_draws(pu, T, 100, SEED, ev, flips=[(6, 0, 999999)])  # never drawn
