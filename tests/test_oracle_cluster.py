"""Pins of the oracle's jet clustering (Sec. 2.4: FastJet's generalized-kT
family, anti-kT by default, on the PFlow collection, with jet pT and
constituent-count cuts).

Expected values come from hand-worked events and from properties of the
algorithms that do not restate the oracle's loop: four-momentum
conservation, the kT algorithm with a radius spanning the whole acceptance
(one jet: the event's total four-momentum), the anti-kT cone property
(isolated hard particles absorb the soft particles around them), the
Cambridge/Aachen two-particle threshold dR < R, and collinear safety; for
the substructure C2 and D2, the two-prong closed form (e3 = 0), the
equilateral three-prong jet (D2 = 1, C2 = a / 3) and rotation invariance;
for the e+e- variant, the opening-angle threshold of p = 0, back-to-back
sprays, and invariance under 3D rotations.
"""
import math

import numpy as np
import pytest

import oracle


def _fm(pt, eta, phi, m=None):
    pt, eta, phi = (np.asarray(x, np.float64) for x in (pt, eta, phi))
    m = np.zeros_like(pt) if m is None else np.asarray(m, np.float64)
    e = np.sqrt((pt * np.cosh(eta)) ** 2 + m ** 2)
    return oracle.four_momenta(pt, eta, phi, e)


def _random_event(rng, n):
    pt = 0.5 * (1 - rng.random(n)) ** (-1 / 2.5)
    eta = rng.uniform(-4, 4, n)
    phi = rng.uniform(-math.pi, math.pi, n)
    m = rng.choice([0.0, 0.13957, 0.49368], n)
    return _fm(pt, eta, phi, m)


def test_hand_worked_event():
    """Two massless particles at dR = 0.1 (pT 10 and 20) and a third 2 units
    away: anti-kT R = 0.4 gives the pair, then the loner.  The pair's mass is
    sqrt(2 pT1 pT2 (cosh 0.1 - 1)) = 1.414803."""
    jets, marg = oracle.cluster(*_fm([10, 20, 5], [0, 0.1, 2], [0, 0, 1]), p=-1, R=0.4)
    assert marg == 0 and len(jets) == 2
    assert jets[0]["pt"] == pytest.approx(30.0, abs=1e-12) and jets[0]["nconst"] == 2
    assert jets[0]["mass"] == pytest.approx(math.sqrt(400 * (math.cosh(0.1) - 1)), rel=1e-9)
    assert jets[0]["eta"] == pytest.approx(math.asinh(20 * math.sinh(0.1) / 30), rel=1e-12)
    assert jets[1]["pt"] == pytest.approx(5.0, abs=1e-12) and jets[1]["eta"] == pytest.approx(2.0, abs=1e-12)
    # pT and constituent cuts
    assert len(oracle.cluster(*_fm([10, 20, 5], [0, 0.1, 2], [0, 0, 1]), p=-1, R=0.4, pt_min=6)[0]) == 1
    assert len(oracle.cluster(*_fm([10, 20, 5], [0, 0.1, 2], [0, 0, 1]), p=-1, R=0.4, nconst_min=2)[0]) == 1


@pytest.mark.parametrize("p", [-1.0, 0.0, 1.0])
def test_four_momentum_is_conserved(p):
    rng = np.random.default_rng(int(10 + p))
    fm = _random_event(rng, 120)
    jets, _ = oracle.cluster(*fm, p=p, R=0.5)
    for k, key in enumerate(("px", "py", "pz", "e")):
        assert jets[key].sum() == pytest.approx(fm[k].sum(), rel=1e-10, abs=1e-9)
    assert jets["nconst"].sum() == 120
    assert np.all(np.diff(jets["pt"]) <= 0)


def test_kt_with_a_radius_spanning_everything_gives_one_jet():
    """|y| < 4 and |dphi| <= pi: every dR^2 < 64 + pi^2 < R^2 for R = 9, so
    d_ij < d_iB for every pair and all objects end in one jet."""
    rng = np.random.default_rng(3)
    fm = _random_event(rng, 60)
    jets, _ = oracle.cluster(*fm, p=1.0, R=9.0)
    assert len(jets) == 1 and jets[0]["nconst"] == 60
    assert jets[0]["pt"] == pytest.approx(math.hypot(fm[0].sum(), fm[1].sum()), rel=1e-12)


def test_anti_kt_cones_around_isolated_hard_particles():
    """Hard particles (pT 100) 2 units apart; soft ones (pT <= 1) within
    R / 2 of one hard particle each: every jet is one hard particle plus its
    soft neighbours (the textbook cone property of anti-kT)."""
    rng = np.random.default_rng(5)
    hard_eta = np.array([-2.0, 0.0, 2.0])
    hard_phi = np.array([0.0, 2.0, -2.0])
    pt, eta, phi, owner = list(100.0 + 10 * np.arange(3)), list(hard_eta), list(hard_phi), [0, 1, 2]
    for h in range(3):
        for _ in range(15):
            r, a = 0.2 * math.sqrt(rng.random()), rng.uniform(0, 2 * math.pi)
            pt.append(rng.uniform(0.1, 1.0)); eta.append(hard_eta[h] + r * math.cos(a))
            phi.append(hard_phi[h] + r * math.sin(a)); owner.append(h)
    fm = _fm(pt, eta, phi)
    jets, marg = oracle.cluster(*fm, p=-1.0, R=0.4)
    assert len(jets) == 3 and marg == 0
    owner = np.array(owner)
    for h in range(3):
        sel = owner == h
        j = jets[2 - h]   # ordered by decreasing pT: the hardest seed is h = 2
        assert j["nconst"] == 16
        for k, key in enumerate(("px", "py", "pz", "e")):
            assert j[key] == pytest.approx(fm[k][sel].sum(), rel=1e-12)


def test_cambridge_pair_threshold():
    """p = 0: d_ij = dR^2 / R^2 against d_iB = 1, so two particles merge iff
    dR < R."""
    for dr, merged in ((0.39, True), (0.41, False)):
        jets, _ = oracle.cluster(*_fm([5, 7], [0.3, 0.3 + dr], [1.0, 1.0]), p=0.0, R=0.4)
        assert (len(jets) == 1) == merged


@pytest.mark.parametrize("p", [-1.0, 0.0, 1.0])
def test_collinear_safety(p):
    """Splitting one particle into two collinear halves leaves the jets."""
    rng = np.random.default_rng(8)
    pt = 0.5 * (1 - rng.random(40)) ** (-1 / 2.5)
    eta = rng.uniform(-3, 3, 40)
    phi = rng.uniform(-math.pi, math.pi, 40)
    base, _ = oracle.cluster(*_fm(pt, eta, phi), p=p, R=0.5)
    k = int(np.argmax(pt))
    pt2 = np.concatenate([pt, [0.5 * pt[k]]])
    pt2[k] *= 0.5
    split, _ = oracle.cluster(*_fm(pt2, np.concatenate([eta, [eta[k]]]), np.concatenate([phi, [phi[k]]])),
                              p=p, R=0.5)
    assert len(split) == len(base)
    for key in ("px", "py", "pz", "e"):
        assert np.allclose(np.sort(split[key]), np.sort(base[key]), rtol=1e-10, atol=1e-9)


def test_symmetric_configuration_is_marginal():
    """Two equal particles at the same distance from a third: the first merge
    is a tie, which the oracle reports as marginal."""
    jets, marg = oracle.cluster(*_fm([10, 3, 3], [0.0, 0.2, -0.2], [0.0, 0.0, 0.0]), p=-1.0, R=0.4)
    assert marg >= 1 and len(jets) == 1


def test_two_prong_energy_correlations():
    """Two massless constituents at dR = 0.3 with pT 30 and 10: z = 3/4, 1/4,
    e2 = (3/16) 0.3 = 0.05625, e3 = 0, C2 = D2 = 0."""
    jets, _ = oracle.cluster(*_fm([30, 10], [0.5, 0.8], [1.0, 1.0]), p=-1.0, R=0.5)
    assert len(jets) == 1
    assert jets[0]["e2"] == pytest.approx(0.05625, rel=1e-12)
    assert jets[0]["e3"] == 0.0 and jets[0]["c2"] == 0.0 and jets[0]["d2"] == 0.0


def test_equilateral_three_prong_has_d2_one():
    """Three equal-pT massless constituents on an equilateral triangle of side
    a in (y, phi): z = 1/3, e2 = 3 a / 9, e3 = a^3 / 27, so C2 = a / 3 and
    D2 = 1."""
    a = 0.2
    eta = [0.0, a, a / 2]
    phi = [0.0, 0.0, a * math.sqrt(3) / 2]
    jets, _ = oracle.cluster(*_fm([20, 20, 20], eta, phi), p=-1.0, R=0.5)
    assert len(jets) == 1 and jets[0]["nconst"] == 3
    assert jets[0]["e2"] == pytest.approx(a / 3, rel=1e-12)
    assert jets[0]["e3"] == pytest.approx(a ** 3 / 27, rel=1e-12)
    assert jets[0]["c2"] == pytest.approx(a / 3, rel=1e-12)
    assert jets[0]["d2"] == pytest.approx(1.0, rel=1e-12)


def test_substructure_is_rotation_invariant():
    rng = np.random.default_rng(12)
    pt = rng.uniform(1, 20, 30)
    eta = rng.normal(0.3, 0.15, 30)
    phi = rng.normal(1.0, 0.15, 30)
    j0, _ = oracle.cluster(*_fm(pt, eta, phi), p=-1.0, R=0.6)
    j1, _ = oracle.cluster(*_fm(pt, eta, phi + 1.7), p=-1.0, R=0.6)
    assert len(j0) == len(j1)
    for key in ("e2", "e3", "c2", "d2"):
        assert np.allclose(j0[key], j1[key], rtol=1e-10, atol=1e-14)


def _dir_fm(E, dirs):
    """Massless four-momenta of energies E along unit vectors dirs."""
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1)[:, None]
    E = np.asarray(E, np.float64)
    return E * d[:, 0], E * d[:, 1], E * d[:, 2], E


@pytest.mark.parametrize("theta,merged", [(0.49, True), (0.51, False)])
def test_ee_cambridge_angle_threshold(theta, merged):
    """e+e- with p = 0: d_ij = (1 - cos theta) / (1 - cos R) against d_iB = 1,
    so two particles merge iff their opening angle is below R."""
    jets, _ = oracle.cluster(*_dir_fm([10, 7], [[1, 0, 0], [math.cos(theta), math.sin(theta), 0]]),
                             p=0.0, R=0.5, ee=True)
    assert (len(jets) == 1) == merged


def test_ee_back_to_back_sprays_and_conservation():
    """Two sprays around opposite directions (opening angles below R / 2):
    the e+e- anti-kT gives two jets, each the sum of its spray; the
    four-momentum of the event is conserved."""
    rng = np.random.default_rng(21)
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    dirs, E, owner = [], [], []
    for side in (1.0, -1.0):
        for _ in range(12):
            v = side * axis + rng.normal(0, 0.08, 3)
            dirs.append(v); E.append(rng.uniform(0.5, 8.0)); owner.append(side)
    fm = _dir_fm(E, dirs)
    jets, _ = oracle.cluster(*fm, p=-1.0, R=0.7, ee=True)
    assert len(jets) == 2 and sorted(jets["nconst"]) == [12, 12]
    owner = np.array(owner)
    for j in jets:
        side = 1.0 if j["px"] * axis[0] + j["py"] * axis[1] + j["pz"] * axis[2] > 0 else -1.0
        sel = owner == side
        assert j["e"] == pytest.approx(fm[3][sel].sum(), rel=1e-12)
        assert j["px"] == pytest.approx(fm[0][sel].sum(), rel=1e-10, abs=1e-12)


def test_ee_rotation_invariance():
    """The e+e- distances depend on energies and opening angles only: a 3D
    rotation of the event rotates the jets and keeps their energies."""
    rng = np.random.default_rng(22)
    n = 40
    dirs = rng.normal(0, 1, (n, 3))
    E = rng.exponential(4.0, n) + 0.2
    fm = _dir_fm(E, dirs)
    a, b = 0.7, -1.1
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    rot = Rx @ Rz
    p3 = np.stack(fm[:3], axis=1) @ rot.T
    j0, _ = oracle.cluster(*fm, p=1.0, R=0.8, ee=True)
    j1, _ = oracle.cluster(p3[:, 0], p3[:, 1], p3[:, 2], fm[3], p=1.0, R=0.8, ee=True)
    assert len(j0) == len(j1)
    assert np.allclose(np.sort(j0["e"]), np.sort(j1["e"]), rtol=1e-10)
    assert sorted(j0["nconst"]) == sorted(j1["nconst"])


def test_forced_runner_up_at_a_tie():
    """The parity protocol's forced branch.  Two soft particles at equal
    distance 0.35 on either side of a hard one, with R = 0.5 anti-kT, and a
    third soft particle 0.65 from the hard one: the first step is a tie
    between merging the left and the right soft particle (d = pT_hard^-2
    0.35^2 / R^2 for both).  Unforced, the lower index wins; forced, the other
    pair is merged first.  Both runs end in the same jets (the cone around
    the hard particle takes both soft particles; the third stays a jet of its
    own), while a step that is not a tie cannot be forced.  Without forced
    steps the result equals the plain call."""
    fm = _fm([100.0, 2.0, 2.0, 1.0], [0.0, -0.35, 0.35, 0.65], [0.0, 0.0, 0.0, 0.0])
    plain, m0 = oracle.cluster(*fm, p=-1.0, R=0.5)
    j0, steps = oracle.cluster_forced(*fm, p=-1.0, R=0.5)
    assert np.array_equal(plain, j0) and m0 == len(steps) >= 1 and steps[0] == 0
    j1, steps1 = oracle.cluster_forced(*fm, p=-1.0, R=0.5, flips=[0])
    assert len(j1) == len(j0) == 2 and list(j0["nconst"]) == [3, 1] == list(j1["nconst"])
    for k in ("px", "py", "pz", "e"):
        assert j1[0][k] == pytest.approx(j0[0][k], rel=1e-12, abs=1e-12)
    with pytest.raises(ValueError):
        oracle.cluster_forced(*fm, p=-1.0, R=0.5, flips=[len(fm[0]) - 1 + 5])  # beyond the last step
    # a clear (non-marginal) step refuses to be forced
    clear = _fm([100.0, 2.0, 2.0], [0.0, 0.1, 0.4], [0.0, 0.0, 0.0])
    _, st = oracle.cluster_forced(*clear, p=-1.0, R=0.5)
    assert 0 not in st
    with pytest.raises(ValueError):
        oracle.cluster_forced(*clear, p=-1.0, R=0.5, flips=[0])


def test_forced_runner_up_changes_a_split():
    """Where the tie decides the result: three equal-pT particles on a line at
    spacing 0.4 with Cambridge/Aachen R = 0.5.  The first step merges the left
    pair (lower indices win the tie); the merged axis then lies 0.6 from the
    third, so two jets: (left pair) + right.  Forcing the runner-up merges the
    right pair first: (right pair) + left.  The jets' constituent counts are
    both (2, 1) but the 2-constituent jet sits on the other side, mirrored."""
    fm = _fm([5.0, 5.0, 5.0], [-0.4, 0.0, 0.4], [0.0, 0.0, 0.0])
    j0, steps = oracle.cluster_forced(*fm, p=0.0, R=0.5)
    assert 0 in steps
    j1, _ = oracle.cluster_forced(*fm, p=0.0, R=0.5, flips=[0])
    two0 = j0[j0["nconst"] == 2][0]
    two1 = j1[j1["nconst"] == 2][0]
    assert two0["eta"] < -0.19 and two1["eta"] == pytest.approx(-two0["eta"], rel=1e-12)


def test_objects_with_only_infinite_distances_become_jets():
    """With p < 0 an object of pT = 0 has d_iB = pT^(2p) = infinity, and so has
    every pair distance among such objects: by the tie rule (the beam
    distance first, then the lowest index) each leaves as a jet of its own,
    after the finite-distance object has left."""
    px = np.array([0.0, 0.0, 10.0])
    py = np.array([0.0, 0.0, 0.0])
    pz = np.array([3.0, -4.0, 1.0])
    e = np.sqrt(px ** 2 + py ** 2 + pz ** 2)
    jets, _ = oracle.cluster(px, py, pz, e, p=-1.0, R=0.5, pt_min=0.0, nconst_min=1)
    assert len(jets) == 3 and list(jets["nconst"]) == [1, 1, 1]
    assert jets[0]["pt"] == pytest.approx(10.0)
