"""Pins of the oracle's simulated annealing (heat bath over the SU(2)
subgroups, readings R7-R11 of culgt_oracle.c).

The paper names simulated annealing combined with overrelaxation
(abstract, Sec. 1) but prints no formula for it, so every pin comes from the
mathematics: published test vectors of the random-number generator, the
exact heat-bath distribution of one SU(2) element (its mean is a ratio of
Bessel functions), its limits T -> 0 (the maximisation of Sec. 2) and
T -> infinity (Haar measure), the covariance of the draw, and the invariance
of the functional under the microcanonical (omega = 2) update.
"""
import numpy as np
import pytest
from scipy import integrate, special, stats

from paper_1412_3655_gb300 import synth

# Random123's known-answer vectors for Philox4x32-10 (Salmon et al., SC 2011):
# (counter, key) -> output
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(orc, ctr, key, want):
    assert orc.philox4x32_10(ctr, key) == want
    got = synth.philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
    assert tuple(int(x) for x in got) == want


def _delta_cdf(alpha):
    """Distribution function of delta = 1 - x0 for the density
    sqrt(delta (2 - delta)) exp(-alpha delta) on [0, 2], by quadrature on a
    grid delta = d_max t^2 (smooth in t)."""
    d_max = min(2.0, 80.0 / alpha)
    t = np.linspace(0.0, 1.0, 40001)
    d = d_max * t * t
    f = np.sqrt(np.clip(d * (2.0 - d), 0.0, None)) * np.exp(-alpha * d) * (2.0 * d_max * t)
    c = integrate.cumulative_trapezoid(f, t, initial=0.0)
    c /= c[-1]
    return lambda x: np.interp(x, d, c)


def _x0_moments(alpha):
    z = integrate.quad(lambda x: np.sqrt(1 - x * x) * np.exp(alpha * (x - 1)), -1, 1, limit=200)[0]
    m2 = integrate.quad(lambda x: x * x * np.sqrt(1 - x * x) * np.exp(alpha * (x - 1)), -1, 1, limit=200)[0]
    return m2 / z


# both sides of the Creutz / Kennedy-Pendleton boundary at alpha = 2
@pytest.mark.parametrize("alpha", [0.05, 0.7, 1.99, 2.0, 4.0, 30.0, 300.0])
def test_heatbath_x0_follows_the_exact_distribution(orc, alpha):
    """E[x0] = I_2(alpha) / I_1(alpha) and a Kolmogorov-Smirnov test against
    the exact distribution of delta = 1 - x0."""
    n = 20000
    d = np.array([orc.hb_delta(alpha, 99, s, 3, s % 3)[0] for s in range(n)])
    assert (d >= 0).all() and (d <= 2).all()
    x0 = 1.0 - d
    mean = special.ive(2, alpha) / special.ive(1, alpha)
    var = _x0_moments(alpha) - mean * mean
    assert abs(x0.mean() - mean) < 5 * np.sqrt(var / n)
    assert stats.kstest(d, _delta_cdf(alpha)).pvalue > 1e-3


@pytest.mark.parametrize("alpha", [0.3, 3.0, 50.0])
def test_heatbath_direction_is_isotropic_and_x_unit(orc, alpha):
    n = 6000
    x = np.array([orc.hb_x(alpha, 5, s, 0, 1) for s in range(n)])
    # delta and eps = 2 - delta come from separate logarithms: |x| = 1 to a few ulp
    assert np.abs(np.linalg.norm(x, axis=1) - 1).max() < 1e-15
    v = x[:, 1:]
    r2 = np.sum(v * v, axis=1)
    assert np.abs(v.mean(axis=0)).max() < 5 * np.sqrt(r2.mean() / 3 / n)
    # the second moments of the direction: r^2 / 3 each, no cross terms
    cov = (v.T @ v) / n
    assert np.abs(np.diag(cov) - r2.mean() / 3).max() < 6 * r2.mean() / 3 * np.sqrt(2 / n)
    assert np.abs(cov - np.diag(np.diag(cov))).max() < 6 * r2.mean() / 3 / np.sqrt(n)


def test_heatbath_attempts_are_bounded_and_reproducible(orc):
    for alpha in (1e-6, 1.0, 2.0, 1e4):
        for s in range(200):
            a = orc.hb_delta(alpha, 1, s, 7, 2)
            assert a == orc.hb_delta(alpha, 1, s, 7, 2)
            assert 1 <= a[1] <= 32
    # different counters give different draws
    assert orc.hb_delta(3.0, 1, 0, 0, 0) != orc.hb_delta(3.0, 1, 0, 1, 0)
    assert orc.hb_delta(3.0, 1, 0, 0, 0) != orc.hb_delta(3.0, 2, 0, 0, 0)


@pytest.mark.parametrize("nc", [2, 3])
def test_zero_temperature_heatbath_is_the_maximisation(orc, nc):
    """At T -> 0 the draw is x = 1 up to delta ~ T/(2k), so a heat-bath sweep
    equals an overrelaxation sweep at omega = 1 (Sec. 2)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 3)
    a = U.copy()
    orc.heatbath_sweep(a, dims, nc, 1e-24, 11, 0)
    b = U.copy()
    orc.sweep(b, dims, nc, 1.0, 1)
    assert np.abs(a - b).max() < 1e-9


@pytest.mark.parametrize("nc", [2, 3])
def test_infinite_temperature_heatbath_is_haar(orc, nc):
    """At T -> infinity every g(x) is Haar distributed: F of the links after
    one sweep averages to 0, and every link is special unitary."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 4)
    orc.heatbath_sweep(U, dims, nc, 1e9, 12, 0)
    th, F = orc.theta(U, dims, nc)
    n = 4 * int(np.prod(dims))
    # Re tr U / Nc of a link between two independent Haar elements has mean 0
    # and variance 1 / (2 Nc^2)
    assert abs(F) < 5 * np.sqrt(1.0 / (2 * nc * nc) / n)
    assert orc.unitarity_error(U, nc) < 1e-13


def test_su2_heatbath_is_covariant_at_the_updated_sites(orc):
    """SU(2): a gauge rotation h(x) at the sites being updated changes K(x) to
    h K(x), the maximiser to v h^+ and the draw to x v h^+; the new links
    x v h^+ h U are those without the rotation (same draws)."""
    dims = (4, 4, 2, 4)
    nc = 2
    U = synth.gauge_config(dims, nc, 0.4, 5)
    V = int(np.prod(dims))
    h = synth.haar(np.arange(V), nc, 77, synth.SLOT_G, 0)
    # canonical order i = x1 + L1 (x2 + L2 (x3 + L3 x0)): coordinates per site
    x0, x3, x2, x1 = np.unravel_index(np.arange(V), (dims[0], dims[3], dims[2], dims[1]))
    par = (x0 + x1 + x2 + x3) & 1
    g = np.where(par[:, None, None] == 0, h, np.eye(2)[None])  # rotate black sites only
    Uh = synth.gauge_transform(U, dims, g)
    a = U.copy()
    b = Uh.copy()
    for arr in (a, b):
        orc.heatbath_sweep(arr, dims, nc, 0.7, 21, 4)
    # the white half-sweep then starts from the same links in both
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_microcanonical_sweep_keeps_the_functional(orc, nc):
    """omega = 2 maps each subgroup element r to r^2, which keeps Re tr[r w]
    (Re tr[v^2 w] = 2k <v^2, v> = 2k v0): F and the plaquette do not change."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 6)
    th0, F0 = orc.theta(U, dims, nc)
    P0 = orc.plaquette(U, dims, nc)
    orc.micro_sweep(U, dims, nc)
    th1, F1 = orc.theta(U, dims, nc)
    assert F1 == pytest.approx(F0, abs=1e-13)
    assert abs(th1 - th0) > 1e-6  # the links did move
    assert orc.plaquette(U, dims, nc) == pytest.approx(P0, abs=1e-13)


def test_su2_microcanonical_halfsweep_is_an_involution(orc):
    """SU(2): r^2 K = k v, whose maximiser is v^+, so a second omega = 2
    half-sweep of the same parity restores the links."""
    dims = (4, 4, 4, 2)
    U = synth.gauge_config(dims, 2, 0.3, 8)
    a = U.copy()
    orc.halfsweep(a, dims, 2, 1, 2.0)
    assert np.abs(a - U).max() > 1e-3
    orc.halfsweep(a, dims, 2, 1, 2.0)
    assert np.abs(a - U).max() < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_anneal_schedule(orc, nc):
    """The schedule of R11 step by step: T linear in the step, draw counter =
    step, n_micro omega = 2 sweeps after each heat-bath sweep."""
    dims = (2, 4, 2, 4)
    U = synth.gauge_config(dims, nc, 0.3, 9)
    a = U.copy()
    orc.anneal(a, dims, nc, 1.2, 0.2, 3, 2, 31)
    b = U.copy()
    for k in range(3):
        orc.heatbath_sweep(b, dims, nc, 1.2 + (0.2 - 1.2) * k / 2, 31, k)
        for _ in range(2):
            orc.micro_sweep(b, dims, nc)
    assert np.array_equal(a, b)
    one = U.copy()
    orc.anneal(one, dims, nc, 0.9, 0.1, 1, 0, 31)
    c = U.copy()
    orc.heatbath_sweep(c, dims, nc, 0.9, 31, 0)
    assert np.array_equal(one, c)


@pytest.mark.parametrize("nc", [2, 3])
def test_anneal_keeps_plaquette_and_unitarity(orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 10)
    P0 = orc.plaquette(U, dims, nc)
    orc.anneal(U, dims, nc, 1.5, 0.05, 40, 2, 3, reunit_every=25)
    assert orc.plaquette(U, dims, nc) == pytest.approx(P0, abs=1e-12)
    assert orc.unitarity_error(U, nc) < 1e-13


def test_annealing_then_overrelaxation_finds_higher_maxima(orc):
    """The purpose of the combination (Sec. 1): starting from random gauge
    copies, annealing before overrelaxation ends on larger local maxima of F
    than overrelaxation alone (mean over copies; fixed seeds)."""
    dims = (4, 4, 4, 4)
    nc = 3
    plain, annealed = [], []
    for c in range(6):
        U = synth.gauge_config(dims, nc, 0.6, 1, copy=c)
        a = U.copy()
        r = orc.landau_fix(a, dims, nc, 1.7, 1e-12, 20000, 10, 50)
        plain.append(r["F"])
        b = U.copy()
        orc.anneal(b, dims, nc, 0.6, 0.01, 300, 3, 100 + c, reunit_every=50)
        r = orc.landau_fix(b, dims, nc, 1.7, 1e-12, 20000, 10, 50)
        assert r["converged"]
        annealed.append(r["F"])
    assert np.mean(annealed) > np.mean(plain)


@pytest.mark.parametrize("T", [0.3, 2.0, 9.0])
def test_su2_site_heatbath_samples_the_boltzmann_weight(orc, T):
    """For a fixed K = k v^+ (k > 0, v in SU(2)) the drawn g has
    Re tr[g K] = 2 k x0 with x0 distributed as sqrt(1 - x0^2) exp(alpha x0),
    alpha = 2 k / T: the weight exp(Re tr[g K] / T) over Haar measure."""
    rng = np.random.default_rng(4)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    k = 1.7
    K = k * np.array([[q[0] + 1j * q[3], q[2] + 1j * q[1]], [-q[2] + 1j * q[1], q[0] - 1j * q[3]]])
    n = 6000
    re = np.array([np.trace(orc.heatbath_gauge(K, T, 8, s, 2) @ K).real for s in range(n)])
    x0 = re / (2 * k)
    alpha = 2 * k / T
    mean = special.ive(2, alpha) / special.ive(1, alpha)
    var = _x0_moments(alpha) - mean * mean
    assert abs(x0.mean() - mean) < 5 * np.sqrt(var / n)
    assert stats.kstest(1 - x0, _delta_cdf(alpha)).pvalue > 1e-3


@pytest.mark.parametrize("nc", [2, 3])
def test_heatbath_sweep_draws_with_the_site_and_sweep_words(orc, nc):
    """R9: the update of site i in a heat-bath half-sweep is the single-site
    draw for its gathered K with counter words (i, sweep); other sweep words
    give other draws."""
    dims = (2, 4, 2, 4)
    U = synth.gauge_config(dims, nc, 0.3, 12)
    V = int(np.prod(dims))
    a = U.copy()
    orc.heatbath_sweep(a, dims, nc, 0.8, 41, 6)
    b = U.copy()
    orc.heatbath_sweep(b, dims, nc, 0.8, 41, 7)
    assert np.abs(a - b).max() > 1e-3
    # a black half-sweep: U_0(i) <- g(i) U_0(i) at black i (its forward
    # neighbour is white), with g(i) the draw for K(i) of the input links
    h = U.copy()
    orc.heatbath_halfsweep(h, dims, nc, 0, 0.8, 41, 6)
    x0, x3, x2, x1 = np.unravel_index(np.arange(V), (dims[0], dims[3], dims[2], dims[1]))
    black = np.flatnonzero(((x0 + x1 + x2 + x3) & 1) == 0)
    for i in black[:8]:
        K = np.zeros((nc, nc), dtype=complex)
        for mu in range(4):
            ib = int(np.flatnonzero(synth.site_neighbour_forward(dims, mu) == i)[0])
            K += U[i, mu] + U[ib, mu].conj().T
        g = orc.heatbath_gauge(K, 0.8, 41, int(i), 6)
        assert np.abs(h[i, 0] - g @ U[i, 0]).max() < 1e-14
        g_other = orc.heatbath_gauge(K, 0.8, 41, int(i) ^ 1, 6)
        assert np.abs(g_other - g).max() > 1e-3


@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_anneal_without_steps_is_coulomb_fix(orc, nc):
    dims = (4, 4, 4, 2)
    U = synth.gauge_config(dims, nc, 0.3, 5)
    a = U.copy()
    ra = orc.coulomb_fix_anneal(a, dims, nc, 0.6, 0.05, 0, 2, 9, 1.7, 1e-12, 3000, 5, 25)
    b = U.copy()
    rb = orc.coulomb_fix(b, dims, nc, 1.7, 1e-12, 3000, 5, 25)
    assert np.array_equal(a, b) and np.array_equal(ra["g"], rb["g"])
    assert list(ra["sweeps"]) == list(rb["sweeps"])


@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_anneal_is_one_gauge_transformation(orc, nc):
    """Annealing then overrelaxing every slice: the output is the input
    transformed by the returned g (spatial links rotated on the way, temporal
    links once at the end), every slice converges, the plaquette stays."""
    dims = (4, 4, 4, 2)
    U = synth.gauge_config(dims, nc, 0.5, 6)
    out = U.copy()
    r = orc.coulomb_fix_anneal(out, dims, nc, 0.6, 0.05, 20, 2, 9, 1.7, 1e-12, 5000, 5, 25)
    assert r["converged"] and (r["theta"] < 1e-12).all()
    assert np.abs(out - synth.gauge_transform(U, dims, r["g"])).max() < 1e-12
    assert orc.plaquette(out, dims, nc) == pytest.approx(orc.plaquette(U, dims, nc), abs=1e-12)
    for t in range(dims[0]):
        th, F = orc.theta_slice(out, dims, nc, t)
        assert th == pytest.approx(r["theta"][t], rel=1e-12) and F == pytest.approx(r["F"][t], rel=1e-14)


def test_coulomb_annealing_raises_the_slice_maxima(orc):
    """Rough field (eps 0.6): over 8 gauge copies the annealed slices end on
    larger maxima of F_t on average than overrelaxation alone."""
    dims = (2, 4, 4, 4)
    plain, ann = [], []
    for c in range(8):
        U = synth.gauge_config(dims, 3, 0.6, 3, copy=c)
        plain += list(orc.coulomb_fix(U.copy(), dims, 3, 1.7, 1e-12, 20000, 10, 50)["F"])
        ann += list(orc.coulomb_fix_anneal(U.copy(), dims, 3, 0.6, 0.01, 200, 3, 40 + c, 1.7, 1e-12, 20000, 10,
                                           50)["F"])
    assert np.mean(ann) > np.mean(plain)


@pytest.mark.parametrize("nc", [2, 3])
def test_heatbath_of_a_zero_K_is_the_identity(orc, nc):
    """k = 0 leaves every block alone (as the maximisation does, reading R4)."""
    g = orc.heatbath_gauge(np.zeros((nc, nc)), 0.7, 1, 0, 0)
    assert np.abs(g - np.eye(nc)).max() == 0
