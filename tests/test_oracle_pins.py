"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test pins a part of the oracle to something other than itself: a closed
form, brute-force maximisation, an exact symmetry, or a library routine. The
paper (Vogt & Schröck, cuLGT, Sec. 2) prints no worked numbers, so no test
compares with printed values.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_1412_3655_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

RNG = np.random.default_rng(20141211)


def haar_su2(n, rng=RNG):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return quat_to_mat(q)


def quat_to_mat(q):
    q = np.atleast_2d(q)
    a0, a1, a2, a3 = q.T
    m = np.empty((q.shape[0], 2, 2), dtype=np.complex128)
    m[:, 0, 0] = a0 + 1j * a3
    m[:, 0, 1] = a2 + 1j * a1
    m[:, 1, 0] = -a2 + 1j * a1
    m[:, 1, 1] = a0 - 1j * a3
    return m


def haar_su3(n, rng=RNG):
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / np.exp(1j * np.angle(det) / 3)[:, None, None]


def retr(a, b):
    """Re tr[a b] for stacks."""
    return np.real(np.einsum("...ij,...ji->...", a, b))


def assert_special_unitary(m, tol):
    n = m.shape[-1]
    eye = np.eye(n)
    assert np.abs(m @ np.swapaxes(m.conj(), -1, -2) - eye).max() < tol
    assert np.abs(np.linalg.det(m) - 1).max() < tol


# ---------------------------------------------------------------- SU(2) max


@pytest.mark.parametrize("seed", range(5))
def test_su2_closed_form_is_the_brute_force_maximum(orc, seed):
    """g = K^+/sqrt(det K^+) (Sec. 2) maximises Re tr[g K] over SU(2):
    Re tr[g K] = 2 sqrt(det K) and no Haar-random s does better."""
    rng = np.random.default_rng(seed)
    K = haar_su2(8, rng).sum(axis=0)
    g = orc.su2_local_max(K)
    assert_special_unitary(g[None], 1e-14)
    best = retr(g, K)
    assert best == pytest.approx(2 * np.sqrt(np.linalg.det(K).real), rel=1e-14)
    s = haar_su2(100_000, rng)
    assert retr(s, K[None]).max() <= best + 1e-12


def test_su2_max_of_a_general_block(orc):
    """For a general 2x2 complex block w the quaternion projection gives the
    SU(2) element maximising Re tr[r w] (brute force + local perturbation)."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        w = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        r = orc.su2_local_max(w)
        assert_special_unitary(r[None], 1e-14)
        best = retr(r, w)
        s = haar_su2(100_000, rng)
        assert retr(s, w[None]).max() <= best + 1e-12
        # second-order local check: rotations near r do not improve
        eps = haar_su2(2000, rng)
        small = np.array([scipy.linalg.fractional_matrix_power(e, 0.01) for e in eps[:200]])
        assert retr(small @ r, w[None]).max() <= best + 1e-12


def test_su2_degenerate_block_is_identity(orc):
    r = orc.su2_local_max(np.zeros((2, 2)))
    assert np.array_equal(r, np.eye(2))


# ---------------------------------------------------------------- SU(3) subgroups


@pytest.mark.parametrize("seed", range(4))
def test_su3_local_update_not_below_any_single_subgroup_maximum(orc, seed):
    """Each subgroup hit does not decrease Re tr[g K]; the first hit is the
    maximum over SU(2) in the (0,1) block, so the final g is at least as good
    as the best element of that subgroup, and at least as good as g = 1."""
    rng = np.random.default_rng(100 + seed)
    K = haar_su3(8, rng).sum(axis=0)
    g = orc.local_gauge(K, 1.0)
    assert_special_unitary(g[None], 1e-14)
    val = retr(g, K)
    assert val >= np.trace(K).real - 1e-12
    s = haar_su2(50_000, rng)
    emb = np.broadcast_to(np.eye(3, dtype=complex), (s.shape[0], 3, 3)).copy()
    emb[:, :2, :2] = s
    assert retr(emb, K[None]).max() <= val + 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_su3_last_subgroup_block_is_maximised(orc, seed):
    """After the (1,2) hit at omega = 1 the (1,2) block of g K has a quaternion
    part proportional to the identity with positive weight: no element of
    that subgroup improves Re tr[g K] further."""
    rng = np.random.default_rng(200 + seed)
    K = haar_su3(8, rng).sum(axis=0)
    g = orc.local_gauge(K, 1.0)
    gk = g @ K
    w = gk[1:, 1:]
    a0 = (w[0, 0] + w[1, 1]).real / 2
    a1 = (w[0, 1] + w[1, 0]).imag / 2
    a2 = (w[0, 1] - w[1, 0]).real / 2
    a3 = (w[0, 0] - w[1, 1]).imag / 2
    assert a0 > 0
    assert max(abs(a1), abs(a2), abs(a3)) < 1e-12 * abs(a0)


def test_su3_update_of_a_su2_embedded_K(orc):
    """K = 2 diag(s, 1) with s in SU(2): the first subgroup hit, on the (0,1)
    block, already reaches the global maximum g = diag(s^+, 1); the later hits
    then see identity blocks and leave it unchanged."""
    rng = np.random.default_rng(3)
    for s in haar_su2(5, rng):
        K = np.eye(3, dtype=complex) * 2.0
        K[:2, :2] = 2.0 * s
        g = orc.local_gauge(K, 1.0)
        expected = np.eye(3, dtype=complex)
        expected[:2, :2] = s.conj().T
        assert np.abs(g - expected).max() < 1e-14


# ---------------------------------------------------------------- overrelaxation


@pytest.mark.parametrize("variant", [0, 1])
def test_overrelax_is_identity_at_omega_one(orc, variant):
    for r in haar_su2(20):
        assert np.abs(orc.overrelax(r, 1.0, variant) - r).max() < 2e-15


def _angle_axis(m):
    c0 = (m[0, 0] + m[1, 1]).real / 2
    v = np.array([(m[0, 1] + m[1, 0]).imag / 2, (m[0, 1] - m[1, 0]).real / 2, (m[0, 0] - m[1, 1]).imag / 2])
    s = np.linalg.norm(v)
    return np.arctan2(s, c0), v / s


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("omega", [1.3, 1.7, 1.95])
def test_overrelax_small_angle_ratio(orc, variant, omega):
    """g^omega rotates about the same axis by omega times the angle, as the
    angle goes to zero (both variants)."""
    axis = np.array([0.3, -0.5, 0.81])
    axis /= np.linalg.norm(axis)
    for phi in [1e-2, 1e-3, 1e-4]:
        q = np.concatenate([[np.cos(phi)], np.sin(phi) * axis])
        r = quat_to_mat(q)[0]
        out = orc.overrelax(r, omega, variant)
        assert_special_unitary(out[None], 1e-14)
        ang, ax = _angle_axis(out)
        assert np.abs(ax - axis).max() < 1e-10
        assert ang / phi == pytest.approx(omega, abs=10 * phi ** 2 + 1e-9)


def test_overrelax_exact_matches_matrix_power(orc):
    for r in haar_su2(20):
        for omega in (1.25, 1.7, 1.9):
            ref = scipy.linalg.fractional_matrix_power(r, omega)
            assert np.abs(orc.overrelax(r, omega, 1) - ref).max() < 1e-12


def test_overrelax_truncated_is_second_order(orc):
    """The truncated series differs from the exact power at third order in the
    angle: halving the angle divides the gap by about 8. A dropped or
    mis-signed second-order term would give a gap of second order."""
    axis = np.array([0.6, 0.0, 0.8])
    for omega in (1.5, 1.7):
        gaps = []
        for phi in (0.08, 0.04, 0.02):
            r = quat_to_mat(np.concatenate([[np.cos(phi)], np.sin(phi) * axis]))[0]
            ref = scipy.linalg.fractional_matrix_power(r, omega)
            gaps.append(np.abs(orc.overrelax(r, omega, 0) - ref).max())
        assert 7.0 < gaps[0] / gaps[1] < 9.0
        assert 7.0 < gaps[1] / gaps[2] < 9.0


def _binomial_series(g, omega, order):
    """sum_{n <= order} binom(omega, n) (g - 1)^n, the series of g^omega."""
    from scipy.special import binom
    D = g - np.eye(2)
    term = np.eye(2, dtype=complex)
    out = np.zeros((2, 2), dtype=complex)
    for n in range(order + 1):
        out = out + binom(omega, n) * term
        term = term @ D
    return out


def test_overrelax_truncated_is_the_second_order_binomial_series(orc):
    """Variant 0 is the binomial series of g^omega cut after (g-1)^2 and put
    back on SU(2). The series itself is checked to converge to the library's
    fractional matrix power, so its coefficients are pinned; cutting it at
    first or third order gives a different element at finite angle."""
    rng = np.random.default_rng(12)
    for _ in range(10):
        # angles below 0.7 keep |g - 1| < 0.7, where the series converges fast
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        phi = rng.uniform(0.05, 0.7)
        g = quat_to_mat(np.concatenate([[np.cos(phi)], np.sin(phi) * axis]))[0]
        for omega in (1.3, 1.7, 1.95):
            full = _binomial_series(g, omega, 200)
            assert np.abs(full - scipy.linalg.fractional_matrix_power(g, omega)).max() < 1e-10
            cut = {k: _binomial_series(g, omega, k) for k in (1, 2, 3)}
            cut = {k: v / np.sqrt(np.linalg.det(v)) for k, v in cut.items()}
            got = orc.overrelax(g, omega, 0)
            assert np.abs(got - cut[2]).max() < 1e-14
            assert np.abs(got - cut[1]).max() > 1e-6
            assert np.abs(got - cut[3]).max() > 1e-6


# ---------------------------------------------------------------- theta, F, plaquette


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 4, 6, 2)])
def test_theta_F_trivial_field(orc, nc, L):
    V = int(np.prod(L))
    U = np.broadcast_to(np.eye(nc, dtype=complex), (V, 4, nc, nc)).copy()
    th, F = orc.theta(U, L, nc)
    assert th == 0.0
    assert F == 1.0
    assert orc.plaquette(U, L, nc) == 1.0


def _single_link(L, nc, eps, site, mu):
    V = int(np.prod(L))
    U = np.broadcast_to(np.eye(nc, dtype=complex), (V, 4, nc, nc)).copy()
    diag = np.ones(nc, dtype=complex)
    diag[0], diag[1] = np.exp(1j * eps), np.exp(-1j * eps)  # exp(i eps sigma_3) / exp(i eps lambda_3)
    U[site, mu] = np.diag(diag)
    return U


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("eps", [0.1, 0.7, 2.0])
@pytest.mark.parametrize("L,site,mu", [((4, 4, 4, 4), 0, 0), ((2, 4, 6, 2), 17, 2), ((4, 2, 2, 6), 5, 1)])
def test_theta_F_plaquette_single_link_closed_forms(orc, nc, eps, L, site, mu):
    """One link exp(i eps T3), the rest 1: theta = 4 sin^2(eps)/V,
    F = 1 - (2 - 2 cos eps)/(Nd Nc V), P = 1 - (2 - 2 cos eps)/(Nc V)."""
    V = int(np.prod(L))
    U = _single_link(L, nc, eps, site, mu)
    th, F = orc.theta(U, L, nc)
    assert th == pytest.approx(4 * np.sin(eps) ** 2 / V, rel=1e-13)
    assert F == pytest.approx(1 - (2 - 2 * np.cos(eps)) / (4 * nc * V), rel=1e-14)
    P = orc.plaquette(U, L, nc)
    assert P == pytest.approx(1 - (2 - 2 * np.cos(eps)) / (nc * V), rel=1e-14)


@pytest.mark.parametrize("nc", [2, 3])
def test_theta_is_the_squared_gradient_of_F(orc, nc):
    """tr[Delta(y)^2] = sum_a (dRe tr[g(y) K(y)]/dt)^2 with g(y) = exp(i t X_a),
    X_a an orthonormal basis of traceless Hermitian matrices: theta is the
    squared gradient of the functional F of Sec. 2, taken here by central
    differences of F alone."""
    L = (2, 2, 2, 4)
    V = int(np.prod(L))
    U = synth.gauge_config(L, nc, 0.4, 11)
    th, _ = orc.theta(U, L, nc)
    X = synth.generators(nc) / np.sqrt(2.0)
    h = 1e-5
    total = 0.0
    for y in range(V):
        for Xa in X:
            vals = []
            for t in (h, -h):
                g = np.broadcast_to(np.eye(nc, dtype=complex), (V, nc, nc)).copy()
                g[y] = scipy.linalg.expm(1j * t * Xa)
                _, F = orc.theta(np.ascontiguousarray(synth.gauge_transform(U, L, g)), L, nc)
                vals.append(F)
            d = (vals[0] - vals[1]) / (2 * h) * (4 * nc * V)
            total += d * d
    assert th == pytest.approx(total / V, rel=1e-7)


@pytest.mark.parametrize("nc", [2, 3])
def test_plaquette_gauge_invariant_and_pure_gauge(orc, nc):
    L = (4, 2, 4, 2)
    U = synth.gauge_config(L, nc, 0.5, 21)
    P = orc.plaquette(U, L, nc)
    g = synth.random_gauge(L, nc, 99, 3)
    Ug = np.ascontiguousarray(synth.gauge_transform(U, L, g))
    assert orc.plaquette(Ug, L, nc) == pytest.approx(P, abs=1e-14)
    assert orc.plaquette(synth.pure_gauge(L, nc, 5), L, nc) == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------- the sweep


@pytest.mark.parametrize("nc", [2, 3])
def test_F_non_decreasing_at_omega_one(orc, nc):
    """Each site update maximises its own local term (Sec. 2), so at omega = 1
    F never decreases, half-sweep by half-sweep."""
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, nc, 0.3, 1)
    _, F = orc.theta(U, L, nc)
    for _ in range(6):
        for p in (0, 1):
            orc.halfsweep(U, L, nc, p, 1.0)
            _, Fn = orc.theta(U, L, nc)
            assert Fn >= F - 1e-15
            F = Fn


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_sweeps_keep_plaquette_and_unitarity(orc, nc, omega):
    L = (4, 4, 2, 6)
    U = synth.gauge_config(L, nc, 0.3, 2)
    P = orc.plaquette(U, L, nc)
    orc.sweep(U, L, nc, omega, 10)
    assert orc.plaquette(U, L, nc) == pytest.approx(P, abs=1e-12)
    assert orc.unitarity_error(U, nc) < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_su2_halfsweep_reaches_the_local_maximum(orc):
    """SU(2), omega = 1: after a half-sweep every active site sits at its local
    maximum, so repeating the same half-sweep changes nothing."""
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, 2, 0.3, 3)
    for p in (0, 1):
        orc.halfsweep(U, L, 2, p, 1.0)
        before = U.copy()
        orc.halfsweep(U, L, 2, p, 1.0)
        assert np.abs(U - before).max() < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_sweep_is_covariant_under_global_rotations(orc, nc):
    """A constant h maps K(x) to h K(x) h^+, so sweep(U^h) = sweep(U)^h: for
    SU(2) for every h, for SU(3) for h in the maximal torus (diagonal phases),
    which maps each SU(2) subgroup into itself."""
    L = (4, 2, 4, 4)
    V = int(np.prod(L))
    U = synth.gauge_config(L, nc, 0.3, 4)
    rng = np.random.default_rng(77)
    if nc == 2:
        h0 = haar_su2(1, rng)[0]
    else:
        a = rng.uniform(-np.pi, np.pi, 2)
        h0 = np.diag([np.exp(1j * a[0]), np.exp(1j * a[1]), np.exp(-1j * a.sum())])
    h = np.broadcast_to(h0, (V, nc, nc))
    Uh = np.ascontiguousarray(synth.gauge_transform(U, L, h))
    orc.sweep(U, L, nc, 1.7, 2)
    orc.sweep(Uh, L, nc, 1.7, 2)
    assert np.abs(Uh - synth.gauge_transform(U, L, h)).max() < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_sweep_is_translation_covariant(orc, nc):
    """Shifting the lattice by an even vector keeps the checkerboard, so it
    commutes with a sweep."""
    L = (4, 4, 2, 6)
    U = synth.gauge_config(L, nc, 0.3, 5)
    shape = (L[0], L[3], L[2], L[1], 4, nc, nc)  # canonical order: x0 slowest, x1 fastest

    def shift(a):
        return np.ascontiguousarray(np.roll(a.reshape(shape), (2, 2, 0, 0), axis=(0, 3, 2, 1)).reshape(U.shape))

    Us = shift(U)
    orc.sweep(U, L, nc, 1.7, 2)
    orc.sweep(Us, L, nc, 1.7, 2)
    assert np.abs(Us - shift(U)).max() < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_pure_gauge_converges_to_F_one(orc, nc):
    """U = g(x) g(x+mu)^+ with g near 1: the iteration reaches theta -> 0 and F -> 1."""
    L = (4, 4, 4, 4)
    U = synth.pure_gauge(L, nc, 6, spread=0.5)
    r = orc.landau_fix(U, L, nc, 1.7, 1e-24, 3000, 10)
    assert r["converged"]
    assert r["F"] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("nc", [2, 3])
def test_landau_fix_contract(orc, nc):
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, nc, 0.3, 1)
    P = orc.plaquette(U, L, nc)
    r = orc.landau_fix(U, L, nc, 1.7, 1e-12, 2000, 5, 20)
    assert r["converged"] and r["sweeps"] % 5 == 0 and r["theta"] < 1e-12
    assert orc.theta(U, L, nc) == (r["theta"], r["F"])
    assert orc.plaquette(U, L, nc) == pytest.approx(P, abs=1e-12)
    U = synth.gauge_config(L, nc, 0.3, 1)
    r = orc.landau_fix(U, L, nc, 1.7, 1e-30, 7, 5, 0)
    assert not r["converged"] and r["sweeps"] == 7


# ---------------------------------------------------------------- reunitarisation


@pytest.mark.parametrize("nc", [2, 3])
def test_reunitarize_idempotent_and_third_row(orc, nc):
    M = haar_su3(50) if nc == 3 else haar_su2(50)
    R = M.copy()
    orc.reunitarize(R, nc)
    assert np.abs(R - M).max() < 1e-15
    noisy = M + 1e-6 * (RNG.standard_normal(M.shape) + 1j * RNG.standard_normal(M.shape))
    orc.reunitarize(noisy, nc)
    assert_special_unitary(noisy, 1e-15)
    if nc == 3:
        broken = M.copy()
        broken[:, 2, :] = 7.0  # discarded third row (12-real storage)
        orc.reunitarize(broken, 3)
        assert np.abs(broken - M).max() < 1e-15


# ---------------------------------------------------------------- Coulomb


def test_coulomb_theta_single_spatial_link(orc):
    L = (4, 4, 2, 2)
    V3 = 16
    U = _single_link(L, 3, 0.4, 2 * V3 + 3, 2)
    th, F = orc.theta_slice(U, L, 3, 2)
    assert th == pytest.approx(4 * np.sin(0.4) ** 2 / V3, rel=1e-13)
    assert F == pytest.approx(1 - (2 - 2 * np.cos(0.4)) / (3 * 3 * V3), rel=1e-14)
    assert orc.theta_slice(U, L, 3, 1) == (0.0, 1.0)


@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_fix_is_one_gauge_transformation(orc, nc):
    """Every slice converges on its own theta_t, and the result is the input
    gauge-transformed by the accumulated g (temporal links included)."""
    L = (4, 4, 4, 2)
    U0 = synth.gauge_config(L, nc, 0.3, 5)
    U = U0.copy()
    r = orc.coulomb_fix(U, L, nc, 1.7, 1e-12, 3000, 1, 25)
    assert r["converged"]
    for t in range(L[0]):
        th, F = orc.theta_slice(U, L, nc, t)
        assert th < 1e-12 and th == r["theta"][t] and F == r["F"][t]
    assert_special_unitary(r["g"], 1e-13)
    assert np.abs(U - synth.gauge_transform(U0, L, r["g"])).max() < 1e-12
    assert orc.plaquette(U, L, nc) == pytest.approx(orc.plaquette(U0, L, nc), abs=1e-12)
