"""Pins of the oracle's first-order error bounds (the per-link tolerances of
the GPU parity tests rest on them).

The bounds say how far a sweep can move each link when its inputs and its
arithmetic carry small errors; a site whose local problem is nearly singular
(a short block quaternion in Sec. 2's maximiser, a MAG block vector near -e3)
amplifies them. They are pinned against the oracle's own response, measured
without them: the exact Jacobian of the site transformation by central
differences, and whole sweeps of perturbed inputs. A bound that dropped a
factor or a term of its derivation would fall below that response somewhere.
"""
import ctypes

import numpy as np
import pytest

import parity as P
from paper_1412_3655_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def gathered_K(U, L):
    """K(x) = sum_mu [U_mu(x) + U_mu(x - mu)^+] for every site."""
    K = U.sum(axis=1)
    for mu in range(4):
        K = K + np.conj(np.swapaxes(U[P.shifted(L, mu, -1), mu], -1, -2))
    return K


def jacobian_norm(f, M, h=1e-7):
    """Largest singular value of the real Jacobian of f at M (central differences)."""
    cols = []
    for idx in np.ndindex(M.shape):
        for z in (1.0, 1j):
            dM = np.zeros(M.shape, dtype=complex)
            dM[idx] = z * h
            D = (f(M + dM) - f(M - dM)) / (2 * h)
            cols.append(np.concatenate([D.real.ravel(), D.imag.ravel()]))
    return np.linalg.svd(np.array(cols).T, compute_uv=False)[0]


def fields(nc, L=(4, 4, 4, 4)):
    U = synth.gauge_config(L, nc, 0.3, 2)
    return U


@pytest.mark.parametrize("omega,variant", [(1.0, 0), (1.75, 1), (1.7, 0)])
def test_su2_local_bound_is_the_jacobian(orc, omega, variant):
    """SU(2): the site transformation is the overrelaxed a/|a| of K's
    quaternion; its bound is exact for omega = 1 and for the exact power,
    and within a factor 2 for the truncated series (whose normalisation the
    bound does not credit)."""
    L = (4, 4, 4, 4)
    U = fields(2, L)
    W = U.copy()
    orc.sweep(W, L, 2, 1.7, 5)
    for X in (U, W):
        K = gathered_K(X, L)
        for k in K[::5]:
            J = jacobian_norm(lambda m: orc.local_gauge(m, omega, variant), k)
            B = orc.local_gauge_bound(k, omega, variant)
            assert J <= B * (1 + 1e-5)
            if omega == 1.0 or variant == 1:
                assert J == pytest.approx(B, rel=1e-5)
            else:
                assert J >= 0.5 * B


@pytest.mark.parametrize("omega,variant", [(1.0, 0), (1.75, 1), (1.7, 0)])
def test_su3_local_bound_holds(orc, omega, variant):
    """SU(3): the bound compounds the three subgroup steps through the rows
    each rotates; it stays above the exact Jacobian norm at every site and
    within a factor 30 of it, on the random start and on warmed fields
    alike (so ratios of bounds compare the sites' conditioning)."""
    L = (4, 4, 4, 4)
    U = fields(3, L)
    W = U.copy()
    orc.sweep(W, L, 3, 1.7, 5)
    for X in (U, W):
        K = gathered_K(X, L)
        for k in K[::7]:
            J = jacobian_norm(lambda m: orc.local_gauge(m, omega, variant), k)
            B = orc.local_gauge_bound(k, omega, variant)
            assert B / 30 <= J <= B * (1 + 1e-5)


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("T", [0.05, 0.5, 2.0, 20.0])
def test_heatbath_local_bound_holds(orc, nc, T):
    """The heat-bath site transformation with its draws held (sites whose
    decisions lie within the difference step are skipped): r = x v moves by
    at most |dx| + |dv| (v the maximiser, x's first component a function of
    alpha = 2 |a| / T), within sqrt2 of the exact Jacobian for SU(2)."""
    L = (4, 4, 4, 4)
    U = fields(nc, L)
    W = U.copy()
    orc.sweep(W, L, nc, 1.7, 5)
    n = 0
    for X in (U, W):
        K = gathered_K(X, L)
        for i in range(0, len(K), 5):
            B, slack = orc.heatbath_gauge_bound(K[i], T, 9, i, 2, dK=1e-6)
            if slack < 1:
                continue
            J = jacobian_norm(lambda m: orc.heatbath_gauge(m, T, 9, i, 2), K[i])
            assert J <= B * (1 + 1e-5)
            assert J >= (0.7 if nc == 2 else 1 / 30) * B
            n += 1
    assert n > 80


def test_local_bound_trivial_field(orc):
    """On the trivial field (K = 8, every block quaternion of length 8 and
    the maximiser 1): SU(2) moves by omega / 8 per unit of K."""
    K = 8 * np.eye(2, dtype=complex)
    for omega in (1.0, 1.5, 1.7):
        assert orc.local_gauge_bound(K, omega, 0) == pytest.approx(omega / 8, rel=1e-12)
        assert orc.local_gauge_bound(K, omega, 1) == pytest.approx(omega / 8, rel=1e-12)


def test_local_bound_degenerate_block_is_infinite(orc):
    """A block with no quaternion part (left alone by the maximiser) has no
    bounded sensitivity: any error picks an arbitrary direction."""
    K = np.diag([1.0, -1.0]).astype(complex)  # quaternion part (K + s2 conj(K) s2) / 2 = 0
    assert orc.local_gauge_bound(K, 1.7, 0) == np.inf


def perturbed_pair(U, delta, seed=0):
    """U and U plus noise whose size varies over two decades from link to
    link (so that a bound charging one link's error for another's fails),
    and each link's perturbation in units of delta."""
    rng = np.random.default_rng(seed)
    scale = delta * 10 ** rng.uniform(-2, 0, U.shape[:2])[..., None, None]
    noise = scale * (rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    e0 = np.sqrt((np.abs(noise) ** 2).sum(axis=(2, 3))) / delta
    return U.copy(), np.ascontiguousarray(U + noise), e0


def moved(a, b, delta):
    return np.sqrt((np.abs(a - b) ** 2).sum(axis=(2, 3))) / delta


# perturbation per element: far above the oracle's own rounding (1e-16 times
# the same amplification), and small enough that the second-order remainder,
# relative size about delta A, stays below 1e-5 where it is checked
DELTA = 1e-11


def assert_bound_holds(A, d, exempt=None):
    """Every link (outside exempt) within its bound, where the bound is
    first order (delta A small); returns the largest ratio."""
    first_order = A * DELTA < 1e-5
    keep = first_order if exempt is None else first_order & ~exempt
    assert keep.mean() > 0.9
    ratio = d[keep] / A[keep]
    assert ratio.max() <= 1 + 1e-4, f"max ratio {ratio.max():.6f}"
    return ratio.max()


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("omega,variant", [(1.7, 0), (1.0, 0), (1.75, 1)])
@pytest.mark.parametrize("warm", [0, 5])
def test_sweep_bound_holds_under_perturbation(orc, nc, omega, variant, warm):
    """One sweep of an input perturbed by 1e-11 per element moves every link
    by no more than the bound carried from the perturbation (rho = 0) through
    the black and the white half-sweep; the sweep itself is unchanged."""
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, nc, 0.3, 2)
    if warm:
        orc.sweep(U, L, nc, 1.7, warm)
    a, b, e0 = perturbed_pair(U, DELTA)
    plain = U.copy()
    orc.sweep(plain, L, nc, omega, 1, variant)
    A = orc.sweep_bound(a, L, nc, omega, variant, e=e0, rho=0.0)
    assert np.array_equal(a, plain)
    orc.sweep(b, L, nc, omega, 1, variant)
    r = assert_bound_holds(A, moved(a, b, DELTA))
    if nc == 2:
        assert r > 0.1  # attained within a factor 10 somewhere


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("kind", ["or", "mag"])
def test_bound_follows_the_perturbed_links(orc, nc, kind):
    """Only the four backward links into one black site x perturbed: x's own
    (forward) links, unperturbed on input, move through g(x), and their
    bound must say so; links far from x neither move nor get a bound."""
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, nc, 0.3, 2)
    orc.sweep(U, L, nc, 1.7, 5)
    x = int(np.flatnonzero(P.parity(L) == 0)[37])
    rng = np.random.default_rng(6)
    b = U.copy()
    e0 = np.zeros((U.shape[0], 4))
    for mu in range(4):
        y = P.shifted(L, mu, -1)[x]
        n = DELTA * (rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc)))
        b[y, mu] += n
        e0[y, mu] = np.linalg.norm(n) / DELTA
    a = U.copy()
    if kind == "or":
        A = orc.sweep_bound(a, L, nc, 1.7, 0, e=e0, rho=0.0)
        orc.sweep(b, L, nc, 1.7, 1)
    else:
        A = orc.mag_sweep_bound(a, L, nc, 1.7, 0, e=e0, rho=0.0)
        orc.mag_sweep(b, L, nc, 1.7, 1)
    d = moved(a, b, DELTA)
    assert (d[x] > 0).all() and (A[x] > 0).all()
    assert (d <= A * (1 + 1e-4)).all()
    far = (P.coords(L) - P.coords(L)[x] + 4) % 8 - 4
    far = np.abs(far).sum(axis=1) > 3
    assert (A[far] == 0).all() and (d[far] == 0).all()


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("T", [0.05, 0.5, 20.0])
@pytest.mark.parametrize("warm", [0, 5])
def test_heatbath_bound_holds_under_perturbation(orc, nc, T, warm):
    """The heat-bath sweep with the same draws: every link outside the sites
    whose decisions the perturbation may flip (slack < delta) and their
    downstream neighbours moves by no more than its bound."""
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, nc, 0.3, 2)
    if warm:
        orc.sweep(U, L, nc, 1.7, warm)
    a, b, e0 = perturbed_pair(U, DELTA, 1)
    plain = U.copy()
    orc.heatbath_sweep(plain, L, nc, T, 7, 3)
    A, slack = orc.heatbath_sweep_bound(a, L, nc, T, 7, 3, e=e0, rho=0.0)
    assert np.array_equal(a, plain)
    orc.heatbath_sweep(b, L, nc, T, 7, 3)
    flagged = slack < DELTA
    black = flagged & (P.parity(L) == 0)
    spread = black.copy()
    for mu in range(4):
        spread |= black[P.shifted(L, mu, 1)] | black[P.shifted(L, mu, -1)]
    assert_bound_holds(A, moved(a, b, DELTA), P.links_touching(L, flagged | spread))


def test_heatbath_slack_predicts_flipped_decisions(orc):
    """One draw with alpha moved by up to dalpha (0.1% to 5% of alpha, where
    the margins are still linear in alpha): wherever its outcome (the
    accepted attempt, or Creutz's method against Kennedy-Pendleton's)
    changes, the slack computed for (alpha, dalpha) is below 1, and it is
    below 1 hardly anywhere else."""
    rng = np.random.default_rng(5)
    flips = low = 0
    for _ in range(15000):
        alpha = float(rng.uniform(0.05, 40.0))
        dalpha = alpha * 10 ** rng.uniform(-3, -1.3)
        site, sub = int(rng.integers(0, 2 ** 31)), int(rng.integers(0, 3))
        s = orc.hb_slack(alpha, dalpha, 0.5, 11, site, 2, sub)
        outcomes = set()
        for x in np.linspace(alpha - dalpha, alpha + dalpha, 9):
            att = ctypes.c_int()
            orc._load().oracle_hb_delta(float(x), orc._key(11), site, 2, sub, ctypes.byref(att))
            outcomes.add((att.value, x < 2.0))
        if len(outcomes) > 1:
            flips += 1
            assert s < 1.0, (alpha, dalpha, site, sub, s)
        low += s < 1.0
    assert flips >= 20
    assert low <= 2 * flips


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("omega,variant", [(1.7, 0), (1.0, 0), (1.5, 1)])
@pytest.mark.parametrize("warm", [0, 5])
def test_mag_sweep_bound_holds_under_perturbation(orc, nc, omega, variant, warm):
    """As for the Landau sweep. The SU(3) MAG bound on the random start is
    large (short block vectors compounded over three subgroups), so there the
    perturbation is 1e-14: the oracle's own rounding then adds about 1% to the
    response, far inside a bound this loose."""
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, nc, 0.3, 2)
    if warm:
        orc.mag_sweep(U, L, nc, 1.7, warm)
    delta = 1e-14 if (nc == 3 and not warm) else DELTA
    a, b, e0 = perturbed_pair(U, delta, 2)
    plain = U.copy()
    orc.mag_sweep(plain, L, nc, omega, 1, variant)
    A = orc.mag_sweep_bound(a, L, nc, omega, variant, e=e0, rho=0.0)
    assert np.array_equal(a, plain)
    orc.mag_sweep(b, L, nc, omega, 1, variant)
    d = moved(a, b, delta)
    first_order = A * delta < 1e-5
    assert first_order.mean() > 0.5
    assert (d[first_order] / A[first_order]).max() <= 1 + 1e-4


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("T", [0.05, 2.0])
def test_mag_heatbath_bound_holds_under_perturbation(orc, nc, T):
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, nc, 0.3, 2)
    orc.mag_sweep(U, L, nc, 1.7, 5)
    a, b, e0 = perturbed_pair(U, DELTA, 3)
    plain = U.copy()
    orc.mag_heatbath_sweep(plain, L, nc, T, 9, 4)
    A = orc.mag_heatbath_sweep_bound(a, L, nc, T, 9, 4, e=e0, rho=0.0)
    assert np.array_equal(a, plain)
    orc.mag_heatbath_sweep(b, L, nc, T, 9, 4)
    d = moved(a, b, DELTA)
    first_order = A * DELTA < 1e-5
    assert first_order.mean() > 0.5
    assert (d[first_order] / A[first_order]).max() <= 1 + 1e-4


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_local_bound_holds(orc, nc):
    """The MAG site transformation moves by at most the bound times
    max_a ||dX_a|| along random directions of every X_a (and along the
    worst single-block direction, X_i and X_j moved oppositely)."""
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, nc, 0.3, 2)
    rng = np.random.default_rng(4)
    for i in range(0, int(np.prod(L)), 11):
        X = np.zeros((nc, nc, nc), dtype=complex)
        for mu in range(4):
            f = U[i, mu]
            bk = U[P.shifted(L, mu, -1)[i], mu]
            for a_ in range(nc):
                Pa = np.zeros((nc, nc))
                Pa[a_, a_] = 1
                X[a_] += f @ Pa @ f.conj().T + bk.conj().T @ Pa @ bk
        B = orc.mag_local_gauge_bound(X, 1.7)
        g0 = orc.mag_local_gauge(X, 1.7)[0]
        h = 1e-8
        for _ in range(8):
            dX = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
            dX = dX + np.conj(np.swapaxes(dX, -1, -2))
            dX /= np.linalg.norm(dX.reshape(nc, -1), axis=1).max()
            g1 = orc.mag_local_gauge(X + h * dX, 1.7)[0]
            assert np.linalg.norm(g1 - g0) / h <= B * (1 + 1e-3)


# --- the tangent bound of an SU(3) site (tight = True) ---

TRACE_POWER = 8 ** (1 / 32)  # (tr M^16)^(1/32) over ||J||_2 is at most this for rank <= 8


def gathered_X(U, L):
    """The MAG X_a(x) = sum_mu [U P_a U^+ + U(x-mu)^+ P_a U(x-mu)] for every site, (V, Nc, Nc, Nc)."""
    nc = U.shape[-1]
    X = np.zeros((U.shape[0], nc, nc, nc), dtype=complex)
    for mu in range(4):
        f = U[:, mu]
        bk = U[P.shifted(L, mu, -1), mu]
        for a in range(nc):
            X[:, a] += np.einsum("vi,vj->vij", f[:, :, a], np.conj(f[:, :, a]))
            X[:, a] += np.einsum("vi,vj->vij", np.conj(bk[:, a, :]), bk[:, a, :])
    return X


def hermitian_jacobian_norms(f, X, h=1e-7):
    """Per a, the largest singular value of the Jacobian of f along an
    orthonormal hermitian basis of X_a (central differences)."""
    nc = X.shape[-1]
    out = []
    for a in range(nc):
        cols = []
        for r in range(nc):
            for c in range(r, nc):
                for z in ((1.0,) if r == c else (1.0, 1j)):
                    E = np.zeros(X.shape, dtype=complex)
                    if r == c:
                        E[a, r, r] = 1.0
                    else:
                        E[a, r, c] = z / np.sqrt(2)
                        E[a, c, r] = np.conj(z) / np.sqrt(2)
                    D = (f(X + h * E) - f(X - h * E)) / (2 * h)
                    cols.append(np.concatenate([D.real.ravel(), D.imag.ravel()]))
        out.append(np.linalg.svd(np.array(cols).T, compute_uv=False)[0])
    return out


TANGENT_KINDS = ["or", "or_power", "hb", "mag", "mag_power", "mag_hb"]


@pytest.mark.parametrize("kind", TANGENT_KINDS)
@pytest.mark.parametrize("warm", [0, 5])
def test_tangent_bound_is_the_jacobian_norm(orc, kind, warm):
    """The tangent bound of an SU(3) site (no rounding) against the exact
    Jacobian of the oracle's own site transformation by central differences:
    Landau per unit ||dK||, MAG per unit max_a ||dX_a|| (the sum over a of
    the hermitian blocks' norms). It is that norm taken from above through
    a trace power, so it lies within [1, 8^(1/32)] of it; a dropped term or
    a wrong sign in any step's derivative moves it out."""
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, 3, 0.3, 2)
    mag = kind.startswith("mag")
    if warm:
        (orc.mag_sweep if mag else orc.sweep)(U, L, 3, 1.7, warm)
    inputs = gathered_X(U, L) if mag else gathered_K(U, L)
    ratios = []
    for i in range(0, int(np.prod(L)), 9):
        M = inputs[i]
        if kind.endswith("hb"):
            for T in (0.05, 2.0):
                B = orc.tangent_bound(M, mag=mag, hb=True, T=T, seed=9, site=i, sweep=4)
                if mag:
                    J = sum(hermitian_jacobian_norms(lambda x: orc.mag_heatbath_gauge(x, T, 9, i, 4), M))
                else:
                    J = jacobian_norm(lambda k: orc.heatbath_gauge(k, T, 9, i, 4), M)
                ratios.append(B / J)
            continue
        omega, variant = (1.5, 1) if kind.endswith("power") else (1.7, 0)
        B = orc.tangent_bound(M, mag=mag, omega=omega, variant=variant)
        if mag:
            J = sum(hermitian_jacobian_norms(lambda x: orc.mag_local_gauge(x, omega, variant)[0], M))
        else:
            J = jacobian_norm(lambda k: orc.local_gauge(k, omega, variant), M)
        ratios.append(B / J)
    ratios = np.array(ratios)
    assert len(ratios) >= 29
    assert ratios.min() >= 1 - 1e-5 and ratios.max() <= TRACE_POWER + 1e-5, (ratios.min(), ratios.max())


def tight_pair(orc, kind, warm):
    L = (8, 8, 8, 8)
    U = synth.gauge_config(L, 3, 0.3, 2)
    if warm:
        (orc.mag_sweep if kind.startswith("mag") else orc.sweep)(U, L, 3, 1.7, warm)
    return L, U


def run_bound(orc, kind, U, L, tight, e=None, rho=1.0):
    """One sweep of this kind in place; (bound, slack or None)."""
    if kind == "or":
        return orc.sweep_bound(U, L, 3, 1.7, 0, e=e, rho=rho, tight=tight), None
    if kind == "mag":
        return orc.mag_sweep_bound(U, L, 3, 1.7, 0, e=e, rho=rho, tight=tight), None
    if kind == "hb":
        return orc.heatbath_sweep_bound(U, L, 3, 0.5, 7, 3, e=e, rho=rho, tight=tight)
    return orc.mag_heatbath_sweep_bound(U, L, 3, 0.5, 7, 3, e=e, rho=rho, tight=tight), None


def run_plain(orc, kind, U, L):
    if kind == "or":
        orc.sweep(U, L, 3, 1.7, 1)
    elif kind == "mag":
        orc.mag_sweep(U, L, 3, 1.7, 1)
    elif kind == "hb":
        orc.heatbath_sweep(U, L, 3, 0.5, 7, 3)
    else:
        orc.mag_heatbath_sweep(U, L, 3, 0.5, 7, 3)


@pytest.mark.parametrize("kind", ["or", "mag", "hb", "mag_hb"])
@pytest.mark.parametrize("warm", [0, 5])
def test_tight_sweep_bound_holds_under_perturbation(orc, kind, warm):
    """SU(3) sweeps with the tangent bound, as for the norm bound: every link
    of a perturbed input moves by no more than its bound (outside the sites
    whose heat-bath decisions the perturbation may flip)."""
    L, U = tight_pair(orc, kind, warm)
    a, b, e0 = perturbed_pair(U, DELTA, 2)
    plain = U.copy()
    run_plain(orc, kind, plain, L)
    A, slack = run_bound(orc, kind, a, L, True, e=e0, rho=0.0)
    assert np.array_equal(a, plain)
    run_plain(orc, kind, b, L)
    exempt = None
    if slack is not None:
        flagged = slack < DELTA
        black = flagged & (P.parity(L) == 0)
        spread = black.copy()
        for mu in range(4):
            spread |= black[P.shifted(L, mu, 1)] | black[P.shifted(L, mu, -1)]
        exempt = P.links_touching(L, flagged | spread)
    assert_bound_holds(A, moved(a, b, DELTA), exempt)


@pytest.mark.parametrize("kind", ["or", "mag", "hb", "mag_hb"])
def test_tight_bound_is_the_smaller(orc, kind):
    """The tangent bound only replaces a site's norm bound where it is
    smaller, so no link's bound grows, and the sweep is the same; on the
    random start it is far smaller (a factor of 10 in the median or more)."""
    L, U = tight_pair(orc, kind, 0)
    a, b = U.copy(), U.copy()
    An, _ = run_bound(orc, kind, a, L, False)
    At, _ = run_bound(orc, kind, b, L, True)
    assert np.array_equal(a, b)
    assert (At <= An).all()
    assert np.median(An / At) >= 10
