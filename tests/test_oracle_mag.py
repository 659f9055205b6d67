"""Pins of the oracle's maximally Abelian gauge (readings R12-R15 of
culgt_oracle.c).

The paper names MAG fixing among cuLGT's gauges (abstract, Sec. 1) without
formulas, so the pins come from the functional itself: brute-force
maximisation of the SU(2) step and of the site functional computed directly
from the links, closed forms for a single off-diagonal link, the trivial
(Abelian) and pure-gauge fields, covariance under global diagonal rotations,
monotonicity at omega = 1 and gauge invariance of the plaquette.
"""
import numpy as np
import pytest

from paper_1412_3655_gb300 import synth

RNG = np.random.default_rng(1412)
S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]])
S3 = np.diag([1.0 + 0j, -1.0])


def haar_su2(n, rng=RNG):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    m = np.empty((n, 2, 2), dtype=complex)
    m[:, 0, 0] = q[:, 0] + 1j * q[:, 3]
    m[:, 0, 1] = q[:, 2] + 1j * q[:, 1]
    m[:, 1, 0] = -q[:, 2] + 1j * q[:, 1]
    m[:, 1, 1] = q[:, 0] - 1j * q[:, 3]
    return m


def embed(r, i, j, nc=3):
    R = np.broadcast_to(np.eye(nc, dtype=complex), r.shape[:-2] + (nc, nc)).copy()
    R[..., i, i], R[..., i, j], R[..., j, i], R[..., j, j] = r[..., 0, 0], r[..., 0, 1], r[..., 1, 0], r[..., 1, 1]
    return R


def random_hermitian(n, rng=RNG):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return a + a.conj().T


def coords(dims):
    V = int(np.prod(dims))
    x0, x3, x2, x1 = np.unravel_index(np.arange(V), (dims[0], dims[3], dims[2], dims[1]))
    return x0, x1, x2, x3


def site_functional(U, dims, i, g=None):
    """sum over the 8 links at site i of sum_a |(link)_aa|^2 after g at site i."""
    nc = U.shape[-1]
    if g is None:
        g = np.eye(nc)
    s = 0.0
    for mu in range(4):
        ib = int(np.flatnonzero(synth.site_neighbour_forward(dims, mu) == i)[0])
        s += np.sum(np.abs(np.diagonal(g @ U[i, mu])) ** 2)
        s += np.sum(np.abs(np.diagonal(U[ib, mu] @ g.conj().T)) ** 2)
    return s


# ---------------------------------------------------------------- SU(2) step


@pytest.mark.parametrize("seed", range(4))
def test_su2_step_is_the_brute_force_maximum(orc, seed):
    """(1/2) tr[s3 B Z B^+] is at most |z| (traceless part z.s of Z), reached
    by the returned B, which rotates z to +|z| e3 about an axis in the
    1-2 plane (the smallest rotation: B_00 real)."""
    rng = np.random.default_rng(seed)
    Z = random_hermitian(2, rng)
    B = orc.mag_su2_max(Z)
    z = np.array([Z[0, 1].real, -Z[0, 1].imag, 0.5 * (Z[0, 0] - Z[1, 1]).real])
    val = 0.5 * np.trace(S3 @ B @ Z @ B.conj().T).real
    assert val == pytest.approx(np.linalg.norm(z), abs=1e-13)
    Bs = haar_su2(20000, rng)
    vals = 0.5 * np.einsum("ij,njk,kl,nil->n", S3, Bs, Z, Bs.conj()).real
    assert vals.max() <= val + 1e-12
    assert np.abs(B @ B.conj().T - np.eye(2)).max() < 1e-14 and abs(np.linalg.det(B) - 1) < 1e-14
    Zt = Z - 0.5 * np.trace(Z) * np.eye(2)
    assert np.abs(B @ Zt @ B.conj().T - np.linalg.norm(z) * S3).max() < 1e-13
    assert abs(B[0, 0].imag) < 1e-15


def test_su2_step_degenerate_blocks(orc):
    assert np.abs(orc.mag_su2_max(np.eye(2) * 3.0) - np.eye(2)).max() == 0
    B = orc.mag_su2_max(-2.0 * S3)
    assert np.abs(B @ (-2.0 * S3) @ B.conj().T - 2.0 * S3).max() < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_su2_site_update_maximises_the_site_functional(orc, seed):
    """SU(2): the site transformation is the global maximum over SU(2) of
    sum_a tr[P_a g X_a g^+]."""
    rng = np.random.default_rng(10 + seed)
    X = np.array([random_hermitian(2, rng) for _ in range(2)])
    g, _ = orc.mag_local_gauge(X, 1.0)

    def f(gs):
        return sum(np.einsum("nj,jk,nk->n", gs[:, a, :], X[a], gs[:, a, :].conj()).real for a in range(2))

    best = f(g[None])[0]
    assert f(haar_su2(20000, rng)).max() <= best + 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_su3_site_update_raises_and_last_block_is_maximal(orc, seed):
    """SU(3): the update does not lower sum_a tr[P_a g X_a g^+], and no SU(2)
    rotation of the last subgroup (1,2) on top of it raises it (each subgroup
    step maximises its block)."""
    rng = np.random.default_rng(20 + seed)
    X = np.array([random_hermitian(3, rng) for _ in range(3)])

    def f(gs):
        return sum(np.einsum("nj,jk,nk->n", gs[:, a, :], X[a], gs[:, a, :].conj()).real for a in range(3))

    g, _ = orc.mag_local_gauge(X, 1.0)
    base = f(np.eye(3)[None])[0]
    val = f(g[None])[0]
    assert val >= base - 1e-12
    Rs = embed(haar_su2(20000, rng), 1, 2)
    assert f(Rs @ g).max() <= val + 1e-12


def test_site_functional_is_maximal_after_an_su2_halfsweep(orc):
    """The gathered X_a describe the links: after a black half-sweep at
    omega = 1, no SU(2) transformation at a black site raises its functional
    computed directly from the links, sum |diagonal|^2 over its 8 links."""
    dims = (4, 4, 2, 4)
    U = synth.gauge_config(dims, 2, 0.5, 3)
    orc.mag_halfsweep(U, dims, 2, 0, 1.0)
    x0, x1, x2, x3 = coords(dims)
    black = np.flatnonzero(((x0 + x1 + x2 + x3) & 1) == 0)
    gs = haar_su2(300, np.random.default_rng(5))
    c = np.random.default_rng(6).standard_normal((100, 3))
    near = synth.expi(np.einsum("na,aij->nij", c, np.array([S1, S2, S3])), 0.05)
    for i in black[:5]:
        f0 = site_functional(U, dims, int(i))
        for g in list(gs) + list(near):
            assert site_functional(U, dims, int(i), g) <= f0 + 1e-12


# ---------------------------------------------------------------- lattice


@pytest.mark.parametrize("nc", [2, 3])
def test_abelian_field_is_fixed(orc, nc):
    """Diagonal links: theta_MAG = 0, F_MAG = 1, and a sweep changes nothing."""
    dims = (4, 2, 4, 2)
    V = int(np.prod(dims))
    rng = np.random.default_rng(7)
    ph = rng.uniform(0, 2 * np.pi, (V, 4, nc - 1))
    U = np.zeros((V, 4, nc, nc), dtype=complex)
    for a in range(nc - 1):
        U[..., a, a] = np.exp(1j * ph[..., a])
    U[..., nc - 1, nc - 1] = np.exp(-1j * ph.sum(axis=-1))
    th, F = orc.mag_theta(U, dims, nc)
    assert th < 1e-28 and F == pytest.approx(1.0, abs=1e-15)
    W = U.copy()
    orc.mag_sweep(W, dims, nc, 1.7)
    assert np.abs(W - U).max() < 1e-15


@pytest.mark.parametrize("nc,eps", [(2, 0.3), (2, 0.7), (3, 0.3), (3, 0.7)])
def test_single_offdiagonal_link_closed_forms(orc, nc, eps):
    """All links 1 except U_0(0) = exp(i eps s1) (SU(3): the (0,1) block):
    theta_MAG = 4 sin^2(2 eps) / V and F_MAG = 1 - 2 sin^2(eps) / (4 Nc V)."""
    dims = (4, 4, 2, 2)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(nc, dtype=complex), (V, 4, nc, nc)).copy()
    r = np.cos(eps) * np.eye(2) + 1j * np.sin(eps) * S1
    U[0, 0] = embed(r, 0, 1, nc) if nc == 3 else r
    th, F = orc.mag_theta(U, dims, nc)
    assert th == pytest.approx(4 * np.sin(2 * eps) ** 2 / V, rel=1e-13)
    assert F == pytest.approx(1 - 2 * np.sin(eps) ** 2 / (4 * nc * V), rel=1e-14)


@pytest.mark.parametrize("nc", [2, 3])
def test_F_mag_non_decreasing_at_omega_one(orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.4, 2)
    last = orc.mag_theta(U, dims, nc)[1]
    for _ in range(6):
        orc.mag_sweep(U, dims, nc, 1.0)
        F = orc.mag_theta(U, dims, nc)[1]
        assert F >= last - 1e-13
        last = F


@pytest.mark.parametrize("nc", [2, 3])
def test_sweep_is_covariant_under_global_diagonal_rotations(orc, nc):
    """A constant diagonal h commutes with the projectors, so
    sweep(h U h^+) = h sweep(U) h^+."""
    dims = (4, 2, 4, 4)
    U = synth.gauge_config(dims, nc, 0.4, 4)
    ph = np.random.default_rng(8).uniform(0, 2 * np.pi, nc - 1)
    d = np.exp(1j * np.append(ph, -ph.sum()))
    h = np.diag(d)
    a = U.copy()
    orc.mag_sweep(a, dims, nc, 1.7)
    b = np.ascontiguousarray(h @ U @ h.conj().T)
    orc.mag_sweep(b, dims, nc, 1.7)
    assert np.abs(b - h @ a @ h.conj().T).max() < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_sweeps_keep_plaquette_and_unitarity(orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 5)
    P0 = orc.plaquette(U, dims, nc)
    orc.mag_sweep(U, dims, nc, 1.7, 5)
    assert orc.plaquette(U, dims, nc) == pytest.approx(P0, abs=1e-13)
    assert orc.unitarity_error(U, nc) < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
def test_pure_gauge_converges_to_the_abelian_field(orc, nc):
    """U = g(x) g(x+mu)^+ with g near 1: MAG fixing reaches F_MAG = 1."""
    dims = (4, 4, 4, 4)
    U = synth.pure_gauge(dims, nc, 6, spread=0.5)
    r = orc.mag_fix(U, dims, nc, 1.7, 1e-14, 4000, 10, 100)
    assert r["converged"]
    assert r["F"] == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_contract(orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    r = orc.mag_fix(U, dims, nc, 1.7, 1e-12, 5000, 10, 50)
    assert r["converged"] and r["theta"] < 1e-12 and r["sweeps"] % 10 == 0
    th, F = orc.mag_theta(U, dims, nc)
    assert th == r["theta"] and F == r["F"]


@pytest.mark.parametrize("omega,variant", [(1.7, 0), (1.5, 1)])
def test_su2_site_update_is_the_overrelaxed_maximiser(orc, omega, variant):
    """The MAG step is overrelaxed like the Landau one: g = (maximiser)^omega
    with the pinned g^omega of reading R3."""
    rng = np.random.default_rng(30)
    X = np.array([random_hermitian(2, rng) for _ in range(2)])
    g1, _ = orc.mag_local_gauge(X, 1.0)
    gw, _ = orc.mag_local_gauge(X, omega, variant)
    assert np.abs(gw - orc.overrelax(g1, omega, variant)).max() < 1e-14
    assert np.abs(gw - g1).max() > 1e-3


# ---------------------------------------------------------------- MAG annealing (R16)


def _u_cdf(beta):
    return lambda u: np.expm1(beta * np.clip(u, 0, 1)) / np.expm1(beta)


@pytest.mark.parametrize("T", [50.0, 3.0, 0.5, 0.05])
def test_mag_heatbath_draw_follows_the_boltzmann_weight(orc, T):
    """For a fixed block Z with |z| = n the drawn B has the subgroup functional
    (1/2) tr[s3 B Z B^+] = n (2u - 1), u exponential on [0, 1] with rate
    2n/T (Haar measure makes u uniform); the residual angles of C = B Bmax^+
    are uniform."""
    from scipy import stats
    rng = np.random.default_rng(40)
    Z = random_hermitian(2, rng)
    n = np.linalg.norm([Z[0, 1].real, Z[0, 1].imag, 0.5 * (Z[0, 0] - Z[1, 1]).real])
    Bmax = orc.mag_su2_max(Z)
    N = 8000
    Bs = np.array([orc.mag_heatbath_su2(Z, T, 3, s, 1, s % 3) for s in range(N)])
    f = 0.5 * np.einsum("ij,njk,kl,nil->n", S3, Bs, Z, Bs.conj()).real
    u = (f / n + 1) / 2
    beta = 2 * n / T
    assert stats.kstest(u, _u_cdf(beta)).pvalue > 1e-3
    C = Bs @ Bmax.conj().T
    c0, c3 = C[:, 0, 0].real, C[:, 0, 0].imag
    c2, c1 = C[:, 0, 1].real, C[:, 0, 1].imag
    assert np.abs(c0 ** 2 + c3 ** 2 - u).max() < 1e-12
    for ang in (np.arctan2(c3, c0), np.arctan2(c2, c1)):
        ok = np.hypot(np.cos(ang), np.sin(ang)) > 0
        assert stats.kstest((ang[ok] + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


@pytest.mark.parametrize("nc", [2, 3])
def test_zero_temperature_mag_heatbath_is_the_maximisation_up_to_U1(orc, nc):
    """T -> 0 draws u = 1: B = e^{i a s3} Bmax, the maximiser up to the
    diagonal rotation MAG leaves free, so the moduli |U_ab| of the links and
    F_MAG equal those after an omega = 1 MAG sweep."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 9)
    a = U.copy()
    orc.mag_heatbath_sweep(a, dims, nc, 1e-24, 5, 0)
    b = U.copy()
    orc.mag_sweep(b, dims, nc, 1.0, 1)
    assert np.abs(np.abs(a) - np.abs(b)).max() < 1e-9
    assert orc.mag_theta(a, dims, nc)[1] == pytest.approx(orc.mag_theta(b, dims, nc)[1], abs=1e-12)
    assert np.abs(a - b).max() > 1e-3  # the diagonal rotations are drawn


@pytest.mark.parametrize("nc", [2, 3])
def test_infinite_temperature_mag_heatbath_is_haar(orc, nc):
    """T -> infinity: g(x) Haar, E|(g U h^+)_aa|^2 = 1/Nc, so F_MAG -> 1/Nc."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 10)
    orc.mag_heatbath_sweep(U, dims, nc, 1e9, 6, 0)
    F = orc.mag_theta(U, dims, nc)[1]
    n = 4 * int(np.prod(dims)) * nc
    assert abs(F - 1.0 / nc) < 6 * 0.5 / np.sqrt(n)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_microcanonical_sweep_keeps_F(orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 11)
    F0 = orc.mag_theta(U, dims, nc)[1]
    orc.mag_sweep(U, dims, nc, 2.0, 1)
    assert orc.mag_theta(U, dims, nc)[1] == pytest.approx(F0, abs=1e-13)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_anneal_schedule(orc, nc):
    dims = (2, 4, 2, 4)
    U = synth.gauge_config(dims, nc, 0.3, 12)
    a = U.copy()
    orc.mag_anneal(a, dims, nc, 1.0, 0.1, 3, 2, 17)
    b = U.copy()
    for k in range(3):
        orc.mag_heatbath_sweep(b, dims, nc, 1.0 + (0.1 - 1.0) * k / 2, 17, k)
        orc.mag_sweep(b, dims, nc, 2.0, 2)
    assert np.array_equal(a, b)


def test_mag_annealing_then_overrelaxation_finds_higher_maxima(orc):
    dims = (4, 4, 4, 4)
    plain, ann = [], []
    for c in range(6):
        U = synth.gauge_config(dims, 3, 0.6, 1, copy=c)
        plain.append(orc.mag_fix(U.copy(), dims, 3, 1.7, 1e-12, 20000, 10, 50)["F"])
        W = U.copy()
        orc.mag_anneal(W, dims, 3, 0.6, 0.01, 300, 3, 60 + c, reunit_every=50)
        ann.append(orc.mag_fix(W, dims, 3, 1.7, 1e-12, 20000, 10, 50)["F"])
    assert np.mean(ann) > np.mean(plain)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_heatbath_draws_depend_on_the_sweep_word(orc, nc):
    dims = (2, 4, 2, 4)
    U = synth.gauge_config(dims, nc, 0.3, 13)
    a, b, c = U.copy(), U.copy(), U.copy()
    orc.mag_heatbath_sweep(a, dims, nc, 0.7, 21, 3)
    orc.mag_heatbath_sweep(b, dims, nc, 0.7, 21, 4)
    orc.mag_heatbath_sweep(c, dims, nc, 0.7, 21, 3)
    assert np.abs(a - b).max() > 1e-3 and np.array_equal(a, c)


def test_mag_heatbath_of_a_zero_block_is_the_identity(orc):
    """z = 0 (a block proportional to 1) leaves the block alone."""
    B = orc.mag_heatbath_su2(2.5 * np.eye(2), 0.7, 1, 0, 0)
    assert np.abs(B - np.eye(2)).max() == 0
