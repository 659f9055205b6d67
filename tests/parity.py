"""Per-link tolerances for comparing one sweep of the CUDA path with the oracle.

The local problem of a site (Sec. 2: the block quaternion a of each SU(2)
subgroup normalised to a/|a|; for MAG, the smallest rotation of a block vector
z onto +e3) amplifies any rounding difference between two implementations by
the inverse length it normalises. The oracle carries a first-order bound of
that amplification through the sweep (``sweep_bound`` and friends): A(link),
how far the link can move per unit error of every input link and every
rounding step. A_ref is the same bound on the trivial field (every link 1),
the best-conditioned input there is. For overrelaxation sweeps (Landau and
MAG) on lattices up to 32^4 sites, an SU(3) site's bound goes through the
site's exact tangent map (``tight``; within 7% of the norm of its Jacobian,
pinned against finite differences); above that, where it would take minutes
per sweep, and for heat-bath sweeps, through the per-step norm rules alone.
The heat-bath draw's own rounding can move the drawn element by thousands
of unit roundoffs where a small cosine multiplies log u2 (the
Kennedy-Pendleton formula, computed differently on each side), which the
per-step rounding charge does not model; the looser norm bound covers it
(measured: a 32^4 FP64 heat-bath sweep put 4 links up to 1.15 times past the
tangent bound's allowance, none past the norm bound's). A and A_ref always
come from the same kind.

The rule, for every link:

    |got - ref| <= tol * max(1, C * A(link) / A_ref)

tol is the tolerance stated for one sweep on well-conditioned input (FP64
1e-13, FP32 5e-6, double-float 3.2e-12). C = 1/2 is fixed once: links whose
bound is at most twice the trivial field's are held to tol itself, and beyond
that the allowance grows in proportion to the link's own bound, never for
other links. The local bound overstates the exact first-order response of a
site by a factor that hardly varies between sites (its pins: 1 to 1.4 for
SU(2), 1 to 1.07 for the SU(3) tangent bound), so A / A_ref compares a link's
conditioning with the trivial field's.

Heat-bath sweeps also take accept/reject decisions. Where a decision's margin
is within its own error bound at the compared precision (the oracle's
per-site slack below that precision's unit roundoff) another implementation
may take it the other way and draw something else entirely; that site's links
are then exempt from the elementwise rule, and so are the links of the white
sites next to such a black site, whose draws gather them later in the same
sweep. Exempt links are still checked to be unitary.
"""
import functools

import numpy as np

C = 0.5
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "df": 2.0 ** -48}
TIGHT_MAX_SITES = 32 ** 4


def tight_for(L):
    """The tangent bound for lattices up to 32^4 sites, the norm bound above."""
    return int(np.prod(L)) <= TIGHT_MAX_SITES


def link_errors(got, ref):
    """Largest entry difference per link, shape (V, 4)."""
    nc = got.shape[-1]
    return np.abs(got - ref).reshape(got.shape[0], 4, nc * nc).max(axis=2)


def coords(L):
    """(V, 4) coordinates of the canonical site order i = x1 + L1 (x2 + L2 (x3 + L3 x0))."""
    i = np.arange(int(np.prod(L)))
    x1 = i % L[1]
    r = i // L[1]
    x2 = r % L[2]
    r //= L[2]
    x3 = r % L[3]
    x0 = r // L[3]
    return np.stack([x0, x1, x2, x3], axis=1)


def index(L, x):
    return x[:, 1] + L[1] * (x[:, 2] + L[2] * (x[:, 3] + L[3] * x[:, 0]))


def shifted(L, mu, step):
    """Site index of x + step mu-hat for every x (periodic)."""
    x = coords(L)
    x[:, mu] = (x[:, mu] + step) % L[mu]
    return index(L, x)


def links_touching(L, sites):
    """(V, 4) mask of the links U_mu(x) with an end in the boolean site mask."""
    m = np.zeros((len(sites), 4), dtype=bool)
    for mu in range(4):
        m[:, mu] = sites | sites[shifted(L, mu, 1)]
    return m


def parity(L):
    return coords(L).sum(axis=1) & 1


def heatbath_exempt(L, slack, precision):
    """Links a heat-bath sweep may draw differently at this precision: those
    of sites with a decision inside its error bound, and those of the white
    sites next to such a black site (black is swept first). Returns the
    (V, 4) mask and the number of such sites."""
    flagged = slack < UNIT_ROUNDOFF[precision]
    black = flagged & (parity(L) == 0)
    spread = black.copy()
    for mu in range(4):
        spread |= black[shifted(L, mu, 1)] | black[shifted(L, mu, -1)]
    return links_touching(L, flagged | spread), int(flagged.sum())


def unit_field(L, nc):
    U = np.zeros((int(np.prod(L)), 4, nc, nc), dtype=np.complex128)
    U[...] = np.eye(nc)
    return U


def reference_bound(bound_fn, nc, L=(4, 4, 4, 4)):
    """A_ref: the largest bound bound_fn(U, L) gives on the trivial field."""
    return float(bound_fn(unit_field(L, nc), L).max())


def allowance(tol, A, A_ref):
    return tol * np.maximum(1.0, C * A / A_ref)


def check_links(got, ref, tol, A, A_ref, exempt=None, unitarity_tol=None):
    """Asserts the per-link rule; returns (worst ratio of error to allowance,
    number of links above tol) for reporting."""
    err = link_errors(got, ref)
    allow = allowance(tol, A, A_ref)
    ok = err <= allow
    if exempt is not None:
        ok |= exempt
        nc = got.shape[-1]
        G = got[exempt]
        dev = np.abs(G @ np.conj(np.swapaxes(G, -1, -2)) - np.eye(nc)).max() if len(G) else 0.0
        assert dev <= (unitarity_tol or 10 * tol), f"exempt links not unitary: {dev:.3e}"
    bad = np.argwhere(~ok)
    assert len(bad) == 0, (f"{len(bad)} links beyond their allowance; first {tuple(bad[0])}: err "
                           f"{err[tuple(bad[0])]:.3e}, allowance {allow[tuple(bad[0])]:.3e}, "
                           f"A/A_ref {A[tuple(bad[0])] / A_ref:.3g}")
    keep = ~exempt if exempt is not None else np.ones_like(ok)
    return float((err / allow)[keep].max()), int((err > tol).sum())


def check_sweep(got, ref, tol, A, A_ref, well_conditioned, exempt=None):
    """The per-link rule above; on well-conditioned input (warmed fields)
    also every (non-exempt) link within tol itself."""
    if well_conditioned:
        err = link_errors(got, ref)
        keep = ~exempt if exempt is not None else np.ones(err.shape, dtype=bool)
        assert err[keep].max() <= tol, f"max {err[keep].max():.3e}"
    check_links(got, ref, tol, A, A_ref, exempt)


# The oracle's sweep with its bound, and the trivial field's bound, per kind.

@functools.lru_cache(maxsize=None)
def _ref_or(orc, nc, omega, variant, tight):
    return reference_bound(lambda U, L: orc.sweep_bound(U, L, nc, omega, variant, tight=tight), nc)


@functools.lru_cache(maxsize=None)
def _ref_mag(orc, nc, omega, variant, tight):
    return reference_bound(lambda U, L: orc.mag_sweep_bound(U, L, nc, omega, variant, tight=tight), nc)


@functools.lru_cache(maxsize=None)
def _ref_hb(orc, nc, T, seed, word, tight):
    return reference_bound(lambda U, L: orc.heatbath_sweep_bound(U, L, nc, T, seed, word, tight=tight)[0], nc)


@functools.lru_cache(maxsize=None)
def _ref_maghb(orc, nc, T, seed, word, tight):
    return reference_bound(lambda U, L: orc.mag_heatbath_sweep_bound(U, L, nc, T, seed, word, tight=tight), nc)


def or_reference(orc, U, L, nc, omega=1.7, variant=0):
    """(oracle after one sweep, bound A, A_ref)."""
    ref = U.copy()
    t = tight_for(L)
    A = orc.sweep_bound(ref, L, nc, omega, variant, tight=t)
    return ref, A, _ref_or(orc, nc, float(omega), int(variant), t)


def mag_reference(orc, U, L, nc, omega=1.7, variant=0):
    ref = U.copy()
    t = tight_for(L)
    A = orc.mag_sweep_bound(ref, L, nc, omega, variant, tight=t)
    return ref, A, _ref_mag(orc, nc, float(omega), int(variant), t)


def heatbath_reference(orc, U, L, nc, T, seed, word, precision):
    """(oracle after one heat-bath sweep, bound A (norm rules), A_ref, exempt mask)."""
    ref = U.copy()
    A, slack = orc.heatbath_sweep_bound(ref, L, nc, T, seed, word)
    exempt, _ = heatbath_exempt(L, slack, precision)
    return ref, A, _ref_hb(orc, nc, float(T), int(seed), int(word), False), exempt


def mag_heatbath_reference(orc, U, L, nc, T, seed, word):
    ref = U.copy()
    A = orc.mag_heatbath_sweep_bound(ref, L, nc, T, seed, word)
    return ref, A, _ref_maghb(orc, nc, float(T), int(seed), int(word), False)
