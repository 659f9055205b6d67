"""FP64 CPU oracle for checkerboard-overrelaxation gauge fixing (test infrastructure).

A thin ctypes binding over ``culgt_oracle.c``: a plain, slow restatement of
lattice Landau/Coulomb gauge fixing as defined in Vogt & Schröck, "cuLGT:
Lattice Gauge Fixing on GPUs", Sec. 2, and of the simulated annealing the paper
combines with it (heat bath over the SU(2) subgroups, readings R7-R11 in
``culgt_oracle.c``), and of maximally Abelian gauge fixing (R12-R15). Only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` use this module; the CUDA library never
does, and the two share no code.

Link arrays are numpy ``complex128`` of shape ``(V, 4, Nc, Nc)`` in the canonical
site order ``i = x1 + L1 (x2 + L2 (x3 + L3 x0))`` with dims ``L = (L0, L1, L2, L3)``,
``L0`` = time.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "culgt_oracle.c")
_LIB = os.path.join(_HERE, "libculgt_oracle.so")

# -ffp-contract=off: no fused multiply-adds, so x86 and Arm builds round alike.
CFLAGS = ["-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (a second or two). Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i, d = ctypes.c_int, ctypes.c_double
    u32p = ctypes.POINTER(ctypes.c_uint32)
    sig = {
        "oracle_halfsweep": (None, [dp, ip, i, i, d, i]),
        "oracle_sweep": (None, [dp, ip, i, d, i, i]),
        "oracle_theta": (None, [dp, ip, i, dp, dp]),
        "oracle_plaquette": (d, [dp, ip, i]),
        "oracle_reunitarize": (None, [dp, ctypes.c_long, i]),
        "oracle_unitarity_error": (d, [dp, ctypes.c_long, i]),
        "oracle_landau_fix": (i, [dp, ip, i, d, i, d, i, i, i, ip, dp, dp]),
        "oracle_theta_slice": (None, [dp, ip, i, i, dp, dp]),
        "oracle_coulomb_fix": (i, [dp, ip, i, d, i, d, i, i, i, dp, ip, dp, dp]),
        "oracle_local_gauge": (None, [dp, i, d, i, dp]),
        "oracle_su2_local_max": (None, [dp, dp]),
        "oracle_overrelax": (None, [dp, d, i, dp]),
        "oracle_philox4x32_10": (None, [u32p, u32p, u32p]),
        "oracle_hb_delta": (d, [d, u32p, ctypes.c_uint32, ctypes.c_uint32, i, ip]),
        "oracle_hb_x": (None, [d, u32p, ctypes.c_uint32, ctypes.c_uint32, i, dp]),
        "oracle_heatbath_gauge": (None, [dp, i, d, u32p, ctypes.c_uint32, ctypes.c_uint32, dp]),
        "oracle_heatbath_halfsweep": (None, [dp, ip, i, i, d, u32p, ctypes.c_uint32, dp]),
        "oracle_heatbath_sweep": (None, [dp, ip, i, d, u32p, ctypes.c_uint32, dp]),
        "oracle_micro_sweep": (None, [dp, ip, i]),
        "oracle_anneal": (None, [dp, ip, i, d, d, i, i, u32p, i]),
        "oracle_mag_halfsweep": (None, [dp, ip, i, i, d, i]),
        "oracle_mag_sweep": (None, [dp, ip, i, d, i, i]),
        "oracle_mag_theta": (None, [dp, ip, i, dp, dp]),
        "oracle_mag_fix": (i, [dp, ip, i, d, i, d, i, i, i, ip, dp, dp]),
        "oracle_mag_local_gauge": (None, [dp, i, d, i, dp]),
        "oracle_mag_su2_max": (None, [dp, dp]),
        "oracle_coulomb_fix_anneal": (i, [dp, ip, i, d, d, i, i, u32p, d, i, d, i, i, i, dp, ip, dp, dp]),
        "oracle_mag_heatbath_halfsweep": (None, [dp, ip, i, i, d, u32p, ctypes.c_uint32]),
        "oracle_mag_heatbath_sweep": (None, [dp, ip, i, d, u32p, ctypes.c_uint32]),
        "oracle_mag_anneal": (None, [dp, ip, i, d, d, i, i, u32p, i]),
        "oracle_mag_heatbath_su2": (None, [dp, d, u32p, ctypes.c_uint32, ctypes.c_uint32, i, dp]),
        "oracle_sweep_bound": (None, [dp, ip, i, d, i, d, dp, i]),
        "oracle_local_gauge_bound": (d, [dp, i, d, i]),
        "oracle_hb_slack": (d, [d, d, d, u32p, ctypes.c_uint32, ctypes.c_uint32, i]),
        "oracle_heatbath_gauge_bound": (d, [dp, i, d, u32p, ctypes.c_uint32, ctypes.c_uint32, d, dp]),
        "oracle_mag_local_gauge_bound": (d, [dp, i, d, i]),
        "oracle_mag_sweep_bound": (None, [dp, ip, i, d, i, d, dp, i]),
        "oracle_heatbath_sweep_bound": (None, [dp, ip, i, d, u32p, ctypes.c_uint32, d, dp, dp, i]),
        "oracle_mag_heatbath_sweep_bound": (None, [dp, ip, i, d, u32p, ctypes.c_uint32, d, dp, i]),
        "oracle_tangent_bound": (d, [dp, i, i, d, i, d, u32p, ctypes.c_uint32, ctypes.c_uint32]),
        "oracle_mag_heatbath_gauge": (None, [dp, i, d, u32p, ctypes.c_uint32, ctypes.c_uint32, dp]),
        "oracle_set_threads": (None, [i]),
        "oracle_get_threads": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    assert a.dtype in (np.float64, np.complex128)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(L):
    arr = (ctypes.c_int * 4)(*[int(x) for x in L])
    return arr


def _check_links(U: np.ndarray, L, nc: int):
    V = int(np.prod(L))
    if U.shape != (V, 4, nc, nc) or U.dtype != np.complex128 or not U.flags["C_CONTIGUOUS"]:
        raise ValueError(f"links must be contiguous complex128 of shape {(V, 4, nc, nc)}")


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def halfsweep(U, L, nc, parity, omega, variant=0):
    """Overrelaxation update of every site of one parity (0 = black = even), in place."""
    _check_links(U, L, nc)
    _load().oracle_halfsweep(_dp(U), _dims(L), nc, int(parity), float(omega), int(variant))


def sweep(U, L, nc, omega, n_sweeps=1, variant=0):
    """n_sweeps x (black half-sweep, white half-sweep), in place."""
    _check_links(U, L, nc)
    _load().oracle_sweep(_dp(U), _dims(L), nc, float(omega), int(variant), int(n_sweeps))


def theta(U, L, nc):
    """Returns (theta, F): theta = (1/V) sum_x tr[Delta Delta^+], F the Landau functional."""
    _check_links(U, L, nc)
    th, F = ctypes.c_double(), ctypes.c_double()
    _load().oracle_theta(_dp(U), _dims(L), nc, ctypes.byref(th), ctypes.byref(F))
    return th.value, F.value


def plaquette(U, L, nc):
    _check_links(U, L, nc)
    return float(_load().oracle_plaquette(_dp(U), _dims(L), nc))


def reunitarize(M, nc):
    """In place over an array of Nc x Nc complex matrices (any leading shape)."""
    assert M.dtype == np.complex128 and M.shape[-2:] == (nc, nc) and M.flags["C_CONTIGUOUS"]
    _load().oracle_reunitarize(_dp(M), int(M.size // (nc * nc)), nc)


def unitarity_error(M, nc):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    return float(_load().oracle_unitarity_error(_dp(M), int(M.size // (nc * nc)), nc))


def landau_fix(U, L, nc, omega, theta_target, max_sweeps, check_every=1, reunit_every=0, variant=0):
    """Iterate sweeps until theta < theta_target or max_sweeps, in place.

    Returns dict(converged, sweeps, theta, F)."""
    _check_links(U, L, nc)
    n, th, F = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    rc = _load().oracle_landau_fix(_dp(U), _dims(L), nc, float(omega), int(variant), float(theta_target),
                                   int(max_sweeps), int(check_every), int(reunit_every), ctypes.byref(n),
                                   ctypes.byref(th), ctypes.byref(F))
    return {"converged": rc == 0, "sweeps": n.value, "theta": th.value, "F": F.value}


def theta_slice(U, L, nc, t):
    """(theta_t, F_t) of time slice t for the Coulomb functional (mu = 1..3)."""
    _check_links(U, L, nc)
    th, F = ctypes.c_double(), ctypes.c_double()
    _load().oracle_theta_slice(_dp(U), _dims(L), nc, int(t), ctypes.byref(th), ctypes.byref(F))
    return th.value, F.value


def coulomb_fix(U, L, nc, omega, theta_target, max_sweeps, check_every=1, reunit_every=0, variant=0):
    """Per-slice Coulomb gauge fixing, in place. Returns dict with per-slice arrays and the
    accumulated gauge transformation g (V, Nc, Nc)."""
    _check_links(U, L, nc)
    V = int(np.prod(L))
    g = np.zeros((V, nc, nc), dtype=np.complex128)
    nt = int(L[0])
    sw = (ctypes.c_int * nt)()
    th = np.zeros(nt)
    F = np.zeros(nt)
    rc = _load().oracle_coulomb_fix(_dp(U), _dims(L), nc, float(omega), int(variant), float(theta_target),
                                    int(max_sweeps), int(check_every), int(reunit_every), _dp(g), sw, _dp(th),
                                    _dp(F))
    return {"converged": rc == 0, "sweeps": np.array(list(sw)), "theta": th, "F": F, "g": g}


def local_gauge(K, omega, variant=0):
    """The overrelaxed local transformation g for one gathered K (Nc x Nc)."""
    K = np.ascontiguousarray(K, dtype=np.complex128)
    nc = K.shape[0]
    g = np.zeros((nc, nc), dtype=np.complex128)
    _load().oracle_local_gauge(_dp(K), nc, float(omega), int(variant), _dp(g))
    return g


def su2_local_max(w):
    w = np.ascontiguousarray(w, dtype=np.complex128)
    r = np.zeros((2, 2), dtype=np.complex128)
    _load().oracle_su2_local_max(_dp(w), _dp(r))
    return r


def overrelax(g, omega, variant=0):
    g = np.ascontiguousarray(g, dtype=np.complex128)
    out = np.zeros((2, 2), dtype=np.complex128)
    _load().oracle_overrelax(_dp(g), float(omega), int(variant), _dp(out))
    return out


# --- simulated annealing (readings R7-R11 of culgt_oracle.c) ---

def _key(seed: int):
    """The Philox key of a 64-bit seed: (low word, high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (ctypes.c_uint32 * 2)(seed & 0xFFFFFFFF, seed >> 32)


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter (4 words) and key (2 words); returns 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (ctypes.c_uint32 * 4)()
    _load().oracle_philox4x32_10(c, k, out)
    return tuple(int(x) for x in out)


def hb_delta(alpha, seed, site, sweep, sub=0):
    """(delta, attempts): delta = 1 - x0 of one heat-bath draw at alpha = 2 k / T."""
    n = ctypes.c_int()
    dlt = _load().oracle_hb_delta(float(alpha), _key(seed), int(site), int(sweep), int(sub), ctypes.byref(n))
    return float(dlt), n.value


def hb_x(alpha, seed, site, sweep, sub=0):
    """The unit quaternion (x0, x1, x2, x3) of one heat-bath draw."""
    x = np.zeros(4)
    _load().oracle_hb_x(float(alpha), _key(seed), int(site), int(sweep), int(sub), _dp(x))
    return x


def heatbath_gauge(K, T, seed, site, sweep):
    """The heat-bath transformation g of one site with gathered K (Nc x Nc)."""
    K = np.ascontiguousarray(K, dtype=np.complex128)
    nc = K.shape[0]
    g = np.zeros((nc, nc), dtype=np.complex128)
    _load().oracle_heatbath_gauge(_dp(K), nc, float(T), _key(seed), int(site), int(sweep), _dp(g))
    return g


def heatbath_sweep(U, L, nc, T, seed, sweep, gacc=None):
    """One heat-bath sweep at temperature T (draw counter word `sweep`), in place.
    gacc (V, Nc, Nc) complex128, if given, accumulates g(x) gacc(x)."""
    _check_links(U, L, nc)
    g = None
    if gacc is not None:
        assert gacc.dtype == np.complex128 and gacc.flags["C_CONTIGUOUS"]
        g = _dp(gacc)
    _load().oracle_heatbath_sweep(_dp(U), _dims(L), nc, float(T), _key(seed), int(sweep), g)


def heatbath_halfsweep(U, L, nc, parity, T, seed, sweep):
    """Heat-bath update of every site of one parity (0 = black), in place."""
    _check_links(U, L, nc)
    _load().oracle_heatbath_halfsweep(_dp(U), _dims(L), nc, int(parity), float(T), _key(seed), int(sweep), None)


def micro_sweep(U, L, nc):
    """One microcanonical (omega = 2) sweep, in place."""
    _check_links(U, L, nc)
    _load().oracle_micro_sweep(_dp(U), _dims(L), nc)


def anneal(U, L, nc, t_start, t_end, steps, n_micro, seed, reunit_every=0):
    """The annealing schedule of R11, in place (no overrelaxation afterwards)."""
    _check_links(U, L, nc)
    _load().oracle_anneal(_dp(U), _dims(L), nc, float(t_start), float(t_end), int(steps), int(n_micro),
                          _key(seed), int(reunit_every))


# --- maximally Abelian gauge (readings R12-R15 of culgt_oracle.c) ---

def mag_halfsweep(U, L, nc, parity, omega, variant=0):
    _check_links(U, L, nc)
    _load().oracle_mag_halfsweep(_dp(U), _dims(L), nc, int(parity), float(omega), int(variant))


def mag_sweep(U, L, nc, omega, n_sweeps=1, variant=0):
    _check_links(U, L, nc)
    _load().oracle_mag_sweep(_dp(U), _dims(L), nc, float(omega), int(variant), int(n_sweeps))


def mag_theta(U, L, nc):
    """(theta_MAG, F_MAG)."""
    _check_links(U, L, nc)
    th, F = ctypes.c_double(), ctypes.c_double()
    _load().oracle_mag_theta(_dp(U), _dims(L), nc, ctypes.byref(th), ctypes.byref(F))
    return th.value, F.value


def mag_fix(U, L, nc, omega, theta_target, max_sweeps, check_every=1, reunit_every=0, variant=0):
    """MAG fixing in place. Returns dict(converged, sweeps, theta, F)."""
    _check_links(U, L, nc)
    n, th, F = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    rc = _load().oracle_mag_fix(_dp(U), _dims(L), nc, float(omega), int(variant), float(theta_target),
                                int(max_sweeps), int(check_every), int(reunit_every), ctypes.byref(n),
                                ctypes.byref(th), ctypes.byref(F))
    return {"converged": rc == 0, "sweeps": n.value, "theta": th.value, "F": F.value}


def mag_local_gauge(X, omega, variant=0):
    """The MAG site transformation for X_0..X_{Nc-1} (array (Nc, Nc, Nc)); returns (g, rotated X)."""
    X = np.ascontiguousarray(X, dtype=np.complex128).copy()
    nc = X.shape[-1]
    g = np.zeros((nc, nc), dtype=np.complex128)
    _load().oracle_mag_local_gauge(_dp(X), nc, float(omega), int(variant), _dp(g))
    return g, X


def mag_su2_max(Z):
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    B = np.zeros((2, 2), dtype=np.complex128)
    _load().oracle_mag_su2_max(_dp(Z), _dp(B))
    return B


def coulomb_fix_anneal(U, L, nc, t_start, t_end, steps, n_micro, seed, omega, theta_target, max_sweeps,
                       check_every=1, reunit_every=0, variant=0):
    """Coulomb gauge fixing with every time slice annealed first (slice t keyed
    by seed + t). Returns the dict of coulomb_fix."""
    _check_links(U, L, nc)
    V = int(np.prod(L))
    g = np.zeros((V, nc, nc), dtype=np.complex128)
    nt = int(L[0])
    sw = (ctypes.c_int * nt)()
    th = np.zeros(nt)
    F = np.zeros(nt)
    rc = _load().oracle_coulomb_fix_anneal(_dp(U), _dims(L), nc, float(t_start), float(t_end), int(steps),
                                           int(n_micro), _key(seed), float(omega), int(variant), float(theta_target),
                                           int(max_sweeps), int(check_every), int(reunit_every), _dp(g), sw, _dp(th),
                                           _dp(F))
    return {"converged": rc == 0, "sweeps": np.array(list(sw)), "theta": th, "F": F, "g": g}


def mag_heatbath_sweep(U, L, nc, T, seed, sweep):
    """One MAG heat-bath sweep at temperature T (draw counter word `sweep`), in place."""
    _check_links(U, L, nc)
    _load().oracle_mag_heatbath_sweep(_dp(U), _dims(L), nc, float(T), _key(seed), int(sweep))


def mag_heatbath_halfsweep(U, L, nc, parity, T, seed, sweep):
    _check_links(U, L, nc)
    _load().oracle_mag_heatbath_halfsweep(_dp(U), _dims(L), nc, int(parity), float(T), _key(seed), int(sweep))


def mag_anneal(U, L, nc, t_start, t_end, steps, n_micro, seed, reunit_every=0):
    """The annealing schedule with MAG heat-bath and microcanonical sweeps, in place."""
    _check_links(U, L, nc)
    _load().oracle_mag_anneal(_dp(U), _dims(L), nc, float(t_start), float(t_end), int(steps), int(n_micro),
                              _key(seed), int(reunit_every))


def mag_heatbath_su2(Z, T, seed, site, sweep, sub=0):
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    B = np.zeros((2, 2), dtype=np.complex128)
    _load().oracle_mag_heatbath_su2(_dp(Z), float(T), _key(seed), int(site), int(sweep), int(sub), _dp(B))
    return B


# --- first-order error bounds of one sweep (for comparing another implementation) ---

def _bound_array(e, V):
    if e is None:
        return np.ones((V, 4))
    e = np.ascontiguousarray(e, dtype=np.float64).copy()
    if e.shape != (V, 4):
        raise ValueError(f"e must have shape {(V, 4)}")
    return e


def sweep_bound(U, L, nc, omega, variant=0, e=None, rho=1.0, tight=False):
    """One overrelaxation sweep, in place, exactly as sweep(); returns the
    first-order bound (V, 4) on how far each output link can move when every
    input link carries the error in e (default: one unit each) and every
    rounding step of the sweep is charged rho units. tight: each SU(3) site's
    g is also bounded through its exact tangent map (tangent_bound), and the
    smaller bound kept (slower)."""
    _check_links(U, L, nc)
    e = _bound_array(e, U.shape[0])
    _load().oracle_sweep_bound(_dp(U), _dims(L), nc, float(omega), int(variant), float(rho), _dp(e), int(tight))
    return e


def mag_sweep_bound(U, L, nc, omega, variant=0, e=None, rho=1.0, tight=False):
    """One MAG sweep, in place, with the bounds of sweep_bound."""
    _check_links(U, L, nc)
    e = _bound_array(e, U.shape[0])
    _load().oracle_mag_sweep_bound(_dp(U), _dims(L), nc, float(omega), int(variant), float(rho), _dp(e),
                                   int(tight))
    return e


def heatbath_sweep_bound(U, L, nc, T, seed, sweep, e=None, rho=1.0, tight=False):
    """One heat-bath sweep, in place, exactly as heatbath_sweep(); returns
    (e, slack): the bounds of sweep_bound and, per site, the smallest slack
    of its draws' decisions (margin over its own error bound, in units of
    the per-step charge): an implementation whose unit roundoff exceeds the
    slack may take that decision the other way. tight bounds the effect of
    input errors through the tangent map but charges the draws' own rounding
    as one step only; comparisons with another implementation take the norm
    bound."""
    _check_links(U, L, nc)
    e = _bound_array(e, U.shape[0])
    slack = np.full(U.shape[0], np.inf)
    _load().oracle_heatbath_sweep_bound(_dp(U), _dims(L), nc, float(T), _key(seed), int(sweep), float(rho),
                                        _dp(e), _dp(slack), int(tight))
    return e, slack


def mag_heatbath_sweep_bound(U, L, nc, T, seed, sweep, e=None, rho=1.0, tight=False):
    """One MAG heat-bath sweep, in place, with the bounds of sweep_bound."""
    _check_links(U, L, nc)
    e = _bound_array(e, U.shape[0])
    _load().oracle_mag_heatbath_sweep_bound(_dp(U), _dims(L), nc, float(T), _key(seed), int(sweep), float(rho),
                                            _dp(e), int(tight))
    return e


def local_gauge_bound(K, omega, variant=0):
    """First-order bound on ||dg|| per unit ||dK|| for the site transformation of K."""
    K = np.ascontiguousarray(K, dtype=np.complex128)
    return float(_load().oracle_local_gauge_bound(_dp(K), K.shape[0], float(omega), int(variant)))


def tangent_bound(inp, mag=False, hb=False, omega=1.7, variant=0, T=1.0, seed=0, site=0, sweep=0):
    """The tangent bound of one SU(3) site transformation, without rounding:
    ||dg|| per unit ||dK|| (inp = K, 3 x 3) or per unit max_a ||dX_a||
    (mag, inp = X, 3 x 3 x 3); overrelaxation, or the heat bath at T with
    the draws of (seed, site, sweep)."""
    inp = np.ascontiguousarray(inp, dtype=np.complex128)
    return float(_load().oracle_tangent_bound(_dp(inp), int(mag), int(hb), float(omega), int(variant), float(T),
                                              _key(seed), int(site), int(sweep)))


def mag_heatbath_gauge(X, T, seed, site, sweep):
    """The MAG heat-bath transformation g of one site with gathered X_a."""
    X = np.ascontiguousarray(X, dtype=np.complex128).copy()
    nc = X.shape[-1]
    g = np.zeros((nc, nc), dtype=np.complex128)
    _load().oracle_mag_heatbath_gauge(_dp(X), nc, float(T), _key(seed), int(site), int(sweep), _dp(g))
    return g


def mag_local_gauge_bound(X, omega, variant=0):
    """First-order bound on ||dg|| per unit max_a ||dX_a|| for the MAG site transformation."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    return float(_load().oracle_mag_local_gauge_bound(_dp(X), X.shape[-1], float(omega), int(variant)))


def hb_slack(alpha, dalpha, T, seed, site, sweep, sub=0):
    """Decision slack of one heat-bath draw whose alpha is known to within dalpha."""
    return float(_load().oracle_hb_slack(float(alpha), float(dalpha), float(T), _key(seed), int(site), int(sweep),
                                         int(sub)))


def heatbath_gauge_bound(K, T, seed, site, sweep, dK=1e-7):
    """(bound on ||dg|| per unit ||dK|| of the heat-bath site transformation
    with its draws' decisions held, smallest decision slack for errors up to dK)."""
    K = np.ascontiguousarray(K, dtype=np.complex128)
    sl = ctypes.c_double()
    b = _load().oracle_heatbath_gauge_bound(_dp(K), K.shape[0], float(T), _key(seed), int(site), int(sweep),
                                            float(dK), ctypes.byref(sl))
    return float(b), sl.value
