"""CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (element by element on the canonical links):
  FP64 storage, after one sweep: 1e-13
  FP32 storage, after one sweep: 5e-6
  (every link, on well-conditioned input that tolerance itself; on the random
  Haar start scaled per link by the oracle's first-order bound of the link's
  conditioning, tests/parity.py)
  converged F: 1e-10 relative;  plaquette unchanged: 1e-12.
FP32 runs start from the FP32-rounded input on both sides, so only the
arithmetic of one sweep is compared. FP32 theta is formed per site in FP32
and accumulated in FP64; its tolerance, 1e-6 relative plus 1e-5 absolute,
follows from per-element rounding of 6e-8 on sums of 16 links.
"""
import numpy as np
import pytest

import parity as P
from paper_1412_3655_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt
    return culgt


def to_dev(U, dtype=np.float64):
    real = np.ascontiguousarray(U).view(np.float64).astype(dtype)
    return torch.from_numpy(real).cuda()


def from_dev(t, shape):
    a = t.cpu().numpy().astype(np.float64)
    return np.ascontiguousarray(a).view(np.complex128).reshape(shape)


def round32(U):
    return U.view(np.float64).astype(np.float32).astype(np.float64).view(np.complex128)


CASES = [
    # dims, nc: several 128-site tiles with a ragged tail, L1 = 2, non-cubic, tiny
    ((8, 8, 8, 8), 3),
    ((6, 4, 6, 10), 3),
    ((4, 2, 6, 4), 3),
    ((2, 2, 2, 2), 3),
    ((8, 8, 8, 8), 2),
    ((6, 4, 6, 10), 2),
    ((2, 2, 2, 2), 2),
]


def warmed(U, dims, nc, orc, n=5):
    """The input after n oracle sweeps: every site's local problem is then
    well conditioned (K dominated by its positive trace part)."""
    W = U.copy()
    orc.sweep(W, dims, nc, 1.7, n)
    return W


@pytest.mark.parametrize("dims,nc", CASES)
@pytest.mark.parametrize("omega,variant", [(1.7, 0), (1.0, 0), (1.75, 1)])
def test_one_sweep_fp64(cu, orc, dims, nc, omega, variant):
    U0 = synth.gauge_config(dims, nc, 0.3, 2)
    storages = [18, 12] if nc == 3 else [4]
    for U, good in [(U0, False), (warmed(U0, dims, nc, orc), True)]:
        ref, A, A_ref = P.or_reference(orc, U, dims, nc, omega, variant)
        for sr in storages:
            d = to_dev(U)
            p = cu.Params.defaults(nc, dims, omega=omega, or_variant=variant, storage_reals=sr)
            cu.culgt_sweep(d, p, 1)
            P.check_sweep(from_dev(d, U.shape), ref, 1e-13, A, A_ref, good)


@pytest.mark.parametrize("dims,nc", CASES)
def test_one_sweep_fp32(cu, orc, dims, nc):
    U0 = synth.gauge_config(dims, nc, 0.3, 3)
    storages = [12, 18] if nc == 3 else [4]
    for U, good in [(round32(U0), False), (round32(warmed(U0, dims, nc, orc)), True)]:
        ref, A, A_ref = P.or_reference(orc, U, dims, nc)
        for sr in storages:
            d = to_dev(U)
            p = cu.Params.defaults(nc, dims, precision=cu.FP32, storage_reals=sr)
            cu.culgt_sweep(d, p, 1)
            P.check_sweep(from_dev(d, U.shape), ref, 5e-6, A, A_ref, good)


@pytest.mark.parametrize("dims,nc", CASES)
def test_one_sweep_double_float(cu, orc, dims, nc):
    """Double-float sweeps (pairs of floats, unit roundoff 2^-48; products of
    unitary factors to a few 2^-47 absolute): one sweep within 32 x the FP64
    bound, 3.2e-12."""
    U0 = synth.gauge_config(dims, nc, 0.3, 2)
    for U, good in [(U0, False), (warmed(U0, dims, nc, orc), True)]:
        d = to_dev(U)
        p = cu.Params.defaults(nc, dims, precision=cu.DF)
        cu.culgt_sweep(d, p, 1)
        ref, A, A_ref = P.or_reference(orc, U, dims, nc)
        P.check_sweep(from_dev(d, U.shape), ref, 3.2e-12, A, A_ref, good)


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("precision", ["df", "mixed_df"])
def test_landau_fix_double_float(cu, orc, nc, precision):
    """Double-float polish: theta < 1e-12 measured in FP64 on the stored
    pairs, F within 1e-10 of the FP64 oracle, plaquette unchanged to 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    prec = cu.DF if precision == "df" else cu.MIXED_DF
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=3000)
    r = cu.culgt_landau_fix(d, p)
    ref = U.copy()
    rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 3000, 1)
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    th, F = orc.theta(from_dev(d, U.shape), dims, nc)
    assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)


@pytest.mark.parametrize("nc", [2, 3])
def test_float_canonical_buffer(cu, orc, nc):
    dims = (4, 4, 4, 4)
    U = round32(synth.gauge_config(dims, nc, 0.3, 4))
    d = to_dev(U, np.float32)
    p = cu.Params.defaults(nc, dims, precision=cu.FP32, dtype_in=1)
    cu.culgt_sweep(d, p, 1)
    ref = U.copy()
    orc.sweep(ref, dims, nc, 1.7, 1)
    assert np.abs(from_dev(d, U.shape) - ref).max() <= 5e-6


@pytest.mark.parametrize("dims,nc", CASES)
def test_theta_F_plaquette(cu, orc, dims, nc):
    U = synth.gauge_config(dims, nc, 0.3, 5)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims)
    th, F = cu.culgt_theta(d, p)
    th_ref, F_ref = orc.theta(U, dims, nc)
    assert th == pytest.approx(th_ref, rel=1e-12)
    assert F == pytest.approx(F_ref, rel=1e-12, abs=1e-14)
    assert cu.culgt_plaquette(d, p) == pytest.approx(orc.plaquette(U, dims, nc), rel=1e-12)
    U32 = round32(U)
    p32 = cu.Params.defaults(nc, dims, precision=cu.FP32)
    th32, F32 = cu.culgt_theta(to_dev(U32), p32)
    th_ref32, F_ref32 = orc.theta(U32, dims, nc)
    assert th32 == pytest.approx(th_ref32, rel=1e-6, abs=1e-5)
    assert F32 == pytest.approx(F_ref32, rel=1e-6)


@pytest.mark.parametrize("nc", [2, 3])
def test_theta_near_convergence(cu, orc, nc):
    """Small theta (a converged field) is resolved in FP64."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    orc.landau_fix(U, dims, nc, 1.7, 1e-14, 3000, 1)
    th_ref, F_ref = orc.theta(U, dims, nc)
    th, F = cu.culgt_theta(to_dev(U), cu.Params.defaults(nc, dims))
    assert th == pytest.approx(th_ref, rel=1e-6, abs=1e-22)
    assert F == pytest.approx(F_ref, rel=1e-13)


@pytest.mark.parametrize("nc", [2, 3])
def test_reunitarize(cu, orc, nc):
    dims = (4, 4, 2, 6)
    U = synth.gauge_config(dims, nc, 0.3, 6)
    noisy = U + 1e-7 * np.random.default_rng(1).standard_normal(U.shape)
    if nc == 2:  # SU(2) links enter through their quaternion part: keep the noise in it
        noisy = U * (1 + 1e-7 * np.random.default_rng(1).standard_normal(U.shape[:2] + (1, 1)))
    d = to_dev(np.ascontiguousarray(noisy))
    cu.culgt_reunitarize(d, cu.Params.defaults(nc, dims))
    ref = np.ascontiguousarray(noisy).copy()
    orc.reunitarize(ref, nc)
    assert np.abs(from_dev(d, U.shape) - ref).max() <= 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_sweeps_keep_plaquette_and_unitarity(cu, orc, nc):
    dims = (8, 8, 8, 8)
    U = synth.gauge_config(dims, nc, 0.3, 7)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims)
    P0 = cu.culgt_plaquette(d, p)
    cu.culgt_sweep(d, p, 20)
    assert cu.culgt_plaquette(d, p) == pytest.approx(P0, abs=1e-12)
    assert orc.unitarity_error(from_dev(d, U.shape), nc) < 1e-13


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("check_every", [1, 7])
def test_landau_fix_fp64_matches_oracle(cu, orc, nc, check_every):
    """4^4, eps = 0.3, seed 1, omega = 1.7, theta < 1e-12: same sweep count,
    F within 1e-10 relative, plaquette unchanged to 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, check_every=check_every, reunit_every=50, max_sweeps=2000)
    r = cu.culgt_landau_fix(d, p)
    ref = U.copy()
    rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 2000, check_every, 50)
    assert r.status == cu.OK and rr["converged"]
    assert r.sweeps_fp64 == rr["sweeps"]
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.theta < 1e-12
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    assert r.unitarity_err < 1e-13
    assert np.abs(from_dev(d, U.shape) - ref).max() < 1e-9


@pytest.mark.parametrize("nc", [2, 3])
def test_landau_fix_mixed(cu, orc, nc):
    """FP32 to theta < 1e-8, then FP64 to 1e-12: same local maximum as the
    FP64 oracle here, F within 1e-10 relative. The switch rebuilds the FP64
    links from the input and the accumulated g, so the result is a gauge
    transform of the input: plaquette to 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, precision=cu.MIXED, check_every=5, reunit_every=50, max_sweeps=3000)
    r = cu.culgt_landau_fix(d, p)
    ref = U.copy()
    rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 3000, 1)
    assert r.status == cu.OK
    assert r.sweeps_fp32 > 0 and r.sweeps_fp64 > 0
    assert r.theta < 1e-12
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    th, F = orc.theta(from_dev(d, U.shape), dims, nc)
    assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_landau_fix_automatic_switch(cu, orc, nc, dims, precision):
    """switch_theta = 0: the FP32 phase runs past theta < 1e-8 until a check
    interval no longer lowers theta, then the orbit-exact switch and the
    FP64-class polish to 1e-12. Final F within 1e-10 of the FP64 oracle's,
    plaquette unchanged to 1e-12, and at least as many FP32 sweeps as with
    the switch at 1e-8."""
    prec = cu.MIXED if precision == "mixed" else cu.MIXED_DF
    U = synth.gauge_config(dims, nc, 0.3, 1)
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=6000,
                           switch_theta=0.0)
    d = to_dev(U)
    r = cu.culgt_landau_fix(d, p)
    r8 = cu.culgt_landau_fix(to_dev(U), cu.Params(**{**p.__dict__, "switch_theta": 1e-8}))
    ref = U.copy()
    rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 6000, 1)
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.sweeps_fp32 >= r8.sweeps_fp32 and r.sweeps_fp64 > 0
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    th, F = orc.theta(from_dev(d, U.shape), dims, nc)
    assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)


def test_not_converged_status(cu):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, 3, 0.3, 1)
    p = cu.Params.defaults(3, dims, max_sweeps=3, check_every=2)
    r = cu.culgt_landau_fix(to_dev(U), p)
    assert r.status == cu.NOT_CONVERGED and r.sweeps_fp64 == 3


def test_nonfinite_input_is_reported(cu):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, 3, 0.3, 1)
    U[17, 2, 1, 1] = np.nan
    with pytest.raises(cu.CulgtError) as e:
        cu.culgt_landau_fix(to_dev(U), cu.Params.defaults(3, dims))
    assert e.value.status == cu.ERR_NONFINITE


def test_host_entry_point_matches_device(cu):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, 3, 0.3, 1)
    p = cu.Params.defaults(3, dims, check_every=5)
    d = to_dev(U)
    r1 = cu.culgt_landau_fix(d, p)
    h = torch.from_numpy(U.view(np.float64).copy())
    r2 = cu.culgt_landau_fix_host(h, p)
    assert r1.sweeps_fp64 == r2.sweeps_fp64 and r1.F == r2.F
    assert torch.equal(h, d.cpu())


@pytest.mark.parametrize("nc", [2, 3])
def test_mixed_switch_is_orbit_exact(cu, orc, nc):
    """Mixed handle: two FP32 sweeps, the switch, one FP64 sweep. After the
    switch the FP64 links are a gauge transform of the FP64 input (plaquette
    to 1e-13, unitary), close to two FP64 oracle sweeps (FP32 accuracy), and
    the FP64 sweep from there matches the oracle's sweep of the same state to 1e-13."""
    dims = (6, 4, 6, 10)
    U = synth.gauge_config(dims, nc, 0.3, 8)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, precision=cu.MIXED)
    with cu.Handle(p) as h:
        h.culgt_load(d)
        h.culgt_handle_sweep(2)
        h.culgt_handle_to_fp64()
        mid = torch.empty_like(d)
        h.culgt_store(mid)
        h.culgt_handle_sweep(1)
        th, F = h.culgt_handle_theta()
        out = torch.empty_like(d)
        h.culgt_store(out)
        torch.cuda.synchronize()
    after_switch = from_dev(mid, U.shape)
    assert orc.plaquette(after_switch, dims, nc) == pytest.approx(orc.plaquette(U, dims, nc), abs=1e-13)
    assert orc.unitarity_error(after_switch, nc) < 1e-14
    two = U.copy()
    orc.sweep(two, dims, nc, 1.7, 2)
    assert np.abs(after_switch - two).max() < 1e-4
    ref = after_switch.copy()
    orc.sweep(ref, dims, nc, 1.7, 1)
    got = from_dev(out, U.shape)
    assert np.abs(got - ref).max() <= 1e-13
    th_ref, F_ref = orc.theta(got, dims, nc)
    assert th == pytest.approx(th_ref, rel=1e-12) and F == pytest.approx(F_ref, rel=1e-13)


@pytest.mark.parametrize("nc", [3, 2])
def test_full_size_32_one_sweep(cu, orc, nc):
    """32^4 (the throughput workload), the whole lattice: one FP64 sweep and
    one FP32 sweep (12-real SU(3), quaternion SU(2)) against the oracle, from
    the random Haar start, and from the same field under a gauge close to 1
    instead (every site well conditioned; a million sites of the random start
    still contain ill-conditioned ones after tens of sweeps)."""
    dims = (32, 32, 32, 32)
    U = synth.gauge_config(dims, nc, 0.3, 2)
    W = synth.gauge_config(dims, nc, 0.3, 2, spread=0.3)
    for X, good in [(U, False), (W, True)]:
        ref, A, A_ref = P.or_reference(orc, X, dims, nc)
        d = to_dev(X)
        cu.culgt_sweep(d, cu.Params.defaults(nc, dims), 1)
        P.check_sweep(from_dev(d, X.shape), ref, 1e-13, A, A_ref, good)
        del d
        X32 = round32(X)
        ref, A, A_ref = P.or_reference(orc, X32, dims, nc)
        d = to_dev(X32)
        cu.culgt_sweep(d, cu.Params.defaults(nc, dims, precision=cu.FP32), 1)
        P.check_sweep(from_dev(d, X.shape), ref, 5e-6, A, A_ref, good)
        del d


def test_full_size_64_one_sweep(cu, orc):
    """64^4 SU(3) (16.8M sites, eps 0.25, seed 3, omega 1.75: the largest
    lattice of the measurements), the whole lattice in the mapping the
    autotuner picks for it: one FP64 18-real sweep and one FP32 12-real sweep
    against the oracle, from the random Haar start (every link within its
    conditioning-scaled tolerance)."""
    dims = (64, 64, 64, 64)
    U = synth.gauge_config(dims, 3, 0.25, 3)
    ref, A, A_ref = P.or_reference(orc, U, dims, 3, 1.75)
    d = to_dev(U)
    cu.culgt_sweep(d, cu.Params.defaults(3, dims, omega=1.75), 1)
    P.check_sweep(from_dev(d, U.shape), ref, 1e-13, A, A_ref, False)
    del d, ref, A
    U = round32(U)
    ref, A, A_ref = P.or_reference(orc, U, dims, 3, 1.75)
    d = to_dev(U)
    cu.culgt_sweep(d, cu.Params.defaults(3, dims, omega=1.75, precision=cu.FP32), 1)
    P.check_sweep(from_dev(d, U.shape), ref, 5e-6, A, A_ref, False)


@pytest.mark.parametrize("nc,precision,storage", [(3, 0, 18), (3, 0, 12), (3, 1, 12), (3, 1, 18), (3, 4, 0),
                                                  (2, 0, 4), (2, 1, 4), (2, 4, 0), (3, 2, 12), (2, 2, 4)])
def test_every_mapping_gives_identical_links(cu, nc, precision, storage):
    """The autotuner's choices (1 or 2 threads per site, 64/128/256 threads per
    block, register limits) all form K in the same order, so the links agree
    bit for bit (the mixed cases cover the FP32 phase that also accumulates g)."""
    dims = (6, 4, 6, 10)
    U = synth.gauge_config(dims, nc, 0.3, 9)
    outs = []
    mappings = [(1, 64, 1), (1, 128, 1), (1, 256, 1), (1, 128, 3), (1, 128, 4), (2, 64, 1), (2, 128, 1),
                (2, 256, 1), (2, 128, 4)]
    for tps, block, minb in mappings:
        if True:
            p = cu.Params.defaults(nc, dims, precision=precision, storage_reals=storage, threads_per_site=tps,
                                   block_size=block, min_blocks_per_sm=minb)
            d = to_dev(U)
            with cu.Handle(p) as h:
                h.culgt_load(d)
                assert h.culgt_handle_tuning() == (tps, block, minb)
                h.culgt_handle_sweep(2)
                if precision == 2:
                    h.culgt_handle_to_fp64()
                    h.culgt_handle_sweep(1)
                out = torch.empty_like(d)
                h.culgt_store(out)
                torch.cuda.synchronize()
            outs.append(out)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_autotuner_picks_a_valid_mapping(cu):
    dims = (16, 16, 16, 32)
    U = synth.gauge_config(dims, 3, 0.3, 1)
    for prec in (cu.FP32, cu.FP64, cu.DF):
        with cu.Handle(cu.Params.defaults(3, dims, precision=prec)) as h:
            h.culgt_load(to_dev(U))
            tps, block, minb = h.culgt_handle_tuning()
            assert tps in (1, 2) and block in (64, 128, 256) and minb in (1, 3, 4)


@pytest.mark.parametrize("nc", [2, 3])
def test_checkpoint_and_resume(cu, nc):
    """culgt_store is the checkpoint and culgt_load the resume: a fix stopped
    at 20 sweeps, written to the canonical buffer and continued in a new
    handle ends bit for bit where the uninterrupted fix ends (FP64-18 and the
    canonical layout round-trip exactly; 20 is a multiple of the theta and
    reunitarisation cadences)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    p = cu.Params.defaults(nc, dims, check_every=10, reunit_every=20, max_sweeps=2000)
    whole = to_dev(U)
    rw = cu.culgt_landau_fix(whole, p)
    assert rw.sweeps_fp64 > 20
    part = to_dev(U)
    first = cu.Params(**{**p.__dict__, "max_sweeps": 20})
    r1 = cu.culgt_landau_fix(part, first)
    assert r1.status == cu.NOT_CONVERGED and r1.sweeps_fp64 == 20
    rest = cu.Params(**{**p.__dict__, "max_sweeps": 2000 - 20})
    r2 = cu.culgt_landau_fix(part, rest)
    assert r2.sweeps_fp64 + 20 == rw.sweeps_fp64
    assert torch.equal(part, whole)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nc", [2, 3])
def test_degenerate_block_is_left_alone(cu, orc, nc, precision):
    """det = 0 (reading 4): all links 1 except the four backward links of the
    origin, -1 (SU(2)) or diag(-1, -1, 1) (SU(3)), so K(0) = 0 (SU(2)) or its
    (0,1) block is 0 (SU(3)). One sweep matches the oracle, which leaves that
    block alone."""
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(nc, dtype=complex), (V, 4, nc, nc)).copy()
    m = -np.eye(2, dtype=complex) if nc == 2 else np.diag([-1.0 + 0j, -1.0, 1.0])
    for mu in range(4):
        ib = int(np.flatnonzero(synth.site_neighbour_forward(dims, mu) == 0)[0])
        U[ib, mu] = m
    ref = U.copy()
    orc.sweep(ref, dims, nc, 1.7, 1)
    prec = cu.FP64 if precision == "fp64" else cu.FP32
    d = to_dev(U)
    cu.culgt_sweep(d, cu.Params.defaults(nc, dims, precision=prec), 1)
    got = from_dev(d, U.shape)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() < (1e-14 if prec == cu.FP64 else 1e-6)
