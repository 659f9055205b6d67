"""Maximally Abelian gauge on the GPU against the FP64 oracle, through the C ABI.

One MAG sweep element by element (FP64 1e-13, FP32 5e-6, on every link of
well-conditioned input; on the random Haar start each link's tolerance scaled
by the oracle's first-order bound of its conditioning, tests/parity.py),
theta_MAG and F_MAG to 1e-12 relative, MAG fixing with the oracle's sweep count
and F_MAG within 1e-10, the plaquette unchanged to 1e-12. The MAG maximiser of
a block turns its vector z onto +e3; where z is short or points close to -e3
the rotation axis is ill conditioned, as |a| small is for the Landau maximiser,
and the bound grows with 1 / sqrt(2 |z| (|z| + z3)).
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


def to_dev(U):
    return torch.from_numpy(np.ascontiguousarray(U).view(np.float64).copy()).cuda()


def from_dev(t, shape):
    return np.ascontiguousarray(t.cpu().numpy()).view(np.complex128).reshape(shape)


def round32(U):
    return U.view(np.float64).astype(np.float32).astype(np.float64).view(np.complex128)


def mag_warmed(U, dims, nc, orc, n=5):
    W = U.copy()
    orc.mag_sweep(W, dims, nc, 1.7, n)
    return W


CASES = [((8, 8, 8, 8), 3), ((6, 4, 6, 10), 3), ((2, 2, 2, 2), 3), ((8, 8, 8, 8), 2), ((6, 4, 6, 10), 2)]


@pytest.mark.parametrize("dims,nc", CASES)
@pytest.mark.parametrize("omega,variant", [(1.7, 0), (1.0, 0), (1.5, 1)])
def test_one_mag_sweep_fp64(cu, orc, dims, nc, omega, variant):
    U0 = synth.gauge_config(dims, nc, 0.3, 2)
    storages = [18, 12] if nc == 3 else [4]
    for U, good in [(U0, False), (mag_warmed(U0, dims, nc, orc), True)]:
        ref, A, A_ref = P.mag_reference(orc, U, dims, nc, omega, variant)
        for sr in storages:
            d = to_dev(U)
            p = cu.Params.defaults(nc, dims, omega=omega, or_variant=variant, storage_reals=sr, gauge=cu.MAG)
            cu.culgt_sweep(d, p, 1)
            P.check_sweep(from_dev(d, U.shape), ref, 1e-13, A, A_ref, good)


@pytest.mark.parametrize("dims,nc", CASES)
def test_one_mag_sweep_fp32(cu, orc, dims, nc):
    U0 = synth.gauge_config(dims, nc, 0.3, 3)
    for U, good in [(round32(U0), False), (round32(mag_warmed(U0, dims, nc, orc)), True)]:
        ref, A, A_ref = P.mag_reference(orc, U, dims, nc)
        for sr in ([12, 18] if nc == 3 else [4]):
            d = to_dev(U)
            p = cu.Params.defaults(nc, dims, precision=cu.FP32, storage_reals=sr, gauge=cu.MAG)
            cu.culgt_sweep(d, p, 1)
            P.check_sweep(from_dev(d, U.shape), ref, 5e-6, A, A_ref, good)


@pytest.mark.parametrize("nc", [2, 3])
def test_one_mag_sweep_double_float(cu, orc, nc):
    dims = (8, 8, 8, 8)
    U = mag_warmed(synth.gauge_config(dims, nc, 0.3, 2), dims, nc, orc)
    ref, A, A_ref = P.mag_reference(orc, U, dims, nc)
    d = to_dev(U)
    cu.culgt_sweep(d, cu.Params.defaults(nc, dims, precision=cu.DF, gauge=cu.MAG), 1)
    P.check_sweep(from_dev(d, U.shape), ref, 3.2e-12, A, A_ref, True)


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mag_theta_and_F(cu, orc, nc, precision):
    dims = (6, 4, 6, 10)
    U = synth.gauge_config(dims, nc, 0.3, 4)
    prec = cu.FP64 if precision == "fp64" else cu.FP32
    if prec == cu.FP32:
        U = round32(U)
    th, F = cu.culgt_theta(to_dev(U), cu.Params.defaults(nc, dims, precision=prec, gauge=cu.MAG))
    rth, rF = orc.mag_theta(U, dims, nc)
    tol = 1e-12 if prec == cu.FP64 else 1e-5
    assert th == pytest.approx(rth, rel=tol)
    assert F == pytest.approx(rF, rel=tol)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_fp64_matches_oracle(cu, orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_mag_fix(d, p)
    ref = U.copy()
    rr = orc.mag_fix(ref, dims, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.sweeps_fp64 == rr["sweeps"]
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    # the functional is unchanged by a global diagonal rotation: compare moduli
    assert np.abs(np.abs(from_dev(d, U.shape)) - np.abs(ref)).max() < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_returns_the_gauge_transformation(cu, orc, nc, precision):
    """culgt_mag_fix_gauge: the output links are the input transformed by the
    returned g (to the accuracy of its accumulation), g is unitary, and the
    fix converges like the FP64 oracle's MAG fix (its sweep count in FP64,
    F_MAG within 1e-10)."""
    prec = {"fp64": cu.FP64, "mixed": cu.MIXED, "mixed_df": cu.MIXED_DF}[precision]
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    gauge = torch.zeros(V * nc * nc * 2, dtype=torch.float64, device="cuda")
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_mag_fix_gauge(d, p, gauge)
    rr = orc.mag_fix(U.copy(), dims, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r.status == cu.OK and r.theta < 1e-12
    if prec == cu.FP64:
        assert r.sweeps_fp64 == rr["sweeps"]
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    g = gauge.cpu().numpy().view(np.complex128).reshape(V, nc, nc)
    assert np.abs(g @ np.swapaxes(g.conj(), 1, 2) - np.eye(nc)).max() < 1e-13
    tol = 1e-12 if prec == cu.FP64 else 1e-10
    assert np.abs(from_dev(d, U.shape) - synth.gauge_transform(U, dims, g)).max() < tol


@pytest.mark.parametrize("precision", ["mixed", "mixed_df", "df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_reduced_and_mixed(cu, orc, nc, precision):
    prec = {"mixed": cu.MIXED, "mixed_df": cu.MIXED_DF, "df": cu.DF}[precision]
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_mag_fix(d, p)
    rr = orc.mag_fix(U.copy(), dims, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    out = from_dev(d, U.shape)
    th, F = orc.mag_theta(out, dims, nc)
    assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)


def test_mag_handle_follows_the_gauge_field(cu, orc):
    """The handle API sweeps and measures the functional p.gauge names."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, 3, 0.3, 2)
    p = cu.Params.defaults(3, dims, gauge=cu.MAG)
    d = to_dev(U)
    with cu.Handle(p) as h:
        h.culgt_load(d)
        h.culgt_handle_sweep(3)
        th, F = h.culgt_handle_theta()
        h.culgt_store(d)
    torch.cuda.synchronize()
    ref = U.copy()
    orc.mag_sweep(ref, dims, 3, 1.7, 3)
    rth, rF = orc.mag_theta(ref, dims, 3)
    assert th == pytest.approx(rth, rel=1e-10) and F == pytest.approx(rF, rel=1e-12)


@pytest.mark.parametrize("nc", [2, 3])
def test_full_size_mag_sweep(cu, orc, nc):
    """32^4: one FP64 MAG sweep of the whole lattice against the oracle."""
    dims = (32, 32, 32, 32)
    U = synth.gauge_config(dims, nc, 0.3, 2)
    ref, A, A_ref = P.mag_reference(orc, U, dims, nc)
    d = to_dev(U)
    cu.culgt_sweep(d, cu.Params.defaults(nc, dims, gauge=cu.MAG), 1)
    P.check_sweep(from_dev(d, U.shape), ref, 1e-13, A, A_ref, False)


SEED = 0x0DDC0FFEE


def mag_heatbath_on_device(cu, U, dims, nc, T, word, **kw):
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, gauge=cu.MAG, **kw)
    with cu.Handle(p) as h:
        h.culgt_load(d)
        h.culgt_handle_heatbath(T, SEED, word)
        h.culgt_store(d)
    torch.cuda.synchronize()
    return from_dev(d, U.shape)


@pytest.mark.parametrize("dims,nc", CASES)
@pytest.mark.parametrize("T", [0.05, 2.0])
def test_one_mag_heatbath_sweep_fp64(cu, orc, dims, nc, T):
    """Cold draws stay near the maximiser, so warmed input stays well
    conditioned through the white half-sweep; hot draws (T = 2) randomise the
    black sites first, and the white sites then see random-start blocks."""
    U0 = synth.gauge_config(dims, nc, 0.3, 2)
    for U, good in [(U0, False), (mag_warmed(U0, dims, nc, orc), T < 0.5)]:
        ref, A, A_ref = P.mag_heatbath_reference(orc, U, dims, nc, T, SEED, 5)
        for sr in ([18, 12] if nc == 3 else [4]):
            got = mag_heatbath_on_device(cu, U, dims, nc, T, 5, storage_reals=sr)
            P.check_sweep(got, ref, 1e-13, A, A_ref, good)


@pytest.mark.parametrize("dims,nc", CASES)
def test_one_mag_heatbath_sweep_fp32(cu, orc, dims, nc):
    U = round32(mag_warmed(synth.gauge_config(dims, nc, 0.3, 3), dims, nc, orc))
    ref, A, A_ref = P.mag_heatbath_reference(orc, U, dims, nc, 0.5, SEED, 2)
    got = mag_heatbath_on_device(cu, U, dims, nc, 0.5, 2, precision=cu.FP32)
    P.check_sweep(got, ref, 5e-6, A, A_ref, False)


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_anneal_fp64_matches_oracle(cu, orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.5, 1)
    ref = U.copy()
    orc.mag_anneal(ref, dims, nc, 0.6, 0.05, 20, 2, SEED, reunit_every=50)
    rr = orc.mag_fix(ref, dims, nc, 1.7, 1e-12, 5000, 5, 50)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_mag_fix_anneal(d, p, cu.AnnealParams(0.6, 0.05, 20, 2, SEED))
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.sweeps_fp64 == rr["sweeps"]
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    # the moduli are free of the diagonal rotations MAG leaves open; the 60
    # annealing sweeps amplify rounding differences (MAG's blocks are worse
    # conditioned than Landau's), the same maximum is pinned by F and the
    # sweep count above
    assert np.abs(np.abs(from_dev(d, U.shape)) - np.abs(ref)).max() < 1e-7


@pytest.mark.parametrize("nc", [2, 3])
def test_mag_fix_anneal_mixed(cu, orc, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.5, 1)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, precision=cu.MIXED, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_mag_fix_anneal(d, p, cu.AnnealParams(0.6, 0.05, 20, 2, SEED))
    assert r.status == cu.OK and r.theta < 1e-12 and r.sweeps_fp32 > 0
    out = from_dev(d, U.shape)
    th, F = orc.mag_theta(out, dims, nc)
    assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)
    assert orc.plaquette(out, dims, nc) == pytest.approx(orc.plaquette(U, dims, nc), abs=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nc", [2, 3])
def test_batched_mag_matches_single_lattice(cu, nc, precision):
    """MAG problems of uneven sizes in shared launches end exactly where
    culgt_mag_fix ends for each of them; with annealing, problem j draws like
    culgt_mag_fix_anneal with seed + j."""
    prec = cu.FP64 if precision == "fp64" else cu.MIXED
    cases = [((4, 4, 4, 4), 1), ((2, 4, 6, 4), 2), ((4, 4, 4, 4), 3)]
    Us = [synth.gauge_config(dims, nc, 0.4, seed) for dims, seed in cases]
    p = cu.Params.defaults(nc, (4, 4, 4, 4), precision=prec, check_every=5, reunit_every=50, max_sweeps=5000,
                           gauge=cu.MAG)
    a = cu.AnnealParams(0.6, 0.05, 10, 2, SEED)
    for anneal in (False, True):
        ds = [to_dev(U) for U in Us]
        res = (cu.culgt_fix_batched_anneal(ds, [c[0] for c in cases], p, a) if anneal
               else cu.culgt_fix_batched(ds, [c[0] for c in cases], p))
        for j, ((dims, _), U, d, r) in enumerate(zip(cases, Us, ds, res)):
            pj = cu.Params(**{**p.__dict__, "dims": dims})
            e = to_dev(U)
            rs = (cu.culgt_mag_fix_anneal(e, pj, cu.AnnealParams(0.6, 0.05, 10, 2, SEED + j)) if anneal
                  else cu.culgt_mag_fix(e, pj))
            assert r.status == cu.OK and rs.status == cu.OK and r.theta < 1e-12
            assert (r.sweeps_fp32, r.sweeps_fp64) == (rs.sweeps_fp32, rs.sweeps_fp64)
            assert r.F == pytest.approx(rs.F, rel=1e-12)
            assert torch.allclose(d, e, atol=1e-12, rtol=0)
