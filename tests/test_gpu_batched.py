"""Batched engine against the oracle: Coulomb gauge (one problem per time
slice) and independent Landau problems of uneven sizes in shared launches.

Each problem retires on its own theta. Sweep counts must equal the oracle's
(theta is checked at the same cadence), converged F agree to 1e-10 relative,
and the plaquette, gauge invariant, stay unchanged to 1e-12.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_fp64_matches_oracle(cu, orc, nc):
    dims = (4, 4, 4, 2)
    U = synth.gauge_config(dims, nc, 0.3, 5)
    d = to_dev(U)
    V = int(np.prod(dims))
    gauge = torch.zeros(V * nc * nc * 2, dtype=torch.float64, device="cuda")
    p = cu.Params.defaults(nc, dims, check_every=1, reunit_every=25, max_sweeps=3000)
    res = cu.culgt_coulomb_fix(d, p, gauge=gauge)
    ref = U.copy()
    rr = orc.coulomb_fix(ref, dims, nc, 1.7, 1e-12, 3000, 1, 25)
    assert rr["converged"] and res[0].status == cu.OK
    for t in range(dims[0]):
        assert res[t].sweeps_fp64 == rr["sweeps"][t]
        assert res[t].theta < 1e-12
        assert res[t].F == pytest.approx(rr["F"][t], rel=1e-10)
    assert res[0].plaq_after == pytest.approx(res[0].plaq_before, abs=1e-12)
    got = from_dev(d, U.shape)
    assert np.abs(got - ref).max() < 1e-9
    g = gauge.cpu().numpy().view(np.complex128).reshape(V, nc, nc)
    assert np.abs(g - rr["g"]).max() < 1e-9
    # the output is the input gauge-transformed by the returned g
    assert np.abs(got - synth.gauge_transform(U, dims, g)).max() < 1e-12


@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_slices_retire_on_their_own(cu, orc, nc):
    """Slices need different sweep counts; each stops at its own theta_t."""
    dims = (6, 6, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 6)
    p = cu.Params.defaults(nc, dims, check_every=5, reunit_every=50, max_sweeps=4000)
    res = cu.culgt_coulomb_fix(to_dev(U), p)
    ref = U.copy()
    rr = orc.coulomb_fix(ref, dims, nc, 1.7, 1e-12, 4000, 5, 50)
    sweeps = [r.sweeps_fp64 for r in res]
    assert sweeps == list(rr["sweeps"])
    assert len(set(sweeps)) > 1
    for t in range(dims[0]):
        assert res[t].F == pytest.approx(rr["F"][t], rel=1e-10)


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_mixed(cu, orc, nc, precision):
    dims = (4, 4, 4, 2)
    U = synth.gauge_config(dims, nc, 0.3, 5)
    d = to_dev(U)
    prec = cu.MIXED if precision == "mixed" else cu.MIXED_DF
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=4000)
    res = cu.culgt_coulomb_fix(d, p)
    ref = U.copy()
    rr = orc.coulomb_fix(ref, dims, nc, 1.7, 1e-12, 4000, 1, 0)
    for t in range(dims[0]):
        assert res[t].status == cu.OK and res[t].sweeps_fp32 > 0 and res[t].sweeps_fp64 > 0
        assert res[t].theta < 1e-12
        assert res[t].F == pytest.approx(rr["F"][t], rel=1e-10)
    assert res[0].plaq_after == pytest.approx(res[0].plaq_before, abs=1e-12)
    got = from_dev(d, U.shape)
    for t in range(dims[0]):
        th, F = orc.theta_slice(got, dims, nc, t)
        assert th < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_batched_uneven_lattices(cu, orc, nc, precision):
    """4^4, 2x4x6x4, 6^4 and two gauge copies of 4^4 in one batch."""
    prec = {"fp64": cu.FP64, "mixed": cu.MIXED, "mixed_df": cu.MIXED_DF}[precision]
    cases = [((4, 4, 4, 4), 1, 0), ((2, 4, 6, 4), 2, 0), ((6, 6, 6, 6), 3, 0), ((4, 4, 4, 4), 1, 1),
             ((4, 4, 4, 4), 1, 2)]
    Us = [synth.gauge_config(dims, nc, 0.3, seed, copy=copy) for dims, seed, copy in cases]
    ds = [to_dev(U) for U in Us]
    p = cu.Params.defaults(nc, (4, 4, 4, 4), precision=prec, check_every=5, reunit_every=50, max_sweeps=5000)
    res = cu.culgt_fix_batched(ds, [c[0] for c in cases], p)
    for (dims, _, _), U, d, r in zip(cases, Us, ds, res):
        ref = U.copy()
        rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 5000, 5, 50)
        assert r.status == cu.OK and r.theta < 1e-12
        if prec == cu.FP64:
            assert r.sweeps_fp64 == rr["sweeps"]
            assert np.abs(from_dev(d, U.shape) - ref).max() < 1e-9
        assert r.F == pytest.approx(rr["F"], rel=1e-10)
        assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
        th, F = orc.theta(from_dev(d, U.shape), dims, nc)
        assert th < 1e-12 and F == pytest.approx(r.F, rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("nc", [2, 3])
def test_batched_single_problem_matches_handle(cu, nc, precision):
    prec = {"fp64": 0, "fp32": 1, "mixed": 2}[precision]
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 1)
    target = 1e-10 if prec == 1 else 1e-12
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, theta_target=target)
    a = to_dev(U)
    ra = cu.culgt_landau_fix(a, p)
    b = to_dev(U)
    rb = cu.culgt_fix_batched([b], [dims], p)[0]
    assert (ra.sweeps_fp32, ra.sweeps_fp64) == (rb.sweeps_fp32, rb.sweeps_fp64)
    assert ra.F == pytest.approx(rb.F, rel=1e-12)
    assert torch.allclose(a, b, atol=1e-12, rtol=0)


@pytest.mark.parametrize("nc", [2, 3])
def test_batched_automatic_switch_matches_handle(cu, nc):
    """The batched engine takes the automatic switch on the device per
    problem, at the same check as the single-lattice handle."""
    dims = (4, 4, 4, 4)
    Us = [synth.gauge_config(dims, nc, 0.3, s) for s in (1, 2)]
    p = cu.Params.defaults(nc, dims, precision=cu.MIXED, check_every=5, reunit_every=50, switch_theta=0.0,
                           max_sweeps=6000)
    res = cu.culgt_fix_batched([to_dev(U) for U in Us], [dims, dims], p)
    for U, rb in zip(Us, res):
        ra = cu.culgt_landau_fix(to_dev(U), p)
        assert rb.status == cu.OK
        assert (ra.sweeps_fp32, ra.sweeps_fp64) == (rb.sweeps_fp32, rb.sweeps_fp64)
        assert ra.F == pytest.approx(rb.F, rel=1e-12)


def test_batched_max_sweeps_and_status(cu):
    dims = (4, 4, 4, 4)
    Us = [synth.gauge_config(dims, 3, 0.3, 1), synth.gauge_config((2, 2, 2, 2), 3, 0.3, 1)]
    p = cu.Params.defaults(3, dims, check_every=3, max_sweeps=7)
    res = cu.culgt_fix_batched([to_dev(U) for U in Us], [dims, (2, 2, 2, 2)], p)
    assert res[0].status == cu.NOT_CONVERGED
    assert [r.sweeps_fp64 for r in res] == [7, 7]


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_landau_fix_returns_the_gauge_transformation(cu, orc, nc, precision):
    """culgt_landau_fix_gauge: the output is the input transformed by the
    returned g (to the accuracy of the accumulation), and converges like the
    FP64 oracle."""
    prec = {"fp64": cu.FP64, "mixed": cu.MIXED, "mixed_df": cu.MIXED_DF}[precision]
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    U = synth.gauge_config(dims, nc, 0.3, 1)
    d = to_dev(U)
    gauge = torch.zeros(V * nc * nc * 2, dtype=torch.float64, device="cuda")
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=3000)
    r = cu.culgt_landau_fix_gauge(d, p, gauge)
    rr = orc.landau_fix(U.copy(), dims, nc, 1.7, 1e-12, 3000, 1)
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    g = gauge.cpu().numpy().view(np.complex128).reshape(V, nc, nc)
    assert np.abs(g @ np.swapaxes(g.conj(), 1, 2) - np.eye(nc)).max() < 1e-13
    tol = 1e-12 if prec == cu.FP64 else 1e-10
    assert np.abs(from_dev(d, U.shape) - synth.gauge_transform(U, dims, g)).max() < tol
