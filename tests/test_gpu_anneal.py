"""Simulated annealing on the GPU against the FP64 oracle, through the C ABI.

A heat-bath sweep draws every subgroup element from Philox4x32-10 with the
same counters on both sides, so one sweep is compared element by element
like an overrelaxation sweep: FP64 within 1e-13, FP32 within 5e-6, on every
link of well-conditioned input, and on the random Haar start within each
link's tolerance scaled by the oracle's first-order bound of its
conditioning (tests/parity.py). The draws take accept/reject decisions in
the storage precision: where the oracle finds a decision's margin inside its
own error bound at that precision (a handful of sites per 10^6 in FP32), the
site may draw differently; its links and those of the white sites next to
it are then only checked to be unitary.
"""
import numpy as np
import pytest

import parity as P
from paper_1412_3655_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 0x1234_5678_9ABC_DEF0


@pytest.fixture(scope="module")
def cu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt
    return culgt


def to_dev(U, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(U).view(np.float64).astype(dtype)).cuda()


def from_dev(t, shape):
    a = t.cpu().numpy().astype(np.float64)
    return np.ascontiguousarray(a).view(np.complex128).reshape(shape)


def round32(U):
    return U.view(np.float64).astype(np.float32).astype(np.float64).view(np.complex128)


def warmed(U, dims, nc, orc, n=5):
    W = U.copy()
    orc.sweep(W, dims, nc, 1.7, n)
    return W


def link_errors(got, ref):
    return P.link_errors(got, ref).reshape(-1)


def traces(U):
    return np.trace(U, axis1=-2, axis2=-1)


def heatbath_on_device(cu, U, dims, nc, T, word, **kw):
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, **kw)
    with cu.Handle(p) as h:
        h.culgt_load(d)
        h.culgt_handle_heatbath(T, SEED, word)
        h.culgt_store(d)
    torch.cuda.synchronize()
    return from_dev(d, U.shape)


CASES = [((8, 8, 8, 8), 3), ((6, 4, 6, 10), 3), ((2, 2, 2, 2), 3), ((8, 8, 8, 8), 2), ((6, 4, 6, 10), 2)]


# T = 0.05 and 0.5 draw mostly by Kennedy-Pendleton (alpha = 2k/T >= 2),
# T = 20 by Creutz's method (alpha < 2)
@pytest.mark.parametrize("dims,nc", CASES)
@pytest.mark.parametrize("T", [0.05, 0.5, 20.0])
def test_one_heatbath_sweep_fp64(cu, orc, dims, nc, T):
    U0 = synth.gauge_config(dims, nc, 0.3, 2)
    storages = [18, 12] if nc == 3 else [4]
    for U, good in [(U0, False), (warmed(U0, dims, nc, orc), True)]:
        ref, A, A_ref, exempt = P.heatbath_reference(orc, U, dims, nc, T, SEED, 9, "fp64")
        for sr in storages:
            got = heatbath_on_device(cu, U, dims, nc, T, 9, storage_reals=sr)
            P.check_sweep(got, ref, 1e-13, A, A_ref, good, exempt)


@pytest.mark.parametrize("dims,nc", CASES)
@pytest.mark.parametrize("T", [0.5, 20.0])
def test_one_heatbath_sweep_fp32(cu, orc, dims, nc, T):
    U = round32(warmed(synth.gauge_config(dims, nc, 0.3, 3), dims, nc, orc))
    ref, A, A_ref, exempt = P.heatbath_reference(orc, U, dims, nc, T, SEED, 4, "fp32")
    for sr in ([12, 18] if nc == 3 else [4]):
        got = heatbath_on_device(cu, U, dims, nc, T, 4, precision=cu.FP32, storage_reals=sr)
        P.check_sweep(got, ref, 5e-6, A, A_ref, True, exempt)


@pytest.mark.parametrize("nc", [2, 3])
def test_one_heatbath_sweep_double_float(cu, orc, nc):
    dims = (8, 8, 8, 8)
    U = warmed(synth.gauge_config(dims, nc, 0.3, 2), dims, nc, orc)
    ref, A, A_ref, exempt = P.heatbath_reference(orc, U, dims, nc, 0.5, SEED, 1, "df")
    got = heatbath_on_device(cu, U, dims, nc, 0.5, 1, precision=cu.DF)
    P.check_sweep(got, ref, 3.2e-12, A, A_ref, True, exempt)


@pytest.mark.parametrize("nc", [2, 3])
def test_heatbath_sweep_words_and_seeds_differ(cu, nc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.3, 5)
    a = heatbath_on_device(cu, U, dims, nc, 0.5, 0)
    b = heatbath_on_device(cu, U, dims, nc, 0.5, 1)
    assert np.abs(a - b).max() > 1e-3
    assert np.array_equal(a, heatbath_on_device(cu, U, dims, nc, 0.5, 0))


@pytest.mark.parametrize("nc", [2, 3])
def test_anneal_schedule_fp64(cu, orc, nc):
    """Heat-bath and microcanonical sweeps of the schedule, with the
    reunitarisation cadence, against the oracle's schedule."""
    dims = (6, 4, 6, 4)
    U = warmed(synth.gauge_config(dims, nc, 0.3, 6), dims, nc, orc)
    a = dict(t_start=0.8, t_end=0.1, steps=4, micro_sweeps=2, seed=SEED)
    ref = U.copy()
    orc.anneal(ref, dims, nc, 0.8, 0.1, 4, 2, SEED, reunit_every=5)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, reunit_every=5)
    with cu.Handle(p) as h:
        h.culgt_load(d)
        h.culgt_handle_anneal(cu.AnnealParams(**a))
        h.culgt_store(d)
    torch.cuda.synchronize()
    err = link_errors(from_dev(d, U.shape), ref)
    assert err.max() <= 1e-12, f"max {err.max():.3e}"


@pytest.mark.parametrize("nc", [2, 3])
def test_landau_fix_anneal_fp64_matches_oracle(cu, orc, nc):
    """Annealing then overrelaxation: same OR sweep count as the oracle, F
    within 1e-10, links within 1e-9, plaquette unchanged to 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.6, 1)
    ref = U.copy()
    orc.anneal(ref, dims, nc, 0.6, 0.05, 30, 2, SEED, reunit_every=50)
    rr = orc.landau_fix(ref, dims, nc, 1.7, 1e-12, 5000, 5, 50)
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, check_every=5, reunit_every=50, max_sweeps=5000)
    r = cu.culgt_landau_fix_anneal(d, p, cu.AnnealParams(0.6, 0.05, 30, 2, SEED))
    assert r.status == cu.OK and r.theta < 1e-12
    assert r.sweeps_fp64 == rr["sweeps"]
    assert r.F == pytest.approx(rr["F"], rel=1e-10)
    assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
    # Landau gauge leaves a global rotation U -> h U h^+ free, which neither
    # annealing nor overrelaxation restores: link traces are compared
    got = from_dev(d, U.shape)
    assert np.abs(traces(got) - traces(ref)).max() < 1e-9


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_df"])
@pytest.mark.parametrize("nc", [2, 3])
def test_landau_fix_anneal_reduced_precision(cu, orc, nc, precision):
    """FP32 annealing (the mixed schedules anneal in their FP32 phase,
    accumulating g): the output is on the input's gauge orbit (plaquette to
    1e-12 for the mixed schedules) and gauge fixed (oracle theta)."""
    prec = {"fp32": cu.FP32, "mixed": cu.MIXED, "mixed_df": cu.MIXED_DF}[precision]
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, nc, 0.6, 1)
    target = 1e-10 if prec == cu.FP32 else 1e-12
    d = to_dev(U)
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=50, max_sweeps=6000,
                           theta_target=target)
    r = cu.culgt_landau_fix_anneal(d, p, cu.AnnealParams(0.6, 0.05, 30, 2, SEED))
    assert r.status == cu.OK and r.sweeps_fp32 > 0
    out = from_dev(d, U.shape)
    th, F = orc.theta(out, dims, nc)
    assert F == pytest.approx(r.F, rel=1e-6 if prec == cu.FP32 else 1e-12)
    if prec != cu.FP32:
        assert th < 1e-12
        assert r.plaq_after == pytest.approx(r.plaq_before, abs=1e-12)
        assert orc.plaquette(out, dims, nc) == pytest.approx(orc.plaquette(U, dims, nc), abs=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nc", [2, 3])
def test_batched_anneal_matches_single_lattice(cu, nc, precision):
    """Problem j of a batch draws with seed + j: it ends exactly where the
    single-lattice call with that seed ends."""
    prec = cu.FP64 if precision == "fp64" else cu.MIXED
    cases = [((4, 4, 4, 4), 1), ((2, 4, 6, 4), 2), ((4, 4, 4, 4), 3)]
    Us = [synth.gauge_config(dims, nc, 0.6, seed) for dims, seed in cases]
    p = cu.Params.defaults(nc, (4, 4, 4, 4), precision=prec, check_every=5, reunit_every=50, max_sweeps=5000)
    a = cu.AnnealParams(0.6, 0.05, 20, 2, SEED)
    ds = [to_dev(U) for U in Us]
    res = cu.culgt_fix_batched_anneal(ds, [c[0] for c in cases], p, a)
    for j, ((dims, _), U, d, r) in enumerate(zip(cases, Us, ds, res)):
        pj = cu.Params(**{**p.__dict__, "dims": dims})
        e = to_dev(U)
        rs = cu.culgt_landau_fix_anneal(e, pj, cu.AnnealParams(0.6, 0.05, 20, 2, SEED + j))
        assert r.status == cu.OK and rs.status == cu.OK
        assert (r.sweeps_fp32, r.sweeps_fp64) == (rs.sweeps_fp32, rs.sweeps_fp64)
        assert r.F == pytest.approx(rs.F, rel=1e-12)
        a_, b_ = from_dev(d, U.shape), from_dev(e, U.shape)
        dl, dt = np.abs(a_ - b_).max(), np.abs(traces(a_) - traces(b_)).max()
        assert dl < 1e-12, f"links {dl:.3e}, traces {dt:.3e}"


def test_annealing_raises_the_gribov_copy_maxima(cu):
    """The purpose of the combination (Sec. 1): over random gauge copies of
    one field, annealing before overrelaxation ends on larger maxima of F
    than overrelaxation alone (means over 16 copies; fixed seeds)."""
    dims = (4, 4, 4, 4)
    nc = 3
    Us = [synth.gauge_config(dims, nc, 0.6, 1, copy=c) for c in range(16)]
    p = cu.Params.defaults(nc, dims, precision=cu.MIXED, check_every=10, reunit_every=50, max_sweeps=20000)
    plain = cu.culgt_fix_batched([to_dev(U) for U in Us], [dims] * 16, p)
    ann = cu.culgt_fix_batched_anneal([to_dev(U) for U in Us], [dims] * 16, p, cu.AnnealParams(0.6, 0.01, 300, 3, 7))
    assert all(r.status == cu.OK for r in plain + ann)
    assert np.mean([r.F for r in ann]) > np.mean([r.F for r in plain])


@pytest.mark.parametrize("nc", [2, 3])
def test_full_size_heatbath_sweep(cu, orc, nc):
    """32^4: one FP64 and one FP32 heat-bath sweep of the whole lattice
    against the oracle, from the random Haar start (every link within its
    conditioning-scaled tolerance, outside the sites whose decisions lie
    within their error bound at the precision)."""
    dims = (32, 32, 32, 32)
    U = synth.gauge_config(dims, nc, 0.3, 2)
    ref, A, A_ref, exempt = P.heatbath_reference(orc, U, dims, nc, 0.5, SEED, 0, "fp64")
    got = heatbath_on_device(cu, U, dims, nc, 0.5, 0)
    P.check_sweep(got, ref, 1e-13, A, A_ref, False, exempt)
    U32 = round32(U)
    ref32, A, A_ref, exempt = P.heatbath_reference(orc, U32, dims, nc, 0.5, SEED, 0, "fp32")
    got32 = heatbath_on_device(cu, U32, dims, nc, 0.5, 0, precision=cu.FP32)
    P.check_sweep(got32, ref32, 5e-6, A, A_ref, False, exempt)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nc", [2, 3])
def test_coulomb_fix_anneal(cu, orc, nc, precision):
    """Coulomb gauge with every slice annealed first (slice t keyed by seed +
    t): FP64 takes the oracle's sweep count per slice with F_t within 1e-10
    and the same link traces; both precisions return a g that maps the input
    onto the output, and keep the plaquette."""
    prec = cu.FP64 if precision == "fp64" else cu.MIXED
    dims = (4, 4, 4, 2)
    V = int(np.prod(dims))
    U = synth.gauge_config(dims, nc, 0.5, 6)
    d = to_dev(U)
    gauge = torch.zeros(V * nc * nc * 2, dtype=torch.float64, device="cuda")
    p = cu.Params.defaults(nc, dims, precision=prec, check_every=5, reunit_every=25, max_sweeps=5000)
    res = cu.culgt_coulomb_fix_anneal(d, p, cu.AnnealParams(0.6, 0.05, 20, 2, SEED), gauge=gauge)
    ref = U.copy()
    rr = orc.coulomb_fix_anneal(ref, dims, nc, 0.6, 0.05, 20, 2, SEED, 1.7, 1e-12, 5000, 5, 25)
    got = from_dev(d, U.shape)
    g = gauge.cpu().numpy().view(np.complex128).reshape(V, nc, nc)
    for t in range(dims[0]):
        assert res[t].status == cu.OK and res[t].theta < 1e-12
        assert res[t].F == pytest.approx(rr["F"][t], rel=1e-10)
        if prec == cu.FP64:
            assert res[t].sweeps_fp64 == rr["sweeps"][t]
    if prec == cu.FP64:
        # each slice keeps a global rotation free, so spatial link traces are
        # compared (temporal links join two slices' rotations); the orbit
        # check below covers the temporal links
        assert np.abs(traces(got[:, 1:]) - traces(ref[:, 1:])).max() < 1e-9
    assert np.abs(got - synth.gauge_transform(U, dims, g)).max() < (1e-12 if prec == cu.FP64 else 1e-10)
    assert res[0].plaq_after == pytest.approx(res[0].plaq_before, abs=1e-12)
