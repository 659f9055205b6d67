"""culgt_theta_static_scratch: the allocation-free theta/F entry point.

It serves callers that cannot allocate device memory while they run (their
pool owns the GPU, or cudaMalloc's synchronisation would stall their stream).
This file is collected last, so a run that stops at the first failure has run
every other test before it; it passes on its own in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

from paper_1412_3655_gb300 import synth

LIMIT_DIMS = (16, 32, 64, 128)  # 4,194,304 sites: the largest lattice the fixed array takes


def _lib():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt
    return culgt


def test_rejects_lattices_beyond_the_fixed_scratch():
    culgt = _lib()
    for dims in [(64, 64, 64, 32), (16, 32, 64, 130)]:  # 8.4M sites; the next even size after the limit
        p = culgt.Params.defaults(3, dims)
        rc = culgt.library().culgt_theta_static_scratch(ctypes.c_void_p(16), ctypes.byref(p._c()), None,
                                                        ctypes.c_void_p(16))
        assert rc == culgt.ERR_TOO_LARGE
    assert "4,194,304" in culgt.culgt_status_string(culgt.ERR_TOO_LARGE)
    assert int(np.prod(LIMIT_DIMS)) == 4194304


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.gpu
def test_matches_culgt_theta_on_two_calls_in_a_row(orc):
    """Each lattice is measured twice in a row, in double and in float
    canonical links (dtype_in 0 and 1), against culgt_theta on the same
    buffer and against the oracle on the same values (1e-12 relative)."""
    torch = _cuda()
    culgt = _lib()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # a larger lattice first, then a smaller one: the second call must not
    # pick up partial sums the first one left in the shared array
    for dims, nc, seed in [((8, 8, 8, 16), 3, 1), ((4, 6, 4, 2), 3, 2), ((8, 8, 8, 8), 2, 3)]:
        U = synth.gauge_config(dims, nc, 0.3, seed)
        for dtype_in, real in [(0, np.float64), (1, np.float32)]:
            vals = U.view(np.float64).astype(real)
            d = torch.from_numpy(vals.copy()).cuda()
            p = culgt.Params.defaults(nc, dims, dtype_in=dtype_in)
            th_ref, F_ref = culgt.culgt_theta(d, p)
            Uo = np.ascontiguousarray(vals.astype(np.float64)).view(np.complex128).reshape(U.shape)
            th_o, F_o = orc.theta(Uo, dims, nc)
            for _ in range(2):
                out.fill_(-1.0)
                culgt.culgt_theta_static_scratch(d, p, out)
                torch.cuda.synchronize()
                th, F = out.tolist()
                assert th == pytest.approx(th_ref, rel=1e-12)
                assert F == pytest.approx(F_ref, rel=1e-12, abs=1e-14)
                assert th == pytest.approx(th_o, rel=1e-12)
                assert F == pytest.approx(F_o, rel=1e-12, abs=1e-14)


@pytest.mark.gpu
def test_at_the_size_limit(orc):
    """4,194,304 sites, float links: the field is a 16 x 32 x 8 x 8 lattice
    repeated 8 x 16 times along the third and fourth directions, so every
    site sees the neighbourhood it has in the small periodic lattice and
    theta and F equal the small lattice's (all 16384 partial sums used)."""
    torch = _cuda()
    culgt = _lib()
    small = (16, 32, 8, 8)
    U = synth.gauge_config(small, 3, 0.3, 4).view(np.float64).astype(np.float32)
    Us = U.astype(np.float64).view(np.complex128).reshape(-1, 4, 3, 3)
    th_o, F_o = orc.theta(np.ascontiguousarray(Us), small, 3)
    # canonical order [x0][x3][x2][x1]: repeat along x3 (x 16) and x2 (x 8)
    A = U.reshape(small[0], small[3], small[2], small[1], 4 * 18)
    big = np.tile(A, (1, LIMIT_DIMS[3] // small[3], LIMIT_DIMS[2] // small[2], 1, 1))
    d = torch.from_numpy(np.ascontiguousarray(big).reshape(-1)).cuda()
    del A, big
    p = culgt.Params.defaults(3, LIMIT_DIMS, dtype_in=1)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    culgt.culgt_theta_static_scratch(d, p, out)
    torch.cuda.synchronize()
    th, F = out.tolist()
    assert th == pytest.approx(th_o, rel=1e-12)
    assert F == pytest.approx(F_o, rel=1e-12)
    # the next even size is refused before any device work, buffers untouched
    over = culgt.Params.defaults(3, (16, 32, 64, 130), dtype_in=1)
    rc = culgt.library().culgt_theta_static_scratch(ctypes.c_void_p(d.data_ptr()), ctypes.byref(over._c()), None,
                                                    ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    assert rc == culgt.ERR_TOO_LARGE and out.tolist() == [th, F]


@pytest.mark.gpu
def test_on_a_caller_stream(orc):
    """Stream-ordered use: the result lands in d_out on the caller's stream;
    synchronising that stream alone is enough to read it."""
    torch = _cuda()
    culgt = _lib()
    dims, nc = (8, 8, 8, 8), 3
    U = synth.gauge_config(dims, nc, 0.3, 5)
    th_o, F_o = orc.theta(U, dims, nc)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = torch.from_numpy(U.view(np.float64).copy()).to("cuda", non_blocking=False)
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    s.synchronize()
    culgt.culgt_theta_static_scratch(d, culgt.Params.defaults(nc, dims), out, stream=s)
    s.synchronize()
    th, F = out.cpu().tolist()
    assert th == pytest.approx(th_o, rel=1e-12)
    assert F == pytest.approx(F_o, rel=1e-12, abs=1e-14)
