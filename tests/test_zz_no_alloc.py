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


def test_rejects_lattices_beyond_the_fixed_scratch():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt
    p = culgt.Params.defaults(3, (64, 64, 64, 32))  # 8.4M sites > 4,194,304
    rc = culgt.library().culgt_theta_static_scratch(ctypes.c_void_p(16), ctypes.byref(p._c()), None,
                                                    ctypes.c_void_p(16))
    assert rc == culgt.ERR_TOO_LARGE
    assert "4,194,304" in culgt.culgt_status_string(rc)


@pytest.mark.gpu
def test_matches_culgt_theta_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt

    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # a larger lattice first, then a smaller one: the second call must not
    # pick up partial sums the first one left in the shared array
    for dims, nc, seed in [((8, 8, 8, 16), 3, 1), ((4, 6, 4, 2), 3, 2), ((8, 8, 8, 8), 2, 3)]:
        U = synth.gauge_config(dims, nc, 0.3, seed)
        d = torch.from_numpy(U.view(np.float64).copy()).cuda()
        p = culgt.Params.defaults(nc, dims)
        out.fill_(-1.0)
        culgt.culgt_theta_static_scratch(d, p, out)
        torch.cuda.synchronize()
        th, F = out.tolist()
        th_ref, F_ref = culgt.culgt_theta(d, p)
        assert th == pytest.approx(th_ref, rel=1e-12)
        assert F == pytest.approx(F_ref, rel=1e-12, abs=1e-14)
