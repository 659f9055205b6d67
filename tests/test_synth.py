"""The seeded input generator: group membership, Haar statistics, determinism."""
import numpy as np
import pytest

from paper_1412_3655_gb300 import synth


@pytest.mark.parametrize("nc", [2, 3])
def test_links_are_special_unitary(nc):
    L = (4, 4, 2, 6)
    U = synth.gauge_config(L, nc, 0.3, 1)
    eye = np.eye(nc)
    assert np.abs(U @ np.swapaxes(U.conj(), -1, -2) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_haar_moments(nc):
    """Haar on SU(N): E[tr g] = 0 and E[|tr g|^2] = 1."""
    g = synth.haar(np.arange(200_000), nc, 123, synth.SLOT_G, 0)
    tr = np.trace(g, axis1=1, axis2=2)
    n = g.shape[0]
    assert abs(tr.mean()) < 5 / np.sqrt(n)
    assert np.mean(np.abs(tr) ** 2) == pytest.approx(1.0, abs=5 * np.sqrt(2.0 / n) * 2)


def test_deterministic_and_split_independent():
    L = (4, 4, 4, 2)
    a = synth.gauge_config(L, 3, 0.3, 9)
    b = synth.gauge_config(L, 3, 0.3, 9, chunk=7)
    assert np.array_equal(a, b)
    c = synth.gauge_config(L, 3, 0.3, 10)
    assert np.abs(a - c).max() > 0.1


def test_philox_uniform_bits():
    ctr = np.zeros((1 << 16, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(1 << 16)
    out = synth.philox4x32_10(ctr, (42, 0))
    bits = np.unpackbits(out.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.002
    # consecutive counters give uncorrelated words
    x = out[:, 0].astype(np.float64)
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 0.02


def test_gaussians_moments():
    z = synth._gaussians(np.arange(100_000), 0, 8, 5, 0)
    assert abs(z.mean()) < 0.01
    assert z.std() == pytest.approx(1.0, abs=0.01)


@pytest.mark.parametrize("nc", [2, 3])
def test_copies_share_the_gauge_orbit(nc):
    """Gribov copies differ by a gauge transformation: same plaquettes, other links."""
    L = (2, 4, 2, 4)
    a = synth.gauge_config(L, nc, 0.3, 4)
    b = synth.gauge_config(L, nc, 0.3, 4, copy=3)
    assert np.abs(a - b).max() > 0.1

    def plaq(U):
        s = 0.0
        for mu in range(4):
            for nu in range(mu + 1, 4):
                fm = synth.site_neighbour_forward(L, mu)
                fn = synth.site_neighbour_forward(L, nu)
                P = U[:, mu] @ U[fm, nu] @ U[fn, mu].conj().transpose(0, 2, 1) @ U[:, nu].conj().transpose(0, 2, 1)
                s += np.trace(P, axis1=1, axis2=2).real.sum()
        return s

    assert plaq(a) == pytest.approx(plaq(b), rel=1e-13)
