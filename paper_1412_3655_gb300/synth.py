"""Seeded synthetic gauge configurations (input generator only).

This module produces the inputs that both the CUDA library and the CPU oracle
are run on; it contains none of the gauge-fixing arithmetic. A configuration is

    U_mu(x) = g(x) exp(i eps H_mu(x)) g(x + mu)^+,

with H_mu(x) = sum_a c_a T_a, c_a ~ N(0, 1), T_a the unscaled Gell-Mann (SU(3))
or Pauli (SU(2)) matrices, and g(x) Haar-random. At eps = 0 it is a pure gauge,
on which Landau gauge fixing can reach F = 1 (Sec. 2 of the paper).

Randomness is counter-based: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC11), keyed by the seed, with
counter (site index, slot, draw, copy). Slots: 0..3 = H_mu, 4 = g of the base
configuration, 5 = random gauge transformation of copy > 0. Uniforms are
(u + 0.5) 2^-32 and Gaussians come from Box-Muller, so every value depends only
on (seed, site, slot, draw, copy) and never on the lattice being split up.

Links are returned as complex128 arrays of shape (V, 4, Nc, Nc) in canonical
site order i = x1 + L1 (x2 + L2 (x3 + L3 x0)), dims (L0, L1, L2, L3), L0 = time.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

SLOT_H = 0  # 0..3: H_mu
SLOT_G = 4
SLOT_COPY = 5


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds. ctr: (N, 4) uint32; key: two uint32. Returns (N, 4) uint32."""
    c = [ctr[:, j].astype(np.uint64) for j in range(4)]
    k0, k1 = np.uint32(key[0]), np.uint32(key[1])
    for r in range(10):
        if r:
            k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=1)


def _uniforms(sites: np.ndarray, slot: int, n_draws: int, seed: int, copy: int) -> np.ndarray:
    """(N, 4 * n_draws) uniforms in (0, 1) for the given sites."""
    n = sites.shape[0]
    out = np.empty((n, 4 * n_draws))
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    for d in range(n_draws):
        ctr = np.empty((n, 4), dtype=np.uint32)
        ctr[:, 0] = sites.astype(np.uint32)
        ctr[:, 1] = slot
        ctr[:, 2] = d
        ctr[:, 3] = copy
        u = philox4x32_10(ctr, key)
        out[:, 4 * d:4 * d + 4] = (u.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    return out


def _gaussians(sites, slot, count, seed, copy):
    """(N, count) standard normals by Box-Muller on consecutive uniform pairs."""
    n_u = count + (count & 1)
    u = _uniforms(sites, slot, (n_u + 3) // 4, seed, copy)[:, :n_u]
    u1, u2 = u[:, 0::2], u[:, 1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((sites.shape[0], n_u))
    z[:, 0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[:, 1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:, :count]


def pauli() -> np.ndarray:
    return np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def generators(nc: int) -> np.ndarray:
    if nc == 2:
        return pauli()
    if nc == 3:
        return gell_mann()
    raise ValueError("nc must be 2 or 3")


def haar(sites: np.ndarray, nc: int, seed: int, slot: int, copy: int) -> np.ndarray:
    """Haar-random SU(Nc) per site. SU(2): normalised 4-Gaussian quaternion.
    SU(3): complex Gaussian matrix, Gram-Schmidt on the rows (Haar on U(3)),
    divided by the principal cube root of its determinant (left-invariant, so
    Haar on SU(3))."""
    n = sites.shape[0]
    if nc == 2:
        q = _gaussians(sites, slot, 4, seed, copy)
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        a0, a1, a2, a3 = q.T
        g = np.empty((n, 2, 2), dtype=np.complex128)
        g[:, 0, 0] = a0 + 1j * a3
        g[:, 0, 1] = a2 + 1j * a1
        g[:, 1, 0] = -a2 + 1j * a1
        g[:, 1, 1] = a0 - 1j * a3
        return g
    z = _gaussians(sites, slot, 18, seed, copy)
    Z = (z[:, 0::2] + 1j * z[:, 1::2]).reshape(n, 3, 3) / np.sqrt(2.0)
    rows = []
    for a in range(3):
        v = Z[:, a, :].copy()
        for r in rows:
            v -= np.sum(r.conj() * v, axis=1, keepdims=True) * r
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        rows.append(v)
    G = np.stack(rows, axis=1)
    det = np.linalg.det(G)
    return G / np.exp(1j * np.angle(det) / 3.0)[:, None, None]


def expi(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) for a stack of Hermitian matrices, by eigendecomposition."""
    w, v = np.linalg.eigh(H)
    return (v * np.exp(1j * eps * w)[:, None, :]) @ v.conj().transpose(0, 2, 1)


def site_neighbour_forward(L, mu: int) -> np.ndarray:
    """Canonical index of x + mu-hat for every site x."""
    L0, L1, L2, L3 = (int(v) for v in L)
    i = np.arange(L0 * L1 * L2 * L3, dtype=np.int64)
    x1 = i % L1
    x2 = (i // L1) % L2
    x3 = (i // (L1 * L2)) % L3
    x0 = i // (L1 * L2 * L3)
    x = [x0, x1, x2, x3]
    x[mu] = (x[mu] + 1) % int(L[mu])
    return x[1] + L1 * (x[2] + L2 * (x[3] + L3 * x[0]))


def gauge_transform(U: np.ndarray, L, g: np.ndarray) -> np.ndarray:
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^+ (the transformation law of Sec. 2)."""
    out = np.empty_like(U)
    for mu in range(4):
        fwd = site_neighbour_forward(L, mu)
        out[:, mu] = g @ U[:, mu] @ g[fwd].conj().transpose(0, 2, 1)
    return out


def random_gauge(L, nc: int, seed: int, copy: int = 0) -> np.ndarray:
    """Haar-random g(x) (slot 4 for copy 0, slot 5 for the Gribov copies)."""
    V = int(np.prod(L))
    sites = np.arange(V, dtype=np.int64)
    return haar(sites, nc, seed, SLOT_G if copy == 0 else SLOT_COPY, copy)


def _gauge_at(sites, L, nc, seed, copy, spread):
    """g at the given sites: Haar (spread None) or exp(i spread H), then for
    copy > 0 the copy's Haar transformation on top, as (g, h) pair."""
    if spread is None:
        g = haar(sites, nc, seed, SLOT_G, 0)
    else:
        T = generators(nc)
        c = _gaussians(sites, SLOT_COPY, T.shape[0], seed, 1 << 20)
        g = expi(np.einsum("na,aij->nij", c, T), spread)
    h = haar(sites, nc, seed, SLOT_COPY, copy) if copy else None
    return g, h


def _forward_sites(L, sites, mu):
    L0, L1, L2, L3 = L
    x1 = sites % L1
    x2 = (sites // L1) % L2
    x3 = (sites // (L1 * L2)) % L3
    x0 = sites // (L1 * L2 * L3)
    x = [x0, x1, x2, x3]
    x[mu] = (x[mu] + 1) % L[mu]
    return x[1] + L1 * (x[2] + L2 * (x[3] + L3 * x[0]))


def _links_for_sites(L, nc, eps, seed, copy, g, h, start, stop):
    """U_mu(x) for the sites x in [start, stop), all mu: (n, 4, Nc, Nc), from
    the gauge transformations g (and h for copy > 0) of every site."""
    sites = np.arange(start, stop, dtype=np.int64)
    n = sites.shape[0]
    T = generators(nc)
    out = np.empty((n, 4, nc, nc), dtype=np.complex128)
    for mu in range(4):
        if eps == 0.0:
            E = np.broadcast_to(np.eye(nc, dtype=np.complex128), (n, nc, nc))
        else:
            c = _gaussians(sites, SLOT_H + mu, T.shape[0], seed, 0)
            E = expi(np.einsum("na,aij->nij", c, T), eps)
        fwd = _forward_sites(L, sites, mu)
        U = g[start:stop] @ E @ g[fwd].conj().transpose(0, 2, 1)
        if copy:
            U = h[start:stop] @ U @ h[fwd].conj().transpose(0, 2, 1)
        out[:, mu] = U
    return out


def _shm_array(name, shape):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)


def _gauge_chunk(args):
    """worker: g (and h) of the sites [a, b) into shared memory"""
    g_name, h_name, V, nc, L, seed, copy, spread, a, b = args
    shm_g, g = _shm_array(g_name, (V, nc, nc))
    shm_h, h = _shm_array(h_name, (V, nc, nc)) if h_name else (None, None)
    try:
        ga, ha = _gauge_at(np.arange(a, b, dtype=np.int64), L, nc, seed, copy, spread)
        g[a:b] = ga
        if h is not None:
            h[a:b] = ha
    finally:
        shm_g.close()
        if shm_h:
            shm_h.close()
    return b - a


def _links_chunk(args):
    """worker: the links of the sites [a, b) into shared memory"""
    u_name, g_name, h_name, V, nc, L, eps, seed, copy, a, b = args
    shm_u, U = _shm_array(u_name, (V, 4, nc, nc))
    shm_g, g = _shm_array(g_name, (V, nc, nc))
    shm_h, h = _shm_array(h_name, (V, nc, nc)) if h_name else (None, None)
    try:
        U[a:b] = _links_for_sites(L, nc, eps, seed, copy, g, h, a, b)
    finally:
        shm_u.close()
        shm_g.close()
        if shm_h:
            shm_h.close()
    return b - a


def _spawn_safe() -> bool:
    """Spawned workers re-import the parent's __main__; that fails when it was
    read from stdin or a path that no longer exists."""
    import os
    import sys
    f = getattr(sys.modules.get("__main__"), "__file__", None)
    return f is None or os.path.exists(f)


def _parallel_config(L, nc, eps, seed, copy, spread, workers):
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context, shared_memory
    V = int(np.prod(L))
    step = -(-V // (4 * workers))
    chunks = [(a, min(V, a + step)) for a in range(0, V, step)]
    shms = []
    try:
        su = shared_memory.SharedMemory(create=True, size=V * 4 * nc * nc * 16)
        shms.append(su)
        sg = shared_memory.SharedMemory(create=True, size=V * nc * nc * 16)
        shms.append(sg)
        sh = None
        if copy:
            sh = shared_memory.SharedMemory(create=True, size=V * nc * nc * 16)
            shms.append(sh)
        hn = sh.name if sh else None
        with ProcessPoolExecutor(max_workers=workers, mp_context=get_context("spawn")) as ex:
            list(ex.map(_gauge_chunk, [(sg.name, hn, V, nc, L, seed, copy, spread, a, b) for a, b in chunks]))
            list(ex.map(_links_chunk, [(su.name, sg.name, hn, V, nc, L, eps, seed, copy, a, b) for a, b in chunks]))
        return np.ndarray((V, 4, nc, nc), dtype=np.complex128, buffer=su.buf).copy()
    finally:
        for m in shms:
            m.close()
            m.unlink()


def gauge_config(L, nc: int, eps: float, seed: int, copy: int = 0, chunk: int = 1 << 18,
                 spread: float | None = None, workers: int | None = None) -> np.ndarray:
    """U_mu(x) = g(x) exp(i eps H_mu(x)) g(x+mu)^+ with Haar g, as (V, 4, Nc, Nc) complex128.

    copy > 0 returns the same configuration under a further Haar-random gauge
    transformation (an independent starting point on the same gauge orbit).
    spread replaces the Haar g by g = exp(i spread H(x)), a gauge close to 1.
    Every site is computed from its own counters, so the result does not
    depend on how the sites are split: lattices of 2^20 sites and more are
    generated by `workers` spawned processes (default: the CPU count, at most
    16) writing into shared memory, in chunks of `chunk` sites otherwise."""
    import os
    L = tuple(int(v) for v in L)
    if len(L) != 4 or any(v < 2 for v in L):
        raise ValueError("dims must be four extents >= 2")
    V = int(np.prod(L))
    if workers is None:
        workers = min(os.cpu_count() or 1, 16) if V >= (1 << 20) else 1
    if workers > 1 and _spawn_safe():
        from concurrent.futures.process import BrokenProcessPool
        try:
            return _parallel_config(L, nc, eps, seed, copy, spread, workers)
        except BrokenProcessPool:
            pass  # a worker could not start: generate here instead
    U = np.empty((V, 4, nc, nc), dtype=np.complex128)
    g, h = _gauge_at(np.arange(V, dtype=np.int64), L, nc, seed, copy, spread)
    for start in range(0, V, chunk):
        stop = min(V, start + chunk)
        U[start:stop] = _links_for_sites(L, nc, eps, seed, copy, g, h, start, stop)
    return U


def near_identity_gauge(L, nc: int, seed: int, spread: float) -> np.ndarray:
    """g(x) = exp(i spread H(x)) with Gaussian H: a gauge transformation close to 1."""
    V = int(np.prod(L))
    sites = np.arange(V, dtype=np.int64)
    T = generators(nc)
    c = _gaussians(sites, SLOT_COPY, T.shape[0], seed, 1 << 20)
    return expi(np.einsum("na,aij->nij", c, T), spread)


def pure_gauge(L, nc: int, seed: int, spread: float | None = None) -> np.ndarray:
    """U_mu(x) = g(x) g(x+mu)^+: Haar g when spread is None, else exp(i spread H)."""
    V = int(np.prod(L))
    g = random_gauge(L, nc, seed) if spread is None else near_identity_gauge(L, nc, seed, spread)
    U = np.broadcast_to(np.eye(nc, dtype=np.complex128), (V, 4, nc, nc)).copy()
    return np.ascontiguousarray(gauge_transform(U, L, g))
