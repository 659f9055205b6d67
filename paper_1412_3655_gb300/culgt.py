"""Python binding of libculgt (include/culgt.h): argument marshalling only.

Every function has the name of the C entry point it calls. Link buffers are
torch tensors in the canonical layout [V][4][Nc][Nc] complex with re/im
interleaved: either complex128/complex64 of shape (V, 4, Nc, Nc) or
float64/float32 of shape (V, 4, Nc, Nc, 2). Device entry points take CUDA
tensors and run on the current torch stream unless a stream is given; the
host entry point takes a CPU tensor. All work happens in libculgt.so; this
module has no fallback and raises if the library cannot be loaded.

Besides Landau and Coulomb gauge fixing (Params.gauge = LANDAU) the library
fixes the maximally Abelian gauge (gauge = MAG, culgt_mag_fix) and combines
either with simulated annealing (AnnealParams and the *_anneal functions).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libculgt.so")

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_DIMS, ERR_NC, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
FP64, FP32, MIXED, MIXED_DF, DF = 0, 1, 2, 3, 4
LANDAU, MAG = 0, 1
# switch_theta of the automatic FP32 -> FP64 switch of the mixed schedules
SWITCH_AUTO = 0.0


class CulgtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {culgt_status_string(status)} ({status})")


class _Params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 4),
        ("nc", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("or_variant", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("storage_reals", ctypes.c_int),
        ("theta_target", ctypes.c_double),
        ("max_sweeps", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("reunit_every", ctypes.c_int),
        ("switch_theta", ctypes.c_double),
        ("dtype_in", ctypes.c_int),
        ("threads_per_site", ctypes.c_int),
        ("block_size", ctypes.c_int),
        ("min_blocks_per_sm", ctypes.c_int),
        ("gauge", ctypes.c_int),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("sweeps_fp32", ctypes.c_int),
        ("sweeps_fp64", ctypes.c_int),
        ("theta", ctypes.c_double),
        ("F", ctypes.c_double),
        ("plaq_before", ctypes.c_double),
        ("plaq_after", ctypes.c_double),
        ("unitarity_err", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]


class _Problem(ctypes.Structure):
    _fields_ = [("d_links", ctypes.c_void_p), ("dims", ctypes.c_int * 4)]


class _AnnealParams(ctypes.Structure):
    _fields_ = [
        ("t_start", ctypes.c_double),
        ("t_end", ctypes.c_double),
        ("steps", ctypes.c_int),
        ("micro_sweeps", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
    ]


@dataclass
class AnnealParams:
    """Mirror of culgt_anneal_params (simulated annealing schedule)."""
    t_start: float = 0.6
    t_end: float = 0.01
    steps: int = 500
    micro_sweeps: int = 3
    seed: int = 0

    def _c(self) -> _AnnealParams:
        a = _AnnealParams()
        for name, _ in _AnnealParams._fields_:
            setattr(a, name, getattr(self, name))
        return a


@dataclass
class Params:
    """Mirror of culgt_params (see include/culgt.h for every field)."""
    dims: tuple
    nc: int
    omega: float = 1.7
    or_variant: int = 0
    precision: int = FP64
    storage_reals: int = 0
    theta_target: float = 1e-12
    max_sweeps: int = 10000
    check_every: int = 10
    reunit_every: int = 100
    switch_theta: float = 1e-8
    dtype_in: int = 0
    threads_per_site: int = 0
    block_size: int = 0
    min_blocks_per_sm: int = 0
    gauge: int = LANDAU

    @classmethod
    def defaults(cls, nc, dims, **kw):
        return cls(dims=tuple(int(d) for d in dims), nc=int(nc), **kw)

    def _c(self) -> _Params:
        p = _Params()
        p.dims = (ctypes.c_int * 4)(*[int(d) for d in self.dims])
        for name, _ in _Params._fields_[1:]:
            setattr(p, name, getattr(self, name))
        return p


@dataclass
class Result:
    sweeps_fp32: int = 0
    sweeps_fp64: int = 0
    theta: float = 0.0
    F: float = 0.0
    plaq_before: float = 0.0
    plaq_after: float = 0.0
    unitarity_err: float = 0.0
    seconds: float = 0.0
    status: int = 0
    extra: dict = field(default_factory=dict)

    @classmethod
    def _from(cls, r: _Result, status: int):
        return cls(**{n: getattr(r, n) for n, _ in _Result._fields_}, status=status)


_lib = None


def library():
    """Loads libculgt.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBRARY_PATH):
        raise ImportError(f"{LIBRARY_PATH} is missing; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIBRARY_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    P, R = ctypes.POINTER(_Params), ctypes.POINTER(_Result)
    A = ctypes.POINTER(_AnnealParams)
    H = ctypes.c_void_p
    sigs = {
        "culgt_status_string": (ctypes.c_char_p, [ip]),
        "culgt_default_params": (ip, [ip, ctypes.POINTER(ctypes.c_int), P]),
        "culgt_validate": (ip, [P]),
        "culgt_kernel_launches": (ctypes.c_longlong, []),
        "culgt_workspace_bytes": (ip, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "culgt_create": (ip, [P, vp, ctypes.POINTER(H)]),
        "culgt_destroy": (None, [H]),
        "culgt_load": (ip, [H, vp]),
        "culgt_store": (ip, [H, vp]),
        "culgt_handle_sweep": (ip, [H, ip]),
        "culgt_handle_theta": (ip, [H, dp, dp]),
        "culgt_handle_plaquette": (ip, [H, dp]),
        "culgt_handle_reunitarize": (ip, [H]),
        "culgt_handle_to_fp64": (ip, [H]),
        "culgt_handle_fix": (ip, [H, R]),
        "culgt_handle_tuning": (ip, [H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
        "culgt_landau_fix": (ip, [vp, P, vp, R]),
        "culgt_landau_fix_host": (ip, [vp, P, vp, R]),
        "culgt_mag_fix": (ip, [vp, P, vp, R]),
        "culgt_sweep": (ip, [vp, P, ip, vp]),
        "culgt_theta": (ip, [vp, P, vp, dp, dp]),
        "culgt_plaquette": (ip, [vp, P, vp, dp]),
        "culgt_theta_static_scratch": (ip, [vp, P, vp, vp]),
        "culgt_coulomb_fix": (ip, [vp, P, vp, R, vp]),
        "culgt_landau_fix_gauge": (ip, [vp, P, vp, R, vp]),
        "culgt_mag_fix_gauge": (ip, [vp, P, vp, R, vp]),
        "culgt_fix_batched": (ip, [ctypes.POINTER(_Problem), ip, P, vp, R]),
        "culgt_reunitarize": (ip, [vp, P, vp]),
        "culgt_default_anneal_params": (ip, [A]),
        "culgt_validate_anneal": (ip, [A]),
        "culgt_handle_heatbath": (ip, [H, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_uint]),
        "culgt_handle_anneal": (ip, [H, A]),
        "culgt_handle_heatbath_tuning": (ip, [H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "culgt_landau_fix_anneal": (ip, [vp, P, A, vp, R]),
        "culgt_fix_batched_anneal": (ip, [ctypes.POINTER(_Problem), ip, P, A, vp, R]),
        "culgt_coulomb_fix_anneal": (ip, [vp, P, A, vp, R, vp]),
        "culgt_mag_fix_anneal": (ip, [vp, P, A, vp, R]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def culgt_status_string(status: int) -> str:
    return library().culgt_status_string(int(status)).decode()


def _check(status: int, where: str) -> int:
    if status < 0:
        raise CulgtError(status, where)
    return status


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _links_ptr(t, params: Params, device: bool):
    import torch
    if device and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError("expected a CPU tensor")
    if not t.is_contiguous():
        raise ValueError("link tensor must be contiguous")
    want = torch.float32 if params.dtype_in else torch.float64
    real = t if not t.is_complex() else torch.view_as_real(t)
    if real.dtype != want:
        raise ValueError(f"link tensor element type must be {want} for dtype_in={params.dtype_in}")
    V = 1
    for d in params.dims:
        V *= int(d)
    if real.numel() != V * 4 * params.nc * params.nc * 2:
        raise ValueError("link tensor size does not match dims and nc")
    return ctypes.c_void_p(t.data_ptr())


def culgt_default_params(nc: int, dims) -> Params:
    p = _Params()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    _check(library().culgt_default_params(int(nc), d, ctypes.byref(p)), "culgt_default_params")
    return Params(dims=tuple(p.dims), **{n: getattr(p, n) for n, _ in _Params._fields_[1:]})


def culgt_kernel_launches() -> int:
    return int(library().culgt_kernel_launches())


def culgt_validate(params: Params) -> int:
    return library().culgt_validate(ctypes.byref(params._c()))


def culgt_workspace_bytes(params: Params) -> int:
    n = ctypes.c_size_t()
    _check(library().culgt_workspace_bytes(ctypes.byref(params._c()), ctypes.byref(n)), "culgt_workspace_bytes")
    return n.value


def culgt_landau_fix(links, params: Params, stream=None) -> Result:
    r = _Result()
    st = _check(library().culgt_landau_fix(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                           _stream(stream), ctypes.byref(r)), "culgt_landau_fix")
    return Result._from(r, st)


def culgt_mag_fix(links, params: Params, stream=None) -> Result:
    """Maximally Abelian gauge fixing in place (theta and F of the result are
    theta_MAG and F_MAG)."""
    r = _Result()
    st = _check(library().culgt_mag_fix(_links_ptr(links, params, True), ctypes.byref(params._c()), _stream(stream),
                                        ctypes.byref(r)), "culgt_mag_fix")
    return Result._from(r, st)


def culgt_landau_fix_host(links, params: Params, stream=None) -> Result:
    r = _Result()
    st = _check(library().culgt_landau_fix_host(_links_ptr(links, params, False), ctypes.byref(params._c()),
                                                _stream(stream), ctypes.byref(r)), "culgt_landau_fix_host")
    return Result._from(r, st)


def _gauge_ptr(gauge, params: Params):
    import torch
    V = 1
    for d in params.dims:
        V *= int(d)
    real = torch.view_as_real(gauge) if gauge.is_complex() else gauge
    if not (gauge.is_cuda and real.dtype == torch.float64 and gauge.is_contiguous()
            and real.numel() == V * params.nc * params.nc * 2):
        raise ValueError("gauge must be a contiguous CUDA float64 tensor of V*Nc*Nc*2 reals")
    return ctypes.c_void_p(gauge.data_ptr())


def culgt_landau_fix_gauge(links, params: Params, gauge, stream=None) -> Result:
    """Landau gauge fixing in place that also writes g(x) into `gauge`
    (CUDA float64/complex128 tensor of V * Nc * Nc complex values)."""
    r = _Result()
    st = _check(library().culgt_landau_fix_gauge(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                                 _stream(stream), ctypes.byref(r), _gauge_ptr(gauge, params)),
                "culgt_landau_fix_gauge")
    return Result._from(r, st)


def culgt_mag_fix_gauge(links, params: Params, gauge, stream=None) -> Result:
    """Maximally Abelian gauge fixing in place that also writes g(x) into
    `gauge` (CUDA float64/complex128 tensor of V * Nc * Nc complex values)."""
    r = _Result()
    st = _check(library().culgt_mag_fix_gauge(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                              _stream(stream), ctypes.byref(r), _gauge_ptr(gauge, params)),
                "culgt_mag_fix_gauge")
    return Result._from(r, st)


def culgt_coulomb_fix(links, params: Params, stream=None, gauge=None):
    """Coulomb gauge fixing in place, one problem per time slice. Returns one
    Result per slice (status on each). gauge: optional CUDA float64 tensor of
    V * Nc * Nc * 2 elements that receives g(x)."""
    nt = int(params.dims[0])
    rs = (_Result * nt)()
    gp = _gauge_ptr(gauge, params) if gauge is not None else None
    st = _check(library().culgt_coulomb_fix(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                            _stream(stream), rs, gp), "culgt_coulomb_fix")
    return [Result._from(r, st) for r in rs]


def _problems(links_list, dims_list, params: Params):
    n = len(links_list)
    if n != len(dims_list) or n == 0:
        raise ValueError("need one dims entry per link tensor")
    probs = (_Problem * n)()
    for i, (t, dims) in enumerate(zip(links_list, dims_list)):
        pi = Params(**{**params.__dict__, "dims": tuple(int(d) for d in dims)})
        probs[i].d_links = _links_ptr(t, pi, True)
        probs[i].dims = (ctypes.c_int * 4)(*[int(d) for d in dims])
    return probs


def culgt_default_anneal_params() -> AnnealParams:
    a = _AnnealParams()
    _check(library().culgt_default_anneal_params(ctypes.byref(a)), "culgt_default_anneal_params")
    return AnnealParams(**{n: getattr(a, n) for n, _ in _AnnealParams._fields_})


def culgt_validate_anneal(anneal: AnnealParams) -> int:
    return int(library().culgt_validate_anneal(ctypes.byref(anneal._c())))


def culgt_landau_fix_anneal(links, params: Params, anneal: AnnealParams, stream=None) -> Result:
    """Simulated annealing (anneal's schedule), then Landau gauge fixing to
    params.theta_target, in place."""
    r = _Result()
    st = _check(library().culgt_landau_fix_anneal(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                                  ctypes.byref(anneal._c()), _stream(stream), ctypes.byref(r)),
                "culgt_landau_fix_anneal")
    return Result._from(r, st)


def culgt_mag_fix_anneal(links, params: Params, anneal: AnnealParams, stream=None) -> Result:
    """Simulated annealing with MAG heat-bath sweeps, then MAG fixing, in place."""
    r = _Result()
    st = _check(library().culgt_mag_fix_anneal(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                               ctypes.byref(anneal._c()), _stream(stream), ctypes.byref(r)),
                "culgt_mag_fix_anneal")
    return Result._from(r, st)


def culgt_coulomb_fix_anneal(links, params: Params, anneal: AnnealParams, stream=None, gauge=None):
    """Coulomb gauge fixing with every time slice annealed first (slice t
    draws with seed + t). One Result per slice; gauge as in culgt_coulomb_fix."""
    nt = int(params.dims[0])
    rs = (_Result * nt)()
    gp = _gauge_ptr(gauge, params) if gauge is not None else None
    st = _check(library().culgt_coulomb_fix_anneal(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                                   ctypes.byref(anneal._c()), _stream(stream), rs, gp),
                "culgt_coulomb_fix_anneal")
    return [Result._from(r, st) for r in rs]


def culgt_fix_batched_anneal(links_list, dims_list, params: Params, anneal: AnnealParams, stream=None):
    """culgt_fix_batched after annealing every problem (problem j draws with
    seed + j). One Result per problem."""
    probs = _problems(links_list, dims_list, params)
    rs = (_Result * len(links_list))()
    st = _check(library().culgt_fix_batched_anneal(probs, len(links_list), ctypes.byref(params._c()),
                                                   ctypes.byref(anneal._c()), _stream(stream), rs),
                "culgt_fix_batched_anneal")
    return [Result._from(r, st) for r in rs]


def culgt_fix_batched(links_list, dims_list, params: Params, stream=None):
    """Landau gauge fixing of several independent lattices (each a CUDA tensor
    in the canonical layout, dims from dims_list) in shared launches; nc,
    precision and the stopping rule come from params. One Result per problem."""
    n = len(links_list)
    if n != len(dims_list) or n == 0:
        raise ValueError("need one dims entry per link tensor")
    probs = (_Problem * n)()
    for i, (t, dims) in enumerate(zip(links_list, dims_list)):
        pi = Params(**{**params.__dict__, "dims": tuple(int(d) for d in dims)})
        probs[i].d_links = _links_ptr(t, pi, True)
        probs[i].dims = (ctypes.c_int * 4)(*[int(d) for d in dims])
    rs = (_Result * n)()
    st = _check(library().culgt_fix_batched(probs, n, ctypes.byref(params._c()), _stream(stream), rs),
                "culgt_fix_batched")
    return [Result._from(r, st) for r in rs]


def culgt_sweep(links, params: Params, n_sweeps: int, stream=None) -> None:
    _check(library().culgt_sweep(_links_ptr(links, params, True), ctypes.byref(params._c()), int(n_sweeps),
                                 _stream(stream)), "culgt_sweep")


def culgt_theta(links, params: Params, stream=None):
    th, F = ctypes.c_double(), ctypes.c_double()
    _check(library().culgt_theta(_links_ptr(links, params, True), ctypes.byref(params._c()), _stream(stream),
                                 ctypes.byref(th), ctypes.byref(F)), "culgt_theta")
    return th.value, F.value


def culgt_theta_static_scratch(links, params: Params, out, stream=None) -> None:
    """theta and F into the CUDA float64 tensor `out` (2 elements), stream-ordered,
    for callers that cannot allocate device memory: the library keeps the
    partial sums in a fixed device array (lattices up to 4,194,304 sites)."""
    import torch
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 2 and out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA float64 tensor with 2 elements")
    _check(library().culgt_theta_static_scratch(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                                _stream(stream), ctypes.c_void_p(out.data_ptr())),
           "culgt_theta_static_scratch")


def culgt_plaquette(links, params: Params, stream=None) -> float:
    P = ctypes.c_double()
    _check(library().culgt_plaquette(_links_ptr(links, params, True), ctypes.byref(params._c()), _stream(stream),
                                     ctypes.byref(P)), "culgt_plaquette")
    return P.value


def culgt_reunitarize(links, params: Params, stream=None) -> None:
    _check(library().culgt_reunitarize(_links_ptr(links, params, True), ctypes.byref(params._c()),
                                       _stream(stream)), "culgt_reunitarize")


class Handle:
    """culgt_create / culgt_destroy around the handle entry points."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self._h = ctypes.c_void_p()
        _check(library().culgt_create(ctypes.byref(params._c()), _stream(stream), ctypes.byref(self._h)),
               "culgt_create")

    def close(self):
        if self._h:
            library().culgt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def culgt_load(self, links):
        _check(library().culgt_load(self._h, _links_ptr(links, self.params, True)), "culgt_load")

    def culgt_store(self, links):
        _check(library().culgt_store(self._h, _links_ptr(links, self.params, True)), "culgt_store")

    def culgt_handle_sweep(self, n: int):
        _check(library().culgt_handle_sweep(self._h, int(n)), "culgt_handle_sweep")

    def culgt_handle_theta(self):
        th, F = ctypes.c_double(), ctypes.c_double()
        _check(library().culgt_handle_theta(self._h, ctypes.byref(th), ctypes.byref(F)), "culgt_handle_theta")
        return th.value, F.value

    def culgt_handle_plaquette(self) -> float:
        P = ctypes.c_double()
        _check(library().culgt_handle_plaquette(self._h, ctypes.byref(P)), "culgt_handle_plaquette")
        return P.value

    def culgt_handle_reunitarize(self):
        _check(library().culgt_handle_reunitarize(self._h), "culgt_handle_reunitarize")

    def culgt_handle_to_fp64(self):
        _check(library().culgt_handle_to_fp64(self._h), "culgt_handle_to_fp64")

    def culgt_handle_tuning(self):
        """(threads per site, block size, min blocks per SM) of the half-sweeps."""
        t, b, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(library().culgt_handle_tuning(self._h, ctypes.byref(t), ctypes.byref(b), ctypes.byref(m)),
               "culgt_handle_tuning")
        return t.value, b.value, m.value

    def culgt_handle_heatbath(self, T: float, seed: int, sweep_word: int):
        _check(library().culgt_handle_heatbath(self._h, float(T), int(seed), int(sweep_word)),
               "culgt_handle_heatbath")

    def culgt_handle_heatbath_tuning(self):
        """(keep links in registers, min blocks per SM) of the heat-bath sweeps."""
        k, m = ctypes.c_int(), ctypes.c_int()
        _check(library().culgt_handle_heatbath_tuning(self._h, ctypes.byref(k), ctypes.byref(m)),
               "culgt_handle_heatbath_tuning")
        return k.value, m.value

    def culgt_handle_anneal(self, anneal: AnnealParams):
        _check(library().culgt_handle_anneal(self._h, ctypes.byref(anneal._c())), "culgt_handle_anneal")

    def culgt_handle_fix(self) -> Result:
        r = _Result()
        st = _check(library().culgt_handle_fix(self._h, ctypes.byref(r)), "culgt_handle_fix")
        return Result._from(r, st)


# loading the module loads the library: a missing build fails here, loudly
library()
