"""ctypes binding of libwcl: argument marshalling only, same names as include/wcl.h.

All arithmetic happens in the CUDA library.  Tensors are torch CUDA tensors
(PyTorch supplies device memory and streams); their ``data_ptr()`` is passed
straight through.  If the library has not been built, every call raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcl.so")

WCL_OK = 0
STATUS_NAMES = {
    0: "WCL_OK", 1: "WCL_ERR_INVALID_ARG", 2: "WCL_ERR_CUDA", 3: "WCL_ERR_OOM", 4: "WCL_ERR_NOT_CONVERGED",
    5: "WCL_ERR_BREAKDOWN", 6: "WCL_ERR_NONFINITE", 7: "WCL_ERR_RECONSTRUCT", 8: "WCL_ERR_TIMEOUT",
    9: "WCL_ERR_NO_GAUGE", 10: "WCL_ERR_NO_PRECOND",
}
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "df64": 4}
SOLVER = {"bicgstab": 0, "cgnr": 1, "fgcr_learned": 2, "gcr": 3, "fgcr_mg": 4, "fgcr_mg_batched": 5}
PTC_NWEIGHTS = 5760
WCL_OPT_TENSOR_CORES = 1
WCL_OPT_SHARED_LINKS = 2
WCL_OPT_AUTOTUNE = 3
WCL_OPT_PTC_TENSOR_CORES = 4
WCL_OPT_STAGED_SPINORS = 5
WCL_OPT_BLOCKED_TILES = 6
WCL_OPT_PAIRED_RHS = 7
WCL_OPT_PREFETCH_SPINORS = 8
WCL_OPT_TMA_STAGING = 9
WCL_OPT_PTC_SPLIT = 10
WCL_OPT_SLOPPY_UPDATES = 11
PTC_CHANNELS = (1, 4, 4, 4, 1)


class wcl_solve_params(ctypes.Structure):
    _fields_ = [
        ("solver", ctypes.c_int), ("outer", ctypes.c_int), ("sloppy", ctypes.c_int), ("tol", ctypes.c_double),
        ("maxiter", ctypes.c_int), ("delta_reliable", ctypes.c_double), ("restart_on_update", ctypes.c_int),
        ("gcr_nkrylov", ctypes.c_int), ("use_graphs", ctypes.c_int), ("check_every", ctypes.c_int),
    ]


class wcl_solve_info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int), ("true_residual", ctypes.c_double), ("reliable_updates", ctypes.c_int),
        ("status", ctypes.c_int), ("seconds", ctypes.c_double),
    ]


class wcl_mg_params(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_int * 4), ("nvec", ctypes.c_int), ("relax_steps", ctypes.c_int), ("pre", ctypes.c_int),
        ("post", ctypes.c_int), ("coarse_tol", ctypes.c_double), ("coarse_maxiter", ctypes.c_int),
        ("coarse_nkrylov", ctypes.c_int),
    ]


class wcl_stats(ctypes.Structure):
    _fields_ = [
        ("kernel_launches", ctypes.c_longlong), ("dslash_launches", ctypes.c_longlong), ("dslash_ms", ctypes.c_double),
        ("dslash_timed", ctypes.c_longlong), ("dslash_bytes", ctypes.c_double), ("dslash_flops", ctypes.c_double),
        ("prec_ms", ctypes.c_double * 5), ("prec_timed", ctypes.c_longlong * 5), ("prec_bytes", ctypes.c_double * 5),
        ("prec_flops", ctypes.c_double * 5),
    ]


class wcl_train_params(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


class WclError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


#: every symbol include/wcl.h declares, with (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "wcl_default_params": (None, [ctypes.POINTER(wcl_solve_params)]),
    "wcl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wcl_last_error": (ctypes.c_char_p, []),
    "wcl_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, _P]),
    "wcl_load_gauge": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double]),
    "wcl_load_gauge_aniso": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double]),
    "wcl_kappa_from_mass_aniso": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.POINTER(ctypes.c_double)]),
    "wcl_apply_D": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "wcl_apply_Mpc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "wcl_fermions_to_propagator": (ctypes.c_int, [_P, _P, _P]),
    "wcl_propagator_to_fermions": (ctypes.c_int, [_P, _P, _P]),
    "wcl_invert": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(wcl_solve_params),
                                  ctypes.POINTER(wcl_solve_info)]),
    "wcl_invert_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                        ctypes.c_int, ctypes.POINTER(wcl_solve_params),
                                        ctypes.POINTER(wcl_solve_info)]),
    "wcl_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "wcl_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "wcl_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(wcl_stats), ctypes.c_int]),
    "wcl_apply_Mpc_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "wcl_default_train_params": (None, [ctypes.POINTER(wcl_train_params)]),
    "wcl_precond_load": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "wcl_precond_get": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "wcl_precond_apply": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "wcl_precond_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    "wcl_precond_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(wcl_train_params),
                                         ctypes.POINTER(ctypes.c_double)]),
    "wcl_gamma": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "wcl_kappa_from_mass": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "wcl_wall_source": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "wcl_sequential_source": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double)]),
    "wcl_contract": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "wcl_destroy": (ctypes.c_int, [_P]),
    "wcl_load_staggered": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "wcl_clover_force": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "wcl_hisq_smear": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double]),
    "wcl_apply_staggered": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "wcl_invert_staggered": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(wcl_solve_params),
                                            ctypes.POINTER(wcl_solve_info)]),
    "wcl_default_mg_params": (None, [ctypes.POINTER(wcl_mg_params)]),
    "wcl_mg_setup": (ctypes.c_int, [_P, _P, ctypes.POINTER(wcl_mg_params)]),
    "wcl_mg_cycle": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "wcl_mg_cycle_batched": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "wcl_mg_restrict": (ctypes.c_int, [_P, _P, _P]),
    "wcl_mg_prolong": (ctypes.c_int, [_P, _P, _P]),
    "wcl_mg_coarse_apply": (ctypes.c_int, [_P, _P, _P]),
    "wcl_mg_get_prolongator": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "wcl_mg_get_stencil": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Open libwcl.so and declare every exported signature; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libwcl.so not built at {path}: run __graft_entry__.build() "
                           "(there is no CPU fallback for the CUDA path)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != WCL_OK:
        msg = load_library().wcl_last_error().decode(errors="replace")
        raise WclError(status, where, msg)


def _ptr(t, dtype=None, numel=None, name="tensor", fermion=False):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda and not (fermion and t.is_pinned()):
        raise ValueError(f"{name} must live on a CUDA device" + (" or in pinned host memory" if fermion else ""))
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (Sec. II.B: contiguous fields only)")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def wcl_default_params(**overrides) -> wcl_solve_params:
    p = wcl_solve_params()
    load_library().wcl_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k in ("outer", "sloppy") and isinstance(v, str):
            v = PREC[v]
        if k == "solver" and isinstance(v, str):
            v = SOLVER[v]
        setattr(p, k, v)
    return p


def wcl_status_string(status: int) -> str:
    return load_library().wcl_status_string(status).decode()


def wcl_gamma(n: int):
    """Gamma(n) in the DeGrand-Rossi basis as a 4 x 4 complex128 numpy array (host only)."""
    import numpy as np

    buf = np.zeros(32, dtype=np.float64)
    _check(load_library().wcl_gamma(int(n), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "wcl_gamma")
    return buf.view(np.complex128).reshape(4, 4)


def wcl_kappa_from_mass(m0: float) -> float:
    k = ctypes.c_double()
    _check(load_library().wcl_kappa_from_mass(float(m0), ctypes.byref(k)), "wcl_kappa_from_mass")
    return k.value


def wcl_kappa_from_mass_aniso(m0: float, xi0: float, nu: float) -> float:
    k = ctypes.c_double()
    _check(load_library().wcl_kappa_from_mass_aniso(float(m0), float(xi0), float(nu), ctypes.byref(k)),
           "wcl_kappa_from_mass_aniso")
    return k.value


def _mom_arg(mom):
    if mom is None:
        return None
    if len(mom) != 3:
        raise ValueError("mom must hold three integers (x, y, z)")
    return (ctypes.c_int * 3)(*(int(v) for v in mom))


def _gamma_arg(gamma):
    import numpy as np

    if gamma is None:
        return None, None
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128))
    if g.shape != (4, 4):
        raise ValueError("gamma must be a 4 x 4 matrix")
    buf = g.view(np.float64).ravel().copy()
    return buf, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """One lattice on one GPU (wcl_create ... wcl_destroy)."""

    def __init__(self, dims: Sequence[int], t_boundary: int = -1, device: int = 0, stream=None):
        import torch

        lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        lx, ly, lz, lt = self.dims
        self.volume = lx * ly * lz * lt
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        handle = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.dims)
        _check(lib.wcl_create(ctypes.byref(handle), d, int(t_boundary), int(device), ctypes.c_void_p(stream.cuda_stream)),
               "wcl_create")
        self.handle = handle

    # fields are complex128 in the QDP layout
    @property
    def fermion_numel(self) -> int:
        return self.volume * 12

    def wcl_load_gauge(self, gauge, kappa: float, csw: float):
        import torch

        _check(load_library().wcl_load_gauge(self.handle, _ptr(gauge, torch.complex128, self.volume * 36, "gauge"),
                                             float(kappa), float(csw)), "wcl_load_gauge")

    def wcl_load_gauge_aniso(self, gauge, kappa: float, xi0: float, nu: float, csw_t: float, csw_r: float):
        import torch

        _check(load_library().wcl_load_gauge_aniso(self.handle, _ptr(gauge, torch.complex128, self.volume * 36, "gauge"),
                                                   float(kappa), float(xi0), float(nu), float(csw_t), float(csw_r)),
               "wcl_load_gauge_aniso")

    def wcl_apply_D(self, out, inp, prec: str = "f64", nrhs: int = 1):
        import torch

        n = self.fermion_numel * nrhs
        _check(load_library().wcl_apply_D(self.handle, _ptr(out, torch.complex128, n, "out", True),
                                          _ptr(inp, torch.complex128, n, "in", True), PREC[prec], nrhs), "wcl_apply_D")

    def wcl_apply_Mpc(self, out_e, in_e, prec: str = "f64", nrhs: int = 1, dagger: bool = False):
        import torch

        n = self.fermion_numel // 2 * nrhs
        _check(load_library().wcl_apply_Mpc(self.handle, _ptr(out_e, torch.complex128, n, "out_e", True),
                                            _ptr(in_e, torch.complex128, n, "in_e", True), PREC[prec], nrhs, int(dagger)),
               "wcl_apply_Mpc")

    def wcl_apply_Mpc_noalloc(self, out_e, in_e, dagger: bool = False):
        """FP64 M_hat (or its adjoint) with the library's fixed scratch array: no allocation in the call."""
        import torch

        n = self.fermion_numel // 2
        _check(load_library().wcl_apply_Mpc_noalloc(self.handle, _ptr(out_e, torch.complex128, n, "out_e"),
                                                    _ptr(in_e, torch.complex128, n, "in_e"), int(dagger)),
               "wcl_apply_Mpc_noalloc")

    # ---- clover fermion force ------------------------------------------------------
    def wcl_clover_force(self, force, x_e, include_logdet: bool = True):
        """force <- F of the two-flavour even-odd clover action for X = (M_hat^+ M_hat)^-1 phi."""
        import torch

        _check(load_library().wcl_clover_force(self.handle, _ptr(force, torch.complex128, self.volume * 36, "force", True),
                                               _ptr(x_e, torch.complex128, self.fermion_numel // 2, "x_e", True),
                                               int(include_logdet)),
               "wcl_clover_force")

    # ---- staggered operator --------------------------------------------------------
    def wcl_hisq_smear(self, fat, long_links, gauge, eps_naik: float = 0.0):
        import torch

        n = self.volume * 36
        _check(load_library().wcl_hisq_smear(self.handle, _ptr(fat, torch.complex128, n, "fat", True),
                                             _ptr(long_links, torch.complex128, n, "long", True),
                                             _ptr(gauge, torch.complex128, n, "gauge", True), float(eps_naik)),
               "wcl_hisq_smear")

    def wcl_load_staggered(self, fat, long_links, mass: float):
        import torch

        n = self.volume * 36
        _check(load_library().wcl_load_staggered(self.handle, _ptr(fat, torch.complex128, n, "fat", True),
                                                 _ptr(long_links, torch.complex128, n, "long", True), float(mass)),
               "wcl_load_staggered")

    def wcl_apply_staggered(self, out, inp, prec: str = "f64", nrhs: int = 1):
        import torch

        n = self.volume * 3 * nrhs
        _check(load_library().wcl_apply_staggered(self.handle, _ptr(out, torch.complex128, n, "out", True),
                                                  _ptr(inp, torch.complex128, n, "in", True), PREC[prec], int(nrhs)),
               "wcl_apply_staggered")

    def wcl_invert_staggered(self, x, b, nrhs: int = 1, params: wcl_solve_params | None = None, check: bool = True):
        import torch

        params = params or wcl_default_params()
        info = (wcl_solve_info * nrhs)()
        n = self.volume * 3 * nrhs
        st = load_library().wcl_invert_staggered(self.handle, _ptr(x, torch.complex128, n, "x", True),
                                                 _ptr(b, torch.complex128, n, "b", True), int(nrhs),
                                                 ctypes.byref(params), info)
        out = [{"iters": i.iters, "true_residual": i.true_residual, "reliable_updates": i.reliable_updates,
                "status": i.status, "seconds": i.seconds} for i in info]
        if check:
            _check(st, "wcl_invert_staggered")
        return st, out

    # ---- multigrid ---------------------------------------------------------------
    def _mg_coarse_numel(self):
        p = self._mg_params
        cs = 1
        for d in range(4):
            cs *= self.dims[d] // p.block[d]
        return cs * 2 * p.nvec

    def wcl_mg_setup(self, starts, params: wcl_mg_params | None = None):
        """Build the two-level hierarchy from `nvec` start vectors ([nvec][QDP fermion] complex128)."""
        import torch

        params = params or wcl_default_mg_params()
        _check(load_library().wcl_mg_setup(self.handle, _ptr(starts, torch.complex128,
                                                             self.fermion_numel * params.nvec, "starts", True),
                                           ctypes.byref(params)), "wcl_mg_setup")
        self._mg_params = params

    def wcl_mg_cycle(self, out, inp) -> int:
        import torch

        it = ctypes.c_int(0)
        _check(load_library().wcl_mg_cycle(self.handle, _ptr(out, torch.complex128, self.fermion_numel, "out", True),
                                           _ptr(inp, torch.complex128, self.fermion_numel, "in", True),
                                           ctypes.byref(it)), "wcl_mg_cycle")
        return it.value

    def wcl_mg_cycle_batched(self, out, inp, nrhs: int):
        import torch

        n = self.fermion_numel * nrhs
        _check(load_library().wcl_mg_cycle_batched(self.handle, _ptr(out, torch.complex128, n, "out", True),
                                                   _ptr(inp, torch.complex128, n, "in", True), int(nrhs)),
               "wcl_mg_cycle_batched")

    def wcl_mg_restrict(self, coarse, fine):
        import torch

        _check(load_library().wcl_mg_restrict(self.handle, _ptr(coarse, torch.complex128, self._mg_coarse_numel(),
                                                                "coarse"),
                                              _ptr(fine, torch.complex128, self.fermion_numel, "fine", True)),
               "wcl_mg_restrict")

    def wcl_mg_prolong(self, fine, coarse):
        import torch

        _check(load_library().wcl_mg_prolong(self.handle, _ptr(fine, torch.complex128, self.fermion_numel, "fine", True),
                                             _ptr(coarse, torch.complex128, self._mg_coarse_numel(), "coarse")),
               "wcl_mg_prolong")

    def wcl_mg_coarse_apply(self, out, inp):
        import torch

        n = self._mg_coarse_numel()
        _check(load_library().wcl_mg_coarse_apply(self.handle, _ptr(out, torch.complex128, n, "out"),
                                                  _ptr(inp, torch.complex128, n, "in")), "wcl_mg_coarse_apply")

    def wcl_mg_get_prolongator(self):
        """P as a numpy array [2][Lt][Lz][Ly][Lx/2][12][2 nvec] complex128 (QDP site order)."""
        import numpy as np

        lx, ly, lz, lt = self.dims
        n = 2 * self._mg_params.nvec
        buf = np.zeros(self.volume * 12 * n * 2, dtype=np.float64)
        _check(load_library().wcl_mg_get_prolongator(self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_mg_get_prolongator")
        return buf.view(np.complex128).reshape(2, lt, lz, ly, lx // 2, 12, n)

    def wcl_mg_get_stencil(self):
        """(X, Yf, Yb) as numpy arrays (Ct, Cz, Cy, Cx, n, n) and (4, Ct, Cz, Cy, Cx, n, n), n = 2 nvec."""
        import numpy as np

        p = self._mg_params
        cd = [self.dims[d] // p.block[d] for d in range(4)]
        nc = cd[0] * cd[1] * cd[2] * cd[3]
        n = 2 * p.nvec
        buf = np.zeros(9 * nc * n * n * 2, dtype=np.float64)
        _check(load_library().wcl_mg_get_stencil(self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_mg_get_stencil")
        y = buf.view(np.complex128).reshape(9, cd[3], cd[2], cd[1], cd[0], n, n)
        return y[0], np.stack([y[1 + 2 * mu] for mu in range(4)]), np.stack([y[2 + 2 * mu] for mu in range(4)])

    def wcl_invert(self, x, b, nrhs: int = 1, params: wcl_solve_params | None = None, check: bool = True):
        import torch

        params = params or wcl_default_params()
        info = (wcl_solve_info * nrhs)()
        n = self.fermion_numel * nrhs
        st = load_library().wcl_invert(self.handle, _ptr(x, torch.complex128, n, "x", True), _ptr(b, torch.complex128, n, "b", True),
                                       nrhs, ctypes.byref(params), info)
        if check:
            _check(st, "wcl_invert")
        return st, [_info_dict(i) for i in info]

    # ---- learned preconditioner (weights are host numpy complex128, WCL_PTC_NWEIGHTS) ----
    def wcl_precond_load(self, weights):
        import numpy as np

        w = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128).ravel())
        if w.size != PTC_NWEIGHTS:
            raise ValueError(f"expected {PTC_NWEIGHTS} complex weights, got {w.size}")
        buf = w.view(np.float64)
        _check(load_library().wcl_precond_load(self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_precond_load")

    def wcl_precond_get(self):
        import numpy as np

        buf = np.zeros(2 * PTC_NWEIGHTS, dtype=np.float64)
        _check(load_library().wcl_precond_get(self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_precond_get")
        return buf.view(np.complex128)

    def wcl_precond_apply(self, out_e, in_e, nrhs: int = 1, bf16: bool = False):
        import torch

        n = self.fermion_numel // 2 * nrhs
        _check(load_library().wcl_precond_apply(self.handle, _ptr(out_e, torch.complex128, n, "out_e"),
                                                _ptr(in_e, torch.complex128, n, "in_e"), nrhs, int(bf16)),
               "wcl_precond_apply")

    def wcl_fermions_to_propagator(self, prop, x12):
        """12 solutions [12][fermion] -> propagator [2][Lt][Lz][Ly][Lx/2][4][4][3][3]."""
        import torch

        n = self.fermion_numel * 12
        _check(load_library().wcl_fermions_to_propagator(self.handle, _ptr(prop, torch.complex128, n, "prop", True),
                                                         _ptr(x12, torch.complex128, n, "x12", True)),
               "wcl_fermions_to_propagator")

    def wcl_propagator_to_fermions(self, x12, prop):
        import torch

        n = self.fermion_numel * 12
        _check(load_library().wcl_propagator_to_fermions(self.handle, _ptr(x12, torch.complex128, n, "x12", True),
                                                         _ptr(prop, torch.complex128, n, "prop", True)),
               "wcl_propagator_to_fermions")

    def wcl_wall_source(self, b12, t0: int, mom=None):
        """Twelve wall sources on timeslice t0 ([12][fermion]), momentum phase exp(+i p.x)."""
        import torch

        n = self.fermion_numel * 12
        _check(load_library().wcl_wall_source(self.handle, _ptr(b12, torch.complex128, n, "b12", True), int(t0),
                                              _mom_arg(mom)), "wcl_wall_source")

    def wcl_sequential_source(self, X, S, t: int, mom=None, gamma=None):
        """X = exp(-i p.x) Gamma S on timeslice t (Gamma = gamma_5 when None); propagators."""
        import torch

        n = self.fermion_numel * 12
        keep, g = _gamma_arg(gamma)
        _check(load_library().wcl_sequential_source(self.handle, _ptr(X, torch.complex128, n, "X", True),
                                                    _ptr(S, torch.complex128, n, "S", True), int(t), _mom_arg(mom), g),
               "wcl_sequential_source")
        del keep

    def wcl_contract(self, out, A, B, gamma=None, mom=None):
        """out[t] = sum_{x in t} exp(-i p.x) conj(A) Gamma B summed over spin and colour (Lt complex128)."""
        import torch

        n = self.fermion_numel * 12
        keep, g = _gamma_arg(gamma)
        _check(load_library().wcl_contract(self.handle, _ptr(out, torch.complex128, self.dims[3], "out", True),
                                           _ptr(A, torch.complex128, n, "A", True), _ptr(B, torch.complex128, n, "B", True), g,
                                           _mom_arg(mom)), "wcl_contract")
        del keep

    def wcl_precond_loss_grad(self, r_e, e_e, npairs: int):
        import numpy as np
        import torch

        n = self.fermion_numel // 2 * npairs
        loss = ctypes.c_double()
        g = np.zeros(2 * PTC_NWEIGHTS, dtype=np.float64)
        _check(load_library().wcl_precond_loss_grad(self.handle, _ptr(r_e, torch.complex128, n, "r_e"),
                                                    _ptr(e_e, torch.complex128, n, "e_e"), npairs, ctypes.byref(loss),
                                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_precond_loss_grad")
        return loss.value, g.view(np.complex128)

    def wcl_precond_train(self, r_e, e_e, npairs: int, params: wcl_train_params | None = None):
        import numpy as np
        import torch

        if params is None:
            params = wcl_train_params()
            load_library().wcl_default_train_params(ctypes.byref(params))
        n = self.fermion_numel // 2 * npairs
        losses = np.zeros(params.epochs, dtype=np.float64)
        _check(load_library().wcl_precond_train(self.handle, _ptr(r_e, torch.complex128, n, "r_e"),
                                                _ptr(e_e, torch.complex128, n, "e_e"), npairs, ctypes.byref(params),
                                                losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "wcl_precond_train")
        return losses

    def wcl_set_option(self, option: int, value: int):
        _check(load_library().wcl_set_option(self.handle, int(option), int(value)), "wcl_set_option")

    def wcl_set_profiling(self, enable: bool = True):
        _check(load_library().wcl_set_profiling(self.handle, int(enable)), "wcl_set_profiling")

    def wcl_get_stats(self, reset: bool = False) -> dict:
        s = wcl_stats()
        _check(load_library().wcl_get_stats(self.handle, ctypes.byref(s), int(reset)), "wcl_get_stats")
        out = {}
        for k, _ in wcl_stats._fields_:
            v = getattr(s, k)
            out[k] = list(v) if k.startswith("prec_") else v
        return out

    def wcl_destroy(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().wcl_destroy(self.handle)
            self.handle = None

    close = wcl_destroy

    def __del__(self):
        try:
            self.wcl_destroy()
        except Exception:
            pass


def wcl_default_train_params(**overrides) -> wcl_train_params:
    p = wcl_train_params()
    load_library().wcl_default_train_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def wcl_default_mg_params(**overrides) -> wcl_mg_params:
    p = wcl_mg_params()
    load_library().wcl_default_mg_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "block":
            p.block = (ctypes.c_int * 4)(*v)
        else:
            setattr(p, k, v)
    return p


def ptc_flatten(layers) -> "numpy.ndarray":
    """Oracle-style list of (Cout, Cin, 9, 4, 4) complex arrays -> the flat weight vector."""
    import numpy as np

    return np.concatenate([np.asarray(w, dtype=np.complex128).ravel() for w in layers])


def ptc_unflatten(flat):
    """Flat weight vector -> list of (Cout, Cin, 9, 4, 4) arrays, channels 1, 4, 4, 4, 1."""
    out, off = [], 0
    for cin, cout in zip(PTC_CHANNELS[:-1], PTC_CHANNELS[1:]):
        n = cout * cin * 9 * 16
        out.append(flat[off:off + n].reshape(cout, cin, 9, 4, 4))
        off += n
    return out


def _info_dict(i: wcl_solve_info) -> dict:
    return {"iters": i.iters, "true_residual": i.true_residual, "reliable_updates": i.reliable_updates,
            "status": i.status, "seconds": i.seconds}


def wcl_invert_batch(ctxs: Sequence[Context], xs, bs, nrhs: int, params: wcl_solve_params | None = None,
                     check: bool = True):
    """Several lattices, one launch per solver step (wcl_invert_batch)."""
    import torch

    params = params or wcl_default_params()
    n = len(ctxs)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    xp = (ctypes.c_void_p * n)(*[_ptr(x, torch.complex128, c.fermion_numel * nrhs, "x", True).value for c, x in zip(ctxs, xs)])
    bp = (ctypes.c_void_p * n)(*[_ptr(b, torch.complex128, c.fermion_numel * nrhs, "b", True).value for c, b in zip(ctxs, bs)])
    info = (wcl_solve_info * (n * nrhs))()
    st = load_library().wcl_invert_batch(hs, n, xp, bp, nrhs, ctypes.byref(params), info)
    if check:
        _check(st, "wcl_invert_batch")
    return st, [_info_dict(i) for i in info]
