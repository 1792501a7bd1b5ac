"""GB300-native even-odd Wilson-clover propagator solver (hot path of arXiv:2411.08461).

The compute path is the CUDA library ``libwcl.so`` (sources in ``csrc/``, C ABI in
``include/wcl.h``); :mod:`paper_2411_08461_gb300.wcl` is its ctypes binding.
Build it with :func:`paper_2411_08461_gb300.build.build`.
"""
from .wcl import (  # noqa: F401
    Context,
    WclError,
    load_library,
    wcl_default_params,
    ptc_flatten,
    ptc_unflatten,
    wcl_default_mg_params,
    wcl_default_train_params,
    wcl_gamma,
    wcl_invert_batch,
    wcl_kappa_from_mass,
    wcl_kappa_from_mass_aniso,
    wcl_status_string,
)


def kappa_from_m0(m0: float, xi0: float = 1.0, nu: float = 1.0) -> float:
    """Hopping parameter from the bare mass: 1/kappa = 2 (m0 + 1 + 3 nu / xi0) (Sec. III.B, below Eq. 5)."""
    return 1.0 / (2.0 * (m0 + 1.0 + 3.0 * nu / xi0))
