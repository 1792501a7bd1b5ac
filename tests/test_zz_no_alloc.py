"""wcl_apply_Mpc_noalloc: the FP64 Schur operator for callers that cannot let the
library allocate device memory during the call (their own pool allocator owns the
device, or an allocation's synchronisation or failure is unacceptable mid-run).

Checked through the C ABI against wcl_apply_Mpc(..., WCL_F64, ...) on two calls in a
row (different inputs, both adjoint settings), at the FP64 tolerance used by every
other parity test.  This file is named to be collected last, so that a run that stops
at the first failure has run every other test already; it also passes on its own.
"""
import numpy as np
import pytest

import workloads as W

from _gpu import TOL, built, cuda, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def test_noalloc_matches_apply_mpc_twice(pkg):
    import torch

    dims = (6, 4, 4, 8)  # Vh = 384 sites per parity, well inside the fixed scratch
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.4, 31)), 0.1235, 1.0)
    free = []
    for call, (seed, dagger) in enumerate([(32, False), (33, True)]):
        psi = cuda(W.gaussian_fermion(dims, seed)[0])
        ref = torch.empty_like(psi)
        ctx.wcl_apply_Mpc(ref, psi, "f64", dagger=dagger)
        out = torch.full_like(psi, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ctx.wcl_apply_Mpc_noalloc(out, psi, dagger=dagger)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert relerr(host(out), host(ref)) <= TOL["f64"], (call, dagger)
    # the second call leaves device memory exactly as it found it
    assert free[3] == free[2]
    ctx.close()


def test_noalloc_rejects_lattices_beyond_the_scratch(pkg):
    from paper_2411_08461_gb300.wcl import WclError

    dims = (16, 16, 16, 16)  # Vh = 32768 > WCL_NOALLOC_MAX_VH
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.3, 1)), 0.1235, 1.0)
    psi = cuda(W.gaussian_fermion(dims, 2)[0])
    out = cuda(np.zeros_like(host(psi)))
    with pytest.raises(WclError) as e:
        ctx.wcl_apply_Mpc_noalloc(out, psi)
    assert e.value.status == 1 and "scratch" in str(e.value)
    ctx.close()
