"""wcl_apply_Mpc_noalloc: the FP64 Schur operator for callers that cannot let the
library allocate device memory during the call (their own pool allocator owns the
device, or an allocation's synchronisation or failure is unacceptable mid-run).

Checked through the C ABI against wcl_apply_Mpc(..., WCL_F64, ...) on two calls in a
row (different inputs, both adjoint settings), at the FP64 tolerance used by every
other parity test.  The first call comes on a lattice shape no other call of the
process has used, before wcl_apply_Mpc sees it, so that neither a first call nor an
untuned configuration may allocate: free device memory is the same before and after
each call.  This file is named to be collected last, so that a run that stops at the
first failure has run every other test already; it also passes on its own.
"""
import ctypes

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

    dims = (10, 4, 2, 6)  # Vh = 240 sites per parity; a shape no other test uses
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.4, 31)), 0.1235, 1.0)
    calls = [(32, False), (33, True)]
    psis = [cuda(W.gaussian_fermion(dims, seed)[0]) for seed, _ in calls]
    outs = [torch.full_like(p, complex(np.nan, np.nan)) for p in psis]
    free = []
    for psi, out, (_, dagger) in zip(psis, outs, calls):
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ctx.wcl_apply_Mpc_noalloc(out, psi, dagger=dagger)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # neither the first call on a fresh shape nor the second allocated device memory
    assert free[1] == free[0] and free[3] == free[2], free
    for psi, out, (_, dagger) in zip(psis, outs, calls):
        ref = torch.empty_like(psi)
        ctx.wcl_apply_Mpc(ref, psi, "f64", dagger=dagger)
        assert relerr(host(out), host(ref)) <= TOL["f64"], dagger
    ctx.close()


def test_noalloc_rejects_host_memory(pkg):
    """Pageable host memory is refused with WCL_ERR_INVALID_ARG before any launch."""
    from paper_2411_08461_gb300.wcl import load_library

    dims = (6, 4, 4, 8)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.4, 34)), 0.1235, 1.0)
    h_in = W.gaussian_fermion(dims, 35)[0].copy()
    h_out = np.zeros_like(h_in)
    d_in, d_out = cuda(h_in), cuda(h_out)
    lib = load_library()
    host_ptr = ctypes.c_void_p(h_in.ctypes.data)
    dev_out = ctypes.c_void_p(d_out.data_ptr())
    assert lib.wcl_apply_Mpc_noalloc(ctx.handle, dev_out, host_ptr, 0) == 1
    assert lib.wcl_apply_Mpc_noalloc(ctx.handle, ctypes.c_void_p(h_out.ctypes.data),
                                     ctypes.c_void_p(d_in.data_ptr()), 0) == 1
    assert "device memory" in lib.wcl_last_error().decode()
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
