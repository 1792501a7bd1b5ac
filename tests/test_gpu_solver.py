"""GPU solves: the true residual recomputed by the FP64 oracle must meet the tolerance."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac
from oracle import lattice as L

from _gpu import built, cuda, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def _oracle_true_residual(op, x_qdp, b_qdp):
    return op.true_residual(L.from_qdp(x_qdp, op.dims), L.from_qdp(b_qdp, op.dims))


@pytest.mark.parametrize("solver", ["bicgstab", "cgnr"])
@pytest.mark.parametrize("graphs", [0, 1])
def test_plain_fp64_point_source(pkg, solver, graphs):
    """4^4, eps 0.2, kappa 0.12, c_sw 1, point source (site 0, spin 0, colour 0), tol 1e-12."""
    dims = (4, 4, 4, 4)
    gauge = W.gauge_links(dims, 0.2, 0)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.12, 1.0)
    b = W.point_source(dims, 0, 0)
    x = cuda(np.zeros_like(b))
    prm = pkg.wcl_default_params(solver=solver, sloppy="f64", tol=1e-12, use_graphs=graphs)
    _, info = ctx.wcl_invert(x, cuda(b), 1, prm)
    op = dirac.from_qdp_problem(gauge, dims, 0.12, 1.0)
    tr = _oracle_true_residual(op, host(x), b)
    assert tr <= 1e-12
    assert abs(tr - info[0]["true_residual"]) <= 1e-3 * tr + 1e-15
    # and the solution itself agrees with the oracle's own solve
    from oracle import solvers
    xo, _ = solvers.solve_even_odd(op, L.from_qdp(b, dims), tol=1e-13)
    assert np.linalg.norm(L.from_qdp(host(x), dims) - xo) <= 1e-10 * np.linalg.norm(xo)
    ctx.close()


@pytest.mark.parametrize("outer", ["df64", "f64"])
@pytest.mark.parametrize("sloppy", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("solver", ["bicgstab", "cgnr"])
def test_mixed_precision_reaches_1e10(pkg, sloppy, solver, outer):
    """Inner FP32/FP16/BF16 solver; residual replacements double-float then FP64, or all FP64."""
    dims = (8, 8, 8, 16)
    gauge = W.gauge_links(dims, 0.3, 0)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    b = W.gaussian_fermion(dims, 1)
    x = cuda(np.zeros_like(b))
    _, info = ctx.wcl_invert(x, cuda(b), 1, pkg.wcl_default_params(solver=solver, sloppy=sloppy, tol=1e-10,
                                                                   outer=outer))
    op = dirac.from_qdp_problem(gauge, dims, 0.1235, 1.0)
    tr = _oracle_true_residual(op, host(x), b)
    assert tr <= 1e-10, (tr, info)
    assert info[0]["reliable_updates"] >= 1
    ctx.close()


@pytest.mark.parametrize("sloppy,k", [("f16", 4), ("bf16", 3), ("f16", 0)])
def test_fp32_early_updates_of_16bit_solves(pkg, sloppy, k):
    """16-bit inner solver whose updates above 10^-k ||b|| evaluate b - M x with the FP32
    operator (k = 0: every intermediate update double-float): 12 RHS, every solution's
    true residual recomputed by the oracle, and the library's FP64 value agrees with it."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_SLOPPY_UPDATES
    dims = (8, 8, 8, 16)
    gauge = W.gauge_links(dims, 0.3, 3)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ctx.wcl_set_option(WCL_OPT_SLOPPY_UPDATES, k)
    b = np.stack([W.point_source(dims, s, c) for s in range(4) for c in range(3)])
    x = cuda(np.zeros_like(b))
    _, info = ctx.wcl_invert(x, cuda(b), 12, pkg.wcl_default_params(sloppy=sloppy, tol=1e-10, delta_reliable=0.01,
                                                                    check_every=2))
    op = dirac.from_qdp_problem(gauge, dims, 0.1235, 1.0)
    xh = host(x)
    for j in range(12):
        tr = _oracle_true_residual(op, xh[j], b[j])
        assert tr <= 1e-10, (j, tr, info[j])
        assert info[j]["status"] == 0 and info[j]["reliable_updates"] >= 2
        assert abs(tr - info[j]["true_residual"]) <= 1e-3 * tr, (tr, info[j])
    ctx.close()


def test_twelve_spin_colour_sources(pkg):
    dims = (4, 4, 4, 8)
    gauge = W.gauge_links(dims, 0.3, 2)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    b = np.stack([W.point_source(dims, s, c) for s in range(4) for c in range(3)])
    x = cuda(np.zeros_like(b))
    _, info = ctx.wcl_invert(x, cuda(b), 12, pkg.wcl_default_params(sloppy="f16", tol=1e-10))
    op = dirac.from_qdp_problem(gauge, dims, 0.1235, 1.0)
    xh = host(x)
    for k in range(12):
        assert _oracle_true_residual(op, xh[k], b[k]) <= 1e-10
        assert info[k]["status"] == 0
    ctx.close()


def test_batch_of_uneven_lattices(pkg):
    shapes = [(4, 4, 4, 8), (6, 6, 6, 12), (8, 4, 4, 8)]
    ctxs, ops, bs, xs = [], [], [], []
    for k, dims in enumerate(shapes):
        g = W.gauge_links(dims, 0.3, 10 + k)
        c = pkg.Context(dims)
        c.wcl_load_gauge(cuda(g), 0.1235, 1.0)
        ctxs.append(c)
        ops.append(dirac.from_qdp_problem(g, dims, 0.1235, 1.0))
        b = W.z2_fermion(dims, 20 + k, nrhs=3)
        bs.append(b)
        xs.append(cuda(np.zeros_like(b)))
    _, info = pkg.wcl_invert_batch(ctxs, xs, [cuda(b) for b in bs], 3, pkg.wcl_default_params(sloppy="f32", tol=1e-10))
    for k in range(len(shapes)):
        xh = host(xs[k])
        for r in range(3):
            assert _oracle_true_residual(ops[k], xh[r], bs[k][r]) <= 1e-10
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("shared_links", [8, 16, 32, 0, "staged", "prefetch", "paired8", "paired16", "paired32"])
@pytest.mark.parametrize("solver", ["bicgstab", "cgnr"])
def test_batch_of_lattices_four_rhs(pkg, solver, shared_links):
    """Two lattices x 4 RHS: the multi-RHS dslash and its fused reductions (per-tile partials),
    with one RHS per thread or two (the packed-pair kernel)."""
    _batch_solve(pkg, solver, shared_links, nrhs=4, sloppy="f32")


@pytest.mark.parametrize("solver", ["bicgstab", "cgnr"])
def test_tma_staged_kernel_in_a_solve(pkg, solver):
    """The TMA-staged kernel with its fused reductions inside BiCGStab and CGNR on a lattice
    with Lx = 32, every true residual recomputed by the oracle."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_TMA_STAGING

    dims = (32, 4, 4, 6)
    g = W.gauge_links(dims, 0.3, 37)
    c = pkg.Context(dims)
    c.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    c.wcl_set_option(WCL_OPT_TMA_STAGING, 1)
    c.wcl_load_gauge(cuda(g), 0.1235, 1.0)
    op = dirac.from_qdp_problem(g, dims, 0.1235, 1.0)
    b = W.z2_fermion(dims, 38, nrhs=5)
    b[2] *= 1e3
    x = cuda(np.zeros_like(b))
    _, info = c.wcl_invert(x, cuda(b), 5, pkg.wcl_default_params(solver=solver, sloppy="f32", tol=1e-10))
    xh = host(x)
    for r in range(5):
        assert _oracle_true_residual(op, xh[r], b[r]) <= 1e-10, (r, info)
    c.close()


@pytest.mark.parametrize("sloppy", ["f32", "bf16", "f16"])
def test_batch_of_lattices_paired_odd_rhs(pkg, sloppy):
    """Five RHS through the packed-pair kernel (the last pair holds one right-hand side) with
    its fused BiCGStab reductions, in FP32 and 16-bit storage."""
    _batch_solve(pkg, "bicgstab", "paired16", nrhs=5, sloppy=sloppy)


def _batch_solve(pkg, solver, shared_links, nrhs, sloppy):
    from paper_2411_08461_gb300.wcl import (WCL_OPT_AUTOTUNE, WCL_OPT_PAIRED_RHS, WCL_OPT_PREFETCH_SPINORS,
                                            WCL_OPT_SHARED_LINKS, WCL_OPT_STAGED_SPINORS)

    staged = shared_links == "staged"
    prefetch = shared_links == "prefetch"
    paired = isinstance(shared_links, str) and shared_links.startswith("paired")
    shared_links = 16 if (staged or prefetch) else int(shared_links[6:]) if paired else shared_links

    shapes = [(4, 4, 4, 8), (6, 6, 2, 10)]
    ctxs, ops, bs, xs = [], [], [], []
    for k, dims in enumerate(shapes):
        g = W.gauge_links(dims, 0.3, 30 + k)
        c = pkg.Context(dims)
        c.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
        c.wcl_set_option(WCL_OPT_SHARED_LINKS, shared_links)
        c.wcl_set_option(WCL_OPT_STAGED_SPINORS, int(staged))
        c.wcl_set_option(WCL_OPT_PAIRED_RHS, int(paired))
        c.wcl_set_option(WCL_OPT_PREFETCH_SPINORS, int(prefetch))
        c.wcl_load_gauge(cuda(g), 0.1235, 1.0)
        ctxs.append(c)
        ops.append(dirac.from_qdp_problem(g, dims, 0.1235, 1.0))
        b = W.z2_fermion(dims, 40 + k, nrhs=nrhs)
        b[2] *= 1e3
        bs.append(b)
        xs.append(cuda(np.zeros_like(b)))
    _, info = pkg.wcl_invert_batch(ctxs, xs, [cuda(b) for b in bs], nrhs,
                                   pkg.wcl_default_params(solver=solver, sloppy=sloppy, tol=1e-10))
    for k in range(len(shapes)):
        xh = host(xs[k])
        for r in range(nrhs):
            assert _oracle_true_residual(ops[k], xh[r], bs[k][r]) <= 1e-10, (k, r, info)
    for c in ctxs:
        c.close()


def test_zero_source_gives_zero(pkg):
    dims = (4, 4, 4, 4)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.2, 0)), 0.12, 1.0)
    b = np.zeros((2, 4, 4, 4, 2, 4, 3), dtype=np.complex128)
    x = cuda(np.ones_like(b))
    _, info = ctx.wcl_invert(x, cuda(b), 1, pkg.wcl_default_params())
    assert np.all(host(x) == 0) and info[0]["status"] == 0
    ctx.close()


# --- failures surface as status codes (all made on the host side) ----------------

def test_errors(pkg):
    from paper_2411_08461_gb300.wcl import WclError

    dims = (4, 4, 4, 4)
    with pytest.raises(WclError) as e:
        pkg.Context((3, 4, 4, 4))
    assert e.value.status == 1
    ctx = pkg.Context(dims)
    b = cuda(W.point_source(dims, 0, 0))
    x = cuda(np.zeros((2, 4, 4, 4, 2, 4, 3), dtype=np.complex128))
    st, _ = ctx.wcl_invert(x, b, 1, check=False)
    assert st == 9  # no gauge
    bad = W.gauge_links(dims, 0.2, 0) * 1.001  # not unitary
    with pytest.raises(WclError) as e:
        ctx.wcl_load_gauge(cuda(bad), 0.12, 1.0)
    assert e.value.status == 7
    nan = W.gauge_links(dims, 0.2, 0)
    nan[0, 0, 0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(WclError) as e:
        ctx.wcl_load_gauge(cuda(nan), 0.12, 1.0)
    assert e.value.status == 6
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.2, 0)), 0.12, 1.0)
    st, info = ctx.wcl_invert(x, b, 1, pkg.wcl_default_params(maxiter=4, check_every=2), check=False)
    assert st == 4 and info[0]["status"] == 4 and info[0]["iters"] >= 4
    assert 0 < info[0]["true_residual"] < 1
    bn = W.point_source(dims, 0, 0)
    bn[0, 0, 0, 0, 1, 0, 0] = np.inf
    st, _ = ctx.wcl_invert(x, cuda(bn), 1, check=False)
    assert st == 6
    st, _ = ctx.wcl_invert(x, b, 1, pkg.wcl_default_params(solver="fgcr_learned"), check=False)
    assert st == 10
    ctx.close()


@pytest.mark.parametrize("solver", ["bicgstab", "cgnr"])
def test_twelve_rhs_f16_tensor_core_solve(pkg, solver):
    """FP16 inner solver with the tensor-core dslash and its fused reductions reaches 1e-10."""
    dims = (8, 8, 8, 16)
    gauge = W.gauge_links(dims, 0.3, 5)
    ctx = pkg.Context(dims)
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_AUTOTUNE, 0)  # the tensor-core kernel, not the tuner's pick
    ctx.wcl_set_option(pkg.wcl.WCL_OPT_TENSOR_CORES, 1)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    b = W.z2_fermion(dims, 6, nrhs=12)
    x = cuda(np.zeros_like(b))
    _, info = ctx.wcl_invert(x, cuda(b), 12, pkg.wcl_default_params(solver=solver, sloppy="f16", tol=1e-10,
                                                                   delta_reliable=0.01))
    op = dirac.from_qdp_problem(gauge, dims, 0.1235, 1.0)
    xh = host(x)
    for k in range(12):
        assert _oracle_true_residual(op, xh[k], b[k]) <= 1e-10, (k, info[k])
    ctx.close()


def test_pinned_host_buffers(pkg):
    """b and x in page-locked host memory give the same solution, bit for bit, as
    device buffers; pageable host memory is refused."""
    import torch

    from paper_2411_08461_gb300.wcl import WclError

    dims = (4, 4, 4, 8)
    gauge = W.gauge_links(dims, 0.3, 3)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    b = W.z2_fermion(dims, 4, nrhs=2)
    prm = pkg.wcl_default_params(sloppy="f32", tol=1e-10)
    xd = cuda(np.zeros_like(b))
    ctx.wcl_invert(xd, cuda(b), 2, prm)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    _, info = ctx.wcl_invert(xh, bh, 2, prm)
    torch.cuda.synchronize()
    assert np.array_equal(xh.numpy(), host(xd))
    yd, yh = cuda(np.zeros_like(b)), torch.zeros_like(bh).pin_memory()
    ctx.wcl_apply_D(yd, xd, "f64", nrhs=2)
    ctx.wcl_apply_D(yh, xh, "f64", nrhs=2)
    torch.cuda.synchronize()
    assert np.array_equal(yh.numpy(), host(yd))
    with pytest.raises((WclError, ValueError)):
        ctx.wcl_invert(torch.zeros_like(bh), torch.from_numpy(b.copy()), 2, prm)
    ctx.close()


def test_propagator_layout_round_trip(pkg):
    """12 solutions -> propagator [.., s, s0, c, c0] (sink-source spin and colour) and back,
    bit exact; compared with the same permutation done by numpy."""
    dims = (4, 2, 2, 6)
    ctx = pkg.Context(dims)
    rng = np.random.default_rng(51)
    shape = (12, 2, dims[3], dims[2], dims[1], dims[0] // 2, 4, 3)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    prop = cuda(np.zeros(shape[1:6] + (4, 4, 3, 3), dtype=np.complex128))
    ctx.wcl_fermions_to_propagator(prop, cuda(x))
    # axes of x as [s0, c0, parity, t, z, y, x/2, s, c] -> [parity, t, z, y, x/2, s, s0, c, c0]
    ref = x.reshape((4, 3) + shape[1:]).transpose(2, 3, 4, 5, 6, 7, 0, 8, 1)
    assert np.array_equal(host(prop), ref)
    back = cuda(np.zeros_like(x))
    ctx.wcl_propagator_to_fermions(back, prop)
    assert np.array_equal(host(back), x)
    ctx.close()
