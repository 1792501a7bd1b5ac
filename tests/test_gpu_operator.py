"""GPU parity of the operator applies (fused dslash + clover) against the FP64 oracle.

Tolerances (normwise relative): FP64 1e-12, FP32 1e-5, FP16/BF16 5e-3.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dirac
from oracle import lattice as L

from _gpu import TOL, built, cuda, host, relerr

pytestmark = pytest.mark.gpu

# several tiles and ragged tails: Vh = 128, 192, 8, 2592, 4096
SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2), (6, 6, 6, 8), (8, 8, 8, 16)]


@pytest.fixture(scope="module")
def pkg():
    return built()


def _setup(pkg, dims, eps=0.3, seed=0, kappa=0.1235, csw=1.0, tb=-1):
    gauge = W.gauge_links(dims, eps, seed)
    ctx = pkg.Context(dims, t_boundary=tb)
    ctx.wcl_load_gauge(cuda(gauge), kappa, csw)
    op = dirac.from_qdp_problem(gauge, dims, kappa, csw, tb)
    return ctx, op, gauge


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("dims", SHAPES)
def test_apply_D_parity(pkg, dims, prec):
    ctx, op, _ = _setup(pkg, dims, seed=1)
    psi = W.gaussian_fermion(dims, 2)
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_D(out, cuda(psi), prec)
    ref = dirac.apply_D_qdp(op, psi)
    assert relerr(host(out), ref) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("tb", [1, -1])
def test_apply_D_time_boundary_and_csw(pkg, tb):
    dims = (4, 2, 2, 6)
    ctx, op, _ = _setup(pkg, dims, eps=0.7, seed=3, kappa=0.13, csw=1.7, tb=tb)
    psi = W.gaussian_fermion(dims, 4)
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_D(out, cuda(psi), "f64")
    assert relerr(host(out), dirac.apply_D_qdp(op, psi)) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_Mpc_parity(pkg, prec, dagger):
    dims = (6, 4, 2, 8)
    ctx, op, _ = _setup(pkg, dims, seed=5)
    psi = W.gaussian_fermion(dims, 6)[0]
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, dagger=dagger)
    ref = dirac.apply_Mhat_qdp(op, psi, dagger)
    assert relerr(host(out), ref) <= TOL[prec]
    ctx.close()


def test_apply_D_multi_rhs(pkg):
    dims = (4, 4, 2, 4)
    ctx, op, _ = _setup(pkg, dims, seed=7)
    psi = W.gaussian_fermion(dims, 8, nrhs=12)
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_D(out, cuda(psi), "f32", nrhs=12)
    got = host(out)
    for k in range(12):
        assert relerr(got[k], dirac.apply_D_qdp(op, psi[k])) <= 1e-5
    ctx.close()


def test_gamma5_hermiticity_on_gpu(pkg):
    """<phi, M psi> = <g5 M g5 phi, psi>, computed with the GPU operator only (any size)."""
    dims = (8, 8, 8, 16)
    ctx, _, _ = _setup(pkg, dims, seed=9)
    phi, psi = W.gaussian_fermion(dims, 10), W.gaussian_fermion(dims, 11)
    g5 = np.array([1, 1, -1, -1])[:, None]
    mpsi, mphi = cuda(np.zeros_like(psi)), cuda(np.zeros_like(psi))
    ctx.wcl_apply_D(mpsi, cuda(psi), "f64")
    ctx.wcl_apply_D(mphi, cuda(g5 * phi), "f64")
    lhs = np.vdot(phi, host(mpsi))
    rhs = np.vdot(g5 * host(mphi), psi)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    ctx.close()


@pytest.mark.parametrize("tensor_cores", [1, 0])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 2, 8), 12), ((4, 4, 4, 4), 5), ((8, 4, 4, 6), 16)])
def test_apply_Mpc_multi_rhs_f16(pkg, dims, nrhs, dagger, tensor_cores):
    """12-RHS 16-bit Schur operator: tensor-core (mma.sync f16, FP32 accumulate) and per-thread kernels."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_SHARED_LINKS, WCL_OPT_TENSOR_CORES

    ctx, op, _ = _setup(pkg, dims, seed=13)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)  # the kernel under test, not the tuner's pick
    ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, 0)
    ctx.wcl_set_option(WCL_OPT_TENSOR_CORES, tensor_cores)
    psi = W.gaussian_fermion(dims, 14, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7  # very different magnitudes per right-hand side
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), "f16", nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL["f16"], k
    ctx.close()


def test_tensor_core_and_per_thread_kernels_agree(pkg):
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_SHARED_LINKS, WCL_OPT_TENSOR_CORES

    dims = (8, 8, 8, 16)
    ctx, _, _ = _setup(pkg, dims, seed=15)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, 0)
    psi = cuda(W.gaussian_fermion(dims, 16, nrhs=12)[:, 0].copy())
    outs = []
    for tc in (1, 0):
        ctx.wcl_set_option(WCL_OPT_TENSOR_CORES, tc)
        o = cuda(np.zeros(psi.shape, dtype=np.complex128))
        ctx.wcl_apply_Mpc(o, psi, "f16", nrhs=12)
        outs.append(host(o))
    assert relerr(outs[0], outs[1]) <= 5e-3
    ctx.close()


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 2, 8), 12), ((6, 6, 6, 8), 4), ((2, 2, 2, 2), 16), ((8, 4, 4, 6), 7)])
def test_apply_Mpc_multi_rhs_shared_links(pkg, dims, nrhs, dagger, prec, tile):
    """Multi-RHS Schur operator with links and clover staged in shared memory (8-, 16- and 32-site
    tiles, ragged last tile for Vh = 96, 1296, 8, 384) against the oracle, RHS of very different
    size; FP64 always runs 16-site tiles."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_SHARED_LINKS

    ctx, op, _ = _setup(pkg, dims, seed=17)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, tile)
    psi = W.gaussian_fermion(dims, 18, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 2, 8), 12), ((6, 6, 6, 8), 4), ((2, 2, 2, 2), 16), ((8, 4, 4, 6), 7)])
def test_apply_Mpc_multi_rhs_paired(pkg, dims, nrhs, dagger, prec, tile):
    """The packed-pair kernel (two right-hand sides per thread in float2 registers, FFMA2):
    8-, 16- and 32-site tiles, ragged last tile for Vh = 96, 1296, 8, 384, an odd RHS count
    (the last pair holds one right-hand side) and RHS of very different size."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_PAIRED_RHS, WCL_OPT_SHARED_LINKS

    ctx, op, _ = _setup(pkg, dims, seed=27)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, tile)
    ctx.wcl_set_option(WCL_OPT_PAIRED_RHS, 1)
    psi = W.gaussian_fermion(dims, 28, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7
    psi[nrhs - 1] *= 1e5
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_multi_rhs_paired_blocked_tile_order(pkg, prec):
    """The packed-pair kernel walking its 16-site tiles in blocks of z planes (32x24x24x4)."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_BLOCKED_TILES, WCL_OPT_PAIRED_RHS

    dims = (32, 24, 24, 4)
    ctx, op, _ = _setup(pkg, dims, seed=29)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_BLOCKED_TILES, 1)
    ctx.wcl_set_option(WCL_OPT_PAIRED_RHS, 1)
    psi = W.gaussian_fermion(dims, 30, nrhs=6)[:, 0].copy()
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=6)
    got = host(out)
    for k in range(6):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], False)) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((32, 4, 2, 4), 12), ((32, 2, 2, 6), 4), ((32, 4, 4, 2), 7), ((32, 6, 2, 2), 16)])
def test_apply_Mpc_multi_rhs_tma_staged(pkg, dims, nrhs, dagger, mode):
    """The persistent FP32 kernel whose links and clover arrive by tensor copies (TMA),
    tiles = whole x-rows of 16 sites (Lx = 32), two stages in flight; more rows than
    CTAs only on the larger shapes, so both one and several tiles per CTA are covered."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_TMA_STAGING

    ctx, op, _ = _setup(pkg, dims, seed=33)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_TMA_STAGING, mode)
    psi = W.gaussian_fermion(dims, 34, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), "f32", nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL["f32"], k
    ctx.close()


def test_tma_staged_many_tiles_per_cta(pkg):
    """32x16x16x16: 4096 rows, several per persistent CTA, so the double-buffered stages
    are reused; the result equals the one-RHS-per-thread kernel's bit for bit."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_TMA_STAGING

    dims = (32, 16, 16, 16)
    ctx, _, _ = _setup(pkg, dims, seed=35)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    psi = cuda(W.gaussian_fermion(dims, 36, nrhs=12)[:, 0].copy())
    outs = []
    for tma in (1, 2, 0):
        ctx.wcl_set_option(WCL_OPT_TMA_STAGING, tma)
        o = cuda(np.zeros(psi.shape, dtype=np.complex128))
        ctx.wcl_apply_Mpc(o, psi, "f32", nrhs=12)
        outs.append(host(o))
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[2])
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_shared_links_and_per_thread_kernels_agree(pkg, prec):
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_SHARED_LINKS

    dims = (8, 8, 8, 16)
    ctx, _, _ = _setup(pkg, dims, seed=19)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    psi = cuda(W.gaussian_fermion(dims, 20, nrhs=12)[:, 0].copy())
    outs = []
    for sl in (1, 0):
        ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, sl)
        o = cuda(np.zeros(psi.shape, dtype=np.complex128))
        ctx.wcl_apply_Mpc(o, psi, prec, nrhs=12)
        outs.append(host(o))
    # same arithmetic in the same order: identical up to FMA contraction differences
    assert relerr(outs[0], outs[1]) <= (1e-14 if prec == "f64" else 1e-6)
    ctx.close()


def test_autotuner_choice_and_cache_file(pkg, tmp_path, monkeypatch):
    """With the tuner on, the first apply of a configuration times the variants, writes the
    choice to WCL_TUNE_CACHE, and the result still matches the oracle."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("WCL_TUNE_CACHE", str(cache))
    dims = (6, 6, 4, 10)  # a shape no other test uses, so the choice is made here
    ctx, op, _ = _setup(pkg, dims, seed=21)
    psi = W.gaussian_fermion(dims, 22, nrhs=12)[:, 0].copy()
    out = cuda(np.zeros_like(psi))
    for _ in range(2):
        ctx.wcl_apply_Mpc(out, cuda(psi), "f32", nrhs=12)
    got = host(out)
    for k in range(12):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], False)) <= TOL["f32"], k
    ctx.close()
    lines = [l.split() for l in cache.read_text().splitlines() if "6x6x4x10" in l]
    assert len(lines) == 2, lines  # the two launches of M_hat, each tuned once
    for v, b, ms, *_ in lines:
        assert (int(v), int(b)) in {(0, 64), (0, 128), (0, 256), (0, 512), (1, 8), (1, 16), (1, 32), (3, 16),
                                    (4, 16), (5, 8), (5, 16), (5, 32), (6, 16), (7, 16), (8, 16), (9, 16),
                                    (10, 16)}
        assert float(ms) > 0


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 2, 8), 12), ((6, 6, 6, 8), 4), ((8, 4, 4, 6), 7)])
def test_apply_Mpc_multi_rhs_staged_spinors(pkg, dims, nrhs, dagger, prec):
    """Multi-RHS kernel whose neighbour spinors arrive through shared memory by cp.async."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_STAGED_SPINORS

    ctx, op, _ = _setup(pkg, dims, seed=23)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_STAGED_SPINORS, 1)
    psi = W.gaussian_fermion(dims, 24, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("blocked", [0, 1])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 2, 8), 12), ((6, 6, 6, 8), 4), ((8, 4, 4, 6), 7), ((32, 24, 24, 4), 5)])
def test_apply_Mpc_multi_rhs_prefetched_spinors(pkg, dims, nrhs, dagger, prec, blocked):
    """Multi-RHS kernel that loads the next hop's neighbour spinor into registers while it
    computes the current hop, in site order and in z-blocked tile order."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_BLOCKED_TILES, WCL_OPT_PREFETCH_SPINORS

    ctx, op, _ = _setup(pkg, dims, seed=31)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_PREFETCH_SPINORS, 1)
    ctx.wcl_set_option(WCL_OPT_BLOCKED_TILES, blocked)
    psi = W.gaussian_fermion(dims, 32, nrhs=nrhs)[:, 0].copy()
    psi[1] *= 1e-7
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "f16", "f64"])
def test_multi_rhs_blocked_tile_order(pkg, prec):
    """32x24x24x4: Ly * Lz > 512 tiles per time slice, so with blocked tiles the
    multi-RHS kernel walks its 16-site tiles in blocks of 12 z planes."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_AUTOTUNE, WCL_OPT_BLOCKED_TILES

    dims = (32, 24, 24, 4)
    ctx, op, _ = _setup(pkg, dims, seed=25)
    ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
    ctx.wcl_set_option(WCL_OPT_BLOCKED_TILES, 1)
    psi = W.gaussian_fermion(dims, 26, nrhs=5)[:, 0].copy()
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=5)
    got = host(out)
    for k in range(5):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], False)) <= TOL[prec], k
    ctx.close()
