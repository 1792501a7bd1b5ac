"""GPU learned preconditioner: network forward and gradient against the FP64 oracle,
training on the GPU, and flexible GCR with the trained network against GCR without it."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, ptc
from oracle import lattice as L

from _gpu import built, cuda, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def identity_weights(noise, seed):
    """Channel 0 passes the field through every layer unchanged, plus small random weights."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout in zip(ptc.DEFAULT_CHANNELS[:-1], ptc.DEFAULT_CHANNELS[1:]):
        w = noise * (rng.standard_normal((cout, cin, 9, 4, 4)) + 1j * rng.standard_normal((cout, cin, 9, 4, 4)))
        w[0, 0, 0] += np.eye(4)
        out.append(w)
    return out


def bf16_round(w):
    """Round real and imaginary parts to bfloat16 (round to nearest even)."""
    def r(x):
        b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(w.real) + 1j * r(w.imag)


def even_embed(dims, half):
    full = np.zeros((2,) + half.shape, dtype=np.complex128)
    full[0] = half
    return L.from_qdp(full, dims)


def oracle_apply(U, ws, dims, r_half):
    out, _ = ptc.forward(U, ws, even_embed(dims, r_half))
    return L.to_qdp(out, dims)[0]


@pytest.mark.parametrize("bf16,split", [(False, None), (True, 3), (True, None)])
def test_forward_parity(pkg, bf16, split):
    """FP32 layers, BF16 layers with inputs split in three BF16 terms (the FP32 layer with
    BF16-rounded weights, to FP32 rounding) and the default BF16 layers (tcgen05, plain
    BF16 inputs: each layer's inputs within 2^-8 of their FP32 values) against the
    oracle's forward pass."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_SPLIT

    dims = (4, 4, 4, 8)
    gauge = W.gauge_links(dims, 0.5, 3)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ws = ptc.init_weights(seed=5, scale=0.3)
    ctx.wcl_precond_load(pkg.ptc_flatten(ws))
    if split is not None:
        ctx.wcl_set_option(WCL_OPT_PTC_SPLIT, split)
    r = W.gaussian_fermion(dims, 6)[0]
    out = cuda(np.zeros_like(r))
    ctx.wcl_precond_apply(out, cuda(r), 1, bf16=bf16)
    U = L.gauge_from_qdp(gauge, dims)
    if bf16 and split == 3:
        assert relerr(host(out), oracle_apply(U, [bf16_round(w) for w in ws], dims, r)) <= 1e-5
        assert relerr(host(out), oracle_apply(U, ws, dims, r)) <= 5e-3
    elif bf16:
        assert relerr(host(out), oracle_apply(U, [bf16_round(w) for w in ws], dims, r)) <= 2e-2
        assert relerr(host(out), oracle_apply(U, ws, dims, r)) <= 2e-2
    else:
        assert relerr(host(out), oracle_apply(U, ws, dims, r)) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 10)])
def test_tensor_core_layers_match_simt(pkg, dims):
    """BF16 network on the tensor cores (mma.sync, inputs split in three BF16 terms) equals
    the FP32 SIMT layers with the same BF16 weights to FP32 accuracy; 6x4x2x10 leaves a
    ragged last tile of sites."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_TENSOR_CORES

    gauge = W.gauge_links(dims, 0.5, 31)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ctx.wcl_precond_load(pkg.ptc_flatten(ptc.init_weights(seed=32, scale=0.3)))
    r = cuda(W.gaussian_fermion(dims, 33, nrhs=3)[:, 0].copy())
    outs = []
    for tc in (1, 0):
        ctx.wcl_set_option(WCL_OPT_PTC_TENSOR_CORES, tc)
        z = cuda(np.zeros(r.shape, dtype=np.complex128))
        ctx.wcl_precond_apply(z, r, 3, bf16=True)
        outs.append(host(z))
    assert relerr(outs[0], outs[1]) <= 1e-5  # the FP32 tolerance
    ctx.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 10), (8, 8, 8, 8)])
def test_tcgen05_layers_match_simt_and_mma_sync(pkg, dims):
    """BF16 network on the fifth-generation tensor cores (tcgen05: 128-site tiles on the
    MMA's M dimension, accumulators in tensor memory, inputs split in three BF16 terms)
    equals the FP32 SIMT layers with the same BF16 weights to FP32 accuracy, and the
    mma.sync layers; 6x4x2x10 (120 sites per parity) is one ragged tile, 8^4 sixteen
    tiles per parity and RHS."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_SPLIT, WCL_OPT_PTC_TENSOR_CORES

    gauge = W.gauge_links(dims, 0.5, 34)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ctx.wcl_precond_load(pkg.ptc_flatten(ptc.init_weights(seed=35, scale=0.3)))
    ctx.wcl_set_option(WCL_OPT_PTC_SPLIT, 3)
    r = cuda(W.gaussian_fermion(dims, 36, nrhs=3)[:, 0].copy())
    outs = {}
    for tc in (2, 1, 0):
        ctx.wcl_set_option(WCL_OPT_PTC_TENSOR_CORES, tc)
        z = cuda(np.zeros(r.shape, dtype=np.complex128))
        ctx.wcl_precond_apply(z, r, 3, bf16=True)
        outs[tc] = host(z)
    assert relerr(outs[2], outs[0]) <= 1e-5  # the FP32 tolerance
    assert relerr(outs[2], outs[1]) <= 1e-5
    for k in range(3):  # every RHS, not only the norm over all of them
        assert relerr(outs[2][k], outs[0][k]) <= 1e-5, k
    ctx.close()


@pytest.mark.parametrize("split,tol", [(2, 1e-4), (1, 2e-2)])
@pytest.mark.parametrize("dims", [(6, 4, 2, 10), (8, 8, 8, 8)])
def test_tcgen05_layers_fewer_input_terms(pkg, dims, split, tol):
    """Inputs split into `split` BF16 terms carry 8 * split significant bits: each input
    is within 2^-(8 split) of its FP32 value, so four layers stay within a few times that
    of the FP32 layers with the same BF16 weights (2^-16 = 1.5e-5, 2^-8 = 3.9e-3)."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_SPLIT, WCL_OPT_PTC_TENSOR_CORES

    gauge = W.gauge_links(dims, 0.5, 37)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ctx.wcl_precond_load(pkg.ptc_flatten(ptc.init_weights(seed=38, scale=0.3)))
    r = cuda(W.gaussian_fermion(dims, 39, nrhs=2)[:, 0].copy())
    outs = {}
    for tc in (2, 0):
        ctx.wcl_set_option(WCL_OPT_PTC_TENSOR_CORES, tc)
        ctx.wcl_set_option(WCL_OPT_PTC_SPLIT, split)
        z = cuda(np.zeros(r.shape, dtype=np.complex128))
        ctx.wcl_precond_apply(z, r, 2, bf16=True)
        outs[tc] = host(z)
    err = relerr(outs[2], outs[0])
    assert err <= tol, err
    assert err > 0.0  # the reduced split did change the arithmetic
    ctx.close()


def test_tcgen05_option_values(pkg):
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_TENSOR_CORES, WclError

    ctx = pkg.Context((4, 4, 4, 4))
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_SPLIT

    for v in (0, 1, 2):
        ctx.wcl_set_option(WCL_OPT_PTC_TENSOR_CORES, v)
    for v in (1, 2, 3):
        ctx.wcl_set_option(WCL_OPT_PTC_SPLIT, v)
    for opt, bad in ((WCL_OPT_PTC_TENSOR_CORES, 3), (WCL_OPT_PTC_SPLIT, 0), (WCL_OPT_PTC_SPLIT, 4)):
        with pytest.raises(WclError) as e:
            ctx.wcl_set_option(opt, bad)
        assert e.value.status == 1
    ctx.close()


def test_loss_and_gradient_parity(pkg):
    dims = (4, 4, 2, 4)
    gauge = W.gauge_links(dims, 0.5, 7)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ws = ptc.init_weights(seed=8, scale=0.25)
    ctx.wcl_precond_load(pkg.ptc_flatten(ws))
    rs = W.gaussian_fermion(dims, 9, nrhs=3)[:, 0]
    es = W.gaussian_fermion(dims, 10, nrhs=3)[:, 0]
    loss, grad = ctx.wcl_precond_loss_grad(cuda(rs), cuda(es), 3)
    U = L.gauge_from_qdp(gauge, dims)
    even = L.parity_mask(dims, 0)
    l_ref, g_ref = ptc.loss_and_grad(U, ws, [even_embed(dims, r) for r in rs], [even_embed(dims, e) for e in es],
                                     mask=even)
    assert abs(loss - l_ref) <= 1e-6 * l_ref
    assert relerr(grad, pkg.ptc_flatten(g_ref)) <= 1e-5
    ctx.close()


def test_adam_steps_match_oracle(pkg):
    """Two training steps on the GPU (its own forward, backward and Adam kernels) against
    the oracle's loss_and_grad + adam_step in FP64: the weight change of each step agrees
    to the FP32 tolerance.  Weights start FP32-exact so that both sides start equal; the
    learning rate is large enough that FP32 rounding of the weights themselves is far
    below the tolerance."""
    dims = (4, 4, 2, 4)
    gauge = W.gauge_links(dims, 0.5, 71)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), 0.1235, 1.0)
    ws = [w.astype(np.complex64).astype(np.complex128) for w in ptc.init_weights(seed=72, scale=0.25)]
    ctx.wcl_precond_load(pkg.ptc_flatten(ws))
    rs = W.gaussian_fermion(dims, 73, nrhs=4)[:, 0]
    es = W.gaussian_fermion(dims, 74, nrhs=4)[:, 0]
    U = L.gauge_from_qdp(gauge, dims)
    even = L.parity_mask(dims, 0)
    lr = 0.05
    state = {}
    prev = pkg.ptc_flatten(ws)
    for step, k in enumerate((0, 2)):
        ctx.wcl_precond_train(cuda(rs[k:k + 2]), cuda(es[k:k + 2]), 2,
                              pkg.wcl_default_train_params(epochs=1, batch=2, lr=lr))
        got = ctx.wcl_precond_get()
        _, g = ptc.loss_and_grad(U, ws, [even_embed(dims, r) for r in rs[k:k + 2]],
                                 [even_embed(dims, e) for e in es[k:k + 2]], mask=even)
        ws = ptc.adam_step(ws, g, state, lr=lr)
        ref = pkg.ptc_flatten(ws)
        assert relerr(got - prev, ref - prev) <= 1e-5, step
        ws = pkg.ptc_unflatten(got)  # continue from the GPU's weights
        prev = got
    ctx.close()


def _pairs(ctx, dims, n, seed):
    """Training pairs (r, e) = (M_hat e, e), e Gaussian on the even sites; r from the GPU operator."""
    import torch

    es = cuda(W.gaussian_fermion(dims, seed, nrhs=n)[:, 0].copy())
    rs = torch.empty_like(es)
    ctx.wcl_apply_Mpc(rs, es, "f64", nrhs=n)
    return rs, es


def test_training_reduces_loss(pkg):
    dims = (4, 4, 4, 8)
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(W.gauge_links(dims, 0.3, 11)), 0.1235, 1.0)
    ctx.wcl_precond_load(pkg.ptc_flatten(identity_weights(1e-3, 12)))
    rs, es = _pairs(ctx, dims, 16, 13)
    l0, _ = ctx.wcl_precond_loss_grad(rs, es, 16)
    losses = ctx.wcl_precond_train(rs, es, 16, pkg.wcl_default_train_params(epochs=20, batch=4, lr=3e-3))
    l1, _ = ctx.wcl_precond_loss_grad(rs, es, 16)
    assert losses[-1] < losses[0] and l1 < 0.7 * l0, (l0, l1, losses)
    ctx.close()


@pytest.mark.parametrize("tc,split", [(1, 3), (2, 3), (2, 1)])
def test_learned_fgcr_gains_over_gcr(pkg, tc, split):
    """The trained network lets flexible GCR reach 1e-10 in fewer iterations than GCR alone,
    with the network's BF16 layers on mma.sync (1) or on tcgen05 (2), the latter also with
    plain BF16 inputs (split 1)."""
    from paper_2411_08461_gb300.wcl import WCL_OPT_PTC_SPLIT, WCL_OPT_PTC_TENSOR_CORES

    train_dims, dims = (4, 4, 4, 8), (8, 8, 8, 16)
    kappa = 0.1235
    tctx = pkg.Context(train_dims)
    tctx.wcl_load_gauge(cuda(W.gauge_links(train_dims, 0.3, 21)), kappa, 1.0)
    tctx.wcl_precond_load(pkg.ptc_flatten(identity_weights(1e-3, 22)))
    rs, es = _pairs(tctx, train_dims, 32, 23)
    tctx.wcl_precond_train(rs, es, 32, pkg.wcl_default_train_params(epochs=30, batch=8, lr=3e-3))
    weights = tctx.wcl_precond_get()
    tctx.close()

    gauge = W.gauge_links(dims, 0.3, 24)  # a fresh configuration: the weights are gauge independent
    ctx = pkg.Context(dims)
    ctx.wcl_load_gauge(cuda(gauge), kappa, 1.0)
    ctx.wcl_precond_load(weights)
    ctx.wcl_set_option(WCL_OPT_PTC_TENSOR_CORES, tc)
    ctx.wcl_set_option(WCL_OPT_PTC_SPLIT, split)
    b = W.gaussian_fermion(dims, 25)
    op = dirac.from_qdp_problem(gauge, dims, kappa, 1.0)
    iters = {}
    for solver in ("gcr", "fgcr_learned"):
        x = cuda(np.zeros_like(b))
        _, info = ctx.wcl_invert(x, cuda(b), 1, pkg.wcl_default_params(solver=solver, sloppy="f32", tol=1e-10,
                                                                     gcr_nkrylov=20, delta_reliable=1e-3))
        tr = op.true_residual(L.from_qdp(host(x), dims), L.from_qdp(b, dims))
        assert tr <= 1e-10, (solver, tr, info)
        iters[solver] = info[0]["iters"]
    assert iters["fgcr_learned"] < iters["gcr"], iters
    ctx.close()
