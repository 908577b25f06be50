"""GPU parity of the learned-warm-start network against the FP64 oracle.

Tolerances from the arithmetic: GEMM operands are BF16 and accumulate in
FP32, so a K-term dot product carries an accumulation error below
K * 2^-24 * sum|a b| (relative ~ K * 6e-8 for same-sign terms) -> rtol
4e-6 * sqrt(K) on outputs normalised by sum|a b| is generous; a BF16-rounded
output adds half an ulp, 2^-9.  Through several layers an FP32/FP64
difference can flip a BF16 rounding of an activation (relative 2^-8): network
outputs and every layer's dW, db are compared element by element against a
bound propagated layer by layer from that arithmetic (_elementwise_bounds).
"""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def GM():
    from paper_2004_02484_gb300 import build as b
    b.build()
    import torch
    torch.cuda.set_device(0)
    from paper_2004_02484_gb300 import mlp as GM
    return GM


def _bf(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda().to(torch.bfloat16).contiguous()


def _f(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("M_,N_,K_", [(1, 8, 8), (1, 512, 8192), (5, 6800, 512), (8, 13, 24),
                                      (9, 130, 72), (37, 130, 72), (128, 128, 32),
                                      (256, 512, 8192), (300, 6800, 512), (512, 64, 4096)])
@pytest.mark.parametrize("gelu", [False, True])
def test_gemm_matches_oracle(GM, M_, N_, K_, gelu):
    import torch
    rng = np.random.default_rng(M_ + N_ + K_)
    A = M.bf16(rng.standard_normal((M_, K_)))
    B = M.bf16(rng.standard_normal((N_, K_)))
    bias = rng.standard_normal(N_).astype(np.float32).astype(np.float64)
    C = torch.zeros((M_, N_), dtype=torch.float32, device="cuda")
    Cb = torch.zeros((M_, N_), dtype=torch.bfloat16, device="cuda")
    GM.nmpc_gemm_bf16(_bf(A), _bf(B), C=C, Cb=Cb, bias=_f(bias), gelu=gelu)
    torch.cuda.synchronize()
    ref = A @ B.T + bias
    scale = np.abs(A) @ np.abs(B).T + np.abs(bias)
    if gelu:
        ref = M.gelu(ref)
        scale = scale  # GELU is 1.13-Lipschitz
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 4e-6 * np.sqrt(K_) * scale + 1e-6)
    gotb = Cb.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gotb - ref) <= 4e-6 * np.sqrt(K_) * scale + np.abs(ref) * 2.0 ** -8 + 1e-6)


def _net(GM, widths, batch, seed):
    return GM.MLP(widths, batch, seed)


U8 = 2.0 ** -8   # BF16 unit roundoff (8 significand bits kept)


def _gamma(K):
    """FP32 accumulation of K products, relative to sum |a b| (a generous
    sqrt(K) multiple of the unit roundoff 2^-24)."""
    return 4e-6 * np.sqrt(K) + 2.0 ** -23


def _elementwise_bounds(p, widths, x, t):
    """Element-wise bounds on |GPU - oracle| for the output y and every
    layer's dW, db, propagated from the arithmetic with the oracle's own
    values: each BF16 copy (activation, dz) may round to the neighbouring
    BF16 value (one ulp, 2^-8 relative) on top of the difference it carries;
    GELU is 1.13-Lipschitz and |GELU''| <= 0.8; FP32 sums add _gamma(K)
    times the sum of absolute products."""
    Ws, bs = M.unpack(p, widths)
    Wb = [np.abs(M.bf16(W)) for W in Ws]
    y, (a, zs) = M.forward(p, widths, x)
    L = len(Ws)
    # forward: dz[l] bounds |z_l(gpu) - z_l(oracle)|
    da = np.zeros_like(a[0])
    dzs = []
    for l in range(L):
        S = np.abs(a[l]) @ Wb[l].T + np.abs(bs[l])
        dz = da @ Wb[l].T + _gamma(widths[l]) * S
        dzs.append(dz)
        if l < L - 1:
            da = 1.13 * dz + U8 * np.abs(a[l + 1])
    n = y.size
    # backward: g is dL/dz of the current layer, e its error bound
    g = 2.0 * (y - t) / n
    e = 2.0 * dzs[-1] / n
    bW, bb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        B = x.shape[0]
        e16 = e + U8 * np.abs(g)            # the BF16 copy of dz
        # the layer input: the network input is rounded to BF16 identically on
        # both sides; a hidden activation carries the forward bound
        ea = (U8 * np.abs(a[l]) + 1.13 * dzs[l - 1]) if l > 0 else np.zeros_like(a[0])
        bW[l] = (e16.T @ np.abs(a[l]) + np.abs(g).T @ ea +
                 _gamma(B) * (np.abs(g).T @ np.abs(a[l])))
        bb[l] = e.sum(axis=0) + _gamma(B) * np.abs(g).sum(axis=0)
        if l > 0:
            dA = np.abs(M.bf16(g)) @ Wb[l]
            eA = e16 @ Wb[l] + _gamma(widths[l + 1]) * (np.abs(g) @ Wb[l])
            gp = M.gelu_grad(zs[l - 1])
            e = eA * np.abs(gp) + dA * 0.8 * dzs[l - 1]
            g = (M.bf16(g) @ M.bf16(Ws[l])) * gp
    return y, dzs[-1], bW, bb


@pytest.mark.parametrize("widths,batch", [([64, 32, 32, 24], 16), ([8192, 512, 512, 512, 6800], 64),
                                          ([2048, 512, 512, 512, 1600], 64)])
def test_forward_and_gradients_match_oracle_elementwise(GM, widths, batch):
    import torch
    net = _net(GM, widths, batch, 3)
    p = net.get_params().astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((batch, widths[0])) * 0.5
    t = rng.standard_normal((batch, widths[-1]))
    y = torch.zeros((batch, widths[-1]), dtype=torch.float32, device="cuda")
    net.forward(_f(x), y)
    torch.cuda.synchronize()
    yo, by, bW, bb = _elementwise_bounds(p, widths, x, t)
    dy = np.abs(y.cpu().numpy() - yo)
    assert np.all(dy <= 2.0 * by + 1e-6), float((dy / (2.0 * by + 1e-6)).max())
    loss = net.backward(_f(x), _f(t))
    lo, go = M.loss_and_grads(p, widths, x, t)
    assert abs(loss - lo) <= 5e-3 * lo
    g = net.get_grads().astype(np.float64)
    o = 0
    for l in range(len(widths) - 1):
        nW, nb = widths[l] * widths[l + 1], widths[l + 1]
        gW, gb = g[o:o + nW].reshape(widths[l + 1], widths[l]), g[o + nW:o + nW + nb]
        oW, ob = go[o:o + nW].reshape(widths[l + 1], widths[l]), go[o + nW:o + nW + nb]
        rW = np.abs(gW - oW) / (2.0 * bW[l] + 1e-9)
        rb = np.abs(gb - ob) / (2.0 * bb[l] + 1e-9)
        assert rW.max() <= 1.0, (l, float(rW.max()))
        assert rb.max() <= 1.0, (l, float(rb.max()))
        o += nW + nb
    net.close()


def test_elementwise_bound_catches_a_single_wrong_column(GM):
    """The bound is tight enough to see one wrong output column: the oracle
    output with column 5 shifted by 10% of its scale fails it."""
    widths, batch = [64, 32, 32, 24], 16
    net = _net(GM, widths, batch, 3)
    p = net.get_params().astype(np.float64)
    net.close()
    rng = np.random.default_rng(4)
    x = rng.standard_normal((batch, widths[0])) * 0.5
    t = rng.standard_normal((batch, widths[-1]))
    yo, by, _, _ = _elementwise_bounds(p, widths, x, t)
    bad = yo.copy()
    bad[:, 5] += 0.1 * np.abs(yo).max()
    assert not np.all(np.abs(bad - yo) <= 2.0 * by + 1e-6)


def test_adam_four_steps_match_oracle(GM):
    """Adam on given (seeded) gradients, four steps with different gradients:
    the moments, beta1, beta2 and both bias corrections all enter."""
    widths = [16, 16, 8]
    net = _net(GM, widths, 8, 5)
    p = net.get_params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    rng = np.random.default_rng(6)
    for step in range(1, 5):
        g = (rng.standard_normal(p.size) * (0.1 + step)).astype(np.float32)
        net.set_grads(g)
        net.adam_step(1e-2)
        p, m, v = M.adam_step(p, g.astype(np.float64), m, v, step, 1e-2)
        got = net.get_params().astype(np.float64)
        # float32 master weights and moments, and float32 constants: beta2 =
        # 0.999 is off by ~1e-8 in float32 while c2 = 1 - beta2^t ~ 1e-3 t, so
        # c2 carries up to ~1e-5 relative error and each step up to lr * 1e-5;
        # a wrong beta or a missing bias correction moves a step by percents
        np.testing.assert_allclose(got, p, rtol=2e-6, atol=step * 1e-2 * 1e-5 + 1e-8)
    net.close()


def test_training_reduces_the_loss(GM):
    """A smooth regression target: 300 Adam steps cut the loss by 20x."""
    widths = [32, 64, 64, 16]
    net = _net(GM, widths, 128, 7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((128, 32))
    Wt = rng.standard_normal((16, 32)) / np.sqrt(32)
    t = np.tanh(x @ Wt.T)
    xd, td = _f(x), _f(t)
    first = net.train_step(xd, td, 3e-3)
    for _ in range(300):
        last = net.train_step(xd, td, 3e-3, want_loss=False)
    last = net.backward(xd, td)
    assert last < first / 20, (first, last)
    net.close()


@pytest.mark.parametrize("M_,N_,K_", [(9, 130, 72), (128, 128, 64), (200, 384, 1024),
                                      (64, 512, 8192), (300, 6800, 512), (4096, 64, 4096)])
def test_tcgen05_gemm_matches_the_mma_sync_gemm_and_the_oracle(GM, M_, N_, K_):
    """The tensor-core path (tcgen05, TMA tiles, TMEM accumulator) and the
    mma.sync path against the float64 product of the BF16 operands, element
    by element at the FP32-accumulation bound; no bounded wait gave up."""
    import torch
    rng = np.random.default_rng(M_ * 7 + N_ + K_)
    A = M.bf16(rng.standard_normal((M_, K_)))
    B = M.bf16(rng.standard_normal((N_, K_)))
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    GM.nmpc_gemm_error(clear=True)
    outs = []
    for path in (0, 1):
        GM.nmpc_gemm_set_path(path)
        C = torch.full((M_, N_), np.nan, dtype=torch.float32, device="cuda")
        GM.nmpc_gemm_bf16(_bf(A), _bf(B), C=C)
        torch.cuda.synchronize()
        outs.append(C.cpu().numpy().astype(np.float64))
    GM.nmpc_gemm_set_path(0)
    assert GM.nmpc_gemm_error(clear=True) == 0
    for got in outs:
        assert np.all(np.abs(got - ref) <= 4e-6 * np.sqrt(K_) * scale + 1e-6)


def test_tcgen05_split_k_inside_the_network_and_no_wait_gave_up(GM):
    """A first layer of 8192 inputs and 64 rows runs as a split-K launch
    (4 tiles, 128 K blocks): the network's output with the tensor-core path
    equals the one with the mma.sync path to the FP32 accumulation bound."""
    import torch
    widths, batch = [8192, 512, 512, 512, 1600], 64
    rng = np.random.default_rng(11)
    x = _f(rng.standard_normal((batch, widths[0])) * 0.5)
    ys = []
    for path in (0, 1):
        GM.nmpc_gemm_set_path(path)
        net = _net(GM, widths, batch, 3)
        y = torch.zeros((batch, widths[-1]), dtype=torch.float32, device="cuda")
        net.forward(x, y)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy().astype(np.float64))
        net.close()
    GM.nmpc_gemm_set_path(0)
    assert GM.nmpc_gemm_error(clear=True) == 0
    p = _net(GM, widths, batch, 3).get_params().astype(np.float64)
    yo, by, _, _ = _elementwise_bounds(p, widths, x.cpu().numpy().astype(np.float64),
                                       np.zeros((batch, widths[-1])))
    for y in ys:
        assert np.all(np.abs(y - yo) <= 2.0 * by + 1e-6)
