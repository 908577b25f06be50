"""GPU parity of the learned-warm-start network against the FP64 oracle.

Tolerances from the arithmetic: GEMM operands are BF16 and accumulate in
FP32, so a K-term dot product carries an accumulation error below
K * 2^-24 * sum|a b| (relative ~ K * 6e-8 for same-sign terms) -> rtol
4e-6 * sqrt(K) on outputs normalised by sum|a b| is generous; a BF16-rounded
output adds half an ulp, 2^-9.  Through several layers an FP32/FP64
difference can flip a BF16 rounding of an activation (relative 2^-8), so
network outputs and gradients are compared at 2e-2 relative (norm-wise).
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


@pytest.mark.parametrize("widths,batch", [([64, 32, 32, 24], 16), ([8192, 512, 512, 512, 6800], 64)])
def test_forward_and_gradients_match_oracle(GM, widths, batch):
    import torch
    net = _net(GM, widths, batch, 3)
    p = net.get_params().astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((batch, widths[0])) * 0.5
    t = rng.standard_normal((batch, widths[-1]))
    y = torch.zeros((batch, widths[-1]), dtype=torch.float32, device="cuda")
    net.forward(_f(x), y)
    torch.cuda.synchronize()
    yo, _ = M.forward(p, widths, x)
    err = np.linalg.norm(y.cpu().numpy() - yo) / np.linalg.norm(yo)
    assert err < 2e-2, err
    loss = net.backward(_f(x), _f(t))
    lo, go = M.loss_and_grads(p, widths, x, t)
    assert abs(loss - lo) <= 2e-2 * lo
    g = net.get_grads()
    o = 0
    for l in range(len(widths) - 1):
        n = widths[l] * widths[l + 1] + widths[l + 1]
        e = np.linalg.norm(g[o:o + n] - go[o:o + n]) / max(np.linalg.norm(go[o:o + n]), 1e-30)
        assert e < 2e-2, (l, e)
        o += n
    net.close()


def test_adam_step_matches_oracle(GM):
    widths = [16, 16, 8]
    net = _net(GM, widths, 8, 5)
    p0 = net.get_params().astype(np.float64)
    rng = np.random.default_rng(6)
    x, t = rng.standard_normal((8, 16)), rng.standard_normal((8, 8))
    net.backward(_f(x), _f(t))
    g = net.get_grads().astype(np.float64)
    net.adam_step(1e-2)
    p1 = net.get_params().astype(np.float64)
    po, _, _ = M.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-2)
    np.testing.assert_allclose(p1, po, rtol=1e-5, atol=1e-6)
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
