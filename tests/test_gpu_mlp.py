"""The predictor network's device kernels against the FP64 oracle network:
forward outputs, loss, every parameter gradient and Adam steps; and that
training reduces the loss."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_07112_gb300 import _lib
    return _lib


@pytest.mark.parametrize("batch", [1, 37, 300])
def test_mlp_forward_and_gradients_match_oracle(lib, batch):
    import torch
    sizes = (12, 64, 64, 2)
    net = lib.MLP(sizes, seed=11)
    params = net.get_params().astype(np.float64)
    rng = np.random.default_rng(batch)
    X = rng.standard_normal((batch, 12)).astype(np.float32)
    T = rng.standard_normal((batch, 2)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    y = net.forward(Xd).cpu().numpy().astype(np.float64)
    y_ref, _ = M.forward(params, sizes, X.astype(np.float64))
    assert np.allclose(y, y_ref, rtol=1e-5, atol=1e-5)
    g, loss = net.gradients(Xd, Td)
    g_ref = M.gradients(params, sizes, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - M.loss(params, sizes, X.astype(np.float64), T.astype(np.float64))) <= 1e-5 * max(1.0, loss)
    scale = np.max(np.abs(g_ref)) + 1e-12
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale, np.max(np.abs(g - g_ref)) / scale
    net.close()


def test_mlp_adam_reduces_loss(lib):
    import torch
    sizes = (12, 64, 64, 2)
    net = lib.MLP(sizes, seed=3)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((512, 12)).astype(np.float32)
    W = rng.standard_normal((12, 2)).astype(np.float32)
    T = (np.tanh(X @ W)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    first = net.train_step(Xd, Td, 1e-3, want_loss=True)
    for _ in range(300):
        net.train_step(Xd, Td, 1e-3)
    last = net.train_step(Xd, Td, 1e-3, want_loss=True)
    assert last < 0.2 * first, (first, last)
    net.close()


def test_mlp_adam_steps_match_oracle(lib):
    """Five Adam steps with weight decay on one batch against the FP64
    oracle optimiser fed the oracle's own gradients."""
    import torch
    sizes = (12, 64, 64, 2)
    net = lib.MLP(sizes, seed=7)
    P = net.get_params().astype(np.float64)
    rng = np.random.default_rng(9)
    X = rng.standard_normal((64, 12)).astype(np.float32)
    T = rng.standard_normal((64, 2)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    opt = M.Adam(P.size)
    lr, wd, steps = 1e-3, 1e-2, 5
    firm = np.ones(P.size, dtype=bool)
    for _ in range(steps):
        net.train_step(Xd, Td, lr, weight_decay=wd)
        g = M.gradients(P, sizes, X.astype(np.float64), T.astype(np.float64))
        # Adam normalises each gradient entry, so an entry whose true value
        # is within FP32 rounding of zero may take either sign: compare
        # those only against the step bound
        firm &= np.abs(g) > 1e-3 * np.max(np.abs(g))
        P = opt.step(P, g, lr, wd)
    got = net.get_params().astype(np.float64)
    d = np.abs(got - P)
    assert firm.mean() > 0.5
    assert np.max(d[firm]) <= 0.02 * lr * steps, np.max(d[firm])
    assert np.max(d) <= 2.2 * lr * steps
    net.close()
