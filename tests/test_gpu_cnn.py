"""Tensor-core convolution network kernels against the NumPy oracle (which
rounds to bfloat16 exactly where the kernels store bfloat16), training, and
the learned correction inside FGMRES."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import cnn as ocnn
from oracle.solver import Solver, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10232_gb300 import _ffi  # noqa: E402
from paper_2010_10232_gb300.learned import Net  # noqa: E402
from paper_2010_10232_gb300.solver import from_problem  # noqa: E402


def _batch(B, H, Wd, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((B, H, Wd, 16))
    x[..., :3] = rng.standard_normal((B, H, Wd, 3))
    t = rng.standard_normal((B, H, Wd, 2))
    return x, t


def _to_dev(x, t):
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    tt = torch.from_numpy(t.astype(np.float32)).cuda().contiguous()
    return xb, tt


@pytest.mark.parametrize("B,H,Wd", [(2, 12, 20), (1, 37, 33)])
def test_forward_matches_oracle(B, H, Wd):
    net = Net(seed=7)
    theta = net.get_params()
    params = ocnn.unflatten(theta.astype(np.float64))
    x, t = _batch(B, H, Wd, 1)
    xb, _ = _to_dev(x, t)
    y = net.forward(xb).cpu().numpy()
    ref, _ = ocnn.forward(params, ocnn.bf16_round(x)[..., :3], bf16=True)
    assert rel_err(y, ref) <= 3e-3


def test_gradient_matches_oracle():
    net = Net(seed=11)
    theta = net.get_params()
    params = ocnn.unflatten(theta.astype(np.float64))
    x, t = _batch(2, 10, 24, 2)
    xb, tt = _to_dev(x, t)
    g, loss = net.grad(xb, tt)
    lo, go = ocnn.loss_and_grad(params, ocnn.bf16_round(x)[..., :3], t.astype(np.float32).astype(np.float64), bf16=True)
    assert abs(loss - lo) <= 1e-3 * abs(lo)
    gref = ocnn.flatten(go)
    # per layer (weights and biases separately)
    k = 0
    for ws, bs in ocnn.param_shapes():
        for shp in (ws, bs):
            nn_ = int(np.prod(shp))
            assert rel_err(g[k:k + nn_], gref[k:k + nn_]) <= 2e-2, shp
            k += nn_


def test_training_reduces_loss():
    net = Net(seed=3)
    x, _ = _batch(8, 16, 16, 5)
    # a learnable target: a fixed random linear 3x3 map of the input channels
    rng = np.random.default_rng(9)
    Wt = rng.standard_normal((2, 3, 3, 3)) * 0.3
    t = ocnn.conv3x3(ocnn.bf16_round(x)[..., :3], Wt, np.zeros(2))
    xb, tt = _to_dev(x, t)
    l0 = net.train_step(xb, tt, lr=3e-3)
    for _ in range(150):
        l1 = net.train_step(xb, tt, lr=3e-3)
    assert l1 < 0.2 * l0, (l0, l1)


def test_params_roundtrip_and_checkpoint(tmp_path):
    net = Net(seed=1)
    th = net.get_params()
    net2 = Net(seed=2)
    assert not np.array_equal(th, net2.get_params())
    p = tmp_path / "w.npy"
    net.save(str(p))
    net2.load(str(p))
    np.testing.assert_array_equal(net2.get_params(), th)
    assert th.size == ocnn.num_params()


def test_learned_fgmres_converges_and_falls_back():
    pr = W.small_2d(n_el=48, p=3, k=30.0)
    s = Solver(pr)
    f = s.load()
    ud = s.direct(f)
    h = from_problem(pr, precision=1)
    x0, it0, *_ = h.solve(torch.from_numpy(f).cuda(), tol=1e-9)
    net = Net(seed=5)
    h.attach(net, gamma=1e-3)
    x1, it1, hist, tr, st = h.solve(torch.from_numpy(f).cuda(), tol=1e-9)
    assert st == 0 and rel_err(x1.cpu().numpy(), ud) <= 1e-6
    # a network that outputs NaN is ignored (plain V-cycle fallback)
    bad = np.full(net.num_params, np.nan, dtype=np.float32)
    net.set_params(bad)
    x2, it2, *_ = h.solve(torch.from_numpy(f).cuda(), tol=1e-9)
    assert it2 == it0 and rel_err(x2.cpu().numpy(), x0.cpu().numpy()) <= 1e-12
    h.attach(None)
