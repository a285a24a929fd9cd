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


@pytest.mark.parametrize("B,H,Wd", [(2, 12, 20), (1, 37, 33), (4, 128, 200)])
def test_forward_matches_oracle(B, H, Wd):
    """Forward pass of the tensor-core (tcgen05) convolutions: ragged 8 x 16
    tiles, and more tiles than resident blocks (the persistent tile loop)."""
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
    # per layer (weights and biases separately): FP32 accumulation against the
    # oracle's FP64 with the same bf16 roundings of the stored tensors
    k = 0
    for ws, bs in ocnn.param_shapes():
        for shp in (ws, bs):
            nn_ = int(np.prod(shp))
            e = rel_err(g[k:k + nn_], gref[k:k + nn_])
            print(f"gradient {shp}: rel err {e:.2e}")
            assert e <= 5e-3, shp
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


@pytest.mark.parametrize("k,n_el", [(80.0, 128), (150.0, 240)])
def test_trained_network_saves_iterations(k, n_el):
    """What the shipped network (weights/cslp_correction.npz, trained on
    residual/error pairs of the FP32 V-cycle at k ~ U[50, 400]) gains: on
    problems it was not trained on (these meshes and wave numbers, centre
    source), FGMRES with the learned correction needs at least two
    iterations fewer than the same FP32-V-cycle FGMRES without it, and
    reaches the same solution.  Wall times of both are printed."""
    import os
    wpath = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2010_10232_gb300", "weights",
                         "cslp_correction.npz")
    d = np.load(wpath)
    net = Net(seed=0)
    net.set_params(d["params"])
    pr = W.Problem(dim=2, p=3, n_el=n_el, kfield=W.constant_k(k), sources=[(0.5, 0.5)])
    h = from_problem(pr, precision=1)
    f = h.point_source(0.5, 0.5)

    def timed():
        x, it, hist, tr, st = h.solve(f, tol=1e-7)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        x, it, hist, tr, st = h.solve(f, tol=1e-7)
        b.record()
        torch.cuda.synchronize()
        return x.cpu().numpy(), it, st, a.elapsed_time(b)

    x0, it0, st0, ms0 = timed()
    h.attach(net, float(d["gamma"]))
    x1, it1, st1, ms1 = timed()
    h.attach(None)
    print(f"k={k} n_el={n_el}: iterations {it0} -> {it1} with the network; ms {ms0:.2f} -> {ms1:.2f}")
    assert st0 == 0 and st1 == 0
    assert it1 <= it0 - 2
    assert rel_err(x1, x0) <= 1e-5
