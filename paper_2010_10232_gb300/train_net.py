"""Train the learned V-cycle correction on residual/error pairs generated by the
solver itself, then measure what it gains inside FGMRES.

    python -m paper_2010_10232_gb300.train_net [--instances 80] [--steps 3000] [--out weights.npz]

Data: for instances with k ~ U[50, 400] (seeded), p = 3 and kh ~ 0.625, the
preconditioner inputs v that FGMRES produces (P A M~^{-1} power sequence from a
point source) give pairs by the V-cycle's error propagation, e = (I - V M_beta) V(v),
r~ = M_beta e (exact: e = M_beta^{-1} r~); random 64 x 64 crops of (r~ / s, e / (s gamma)) form the set
(instances x 8 vectors x 16 crops, about 10^4 samples).  Training: Adam on
the relative L2 loss.  Evaluation: FGMRES iterations and time to 1e-7 with
and without the network on unseen wave numbers.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from .learned import Net, make_pairs, preconditioner_inputs, target_scale
from .solver import Helmholtz


def n_el_for(k: float) -> int:
    return int(min(640, max(48, 16 * round(k / (0.625 * 16)))))


def build_dataset(n_inst: int, seed: int, crop: int = 64, vecs: int = 8, crops: int = 16, log=print):
    rng = np.random.default_rng(seed)
    Xs, Ts = [], []
    gamma = None
    t0 = time.time()
    for i in range(n_inst):
        k = float(rng.uniform(50.0, 400.0))
        h = Helmholtz(dim=2, p=3, n_el=n_el_for(k), kfield=k, precision=1)
        f = h.point_source(*rng.uniform(0.1, 0.9, 2))
        vs = preconditioner_inputs(h, f, vecs)
        if gamma is None:
            gamma = target_scale(h, vs[1], 1)
        X, T = make_pairs(h, vs, crops, crop, gamma, 1, rng)
        Xs.append(X)
        Ts.append(T)
        h.close()
        if (i + 1) % 10 == 0:
            log(f"  data: {i + 1}/{n_inst} instances, {time.time() - t0:.1f} s")
    return torch.cat(Xs), torch.cat(Ts), gamma


def train(net: Net, X, T, steps: int, batch: int = 32, lr: float = 1e-3, seed: int = 0, log=print):
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    hist = []
    t0 = time.time()
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).cuda()
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        cur = lr * (0.1 ** (s / max(1, steps)))           # exponential decay to lr/10
        loss = net.train_step(xb, tb, lr=cur)
        if s % 100 == 0 or s == steps - 1:
            hist.append((s, loss))
            log(f"  step {s}: loss {loss:.4f} ({time.time() - t0:.1f} s)")
    return hist


def evaluate(net: Net, gamma: float, ks=(75.0, 150.0, 275.0), p: int = 3, log=print):
    out = []
    for k in ks:
        h = Helmholtz(dim=2, p=p, n_el=n_el_for(k), kfield=k, precision=1)
        f = h.point_source(0.5, 0.5)
        res = {}
        for name, attach in (("plain", False), ("learned", True)):
            h.attach(net if attach else None, gamma)
            x, it, hist, tr, st = h.solve(f, tol=1e-7)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                h.solve(f, x=x)
            torch.cuda.synchronize()
            res[name] = {"iters": it, "ms": (time.perf_counter() - t0) / 3 * 1e3, "true_res": tr, "status": st}
        h.attach(None)
        out.append({"k": k, "n_el": n_el_for(k), **res})
        log(f"  k={k}: plain {res['plain']['iters']} its {res['plain']['ms']:.2f} ms, "
            f"learned {res['learned']['iters']} its {res['learned']['ms']:.2f} ms")
        h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=80)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", default="")
    ap.add_argument("--report", default="")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    X, T, gamma = build_dataset(args.instances, args.seed)
    print(f"dataset: {X.shape[0]} samples of {X.shape[1]}x{X.shape[2]}, gamma {gamma:.4g}, {time.time() - t0:.1f} s")
    net = Net(seed=args.seed)
    hist = train(net, X, T, args.steps)
    ev = evaluate(net, gamma)
    if args.out:
        np.savez(args.out, params=net.get_params(), gamma=gamma)
    rep = {"samples": int(X.shape[0]), "gamma": gamma, "loss_history": hist, "evaluation": ev,
           "seconds": time.time() - t0}
    if args.report:
        json.dump(rep, open(args.report, "w"), indent=1)
    print(json.dumps(rep["evaluation"]))


if __name__ == "__main__":
    main()
