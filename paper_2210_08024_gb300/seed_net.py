"""Training data, training loop and export of the seed network.

The network (include/tc_mlp.h) predicts the root of one backward-Euler step of length
dt, as changes from the cell's state, from its state, fields and dt.  The seeded step
modes start each substep's Newton iteration from that prediction and still iterate to
the solver's own tolerance, so the prediction only shortens the iteration.

Training data: cells drawn like the 128^3 slab (synthgen.training_samples: lognormal
density, two-phase temperatures, six-ray fields) with Z' log-uniform in [0.1, 3] and
step lengths log-uniform in [1e-6, 1] x 1e4 yr, wide enough to cover the substeps that
the 0.1 limiter produces.  Labels come from the library's plain FP64 solver
(TC_MODE_NEWTON_FP64, checked against the CPU oracle by the parity tests) run with the
substep limiter switched off, so each label is a single backward-Euler root.  Each
sample's step length is one of `nbins` log-spaced values so that a bin is one tc_step.
Training: Adam on mini-batches with the library's forward/backward kernels
(tc_mlp_train_step); everything numerical runs on the GPU in those kernels.

    python -m paper_2210_08024_gb300.seed_net --samples 4000000 --epochs 6 --out seed.bin
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthgen  # noqa: E402

from . import tc  # noqa: E402

DEFAULT_BLOB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "seed_slab.bin")


def features(cells: dict, T, xH2, xHp, dt) -> np.ndarray:
    """Raw (unnormalised) features in the order of include/tc_mlp.h, float32 [N, 10]."""
    n = np.asarray(cells["n"], dtype=np.float64)
    N = n.size
    bc = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (N,))  # noqa: E731
    chi_fuv = (1.8e-4 * bc(cells["chi_pe"]) + 3.0e-5 * bc(cells["chi_lw"])) / 2.1e-4
    X = np.empty((N, 10), dtype=np.float32)
    X[:, 0] = np.log10(n)
    X[:, 1] = np.log10(bc(T))
    X[:, 2] = bc(xH2)
    X[:, 3] = bc(xHp)
    X[:, 4] = np.log10(np.maximum(chi_fuv, 1e-30))
    X[:, 5] = np.log10(np.maximum(bc(cells["f_h2"]), 1e-30))
    X[:, 6] = np.log10(bc(cells["F_lyc"]) + 1.0)
    X[:, 7] = np.log10(np.maximum(bc(cells["xi"]), 1e-30))
    X[:, 8] = np.log10(bc(dt))
    X[:, 9] = np.log10(np.maximum(bc(cells["Zd"]), 1e-30))
    return X


def targets(T0, xH2_0, xHp_0, xe0, T1, xH2_1, xHp_1, xe1) -> np.ndarray:
    """Changes over one backward-Euler step, float32 [N, 3]: (x_H2' - x_H2)/0.5,
    x_H+' - x_H+ and log10 T' - log10 T, where T' = mu_0 T_mu' is the root's temperature
    at the step's start mu (the frozen mu of the residual).  The solver returns
    T1 = mu_1 T_mu', so T' = T1 mu_0 / mu_1 with mu = mu_H / (1.1 + x_e - x_H2)."""
    ratio = (1.1 + np.asarray(xe1) - np.asarray(xH2_1)) / (1.1 + np.asarray(xe0) - np.asarray(xH2_0))
    Y = np.empty((np.size(T0), 3), dtype=np.float32)
    Y[:, 0] = (np.asarray(xH2_1) - np.asarray(xH2_0)) / 0.5
    Y[:, 1] = np.asarray(xHp_1) - np.asarray(xHp_0)
    Y[:, 2] = np.log10(np.asarray(T1) * ratio) - np.log10(np.asarray(T0))
    return Y


def make_dataset(n: int, key: int = 4, nbins: int = 48, dt_range=(1e-6, 1.0), log=print):
    """Returns (X, Y, cells, dt).  Labels: one backward-Euler step of length dt per sample
    (the substep rule switched off by a huge limiter), solved by the library's plain FP64
    Newton; samples whose solve needed a halved substep are dropped."""
    import torch
    cells = synthgen.training_samples(n, key)
    cells.pop("dt")
    g = np.random.default_rng(key + 1)
    lo, hi = math.log10(synthgen.DT_1E4YR * dt_range[0]), math.log10(synthgen.DT_1E4YR * dt_range[1])
    edges = np.linspace(lo, hi, nbins + 1)
    b = g.integers(0, nbins, n)
    centers = 10.0 ** (0.5 * (edges[:-1] + edges[1:]))
    dt = centers[b]
    st0 = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    st1 = tc.Stepper(tc.TC_MODE_NEWTON_FP64, limiter=1e30)
    out = {k: np.empty(n) for k in ("xe0", "T1", "x21", "xp1", "xe1")}
    nsub = np.empty(n, dtype=np.int32)
    t0 = time.time()
    for k in range(nbins):
        idx = np.nonzero(b == k)[0]
        if idx.size == 0:
            continue
        sub = synthgen.subset(cells, idx)
        d = tc.to_device(sub)
        st0.step(d, 0.0)                 # dt = 0: the initial C/O/e equilibrium only
        torch.cuda.synchronize()
        out["xe0"][idx] = d["xe"].cpu().numpy()
        d = tc.to_device(sub)
        st1.step(d, float(centers[k]))
        torch.cuda.synchronize()
        out["T1"][idx] = d["T"].cpu().numpy()
        out["x21"][idx] = d["xH2"].cpu().numpy()
        out["xp1"][idx] = d["xHp"].cpu().numpy()
        out["xe1"][idx] = d["xe"].cpu().numpy()
        nsub[idx] = d["nsub"].cpu().numpy()
    st0.close()
    st1.close()
    log("labels for %d samples in %.1f s (%d needed more than one substep)" % (n, time.time() - t0,
                                                                           int(np.sum(nsub != 1))))
    X = features(cells, cells["T"], cells["xH2"], cells["xHp"], dt)
    Y = targets(cells["T"], cells["xH2"], cells["xHp"], out["xe0"], out["T1"], out["x21"], out["xp1"], out["xe1"])
    ok = np.all(np.isfinite(X), axis=1) & np.all(np.isfinite(Y), axis=1) & (nsub == 1)
    return X[ok], Y[ok], synthgen.subset(cells, np.nonzero(ok)[0]), dt[ok]


def train(X: np.ndarray, Y: np.ndarray, epochs: int = 6, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          val_frac: float = 0.05, log=print) -> tuple:
    """Trains a SeedNet on (X, Y); returns (net, history) with per-epoch train/val loss."""
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    perm = rng.permutation(X.shape[0])
    nval = max(1, int(val_frac * X.shape[0]))
    vi, ti = perm[:nval], perm[nval:]
    mean = X[ti].mean(axis=0, dtype=np.float64)
    std = X[ti].std(axis=0, dtype=np.float64)
    std = np.where(std > 1e-6, std, 1.0)
    net = tc.SeedNet(seed)
    net.set_norm(mean, std)
    Xt = torch.from_numpy(X[ti]).to(dev)
    Yt = torch.from_numpy(Y[ti]).to(dev)
    Xv = torch.from_numpy(X[vi]).to(dev)
    Yv = torch.from_numpy(Y[vi]).to(dev)
    nb = Xt.shape[0] // batch
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    step, total = 0, epochs * nb
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(Xt.shape[0])[: nb * batch]).to(dev).view(nb, batch)
        acc = torch.zeros(1, dtype=torch.float32, device=dev)
        for i in range(nb):
            # cosine decay from lr to lr/20
            lr_i = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * step / max(1, total))))
            xb = Xt.index_select(0, order[i])
            yb = Yt.index_select(0, order[i])
            net.train_step(xb, yb, lr_i, loss)
            acc += loss
            step += 1
        _, vloss = net.grad(Xv, Yv)
        hist.append((float(acc.item()) / max(1, nb), float(vloss.item())))
        log("epoch %d: train %.5f  val %.5f" % (ep, hist[-1][0], hist[-1][1]))
    return net, hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=4_000_000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_BLOB)
    a = ap.parse_args()
    X, Y, _, _ = make_dataset(a.samples)
    net, hist = train(X, Y, a.epochs, a.batch, a.lr, a.seed)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "wb") as fh:
        fh.write(net.export())
    print("wrote %s (val loss %.5f)" % (a.out, hist[-1][1]))


if __name__ == "__main__":
    main()
