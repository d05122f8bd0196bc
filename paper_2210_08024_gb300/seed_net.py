"""Training data, training loop and export of the seed network.

The network (include/tc_mlp.h) predicts the root of one backward-Euler step of length
dt, as changes from the cell's state beyond the explicit-Euler ones, from its state,
fields, dt and those explicit changes.  The seeded step modes start each substep's
Newton iteration from that prediction and still iterate to the solver's own tolerance,
so the prediction only shortens the iteration.

Training data: cells drawn like the 128^3 slab (synthgen.training_samples: lognormal
density, two-phase temperatures, six-ray fields) with Z' log-uniform in [0.1, 3].
Each sample's step is the first substep that the substep rule of Sec. 6.1 gives for a
step of 1e4 yr (tc_rates, from the library's own start-state source terms), or for 30%
of the samples a fraction log-uniform in [1e-3, 1] of it, as a truncated last substep
is: the steps the seed is asked about.  Step lengths are rounded to 20 per decade so
that one length is one tc_step.  Labels come from the library's plain FP64 solver
(TC_MODE_NEWTON_FP64, checked against the CPU oracle by the parity tests and, for a
sample of labels, by tests/test_gpu_mlp.py) run with the substep limiter switched off,
so each label is a single backward-Euler root.  Training: Adam on mini-batches with the
library's forward/backward kernels (tc_mlp_train_step), each output's squared error
weighted by the inverse variance of its target; everything numerical runs on the GPU
in those kernels.

    python -m paper_2210_08024_gb300.seed_net --samples 8000000 --epochs 40 --out seed.bin
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
LN10 = math.log(10.0)


def explicit_changes(rate: np.ndarray, dt) -> np.ndarray:
    """Explicit-Euler changes over a step dt in the output units, float64 [N, 3]:
    dt C_H2 / 0.5, dt C_H+, dt H / (K T_mu ln 10), from tc_rates' rates [N, 3]."""
    r = np.asarray(rate, dtype=np.float64).reshape(-1, 3)
    d = np.asarray(dt, dtype=np.float64)
    return np.stack([d * r[:, 0] / 0.5, d * r[:, 1], d * r[:, 2] / LN10], axis=1)


def features(cells: dict, T, xH2, xHp, dt, g) -> np.ndarray:
    """Raw (unnormalised) features in the order of include/tc_mlp.h, float32 [N, 13]."""
    n = np.asarray(cells["n"], dtype=np.float64)
    N = n.size
    bc = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (N,))  # noqa: E731
    chi_fuv = (1.8e-4 * bc(cells["chi_pe"]) + 3.0e-5 * bc(cells["chi_lw"])) / 2.1e-4
    X = np.empty((N, 13), dtype=np.float32)
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
    X[:, 10:13] = g
    return X


def targets(T0, xH2_0, xHp_0, xe0, T1, xH2_1, xHp_1, xe1, g) -> np.ndarray:
    """Changes over one backward-Euler step minus the explicit ones g, float32 [N, 3]:
    (x_H2' - x_H2)/0.5 - g0, x_H+' - x_H+ - g1 and log10 T' - log10 T - g2, where
    T' = mu_0 T_mu' is the root's temperature at the step's start mu (the frozen mu of the
    residual).  The solver returns T1 = mu_1 T_mu', so T' = T1 mu_0 / mu_1 with
    mu = mu_H / (1.1 + x_e - x_H2)."""
    ratio = (1.1 + np.asarray(xe1) - np.asarray(xH2_1)) / (1.1 + np.asarray(xe0) - np.asarray(xH2_0))
    Y = np.empty((np.size(T0), 3), dtype=np.float32)
    Y[:, 0] = (np.asarray(xH2_1) - np.asarray(xH2_0)) / 0.5 - g[:, 0]
    Y[:, 1] = np.asarray(xHp_1) - np.asarray(xHp_0) - g[:, 1]
    Y[:, 2] = np.log10(np.asarray(T1) * ratio) - np.log10(np.asarray(T0)) - g[:, 2]
    return Y


def label_states(cells: dict, b: np.ndarray, per_decade: int, ok: np.ndarray) -> dict:
    """One backward-Euler step of length 10^(b / per_decade) s for each cell where `ok`
    (the library's FP64 Newton with the substep limiter switched off, one tc_step per
    distinct length): the end states T, xH2, xHp, xe and the substep counts nsub."""
    import torch
    n = np.asarray(cells["n"]).size
    out = {k: np.full(n, np.nan) for k in ("T", "xH2", "xHp", "xe")}
    out["nsub"] = np.zeros(n, dtype=np.int32)
    st1 = tc.Stepper(tc.TC_MODE_NEWTON_FP64, limiter=1e30)
    for bk in np.unique(b[ok]):
        idx = np.nonzero((b == bk) & ok)[0]
        dd = tc.to_device(synthgen.subset(cells, idx))
        st1.step(dd, float(10.0 ** (bk / per_decade)))
        torch.cuda.synchronize()
        for k in ("T", "xH2", "xHp", "xe", "nsub"):
            out[k][idx] = dd[k].cpu().numpy()
    st1.close()
    return out


def make_dataset(n: int, key: int = 4, per_decade: int = 20, short_frac: float = 0.3, log=print):
    """Returns (X, Y, cells, dt).  Labels: one backward-Euler step of length dt per sample
    (the substep rule switched off by a huge limiter), solved by the library's plain FP64
    Newton; samples whose solve needed a halved substep are dropped."""
    import torch
    cells = synthgen.training_samples(n, key)
    cells.pop("dt")
    st0 = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    d = tc.to_device(cells)
    rate = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    dts = torch.empty(n, dtype=torch.float64, device="cuda")
    tc.tc_rates(st0.h, tc.make_fields(d), synthgen.DT_1E4YR, rate, dts)
    st0.step(d, 0.0)                     # dt = 0: the initial C/O/e equilibrium only
    torch.cuda.synchronize()
    rate = rate.cpu().numpy().reshape(n, 3)
    xe0 = d["xe"].cpu().numpy()
    del d
    g = np.random.default_rng(key + 1)
    frac = np.where(g.random(n) < short_frac, 10.0 ** g.uniform(-3.0, 0.0, n), 1.0)
    step = dts.cpu().numpy() * frac
    ok = np.isfinite(step) & (step > 0)
    b = np.round(np.log10(np.where(ok, step, 1.0)) * per_decade).astype(np.int64)
    dt = 10.0 ** (b / per_decade)
    out = label_states(cells, b, per_decade, ok)
    nsub = out["nsub"]
    log("labels for %d samples (%d needed more than one substep)" % (int(ok.sum()), int(np.sum(ok & (nsub != 1)))))
    gx = explicit_changes(rate, dt)
    X = features(cells, cells["T"], cells["xH2"], cells["xHp"], dt, gx)
    Y = targets(cells["T"], cells["xH2"], cells["xHp"], xe0, out["T"], out["xH2"], out["xHp"], out["xe"], gx)
    ok &= np.all(np.isfinite(X), axis=1) & np.all(np.isfinite(Y), axis=1) & (nsub == 1)
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
    w3 = tuple(float(v) for v in 1.0 / np.maximum(Y[ti].var(axis=0, dtype=np.float64), 1e-30))
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    step, total = 0, epochs * nb
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(Xt.shape[0])[: nb * batch]).to(dev).view(nb, batch)
        acc = torch.zeros(1, dtype=torch.float32, device=dev)
        for i in range(nb):
            # cosine decay from lr to lr/100
            lr_i = lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * step / max(1, total))))
            xb = Xt.index_select(0, order[i])
            yb = Yt.index_select(0, order[i])
            net.train_step(xb, yb, lr_i, loss, w=w3)
            acc += loss
            step += 1
        _, vloss = net.grad(Xv, Yv, w=w3)
        hist.append((float(acc.item()) / max(1, nb), float(vloss.item())))
        log("epoch %d: train %.5f  val %.5f" % (ep, hist[-1][0], hist[-1][1]))
    return net, hist


def accuracy(net, X: np.ndarray, Y: np.ndarray) -> dict:
    """RMS and 99th-percentile error of the network's changes on (X, Y), with those of
    the explicit-Euler changes (a zero network output) beside them."""
    import torch
    o = net.predict(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    e = o - Y
    z = -Y.astype(np.float64)
    r = lambda a: [float(v) for v in np.sqrt(np.mean(a ** 2, axis=0))]  # noqa: E731
    q = lambda a: [float(v) for v in np.percentile(np.abs(a), 99, axis=0)]  # noqa: E731
    return {"rms": r(e), "p99": q(e), "explicit_rms": r(z), "explicit_p99": q(z)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=8_000_000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_BLOB)
    a = ap.parse_args()
    X, Y, _, _ = make_dataset(a.samples)
    net, hist = train(X, Y, a.epochs, a.batch, a.lr, a.seed)
    Xh, Yh, _, _ = make_dataset(200_000, key=44, log=lambda *x: None)
    print("held-out accuracy (outputs x_H2/0.5, x_H+, log10 T):", accuracy(net, Xh, Yh))
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "wb") as fh:
        fh.write(net.export())
    print("wrote %s (val loss %.5f)" % (a.out, hist[-1][1]))


if __name__ == "__main__":
    main()
