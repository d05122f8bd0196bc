"""The seed network on the GPU: forward pass and gradients against the CPU FP64
reference (oracle/mlp.py, same BF16-rounded weights), training, the weight blob, and
the seeded step modes: the same roots as the unseeded solver, with the Newton
iteration counts reported."""
import os

import numpy as np
import pytest

import oracle
import synthgen
from oracle import mlp as ref_mlp
from tests._parity import assert_fp64_parity, assert_mixed_parity

pytestmark = pytest.mark.gpu

DT = synthgen.DT_1E4YR


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _rounded(theta):
    """The weights the kernels use: BF16-rounded weights, FP32 biases."""
    parts = ref_mlp.unflatten(theta)
    out = []
    for i, p in enumerate(parts):
        out.append(ref_mlp.bf16_round(p) if i % 2 == 0 else np.asarray(p, dtype=np.float32).astype(np.float64))
    return ref_mlp.flatten(out)


def _random_net(tc, seed=0):
    g = np.random.default_rng(seed)
    theta = (g.normal(0.0, 0.25, ref_mlp.n_params())).astype(np.float32)
    net = tc.SeedNet(1)
    net.set_params(theta)
    net.set_norm(np.zeros(ref_mlp.N_IN), np.ones(ref_mlp.N_IN))
    return net, theta.astype(np.float64)


def test_forward_matches_fp64_reference(tc):
    import torch
    net, theta = _random_net(tc)
    x = np.random.default_rng(1).normal(0, 1, (1000, ref_mlp.N_IN)).astype(np.float32)
    o = net.predict(torch.from_numpy(x).cuda()).cpu().numpy()
    r, _, _ = ref_mlp.forward(_rounded(theta), x.astype(np.float64))
    np.testing.assert_allclose(o, r, rtol=1e-4, atol=1e-5)
    net.close()


def test_tensor_core_inference_matches_bf16_reference(tc):
    # The seeded step kernels evaluate the network with warp-level BF16 tensor-core
    # instructions (every layer's inputs rounded to BF16, FP32 accumulation).  On random
    # weights and features, including row counts that leave a warp partly empty, the
    # outputs must equal the CPU reference of that rounding, and stay within the BF16
    # rounding of the FP32-activation forward pass of the training kernels.
    import torch
    net, theta = _random_net(tc, 5)
    g = np.random.default_rng(6)
    mean = g.normal(0, 1, ref_mlp.N_IN)
    std = g.uniform(0.5, 2.0, ref_mlp.N_IN)
    net.set_norm(mean, std)
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64_SEEDED)
    st.load_mlp(net.export())
    for B in (1, 31, 1000, 4097):
        x = (mean + std * g.normal(0, 1, (B, ref_mlp.N_IN))).astype(np.float32)
        out = torch.empty((B, 3), dtype=torch.float32, device="cuda")
        tc.tc_seed_predict(st.h, torch.from_numpy(x).cuda(), out)
        o = out.cpu().numpy()
        xn = (x.astype(np.float64) - np.float32(mean).astype(np.float64)) * (1.0 / std.astype(np.float32)).astype(np.float64)
        r = ref_mlp.forward_bf16_inputs(_rounded(theta), xn)
        scale = np.abs(r).max()
        np.testing.assert_allclose(o, r, rtol=0, atol=2e-2 * scale)
        assert np.median(np.abs(o - r)) < 2e-3 * scale
        full = net.predict(torch.from_numpy(x).cuda()).cpu().numpy()
        np.testing.assert_allclose(o, full, rtol=0, atol=5e-2 * scale)
    st.close()
    net.close()


def test_gradient_matches_fp64_reference(tc):
    import torch
    net, theta = _random_net(tc, 2)
    g = np.random.default_rng(3)
    x = g.normal(0, 1, (4096, ref_mlp.N_IN)).astype(np.float32)
    y = g.normal(0, 1, (4096, 3)).astype(np.float32)
    w = (1.0, 2.0, 0.5)
    grad, loss = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), w)
    grad = grad.cpu().numpy().astype(np.float64)
    th = _rounded(theta)
    gr = ref_mlp.grad(th, x.astype(np.float64), y.astype(np.float64), w)
    lr = ref_mlp.loss(th, x.astype(np.float64), y.astype(np.float64), w)
    assert float(loss.item()) == pytest.approx(lr, rel=1e-4)
    # whole-vector and per-block relative errors, FP32 accumulation over 4096 samples
    assert np.linalg.norm(grad - gr) <= 1e-4 * np.linalg.norm(gr)
    k = 0
    for s in ref_mlp.SHAPES:
        m = int(np.prod(s))
        a, b = grad[k:k + m], gr[k:k + m]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-9, s
        k += m
    net.close()


def test_training_reduces_loss(tc):
    import torch
    g = np.random.default_rng(4)
    x = g.normal(0, 1, (16384, ref_mlp.N_IN)).astype(np.float32)
    y = np.stack([np.tanh(x[:, 0] - x[:, 1]), 0.5 * x[:, 2] * x[:, 3], np.sin(x[:, 4])], axis=1).astype(np.float32)
    net = tc.SeedNet(5)
    X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    _, l0 = net.grad(X, Y)
    loss = torch.zeros(1, device="cuda")
    for i in range(300):
        idx = torch.randint(0, 16384, (1024,), device="cuda")
        net.train_step(X[idx], Y[idx], 3e-3, loss)
    _, l1 = net.grad(X, Y)
    assert float(l1.item()) < 0.1 * float(l0.item())
    net.close()


def test_blob_roundtrip_and_validation(tc):
    net, _ = _random_net(tc, 6)
    blob = net.export()
    assert len(blob) == int(tc.lib.tc_mlp_blob_bytes())
    st = tc.Stepper(tc.TC_MODE_MIXED_SEEDED)
    st.load_mlp(blob)
    with pytest.raises(tc.TcError):
        st.load_mlp(blob[:-16])
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(tc.TcError):
        st.load_mlp(bytes(bad))
    st.close()
    s2 = tc.Stepper(tc.TC_MODE_NEWTON_FP64_SEEDED)
    d = tc.to_device(synthgen.cells_4096(n=64, key=8))
    with pytest.raises(tc.TcError):   # seeded mode without weights
        s2.step(d, DT)
    s2.close()
    net.close()


@pytest.fixture(scope="module")
def trained_blob(tc):
    from paper_2210_08024_gb300 import seed_net
    if os.path.exists(seed_net.DEFAULT_BLOB):
        return open(seed_net.DEFAULT_BLOB, "rb").read()
    X, Y, _, _ = seed_net.make_dataset(300_000, key=40, log=lambda *a: None)
    net, _ = seed_net.train(X, Y, epochs=3, batch=4096, log=lambda *a: None)
    blob = net.export()
    net.close()
    return blob


def _run(tc, cells, mode, blob=None):
    import torch
    d = tc.to_device(cells)
    st = tc.Stepper(mode)
    if blob is not None:
        st.load_mlp(blob)
    st.step(d, DT)
    torch.cuda.synchronize()
    out = tc.from_device(d)
    st.close()
    return out


def test_training_labels_match_oracle(tc):
    # The seed network's labels are single backward-Euler roots from the library's FP64
    # solver with the substep limiter off; 10k of them re-checked against the CPU
    # oracle's coupled scheme at the FP64 bound, over step lengths 1e4 .. 1e11 s.
    from paper_2210_08024_gb300 import seed_net
    n = 10000
    cells = synthgen.training_samples(n, key=45)
    cells.pop("dt")
    b = np.random.default_rng(3).integers(80, 221, n)
    ok = np.ones(n, dtype=bool)
    lab = seed_net.label_states(cells, b, 20, ok)
    p = oracle.default_params(mode=1, limiter=1e30)
    for bk in np.unique(b):
        idx = np.nonzero(b == bk)[0]
        ref = oracle.step(synthgen.subset(cells, idx), 10.0 ** (bk / 20), p)
        assert np.array_equal(lab["nsub"][idx], ref["nsub"])
        assert_fp64_parity({k: lab[k][idx] for k in ("T", "xH2", "xHp")}, ref, "labels dt=%g" % 10.0 ** (bk / 20))


@pytest.mark.parametrize("workload", ["slab", "random"])
def test_seeded_fp64_same_root(tc, trained_blob, workload):
    # The seeded FP64 solve (FP64 chord iterations from the network's prediction on an
    # FP32 Jacobian built there, the plain Newton solve from the start state where the
    # seed is missing or fails) must reach the same FP64 roots as the unseeded solver.
    # On the slab most cells start some substep from the seed.  Iteration counts are
    # printed with -s; they are not comparable with the plain solve's (a chord
    # iteration evaluates f once, a full Newton iteration four times).
    c = synthgen.slab(ncell=20000, key=41) if workload == "slab" else synthgen.cells_4096(n=2048, key=43)
    plain = _run(tc, c, tc.TC_MODE_NEWTON_FP64)
    seeded = _run(tc, c, tc.TC_MODE_NEWTON_FP64_SEEDED, trained_blob)
    assert np.array_equal(seeded["status"] & tc.TC_ST_ERROR_MASK, plain["status"] & tc.TC_ST_ERROR_MASK)
    assert_fp64_parity(seeded, plain, "seeded-vs-plain")
    assert np.array_equal(seeded["nsub"], plain["nsub"])
    ref = oracle.step(synthgen.subset(c, slice(0, 2000)), DT, oracle.default_params(mode=1))
    assert_fp64_parity(synthgen.subset(seeded, slice(0, 2000)), ref, "seeded-vs-oracle")
    print("%s: iterations per cell: plain %.3f, seeded %.3f; cells with a seeded solve %.3f, with a failed seed %.4f"
          % (workload, plain["iters"].mean(), seeded["iters"].mean(),
             np.mean((seeded["status"] & tc.TC_ST_SEEDED) != 0), np.mean((seeded["status"] & tc.TC_ST_SEED_FAIL) != 0)))
    if workload == "slab":
        assert np.mean((seeded["status"] & tc.TC_ST_SEEDED) != 0) > 0.5
        assert np.mean((seeded["status"] & tc.TC_ST_SEED_FAIL) != 0) < 0.05


def test_seeded_mixed_needs_fewer_iterations_on_slab(tc, trained_blob):
    # The mixed solve's FP32 Newton iterations from the seed (measured on the 128^3 slab:
    # 10.44 against 11.30 per cell; seeded mixed 111 ms against 129 ms unseeded).
    c = synthgen.slab(ncell=20000, key=41)
    plain = _run(tc, c, tc.TC_MODE_MIXED)
    seeded = _run(tc, c, tc.TC_MODE_MIXED_SEEDED, trained_blob)
    print("slab mixed: FP32 iterations per cell: plain %.3f, seeded %.3f" % (plain["iters"].mean(),
                                                                          seeded["iters"].mean()))
    assert seeded["iters"].sum() <= 0.95 * plain["iters"].sum()
    assert_mixed_parity(seeded, plain, "seeded-vs-plain mixed")


def test_seeded_mixed_within_tolerance(tc, trained_blob):
    # Random states include hot molecular gas that cools through 1e4 K over ~100
    # substeps; no substep of this workload is halved by either side, so the bound is
    # the plain mixed one, cell by cell.
    c = synthgen.cells_4096(n=4096, key=42)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    assert np.all((ref["status"] & tc.TC_ST_ERROR_MASK) == 0)
    g = _run(tc, c, tc.TC_MODE_MIXED_SEEDED, trained_blob)
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert_mixed_parity(g, ref, "mixed-seeded")
