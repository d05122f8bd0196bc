"""Full-size parity cases of the larger workloads, in every headline mode, on sampled
cells checked one by one against the CPU oracle's coupled implicit scheme.

* 256^3 stiff grid (16.8M cells): the slab plus 16 H II regions (ionising flux
  1e7..1e11 cm^-2 s^-1 falling as r^-2) and 16 supernova-remnant interiors
  (1e6..1e8 K, 1% density), plain FP64 and mixed precision on the persistent work
  queue; the sample includes 500 sphere cells.
* 128^3 slab with the seed network: seeded mixed and seeded FP64.
* 48 independent boxes of 32^3..128^3 cells with per-box Z', field and CR scales,
  advanced by one batched launch replayed from a CUDA graph: plain FP64, mixed and
  seeded mixed.

FP64 modes are held to the FP64 bound and the oracle's substep counts; mixed modes to
1e-5 relative on T and 1e-6 absolute on the abundances.  No allowance per cell.
"""
import os

import numpy as np
import pytest

import oracle
import synthgen
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


@pytest.fixture(scope="module")
def blob():
    from paper_2210_08024_gb300 import seed_net
    assert os.path.exists(seed_net.DEFAULT_BLOB)
    return open(seed_net.DEFAULT_BLOB, "rb").read()


def _no_errors(tc, status):
    bad = (status & tc.TC_ST_ERROR_MASK) != 0
    assert int(bad.sum().item()) == 0


def _check(tc, mode, g, ref, label):
    assert np.all((ref["status"] & tc.TC_ST_ERROR_MASK) == 0)
    if mode in (tc.TC_MODE_NEWTON_FP64, tc.TC_MODE_NEWTON_FP64_SEEDED):
        assert_fp64_parity(g, ref, label)
        assert np.array_equal(g["nsub"], ref["nsub"]), label
    else:
        assert_mixed_parity(g, ref, label)


@pytest.fixture(scope="module")
def stiff():
    c = synthgen.stiff()
    n = c["n"].size
    sphere = np.nonzero((c["F_lyc"] > 0) | (c["T"] >= 1e6))[0]
    rng = np.random.default_rng(11)
    idx = np.concatenate([rng.choice(n, 1500, replace=False), rng.choice(sphere, 500, replace=False)])
    ref = oracle.step(synthgen.subset(c, idx), DT, oracle.default_params(mode=1))
    return c, idx, ref


@pytest.mark.parametrize("mode", ["newton_fp64", "mixed"])
def test_stiff_grid_full_size(tc, stiff, mode):
    import torch
    m = {"newton_fp64": tc.TC_MODE_NEWTON_FP64, "mixed": tc.TC_MODE_MIXED}[mode]
    c, idx, ref = stiff
    d = tc.to_device(c)
    st = tc.Stepper(m)
    st.step(d, DT)
    torch.cuda.synchronize()
    _no_errors(tc, d["status"])
    st.close()
    ti = torch.from_numpy(idx).cuda()
    g = {k: d[k][ti].cpu().numpy() for k in ("T", "xH2", "xHp", "nsub")}
    del d
    _check(tc, m, g, ref, "stiff256 " + mode)


@pytest.fixture(scope="module")
def slab():
    c = synthgen.slab()
    idx = np.random.default_rng(13).choice(c["n"].size, 3000, replace=False)
    ref = oracle.step(synthgen.subset(c, idx), DT, oracle.default_params(mode=1))
    return c, idx, ref


@pytest.mark.parametrize("mode", ["mixed_seeded", "newton_fp64_seeded"])
def test_seeded_slab_full_size(tc, blob, slab, mode):
    import torch
    m = {"mixed_seeded": tc.TC_MODE_MIXED_SEEDED, "newton_fp64_seeded": tc.TC_MODE_NEWTON_FP64_SEEDED}[mode]
    c, idx, ref = slab
    d = tc.to_device(c)
    st = tc.Stepper(m)
    st.load_mlp(blob)
    st.step(d, DT)
    torch.cuda.synchronize()
    _no_errors(tc, d["status"])
    st.close()
    ti = torch.from_numpy(idx).cuda()
    g = {k: d[k][ti].cpu().numpy() for k in ("T", "xH2", "xHp", "nsub")}
    _check(tc, m, g, ref, "slab128 " + mode)


@pytest.fixture(scope="module")
def boxes():
    bx = synthgen.boxes()
    assert len(bx) == 48
    rng = np.random.default_rng(12)
    out = []
    for cells, meta in bx:
        idx = rng.choice(cells["n"].size, 24, replace=False)
        ref = oracle.step(synthgen.subset(cells, idx), DT, oracle.default_params(mode=1))
        out.append((cells, meta, idx, ref))
    return out


@pytest.mark.parametrize("mode", ["mixed", "mixed_seeded", "newton_fp64"])
def test_batched_boxes_full_size_graph(tc, blob, boxes, mode):
    import torch
    m = {"mixed": tc.TC_MODE_MIXED, "mixed_seeded": tc.TC_MODE_MIXED_SEEDED,
         "newton_fp64": tc.TC_MODE_NEWTON_FP64}[mode]
    devs, fields, pristine = [], [], []
    for cells, meta, idx, ref in boxes:
        d = tc.to_device(cells)
        devs.append(d)
        fields.append(tc.make_fields(d))
        pristine.append({k: d[k].clone() for k in ("T", "xH2", "xHp")})
    st = tc.Stepper(m)
    if m == tc.TC_MODE_MIXED_SEEDED:
        st.load_mlp(blob)
    tc.tc_step_batch(st.h, fields, DT)
    torch.cuda.synchronize()
    for (cells, meta, idx, ref), d in zip(boxes, devs):
        _no_errors(tc, d["status"])
        ti = torch.from_numpy(idx).cuda()
        g = {k: d[k][ti].cpu().numpy() for k in ("T", "xH2", "xHp", "nsub")}
        _check(tc, m, g, ref, "%s box side %d Z %.2f" % (mode, meta["side"], meta["Z"]))
    if mode == "mixed":
        # the second call replays the captured graph: identical results from the same inputs
        first = [d["T"].clone() for d in devs]
        for d, p in zip(devs, pristine):
            for k in p:
                d[k].copy_(p[k])
        tc.tc_step_batch(st.h, fields, DT)
        torch.cuda.synchronize()
        for d, f0 in zip(devs, first):
            assert torch.equal(d["T"], f0)
    st.close()
