"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import synthgen
from tests._parity import assert_fp64_parity, ulp_spread

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
def cfg1():
    c = synthgen.cells_4096()
    r0, spread0 = ulp_spread(oracle, c, DT, oracle.default_params(mode=0))
    ref = {0: r0, 1: oracle.step(c, DT, oracle.default_params(mode=1)), "spread0": spread0}
    return c, ref


def test_config1_paper_scheme_fp64(tc, cfg1):
    c, ref = cfg1
    g = tc.step_numpy(c, DT, tc.TC_MODE_PAPER_FP64)
    assert np.all(g["status"] == 0)
    assert_fp64_parity(g, ref[0], "mode0", spread=ref["spread0"])
    assert np.mean(g["nsub"] != ref[0]["nsub"]) < 0.01


def test_config1_newton_fp64(tc, cfg1):
    c, ref = cfg1
    g = tc.step_numpy(c, DT, tc.TC_MODE_NEWTON_FP64)
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert_fp64_parity(g, ref[1], "mode1")


@pytest.mark.parametrize("key", [42, 43])
def test_newton_fp64_hot_random_states_strict(tc, key):
    # 4096 random states that hold hot molecular cells (1e7 K, x_H2 ~ 0.49) whose Newton
    # solve from the start state fails and restarts from the block predictor: plain
    # FP64 bound, same substep counts, no halved substep on either side.
    c = synthgen.cells_4096(n=4096, key=key)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    assert np.any(ref["status"] & oracle.ST_PREDICTOR)
    assert np.all((ref["status"] & tc.TC_ST_ERROR_MASK) == 0)
    g = tc.step_numpy(c, DT, tc.TC_MODE_NEWTON_FP64)
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert np.array_equal(g["nsub"], ref["nsub"])
    assert_fp64_parity(g, ref, "mode1 key%d" % key)


@pytest.mark.parametrize("n", [1, 31, 33, 4097])
def test_ragged_sizes_paper(tc, n):
    c = synthgen.cells_4096(n=n, key=77)
    ref, spread = ulp_spread(oracle, c, DT, oracle.default_params(mode=0))
    g = tc.step_numpy(c, DT, tc.TC_MODE_PAPER_FP64)
    assert_fp64_parity(g, ref, "ragged%d" % n, spread=spread)


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_ragged_sizes_newton(tc, n):
    c = synthgen.cells_4096(n=n, key=78)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    g = tc.step_numpy(c, DT, tc.TC_MODE_NEWTON_FP64)
    assert_fp64_parity(g, ref, "ragged-newton%d" % n)


def test_zero_cells_and_zero_dt(tc):
    import torch
    c = synthgen.cells_4096(n=64, key=5)
    st = tc.Stepper(tc.TC_MODE_PAPER_FP64)
    d = tc.to_device(c)
    empty = tc.make_fields(d, ncell=0)
    tc.tc_step(st.h, empty, DT)          # no-op
    T0 = d["T"].clone()
    st.step(d, 0.0)
    torch.cuda.synchronize()
    assert torch.allclose(d["T"], T0, rtol=1e-14, atol=0)
    assert int(d["nsub"].max()) == 0
    with pytest.raises(tc.TcError):
        st.step(d, -1.0)
    st.close()


def test_host_buffer_entry_matches_device(tc, cfg1):
    c, ref = cfg1
    sub = synthgen.subset(c, slice(0, 1000))
    host = {k: np.array(np.broadcast_to(sub[k], (1000,)), dtype=np.float64) for k in tc.INPUT_KEYS + ("T", "xH2", "xHp")}
    for k in ("xe", "xCp", "xCO"):
        host[k] = np.zeros(1000)
    host["nsub"] = np.zeros(1000, dtype=np.int32)
    host["status"] = np.zeros(1000, dtype=np.int32)
    st = tc.Stepper(tc.TC_MODE_PAPER_FP64)
    st.step_host(host, DT)
    g = tc.step_numpy(sub, DT, tc.TC_MODE_PAPER_FP64)
    for k in ("T", "xH2", "xHp", "xe"):
        assert np.array_equal(host[k], g[k]), k
    st.close()


def test_batched_alternating_box_sets_without_sync(tc):
    # Two box sets launched in turn, twice each, with no synchronisation between calls:
    # every call re-captures the batched graph while the previous one may still run, so
    # each launch must still read its own box table.  Both sets end two steps on.
    import torch
    sets = [[synthgen.cells_4096(n=n, key=400 + 10 * s + i, Z=z) for i, (n, z) in enumerate(shape)]
            for s, shape in enumerate([[(700, 0.5), (300, 2.0)], [(999, 1.0), (64, 0.2), (257, 3.0)]])]
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    devs = [[tc.to_device(b) for b in bs] for bs in sets]
    for ds in devs:
        for d in ds:
            d.pop("Zg"); d.pop("Zd")
    fields = [[tc.make_fields(d, Zg=float(b["Zg"][0]), Zd=float(b["Zd"][0])) for d, b in zip(ds, bs)]
              for ds, bs in zip(devs, sets)]
    for _ in range(2):
        tc.tc_step_batch(st.h, fields[0], DT)
        tc.tc_step_batch(st.h, fields[1], DT)
    torch.cuda.synchronize()
    p1 = oracle.default_params(mode=1)
    for ds, bs in zip(devs, sets):
        for d, b in zip(ds, bs):
            r1 = oracle.step(b, DT, p1)
            b2 = dict(b, T=r1["T"], xH2=r1["xH2"], xHp=r1["xHp"])
            ref = oracle.step(b2, DT, p1)
            assert_fp64_parity({k: d[k].cpu().numpy() for k in ("T", "xH2", "xHp")}, ref, "alternating")
    st.close()


def test_batched_boxes_match_oracle_and_replay(tc):
    import torch
    boxes = [synthgen.cells_4096(n=n, key=300 + i, Z=z) for i, (n, z) in enumerate([(512, 0.3), (1000, 1.0), (77, 2.5)])]
    st = tc.Stepper(tc.TC_MODE_PAPER_FP64)
    devs = [tc.to_device(b) for b in boxes]
    fields = [tc.make_fields(d, Zg=float(b["Zg"][0]), Zd=float(b["Zd"][0])) for d, b in zip(devs, boxes)]
    for d in devs:
        d.pop("Zg"); d.pop("Zd")
    fields = [tc.make_fields(d, Zg=float(b["Zg"][0]), Zd=float(b["Zd"][0])) for d, b in zip(devs, boxes)]
    tc.tc_step_batch(st.h, fields, DT)
    torch.cuda.synchronize()
    # Each box against the oracle at its own metallicity.  (The batched kernel is a
    # separate instantiation; FMA contraction may differ from the single-box kernel at
    # the rounding level, so the bar is the parity tolerance, not bit equality.)
    for d, b in zip(devs, boxes):
        ref, spread = ulp_spread(oracle, b, DT, oracle.default_params(mode=0))
        assert_fp64_parity({k: d[k].cpu().numpy() for k in ("T", "xH2", "xHp")}, ref, "batch", spread=spread)
    # replay of the captured graph on restored inputs gives the same answer
    first = [d["T"].clone() for d in devs]
    for d, b in zip(devs, boxes):
        for k in ("T", "xH2", "xHp"):
            d[k].copy_(torch.from_numpy(np.ascontiguousarray(b[k])).cuda())
    tc.tc_step_batch(st.h, fields, DT)
    torch.cuda.synchronize()
    for d, f0 in zip(devs, first):
        assert torch.equal(d["T"], f0)
    st.close()


def test_status_and_substep_cap(tc):
    import torch
    c = synthgen.cells_4096(n=2048, key=9)
    st = tc.Stepper(tc.TC_MODE_PAPER_FP64, max_substeps=2)
    d = tc.to_device(c)
    st.step(d, DT)
    nbad = tc.tc_sync_status(st.h, d["status"])
    ref = oracle.step(c, DT, oracle.default_params(mode=0, max_substeps=2))
    assert nbad == int(np.sum(ref["status"] != 0)) and nbad > 0
    assert np.array_equal(d["status"].cpu().numpy(), ref["status"])
    st.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_config2_slab_sampled_full_size(tc, mode):
    # Full 128^3 slab on the GPU in the benchmark's launch configuration; sampled cells
    # checked one by one against the oracle.
    import torch
    c = synthgen.slab()
    d = tc.to_device(c)
    st = tc.Stepper(mode)
    st.step(d, DT)
    torch.cuda.synchronize()
    g = tc.from_device(d)
    st.close()
    assert int(np.sum(g["status"] != 0)) == 0
    idx = np.random.default_rng(mode).choice(c["n"].size, 3000, replace=False)
    sub = synthgen.subset(c, idx)
    if mode == 0:
        ref, spread = ulp_spread(oracle, sub, DT, oracle.default_params(mode=0))
    else:
        ref, spread = oracle.step(sub, DT, oracle.default_params(mode=1)), None
    assert_fp64_parity(synthgen.subset(g, idx), ref, "slab-mode%d" % mode, spread=spread)
