"""Pins of the oracle's coupled implicit scheme (mode B, Sec. 6.1) that do not come from
the oracle itself: its result must be the backward-Euler root of each substep, which
does not depend on how the Newton iteration reaches it.

* No substep of the random-state workloads is halved: each solve converges at the
  length the substep rule of Sec. 6.1 gives, restarting from the block predictor where
  the iteration from the start state fails (hot molecular cells next to x_H = 0).
* Path independence: moving an input state variable by one unit in the last place
  moves the outputs by rounding only (a halved substep, or a solve that lands on
  another root, would move them by the scheme's discretisation error, ~1e-4).
* The predictor's start point leads to the same roots as the start state on the
  workloads that exercise it.  (Not everywhere: thermally unstable gas can give a
  substep's backward-Euler system a second root, and the predictor reaches it in about
  one cell in 10^4 of the random states, e.g. n = 5e3 cm^-3 cooling from 353 K.  That
  is why the predictor is a fallback, used only where the iteration from the start
  state fails.)
"""
import numpy as np
import pytest

import oracle
import synthgen

DT = synthgen.DT_1E4YR


@pytest.mark.parametrize("key", [0, 42, 43, 91])
def test_no_substep_halved_on_random_states(key):
    r = oracle.step(synthgen.cells_4096(key=key), DT, oracle.default_params(mode=1))
    assert np.all((r["status"] & (oracle.ST_NEWTON | oracle.ST_NONFINITE | oracle.ST_MAX_SUBSTEPS)) == 0)
    if key in (42, 43):
        assert np.any(r["status"] & oracle.ST_PREDICTOR)


@pytest.mark.parametrize("key", [42, 43])
def test_one_ulp_changes_move_mode_b_by_rounding_only(key):
    c = synthgen.cells_4096(key=key)
    p = oracle.default_params(mode=1)
    base = oracle.step(c, DT, p)
    worst = 0.0
    for k in ("T", "xH2", "xHp"):
        for d in (np.inf, 0.0):
            c2 = dict(c)
            c2[k] = np.nextafter(np.asarray(c[k], dtype=np.float64), d)
            r = oracle.step(c2, DT, p)
            assert np.array_equal(r["nsub"], base["nsub"])
            worst = max(worst, float(np.max(np.abs(r["T"] - base["T"]) / base["T"])))
    assert worst < 1e-10, worst


@pytest.mark.parametrize("workload", ["key42", "key43", "slab"])
def test_predictor_start_reaches_the_start_state_root(workload):
    # Every solve started from the predictor (oracle-only flag) must land on the roots
    # the plain solve reaches from the start state: the same substeps, the same result.
    c = synthgen.slab(ncell=8192, key=2) if workload == "slab" else synthgen.cells_4096(key=int(workload[3:]))
    plain = oracle.step(c, DT, oracle.default_params(mode=1))
    pred = oracle.step(c, DT, oracle.default_params(mode=1, flags=oracle.F_PREDICTOR))
    assert np.all(pred["status"] & oracle.ST_PREDICTOR)
    assert np.all((pred["status"] & (oracle.ST_NEWTON | oracle.ST_NONFINITE)) == 0)
    assert np.array_equal(pred["nsub"], plain["nsub"])
    np.testing.assert_allclose(pred["T"], plain["T"], rtol=1e-10)
    np.testing.assert_allclose(pred["xH2"], plain["xH2"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(pred["xHp"], plain["xHp"], rtol=1e-10, atol=1e-14)
