"""Shared helpers of the parity tests (tolerances and comparisons).

FP64 paths vs the FP64 oracle: relative 1e-9 on T, and on x_H2, x_H+ relative 1e-9 with
an absolute floor of 1e-14.  Every abundance passes through the closure
x_H = 1 - 2 x_H2 - x_H+, whose FP64 rounding is a few 1e-16 in absolute terms; when
x_H+ -> 1 (or x_H2 -> 0.5) the trace species inherit that absolute error, so a purely
relative bound on a 1e-7 abundance would ask for more digits than the closure carries.

The paper's sequential scheme (Sec. 6.1, mode 0) is, in addition, ill-conditioned with
respect to rounding: its finite-difference dH/dT_mu divides a difference of two nearly
equal source terms by 1e-3 T_mu, and the substep lengths (0.1 e/|H|, 0.1/|C|) feed
back into the elapsed time at which the truncated last substep ends.  Perturbing the
input temperature by one unit in the last place moves the oracle's own result by up
to ~1e-9.  The mode-0 bound therefore adds four times that measured one-ulp spread
(``ulp_spread``) to the 1e-9 relative bound, cell by cell.

Mixed path vs the FP64 oracle: 1e-5 relative on T and 1e-6 absolute on abundances.

The coupled scheme (mode 1) carries no such allowance: its result is the backward-Euler
root of each substep, which does not depend on the path the Newton iteration takes to
it, and no substep of the test workloads is halved (a solve that fails from the start
state restarts from the block predictor first), so every FP64 and mixed comparison of
mode 1 uses the plain bounds above.
"""
import numpy as np

RTOL_FP64 = 1e-9
ATOL_X_FP64 = 1e-14
SPREAD_FACTOR = 4.0
RTOL_T_MIXED = 1e-5
ATOL_X_MIXED = 1e-6


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def ulp_spread(oracle_mod, cells, dt, params, inputs=("T",)):
    """Largest change of the oracle's outputs when one input state variable (each of
    `inputs` in turn) moves by one unit in the last place (up or down): a per-cell
    measure of how much rounding the paper's sequential scheme amplifies."""
    base = oracle_mod.step(cells, dt, params)
    spread = {k: np.zeros_like(base[k]) for k in ("T", "xH2", "xHp")}
    for key in inputs:
        for direction in (np.inf, 0.0):
            c2 = dict(cells)
            c2[key] = np.nextafter(np.asarray(cells[key], dtype=np.float64), direction)
            r2 = oracle_mod.step(c2, dt, params)
            for k in spread:
                spread[k] = np.maximum(spread[k], np.abs(r2[k] - base[k]))
    return base, spread


def assert_fp64_parity(gpu, ref, label="", spread=None):
    for k in ("T", "xH2", "xHp"):
        a = np.asarray(gpu[k], dtype=np.float64)
        b = np.asarray(ref[k], dtype=np.float64)
        tol = RTOL_FP64 * np.abs(b)
        if k != "T":
            tol = tol + ATOL_X_FP64
        if spread is not None:
            tol = tol + SPREAD_FACTOR * spread[k]
        err = np.abs(a - b)
        bad = np.where(~(err <= tol))[0]
        assert bad.size == 0, "%s %s: %d cells over tolerance (worst rel %.3e at %d: gpu %r oracle %r)" % (
            label, k, bad.size, np.nanmax(err / np.maximum(np.abs(b), 1e-300)), bad[0], a[bad[0]], b[bad[0]])


def assert_mixed_parity(gpu, ref, label=""):
    b = np.asarray(ref["T"], dtype=np.float64)
    err = np.abs(np.asarray(gpu["T"], dtype=np.float64) - b)
    tol = RTOL_T_MIXED * np.abs(b)
    assert np.all(err <= tol), "%s T: max rel %.3e" % (label, np.nanmax(err / np.abs(b)))
    for k in ("xH2", "xHp"):
        ea = np.abs(np.asarray(gpu[k]) - np.asarray(ref[k]))
        assert np.all(ea <= ATOL_X_MIXED), "%s %s: max abs %.3e" % (label, k, np.nanmax(ea))
