"""GPU parity of the six-ray fields (tc_sixray, Secs. 5.2, 5.3) against the oracle
(oracle/sixray.py): ragged and degenerate grid shapes, deep columns whose fields
underflow, no dust, the full 128^3 slab, and the fields feeding the step."""
import numpy as np
import pytest

import oracle
import synthgen
from oracle import sixray as sr
from tests._parity import assert_fp64_parity

pytestmark = pytest.mark.gpu

PC = 3.0856775814913673e18
RTOL = 1e-10


@pytest.fixture(scope="module")
def tc():
    import torch
    assert torch.cuda.is_available()
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _grid(shape, key, mu=1.0, sig=1.5):
    rng = np.random.default_rng(key)
    n = rng.lognormal(mu, sig, shape)
    x = rng.uniform(0.0, 0.5, shape)
    return n, x


def _gpu(tc, n, x, dx, **kw):
    import torch
    out = tc.tc_sixray(torch.from_numpy(n).cuda(), torch.from_numpy(x).cuda(), dx, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(g, r, rtol=RTOL):
    for k in ("chi_pe", "chi_lw", "f_h2", "N_eff", "xi"):
        np.testing.assert_allclose(g[k], r[k], rtol=rtol, atol=0, err_msg=k)


@pytest.mark.parametrize("shape", [(41, 29, 37), (1, 1, 1), (1, 1, 33), (70, 1, 1), (1, 65, 3), (5, 3, 200)])
def test_ragged_and_degenerate_shapes(tc, shape):
    n, x = _grid(shape, key=sum(shape))
    dx = 0.5 * PC
    g = _gpu(tc, n, x, dx, chi0=2.0, xi0=3e-16, Zd=0.7)
    r = sr.sixray(n, x, dx, chi0=2.0, xi0=3e-16, Zd=0.7)
    _compare(g, r)


def test_deep_columns_underflow(tc):
    # ~3000 cm^-3 in 10 pc cells: tau ~ 90 per cell, ~1800 to the centre of a 40^3 cube,
    # so exp(-tau) underflows in the interior while the relative ray sums do not
    n, x = _grid((40, 40, 40), key=5, mu=8.0, sig=0.3)
    g = _gpu(tc, n, x, 10.0 * PC)
    r = sr.sixray(n, x, 10.0 * PC)
    assert np.all(r["chi_pe"][15:25, 15:25, 15:25] == 0.0)
    for k in ("f_h2", "N_eff", "xi"):
        np.testing.assert_allclose(g[k], r[k], rtol=RTOL, atol=0, err_msg=k)
    for k in ("chi_pe", "chi_lw"):
        np.testing.assert_allclose(g[k], r[k], rtol=RTOL, atol=1e-300, err_msg=k)


def test_no_dust(tc):
    n, x = _grid((9, 10, 11), key=6)
    g = _gpu(tc, n, x, 1.0 * PC, Zd=0.0)
    r = sr.sixray(n, x, 1.0 * PC, Zd=0.0)
    _compare(g, r)
    assert np.all(g["xi"] == 2e-16) and np.all(g["N_eff"] == 0.0)


def test_full_slab_grid(tc):
    # the 128^3 slab's densities and H2 fractions laid out on a 128^3 grid of 4 pc cells
    c = synthgen.slab()
    n = np.ascontiguousarray(c["n"].reshape(128, 128, 128))
    x = np.ascontiguousarray(np.broadcast_to(c["xH2"], c["n"].shape).reshape(128, 128, 128))
    g = _gpu(tc, n, x, 4.0 * PC)
    r = sr.sixray(n, x, 4.0 * PC)
    _compare(g, r)


def test_fields_feed_the_step(tc):
    import torch
    n, x = _grid((24, 24, 24), key=7, mu=2.0, sig=1.2)
    dx = 1.0 * PC
    f = tc.tc_sixray(torch.from_numpy(n).cuda(), torch.from_numpy(x).cuda(), dx)
    cells = {"n": n.ravel(), "f_c": 1.0, "F_lyc": 0.0, "Zg": 1.0, "Zd": 1.0, "T": np.full(n.size, 100.0),
             "xH2": x.ravel(), "xHp": np.full(n.size, 1e-3), "chi_pe": 0.0, "chi_lw": 0.0, "f_h2": 0.0, "xi": 0.0}
    d = tc.to_device(cells)
    for k in ("chi_pe", "chi_lw", "f_h2", "xi"):
        d[k].copy_(f[k].reshape(-1))
    st = tc.Stepper(tc.TC_MODE_NEWTON_FP64)
    st.step(d, synthgen.DT_1E4YR)
    torch.cuda.synchronize()
    st.close()
    g = tc.from_device(d)
    r = sr.sixray(n, x, dx)
    oc = dict(cells, chi_pe=r["chi_pe"].ravel(), chi_lw=r["chi_lw"].ravel(), f_h2=r["f_h2"].ravel(),
              xi=r["xi"].ravel())
    idx = np.random.default_rng(8).choice(n.size, 1500, replace=False)
    ref = oracle.step(synthgen.subset(oc, idx), synthgen.DT_1E4YR, oracle.default_params(mode=1))
    assert_fp64_parity(synthgen.subset(g, idx), ref, "sixray+step")


def test_invalid_grids_rejected(tc):
    import torch
    n = torch.ones((2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(tc.TcError):
        tc.tc_sixray(n, n, -1.0)
    with pytest.raises(tc.TcError):
        tc.tc_sixray(n, n, 1.0, Zd=-1.0)
