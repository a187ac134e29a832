"""The g-space route to P~ (gw_build_PG): sphere transforms of the pair densities and an
N_g x N_g rank-k update, against Eq. (gpsaceP) in FP64 (the oracle's g-space route), against the
r-space route of the same library, and through eps^-1."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gspace(psi, E, nv, dims, gcut, prec="fp16x3"):
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, nv)
        g = ctx.build_PG(gcut, prec)
        ng = len(g)
        PG = torch.empty((ng, ng), dtype=torch.complex64, device=dev)
        ctx.build_PG(gcut, prec, PG_out=PG)
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
        resid = float((inv @ eps - torch.eye(ng, dtype=torch.complex128, device=dev)).abs().max())
        return g, PG.cpu().numpy(), inv.cpu().numpy(), resid


@pytest.fixture(scope="module")
def small():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    g = O.sphere(dims, w.gcut)
    return w, psi, E, dims, g, O.P_gspace(psi, E, w.nv, dims, g)


@pytest.mark.parametrize("prec,tol", [("fp16x3", 1e-6), ("bf16x3", 1e-4)])
def test_small_matches_oracle(small, prec, tol):
    w, psi, E, dims, gref, Pt = small
    g, PG, inv, resid = gspace(psi, E, w.nv, dims, w.gcut, prec)
    assert np.array_equal(g, gref)
    assert rel(PG, Pt) <= tol
    assert np.array_equal(PG, PG.conj().T)       # Hermitian by construction (mirrored writes)
    assert np.all(PG.diagonal().imag == 0)
    assert resid <= 1e-12


def test_small_equals_rspace_route(small):
    w, psi, E, dims, gref, Pt = small
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, w.nv)
        ctx.build_P("fp16x3")
        ctx.P_to_G(w.gcut)
        PG_r = ctx.view("PG").cpu().numpy()
        ctx.build_PG(w.gcut)
        PG_g = ctx.view("PG").cpu().numpy()
        with pytest.raises(gw.GwError):   # the g-space route does not form P(r,r')
            ctx.view("P")
    assert rel(PG_g, PG_r) <= 1e-6


def test_ragged_noncubic_grid():
    dims, nv, nc, gcut = (10, 12, 14), 3, 20, 4
    psi, E = inputs.make_states(0, nv, nc, 17, dims=dims)
    gref = O.sphere(dims, gcut)
    g, PG, inv, resid = gspace(psi, E, nv, dims, gcut)
    assert np.array_equal(g, gref)
    assert rel(PG, O.P_gspace(psi, E, nv, dims, gref)) <= 1e-6
    assert resid <= 1e-12


def test_plane_wave_closed_form():
    """psi_v = exp(iG_a.r)/sqrt(N_r), psi_c = exp(iG_b.r)/sqrt(N_r): M is a Kronecker delta at
    G_b - G_a, so P~ has the single entry 2/(E_v - E_c) (Hartree) there and zeros elsewhere."""
    dims = (8, 8, 8)
    psi, E = inputs.plane_wave_states(dims, [(0, 0, 0), (1, 0, 0)], [-3.0, 5.0])
    g, PG, inv, resid = gspace(psi, E, 1, dims, 3)
    i = int(np.flatnonzero((g == [1, 0, 0]).all(axis=1))[0])
    want = 2.0 / ((E[0] - E[1]) / 27.211386245988)
    assert abs(PG[i, i].real - want) <= 1e-6 * abs(want)
    off = PG.copy()
    off[i, i] = 0
    assert np.abs(off).max() <= 1e-6 * abs(want)


def test_call_order_and_arguments(small):
    w, psi, E, dims, gref, Pt = small
    with gw.Context(0) as ctx:
        with pytest.raises(gw.GwError):
            ctx.build_PG(w.gcut)                    # before gw_load_states
        ctx.load_states(psi, E, dims, w.nv)
        with pytest.raises(gw.GwError):
            ctx.build_PG(w.gcut, "tf32x3")          # only the 16-bit update is offered here
        with pytest.raises(gw.GwError):
            ctx.build_PG(100)                       # sphere outside the grid


def test_plain_workload_full_size():
    """24^3, N_v = 32, N_c = 480 (k = 15360, N_g = 691): all of P~ against Eq. (gpsaceP), eps^-1
    against the oracle's inverse."""
    w = inputs.PLAIN
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    g, PG, inv, resid = gspace(psi, E, w.nv, dims, w.gcut)
    gref = O.sphere(dims, w.gcut)
    assert np.array_equal(g, gref) and len(g) == 691
    Pt = O.P_gspace(psi, E, w.nv, dims, gref)
    assert rel(PG, Pt) <= 1e-6
    inv_ref = O.inverse_cholesky(O.eps_build(Pt, gref, w.cell_L))
    assert np.max(np.abs(inv - inv_ref)) <= 1e-6
    assert resid <= 1e-12


@pytest.mark.slow
def test_largest_grid_gspace_route():
    """The largest grid gw_load_states takes, 64^3 (N_r = 262144), by the g-space route: P(r,r')
    would be 550 GB, the route needs k N_r complex64 (0.14 GB here).  N_v = 4, N_c = 32, gcut 40
    (about a thousand G): all of P~ against Eq. (gpsaceP), then eps^-1."""
    dims, nv, nc, gcut = (64, 64, 64), 4, 32, 40
    psi, E = inputs.make_states(64, nv, nc, 29)
    gref = O.sphere(dims, gcut)
    g, PG, inv, resid = gspace(psi, E, nv, dims, gcut)
    assert np.array_equal(g, gref) and len(g) > 1000
    assert rel(PG, O.P_gspace(psi, E, nv, dims, gref)) <= 1e-6
    assert resid <= 1e-12
