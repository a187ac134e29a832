"""eps^q at q != 0 (gw_set_q): V(q + G) in eps, the head no longer zero, against the oracle's
eps^q and the constant-state closed form, through the r-space and the g-space routes."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

Q = (0.25, -0.1, 0.05)
L = 1.7


def run(psi, E, nv, dims, gcut, q, route, cell_L=L):
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, nv, cell_L=cell_L)
        ctx.set_q(q)
        if route == "gspace":
            g = ctx.build_PG(gcut)
        else:
            ctx.build_P("fp16x3")
            g = ctx.P_to_G(gcut)
        ng = len(g)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
        return g, eps.cpu().numpy(), inv.cpu().numpy()


@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_constant_states_head(route):
    """u_v = u_c = 1/sqrt(N_r): P~ is a head entry only, eps^q_00 = 1 + 8 pi/(Omega |q|^2 (E_c - E_v))."""
    dims = (8, 8, 8)
    psi, E = inputs.plane_wave_states(dims, [(0, 0, 0), (0, 0, 0)], [-2.0, 3.0])
    g, eps, inv = run(psi, E, 1, dims, 3, Q, route)
    q2 = (2 * np.pi / L) ** 2 * np.sum(np.asarray(Q) ** 2)
    e00 = 1.0 + 8 * np.pi / (L ** 3 * q2 * ((E[1] - E[0]) / 27.211386245988))
    assert abs(eps[0, 0].real - e00) <= 1e-6 * e00
    assert abs(inv[0, 0].real - 1.0 / e00) <= 1e-6
    off = inv - np.diag(np.diag(inv))
    assert np.abs(off).max() <= 1e-6   # FP32 transforms leave ~1e-9 off the head


def kq_states(w):
    """u_{v,k+q} and u_{c,k} from two independent draws: each set orthonormal, the two sets not
    orthogonal to each other (as for a real q != 0), so P~ and eps^q have a non-zero head."""
    pa, E = inputs.make_states(w.n, w.nv, w.nc, w.seed)
    pb, _ = inputs.make_states(w.n, w.nv, w.nc, w.seed + 1000)
    return np.concatenate([pa[: w.nv], pb[w.nv:]]), E


@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_random_states_match_oracle(route):
    w = inputs.SMALL
    psi, E = kq_states(w)
    dims = (w.n,) * 3
    g, eps, inv = run(psi, E, w.nv, dims, w.gcut, Q, route)
    ref = O.eps_inv_path(psi, E, w.nv, dims, w.gcut, L, route="gspace", q=Q)
    assert np.array_equal(g, ref["gvec"])
    assert np.max(np.abs(eps - ref["eps"])) <= 1e-6
    assert np.max(np.abs(inv - ref["epsinv"])) <= 1e-6
    assert abs(inv[0, 0] - ref["epsinv"][0, 0]) <= 1e-6 and abs(ref["epsinv"][0, 0] - 1.0) > 1e-3  # a real head


def test_q_change_takes_effect():
    w = inputs.SMALL
    psi, E = kq_states(w)
    dims = (w.n,) * 3
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, w.nv, cell_L=L)
        ctx.build_PG(w.gcut)
        ctx.eps_inv("cholesky")
        e0 = ctx.view("eps").cpu().numpy().copy()
        ctx.set_q(Q)                         # V(q + G) for the current sphere at once
        ctx.eps_inv("cholesky")
        e1 = ctx.view("eps").cpu().numpy()
        with pytest.raises(gw.GwError):
            ctx.set_q((float("nan"), 0.0, 0.0))
    assert e0[0, 0] == 1.0 and abs(e1[0, 0] - 1.0) > 1e-3   # V(0) := 0 at q = 0 only
    ref = O.eps_inv_path(psi, E, w.nv, dims, w.gcut, L, route="gspace", q=Q)
    assert np.max(np.abs(e1 - ref["eps"])) <= 1e-6
