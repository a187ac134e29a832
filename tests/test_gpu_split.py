"""The split-precision workload at full size: 36^3 grid (N_r = 46656), N_v = 64, N_c = 1000
(k = 64000), N_g = 2007.  The whole 2007 x 2007 P~ against Eq. (gpsaceP) in FP64 (the oracle's
FFT route, itself pinned on the CPU against the entry-by-entry phase sums, and checked here against
them on a spread of G), sampled rows of P against the FP64 loop, and eps^-1 eps = I.

Bars: BF16X3 (8 + 8-bit split) relative error <= 1e-4; FP16X3 <= 1e-6."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def split_case():
    w = inputs.SPLIT
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    g = O.sphere(dims, w.gcut)
    sel = np.array([0, 1, 6, 57, 300, 1000, 1500, len(g) - 1])
    ref = O.P_gspace(psi, E, w.nv, dims, g)
    ent = O.P_gspace_entries(psi, E, w.nv, dims, g[sel])
    assert np.linalg.norm(ref[np.ix_(sel, sel)] - ent) <= 1e-12 * np.linalg.norm(ent)
    rows = list(range(0, w.nr, w.nr // 16))[:16]
    Prows = O.P_rows_loop(psi, E, w.nv, 0, 0)  # warm the C library
    Prows = np.concatenate([O.P_rows_loop(psi, E, w.nv, r, r + 1) for r in rows[:4]])
    return dict(w=w, psi=psi, E=E, dims=dims, g=g, sel=sel, ref=ref, rows=rows[:4], Prows=Prows)


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("fp16x3", 1e-6)])
def test_split_workload(split_case, prec, tol):
    s = split_case
    w = s["w"]
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(s["psi"].astype(np.complex64)).to(dev), s["E"], s["dims"], w.nv)
        ctx.build_P(prec)
        rows = ctx.view("P")[s["rows"]].cpu().numpy()
        g = ctx.P_to_G(w.gcut)
        assert np.array_equal(g, s["g"]) and len(g) == 2007
        ng = len(g)
        PG = ctx.view("PG").cpu().numpy()
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
        resid = float((inv @ eps - torch.eye(ng, dtype=torch.complex128, device=dev)).abs().max())
    ref = s["ref"]
    assert np.linalg.norm(PG - ref) / np.linalg.norm(ref) <= tol
    assert np.linalg.norm(rows - s["Prows"]) / np.linalg.norm(s["Prows"]) <= tol
    assert resid <= 1e-12


def test_split_workload_gspace_route(split_case):
    """The same system by the g-space route (no 17 GB P(r,r')): FP16X3 within 1e-6 on the whole P~."""
    s = split_case
    w = s["w"]
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(s["psi"].astype(np.complex64)).to(dev), s["E"], s["dims"], w.nv)
        g = ctx.build_PG(w.gcut, "fp16x3")
        assert np.array_equal(g, s["g"])
        PG = ctx.view("PG").cpu().numpy()
        ctx.eps_inv("cholesky")
    ref = s["ref"]
    assert np.linalg.norm(PG - ref) / np.linalg.norm(ref) <= 1e-6
