"""The plasmon-pole model of Sec. 5.2 (gw_pp_modes, gw_pp_eval) against the oracle's LAPACK
eigendecomposition of S = sqrt(V)(eps^-1 - I)sqrt(V), its Johnson-sum-rule frequencies and
S(omega), on the library's own eps^-1, plus a plane-wave closed form through the whole path."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def run_pp(psi, E, nv, dims, gcut, nmodes, inv_method="cholesky", cell_L=1.0, q=None, omegas=(0.0, 0.5)):
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, nv, cell_L=cell_L)
        if q is not None:
            ctx.set_q(q)
        g = ctx.build_PG(gcut)
        ng = len(g)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=DEV)
        ctx.eps_inv(inv_method, epsinv_out=inv)
        modes = ctx.pp_modes(nmodes, tol=1e-12)
        S_w = {w: ctx.pp_eval(w, nmodes) for w in omegas}
        psiT = ctx.view("psiT").cpu().numpy()
    return g, inv.cpu().numpy(), modes, S_w, psiT.T


@pytest.mark.parametrize("w,nmodes,inv_method", [(inputs.SMALL, 6, "cholesky"), (inputs.PLAIN, 6, "newton_tc")])
def test_modes_match_oracle(w, nmodes, inv_method):
    """nmodes sits on a gap of the spectrum (the next eigenvalue is far), so the span of the modes
    is unique; sigma to 1e-11 of |sigma_0|, omega^2 to 1e-7, the projector onto the modes to 1e-9,
    and S(omega) from those modes to 1e-7 of max |S|."""
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    g, inv, m, S_w, states = run_pp(psi, E, w.nv, dims, w.gcut, nmodes, inv_method)
    rho = O.density_g(states.astype(np.complex128), w.nv, dims)   # the density of the states the GPU used
    sig, w2, A = O.pp_modes(inv, g, w.cell_L, rho, dims, nmodes + 1)
    assert abs(sig[nmodes] - sig[nmodes - 1]) > 0.2 * abs(sig[nmodes - 1])   # the gap
    sig, w2, A = sig[:nmodes], w2[:nmodes], A[:, :nmodes]
    assert np.max(np.abs(m["sigma"] - sig)) <= 1e-11 * abs(sig[0])
    # modes inside a close cluster are fixed only to residual / gap, which enters omega^2
    assert np.max(np.abs(m["omega2"] - w2) / w2) <= 1e-7
    assert np.max(m["resid"]) <= 1e-12 * abs(sig[0])
    P_gpu = m["A"] @ m["A"].conj().T
    assert np.max(np.abs(P_gpu - A @ A.conj().T)) <= 1e-9
    S_ref = O.pp_S(inv, g, w.cell_L)
    for om, S in S_w.items():
        ref = O.pp_S_omega(sig, w2, A, om)
        assert np.max(np.abs(S - ref)) <= 1e-7 * np.max(np.abs(S_ref))
        assert np.max(np.abs(S - S.conj().T)) <= 1e-12 * np.max(np.abs(S_ref))


def test_plane_wave_closed_form():
    """One occupied plane wave (0,0,0) and one unoccupied (1,0,0): eps is diagonal, S has the one
    entry sigma = -2 V^2 / (dE + 2 V) at G = (1,0,0) (dE = E_c - E_v, Hartree), the density is the
    constant 2 electrons, and the sum rule gives omega^2 = |G|^2 (dE + 2 V)."""
    dims, L = (8, 8, 8), 1.0
    psi, E = inputs.plane_wave_states(dims, [(0, 0, 0), (1, 0, 0)], [-3.0, 5.0])
    g, inv, m, S_w, _ = run_pp(psi, E, 1, dims, 3, 1, omegas=(0.0,))
    dE = (E[1] - E[0]) / 27.211386245988
    G2 = (2 * np.pi / L) ** 2
    V = 4 * np.pi / (L ** 3 * G2)
    want_sig = -2 * V * V / (dE + 2 * V)
    assert abs(m["sigma"][0] - want_sig) <= 1e-6 * abs(want_sig)     # P~ carries FP32 rounding
    assert abs(m["omega2"][0] - G2 * (dE + 2 * V)) <= 1e-6 * G2 * (dE + 2 * V)
    i = int(np.flatnonzero((g == [1, 0, 0]).all(axis=1))[0])
    assert abs(abs(m["A"][i, 0]) - 1) <= 1e-9


def test_finite_q_modes():
    """q != 0: V(q + G) everywhere, the head included; the modes still match the oracle."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    q = (0.25, -0.1, 0.05)
    g, inv, m, S_w, states = run_pp(psi, E, w.nv, dims, w.gcut, 3, q=q, omegas=(0.3,))
    rho = O.density_g(states.astype(np.complex128), w.nv, dims)
    sig, w2, A = O.pp_modes(inv, g, w.cell_L, rho, dims, 3, q=q)
    assert np.max(np.abs(m["sigma"] - sig)) <= 1e-11 * abs(sig[0])
    assert np.max(np.abs(m["omega2"] - w2) / np.abs(w2)) <= 1e-7


def test_pp_call_order_and_arguments():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    with gw.Context(0) as ctx:
        ctx.load_states(psi, E, dims, w.nv)
        ctx.build_PG(w.gcut)
        with pytest.raises(gw.GwError):
            ctx.pp_modes(3)                           # before gw_eps_inv
        ctx.eps_inv("cholesky")
        with pytest.raises(gw.GwError):
            ctx.pp_eval(0.0, 1)                       # before gw_pp_modes
        with pytest.raises(gw.GwError):
            ctx.pp_modes(17)
        ctx.pp_modes(2)
        with pytest.raises(gw.GwError):
            ctx.pp_eval(0.0, 3)                       # more modes than computed
