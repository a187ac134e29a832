"""States given as plane-wave coefficients (gw_load_states_g, Sec. 4.1's u_nk = FFT[u~_nk]) and
the (1/N_k) sum over k-points of P~^q (gw_set_kweight), against the oracle's phase-sum transform
and its k-point sum of Eq. (gpsaceP)."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small_g():
    w = inputs.SMALL
    dims = (w.n,) * 3
    coef, gvec, E = inputs.make_states_g(dims, 8, w.nv, w.nc, 31)
    return w, dims, coef, gvec, E


def test_states_match_phase_sum(small_g):
    w, dims, coef, gvec, E = small_g
    ref = O.states_from_g(coef, gvec, dims)                  # [nb][N_r]
    with gw.Context(0) as ctx:
        ctx.load_states_g(coef, gvec, E, dims, w.nv)          # host complex128
        u = ctx.view("psiT").cpu().numpy().T
        ctx.load_states_g(torch.from_numpy(coef.astype(np.complex64)).to(DEV), gvec, E, dims, w.nv)
        u2 = ctx.view("psiT").cpu().numpy().T
    assert np.max(np.abs(u - ref)) <= 1e-6 * np.max(np.abs(ref))
    assert np.max(np.abs(u2 - ref)) <= 1e-6 * np.max(np.abs(ref))
    assert np.allclose(u.conj() @ u.T, np.eye(u.shape[0]), atol=1e-6)   # still orthonormal


def test_noncubic_grid_and_aliased_indices():
    dims = (10, 12, 14)
    coef, gvec, E = inputs.make_states_g(dims, 6, 3, 20, 32)
    shifted = gvec + np.array(dims) * np.array([1, 0, -1])   # the same grid functions
    ref = O.states_from_g(coef, gvec, dims)
    with gw.Context(0) as ctx:
        ctx.load_states_g(coef, shifted, E, dims, 3)
        u = ctx.view("psiT").cpu().numpy().T
    assert np.max(np.abs(u - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("route", ["gspace", "rspace"])
def test_P_from_g_states_matches_oracle(small_g, route):
    w, dims, coef, gvec, E = small_g
    psi = O.states_from_g(coef, gvec, dims)
    g_ref = O.sphere(dims, w.gcut)
    Pt = O.P_gspace(psi, E, w.nv, dims, g_ref)
    with gw.Context(0) as ctx:
        ctx.load_states_g(coef, gvec, E, dims, w.nv)
        if route == "gspace":
            g = ctx.build_PG(w.gcut)
        else:
            ctx.build_P("fp16x3")
            g = ctx.P_to_G(w.gcut)
        PG = ctx.view("PG").cpu().numpy()
    assert np.array_equal(g, g_ref)
    assert rel(PG, Pt) <= 1e-6


def test_plane_wave_coefficients_closed_form():
    """Occupied = plane wave m_a, unoccupied = plane wave m_b, given as single coefficients:
    P~ is 2/(E_v - E_c) (Hartree) at G = m_b - m_a and zero elsewhere."""
    dims = (8, 8, 8)
    gvec = np.array([(0, 0, 0), (1, 0, 0), (0, 1, 1)])
    coef = np.array([[0, 1, 0], [0, 0, 1]], dtype=np.complex128)   # states m_a = (1,0,0), m_b = (0,1,1)
    E = np.array([-3.0, 5.0])
    with gw.Context(0) as ctx:
        ctx.load_states_g(coef, gvec, E, dims, 1)
        g = ctx.build_PG(3)
        PG = ctx.view("PG").cpu().numpy()
    i = int(np.flatnonzero((g == [-1, 1, 1]).all(axis=1))[0])
    want = 2.0 / ((E[0] - E[1]) / 27.211386245988)
    assert abs(PG[i, i].real - want) <= 1e-6 * abs(want)
    off = PG.copy()
    off[i, i] = 0
    assert np.abs(off).max() <= 1e-6 * abs(want)


def test_load_states_g_arguments():
    dims = (6, 6, 6)
    coef, gvec, E = inputs.make_states_g(dims, 3, 2, 3, 33)
    with gw.Context(0) as ctx:
        bad = gvec.copy()
        bad[1] = bad[0] + np.array([6, 0, 0])                 # aliases plane wave 0
        with pytest.raises(gw.GwError):
            ctx.load_states_g(coef, bad, E, dims, 2)
        with pytest.raises(gw.GwError):                       # more plane waves than grid points
            ctx.load_states_g(np.zeros((5, 300), np.complex128), np.zeros((300, 3), np.int32), E, dims, 2)
        ctx.load_states_g(coef, gvec, E, dims, 2)             # the context is still usable


def test_kpoint_sum_both_routes():
    """Two k-points with weights 1/2: the accumulated P~ equals the oracle's (1/N_k) sum; eps^-1
    is then formed from the sum."""
    w = inputs.SMALL
    dims = (w.n,) * 3
    ka = inputs.make_states(w.n, w.nv, w.nc, 41)
    kb = inputs.make_states(w.n, w.nv, w.nc, 42)
    g_ref = O.sphere(dims, w.gcut)
    Pt = O.P_gspace_ksum([ka, kb], w.nv, dims, g_ref)
    for route in ("gspace", "rspace"):
        with gw.Context(0) as ctx:
            for i, (psi, E) in enumerate((ka, kb)):
                ctx.load_states(psi, E, dims, w.nv)
                ctx.set_kweight(0.5, accumulate=i > 0)
                if route == "gspace":
                    ctx.build_PG(w.gcut)
                else:
                    ctx.build_P("fp16x3")
                    ctx.P_to_G(w.gcut)
            PG = ctx.view("PG").cpu().numpy()
            inv = torch.empty((len(g_ref), len(g_ref)), dtype=torch.complex128, device=DEV)
            ctx.eps_inv("cholesky", epsinv_out=inv)
        assert rel(PG, Pt) <= 1e-6
        ref_inv = O.inverse_cholesky(O.eps_build(Pt, g_ref, w.cell_L))
        assert np.max(np.abs(inv.cpu().numpy() - ref_inv)) <= 1e-6


def test_kpoint_accumulate_needs_a_matching_sum():
    w = inputs.SMALL
    dims = (w.n,) * 3
    psi, E = inputs.make_states(w.n, w.nv, w.nc, 43)
    with gw.Context(0) as ctx:
        ctx.load_states(psi, E, dims, w.nv)
        ctx.set_kweight(1.0, accumulate=True)
        with pytest.raises(gw.GwError) as e:
            ctx.build_PG(w.gcut)                              # nothing to add to yet
        assert e.value.status == gw.GW_E_NOT_READY
        ctx.set_kweight(1.0, accumulate=False)
        ctx.build_PG(w.gcut)
        ctx.set_kweight(1.0, accumulate=True)
        with pytest.raises(gw.GwError):
            ctx.build_PG(w.gcut - 2)                          # another sphere
        with pytest.raises(gw.GwError):
            ctx.set_kweight(float("inf"))
