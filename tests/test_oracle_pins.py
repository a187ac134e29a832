"""Pins for the FP64 oracle: what the paper and the mathematics fix, independent of the oracle.

Each test names the passage (Kim et al., arXiv 1810.07772) or the mathematical fact it checks and
is chosen so that a plausible slip in the oracle (a dropped term, a flipped sign or exponent, a
transposed operand, a wrong unit) fails at least one of them.
"""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import inputs

TINY = (3, 3, 2)


def tiny_states(seed=7, nv=2, nc=3, dims=TINY):
    return inputs.make_states(0, nv, nc, seed, dims=dims)


# --------------------------------------------------------------------------- real-space P


def test_quadruple_loop_equals_C_loop_and_outer_product():
    """Eq. (Pstatic) three ways on a tiny grid: pure-Python loop, the C loop, and f f^H."""
    psi, E = tiny_states()
    nv = 2
    P_py = O.P_quadruple_loop(psi, E, nv)
    P_c = O.P_rows_loop(psi, E, nv, 0, psi.shape[1])
    P_mm = O.P_rspace(psi, E, nv)
    assert np.max(np.abs(P_c - P_py)) < 1e-14 * np.max(np.abs(P_py))
    assert np.max(np.abs(P_mm - P_py)) < 1e-14 * np.max(np.abs(P_py))


def test_C_loop_row_block_matches_full():
    psi, E = inputs.make_states(4, 2, 5, 11)
    P = O.P_rspace(psi, E, 2)
    rows = O.P_rows_loop(psi, E, 2, 5, 17)
    assert np.allclose(rows, P[5:17], rtol=0, atol=1e-15 * np.max(np.abs(P)))


def test_hand_computed_single_pair():
    """One occupied and one unoccupied state on a 2-point grid, evaluated by hand:
    psi_v = (1, 1)/sqrt2, psi_c = (1, -1)/sqrt2, E_v = -1 Ha, E_c = +1 Ha.
    rho = conj(psi_v) psi_c = (1, -1)/2, so P = 2/(E_v - E_c) rho rho^H = -(1/4) [[1, -1], [-1, 1]]."""
    s = 1 / np.sqrt(2)
    psi = np.array([[s, s], [s, -s]], dtype=np.complex128)
    E = np.array([-1.0, 1.0]) * O.HARTREE_EV
    P = O.P_rspace(psi, E, 1)
    expect = -0.25 * np.array([[1, -1], [-1, 1]])
    assert np.allclose(P, expect, atol=1e-15)
    assert np.allclose(O.P_rows_loop(psi, E, 1, 0, 2), expect, atol=1e-15)


def test_hand_computed_orientation_with_complex_states():
    """Orientation of Eq. (Pstatic) on a 3-point grid, by hand: psi_v = (1, 1, 1)/sqrt3,
    psi_c = (1, w, w^2)/sqrt3 with w = exp(2 pi i/3), E_c - E_v = 2 Ha.  Then
    rho = conj(psi_v) psi_c = (1, w, w^2)/3 and P[a][b] = -(1/9) w^(a-b), so
    P[0][1] = -(1/9) exp(-2 pi i/3) = (1 + i sqrt3)/18; the transposed orientation would give
    (1 - i sqrt3)/18."""
    s = 1 / np.sqrt(3)
    w = np.exp(2j * np.pi / 3)
    psi = np.array([[s, s, s], [s, s * w, s * w * w]], dtype=np.complex128)
    E = np.array([-1.0, 1.0]) * O.HARTREE_EV
    for P in (O.P_rspace(psi, E, 1), O.P_rows_loop(psi, E, 1, 0, 3)):
        assert abs(P[0, 1] - (1 + 1j * np.sqrt(3)) / 18) < 1e-15
        assert abs(P[1, 0] - (1 - 1j * np.sqrt(3)) / 18) < 1e-15
        assert abs(P[2, 2] - (-1 / 9)) < 1e-15


def test_paper_outer_product_orientation_is_transpose():
    """Reading 1: the form -sum f^*(x) f(x') printed after Eq. (fdef) is P^T of Eq. (Pstatic)."""
    psi, E = tiny_states(seed=3)
    f = O.pair_density(psi, E, 2)
    P = O.P_from_f(f)
    P_paper = -(np.conj(f).T @ f)
    assert np.allclose(P_paper, P.T, atol=1e-15)


def test_P_hermitian_negative_semidefinite_rank():
    psi, E = inputs.make_states(6, 3, 9, 5)
    P = O.P_rspace(psi, E, 3)
    assert np.max(np.abs(P - np.conj(P.T))) < 1e-16
    lam = np.linalg.eigvalsh(P)
    assert lam.max() < 1e-15 * np.abs(lam).max()
    assert np.sum(np.abs(lam) > 1e-12 * np.abs(lam).max()) == 27     # rank k = nv * nc


def test_phase_invariance_and_partition_linearity():
    psi, E = inputs.make_states(4, 2, 6, 9)
    P = O.P_rspace(psi, E, 2)
    ph = np.exp(1j * np.linspace(0.1, 5.0, psi.shape[0]))
    assert np.allclose(O.P_rspace(psi * ph[:, None], E, 2), P, atol=1e-16)
    A = np.r_[0:2, 2:5]
    B = np.r_[0:2, 5:8]
    PA = O.P_rspace(psi[A], E[A], 2)
    PB = O.P_rspace(psi[B], E[B], 2)
    assert np.allclose(PA + PB, P, atol=1e-16)


def test_pair_weights_units():
    """eV -> Hartree with 27.211386245988 eV/Ha, and w = 2/(E_c - E_v) > 0."""
    E = np.array([-O.HARTREE_EV, 0.0, O.HARTREE_EV])
    w = O.pair_weights(E, 1)
    assert np.allclose(w, [[2.0 / 1.0, 2.0 / 2.0]])


# --------------------------------------------------------------------------- sphere and FFTs


def test_sphere_counts_and_order():
    """Lattice points with |m|^2 <= K: 1 + r3(1) + ... ; r3 = 6, 12, 8, 6, 24, 24, 0, 12 for 1..8."""
    g = O.sphere((12, 12, 12), 8)
    assert g.shape == (93, 3)
    assert tuple(g[0]) == (0, 0, 0)
    m2 = np.sum(g * g, axis=1)
    assert np.all(np.diff(m2) >= 0)
    assert len(O.sphere((24, 24, 24), 29)) == 691
    assert len(O.sphere((36, 36, 36), 61)) == 2007
    # even grid: -n/2 is in range, +n/2 is not
    g4 = O.sphere((4, 4, 4), 4)
    assert (-2, 0, 0) in map(tuple, g4) and (2, 0, 0) not in map(tuple, g4)


def test_fft_route_equals_explicit_dft():
    psi, E = inputs.make_states(0, 2, 4, 21, dims=(4, 3, 5))
    dims = (4, 3, 5)
    P = O.P_rspace(psi, E, 2)
    g = O.sphere(dims, 3)
    assert np.allclose(O.P_to_G(P, dims, g), O.P_to_G_direct(P, dims, g), atol=1e-14)


def test_plane_wave_closed_form():
    """Plane waves psi = exp(i G.r)/sqrt(N_r): rho_vc = exp(i (G_c - G_v).r)/N_r, so
    M_vc(G) = delta(G, G_c - G_v) and P~ is 2/(E_v - E_c) at (G_c - G_v, G_c - G_v) only.
    Pins the sign of both exponents, the orientation, the factor 2 and the unit conversion."""
    dims = (6, 6, 6)
    mv = [(0, 0, 0), (1, 0, 0)]
    mc = [(0, 1, 0), (1, 1, 1), (-1, 0, 2)]
    Ev = [-5.0, -2.0]
    Ec = [3.0, 7.0, 11.0]
    psi, E = inputs.plane_wave_states(dims, mv + mc, Ev + Ec)
    g = O.sphere(dims, 9)
    expect = np.zeros((len(g), len(g)), dtype=np.complex128)
    pos = {tuple(x): i for i, x in enumerate(g)}
    for iv, a in enumerate(mv):
        for ic, b in enumerate(mc):
            d = tuple(np.array(b) - np.array(a))
            i = pos[d]
            expect[i, i] += 2.0 / ((Ev[iv] - Ec[ic]) / O.HARTREE_EV)
    Pr = O.P_to_G(O.P_rspace(psi, E, 2), dims, g)
    Pg = O.P_gspace(psi, E, 2, dims, g)
    assert np.max(np.abs(Pr - expect)) < 1e-12
    assert np.max(np.abs(Pg - expect)) < 1e-12
    # closed-form eps^-1 on those entries (V = 4 pi/(|G|^2 Omega), L = 1)
    eps = O.eps_build(expect, g, 1.0)
    inv = O.inverse_cholesky(eps)
    for iv, a in enumerate(mv):
        for ic, b in enumerate(mc):
            d = np.array(b) - np.array(a)
            i = pos[tuple(d)]
            V = 4 * np.pi / ((2 * np.pi) ** 2 * np.sum(d * d))
            assert abs(inv[i, i] - 1.0 / (1.0 - V * expect[i, i].real)) < 1e-13


def test_parseval_on_full_grid():
    """With every G of the grid kept, P~ = D P D^H with D unitary up to sqrt(N_r):
    tr P~ = N_r tr P and ||P~||_F = N_r ||P||_F."""
    dims = (4, 4, 3)
    psi, E = inputs.make_states(0, 2, 5, 4, dims=dims)
    P = O.P_rspace(psi, E, 2)
    g = O.sphere(dims, 10 ** 6)
    assert len(g) == 48
    Pt = O.P_to_G(P, dims, g)
    nr = 48
    assert abs(np.trace(Pt) - nr * np.trace(P)) < 1e-13
    assert abs(np.linalg.norm(Pt) - nr * np.linalg.norm(P)) < 1e-13


def test_head_row_vanishes_by_orthogonality():
    """G = 0 row and column of P~ vanish at q = 0 because occupied and unoccupied states are
    orthogonal: M_vc(0) = <psi_v|psi_c> = 0."""
    psi, E = inputs.make_states(8, 3, 10, 13)
    g = O.sphere((8, 8, 8), 6)
    Pt = O.P_gspace(psi, E, 3, (8, 8, 8), g)
    scale = np.max(np.abs(Pt))
    assert np.max(np.abs(Pt[0])) < 1e-14 * scale
    assert np.max(np.abs(Pt[:, 0])) < 1e-14 * scale


def test_rspace_route_equals_gspace_route():
    """Sec. 4.1: the r-space route (P then row/column FFTs) and Eq. (gpsaceP) agree exactly on a
    grid that holds the states (a discrete identity)."""
    dims = (6, 5, 4)
    psi, E = inputs.make_states(0, 3, 7, 17, dims=dims)
    g = O.sphere(dims, 5)
    Pr = O.P_to_G(O.P_rspace(psi, E, 3), dims, g)
    Pg = O.P_gspace(psi, E, 3, dims, g)
    assert np.linalg.norm(Pr - Pg) < 1e-14 * np.linalg.norm(Pg)


# --------------------------------------------------------------------------- eps and inverse


def test_coulomb_values():
    g = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]])
    V = O.coulomb(g, 2.0)
    # G = 2 pi m / 2 = pi m, Omega = 8: V = 4 pi / (8 pi^2 |m|^2) = 1/(2 pi |m|^2)
    assert V[0] == 0.0
    assert np.allclose(V[1:], [1 / (2 * np.pi), 1 / (4 * np.pi), 1 / (6 * np.pi)])


def test_eps_hpd_and_inverse_against_library():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    res = O.eps_inv_path(psi, E, w.nv, (w.n,) * 3, w.gcut, w.cell_L)
    eps = res["eps"]
    assert eps.shape == (93, 93)
    assert np.max(np.abs(eps - np.conj(eps.T))) < 1e-14
    lam = np.linalg.eigvalsh(eps)
    assert lam.min() > 1 - 1e-12            # -sqrt(V) P~ sqrt(V) is PSD, so eps >= I
    assert abs(eps[0, 0] - 1) < 1e-15 and np.max(np.abs(eps[0, 1:])) < 1e-15
    inv = res["epsinv"]
    assert np.max(np.abs(inv @ eps - np.eye(93))) < 1e-12
    assert np.max(np.abs(inv - np.linalg.inv(eps))) < 1e-12
    L = O.cholesky_lower(eps)
    assert np.max(np.abs(L - np.linalg.cholesky(eps))) < 1e-13


def test_newton_iteration_matches_cholesky():
    """Sec. 5.1 Newton iteration X <- X(2I - AX) converges to the same inverse."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    res = O.eps_inv_path(psi, E, w.nv, (w.n,) * 3, w.gcut, w.cell_L)
    X, it = O.inverse_newton(res["eps"], tol=1e-11)
    assert it < 40
    assert np.max(np.abs(X - res["epsinv"])) < 1e-11


def test_newton_start_for_a_general_complex_matrix():
    """Reading 7: the start alpha A^H (with |.| in alpha) makes A X0 Hermitian positive definite, so
    the iteration converges for any nonsingular A, here a non-normal, non-Hermitian complex matrix
    (the start alpha A^T would diverge on it: A A^T has eigenvalues of negative real part)."""
    A = np.array([[1j, 0.3, 0.0], [0.0, 2j, 0.1 - 0.2j], [0.05, 0.0, -1.5j]])
    X, it = O.inverse_newton(A, tol=1e-14)
    assert it < 100
    assert np.max(np.abs(X @ A - np.eye(3))) < 1e-12
    assert np.max(np.abs(X - np.linalg.inv(A))) < 1e-12
    # alpha from the row sums of |A A^H|: here the signed row sums cancel to 0.01, and a start
    # 100 A would diverge (A X0 would reach 361 I on one eigenvector)
    A = np.array([[1.0, -0.9], [-0.9, 1.0]], dtype=np.complex128)
    X, it = O.inverse_newton(A, tol=1e-14)
    assert it < 100
    assert np.max(np.abs(X - np.linalg.inv(A))) < 1e-12


def test_cholesky_rejects_indefinite():
    """An indefinite matrix and a singular positive semidefinite one (second pivot exactly 0) both
    have no Cholesky factor with a positive diagonal."""
    for A in ([[1.0, 2.0], [2.0, 1.0]], [[1.0, 1j], [-1j, 1.0]]):
        with pytest.raises(O.NotPositiveDefinite):
            O.cholesky_lower(np.array(A, dtype=np.complex128))


def test_small_workload_rspace_vs_gspace():
    """The 12^3 workload end to end: both routes agree to FP64 rounding."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    a = O.eps_inv_path(psi, E, w.nv, dims, w.gcut, w.cell_L, route="rspace")
    b = O.eps_inv_path(psi, E, w.nv, dims, w.gcut, w.cell_L, route="gspace")
    assert np.linalg.norm(a["Pt"] - b["Pt"]) < 1e-13 * np.linalg.norm(b["Pt"])
    assert np.max(np.abs(a["epsinv"] - b["epsinv"])) < 1e-13


def test_selected_entries_equal_full_gspace_route():
    """P_gspace_entries (explicit phase sums on chosen G) equals the FFT-based Eq. (gpsaceP) on the
    same entries, and the r-space route on a tiny grid."""
    dims = (6, 5, 4)
    psi, E = inputs.make_states(0, 3, 8, 23, dims=dims)
    g = O.sphere(dims, 5)
    sel = np.array([0, 3, 7, len(g) - 1])
    full = O.P_gspace(psi, E, 3, dims, g)
    part = O.P_gspace_entries(psi, E, 3, dims, g[sel])
    assert np.max(np.abs(part - full[np.ix_(sel, sel)])) < 1e-15 * np.max(np.abs(full)) * 10
    Pr = O.P_to_G(O.P_rspace(psi, E, 3), dims, g)
    assert np.max(np.abs(part - Pr[np.ix_(sel, sel)])) < 1e-13


def test_finite_q_closed_forms():
    """q != 0 (Sec. 4.1 and 5.1).  (a) u_v = u_c = 1/sqrt(N_r), allowed when the two sets belong to
    k + q and k: M(G) is a Kronecker delta at G = 0, so P~ has only a head entry 2/(E_v - E_c) and
    eps^q_00 = 1 + 4 pi * 2 / (Omega |q|^2 (E_c - E_v)), with V(q) = 4 pi / (Omega |2 pi q / L|^2).
    (b) plane waves m_a, m_b: the single entry sits at G = m_b - m_a with V(q + G)."""
    dims, L, q = (6, 6, 6), 1.7, (0.25, -0.1, 0.05)
    Eh = lambda e: e / 27.211386245988  # noqa: E731
    psi, E = inputs.plane_wave_states(dims, [(0, 0, 0), (0, 0, 0)], [-2.0, 3.0])
    r = O.eps_inv_path(psi, E, 1, dims, 3, L, route="gspace", q=q)
    g = r["gvec"]
    assert np.array_equal(g[0], [0, 0, 0])
    want_P = 2.0 / (Eh(E[0]) - Eh(E[1]))
    assert abs(r["Pt"][0, 0] - want_P) <= 1e-12 * abs(want_P)
    assert np.abs(r["Pt"]).sum() - abs(r["Pt"][0, 0]) <= 1e-12 * abs(want_P)
    q2 = (2 * np.pi / L) ** 2 * np.sum(np.asarray(q) ** 2)
    e00 = 1.0 + 4 * np.pi * 2.0 / (L ** 3 * q2 * (Eh(E[1]) - Eh(E[0])))
    assert abs(r["eps"][0, 0] - e00) <= 1e-12 * e00
    assert abs(r["epsinv"][0, 0] - 1.0 / e00) <= 1e-12
    # (b) plane waves at distinct m: entry at m_b - m_a, with |q + G|
    psi, E = inputs.plane_wave_states(dims, [(1, 0, 0), (0, 1, 1)], [-1.0, 4.0])
    r = O.eps_inv_path(psi, E, 1, dims, 3, L, route="gspace", q=q)
    i = int(np.flatnonzero((r["gvec"] == [-1, 1, 1]).all(axis=1))[0])
    qg2 = (2 * np.pi / L) ** 2 * np.sum((np.array([-1, 1, 1]) + np.asarray(q)) ** 2)
    eii = 1.0 + 4 * np.pi * 2.0 / (L ** 3 * qg2 * (Eh(E[1]) - Eh(E[0])))
    assert abs(r["epsinv"][i, i] - 1.0 / eii) <= 1e-12
    # and the q -> 0 limit of V keeps the q = 0 convention (head 0) only at q = 0 itself
    assert O.coulomb(np.array([[0, 0, 0]]), L)[0] == 0.0
    assert O.coulomb(np.array([[0, 0, 0]]), L, q)[0] > 0.0


def test_states_from_g_plane_wave_translation():
    """One coefficient at m: the grid state has constant modulus N_r^-1/2 and picks up
    exp(2 pi i m_a / n_a) under a one-point shift along axis a (this fixes the sign, the axis order
    and the C-order index), and it sums to zero over the grid unless m = 0 (mod n)."""
    dims = (6, 5, 4)
    nr = 6 * 5 * 4
    for m in [(1, 0, 0), (0, -2, 1), (2, 1, -1), (0, 0, 0)]:
        u = O.states_from_g(np.array([[1.0 + 0j]]), np.array([m]), dims)[0].reshape(dims)
        assert np.allclose(np.abs(u), nr ** -0.5, atol=1e-15)
        for a in range(3):
            shifted = np.roll(u, -1, axis=a)     # u at j + e_a
            assert np.allclose(shifted, u * np.exp(2j * np.pi * m[a] / dims[a]), atol=1e-14)
        assert abs(u.sum()) < 1e-12 or m == (0, 0, 0)


def test_states_from_g_unitary_and_equals_inverse_fft():
    """Orthonormal coefficient rows give orthonormal grid states (Parseval), and the phase sum
    equals N_r^(1/2) times numpy's inverse FFT of the coefficients scattered on the grid (an
    independent route: library FFT, modular index placement); m and m + n alias."""
    dims = (8, 6, 5)
    coef, gvec, _ = inputs.make_states_g(dims, 5, 3, 9, 4)
    u = O.states_from_g(coef, gvec, dims)
    assert np.allclose(u.conj() @ u.T, np.eye(12), atol=1e-13)
    grid = np.zeros((12,) + dims, dtype=np.complex128)
    for p, m in enumerate(gvec):
        grid[:, m[0] % dims[0], m[1] % dims[1], m[2] % dims[2]] = coef[:, p]
    ref = np.sqrt(np.prod(dims)) * np.fft.ifftn(grid, axes=(1, 2, 3)).reshape(12, -1)
    assert np.allclose(u, ref, atol=1e-13)
    shifted = gvec + np.array(dims) * np.array([1, -1, 2])
    assert np.allclose(O.states_from_g(coef, shifted, dims), u, atol=1e-12)


def test_ksum_identical_points_and_linearity():
    """The (1/N_k) sum over k of identical k-points is the one-point result; with two different
    point sets it is linear in the weights."""
    w = inputs.SMALL
    dims = (w.n,) * 3
    g = O.sphere(dims, w.gcut)
    a = inputs.make_states(w.n, w.nv, w.nc, 5)
    b = inputs.make_states(w.n, w.nv, w.nc, 6)
    Pa = O.P_gspace(a[0], a[1], w.nv, dims, g)
    assert np.allclose(O.P_gspace_ksum([a, a, a], w.nv, dims, g), Pa, atol=1e-15)
    Pb = O.P_gspace(b[0], b[1], w.nv, dims, g)
    assert np.allclose(O.P_gspace_ksum([a, b], w.nv, dims, g, [0.25, 0.75]), 0.25 * Pa + 0.75 * Pb, atol=1e-15)


def test_pp_single_pole_closed_form():
    """Sec. 5.2 with a diagonal single-pole eps^-1 = 1 - wp^2 / w_g^2 (wp^2 = 4 pi rho(0)/Omega) and
    a constant density: every mode is one G and its Johnson-sum-rule frequency is w_g (this fixes
    the sign of Eq. ppfreq, the V factors, |q+G|^2 and the density normalisation rho(0) = N_el)."""
    dims, L = (8, 8, 8), 1.3
    g = O.sphere(dims, 3)[1:]                     # no G = 0 (V(0) = 0 at q = 0)
    n = len(g)
    nel = 6.0
    rhoG = np.zeros(dims, dtype=np.complex128)
    rhoG[0, 0, 0] = nel
    wp2 = 4 * np.pi * nel / L ** 3
    wt2 = np.linspace(2.0, 9.0, n) * wp2          # distinct poles, eps^-1 - 1 in (-1, 0)
    inv = np.diag(1.0 - wp2 / wt2).astype(np.complex128)
    sig, w2, A = O.pp_modes(inv, g, L, rhoG, dims, n)
    for a in range(n):
        gi = int(np.argmax(np.abs(A[:, a])))
        assert abs(abs(A[gi, a]) - 1) < 1e-12
        assert abs(w2[a] - wt2[gi]) <= 1e-12 * wt2[gi]
    assert np.all(sig < 0)
    # fewer modes than G vectors: the most negative sigma first (the leading modes of Sec. 5.2),
    # here the five smallest of the closed-form diagonal -V(g) wp^2 / w_g^2
    V = O.coulomb(g, L)
    s_diag = -V * wp2 / wt2
    sig5, _, A5 = O.pp_modes(inv, g, L, rhoG, dims, 5)
    order = np.argsort(s_diag)[:5]
    assert np.max(np.abs(sig5 - s_diag[order])) <= 1e-12 * np.max(np.abs(s_diag))
    assert np.all(np.abs(np.abs(A5[order, np.arange(5)]) - 1) < 1e-12)
    # away from w = 0 the model follows the single-oscillator form eps^-1(w) - 1 = wp^2 / (w^2 - w_g^2)
    # (its w = 0 value is the static eps^-1 above), so S(w) = V(g) wp^2 / (w^2 - w_g^2) on the
    # diagonal: below every pole, between two poles and above them all
    for w_sq in (0.5 * wp2, 5.0 * wp2, 20.0 * wp2):
        S = O.pp_S_omega(sig, w2, A, np.sqrt(w_sq))
        want = V * wp2 / (w_sq - wt2)
        assert np.max(np.abs(np.diag(S) - want)) <= 1e-10 * np.max(np.abs(want))
        assert np.max(np.abs(S - np.diag(np.diag(S)))) <= 1e-12 * np.max(np.abs(want))


def test_pp_density_and_S_omega_limits():
    """Occupied plane waves give a constant density, rho(G) = 2 N_v at G = 0 only; S(w) from every
    mode is S at w = 0 and vanishes as w grows; all-mode S(w) is Hermitian."""
    dims = (6, 6, 6)
    psi, E = inputs.plane_wave_states(dims, [(0, 0, 0), (1, 0, 0), (0, 1, 0)], [-3.0, -2.0, 4.0])
    rhoG = O.density_g(psi, 2, dims)
    assert abs(rhoG[0, 0, 0] - 4.0) < 1e-12
    rhoG0 = rhoG.copy()
    rhoG0[0, 0, 0] = 0
    assert np.max(np.abs(rhoG0)) < 1e-12
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    d3 = (w.n,) * 3
    r = O.eps_inv_path(psi, E, w.nv, d3, w.gcut, w.cell_L, route="gspace")
    g = O.sphere(d3, w.gcut)
    rho = O.density_g(psi, w.nv, d3)
    assert abs(rho[0, 0, 0] - 2 * w.nv) < 1e-12
    sig, w2, A = O.pp_modes(r["epsinv"], g, w.cell_L, rho, d3, len(g))
    S = O.pp_S(r["epsinv"], g, w.cell_L)
    keep = np.abs(sig) > 1e-14                    # the G = 0 null mode carries no pole
    S0 = O.pp_S_omega(sig[keep], w2[keep], A[:, keep], 0.0)
    assert np.max(np.abs(S0 - S)) < 1e-12 * np.max(np.abs(S))
    Sinf = O.pp_S_omega(sig[keep], w2[keep], A[:, keep], 1e6)
    assert np.max(np.abs(Sinf)) < 1e-6 * np.max(np.abs(S))
    assert np.all(w2[keep] > 0)
