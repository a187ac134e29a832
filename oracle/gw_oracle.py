"""FP64 CPU oracle for the static polarizability -> P~_GG' -> eps -> eps^-1 path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  It shares no code with the CUDA library: it has
its own G-sphere ordering, its own twiddles (through numpy's FFT), its own units and its own
linear algebra.

Every function follows a passage of Kim et al., "Scalable GW software for quasiparticle
properties using OpenAtom" (arXiv 1810.07772), at q = 0 and a single k-point, in Hartree atomic
units with e^2 = 1:

* Eq. (Pstatic), Sec. 2 -- the static polarizability in real space.
* Eq. (fdef), Sec. 4.1 -- the energy-weighted pair densities f_vc(r).
* The outer-product equation right after Eq. (fdef) -- P as a sum of f f^H.
* The row and column FFT equations of Sec. 4.1 -- P(r,r') -> P^(G,r') -> P~(G,G').
* Eq. (gpsaceP), Sec. 4.1 -- the Adler-Wiser g-space sum over states (the second route).
* Sec. 5.1 (static inverse dielectric matrix) -- eps = I - sqrt(V) P~ sqrt(V), V = 4 pi/(Omega |G|^2),
  and the Newton iteration X <- X (2I - A X) the paper uses to invert it.
* Sec. 4.1, u_nk(x) = FFT[u~_nk(g)] -- states given as plane-wave coefficients, transformed to
  the grid (`states_from_g`), and the (1/N_k) sum over k-points of P^q (`P_gspace_ksum`).
* Sec. 5.2, Eqs. (eigdecomp), (ppform), (ppfreq) -- the plasmon-pole model: S = sqrt(V)(eps^-1 - I)
  sqrt(V), its eigenpairs, the Johnson-sum-rule frequencies and S(omega) (`pp_*`).
* Sec. 2 (band truncation of the sum over c in Eq. Pstatic) -- the closure estimate of the omitted
  part from the loaded states and the omitted states' energies (`closure_weights`, `P_closure`).

Readings of the paper taken here (where it is silent or inconsistent):

1. Orientation.  Eq. (Pstatic) pairs psi_c(x) psi_v^*(x) with psi_c^*(x') psi_v(x'); Eq. (fdef) and
   the outer product built from it give the transpose.  The oracle follows Eq. (Pstatic):
   P(r,r') = -sum_k f_k(r) conj(f_k(r')) with f_vc = conj(psi_v) psi_c sqrt(2/(E_c-E_v)).  The
   g-space matrix element is then M_vc(G) = sum_r exp(-i G.r) conj(psi_v(r)) psi_c(r).
2. The factor 2 of Eq. (Pstatic) is the whole spin/time-ordering factor; no extra spin sum.
3. Transform signs: exp(-i G.r) on the row index r and exp(+i G'.r') on the column index r',
   unnormalised (the states are orthonormal on the discrete grid, which absorbs the paper's
   1/sqrt(Omega) factors).
4. Units: energies arrive in eV and are divided by 27.211386245988; the cell is cubic with edge L
   (bohr), Omega = L^3, G = 2 pi m / L for integer m in FFT order.
5. Sphere: all m with |m|^2 <= gcut, ordered by (|m|^2, m1, m2, m3) ascending, so G = 0 is first.
6. Head at q = 0: V(G=0) is set to 0, so eps has a unit head and zero wings.  For q != 0 (given
   in units of 2 pi / L) V(q + G) = 4 pi / (Omega |q + G|^2) for every G; the states are then the
   periodic parts u_{v,k+q} (occupied rows) and u_{c,k} (unoccupied rows) of Sec. 4.1, and the
   transforms are the same as at q = 0.
7. Newton start: alpha = 1 / max_i sum_j |(A A^H)_ij| (the paper's A^T read as A^H for complex A,
   with absolute values so the row sums bound the spectral radius).
8. Plane-wave states: u(r_j) = N_r^(-1/2) sum_g c(g) exp(+i g.r_j), the discrete form of the
   paper's 1/sqrt(Omega) normalisation (unit-norm coefficients give unit-norm grid states); a
   Miller index m and m + n (per axis) are the same grid function.
9. Plasmon-pole frequencies: omega_a^2 = -(1/sigma_a) A_a^H Omega A_a.  The paper prints the
   quotient without the minus sign; with sigma_a < 0 (S is negative semidefinite) and Omega positive
   semidefinite that would give omega^2 < 0.  The sign follows from the sum rule with the pole form
   of Eq. (ppform): int_0^inf w Im S(w) dw = (pi/2) sum_a A sigma omega^2 A^H = -(pi/2) Omega.  The
   density is rho(G) = sum_r e^{-iG.r} rho(r) with rho(r) = 2 sum_v |psi_v(r)|^2 per grid point, so
   rho(0) = 2 N_v is the number of electrons per cell; with it a single-pole eps^-1 = 1 - wp^2/w~^2
   (wp^2 = 4 pi rho(0)/Omega) returns omega = w~ exactly.  g - g' is taken modulo the grid.
10. Band truncation: the paper names the cut of the sum over c as a cost and gives no correction.
   The estimate of the omitted part (`P_closure`) takes the omitted states as unknown members of
   the complement of the loaded ones, each with mean projector (I - Pi)/(N_r - n_in), and uses
   their energies exactly; it is the mean of the omitted sum over such states.
"""
from __future__ import annotations

import ctypes

import numpy as np
import scipy.fft

HARTREE_EV = 27.211386245988


# ----------------------------------------------------------------------------- energies


def to_hartree(E_eV):
    return np.asarray(E_eV, dtype=np.float64) / HARTREE_EV


def pair_weights(E_eV, nv):
    """w_vc = 2 / (E_c - E_v) in 1/Hartree: the energy factor of Eq. (fdef), before the root."""
    E = to_hartree(E_eV)
    return 2.0 / (E[None, nv:] - E[:nv, None])


# ----------------------------------------------------------------------------- real space


def pair_density(psi, E_eV, nv):
    """Eq. (fdef) at q = 0: f_vc(r) = conj(psi_v(r)) psi_c(r) sqrt(2/(E_c - E_v)), row k = v*N_c + c."""
    psi = np.asarray(psi, dtype=np.complex128)
    nb, nr = psi.shape
    nc = nb - nv
    w = pair_weights(E_eV, nv)
    f = np.conj(psi[:nv])[:, None, :] * psi[nv:][None, :, :] * np.sqrt(w)[:, :, None]
    return f.reshape(nv * nc, nr)


def P_from_f(f):
    """The outer product after Eq. (fdef), in the orientation of Eq. (Pstatic):
    P(r, r') = -sum_k f_k(r) conj(f_k(r')).  (The matmul is the only library step.)"""
    f = np.asarray(f, dtype=np.complex128)
    return -(f.T @ np.conj(f))


def P_rspace(psi, E_eV, nv):
    """P(r, r') from the states through f (Eq. fdef and the outer product)."""
    return P_from_f(pair_density(psi, E_eV, nv))


_clib = None


def _load_clib():
    global _clib
    if _clib is None:
        from . import build as _b
        path = _b.build()
        lib = ctypes.CDLL(path)
        lib.oracle_P_rows.restype = ctypes.c_int
        lib.oracle_P_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _clib = lib
    return _clib


def clib_threads() -> int:
    return int(_load_clib().oracle_num_threads())


def P_rows_loop(psi, E_eV, nv, r0, r1):
    """Rows [r0, r1) of Eq. (Pstatic) by the plain FP64 C loop over r, r', v, c."""
    lib = _load_clib()
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    nb, nr = psi.shape
    E = np.ascontiguousarray(to_hartree(E_eV))
    out = np.zeros((r1 - r0, nr), dtype=np.complex128)
    rc = lib.oracle_P_rows(nr, nv, nb - nv, psi.ctypes.data, E.ctypes.data, r0, r1, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_P_rows rejected its arguments")
    return out


def P_quadruple_loop(psi, E_eV, nv):
    """Eq. (Pstatic) as a pure-Python loop over v, c, r, r' (tiny inputs only)."""
    psi = np.asarray(psi, dtype=np.complex128)
    E = to_hartree(E_eV)
    nb, nr = psi.shape
    P = np.zeros((nr, nr), dtype=np.complex128)
    for v in range(nv):
        for c in range(nv, nb):
            for r in range(nr):
                for rp in range(nr):
                    P[r, rp] += (2.0 * np.conj(psi[v, r]) * psi[c, r] * np.conj(psi[c, rp]) * psi[v, rp]
                                 / (E[v] - E[c]))
    return P


# ----------------------------------------------------------------------------- G sphere


def sphere(dims, gcut):
    """Integer G-vectors m (FFT order, each component in [-n/2, n - n/2)) with |m|^2 <= gcut,
    sorted by (|m|^2, m1, m2, m3).  Returns an int64 array of shape (N_g, 3)."""
    ranges = [range(-(n // 2), n - n // 2) for n in dims]
    pts = []
    for a in ranges[0]:
        for b in ranges[1]:
            for c in ranges[2]:
                if a * a + b * b + c * c <= gcut:
                    pts.append((a * a + b * b + c * c, a, b, c))
    pts.sort()
    return np.array([p[1:] for p in pts], dtype=np.int64).reshape(-1, 3)


def states_from_g(coef, gvec, dims):
    """Sec. 4.1's u_nk(x) = sum_g u~_nk(g) e^{i g.x} / sqrt(Omega) on the grid (reading 8):
    u[n][j] = N_r^(-1/2) sum_p coef[n][p] exp(+2 pi i sum_a m_pa j_a / n_a), j in C order.  A plain
    phase sum in FP64 (an [npw x N_r] phase matrix: small grids only)."""
    n1, n2, n3 = dims
    j = np.indices((n1, n2, n3)).reshape(3, -1).astype(np.float64)
    m = np.asarray(gvec, dtype=np.float64)
    phase = np.outer(m[:, 0], j[0] / n1) + np.outer(m[:, 1], j[1] / n2) + np.outer(m[:, 2], j[2] / n3)
    return (np.asarray(coef, dtype=np.complex128) @ np.exp(2j * np.pi * phase)) / np.sqrt(n1 * n2 * n3)


def P_gspace_ksum(kpoints, nv, dims, gvec, weights=None):
    """Sec. 4.1's (1/N_k) sum over k of the one-k-point P~^q: kpoints is a list of (psi, E_eV),
    each psi holding u_{v,k+q} (occupied rows) and u_{c,k}; weights default to 1/N_k."""
    if weights is None:
        weights = [1.0 / len(kpoints)] * len(kpoints)
    out = None
    for (psi, E), w in zip(kpoints, weights):
        t = w * P_gspace(psi, E, nv, dims, gvec)
        out = t if out is None else out + t
    return out


def density_g(psi, nv, dims):
    """rho(G) on the whole grid (reading 9): numpy's forward FFT (e^{-iG.r}) of
    rho(r) = 2 sum_v |psi_v(r)|^2, indexed by m modulo the grid."""
    rho = 2.0 * np.sum(np.abs(np.asarray(psi)[:nv]) ** 2, axis=0).reshape(dims)
    return np.fft.fftn(rho)


def pp_S(epsinv, gvec, cell_L, q=None):
    """Sec. 5.2: S = sqrt(V) (eps^-1 - I) sqrt(V) (Hermitian part)."""
    sv = np.sqrt(coulomb(gvec, cell_L, q))
    S = sv[:, None] * (np.asarray(epsinv) - np.eye(len(gvec))) * sv[None, :]
    return 0.5 * (S + S.conj().T)


def pp_omega_matrix(gvec, cell_L, rhoG, dims, q=None):
    """Omega_gg' = V(q+g) V(q+g') ((q+g).(q+g')) rho(g - g') of Eq. (ppfreq)."""
    V = coulomb(gvec, cell_L, q)
    m = np.asarray(gvec, dtype=np.float64) + (np.zeros(3) if q is None else np.asarray(q, dtype=np.float64))
    k = (2.0 * np.pi / cell_L) * m
    g = np.asarray(gvec)
    d = g[:, None, :] - g[None, :, :]
    rho = rhoG[d[..., 0] % dims[0], d[..., 1] % dims[1], d[..., 2] % dims[2]]
    return V[:, None] * V[None, :] * (k @ k.T) * rho


def pp_modes(epsinv, gvec, cell_L, rhoG, dims, nmodes, q=None):
    """Eq. (eigdecomp) by LAPACK (numpy.linalg.eigh, ascending) and Eq. (ppfreq) with reading 9:
    returns (sigma[:nmodes], omega2[:nmodes], A[:, :nmodes])."""
    S = pp_S(epsinv, gvec, cell_L, q)
    w, A = np.linalg.eigh(S)
    A = A[:, :nmodes]
    Om = pp_omega_matrix(gvec, cell_L, rhoG, dims, q)
    quad = np.real(np.einsum("ga,gh,ha->a", A.conj(), Om, A))
    sig = w[:nmodes]
    # a mode with sigma = 0 (the G = 0 row at q = 0) screens nothing and has no pole: omega^2 := 0
    return sig, np.where(sig != 0, -quad / np.where(sig != 0, sig, 1.0), 0.0), A


def pp_S_omega(sigma, omega2, A, w):
    """Eq. (ppform): S(w) = sum_a A_a sigma_a omega_a^2 / (omega_a^2 - w^2) A_a^H."""
    f = sigma * omega2 / (omega2 - w * w)
    return (A * f) @ A.conj().T


def _flat_index(dims, m):
    n1, n2, n3 = dims
    return ((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (m[:, 2] % n3)


def P_to_G(P, dims, gvec):
    """The two FFT phases of Sec. 4.1 restricted to the sphere:
    P^(G, r') = sum_r exp(-i G.r) P(r, r');  P~(G, G') = sum_r' P^(G, r') exp(+i G'.r').
    numpy's forward FFT carries exp(-i...) and its inverse exp(+i...)/N, undone by the factor N_r."""
    n1, n2, n3 = dims
    nr = n1 * n2 * n3
    idx = _flat_index(dims, gvec)
    Phat = np.fft.fftn(np.asarray(P).reshape(n1, n2, n3, nr), axes=(0, 1, 2)).reshape(nr, nr)[idx]
    Pt = np.fft.ifftn(Phat.reshape(-1, n1, n2, n3), axes=(1, 2, 3)).reshape(-1, nr)[:, idx]
    return Pt * nr


def dft_matrix(dims, gvec):
    """D[g, r] = exp(-i 2 pi (m1 j1/n1 + m2 j2/n2 + m3 j3/n3)) written out element by element."""
    n1, n2, n3 = dims
    j1, j2, j3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    j1, j2, j3 = j1.reshape(-1), j2.reshape(-1), j3.reshape(-1)
    ph = (np.outer(gvec[:, 0], j1) / n1 + np.outer(gvec[:, 1], j2) / n2
          + np.outer(gvec[:, 2], j3) / n3)
    return np.exp(-2j * np.pi * ph)


def P_to_G_direct(P, dims, gvec):
    """Same transform as P_to_G as explicit sums, P~ = D P D^H (tiny inputs)."""
    D = dft_matrix(dims, gvec)
    return D @ np.asarray(P) @ np.conj(D.T)


def matrix_elements(psi, nv, dims, gvec, v_list=None):
    """M_vc(G) = sum_r exp(-i G.r) conj(psi_v(r)) psi_c(r) for the listed v (Eq. gpsaceP's M, read
    in the orientation of Eq. Pstatic).  Returns [len(v_list) * N_c][N_g]."""
    psi = np.asarray(psi, dtype=np.complex128)
    n1, n2, n3 = dims
    nb = psi.shape[0]
    nc = nb - nv
    idx = _flat_index(dims, gvec)
    if v_list is None:
        v_list = range(nv)
    out = []
    for v in v_list:
        rho = np.conj(psi[v])[None, :] * psi[nv:]
        # the library FFT step (scipy's, the same unnormalised exp(-i...) convention as numpy's),
        # on every host core: the 36^3 workload needs 64000 of these transforms
        out.append(scipy.fft.fftn(rho.reshape(nc, n1, n2, n3), axes=(1, 2, 3), workers=-1).reshape(nc, -1)[:, idx])
    return np.concatenate(out, axis=0)


def P_gspace(psi, E_eV, nv, dims, gvec, v_chunk=4):
    """Eq. (gpsaceP): P~(G, G') = sum_vc 2 M_vc(G) conj(M_vc(G')) / (E_v - E_c)."""
    psi = np.asarray(psi, dtype=np.complex128)
    E = to_hartree(E_eV)
    nc = psi.shape[0] - nv
    ng = gvec.shape[0]
    Pt = np.zeros((ng, ng), dtype=np.complex128)
    for v0 in range(0, nv, v_chunk):
        vs = list(range(v0, min(nv, v0 + v_chunk)))
        M = matrix_elements(psi, nv, dims, gvec, vs)
        d = np.concatenate([2.0 / (E[v] - E[nv:]) for v in vs])
        Pt += (M.T * d[None, :]) @ np.conj(M)
    return Pt


def P_gspace_entries(psi, E_eV, nv, dims, gsel):
    """Eq. (gpsaceP) on a chosen set of G only: P~(Ga, Gb) for Ga, Gb in gsel, with
    M_vc(G) = sum_r exp(-i G.r) conj(psi_v(r)) psi_c(r) written as explicit phase sums (no FFT), so
    single entries of large systems can be checked one by one."""
    psi = np.asarray(psi, dtype=np.complex128)
    E = to_hartree(E_eV)
    n1, n2, n3 = dims
    j1, j2, j3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    j1, j2, j3 = j1.reshape(-1), j2.reshape(-1), j3.reshape(-1)
    gsel = np.asarray(gsel).reshape(-1, 3)
    phases = np.exp(-2j * np.pi * (np.outer(gsel[:, 0], j1) / n1 + np.outer(gsel[:, 1], j2) / n2
                                   + np.outer(gsel[:, 2], j3) / n3))          # [ns][N_r]
    ns = len(gsel)
    out = np.zeros((ns, ns), dtype=np.complex128)
    for v in range(nv):
        weighted = phases * np.conj(psi[v])[None, :]                           # [ns][N_r]
        M = weighted @ psi[nv:].T                                              # [ns][N_c]: M_vc(G)
        d = 2.0 / (E[v] - E[nv:])
        out += (M * d[None, :]) @ np.conj(M.T)
    return out


# ----------------------------------------------------------------------------- band truncation


def closure_weights(E_in_eV, nv, E_omit_eV):
    """W_v = sum over the omitted unoccupied states c of 2 / (E_v - E_c), in 1/Hartree (negative):
    the energy factor of Eq. (Pstatic) summed over the states beyond the cut, one per occupied v."""
    E = to_hartree(E_in_eV)
    Eo = to_hartree(E_omit_eV)
    return np.sum(2.0 / (E[:nv, None] - Eo[None, :]), axis=1)


def P_closure(psi_in, E_in_eV, nv, E_omit_eV, dims, gvec):
    """Estimate of the omitted part of Eq. (gpsaceP) when the sum over c stops after the loaded
    states psi_in (occupied first) and only the energies E_omit of the states beyond the cut are
    known.  Written from the closure relation: on the grid sum_n psi_n(r) conj(psi_n(r')) =
    delta_rr' over a complete set, so the omitted states span the complement of the loaded ones,
    and for states drawn without preference inside that complement the mean of
    psi_c(r) conj(psi_c(r')) is (delta_rr' - Pi(r, r')) / (N_r - n_in), Pi = sum_{n loaded}
    psi_n psi_n^H.  Inserted into Eq. (Pstatic) (reading: the omitted c enter only through this
    mean and their known energies):
        dP(r, r') = sum_v W_v / (N_r - n_in) conj(psi_v(r)) psi_v(r') (delta_rr' - Pi(r, r'))
    and, transformed as P~ is,
        dP~(G, G') = [rho_W(G - G') - sum_v W_v sum_{n loaded} M_vn(G) conj(M_vn(G'))] / (N_r - n_in)
    with rho_W(q) = sum_r e^{-i q.r} sum_v W_v |psi_v(r)|^2 and M_vn(G) = sum_r e^{-iG.r}
    conj(psi_v(r)) psi_n(r).  It is exact when the omitted states complete the set and share one
    energy."""
    psi = np.asarray(psi_in, dtype=np.complex128)
    n_in = psi.shape[0]
    n1, n2, n3 = dims
    nr = n1 * n2 * n3
    W = closure_weights(E_in_eV, nv, E_omit_eV)
    g = np.asarray(gvec)
    # term 1: rho_W at every difference G - G' (taken modulo the grid)
    rhoW = np.sum(W[:, None] * np.abs(psi[:nv]) ** 2, axis=0).reshape(n1, n2, n3)
    rhoG = np.fft.fftn(rhoW)
    d = g[:, None, :] - g[None, :, :]
    T1 = rhoG[d[..., 0] % n1, d[..., 1] % n2, d[..., 2] % n3]
    # term 2: the projector on the loaded states, through the matrix elements M_vn for all loaded n
    idx = _flat_index(dims, g)
    T2 = np.zeros((len(g), len(g)), dtype=np.complex128)
    for v in range(nv):
        rho = np.conj(psi[v])[None, :] * psi
        M = np.fft.fftn(rho.reshape(n_in, n1, n2, n3), axes=(1, 2, 3)).reshape(n_in, -1)[:, idx]   # [n][G]
        T2 += W[v] * (M.T @ np.conj(M))
    return (T1 - T2) / (nr - n_in)


# ----------------------------------------------------------------------------- eps


def coulomb(gvec, cell_L, q=None):
    """V_c(q + G) = 4 pi / (Omega |q + G|^2) with G = 2 pi m / L, q = 2 pi q_frac / L and
    Omega = L^3 (Sec. 5.1); V_c := 0 where q + G = 0 (the head at q = 0)."""
    m = np.asarray(gvec, dtype=np.float64)
    if q is not None:
        m = m + np.asarray(q, dtype=np.float64)[None, :]
    m2 = np.sum(m ** 2, axis=1)
    G2 = (2.0 * np.pi / cell_L) ** 2 * m2
    omega = cell_L ** 3
    V = np.zeros_like(G2)
    nz = m2 > 0
    V[nz] = 4.0 * np.pi / (omega * G2[nz])
    return V


def eps_build(Pt, gvec, cell_L, q=None):
    """eps^q_GG' = delta_GG' - sqrt(V(q + G)) P~^q_GG' sqrt(V(q + G')) (Sec. 5.1)."""
    s = np.sqrt(coulomb(gvec, cell_L, q))
    return np.eye(Pt.shape[0], dtype=np.complex128) - s[:, None] * np.asarray(Pt, np.complex128) * s[None, :]


class NotPositiveDefinite(ArithmeticError):
    pass


def cholesky_lower(A):
    """A = L L^H column by column (Cholesky-Crout), raising on a non-positive pivot."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        d = A[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
        if not d > 0.0:
            raise NotPositiveDefinite(f"pivot {j} is {d}")
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ np.conj(L[j, :j])) / L[j, j]
    return L


def forward_substitute(L, B):
    """Solve L Y = B for lower-triangular L, one row at a time."""
    L = np.asarray(L)
    Y = np.zeros(np.shape(B), dtype=np.complex128)
    for i in range(L.shape[0]):
        Y[i] = (B[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def inverse_cholesky(A):
    """A^-1 = L^-H L^-1 from the Cholesky factor (the method fixed for eps^-1 in FP64)."""
    L = cholesky_lower(A)
    Y = forward_substitute(L, np.eye(L.shape[0], dtype=np.complex128))
    return np.conj(Y.T) @ Y


def inverse_newton(A, tol=1e-11, max_iter=100):
    """Sec. 5.1: X_{n+1} = X_n (2I - A X_n), X_0 = alpha A^H, stopped when every entry moves < tol.
    Returns (X, iterations)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    alpha = 1.0 / np.max(np.sum(np.abs(A @ np.conj(A.T)), axis=1))
    X = alpha * np.conj(A.T)
    I2 = 2.0 * np.eye(n)
    for it in range(1, max_iter + 1):
        Xn = X @ (I2 - A @ X)
        if np.max(np.abs(Xn - X)) < tol:
            return Xn, it
        X = Xn
    return X, max_iter


# ----------------------------------------------------------------------------- whole path


def eps_inv_path(psi, E_eV, nv, dims, gcut, cell_L, route="gspace", q=None):
    """States -> P~ -> eps -> eps^-1.  route 'rspace' goes through P(r,r') (small grids),
    'gspace' through Eq. (gpsaceP).  For q != 0 the occupied rows of psi are u_{v,k+q} and the
    unoccupied ones u_{c,k} (Sec. 4.1); the transforms are unchanged.  Returns dict(gvec, Pt, eps,
    epsinv)."""
    gvec = sphere(dims, gcut)
    if route == "rspace":
        Pt = P_to_G(P_rspace(psi, E_eV, nv), dims, gvec)
    else:
        Pt = P_gspace(psi, E_eV, nv, dims, gvec)
    eps = eps_build(Pt, gvec, cell_L, q)
    return {"gvec": gvec, "Pt": Pt, "eps": eps, "epsinv": inverse_cholesky(eps)}
