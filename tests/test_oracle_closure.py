"""Pins for the oracle's closure estimate of the band-truncated part of P~ (Sec. 2; Eq. Pstatic,
Eq. gpsaceP).  The estimate must equal the exact omitted sum when the omitted states complete
the set and share one energy (the closure relation is then an identity), keep the G = 0 row and
column at zero (occupied states are orthogonal to all others), be Hermitian, and be the mean of
the omitted sum over random completions of the loaded states."""
import numpy as np

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import inputs

HA = 27.211386245988


def test_closure_weights_by_hand():
    """One occupied state at -1 Ha, omitted states at +1 and +3 Ha: W = 2/(-2) + 2/(-4) = -1.5."""
    W = O.closure_weights(np.array([-1.0, 0.5]) * HA, 1, np.array([1.0, 3.0]) * HA)
    assert np.allclose(W, [-1.5], rtol=0, atol=1e-14)


def _complete_system(dims, nv, keep, seed):
    nr = int(np.prod(dims))
    psi, E = inputs.make_states(0, nv, nr - nv, seed, dims=dims)    # a full orthonormal basis
    return psi, E, nv + keep


def test_closure_is_exact_for_a_complete_set_with_one_omitted_energy():
    dims, nv, keep = (4, 4, 4), 2, 5
    psi, E, n_in = _complete_system(dims, nv, keep, 11)
    E = E.copy()
    E[n_in:] = 7.0                                  # every omitted state at 7 eV
    g = O.sphere(dims, 2)
    full = O.P_gspace(psi, E, nv, dims, g)
    kept = O.P_gspace(psi[:n_in], E[:n_in], nv, dims, g)
    est = O.P_closure(psi[:n_in], E[:n_in], nv, E[n_in:], dims, g)
    exact = full - kept
    assert np.linalg.norm(exact) > 1e-3
    assert np.linalg.norm(est - exact) <= 1e-12 * np.linalg.norm(exact)


def test_closure_with_uneven_energies_differs_and_keeps_head_zero():
    """With spread omitted energies the estimate is no longer exact, but it stays Hermitian with a
    zero G = 0 row and column, and it still beats the diagonal shift alone."""
    dims, nv, keep = (4, 4, 4), 2, 5
    psi, E, n_in = _complete_system(dims, nv, keep, 12)
    g = O.sphere(dims, 2)
    exact = O.P_gspace(psi, E, nv, dims, g) - O.P_gspace(psi[:n_in], E[:n_in], nv, dims, g)
    est = O.P_closure(psi[:n_in], E[:n_in], nv, E[n_in:], dims, g)
    nr = int(np.prod(dims))
    assert np.linalg.norm(est - exact) > 1e-6 * np.linalg.norm(exact)
    assert np.max(np.abs(est - est.conj().T)) <= 1e-14 * np.max(np.abs(est))
    assert np.max(np.abs(est[0])) <= 1e-14 * np.max(np.abs(est))
    assert np.max(np.abs(est[:, 0])) <= 1e-14 * np.max(np.abs(est))
    diag = np.diag(np.full(len(g), np.sum(O.closure_weights(E[:n_in], nv, E[n_in:])) / (nr - n_in)))
    diag[0, 0] = 0
    assert np.linalg.norm(est - exact) < np.linalg.norm(diag - exact)


def test_closure_is_the_mean_over_random_completions():
    """Fix the loaded states of a 3 x 3 x 4 grid and the omitted energies; draw 3000 random
    orthonormal sets of omitted states inside the complement; the mean of the exact omitted part
    approaches the estimate like 1/sqrt(draws)."""
    dims, nv, keep, n_om = (3, 3, 4), 2, 3, 6
    nr = int(np.prod(dims))
    psi, E = inputs.make_states(0, nv, keep, 21, dims=dims)
    n_in = nv + keep
    rng = np.random.default_rng(5)
    E_om = np.sort(rng.uniform(0.5, 20.0, n_om))
    g = O.sphere(dims, 1)
    est = O.P_closure(psi, E, nv, E_om, dims, g)
    proj = np.eye(nr) - psi.T @ psi.conj()          # onto the complement of the loaded states
    acc = np.zeros_like(est)
    draws = 3000
    for _ in range(draws):
        a = proj @ (rng.standard_normal((nr, n_om)) + 1j * rng.standard_normal((nr, n_om)))
        q, _ = np.linalg.qr(a)
        om = np.concatenate([psi[:nv], q.T])
        acc += O.P_gspace(om, np.concatenate([E[:nv], E_om]), nv, dims, g)
    mean = acc / draws
    spread = np.linalg.norm(est)
    assert np.linalg.norm(mean - est) <= 0.03 * spread      # measured 0.011; without the projector term 0.57
