"""The closure estimate of the band-truncated part of P~ on the GPU (gw_corr_closure) against the
FP64 oracle (oracle.P_closure), and against the exact omitted sum where the estimate is exact
(omitted states that complete the set and share one energy).  Bar: 1e-5 relative Frobenius (the
projector term is an FP16X3 rank-k update, 6.5e-7 at 24^3; the density term is FP64)."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def closure_gpu(psi_in, E_in, nv, E_omit, dims, gcut):
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(np.asarray(psi_in).astype(np.complex64)).cuda(), E_in, dims, nv)
        out = ctx.corr_closure(gcut, E_omit)
        ctx.sync()
        return out.cpu().numpy()


@pytest.mark.parametrize("dims,nv,keep,nc_all,gcut,seed", [((12, 12, 12), 4, 20, 60, 8, 3),
                                                            ((10, 12, 9), 3, 11, 40, 5, 4)])
def test_closure_matches_oracle(dims, nv, keep, nc_all, gcut, seed):
    psi, E = inputs.make_states(0, nv, nc_all, seed, dims=dims)
    n_in = nv + keep
    got = closure_gpu(psi[:n_in], E[:n_in], nv, E[n_in:], dims, gcut)
    g = O.sphere(dims, gcut)
    ref = O.P_closure(psi[:n_in], E[:n_in], nv, E[n_in:], dims, g)
    assert got.shape == ref.shape
    assert rel(got, ref) <= 1e-5
    assert np.max(np.abs(got[0])) <= 1e-5 * np.max(np.abs(ref))


def test_closure_exact_for_a_complete_set_with_one_energy():
    dims, nv, keep = (8, 8, 8), 2, 6
    nr = 512
    psi, E = inputs.make_states(0, nv, nr - nv, 31, dims=dims)
    n_in = nv + keep
    E = E.copy()
    E[n_in:] = 9.0
    got = closure_gpu(psi[:n_in], E[:n_in], nv, E[n_in:], dims, 3)
    g = O.sphere(dims, 3)
    exact = O.P_gspace(psi, E, nv, dims, g) - O.P_gspace(psi[:n_in], E[:n_in], nv, dims, g)
    assert rel(got, exact) <= 1e-5


def test_closure_rejects_bad_input():
    dims, nv = (8, 8, 8), 2
    psi, E = inputs.make_states(0, nv, 10, 5, dims=dims)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        with pytest.raises(gw.GwError) as e:
            ctx.corr_closure(3, np.array([-20.0]))          # below an occupied energy
        assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.corr_closure(3, np.array([5.0]), out=torch.empty((4, 4), dtype=torch.complex64))   # host output
        assert e.value.status == gw.GW_E_INVALID


def test_closure_learned_shape_24cubed():
    """24^3 grid, N_v = 32, 200 kept of 2000 unoccupied states (the learned workload's shape)."""
    n, nv, keep, nc_all, gcut = 24, 32, 200, 2000, 29
    dims = (n,) * 3
    psi, E = inputs.make_states(n, nv, nc_all, 2000)
    n_in = nv + keep
    got = closure_gpu(psi[:n_in], E[:n_in], nv, E[n_in:], dims, gcut)
    g = O.sphere(dims, gcut)
    ref = O.P_closure(psi[:n_in], E[:n_in], nv, E[n_in:], dims, g)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("dims,nv,keep,nc_all,gcut,seed", [((12, 12, 12), 4, 20, 60, 8, 3),
                                                            ((24, 24, 24), 32, 200, 2000, 29, 2000)])
def test_closure_after_build_PG_reuses_its_transforms(dims, nv, keep, nc_all, gcut, seed):
    """After gw_build_PG on the same states and sphere, the closure's projector term takes the
    unoccupied pairs' matrix elements from that call's transforms (rescaled to the closure weight)
    and transforms only the occupied pairs: the same estimate to rounding, against a context that
    transforms every pair itself and against the oracle; another sphere in between falls back."""
    psi, E = inputs.make_states(0, nv, nc_all, seed, dims=dims)
    n_in = nv + keep
    psi_d = torch.from_numpy(np.asarray(psi[:n_in]).astype(np.complex64)).cuda()
    fresh = closure_gpu(psi[:n_in], E[:n_in], nv, E[n_in:], dims, gcut)
    with gw.Context(0) as ctx:
        ctx.load_states(psi_d, E[:n_in], dims, nv)
        ctx.build_PG(gcut)
        reused = ctx.corr_closure(gcut, E[n_in:]).cpu().numpy()
        again = ctx.corr_closure(gcut, E[n_in:]).cpu().numpy()          # Q is still the pair transforms
        ctx.build_PG(gcut - 1)                                         # another sphere, then back
        other = ctx.corr_closure(gcut, E[n_in:]).cpu().numpy()
    assert np.array_equal(reused, again)
    assert rel(reused, fresh) <= 1e-6
    assert np.array_equal(other, fresh)
    # the one-kernel transform leaves the same pair transforms for the closure to reuse
    with gw.Context(0) as ctx:
        ctx.set_transform_kernel("fused")
        ctx.load_states(psi_d, E[:n_in], dims, nv)
        ctx.build_PG(gcut)
        fused = ctx.corr_closure(gcut, E[n_in:]).cpu().numpy()
    assert rel(fused, fresh) <= 1e-6
    if dims[0] == 12:
        ref = O.P_closure(psi[:n_in], E[:n_in], nv, E[n_in:], dims, O.sphere(dims, gcut))
        assert rel(reused, ref) <= 1e-5
