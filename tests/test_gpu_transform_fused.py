"""The one-kernel sphere transform (GW_TRANSFORM_FUSED: rows streamed plane by plane into shared
memory, axes j1, j2, j3 transformed there with the j / n - j pairing) against the two-kernel form
and the FP64 oracle: the row and column passes of gw_P_to_G, the pair-density rows of gw_build_PG
and of the closure estimate, on cubic, mixed and ragged grids (the ragged one takes the two-kernel
form), and the bounded waits."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(ctx, kind, route, gcut):
    ctx.set_transform_kernel(kind)
    if route == "rspace":
        ctx.build_P("fp16x3")
        g = ctx.P_to_G(gcut)
    else:
        g = ctx.build_PG(gcut, "fp16x3")
    ctx.sync()
    return g, ctx.view("PG").cpu().numpy()


CASES = [((12, 12, 12), 4, 28, 8, 1), ((10, 12, 9), 3, 30, 5, 2), ((8, 8, 8), 2, 20, 5, 3),
         ((16, 16, 16), 8, 120, 13, 4), ((7, 9, 11), 3, 20, 3, 5)]


@pytest.mark.parametrize("dims,nv,nc,gcut,seed", CASES)
@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_fused_matches_two_kernel_and_oracle(dims, nv, nc, gcut, seed, route):
    psi, E = inputs.make_states(0, nv, nc, seed, dims=dims)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        g2, PG2 = run(ctx, "two_kernel", route, gcut)
        g1, PG1 = run(ctx, "fused", route, gcut)
    assert np.array_equal(g1, g2)
    ref = O.P_gspace(psi, E, nv, dims, O.sphere(dims, gcut))
    assert rel(PG1, ref) <= 1e-6
    assert rel(PG1, PG2) <= 5e-7


def test_fused_closure_matches_two_kernel():
    dims, nv, keep, nc_all, gcut = (12, 12, 12), 4, 20, 60, 8
    psi, E = inputs.make_states(0, nv, nc_all, 3, dims=dims)
    n_in = nv + keep
    out = {}
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi[:n_in].astype(np.complex64)).cuda(), E[:n_in], dims, nv)
        for kind in ("two_kernel", "fused"):
            ctx.set_transform_kernel(kind)
            out[kind] = ctx.corr_closure(gcut, E[n_in:]).cpu().numpy()
    assert rel(out["fused"], out["two_kernel"]) <= 1e-6


def test_fused_full_size_24cubed():
    """The 24^3 workload through both routes with the fused transforms, against Eq. (gpsaceP); the
    row pass reads P from HBM once."""
    w = inputs.PLAIN
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, w.nv)
        g, PGr = run(ctx, "fused", "rspace", w.gcut)
        _, PGg = run(ctx, "fused", "gspace", w.gcut)
    ref = O.P_gspace(psi, E, w.nv, dims, g)
    assert rel(PGr, ref) <= 1e-6
    assert rel(PGg, ref) <= 1e-6


def test_fused_wait_limit_expires_cleanly():
    """A wait limit far below the transform's run time: GW_E_TIMEOUT, and the context then
    reproduces the earlier P~ bit for bit."""
    dims, nv, nc, gcut = (16, 16, 16), 8, 120, 13
    psi, E = inputs.make_states(0, nv, nc, 7, dims=dims)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        ctx.set_transform_kernel("fused")
        ctx.build_P("fp16x3")
        ctx.P_to_G(gcut)
        ctx.sync()
        PG1 = ctx.view("PG").clone()
        ctx.set_wait_limit(1e-6)
        ctx.P_to_G(gcut)
        with pytest.raises(gw.GwError) as e:
            ctx.sync()
        assert e.value.status == gw.GW_E_TIMEOUT
        ctx.set_wait_limit(2000.0)
        ctx.P_to_G(gcut)
        ctx.sync()
        assert torch.equal(PG1, ctx.view("PG"))
