"""The sphere transforms of Sec. 4.1 (e^{+iG.r} on rows of P in gw_P_to_G, e^{-iG.r} on the pair
densities in gw_build_PG) on grids that reach every branch of the paired sums: odd and even axis
lengths (with and without the middle term x_{n/2}), the register stage 1 (compiled n3: 24, 27)
and the generic one (n3 = 11, 13), non-cubic grids.  Each P~ is compared with the oracle's FP64
route of Eq. (gpsaceP), which shares nothing with the kernels."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


GRIDS = [
    ((27, 27, 27), 40),   # compiled odd n3, odd n1 and n2: no middle term anywhere
    ((9, 15, 27), 16),    # odd n1, n2 with the compiled odd stage 1
    ((7, 9, 24), 12),     # compiled even n3 (middle term in stage 1 only)
    ((12, 10, 13), 8),    # generic odd n3, even n1 and n2 (middle terms in stages 2 and 3)
    ((11, 11, 11), 20),   # generic stage 1, all odd
]


@pytest.mark.parametrize("dims,gcut", GRIDS)
@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_paired_transforms_match_oracle(dims, gcut, route):
    nv, nc = 3, 9
    psi, E = inputs.make_states(0, nv, nc, 61 + sum(dims), dims=dims)
    g_ref = O.sphere(dims, gcut)
    Pt = O.P_gspace(psi, E, nv, dims, g_ref)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, nv)
        if route == "rspace":
            ctx.build_P("fp16x3")
            g = ctx.P_to_G(gcut)
        else:
            g = ctx.build_PG(gcut)
        PG = ctx.view("PG").cpu().numpy()
    assert np.array_equal(g, g_ref)
    assert rel(PG, Pt) <= 1e-6
    # the G = 0 row vanishes at q = 0 (occupied and unoccupied states are orthogonal)
    i0 = int(np.flatnonzero((g_ref == 0).all(axis=1))[0])
    assert np.max(np.abs(Pt[i0])) <= 1e-12 * np.linalg.norm(Pt)
    assert np.max(np.abs(PG[i0])) <= 1e-6 * np.linalg.norm(Pt)


# At q = 0, square planes (n2 = n3 <= 27, a compiled size) take the stages 1 and 2 with
# compile-time twiddles by default, and a compiled n1 takes stage 3 with them;
# GW_TRANSFORM_TABLES runs the same sums with twiddle tables.
CONST_CASES = [
    ((12, 12, 12), 8),    # even N: middle terms x_{N/2} in every stage
    ((16, 16, 16), 20),
    ((10, 18, 18), 14),   # n1 != n2 = n3 (stage 3 from tables)
    ((16, 12, 18), 10),   # n2 != n3 (stages 1 and 2 from tables, stage 3 constant)
    ((27, 27, 27), 40),   # odd N
    ((20, 20, 20), 1),    # M = 1: seven G-vectors
    ((9, 12, 12), 8),     # odd n1 with even N: an odd task count (a last pair of one plane)
    ((15, 16, 16), 12),   # odd n1 again, both passes through the asynchronous plane staging
    ((24, 24, 24), 58),   # the largest sphere of the constant form: 15 m3 values, 185 disk points
]


@pytest.mark.parametrize("dims,gcut", CONST_CASES)
@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_constant_twiddles_match_tables_and_oracle(dims, gcut, route):
    nv, nc = 3, 9
    psi, E = inputs.make_states(0, nv, nc, 7 + sum(dims), dims=dims)
    g_ref = O.sphere(dims, gcut)
    Pt = O.P_gspace(psi, E, nv, dims, g_ref)
    out = {}
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, nv)
        for kind in ("two_kernel", "tables"):
            ctx.set_transform_kernel(kind)
            if route == "rspace":
                ctx.build_P("fp16x3")
                g = ctx.P_to_G(gcut)
            else:
                g = ctx.build_PG(gcut)
            assert np.array_equal(g, g_ref)
            out[kind] = ctx.view("PG").cpu().numpy()
    # the same FP32 sums in the same order; the twiddles differ only where the table's FP64 cosine
    # of an exact zero (pi/2, ...) left ~1e-17
    assert rel(out["two_kernel"], out["tables"]) <= 1e-7
    assert rel(out["two_kernel"], Pt) <= 1e-6
