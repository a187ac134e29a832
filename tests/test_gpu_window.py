"""The error target of the 16-bit rank-k update (gw_set_error_target): the window it picks for each
precision, the errors it then reaches against the oracle's FP64 g-space route of Eq. (gpsaceP),
and its argument checks."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def small():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    g = O.sphere(dims, w.gcut)
    return w, psi, E, dims, O.P_gspace(psi, E, w.nv, dims, g)


@pytest.mark.parametrize("prec,target,W", [("fp16x3", 1e-6, 3), ("fp16x3", 1e-4, 16), ("bf16x3", 1e-4, 16),
                                           ("fp16x3", 5e-7, 1)])
@pytest.mark.parametrize("route", ["rspace", "gspace"])
def test_target_picks_window_and_holds(small, prec, target, W, route):
    w, psi, E, dims, Pt = small
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, w.nv)
        ctx.set_error_target(target)
        if route == "rspace":
            ctx.build_P(prec)
            ctx.P_to_G(w.gcut)
        else:
            ctx.build_PG(w.gcut, prec)
        assert ctx.stats()["window_chunks"] == W
        PG = ctx.view("PG").cpu().numpy()
    assert np.linalg.norm(PG - Pt) / np.linalg.norm(Pt) <= target


def test_target_arguments(small):
    w, psi, E, dims, _ = small
    with gw.Context(0) as ctx:
        ctx.load_states(psi, E, dims, w.nv)
        with pytest.raises(gw.GwError) as e:
            ctx.set_error_target(-1.0)
        assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.set_error_target(1e-7)              # below every window's prediction
        assert e.value.status == gw.GW_E_UNSUPPORTED
        ctx.set_error_target(1e-6)
        with pytest.raises(gw.GwError) as e:
            ctx.build_P("bf16x3")                   # BF16 cannot meet 1e-6
        assert e.value.status == gw.GW_E_UNSUPPORTED
        ctx.set_herk_window(5, 256)                 # an explicit window clears the target
        ctx.build_P("bf16x3")
        assert ctx.stats()["window_chunks"] == 5
        ctx.set_error_target(0.0)                   # back to the explicit window
        ctx.build_P("fp16x3")
        assert ctx.stats()["window_chunks"] == 5
