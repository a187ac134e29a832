"""The batched path at the exact shapes of the eight-system workload: grids 16^3, 18^3, 20^3,
24^3, 24^3, 27^3, 30^3, 32^3 with N_v = 8 .. 48 and N_c = 100 .. 800, sphere cuts
floor((n / 4.4)^2) (N_g = 203 .. 1575).  One persistent launch walks tens of thousands of tiles
across all instances (several tiles per CTA); the pass is replayed from a CUDA graph.  Every
instance's whole P~ is compared with Eq. (gpsaceP) in FP64, and its eps^-1 with eps."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

NG = [203, 257, 389, 691, 691, 949, 1357, 1575]   # lattice points |m|^2 <= floor((n / 4.4)^2)


def test_batch_workload_every_instance_against_oracle():
    ws = inputs.batch_workloads()
    assert [w.n for w in ws] == [16, 18, 20, 24, 24, 27, 30, 32]
    assert [w.nc for w in ws] == [100 * (i + 1) for i in range(8)]
    states = [inputs.make_workload_states(w) for w in ws]
    ctxs = []
    for w, (psi, E) in zip(ws, states):
        c = gw.Context(0)
        c.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, (w.n,) * 3, w.nv)
        ctxs.append(c)
    b = gw.Batch(ctxs, [w.gcut for w in ws], precision="fp16x3")
    for _ in range(3):                 # eager, capture, replay: the replay's results are checked
        b.run(use_graph=True)
    torch.cuda.synchronize()
    tiles = b.stats()["tiles"]
    got = []
    for c in ctxs:
        ng = c.ng
        eps = c.view("eps").clone()
        inv = c.view("epsinv").clone()
        resid = float((inv @ eps - torch.eye(ng, dtype=torch.complex128, device="cuda:0")).abs().max())
        got.append((c.view("PG").cpu().numpy(), resid))
    b.close()
    for c in ctxs:
        c.close()
    assert tiles > 10 * 152, "the persistent walk should give every CTA many tiles"
    for w, (psi, E), (PG, resid), ng in zip(ws, states, got, NG):
        dims = (w.n,) * 3
        g = O.sphere(dims, w.gcut)
        assert len(g) == ng == PG.shape[0]
        ref = O.P_gspace(psi, E, w.nv, dims, g)
        err = np.linalg.norm(PG - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, f"{w.name}: P~ relative error {err:.3e}"
        assert abs(PG[0]).max() <= 1e-5 * abs(PG).max()       # G = 0 row: occupied and unoccupied orthogonal
        assert resid <= 1e-10, f"{w.name}: |eps^-1 eps - I| = {resid:.3e}"
