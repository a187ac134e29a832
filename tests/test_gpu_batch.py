"""Batched path on the GPU: uneven independent systems in one pass (one persistent launch of the
rank-k update, optional CUDA-graph replay, autotuned window length), checked against the
single-instance path (bit for bit) and against the FP64 oracle."""
import json

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# uneven grids (one non-cubic and one ragged), occupied/unoccupied counts and sphere cuts
SYSTEMS = [((10, 10, 10), 3, 20, 5, 71), ((12, 12, 12), 4, 28, 8, 72), ((8, 10, 12), 2, 30, 6, 73),
           ((9, 11, 7), 5, 17, 4, 74)]


def load(dims, nv, nc, seed):
    psi, E = inputs.make_states(0, nv, nc, seed, dims=dims)
    ctx = gw.Context(0)
    ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
    return ctx, psi, E


def single_path(dims, nv, nc, seed, gcut, W=2, L=256, inv_method="newton_tc"):
    ctx, psi, E = load(dims, nv, nc, seed)
    ctx.set_herk_window(W, L)
    ctx.build_P("fp16x3")
    g = ctx.P_to_G(gcut)
    ng = len(g)
    PG = torch.empty((ng, ng), dtype=torch.complex64, device="cuda:0")
    inv = torch.empty((ng, ng), dtype=torch.complex128, device="cuda:0")
    ctx.P_to_G(gcut, PG_out=PG)
    ctx.eps_inv(inv_method, epsinv_out=inv)
    ctx.close()
    return PG.cpu().numpy(), inv.cpu().numpy(), g


@pytest.fixture(scope="module")
def batch_results():
    ctxs, states = [], []
    for dims, nv, nc, gcut, seed in SYSTEMS:
        ctx, psi, E = load(dims, nv, nc, seed)
        ctxs.append(ctx)
        states.append((psi, E))
    b = gw.Batch(ctxs, [s[3] for s in SYSTEMS])
    out = {}
    for mode, graph in (("eager", False), ("graph_first", True), ("graph_capture", True), ("graph_replay", True)):
        b.run(use_graph=graph)
        out[mode] = [(c.view("PG").cpu().numpy(), c.view("epsinv").cpu().numpy()) for c in ctxs]
    out["stats"] = b.stats()
    b.close()
    for c in ctxs:
        c.close()
    return out, states


def test_batch_equals_single_instance_path_bit_for_bit(batch_results):
    out, _ = batch_results
    for (dims, nv, nc, gcut, seed), (PG, inv) in zip(SYSTEMS, out["eager"]):
        PGs, invs, _ = single_path(dims, nv, nc, seed, gcut)
        assert np.array_equal(PG, PGs)
        assert np.array_equal(inv, invs)


def test_batch_cholesky_inverse_bit_for_bit():
    """gw_batch_set_inverse(GW_INV_CHOLESKY): the replayed graph equals the single-instance
    Cholesky path bit for bit, and switching back re-captures the Newton inverse."""
    ctxs = [load(dims, nv, nc, seed)[0] for dims, nv, nc, gcut, seed in SYSTEMS]
    b = gw.Batch(ctxs, [s[3] for s in SYSTEMS])
    b.set_inverse("cholesky")
    for _ in range(3):
        b.run(use_graph=True)
    chol = [c.view("epsinv").cpu().numpy() for c in ctxs]
    b.set_inverse("newton_tc")
    for _ in range(2):
        b.run(use_graph=True)
    tc = [c.view("epsinv").cpu().numpy() for c in ctxs]
    with pytest.raises(gw.GwError):
        b.set_inverse("newton")          # the FP64 Newton iteration is not offered in the batch
    b.close()
    for c in ctxs:
        c.close()
    for (dims, nv, nc, gcut, seed), inv_c, inv_t in zip(SYSTEMS, chol, tc):
        _, ref, _ = single_path(dims, nv, nc, seed, gcut, inv_method="cholesky")
        assert np.array_equal(inv_c, ref)
        assert np.max(np.abs(inv_t - ref)) <= 1e-12


def test_graph_replay_equals_eager(batch_results):
    out, _ = batch_results
    for mode in ("graph_first", "graph_capture", "graph_replay"):
        for (a, ai), (b, bi) in zip(out["eager"], out[mode]):
            assert np.array_equal(a, b) and np.array_equal(ai, bi), mode


def test_batch_against_oracle(batch_results):
    out, states = batch_results
    for (dims, nv, nc, gcut, seed), (psi, E), (PG, inv) in zip(SYSTEMS, states, out["graph_replay"]):
        ref = O.eps_inv_path(psi, E, nv, dims, gcut, 1.0, route="rspace")
        assert np.linalg.norm(PG - ref["Pt"]) / np.linalg.norm(ref["Pt"]) <= 1e-6
        assert np.max(np.abs(inv - ref["epsinv"])) <= 1e-6


def test_batch_stats(batch_results):
    out, _ = batch_results
    st = out["stats"]
    assert st["tiles"] >= len(SYSTEMS) and st["herk_ms"] > 0
    assert st["window_chunks"] == 2 and st["flush_windows"] == 256


def test_autotune_respects_error_target_and_caches(tmp_path):
    ctxs = [load(d, nv, nc, seed)[0] for d, nv, nc, g, seed in SYSTEMS[:2]]
    cache = str(tmp_path / "tune.jsonl")
    with gw.Batch(ctxs, [s[3] for s in SYSTEMS[:2]]) as b:
        st = b.autotune(cache, target_error=1e-6)
        # the candidates whose predicted error x 1.25 <= 1e-6: W = 1, 2, 3 (6.5e-7 x 1.25 at W = 3;
        # W = 4 measures 8.1e-7, x 1.25 above the target)
        assert 1 <= st["window_chunks"] <= 3
        lines = [json.loads(l) for l in open(cache)]
        assert len(lines) == 1 and lines[0]["W"] == st["window_chunks"]
        b.set_window(1, 1)
        st2 = b.autotune(cache, target_error=1e-6)      # reused from the cache, no new line
        assert st2["window_chunks"] == st["window_chunks"]
        assert len(open(cache).read().strip().split("\n")) == 1
        # a tighter target admits only W = 1 (2.9e-7 x 1.25 <= 5e-7 < 4.6e-7 x 1.25) and is cached
        # under its own key
        st3 = b.autotune(cache, target_error=5e-7)
        assert st3["window_chunks"] == 1
        assert len(open(cache).read().strip().split("\n")) == 2
        b.run(use_graph=True)
        b.run(use_graph=True)
    for c in ctxs:
        c.close()


def test_batch_rejects_mixed_or_unloaded_contexts():
    ctx, _, _ = load((8, 8, 8), 2, 6, 5)
    empty = gw.Context(0)
    with pytest.raises(gw.GwError) as e:
        gw.Batch([ctx, empty], [3, 3])
    assert e.value.status == gw.GW_E_NOT_READY
    with pytest.raises(gw.GwError) as e:
        gw.Batch([ctx], [16])                            # sphere leaves the 8^3 grid
    assert e.value.status == gw.GW_E_INVALID
    with pytest.raises(gw.GwError) as e:
        gw.Batch([ctx], [3], precision="tf32x3")
    assert e.value.status == gw.GW_E_UNSUPPORTED
    ctx.close()
    empty.close()
