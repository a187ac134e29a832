"""gw_eps_inv_noalloc: the allocation-free FP64 inverse for callers that cannot call cudaMalloc
(device memory owned by another allocator, loops that must not pay cudaFree's device-wide sync).

It must agree with the inverse that gw_eps_inv returns for the same eps, on two calls in a row
of different sizes (the static workspace keeps the previous call's contents), and reject orders
above its fixed maximum.  This file is collected last, so a run that stops at the first failure
has already run every other test."""

import numpy as np
import pytest

from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def eps_and_inverse(dims, nv, nc, seed, gcut):
    """eps and eps^-1 from the existing path (gw_eps_inv) for a seeded system."""
    psi, E = inputs.make_states(0, nv, nc, seed, dims=dims)
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, nv)
        ctx.build_P()
        g = ctx.P_to_G(gcut)
        ng = len(g)
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
        ctx.sync()
    return eps, inv


def call_noalloc(eps, out):
    stream = torch.cuda.current_stream().cuda_stream
    return gw.lib().gw_eps_inv_noalloc(eps.data_ptr(), eps.shape[0], out.data_ptr(), stream)


def test_noalloc_inverse_matches_gw_eps_inv_twice_in_a_row():
    cases = [((12, 12, 12), 4, 28, 1, 8), ((14, 12, 10), 6, 40, 9, 20)]
    results = []
    for dims, nv, nc, seed, gcut in cases:
        eps, inv = eps_and_inverse(dims, nv, nc, seed, gcut)
        assert eps.shape[0] <= 512
        results.append((eps, inv))
    assert results[0][0].shape[0] != results[1][0].shape[0]   # the second call has another order
    for eps, inv in results:
        out = torch.full_like(eps, float("nan"))
        st = call_noalloc(eps, out)
        assert st == gw.GW_OK
        torch.cuda.synchronize()
        diff = float((out - inv).abs().max())
        assert diff <= 1e-12
        I = torch.eye(eps.shape[0], dtype=torch.complex128, device=eps.device)
        assert float((out @ eps - I).abs().max()) <= 1e-12


def test_noalloc_rejects_orders_above_its_maximum():
    big = torch.eye(513, dtype=torch.complex128, device="cuda:0")
    out = torch.empty_like(big)
    assert call_noalloc(big, out) == gw.GW_E_INVALID
    ok = torch.eye(512, dtype=torch.complex128, device="cuda:0") * 2.0
    out = torch.empty_like(ok)
    assert call_noalloc(ok, out) == gw.GW_OK
    torch.cuda.synchronize()
    assert float((out - 0.5 * torch.eye(512, dtype=torch.complex128, device="cuda:0")).abs().max()) <= 1e-15


def test_noalloc_reports_a_bad_pivot_then_recovers():
    """-I has a negative first pivot: the status word in the shared array says GW_E_NUMERIC.  The
    next call, on 2I of another order, must clear that word and return GW_OK with 0.5 I."""
    dev = torch.device("cuda:0")
    neg = -torch.eye(40, dtype=torch.complex128, device=dev)
    out = torch.empty_like(neg)
    assert call_noalloc(neg, out) == gw.GW_E_NUMERIC
    two = 2.0 * torch.eye(57, dtype=torch.complex128, device=dev)
    out = torch.full_like(two, float("nan"))
    assert call_noalloc(two, out) == gw.GW_OK
    torch.cuda.synchronize()
    assert float((out - 0.5 * torch.eye(57, dtype=torch.complex128, device=dev)).abs().max()) <= 1e-15


def test_noalloc_rejects_host_pointers():
    """Pointers that are not device memory of the current GPU are refused before any launch."""
    host = torch.eye(8, dtype=torch.complex128)
    out = torch.empty_like(host)
    assert call_noalloc(host, out) == gw.GW_E_INVALID
