"""The tensor-core Newton inverse of Sec. 5.1 (gw_eps_inv with GW_INV_NEWTON_TC, gw_zinv_tc) and
the sliced complex GEMM under it (gw_zgemm_tc): integer slices against exact integer products and
FP64 products, the FP16X3 split, and eps^-1 against the oracle's FP64 Cholesky inverse."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def crand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def exact_product(Ar, Ai, Br, Bi):
    """(Ar + i Ai)(Br + i Bi) for int64 matrices, in int64 (no rounding anywhere)."""
    return Ar @ Br - Ai @ Bi, Ar @ Bi + Ai @ Br


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 77, 45), (257, 300, 691), (64, 40, 2100)])
def test_slices_exact_on_small_integers(M, N, K):
    """Entries with |Re|, |Im| <= 31 are one slice each, every product and partial sum is an
    integer below 2^24, so C equals the integer product exactly (K = 2100 uses two K ranges)."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    Ar, Ai = rng.integers(-31, 32, (M, K)), rng.integers(-31, 32, (M, K))
    Br, Bi = rng.integers(-31, 32, (K, N)), rng.integers(-31, 32, (K, N))
    Cr, Ci = exact_product(Ar, Ai, Br, Bi)
    with gw.Context(0) as ctx:
        C = ctx.zgemm_tc(dev(Ar + 1j * Ai), dev(Br + 1j * Bi), "slices").cpu().numpy()
    assert np.array_equal(C.real, Cr.astype(np.float64))
    assert np.array_equal(C.imag, Ci.astype(np.float64))


def test_slices_fp64_accuracy_and_strided_rows():
    """Random FP64 operands (one with rows spread over 2^-20 .. 1): error per entry within
    K 2^-52 max|A| max|B| of the FP64 product, as the slicing bounds it."""
    rng = np.random.default_rng(5)
    M, N, K = 300, 200, 517
    A = crand(rng, M, K) * 2.0 ** rng.uniform(-20, 0, (M, 1))
    Bfull = crand(rng, K, N + 9)
    B = dev(Bfull)[:, :N]                      # row stride N + 9
    with gw.Context(0) as ctx:
        C = ctx.zgemm_tc(dev(A), B, "slices").cpu().numpy()
    ref = A @ Bfull[:, :N]
    bound = K * 2.0 ** -52 * np.abs(A).max() * np.abs(Bfull).max()
    assert np.max(np.abs(C - ref)) <= bound
    assert np.max(np.abs(C - ref)) / np.max(np.abs(ref)) < 1e-14


def test_fp16x3_split():
    rng = np.random.default_rng(6)
    A, B = crand(rng, 200, 333), crand(rng, 333, 150)
    with gw.Context(0) as ctx:
        C = ctx.zgemm_tc(dev(A), dev(B), "fp16x3").cpu().numpy()
    ref = A @ B
    assert np.max(np.abs(C - ref)) / np.max(np.abs(ref)) < 1e-5


def test_arguments_rejected():
    with gw.Context(0) as ctx:
        A = dev(np.eye(4))
        with pytest.raises(gw.GwError):
            ctx.zgemm_tc(A, A, mode=3)
        with pytest.raises(gw.GwError):
            ctx.zgemm_tc(A.cpu(), A.cpu())        # host pointers
        with pytest.raises(gw.GwError):
            ctx.zinv_tc(A.cpu())


def hpd(rng, n, lo, hi):
    Q, _ = np.linalg.qr(crand(rng, n, n))
    lam = rng.uniform(lo, hi, n)
    return (Q * lam) @ Q.conj().T


@pytest.mark.parametrize("n", [1, 93, 200, 517])
def test_zinv_tc_random_hpd(n):
    rng = np.random.default_rng(n)
    A = hpd(rng, n, 1.0, 10.0)
    with gw.Context(0) as ctx:
        try:
            X = ctx.zinv_tc(dev(A)).cpu().numpy()
        finally:
            print(n, ctx.newton_tc_report())
        iters = ctx.stats()["newton_iters"]
        rep = ctx.newton_tc_report()
    ref = np.linalg.inv(A)
    assert np.max(np.abs(X - ref)) <= 1e-12
    assert np.max(np.abs(X @ A - np.eye(n))) <= 1e-12
    assert 0 <= iters < 16 and iters == rep["steps"]
    assert 1 <= rep["refinements"] <= 3 and rep["res_last"] <= 1e-8


def test_zinv_tc_jacobi_start():
    """A = D^1/2 C D^1/2 with C of unit diagonal (eigenvalues 1..3 before the scaling) and D in
    [1, 16]: the Jacobi-scaled start sees C's conditioning (3) instead of A's (21).  In FP64 the
    iteration from 2/(1+u) I needs 9 steps to max |I - A X| < 3e-5 and from the Jacobi start 6;
    the tensor-core phase 1 must stay within one step of the latter."""
    rng = np.random.default_rng(23)
    n = 300
    Q, _ = np.linalg.qr(crand(rng, n, n))
    C = (Q * rng.uniform(1.0, 3.0, n)) @ Q.conj().T
    c = np.real(np.diag(C))
    C = C / np.sqrt(c[:, None] * c[None, :])
    d = rng.uniform(1, 16, n)
    A = C * np.sqrt(d[:, None] * d[None, :])
    with gw.Context(0) as ctx:
        X = ctx.zinv_tc(dev(A)).cpu().numpy()
        rep = ctx.newton_tc_report()
    ref = np.linalg.inv(A)
    assert rep["steps"] <= 7
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(X @ A - np.eye(n))) <= 1e-11


def test_zinv_tc_indefinite_is_numeric_error():
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(crand(rng, 64, 64))
    lam = np.concatenate([rng.uniform(-1.0, -0.5, 8), rng.uniform(1.0, 2.0, 56)])
    A = (Q * lam) @ Q.conj().T
    with gw.Context(0) as ctx:
        with pytest.raises(gw.GwError) as e:
            ctx.zinv_tc(dev(A))
        assert e.value.status == gw.GW_E_NUMERIC
        # the context stays usable
        X = ctx.zinv_tc(dev(np.eye(8) * 2.0)).cpu().numpy()
    assert np.allclose(X, np.eye(8) * 0.5, rtol=0, atol=1e-15)


def eps_pair(w, route):
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, w.nv)
        if route == "gspace":
            g = ctx.build_PG(w.gcut)
        else:
            ctx.build_P("fp16x3")
            g = ctx.P_to_G(w.gcut)
        ng = len(g)
        out = {}
        for m in ("cholesky", "newton_tc"):
            eps = torch.empty((ng, ng), dtype=torch.complex128, device=DEV)
            inv = torch.empty_like(eps)
            ctx.eps_inv(m, eps_out=eps, epsinv_out=inv)
            resid = float((inv @ eps - torch.eye(ng, dtype=torch.complex128, device=DEV)).abs().max())
            out[m] = (eps.cpu().numpy(), inv.cpu().numpy(), resid, ctx.stats()["newton_iters"])
    return out


@pytest.mark.parametrize("w,route", [(inputs.SMALL, "rspace"), (inputs.PLAIN, "gspace")])
def test_eps_inv_newton_tc_matches_cholesky(w, route):
    out = eps_pair(w, route)
    eps, inv_c, res_c, _ = out["cholesky"]
    eps2, inv_t, res_t, iters = out["newton_tc"]
    assert np.array_equal(eps, eps2)
    ref = O.inverse_cholesky(eps)
    assert np.max(np.abs(inv_t - ref)) <= 1e-12
    assert np.max(np.abs(inv_t - inv_c)) <= 1e-12
    assert res_t <= 1e-12
    assert 0 <= iters < 16


def test_eps_inv_graph_replay_matches_eager():
    """gw_eps_inv replays its tensor-core inverse from a captured CUDA graph (graph-safe steps,
    device flags) and recaptures when the order changes; gw_zinv_tc queues the same kernels
    eagerly with host reads of the convergence flag (and, for another order, drops the graph,
    whose tables it overwrites).  The kernels that run are the same, so the results agree bit for
    bit."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, w.nv)
        for gcut in (w.gcut, w.gcut - 2, w.gcut):
            g = ctx.build_PG(gcut)
            ng = len(g)
            eps = torch.empty((ng, ng), dtype=torch.complex128, device=DEV)
            first = torch.empty_like(eps)
            ctx.eps_inv("newton_tc", eps_out=eps, epsinv_out=first)          # capture
            again = torch.empty_like(eps)
            ctx.eps_inv("newton_tc", epsinv_out=again)                      # replay
            eager = ctx.zinv_tc(eps)
            other = ctx.zinv_tc(torch.eye(5, dtype=torch.complex128, device=DEV) * 2.0)  # another order
            last = torch.empty_like(eps)
            ctx.eps_inv("newton_tc", epsinv_out=last)                       # recapture
            a, b, c, d, e = (t.cpu().numpy() for t in (first, again, eager, last, eps))
            assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)
            assert np.max(np.abs(a - O.inverse_cholesky(e))) <= 1e-12
            assert np.allclose(other.cpu().numpy(), np.eye(5) * 0.5, rtol=0, atol=1e-15)


def test_eps_inv_graph_finishes_an_eps_that_needs_more_steps():
    """gw_eps_inv's graph queues 8 FP16X3 steps.  An eps with condition number ~2e3 needs about 14
    from the Jacobi-scaled start; the graph's refinements then fail with the phase-1 flag, and the
    call finishes the inverse with the eager form.  The result matches the FP64 Cholesky inverse of
    the same eps, and a well-conditioned eps afterwards still takes the graph."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, dims, w.nv)
        g = ctx.build_PG(w.gcut)
        ng = len(g)
        PG_plain = ctx.view("PG").clone()
        # eps = I + M, M Hermitian positive semidefinite with eigenvalues 1e-3 .. 2e3, zero row and
        # column 0 (V(0) = 0): P~ = -M / (sqrt(V) sqrt(V)^T) off the head
        rng = np.random.default_rng(3)
        Q, _ = np.linalg.qr(rng.standard_normal((ng - 1, ng - 1)) + 1j * rng.standard_normal((ng - 1, ng - 1)))
        M = (Q * np.geomspace(1e-3, 2e3, ng - 1)) @ Q.conj().T
        sv = np.sqrt(O.coulomb(g, 1.0))
        P = np.zeros((ng, ng), dtype=np.complex128)
        P[1:, 1:] = -M / np.outer(sv[1:], sv[1:])
        ctx.view("PG").copy_(torch.from_numpy(P.astype(np.complex64)))
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=DEV)
        inv_c = torch.empty_like(eps)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv_c)
        inv_n = torch.empty_like(eps)
        ctx.eps_inv("newton_tc", epsinv_out=inv_n)
        rep = ctx.newton_tc_report()
        e, c, n = (t.cpu().numpy() for t in (eps, inv_c, inv_n))
        ctx.view("PG").copy_(PG_plain)
        ctx.eps_inv("newton_tc", epsinv_out=inv_n)
        rep2 = ctx.newton_tc_report()
    assert np.linalg.cond(e) > 1e3
    assert rep["steps"] > 8                 # more than the graph queues: the eager form ran
    assert np.linalg.norm(n - c) / np.linalg.norm(c) <= 1e-11
    assert np.max(np.abs(n @ e - np.eye(ng))) <= 1e-9
    assert rep2["steps"] <= 8


def test_eps_inv_refuses_a_stream_under_capture():
    """gw_eps_inv synchronises its stream to read the device status back, which a stream under
    capture does not allow: the call returns GW_E_INVALID before it queues anything into the
    caller's graph, the caller's capture stays valid, and the context works afterwards."""
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    s = torch.cuda.Stream(device=DEV)
    with gw.Context(0, s) as ctx:
        with torch.cuda.stream(s):
            ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(DEV), E, (w.n,) * 3, w.nv)
            ctx.build_PG(w.gcut)
            ref = torch.empty((ctx.ng, ctx.ng), dtype=torch.complex128, device=DEV)
            ctx.eps_inv("newton_tc", epsinv_out=ref)
            x = torch.zeros(4, device=DEV)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin(capture_error_mode="relaxed")
            try:
                x.add_(1.0)
                with pytest.raises(gw.GwError) as ei:
                    ctx.eps_inv("newton_tc")
            finally:
                g.capture_end()
        assert ei.value.status == gw.GW_E_INVALID
        g.replay()                       # the caller's graph holds its own work only
        torch.cuda.synchronize()
        assert torch.equal(x.cpu(), torch.ones(4))
        with torch.cuda.stream(s):
            again = torch.empty_like(ref)
            ctx.eps_inv("newton_tc", epsinv_out=again)
        s.synchronize()
        assert torch.equal(again, ref)
