"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances.  The bar for the plain FP32 path is a relative Frobenius error of 1e-6 on P~; the
split forms must stay within 1e-4.
* FP16X3 (the plain FP32 path: 11+11-bit split, short TMEM windows promoted to FP32) and the
  CUDA-core FP32 path: relative Frobenius error <= 1e-6 on P and P~ at the 12^3 size; element-wise
  max error <= 1e-5 * max|P|.  Inputs are rounded to complex64 (6e-8 relative) and the sums are
  FP32, so the expected error is a few 1e-7.
* BF16X3 (8+8-bit split): <= 1e-4.
* TF32X3 accumulates the whole k range in one TMEM accumulator whose truncating FP32 additions
  cost about 2e-8 per MMA, so its bar scales with k: 5e-6 at k = 112.  TF32X1: 2e-3.
* eps and eps^-1 are FP64 built from FP32 P~: max |error| <= 1e-6 (|V P~| is O(1)); the GPU's own
  eps^-1 times its own eps equals I to 1e-12 (that part is pure FP64).
"""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PLAIN = "fp16x3"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def device_bytes(ptr, nbytes, dtype):
    src = torch.as_tensor(gw.DeviceView(ptr, (nbytes,), "|u1"), device="cuda:0")
    return src.cpu().numpy().view(dtype)


def run(psi, E, nv, dims, gcut=None, prec=PLAIN, method="cholesky", cell_L=1.0, want_P=True, want_F=False):
    dev = torch.device("cuda:0")
    out = {}
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64)).to(dev), E, dims, nv,
                        cell_L=cell_L)
        nr = int(np.prod(dims))
        if want_P:
            P = torch.empty((nr, nr), dtype=torch.complex64, device=dev)
            ctx.build_P(prec, P_out=P)
        else:
            ctx.build_P(prec)
        if want_F:
            ptr, nbytes = ctx.buffer("F")
            torch.cuda.synchronize()
            out["F"] = device_bytes(ptr, nbytes, np.uint8)
            out["nr_pad"] = ctx.dims8()[7]
        if gcut is not None:
            g = ctx.P_to_G(gcut)
            ng = len(g)
            PG = torch.empty((ng, ng), dtype=torch.complex64, device=dev)
            ctx.P_to_G(gcut, PG_out=PG)
            eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
            inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
            ctx.eps_inv(method, eps_out=eps, epsinv_out=inv)
            out.update(gvec=g, PG=PG.cpu().numpy(), eps=eps.cpu().numpy(), epsinv=inv.cpu().numpy())
        ctx.sync()
        if want_P:
            out["P"] = P.cpu().numpy()
    return out


@pytest.fixture(scope="module")
def small():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    P = O.P_rows_loop(psi, E, w.nv, 0, w.nr)
    gvec = O.sphere(dims, w.gcut)
    Pt = O.P_to_G(P, dims, gvec)
    eps = O.eps_build(Pt, gvec, w.cell_L)
    return dict(w=w, psi=psi, E=E, dims=dims, P=P, gvec=gvec, Pt=Pt, eps=eps, epsinv=O.inverse_cholesky(eps))


@pytest.mark.parametrize("prec,tol", [("fp16x3", 1e-6), ("fp32_simt", 1e-6), ("bf16x3", 1e-4), ("tf32x3", 5e-6),
                                      ("tf32x1", 2e-3)])
def test_small_P_matches_C_loop(small, prec, tol):
    w = small["w"]
    P = run(small["psi"], small["E"], w.nv, small["dims"], prec=prec)["P"]
    assert rel(P, small["P"]) <= tol
    if tol <= 1e-6:
        assert np.max(np.abs(P - small["P"])) <= 1e-5 * np.max(np.abs(small["P"]))


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_small_P_hermitian_by_construction(small, prec):
    w = small["w"]
    P = run(small["psi"], small["E"], w.nv, small["dims"], prec=prec)["P"]
    assert np.array_equal(P, np.conj(P.T))
    assert np.all(np.diag(P).imag == 0)


def _decode_tf32(F, nr_pad, nr, k):
    F = F.view(np.float32)
    rr = np.arange(nr)[:, None]
    kk = np.arange(k)[None, :]
    off = (((kk // 8) * 4) * nr_pad + (rr // 8) * 8) * 8 + ((kk % 8) // 4) * 32 + (rr % 8) * 4 + kk % 4
    per = nr_pad * 8
    pl = [F[off + p * per].astype(np.float64) for p in range(4)]
    return (pl[0] + pl[1]) + 1j * (pl[2] + pl[3]), F


def _decode_16(F, nr_pad, nr, k, bf16, npl=4):
    """Block layout of gw.h: per 16-k chunk and 128-row block, the block's planes side by side
    (four: Im hi, Re hi, Im lo, Re lo; six: Im hi, Im lo, Re hi, Re lo, -Im hi, -Im lo)."""
    u = F.view(np.uint16)
    rr = np.arange(nr)[:, None]
    kk = np.arange(k)[None, :]
    nblk = nr_pad // 128
    blk = ((kk // 16) * nblk + rr // 128) * npl
    off = ((rr % 128) // 8) * 128 + ((kk % 16) // 8) * 64 + (rr % 8) * 8 + kk % 8
    if bf16:
        val = lambda x: (x.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        val = lambda x: x.view(np.float16).astype(np.float64)
    slots = {"rh": 1, "rl": 3, "ih": 0, "il": 2} if npl == 4 else {"rh": 2, "rl": 3, "ih": 0, "il": 1}
    pl = {n: val(u[(blk + p) * 2048 + off]) for n, p in slots.items()}
    assert len(u) // (nr_pad * 16 * ((k + 15) // 16)) == npl
    return (pl["rh"] + pl["rl"]) + 1j * (pl["ih"] + pl["il"]), u


def test_small_operand_planes(small):
    """The operand planes decode (layouts documented in gw.h) to the oracle's f: TF32 parts with 13
    low bits zero; FP16 parts that carry one power-of-two scale; zero padding."""
    w = small["w"]
    k = w.nv * w.nc
    f_ref = O.pair_density(small["psi"], small["E"], w.nv).T
    r = run(small["psi"], small["E"], w.nv, small["dims"], prec="tf32x3", want_P=False, want_F=True)
    f, F = _decode_tf32(r["F"], r["nr_pad"], w.nr, k)
    assert rel(f, f_ref) < 1e-6
    assert np.all(F.view(np.uint32) & 0x1FFF == 0)
    assert np.count_nonzero(F) <= 4 * w.nr * k
    r = run(small["psi"], small["E"], w.nv, small["dims"], prec="fp16x3", want_P=False, want_F=True)
    f, u = _decode_16(r["F"], r["nr_pad"], w.nr, k, bf16=False)
    ratio = np.max(np.abs(f)) / np.max(np.abs(f_ref))
    scale = 2.0 ** np.round(np.log2(ratio))                   # one power of two for every value
    assert abs(ratio / scale - 1) < 1e-3
    assert np.max(np.abs(f)) < 2 ** 15                        # FP16 range respected
    assert rel(f / scale, f_ref) < 1e-6
    r = run(small["psi"], small["E"], w.nv, small["dims"], prec="bf16x3", want_P=False, want_F=True)
    f, _ = _decode_16(r["F"], r["nr_pad"], w.nr, k, bf16=True)
    assert rel(f, f_ref) < 1e-4


def test_small_PG_eps_and_inverse(small):
    w = small["w"]
    r = run(small["psi"], small["E"], w.nv, small["dims"], gcut=w.gcut)
    assert np.array_equal(r["gvec"], small["gvec"])
    assert rel(r["PG"], small["Pt"]) <= 1e-6
    assert np.max(np.abs(r["PG"][0])) <= 1e-5 * np.max(np.abs(small["Pt"]))    # orthogonality head
    assert np.max(np.abs(r["eps"] - small["eps"])) <= 1e-6
    assert np.max(np.abs(r["epsinv"] - small["epsinv"])) <= 1e-6
    ng = len(r["gvec"])
    assert np.max(np.abs(r["epsinv"] @ r["eps"] - np.eye(ng))) <= 1e-12
    assert abs(r["epsinv"][0, 0] - 1) <= 1e-12            # V(0) = 0: unit head, zero wings


def test_newton_matches_cholesky(small):
    w = small["w"]
    a = run(small["psi"], small["E"], w.nv, small["dims"], gcut=w.gcut, want_P=False)
    b = run(small["psi"], small["E"], w.nv, small["dims"], gcut=w.gcut, method="newton", want_P=False)
    assert np.max(np.abs(a["epsinv"] - b["epsinv"])) <= 1e-10


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3", "fp32_simt"])
def test_ragged_noncubic_grid(prec):
    """N_r = 693 (not a multiple of any tile), k = 15 (not a multiple of the 8- or 16-wide chunk)."""
    dims = (7, 9, 11)
    nv, nc, gcut = 3, 5, 12
    psi, E = inputs.make_states(0, nv, nc, 31, dims=dims)
    r = run(psi, E, nv, dims, gcut=gcut, prec=prec)
    P = O.P_rspace(psi, E, nv)
    assert rel(r["P"], P) <= 1e-6
    g = O.sphere(dims, gcut)
    assert np.array_equal(r["gvec"], g)
    assert rel(r["PG"], O.P_to_G(P, dims, g)) <= 1e-6


def test_single_pair_rank_one():
    dims = (4, 4, 4)
    psi, E = inputs.make_states(4, 1, 1, 3)
    P = O.P_rspace(psi, E, 1)
    for prec in ("fp16x3", "tf32x3", "fp32_simt"):
        r = run(psi, E, 1, dims, gcut=3, prec=prec)
        assert rel(r["P"], P) <= 1e-6, prec


@pytest.mark.parametrize("W,L", [(1, 1), (3, 2), (64, 4096)])
def test_window_settings_agree(small, W, L):
    """Any window / flush setting computes the same P (window length only trades accuracy)."""
    w = small["w"]
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(small["psi"].astype(np.complex64)).to(dev), small["E"], small["dims"], w.nv)
        ctx.set_herk_window(W, L)
        P = torch.empty((w.nr, w.nr), dtype=torch.complex64, device=dev)
        ctx.build_P("fp16x3", P_out=P)
        ctx.sync()
    assert rel(P.cpu().numpy(), small["P"]) <= 2e-6


def test_plane_wave_closed_form_on_gpu():
    dims = (8, 8, 8)
    mv = [(0, 0, 0), (1, 0, 0)]
    mc = [(0, 1, 0), (1, 1, 1), (-1, 0, 2), (2, -1, 0)]
    Ev, Ec = [-6.0, -1.5], [2.0, 4.0, 9.0, 13.0]
    psi, E = inputs.plane_wave_states(dims, mv + mc, Ev + Ec)
    gcut = 9
    r = run(psi, E, 2, dims, gcut=gcut)
    g = O.sphere(dims, gcut)
    pos = {tuple(x): i for i, x in enumerate(g)}
    expect = np.zeros((len(g), len(g)))
    for iv, a in enumerate(mv):
        for ic, b in enumerate(mc):
            i = pos[tuple(np.array(b) - np.array(a))]
            expect[i, i] += 2.0 / ((Ev[iv] - Ec[ic]) / O.HARTREE_EV)
    assert np.max(np.abs(r["PG"] - expect)) <= 1e-5 * np.max(np.abs(expect))


def test_invalid_arguments_and_call_order():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    with gw.Context(0) as ctx:
        with pytest.raises(gw.GwError) as e:
            ctx.build_P()
        assert e.value.status == gw.GW_E_NOT_READY
        bad = E.copy()
        bad[w.nv - 1] = bad[w.nv] + 1.0        # highest occupied above lowest unoccupied
        with pytest.raises(gw.GwError) as e:
            ctx.load_states(psi.astype(np.complex64), bad, (w.n,) * 3, w.nv)
        assert e.value.status == gw.GW_E_INVALID
        bad = E.copy()
        bad[0] = np.nan
        with pytest.raises(gw.GwError) as e:
            ctx.load_states(psi.astype(np.complex64), bad, (w.n,) * 3, w.nv)
        assert e.value.status == gw.GW_E_INVALID
        # empty sums of Eq. (Pstatic): no occupied or no unoccupied state, or no state at all; a
        # grid outside [2, 64]^3.  All are host checks, made before psi is read.
        for nv_bad in (0, len(E)):
            with pytest.raises(gw.GwError) as e:
                ctx.load_states(psi.astype(np.complex64), E, (w.n,) * 3, nv_bad)
            assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.load_states(np.zeros((0, w.nr), np.complex64), np.zeros(0), (w.n,) * 3, 0)
        assert e.value.status == gw.GW_E_INVALID
        # a grid that does not match psi's rows (the binding) and one outside [2, 64]^3 (the library)
        for dims in ((w.n, w.n, w.n + 1), (1, w.n, w.n * w.n)):
            with pytest.raises(gw.GwError) as e:
                ctx.load_states(psi.astype(np.complex64), E, dims, w.nv)
            assert e.value.status == gw.GW_E_INVALID
        ctx.load_states(psi.astype(np.complex64), E, (w.n,) * 3, w.nv)   # host input path
        with pytest.raises(gw.GwError) as e:
            ctx.P_to_G(8)
        assert e.value.status == gw.GW_E_NOT_READY
        with pytest.raises(gw.GwError) as e:
            ctx.build_P(7)
        assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.set_herk_window(0, 1)
        ctx.build_P()
        with pytest.raises(gw.GwError) as e:
            ctx.P_to_G(36)                      # 4 * 36 >= 12^2: sphere leaves the grid
        assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.P_to_G(-1)
        assert e.value.status == gw.GW_E_INVALID
        # output buffers smaller than the call writes are rejected before the library runs
        with pytest.raises(gw.GwError) as e:
            ctx.build_P(P_out=np.zeros(16, np.complex64))
        assert e.value.status == gw.GW_E_INVALID
        with pytest.raises(gw.GwError) as e:
            ctx.P_to_G(w.gcut, PG_out=np.zeros((4, 4), np.complex64))
        assert e.value.status == gw.GW_E_INVALID
        g = ctx.P_to_G(w.gcut)
        with pytest.raises(gw.GwError) as e:
            ctx.eps_inv("cholesky", epsinv_out=np.zeros((len(g) - 1, len(g)), np.complex128))
        assert e.value.status == gw.GW_E_INVALID
        ctx.eps_inv("cholesky", epsinv_out=np.zeros((len(g), len(g)), np.complex128))


def test_host_complex128_input_matches_device_input(small):
    w = small["w"]
    dev = torch.device("cuda:0")
    outs = []
    for psi in (small["psi"], torch.from_numpy(small["psi"].astype(np.complex64)).to(dev)):
        with gw.Context(0) as ctx:
            ctx.load_states(psi, small["E"], small["dims"], w.nv)
            P = torch.empty((w.nr, w.nr), dtype=torch.complex64, device=dev)
            ctx.build_P(P_out=P)
            ctx.sync()
            outs.append(P.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_non_finite_state_is_reported():
    w = inputs.SMALL
    psi, E = inputs.make_workload_states(w)
    psi = psi.astype(np.complex64)
    psi[3, 100] = np.inf
    with gw.Context(0) as ctx:
        ctx.load_states(psi, E, (w.n,) * 3, w.nv)
        with pytest.raises(gw.GwError) as e:
            ctx.sync()
        assert e.value.status == gw.GW_E_INVALID


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_wait_limit_expires_cleanly_and_context_recovers(prec):
    """A wait limit far below the kernel's run time makes the rank-k update's waits run out:
    the kernel records GW_E_TIMEOUT and returns early; the context stays usable and the next
    call with the default limit reproduces the earlier result bit for bit."""
    dims = (16, 16, 16)
    nv, nc = 16, 512                      # k = 8192: each tile's main loop lasts about a millisecond
    psi, E = inputs.make_states(16, nv, nc, 41)
    nr = 4096
    dev = torch.device("cuda:0")
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, nv)
        P1 = torch.empty((nr, nr), dtype=torch.complex64, device=dev)
        ctx.build_P(prec, P_out=P1)
        ctx.sync()
        ctx.set_wait_limit(1e-6)
        ctx.build_P(prec)
        with pytest.raises(gw.GwError) as e:
            ctx.sync()
        assert e.value.status == gw.GW_E_TIMEOUT
        ctx.set_wait_limit(2000.0)
        P2 = torch.empty((nr, nr), dtype=torch.complex64, device=dev)
        ctx.build_P(prec, P_out=P2)
        ctx.sync()
        assert torch.equal(P1, P2)
    if prec == PLAIN:
        rows = [0, 1777, 4095]
        ref = np.concatenate([O.P_rows_loop(psi, E, nv, r, r + 1) for r in rows])
        assert rel(P1.cpu().numpy()[rows], ref) <= 1e-6


def test_plain_workload_full_size():
    """The 24^3 workload (N_r = 13824, k = 15360) in the launch configuration the benchmark
    times: sampled rows of P against the FP64 loop, all of P~ against Eq. (gpsaceP), eps^-1."""
    w = inputs.PLAIN
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    dev = torch.device("cuda:0")
    rows = [0, 4097, 9000, 13823]
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).to(dev), E, dims, w.nv)
        Pv = torch.empty((w.nr, w.nr), dtype=torch.complex64, device=dev)
        ctx.build_P(PLAIN, P_out=Pv)
        got_rows = Pv[rows].cpu().numpy()
        herm = float((Pv[:512, :512] - Pv[:512, :512].conj().T).abs().max())
        g = ctx.P_to_G(w.gcut)
        ng = len(g)
        PG = torch.empty((ng, ng), dtype=torch.complex64, device=dev)
        ctx.P_to_G(w.gcut, PG_out=PG)
        inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
        ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
    assert herm == 0.0
    ref_rows = np.concatenate([O.P_rows_loop(psi, E, w.nv, r, r + 1) for r in rows])
    assert rel(got_rows, ref_rows) <= 1e-6
    gref = O.sphere(dims, w.gcut)
    assert np.array_equal(g, gref) and ng == 691
    Pt = O.P_gspace(psi, E, w.nv, dims, gref)
    assert rel(PG.cpu().numpy(), Pt) <= 1e-6
    inv_ref = O.inverse_cholesky(O.eps_build(Pt, gref, w.cell_L))
    invh = inv.cpu().numpy()
    assert np.max(np.abs(invh - inv_ref)) <= 1e-6
    assert np.max(np.abs(np.diag(invh) - np.diag(inv_ref))) <= 1e-6
    assert np.max(np.abs(invh @ eps.cpu().numpy() - np.eye(ng))) <= 1e-12
