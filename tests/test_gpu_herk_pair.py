"""The rank-k update on CTA pairs (GW_HERK_PAIR: 2-SM tensor-core MMAs, 256 x 128 complex tiles)
against the one-CTA kernel and the FP64 oracle.

Both kernels issue the same products in the same order for every element of P (per 16-k chunk:
Ai Bi and Ai Br, hi*hi + hi*lo + lo*hi, then Ar Br and -Ar Bi), so P must agree bit for bit;
negating the B operand (the pair kernel's -Im planes) instead of the A operand (the one-CTA
kernel's negate bit) changes no bit, since every product and sum is sign-symmetric.  Against the
FP64 loop of Eq. (Pstatic) the FP16X3 bar is 1e-6 relative (as in test_gpu_parity)."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_1810_07772_gb300 import gw, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def build(ctx, kind, prec, window=None):
    nr = int(np.prod(ctx.dims))
    ctx.set_herk_kernel(kind)
    if window:
        ctx.set_herk_window(*window)
    P = torch.empty((nr, nr), dtype=torch.complex64, device="cuda:0")
    ctx.build_P(prec, P_out=P)
    ctx.sync()
    return P


CASES = [((12, 12, 12), 4, 28, 1), ((7, 9, 11), 3, 20, 5), ((8, 8, 8), 2, 5, 6)]


@pytest.mark.parametrize("dims,nv,nc,seed", CASES)
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("window", [None, (8, 256), (2, 1)])
def test_pair_equals_single_bit_for_bit(dims, nv, nc, seed, prec, window):
    """Cubic, ragged (N_r = 693 in a 768-row padding) and tiny grids; the default window, a window
    longer than the pipeline (its own window commit) and flushes after every window."""
    psi, E = inputs.make_states(0, nv, nc, seed, dims=dims)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        Ps = build(ctx, "single", prec, window)
        Pp = build(ctx, "pair", prec, window)
        assert ctx.stats()["herk_tiles"] == len([1 for I in range((ctx.dims8()[7]) // 256)
                                                 for J in range(ctx.dims8()[7] // 128) if J >= 2 * I])
    assert torch.equal(Ps, Pp)
    if prec == "fp16x3":
        ref = O.P_rows_loop(psi, E, nv, 0, int(np.prod(dims)))
        assert rel(Pp.cpu().numpy(), ref) <= 1e-6


def test_pair_operand_holds_negated_im_planes():
    """The pair kernel's operand has six planes per 128-row block and 16-k chunk (Im hi, Im lo,
    Re hi, Re lo, -Im hi, -Im lo); the last two are the first two with the sign bit flipped, and
    the four-plane decoding of the first four gives the same f as the one-CTA kernel's operand."""
    from test_gpu_parity import _decode_16
    dims, nv, nc = (12, 12, 12), 4, 28
    psi, E = inputs.make_states(0, nv, nc, 1, dims=dims)
    k = nv * nc
    nr = int(np.prod(dims))
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        nr_pad = ctx.dims8()[7]
        kpad = (k + 15) // 16 * 16
        got = {}
        for kind, npl in (("pair", 6), ("single", 4)):
            build(ctx, kind, "fp16x3")
            ptr, nbytes = ctx.buffer("F")
            F = torch.as_tensor(gw.DeviceView(ptr, (nbytes,), "|u1"), device="cuda:0").view(torch.int16)
            F = F[: kpad * nr_pad * npl].clone()
            got[kind] = F
        F6 = got["pair"].view(kpad // 16, nr_pad // 128, 6, 2048)
        assert torch.equal(F6[:, :, 4], F6[:, :, 0] ^ -32768)
        assert torch.equal(F6[:, :, 5], F6[:, :, 1] ^ -32768)
        assert int((F6[:, :, 0] != 0).sum()) > 0
    f6, _ = _decode_16(got["pair"].cpu().numpy().view(np.uint8), nr_pad, nr, k, False, npl=6)
    f4, _ = _decode_16(got["single"].cpu().numpy().view(np.uint8), nr_pad, nr, k, False, npl=4)
    assert np.array_equal(f6, f4)
    f_ref = O.pair_density(psi, E, nv).T
    scale = 2.0 ** np.round(np.log2(np.max(np.abs(f4)) / np.max(np.abs(f_ref))))
    assert rel(f4 / scale, f_ref) < 1e-6


def test_pair_full_size_24cubed():
    """The 24^3 workload (N_r = 13824, k = 15360, 2970 pairs): equal to the one-CTA kernel bit for
    bit, sampled rows against the FP64 loop, and P~ against Eq. (gpsaceP)."""
    w = inputs.PLAIN
    psi, E = inputs.make_workload_states(w)
    dims = (w.n,) * 3
    rows = [0, 4097, 9000, 13823]
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, w.nv)
        Ps = build(ctx, "single", "fp16x3")
        Pp = build(ctx, "pair", "fp16x3")
        assert ctx.stats()["herk_tiles"] == 2970
        same = torch.equal(Ps, Pp)
        got_rows = Pp[rows].cpu().numpy()
        del Ps
        g = ctx.P_to_G(w.gcut)
        PG = ctx.view("PG").cpu().numpy()
    assert same
    ref_rows = np.concatenate([O.P_rows_loop(psi, E, w.nv, r, r + 1) for r in rows])
    assert rel(got_rows, ref_rows) <= 1e-6
    assert rel(PG, O.P_gspace(psi, E, w.nv, dims, g)) <= 1e-6


def test_pair_wait_limit_expires_cleanly_and_context_recovers():
    """A wait limit far below the kernel's run time: both CTAs of every pair run out of their
    waits, record GW_E_TIMEOUT, drain and leave together; the context stays usable and the next
    build reproduces the earlier P bit for bit."""
    dims, nv, nc = (16, 16, 16), 16, 512
    psi, E = inputs.make_states(16, nv, nc, 41)
    with gw.Context(0) as ctx:
        ctx.load_states(torch.from_numpy(psi.astype(np.complex64)).cuda(), E, dims, nv)
        P1 = build(ctx, "pair", "fp16x3")
        ctx.set_wait_limit(1e-6)
        ctx.build_P("fp16x3")
        with pytest.raises(gw.GwError) as e:
            ctx.sync()
        assert e.value.status == gw.GW_E_TIMEOUT
        ctx.set_wait_limit(2000.0)
        P2 = build(ctx, "pair", "fp16x3")
    assert torch.equal(P1, P2)
