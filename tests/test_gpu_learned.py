"""Learned truncation correction on the GPU.

* The network's gradient, loss and forward pass (the library's kernels, FP16 weights, FP32
  accumulation) against the FP64 oracle network evaluated with the same FP16-rounded weights.
* One Adam step against the oracle's Adam.
* The per-entry features, targets and the correction rule against the oracle, on a seeded
  synthetic Hermitian P~.
* End to end on the 24^3 workload: 64 systems with N_v = 32 and N_c = 200 of 2000 kept, trained
  on the GPU and judged on held-out systems against the full N_c = 2000 sum of the plain method.
  The network learns what the closure estimate of the omitted part leaves.  The closure estimate
  is the mean of the omitted sum over the unknown omitted states (they are drawn without
  preference in the complement of the kept ones), so no predictor can beat it on average here:
  the learned form must stay within 2 % of it, beat the diagonal shift alone and gain over
  truncation alone; the full sum is itself checked against the FP64 oracle at sampled entries.
"""
import math

import numpy as np
import pytest

from oracle import gw_oracle as O
from oracle import mlp as M
from paper_1810_07772_gb300 import gw, inputs, learned

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_IN, HID = M.N_FEATURES, 256


def _blocks(vec):
    """Split a flat parameter vector into its 8 blocks (W1, b1, ..., W4, b4)."""
    out, o = [], 0
    for r, c in [(HID, N_IN), (HID, HID), (HID, HID), (2, HID)]:
        out.append(vec[o:o + r * c])
        o += r * c
        out.append(vec[o:o + r])
        o += r
    return out


def _theta(seed):
    th = inputs.mlp_init(N_IN, HID, seed).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    for blk in _blocks(th)[1::2]:        # non-zero biases so their paths are exercised
        blk[:] = 0.1 * rng.standard_normal(blk.size)
    return th.astype(np.float32)


def test_gradient_and_forward_match_oracle():
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(11)
    S, B = 1000, 300                      # ragged: neither is a multiple of the 128-row tile
    X = rng.standard_normal((S, N_IN)).astype(np.float32)
    T = rng.standard_normal((S, 2)).astype(np.float32)
    rows = rng.permutation(S)[:B].astype(np.int32)
    th = _theta(5)
    params = M.unpack(M.to_fp16_weights(th.astype(np.float64), N_IN, HID), N_IN, HID)
    loss_ref, grads = M.loss_and_grad(params, X[rows].astype(np.float64), T[rows].astype(np.float64))
    g_ref = M.flatten(grads)
    y_ref, _ = M.forward(params, X.astype(np.float64))
    with gw.Mlp(N_IN, HID, max_batch=384, device=0) as net:
        net.set_params(th)
        assert np.array_equal(net.get_params(), th)
        g, loss = net.grad(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), torch.from_numpy(rows).to(dev))
        Y = net.forward(torch.from_numpy(X).to(dev)).cpu().numpy()   # 1000 rows in chunks of 384
    g = g.cpu().numpy().astype(np.float64)
    # The products take each FP32 operand as three BF16 parts and drop only terms below 2^-24 of a
    # product; FP32 accumulation over at most 300 terms in each of the 8 product stages: about
    # sqrt(300) u_32 = 1e-6 relative per stage, compounded over the stages.
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    for gb, rb in zip(_blocks(g), _blocks(g_ref)):
        assert np.linalg.norm(gb - rb) <= 2e-5 * np.linalg.norm(rb)
    assert np.linalg.norm(Y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)


def test_gradient_at_shapes_off_the_tile_grid():
    """n_in = 5 and hidden = 200: partial 16-wide K chunks, a partial second 128-column tile with
    its last 8 columns on the scalar epilogue path, a weight gradient with 5 columns (rows of 20
    bytes, scalar stores throughout); batch 257 is one row past two 128-row tiles.  Same bars as
    the full-width test."""
    dev = torch.device("cuda:0")
    n_in, hid, S, B = 5, 200, 600, 257
    rng = np.random.default_rng(21)
    X = rng.standard_normal((S, n_in)).astype(np.float32)
    T = rng.standard_normal((S, 2)).astype(np.float32)
    rows = rng.permutation(S)[:B].astype(np.int32)
    th = inputs.mlp_init(n_in, hid, 3).astype(np.float64)
    sizes = [(hid, n_in), (hid, hid), (hid, hid), (2, hid)]
    o = 0
    for r, c in sizes:                    # non-zero biases
        o += r * c
        th[o:o + r] = 0.1 * rng.standard_normal(r)
        o += r
    th = th.astype(np.float32)
    params = M.unpack(M.to_fp16_weights(th.astype(np.float64), n_in, hid), n_in, hid)
    loss_ref, grads = M.loss_and_grad(params, X[rows].astype(np.float64), T[rows].astype(np.float64))
    g_ref = M.flatten(grads)
    y_ref, _ = M.forward(params, X.astype(np.float64))
    with gw.Mlp(n_in, hid, max_batch=300, device=0) as net:
        net.set_params(th)
        g, loss = net.grad(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), torch.from_numpy(rows).to(dev))
        Y = net.forward(torch.from_numpy(X).to(dev)).cpu().numpy()
        net.check()
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    o = 0
    for r, c in sizes:
        for n in (r * c, r):              # W_l, then b_l
            assert np.linalg.norm(g[o:o + n] - g_ref[o:o + n]) <= 2e-5 * np.linalg.norm(g_ref[o:o + n])
            o += n
    assert np.linalg.norm(Y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)


def test_tensor_core_inference_matches_oracle():
    """gw_mlp_infer (tcgen05 kind::f16 on CTA pairs, FP16 activations into the 256-wide products)
    against the oracle forward with the same FP16 roundings; 1000 rows = several 256-row tiles and
    a ragged last tile.  Tolerance: the kernel's tanh is the hardware approximation (relative error
    about 2^-11 per activation, against exact tanh in the oracle), which with the FP16 roundings
    moves the output by about 1e-4 relative (measured 9.6e-5 on these inputs); 1e-3 bounds it."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(13)
    X = rng.standard_normal((1000, N_IN)).astype(np.float32)
    th = _theta(9)
    params = M.unpack(M.to_fp16_weights(th.astype(np.float64), N_IN, HID), N_IN, HID)
    y_ref = M.forward_f16act(params, X.astype(np.float64))
    y_fp32 = M.forward(params, X.astype(np.float64))[0]
    with gw.Mlp(N_IN, HID, max_batch=384, device=0) as net:
        net.set_params(th)
        Y = net.infer(torch.from_numpy(X).to(dev))
        net.check()
        Y = Y.cpu().numpy()
        # a parameter update invalidates the tiled weights: inference must follow it
        th2 = th.copy()
        th2[: HID * N_IN] *= -1.0
        net.set_params(th2)
        Y2 = net.infer(torch.from_numpy(X).to(dev)).cpu().numpy()
    assert np.linalg.norm(Y - y_ref) <= 1e-3 * np.linalg.norm(y_ref)
    assert np.linalg.norm(Y - y_fp32) <= 1e-2 * np.linalg.norm(y_fp32)
    p2 = M.unpack(M.to_fp16_weights(th2.astype(np.float64), N_IN, HID), N_IN, HID)
    assert np.linalg.norm(Y2 - M.forward_f16act(p2, X.astype(np.float64))) <= 1e-3 * np.linalg.norm(Y2)


def test_adam_step_matches_oracle():
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(12)
    X = rng.standard_normal((512, N_IN)).astype(np.float32)
    T = rng.standard_normal((512, 2)).astype(np.float32)
    th = _theta(6)
    params = M.unpack(M.to_fp16_weights(th.astype(np.float64), N_IN, HID), N_IN, HID)
    _, grads = M.loss_and_grad(params, X.astype(np.float64), T.astype(np.float64))
    g = M.flatten(grads)
    lr = 1e-3
    want, _, _ = M.adam_step(th.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    rows = torch.arange(512, dtype=torch.int32, device=dev)
    with gw.Mlp(N_IN, HID, max_batch=512, device=0) as net:
        net.set_params(th)
        net.train_step(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), rows, lr)
        got = net.get_params().astype(np.float64)
    # The first step moves every parameter by ~lr sign(g); where |g| is within rounding of 0 the
    # sign is not fixed by FP32 arithmetic, so those entries are excluded.
    firm = np.abs(g) > 1e-4 * np.abs(g).max()
    assert firm.mean() > 0.9
    assert np.max(np.abs(got - want)[firm]) <= 1e-6


def _synthetic_PG(ng, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((ng, 3 * ng)) + 1j * rng.standard_normal((ng, 3 * ng))
    P = -(A @ A.conj().T) / (3 * ng)
    P = 0.5 * (P + P.conj().T)
    P[np.diag_indices(ng)] = P.diagonal().real
    P[0, :] = 0
    P[:, 0] = 0
    return P.astype(np.complex64)


def test_features_targets_apply_match_oracle():
    dev = torch.device("cuda:0")
    dims, gcut = (12, 12, 12), 8
    g = O.sphere(dims, gcut)
    ng = len(g)                           # 93: one full 64-row block and a ragged one
    lo, hi = _synthetic_PG(ng, 21), _synthetic_PG(ng, 22)
    hi = lo + 0.3 * hi
    dc = (0.2 * _synthetic_PG(ng, 24)).astype(np.complex64)          # a stand-in closure estimate
    psi, E = inputs.make_states(12, 4, 40, 3)
    nv, keep = 4, 10
    w_om, w_in = M.omitted_weights(E, nv, keep)
    X_ref, s_ref = M.features(lo.astype(np.complex128), g, gcut, w_om, w_in, dc.astype(np.complex128))
    T_ref = M.targets(lo.astype(np.complex128), hi.astype(np.complex128), dc.astype(np.complex128))
    Y = np.random.default_rng(23).standard_normal((ng * (ng + 1) // 2, 2)).astype(np.float32)
    P_ref = M.apply_correction(lo.astype(np.complex128), Y.astype(np.float64), s_ref, dc.astype(np.complex128))

    lo_d, hi_d, dc_d = torch.from_numpy(lo).to(dev), torch.from_numpy(hi).to(dev), torch.from_numpy(dc).to(dev)
    ratio = gw.corr_weight_ratio(E, nv, keep)
    X, scale = gw.corr_features(lo_d, g, gcut, ratio, dc_d)
    T = gw.corr_targets(lo_d, hi_d, scale, dc_d)
    P = lo_d.clone()
    gw.corr_apply(P, torch.from_numpy(Y).to(dev), scale, dc_d)
    X0, _ = gw.corr_features(lo_d, g, gcut, ratio)                      # without a closure estimate
    X, T, P, X0 = X.cpu().numpy(), T.cpu().numpy(), P.cpu().numpy(), X0.cpu().numpy()
    assert np.array_equal(X0[:, :10], X[:, :10]) and not X0[:, 10:].any()
    assert abs(float(ratio.item()) - w_om / w_in) <= 1e-7 * (w_om / w_in)
    assert abs(float(scale.item()) - s_ref) <= 1e-6 * s_ref
    assert X.shape == X_ref.shape and T.shape == T_ref.shape
    for j in range(M.N_FEATURES):
        assert np.allclose(X[:, j], X_ref[:, j], rtol=2e-6, atol=2e-7 * max(1.0, np.abs(X_ref[:, j]).max())), j
    assert np.array_equal(X[:, [7, 9]], X_ref[:, [7, 9]])
    assert np.allclose(T, T_ref, rtol=0, atol=2e-6 * np.abs(T_ref).max())
    assert np.allclose(P, P_ref, rtol=0, atol=2e-6 * np.abs(P_ref).max())
    assert np.array_equal(P[0], lo[0]) and np.array_equal(P[:, 0], lo[:, 0])
    assert np.array_equal(P, P.conj().T)


def _rel(A, B):
    return float(torch.linalg.norm(A - B) / torch.linalg.norm(B))


@pytest.mark.slow
def test_weight_ratio_at_the_occupied_limit():
    """The omitted/kept weight ratio of Eq. (Pstatic) at the largest supported nv (1024) and with
    more unoccupied states than one pass of the block (3000), against the FP64 sums; nv = 1025 is
    rejected."""
    rng = np.random.default_rng(31)
    nv, nc_all, keep = 1024, 3000, 1100
    E = np.concatenate([np.sort(rng.uniform(-25.0, -0.2, nv)), np.sort(rng.uniform(0.05, 80.0, nc_all))])
    w_om, w_in = M.omitted_weights(E, nv, keep)
    ratio = float(gw.corr_weight_ratio(E, nv, keep).item())
    assert abs(ratio - w_om / w_in) <= 1e-7 * (w_om / w_in)
    with pytest.raises(gw.GwError):
        gw.corr_weight_ratio(np.concatenate([E[:1], E]), nv + 1, keep)


def test_learned_correction_gain_24cubed():
    """24^3, N_v = 32, N_c = 200 kept of 2000; 64 training systems, 8 held-out systems, band-
    structured states (energy-ordered plane-wave shells): the closure estimate assumes the omitted
    states spread evenly over the complement of the kept ones, which band structure breaks, and the
    network has to learn the rest."""
    dev = torch.device("cuda:0")
    n, nv, keep, nc_all, gcut = 24, 32, 200, 2000, 29
    dims = (n,) * 3
    nr = n ** 3

    with gw.Context(0) as ctx:
        def states(seed):
            coef, gvec, E = inputs.make_states_g_structured_device(dims, nv, nc_all, seed, dev)
            return learned.states_in_real_space(ctx, coef, gvec, E, dims, nv), E

        X, T = learned.training_set(ctx, states, range(1000, 1064), nv, keep, dims, gcut)
        assert X.shape[0] == 64 * 691 * 692 // 2
        with gw.Mlp(N_IN, HID, max_batch=8192, device=0) as net:
            net.set_params(inputs.mlp_init(N_IN, HID, 7))
            losses = learned.train(net, X, T, epochs=6, batch=8192, lr=1e-3, seed=0, diag_repeat=32)
            del X, T
            e_trunc, e_mlp, e_clos, e_full = [], [], [], []
            for seed in range(2000, 2008):
                psi, E = states(seed)
                d = learned.system_samples(ctx, psi, E, nv, keep, dims, gcut)
                P_ml = learned.correct(net, d["PG_keep"], d["gvec"], gcut, E, nv, keep, d["clos"])
                w_om, _ = M.omitted_weights(E, nv, keep)
                clos = d["PG_keep"].clone()                   # the diagonal shift alone
                idx = torch.arange(1, clos.shape[0], device=dev)
                clos[idx, idx] -= w_om / (nr - (nv + keep))
                e_trunc.append(_rel(d["PG_keep"], d["PG_all"]))
                e_mlp.append(_rel(P_ml, d["PG_all"]))
                e_clos.append(_rel(clos, d["PG_all"]))
                e_full.append(_rel(d["PG_keep"] + d["clos"], d["PG_all"]))
                if seed == 2000:
                    # the learned form goes on to eps^-1 like any P~
                    ctx.view("PG").copy_(P_ml)
                    ng = P_ml.shape[0]
                    eps = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
                    inv = torch.empty((ng, ng), dtype=torch.complex128, device=dev)
                    ctx.eps_inv("cholesky", eps_out=eps, epsinv_out=inv)
                    I = torch.eye(ng, dtype=torch.complex128, device=dev)
                    assert float((inv @ eps - I).abs().max()) <= 1e-12
                    # the reference of the learned form, P~ of the full sum, against the FP64 oracle at sampled entries
                    sel = np.array([0, 1, 7, 100, 350, 690])
                    ref = O.P_gspace_entries(psi.cpu().numpy().astype(np.complex128), E, nv, dims, d["gvec"][sel])
                    sub = d["PG_all"][sel][:, sel].cpu().numpy()
                    assert np.linalg.norm(sub - ref) / np.linalg.norm(ref) <= 1e-6
    e_trunc, e_mlp, e_clos, e_full = map(np.mean, (e_trunc, e_mlp, e_clos, e_full))
    print(f"losses {losses}  rel. error of P~: truncated {e_trunc:.4f}  learned {e_mlp:.4f}  "
          f"closure {e_full:.4f}  diagonal shift {e_clos:.4f}")
    assert losses[-1] <= losses[0]
    assert e_mlp < 0.5 * e_trunc
    assert e_mlp < e_clos
    assert e_mlp < 0.5 * e_full             # the network improves on the closure estimate


def _order_keys(seed, e, S):
    """The library's minibatch keys, written out with numpy's wrapping uint64 arithmetic."""
    u = np.uint64
    base = (np.array([seed], dtype=u) * u(0x9E3779B97F4A7C15) + np.array([e + 1], dtype=u) * u(0xD1B54A32D192ED03))
    z = base + np.arange(S, dtype=u)
    z ^= z >> u(30)
    z *= u(0xBF58476D1CE4E5B9)
    z ^= z >> u(27)
    z *= u(0x94D049BB133111EB)
    z ^= z >> u(31)
    return z


def test_corr_train_equals_the_loop_it_replaces():
    """gw_corr_train against the same loop driven from Python through gw_mlp_train_step: the pool
    (all rows, then the diagonal rows three more times), each pass in the order of the documented
    keys, the cosine rate, the per-pass loss.  Same kernels in the same order: parameters and
    losses agree bit for bit."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(31)
    n, batch, epochs, rep, seed = 5000, 256, 3, 4, 12345
    X = rng.standard_normal((n, N_IN)).astype(np.float32)
    X[:, 7] = (rng.random(n) < 0.05).astype(np.float32)           # diagonal flags
    T = rng.standard_normal((n, 2)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    th = _theta(17)
    with gw.Mlp(N_IN, HID, max_batch=batch, device=0) as a, gw.Mlp(N_IN, HID, max_batch=batch, device=0) as b:
        a.set_params(th)
        b.set_params(th)
        la = a.train_corr(Xd, Td, epochs, batch, 2e-3, lr_final=1e-4, seed=seed, diag_repeat=rep)
        diag = np.flatnonzero(X[:, 7] == 1)
        pool = np.concatenate([np.arange(n)] + [diag] * (rep - 1)).astype(np.int32)
        steps = len(pool) // batch
        total, t, lb = epochs * steps, 0, []
        acc = torch.zeros(1, dtype=torch.float32, device=dev)
        for e in range(epochs):
            order = pool[np.argsort(_order_keys(seed, e, len(pool)), kind="stable")]
            rows = torch.from_numpy(order).to(dev)
            acc.zero_()
            for i in range(steps):
                lr_t = 1e-4 + 0.5 * (2e-3 - 1e-4) * (1.0 + math.cos(math.pi * t / total))
                b.train_step(Xd, Td, rows[i * batch:(i + 1) * batch], lr_t, loss_accum=acc)
                t += 1
            lb.append(float(acc.item()) / steps)
        pa, pb = a.get_params(), b.get_params()
    assert np.array_equal(pa, pb)
    assert np.allclose(la, lb, rtol=1e-6, atol=0)
    assert la[-1] < la[0]
