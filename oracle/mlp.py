"""FP64 CPU oracle of the learned truncation correction (test infrastructure only).

The paper names band truncation (the sum over unoccupied states c in Eq. Pstatic cut at some N_c)
as an open issue and prescribes no correction; the network below is this build's extension.
Everything here is written from definitions:

* features of one entry (G, G') of a truncated P~ (upper triangle, G index <= G' index);
* a multilayer perceptron  h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
  y = W4 h3 + b4, with loss  L = (1 / (2 B)) sum_{samples, outputs} (y - t)^2;
* its gradient by the chain rule, pinned in the tests by central finite differences.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 12


def entry_scale(PG_lo):
    """s = 1 / mean_{G != 0} |P~_lo(G, G)|: makes features and targets O(1) for any system."""
    d = np.abs(np.real(np.diag(PG_lo)))[1:]
    return 1.0 / np.mean(d)


def omitted_weights(E_eV, nv, nc_lo):
    """(sum over omitted c, sum over kept c) of sum_v 2 / (E_c - E_v), energies in Hartree."""
    E = np.asarray(E_eV, dtype=np.float64) / 27.211386245988
    w = 2.0 / (E[None, nv:] - E[:nv, None])
    return float(np.sum(w[:, nc_lo:])), float(np.sum(w[:, :nc_lo]))


def features(PG_lo, gvec, gcut, w_om, w_in, dclos=None):
    """Rows (g, h), g <= h in basis order (row-major over the upper triangle):
    |m_g|^2/gcut, |m_h|^2/gcut, |m_g - m_h|^2/(4 gcut), s Re P~(g,h), s Im P~(g,h), s P~(g,g),
    s P~(h,h), [g == h], w_om / w_in, [g == 0 or h == 0], s Re dP~(g,h), s Im dP~(g,h), where dP~ is
    the closure estimate of the omitted part (zero when dclos is None)."""
    PG_lo = np.asarray(PG_lo, dtype=np.complex128)
    gvec = np.asarray(gvec, dtype=np.float64)
    ng = gvec.shape[0]
    s = entry_scale(PG_lo)
    gi, hi = np.triu_indices(ng)
    m2 = np.sum(gvec * gvec, axis=1)
    dm = gvec[gi] - gvec[hi]
    diag = np.real(np.diag(PG_lo))
    dc = np.zeros(gi.shape, dtype=np.complex128) if dclos is None else np.asarray(dclos, np.complex128)[gi, hi]
    X = np.stack([m2[gi] / gcut, m2[hi] / gcut, np.sum(dm * dm, axis=1) / (4.0 * gcut),
                  s * np.real(PG_lo[gi, hi]), s * np.imag(PG_lo[gi, hi]), s * diag[gi], s * diag[hi],
                  (gi == hi).astype(np.float64), np.full(gi.shape, w_om / w_in),
                  ((gi == 0) | (hi == 0)).astype(np.float64), s * np.real(dc), s * np.imag(dc)], axis=1)
    return X, s


def targets(PG_lo, PG_hi, dclos=None):
    """t = s (P~_hi - P~_lo - dP~)(g, h) as (Re, Im) over the upper triangle, s from the truncated P~
    and dP~ the closure estimate (zero when dclos is None): the network learns what the closure
    estimate leaves."""
    s = entry_scale(PG_lo)
    ng = PG_lo.shape[0]
    gi, hi = np.triu_indices(ng)
    D = np.asarray(PG_hi, np.complex128) - np.asarray(PG_lo, np.complex128)
    if dclos is not None:
        D = D - np.asarray(dclos, np.complex128)
    d = D[gi, hi] * s
    return np.stack([np.real(d), np.imag(d)], axis=1)


def unpack(theta, n_in, hidden, n_out=2):
    """Flat parameter vector -> [(W1, b1), ..., (W4, b4)], W_l of shape (out, in)."""
    sizes = [(hidden, n_in), (hidden, hidden), (hidden, hidden), (n_out, hidden)]
    out, o = [], 0
    for r, c in sizes:
        W = theta[o:o + r * c].reshape(r, c)
        o += r * c
        b = theta[o:o + r]
        o += r
        out.append((W, b))
    assert o == theta.size
    return out


def n_params(n_in, hidden, n_out=2):
    return hidden * n_in + hidden + 2 * (hidden * hidden + hidden) + n_out * hidden + n_out


def forward(params, X):
    """Returns (y, activations) with activations = [x, h1, h2, h3]."""
    acts = [np.asarray(X, dtype=np.float64)]
    a = acts[0]
    for W, b in params[:-1]:
        a = np.tanh(a @ W.T + b)
        acts.append(a)
    W, b = params[-1]
    return a @ W.T + b, acts


def loss_and_grad(params, X, T):
    """L = (1/(2B)) sum (y - t)^2 and dL/d(each W_l, b_l) by the chain rule."""
    y, acts = forward(params, X)
    B = X.shape[0]
    r = y - np.asarray(T, dtype=np.float64)
    loss = 0.5 * np.sum(r * r) / B
    grads = [None] * len(params)
    delta = r / B                                   # dL/dy
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        a_in = acts[l]
        grads[l] = (delta.T @ a_in, np.sum(delta, axis=0))
        if l > 0:
            da = delta @ W                          # dL/d(activation of layer l)
            delta = da * (1.0 - acts[l] ** 2)       # through tanh
    return loss, grads


def flatten(grads):
    return np.concatenate([np.concatenate([g.reshape(-1), b]) for g, b in grads])


def to_fp16_weights(theta, n_in, hidden):
    """The weights the GPU multiplies with: every W_l rounded to FP16 (biases stay FP32)."""
    out = np.array(theta, dtype=np.float64)
    o = 0
    for r, c in [(hidden, n_in), (hidden, hidden), (hidden, hidden), (2, hidden)]:
        out[o:o + r * c] = out[o:o + r * c].astype(np.float16).astype(np.float64)
        o += r * c + r
    return out


def apply_correction(PG_lo, Y, s, dclos=None):
    """P~ = P~_lo + dP~ + (y0 + i y1) / s on the upper triangle, mirrored as the conjugate below it
    (dP~ the closure estimate, zero when dclos is None).  The diagonal takes the real part only (a
    Hermitian matrix has a real diagonal) and the G = 0 row and column are left unchanged (they
    vanish exactly, because occupied and unoccupied states are orthogonal, at any N_c)."""
    P = np.array(PG_lo, dtype=np.complex128)
    ng = P.shape[0]
    gi, hi = np.triu_indices(ng)
    d = (np.asarray(Y[:, 0], dtype=np.float64) + 1j * np.asarray(Y[:, 1], dtype=np.float64)) / s
    if dclos is not None:
        d = d + np.asarray(dclos, np.complex128)[gi, hi]
    keep = (gi != 0) & (hi != 0)
    gi, hi, d = gi[keep], hi[keep], d[keep]
    on = gi == hi
    P[gi[on], gi[on]] += np.real(d[on])
    P[gi[~on], hi[~on]] += d[~on]
    P[hi[~on], gi[~on]] += np.conj(d[~on])
    return P


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015): moment updates, bias correction by 1 - beta^t, then
    theta -= lr * m_hat / (sqrt(v_hat) + eps).  Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def forward_f16act(params, X):
    """Inference arithmetic of the tensor-core path: the outputs of layers 1 and 2 (the inputs of
    the two 256 x 256 products, FP16 operands on both sides) are rounded to FP16; layer 3's output
    feeds the last layer unrounded.  params should hold FP16-rounded weights (to_fp16_weights)."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = params
    f16 = lambda a: a.astype(np.float16).astype(np.float64)  # noqa: E731
    h1 = f16(np.tanh(np.asarray(X, dtype=np.float64) @ W1.T + b1))
    h2 = f16(np.tanh(h1 @ W2.T + b2))
    h3 = np.tanh(h2 @ W3.T + b3)
    return h3 @ W4.T + b4
