"""Pins for the oracle of the learned truncation correction: the analytic gradient against central
finite differences, a one-layer case against the closed-form least-squares gradient, the
features against a hand-made 2-vector system, the kept/omitted energy weights against hand sums,
and the FP16 weight copy against hand-known FP16 values at hand-counted offsets."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n_in, hidden, B = 5, 7, 9
    theta = rng.standard_normal(M.n_params(n_in, hidden)) * 0.4
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, 2))
    loss, grads = M.loss_and_grad(M.unpack(theta, n_in, hidden), X, T)
    g = M.flatten(grads)
    eps = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp, _ = M.loss_and_grad(M.unpack(tp, n_in, hidden), X, T)
        lm, _ = M.loss_and_grad(M.unpack(tm, n_in, hidden), X, T)
        assert abs((lp - lm) / (2 * eps) - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_output_layer_gradient_is_least_squares_gradient():
    """With all hidden layers fixed, dL/dW4 = (1/B) (y - t)^T h3 and dL/db4 = mean(y - t): the
    closed form of linear least squares."""
    rng = np.random.default_rng(5)
    n_in, hidden, B = 3, 4, 11
    params = M.unpack(rng.standard_normal(M.n_params(n_in, hidden)), n_in, hidden)
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, 2))
    y, acts = M.forward(params, X)
    _, grads = M.loss_and_grad(params, X, T)
    h3 = acts[-1]
    assert np.allclose(grads[-1][0], (y - T).T @ h3 / B, atol=1e-14)
    assert np.allclose(grads[-1][1], np.mean(y - T, axis=0), atol=1e-14)
    # and h3 really is tanh of the previous layer
    W3, b3 = params[2]
    assert np.allclose(h3, np.tanh(acts[2] @ W3.T + b3))


def test_features_by_hand():
    """Two G-vectors m0 = 0, m1 = (1, 0, 0), gcut = 1, P~_lo = [[0, 1+2i], [1-2i, 4]], closure
    estimate dP~ = [[0, 8-4i], [8+4i, -12]]: s = 1/4 (mean |diagonal| over G != 0), three
    upper-triangle rows (0,0), (0,1), (1,1); the last two features are s dP~(g, h)."""
    PG = np.array([[0.0, 1 + 2j], [1 - 2j, 4.0]])
    dc = np.array([[0.0, 8 - 4j], [8 + 4j, -12.0]])
    g = np.array([[0, 0, 0], [1, 0, 0]])
    X, s = M.features(PG, g, 1, 3.0, 6.0, dc)
    assert s == 0.25
    assert X.shape == (3, M.N_FEATURES) == (3, 12)
    assert np.allclose(X[1], [0, 1, 0.25, 0.25, 0.5, 0, 1, 0, 0.5, 1, 2, -1])
    assert np.allclose(X[0], [0, 0, 0, 0, 0, 0, 0, 1, 0.5, 1, 0, 0])
    assert np.allclose(X[2], [1, 1, 0, 1, 0, 1, 1, 1, 0.5, 0, -3, 0])
    X0, _ = M.features(PG, g, 1, 3.0, 6.0)
    assert np.array_equal(X0[:, :10], X[:, :10]) and not X0[:, 10:].any()
    hi = PG + np.array([[0, 4j], [-4j, 8]])
    T = M.targets(PG, hi)
    assert np.allclose(T, [[0, 0], [0, 1], [2, 0]])
    # with the closure estimate the targets are what it leaves: s (hi - lo - dP~)
    T = M.targets(PG, hi, dc)
    assert np.allclose(T, [[0, 0], [-2, 2], [5, 0]])


def test_apply_correction_by_hand():
    """3x3 P~_lo = 0, three upper-triangle predictions per row: head row/column untouched,
    diagonal takes the real part only, (1,2) and (2,1) are conjugates; s = 2 halves everything.
    With a closure estimate dP~ it is added on the same entries under the same rules."""
    Y = np.array([[9, 9], [9, 9], [9, 9], [2, 4], [4, 6], [6, 8]], dtype=float)
    P = M.apply_correction(np.zeros((3, 3)), Y, 2.0)
    want = np.array([[0, 0, 0], [0, 1, 2 + 3j], [0, 2 - 3j, 3]])
    assert np.array_equal(P, want)
    dc = np.array([[5, 5j, 5], [-5j, 10, 1 - 1j], [5, 1 + 1j, 20]])
    P = M.apply_correction(np.zeros((3, 3)), Y, 2.0, dc)
    want = np.array([[0, 0, 0], [0, 11, 3 + 2j], [0, 3 - 2j, 23]])
    assert np.array_equal(P, want)


def test_adam_first_step_is_signed_learning_rate():
    """From zero moments the bias-corrected first step is lr * g / (|g| + eps): lr * sign(g) up to
    eps; a second identical gradient repeats it exactly (m_hat = g, v_hat = g^2 again)."""
    g = np.array([3.0, -0.5, 2e-3, -7.0])
    th, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=0, atol=1e-15)
    th2, _, _ = M.adam_step(th, g, m, v, 2, 0.01, eps=0.0)
    assert np.allclose(th2, -0.02 * np.sign(g), rtol=0, atol=1e-15)


def test_f16_activation_forward_equals_forward_when_activations_are_exact():
    """With W1 = W2 = 0 and biases atanh(1/2), atanh(1/4), the activations feeding the 256-wide
    products are 1/2 and 1/4, exact in FP16: both forwards then agree bit for bit; with a random
    network they differ by FP16 rounding only (2^-11 relative per activation)."""
    rng = np.random.default_rng(8)
    n_in, hidden = 4, 16
    params = M.unpack(rng.standard_normal(M.n_params(n_in, hidden)) * 0.3, n_in, hidden)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = params
    W1[:] = 0
    b1[:] = np.arctanh(0.5)
    W2[:] = 0
    b2[:] = np.arctanh(0.25)
    X = rng.standard_normal((7, n_in))
    assert np.array_equal(M.forward_f16act(params, X), M.forward(params, X)[0])
    params = M.unpack(rng.standard_normal(M.n_params(n_in, hidden)) * 0.3, n_in, hidden)
    a, b = M.forward_f16act(params, X), M.forward(params, X)[0]
    assert 0 < np.abs(a - b).max() <= 2.0 ** -9 * np.abs(b).max()


def test_f16_activation_forward_rounds_exactly_the_square_products_inputs():
    """The inference arithmetic rounds the outputs of layers 1 and 2 (the operands of the two
    256-wide products) to FP16 and nothing else: nudging b1 or b2 by 1e-10 moves those outputs by
    far less than an FP16 step, so the result does not change at all, while the same nudge of b3
    (layer 3 feeds the last product unrounded) does change it."""
    rng = np.random.default_rng(9)
    n_in, hidden = 12, 16
    theta = M.to_fp16_weights(rng.standard_normal(M.n_params(n_in, hidden)) * 0.3, n_in, hidden)
    X = rng.standard_normal((8, n_in))
    y0 = M.forward_f16act(M.unpack(theta, n_in, hidden), X)
    for layer, changes in ((0, False), (1, False), (2, True)):
        params = M.unpack(theta.copy(), n_in, hidden)
        params[layer][1][:] += 1e-10
        y = M.forward_f16act(params, X)
        assert (not np.array_equal(y, y0)) == changes, layer


HA = 27.211386245988   # eV per Hartree


def test_omitted_weights_by_hand():
    """One occupied state at -1 Ha, four unoccupied at +1, +2, +3, +4 Ha, the sum cut after two of
    them: kept = 2/2 + 2/3, omitted = 2/4 + 2/5 (weights 2 / (E_c - E_v) in 1/Hartree, inputs in
    eV).  A second occupied state at -2 Ha adds 2/3 + 2/4 to the kept and 2/5 + 2/6 to the omitted
    sum: the sum runs over v as well, and swapping kept and omitted fails both cases."""
    E = np.array([-1.0, 1.0, 2.0, 3.0, 4.0]) * HA
    om, kept = M.omitted_weights(E, 1, 2)
    assert abs(kept - (1.0 + 2.0 / 3.0)) < 1e-14
    assert abs(om - (0.5 + 0.4)) < 1e-14
    E2 = np.array([-2.0, -1.0, 1.0, 2.0, 3.0, 4.0]) * HA
    om2, kept2 = M.omitted_weights(E2, 2, 2)
    assert abs(kept2 - (1.0 + 2.0 / 3.0 + 2.0 / 3.0 + 0.5)) < 1e-14
    assert abs(om2 - (0.5 + 0.4 + 0.4 + 2.0 / 6.0)) < 1e-14
    # nothing omitted: the whole sum is kept
    om3, kept3 = M.omitted_weights(E, 1, 4)
    assert om3 == 0.0 and abs(kept3 - (1.0 + 2.0 / 3.0 + 0.5 + 0.4)) < 1e-14


def test_to_fp16_weights_rounds_weights_and_keeps_biases():
    """A 2 -> 3 -> 3 -> 3 -> 2 network has 41 parameters laid out as W1 [0, 6), b1 [6, 9),
    W2 [9, 18), b2 [18, 21), W3 [21, 30), b3 [30, 33), W4 [33, 39), b4 [39, 41).  With every
    parameter 1/3, the weights must become FP16's nearest value 0.333251953125 (0x3555) and the
    biases stay 1/3 bit for bit; 2049 rounds to 2048 (FP16 spacing 2 there, tie to even) and 0.1
    to 0.0999755859375 (0x2E66)."""
    assert M.n_params(2, 3) == 41
    theta = np.full(41, 1.0 / 3.0)
    theta[0], theta[40] = 2049.0, 2049.0        # a weight of W1 and the last bias of b4
    theta[33], theta[8] = 0.1, 0.1              # the first weight of W4 and the last bias of b1
    out = M.to_fp16_weights(theta, 2, 3)
    weight = np.zeros(41, dtype=bool)
    for a, b in [(0, 6), (9, 18), (21, 30), (33, 39)]:
        weight[a:b] = True
    want = np.where(weight, 0.333251953125, 1.0 / 3.0)
    want[0], want[40] = 2048.0, 2049.0
    want[33], want[8] = 0.0999755859375, 0.1
    assert np.array_equal(out, want)
    assert np.array_equal(theta[~weight], out[~weight])    # biases untouched, bit for bit
