"""Pins for the oracle MLP: analytic gradient against central finite
differences, and the output-to-parameter map at its fixed points.  CPU only."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = mlp.init(1) * 0.5
    x = rng.standard_normal((7, mlp.IN))
    t = rng.random((7, mlp.OUT))
    g = mlp.grad(w, x, t)
    idx = rng.choice(mlp.N_PARAMS, size=80, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, mlp.N_PARAMS - 3]])  # include biases of the last layer
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, x, t) - mlp.loss(wm, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_param_map():
    o = np.array([[0.0, 0.0], [-50.0, -50.0], [50.0, 50.0]])
    cut, hf = mlp.params_from_output(o)
    assert cut.tolist() == [16, 3, 30]  # 3 + 27/2 = 16.5 -> 16 (round half to even)
    np.testing.assert_allclose(hf, [0.75, 0.5, 1.0], atol=1e-12)


def test_pack_roundtrip():
    w = mlp.init(3)
    assert w.size == mlp.N_PARAMS == 16706
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(w)), w)


def test_forward_hand_computed_2_2_2():
    """A 2-2-2 network worked by hand, embedded in the packed 64-128-64-2
    parameter vector (every other weight and bias 0, so the other hidden units
    stay at ReLU(0) = 0).  The offsets are written out here, not taken from
    unpack(), so the packing order W1, b1, W2, b2, W3, b3 is pinned too.

      x  = (1, -2)
      z1 = W1 x + b1 = (1*1 + 2*-2 + 0.5, 3*1 + -1*-2 - 1) = (-2.5, 4)  -> a1 = (0, 4)
      z2 = W2 a1 + b2 = (2*0 + -1*4 + 1, 0.5*0 + 1*4 - 3) = (-3, 1)    -> a2 = (0, 1)
      o  = W3 a2 + b3 = (4*0 + 2*1 + 0.25, -1*0 + 3*1 - 0.5) = (2.25, 2.5)

    A transposed weight matrix, a missing or misplaced ReLU, or a dropped bias
    each changes o."""
    w = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = 0, 128 * 64, 128 * 64 + 128, 2 * 128 * 64 + 128, 2 * 128 * 64 + 128 + 64, \
        2 * 128 * 64 + 128 + 64 + 2 * 64
    assert b3 + 2 == mlp.N_PARAMS
    w[W1 + 0 * 64 + 0], w[W1 + 0 * 64 + 1], w[W1 + 1 * 64 + 0], w[W1 + 1 * 64 + 1] = 1.0, 2.0, 3.0, -1.0
    w[b1 + 0], w[b1 + 1] = 0.5, -1.0
    w[W2 + 0 * 128 + 0], w[W2 + 0 * 128 + 1], w[W2 + 1 * 128 + 0], w[W2 + 1 * 128 + 1] = 2.0, -1.0, 0.5, 1.0
    w[b2 + 0], w[b2 + 1] = 1.0, -3.0
    w[W3 + 0 * 64 + 0], w[W3 + 0 * 64 + 1], w[W3 + 1 * 64 + 0], w[W3 + 1 * 64 + 1] = 4.0, 2.0, -1.0, 3.0
    w[b3 + 0], w[b3 + 1] = 0.25, -0.5
    x = np.zeros((1, mlp.IN))
    x[0, 0], x[0, 1] = 1.0, -2.0
    o, (_, z1, a1, z2, a2, _) = mlp.forward(w, x)
    np.testing.assert_array_equal(z1[0, :2], [-2.5, 4.0])
    np.testing.assert_array_equal(a1[0, :3], [0.0, 4.0, 0.0])
    np.testing.assert_array_equal(z2[0, :2], [-3.0, 1.0])
    np.testing.assert_array_equal(a2[0, :3], [0.0, 1.0, 0.0])
    np.testing.assert_array_equal(o[0], [2.25, 2.5])
    # loss against t = (1, 0): (sigmoid(2.25) - 1)^2 + sigmoid(2.5)^2, sigmoid written out
    s0, s1 = 1.0 / (1.0 + np.exp(-2.25)), 1.0 / (1.0 + np.exp(-2.5))
    assert abs(mlp.loss(w, x, np.array([[1.0, 0.0]])) - ((s0 - 1.0) ** 2 + s1 ** 2)) <= 1e-15
    # the parameter map: cut = round(3 + 27 * 0.904651) = round(27.43) = 27, hf = 0.5 + 0.5 * 0.924142
    cut, hf = mlp.params_from_output(o)
    assert cut.tolist() == [27]
    assert abs(hf[0] - 0.962071) <= 1e-6
