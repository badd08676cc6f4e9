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
