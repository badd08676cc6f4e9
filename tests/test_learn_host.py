"""Host logic of the learned-parameter trainer (CPU only): the network
trained on standardized features, folded into its first layer, gives the
outputs of the unfolded network on the standardized features (through the
oracle's fp64 MLP forward, which shares nothing with the trainer)."""
import numpy as np
import pytest

from oracle import mlp


@pytest.fixture(scope="module")
def learn():
    import __graft_entry__
    __graft_entry__._builder().build()  # the binding refuses to import without the library
    from paper_2509_24815_gb300 import learn as m
    return m


def test_folded_input_scaling_equals_standardized_inputs(learn):
    rng = np.random.default_rng(3)
    # features on very different scales, one of them constant
    x = rng.standard_normal((50, mlp.IN)) * np.logspace(-1, 2, mlp.IN) + rng.standard_normal(mlp.IN) * 10
    x[:, 7] = 4.0
    mu, sd = learn.standardize(x)
    assert sd[7] == 1.0 and np.all(sd > 0)
    w = (mlp.init(5) * 0.5).astype(np.float32)
    w[-130:] = rng.standard_normal(130).astype(np.float32) * 0.1  # a non-trivial last layer
    o_std, _ = mlp.forward(w.astype(np.float64), (x - mu) / sd)
    o_fold, _ = mlp.forward(learn.fold_input_scaling(w, mu, sd).astype(np.float64), x)
    np.testing.assert_allclose(o_fold, o_std, rtol=2e-4, atol=2e-4)
    # only the first layer changes
    f = learn.fold_input_scaling(w, mu, sd)
    np.testing.assert_array_equal(f[128 * 64 + 128:], w[128 * 64 + 128:])
