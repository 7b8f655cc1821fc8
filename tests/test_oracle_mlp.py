"""Pin P12 (CPU): the FP64 MLP oracle's backward pass against central finite differences of its
loss, GELU's derivative against differences of GELU, the BF16 rounding against its definition,
and Adam against a hand-computed first step."""
import numpy as np
import pytest

from oracle import mlp


def test_gelu_values_and_derivative():
    z = np.linspace(-6, 6, 121)
    # tanh form: gelu(0) = 0, gelu(z) -> z for large z, -> 0 for very negative z
    g = mlp.gelu(z)
    assert g[60] == 0.0 and abs(g[-1] - 6.0) < 1e-6 and abs(g[0]) < 1e-6
    # close to the exact erf form z Phi(z)
    from scipy.special import erf

    assert np.max(np.abs(g - 0.5 * z * (1 + erf(z / np.sqrt(2))))) < 2e-3
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(37, 6))
    T = rng.normal(size=(37, 6))
    loss, g = mlp.loss_and_grads(p, X, T)
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        idx = [tuple(rng.integers(0, s) for s in p[name].shape) for _ in range(8)]
        for ix in idx:
            # fourth-order central difference (truncation ~h^4, rounding ~1e-16/h)
            h = 1e-3

            def f(delta):
                q = {k: v.copy() for k, v in p.items()}
                q[name][ix] += delta
                return mlp.loss_and_grads(q, X, T)[0]

            fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
            assert g[name][ix] == pytest.approx(fd, rel=1e-7, abs=1e-12), (name, ix)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-9, 1.0 + 3 * 2**-9, -2.5, 3.0e-3])
    r = mlp.round_bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2**-7 or r[1] == 1.0  # 2^-8 is exactly half an ulp: ties to even -> 1.0
    assert r[1] == 1.0
    assert r[2] == 1.0
    assert r[3] == 1.0 + 2**-7
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) / 3.0e-3 < 2**-8


def test_adam_first_step():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.5, -0.25])}
    m = {"w": np.zeros(2)}
    v = {"w": np.zeros(2)}
    mlp.adam_update(p, g, m, v, 1, lr=0.1)
    # bias-corrected first step moves every parameter by lr * sign(g) (up to eps)
    np.testing.assert_allclose(p["w"], [0.9, -1.9], rtol=1e-7)


def test_pack_roundtrip():
    p = mlp.init_params(3)
    q = mlp.unpack(mlp.pack(p))
    for k in p:
        np.testing.assert_array_equal(p[k], q[k])
    assert len(mlp.pack(p)) == mlp.NPARAMS == 4998
