"""Pins of the FP64 reference of the warm-start network: analytic gradients
against central finite differences, the neighbour average and its adjoint,
and bfloat16 rounding on values whose rounding is known."""
import numpy as np

from oracle.wsnet import (HIDDEN, N_MP, WarmStartNet, bf16, init_params, neighbour_matrix,
                          param_shapes)


def _tiny(seed=0, T=2, F=3):
    rng = np.random.default_rng(seed)
    N = 6
    lf = np.array([0, 1, 2, 3, 0, 4])
    lt = np.array([1, 2, 3, 4, 2, 5])
    lb = rng.uniform(5, 20, len(lf))
    net = WarmStartNet(N, lf, lt, lb, T)
    X = rng.normal(size=(T * N, F))
    Yt = rng.normal(size=(T * N, 2))
    return net, X, Yt


def test_bf16_rounding_known_values():
    one = 1.0
    assert bf16(np.float32(one)) == 1.0
    assert bf16(np.float32(1 + 2 ** -8)) == 1.0                 # tie -> even
    assert bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6     # tie -> even (up)
    assert bf16(np.float32(1 + 2 ** -8 + 2 ** -20)) == 1 + 2 ** -7
    assert bf16(np.float32(-2.5)) == -2.5


def test_neighbour_average_rows_and_adjoint():
    rng = np.random.default_rng(1)
    lf, lt = np.array([0, 1, 1]), np.array([1, 2, 3])
    lb = np.array([2.0, 6.0, 2.0])
    A = neighbour_matrix(5, lf, lt, lb)      # node 4 has no line
    np.testing.assert_allclose(A.sum(axis=1)[:4], 1.0)
    assert np.all(A[4] == 0)
    assert A[1, 2] == 6.0 / 10.0 and A[2, 1] == 1.0
    net = WarmStartNet(5, lf, lt, lb, 3)
    H = rng.normal(size=(15, 4))
    G = rng.normal(size=(15, 4))
    assert abs(np.sum(net._agg(H) * G) - np.sum(H * net._agg_t(G))) < 1e-12


def test_gradients_match_finite_differences():
    net, X, Yt = _tiny()
    params = [p.astype(np.float64) for p in init_params(X.shape[1], seed=3)]
    # non-zero biases so every term of the gradient is exercised
    rng = np.random.default_rng(4)
    params = [p + (0.1 * rng.normal(size=p.shape) if p.ndim == 1 else 0) for p in params]
    scale = np.array([1.0, 3.0])
    loss, grads = net.loss_and_grads(params, X, Yt, scale, round_bf16=False)
    h = 1e-6
    for i, p in enumerate(params):
        flat = p.ravel()
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for j in idx:
            q = [x.copy() for x in params]
            q[i].ravel()[j] += h
            lp = net.loss_and_grads(q, X, Yt, scale, round_bf16=False)[0]
            q[i].ravel()[j] -= 2 * h
            lm = net.loss_and_grads(q, X, Yt, scale, round_bf16=False)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[i].ravel()[j]) <= 1e-6 * (1 + abs(fd)), (i, j, fd, grads[i].ravel()[j])


def test_shapes_and_layer_count():
    shapes = param_shapes(7)
    assert len(shapes) == 2 + 3 * N_MP + 2
    assert shapes[0] == (7, HIDDEN) and shapes[-2] == (HIDDEN, 2)
    net, X, _ = _tiny(F=7)
    Y = net.forward(init_params(7, seed=0), X)
    assert Y.shape == (X.shape[0], 2)
