"""The warm-start network's CUDA kernels against the FP64 reference
(oracle/wsnet.py): forward outputs, the gradient of the loss, and one Adam
step, on a 30-bus grid with a ragged number of rows (not a multiple of the
kernels' row tiles)."""
import numpy as np
import pytest

from gridgen import make_case
from oracle.wsnet import WarmStartNet as RefNet
from oracle.wsnet import init_params, param_shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2410_17203_gb300 import load_library
    load_library()


def _setup(T=5, F=6, seed=0, case=None):
    import torch
    case = case or make_case("tiny")
    N = case["n_nodes"]
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(T * N, F)).astype(np.float32)
    Yt = rng.normal(size=(T * N, 2)).astype(np.float32)
    params = init_params(F, seed=seed + 1)
    params = [p + (0.05 * rng.normal(size=p.shape)).astype(np.float32) if p.ndim == 1 else p for p in params]
    flat = np.concatenate([p.ravel() for p in params]).astype(np.float32)
    ref = RefNet(N, case["line_from"], case["line_to"], case["line_b"], T)
    dev = torch.device("cuda")
    return case, N, T, F, X, Yt, params, flat, ref, torch.from_numpy(X).to(dev), torch.from_numpy(Yt).to(dev)


def _unflatten(flat, F):
    out, o = [], 0
    for shp in param_shapes(F):
        n = int(np.prod(shp))
        out.append(flat[o:o + n].reshape(shp))
        o += n
    return out


def test_forward_matches_reference():
    import torch
    from paper_2410_17203_gb300 import WarmStartNet
    case, N, T, F, X, Yt, params, flat, ref, xd, _ = _setup()
    net = WarmStartNet(N, case["line_from"], case["line_to"], case["line_b"], T, F, params=flat)
    y = torch.zeros((T * N, 2), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    want = ref.forward(params, X)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    np.testing.assert_array_equal(net.params(), flat)
    net.close()


def test_gradient_matches_reference():
    from paper_2410_17203_gb300 import WarmStartNet
    case, N, T, F, X, Yt, params, flat, ref, xd, yd = _setup(seed=3)
    net = WarmStartNet(N, case["line_from"], case["line_to"], case["line_b"], T, F, params=flat)
    scale = (1.0, 4.0)
    loss, g = net.gradient(xd, yd, scale)
    rl, rg = ref.loss_and_grads(params, X, Yt, np.array(scale))
    assert loss == pytest.approx(rl, rel=1e-5)
    for i, (a, b) in enumerate(zip(_unflatten(g, F), rg)):
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-9, i
    net.close()


def test_adam_step_matches_reference_and_training_lowers_the_loss():
    from paper_2410_17203_gb300 import WarmStartNet
    case, N, T, F, X, Yt, params, flat, ref, xd, yd = _setup(seed=5)
    net = WarmStartNet(N, case["line_from"], case["line_to"], case["line_b"], T, F, params=flat)
    scale, lr = (1.0, 1.0), 1e-3
    l0 = net.train_step(xd, yd, scale, lr)
    # one Adam step from zero moments moves every parameter by about lr * sign(g)
    _, rg = ref.loss_and_grads(params, X, Yt, np.array(scale))
    g = np.concatenate([x.ravel() for x in rg])
    m, v = 0.1 * g, 0.001 * g * g
    want = flat - lr * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    got = net.params()
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(got[big], want[big], rtol=0, atol=2e-6)
    losses = [l0] + [net.train_step(xd, yd, scale, lr) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]
    net.close()


@pytest.mark.parametrize("F", [9, 64])
def test_forward_and_gradient_over_many_row_tiles(F):
    """A 300-bus grid over 24 steps (7,200 rows: 56 full tiles of the
    register-tiled layers and a ragged one), with the bench's nine features
    and with the largest feature count the network takes (forward only: with
    64 unit-variance inputs many first-layer pre-activations sit within FP32
    rounding of the ReLU kink, where the FP32 and FP64 gradients take
    different branches)."""
    import torch
    from gridgen import scale_case
    from paper_2410_17203_gb300 import WarmStartNet
    case, N, T, F, X, Yt, params, flat, ref, xd, yd = _setup(T=24, F=F, seed=7,
                                                             case=make_case(scale_case(300, 24, 0, seed=8)))
    assert (T * N) % 128 != 0
    net = WarmStartNet(N, case["line_from"], case["line_to"], case["line_b"], T, F, params=flat)
    y = torch.zeros((T * N, 2), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    want = ref.forward(params, X)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    if F <= 9:
        scale = (1.0, 4.0)
        loss, g = net.gradient(xd, yd, scale)
        rl, rg = ref.loss_and_grads(params, X, Yt, np.array(scale))
        assert loss == pytest.approx(rl, rel=1e-5)
        for i, (a, b) in enumerate(zip(_unflatten(g, F), rg)):
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-9, i
    net.close()
