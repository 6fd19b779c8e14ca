"""GPU parity of the learned reconstructor's kernels against the FP64 oracle.

The GPU runs the contractions in bf16 with FP32 accumulation, so outputs and
gradients agree with the FP64 oracle at the bf16 level: per tensor relative
L2 error <= 2e-2 and cosine similarity >= 0.999.  Adam itself is FP32 and is
checked tightly on identical gradients."""
import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

SIZES = [200, 256, 384, 50]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _params32(sizes, seed):
    return [(W.astype(np.float32), b.astype(np.float32)) for W, b in omlp.init_params(sizes, seed)]


def _model(sp, ctx, params, sizes, bmax):
    m = sp.MLP(ctx, sizes, bmax)
    for l, (W, b) in enumerate(params):
        m.set_layer(l, W, b)
    return m


def _close(a, b, rel=2e-2, cos=0.999):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    r = np.linalg.norm(a - b) / np.linalg.norm(b)
    c = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
    return r <= rel and c >= cos, (r, c)


def test_set_get_roundtrip_and_forward_parity(env):
    torch, sp, ctx = env
    params = _params32(SIZES, seed=1)
    m = _model(sp, ctx, params, SIZES, 200)
    for l, (W, b) in enumerate(params):
        W2, b2 = m.get_layer(l)
        assert np.array_equal(W2, W) and np.array_equal(b2, b)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((150, SIZES[0])).astype(np.float32)
    Y = torch.empty(150, SIZES[3], device="cuda")
    m.forward(torch.tensor(X, device="cuda"), Y)
    torch.cuda.synchronize()
    ref, _ = omlp.forward([(W.astype(np.float64), b.astype(np.float64)) for W, b in params], X)
    ok, info = _close(Y.cpu().numpy(), ref)
    assert ok, info


def test_gradients_match_oracle(env):
    torch, sp, ctx = env
    params = _params32(SIZES, seed=3)
    m = _model(sp, ctx, params, SIZES, 256)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((256, SIZES[0])).astype(np.float32)
    T = rng.standard_normal((256, SIZES[3])).astype(np.float32)
    loss = torch.empty(1, device="cuda")
    m.forward(torch.tensor(X, device="cuda"))
    m.backward(torch.tensor(T, device="cuda"), loss)
    torch.cuda.synchronize()
    p64 = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    Yr, cache = omlp.forward(p64, X)
    grads = omlp.backward(p64, cache, Yr, T.astype(np.float64))
    assert abs(loss.item() - omlp.mse(Yr, T)) <= 2e-2 * omlp.mse(Yr, T)
    for l in range(3):
        gW, gb = m.get_grad(l)
        for got, ref, name in ((gW, grads[l][0], "W"), (gb, grads[l][1], "b")):
            ok, info = _close(got, ref)
            assert ok, (l, name, info)


def test_adam_step_matches_oracle_on_same_gradients(env):
    torch, sp, ctx = env
    params = _params32(SIZES, seed=5)
    m = _model(sp, ctx, params, SIZES, 128)
    rng = np.random.default_rng(6)
    X = torch.tensor(rng.standard_normal((128, SIZES[0])).astype(np.float32), device="cuda")
    T = torch.tensor(rng.standard_normal((128, SIZES[3])).astype(np.float32), device="cuda")
    p = [(W.astype(np.float64), b.astype(np.float64)) for W, b in params]
    opt = omlp.Adam(p, lr=1e-3)
    for _ in range(3):
        m.forward(X)
        m.backward(T)
        g = [tuple(x.astype(np.float64) for x in m.get_grad(l)) for l in range(3)]
        m.adam(1e-3)
        p = opt.step(p, g)
    for l in range(3):
        W, b = m.get_layer(l)
        assert np.max(np.abs(W - p[l][0])) <= 1e-6 * (1 + np.abs(p[l][0]).max())
        assert np.max(np.abs(b - p[l][1])) <= 1e-6 * (1 + np.abs(p[l][1]).max())


def _train(torch, sp, ctx, steps, seed):
    sizes = [64, 128, 128, 8]
    params = _params32(sizes, seed=seed)
    m = _model(sp, ctx, params, sizes, 256)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((256, 64)).astype(np.float32)
    T = np.tanh(X[:, :8] * 1.5 + 0.3 * X[:, 8:16] ** 2).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    loss = torch.empty(1, device="cuda")
    losses = []
    for _ in range(steps):
        m.forward(Xd)
        m.backward(Td, loss)
        m.adam(3e-3)
        losses.append(loss.item())
    return m, losses


def test_training_reduces_loss_and_is_deterministic(env):
    torch, sp, ctx = env
    m1, l1 = _train(torch, sp, ctx, 150, seed=9)
    m2, l2 = _train(torch, sp, ctx, 150, seed=9)
    assert l1[-1] < 0.2 * l1[0], (l1[0], l1[-1])
    assert l1 == l2
    for l in range(3):
        assert np.array_equal(m1.get_layer(l)[0], m2.get_layer(l)[0])


def test_model_outliving_its_context_leaves_no_error(env):
    """Closing a context closes the models made on it; a model used after
    that raises, and later contexts and models work normally."""
    torch, sp, _ = env
    c2 = sp.Context(0)
    m = sp.MLP(c2, SIZES, 128)
    c2.close()
    assert m.handle is None
    with pytest.raises(sp.SpeculaError):
        m.forward(torch.zeros(4, SIZES[0], device="cuda"))
    c3 = sp.Context(0)
    m3 = _model(sp, c3, _params32(SIZES, seed=3), SIZES, 128)
    Y = torch.empty(4, SIZES[3], device="cuda")
    m3.forward(torch.zeros(4, SIZES[0], device="cuda"), Y)
    torch.cuda.synchronize()
    assert torch.isfinite(Y).all()
    c3.close()


@pytest.mark.parametrize("nb", [1, 3, 9])
def test_infer_matches_oracle(env, nb):
    """The inference entry point (weight streaming for batch <= 4, the forward
    pass above) against the FP64 oracle on the bf16-rounded weights."""
    torch, sp, ctx = env
    sizes = [203, 256, 384, 77]   # an input width that is not a multiple of 8
    params = _params32(sizes, seed=4)
    m = _model(sp, ctx, params, sizes, 128)
    rng = np.random.default_rng(nb)
    X = rng.standard_normal((nb, sizes[0])).astype(np.float32)
    Y = torch.empty(nb, sizes[3], device="cuda")
    m.infer(torch.tensor(X, device="cuda"), Y)
    torch.cuda.synchronize()
    bf = lambda a: torch.tensor(a).to(torch.bfloat16).float().numpy().astype(np.float64)
    ref, _ = omlp.forward([(bf(W), b.astype(np.float64)) for W, b in params], X)
    ok, info = _close(Y.cpu().numpy(), ref, rel=1e-2 if nb > 4 else 1e-4)
    assert ok, info
    m.close()
