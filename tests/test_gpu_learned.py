"""Learned sizing on the GPU: the predictor's CUDA forward and backward
against the float64 reference, training that lowers the loss, and learned
products whose rows equal the two-phase path bit for bit -- with slots that
fit, with forced overflow (every row re-run), and for every value type."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


def test_forward_and_gradient_match_reference(sg):
    import torch
    rng = np.random.default_rng(3)
    N = 1000
    X = (rng.random((N, mlp.F)) * 12).astype(np.float32)
    t = (rng.random(N) * 10).astype(np.float32)
    p = (rng.normal(size=mlp.param_count()) * 0.2).astype(np.float32)
    dX, dt, dp = (torch.from_numpy(a).cuda() for a in (X, t, p))
    y = sg.sizer_forward(dX, dp).cpu().numpy()
    yr, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y, yr, rtol=1e-4, atol=1e-4)
    g, loss = sg.sizer_grad(dX, dt, dp)
    lr, gr = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - lr) <= 1e-4 * max(1, lr)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    np.testing.assert_allclose(g[big], gr[big], rtol=1e-3, atol=1e-5 * np.abs(gr).max())


def train_small(sg):
    pairs = [(inputs.rmat(s, seed=300 + s), None) for s in (9, 10, 11)]
    pairs += [(inputs.er_column_regular(2048, d, 400 + d), None) for d in (4, 8, 16)]
    dev = [(sg.to_device(A), sg.to_device(A)) for A, _ in pairs]
    X, T = sg.sizer_training_set(dev)
    params = sg.sizer_init(seed=1)
    trace = sg.sizer_train(X, T, params, steps=400, batch=1024, lr=3e-3, seed=2)
    return params, trace, X, T


def test_training_lowers_the_loss(sg):
    params, trace, X, T = train_small(sg)
    tr = trace.cpu().numpy()
    assert tr[-20:].mean() < 0.25 * tr[:20].mean()
    y = sg.sizer_forward(X, params)
    rmse = float(((y - T) ** 2).mean().sqrt())
    assert rmse < 1.0      # log2 units


@pytest.fixture(scope="module")
def trained(sg):
    return train_small(sg)[0]


@pytest.mark.parametrize("margin", [0.3, -4.0, 40.0])
def test_learned_product_equals_two_phase(sg, trained, margin):
    import torch
    A = inputs.rmat(12, seed=77)
    dA = sg.to_device(A)
    C, stats = sg.learned_multiply(dA, dA, trained, margin=margin)
    P = sg.spgemm(dA, dA)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all())
    assert bool((Cc.col == P.col).all()) and bool((Cc.val == P.val).all())
    if margin == -4.0:
        assert stats["overflow_rows"] > 0 and not stats["slots"]
    if margin == 40.0:
        assert stats["overflow_rows"] == 0 and stats["slots"]


@pytest.mark.parametrize("value", ["u11_f32", "int", "none"])
def test_learned_value_types(sg, trained, value):
    A = inputs.er_column_regular(4096, 12, 9, value=value)
    dA = sg.to_device(A)
    semiring = 1 if value == "none" else 0
    C, _ = sg.learned_multiply(dA, dA, trained, margin=0.1, semiring=semiring)
    P = sg.spgemm(dA, dA, semiring=semiring)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all()) and bool((Cc.col == P.col).all())
    if value != "none":
        assert bool((Cc.val == P.val).all())
    R = oracle.spgemm(A, A, semiring="or_and" if value == "none" else "plus_times")
    assert_pattern_equal(Cc, R)
