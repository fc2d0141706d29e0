"""GPU parity of the MLP kernels (tensor-core forward, backward, Adam)
against the numpy oracle run with the same BF16 rounding points.

Tolerances: forward relative 2-norm <= 5e-3 and gradient blocks <= 2e-2
(FP32 accumulation against FP64, and an occasional BF16 rounding of a hidden
activation landing on the other side of a tie)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2208_01339_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2208_01339_gb300.polyprec")


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [1, 7, 16, 100, 1000])
def test_forward_and_gradients_match_oracle(B):
    net = P.Mlp(max_batch=1024, seed=3)
    p = net.params().astype(np.float64)
    x = I.normal(5, 9, B * M.NIN).reshape(B, M.NIN)
    t = I.normal(6, 9, B * M.NOUT).reshape(B, M.NOUT)
    y = net.forward(x)
    _, _, _, yo = M.forward(p, x)
    assert rel(y, yo[:, :M.NOUT]) <= 5e-3
    loss, g = net.grad(x, t)
    lo, go = M.loss_and_grad(p, x, t)
    assert loss == pytest.approx(lo, rel=1e-2)
    for a, b in ((M.OW1, M.OB1), (M.OB1, M.OW2), (M.OW2, M.OB2), (M.OB2, M.OW3), (M.OW3, M.OB3), (M.OB3, M.NPARAM)):
        assert rel(g[a:b], go[a:b]) <= 2e-2, (a, b)


def test_padding_parameters_stay_zero_and_training_fits():
    net = P.Mlp(max_batch=512, seed=4)
    B = 512
    x = I.normal(7, 9, B * M.NIN).reshape(B, M.NIN)
    Wt = I.normal(8, 9, M.NIN * M.NOUT).reshape(M.NIN, M.NOUT) / np.sqrt(M.NIN)
    t = np.tanh(x @ Wt)
    first = net.train_step(x, t, 3e-3)
    for _ in range(400):
        last = net.train_step(x, t, 3e-3)
    assert last < 0.1 * first
    p = net.params()
    assert not p[M.OW1:M.OB1].reshape(M.NH, M.NINP)[:, M.NIN:].any()
    assert not p[M.OW3:M.OB3].reshape(M.NOUTP, M.NH)[M.NOUT:, :].any()
    assert not p[M.OB3 + M.NOUT:].any()


def test_params_roundtrip():
    net = P.Mlp(max_batch=16, seed=1)
    p = net.params()
    q = p * 0.5
    net.params(q)
    np.testing.assert_array_equal(net.params(), q.astype(np.float32))
