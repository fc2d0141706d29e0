"""Pins of the MLP oracle: analytic gradients against central finite
differences (pure FP64), the BF16 rounding against exact values, and the
parameter count against the C header."""
import os
import re

import numpy as np
import pytest

from oracle import mlp as M
from paper_2208_01339_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_param_count_matches_header():
    h = open(os.path.join(ROOT, "include", "polyprec.h")).read()
    assert int(re.search(r"#define PP_MLP_NPARAM (\d+)", h).group(1)) == M.NPARAM


def test_bf16_rounding_exact_cases():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.140625, 1.0 + 2.0 ** -7])
    want = np.array([1.0, 1.0, 1.0 + 4 * 2.0 ** -8, 1.0, -2.5, 3.140625, 1.0 + 2.0 ** -7])
    np.testing.assert_array_equal(M.bf16(x), want)


def params(seed=1, scale=0.3):
    p = np.zeros(M.NPARAM)
    rnd = I.normal(seed, 9, M.NPARAM) * scale
    W1 = rnd[M.OW1:M.OB1].reshape(M.NH, M.NINP)
    W1[:, M.NIN:] = 0.0
    p[M.OW1:M.OB1] = W1.ravel()
    p[M.OB1:M.OW2] = 0.05 * rnd[M.OB1:M.OW2]
    p[M.OW2:M.OB2] = rnd[M.OW2:M.OB2] / np.sqrt(M.NH)
    p[M.OB2:M.OW3] = 0.05 * rnd[M.OB2:M.OW3]
    W3 = rnd[M.OW3:M.OB3].reshape(M.NOUTP, M.NH) / np.sqrt(M.NH)
    W3[M.NOUT:, :] = 0.0
    p[M.OW3:M.OB3] = W3.ravel()
    b3 = 0.1 * rnd[M.OB3:]
    b3[M.NOUT:] = 0.0
    p[M.OB3:] = b3
    return p


def test_gradients_match_finite_differences():
    p = params()
    x = I.normal(2, 9, 6 * M.NIN).reshape(6, M.NIN)
    t = I.normal(3, 9, 6 * M.NOUT).reshape(6, M.NOUT)
    loss, g = M.loss_and_grad(p, x, t, rounded=False)
    idx = np.concatenate([np.arange(M.OW1, M.OW1 + 40), np.arange(M.OB1, M.OB1 + 10),
                          np.arange(M.OW2, M.OW2 + 40), np.arange(M.OB2, M.OB2 + 10),
                          np.arange(M.OW3, M.OW3 + 3 * M.NH, 37), np.arange(M.OB3, M.OB3 + 3)])
    h = 1e-6
    for j in idx:
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        fd = (M.loss_and_grad(pp, x, t, rounded=False)[0] - M.loss_and_grad(pm, x, t, rounded=False)[0]) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    assert loss > 0
