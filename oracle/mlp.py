"""Oracle of the learned interval predictor (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  A plain numpy FP64
restatement of the 3-layer MLP the library trains on the GPU, with the same
parameter layout and, when `rounded=True`, the same BF16 rounding points
(inputs, weights, hidden activations and back-propagated signals rounded to
BF16; every product accumulated exactly here, in FP32 on the GPU):

  x0 = r(x); h1 = relu(x0 W1^T + b1); h2 = relu(r(h1) W2^T + b2); y = r(h2) W3^T + b3
  L = sum (y - t)^2 / (2B); dY = (y - t)/B
  dW3 = r(dY)^T r(h2), db3 = sum dY, dZ2 = (r(dY) W3) o [h2 > 0]
  dW2 = r(dZ2)^T r(h1), db2 = sum dZ2, dZ1 = (r(dZ2) W2) o [h1 > 0]
  dW1 = r(dZ1)^T x0,   db1 = sum dZ1
with W = r(master) and r = round to BF16 (identity when rounded=False).
"""
import numpy as np

NIN, NINP, NH, NOUT, NOUTP = 8, 16, 128, 3, 8
OW1 = 0
OB1 = OW1 + NH * NINP
OW2 = OB1 + NH
OB2 = OW2 + NH * NH
OW3 = OB2 + NH
OB3 = OW3 + NOUTP * NH
NPARAM = OB3 + NOUTP


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) through FP32."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OW1:OB1].reshape(NH, NINP), p[OB1:OW2], p[OW2:OB2].reshape(NH, NH), p[OB2:OW3],
            p[OW3:OB3].reshape(NOUTP, NH), p[OB3:NPARAM])


def forward(p, x, rounded=True):
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    B = x.shape[0]
    x0 = np.zeros((B, NINP))
    x0[:, :NIN] = r(x)
    z1 = x0 @ r(W1).T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    y = r(h2) @ r(W3).T + b3
    return x0, h1, h2, y


def loss_and_grad(p, x, t, rounded=True):
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    B = x.shape[0]
    x0, h1, h2, y = forward(p, x, rounded)
    res = y[:, :NOUT] - t
    loss = float((res ** 2).sum() / (2.0 * B))
    dY = np.zeros((B, NOUTP))
    dY[:, :NOUT] = res / B
    g = np.zeros(NPARAM)
    g[OW3:OB3] = (r(dY).T @ r(h2)).ravel()
    g[OB3:NPARAM] = dY.sum(axis=0)
    dZ2 = (r(dY) @ r(W3)) * (h2 > 0)
    g[OW2:OB2] = (r(dZ2).T @ r(h1)).ravel()
    g[OB2:OW3] = dZ2.sum(axis=0)
    dZ1 = (r(dZ2) @ r(W2)) * (h1 > 0)
    g[OW1:OB1] = (r(dZ1).T @ x0).ravel()
    g[OB1:OW2] = dZ1.sum(axis=0)
    return loss, g
