"""FP64 reference of the proposer network (test infrastructure).

A plain numpy forward / backward of y = relu(relu(X W1^T + b1) W2^T + b2) . w3 + b3 with
the MSE loss and one Adam step.  With rounding=True it rounds to BF16 exactly where the
CUDA kernels do (weights, the stored activations H1 / H2 and the products' gradient
operands), so the two differ only by the order of FP32 sums; with rounding=False it is
the exact FP64 network, pinned by finite differences and torch autograd.
"""
import numpy as np

F_IN, HID = 48, 256
SIZES = [("W1", (HID, F_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def bf16(x):
    """Round to the nearest BF16 (ties to even) through the FP32 value."""
    b = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(P):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(P[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def forward(P, X, rounding=True):
    p = unpack(P)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    X = r(X)
    W1, W2, w3 = r(p["W1"]), r(p["W2"]), r(p["w3"])
    H1 = r(np.maximum(X @ W1.T + p["b1"], 0.0))
    H2 = r(np.maximum(H1 @ W2.T + p["b2"], 0.0))
    y = H2 @ w3 + p["b3"][0]
    return dict(X=X, W1=W1, W2=W2, w3=w3, H1=H1, H2=H2, y=y)


def gradients(P, X, t, rounding=True):
    """(loss, gradient in the parameter layout) of mean((y - t)^2)."""
    f = forward(P, X, rounding)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    t = np.asarray(t, np.float64)
    B = len(t)
    d = f["y"] - t
    loss = np.mean(d * d)
    dy = 2.0 * d / B
    dw3 = f["H2"].T @ dy
    db3 = np.array([dy.sum()])
    G2 = np.outer(dy, f["w3"]) * (f["H2"] > 0)
    db2 = G2.sum(axis=0)
    G2r = r(G2)
    dW2 = G2r.T @ f["H1"]
    dH1 = G2r @ f["W2"]
    G1 = dH1 * (f["H1"] > 0)
    db1 = G1.sum(axis=0)
    dW1 = r(G1).T @ f["X"]
    return loss, pack(dict(W1=dW1, b1=db1, W2=dW2, b2=db2, w3=dw3, b3=db3))


def adam(P, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    P = P - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return P, m, v
