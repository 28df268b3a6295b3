"""Tensor-core (tcgen05) GEMM of the learned proposer against an FP64 numpy product of
the same BF16-rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ref(A, B, transA, transB):
    a = A.float().cpu().numpy().astype(np.float64)
    b = B.float().cpu().numpy().astype(np.float64)
    a = a.T if transA else a
    b = b.T if transB else b
    return a @ b.T


@pytest.mark.parametrize("M,N,K,tA,tB", [(128, 256, 48, 0, 0), (128, 16, 16, 0, 0), (256, 256, 256, 0, 0),
                                         (300, 48, 64, 0, 0), (200, 256, 80, 1, 0), (256, 48, 384, 1, 1),
                                         (384, 512, 32, 0, 1), (130, 32, 4096, 1, 1)])
def test_gemm_matches_fp64(M, N, K, tA, tB):
    import torch
    from paper_1901_06229_b300 import mlp
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((K, M) if tA else (M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((K, N) if tB else (N, K), generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    mlp.gemm(A, B, M, N, K, transA=tA, transB=tB, C_out=C, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = _ref(A, B, tA, tB)
    got = C.cpu().numpy()
    # FP32 accumulation of K products of O(1) BF16 values; a layout error is O(1)
    bound = 1e-4 * np.sqrt(K)
    assert np.isfinite(got).all()
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=bound)


def test_gemm_epilogue_bias_relu_bf16_and_dot():
    import torch
    from paper_1901_06229_b300 import mlp
    g = torch.Generator(device="cpu").manual_seed(5)
    M, N, K = 256, 256, 48
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    w = torch.randn(N, generator=g).cuda()
    Cb = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(M, device="cuda")
    mlp.gemm(A, B, M, N, K, Cb_out=Cb, bias=bias, relu=True, dotw=w, dot_bias=0.25, dot_out=y)
    torch.cuda.synchronize()
    x = np.maximum(_ref(A, B, 0, 0) + bias.cpu().numpy()[None, :], 0.0)
    xb = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float().numpy()
    got = Cb.float().cpu().numpy()
    # the kernel rounds its FP32 value to BF16: at most one BF16 ulp from rounding the FP64 value
    np.testing.assert_allclose(got, xb, rtol=2 ** -7, atol=1e-6)
    np.testing.assert_allclose(y.cpu().numpy(), got.astype(np.float64) @ w.cpu().numpy() + 0.25, rtol=1e-4, atol=1e-3)


def _net_case(seed, B):
    rng = np.random.default_rng(seed)
    from oracle import mlp as om
    P = (rng.normal(scale=0.15, size=om.NPARAM)).astype(np.float32)
    X = rng.uniform(0, 1, size=(B, 48)).astype(np.float32)
    t = rng.uniform(0, 1, size=B).astype(np.float32)
    return P, X, t


STEPS = 4  # BF16 steps (2^-7 relative) of an element's absolute mass the device may differ by


def grad_mass(P, X, t):
    """Each gradient element's absolute mass: its sum over the batch with every factor
    replaced by its absolute value (|G2|^T |H1| for dW2, and so on down the backward
    pass).  The device and the oracle round the same operands (H1, H2, G2, G1) to BF16;
    where an FP32 and an FP64 value straddle a BF16 rounding boundary the operand moves by
    one BF16 step (at most 2^-7 of it), and through y such a move shifts every later
    factor of its row by a comparable share.  An element's difference is therefore a
    small number of BF16 steps of its mass -- not of the (often cancelling) gradient."""
    from oracle import mlp as om
    f = om.forward(P, X, rounding=True)
    B = len(t)
    dy = np.abs(2.0 * (f["y"] - np.asarray(t, np.float64)) / B)
    aw3, aH1, aH2, aX = np.abs(f["w3"]), np.abs(f["H1"]), np.abs(f["H2"]), np.abs(f["X"])
    G2 = np.outer(dy, aw3) * (f["H2"] > 0)
    G1 = (G2 @ np.abs(f["W2"])) * (f["H1"] > 0)
    return om.pack(dict(W1=G1.T @ aX, b1=G1.sum(0), W2=G2.T @ aH1, b2=G2.sum(0), w3=aH2.T @ dy,
                        b3=np.array([dy.sum()])))


# 512 rows: 8 K ranges of the weight-gradient GEMMs; 1,008: 16, the last one 48 rows;
# 4,096: the 64-range maximum
@pytest.mark.parametrize("B", [512, 1008, 4096])
def test_network_forward_and_gradients_match_oracle(B):
    import torch
    from oracle import mlp as om
    from paper_1901_06229_b300 import mlp
    P, X, t = _net_case(7, B)
    net = mlp.MLP(0, seed=1, max_batch=4096)
    net.set_params(P)
    Xb = torch.tensor(X).to(torch.bfloat16).cuda()
    tt = torch.tensor(t).cuda()
    y = torch.zeros(B, device="cuda")
    net.predict(Xb, y)
    grad = torch.zeros(net.nparam, device="cuda")
    loss = torch.zeros(1, device="cuda")
    net.gradients(Xb, tt, grad, loss)
    torch.cuda.synchronize()
    assert net.error() == 0
    Xr = Xb.float().cpu().numpy()
    f = om.forward(P, Xr, rounding=True)
    np.testing.assert_allclose(y.cpu().numpy(), f["y"], rtol=1e-3, atol=2e-3)
    ref_loss, ref = om.gradients(P, Xr, t, rounding=True)
    assert abs(loss.item() - ref_loss) <= 1e-3 * ref_loss + 1e-6
    g = grad.cpu().numpy().astype(np.float64)
    mass = grad_mass(P, Xr, t)
    o = 0
    for name, shape in om.SIZES:
        n = int(np.prod(shape))
        a, b, lim = g[o:o + n], ref[o:o + n], STEPS * 2.0 ** -7 * mass[o:o + n] + 1e-7
        err = np.abs(a - b)
        worst = int(np.argmax(err / lim))
        print(name, "largest error in BF16 steps of the element's mass:",
              float(err[worst] / (2.0 ** -7 * mass[o + worst] + 1e-30)))
        assert np.all(err <= lim), (name, worst, a[worst], b[worst], lim[worst])
        assert np.corrcoef(a, b)[0, 1] > 0.9999 if n > 1 else True
        o += n
    net.close()


def test_training_reduces_loss():
    import torch
    from paper_1901_06229_b300 import mlp
    rng = np.random.default_rng(9)
    N = 8192
    X = rng.uniform(0, 1, size=(N, 48)).astype(np.float32)
    t = (0.5 + 0.3 * np.sin(3 * X[:, 0]) * X[:, 5] + 0.2 * X[:, 30] ** 2).astype(np.float32)
    Xb = torch.tensor(X).to(torch.bfloat16).cuda()
    tt = torch.tensor(t).cuda()
    net = mlp.MLP(0, seed=3, max_batch=1024)
    loss = torch.zeros(1, device="cuda")
    losses = []
    for epoch in range(8):
        perm = torch.randperm(N, generator=torch.Generator().manual_seed(epoch)).to(torch.int32).cuda()
        for b in range(N // 1024):
            net.train_step(Xb, tt, 1e-3, loss=loss, idx=perm[b * 1024:(b + 1) * 1024], B=1024)
            losses.append(loss.item())
    assert net.error() == 0
    first, last = np.mean(losses[:4]), np.mean(losses[-4:])
    print(first, last)
    assert last < 0.05 * first
    net.close()


@pytest.mark.parametrize("M", [1, 127, 1000, 70000, 262221])
def test_fused_predict_matches_oracle(M):
    import torch
    from oracle import mlp as om
    from paper_1901_06229_b300 import mlp
    P, X, _ = _net_case(11, M)
    net = mlp.MLP(0, seed=1, max_batch=1024)
    net.set_params(P)
    Xb = torch.tensor(X).to(torch.bfloat16).cuda()
    y = torch.full((M + 5,), float("nan"), device="cuda")
    net.predict(Xb, y[:M])
    torch.cuda.synchronize()
    assert net.error() == 0
    got = y.cpu().numpy()
    assert np.isnan(got[M:]).all(), "wrote past the last row"
    f = om.forward(P, Xb.float().cpu().numpy(), rounding=True)
    err = np.abs(got[:M] - f["y"])
    # a hidden activation whose FP32 and FP64 sums round to neighbouring BF16 values moves
    # y by one BF16 ulp (2^-8 relative) of that unit's contribution: bound per row by the
    # row's total |H2 w3| mass; typical rows agree to FP32 summation error
    mass = np.abs(f["H2"]) @ np.abs(f["w3"])
    assert np.all(err <= 2.0 ** -7 * mass + 1e-3), err.max()
    assert np.median(err) <= 1e-4
    net.close()
