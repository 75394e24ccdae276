"""Tensor-core MLP of the learned column closure against the FP64 oracle (oracle/mlp.py).

Tolerance for BF16 products (written here, derived from the arithmetic): BF16 keeps 8
significand bits, unit roundoff u = 2^-9.  Every product rounds both operands (inputs,
weights, activations or output errors) to BF16 and accumulates in FP32, so each layer adds
a relative perturbation of order 2u to what flows through it; four layers forward and four
back give a normwise relative error of a few u (a CPU emulation of the rounding gives
about 2.5u).  The kernels evaluate GELU in its tanh form, at most 4.7e-4 from the erf
definition the oracle uses (1.8e-4 relative where that maximum occurs), below the BF16
rounding each activation receives next.  Tests allow 16u = 2^-5 normwise on every output and
gradient tensor.  The
bare GEMM has exactly representable products (8 x 8 significand bits fit FP32), so only
FP32 accumulation remains: |D - AB^T| <= K 2^-23 (|A||B|^T) elementwise.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -9
TOL_BF16 = 16 * U_BF16


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bf16_round(x):
    torch = _torch()
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("M,N,K", [(128, 16, 32), (300, 128, 128), (256, 256, 200), (77, 32, 8), (1000, 48, 520)])
def test_gemm_bf16_matches_exact_products(M, N, K):
    torch = _torch()
    from paper_2502_14148_gb300 import ocn
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = _bf16_round(rng.standard_normal((M, K)))
    B = _bf16_round(rng.standard_normal((N, K)))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    D = ocn.gemm_bf16(A.cuda(), B.cuda(), status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a, b = A.double().numpy(), B.double().numpy()
    ref = a @ b.T
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(D.cpu().double().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_gemm_rejects_unsupported_shapes():
    torch = _torch()
    from paper_2502_14148_gb300 import ocn
    A = torch.zeros((128, 32), dtype=torch.bfloat16, device="cuda")
    for N, K in [(8, 32), (24, 32), (272, 32)]:
        B = torch.zeros((N, K), dtype=torch.bfloat16, device="cuda")
        with pytest.raises(ocn.OcnError) as ei:
            ocn.gemm_bf16(A, B)
        assert ei.value.status == -1
    A2 = torch.zeros((128, 12), dtype=torch.bfloat16, device="cuda")   # K not a multiple of 8
    with pytest.raises(ocn.OcnError):
        ocn.gemm_bf16(A2, torch.zeros((16, 12), dtype=torch.bfloat16, device="cuda"))


def _net(M=1000, seed=7, sizes=inputs.MLP_SIZES):
    _torch()
    from paper_2502_14148_gb300 import ocn
    params = inputs.mlp_init(seed=seed, sizes=sizes)
    X, T, mask = inputs.mlp_batch(seed=seed, M=M, n_in=sizes[0], n_out=sizes[-1])
    net = ocn.MLP(sizes, max_batch=max(M, 4096))
    net.set_params(params)
    # the oracle sees the same FP32-rounded master weights the device holds
    params32 = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
                for W, b in params]
    return net, params32, X, T, mask


@pytest.mark.parametrize("M", [1000, 128, 37])
def test_forward_matches_oracle(M):
    net, params, X, T, mask = _net(M=M)
    y = net.forward(X).cpu().numpy()
    y_ref, _ = omlp.forward(params, X)
    assert _rel(y, y_ref) < TOL_BF16
    assert np.isfinite(y).all()


def test_gradients_match_oracle():
    """Gradient check: the device's hand-written backward pass against the oracle's chain
    rule (itself pinned by finite differences in the CPU suite), every tensor."""
    net, params, X, T, mask = _net(M=1000)
    loss, g = net.gradients(X, T, mask)
    y, cache = omlp.forward(params, X)
    grads = omlp.backward(params, cache, y, T, mask)
    assert abs(loss - omlp.loss(y, T, mask)) < TOL_BF16 * omlp.loss(y, T, mask)
    got = net.unflatten(g.cpu().numpy())
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, grads)):
        assert _rel(gW, rW) < TOL_BF16, (l, "W", _rel(gW, rW))
        assert _rel(gb, rb) < TOL_BF16, (l, "b", _rel(gb, rb))


def test_gradient_directional_finite_difference():
    """The device gradient predicts the oracle loss change along a random direction."""
    net, params, X, T, mask = _net(M=512)
    _, g = net.gradients(X, T, mask)
    got = net.unflatten(g.cpu().numpy())
    rng = np.random.default_rng(3)
    d = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    h = 1e-4
    plus = [(W + h * dW, b + h * db) for (W, b), (dW, db) in zip(params, d)]
    minus = [(W - h * dW, b - h * db) for (W, b), (dW, db) in zip(params, d)]
    fd = (omlp.loss(omlp.forward(plus, X)[0], T, mask) - omlp.loss(omlp.forward(minus, X)[0], T, mask)) / (2 * h)
    an = sum(float((gW * dW).sum() + (gb * db).sum()) for (gW, gb), (dW, db) in zip(got, d))
    assert abs(an - fd) < TOL_BF16 * abs(fd)


def test_adam_matches_oracle():
    torch = _torch()
    net, params, X, T, mask = _net(M=256, sizes=(32, 64, 64, 16))
    rng = np.random.default_rng(11)
    state = {}
    ref = params
    for step in range(3):
        grads = [(rng.standard_normal(W.shape) * 10.0 ** (-step), rng.standard_normal(b.shape)) for W, b in ref]
        grads = [(gW.astype(np.float32).astype(np.float64), gb.astype(np.float32).astype(np.float64))
                 for gW, gb in grads]
        net.adam(torch.tensor(net.flatten(grads)), lr=1e-3)
        ref = omlp.adam_step(ref, grads, state, lr=1e-3)
    got = net.get_params()
    for (gW, gb), (rW, rb) in zip(got, ref):
        assert np.allclose(gW, rW, rtol=1e-6, atol=3e-6)
        assert np.allclose(gb, rb, rtol=1e-6, atol=3e-6)


def test_training_reduces_loss():
    net, params, X, T, mask = _net(M=2048, sizes=(32, 64, 64, 64, 16))
    T = T.copy()
    T[:, :3] = np.tanh(X[:, :3]) * np.cos(X[:, 3:6])
    losses = [net.train_step(X, T, mask, lr=3e-3) for _ in range(300)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    final, _ = net.gradients(X, T, mask)
    y, _ = omlp.forward([(W.astype(np.float64), b.astype(np.float64)) for W, b in net.get_params()], X)
    assert abs(omlp.loss(y, T, mask) - final) < 0.1 * final


def test_bad_batch_sizes_are_rejected():
    torch = _torch()
    from paper_2502_14148_gb300 import ocn
    net = ocn.MLP((32, 64, 16), max_batch=256)
    with pytest.raises(ocn.OcnError):
        net.forward(np.zeros((257, 32), np.float32))
    with pytest.raises(ocn.OcnError):
        ocn.MLP((32, 60, 16), max_batch=256)


def test_bounded_wait_times_out_and_reports():
    """Failure detection without a fault: a tensor-core kernel whose MMA is never issued gives up its
    bounded wait, reports through its status word and leaves the context usable (a normal GEMM after
    it is still exact)."""
    torch = _torch()
    import time
    from paper_2502_14148_gb300 import ocn
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    ocn._check(ocn.lib().ocn_gemm_timeout_test(ocn.C.c_void_p(status.data_ptr()),
                                               ocn.C.c_void_p(torch.cuda.current_stream().cuda_stream)), "timeout")
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(status.item()) == 1
    assert 0.2 < waited < 10.0
    A = _bf16_round(np.eye(128, 32)).cuda()
    D = ocn.gemm_bf16(A, A[:16].contiguous())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(D.cpu().numpy(), np.eye(128, 32) @ np.eye(128, 32)[:16].T)
