"""Proposal network on the tcgen05 tensor cores against the FP64 oracle:
the raw BF16 GEMM (ragged shapes), the forward pass and the backprop gradient
(the oracle mirrors the BF16 rounding points, so only accumulation order
differs), and training reducing the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402
from paper_2409_10469_gb300 import _mppi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("M_,N_,K_", [(128, 64, 64), (300, 48, 62), (256, 256, 256), (77, 200, 1000),
                                       (1024, 256, 64), (300, 48, 64), (130, 64, 1024), (129, 256, 24),
                                       (39013, 256, 256), (5, 16, 8), (12000, 256, 256), (20000, 200, 128)])
def test_tc_gemm_bf16(M_, N_, K_):
    """K a multiple of 8 takes the TMA-fed pipeline: 64-wide column tiles for few
    row tiles (77 x 200: four column tiles, the last one ragged), 128-wide for
    12000 rows, 256-wide from 152 row tiles on (39013 rows: several tiles per
    persistent CTA and both accumulators); K = 24 and 8: one partial chunk
    zero-filled by TMA.  K = 62 takes the thread-staged kernel"""
    g = torch.Generator().manual_seed(M_ + N_ + K_)
    A = torch.randn(M_, K_, generator=g).to(torch.bfloat16)
    B = torch.randn(N_, K_, generator=g).to(torch.bfloat16)
    D = torch.full((M_, N_), float("nan"), device="cuda")
    Ab = A.contiguous().view(torch.int16).cuda()
    Bb = B.contiguous().view(torch.int16).cuda()
    rc = _mppi.tc_gemm_bf16(Ab, Bb, M_, N_, K_, D)
    assert rc == _mppi.MPPI_OK
    torch.cuda.synchronize()
    ref = A.double().numpy() @ B.double().numpy().T
    got = D.cpu().double().numpy()
    # bf16 products are exact in FP32; only the FP32 accumulation order differs
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.sqrt(K_) * max(1.0, np.max(np.abs(ref)))


def data(B, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, 62)).astype(np.float32), (0.3 * rng.normal(size=(B, 48))).astype(np.float32)


@pytest.mark.parametrize("B", [1, 2, 3, 7, 9, 64, 128, 129, 300])
def test_forward_matches_oracle(B):
    """batches up to 128 take the CUDA-core cluster forward (1, 2, 4 or 8
    samples per 8-CTA cluster: B = 1, 2, 3, 7, one ragged second cluster at 9,
    8 and 16 clusters), larger ones the tensor cores; both mirror the oracle's
    BF16 rounding points"""
    net = _mppi.MLP(512)
    p = M.init_params(5)
    net.set_params(p)
    X, _ = data(B, 1)
    Y = net.forward(X)
    Yo, _ = M.forward(p, X, mirror=True)
    err = np.max(np.abs(Y - Yo)) / max(1.0, np.max(np.abs(Yo)))
    # FP32 vs FP64 accumulation can put a hidden pre-activation on the other side
    # of a BF16 rounding boundary (a 2^-8 flip of one activation): 1e-3 bound
    assert err <= 1e-3, err
    assert np.array_equal(net.get_params(), p)
    # device output buffers too
    Yd = torch.empty((B, 48), device="cuda")
    net.forward(torch.as_tensor(X).cuda(), out=Yd)
    assert np.array_equal(Yd.cpu().numpy(), Y)


@pytest.mark.parametrize("B", [256, 129, 1000, 3, 4096])
def test_gradient_matches_oracle(B):
    """the backward pass reads K-major transposed copies; the weight gradients
    sum over the batch in K ranges (1000 samples: 16 chunks, 4 ranges; 4096: 64
    chunks, 16 ranges, and the forward in 64-wide column tiles)"""
    net = _mppi.MLP(4096)
    p = M.init_params(6)
    net.set_params(p)
    X, T = data(B, 2)
    loss, g = net.train_step(X, T, lr=0.0, grad=True)
    lo, go = M.loss_grad(p, X, T, mirror=True)
    assert abs(loss - lo) <= 1e-4 * max(1.0, abs(lo))
    for (a, b) in _blocks(g, go):
        err = np.max(np.abs(a - b)) / max(1e-12, np.max(np.abs(b)))
        assert err <= 1e-2, err
    # the parameters are untouched when lr = 0
    assert np.array_equal(net.get_params(), p)


def _blocks(g, go):
    o = 0
    for no, ni in M.SIZES:
        yield g[o:o + no * ni], go[o:o + no * ni]
        o += no * ni
        yield g[o:o + no], go[o:o + no]
        o += no


def test_adamw_step_matches_oracle_and_training_converges():
    net = _mppi.MLP(512)
    p = M.init_params(7)
    net.set_params(p)
    X, T = data(512, 3)
    _, g = net.train_step(X, T, lr=1e-3, weight_decay=1e-4, grad=True)
    po, _, _ = M.adamw(p.astype(np.float64), g.astype(np.float64), np.zeros(p.size), np.zeros(p.size), 1,
                       1e-3, 1e-4)
    assert np.max(np.abs(net.get_params() - po)) <= 1e-6
    # a learnable target: T = tanh of a fixed linear map of X
    rng = np.random.default_rng(4)
    Wt = rng.normal(size=(62, 48)) / 8
    Xt = rng.normal(size=(512, 62)).astype(np.float32)
    Tt = np.tanh(Xt @ Wt).astype(np.float32)
    net.set_params(M.init_params(8))
    first = net.train_step(Xt, Tt, lr=2e-3)
    for _ in range(300):
        last = net.train_step(Xt, Tt, lr=2e-3)
    assert last < 0.2 * first, (first, last)


def test_gradient_after_update_uses_updated_transposed_weights():
    """AdamW refreshes W and its transposed BF16 copy W^T together: the next
    gradient (whose dH products read W^T) matches the oracle at the new parameters"""
    net = _mppi.MLP(512)
    net.set_params(M.init_params(9))
    X, T = data(300, 5)
    for _ in range(3):
        net.train_step(X, T, lr=5e-3)
    p1 = net.get_params()
    loss, g = net.train_step(X, T, lr=0.0, grad=True)
    lo, go = M.loss_grad(p1.astype(np.float64), X, T, mirror=True)
    assert abs(loss - lo) <= 1e-4 * max(1.0, abs(lo))
    for (a, b) in _blocks(g, go):
        assert np.max(np.abs(a - b)) / max(1e-12, np.max(np.abs(b))) <= 1e-2


def test_bounded_wait_times_out_and_context_survives():
    """a tensor-core wait that is never signalled runs out after its limit; the
    kernel returns an error status and the GPU stays usable"""
    assert _mppi.lib().mppi_selftest_wait_timeout(None) == _mppi.MPPI_ERR_TIMEOUT
    A = torch.ones(128, 64, dtype=torch.bfloat16).view(torch.int16).cuda()
    B = torch.ones(64, 64, dtype=torch.bfloat16).view(torch.int16).cuda()
    D = torch.zeros(128, 64, device="cuda")
    assert _mppi.tc_gemm_bf16(A, B, 128, 64, 64, D) == _mppi.MPPI_OK
    torch.cuda.synchronize()
    assert torch.all(D == 64.0)
