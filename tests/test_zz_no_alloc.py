"""mppi_update_noalloc -- the update for callers that cannot allocate device
memory (a hard real-time loop that must not block in the allocator, code inside
another framework's memory pool).  Through the C ABI it must give the FP64
oracle's Eq. 1 / Eq. 2 mean and shift, and the same result as the handle-based
mppi_update on the same costs and knots, on two calls in a row (the second
reuses the library's fixed scratch array, whose completion counter the call
clears), for every knot representation; and a call must allocate nothing on the
device.  Kept in its own file so that pytest collects it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import _mppi, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def rel(g, r):
    return float(np.max(np.abs(g - r) / np.maximum(np.abs(r), 1.0)))


@pytest.mark.parametrize("interp", ["cubic", "zero", "linear"])
def test_noalloc_update_matches_oracle_and_handle_twice(interp):
    cfg = W.config_trot()
    K = 3000
    m = dict(cfg.mppi, K=K, interp=interp)
    rng = np.random.default_rng(8)
    for call in range(2):
        Uh = (np.tile(W.stand_mu(), (K, 1)) + rng.normal(0, 0.3, (K, 48))).astype(np.float32)
        Lh = (100 + 7 * rng.random(K)).astype(np.float32)
        U, L = torch.tensor(Uh).cuda(), torch.tensor(Lh).cuda()
        mu_in = torch.tensor(W.stand_mu() + np.float32(0.01 * call)).cuda()
        # the existing entry point, through its handle
        ctl = _mppi.Controller(cfg.robot, cfg.cost, m)
        ctl.set_nominal(mu_in)
        mu_upd_ref = torch.empty(48, device="cuda")
        u0_ref = torch.empty(12, device="cuda")
        assert ctl.update(L, U, n=K, mu_out=mu_upd_ref, u0_out=u0_ref) == 0
        nominal_ref = torch.tensor(ctl.get_nominal()).cuda()
        ctl.close()
        # the allocation-free entry point
        mu_out = torch.empty(48, device="cuda")
        mu_upd = torch.empty(48, device="cuda")
        u0 = torch.empty(12, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = _mppi.update_noalloc(L, U, K, m["H"], m["ctrl_steps"], m["lam"], mu_in, mu_out, u0,
                                  mu_upd_out=mu_upd, status_out=status, interp=interp)
        assert rc == _mppi.MPPI_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for got, ref in ((mu_upd, mu_upd_ref), (u0, u0_ref), (mu_out, nominal_ref)):
            assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-6, (interp, call)
        # the oracle: Eq. 1 / Eq. 2 on the same FP32 costs and knots, then the
        # representation's shift of the GPU's mean
        _, mu_o, _ = O.update(Lh, Uh, m["lam"])
        g = mu_upd.cpu().numpy()
        assert rel(g, mu_o) <= 1e-6, (interp, call)
        assert np.array_equal(u0.cpu().numpy(), g[:12])
        assert rel(mu_out.cpu().numpy(), O.shift(g, m["H"], m["ctrl_steps"], interp)) <= 1e-6, (interp, call)


def test_noalloc_allocates_nothing():
    """after a first call (which looks up the scratch array's address), a call
    changes neither the device's free memory nor torch's allocated bytes"""
    cfg = W.config_trot()
    K = 1024
    m = dict(cfg.mppi, K=K)
    rng = np.random.default_rng(9)
    U = torch.tensor((np.tile(W.stand_mu(), (K, 1)) + rng.normal(0, 0.3, (K, 48))).astype(np.float32)).cuda()
    L = torch.tensor((50 + rng.random(K)).astype(np.float32)).cuda()
    mu = torch.tensor(W.stand_mu()).cuda()
    u0 = torch.empty(12, device="cuda")
    assert _mppi.update_noalloc(L, U, K, m["H"], m["ctrl_steps"], m["lam"], mu, mu, u0) == _mppi.MPPI_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert _mppi.update_noalloc(L, U, K, m["H"], m["ctrl_steps"], m["lam"], mu, mu, u0) == _mppi.MPPI_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_out_of_range_sizes():
    K = 8
    buf = torch.zeros(K * 48, device="cuda")
    small = torch.zeros(48, device="cuda")
    u0 = torch.zeros(12, device="cuda")
    big = (1 << 20) + 1
    assert _mppi.update_noalloc(buf[:K], buf, big, 100, 2, 0.1, small, small, u0) == _mppi.MPPI_ERR_ARG
    assert _mppi.update_noalloc(buf[:K], buf, 0, 100, 2, 0.1, small, small, u0) == _mppi.MPPI_ERR_ARG
    host = np.zeros(48, np.float32)
    assert _mppi.update_noalloc(buf[:K], buf, K, 100, 2, 0.1, host, small, u0) == _mppi.MPPI_ERR_ARG
    # direct targets have 12 H parameters per sample, not 48
    assert _mppi.update_noalloc(buf[:K], buf, K, 100, 2, 0.1, small, small, u0,
                                interp="direct") == _mppi.MPPI_ERR_ARG


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second GPU")
def test_noalloc_rejects_buffers_of_another_gpu():
    K = 8
    other = torch.zeros(K * 48, device="cuda:1")
    small = torch.zeros(48, device="cuda:0")
    u0 = torch.zeros(12, device="cuda:0")
    with torch.cuda.device(0):
        assert _mppi.update_noalloc(other[:K], other, K, 100, 2, 0.1, small, small, u0) == _mppi.MPPI_ERR_ARG
