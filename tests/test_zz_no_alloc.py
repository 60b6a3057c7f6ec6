"""mppi_update_noalloc -- the update for callers that cannot allocate device
memory (a hard real-time loop that must not block in the allocator, code inside
another framework's memory pool).  Through the C ABI it must give the same
result as the handle-based mppi_update on the same costs and knots, on two calls
in a row (the second reuses the library's fixed scratch array, whose completion
counter the call clears).  Kept in its own file so that pytest collects it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_10469_gb300 import _mppi, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_noalloc_update_matches_handle_update_twice():
    cfg = W.config_trot()
    K = 3000
    m = dict(cfg.mppi, K=K)
    rng = np.random.default_rng(8)
    for call in range(2):
        U = torch.tensor((np.tile(W.stand_mu(), (K, 1)) + rng.normal(0, 0.3, (K, 48))).astype(np.float32)).cuda()
        L = torch.tensor((100 + 7 * rng.random(K)).astype(np.float32)).cuda()
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
                                  mu_upd_out=mu_upd, status_out=status)
        assert rc == _mppi.MPPI_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for got, ref in ((mu_upd, mu_upd_ref), (u0, u0_ref), (mu_out, nominal_ref)):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(g - r) / np.maximum(np.abs(r), 1.0)) <= 1e-6, call


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
