"""Serving runtime (mppi_server_*): a robot's control is bit-identical alone and
inside a busy mix of concurrent requests, within the update tolerance of the
single-instance step, and equal to the FP64 oracle's update of the same samples;
admission respects the memory budget; a second request for a busy robot is
refused."""
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


def robot(task, K, H, inst):
    cfg = W.task_config(task, K, H)
    c = _mppi.Controller(cfg.robot, cfg.cost, dict(cfg.mppi, inst=inst))
    c.set_nominal(cfg.mu0)
    return c, cfg


def ws_bytes(K):
    al = lambda x: (x + 255) // 256 * 256
    return al(K * 48 * 4) + al(K * 4)


def test_result_same_alone_and_in_the_mix():
    # alone
    srv = _mppi.Server(64 << 20, 4, 2048)
    x, cfg = robot("trot", 700, 80, inst=5)
    rid = srv.add_robot(x)
    outs_alone = []
    for step in range(2):
        srv.submit(rid, cfg.x0, step)
        srv.drain()
        u0, lat = srv.poll(rid)
        outs_alone.append(u0)
    # in a mix of 24 robots with concurrent requests, twice
    specs = W.serving_robots(23, seed=11, K_range=(256, 2048), H_range=(50, 150))
    srv2 = _mppi.Server(256 << 20, 24, 2048)
    others = []
    for i, (task, K, H) in enumerate(specs):
        c, cf = robot(task, K, H, inst=100 + i)
        others.append((srv2.add_robot(c), c, cf))
    x2, cfg2 = robot("trot", 700, 80, inst=5)
    rid2 = srv2.add_robot(x2)
    for step in range(2):
        for j, (r, c, cf) in enumerate(others[: 12]):
            srv2.submit(r, cf.x0, step)
        srv2.tick()
        srv2.submit(rid2, cfg2.x0, step)       # arrives while others are on the GPU
        for j, (r, c, cf) in enumerate(others[12:]):
            srv2.submit(r, cf.x0, step)
        srv2.drain()
        u0, lat = srv2.poll(rid2)
        assert np.array_equal(u0.view(np.uint32), outs_alone[step].view(np.uint32)), step
        for r, c, cf in others:
            assert srv2.poll(r) is not None
    assert np.array_equal(x.get_nominal(), x2.get_nominal())
    st = srv2.stats()
    assert st["completed"] == 48 and st["launches"] >= 2
    # and close to the single-instance step of the same robot
    single, cfg3 = robot("trot", 700, 80, inst=5)
    u0s = np.zeros(12, np.float32)
    single.step(cfg3.x0.astype(np.float32), 0, u0_out=u0s)
    assert np.max(np.abs(u0s - outs_alone[0]) / np.maximum(np.abs(u0s), 1)) <= 1e-6


def test_served_robot_matches_oracle_in_the_mix():
    """one robot (trot, K = 700, H = 80) inside a 24-robot mix with concurrent
    requests, three control steps: its samples are the oracle's Philox knots of
    the nominal it held; their rollout costs (the single-instance kernel, whose
    arithmetic the persistent kernel shares) are the oracle's rollouts of them
    (at most 1% of them beyond both 1e-3 and their chaotic sensitivity); and the
    served control and the robot's next nominal are the oracle's
    Eq. 1 / Eq. 2 mean and shift of those samples and costs to 1e-6"""
    specs = W.serving_robots(23, seed=12, K_range=(256, 2048), H_range=(50, 150))
    srv = _mppi.Server(256 << 20, 24, 2048)
    others = []
    for i, (task, K, H) in enumerate(specs):
        c, cf = robot(task, K, H, inst=200 + i)
        others.append((srv.add_robot(c), c, cf))
    x, cfg = robot("trot", 700, 80, inst=7)
    rid = srv.add_robot(x)
    m = dict(cfg.mppi, inst=7)
    costs = _mppi.Controller(cfg.robot, cfg.cost, m)
    world = O.World(cfg.robot)
    x0 = cfg.x0.astype(np.float32)
    for step in range(3):
        nominal = x.get_nominal().copy()
        for r, c, cf in others[:12]:
            srv.submit(r, cf.x0, step)
        srv.tick()
        srv.submit(rid, x0, step)
        for r, c, cf in others[12:]:
            srv.submit(r, cf.x0, step)
        srv.drain()
        u0, _ = srv.poll(rid)
        U_o = O.sample(m, nominal, step)
        t0 = step * m["ctrl_steps"] * m["dt"]
        L = torch.empty(700, device="cuda")
        costs.rollouts(torch.tensor(x0).cuda(), U=torch.tensor(U_o).cuda(), n=700, t0=t0, L_out=L)
        Lg = L.cpu().numpy()
        x0d = x0.astype(np.float64)
        Lo = O.rollouts(world, cfg.cost, m, t0, x0d, U_o)
        rel = np.abs(Lg - Lo) / np.maximum(np.abs(Lo), 1.0)
        # an 80-step rollout with contacts is chaotic (a contact that switches one
        # sub-step apart changes the rest of the rollout): at most 1% of the
        # samples beyond both 1e-3 and 3x the oracle's own sensitivity to a 1e-7
        # perturbation of x0
        sens = np.zeros(700)
        for sd in range(2):
            xp = x0d * (1 + 1e-7 * np.random.default_rng(sd).standard_normal(x0d.shape))
            Lp = O.rollouts(world, cfg.cost, m, t0, xp, U_o)
            sens = np.maximum(sens, np.abs(Lp - Lo) / np.maximum(np.abs(Lo), 1.0))
        assert np.mean(rel > np.maximum(1e-3, 3 * sens)) <= 0.01, (step, np.percentile(rel, 99), rel.max())
        _, mu_o, _ = O.update(Lg, U_o, m["lam"])
        assert np.max(np.abs(u0 - mu_o[:12]) / np.maximum(np.abs(mu_o[:12]), 1.0)) <= 1e-6, step
        sh = O.shift(mu_o, m["H"], m["ctrl_steps"])
        assert np.max(np.abs(x.get_nominal() - sh) / np.maximum(np.abs(sh), 1.0)) <= 1e-6, step
        for r, c, cf in others:
            assert srv.poll(r) is not None
    costs.close()


def test_admission_by_memory_budget():
    K = 1024
    budget = 2 * ws_bytes(K) + 100        # room for two solves at a time
    srv = _mppi.Server(budget, 6, K)
    rs = []
    for i in range(6):
        c, cfg = robot("stand", K, 50, inst=i)
        rs.append((srv.add_robot(c), c, cfg))
    for r, c, cfg in rs:
        srv.submit(r, cfg.x0, 0)
    srv.tick()
    st = srv.stats()
    assert st["in_flight"] <= 2 and st["queued"] >= 4 and st["pool_in_use"] <= budget
    srv.drain()
    st = srv.stats()
    assert st["completed"] == 6 and st["pool_peak"] <= budget and st["pool_in_use"] == 0
    # a robot whose single solve exceeds the budget is refused at registration
    big, _ = robot("stand", 4 * K, 50, inst=9)
    with pytest.raises(_mppi.MppiError):
        srv.add_robot(big)


def test_busy_robot_refused_until_done():
    srv = _mppi.Server(32 << 20, 2, 512)
    c, cfg = robot("stand", 512, 50, inst=1)
    r = srv.add_robot(c)
    assert srv.submit(r, cfg.x0, 0) == _mppi.MPPI_OK
    assert srv.submit(r, cfg.x0, 1) == _mppi.MPPI_ERR_BUSY
    srv.drain()
    assert srv.poll(r) is not None
    assert srv.submit(r, cfg.x0, 1) == _mppi.MPPI_OK
    srv.drain()


def test_serving_loop_small():
    from paper_2409_10469_gb300 import serve
    out = serve.run(n_robots=8, rate_hz=50.0, duration=0.3, K_range=(512, 1024), H_range=(50, 80),
                    warmup=0.05)
    assert out["requests"] > 0 and out["latency_ms"]["p99"] is not None
    assert out["pool_peak_bytes"] <= out["budget_bytes"]


def test_device_buffers_refused_where_host_memory_is_read():
    """The server reads x0 and writes u0 on the host: device memory there is an
    argument error, returned before anything is read or written."""
    import ctypes as C
    srv = _mppi.Server(32 << 20, 1, 512)
    c, cfg = robot("stand", 512, 50, inst=1)
    r = srv.add_robot(c)
    x_dev = torch.tensor(cfg.x0, dtype=torch.float32, device="cuda")
    u_dev = torch.zeros(12, device="cuda")
    L = _mppi.lib()
    assert L.mppi_server_submit(srv.s, r, C.c_void_p(x_dev.data_ptr()), 0) == _mppi.MPPI_ERR_ARG
    assert srv.submit(r, cfg.x0, 0) == _mppi.MPPI_OK
    srv.drain()
    lat, ready = C.c_double(), C.c_int()
    assert L.mppi_server_poll(srv.s, r, C.c_void_p(u_dev.data_ptr()), C.byref(lat),
                              C.byref(ready)) == _mppi.MPPI_ERR_ARG
    assert srv.poll(r) is not None  # the result is still waiting after the refused poll
