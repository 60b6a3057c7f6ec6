"""Multi-instance persistent launch (mppi_batch_*): every instance's samples,
costs and update agree with the FP64 oracle (Alg. 1, Eq. 1-2 per instance), its
step equals the single-instance path within the update tolerance, an instance's
result is bit-identical alone and inside a mixed batch, inactive instances are
untouched, the autotuner picks a valid shape and restores the nominals."""
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


def make(cfg, K, H, seed=0, inst=0):
    m = dict(cfg.mppi, K=K, H=H, seed=seed, inst=inst)
    c = _mppi.Controller(cfg.robot, cfg.cost, m)
    c.set_nominal(cfg.mu0)
    return c, m


def x0_row(cfg):
    x = np.zeros(50, np.float32)
    x[:len(cfg.x0)] = cfg.x0
    return x


def mix():
    return [(W.config_stand(), 100, 50), (W.config_terrain(), 64, 60), (W.config_push(), 96, 100),
            (W.config_trot(), 300, 100)]


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def test_batch_matches_oracle_per_instance():
    """each instance of a mixed batch (stand, heightfield + step box, push,
    trot), two control steps: its knots are the oracle's Philox samples
    bit for bit, its costs are the oracle's rollouts of those knots (at most 1%
    of the samples, or one, beyond both 1e-3 and 3x the oracle's own
    sensitivity to a 1e-7 perturbation of x0: a 100-step rollout with contacts
    is chaotic), and
    its mean, applied control and shifted
    nominal are the oracle's Eq. 1 / Eq. 2 and shift on those knots and costs
    (<= 1e-6)"""
    items = mix()
    members = [make(c, K, H, inst=i) for i, (c, K, H) in enumerate(items)]
    batch = _mppi.Batch([c for c, _ in members])
    x0s = np.stack([x0_row(c) for c, _, _ in items])
    for step in (0, 1):
        before = [c.get_nominal().copy() for c, _ in members]
        u0b = np.zeros((len(items), 12), np.float32)
        batch.step(x0s, np.full(len(items), step), u0s=u0b)
        mu_upds = np.zeros((len(items), 48), np.float32)
        noms = np.zeros((len(items), 48), np.float32)
        batch.means(mu_upds, noms)
        for i, ((cfg, K, H), (ctl, m)) in enumerate(zip(items, members)):
            Ub, Lb = ctl.last_samples()
            assert np.array_equal(Ub.view(np.uint32), O.sample(m, before[i], step).view(np.uint32)), (i, step)
            world = O.World(cfg.robot)
            t0 = step * m["ctrl_steps"] * m["dt"]
            x0 = cfg.x0.astype(np.float32).astype(np.float64)
            Lo = O.rollouts(world, cfg.cost, m, t0, x0, Ub)
            r = rel(Lb.astype(np.float64), Lo)
            sens = np.zeros(K)
            for sd in range(2):
                xp = x0 * (1 + 1e-7 * np.random.default_rng(sd).standard_normal(x0.shape))
                sens = np.maximum(sens, rel(O.rollouts(world, cfg.cost, m, t0, xp, Ub), Lo))
            n_out = int(np.sum(r > np.maximum(1e-3, 3 * sens)))
            assert n_out <= max(1, K // 100), (i, step, n_out, np.percentile(r, 95), r.max())
            _, mu_o, _ = O.update(Lb, Ub, m["lam"])
            assert rel(mu_upds[i], mu_o).max() <= 1e-6, (i, step)
            assert np.array_equal(u0b[i], mu_upds[i][:12])
            assert rel(noms[i], O.shift(mu_upds[i], H, m["ctrl_steps"])).max() <= 1e-6, (i, step)
            assert np.array_equal(noms[i], ctl.get_nominal())


def test_batch_matches_single_instance_steps():
    items = mix()
    singles = [make(c, K, H, inst=i) for i, (c, K, H) in enumerate(items)]
    batched = [make(c, K, H, inst=i) for i, (c, K, H) in enumerate(items)]
    batch = _mppi.Batch([c for c, _ in batched])
    x0s = np.stack([x0_row(c) for c, _, _ in items])
    for step in (0, 1):
        u0b = np.zeros((len(items), 12), np.float32)
        batch.step(x0s, np.full(len(items), step), u0s=u0b)
        for i, ((cfg, K, H), (ctl, m)) in enumerate(zip(items, singles)):
            u0 = np.zeros(12, np.float32)
            ctl.step(cfg.x0.astype(np.float32), step, u0_out=u0)
            assert np.max(np.abs(u0b[i] - u0) / np.maximum(np.abs(u0), 1)) <= 1e-6, (i, step)
            nb, ns = batched[i][0].get_nominal(), ctl.get_nominal()
            assert np.max(np.abs(nb - ns) / np.maximum(np.abs(ns), 1)) <= 1e-6, (i, step)
    assert batch.launch_count() == 2


def test_shared_model_batch_matches_single_instance_steps():
    """three heightfield controllers (each handle uploads its own copy of the
    same heights) with different K, H and noise streams share one model: the
    batch takes the parameter-bank kernel and matches the single-instance path;
    a mix of tasks does not share"""
    items = [(W.config_terrain(), 64, 60), (W.config_terrain(), 200, 100), (W.config_terrain(), 96, 50)]
    singles = [make(c, K, H, seed=11, inst=i) for i, (c, K, H) in enumerate(items)]
    batched = [make(c, K, H, seed=11, inst=i) for i, (c, K, H) in enumerate(items)]
    batch = _mppi.Batch([c for c, _ in batched])
    assert batch.shared_model()
    x0s = np.stack([x0_row(c) for c, _, _ in items])
    for step in (0, 1, 2):
        u0b = np.zeros((len(items), 12), np.float32)
        batch.step(x0s, np.full(len(items), step), u0s=u0b)
        for i, ((cfg, K, H), (ctl, m)) in enumerate(zip(items, singles)):
            u0 = np.zeros(12, np.float32)
            ctl.step(cfg.x0.astype(np.float32), step, u0_out=u0)
            assert np.max(np.abs(u0b[i] - u0) / np.maximum(np.abs(u0), 1)) <= 1e-6, (i, step)
    mixed = _mppi.Batch([make(c, K, H, inst=i)[0] for i, (c, K, H) in enumerate(mix())])
    assert not mixed.shared_model()


def push_on_steps():
    """the push task on a model that also has a static box (out of the robot's
    reach): the free box and the static-environment code in one model"""
    cfg = W.config_push()
    rb = W.robot(box=True, static_boxes=[((2.5, -0.5, -0.2), (3.0, 0.5, 0.1))])
    return W.Workload("push_static_box", rb, cfg.cost, cfg.mppi, cfg.x0, cfg.mu0, cfg.steps)


ALONE = {"trot": W.config_trot, "terrain": W.config_terrain, "push": W.config_push,
         "push_static_box": push_on_steps}


@pytest.mark.parametrize("task", list(ALONE))
def test_batch_alone_equals_mixed_bit_exact(task):
    """a one-instance batch takes the parameter-bank kernel of its model's
    terrain / free-box variant (flat, terrain, free box, free box with a static
    box), the mixed batch the general one: the same instance's results are
    bit-identical"""
    cfg = ALONE[task]()
    alone, _ = make(cfg, 256, 50, seed=7, inst=3)
    b1 = _mppi.Batch([alone])
    assert b1.shared_model()
    twin, _ = make(cfg, 256, 50, seed=7, inst=3)
    others = [make(W.config_terrain(), 512, 150, inst=9)[0], make(W.config_stand(), 1024, 100, inst=4)[0],
              make(W.config_push(), 128, 100, inst=5)[0]]
    b2 = _mppi.Batch([others[0], twin, others[1], others[2]])
    assert not b2.shared_model()
    x0 = x0_row(cfg)
    x0s = np.stack([x0_row(W.config_terrain()), x0, x0_row(W.config_stand()), x0_row(W.config_push())])
    for step in range(3):
        u1 = np.zeros((1, 12), np.float32)
        u2 = np.zeros((4, 12), np.float32)
        b1.step(x0[None], [step], u0s=u1)
        b2.step(x0s, [step] * 4, u0s=u2)
        assert np.array_equal(u1[0].view(np.uint32), u2[1].view(np.uint32)), step
        assert np.array_equal(alone.get_nominal().view(np.uint32), twin.get_nominal().view(np.uint32)), step


def test_batch_inactive_untouched_and_device_io():
    items = mix()
    ctls = [make(c, K, H, inst=i)[0] for i, (c, K, H) in enumerate(items)]
    batch = _mppi.Batch(ctls)
    before = [c.get_nominal().copy() for c in ctls]
    x0s = torch.tensor(np.stack([x0_row(c) for c, _, _ in items])).cuda()
    u0s = torch.zeros((len(items), 12), device="cuda")
    batch.step(x0s, np.zeros(len(items)), u0s=u0s, active=[1, 0, 1, 0])
    torch.cuda.synchronize()
    assert np.array_equal(ctls[1].get_nominal(), before[1]) and np.array_equal(ctls[3].get_nominal(), before[3])
    assert not np.array_equal(ctls[0].get_nominal(), before[0])
    assert torch.all(u0s[1] == 0) and torch.any(u0s[0] != 0)


def test_batch_autotune_valid_and_restores_nominals():
    items = mix()
    ctls = [make(c, K, H, inst=i)[0] for i, (c, K, H) in enumerate(items)]
    batch = _mppi.Batch(ctls)
    before = [c.get_nominal().copy() for c in ctls]
    x0s = np.stack([x0_row(c) for c, _, _ in items])
    blk, bpsm, ms = batch.autotune(x0s, trials=2)
    assert blk in (64, 128, 256) and bpsm >= 1 and ms > 0
    assert batch.shape() == (blk, bpsm)
    for c, b in zip(ctls, before):
        assert np.array_equal(c.get_nominal(), b)
    with pytest.raises(_mppi.MppiError):
        batch.set_shape(96, 1)
