"""Learned proposal (pattern 4), judged by the FP64 oracle's task cost:
features match the oracle, proposal sampling (incl. the non-finite fallback)
is bit-exact, and on the box-pushing task a network trained on the plain
controller's own updated means lowers the oracle-judged cost of closed-loop
episodes at equal K and matches plain MPPI with 2x the samples.  Episodes are
paired (same starts and goals for every variant) and the pipeline is
deterministic.  The config-4 scale run is opt-in (MPPI_FULL=1, several
GPU-minutes)."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import features as OF  # noqa: E402
from paper_2409_10469_gb300 import _mppi, proposal as P, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def oracle_task_cost(states, controls, cfgs):
    """oracle L_walk + L_box of each realised episode: the stage cost of every
    visited state with the control applied from it"""
    out = []
    for e, cfg in enumerate(cfgs):
        w = O.World(cfg.robot)
        S = states.shape[0]
        t = np.arange(S) * cfg.mppi["ctrl_steps"] * cfg.mppi["dt"]
        out.append(O.stage_costs(w, cfg.cost, states[:, e], controls[:, e].astype(np.float64), t).sum())
    return np.array(out)


def test_features_match_oracle():
    cfg = W.config_push(seed=103)
    c = _mppi.Controller(cfg.robot, cfg.cost, cfg.mppi)
    X = W.random_states(64, 5, box=True).astype(np.float32)
    for step in (0, 37):
        F = c.features(X, step)
        Fo = np.array([OF.features(x, cfg.cost, cfg.mppi["ctrl_steps"], cfg.mppi["dt"], step)
                       for x in X.astype(np.float64)])
        assert np.max(np.abs(F - Fo)) <= 2e-6
    ct = W.config_trot()
    c2 = _mppi.Controller(ct.robot, ct.cost, ct.mppi)
    Xr = W.random_states(8, 6).astype(np.float32)
    Fo = np.array([OF.features(x, ct.cost, ct.mppi["ctrl_steps"], ct.mppi["dt"], 3) for x in Xr.astype(np.float64)])
    assert np.max(np.abs(c2.features(Xr, 3) - Fo)) <= 2e-6


def test_proposal_sampling_and_fallback_bit_exact():
    cfg = W.config_push()
    m = dict(cfg.mppi, K=200, n_prop=100)
    c = _mppi.Controller(cfg.robot, cfg.cost, m)
    mu = W.stand_mu()
    c.set_nominal(mu)
    mp = mu + np.float32(0.05)
    mp[[3, 17, 40]] = np.nan                       # non-finite entries fall back to the plain mean
    U = torch.empty((200, 48), device="cuda")
    c.sample(9, mu_prop=torch.tensor(mp).cuda(), out=U)
    Uo = O.sample(m, mu, 9, mu_prop=mp)
    assert np.array_equal(U.cpu().numpy().view(np.uint32), Uo.view(np.uint32))
    assert np.all(np.isfinite(Uo))


def make_push(e):
    return W.config_push(K=1024, H=60, seed=100 + e)


def test_learned_proposal_gain():
    E, S = 48, 60
    F, T = P.generate(make_push, E, 2048, 60, S, seed=1)
    net, hist = P.train(F, T, epochs=60, batch=256)
    assert hist[-1] < 0.3 * hist[0]
    cost = {}
    for name, K, use in (("plain512", 512, False), ("prop512", 512, True), ("plain1024", 1024, False)):
        st, ct, cfgs = P.run_episodes(make_push, E, K, 60, S, seed=7, net=net if use else None, n_prop=K // 2)
        assert np.all(np.isfinite(st))
        cost[name] = oracle_task_cost(st, ct, cfgs)
    gain = cost["plain512"] - cost["prop512"]
    print("oracle task cost mean:", {k: float(v.mean()) for k, v in cost.items()},
          "paired gain at K=512: %.1f +- %.1f" % (gain.mean(), gain.std() / np.sqrt(E)))
    # what the trained network gains over plain MPPI at the same K ...
    assert gain.mean() > 0
    # ... and the proposal at K matches plain MPPI at 2K
    assert cost["prop512"].mean() <= cost["plain1024"].mean() * 1.02


def test_learned_proposal_config4_reduced_scale():
    """Config 4 at a reduced scale that the default suite runs: the push task at
    H = 100, teacher plain K = 4096 (24 episodes x 80 control steps: 1,920
    pairs), and the learned-proposal form at K = 2048 (half the samples around
    the network's mean) against plain K = 4096 and plain K = 2048, 24 paired
    episodes x 80 steps judged by the FP64 oracle's task cost.  The network must
    gain over plain MPPI at the same K, and the proposal form at K = 2048 must
    reach plain K = 4096's task cost (the pipeline is deterministic; measured on
    GB300: 4147 +- 298 against 4714 +- 365, plain K = 2048 4695 +- 352); the
    numbers are printed as a record."""
    def make(e):
        return W.config_push(K=4096, H=100, seed=2000 + e)
    E, S = 24, 80
    F, T = P.generate(make, E, 4096, 100, S, seed=21)
    net, hist = P.train(F, T, epochs=60, batch=256)
    assert hist[-1] < 0.5 * hist[0]
    cost = {}
    for name, K, use in (("plain4096", 4096, False), ("prop2048", 2048, True), ("plain2048", 2048, False)):
        st, ct, cfgs = P.run_episodes(make, E, K, 100, S, seed=31, net=net if use else None, n_prop=K // 2)
        assert np.all(np.isfinite(st))
        cost[name] = oracle_task_cost(st, ct, cfgs)
    res = {"pairs": int(F.shape[0]), "episodes": E, "steps": S,
           "mean": {k: float(v.mean()) for k, v in cost.items()},
           "sem": {k: float(v.std() / np.sqrt(E)) for k, v in cost.items()},
           "paired_gain_vs_plain2048": float((cost["plain2048"] - cost["prop2048"]).mean()),
           "paired_diff_vs_plain4096": float((cost["prop2048"] - cost["plain4096"]).mean())}
    print(json.dumps(res))
    assert res["paired_gain_vs_plain2048"] > 0
    assert res["paired_diff_vs_plain4096"] < 0


@pytest.mark.skipif(os.environ.get("MPPI_FULL") != "1", reason="config-4 scale run: set MPPI_FULL=1")
def test_learned_proposal_config4_scale():
    """Config 4: teacher plain K=4096 H=100, ~1e5 pairs; proposal K=2048 (half
    from the proposal) against plain K=4096 and plain K=2048, 64 paired episodes."""
    def make(e):
        return W.config_push(K=4096, H=100, seed=1000 + e)
    E, S_gen, rounds = 64, 400, 4
    Fs, Ts = [], []
    for r in range(rounds):
        F, T = P.generate(make, E, 4096, 100, S_gen, seed=10 + r)
        Fs.append(F)
        Ts.append(T)
    F, T = np.concatenate(Fs), np.concatenate(Ts)
    net, hist = P.train(F, T, epochs=30, batch=512)
    S = 200
    cost = {}
    for name, K, use in (("plain4096", 4096, False), ("prop2048", 2048, True), ("plain2048", 2048, False)):
        st, ct, cfgs = P.run_episodes(make, E, K, 100, S, seed=77, net=net if use else None, n_prop=K // 2)
        cost[name] = oracle_task_cost(st, ct, cfgs)
    res = {"pairs": int(F.shape[0]), "loss_first_last": [hist[0], hist[-1]],
           "mean": {k: float(v.mean()) for k, v in cost.items()},
           "sem": {k: float(v.std() / np.sqrt(E)) for k, v in cost.items()},
           "paired_gain_vs_plain2048": float((cost["plain2048"] - cost["prop2048"]).mean()),
           "paired_diff_vs_plain4096": float((cost["prop2048"] - cost["plain4096"]).mean())}
    print(json.dumps(res))
    path = os.environ.get("MPPI_FULL_OUT")
    if path:
        with open(path, "w") as f:
            json.dump(res, f, indent=1)
    assert np.all(np.isfinite([v.mean() for v in cost.values()]))


def test_step_proposal_one_call_equals_four_calls():
    """mppi_step_proposal (features, forward, proposal, step on the handle's stream)
    gives bit-for-bit the outputs of features -> forward -> set_proposal -> step,
    over a short closed loop, with host and with device x0"""
    cfg = W.config_push(K=1024, H=60, seed=11)
    m = dict(cfg.mppi, n_prop=512)
    rng = np.random.default_rng(5)
    net = _mppi.MLP(64)
    net.set_params((rng.standard_normal(net.nparam) * 0.05).astype(np.float32))
    a = _mppi.Controller(cfg.robot, cfg.cost, m)
    b = _mppi.Controller(cfg.robot, cfg.cost, m)
    x = W.random_states(1, 3, box=True)[0].astype(np.float32)
    for c in (a, b):
        c.set_nominal(W.stand_mu())
    ua, ub = np.zeros(12, np.float32), np.zeros(12, np.float32)
    mua, mub = np.zeros(48, np.float32), np.zeros(48, np.float32)
    for step in range(4):
        F = a.features(x[None], step)
        mp = net.forward(F)[0]
        a.set_proposal(mp)
        a.step(x, step, ua, mua)
        xin = x if step % 2 == 0 else torch.tensor(x).cuda()
        b.step_proposal(net, xin, step, ub, mub)
        assert np.array_equal(ua.view(np.uint32), ub.view(np.uint32)), step
        assert np.array_equal(mua.view(np.uint32), mub.view(np.uint32)), step
        x = x + np.float32(0.01) * np.float32(step + 1)
    c0 = _mppi.Controller(cfg.robot, cfg.cost, cfg.mppi)
    assert c0.step_proposal(net, x, 0, ub, mub, check=False) == _mppi.MPPI_ERR_ARG
