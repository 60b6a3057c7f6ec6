"""The sampling-representation ablation (Sec. IV-E, Fig. 5) on the GPU path:
closed-loop episodes of the trot task (and of the terrain task with its 0.3 m
step box, standing in for the paper's box climb) with each control
representation, scored by the FP64 oracle's L_walk along the realised
trajectory.  The paper ranks Direct far behind the knot representations and
Cubic < Linear < Zeroth-order; the relative ranking, not MuJoCo's cost values,
is what carries over to this simulator."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2409_10469_gb300 import proposal as P, workloads as W  # noqa: E402

MODES = ["direct", "zero", "linear", "cubic"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def oracle_task_cost(states, controls, cfgs):
    """oracle stage cost of every visited state with the control applied from it"""
    out = []
    for e, cfg in enumerate(cfgs):
        w = O.World(cfg.robot)
        S = states.shape[0]
        t = np.arange(S) * cfg.mppi["ctrl_steps"] * cfg.mppi["dt"]
        out.append(O.stage_costs(w, cfg.cost, states[:, e], controls[:, e].astype(np.float64), t).sum())
    return np.array(out)


def ablation(make, E, K, H, S, seed):
    cost = {}
    for mode in MODES:
        st, ct, cfgs = P.run_episodes(make, E, K, H, S, seed=seed, interp=mode)
        cost[mode] = oracle_task_cost(st, ct, cfgs)
    return cost


def summary(cost):
    E = len(next(iter(cost.values())))
    return {"mean": {k: float(v.mean()) for k, v in cost.items()},
            "sem": {k: float(v.std() / np.sqrt(E)) for k, v in cost.items()}}


def test_direct_sampling_is_worst_on_trot():
    def make(e):
        return W.config_trot(K=256, H=60)
    cost = ablation(make, 12, 256, 60, 80, seed=3)
    print(json.dumps(summary(cost)))
    for mode in MODES:
        assert np.all(np.isfinite(cost[mode])), mode
    for mode in ("zero", "linear", "cubic"):
        # paired over the same start states and noise streams
        assert (cost["direct"] - cost[mode]).mean() > 0, mode


@pytest.mark.skipif(os.environ.get("MPPI_FULL") != "1", reason="ablation-scale run: set MPPI_FULL=1")
def test_sampling_representation_ablation_full():
    """Trot, the terrain step and the 0.24 m box climb (K = 1024, H = 100), 32
    paired episodes of 2 s each per representation."""
    res = {}
    for task, make in (("trot", lambda e: W.config_trot(K=1024, H=100)),
                       ("terrain_step", lambda e: W.config_terrain(K=1024, H=100, seed=3)),
                       ("box_climb_24cm", lambda e: W.config_climb(K=1024, H=100, box_height=0.24))):
        cost = ablation(make, 32, 1024, 100, 200, seed=11)
        res[task] = summary(cost)
        res[task]["paired_vs_cubic"] = {k: float((v - cost["cubic"]).mean()) for k, v in cost.items()}
    print(json.dumps(res))
    path = os.environ.get("MPPI_FULL_OUT")
    if path:
        with open(path, "w") as f:
            json.dump(res, f, indent=1)
    for task in res:
        assert all(np.isfinite(v) for v in res[task]["mean"].values())
