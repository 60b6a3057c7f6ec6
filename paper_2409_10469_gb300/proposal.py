"""Learned proposal for the spline knots, end to end on the C ABI.

The paper points to better sampling distributions as future work (arXiv
2409.10469, Sec. V-B) and cites learning one offline (Sec. II-B).  Here:
  1. plain MPPI (the teacher) runs closed-loop episodes of a task; at every
     control step the robot + task features and the teacher's updated mean
     (Eq. 2) form one training pair;
  2. the proposal network (62 -> 256 -> 256 -> 256 -> 48, BF16 on the tensor
     cores) is trained on those pairs by the library's forward / backward /
     AdamW kernels;
  3. at control time the network maps the current features to a mean, and the
     controller draws the last n_prop of its K samples around it (the first
     of them is the prediction itself); the other samples stay around the
     plain warm-started mean, so plain MPPI remains in every step, and a
     non-finite prediction falls back to the plain mean.
Episodes run on the GPU: the controllers step as one batch, and the plant is
the same simulator advanced one control period with the applied targets held.
The task cost of a realised episode is scored afterwards by the caller (the
tests and scripts use the FP64 oracle as the arbiter).
"""
from __future__ import annotations

import numpy as np

from . import _mppi
from . import workloads as W


class Episodes:
    """E closed-loop episodes of one task, stepped together."""

    def __init__(self, make_cfg, E: int, K: int, H: int, seed: int = 0, n_prop: int = 0,
                 perturb: float = 0.05, inst0: int = 0, interp="cubic"):
        import torch
        self.torch = torch
        self.E, self.K, self.H = E, K, H
        rng = np.random.default_rng(seed)
        self.cfgs, self.ctls = [], []
        for e in range(E):
            cfg = make_cfg(e)
            m = dict(cfg.mppi, K=K, H=H, n_prop=n_prop, inst=inst0 + e, seed=seed, interp=interp)
            c = _mppi.Controller(cfg.robot, cfg.cost, m)
            # the warm start: the task's knots, or its first knot held over the horizon (direct)
            c.set_nominal(cfg.mu0 if c.D == 48 else np.tile(cfg.mu0[:12], c.D // 12).astype(np.float32))
            self.cfgs.append(cfg)
            self.ctls.append(c)
        cfg0 = self.cfgs[0]
        self.nx = len(cfg0.x0)
        self.ctrl_steps = cfg0.mppi["ctrl_steps"]
        self.dt = cfg0.mppi["dt"]
        # knot representations step as one batch; direct targets step controller by controller
        self.batch = _mppi.Batch(self.ctls) if self.ctls[0].D == 48 else None
        # plant: the same simulator, E rollouts over one control period
        pm = dict(cfg0.mppi, K=E, H=max(2, self.ctrl_steps))
        self.plant = _mppi.Controller(cfg0.robot, cfg0.cost, pm)
        X = np.zeros((E, 50), np.float32)
        for e, cfg in enumerate(self.cfgs):
            x = cfg.x0.copy()
            x[7:19] += rng.uniform(-perturb, perturb, 12)
            X[e, :self.nx] = x
        self.X = torch.tensor(X).cuda()
        self.u0 = torch.zeros((E, 12), device="cuda")
        self.step_idx = 0
        self.states, self.controls = [], []

    def features(self):
        torch = self.torch
        F = torch.empty((self.E, 62), device="cuda")
        for e, c in enumerate(self.ctls):
            c.features(self.X[e:e + 1, :self.nx].contiguous(), self.step_idx, out=F[e:e + 1])
        return F

    def control(self, mu_props=None):
        """One MPPI step of every episode (with the given proposal means, if any)."""
        if mu_props is not None:
            for e, c in enumerate(self.ctls):
                c.set_proposal(mu_props[e])
        if self.batch is not None:
            self.batch.step(self.X, np.full(self.E, self.step_idx), u0s=self.u0)
        else:
            for e, c in enumerate(self.ctls):
                c.step(self.X[e, :self.nx].contiguous(), self.step_idx, u0_out=self.u0[e])

    def advance(self):
        """Apply u0 for one control period on the plant, record the visited state."""
        torch = self.torch
        self.states.append(self.X[:, :self.nx].cpu().numpy().copy())
        self.controls.append(self.u0.cpu().numpy().copy())
        U = self.u0.repeat(1, 4).contiguous()
        Hp = max(2, self.ctrl_steps)
        traj = torch.empty((self.E, Hp + 1, self.nx), device="cuda")
        L = torch.empty(self.E, device="cuda")
        x0 = self.X[:, :self.nx].contiguous()
        self.plant.rollouts(x0, U=U, n=self.E, L_out=L, traj_out=traj, x0_per_sample=True)
        self.X[:, :self.nx] = traj[:, self.ctrl_steps]
        self.step_idx += 1

    def updated_means(self):
        torch = self.torch
        mu = torch.empty((self.E, 48), device="cuda")
        self.batch.means(mu_upds=mu)
        return mu

    def close(self):
        if self.batch is not None:
            self.batch.close()
        self.plant.close()
        for c in self.ctls:
            c.close()


def generate(make_cfg, E, K, H, steps, seed=0):
    """Plain-MPPI teacher episodes: (features [N][62], updated means [N][48])."""
    ep = Episodes(make_cfg, E, K, H, seed=seed)
    Fs, Ms = [], []
    for s in range(steps):
        F = ep.features()
        ep.control()
        Fs.append(F.cpu().numpy())
        Ms.append(ep.updated_means().cpu().numpy())
        ep.advance()
    ep.close()
    return np.concatenate(Fs), np.concatenate(Ms)


def train(F, T, epochs=40, batch=512, lr=2e-3, wd=1e-4, seed=0, params=None):
    """Train the proposal network on (F, T); returns (net, loss history)."""
    rng = np.random.default_rng(seed)
    net = _mppi.MLP(batch)
    p = W.mlp_init(seed) if params is None else params
    p = p.copy()
    p[-48:] = T.mean(0)          # output bias starts at the mean target
    net.set_params(p)
    hist = []
    n = F.shape[0]
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        nb = 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            tot += net.train_step(F[idx], T[idx], lr=lr, weight_decay=wd)
            nb += 1
        hist.append(tot / max(nb, 1))
    return net, hist


def run_episodes(make_cfg, E, K, H, steps, seed, net=None, n_prop=0, interp="cubic"):
    """Closed-loop episodes; with `net`, n_prop samples come from the proposal;
    `interp` selects the control representation (Sec. III-B, Fig. 5).
    Returns the visited states [steps][E][nx] and applied controls [steps][E][12]."""
    torch = __import__("torch")
    ep = Episodes(make_cfg, E, K, H, seed=seed, n_prop=n_prop if net is not None else 0, interp=interp)
    for s in range(steps):
        props = None
        if net is not None:
            F = ep.features()
            Y = torch.empty((E, 48), device="cuda")
            net.forward(F, out=Y)
            props = [Y[e] for e in range(E)]
        ep.control(props)
        ep.advance()
    out = (np.array(ep.states), np.array(ep.controls), ep.cfgs)
    ep.close()
    return out
