"""Learned warm start of the Sinkhorn solves (not part of the paper).

Each solve of an outer iteration starts from the cold first column update
v1 that fa_align_iter leaves in ``log_v``; its converged column scaling v*
differs from it by the correction c = log v* - log v1.  Consecutive outer
iterations have similar corrections, so the warm start is

    warm_log_v = log v1 + c_prev + clamp(f(features)),

where c_prev is the previous solve's correction (0 at the first) and f, a
2-layer graph network on the column graph G2 (hidden width 64, BF16
weights), predicts the change of the correction, c - c_prev, from per-column
inputs: the cold update log v1, c_prev, the previous converged potential
log v*_prev, the degree, the anchor flag and the outer-iteration index.  With f = 0
this is the "previous correction" warm start; the network learns what that
misses.  The plain cold start (no warm start) stays available and is the
reference the model is judged against.  The model's forward, backward and Adam kernels are the library's
(fa_gnn_*); this module only moves tensors and decides what to call.

Training data are the method's own solves: Chung-Lu pairs with n uniform in
[2000, 5000], degree exponent in [2.1, 2.8] and 5-20% edge noise; every
outer iteration contributes one (features, target) sample.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np
import torch

from . import _lib as L
from . import api, synth

NP = L.FA_GNN_NPARAMS
FIN, HID = L.FA_GNN_FIN, L.FA_GNN_HIDDEN
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gnn_weights.json")


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters (He-scaled W1, small w2, zero biases),
    rounded to values BF16 represents exactly."""
    from .synth import bf16_representable
    rng = synth.rng_for(seed)
    th = np.zeros(NP, np.float32)
    th[: FIN * HID] = rng.standard_normal(FIN * HID) * np.sqrt(2.0 / FIN)
    th[FIN * HID + HID: FIN * HID + 2 * HID] = rng.standard_normal(HID) * np.sqrt(1.0 / HID)
    return bf16_representable(th)


class WarmStartModel:
    """The device-resident model with its optimiser state and workspaces."""

    def __init__(self, theta: np.ndarray | None = None, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        self.h = L.fa_gnn_create()
        L.fa_gnn_set_params(self.h, init_params(seed) if theta is None else theta)
        self.grad = torch.zeros(NP, dtype=torch.float32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self._ws = {}

    def ws(self, n: int) -> torch.Tensor:
        w = self._ws.get(n)
        if w is None:
            w = torch.empty(L.fa_gnn_workspace_floats(n), dtype=torch.float32, device=self.device)
            self._ws[n] = w
        return w

    def features(self, graph: api.Graph, log_v1, corr_prev, pot_prev=None, anchor_mask=None,
                 outer_index: int = 0, F=None):
        F = torch.empty((graph.n, FIN), dtype=torch.float32, device=self.device) if F is None else F
        L.fa_gnn_features(graph.handle, log_v1, corr_prev, pot_prev, anchor_mask, outer_index,
                          F, self.ws(graph.n))
        return F

    def predict(self, graph: api.Graph, F, out=None):
        out = torch.empty(graph.n, dtype=torch.float32, device=self.device) if out is None else out
        L.fa_gnn_forward(self.h, graph.handle, F, self.ws(graph.n), out)
        return out

    def train_step(self, graph: api.Graph, F, y, lr: float):
        a = self.predict(graph, F)
        L.fa_gnn_backward(self.h, graph.handle, self.ws(graph.n), a, y, self.grad, self.loss)
        L.fa_gnn_adam_step(self.h, self.grad, lr)
        return self.loss

    def params(self) -> np.ndarray:
        return L.fa_gnn_get_params(self.h)

    def save(self, path: str = WEIGHTS_PATH, meta: dict | None = None):
        with open(path, "w") as f:
            json.dump({"nparams": NP, "theta": [float(x) for x in self.params()],
                       "meta": meta or {}}, f, indent=0)

    @staticmethod
    def load(path: str = WEIGHTS_PATH, device="cuda") -> "WarmStartModel":
        d = json.load(open(path))
        return WarmStartModel(np.asarray(d["theta"], np.float32), device=device)

    def close(self):
        if getattr(self, "h", None):
            L.fa_gnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmStarter:
    """Warm-start protocol for the solves of one alignment.

    mode "cold":    no warm start (fa_sinkhorn's first b update uses v1).
    mode "prev":    warm_log_v = log v1 + c_prev (the previous solve's correction).
    mode "learned": warm_log_v = log v1 + c_prev + alpha clamp(model(features)),
                    alpha in [0, 1] the least-squares scale of the previous
                    solve's prediction against the change it predicted (1
                    before the first fit): the previous solve calibrates how
                    far the network is trusted on this pair.
    Call ``before_solve`` right after fa_align_iter and ``after_solve``
    after fa_sinkhorn, or ``solve`` for both with the cold-start fallback."""

    MAX_CORR = 20.0     # bound on a predicted change of the correction (log units)
    CALIBRATE = True    # fit the trust alpha after every solve (False: alpha = 1)
    SHRINK = 0          # alpha alone (1: alpha rho^2, 2: alpha |rho|, rho the correlation)

    def __init__(self, aligner: api.Aligner, mode: str = "learned",
                 model: WarmStartModel | None = None, anchors=None):
        if mode == "learned" and model is None:
            raise ValueError("learned warm start needs a model")
        self.al, self.mode, self.model = aligner, mode, model
        dev = aligner.device
        n2 = aligner.n2
        self.log_v1 = torch.empty(n2, dtype=torch.float32, device=dev)
        self.corr = torch.zeros(n2, dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n2, dtype=torch.float32, device=dev)    # previous log v*
        self.warm = torch.empty(n2, dtype=torch.float32, device=dev)
        self.base = torch.empty(n2, dtype=torch.float32, device=dev)
        self.F = torch.empty((n2, FIN), dtype=torch.float32, device=dev)
        self.t = 0                      # solves done
        self._anchors = anchors         # default: the aligner's, at the first solve
        self.anchor_mask = None
        self.pred = torch.zeros(n2, dtype=torch.float32, device=dev)   # last prediction
        self.change = torch.empty(n2, dtype=torch.float32, device=dev)
        self.alpha = torch.ones(1, dtype=torch.float32, device=dev)    # trust in the network
        self.predicted = False

    def _mask(self):
        """1 at every column that is an anchor's partner (built once)."""
        if self.anchor_mask is None:
            a = self._anchors if self._anchors is not None else getattr(self.al, "anchors", None)
            m = torch.zeros(self.al.n2, dtype=torch.float32)
            if a is not None and len(a):
                m[torch.as_tensor(np.asarray(a)[:, 1], dtype=torch.long)] = 1.0
            self.anchor_mask = m.to(self.al.device)
        return self.anchor_mask

    def before_solve(self):
        L.fa_vec_axpby(self.al.n2, 1.0, self.al.log_v, 0.0, None, self.log_v1)
        if self.mode == "cold":
            return None
        if self.mode == "prev":
            L.fa_vec_axpby(self.al.n2, 1.0, self.log_v1, 1.0, self.corr, self.warm)
            return self.warm
        self.model.features(self.al.g2, self.log_v1, self.corr,
                            self.pot if self.t > 0 else None, self._mask(), self.t, self.F)
        self.model.predict(self.al.g2, self.F, out=self.pred)
        self.predicted = True
        # base = log v1 + c_prev, then warm = base + alpha clamp(pred)
        L.fa_vec_axpby(self.al.n2, 1.0, self.log_v1, 1.0, self.corr, self.base)
        L.fa_gnn_warm_start(self.al.n2, self.base, self.pred, self.MAX_CORR, self.warm,
                            scale=self.alpha)
        return self.warm

    def after_solve(self):
        if self.predicted and self.CALIBRATE:
            # the change of the correction this solve produced, c - c_prev,
            # against the prediction: the next solve's trust alpha
            L.fa_vec_axpby(self.al.n2, 1.0, self.al.log_v, -1.0, self.log_v1, self.change)
            L.fa_vec_axpby(self.al.n2, 1.0, self.change, -1.0, self.corr, self.change)
            L.fa_gnn_fit_scale(self.al.n2, self.pred, self.change, self.MAX_CORR, self.alpha,
                               shrink=self.SHRINK)
            self.predicted = False
        L.fa_vec_axpby(self.al.n2, 1.0, self.al.log_v, -1.0, self.log_v1, self.corr)
        L.fa_vec_axpby(self.al.n2, 1.0, self.al.log_v, 0.0, None, self.pot)
        self.t += 1

    def state(self) -> dict:
        """What the next solve depends on besides the plan: the previous
        solve's correction and converged potential, and the number of
        solves done (host copies, for checkpoints)."""
        return {"mode": self.mode, "corr": self.corr.cpu(), "pot": self.pot.cpu(), "t": self.t,
                "alpha": self.alpha.cpu()}

    def load_state(self, st: dict) -> None:
        if st.get("mode") != self.mode or tuple(st["corr"].shape) != tuple(self.corr.shape):
            raise ValueError("warm-start state of another mode or size")
        self.corr.copy_(st["corr"])
        self.pot.copy_(st["pot"])
        self.alpha.copy_(st["alpha"])
        self.t = int(st["t"])

    def solve(self, max_iter: int, tol: float, check_every: int = 5):
        """One warm-started solve; if it meets NaN/Inf (a bad prediction),
        the cold start runs from the same kernel instead.  Returns
        (iterations, error, status, used_fallback)."""
        warm = self.before_solve()
        try:
            it, err, st = self.al.sinkhorn(max_iter, tol, check_every, warm)
            fell_back = False
        except L.FastAlignError as e:
            if warm is None or e.status != L.FA_ERR_NUMERIC:
                raise
            L.fa_vec_axpby(self.al.n2, 1.0, self.log_v1, 0.0, None, self.al.log_v)
            it, err, st = self.al.sinkhorn(max_iter, tol, check_every, None)
            fell_back = True
        self.after_solve()
        return it, err, st, fell_back


@dataclasses.dataclass
class Sample:
    graph: api.Graph          # column graph G2 (kept alive)
    F: torch.Tensor           # n x FIN features
    y: torch.Tensor           # n targets: change of the correction, c - c_prev


def training_pair(k: int, seed: int) -> synth.GraphPair:
    """The k-th training pair: n ~ U[2000, 5000], exponent ~ U[2.1, 2.8],
    edge noise ~ U[5%, 20%], 64-dim attributes, 5% anchors."""
    rng = synth.rng_for(seed * 100003 + k)
    n = int(rng.integers(2000, 5001))
    gamma = float(rng.uniform(2.1, 2.8))
    noise = float(rng.uniform(0.05, 0.20))
    e1 = synth.chung_lu(n, gamma, 10.0, rng)
    return synth.make_pair(e1, n, d=64, sigma=0.1, anchor_frac=0.05, frac_del=noise,
                           frac_add=noise, rng=rng, name=f"train{k}", seed=seed)


def large_training_pair(k: int, seed: int) -> synth.GraphPair:
    """The k-th larger training pair: n ~ U[10000, 30000], exponent ~
    U[2.1, 2.8], edge noise ~ U[5%, 20%], 64- or 128-dim attributes, 5%
    anchors.  Solves on pairs this size teach the network the dynamics of
    the large workloads, which the 2k-5k pairs alone do not."""
    rng = synth.rng_for(seed * 100003 + k)
    n = int(rng.integers(10000, 30001))
    gamma = float(rng.uniform(2.1, 2.8))
    noise = float(rng.uniform(0.05, 0.20))
    d = int(rng.choice([64, 128]))
    e1 = synth.chung_lu(n, gamma, 10.0, rng)
    return synth.make_pair(e1, n, d=d, sigma=0.1, anchor_frac=0.05, frac_del=noise,
                           frac_add=noise, rng=rng, name=f"trainL{k}", seed=seed)


def generate_solves(n_pairs: int, outer: int, seed: int = 7, tol: float = 1e-5,
                    max_sweeps: int = 20000, dtype: str = "f32", log=None,
                    pair_fn=None):
    """Run the method on training pairs and record, for every outer
    iteration, the features and the change of the converged correction
    c - c_prev.  The solves start from the previous correction (the
    converged potentials do not depend on the start, only the number of
    iterations does)."""
    samples = []
    model = WarmStartModel(seed=seed)            # only for its feature kernel
    for k in range(n_pairs):
        g = (pair_fn or training_pair)(k, seed)
        G1, G2 = api.Graph(g.n1, g.edges1), api.Graph(g.n2, g.edges2)
        al = api.Aligner(G1, G2, api.Params(dtype=dtype))
        ws = WarmStarter(al, "prev")
        al.node_cost(g.X1, g.X2, g.anchors)
        al.plan_init()
        for t in range(outer):
            al.align_iter()
            warm = ws.before_solve()
            F = model.features(G2, ws.log_v1, ws.corr, ws.pot if ws.t > 0 else None,
                               ws._mask(), ws.t)
            c_prev = ws.corr.clone()
            al.sinkhorn(max_sweeps, tol, 10, warm)
            ws.after_solve()
            samples.append(Sample(G2, F.clone(), ws.corr - c_prev))
        al.close()
        if log and (k + 1) % 25 == 0:
            log(f"generated {len(samples)} solves from {k + 1} pairs")
    model.close()
    return samples


def train(samples, epochs: int = 20, lr: float = 3e-3, seed: int = 0, log=None):
    model = WarmStartModel(seed=seed)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        losses = []
        for i in order:
            s = samples[i]
            losses.append(model.train_step(s.graph, s.F, s.y, lr).clone())
        ep_loss = float(torch.stack(losses).mean().item())
        hist.append(ep_loss)
        if log:
            log(f"epoch {ep}: mean loss {ep_loss:.4e}")
    return model, hist
