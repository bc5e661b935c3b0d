"""Transport-data surrogate workflow.

The local-field fluid model of the paper reads flux transport data versus the
reduced field (Sec. 2.2.4, computed there by Monte Carlo swarms).  This module
builds such tables with the library's batched swarms, fits the 2-128-128-6
network of ``mlp_train`` to them and answers queries with ``mlp_forward``;
where the network is not trusted, running a swarm remains the answer and
the reference its error is measured against.

Inputs: log10(E/N in Td) and the O2 fraction.  Targets: natural logarithms
of mu N (1/(V m s)), D_L N and D_T N (1/(m s)), max(alpha / N, 1e-25 m^2),
max(eta / N, 1e-25 m^2) and the mean energy (eV).  Both are standardized
with the training set's column means and standard deviations.  Everything
here is argument marshalling and table bookkeeping; the network's arithmetic
runs in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import picmcc as P

TD = 1e-21  # V m^2
FLOOR = 1e-25
TARGET_NAMES = ("log_muN", "log_DLN", "log_DTN", "log_alpha_N", "log_eta_N", "log_mean_eps")
# columns of swarm_result used: W_flux, DL_flux, DT_flux, mean_eps, alpha, eta
R_W, R_DL, R_DT, R_EPS, R_ALPHA, R_ETA = 0, 2, 3, 6, 9, 10


def features(EN_Td, f_o2) -> np.ndarray:
    EN_Td = np.asarray(EN_Td, np.float64)
    return np.stack([np.log10(EN_Td), np.broadcast_to(np.asarray(f_o2, np.float64), EN_Td.shape)], axis=-1)


def targets(res: np.ndarray, EN_Td, n_gas: float) -> np.ndarray:
    """The six log targets from swarm_run results [n][24] at E/N values EN_Td."""
    EN = np.asarray(EN_Td, np.float64)
    muN = res[:, R_W] / (EN * TD)
    return np.stack([np.log(muN), np.log(res[:, R_DL] * n_gas), np.log(res[:, R_DT] * n_gas),
                     np.log(np.maximum(res[:, R_ALPHA] / n_gas, FLOOR)),
                     np.log(np.maximum(res[:, R_ETA] / n_gas, FLOOR)), np.log(res[:, R_EPS])], axis=1)


def swarm_points(gas, EN_Td, fractions, n_gas: float, **swarm_kw):
    """Runs the batched swarms of every (O2 fraction, E/N) pair in one batched
    call (each swarm with its own gas composition); returns (features [n][2],
    targets [n][6], raw results [n][24]), fraction-major.  gas: the N2/O2 gas
    with its species tagged."""
    EN = np.asarray(EN_Td, np.float64)
    fr = np.atleast_1d(np.asarray(fractions, np.float64))
    ENs = np.tile(EN, len(fr))
    fs = np.repeat(fr, len(EN))
    res, _, _ = P.swarm_run(gas, ENs, o2_frac=fs, batched=True, **swarm_kw)
    return features(ENs, fs), targets(res, ENs, n_gas), res


class Standardizer:
    def __init__(self, a: np.ndarray):
        self.mean = a.mean(axis=0)
        self.std = np.where(a.std(axis=0) > 0, a.std(axis=0), 1.0)

    def fwd(self, a):
        return (np.asarray(a) - self.mean) / self.std

    def inv(self, a):
        return np.asarray(a) * self.std + self.mean


class Surrogate:
    """Network parameters and Adam state on the device plus the input and
    target standardizers of its training set."""

    def __init__(self, params0: np.ndarray, x: np.ndarray, y: np.ndarray):
        import torch
        self.sx, self.sy = Standardizer(x), Standardizer(y)
        self.params = torch.as_tensor(np.asarray(params0, np.float32)).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._folded, self._folded_step = None, -1
        self.x = torch.as_tensor(self.sx.fwd(x).astype(np.float32)).cuda()
        self.y = torch.as_tensor(self.sy.fwd(y).astype(np.float32)).cuda()

    def fit(self, n_steps: int, lr: float = 1e-3, chunk: int = 1000):
        """Full-batch Adam; returns (loss trace [(step, loss)], seconds)."""
        import torch
        trace = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        while done < n_steps:
            k = min(chunk, n_steps - done)
            loss = P.mlp_train(self.params, self.m, self.v, self.step, self.x, self.y, k, lr=lr)
            self.step += k
            done += k
            trace.append((self.step, float(loss.item())))
        torch.cuda.synchronize()
        return trace, time.perf_counter() - t0

    def predict_std(self, xs_dev):
        """Standardized outputs for standardized device inputs (no host copies)."""
        return P.mlp_forward(self.params, xs_dev)

    def folded(self):
        """Parameters that take raw inputs and give raw log targets
        (mlp_fold_standardization), refolded after every fit."""
        if self._folded is None or self._folded_step != self.step:
            self._folded = P.mlp_fold_standardization(self.params, self.sx.mean, self.sx.std, self.sy.mean,
                                                      self.sy.std)
            self._folded_step = self.step
        return self._folded

    def predict_dev(self, EN_dev, f_dev):
        """Log targets [n][6] on the device for float64 CUDA tensors of E/N (Td)
        and O2 fraction: the feature kernel, then the network with the
        standardizations folded in."""
        return P.mlp_forward(self.folded(), P.mlp_features(EN_dev, f_dev))

    def predict(self, EN_Td, f_o2) -> np.ndarray:
        """Log targets at raw inputs (host arrays in, host array out)."""
        import torch
        EN = torch.as_tensor(np.ascontiguousarray(EN_Td, np.float64)).cuda()
        f = torch.as_tensor(np.ascontiguousarray(np.broadcast_to(np.asarray(f_o2, np.float64), EN.shape))).cuda()
        return self.predict_dev(EN, f).cpu().numpy().astype(np.float64)


def table_interp(EN_grid, f_grid, table: np.ndarray, EN_Td, f_o2) -> np.ndarray:
    """Bilinear interpolation in (log10 E/N, f) of targets tabulated on the
    grid table[len(f_grid)][len(EN_grid)][6] (the method without the network)."""
    lx = np.log10(np.asarray(EN_grid, np.float64))
    fg = np.asarray(f_grid, np.float64)
    qx = np.log10(np.asarray(EN_Td, np.float64))
    qf = np.asarray(f_o2, np.float64)
    i = np.clip(np.searchsorted(lx, qx) - 1, 0, len(lx) - 2)
    j = np.clip(np.searchsorted(fg, qf) - 1, 0, len(fg) - 2)
    a = np.clip((qx - lx[i]) / (lx[i + 1] - lx[i]), 0.0, 1.0)[:, None]
    b = np.clip((qf - fg[j]) / (fg[j + 1] - fg[j]), 0.0, 1.0)[:, None]
    return ((1 - a) * (1 - b) * table[j, i] + a * (1 - b) * table[j, i + 1] + (1 - a) * b * table[j + 1, i] +
            a * b * table[j + 1, i + 1])
