"""Learned gridding kernel: a small MLP over the sub-cell offset, trained through the
imager's own forward and adjoint kernels to minimise the image error against the
direct transform at a fixed support.

The paper grids with a Gaussian of 7 cells (section 2, Eq. 3) and lists better
(tabulated) kernels as future work in its conclusions.  Here:

* ``KernelMLP``: 1 -> 32 -> 32 -> 1 with tanh, input x / (W/2) for x in [-W/2, W/2];
  the kernel is g(x) = f(x) + f(-x), even by construction, so its Fourier transform
  (the grid correction) is real.
* ``tabulate``: samples of g at ``per_cell`` points per cell, the WST_KERNEL_TABLE
  form the CUDA gridder interpolates linearly.
* ``correction_matrix``: Ghat(nu_a) = M @ table, the integral of the piecewise-linear
  table times cos(2 pi nu x) (3-point Gauss-Legendre per table interval, exact to
  rounding for these interval lengths); 1/Ghat is the grid correction, differentiable
  in torch.
* ``Trainer``: per step one synthetic point-source sky; visibilities by Eq. 1
  (``wst_predict_points``), target = direct transform (``wst_dft``) at pixels sampled
  in the central 3/4 of the image; prediction = U(table) (``autograd.kernel_image``:
  ``wst_image`` forward, ``wst_kernel_grad`` backward) times the correction; loss =
  relative squared error; Adam on the MLP parameters.
* ``save_checkpoint`` / ``load_checkpoint``: the training state (MLP parameters, Adam's
  moments, completed steps, losses) written atomically every few steps, so that an
  interrupted training resumes where it stopped and ends as an uninterrupted one does.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np
import torch
from torch import nn

from . import autograd, synth, wst


class KernelMLP(nn.Module):
    def __init__(self, support: int = 8, hidden: int = 32):
        super().__init__()
        self.half = 0.5 * support
        self.net = nn.Sequential(nn.Linear(1, hidden), nn.Tanh(), nn.Linear(hidden, hidden), nn.Tanh(),
                                 nn.Linear(hidden, 1))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        z = (x / self.half).unsqueeze(-1)
        return (self.net(z) + self.net(-z)).squeeze(-1)


def table_nodes(support: int, per_cell: int, device=None) -> torch.Tensor:
    return torch.linspace(-0.5 * support, 0.5 * support, support * per_cell + 1, dtype=torch.float32,
                          device=device)


def tabulate(mlp: KernelMLP, support: int, per_cell: int = 1024, device=None) -> torch.Tensor:
    return mlp(table_nodes(support, per_cell, device))


def gaussian_table(support: int, sigma: float, per_cell: int = 1024, device=None) -> torch.Tensor:
    x = table_nodes(support, per_cell, device)
    return torch.exp(-x * x / (2.0 * sigma * sigma))


def correction_matrix(n: int, support: int, table_len: int) -> np.ndarray:
    """M[a, i]: Ghat(nu_a) = sum_i M[a, i] table[i], nu_a = (a - n/2)/n."""
    xs = np.linspace(-0.5 * support, 0.5 * support, table_len)
    h = xs[1] - xs[0]
    gx, gw = np.polynomial.legendre.leggauss(3)
    s = 0.5 * (gx + 1.0)  # nodes on [0, 1]
    wq = 0.5 * gw
    nu = (np.arange(n) - n // 2) / n
    M = np.zeros((n, table_len))
    for si, wi in zip(s, wq):
        x = xs[:-1] + si * h  # (L-1,)
        c = np.cos(2.0 * math.pi * np.outer(nu, x)) * (h * wi)  # (n, L-1)
        M[:, :-1] += c * (1.0 - si)
        M[:, 1:] += c * si
    return M


def fit_to_table(mlp: KernelMLP, target: torch.Tensor, support: int, per_cell: int, steps: int = 1500,
                 lr: float = 3e-3) -> float:
    """Least-squares fit of the MLP to a given table (initialisation)."""
    x = table_nodes(support, per_cell, target.device)
    opt = torch.optim.Adam(mlp.parameters(), lr=lr)
    loss = torch.tensor(0.0)
    for _ in range(steps):
        opt.zero_grad()
        loss = torch.mean((mlp(x) - target) ** 2)
        loss.backward()
        opt.step()
    return float(loss.item())


@dataclass
class SkyCase:
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    vis: torch.Tensor
    pa: torch.Tensor
    pb: torch.Tensor
    target: torch.Tensor


class Trainer:
    """Trains KernelMLP on synthetic skies (512^2, FoV 0.1 rad, 8 planes, W = 8)."""

    def __init__(self, n: int = 512, fov: float = 0.1, n_w: int = 8, support: int = 8, per_cell: int = 1024,
                 n_vis: int = 200_000, pixels: int = 2048, region: float = 0.375, snap_w: bool = True,
                 device="cuda"):
        self.n, self.fov, self.n_w, self.support, self.per_cell = n, fov, n_w, support, per_cell
        self.n_vis, self.pixels, self.region, self.snap_w = n_vis, pixels, region, snap_w
        self.device = torch.device(device)
        self.L = support * per_cell + 1
        self.w_lo, self.w_hi = -200.0, 200.0
        cfg = wst.Config(n=n, fov=fov, n_w=n_w, w_min=self.w_lo, w_max=self.w_hi, support=support,
                         kernel=wst.WST_KERNEL_TABLE, ktable_len=self.L)
        self.plan = wst.Plan(cfg, device=self.device)
        self.M = torch.from_numpy(correction_matrix(n, support, self.L)).to(self.device)

    # -- data --------------------------------------------------------------------------
    def sky_case(self, index: int) -> SkyCase:
        work = synth.learned_sky(index, n=self.n, fov=self.fov, n_vis=self.n_vis)
        w = work.w.astype(np.float64)
        if self.snap_w:  # put every w on its plane centre: the remaining error is the (u,v) kernel's
            dw = (self.w_hi - self.w_lo) / self.n_w
            k = np.clip(np.floor((w - self.w_lo) * (self.n_w / (self.w_hi - self.w_lo))), 0, self.n_w - 1)
            w = self.w_lo + (k + 0.5) * dw
        dev = self.device
        u = torch.from_numpy(work.u).to(dev)
        v = torch.from_numpy(work.v).to(dev)
        wt = torch.from_numpy(w.astype(np.float32)).to(dev)
        vis = torch.empty(work.n_vis, dtype=torch.complex64, device=dev)
        l = torch.from_numpy(work.sky.l).to(dev)
        m = torch.from_numpy(work.sky.m).to(dev)
        f = torch.from_numpy(work.sky.flux).to(dev)
        wst.wst_predict_points(u, v, wt, l, m, f, vis)
        rng = np.random.default_rng(100_000 + index)
        r = int(self.region * self.n)
        pa = torch.from_numpy(rng.integers(self.n // 2 - r, self.n // 2 + r, self.pixels).astype(np.int32)).to(dev)
        pb = torch.from_numpy(rng.integers(self.n // 2 - r, self.n // 2 + r, self.pixels).astype(np.int32)).to(dev)
        target = torch.empty(self.pixels, dtype=torch.complex64, device=dev)
        wst.wst_dft(u, v, wt, vis, self.n, self.fov, pa, pb, target)
        return SkyCase(u, v, wt, vis, pa, pb, target)

    # -- model -------------------------------------------------------------------------
    def image_at(self, table: torch.Tensor, case: SkyCase) -> torch.Tensor:
        """Corrected image at the case's pixels, differentiable in the table."""
        U = autograd.kernel_image(table, self.plan, case.u, case.v, case.w, case.vis)[0]
        ghat = self.M.to(table.dtype) @ table if table.dtype == torch.float64 else (self.M @ table.double()).float()
        ia, ib = case.pa.long(), case.pb.long()
        corr = 1.0 / (ghat[ia] * ghat[ib])
        return U[ib, ia] * corr

    @staticmethod
    def rel_error(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
        return torch.sum(torch.abs(pred - target) ** 2) / torch.sum(torch.abs(target) ** 2)

    def loss(self, table: torch.Tensor, case: SkyCase) -> torch.Tensor:
        return self.rel_error(self.image_at(table, case), case.target)

    def evaluate(self, table: torch.Tensor, indices) -> float:
        with torch.no_grad():
            errs = [math.sqrt(float(self.loss(table.detach(), self.sky_case(i)))) for i in indices]
        return float(np.mean(errs))

    def train(self, mlp: KernelMLP, indices, lr: float = 1e-3, log_every: int = 0, checkpoint: str | None = None,
              checkpoint_every: int = 0):
        """One Adam step per sky of ``indices``; with ``checkpoint``, resume from it if it
        exists and rewrite it every ``checkpoint_every`` steps."""
        opt = torch.optim.Adam(mlp.parameters(), lr=lr)
        indices = list(indices)
        start, history = 0, []
        if checkpoint and os.path.exists(checkpoint):
            start, history = load_checkpoint(checkpoint, mlp, opt)
        for step in range(start, len(indices)):
            case = self.sky_case(indices[step])
            opt.zero_grad()
            table = tabulate(mlp, self.support, self.per_cell, self.device)
            loss = self.loss(table, case)
            loss.backward()
            opt.step()
            history.append(float(loss.item()))
            if log_every and step % log_every == 0:
                print(f"step {step} loss {history[-1]:.4e}", flush=True)
            if checkpoint and checkpoint_every and (step + 1) % checkpoint_every == 0:
                save_checkpoint(checkpoint, mlp, opt, step + 1, history)
        return history


def save_checkpoint(path: str, mlp: KernelMLP, opt: torch.optim.Optimizer, step: int, history) -> None:
    """Training state after ``step`` completed steps; written to a temporary file and
    renamed, so a crash while saving leaves the previous checkpoint intact."""
    tmp = path + ".tmp"
    torch.save({"mlp": mlp.state_dict(), "opt": opt.state_dict(), "step": int(step),
                "history": [float(h) for h in history]}, tmp)
    os.replace(tmp, path)


def load_checkpoint(path: str, mlp: KernelMLP, opt: torch.optim.Optimizer):
    """Restore parameters and optimiser state in place; returns (completed steps, losses)."""
    state = torch.load(path, map_location="cpu")
    mlp.load_state_dict(state["mlp"])
    opt.load_state_dict(state["opt"])
    return int(state["step"]), list(state["history"])


def train_default(n_skies: int = 10_000, held_out: int = 500, device="cuda", log_every: int = 500,
                  checkpoint: str | None = None, checkpoint_every: int = 500):
    """The full training of the learned W = 8 kernel; returns (mlp, table, report)."""
    torch.manual_seed(20230106)
    mlp = KernelMLP(8).to(device)
    gauss = gaussian_table(8, wst.DEFAULT_SIGMA[8], device=device)
    fit_to_table(mlp, gauss, 8, 1024)
    tr = Trainer(device=device)
    tr.train(mlp, range(n_skies), log_every=log_every, checkpoint=checkpoint, checkpoint_every=checkpoint_every)
    table = tabulate(mlp, 8, 1024, device).detach()
    test_idx = range(1_000_000, 1_000_000 + held_out)
    report = {"gauss_err": tr.evaluate(gauss, test_idx), "learned_err": tr.evaluate(table, test_idx)}
    return mlp, table, report


def save(path: str, mlp: KernelMLP, table: torch.Tensor, report: dict) -> None:
    state = {k: v.detach().cpu().numpy() for k, v in mlp.state_dict().items()}
    np.savez(path, table=table.detach().cpu().numpy().astype(np.float32), support=8, per_cell=1024,
             report_keys=np.array(list(report.keys())), report_vals=np.array(list(report.values()), np.float64),
             **{"mlp." + k: v for k, v in state.items()})


def load_table(path: str) -> np.ndarray:
    with np.load(path) as f:
        return f["table"].astype(np.float32)


def load_mlp(path: str) -> KernelMLP:
    """The trained network saved beside the table (its parameters under "mlp.")."""
    with np.load(path) as f:
        mlp = KernelMLP(int(f["support"]))
        mlp.load_state_dict({k[4:]: torch.from_numpy(f[k]) for k in f.files if k.startswith("mlp.")})
    return mlp


def table_at(path: str, per_cell: int) -> np.ndarray:
    """The trained kernel tabulated at per_cell samples per cell (FP32): the stored table
    when per_cell is its own resolution, else the network sampled afresh."""
    with np.load(path) as f:
        if int(f["per_cell"]) == per_cell:
            return f["table"].astype(np.float32)
        support = int(f["support"])
    with torch.no_grad():
        return tabulate(load_mlp(path), support, per_cell).numpy().astype(np.float32)


def load_report(path: str) -> dict:
    with np.load(path) as f:
        return dict(zip([str(k) for k in f["report_keys"]], [float(v) for v in f["report_vals"]]))


if __name__ == "__main__":
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description="train the learned W = 8 gridding kernel")
    ap.add_argument("--skies", type=int, default=10_000)
    ap.add_argument("--held-out", type=int, default=500)
    ap.add_argument("--out", default="learned_kernel_w8.npz")
    ap.add_argument("--checkpoint", default=None, help="resume from / save the training state to this file")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    a = ap.parse_args()
    t0 = time.time()
    mlp, table, report = train_default(a.skies, a.held_out, checkpoint=a.checkpoint,
                                       checkpoint_every=a.checkpoint_every)
    report.update({"skies": a.skies, "held_out": a.held_out, "train_seconds": time.time() - t0})
    save(a.out, mlp, table, report)
    print(json.dumps(report))
