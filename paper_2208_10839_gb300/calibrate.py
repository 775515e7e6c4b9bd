"""Array self-calibration by gradient descent through the energyscape.

A recording of a known scene, made by an array whose microphone positions,
gains and delays are off their nominal values, is beamformed with the
current estimate; the estimate moves to make that energyscape match the one
the known scene should give (L = sum (E - E_ref)^2).  Each step is three
native calls on the plan's stream (rtis_process, rtis_loss_l2,
rtis_backward) and an Adam update of the 5 M parameters.  The parameters
are optimised in scaled units (positions / pos_scale, (gain - 1) /
gain_scale, delay / delay_scale) so one learning rate suits all three.
State (estimate, optimiser moments, step count) saves to and loads from
.npz.
"""
from __future__ import annotations

import numpy as np

from . import _native as nat


class Calibrator:
    def __init__(self, plan, mic_xyz, *, lr=0.05, pos_scale=1e-3, gain_scale=0.1, delay_scale=1e-6,
                 betas=(0.9, 0.999), eps=1e-12, fit=("xyz", "gain", "delay")):
        import torch
        self._torch = torch
        self.plan = plan
        self.dev = torch.device("cuda", torch.cuda.current_device())
        M = plan.M
        self.p0 = torch.as_tensor(np.asarray(mic_xyz, dtype=np.float32), device=self.dev).reshape(M, 3)
        self.scale = {"xyz": pos_scale, "gain": gain_scale, "delay": delay_scale}
        self.z = {"xyz": torch.zeros((M, 3), dtype=torch.float32, device=self.dev),
                  "gain": torch.zeros(M, dtype=torch.float32, device=self.dev),
                  "delay": torch.zeros(M, dtype=torch.float32, device=self.dev)}
        self.m1 = {k: torch.zeros_like(v) for k, v in self.z.items()}
        self.m2 = {k: torch.zeros_like(v) for k, v in self.z.items()}
        self.lr, self.betas, self.eps = float(lr), betas, float(eps)
        self.fit = tuple(fit)
        self.t = 0
        self._E = torch.empty((plan.D, plan.n_out), dtype=torch.float32, device=self.dev)
        self._G = torch.empty_like(self._E)
        self._loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        self._gx = torch.empty((M, 3), dtype=torch.float32, device=self.dev)
        self._gg = torch.empty(M, dtype=torch.float32, device=self.dev)
        self._gd = torch.empty(M, dtype=torch.float32, device=self.dev)

    # -- current estimate ---------------------------------------------------
    def params(self):
        return (self.p0 + self.scale["xyz"] * self.z["xyz"], 1.0 + self.scale["gain"] * self.z["gain"],
                self.scale["delay"] * self.z["delay"])

    def loss_and_grad(self, x, E_ref):
        """L and dL/d(xyz, gain, delay) at the current estimate (device tensors)."""
        p, g, d = self.params()
        self.plan.set_calibration(p, g, d)
        self.plan.process(x, self._E)
        h = self.plan.handle
        nat.rtis_loss_l2(h, self._E, E_ref, self._G, self._loss)
        nat.rtis_backward(h, x, self._G, self._gx, self._gg, self._gd)
        return self._loss, (self._gx, self._gg, self._gd)

    def step(self, x, E_ref):
        """One descent step; returns the loss before it (a device scalar)."""
        loss, (gx, gg, gd) = self.loss_and_grad(x, E_ref)
        self.t += 1
        b1, b2 = self.betas
        grads = {"xyz": gx * self.scale["xyz"], "gain": gg * self.scale["gain"], "delay": gd * self.scale["delay"]}
        for k in self.fit:
            self.m1[k].mul_(b1).add_(grads[k], alpha=1 - b1)
            self.m2[k].mul_(b2).addcmul_(grads[k], grads[k], value=1 - b2)
            mh = self.m1[k] / (1 - b1 ** self.t)
            vh = self.m2[k] / (1 - b2 ** self.t)
            self.z[k].sub_(self.lr * mh / (vh.sqrt() + self.eps))
        return loss.clone()

    # -- checkpoint -----------------------------------------------------------
    def state_dict(self):
        out = {"t": np.int64(self.t), "lr": np.float64(self.lr), "p0": self.p0.cpu().numpy()}
        for k in self.z:
            out[f"z_{k}"] = self.z[k].cpu().numpy()
            out[f"m1_{k}"] = self.m1[k].cpu().numpy()
            out[f"m2_{k}"] = self.m2[k].cpu().numpy()
            out[f"scale_{k}"] = np.float64(self.scale[k])
        return out

    def load_state_dict(self, st):
        torch = self._torch
        self.t = int(st["t"])
        self.lr = float(st["lr"])
        self.p0 = torch.as_tensor(np.asarray(st["p0"]), device=self.dev)
        for k in self.z:
            self.z[k] = torch.as_tensor(np.asarray(st[f"z_{k}"]), device=self.dev)
            self.m1[k] = torch.as_tensor(np.asarray(st[f"m1_{k}"]), device=self.dev)
            self.m2[k] = torch.as_tensor(np.asarray(st[f"m2_{k}"]), device=self.dev)
            self.scale[k] = float(st[f"scale_{k}"])

    def save(self, path):
        np.savez(path, **self.state_dict())

    def load(self, path):
        with np.load(path) as f:
            self.load_state_dict({k: f[k] for k in f.files})
