"""Potential fitting: a torch.autograd.Function over the library's force
evaluation and its parameter adjoint (md_param_grad).

forward(theta) sets the potential parameters of a batch of fixed
configurations (md_batch_set_potential re-evaluates forces at the stored
positions and neighbour lists) and returns forces [N, 3] and per-box
energies [B]; backward(dL/dF, dL/dE) returns dL/dtheta from the adjoint
kernels. theta is a float64 tensor: (A, xi, p, q, r0) for RGL, the
concatenated V, rho and F knot values for a spline model, or for several
species all V pair tables, then all rho pair tables, then the F tables.
"""
from __future__ import annotations

import numpy as np
import torch

from .md import System

RGL_KEYS = ("A", "xi", "p", "q", "r0")


def theta_of(spec: dict) -> torch.Tensor:
    if spec["kind"] == "rgl":
        return torch.tensor([spec[k] for k in RGL_KEYS], dtype=torch.float64)
    if spec["kind"] == "spline":
        return torch.tensor(np.concatenate([spec["phi"], spec["f"], spec["F"]]), dtype=torch.float64)
    if spec["kind"] == "alloy":
        tabs = [np.asarray(t, dtype=np.float64) for key in ("phi", "f", "F") for t in spec[key]]
        return torch.tensor(np.concatenate(tabs), dtype=torch.float64)
    raise ValueError("fitting supports RGL, spline and alloy potentials")


def spec_of(theta: torch.Tensor, template: dict) -> dict:
    vals = theta.detach().cpu().numpy().astype(np.float64)
    spec = dict(template)
    if template["kind"] == "rgl":
        spec.update({k: float(v) for k, v in zip(RGL_KEYS, vals)})
    elif template["kind"] == "alloy":
        off = 0
        for key in ("phi", "f", "F"):
            tabs = []
            for t in template[key]:
                tabs.append(vals[off:off + len(t)].copy())
                off += len(t)
            spec[key] = tabs
    else:
        a, b = len(template["phi"]), len(template["f"])
        spec["phi"], spec["f"], spec["F"] = vals[:a].copy(), vals[a:a + b].copy(), vals[a + b:].copy()
    return spec


class ForceField(torch.autograd.Function):
    """(forces [N, 3], per-box energies [B]) as a differentiable function of
    the potential parameters, at the fixed positions held by `system`."""

    @staticmethod
    def forward(ctx, theta, system: System, template: dict):
        system.set_potential(spec_of(theta, template))
        f = system.get_forces(e_atom=False, rho=False)["f"]
        e_box = system.batch_thermo()[:, 1].contiguous()
        ctx.system = system
        ctx.dev = theta.device
        return f, e_box

    @staticmethod
    def backward(ctx, g_f, g_e):
        sysm = ctx.system
        g_f = torch.zeros(sysm.n, 3, dtype=torch.float64, device="cuda") if g_f is None else g_f.contiguous()
        g_e = torch.zeros(sysm.n_boxes, dtype=torch.float64, device="cuda") if g_e is None else g_e.contiguous()
        grad = sysm.param_grad(g_f, g_e)
        return grad.to(ctx.dev), None, None


def config_index(counts: torch.Tensor) -> torch.Tensor:
    """Configuration of every atom (configurations back to back). Building
    it waits for the device (the output size depends on the counts), so a
    fitting loop builds it once and passes it to force_matching_loss."""
    return torch.repeat_interleave(torch.arange(counts.shape[0], device=counts.device), counts.long())


def force_matching_loss(f, e_box, f_tgt, e_tgt, counts, w_e: float = 0.1, idx=None):
    """Mean over configurations of mean squared force error plus w_e times
    the squared per-atom energy error. idx: config_index(counts), built
    here when not given."""
    n_cfg = counts.shape[0]
    if idx is None:
        idx = config_index(counts)
    sq = ((f - f_tgt) ** 2).sum(dim=1)
    per_cfg = torch.zeros(n_cfg, dtype=f.dtype, device=f.device).index_add_(0, idx, sq) / (3.0 * counts)
    de = (e_box - e_tgt) / counts
    return (per_cfg + w_e * de * de).mean()


def make_batch(spec: dict, configs, skin: float = 0.0, precision: str = "fp64", mass: float = 63.546,
               types=None, deferred: bool = True) -> System:
    """A batch System holding fixed configurations (inputs.Box objects);
    types (one label per atom, configurations concatenated) for a potential
    with several species. deferred: the forward and adjoint calls of a
    fitting loop return without waiting for the device status word
    (System.set_deferred_status); call System.sync() to check it."""
    offs = np.zeros(len(configs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([c.n for c in configs])
    s = System(spec, boxes=np.stack([c.box for c in configs]), atom_offsets=offs, skin=skin, mass=mass,
               precision=precision)
    if types is not None:
        s.set_types(types)
    x = torch.tensor(np.concatenate([c.x for c in configs]), device="cuda")
    s.set_state(x)
    if deferred:
        s.set_deferred_status(True)
    return s
