#!/usr/bin/env python
"""Throughput of the many-body MD step on one GB300 (atom-steps/s).

Default workload: fcc Cu, 100 x 100 x 100 conventional cells = 4,000,000
atoms, a = 3.615 A, RGL (Cleri-Rosato) Cu with a quintic taper 4.5-5.0 A,
skin 0.3 A, 300 K Maxwell velocities (seed 1), dt = 1 fs, float64. One bench
step is one velocity-Verlet MD step of the whole box through the C ABI
(kick-drift, device-decided list rebuild, density pass, force pass,
second half-kick); inputs are resident in HBM when the timed region starts.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica of the box on its own
GPU (the single-box path does not shard); value = all ranks' atom-steps over
the slowest rank's time. --impl reference times the CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import pathlib
import subprocess
import sys
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1212_6332_gb300 import inputs as I  # noqa: E402

METRIC = "atom-steps/s on 1 GB300: 4M-atom box, 4096-box batch; FP64 vs mixed; grad/s"
UNIT = "atom-steps/s"
N_CELLS = 100            # fcc repeats per axis of the bench box
SEED = 1
TEMP = 300.0
SKIN = 0.3
DT = 1.0
ORACLE_CELLS = 50        # CPU sample: 500,000 atoms of the same lattice

# Algorithmic float64 work per neighbour-list entry, counting each add, mul
# and compare as 1 flop, an FMA as 2, and exp, sqrt (or rsqrt) and a
# division as 15, 8 and 8 flops (the cost of a table-free float64 evaluation
# by polynomial / Newton steps). K = list length, K_in = entries inside r_cut.
# Pair pass (k_pairs_half), RGL, per pair evaluated (the K/2 upper entries):
# separation 3, r^2 5, rsqrt 8, r 1, two exp arguments 4, two exp 30,
# prefactors 2, A = V'/r and B = rho'/r 6 -> 59 inside r_cut, 8 outside.
# Density sums (k_rho_sum): 2 per entry. Force pass (k_force): separation
# 3, s = A + (F'_i + F'_j) B 3, F_i += s d 6 -> 12 per entry inside r_cut.
KERNELS = {
    # phase: (kernel, flops(K, K_in), bytes(K, K_in)) per atom
    "pairs": ("k_pairs_half (float64 pair functions)",
              lambda K, Ki: Ki / 2 * 59.0 + (K - Ki) / 2 * 8.0,
              # list 4K, reverse index 2K, (A,B) and (rho,V) written to both slots 32K, x 32
              lambda K, Ki: 38.0 * K + 32.0),
    "density": ("k_rho_sum (float64 density sums)", lambda K, Ki: 2.0 * K,
                # count 4, (rho, V) reads 16K, rho/F'/E_i writes 24
                lambda K, Ki: 16.0 * K + 28.0),
    "force": ("k_force (float64 force pass)", lambda K, Ki: 10.0 * Ki,
              # list 4K, (A,B) reads 16K, count 4, x_i 32, F'_i 8, F 24, v 48
              lambda K, Ki: 20.0 * K + 116.0),
}
# GB300 float64 peak from unit counts and clock (no measured float64 peak
# is provided): 152 SMs x 2 float64 FMA per clock x 2 flop x 2.07 GHz
# (an FMA-chain probe measured 1.20 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per atom of one k_pairs_half launch, from an ncu
# capture of 1,048,576 atoms of the same lattice, potential and temperature
# (0.454 GB read + 1.772 GB written); traffic grows in proportion to the
# atom count.
PAIRS_DRAM_BYTES_PER_ATOM = (0.453648e9 + 1.771678e9) / 1048576

REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to MD_CLOCKS_DIR (default: the system's temporary
        # directory); the JSON line carries their summary
        import tempfile
        base = pathlib.Path(os.environ.get("MD_CLOCKS_DIR", tempfile.gettempdir()))
        self.path = base / f"clocks_bench_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.path.parent.mkdir(parents=True, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        try:
            for line in self.path.read_text().splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 4:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                    bits = int(parts[3], 16)
                except ValueError:
                    continue
                for b, name in REASONS.items():
                    if bits & b and name != "gpu_idle":
                        reasons.add(name)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_ranks(local_ms: float, atoms_per_rank: int, steps: int, dist=None, device="cuda") -> tuple[float, float]:
    """Whole-job rate of independent replicas: every rank advances its own
    box; the job's time is the slowest rank's. Returns (atom-steps/s over
    all ranks, slowest rank's ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms = float(t.item())
    return world * atoms_per_rank * steps / (ms * 1e-3), ms


def list_stats(sysm, x_dev, box, rc, sample: int = 65536):
    """Mean list length K and mean entries inside r_cut over a sample of atoms."""
    import torch
    nn, nl = sysm.neighbors()
    n = nn.shape[0]
    idx = torch.linspace(0, n - 1, min(sample, n), device="cuda").long()
    nns = nn[idx].long()
    cols = nl[idx].long()
    valid = torch.arange(cols.shape[1], device="cuda")[None, :] < nns[:, None]
    cols = torch.where(valid, cols, torch.zeros_like(cols))
    d = x_dev[cols] - x_dev[idx][:, None, :]
    bt = torch.tensor(box, device="cuda", dtype=torch.float64)
    d = d - bt * torch.round(d / bt)
    r2 = (d * d).sum(-1)
    inside = ((r2 < rc * rc) & valid).sum(1).double().mean().item()
    K = nns.double().mean().item()
    del nn, nl
    return K, inside


def oracle_sample(steps: int, cells: int = ORACLE_CELLS) -> dict:
    """The CPU oracle (single thread) on a bounded sample of the workload: a
    cells^3 fcc box of the same lattice, potential, temperature and seed."""
    import oracle as O
    bx = I.perturbed_fcc(cells, I.A_CU, TEMP, I.MASS_CU, SEED)
    pot = O.Potential(I.RGL_CU)
    t0 = time.perf_counter()
    O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, DT, SKIN, 0)
    t1 = time.perf_counter()
    O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, DT, SKIN, steps)
    t2 = time.perf_counter()
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / steps
    return dict(value=bx.n / per_step, per_step_s=per_step, n=bx.n, setup_s=t1 - t0,
                sample=f"oracle on a {cells}^3-cell fcc Cu box ({bx.n} atoms, same lattice, RGL, {TEMP:.0f} K, "
                       f"seed {SEED}), {steps} velocity-Verlet steps minus its setup run")


def oracle_batch_sample(steps: int = 3, n_sample: int = 16) -> dict:
    """The CPU oracle on the first n_sample boxes of the 4096-box batch
    (same seed), each box on its own: atom-steps/s of the sample."""
    import oracle as O
    bt = I.batch_of_boxes(n_sample, I.A_CU, I.MASS_CU, seed=2024)
    pot = O.Potential(I.RGL_CU)
    t_setup = t_run = 0.0
    for k in range(n_sample):
        lo, hi = int(bt.atom_offsets[k]), int(bt.atom_offsets[k + 1])
        t0 = time.perf_counter()
        O.md_run(pot, bt.x[lo:hi], bt.v[lo:hi], bt.box[k], I.MASS_CU, DT, SKIN, 0)
        t1 = time.perf_counter()
        O.md_run(pot, bt.x[lo:hi], bt.v[lo:hi], bt.box[k], I.MASS_CU, DT, SKIN, steps)
        t2 = time.perf_counter()
        t_setup += t1 - t0
        t_run += t2 - t1
    n = int(bt.atom_offsets[n_sample])
    per_step = max(t_run - t_setup, 1e-9) / steps
    return dict(value=n / per_step, unit=UNIT, cores=1,
                sample=f"oracle on the first {n_sample} boxes of the batch ({n} atoms), {steps} steps each")


def oracle_grad_sample(n_cfg: int = 8) -> dict:
    """The CPU oracle's parameter gradient (forward mode, RGL, 5 parameters)
    on n_cfg configurations of the 256-configuration fitting set, scaled to
    (gradient over 256 configurations)/s."""
    import oracle as O
    cfgs = [I.strained_fcc(6, I.A_CU, seed=5000 + k) for k in range(n_cfg)]
    pot = O.Potential(I.RGL_CU)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    for c in cfgs:
        O.param_grad(pot, c.x, c.box, rng.normal(size=(c.n, 3)), 1.0)
    dt = time.perf_counter() - t0
    return dict(value=n_cfg / dt / 256.0, unit="(gradient over 256 configs)/s", cores=1,
                sample=f"oracle forward-mode gradient on {n_cfg} of the 256 configurations, scaled to 256")


def workload_name(cells: int, precision: str) -> str:
    """The timed single-box workload, named by what it is."""
    return (f"fcc Cu {cells}^3 cells ({4 * cells ** 3} atoms), RGL Cu taper 4.5-5.0 A, skin {SKIN} A, "
            f"{TEMP:.0f} K, dt {DT} fs, " + ("float64" if precision == "fp64" else "mixed precision"))


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    W, K = args.warmup, args.steps
    cells = ORACLE_CELLS
    bx = I.perturbed_fcc(cells, I.A_CU, TEMP, I.MASS_CU, SEED)
    pot = O.Potential(I.RGL_CU)
    st = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, DT, SKIN, max(W, 0))
    t0 = time.perf_counter()
    O.md_run(pot, st["x"], st["v"], bx.box, I.MASS_CU, DT, SKIN, 0)
    t1 = time.perf_counter()
    O.md_run(pot, st["x"], st["v"], bx.box, I.MASS_CU, DT, SKIN, K)
    t2 = time.perf_counter()
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / max(K, 1)
    value = bx.n / per_step
    sample = (f"oracle on a {cells}^3-cell fcc Cu box ({bx.n} atoms, same lattice, RGL, {TEMP:.0f} K, seed {SEED}); "
              f"per-step time = ({K} steps run - setup run) / {K}")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": per_step * 1e3 * (4 * args.cells ** 3 / bx.n), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(args.cells, "fp64"), "atoms": 4 * args.cells ** 3,
                      "sample_atoms": bx.n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_variant(precision: str, W: int, K: int, x_h, v_h, box, spec=None, mass=None, thermostat=None,
                barostat=None, types=None, newton3=False) -> dict:
    """atom-steps/s of a box in another precision or potential (same timing
    rules), with its per-phase times; optionally with the friction of
    Eq. (4) (thermostat = (T_e, tau_T)), the pressure coupling of Eq. (5)
    (barostat = (P0, tau_p, beta)) or the half-list sums with Newton's
    third law."""
    import torch
    from paper_1212_6332_gb300.md import System
    spec = spec or I.RGL_CU
    s = System(spec, box=box, n_atoms=len(x_h), skin=SKIN, dt=DT, mass=mass or I.MASS_CU, precision=precision)
    if types is not None:
        s.set_types(types)
    if newton3:
        s.set_newton3(True)
    if thermostat:
        s.set_thermostat(*thermostat)
    if barostat:
        s.set_barostat(*barostat)
    s.set_state(torch.tensor(x_h, device="cuda"), torch.tensor(v_h, device="cuda"))
    s.step(W)
    torch.cuda.synchronize()
    s.profile_start(timing=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    th = s.step(K)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    prof = s.profile_read()
    s.close()
    return dict(value=len(x_h) * K / (ms * 1e-3), ms_per_step=ms / K, n_rebuild=th["n_rebuild"],
                phase_ms_per_step={k: v / max(K, 1) for k, v in prof["ms"].items()})


def run_small(K: int, use_graph: bool) -> dict:
    """The 2048-atom Cu box (8^3 cells, RGL Cu, 300 K, seed 12345), K
    velocity-Verlet steps in one call: launch-bound, the working set sits in
    L2 (a latency figure, not an HBM one)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(8, I.A_CU, 300.0, I.MASS_CU, 12345)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=SKIN, dt=DT, mass=I.MASS_CU)
    s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    s.step(K, use_graph=use_graph)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    th = s.step(K, use_graph=use_graph)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    s.close()
    return dict(value=bx.n * K / (ms * 1e-3), ms_per_step=ms / K, steps=K, n_rebuild=th["n_rebuild"],
                graph=use_graph, l2="working set inside L2")


def run_batch(precision: str, K: int, W: int, n_boxes: int = 4096, use_graph: bool = True,
              schedule: str = "tile") -> dict:
    """The 4096-box batch (n ~ U{3..10} fcc Cu repeats, T ~ U(300, 1500) K,
    RGL Cu): all boxes advance together, one launch per phase (graph-replayed)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(n_boxes, I.A_CU, I.MASS_CU, seed=2024)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=SKIN, dt=DT, mass=I.MASS_CU,
               precision=precision)
    s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
    s.batch_step(W, schedule=schedule, use_graph=use_graph, per_box=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    s.batch_step(K, schedule=schedule, use_graph=use_graph, per_box=False)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    n = int(bt.atom_offsets[-1])
    phases = None
    if schedule == "tile":
        # phase split from a further, untimed stretch of the same run (phase
        # events turn graph replay off, so they stay out of the timed steps)
        s.profile_start(timing=True)
        s.batch_step(K, schedule=schedule, use_graph=False, per_box=False)
        prof = s.profile_read()
        phases = {k: v / max(K, 1) for k, v in prof["ms"].items()}
    s.close()
    return dict(value=n * K / (ms * 1e-3), ms_per_step=ms / K, atoms=n, boxes=n_boxes, schedule=schedule,
                graph=use_graph and schedule == "tile", phase_ms_per_step=phases)


def run_per_box_sample(K: int, n_sample: int = 64, n_boxes: int = 4096) -> dict:
    """One launch sequence per box: the first n_sample boxes of the same
    batch, each in its own single-box context stepped on its own,
    extrapolated to all boxes by atom count."""
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(n_boxes, I.A_CU, I.MASS_CU, seed=2024)
    systems = []
    for k in range(n_sample):
        lo, hi = int(bt.atom_offsets[k]), int(bt.atom_offsets[k + 1])
        s = System(I.RGL_CU, box=bt.box[k], n_atoms=hi - lo, skin=SKIN, dt=DT, mass=I.MASS_CU)
        s.set_state(torch.tensor(bt.x[lo:hi], device="cuda"), torch.tensor(bt.v[lo:hi], device="cuda"))
        s.step(2)
        systems.append(s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in systems:
        s.step(K)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_s = int(bt.atom_offsets[n_sample])
    for s in systems:
        s.close()
    return dict(value=n_s * K / dt, sample_boxes=n_sample, sample_atoms=n_s,
                note="each box its own context and launch sequence; rate extrapolates to any box count")


def run_grad(K: int, W: int, precision: str = "fp64", kind: str = "rgl") -> dict:
    """Force-matching loss + gradient over 256 configurations of 864 atoms
    (6^3 fcc Cu, strain U(0.98, 1.02), N(0, 0.1 A) displacements); targets
    from RGL Cu at the reference parameters, model RGL perturbed by 5%
    (or its 3 x 200-knot spline tabulation, or the two-species alloy_model
    with U{0, 1} labels: 3 V + 3 rho + 2 F tables of 200 knots)."""
    import torch
    from paper_1212_6332_gb300.fit import ForceField, force_matching_loss, make_batch, theta_of
    cfgs = [I.strained_fcc(6, I.A_CU, seed=5000 + k) for k in range(256)]
    n = sum(c.n for c in cfgs)
    ref = make_batch(I.RGL_CU, cfgs)
    f_tgt = ref.get_forces()["f"].clone()
    e_tgt = ref.batch_thermo()[:, 1].clone()
    ref.close()
    signs = np.where(I.uniform(77, 5) < 0.5, -1.0, 1.0)
    model = dict(I.RGL_CU, **{k: I.RGL_CU[k] * (1 + 0.05 * sg) for k, sg in zip(("A", "xi", "p", "q", "r0"), signs)})
    types = None
    if kind == "spline":
        model = spline_model(model)
    elif kind == "alloy":
        # two species, labels U{0, 1} per atom
        model = alloy_model()
        types = (I.uniform(78, n) < 0.5).astype(np.int32)
    s = make_batch(model, cfgs, precision=precision, types=types)
    counts = torch.tensor([c.n for c in cfgs], device="cuda", dtype=torch.float64)
    theta = theta_of(model).cuda().requires_grad_(True)

    def once():
        f, e = ForceField.apply(theta, s, model)
        L = force_matching_loss(f, e, f_tgt, e_tgt, counts)
        (g,) = torch.autograd.grad(L, theta)
        return L, g

    for _ in range(W):
        once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        L, g = once()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return dict(value=K / dt, unit="(loss + gradient over 256 configs)/s", atom_grads_per_s=n * K / dt,
                n_params=int(theta.numel()), loss=float(L.item()), precision=precision, model=kind)


def spline_model(spec: dict) -> dict:
    """Spline model tabulated from an RGL potential by the library itself
    (md_eval of V, rho on 200 knots over [1.5, 5.0] A and F on 200 knots over
    [0, 2 rho_eq])."""
    import torch
    from paper_1212_6332_gb300.md import System
    x, box = I.fcc_lattice(6, I.A_CU)
    s = System(spec, box=box, n_atoms=len(x), skin=0.0, mass=I.MASS_CU)
    rho_eq = float(s.compute_forces(torch.tensor(x, device="cuda"))["rho"].mean().item())
    s.close()
    r = np.linspace(1.5, 5.0, 200)
    pair = np.zeros((2, 200))
    # V(r) and rho(r) from a two-atom box at each knot (the library's own evaluation)
    d = System(spec, box=[20.0, 20.0, 20.0], n_atoms=2, skin=0.0, mass=I.MASS_CU)
    for k, rk in enumerate(r):
        xx = np.array([[1.0, 1.0, 1.0], [1.0 + rk, 1.0, 1.0]])
        o = d.compute_forces(torch.tensor(xx, device="cuda"))
        pair[1, k] = o["rho"][0].item()
        pair[0, k] = o["e_atom"].sum().item() - 2 * (-spec_f_scale(spec) * np.sqrt(pair[1, k]))
    d.close()
    rg = np.linspace(0.0, 2 * rho_eq, 200)
    F = -spec_f_scale(spec) * np.sqrt(rg)
    return dict(kind="spline", phi=pair[0], f=pair[1], F=F, r_lo=1.5, r_hi=5.0, rho_lo=0.0, rho_hi=2 * rho_eq)


def alloy_model() -> dict:
    """Two-species spline model tabulated by the library itself (as
    spline_model): RGL Cu for the (0, 0) pair, RGL Ni with the Cu taper for
    (1, 1), the parameter means for (0, 1); V and rho on 200 knots over
    [1.5, 5.0] A, F = -sqrt(rho) for both species on 200 knots over [0, 45]."""
    import torch
    from paper_1212_6332_gb300.md import System
    cuni = dict(kind="rgl", A=0.5 * (0.0855 + 0.0376), xi=float(np.sqrt(1.224 * 1.070)), p=0.5 * (10.960 + 16.999),
                q=0.5 * (2.278 + 1.189), r0=0.5 * (2.5562 + 2.4911), r_taper=4.5, r_cut=5.0)
    r = np.linspace(1.5, 5.0, 200)
    phi, f = [], []
    for spec in (I.RGL_CU, cuni, dict(I.RGL_NI, r_taper=4.5, r_cut=5.0)):
        d = System(spec, box=[20.0, 20.0, 20.0], n_atoms=2, skin=0.0, mass=I.MASS_CU)
        v, rho = np.zeros(200), np.zeros(200)
        for k, rk in enumerate(r):
            xx = np.array([[1.0, 1.0, 1.0], [1.0 + rk, 1.0, 1.0]])
            o = d.compute_forces(torch.tensor(xx, device="cuda"))
            rho[k] = o["rho"][0].item()
            v[k] = o["e_atom"].sum().item() + 2.0 * np.sqrt(rho[k])
        d.close()
        phi.append(v)
        f.append(rho)
    F = -np.sqrt(np.linspace(0.0, 45.0, 200))
    return dict(kind="alloy", n_types=2, phi=phi, f=f, F=[F, F], r_lo=1.5, r_hi=5.0, rho_lo=0.0, rho_hi=45.0)


def spec_f_scale(spec: dict) -> float:
    return spec["c"] * spec["eps"] if spec["kind"] == "sc" else 1.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=N_CELLS)
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-precision, batch, gradient and oracle legs")
    ap.add_argument("--e2e-steps", type=int, default=10, help="host-buffer end-to-end steps (0 skips the leg)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the headline box (default float64)")
    ap.add_argument("--batch-boxes", type=int, default=0,
                    help="only the tile-schedule batch leg with this many boxes (profiling runs; prints its dict)")
    ap.add_argument("--alloy-only", action="store_true",
                    help="only the two-species spline alloy box of --cells (profiling runs; prints its dict)")
    ap.add_argument("--grad-only", default="", choices=["", "rgl", "spline", "alloy"],
                    help="only the fitting-gradient leg of this model, K iterations (profiling runs; prints its dict)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    W = max(args.warmup, 3)
    K = args.steps
    world, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1212_6332_gb300 import build
    build.build()
    if args.batch_boxes:
        print(json.dumps(run_batch(args.precision, K, W, n_boxes=args.batch_boxes)))
        return
    if args.grad_only:
        print(json.dumps(run_grad(K, W, args.precision, args.grad_only)))
        return
    if args.alloy_only:
        al = I.perturbed_fcc(args.cells, 3.57, TEMP, I.MASS_CU, 5)
        al_types = np.random.default_rng(5).integers(0, 2, al.n).astype(np.int32)
        print(json.dumps(run_variant(args.precision, W, K, al.x, al.v, al.box, spec=alloy_model(), types=al_types)))
        return
    from paper_1212_6332_gb300.md import System

    bx = I.perturbed_fcc(args.cells, I.A_CU, TEMP, I.MASS_CU, SEED)
    N = bx.n
    x_dev = torch.tensor(bx.x, device="cuda")
    v_dev = torch.tensor(bx.v, device="cuda")
    s = System(I.RGL_CU, box=bx.box, n_atoms=N, skin=SKIN, dt=DT, mass=I.MASS_CU, precision=args.precision)
    s.set_state(x_dev, v_dev)
    K_list, K_in = list_stats(s, x_dev, bx.box, I.RGL_CU["r_cut"])
    s.step(W)

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.profile_start(timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        th = s.step(K)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    prof = s.profile_read()
    ms = ev0.elapsed_time(ev1)
    value, ms_max = combine_ranks(ms, N, K, dist)

    # dominant kernel (event-timed on the launching stream)
    dom = max(KERNELS, key=lambda k: prof["ms"][k])
    k_ms = prof["ms"][dom] / max(prof["timed"][dom], 1)
    kname, ffl, fby = KERNELS[dom]
    flops = N * ffl(K_list, K_in)
    achieved = flops / (k_ms * 1e-3) / 1e12
    bytes_k = N * fby(K_list, K_in)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SM x 2 float64 FMA/clock x 2 flop x 2.07 GHz",
                "traffic": (PAIRS_DRAM_BYTES_PER_ATOM * N if dom == "pairs" and args.precision == "fp64" else None),
                "traffic_source": "ncu capture of 1,048,576 atoms scaled by the atom count",
                "flops_per_launch": flops, "launch_ms": k_ms,
                "hbm": {"achieved": bytes_k / (k_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": bytes_k / (k_ms * 1e-3) / 1e9 / hbm,
                        "peak_source": "measured" if "fallback" not in peaks else "fallback",
                        "bytes_per_launch": bytes_k}}
    phase_ms = {k: prof["ms"][k] / max(K, 1) for k in prof["ms"]}

    # end to end through the C ABI with pinned host buffers: every step
    # uploads the state, advances one step and downloads the state
    xh = torch.empty((N, 3), dtype=torch.float64, pin_memory=True)
    vh = torch.empty((N, 3), dtype=torch.float64, pin_memory=True)
    s.get_state(xh, vh)
    K_e2e = min(args.e2e_steps, max(K, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K_e2e):
        s.set_state(xh, vh)
        s.step(1)
        s.get_state(xh, vh)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_value = combine_ranks(t_e2e * 1e3, N, K_e2e, dist)[0] if K_e2e > 0 else None
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": 2 * N * 3 * 8,
           "d2h_bytes_per_step": 2 * N * 3 * 8 + 56,
           "call": "md_set_state(host) + md_step(1) + md_get_state(host) per step", "steps": K_e2e}

    variants = {}
    cpu = None
    batch = grad = None
    if rank == 0 and not args.no_extras:
        s.close()
        del s
        variants["mixed"] = run_variant("mixed", W, K, bx.x, bx.v, bx.box)
        variants["fp64"] = {"value": value, "ms_per_step": ms_max / K}
        hot = I.perturbed_fcc(args.cells, I.A_CU, 1200.0, I.MASS_CU, 2)
        variants["fp64_1200K"] = run_variant("fp64", W, K, hot.x, hot.v, hot.box)
        variants["mixed_1200K"] = run_variant("mixed", W, K, hot.x, hot.v, hot.box)
        variants["sc_fp64"] = run_variant("fp64", W, max(5, K // 3), bx.x, bx.v, bx.box, spec=I.SC_CU)
        variants["sc_mixed"] = run_variant("mixed", W, K, bx.x, bx.v, bx.box, spec=I.SC_CU)
        del hot
        ni = I.perturbed_fcc(80, I.A_NI, 600.0, I.MASS_NI, 3)
        variants["ni_2m_fp64"] = run_variant("fp64", W, K, ni.x, ni.v, ni.box, spec=I.RGL_NI, mass=I.MASS_NI)
        variants["ni_2m_mixed"] = run_variant("mixed", W, K, ni.x, ni.v, ni.box, spec=I.RGL_NI, mass=I.MASS_NI)
        del ni
        # full-list sums against Newton's third law, both with phase events
        variants["fp64_phases"] = run_variant("fp64", W, K, bx.x, bx.v, bx.box)
        variants["fp64_newton3"] = run_variant("fp64", W, K, bx.x, bx.v, bx.box, newton3=True)
        variants["fp64_thermostat"] = run_variant("fp64", W, K, bx.x, bx.v, bx.box, thermostat=(300.0, 100.0))
        variants["fp64_barostat"] = run_variant("fp64", W, K, bx.x, bx.v, bx.box,
                                                barostat=(0.0, 1000.0, 160.21766208 / 140.0))
        al = I.perturbed_fcc(args.cells, 3.57, TEMP, I.MASS_CU, 5)
        al_types = np.random.default_rng(5).integers(0, 2, al.n).astype(np.int32)
        al_spec = alloy_model()
        variants["alloy_cuni_fp64"] = run_variant("fp64", W, K, al.x, al.v, al.box, spec=al_spec, types=al_types)
        variants["alloy_cuni_mixed"] = run_variant("mixed", W, K, al.x, al.v, al.box, spec=al_spec, types=al_types)
        del al
        variants["cu_2048_graph"] = run_small(200, True)
        variants["cu_2048_nograph"] = run_small(200, False)
        del x_dev, v_dev
        torch.cuda.empty_cache()
        kb = max(5, min(K, 20))
        batch = {"fp64": run_batch("fp64", kb, W), "fp64_box": run_batch("fp64", kb, W, schedule="box"),
                 "mixed": run_batch("mixed", kb, W),
                 "one_launch_per_box": run_per_box_sample(kb)}
        kg = max(3, min(K, 10))
        grad = {"rgl_fp64": run_grad(kg, 2, "fp64", "rgl"), "rgl_mixed": run_grad(kg, 2, "mixed", "rgl"),
                "spline_fp64": run_grad(kg, 2, "fp64", "spline"),
                "spline_mixed": run_grad(kg, 2, "mixed", "spline"),
                "alloy_fp64": run_grad(kg, 2, "fp64", "alloy"), "alloy_mixed": run_grad(kg, 2, "mixed", "alloy")}
    if rank == 0 and not args.no_extras:
        import oracle as O
        O.build()
        smp = oracle_sample(3)
        cpu = {"value": smp["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": smp["sample"],
               "batch_sample": oracle_batch_sample(), "grad_sample": oracle_grad_sample()}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
               "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
               "config": {"workload": workload_name(args.cells, args.precision),
                          "atoms": N, "parallelism": "replicas" if world > 1 else "single",
                          "l2": "working set (list + positions) larger than L2",
                          "mean_list_len": K_list, "mean_in_cutoff": K_in,
                          "n_rebuild": th["n_rebuild"], "phase_ms_per_step": phase_ms},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": prof["launches"],
               "clocks": clk.summary(), "variants": variants, "batch": batch, "grad": grad}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
