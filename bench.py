#!/usr/bin/env python
"""Throughput of the many-body MD step on one GB300 (atom-steps/s).

Default workload: fcc Cu, 100 x 100 x 100 conventional cells = 4,000,000
atoms, a = 3.615 A, RGL (Cleri-Rosato) Cu with a quintic taper 4.5-5.0 A,
skin 0.3 A, 300 K Maxwell velocities (seed 1), dt = 1 fs, float64. One bench
step is one velocity-Verlet MD step of the whole box through the C ABI
(kick-drift, device-decided list rebuild, density pass, force pass,
second half-kick); inputs are resident in HBM when the timed region starts.

The timed steps are the ones a user runs: md_step with CUDA-graph replay.
Per-kernel times come from a further, untimed stretch of the same run with
per-phase CUDA events (which turn graph replay off). The roofline
denominators are measured in the same process: float64 and float32 FMA
rates by the library's probe kernel, HBM bandwidth from MEASURED_PEAKS.json.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica of the box on its own
GPU (the single-box path does not shard); value = all ranks' atom-steps over
the slowest rank's time. --impl reference times the CPU oracle on the same
4M-atom box on all host cores (OpenMP).
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

# Algorithmic work per atom of each hot kernel, counting each add, mul and
# compare as 1 flop, an FMA as 2, and exp, sqrt (or rsqrt) and a division
# as 15, 8 and 8 flops in float64 (the cost of a table-free evaluation by
# polynomial / Newton steps) and 4 in float32 (one special-function
# instruction and its scaling). K = list length, Ki = entries inside r_cut;
# positions and F' of partners are counted once per atom (ideal L2 reuse in
# cell order). Counted by hand from the kernel sources.
#
# float64 pair pass (k_pairs_half), per pair evaluated (the K/2 upper entries):
#   RGL: separation 3, r^2 5, rsqrt 8, r 1, two exp arguments 4, two exp 30,
#        prefactors 2, A = V'/r and B = rho'/r 6 -> 59 inside r_cut, 8 outside
#   Sutton-Chen: separation 3, r^2 5, rsqrt 8, r 1, a/r 1, (a/r)^9 and
#        (a/r)^6 by squarings 9, eps 1, A and B 6 -> 34 (+ taper share 1)
#   spline: separation 3, r^2 5, rsqrt 8, r 1, u 1, V, V', rho, rho' 20,
#        A and B 2 -> 40
#   bytes: list 4K, reverse index 2K, the 32-byte cache entry written to
#   both slots 32K, x 32, the fixed-point density totals (4 words) 32
# float64 density finish (k_embed_sums): F, F' and E_i from the fixed-point
#   totals, 6 per atom; totals 32, count 4, rho/F'/E_i writes 24
# float64 force pass (k_force): separation 3, s = A + (F'_i + F'_j) B 3 and
#   F_i += s d 6 -> 12 per entry inside r_cut (the kernel executes s in
#   float64 and the rest as float32 pieces); list 4K, (A, B) 16K, count 4,
#   fixed-point x_i 32, F'_i 8, F 24, v 48
# float32 density pass (k_density_mixed): separation 9, r^2 5, compare 1 per
#   entry; rsqrt 4, r 1, exp argument 2, exp 5, f = xi^2 e S 2, sum 2 per
#   pair inside r_cut (SC: (a/r)^6 6 instead of the exponential); list 4K,
#   offset 16, count 4, rho/F'/F'32/E_i writes 28
# float32 force pass (k_force_mixed): 15 per entry as above; rsqrt 4, r 1,
#   two exponentials 14, V, V', rho, rho' 6, s 4, three products and four
#   sums 7, taper share 3 per pair inside r_cut -> 39; list 4K, offset 16,
#   count 4, F' 4, F 24, E_i 16, v 48
# adjoint (md_param_grad, the fitting leg): per entry inside r_cut, float64
#   with cached pair values: u_i terms 12 and the five RGL parameter terms
#   30 -> 42; float32 from offsets: 15 per entry + 60 per pair; bytes: two
#   passes over list and cache (2 x (4K + 32K)) float64, 2 x 4K float32
SEP64 = 3.0
PAIR64 = {"rgl": 59.0, "sc": 35.0, "spline": 40.0, "alloy": 40.0}


def kernel_model(phase: str, precision: str, kind: str, K: float, Ki: float):
    """(kernel name, flops per atom, bytes per atom, pipe) of a phase's
    dominant kernel, after the counts above."""
    if precision == "fp64":
        if phase == "pairs":
            return ("k_pairs_half (float64 pair functions)",
                    Ki / 2 * PAIR64.get(kind, 40.0) + (K - Ki) / 2 * 8.0, 38.0 * K + 64.0, "fp64")
        if phase == "density":
            return "k_embed_sums (fixed-point density totals, F, F')", 6.0, 60.0, "fp64"
        if phase == "force":
            return "k_force (float64 force pass)", 12.0 * Ki, 20.0 * K + 116.0, "fp64"
        if phase == "grad":
            return "adjoint kernels (float64, cached pair values)", 42.0 * Ki, 72.0 * K + 64.0, "fp64"
    else:
        dens = 16.0 if kind == "rgl" else 17.0
        if phase == "density":
            return "k_density_mixed (float32 pair math)", 15.0 * K + dens * Ki, 4.0 * K + 48.0, "fp32"
        if phase == "force":
            return "k_force_mixed (float32 pair math)", 15.0 * K + 39.0 * Ki, 4.0 * K + 116.0, "fp32"
        if phase == "grad":
            return "adjoint kernels (float32 pair math)", 15.0 * K + 60.0 * Ki, 8.0 * K + 64.0, "fp32"
    return f"{phase} phase", None, None, None


# Derived float64 peak, kept as a note beside the measured one: 152 SMs x 2
# float64 FMA per clock x 2 flop x 2.07 GHz.
FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Algorithmic bytes per atom-step of the whole step: the list (4 B per
# entry) and positions (24 B) read by both force passes.
STEP_BYTES = lambda K: 2 * 4.0 * K + 2 * 24.0  # noqa: E731
# DRAM bytes (read + write) per atom of one k_pairs_half launch, from an ncu
# capture of 1,048,576 atoms of the same lattice, potential and temperature
# (0.464 GB read + 1.792 GB written, a step that forms no pair-energy
# totals; profiles/k_pairs_half_rgl_cu_1m_fp64.md); traffic grows in
# proportion to the atom count.
PAIRS_DRAM_BYTES_PER_ATOM = (0.463907e9 + 1.791848e9) / 1048576
# What the same capture counts per evaluated pair (22.03M pairs): executed
# float64 instructions (DFMA + DMUL + DADD) and their flops (an FMA as 2),
# and the share of issue slots in use. The pass takes r^2, 1/r, r, the
# table index and the exponentials' high-order terms on the integer and
# float32 pipes, so it executes fewer float64 flops than the algorithm
# counts (59 per RGL pair).
PAIRS_FP64_INST_PER_PAIR = 13.51
PAIRS_FP64_FLOPS_PER_PAIR = 20.75
PAIRS_ISSUE_ACTIVE = 0.676

REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {"hbm_gbs": 6800.0, "fallback": True}


def probe_peaks(gpu_index: int) -> dict:
    """float64 and float32 FMA rates of this GPU by the library's probe
    kernel (md_fma_probe), each launch sized to about 5 ms, best of three,
    with the SM clock sampled meanwhile."""
    from paper_1212_6332_gb300 import md
    res = {}
    with ClockSampler(gpu_index) as clk:
        for prec, it0 in (("fp64", 512), ("fp32", 16384)):
            md.fma_probe(prec, it0)
            r = md.fma_probe(prec, it0)
            iters = int(it0 * max(1.0, 5.0 / max(r["ms"], 1e-3)))
            res[prec] = max((md.fma_probe(prec, iters) for _ in range(3)), key=lambda d: d["flops"])
    c = clk.summary()
    return {"fp64_tflops": res["fp64"]["flops"] / 1e12, "fp32_tflops": res["fp32"]["flops"] / 1e12,
            "sm_count": res["fp64"]["n_sm"], "fp64_launch_ms": res["fp64"]["ms"],
            "fp32_launch_ms": res["fp32"]["ms"], "clocks": c,
            "how": "md_fma_probe: every resident thread runs 8 independent FMA chains; best of 3 launches of ~5 ms",
            "fp64_derived_tflops": FP64_DERIVED_TFLOPS}


def cpu_info() -> dict:
    """Host CPU: logical cores and the model line(s) of /proc/cpuinfo."""
    model = None
    try:
        txt = pathlib.Path("/proc/cpuinfo").read_text()
        for key in ("model name", "Model", "CPU part"):
            for line in txt.splitlines():
                if line.lower().startswith(key.lower()):
                    model = line.split(":", 1)[1].strip()
                    if key == "CPU part":
                        impl = [ln.split(":", 1)[1].strip() for ln in txt.splitlines()
                                if ln.startswith("CPU implementer")]
                        model = f"CPU implementer {impl[0] if impl else '?'}, part {model}"
                    break
            if model:
                break
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def roofline_block(prof: dict, N: int, precision: str, kind: str, K: float, Ki: float, peaks: dict,
                   hbm_gbs: float, phases=("pairs", "density", "force", "grad"), note: str | None = None) -> dict:
    """The dominant kernel of one run (largest event time among the hot
    phases) against both ceilings: algorithmic bytes over time against the
    measured HBM bandwidth, algorithmic flops over time against the measured
    FMA rate of its pipe (float64 or float32); the binding ceiling is the
    larger fraction."""
    ms = {p: prof["ms"].get(p, 0.0) for p in phases if prof["ms"].get(p, 0.0) > 0}
    if not ms:
        return {"kernel": None, "note": "no timed hot phase"}
    dom = max(ms, key=ms.get)
    launches = max(prof["timed"].get(dom, 1), 1)
    launch_ms = ms[dom] / launches
    kname, fl, by, pipe = kernel_model(dom, precision, kind, K, Ki)
    out = {"phase": dom, "kernel": kname, "launch_ms": launch_ms, "launches": launches,
           "share_of_timed": ms[dom] / max(sum(prof["ms"].values()), 1e-12), "mean_list_len": K, "mean_in_cutoff": Ki}
    if fl is None:
        out["note"] = "no work model for this phase"
        return out
    peak_alu = peaks["fp64_tflops"] if pipe == "fp64" else peaks["fp32_tflops"]
    a_alu = N * fl / (launch_ms * 1e-3) / 1e12
    a_hbm = N * by / (launch_ms * 1e-3) / 1e9
    out["alu"] = {"pipe": pipe, "achieved": a_alu, "peak": peak_alu, "unit": "TFLOP/s", "frac": a_alu / peak_alu,
                  "flops_per_launch": N * fl, "peak_source": "measured (md_fma_probe)"}
    out["hbm"] = {"achieved": a_hbm, "peak": hbm_gbs, "unit": "GB/s", "frac": a_hbm / hbm_gbs,
                  "bytes_per_launch": N * by, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    fa, fh = a_alu / peak_alu, a_hbm / hbm_gbs
    out["binding"] = pipe if fa >= fh else "hbm"
    if max(fa, fh) < 0.5:
        out["binding_note"] = "both below half: latency / issue bound"
    if note:
        out["note"] = note
    return out


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
    """Mean list length K and mean entries inside r_cut over a sample of
    atoms. box: [3] or per-atom [N, 3] box lengths."""
    import torch
    nn, nl = sysm.neighbors()
    n = nn.shape[0]
    idx = torch.linspace(0, n - 1, min(sample, n), device="cuda").long()
    nns = nn[idx].long()
    cols = nl[idx].long()
    valid = torch.arange(cols.shape[1], device="cuda")[None, :] < nns[:, None]
    cols = torch.where(valid, cols, torch.zeros_like(cols))
    d = x_dev[cols] - x_dev[idx][:, None, :]
    bt = torch.as_tensor(np.asarray(box, dtype=np.float64), device="cuda")
    if bt.dim() == 2:
        bt = bt[idx][:, None, :]
    d = d - bt * torch.round(d / bt)
    r2 = (d * d).sum(-1)
    inside = ((r2 < rc * rc) & valid).sum(1).double().mean().item()
    K = nns.double().mean().item()
    del nn, nl
    return K, inside


def oracle_sample(steps: int, cells: int = ORACLE_CELLS, threads: int = 1, spec=None, a=I.A_CU, mass=I.MASS_CU,
                  temp=TEMP, seed=SEED, label="fcc Cu, RGL Cu") -> dict:
    """The CPU oracle on a cells^3 fcc box of the workload's lattice,
    potential, temperature and seed: `steps` velocity-Verlet steps, minus a
    run of no steps (its list build and first forces). threads > 1 runs the
    oracle's all-cores form (OpenMP, thread-private sums)."""
    import oracle as O
    spec = spec or I.RGL_CU
    bx = I.perturbed_fcc(cells, a, temp, mass, seed)
    pot = O.Potential(spec)
    used = O.set_threads(threads)
    try:
        t0 = time.perf_counter()
        O.md_run(pot, bx.x, bx.v, bx.box, mass, DT, SKIN, 0)
        t1 = time.perf_counter()
        O.md_run(pot, bx.x, bx.v, bx.box, mass, DT, SKIN, steps)
        t2 = time.perf_counter()
    finally:
        O.set_threads(1)
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / steps
    return dict(value=bx.n / per_step, unit=UNIT, cores=used, per_step_s=per_step, n=bx.n, setup_s=t1 - t0,
                sample=f"oracle on a {cells}^3-cell box ({bx.n} atoms; {label}, {temp:.0f} K, seed {seed}), "
                       f"{steps} velocity-Verlet steps minus a run of none, {used} thread(s)")


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


# Single-box workloads of the --spec option (profiling runs; the default
# is the timed 4M-atom Cu box): potential, lattice constant, mass,
# temperature, seed and name.
SPECS = {
    "rgl_cu": (I.RGL_CU, I.A_CU, I.MASS_CU, TEMP, SEED, "fcc Cu", "RGL Cu taper 4.5-5.0 A"),
    "sc_cu": (I.SC_CU, I.A_CU, I.MASS_CU, TEMP, SEED, "fcc Cu", "Sutton-Chen Cu taper 6.92-7.22 A"),
    "rgl_ni": (I.RGL_NI, I.A_NI, I.MASS_NI, 600.0, 3, "fcc Ni", "RGL Ni taper 4.3-4.8 A"),
}


def workload_name(cells: int, precision: str, spec: str = "rgl_cu") -> str:
    """The timed single-box workload, named by what it is."""
    _, _, _, temp, _, lat, pot = SPECS[spec]
    return (f"{lat} {cells}^3 cells ({4 * cells ** 3} atoms), {pot}, skin {SKIN} A, "
            f"{temp:.0f} K, dt {DT} fs, " + ("float64" if precision == "fp64" else "mixed precision"))


def run_reference(args):
    """The CPU oracle on the timed arm's own box (fcc Cu, --cells^3 cells,
    RGL Cu, 300 K, seed 1) on all host cores: W untimed steps, then K timed
    steps minus a run of none (the list build and first forces every run
    starts with)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    W, K = args.warmup, max(args.steps, 1)
    threads = O.max_threads()
    bx = I.perturbed_fcc(args.cells, I.A_CU, TEMP, I.MASS_CU, SEED)
    pot = O.Potential(I.RGL_CU)
    used = O.set_threads(threads)
    try:
        st = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, DT, SKIN, max(W, 0))
        t0 = time.perf_counter()
        O.md_run(pot, st["x"], st["v"], bx.box, I.MASS_CU, DT, SKIN, 0)
        t1 = time.perf_counter()
        run = O.md_run(pot, st["x"], st["v"], bx.box, I.MASS_CU, DT, SKIN, K)
        t2 = time.perf_counter()
    finally:
        O.set_threads(1)
    per_step = max((t2 - t1) - (t1 - t0), 1e-9) / K
    value = bx.n / per_step
    cpu = cpu_info()
    sample = (f"the oracle on the whole timed box ({bx.n} atoms) on {used} thread(s) (OpenMP, thread-private "
              f"sums); per-step time = ({K} steps - a run of none) / {K}, after {W} untimed steps")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": per_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(args.cells, "fp64"), "atoms": bx.n, "n_rebuild": run["n_rebuild"],
                      "timed_s": t2 - t1, "setup_s": t1 - t0},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                            "nproc": cpu["nproc"], "cpu_model": cpu["model"]},
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
    x_dev = torch.tensor(x_h, device="cuda")
    s.set_state(x_dev, torch.tensor(v_h, device="cuda"))
    Kl, Ki = list_stats(s, x_dev, box, spec.get("r_cut", spec.get("r_hi", 5.0)))
    del x_dev
    th_w = s.step(W, use_graph=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    th = s.step(K, use_graph=True)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    # per-phase event times from a further, untimed stretch (events turn
    # graph replay off)
    s.profile_start(timing=True)
    s.step(K)
    prof = s.profile_read()
    s.close()
    return dict(value=len(x_h) * K / (ms * 1e-3), ms_per_step=ms / K, n_rebuild=th["n_rebuild"] - th_w["n_rebuild"],
                graph=True,
                phase_ms_per_step={k: v / max(K, 1) for k, v in prof["ms"].items()},
                mean_list_len=Kl, mean_in_cutoff=Ki, _prof=prof)


def run_small(K: int, use_graph: bool) -> dict:
    """The 2048-atom Cu box (8^3 cells, RGL Cu, 300 K, seed 12345), K
    velocity-Verlet steps in one call: launch-bound, the working set sits in
    L2 (a latency figure, not an HBM one)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(8, I.A_CU, 300.0, I.MASS_CU, 12345)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=SKIN, dt=DT, mass=I.MASS_CU)
    x_dev = torch.tensor(bx.x, device="cuda")
    s.set_state(x_dev, torch.tensor(bx.v, device="cuda"))
    Kl, Ki = list_stats(s, x_dev, bx.box, I.RGL_CU["r_cut"])
    th_w = s.step(K, use_graph=use_graph)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    th = s.step(K, use_graph=use_graph)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    s.profile_start(timing=True)
    s.step(K)
    prof = s.profile_read()
    s.close()
    return dict(value=bx.n * K / (ms * 1e-3), ms_per_step=ms / K, steps=K, n_rebuild=th["n_rebuild"] - th_w["n_rebuild"],
                graph=use_graph, l2="working set inside L2", mean_list_len=Kl, mean_in_cutoff=Ki, atoms=bx.n,
                phase_ms_per_step={k: v / max(K, 1) for k, v in prof["ms"].items()}, _prof=prof)


def run_batch(precision: str, K: int, W: int, n_boxes: int = 4096, use_graph: bool = True,
              schedule: str = "tile") -> dict:
    """The 4096-box batch (n ~ U{3..10} fcc Cu repeats, T ~ U(300, 1500) K,
    RGL Cu): all boxes advance together, one launch per phase (graph-replayed)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(n_boxes, I.A_CU, I.MASS_CU, seed=2024)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=SKIN, dt=DT, mass=I.MASS_CU,
               precision=precision)
    x_dev = torch.tensor(bt.x, device="cuda")
    s.set_state(x_dev, torch.tensor(bt.v, device="cuda"))
    counts = np.diff(np.asarray(bt.atom_offsets))
    Kl, Ki = list_stats(s, x_dev, np.repeat(np.asarray(bt.box), counts, axis=0), I.RGL_CU["r_cut"])
    del x_dev
    s.batch_step(W, schedule=schedule, use_graph=use_graph, per_box=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    s.batch_step(K, schedule=schedule, use_graph=use_graph, per_box=False)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    n = int(bt.atom_offsets[-1])
    phases = prof = None
    if schedule == "tile":
        # phase split from a further, untimed stretch of the same run (phase
        # events turn graph replay off, so they stay out of the timed steps)
        s.profile_start(timing=True)
        s.batch_step(K, schedule=schedule, use_graph=False, per_box=False)
        prof = s.profile_read()
        phases = {k: v / max(K, 1) for k, v in prof["ms"].items()}
    s.close()
    return dict(value=n * K / (ms * 1e-3), ms_per_step=ms / K, atoms=n, boxes=n_boxes, schedule=schedule,
                graph=use_graph and schedule == "tile", phase_ms_per_step=phases, mean_list_len=Kl,
                mean_in_cutoff=Ki, _prof=prof)


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
    from paper_1212_6332_gb300.fit import ForceField, config_index, force_matching_loss, make_batch, theta_of
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
    idx = config_index(counts)
    theta = theta_of(model).cuda().requires_grad_(True)

    def once():
        f, e = ForceField.apply(theta, s, model)
        L = force_matching_loss(f, e, f_tgt, e_tgt, counts, idx=idx)
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
    # per-phase device time of one further iteration (forward passes and
    # the adjoint), untimed
    s.profile_start(timing=True)
    once()
    prof = s.profile_read()
    Kl = Ki = None
    if kind == "rgl":
        x_all = torch.tensor(np.concatenate([c.x for c in cfgs]), device="cuda")
        boxes = np.repeat(np.stack([c.box for c in cfgs]), [c.n for c in cfgs], axis=0)
        Kl, Ki = list_stats(s, x_all, boxes, I.RGL_CU["r_cut"])
    s.close()
    return dict(value=K / dt, unit="(loss + gradient over 256 configs)/s", atom_grads_per_s=n * K / dt,
                n_params=int(theta.numel()), loss=float(L.item()), precision=precision, model=kind, atoms=n,
                phase_ms_per_iter=prof["ms"], mean_list_len=Kl, mean_in_cutoff=Ki, _prof=prof)


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
                    help="only the batch leg with this many boxes (profiling runs; prints its dict)")
    ap.add_argument("--schedule", default="tile", choices=["tile", "box"],
                    help="schedule of the --batch-boxes leg")
    ap.add_argument("--spec", default="rgl_cu", choices=sorted(SPECS),
                    help="potential and lattice of the single box (profiling runs; the timed workload is rgl_cu)")
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
        print(json.dumps(run_batch(args.precision, K, W, n_boxes=args.batch_boxes, schedule=args.schedule)))
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

    peaks = probe_peaks(local)
    mp = measured_peaks()
    hbm = mp.get("hbm_gbs", 6800.0)
    hbm_src = "fallback" if "fallback" in mp else "measured"

    pspec, a_lat, mass, temp, seed, _, _ = SPECS[args.spec]
    bx = I.perturbed_fcc(args.cells, a_lat, temp, mass, seed)
    N = bx.n
    x_dev = torch.tensor(bx.x, device="cuda")
    v_dev = torch.tensor(bx.v, device="cuda")
    s = System(pspec, box=bx.box, n_atoms=N, skin=SKIN, dt=DT, mass=mass, precision=args.precision)
    s.set_state(x_dev, v_dev)
    K_list, K_in = list_stats(s, x_dev, bx.box, pspec["r_cut"])
    th_w = s.step(W, use_graph=True)

    def barrier():
        if dist is not None:
            dist.barrier()

    # the timed steps: md_step with CUDA-graph replay, as a user runs it;
    # launches are counted (not timed) meanwhile
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.profile_start(timing=False)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        th = s.step(K, use_graph=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = s.profile_read()["launches"]
    ms = ev0.elapsed_time(ev1)
    value, ms_max = combine_ranks(ms, N, K, dist)

    # per-kernel times: K further steps with per-phase CUDA events on the
    # launching stream (graph replay off while they record), untimed
    s.profile_start(timing=True)
    th_p = s.step(K)
    prof = s.profile_read()
    phase_ms = {k: prof["ms"][k] / max(K, 1) for k in prof["ms"]}
    phase_sum = sum(phase_ms.values())
    # the stretch may catch another number of list builds than the timed
    # steps: the phase sum with its build time rescaled to the timed count
    # (md_step counts builds since the state was set: differences per stretch)
    reb_timed = th["n_rebuild"] - th_w["n_rebuild"]
    reb_stretch = th_p["n_rebuild"] - th["n_rebuild"]
    reb_fixed = phase_ms.get("rebuild", 0.0) * (reb_timed / reb_stretch if reb_stretch else 1.0)
    phase_sum_same_builds = phase_sum - phase_ms.get("rebuild", 0.0) + reb_fixed

    # dominant kernel of the headline against the measured float64 FMA rate
    kind = pspec["kind"]
    main_block = roofline_block(prof, N, args.precision, kind, K_list, K_in, peaks, hbm)
    dom = main_block["phase"]
    alu = main_block.get("alu", {})
    roofline = {"bound": "alu", "kernel": main_block["kernel"], "achieved": alu.get("achieved"),
                "peak": alu.get("peak"), "unit": "TFLOP/s", "frac": alu.get("frac"),
                "peak_source": f"measured: md_fma_probe {'float64' if alu.get('pipe') == 'fp64' else 'float32'} "
                               f"FMA rate in this run ({peaks['sm_count']} SMs, "
                               f"SM clock {peaks['clocks'].get('sm_mhz')} MHz); derived "
                               f"{FP64_DERIVED_TFLOPS:.3f} TFLOP/s float64 from unit counts",
                "traffic": (PAIRS_DRAM_BYTES_PER_ATOM * N
                            if dom == "pairs" and args.precision == "fp64" and args.spec == "rgl_cu" else None),
                "traffic_source": "ncu capture of 1,048,576 atoms scaled by the atom count",
                "flops_per_launch": alu.get("flops_per_launch"), "launch_ms": main_block["launch_ms"],
                "launch_ms_source": "CUDA events around each launch of the kernel on its stream, over K steps "
                                    "after the timed ones",
                "hbm": main_block.get("hbm"), "binding": main_block.get("binding"),
                "peaks": peaks}
    if dom == "pairs" and args.precision == "fp64" and args.spec == "rgl_cu" and alu.get("frac"):
        # the algorithm's float64 flops per second exceed the float64 pipe's
        # peak because part of the work runs exactly on other pipes: the
        # executed float64 flops (ncu count per pair) against the same peak
        # say how busy the float64 pipe is, the issue share what binds
        pairs_n = N * K_in / 2.0
        ex = pairs_n * PAIRS_FP64_FLOPS_PER_PAIR / (main_block["launch_ms"] * 1e-3) / 1e12
        roofline["executed_fp64"] = {
            "flops_per_pair": PAIRS_FP64_FLOPS_PER_PAIR, "inst_per_pair": PAIRS_FP64_INST_PER_PAIR,
            "achieved": ex, "peak": alu.get("peak"), "unit": "TFLOP/s", "frac": ex / alu.get("peak"),
            "source": "float64 instruction counts per evaluated pair from the ncu capture of 1,048,576 atoms "
                      "(profiles/k_pairs_half_rgl_cu_1m_fp64.md) over this run's launch time"}
        roofline["issue_active"] = PAIRS_ISSUE_ACTIVE
        roofline["note"] = ("achieved/frac: the algorithm's float64 flops (59 per RGL pair, counted for a plain "
                            "float64 evaluation) over the launch time; above 1 because r^2, 1/r, r, the table "
                            "index and the exponentials' high-order terms run exactly on the integer and float32 "
                            "pipes. The pass is bound by instruction issue (issue_active, ncu) with the float64 "
                            "pipe at executed_fp64.frac")
    # the whole step against HBM by its algorithmic byte count (list and
    # positions read by both force passes)
    step_bytes = N * STEP_BYTES(K_list)
    roofline["step_hbm"] = {"bytes_per_step": step_bytes, "achieved": step_bytes / (ms_max / K * 1e-3) / 1e9,
                            "peak": hbm, "unit": "GB/s",
                            "frac": step_bytes / (ms_max / K * 1e-3) / 1e9 / hbm, "peak_source": hbm_src,
                            "definition": "2 x 4K + 2 x 24 B per atom-step, K the mean list length"}
    configs = {"C2_rgl_fp64_300K": main_block}

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
        s.step(1, use_graph=True)
        s.get_state(xh, vh)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_value = combine_ranks(t_e2e * 1e3, N, K_e2e, dist)[0] if K_e2e > 0 else None
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": 2 * N * 3 * 8,
           "d2h_bytes_per_step": 2 * N * 3 * 8 + 56,
           "call": "md_set_state(host) + md_step(1, graph replay) + md_get_state(host) per step",
           "steps": K_e2e}

    def strip(d):
        return {k: v for k, v in d.items() if not k.startswith("_")}

    variants = {}
    cpu = None
    batch = grad = None
    if rank == 0 and not args.no_extras:
        s.close()
        del s
        v = run_variant("mixed", W, K, bx.x, bx.v, bx.box)
        configs["C2_rgl_mixed_300K"] = roofline_block(v["_prof"], N, "mixed", "rgl", v["mean_list_len"],
                                                      v["mean_in_cutoff"], peaks, hbm)
        variants["mixed"] = strip(v)
        variants["fp64"] = {"value": value, "ms_per_step": ms_max / K}
        hot = I.perturbed_fcc(args.cells, I.A_CU, 1200.0, I.MASS_CU, 2)
        variants["fp64_1200K"] = strip(run_variant("fp64", W, K, hot.x, hot.v, hot.box))
        variants["mixed_1200K"] = strip(run_variant("mixed", W, K, hot.x, hot.v, hot.box))
        del hot
        v = run_variant("fp64", W, max(5, K // 3), bx.x, bx.v, bx.box, spec=I.SC_CU)
        configs["C2_sc_fp64"] = roofline_block(v["_prof"], N, "fp64", "sc", v["mean_list_len"], v["mean_in_cutoff"],
                                               peaks, hbm)
        variants["sc_fp64"] = strip(v)
        v = run_variant("mixed", W, K, bx.x, bx.v, bx.box, spec=I.SC_CU)
        configs["C2_sc_mixed"] = roofline_block(v["_prof"], N, "mixed", "sc", v["mean_list_len"], v["mean_in_cutoff"],
                                                peaks, hbm)
        variants["sc_mixed"] = strip(v)
        ni = I.perturbed_fcc(80, I.A_NI, 600.0, I.MASS_NI, 3)
        for prec in ("fp64", "mixed"):
            v = run_variant(prec, W, K, ni.x, ni.v, ni.box, spec=I.RGL_NI, mass=I.MASS_NI)
            configs[f"C3_ni_{prec}"] = roofline_block(v["_prof"], ni.n, prec, "rgl", v["mean_list_len"],
                                                      v["mean_in_cutoff"], peaks, hbm)
            variants[f"ni_2m_{prec}"] = strip(v)
        del ni
        variants["fp64_newton3"] = strip(run_variant("fp64", W, K, bx.x, bx.v, bx.box, newton3=True))
        variants["fp64_thermostat"] = strip(run_variant("fp64", W, K, bx.x, bx.v, bx.box, thermostat=(300.0, 100.0)))
        variants["fp64_barostat"] = strip(run_variant("fp64", W, K, bx.x, bx.v, bx.box,
                                                      barostat=(0.0, 1000.0, 160.21766208 / 140.0)))
        al = I.perturbed_fcc(args.cells, 3.57, TEMP, I.MASS_CU, 5)
        al_types = np.random.default_rng(5).integers(0, 2, al.n).astype(np.int32)
        al_spec = alloy_model()
        variants["alloy_cuni_fp64"] = strip(run_variant("fp64", W, K, al.x, al.v, al.box, spec=al_spec,
                                                        types=al_types))
        variants["alloy_cuni_mixed"] = strip(run_variant("mixed", W, K, al.x, al.v, al.box, spec=al_spec,
                                                         types=al_types))
        del al
        v = run_small(200, True)
        configs["C1_cu_2048_fp64"] = roofline_block(
            v["_prof"], v["atoms"], "fp64", "rgl", v["mean_list_len"], v["mean_in_cutoff"], peaks, hbm,
            note="2048 atoms: the working set sits in L2 and the step is launch-bound; the kernel figures are "
                 "from per-phase events with graph replay off")
        variants["cu_2048_graph"] = strip(v)
        variants["cu_2048_nograph"] = strip(run_small(200, False))
        del x_dev, v_dev
        torch.cuda.empty_cache()
        kb = max(5, min(K, 20))
        b64 = run_batch("fp64", kb, W)
        bmx = run_batch("mixed", kb, W)
        configs["C4_batch_fp64"] = roofline_block(b64["_prof"], b64["atoms"], "fp64", "rgl", b64["mean_list_len"],
                                                  b64["mean_in_cutoff"], peaks, hbm)
        configs["C4_batch_mixed"] = roofline_block(bmx["_prof"], bmx["atoms"], "mixed", "rgl",
                                                   bmx["mean_list_len"], bmx["mean_in_cutoff"], peaks, hbm)
        batch = {"fp64": strip(b64), "fp64_box": strip(run_batch("fp64", kb, W, schedule="box")),
                 "mixed": strip(bmx), "one_launch_per_box": run_per_box_sample(kb)}
        kg = max(3, min(K, 10))
        grad = {}
        for name, prec, model in (("rgl_fp64", "fp64", "rgl"), ("rgl_mixed", "mixed", "rgl"),
                                  ("spline_fp64", "fp64", "spline"), ("spline_mixed", "mixed", "spline"),
                                  ("alloy_fp64", "fp64", "alloy"), ("alloy_mixed", "mixed", "alloy")):
            g = run_grad(kg, 2, prec, model)
            if model == "rgl":
                configs[f"C5_grad_rgl_{prec}"] = roofline_block(
                    g["_prof"], g["atoms"], prec, "rgl", g["mean_list_len"], g["mean_in_cutoff"], peaks, hbm,
                    note="one loss + gradient iteration: forward passes of the new parameters and the adjoint")
            grad[name] = strip(g)
    if rank == 0 and not args.no_extras:
        import oracle as O
        O.build()
        info = cpu_info()
        all_cores = O.max_threads()
        one = oracle_sample(3)
        full = oracle_sample(3, cells=args.cells, threads=all_cores)
        sc = oracle_sample(2, cells=args.cells, threads=all_cores, spec=I.SC_CU, label="fcc Cu, Sutton-Chen Cu")
        ni_o = oracle_sample(100, cells=80, threads=all_cores, spec=I.RGL_NI, a=I.A_NI, mass=I.MASS_NI, temp=600.0,
                             seed=3, label="fcc Ni, RGL Ni")
        cpu = {"value": full["value"], "unit": UNIT, "cores": full["cores"], "kind": "oracle",
               "sample": full["sample"], "nproc": info["nproc"], "cpu_model": info["model"],
               "one_core": {k: one[k] for k in ("value", "cores", "sample")},
               "all_cores": {k: full[k] for k in ("value", "cores", "sample")},
               "sc_all_cores": {k: sc[k] for k in ("value", "cores", "sample")},
               "ni_2m_all_cores_100_steps": {k: ni_o[k] for k in ("value", "cores", "sample")},
               "batch_sample": oracle_batch_sample(), "grad_sample": oracle_grad_sample()}
    roofline["configs"] = configs

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
               "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
               "config": {"workload": workload_name(args.cells, args.precision, args.spec),
                          "atoms": N, "parallelism": "replicas" if world > 1 else "single",
                          "l2": "working set (list + positions) larger than L2",
                          "timing": "md_step with CUDA-graph replay (the user path); phases from K further "
                                    "steps with per-phase events",
                          "mean_list_len": K_list, "mean_in_cutoff": K_in,
                          "n_rebuild": reb_timed, "phase_ms_per_step": phase_ms,
                          "phase_sum_ms": phase_sum, "phase_stretch_n_rebuild": reb_stretch,
                          "phase_sum_same_builds_ms": phase_sum_same_builds},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "variants": variants, "batch": batch, "grad": grad}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
