"""The 2,048,000-atom Ni box (80^3 fcc cells, RGL Ni, 600 K) run for 10,000
velocity-Verlet steps at 1 fs in float64 and in mixed precision from the
same start: total-energy drift of both, and the per-atom force error of each
against the oracle on snapshots every 1000 steps, computed from the sampled
atoms' 2 r_cut neighbourhoods (see test_gpu_fullsize)."""
import numpy as np
import pytest

from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STEPS = 10000
SNAP = 1000


def test_nickel_box_drift_and_snapshot_errors():
    import torch
    from paper_1212_6332_gb300.md import System
    from test_gpu_fullsize import cluster_values
    bx = I.perturbed_fcc(80, I.A_NI, 600.0, I.MASS_NI, seed=3)
    rng = np.random.default_rng(12)
    out = {}
    for prec in ("fp64", "mixed"):
        s = System(I.RGL_NI, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_NI, precision=prec)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        e0 = s.thermo()["etot"]
        hist, errs = [], []
        for _ in range(STEPS // SNAP):
            th = s.step(SNAP, history=True, use_graph=True)
            hist.append(th["history"][:, 2].cpu().numpy())
            x, _ = s.get_state()
            x = x.cpu().numpy()
            f = s.get_forces()["f"].cpu().numpy()
            rms = np.sqrt(np.mean(np.sum(f ** 2, axis=1)))
            for i in rng.choice(bx.n, 4, replace=False):
                _, _, fr = cluster_values(I.RGL_NI, x, bx.box, i)
                errs.append(np.linalg.norm(f[i] - fr) / rms)
        et = np.concatenate(hist) / bx.n
        slope = np.polyfit(np.arange(len(et)), et, 1)[0]  # eV/atom per fs
        out[prec] = dict(slope=slope, span=np.abs(et - e0 / bx.n).max(), err=max(errs))
        s.close()
    print("nickel 10k steps:", out)
    assert out["fp64"]["err"] <= 1e-9  # relative to the RMS force
    assert out["mixed"]["err"] <= 5e-5 + 1e-6
    for prec in ("fp64", "mixed"):
        assert abs(out[prec]["slope"]) < 1e-8, out
        assert out[prec]["span"] < 5e-5, out
