"""Temperature control of Eq. (4) (electron-phonon friction) on the GPU
against the oracle's integrator, across schedules and precisions."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TAU, T_E = 60.0, 300.0


def test_thermostat_trajectory_matches_oracle():
    """The 2048-atom Cu box started at 900 K and coupled to a 300 K electron
    gas: 200 steps on the GPU (with and without CUDA graphs) against the
    oracle's trajectory."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(8, I.A_CU, 900.0, I.MASS_CU, seed=77)
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 200, tau_T=TAU, T_e=T_E)
    for use_graph in (False, True):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
        s.set_thermostat(T_E, TAU)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        out = s.step(200, history=True, use_graph=use_graph)
        x, v = (t.cpu().numpy() for t in s.get_state())
        d = x - ref["x"]
        d -= bx.box * np.round(d / bx.box)
        assert np.abs(d).max() < 1e-9
        assert np.abs(v - ref["v"]).max() < 1e-8 * np.abs(ref["v"]).max()
        hist = out["history"].cpu().numpy()
        assert np.allclose(hist, ref["thermo"][1:], rtol=1e-9, atol=1e-9)
        # the coupling cooled the crystal
        assert hist[-1, 3] < 0.8 * hist[0, 3]


def test_thermostat_off_is_plain_verlet():
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(5, I.A_CU, 600.0, I.MASS_CU, seed=3)
    runs = []
    for tau in (None, 0.0):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
        if tau is not None:
            s.set_thermostat(1000.0, tau)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        s.step(30)
        runs.append([t.cpu().numpy() for t in s.get_state()])
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_thermostat_box_and_tile_schedules_give_the_same_bits():
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(12, I.A_CU, I.MASS_CU, seed=19)
    out = []
    for sched in ("tile", "box"):
        s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU)
        s.set_thermostat(T_E, TAU)
        s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
        s.batch_step(40, schedule=sched)
        out.append([t.cpu().numpy() for t in s.get_state()])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_mixed_precision_thermostat_follows_float64():
    """Mixed precision under the same coupling: the temperature history
    stays within 1% of the float64 run's over 300 steps of cooling."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(6, I.A_CU, 900.0, I.MASS_CU, seed=5)
    hist = {}
    for prec in ("fp64", "mixed"):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, precision=prec)
        s.set_thermostat(T_E, TAU)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        hist[prec] = s.step(300, history=True)["history"].cpu().numpy()[:, 3]
    assert np.abs(hist["mixed"] - hist["fp64"]).max() <= 0.01 * hist["fp64"].max()
    assert hist["fp64"][-1] < 0.8 * hist["fp64"][0]
