"""Float64 half-list sums with Newton's third law (md_set_newton3, the CPU
scheme of Sec. 4.3) on the GPU: against the oracle, against the default
full-list sums, and through trajectories with list rebuilds, friction,
pressure coupling and a batch of boxes."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BETA = 160.21766208 / 140.0  # A^3/eV: 1/(140 GPa)


def alloy():
    sp = O.tabulate_spline(I.RGL_CU, n_knots=120, rho_hi=45.0)
    sc = [1.0, 0.95, 1.1]
    return dict(kind="alloy", n_types=2, phi=[sp["phi"] * c for c in sc], f=[sp["f"] * c for c in sc[::-1]],
                F=[sp["F"], sp["F"] * 0.95], r_lo=sp["r_lo"], r_hi=sp["r_hi"], rho_lo=0.0, rho_hi=45.0)


CASES = {
    "rgl_cu": lambda: (I.RGL_CU, I.A_CU, 7, I.MASS_CU),
    "sc_cu": lambda: (I.SC_CU, I.A_CU, 6, I.MASS_CU),
    "spline_cu": lambda: (O.tabulate_spline(I.RGL_CU, n_knots=150, rho_hi=45.0), I.A_CU, 6, I.MASS_CU),
    "alloy": lambda: (alloy(), I.A_CU, 6, I.MASS_CU),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_newton3_forces_match_oracle_and_full_list(case):
    import torch
    from paper_1212_6332_gb300.md import System
    spec, a, n, mass = CASES[case]()
    bx = I.perturbed_fcc(n, a, 600.0, mass, seed=70 + n)
    types = np.random.default_rng(n).integers(0, 2, bx.n) if spec["kind"] == "alloy" else None
    ref = O.forces(O.Potential(spec), bx.x, bx.box, skin=0.3, types=types)
    out = {}
    for n3 in (False, True):
        s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=mass)
        if types is not None:
            s.set_types(types)
        s.set_newton3(n3)
        o = s.compute_forces(torch.tensor(bx.x, device="cuda"))
        out[n3] = {k: v.cpu().numpy() for k, v in o.items()}
        s.close()
    got, full = out[True], out[False]
    fscale = np.linalg.norm(ref["f"], axis=1).max()
    assert np.linalg.norm(got["f"] - ref["f"], axis=1).max() <= 1e-10 * fscale
    assert abs(float(got["energy"][0]) - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert np.allclose(got["rho"], ref["rho"], rtol=1e-12, atol=0)
    assert np.allclose(got["e_atom"].sum(), ref["E"], rtol=1e-12, atol=0)
    # against the reproducible full-list sums: rounding only
    assert np.linalg.norm(got["f"] - full["f"], axis=1).max() <= 1e-12 * fscale
    assert np.allclose(got["rho"], full["rho"], rtol=1e-13, atol=0)
    assert np.allclose(got["e_atom"], full["e_atom"], rtol=1e-12, atol=1e-15)
    # Newton's third law: the half-list forces still sum to zero
    assert np.abs(got["f"].sum(axis=0)).max() <= 1e-10 * fscale


def test_newton3_trajectory_matches_oracle():
    """200 steps at 1200 K (several list rebuilds), with and without CUDA
    graphs, against the oracle's trajectory."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(6, I.A_CU, 1200.0, I.MASS_CU, seed=81)
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 200)
    for use_graph in (False, True):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
        s.set_newton3(True)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        out = s.step(200, history=True, use_graph=use_graph)
        assert out["n_rebuild"] >= 2
        x, v = (t.cpu().numpy() for t in s.get_state())
        d = x - ref["x"]
        d -= bx.box * np.round(d / bx.box)
        assert np.abs(d).max() < 1e-9
        assert np.abs(v - ref["v"]).max() < 1e-8 * np.abs(ref["v"]).max()
        assert np.allclose(out["history"].cpu().numpy(), ref["thermo"][1:], rtol=1e-9, atol=1e-9)
        s.close()


def test_newton3_with_friction_and_pressure_coupling():
    """Eq. (4) friction and the Eq. (5) coupling on top of the half-list sums
    (the second half-kick is its own launch there): 150 steps against the
    oracle, box included."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(5, I.A_CU, 900.0, I.MASS_CU, seed=83)
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 150, tau_T=200.0, T_e=300.0,
                   tau_p=50.0, P0=0.0, beta=BETA)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_newton3(True)
    s.set_thermostat(300.0, 200.0)
    s.set_barostat(0.0, 50.0, BETA)
    s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    out = s.step(150, history=True)
    box = s.box()[0]
    assert np.allclose(box, ref["box"], rtol=1e-11, atol=0)
    x, v = (t.cpu().numpy() for t in s.get_state())
    d = x - ref["x"]
    d -= box * np.round(d / box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(v - ref["v"]).max() < 1e-8 * np.abs(ref["v"]).max()
    assert np.allclose(out["history"].cpu().numpy(), ref["thermo"][1:], rtol=1e-9, atol=1e-9)


def test_newton3_pressure_matches_full_list():
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(7, I.A_CU, 600.0, I.MASS_CU, seed=85)
    p = {}
    for n3 in (False, True):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
        s.set_newton3(n3)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        p[n3] = float(s.pressure().cpu()[0])
        s.close()
    W = O.virial(O.Potential(I.RGL_CU), bx.x, bx.box)
    assert abs(p[True] - p[False]) <= 1e-12 * abs(W / (3.0 * np.prod(bx.box)))


def test_newton3_batch_matches_oracle_per_box():
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(5, I.A_CU, I.MASS_CU, seed=87)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU)
    s.set_newton3(True)
    s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
    s.batch_step(60, schedule="tile")
    x, v = (t.cpu().numpy() for t in s.get_state())
    pot = O.Potential(I.RGL_CU)
    for k in range(5):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        ref = O.md_run(pot, bt.x[lo:hi], bt.v[lo:hi], bt.box[k], I.MASS_CU, 1.0, 0.3, 60)
        d = x[lo:hi] - ref["x"]
        d -= bt.box[k] * np.round(d / bt.box[k])
        assert np.abs(d).max() < 1e-9, k
        assert np.abs(v[lo:hi] - ref["v"]).max() < 1e-8 * np.abs(ref["v"]).max(), k


def test_newton3_switch_back_is_reproducible_and_mixed_is_refused():
    import torch
    from paper_1212_6332_gb300.md import MDError, System
    bx = I.perturbed_fcc(6, I.A_CU, 600.0, I.MASS_CU, seed=89)
    x = torch.tensor(bx.x, device="cuda")
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    f0 = s.compute_forces(x)["f"].clone()
    s.set_newton3(True)
    s.compute_forces(x)
    s.set_newton3(False)
    f1 = s.compute_forces(x)["f"]
    assert torch.equal(f0, f1)
    m = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, precision="mixed")
    with pytest.raises(MDError) as err:
        m.set_newton3(True)
    assert err.value.code == 7


@pytest.mark.parametrize("newton3", [False, True])
def test_list_overflow_under_compression_regrows_mid_run(newton3):
    """Pressure coupling towards 20 GPa shrinks the box by a few per cent, so
    the neighbour counts outgrow a list sized to the initial maximum: the
    overflow is caught on the device, the lists regrow and the trajectory
    stays the oracle's, with plain launches and with graph replay alike (bit
    for bit alike with the full-list sums)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(7, I.A_CU, 600.0, I.MASS_CU, seed=91)
    P0 = 20.0 / 160.21766208  # eV/A^3
    probe = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    probe.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    cap = probe.max_count()
    probe.close()
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 150, tau_p=50.0, P0=P0,
                   beta=BETA)
    assert ref["box"][0] < 0.975 * bx.box[0]
    runs = []
    for use_graph in (False, True):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, max_neighbors=cap)
        s.set_newton3(newton3)
        s.set_barostat(P0, 50.0, BETA)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        s.step(150, use_graph=use_graph)
        assert s.max_count() > cap
        box = s.box()[0]
        assert np.allclose(box, ref["box"], rtol=1e-11, atol=0)
        x, v = (t.cpu().numpy() for t in s.get_state())
        d = x - ref["x"]
        d -= box * np.round(d / box)
        assert np.abs(d).max() < 1e-9
        assert np.abs(v - ref["v"]).max() < 1e-8 * np.abs(ref["v"]).max()
        runs.append((x, v))
        s.close()
    if not newton3:  # the half-list partner updates are atomic adds in no fixed order
        assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
