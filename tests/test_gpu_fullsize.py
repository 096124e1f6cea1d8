"""Parity at the full workload sizes, on sampled outputs.

The oracle cannot evaluate millions of atoms, but an atom's density, energy
and force depend only on atoms within 2 r_cut of it. For each sampled atom
the test cuts that cluster (minimum image, plus a margin) out of the full
box, places it in a large isolated box, and lets the oracle compute the
centre atom's values, which must then equal the GPU's at the usual bars.
Workloads: the 4,000,000-atom Cu box (RGL and Sutton-Chen, float64), the
4,000,000-atom two-species spline alloy (float64), the 2,048,000-atom Ni
box (mixed precision), the 4096-box batch, and the gradient over the
256-configuration fitting set.
"""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def cluster_values(spec, x, box, idx, margin=0.5, types=None):
    """Oracle rho, E_i, F_i of atom idx from its 2 r_cut neighbourhood."""
    rc = spec.get("r_cut", spec.get("r_hi"))
    d = x - x[idx]
    d -= box * np.round(d / box)
    keep = np.where(np.sum(d * d, axis=1) < (2 * rc + margin) ** 2)[0]
    centre = int(np.where(keep == idx)[0][0])
    L = 4 * (2 * rc + margin) + 10.0
    xc = d[keep] + L / 2
    out = O.forces(O.Potential(spec), xc, np.array([L, L, L]), method="pairs",
                   types=None if types is None else types[keep])
    return out["rho"][centre], out["e_atom"][centre], out["f"][centre]


def gpu_full(spec, bx, precision="fp64"):
    import torch
    from paper_1212_6332_gb300.md import System
    s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, precision=precision)
    out = s.compute_forces(torch.tensor(bx.x, device="cuda"))
    res = {k: v.cpu().numpy() for k, v in out.items()}
    s.close()
    return res


@pytest.mark.parametrize("spec,name", [(I.RGL_CU, "rgl"), (I.SC_CU, "sc")])
def test_4m_atom_box_sampled_atoms(spec, name):
    bx = I.perturbed_fcc(100, I.A_CU, 300.0, I.MASS_CU, seed=1)
    got = gpu_full(spec, bx)
    rng = np.random.default_rng(7)
    sample = np.concatenate([rng.choice(bx.n, 12, replace=False), [0, bx.n - 1]])
    fscale = np.abs(got["f"]).max()
    for i in sample:
        rho, e, f = cluster_values(spec, bx.x, bx.box, i)
        assert got["rho"][i] == pytest.approx(rho, rel=1e-12)
        assert got["e_atom"][i] == pytest.approx(e, rel=1e-10)
        assert np.abs(got["f"][i] - f).max() <= 1e-10 * fscale
    # properties of the whole box: net force, energy per atom near the lattice value
    assert np.abs(got["f"].sum(axis=0)).max() <= 1e-9 * bx.n * 1e-3
    assert -3.6 < got["energy"][0] / bx.n < -3.3


def test_4m_atom_alloy_box_sampled_atoms():
    """The 4,000,000-atom two-species spline alloy (a = 3.57 A, random 50/50
    labels), float64: the tabulated pair path at full size."""
    import torch
    from paper_1212_6332_gb300.md import System
    ni = dict(I.RGL_NI, r_taper=4.5, r_cut=5.0)
    cuni = dict(kind="rgl", A=0.5 * (0.0855 + 0.0376), xi=np.sqrt(1.224 * 1.070), p=0.5 * (10.960 + 16.999),
                q=0.5 * (2.278 + 1.189), r0=0.5 * (2.5562 + 2.4911), r_taper=4.5, r_cut=5.0)
    tabs = [O.tabulate_spline(sp, n_knots=200, rho_hi=45.0) for sp in (I.RGL_CU, cuni, ni)]
    spec = dict(kind="alloy", n_types=2, phi=[t["phi"] for t in tabs], f=[t["f"] for t in tabs],
                F=[tabs[0]["F"], tabs[2]["F"]], r_lo=tabs[0]["r_lo"], r_hi=tabs[0]["r_hi"], rho_lo=0.0,
                rho_hi=45.0)
    bx = I.perturbed_fcc(100, 3.57, 300.0, I.MASS_CU, seed=5)
    types = np.random.default_rng(5).integers(0, 2, bx.n).astype(np.int32)
    s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_types(types)
    got = {k: v.cpu().numpy() for k, v in s.compute_forces(torch.tensor(bx.x, device="cuda")).items()}
    s.close()
    rng = np.random.default_rng(8)
    sample = np.concatenate([rng.choice(bx.n, 12, replace=False), [0, bx.n - 1]])
    fscale = np.abs(got["f"]).max()
    for i in sample:
        rho, e, f = cluster_values(spec, bx.x, bx.box, i, types=types)
        assert got["rho"][i] == pytest.approx(rho, rel=1e-12)
        assert got["e_atom"][i] == pytest.approx(e, rel=1e-10)
        assert np.abs(got["f"][i] - f).max() <= 1e-10 * fscale
    assert np.abs(got["f"].sum(axis=0)).max() <= 1e-9 * bx.n * 1e-3


def test_2m_atom_nickel_box_mixed_precision():
    bx = I.perturbed_fcc(80, I.A_NI, 600.0, I.MASS_NI, seed=3)
    got = gpu_full(I.RGL_NI, bx, precision="mixed")
    rng = np.random.default_rng(8)
    rms = np.sqrt(np.mean(np.sum(got["f"] ** 2, axis=1)))
    for i in rng.choice(bx.n, 12, replace=False):
        rho, e, f = cluster_values(I.RGL_NI, bx.x, bx.box, i)
        assert np.linalg.norm(got["f"][i] - f) <= 5e-5 * rms + 1e-6
        assert abs(got["e_atom"][i] - e) <= 1e-5
        assert got["rho"][i] == pytest.approx(rho, rel=1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_4096_box_batch_sampled_boxes(precision):
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(4096, I.A_CU, I.MASS_CU, seed=2024)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU,
               precision=precision)
    f, e_box = s.batch_compute_forces(torch.tensor(bt.x, device="cuda"))
    f, e_box = f.cpu().numpy(), e_box.cpu().numpy()
    rng = np.random.default_rng(9)
    sizes = bt.atom_offsets[1:] - bt.atom_offsets[:-1]
    picks = list(rng.choice(4096, 6, replace=False)) + [int(np.argmin(sizes)), int(np.argmax(sizes))]
    pot = O.Potential(I.RGL_CU)
    for b in picks:
        lo, hi = bt.atom_offsets[b], bt.atom_offsets[b + 1]
        ref = O.forces(pot, bt.x[lo:hi], bt.box[b], skin=0.3)
        fb = f[lo:hi]
        if precision == "fp64":
            assert np.linalg.norm(fb - ref["f"], axis=1).max() <= 1e-10 * np.linalg.norm(ref["f"], axis=1).max()
            assert e_box[b] == pytest.approx(ref["E"], rel=1e-10)
        else:
            rms = np.sqrt(np.mean(np.sum(ref["f"] ** 2, axis=1)))
            assert np.linalg.norm(fb - ref["f"], axis=1).max() <= 5e-5 * rms + 1e-6
            assert abs(e_box[b] - ref["E"]) / (hi - lo) <= 1e-6


def test_fitting_set_gradient_on_a_subset():
    """The gradient over the 256-configuration set with dL/dF and dL/dE set
    to zero outside two configurations equals the oracle's gradient of those
    two configurations."""
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    cfgs = [I.strained_fcc(6, I.A_CU, seed=5000 + k) for k in range(256)]
    model = dict(I.RGL_CU, A=0.0855 * 1.05, xi=1.224 * 0.95, p=10.96 * 1.05, q=2.278 * 0.95, r0=2.5562 * 0.95)
    s = make_batch(model, cfgs)
    n = sum(c.n for c in cfgs)
    rng = np.random.default_rng(11)
    g_f = np.zeros((n, 3))
    g_e = np.zeros(256)
    chosen = [3, 200]
    for c in chosen:
        g_f[c * 864:(c + 1) * 864] = rng.normal(size=(864, 3))
        g_e[c] = rng.normal()
    got = s.param_grad(torch.tensor(g_f, device="cuda"), torch.tensor(g_e, device="cuda")).cpu().numpy()
    pot = O.Potential(model)
    ref = np.zeros(5)
    for c in chosen:
        O.param_grad(pot, cfgs[c].x, cfgs[c].box, g_f[c * 864:(c + 1) * 864], g_e[c], ref)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
