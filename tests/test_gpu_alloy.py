"""Several species (Eq. 1-3 with type labels, spline tables per type pair)
on the GPU against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RGL_CUNI = dict(kind="rgl", A=0.5 * (0.0855 + 0.0376), xi=np.sqrt(1.224 * 1.070), p=0.5 * (10.960 + 16.999),
                q=0.5 * (2.278 + 1.189), r0=0.5 * (2.5562 + 2.4911), r_taper=4.5, r_cut=5.0)


def cuni_alloy(n_knots=150, rho_hi=45.0):
    ni = dict(I.RGL_NI, r_taper=4.5, r_cut=5.0)
    tabs = [O.tabulate_spline(sp, n_knots=n_knots, rho_hi=rho_hi) for sp in (I.RGL_CU, RGL_CUNI, ni)]
    return dict(kind="alloy", n_types=2, phi=[t["phi"] for t in tabs], f=[t["f"] for t in tabs],
                F=[tabs[0]["F"], tabs[2]["F"] * 0.9], r_lo=tabs[0]["r_lo"], r_hi=tabs[0]["r_hi"],
                rho_lo=0.0, rho_hi=rho_hi)


def three_species():
    """Three species with distinct tables from scaled Cu tables."""
    sp = O.tabulate_spline(I.RGL_CU, n_knots=120, rho_hi=45.0)
    sc = [1.0, 0.95, 1.1, 1.05, 0.9, 1.0]
    return dict(kind="alloy", n_types=3, phi=[sp["phi"] * c for c in sc], f=[sp["f"] * c for c in sc[::-1]],
                F=[sp["F"], sp["F"] * 0.95, sp["F"] * 1.08], r_lo=sp["r_lo"], r_hi=sp["r_hi"], rho_lo=0.0,
                rho_hi=45.0)


def check(got, ref):
    fscale = np.linalg.norm(ref["f"], axis=1).max()
    assert np.linalg.norm(got["f"] - ref["f"], axis=1).max() <= 1e-10 * fscale
    assert abs(got["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert np.allclose(got["rho"], ref["rho"], rtol=1e-12, atol=0)


def gpu(spec, bx, types, precision="fp64", types_first=True):
    import torch
    from paper_1212_6332_gb300.md import System
    s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, precision=precision)
    if types_first:
        s.set_types(types)
        out = s.compute_forces(torch.tensor(bx.x, device="cuda"))
    else:
        s.compute_forces(torch.tensor(bx.x, device="cuda"))
        s.set_types(types)
        out = dict(s.get_forces(), energy=torch.tensor([s.thermo()["pe"]], dtype=torch.float64))
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["E"] = float(res.pop("energy")[0])
    return s, res


@pytest.mark.parametrize("spec_fn,n", [(cuni_alloy, 6), (three_species, 5)])
def test_alloy_forces_match_oracle(spec_fn, n):
    spec = spec_fn()
    bx = I.perturbed_fcc(n, 3.57, 600.0, I.MASS_CU, seed=50 + n)
    types = np.random.default_rng(n).integers(0, spec["n_types"], bx.n)
    ref = O.forces(O.Potential(spec), bx.x, bx.box, skin=0.3, types=types)
    for first in (True, False):
        _, got = gpu(spec, bx, types, types_first=first)
        check(got, ref)


def test_alloy_trajectory_matches_oracle():
    import torch
    from paper_1212_6332_gb300.md import System
    spec = cuni_alloy()
    bx = I.perturbed_fcc(6, 3.57, 600.0, I.MASS_CU, seed=5)
    types = np.random.default_rng(1).integers(0, 2, bx.n)
    ref = O.md_run(O.Potential(spec), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 100, types=types)
    s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_types(types)
    s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    out = s.step(100, history=True, use_graph=True)
    x, v = (t.cpu().numpy() for t in s.get_state())
    d = x - ref["x"]
    d -= bx.box * np.round(d / bx.box)
    assert np.abs(d).max() < 1e-9
    assert np.allclose(out["history"].cpu().numpy(), ref["thermo"][1:], rtol=1e-10, atol=1e-10)
    assert out["n_rebuild"] >= 1


def test_alloy_mixed_precision_within_bound():
    spec = cuni_alloy()
    bx = I.perturbed_fcc(6, 3.57, 600.0, I.MASS_CU, seed=7)
    types = np.random.default_rng(2).integers(0, 2, bx.n)
    ref = O.forces(O.Potential(spec), bx.x, bx.box, skin=0.3, types=types)
    _, got = gpu(spec, bx, types, precision="mixed")
    rms = np.sqrt(np.mean(np.sum(ref["f"] ** 2, axis=1)))
    assert np.linalg.norm(got["f"] - ref["f"], axis=1).max() <= 5e-5 * rms + 1e-6
    assert abs(got["E"] - ref["E"]) / bx.n <= 1e-6


def test_alloy_batch_per_box_types():
    import torch
    from paper_1212_6332_gb300.md import System
    spec = cuni_alloy()
    bt = I.batch_of_boxes(4, 3.57, I.MASS_CU, seed=31)
    types = np.random.default_rng(3).integers(0, 2, int(bt.atom_offsets[-1]))
    s = System(spec, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU)
    s.set_types(types)
    f, e_box = s.batch_compute_forces(torch.tensor(bt.x, device="cuda"))
    f, e_box = f.cpu().numpy(), e_box.cpu().numpy()
    pot = O.Potential(spec)
    for k in range(4):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        ref = O.forces(pot, bt.x[lo:hi], bt.box[k], skin=0.3, types=types[lo:hi])
        assert np.linalg.norm(f[lo:hi] - ref["f"], axis=1).max() <= 1e-10 * np.linalg.norm(ref["f"], axis=1).max()
        assert e_box[k] == pytest.approx(ref["E"], rel=1e-10)


def test_alloy_limits_are_reported():
    import torch
    from paper_1212_6332_gb300.md import MDError, System
    spec = cuni_alloy()
    bt = I.batch_of_boxes(3, 3.57, I.MASS_CU, seed=2)
    s = System(spec, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU)
    with pytest.raises(MDError):
        s.set_types(np.full(int(bt.atom_offsets[-1]), 2))  # type out of range
    s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
    with pytest.raises(MDError) as err:
        s.batch_step(2, schedule="box")
    assert err.value.code == 7


def alloy_grad_case(spec, precision, seed):
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    cfgs = [I.strained_fcc(n, I.A_CU, seed=seed + k) for k, n in enumerate((3, 4, 3))]
    n = sum(c.n for c in cfgs)
    rng = np.random.default_rng(seed)
    types = rng.integers(0, spec["n_types"], n)
    s = make_batch(spec, cfgs, precision=precision, types=types)
    g_f = rng.normal(size=(n, 3))
    g_e = rng.normal(size=len(cfgs))
    got = s.param_grad(torch.tensor(g_f, device="cuda"), torch.tensor(g_e, device="cuda")).cpu().numpy()
    pot = O.Potential(spec)
    ref = np.zeros(pot.n_param)
    off = 0
    for c, ge in zip(cfgs, g_e):
        O.param_grad(pot, c.x, c.box, g_f[off:off + c.n], ge, ref, types=types[off:off + c.n])
        off += c.n
    assert got.shape == ref.shape == (s.n_params,)
    return got, ref


@pytest.mark.parametrize("spec_fn", [cuni_alloy, three_species])
def test_alloy_adjoint_matches_oracle_forward_mode(spec_fn):
    """Knot gradient for several species (every V and rho pair table and
    every F table) against the oracle's forward-mode derivatives."""
    got, ref = alloy_grad_case(spec_fn(), "fp64", 40)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    # every table receives gradient: no table offset collapsed onto another
    spec = spec_fn()
    off = 0
    for key in ("phi", "f", "F"):
        for t in spec[key]:
            assert np.abs(ref[off:off + len(t)]).max() > 0
            off += len(t)


def test_alloy_mixed_adjoint_within_bound():
    """Mixed precision: each component within 1e-4 of the largest, as for one
    species."""
    got, ref = alloy_grad_case(cuni_alloy(), "mixed", 41)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_alloy_fit_gradient_matches_finite_differences():
    """Autograd through ForceField for an alloy: a few knots of each table
    kind against central differences of the force-matching loss."""
    import torch
    from paper_1212_6332_gb300.fit import ForceField, force_matching_loss, make_batch, theta_of
    spec = cuni_alloy(n_knots=60)
    cfgs = [I.strained_fcc(3, I.A_CU, seed=60 + k) for k in range(3)]
    n = sum(c.n for c in cfgs)
    types = np.random.default_rng(9).integers(0, 2, n)
    ref = make_batch(spec, cfgs, types=types)
    f_tgt = (ref.get_forces()["f"] * 1.02).clone()
    e_tgt = (ref.batch_thermo()[:, 1] * 0.99).clone()
    counts = torch.tensor([c.n for c in cfgs], device="cuda", dtype=torch.float64)
    s = make_batch(spec, cfgs, types=types)
    theta = theta_of(spec).requires_grad_(True)

    def loss_at(th):
        f, e = ForceField.apply(th, s, spec)
        return force_matching_loss(f, e, f_tgt, e_tgt, counts)

    (g,) = torch.autograd.grad(loss_at(theta), theta)
    nphi, nf, nF = len(spec["phi"][0]), len(spec["f"][0]), len(spec["F"][0])
    order = np.argsort(-np.abs(g.detach().numpy()))
    picks = [k for k in order if k < 3 * nphi][:2] + [k for k in order if 3 * nphi <= k < 3 * (nphi + nf)][:2] + \
        [k for k in order if k >= 3 * (nphi + nf)][:2]
    for k in picks:
        h = 1e-6 * max(abs(theta[k].item()), 1e-2)
        tp, tm = theta.detach().clone(), theta.detach().clone()
        tp[k] += h
        tm[k] -= h
        fd = (loss_at(tp).item() - loss_at(tm).item()) / (2 * h)
        assert g[k].item() == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g.detach().numpy()).max()), k
