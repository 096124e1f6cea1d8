"""State loads that keep the neighbour lists.

A handle that already has lists keeps them when new positions stay within
half the skin of the positions the lists were built from (the rule the
steps follow); boxes that moved farther are rebuilt. Positions that crossed
a periodic face since the build are taken as the image next to the build
position. Every case is checked against the oracle on the same positions."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F_TOL = 1e-10


def check(got, ref):
    err = np.linalg.norm(got["f"] - ref["f"], axis=1).max() / np.linalg.norm(ref["f"], axis=1).max()
    assert err <= F_TOL, err
    assert abs(got["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])


def forces_of(s, x):
    out = s.compute_forces(x)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["E"] = float(res.pop("energy")[0])
    return res


def test_small_moves_keep_lists_and_match_oracle():
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(6, I.A_CU, 300.0, I.MASS_CU, seed=31)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    pot = O.Potential(I.RGL_CU)
    check(forces_of(s, bx.x.copy()), O.forces(pot, bx.x, bx.box, skin=0.3))
    rng = np.random.default_rng(5)
    # moves below skin/2 = 0.15 A (|d| <= 0.13 A): no box rebuilds, and the
    # atoms near a face that are pushed across it come back wrapped
    x = bx.x + rng.uniform(-0.05, 0.05, bx.x.shape)
    near = np.where(bx.x[:, 0] < 0.03)[0][:5]
    assert len(near) > 0
    x[near, 0] -= 0.06
    x = I.wrap(x, bx.box)
    check(forces_of(s, x.copy()), O.forces(pot, x, bx.box, skin=0.3))
    # a large move rebuilds the lists and is still exact
    x2 = I.wrap(x + rng.uniform(-0.4, 0.4, x.shape), bx.box)
    check(forces_of(s, x2.copy()), O.forces(pot, x2, bx.box, skin=0.3))


def test_batch_rebuilds_only_the_boxes_that_moved():
    import torch
    from paper_1212_6332_gb300.md import System
    bt = I.batch_of_boxes(6, I.A_CU, I.MASS_CU, seed=17)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, skin=0.3, mass=I.MASS_CU)
    s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
    rng = np.random.default_rng(8)
    x = bt.x.copy()
    for k in range(6):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        amp = 0.5 if k == 2 else 0.05
        x[lo:hi] = I.wrap(x[lo:hi] + rng.uniform(-amp, amp, (hi - lo, 3)), bt.box[k])
    f, e_box = s.batch_compute_forces(torch.tensor(x, device="cuda"))
    f, e_box = f.cpu().numpy(), e_box.cpu().numpy()
    pot = O.Potential(I.RGL_CU)
    for k in range(6):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        ref = O.forces(pot, x[lo:hi], bt.box[k], skin=0.3)
        fb = f[lo:hi]
        assert np.linalg.norm(fb - ref["f"], axis=1).max() <= F_TOL * np.linalg.norm(ref["f"], axis=1).max()
        assert e_box[k] == pytest.approx(ref["E"], rel=1e-10)


def test_reloading_the_own_state_continues_the_trajectory():
    """Loading a handle's own state back (the end-to-end pattern: download,
    upload, step) keeps its lists and follows the same trajectory as a
    fresh handle loaded with that state."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(5, I.A_CU, 900.0, I.MASS_CU, seed=8)
    a = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    a.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    a.step(40)
    xa, va = (t.cpu().numpy().copy() for t in a.get_state())
    b = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    b.set_state(xa.copy(), va.copy())
    a.set_state(xa.copy(), va.copy())
    assert a.thermo()["n_rebuild"] == 0
    a.step(40)
    b.step(40)
    (x1, v1), (x2, v2) = a.get_state(), b.get_state()
    d = (x1 - x2).cpu().numpy()
    d -= bx.box * np.round(d / bx.box)
    assert np.abs(d).max() < 1e-11
    assert torch.allclose(v1, v2, rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_round_trip_of_the_state_changes_nothing(precision):
    """A state read back with md_get_state and loaded again is the current
    state: the forces are kept, and a run interrupted by such a round trip
    (through host buffers) follows the uninterrupted run bit for bit."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(6, I.A_CU, 900.0, I.MASS_CU, seed=41)
    runs = []
    for split in (False, True):
        s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU, precision=precision)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        if split:
            s.step(60)
            xh = torch.empty((bx.n, 3), dtype=torch.float64, pin_memory=True)
            vh = torch.empty((bx.n, 3), dtype=torch.float64, pin_memory=True)
            s.get_state(xh, vh)
            f0 = s.get_forces()["f"].clone()
            s.set_state(xh, vh)
            assert torch.equal(s.get_forces()["f"], f0)
            s.step(60)
        else:
            s.step(120)
        runs.append([t.cpu() for t in s.get_state()] + [s.get_forces()["f"].cpu()])
        s.close()
    for a, b in zip(*runs):
        assert torch.equal(a, b)


def test_new_velocities_keep_forces_and_new_positions_do_not():
    """Loading the current positions with new velocities (a host-side
    velocity change) keeps the forces; loading moved positions recomputes
    them. Both continue like a fresh handle given the same state."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(6, I.A_CU, 600.0, I.MASS_CU, seed=43)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    s.step(30)
    x, v = s.get_state()
    v2 = v * 0.5
    s.set_state(x, v2)
    th = s.thermo()
    assert th["ke"] == pytest.approx(0.25 * float((0.5 * I.MASS_CU * I.MVV_EV * (v * v).sum()).item()), rel=1e-12)
    out = s.step(40, history=True)
    fresh = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    fresh.set_state(x.clone(), v2.clone())
    ref = fresh.step(40, history=True)
    xa, va = (t.cpu().numpy() for t in s.get_state())
    xb, vb = (t.cpu().numpy() for t in fresh.get_state())
    d = xa - xb
    d -= bx.box * np.round(d / bx.box)
    assert np.abs(d).max() < 1e-11
    assert np.abs(va - vb).max() < 1e-10 * np.abs(vb).max()
    assert np.allclose(out["history"].cpu().numpy(), ref["history"].cpu().numpy(), rtol=1e-11, atol=1e-12)
    # moved positions: forces recomputed, equal to the oracle's
    x3 = I.wrap(x.cpu().numpy() + 0.01, bx.box)
    s.set_state(torch.tensor(x3, device="cuda"), v2)
    got = s.get_forces()["f"].cpu().numpy()
    ref_f = O.forces(O.Potential(I.RGL_CU), x3, bx.box, skin=0.3)["f"]
    assert np.linalg.norm(got - ref_f, axis=1).max() <= F_TOL * np.linalg.norm(ref_f, axis=1).max()


def test_round_trip_after_pressure_coupling_recomputes_forces():
    """With the Eq. (5) coupling the box scaling follows the last force
    pass, so the forces held after a step are not those of the final
    positions: a state load of those positions must evaluate them again
    (they then equal a fresh handle's forces at the same positions)."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(5, I.A_CU, 300.0, I.MASS_CU, seed=45)
    beta = 160.21766208 / 140.0
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_barostat(0.0, 50.0, beta)
    s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    s.step(20)
    box = s.box()[0]
    assert not np.allclose(box, bx.box)
    x, v = s.get_state()
    held = s.get_forces()["f"].clone()
    s.set_state(x, v)
    got = s.get_forces()["f"]
    fresh = System(I.RGL_CU, box=box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    ref = fresh.compute_forces(x.clone())["f"]
    scale = ref.abs().max().item()
    assert (got - ref).abs().max().item() <= 1e-12 * scale
    assert (held - ref).abs().max().item() > 1e-9 * scale  # the held forces were of the unscaled positions


def test_far_unwrapped_positions_wrap_by_the_oracle_rule():
    """Positions given several box lengths away (and a few ulp below a
    multiple of L, where x - L floor(x/L) rounds below zero) are wrapped on
    the device by the same rule as the oracle: md_get_state returns exactly
    the oracle's wrapped coordinates, all in [0, L), and the forces are
    those of the wrapped box."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(5, I.A_CU, 300.0, I.MASS_CU, seed=57)
    k = np.zeros_like(bx.x)
    k[0::4, 0], k[1::4, 1], k[2::4, 2], k[3::4] = 3.0, -5.0, 7.0, -2.0
    x_far = bx.x + k * bx.box
    # atoms placed a few ulp below k*L on one axis
    for i, kk in zip(range(0, 40, 4), range(-6, 4)):
        x_far[i, 0] = np.nextafter(kk * bx.box[0], -np.inf)
    want = O.wrap(x_far, bx.box)
    assert np.all(want >= 0.0) and np.all(want < bx.box)
    s = System(I.RGL_CU, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    s.set_state(torch.tensor(x_far, device="cuda"))
    x, _ = (t.cpu().numpy() for t in s.get_state())
    assert np.array_equal(x, want)
    check(forces_of(s, torch.tensor(x_far, device="cuda")),
          O.forces(O.Potential(I.RGL_CU), want, bx.box, skin=0.3))
