"""Batches of independent boxes (Sec. 4.4): the tile schedule (one launch per
phase over all boxes) and the block-per-box schedule (one thread block per
box for all steps) against each other, against single-box runs and against
the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def batch_system(bt, **kw):
    import torch
    from paper_1212_6332_gb300.md import System
    kw.setdefault("skin", 0.3)
    s = System(I.RGL_CU, boxes=bt.box, atom_offsets=bt.atom_offsets, mass=I.MASS_CU, **kw)
    s.set_state(torch.tensor(bt.x, device="cuda"), torch.tensor(bt.v, device="cuda"))
    return s


def small_batch(n_boxes=24, seed=77):
    return I.batch_of_boxes(n_boxes, I.A_CU, I.MASS_CU, seed=seed)


def test_box_and_tile_schedules_give_the_same_bits():
    bt = small_batch()
    a, b = batch_system(bt), batch_system(bt)
    ta = a.batch_step(60, schedule="tile").cpu().numpy()
    tb = b.batch_step(60, schedule="box").cpu().numpy()
    (xa, va), (xb, vb) = a.get_state(), b.get_state()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    assert np.array_equal(va.cpu().numpy(), vb.cpu().numpy())
    assert np.array_equal(ta, tb)


def test_each_box_equals_its_own_single_box_run():
    import torch
    from paper_1212_6332_gb300.md import System
    bt = small_batch(8, seed=5)
    s = batch_system(bt)
    s.batch_step(40, schedule="box")
    x, v = (t.cpu().numpy() for t in s.get_state())
    for k in (0, 3, 7):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        one = System(I.RGL_CU, box=bt.box[k], n_atoms=hi - lo, skin=0.3, mass=I.MASS_CU)
        one.set_state(torch.tensor(bt.x[lo:hi], device="cuda"), torch.tensor(bt.v[lo:hi], device="cuda"))
        one.step(40)
        x1, v1 = (t.cpu().numpy() for t in one.get_state())
        assert np.array_equal(x1, x[lo:hi]) and np.array_equal(v1, v[lo:hi])


def test_batch_trajectory_matches_oracle_per_box():
    bt = small_batch(6, seed=9)
    s = batch_system(bt)
    s.batch_step(50, schedule="box")
    x, v = (t.cpu().numpy() for t in s.get_state())
    pot = O.Potential(I.RGL_CU)
    for k in range(6):
        lo, hi = bt.atom_offsets[k], bt.atom_offsets[k + 1]
        ref = O.md_run(pot, bt.x[lo:hi], bt.v[lo:hi], bt.box[k], I.MASS_CU, 1.0, 0.3, 50)
        # positions in [0, L), compared without a periodic fold
        assert np.all(x[lo:hi] >= 0.0) and np.all(x[lo:hi] < bt.box[k])
        assert np.abs(x[lo:hi] - ref["x"]).max() < 1e-9
        assert np.abs(v[lo:hi] - ref["v"]).max() < 1e-9


def test_box_schedule_regrows_an_overflowing_list():
    bt = small_batch(10, seed=3)
    a = batch_system(bt)
    b = batch_system(bt, max_neighbors=16)
    a.batch_step(30, schedule="box")
    b.batch_step(30, schedule="box")
    (xa, _), (xb, _) = a.get_state(), b.get_state()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())


def test_autotuner_picks_a_schedule_and_keeps_the_bits():
    bt = small_batch(32, seed=11)
    a, b = batch_system(bt), batch_system(bt)
    a.batch_step(40, schedule="auto")
    b.batch_step(40, schedule="tile")
    sched = a.schedule()
    assert sched["choice"] in ("tile", "box") and sched["ms_tile"] > 0 and sched["ms_box"] > 0
    assert np.array_equal(a.get_state()[0].cpu().numpy(), b.get_state()[0].cpu().numpy())


def test_mixed_precision_batch_uses_the_tile_schedule():
    from paper_1212_6332_gb300.md import MDError
    bt = small_batch(4, seed=1)
    s = batch_system(bt, precision="mixed")
    with pytest.raises(MDError):
        s.batch_step(2, schedule="box")
    s.batch_step(10, schedule="auto")
    assert s.schedule()["choice"] == "tile"


@pytest.mark.parametrize("spec,n_cells,temp", [(I.RGL_CU, 8, 300.0), (I.SC_CU, 6, 1200.0)])
def test_small_single_box_kernels_give_the_box_schedule_bits(spec, n_cells, temp):
    """A single box of a few thousand atoms takes the small-system float64
    kernels (one thread per pair row; sums staged in shared memory); its
    trajectory equals, bit for bit, the block-per-box schedule's (whose
    passes equal the large-system kernels', as the test above checks).
    Sutton-Chen lists (140 entries) span several staged chunks."""
    import torch
    from paper_1212_6332_gb300.md import System
    bx = I.perturbed_fcc(n_cells, I.A_CU, temp, I.MASS_CU, seed=90 + n_cells)
    one = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    one.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    th = one.step(60, history=True, use_graph=True)
    offs = np.array([0, bx.n], dtype=np.int64)
    b = System(spec, boxes=bx.box[None, :], atom_offsets=offs, skin=0.3, mass=I.MASS_CU)
    b.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    b.batch_step(60, schedule="box")
    (x1, v1), (x2, v2) = one.get_state(), b.get_state()
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())
    assert th["n_rebuild"] >= 1
    f1, f2 = one.get_forces(), b.get_forces()
    assert np.array_equal(f1["f"].cpu().numpy(), f2["f"].cpu().numpy())


def test_small_batch_tile_equals_box_schedule():
    """Sixteen boxes (under the small-system threshold, per-box geometry):
    the tile schedule's small kernels and the box schedule agree bit for bit."""
    bt = small_batch(16, seed=21)
    assert int(bt.atom_offsets[-1]) <= 32768
    a, b = batch_system(bt), batch_system(bt)
    ta = a.batch_step(50, schedule="tile").cpu().numpy()
    tb = b.batch_step(50, schedule="box").cpu().numpy()
    (xa, va), (xb, vb) = a.get_state(), b.get_state()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    assert np.array_equal(va.cpu().numpy(), vb.cpu().numpy())
    assert np.array_equal(ta, tb)
