"""The force sums of Eq. (3) in float32 pieces: the separation exact in the
fixed point of the box (x 2^kq, kq = 60 - ex for the longest side L =
f 2^ex), s_ij times it in float32 pieces with float-float totals, the same
operations in every force kernel. A box longer than 512 A (kq = 50, a
coarser fixed point than any other test box) against the oracle, and a box
of more than 32,768 atoms (the large-system kernels) giving the same bits
alone and inside a batch (the batch kernels)."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def perturbed(nx, ny, nz, amplitude, temperature, seed):
    x, box = I.fcc_lattice(nx, I.A_CU, ny, nz)
    u = I.uniform(I.derive_seed(seed, 0), x.size).reshape(x.shape)
    x = I.wrap(x + (2.0 * u - 1.0) * amplitude, box)
    v = I.maxwell_velocities(x.shape[0], temperature, I.MASS_CU, I.derive_seed(seed, 1))
    return x, v, box


def test_long_box_beyond_512_A_matches_oracle():
    import torch
    from paper_1212_6332_gb300.md import System
    x, _, box = perturbed(170, 8, 8, 0.1, 300.0, seed=616)  # 614.6 x 28.9 x 28.9 A, 43,520 atoms
    assert box.max() > 512.0 and len(x) > 32768
    ref = O.forces(O.Potential(I.RGL_CU), x, box)
    s = System(I.RGL_CU, box=box, n_atoms=len(x), skin=0.3, mass=I.MASS_CU)
    out = s.compute_forces(torch.tensor(x, device="cuda"))
    got = {k: out[k].cpu().numpy() for k in ("f", "rho", "energy")}
    s.close()
    assert np.abs(got["f"] - ref["f"]).max() <= 1e-10 * np.abs(ref["f"]).max()
    assert np.abs(got["rho"] - ref["rho"]).max() <= 1e-12 * np.abs(ref["rho"]).max()
    assert abs(got["energy"][0] - ref["E"]) <= 1e-10 * abs(ref["E"])
    # the sums' own bias: the net force of a box is zero
    assert np.abs(got["f"].sum(axis=0)).max() < 1e-10


def test_large_box_gives_the_same_bits_alone_and_in_a_batch():
    import torch
    from paper_1212_6332_gb300.md import System
    xb, vb, bb = perturbed(20, 20, 22, 0.05, 600.0, seed=617)  # 35,200 atoms
    small = I.perturbed_fcc(4, I.A_CU, 600.0, I.MASS_CU, seed=618)
    assert len(xb) > 32768
    n_big = len(xb)
    one = System(I.RGL_CU, box=bb, n_atoms=n_big, skin=0.3, mass=I.MASS_CU)
    one.set_state(torch.tensor(xb, device="cuda"), torch.tensor(vb, device="cuda"))
    one.step(12)
    x1, v1 = (t.cpu().numpy() for t in one.get_state())
    one.close()
    boxes = np.stack([bb, small.box])
    offs = np.array([0, n_big, n_big + small.n], dtype=np.int64)
    bt = System(I.RGL_CU, boxes=boxes, atom_offsets=offs, skin=0.3, mass=I.MASS_CU)
    bt.set_state(torch.tensor(np.concatenate([xb, small.x]), device="cuda"),
                 torch.tensor(np.concatenate([vb, small.v]), device="cuda"))
    bt.batch_step(12, schedule="tile")
    x2, v2 = (t.cpu().numpy() for t in bt.get_state())
    bt.close()
    assert np.array_equal(x1, x2[:n_big]) and np.array_equal(v1, v2[:n_big])
