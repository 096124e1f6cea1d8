"""md_forces_noalloc, the entry point for callers that cannot call cudaMalloc
(plug-ins whose host application owns all device memory, latency-bound loops
that must not enter the driver's allocator). It keeps its working memory in
a fixed device array inside the library; here it is called through the C ABI
twice in a row, on two different boxes, and each result is compared with
md_compute_forces (the regular entry point) and with the CPU oracle at the
tolerance of the float64 parity tests. This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F_TOL = 1e-10
E_TOL = 1e-10


def regular(spec, bx):
    import torch
    from paper_1212_6332_gb300.md import System
    s = System(spec, box=bx.box, n_atoms=bx.n, skin=0.3, mass=I.MASS_CU)
    out = s.compute_forces(torch.tensor(bx.x, device="cuda"))
    res = {k: v.cpu().numpy() for k, v in out.items()}
    s.close()
    return res


def from_oracle(spec, bx):
    r = O.forces(O.Potential(spec), bx.x, bx.box)
    return dict(f=r["f"], e_atom=r["e_atom"], energy=np.array([r["E"]]))


def noalloc(spec, bx, x_in=None):
    """Direct C-ABI call with caller-owned device buffers."""
    import torch
    from paper_1212_6332_gb300 import md
    lib = md.load()
    x = torch.tensor(bx.x if x_in is None else x_in, device="cuda")
    f = torch.full((bx.n, 3), np.nan, dtype=torch.float64, device="cuda")
    e = torch.full((bx.n,), np.nan, dtype=torch.float64, device="cuda")
    et = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    pot, keep = md.potential_struct(spec)
    box = np.ascontiguousarray(bx.box)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.md_forces_noalloc(ctypes.byref(pot), ctypes.c_void_p(box.ctypes.data), bx.n,
                               ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                               ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(et.data_ptr()), stream)
    assert rc == 0, md.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return dict(f=f.cpu().numpy(), e_atom=e.cpu().numpy(), energy=et.cpu().numpy())


def check(got, ref):
    err = np.linalg.norm(got["f"] - ref["f"], axis=1).max() / np.linalg.norm(ref["f"], axis=1).max()
    assert err <= F_TOL, err
    assert np.allclose(got["e_atom"], ref["e_atom"], rtol=E_TOL, atol=1e-13)
    assert abs(got["energy"][0] - ref["energy"][0]) <= E_TOL * abs(ref["energy"][0])


def test_noalloc_matches_compute_forces_on_two_calls_in_a_row():
    first = I.perturbed_fcc(5, I.A_CU, 900.0, I.MASS_CU, seed=41)   # 500 atoms, RGL Cu
    second = I.perturbed_fcc(6, I.A_CU, 300.0, I.MASS_CU, seed=42)  # 864 atoms, Sutton-Chen Cu
    got1 = noalloc(I.RGL_CU, first)
    got2 = noalloc(I.SC_CU, second)
    check(got1, regular(I.RGL_CU, first))
    check(got2, regular(I.SC_CU, second))
    check(got1, from_oracle(I.RGL_CU, first))
    check(got2, from_oracle(I.SC_CU, second))
    # and back to the first box: nothing left over from the larger call
    check(noalloc(I.RGL_CU, first), regular(I.RGL_CU, first))


def test_noalloc_takes_unwrapped_positions():
    """Atoms shifted by whole box lengths (+-2L, as an MD loop that never
    wraps would leave them) give the forces of the wrapped box."""
    bx = I.perturbed_fcc(5, I.A_CU, 600.0, I.MASS_CU, seed=43)
    k = np.zeros_like(bx.x)
    k[0::3, 0], k[1::3, 1], k[2::3, 2] = 2.0, -2.0, 3.0
    k[5::7] *= -1.0
    got = noalloc(I.RGL_CU, bx, x_in=bx.x + k * bx.box)
    check(got, regular(I.RGL_CU, bx))
    check(got, from_oracle(I.RGL_CU, bx))


def test_noalloc_with_no_atoms_sets_the_energy_to_zero():
    import torch
    from paper_1212_6332_gb300 import md
    lib = md.load()
    et = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    pot, keep = md.potential_struct(I.RGL_CU)
    box = np.full(3, 30.0)
    rc = lib.md_forces_noalloc(ctypes.byref(pot), ctypes.c_void_p(box.ctypes.data), 0, None, None, None,
                               ctypes.c_void_p(et.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert et.item() == 0.0


def test_noalloc_rejects_host_memory():
    """Pointer checks run on the host before anything is enqueued."""
    import torch
    from paper_1212_6332_gb300 import md
    lib = md.load()
    bx = I.perturbed_fcc(3, I.A_CU, 300.0, I.MASS_CU, seed=44)
    x_host = np.ascontiguousarray(bx.x)
    f = torch.zeros((bx.n, 3), dtype=torch.float64, device="cuda")
    pot, keep = md.potential_struct(I.RGL_CU)
    box = np.ascontiguousarray(bx.box) * 2.0
    rc = lib.md_forces_noalloc(ctypes.byref(pot), ctypes.c_void_p(box.ctypes.data), bx.n,
                               ctypes.c_void_p(x_host.ctypes.data), ctypes.c_void_p(f.data_ptr()), None, None, None)
    assert rc == 1  # MD_ERR_ARG


def test_noalloc_rejects_more_atoms_than_its_scratch():
    import torch
    from paper_1212_6332_gb300 import md
    lib = md.load()
    n = md.NOALLOC_MAX_ATOMS + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    pot, keep = md.potential_struct(I.RGL_CU)
    box = np.full(3, 200.0)
    rc = lib.md_forces_noalloc(ctypes.byref(pot), ctypes.c_void_p(box.ctypes.data), n,
                               ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(f.data_ptr()), None, None, None)
    assert rc == 1  # MD_ERR_ARG, nothing launched
