"""CUDA path against the CPU oracle through the C ABI (float64 path).

Bars: neighbour sets bit-exact; forces max_i|dF_i| / max_i|F_i| <= 1e-10;
energies |dE|/|E| <= 1e-10; densities relative <= 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F_TOL = 1e-10
E_TOL = 1e-10
RHO_TOL = 1e-12


def torch_cuda():
    import torch
    return torch


def make_system(spec, box, n, **kw):
    from paper_1212_6332_gb300.md import System
    kw.setdefault("skin", 0.3)
    kw.setdefault("mass", I.MASS_CU)
    return System(spec, box=box, n_atoms=n, **kw)


def gpu_forces(spec, x, box, **kw):
    torch = torch_cuda()
    s = make_system(spec, box, len(x), **kw)
    out = s.compute_forces(torch.tensor(x, device="cuda"))
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["E"] = float(res.pop("energy")[0])
    return s, res


def assert_force_parity(got, ref, f_tol=F_TOL):
    fmax = np.abs(ref["f"]).max()
    err = np.linalg.norm(got["f"] - ref["f"], axis=1).max() / max(np.linalg.norm(ref["f"], axis=1).max(), 1e-300)
    assert err <= f_tol, f"force rel err {err:.3e}"
    assert abs(got["E"] - ref["E"]) <= E_TOL * abs(ref["E"]), (got["E"], ref["E"])
    assert np.allclose(got["rho"], ref["rho"], rtol=RHO_TOL, atol=0), np.abs(got["rho"] - ref["rho"]).max()
    assert np.allclose(got["e_atom"], ref["e_atom"], rtol=1e-10, atol=1e-13)
    return fmax


def oracle_sets(x, box, rl):
    pi, pj = O.pairs(x, box, rl)
    return O.full_neighbor_lists(len(x), pi, pj)


CASES = [
    ("rgl_cu_8", I.RGL_CU, I.A_CU, 8, 300.0),     # 2048 atoms, the small single-box workload
    ("rgl_cu_3", I.RGL_CU, I.A_CU, 3, 300.0),     # 2 cells per axis: de-duplicated stencil
    ("rgl_cu_4", I.RGL_CU, I.A_CU, 4, 1200.0),
    ("rgl_ni_6", I.RGL_NI, I.A_NI, 6, 600.0),
    ("sc_cu_7", I.SC_CU, I.A_CU, 7, 1200.0),      # long list (140 per atom)
]


@pytest.mark.parametrize("name,spec,a,n,T", CASES, ids=[c[0] for c in CASES])
def test_neighbour_lists_are_bit_exact(name, spec, a, n, T):
    bx = I.perturbed_fcc(n, a, T, I.MASS_CU, seed=100 + n)
    s = make_system(spec, bx.box, bx.n)
    torch = torch_cuda()
    s.set_state(torch.tensor(bx.x, device="cuda"))
    nn, nl = s.neighbors()
    nn, nl = nn.cpu().numpy(), nl.cpu().numpy()
    ref = oracle_sets(bx.x, bx.box, spec["r_cut"] + 0.3)
    for i in range(bx.n):
        got = np.sort(nl[i, :nn[i]])
        assert np.array_equal(got, ref[i]), (i, got, ref[i])


@pytest.mark.parametrize("name,spec,a,n,T", CASES, ids=[c[0] for c in CASES])
def test_forces_match_oracle(name, spec, a, n, T):
    bx = I.perturbed_fcc(n, a, T, I.MASS_CU, seed=200 + n)
    _, got = gpu_forces(spec, bx.x, bx.box)
    ref = O.forces(O.Potential(spec), bx.x, bx.box, skin=0.3)
    assert_force_parity(got, ref)


def test_spline_forces_match_oracle():
    sp = O.tabulate_spline(dict(I.RGL_CU, A=0.0855 * 1.05, p=10.96 * 0.95), n_knots=200,
                           rho_hi=2 * 20.620605425592796)
    bx = I.strained_fcc(6, I.A_CU, seed=5)
    _, got = gpu_forces(sp, bx.x, bx.box, skin=0.0)
    ref = O.forces(O.Potential(sp), bx.x, bx.box, skin=0.0)
    assert_force_parity(got, ref)


def test_perfect_lattice_and_net_force():
    x, box = I.fcc_lattice(8, I.A_CU)
    _, got = gpu_forces(I.RGL_CU, x, box)
    assert np.abs(got["f"]).max() < 1e-12
    ref_e = O.forces(O.Potential(I.RGL_CU), x, box, skin=0.3)["E"]
    assert abs(got["E"] - ref_e) <= 1e-12 * abs(ref_e)
    bx = I.perturbed_fcc(8, I.A_CU, 300.0, I.MASS_CU, seed=9)
    _, got = gpu_forces(I.RGL_CU, bx.x, bx.box)
    assert np.abs(got["f"].sum(axis=0)).max() < 1e-11


def test_ragged_box_and_sparse_gas():
    """Non-cubic box whose atom count is no multiple of 32, and a dilute gas
    with empty cells, isolated atoms (rho = 0) and a close dimer."""
    rng = np.random.default_rng(3)
    x, box = I.fcc_lattice(5, I.A_CU, 6, 7)
    x = I.wrap(x + rng.uniform(-0.05, 0.05, x.shape), box)[:-7]  # 833 atoms
    _, got = gpu_forces(I.RGL_CU, x, box)
    assert_force_parity(got, O.forces(O.Potential(I.RGL_CU), x, box, skin=0.3))
    box = np.array([40.0, 33.0, 47.0])
    x = rng.uniform(0, 1, (61, 3)) * box
    x = np.concatenate([x, [[5.0, 5.0, 5.0], [7.4, 5.0, 5.0]]])
    _, got = gpu_forces(I.RGL_CU, x, box)
    ref = O.forces(O.Potential(I.RGL_CU), x, box, skin=0.3)
    assert np.abs(got["f"] - ref["f"]).max() <= 1e-10 * np.abs(ref["f"]).max()
    assert abs(got["E"] - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert (got["rho"] == 0).sum() == (ref["rho"] == 0).sum() > 0


def test_empty_system():
    torch = torch_cuda()
    s = make_system(I.RGL_CU, [30.0, 30.0, 30.0], 0)
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    s.set_state(x)
    th = s.step(3)
    assert th["ke"] == 0.0 and th["pe"] == 0.0 and th["step"] == 3


def test_neighbour_overflow_regrows_and_stays_exact():
    bx = I.perturbed_fcc(6, I.A_CU, 300.0, I.MASS_CU, seed=77)
    s, got = gpu_forces(I.RGL_CU, bx.x, bx.box, max_neighbors=8)
    assert s.max_count() > 8
    assert_force_parity(got, O.forces(O.Potential(I.RGL_CU), bx.x, bx.box, skin=0.3))


def test_trajectory_matches_oracle_small_box():
    """The 2048-atom RGL Cu box, 200 velocity-Verlet steps at 1 fs."""
    torch = torch_cuda()
    bx = I.perturbed_fcc(8, I.A_CU, 300.0, I.MASS_CU, seed=12345)
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 200)
    for use_graph in (False, True):
        s = make_system(I.RGL_CU, bx.box, bx.n)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        out = s.step(200, history=True, use_graph=use_graph)
        x, v = (t.cpu().numpy() for t in s.get_state())
        # both sides wrap by the same rule: positions lie in [0, L) and are
        # compared as they are, with no periodic fold
        assert np.all(x >= 0.0) and np.all(x < bx.box)
        assert np.abs(x - ref["x"]).max() < 1e-9
        assert np.abs(v - ref["v"]).max() < 1e-10 * np.abs(ref["v"]).max()
        hist = out["history"].cpu().numpy()
        assert np.allclose(hist, ref["thermo"][1:], rtol=1e-10, atol=1e-10)
        assert out["step"] == 200 and out["n_rebuild"] >= 1


def test_graph_replay_gates_the_rebuild_and_matches_plain_launches():
    """Graph-replayed steps of one box skip the binning and list kernels on
    the steps that rebuild nothing (a conditional node set on the device by
    the half-skin test), and end bit for bit where plain launches end."""
    torch = torch_cuda()
    bx = I.perturbed_fcc(8, I.A_CU, 600.0, I.MASS_CU, seed=12346)
    K = 400
    res = {}
    for use_graph in (False, True):
        s = make_system(I.RGL_CU, bx.box, bx.n)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        s.profile_start()
        out = s.step(K, use_graph=use_graph)
        res[use_graph] = (out["n_rebuild"], s.profile_read()["launches"], [t.cpu().numpy() for t in s.get_state()])
        s.close()
    (nr, ln, sn), (ng, lg, sg) = res[False], res[True]
    assert nr == ng and 1 <= nr < K // 4
    assert np.array_equal(sn[0], sg[0]) and np.array_equal(sn[1], sg[1])
    # plain launches: L per step; replays: L + 1 (the gate) less the body on
    # each of the K - n_rebuild steps without a list build
    saved = ln - lg + K
    assert saved % (K - nr) == 0 and saved // (K - nr) >= 10


def test_runs_are_bitwise_deterministic():
    torch = torch_cuda()
    bx = I.perturbed_fcc(6, I.A_CU, 1200.0, I.MASS_CU, seed=4)
    res = []
    for _ in range(2):
        s = make_system(I.RGL_CU, bx.box, bx.n)
        s.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
        s.step(60)
        res.append([t.cpu().numpy() for t in s.get_state()])
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_checkpoint_resume():
    torch = torch_cuda()
    bx = I.perturbed_fcc(5, I.A_CU, 900.0, I.MASS_CU, seed=8)
    a = make_system(I.RGL_CU, bx.box, bx.n)
    a.set_state(torch.tensor(bx.x, device="cuda"), torch.tensor(bx.v, device="cuda"))
    a.step(40)
    xa, va = a.get_state()
    b = make_system(I.RGL_CU, bx.box, bx.n)
    b.set_state(xa.cpu().numpy().copy(), va.cpu().numpy().copy())  # host buffers
    a.step(40)
    b.step(40)
    (x1, v1), (x2, v2) = a.get_state(), b.get_state()
    assert torch.allclose(x1, x2, rtol=0, atol=1e-11) and torch.allclose(v1, v2, rtol=0, atol=1e-12)


def test_host_and_device_buffers_agree():
    torch = torch_cuda()
    bx = I.perturbed_fcc(4, I.A_CU, 300.0, I.MASS_CU, seed=6)
    s = make_system(I.RGL_CU, bx.box, bx.n)
    dev = s.compute_forces(torch.tensor(bx.x, device="cuda"))
    f_host = np.zeros((bx.n, 3))
    e_host = np.zeros(1)
    s.compute_forces(bx.x.copy(), f=f_host, energy=e_host)
    assert np.array_equal(f_host, dev["f"].cpu().numpy())
    assert e_host[0] == dev["energy"].item()


def test_non_finite_inputs_are_reported():
    """Failure injected on the host: a NaN position or an infinite velocity
    makes set_state return MD_ERR_NONFINITE; the handle stays usable."""
    from paper_1212_6332_gb300.md import MDError
    bx = I.perturbed_fcc(4, I.A_CU, 300.0, I.MASS_CU, seed=6)
    s = make_system(I.RGL_CU, bx.box, bx.n)
    x = bx.x.copy()
    x[17, 1] = np.nan
    with pytest.raises(MDError) as err:
        s.set_state(x, bx.v.copy())
    assert err.value.code == 5
    v = bx.v.copy()
    v[3, 0] = np.inf
    with pytest.raises(MDError) as err:
        s.set_state(bx.x.copy(), v)
    assert err.value.code == 5
    s.set_state(bx.x.copy(), bx.v.copy())
    assert s.step(5)["step"] == 5
