"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a closed form, a literature value, an
independent library routine (scipy), brute force, a physical invariant, or
a finite difference, chosen so that a dropped term, a wrong sign or index,
or a wrong convention in the oracle fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I


def fcc_shells(a, rmax):
    """Distances of all fcc lattice sites within rmax of the origin, by
    enumerating conventional cells (independent of any neighbour search)."""
    n = int(rmax / a) + 2
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    out = []
    for i, j, k in itertools.product(range(-n, n + 1), repeat=3):
        p = (np.array([i, j, k]) + basis) * a
        r = np.linalg.norm(p, axis=1)
        out.append(r[(r > 0) & (r < rmax)])
    return np.concatenate(out)


def smoothstep(r, rs, rc):
    x = np.clip((r - rs) / (rc - rs), 0.0, 1.0)
    return np.where(r < rc, 1 - 10 * x ** 3 + 15 * x ** 4 - 6 * x ** 5, 0.0)


def rgl_lattice_energy(spec, a):
    """Cohesive energy per atom of the perfect fcc lattice as a shell sum:
    E = -sqrt(sum_s rho(r_s)) + 1/2 sum_s V(r_s)."""
    r = fcc_shells(a, spec["r_cut"])
    S = smoothstep(r, spec["r_taper"], spec["r_cut"])
    V = 2 * spec["A"] * np.exp(-spec["p"] * (r / spec["r0"] - 1)) * S
    rho = spec["xi"] ** 2 * np.exp(-2 * spec["q"] * (r / spec["r0"] - 1)) * S
    return -np.sqrt(rho.sum()) + 0.5 * V.sum(), rho.sum()


def sc_lattice_energy(spec, a):
    r = fcc_shells(a, spec["r_cut"])
    S = smoothstep(r, spec["r_taper"], spec["r_cut"])
    V = spec["eps"] * (spec["a"] / r) ** spec["n"] * S
    rho = (spec["a"] / r) ** spec["m"] * S
    return -spec["c"] * spec["eps"] * np.sqrt(rho.sum()) + 0.5 * V.sum(), rho.sum()


# ---------------------------------------------------------------- lists

@pytest.mark.parametrize("n,spec,skin", [(3, I.RGL_CU, 0.3), (4, I.RGL_CU, 0.3), (5, I.RGL_CU, 0.3),
                                         (6, I.RGL_CU, 0.3), (7, I.SC_CU, 0.3)])
def test_linked_cells_equal_brute_force(n, spec, skin):
    bx = I.perturbed_fcc(n, I.A_CU, 300.0, I.MASS_CU, seed=7 + n)
    rl = spec["r_cut"] + skin
    a = O.pairs(bx.x, bx.box, rl, "cells")
    b = O.pairs(bx.x, bx.box, rl, "brute")
    sa = set(zip(a[0].tolist(), a[1].tolist()))
    sb = set(zip(b[0].tolist(), b[1].tolist()))
    assert sa == sb and len(sa) == len(a[0])
    assert all(i < j for i, j in sa)


def test_pairs_match_scipy_periodic_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    bx = I.perturbed_fcc(6, I.A_CU, 300.0, I.MASS_CU, seed=99)
    rl = 5.3
    pi, pj = O.pairs(bx.x, bx.box, rl)
    tree = spatial.cKDTree(bx.x, boxsize=bx.box)
    ref = tree.query_pairs(rl, output_type="ndarray")
    ref = set(map(tuple, np.sort(ref, axis=1).tolist()))
    assert set(zip(pi.tolist(), pj.tolist())) == ref


@pytest.mark.parametrize("spec,a,rc_count,rl_count", [(I.RGL_CU, I.A_CU, 42, 54), (I.SC_CU, I.A_CU, 134, 140),
                                                      (I.RGL_NI, I.A_NI, 42, 54)])
def test_neighbour_counts_on_perfect_lattice(spec, a, rc_count, rl_count):
    n = 6 if spec is not I.SC_CU else 7
    x, box = I.fcc_lattice(n, a)
    lists = O.full_neighbor_lists(len(x), *O.pairs(x, box, spec["r_cut"] + 0.3))
    counts = np.array([len(l) for l in lists])
    assert (counts == rl_count).all()
    inner = O.full_neighbor_lists(len(x), *O.pairs(x, box, spec["r_cut"]))
    assert all(len(l) == rc_count for l in inner)
    assert rc_count == len(fcc_shells(a, spec["r_cut"]))


# ---------------------------------------------------------------- energies

@pytest.mark.parametrize("scale", [1.0, 0.98, 1.02])
def test_rgl_cu_lattice_shell_sum(scale):
    a = I.A_CU * scale
    x, box = I.fcc_lattice(6, a)
    r = O.forces(O.Potential(I.RGL_CU), x, box, skin=0.3)
    e_ref, rho_ref = rgl_lattice_energy(I.RGL_CU, a)
    assert r["E"] / len(x) == pytest.approx(e_ref, rel=1e-13)
    assert np.allclose(r["rho"], rho_ref, rtol=1e-13)
    assert np.allclose(r["e_atom"], e_ref, rtol=1e-13)


def test_rgl_ni_lattice_shell_sum():
    x, box = I.fcc_lattice(6, I.A_NI)
    r = O.forces(O.Potential(I.RGL_NI), x, box, skin=0.3)
    assert r["E"] / len(x) == pytest.approx(rgl_lattice_energy(I.RGL_NI, I.A_NI)[0], rel=1e-13)


def test_sutton_chen_lattice_shell_sum():
    x, box = I.fcc_lattice(7, I.A_CU)
    r = O.forces(O.Potential(I.SC_CU), x, box, skin=0.3)
    assert r["E"] / len(x) == pytest.approx(sc_lattice_energy(I.SC_CU, I.A_CU)[0], rel=1e-13)


def test_rgl_cu_literature_cohesive_energy():
    """Cleri and Rosato (Phys. Rev. B 48, 22 (1993)) fitted these Cu
    parameters with interactions out to the fifth neighbour shell to the
    cohesive energy 3.544 eV/atom. A hard cut between the 5th (5.72 A) and
    6th (6.26 A) shells reproduces it; the taper is switched off by
    r_taper = r_cut."""
    spec = dict(I.RGL_CU, r_taper=6.0, r_cut=6.0)
    x, box = I.fcc_lattice(8, I.A_CU)
    r = O.forces(O.Potential(spec), x, box, skin=0.0)
    assert r["E"] / len(x) == pytest.approx(-3.544, abs=2e-3)


def test_dimer_closed_form():
    """Two atoms: rho_1 = rho_2 = rho(r), E = V(r) + 2 F(rho(r)),
    |F| = dE/dr (by a central difference of the closed form)."""
    pot = O.Potential(I.RGL_CU)
    box = np.array([40.0, 40.0, 40.0])
    for r in (2.2, 3.0, 4.7):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        out = O.forces(pot, x, box, method="brute")
        e = lambda s: 2 * I.RGL_CU["A"] * np.exp(-I.RGL_CU["p"] * (s / I.RGL_CU["r0"] - 1)) * smoothstep(s, 4.5, 5.0) \
            - 2 * np.sqrt(I.RGL_CU["xi"] ** 2 * np.exp(-2 * I.RGL_CU["q"] * (s / I.RGL_CU["r0"] - 1))
                          * smoothstep(s, 4.5, 5.0))
        assert out["E"] == pytest.approx(float(e(r)), rel=1e-13)
        h = 1e-6
        dEdr = (e(r + h) - e(r - h)) / (2 * h)
        # atom 1 sits at larger x: F_1x = -dE/dr, F_0x = +dE/dr
        assert out["f"][1, 0] == pytest.approx(-dEdr, rel=1e-7, abs=1e-10)
        assert out["f"][0, 0] == pytest.approx(dEdr, rel=1e-7, abs=1e-10)
        assert np.abs(out["f"][:, 1:]).max() == 0.0
    far = np.array([[1.0, 1.0, 1.0], [20.0, 1.0, 1.0]])
    out = O.forces(pot, far, box, method="brute")
    assert out["E"] == 0.0 and np.abs(out["f"]).max() == 0.0


# ---------------------------------------------------------------- forces

@pytest.mark.parametrize("spec,a,n", [(I.RGL_CU, I.A_CU, 5), (I.SC_CU, I.A_CU, 7), (I.RGL_NI, I.A_NI, 5)])
def test_perfect_lattice_has_zero_force(spec, a, n):
    x, box = I.fcc_lattice(n, a)
    r = O.forces(O.Potential(spec), x, box, skin=0.3)
    assert np.abs(r["f"]).max() < 1e-12


@pytest.mark.parametrize("spec", [I.RGL_CU, I.SC_CU])
def test_half_list_equals_double_sums(spec):
    bx = I.perturbed_fcc(5 if spec is I.RGL_CU else 7, I.A_CU, 300.0, I.MASS_CU, seed=3)
    pot = O.Potential(spec)
    a = O.forces(pot, bx.x, bx.box, skin=0.3)
    b = O.forces(pot, bx.x, bx.box, method="brute")
    assert a["E"] == pytest.approx(b["E"], rel=1e-13)
    assert np.allclose(a["rho"], b["rho"], rtol=1e-13)
    assert np.allclose(a["e_atom"], b["e_atom"], rtol=1e-12, atol=1e-13)
    assert np.abs(a["f"] - b["f"]).max() <= 1e-12 * np.abs(b["f"]).max()


def test_net_force_vanishes():
    bx = I.perturbed_fcc(5, I.A_CU, 300.0, I.MASS_CU, seed=11)
    r = O.forces(O.Potential(I.RGL_CU), bx.x, bx.box, skin=0.3, method="brute")
    assert np.abs(r["f"].sum(axis=0)).max() < 1e-12


def test_translation_and_permutation_invariance():
    bx = I.perturbed_fcc(5, I.A_CU, 300.0, I.MASS_CU, seed=5)
    pot = O.Potential(I.RGL_CU)
    a = O.forces(pot, bx.x, bx.box, skin=0.3)
    shifted = I.wrap(bx.x + np.array([1.234, -0.77, 5.5]), bx.box)
    b = O.forces(pot, shifted, bx.box, skin=0.3)
    assert b["E"] == pytest.approx(a["E"], rel=1e-12)
    assert np.abs(a["f"] - b["f"]).max() < 1e-11
    perm = np.random.default_rng(0).permutation(len(bx.x))
    c = O.forces(pot, bx.x[perm], bx.box, skin=0.3)
    assert c["E"] == pytest.approx(a["E"], rel=1e-13)
    assert np.abs(c["f"] - a["f"][perm]).max() < 1e-12


@pytest.mark.parametrize("spec", [I.RGL_CU, I.SC_CU])
def test_forces_are_minus_energy_gradient(spec):
    """Central differences of E_T against the force of Eq. (3)."""
    bx = I.perturbed_fcc(5 if spec is I.RGL_CU else 7, I.A_CU, 300.0, I.MASS_CU, seed=21)
    pot = O.Potential(spec)
    f = O.forces(pot, bx.x, bx.box, skin=0.3)["f"]
    h = 1e-5
    rng = np.random.default_rng(1)
    for i in rng.choice(len(bx.x), 6, replace=False):
        for a in range(3):
            xp, xm = bx.x.copy(), bx.x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            ep = O.forces(pot, xp, bx.box, skin=0.3)["E"]
            em = O.forces(pot, xm, bx.box, skin=0.3)["E"]
            assert -(ep - em) / (2 * h) == pytest.approx(f[i, a], abs=2e-7 * max(1.0, abs(f[i, a])))


# ---------------------------------------------------------------- functions

def test_taper_and_pair_derivatives():
    pot = O.Potential(I.RGL_CU)
    r = np.linspace(2.0, 4.999, 301)
    V, dV, rho, drho = pot.pair(r)
    h = 1e-6
    Vp, _, rp, _ = pot.pair(r + h)
    Vm, _, rm, _ = pot.pair(r - h)
    assert np.allclose(dV, (Vp - Vm) / (2 * h), rtol=1e-7, atol=1e-9)
    assert np.allclose(drho, (rp - rm) / (2 * h), rtol=1e-7, atol=1e-9)
    # taper: value and slope continuous at r_taper, zero at and beyond r_cut
    lo = pot.pair(np.array([4.5 - 1e-9, 4.5 + 1e-9]))
    assert abs(lo[0][0] - lo[0][1]) < 1e-9 and abs(lo[1][0] - lo[1][1]) < 1e-8
    hi = pot.pair(np.array([5.0 - 1e-4, 5.0, 5.2]))
    assert abs(hi[0][0]) < 1e-10 and abs(hi[1][0]) < 1e-6
    assert (hi[0][1:] == 0).all() and (hi[1][1:] == 0).all() and (hi[2][1:] == 0).all()
    F, Fp, Fpp = pot.embed(np.array([0.0, 4.0, 20.0]))
    assert F[0] == 0 and Fp[0] == 0
    assert F[1] == pytest.approx(-2.0) and Fp[1] == pytest.approx(-0.25) and Fpp[1] == pytest.approx(1 / 32)


def test_natural_spline_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(3)
    n = 23
    spec = dict(kind="spline", phi=rng.normal(size=n), f=rng.normal(size=n), F=rng.normal(size=n),
                r_lo=1.5, r_hi=5.0, rho_lo=0.0, rho_hi=40.0)
    pot = O.Potential(spec)
    t = np.linspace(1.5, 5.0, n)
    cs = interp.CubicSpline(t, spec["phi"], bc_type="natural")
    r = np.linspace(1.5, 4.999, 777)
    V, dV, rho, drho = pot.pair(r)
    assert np.allclose(V, cs(r), atol=1e-12) and np.allclose(dV, cs(r, 1), atol=1e-11)
    cf = interp.CubicSpline(t, spec["f"], bc_type="natural")
    assert np.allclose(rho, cf(r), atol=1e-12)
    tF = np.linspace(0.0, 40.0, n)
    cF = interp.CubicSpline(tF, spec["F"], bc_type="natural")
    g = np.linspace(0.0, 40.0, 501)
    F, Fp, Fpp = pot.embed(g)
    assert np.allclose(F, cF(g), atol=1e-12) and np.allclose(Fp, cF(g, 1), atol=1e-11)
    assert np.allclose(Fpp, cF(g, 2), atol=1e-10)
    # linear extrapolation beyond the F range, zero beyond r_hi
    Fo, Fpo, _ = pot.embed(np.array([45.0]))
    assert Fo[0] == pytest.approx(cF(40.0) + 5.0 * cF(40.0, 1)) and Fpo[0] == pytest.approx(cF(40.0, 1))
    assert pot.pair(np.array([5.0, 6.0]))[0].tolist() == [0.0, 0.0]


# ---------------------------------------------------------------- dynamics

def test_nve_energy_drift_bounded():
    bx = I.perturbed_fcc(4, I.A_CU, 300.0, I.MASS_CU, seed=12345)
    out = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 200)
    et = out["thermo"][:, 2]
    n = len(bx.x)
    assert np.abs(et - et[0]).max() / n < 2e-5
    slope = np.polyfit(np.arange(len(et)), et / n, 1)[0]
    assert abs(slope) < 2e-8  # eV/atom per fs
    assert out["n_rebuild"] >= 1
    # the initial temperature is the fixture's exact 300 K
    assert out["thermo"][0, 3] == pytest.approx(300.0, rel=1e-12)


def test_time_reversibility():
    bx = I.perturbed_fcc(4, I.A_CU, 600.0, I.MASS_CU, seed=4)
    pot = O.Potential(I.RGL_CU)
    fwd = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 50)
    back = O.md_run(pot, fwd["x"], -fwd["v"], bx.box, I.MASS_CU, 1.0, 0.3, 50)
    d = back["x"] - bx.x
    d -= bx.box * np.round(d / bx.box)
    assert np.abs(d).max() < 1e-9
    assert np.abs(back["v"] + bx.v).max() < 1e-10


def exact_residue(x, L):
    """x mod L in exact rational arithmetic, in [0, L)."""
    from fractions import Fraction
    import math
    fx, fL = Fraction(float(x)), Fraction(float(L))
    return fx - fL * math.floor(fx / fL)


@pytest.mark.parametrize("L", [3.615, 28.92, 361.5, 281.84])
def test_wrap_rule_special_values(L):
    """Periodic wrap of Sec. 3.2 into [0, L): named values, including the case
    where x - L*floor(x/L) rounds to L (x = -1e-17) and must become 0."""
    ulp_below_L = np.nextafter(L, 0.0)
    cases = {-L: 0.0, -1e-17: 0.0, -np.nextafter(0.0, 1.0): 0.0, 0.0: 0.0, ulp_below_L: ulp_below_L, L: 0.0,
             2 * L: 0.0, 1.25: 1.25 if 1.25 < L else None}
    for x, want in cases.items():
        if want is None:
            continue
        got = O.wrap(np.array([[x, x, x]]), np.array([L, L, L]))[0]
        assert got.tolist() == [want] * 3, (x, got)
    delta = 0.3125
    got = O.wrap(np.array([[2 * L + delta] * 3]), np.array([L] * 3))[0, 0]
    assert got == pytest.approx(delta, abs=4 * np.spacing(2 * L)) and 0.0 <= got < L


@pytest.mark.parametrize("L", [3.615, 28.92, 361.5, 281.84, 10.845, 0.1, 7.0])
def test_wrap_lands_in_the_box_next_to_every_multiple(L):
    """Coordinates a few ulp either side of k*L, |k| <= 150, land in [0, L) and
    equal the exact residue x mod L (rational arithmetic) to a few ulp, or
    its image across the boundary. Without the fold of negative results,
    x just below k*L (|k| >= 2) wraps to about -1e-14."""
    xs = []
    for k in range(-150, 151):
        c = k * L
        lo = hi = c
        xs.append(c)
        for _ in range(3):
            lo, hi = np.nextafter(lo, -np.inf), np.nextafter(hi, np.inf)
            xs += [lo, hi]
    xs = np.array(xs)
    got = O.wrap(np.repeat(xs[:, None], 3, axis=1), np.array([L, L, L]))[:, 0]
    assert np.all(got >= 0.0) and np.all(got < L)
    for x, y in zip(xs, got):
        r = float(exact_residue(x, L))
        tol = 4 * np.spacing(max(abs(x), L))
        assert min(abs(y - r), abs(y - r + L), abs(y - r - L)) <= tol, (x, y, r)


def test_trajectory_positions_stay_in_the_box():
    """Every position that velocity Verlet returns lies in [0, L), also from
    a start given far outside the box (unwrapped by several box lengths)."""
    bx = I.perturbed_fcc(4, I.A_CU, 1200.0, I.MASS_CU, seed=31)
    shift = np.array([-3.0, 2.0, 7.0]) * bx.box
    x0 = bx.x + shift[None, :] * (np.arange(len(bx.x)) % 2)[:, None]
    out = O.md_run(O.Potential(I.RGL_CU), x0, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30)
    assert np.all(out["x"] >= 0.0) and np.all(out["x"] < bx.box)
    ref = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30)
    d = out["x"] - ref["x"]
    d -= bx.box * np.round(d / bx.box)
    assert np.abs(d).max() < 1e-9


def gas(n_side=4, spacing=6.5, temperature=600.0, seed=21):
    """Atoms on a simple cubic grid farther apart than r_cut + skin: no
    forces act, only the friction of Eq. (4)."""
    g = np.arange(n_side) * spacing + 1.0
    x = np.array(list(itertools.product(g, g, g)), dtype=float)
    box = np.full(3, n_side * spacing)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=x.shape) * np.sqrt(I.KB_EV_PER_K * temperature / (I.MASS_CU * I.MVV_EV))
    return x, v, box


def atom_temperatures(v):
    return I.MASS_CU * I.MVV_EV * np.sum(v * v, axis=1) / (3.0 * I.KB_EV_PER_K)


def test_friction_free_atoms_follow_the_closed_form():
    """With no forces, Eq. (4) reads dv/dt = -(1/tau)(1 - T_e/T_i) v, so each
    atom keeps its direction and its temperature T_i = m v^2 / (3 k_B) obeys
    dT_i/dt = -(2/tau)(T_i - T_e): T_i(t) = T_e + (T_i(0) - T_e) exp(-2t/tau)."""
    x, v, box = gas()
    tau, T_e, dt, n = 40.0, 300.0, 1.0, 60
    out = O.md_run(O.Potential(I.RGL_CU), x, v, box, I.MASS_CU, dt, 0.3, n, tau_T=tau, T_e=T_e)
    T0, T1 = atom_temperatures(v), atom_temperatures(out["v"])
    expect = T_e + (T0 - T_e) * np.exp(-2.0 * n * dt / tau)
    assert np.allclose(T1, expect, rtol=1e-12, atol=0)
    cos = np.sum(out["v"] * v, axis=1) / np.linalg.norm(out["v"], axis=1) / np.linalg.norm(v, axis=1)
    assert np.allclose(cos, 1.0, rtol=0, atol=1e-14)
    # positions advance with the velocities (no forces): ballistic drift
    assert out["thermo"][:, 1].max() == 0.0


def test_friction_without_coupling_is_plain_verlet():
    bx = I.perturbed_fcc(3, I.A_CU, 600.0, I.MASS_CU, seed=8)
    pot = O.Potential(I.RGL_CU)
    a = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30)
    b = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30, tau_T=0.0, T_e=1000.0)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])


def test_friction_brings_a_hot_crystal_to_the_electron_temperature():
    """A 900 K crystal coupled to a 300 K electron bath (tau = 50 fs) cools
    to 300 K: the kinetic temperature, averaged over the last 300 of 1500
    steps, is within 5% of T_e, and the energy it lost went to the bath."""
    bx = I.perturbed_fcc(4, I.A_CU, 900.0, I.MASS_CU, seed=13)
    out = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 1500, tau_T=50.0, T_e=300.0)
    T = out["thermo"][:, 3]
    assert T[-300:].mean() == pytest.approx(300.0, rel=0.05)
    assert out["thermo"][-1, 2] < out["thermo"][0, 2]


# ---------------------------------------------------------------- pressure (Eq. 5-6)

@pytest.mark.parametrize("case", ["rgl_cu", "rgl_ni", "sc_cu", "spline"])
def test_virial_is_minus_the_volume_derivative(case):
    """For a static configuration the interaction part of Eq. (6), W/(3V),
    is -dE/dV: scaling every coordinate and the box by lambda changes V by
    lambda^3, and dE/dlambda at 1 is -W."""
    spec, a, n = {"rgl_cu": (I.RGL_CU, I.A_CU, 4), "rgl_ni": (I.RGL_NI, I.A_NI, 4),
                  "sc_cu": (I.SC_CU, I.A_CU, 5), "spline": (None, I.A_CU, 4)}[case]
    if spec is None:
        spec = O.tabulate_spline(dict(I.RGL_CU, A=0.0855 * 1.05), n_knots=120, rho_hi=41.2)
    bx = I.perturbed_fcc(n, a, 300.0, I.MASS_CU, seed=17)
    pot = O.Potential(spec)
    V = np.prod(bx.box)
    W = O.virial(pot, bx.x, bx.box)
    h = 1e-5
    E = [O.forces(pot, bx.x * lam, bx.box * lam)["E"] for lam in (1 + h, 1 - h)]
    dEdV = (E[0] - E[1]) / (2 * h) / (3 * V)
    assert W / (3 * V) == pytest.approx(-dEdV, rel=1e-6)


def test_pressure_of_free_atoms_is_the_ideal_gas_law():
    x, v, box = gas()
    out = O.md_run(O.Potential(I.RGL_CU), x, v, box, I.MASS_CU, 1.0, 0.3, 0, want_pressure=True)
    n = len(x)
    T = out["thermo"][0, 3]
    assert out["pressure"][0] == pytest.approx(n * I.KB_EV_PER_K * T / np.prod(box), rel=1e-14)


def test_barostat_drives_the_pressure_to_its_target():
    """A Cu crystal at the fcc lattice constant is under ~2 GPa at 300 K
    with this potential; the coupling of Eq. (5) (P0 = 0, beta = 1/140 GPa,
    tau_p = 100 fs) expands the box until the mean pressure over the last
    1000 of 3000 steps is zero within 1e-4 eV/A^3 (16 MPa)."""
    bx = I.perturbed_fcc(4, I.A_CU, 300.0, I.MASS_CU, seed=1)
    beta = 160.21766208 / 140.0
    out = O.md_run(O.Potential(I.RGL_CU), bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 3000, tau_p=100.0, P0=0.0,
                   beta=beta)
    P = out["pressure"]
    assert P[0] > 0.01
    assert abs(P[-1000:].mean()) < 1e-4
    assert out["box"][0] > bx.box[0] * 1.004 and np.allclose(out["box"], out["box"][0])


def test_barostat_off_is_plain_verlet():
    bx = I.perturbed_fcc(3, I.A_CU, 600.0, I.MASS_CU, seed=8)
    pot = O.Potential(I.RGL_CU)
    a = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30)
    b = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 30, tau_p=0.0, P0=1.0, beta=1.0)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
    assert np.array_equal(b["box"], bx.box)


# ---------------------------------------------------------------- several species (Eq. 1-3 with types)

RGL_CUNI = dict(kind="rgl", A=0.5 * (0.0855 + 0.0376), xi=np.sqrt(1.224 * 1.070), p=0.5 * (10.960 + 16.999),
                q=0.5 * (2.278 + 1.189), r0=0.5 * (2.5562 + 2.4911), r_taper=4.5, r_cut=5.0)


def cuni_alloy(n_knots=150, rho_hi=45.0):
    """Binary alloy tables: RGL Cu for (0, 0), RGL Ni (with the Cu taper) for
    (1, 1), parameter means for (0, 1); F = -sqrt(rho) for both types."""
    ni = dict(I.RGL_NI, r_taper=4.5, r_cut=5.0)
    tabs = [O.tabulate_spline(sp, n_knots=n_knots, rho_hi=rho_hi) for sp in (I.RGL_CU, RGL_CUNI, ni)]
    return dict(kind="alloy", n_types=2, phi=[t["phi"] for t in tabs], f=[t["f"] for t in tabs],
                F=[tabs[0]["F"], tabs[2]["F"] * 0.9], r_lo=tabs[0]["r_lo"], r_hi=tabs[0]["r_hi"],
                rho_lo=0.0, rho_hi=rho_hi)


def alloy_box(seed=4):
    bx = I.perturbed_fcc(4, 3.57, 300.0, I.MASS_CU, seed=seed)
    types = np.random.default_rng(seed).integers(0, 2, bx.n)
    return bx, types


def test_alloy_with_identical_tables_equals_one_species():
    sp = O.tabulate_spline(I.RGL_CU, n_knots=100, rho_hi=41.2)
    al = dict(kind="alloy", n_types=3, phi=[sp["phi"]] * 6, f=[sp["f"]] * 6, F=[sp["F"]] * 3, r_lo=sp["r_lo"],
              r_hi=sp["r_hi"], rho_lo=sp["rho_lo"], rho_hi=sp["rho_hi"])
    bx = I.perturbed_fcc(4, I.A_CU, 300.0, I.MASS_CU, seed=1)
    one = O.forces(O.Potential(sp), bx.x, bx.box)
    many = O.forces(O.Potential(al), bx.x, bx.box, types=np.arange(bx.n) % 3)
    assert one["E"] == many["E"] and np.array_equal(one["f"], many["f"])


def test_alloy_half_list_equals_double_sums():
    bx, t = alloy_box()
    pot = O.Potential(cuni_alloy())
    a = O.forces(pot, bx.x, bx.box, types=t)
    b = O.forces(pot, bx.x, bx.box, method="brute", types=t)
    assert a["E"] == pytest.approx(b["E"], rel=1e-13)
    assert np.abs(a["f"] - b["f"]).max() < 1e-12
    assert np.allclose(a["rho"], b["rho"], rtol=1e-13)


def test_alloy_forces_are_minus_energy_gradient():
    bx, t = alloy_box(seed=6)
    pot = O.Potential(cuni_alloy())
    f = O.forces(pot, bx.x, bx.box, types=t)["f"]
    h = 1e-4  # central differences: O(h^2) truncation, roundoff of E ~ 1e3 eV
    for i, a in [(0, 0), (17, 1), (100, 2), (255, 0)]:
        xp, xm = bx.x.copy(), bx.x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = -(O.forces(pot, xp, bx.box, types=t)["E"] - O.forces(pot, xm, bx.box, types=t)["E"]) / (2 * h)
        assert f[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_alloy_dimer_closed_form():
    """An isolated a-b pair: E = V^(ab)(r) + F_a(rho^(ab)(r)) + F_b(rho^(ab)(r))
    and the force on each atom is -dE/dr along the bond, with every table
    taken as scipy's natural cubic spline of the same knots."""
    import scipy.interpolate as interp
    al = cuni_alloy()
    pot = O.Potential(al)
    t = np.linspace(al["r_lo"], al["r_hi"], len(al["phi"][0]))
    tF = np.linspace(al["rho_lo"], al["rho_hi"], len(al["F"][0]))
    V = interp.CubicSpline(t, al["phi"][1], bc_type="natural")
    R = interp.CubicSpline(t, al["f"][1], bc_type="natural")
    Fa = interp.CubicSpline(tF, al["F"][0], bc_type="natural")
    Fb = interp.CubicSpline(tF, al["F"][1], bc_type="natural")
    box = np.array([30.0, 30.0, 30.0])
    for r in (2.3, 2.7, 3.4, 4.7):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        out = O.forces(pot, x, box, types=np.array([0, 1]))
        rho = R(r)
        E = V(r) + Fa(rho) + Fb(rho)
        dE = V(r, 1) + (Fa(rho, 1) + Fb(rho, 1)) * R(r, 1)
        assert out["E"] == pytest.approx(E, rel=1e-12)
        assert out["f"][1, 0] == pytest.approx(-dE, rel=1e-10, abs=1e-12)
        assert out["f"][0, 0] == pytest.approx(dE, rel=1e-10, abs=1e-12)


def test_alloy_relabelling_species_changes_nothing():
    bx, t = alloy_box(seed=9)
    al = cuni_alloy()
    sw = dict(al, phi=al["phi"][::-1], f=al["f"][::-1], F=al["F"][::-1])
    a = O.forces(O.Potential(al), bx.x, bx.box, types=t)
    b = O.forces(O.Potential(sw), bx.x, bx.box, types=1 - t)
    assert a["E"] == pytest.approx(b["E"], rel=1e-14)
    assert np.abs(a["f"] - b["f"]).max() < 1e-13


def test_alloy_knot_derivatives_match_finite_differences():
    """Forward-mode derivatives of E_T and of the forces with respect to
    knot values of every kind of table (V pair, rho pair, F type) equal
    central differences of the oracle's own energy and forces."""
    al = cuni_alloy(n_knots=40)
    bx, t = alloy_box()
    pot = O.Potential(al)
    knots = pot._knots
    nr, P = len(al["phi"][0]), 3

    def spec_with(k2):
        return dict(al, phi=[k2[i * nr:(i + 1) * nr] for i in range(P)],
                    f=[k2[(P + i) * nr:(P + i + 1) * nr] for i in range(P)],
                    F=[k2[2 * P * nr + i * nr:2 * P * nr + (i + 1) * nr] for i in range(2)])

    h = 1e-6
    for which in (5, 45, 85, 130, 205):
        dE, dF = O.param_deriv(pot, which, bx.x, bx.box, types=t)
        kp, km = knots.copy(), knots.copy()
        kp[which] += h
        km[which] -= h
        op = O.forces(O.Potential(spec_with(kp)), bx.x, bx.box, types=t)
        om = O.forces(O.Potential(spec_with(km)), bx.x, bx.box, types=t)
        assert dE == pytest.approx((op["E"] - om["E"]) / (2 * h), rel=1e-5, abs=1e-6)
        assert np.abs(dF - (op["f"] - om["f"]) / (2 * h)).max() < 1e-5


def test_dimer_small_oscillation_period():
    """A dimer near its bond length oscillates at omega = sqrt(k/mu), with
    k = E''(r_eq) of the closed-form dimer energy and mu = m/2."""
    pot = O.Potential(I.RGL_CU)
    box = np.array([40.0, 40.0, 40.0])

    def energy(r):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        return O.forces(pot, x, box, method="brute")["E"]

    rs = np.linspace(2.0, 2.6, 6001)
    req = rs[np.argmin([energy(r) for r in rs])]
    h = 1e-4
    k = (energy(req + h) - 2 * energy(req) + energy(req - h)) / h ** 2
    mu = I.MASS_CU / 2 * I.MVV_EV
    period = 2 * np.pi / np.sqrt(k / mu)
    x0 = np.array([[10.0, 10.0, 10.0], [10.0 + req + 0.002, 10.0, 10.0]])
    n_steps = int(3 * period)
    out = O.md_run(pot, x0, np.zeros((2, 3)), box, I.MASS_CU, 0.5, 0.3, 2 * n_steps)
    # sample the bond length by re-running step by step
    xs = [x0]
    x, v = x0, np.zeros((2, 3))
    for _ in range(2 * n_steps):
        o = O.md_run(pot, x, v, box, I.MASS_CU, 0.5, 0.3, 1)
        x, v = o["x"], o["v"]
        xs.append(x)
    b = np.array([xx[1, 0] - xx[0, 0] for xx in xs]) - req
    crossings = np.where(np.diff(np.sign(b)) != 0)[0]
    measured = 2 * 0.5 * np.mean(np.diff(crossings))
    assert measured == pytest.approx(period, rel=0.02)
    assert out["thermo"][:, 2].std() < 1e-6


# ---------------------------------------------------------------- gradients

def loss_of(pot, configs, targets):
    L = 0.0
    for (x, box), (ft, et) in zip(configs, targets):
        r = O.forces(pot, x, box)
        n = len(x)
        L += np.mean((r["f"] - ft) ** 2) + 0.1 * (r["E"] / n - et / n) ** 2
    return L / len(configs)


def test_rgl_param_derivatives_match_finite_differences():
    bx = I.strained_fcc(3, I.A_CU, seed=8)
    pot = O.Potential(I.RGL_CU)
    for k, name in enumerate(O.RGL_ORDER):
        dE, dF = O.param_deriv(pot, k, bx.x, bx.box)
        h = 1e-6 * abs(I.RGL_CU[name])
        rp = O.forces(O.Potential(dict(I.RGL_CU, **{name: I.RGL_CU[name] + h})), bx.x, bx.box)
        rm = O.forces(O.Potential(dict(I.RGL_CU, **{name: I.RGL_CU[name] - h})), bx.x, bx.box)
        assert dE == pytest.approx((rp["E"] - rm["E"]) / (2 * h), rel=1e-6)
        fd = (rp["f"] - rm["f"]) / (2 * h)
        assert np.abs(dF - fd).max() <= 1e-6 * np.abs(fd).max()


def test_sutton_chen_param_derivatives_match_finite_differences():
    """Forward-mode derivatives for Sutton-Chen (eps, c, a, n, m), including
    the c*eps factor of its embedding, against central differences."""
    bx = I.strained_fcc(5, I.A_CU, seed=9)
    pot = O.Potential(I.SC_CU)
    for k, name in enumerate(O.SC_ORDER):
        dE, dF = O.param_deriv(pot, k, bx.x, bx.box)
        h = 1e-6 * abs(I.SC_CU[name])
        rp = O.forces(O.Potential(dict(I.SC_CU, **{name: I.SC_CU[name] + h})), bx.x, bx.box)
        rm = O.forces(O.Potential(dict(I.SC_CU, **{name: I.SC_CU[name] - h})), bx.x, bx.box)
        assert dE == pytest.approx((rp["E"] - rm["E"]) / (2 * h), rel=1e-6), name
        fd = (rp["f"] - rm["f"]) / (2 * h)
        assert np.abs(dF - fd).max() <= 1e-6 * np.abs(fd).max(), name


def test_loss_gradient_matches_finite_differences():
    """d/dtheta of the force-matching loss, RGL and spline models."""
    configs = [(b.x, b.box) for b in (I.strained_fcc(3, I.A_CU, seed=s) for s in (1, 2))]
    ref = O.Potential(I.RGL_CU)
    targets = [(O.forces(ref, x, box)["f"], O.forces(ref, x, box)["E"]) for x, box in configs]
    model = dict(I.RGL_CU, A=0.0855 * 1.05, xi=1.224 * 0.95, p=10.96 * 1.05, q=2.278 * 0.95, r0=2.5562 * 1.05)
    pot = O.Potential(model)
    grad = np.zeros(5)
    for (x, box), (ft, et) in zip(configs, targets):
        r = O.forces(pot, x, box)
        n = len(x)
        gF = 2 * (r["f"] - ft) / (3 * n) / len(configs)
        gE = 0.2 * (r["E"] / n - et / n) / n / len(configs)
        O.param_grad(pot, x, box, gF, gE, grad)
    for k, name in enumerate(O.RGL_ORDER):
        h = 1e-6 * abs(model[name])
        lp = loss_of(O.Potential(dict(model, **{name: model[name] + h})), configs, targets)
        lm = loss_of(O.Potential(dict(model, **{name: model[name] - h})), configs, targets)
        assert grad[k] == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    # spline model tabulated from the perturbed RGL, gradient on a few knots
    sp = O.tabulate_spline(model, n_knots=40, rho_hi=2 * 20.620605425592796)
    spot = O.Potential(sp)
    grad = np.zeros(spot.n_param)
    for (x, box), (ft, et) in zip(configs, targets):
        r = O.forces(spot, x, box)
        n = len(x)
        gF = 2 * (r["f"] - ft) / (3 * n) / len(configs)
        gE = 0.2 * (r["E"] / n - et / n) / n / len(configs)
        O.param_grad(spot, x, box, gF, gE, grad)
    keys = [("phi", 8), ("phi", 20), ("f", 15), ("f", 30), ("F", 19), ("F", 21)]
    offs = {"phi": 0, "f": 40, "F": 80}
    for key, idx in keys:
        h = 1e-6 * max(abs(sp[key][idx]), 1e-3)
        up, dn = dict(sp), dict(sp)
        up[key] = sp[key].copy()
        dn[key] = sp[key].copy()
        up[key][idx] += h
        dn[key][idx] -= h
        fd = (loss_of(O.Potential(up), configs, targets) - loss_of(O.Potential(dn), configs, targets)) / (2 * h)
        g = grad[offs[key] + idx]
        assert g == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(grad).max()))


# ---------------------------------------------------------------- all-cores form

@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_pair_list_is_the_serial_list(threads):
    """The all-cores linked-cell list joins per-slab buffers in slab order:
    the same pairs in the same order as the serial linked-cell list."""
    bx = I.perturbed_fcc(7, I.A_CU, 600.0, I.MASS_CU, seed=61)
    a = O.pairs(bx.x, bx.box, 5.3)
    b = O.pairs(bx.x, bx.box, 5.3, threads=threads)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_threaded_sums_with_one_thread_are_the_serial_sums_bit_for_bit():
    bx = I.perturbed_fcc(6, I.A_CU, 900.0, I.MASS_CU, seed=62)
    for spec in (I.RGL_CU, I.SC_CU):
        if spec is I.SC_CU:
            bx = I.perturbed_fcc(7, I.A_CU, 900.0, I.MASS_CU, seed=63)
        pot = O.Potential(spec)
        a = O.forces(pot, bx.x, bx.box, skin=0.3)
        b = O.forces(pot, bx.x, bx.box, skin=0.3, threads=1)
        assert a["E"] == b["E"]
        for k in ("rho", "Fp", "e_atom", "f"):
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("threads", [2, 5, 8])
def test_threaded_sums_equal_the_serial_sums_to_rounding(threads):
    bx = I.perturbed_fcc(6, I.A_CU, 900.0, I.MASS_CU, seed=64)
    pot = O.Potential(I.RGL_CU)
    a = O.forces(pot, bx.x, bx.box, skin=0.3)
    b = O.forces(pot, bx.x, bx.box, skin=0.3, threads=threads)
    assert abs(a["E"] - b["E"]) <= 1e-13 * abs(a["E"])
    assert np.abs(a["rho"] - b["rho"]).max() <= 1e-13 * np.abs(a["rho"]).max()
    assert np.abs(a["f"] - b["f"]).max() <= 1e-12 * np.abs(a["f"]).max()


def test_threaded_trajectory_follows_the_serial_one():
    bx = I.perturbed_fcc(5, I.A_CU, 600.0, I.MASS_CU, seed=65)
    pot = O.Potential(I.RGL_CU)
    ref = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 40)
    try:
        O.set_threads(4)
        par = O.md_run(pot, bx.x, bx.v, bx.box, I.MASS_CU, 1.0, 0.3, 40)
    finally:
        O.set_threads(1)
    assert par["n_rebuild"] == ref["n_rebuild"]
    assert np.abs(par["x"] - ref["x"]).max() < 1e-10
    assert np.allclose(par["thermo"], ref["thermo"], rtol=1e-11, atol=1e-11)
