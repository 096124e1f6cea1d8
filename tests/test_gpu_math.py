"""The float64 hot-path functions (table-driven exp, refined rsqrt) against
CUDA's own exp / rsqrt and the host's libm, through md_eval_math."""
import numpy as np
import pytest

from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sysm():
    from paper_1212_6332_gb300.md import System
    return System(I.RGL_CU, box=[30.0, 30.0, 30.0], n_atoms=4)


def ulp_err(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_table_exp_within_two_ulp(sysm):
    import torch
    rng = np.random.default_rng(0)
    y = np.concatenate([rng.uniform(-60.0, 20.0, 1 << 20), np.linspace(-0.01, 0.01, 4097),
                        np.arange(-40, 21, dtype=np.float64) * np.log(2.0) / 256.0 * 997.0, [0.0, -0.0]])
    yt = torch.tensor(y, device="cuda")
    mine = sysm.eval_math("exp", yt).cpu().numpy()
    ref = sysm.eval_math("exp_ref", yt).cpu().numpy()
    host = np.exp(y)
    assert ulp_err(mine, ref).max() <= 2.0
    assert ulp_err(mine, host).max() <= 2.0
    assert mine[-2] == 1.0 and mine[-1] == 1.0


def test_refined_rsqrt_within_two_ulp(sysm):
    """Two ulp against the host's 1/sqrt(x), itself two roundings away from
    the exact value."""
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(0.5, 60.0, 1 << 20), 10.0 ** rng.uniform(-6, 6, 1 << 16), [1.0, 4.0, 25.0]])
    xt = torch.tensor(x, device="cuda")
    mine = sysm.eval_math("rsqrt", xt).cpu().numpy()
    ref = sysm.eval_math("rsqrt_ref", xt).cpu().numpy()
    host = 1.0 / np.sqrt(x)
    assert ulp_err(mine, host).max() <= 2.0
    assert ulp_err(ref, host).max() <= 2.0
    assert mine[-3] == 1.0 and mine[-2] == 0.5 and abs(mine[-1] - 0.2) <= np.spacing(0.2)


def test_integer_pipe_rsqrt_and_sqrt_within_0_51_ulp(sysm):
    """The float64 pair functions' 1/sqrt(r^2) and r, formed in fixed point on
    the integer pipe: within 0.51 ulp of the exact values (50-digit decimal
    arithmetic on a sample; the host's sqrt, correctly rounded, on all), and
    exact at powers of four."""
    import decimal
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(0.5, 60.0, 1 << 20), 10.0 ** rng.uniform(-6, 6, 1 << 16),
                        np.nextafter(np.float64(4.0), 0.0) * np.ones(1), [1.0, 4.0, 16.0, 0.25]])
    xt = torch.tensor(x, device="cuda")
    y = sysm.eval_math("rsqrt_int", xt).cpu().numpy()
    r = sysm.eval_math("sqrt_int", xt).cpu().numpy()
    host_r = np.sqrt(x)
    assert ulp_err(r, host_r).max() <= 1.0
    assert ulp_err(y, 1.0 / host_r).max() <= 2.0
    assert list(y[-4:]) == [1.0, 0.5, 0.25, 2.0] and list(r[-4:]) == [1.0, 2.0, 4.0, 0.5]
    decimal.getcontext().prec = 50
    worst = 0.0
    for k in np.concatenate([rng.integers(0, x.size, 4000), np.arange(x.size - 5, x.size)]):
        s = decimal.Decimal(float(x[k])).sqrt()
        for got, want in ((float(r[k]), s), (float(y[k]), 1 / s)):
            worst = max(worst, float(abs(decimal.Decimal(got) - want) / decimal.Decimal(np.spacing(got))))
    assert worst <= 0.51, worst


@pytest.mark.parametrize("spec", [I.RGL_CU, I.RGL_NI])
def test_rgl_pair_functions_from_the_r_table(spec):
    """The float64 pair path takes both RGL exponentials from a table over r
    (points 1/1024 A apart, a degree-4 correction). Two-atom boxes at 6001
    separations from 0.5 A (below the table: the exp_tab path) to r_cut,
    through every taper and table cell boundary: rho_i within 1e-14 and the
    pair force within 1e-13 (inside r_taper) of the oracle's libm evaluation
    (plus 1e-15 absolute: next to r_cut the taper itself cancels to ~1e-25). The two
    sides form r differently (refined rsqrt against sqrt, an ulp or two),
    and exp(-b r) amplifies that by b r (up to ~20), so a few tens of ulp
    separate them; a table off by one point would be 1e-3 off, a wrong
    correction coefficient 1e-6."""
    import torch
    import oracle as O
    from paper_1212_6332_gb300.md import System
    rc = spec["r_cut"]
    r = np.concatenate([np.linspace(0.5, rc - 1e-9, 6001), np.arange(1536, int(rc * 1024)) / 1024.0])
    n = len(r)
    L = 2.0 * rc + 2.0
    x = np.zeros((n, 2, 3))
    x[:, :] = [1.0, 1.0, 1.0]
    x[:, 1, 0] = 1.0 + r * 0.6
    x[:, 1, 1] = 1.0 + r * 0.8
    boxes = np.full((n, 3), L)
    offs = np.arange(n + 1, dtype=np.int64) * 2
    s = System(spec, boxes=boxes, atom_offsets=offs, skin=0.0, mass=I.MASS_CU)
    f, _ = s.batch_compute_forces(torch.tensor(x.reshape(-1, 3), device="cuda"))
    rho = s.get_forces()["rho"].cpu().numpy().reshape(n, 2)[:, 0]
    f = f.cpu().numpy().reshape(n, 2, 3)[:, 0]
    pot = O.Potential(spec)
    ref_rho = np.empty(n)
    ref_f = np.empty((n, 3))
    for k in range(n):
        o = O.forces(pot, x[k], boxes[k], method="brute")
        ref_rho[k] = o["rho"][0]
        ref_f[k] = o["f"][0]
    inside = r < rc
    rerr = np.abs(rho[inside] - ref_rho[inside]) / (np.abs(ref_rho[inside]) + 1e-1)
    assert rerr.max() <= 1e-14, (rerr.max(), r[inside][np.argmax(rerr)])
    fmag = np.linalg.norm(ref_f, axis=1)
    ferr = np.linalg.norm(f - ref_f, axis=1)
    # the pair force is the difference of a repulsive and an attractive term
    # (it vanishes at the dimer's equilibrium): measure it against their
    # sum, |V'| + 2 |F'(rho) rho'| = 2A (p/r0) e^(p(1 - r/r0)) + (2q/r0) sqrt(rho)
    # inside r_taper; inside the taper rho carries the taper's cancellation
    # (rho -> 1e-9 at r_cut) and F'(rho) = -1/(2 sqrt(rho)) amplifies it on
    # both sides alike
    scale = 2 * spec["A"] * spec["p"] / spec["r0"] * np.exp(spec["p"] * (1 - r / spec["r0"])) + \
        2 * spec["q"] / spec["r0"] * np.sqrt(ref_rho)
    flat = r < spec["r_taper"]
    worst = np.max(ferr[flat] / scale[flat])
    assert worst <= 1e-13, (worst, r[flat][np.argmax(ferr[flat] / scale[flat])])
    # (next to r_cut S ~ 1e-7 and its float64 polynomial carries ~1e-9 of
    # relative rounding on either side, 4e-9 of the force at r_cut - 1e-3 A
    # for Ni, and the force crosses zero inside the taper too: the bound is
    # taken against the region's largest force; a table error would be 1e-6
    # of it or more)
    tap = inside & ~flat
    assert ferr[tap].max() <= 1e-8 * fmag[tap].max(), (ferr[tap].max(), r[tap][np.argmax(ferr[tap])])


def test_fma_probe_measures_both_pipes():
    """md_fma_probe (the roofline denominators): a positive float64 and a
    larger float32 FMA rate, and the device's multiprocessor count."""
    import torch
    from paper_1212_6332_gb300 import md
    r64 = md.fma_probe("fp64", 256)
    r32 = md.fma_probe("fp32", 4096)
    assert r64["n_sm"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert r64["flops"] > 1e11 and r32["flops"] > 8 * r64["flops"]
    assert r64["ms"] > 0 and r32["ms"] > 0
