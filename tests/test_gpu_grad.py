"""Parameter adjoint (md_param_grad) against the oracle's forward-mode
derivatives and against central finite differences of the loss."""
import numpy as np
import pytest

import oracle as O
from paper_1212_6332_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RHO_EQ = 20.620605425592796
MODEL = dict(I.RGL_CU, A=0.0855 * 1.05, xi=1.224 * 0.95, p=10.96 * 1.05, q=2.278 * 0.95, r0=2.5562 * 1.05)


def configs(ns=(3, 4, 3), seed=10):
    return [I.strained_fcc(n, I.A_CU, seed=seed + k) for k, n in enumerate(ns)]


def oracle_grad(spec, cfgs, g_f, g_e):
    pot = O.Potential(spec)
    grad = np.zeros(pot.n_param)
    off = 0
    for c, ge in zip(cfgs, g_e):
        O.param_grad(pot, c.x, c.box, g_f[off:off + c.n], ge, grad)
        off += c.n
    return grad


@pytest.mark.parametrize("kind", ["rgl", "spline"])
def test_adjoint_matches_oracle_forward_mode(kind):
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    spec = MODEL if kind == "rgl" else O.tabulate_spline(MODEL, n_knots=60, rho_hi=2 * RHO_EQ)
    cfgs = configs()
    s = make_batch(spec, cfgs)
    n = sum(c.n for c in cfgs)
    rng = np.random.default_rng(5)
    g_f = rng.normal(size=(n, 3))
    g_e = rng.normal(size=len(cfgs))
    got = s.param_grad(torch.tensor(g_f, device="cuda"), torch.tensor(g_e, device="cuda")).cpu().numpy()
    ref = oracle_grad(spec, cfgs, g_f, g_e)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_autograd_loss_gradient_matches_finite_differences():
    import torch
    from paper_1212_6332_gb300.fit import ForceField, force_matching_loss, make_batch, spec_of, theta_of
    cfgs = configs((3, 3, 4, 3), seed=20)
    ref = make_batch(I.RGL_CU, cfgs)
    f_tgt = ref.get_forces()["f"].clone()
    e_tgt = ref.batch_thermo()[:, 1].clone()
    counts = torch.tensor([c.n for c in cfgs], device="cuda", dtype=torch.float64)
    s = make_batch(MODEL, cfgs)
    theta = theta_of(MODEL).requires_grad_(True)

    def loss_at(th):
        f, e = ForceField.apply(th, s, MODEL)
        return force_matching_loss(f, e, f_tgt, e_tgt, counts)

    L = loss_at(theta)
    (g,) = torch.autograd.grad(L, theta)
    for k in range(5):
        h = 1e-6 * abs(theta[k].item())
        tp, tm = theta.detach().clone(), theta.detach().clone()
        tp[k] += h
        tm[k] -= h
        fd = (loss_at(tp).item() - loss_at(tm).item()) / (2 * h)
        assert g[k].item() == pytest.approx(fd, rel=1e-6), (k, g[k].item(), fd)


def test_adjoint_with_zero_upstream_is_zero():
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    cfgs = configs((3,), seed=3)
    s = make_batch(MODEL, cfgs)
    z = torch.zeros(cfgs[0].n, 3, dtype=torch.float64, device="cuda")
    g = s.param_grad(z, torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(g) == 0


@pytest.mark.parametrize("kind", ["rgl", "spline"])
def test_mixed_precision_adjoint_within_bound(kind):
    """Mixed precision (float32 pair geometry and pair terms, float64
    parameter sums) against the oracle's float64 forward-mode gradient: each
    component within 1e-4 of the largest (the pair terms carry ~1e-6
    relative float32 error, and the gradient is a sum of many such terms
    with partial cancellation)."""
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    spec = MODEL if kind == "rgl" else O.tabulate_spline(MODEL, n_knots=60, rho_hi=2 * RHO_EQ)
    cfgs = configs((3, 4, 4), seed=31)
    s = make_batch(spec, cfgs, precision="mixed")
    n = sum(c.n for c in cfgs)
    rng = np.random.default_rng(6)
    g_f = rng.normal(size=(n, 3))
    g_e = rng.normal(size=len(cfgs))
    got = s.param_grad(torch.tensor(g_f, device="cuda"), torch.tensor(g_e, device="cuda")).cpu().numpy()
    ref = oracle_grad(spec, cfgs, g_f, g_e)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("kind", ["rgl", "spline"])
def test_adjoint_from_the_forward_cache_equals_the_recomputed_one(kind):
    """The float64 adjoint reads the forward pass's pair cache, rho and F'
    when they are current; after a call that leaves them stale it evaluates
    the pair functions again. Both paths give the same gradient (to
    rounding), and with the Newton's-third-law sums on (lower cache slots
    unwritten) the recomputing path serves and still matches the oracle."""
    import torch
    from paper_1212_6332_gb300.fit import make_batch
    spec = MODEL if kind == "rgl" else O.tabulate_spline(MODEL, n_knots=60, rho_hi=2 * RHO_EQ)
    cfgs = configs((3, 4), seed=71)
    s = make_batch(spec, cfgs)
    n = sum(c.n for c in cfgs)
    rng = np.random.default_rng(8)
    g_f = torch.tensor(rng.normal(size=(n, 3)), device="cuda")
    g_e = torch.tensor(rng.normal(size=len(cfgs)), device="cuda")
    cached = s.param_grad(g_f, g_e).cpu().numpy()
    s.set_newton3(True)  # the adjoint may no longer read the cache
    recomputed = s.param_grad(g_f, g_e).cpu().numpy()
    ref = oracle_grad(spec, cfgs, g_f.cpu().numpy(), g_e.cpu().numpy())
    scale = np.abs(ref).max()
    assert np.abs(cached - recomputed).max() <= 1e-12 * scale
    assert np.abs(recomputed - ref).max() <= 1e-10 * scale


def test_deferred_status_gives_the_same_fit_and_reports_at_sync():
    """A fitting loop with deferred device status (the calls return without
    waiting for the status word) gives the bits of the waiting loop; sync()
    reports a clean status; argument errors still come back at once."""
    import torch
    from paper_1212_6332_gb300.fit import ForceField, config_index, force_matching_loss, make_batch, theta_of
    from paper_1212_6332_gb300.md import MDError
    cfgs = configs((3, 4, 3), seed=33)
    ref = make_batch(I.RGL_CU, cfgs, deferred=False)
    f_tgt = ref.get_forces()["f"].clone()
    e_tgt = ref.batch_thermo()[:, 1].clone()
    ref.close()
    counts = torch.tensor([c.n for c in cfgs], device="cuda", dtype=torch.float64)
    idx = config_index(counts)
    out = {}
    for deferred in (False, True):
        s = make_batch(MODEL, cfgs, deferred=deferred)
        theta = theta_of(MODEL).cuda().requires_grad_(True)
        hist = []
        for _ in range(3):
            f, e = ForceField.apply(theta, s, MODEL)
            L = force_matching_loss(f, e, f_tgt, e_tgt, counts, idx=idx)
            (g,) = torch.autograd.grad(L, theta)
            hist.append((L.item(), g.cpu().numpy(), f.detach().cpu().numpy()))
            with torch.no_grad():
                theta -= 1e-3 * g
        s.sync()
        if deferred:
            with pytest.raises(MDError):
                s.param_grad(torch.zeros(s.n, 3, dtype=torch.float64, device="cuda"),
                             torch.zeros(s.n_boxes, dtype=torch.float64, device="cuda"),
                             grad=torch.zeros(s.n_params, dtype=torch.float64))  # host tensor: rejected
        s.close()
        out[deferred] = hist
    # (the loss itself goes through torch's index_add_, whose float64 atomics
    # land in any order: compared to rounding; forces and gradients by bits)
    for (la, ga, fa), (lb, gb, fb) in zip(out[False], out[True]):
        assert abs(la - lb) <= 1e-14 * abs(la)
        assert np.array_equal(ga, gb) and np.array_equal(fa, fb)
