"""Host-side parameter plumbing of the fitting module (no GPU): theta <->
potential spec for every kind, in the knot order md_param_grad and
md_num_params use."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1212_6332_gb300 import inputs as I  # noqa: E402
from paper_1212_6332_gb300.fit import spec_of, theta_of  # noqa: E402


def test_rgl_theta_round_trip():
    th = theta_of(I.RGL_CU)
    assert th.dtype == torch.float64 and th.numel() == 5
    assert np.allclose(th.numpy(), [I.RGL_CU[k] for k in ("A", "xi", "p", "q", "r0")])
    back = spec_of(th * 1.5, I.RGL_CU)
    assert back["A"] == pytest.approx(1.5 * I.RGL_CU["A"]) and back["r_cut"] == I.RGL_CU["r_cut"]


def test_alloy_theta_is_pair_tables_then_rho_then_embedding():
    rng = np.random.default_rng(0)
    T, n = 3, 7
    P = T * (T + 1) // 2
    spec = dict(kind="alloy", n_types=T, phi=[rng.normal(size=n) for _ in range(P)],
                f=[rng.normal(size=n) for _ in range(P)], F=[rng.normal(size=n + 2) for _ in range(T)],
                r_lo=1.5, r_hi=5.0, rho_lo=0.0, rho_hi=40.0)
    th = theta_of(spec)
    assert th.numel() == P * n + P * n + T * (n + 2)  # P (n_phi + n_f) + T n_F
    flat = np.concatenate(spec["phi"] + spec["f"] + spec["F"])
    assert np.array_equal(th.numpy(), flat)
    back = spec_of(th + 1.0, spec)
    for key in ("phi", "f", "F"):
        assert len(back[key]) == len(spec[key])
        for a, b in zip(back[key], spec[key]):
            assert np.array_equal(a, b + 1.0)
    assert back["n_types"] == T and back["r_hi"] == 5.0


def test_spline_theta_round_trip():
    spec = dict(kind="spline", phi=np.linspace(1, 0, 5), f=np.linspace(2, 0, 5), F=-np.sqrt(np.linspace(0, 4, 6)),
                r_lo=1.5, r_hi=5.0, rho_lo=0.0, rho_hi=4.0)
    th = theta_of(spec)
    assert th.numel() == 16
    back = spec_of(th, spec)
    for key in ("phi", "f", "F"):
        assert np.array_equal(back[key], spec[key])
