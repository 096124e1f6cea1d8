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
