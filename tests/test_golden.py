"""Stored oracle values (tests/golden/*.json, written by
tests/golden/make_golden.py from the CPU oracle alone): the oracle still
gives them (CPU), and the CUDA path matches them at the parity bars of
forces and energies, 1e-10 relative (GPU)."""
import json
import pathlib

import numpy as np
import pytest

import oracle as O

GOLDEN = sorted((pathlib.Path(__file__).resolve().parent / "golden").glob("*.json"))


def load(p):
    d = json.loads(p.read_text())
    return d, np.array(d["x"]), np.array(d["box"]), np.array(d["f"]), np.array(d["rho"])


@pytest.mark.parametrize("path", GOLDEN, ids=[p.stem for p in GOLDEN])
def test_oracle_reproduces_its_stored_values(path):
    d, x, box, f, rho = load(path)
    out = O.forces(O.Potential(d["potential"]), x, box)
    assert abs(out["E"] - d["E"]) <= 1e-13 * abs(d["E"])
    assert np.abs(out["f"] - f).max() <= 1e-13 * np.abs(f).max()
    assert np.abs(out["rho"] - rho).max() <= 1e-13 * np.abs(rho).max()


@pytest.mark.gpu
@pytest.mark.parametrize("path", GOLDEN, ids=[p.stem for p in GOLDEN])
def test_cuda_path_matches_stored_oracle_values(path):
    import torch
    from paper_1212_6332_gb300.md import System
    d, x, box, f, rho = load(path)
    s = System(d["potential"], box=box, n_atoms=len(x), skin=0.3, mass=63.546)
    out = s.compute_forces(torch.tensor(x, device="cuda"))
    got_f = out["f"].cpu().numpy()
    assert np.abs(got_f - f).max() <= 1e-10 * np.abs(f).max()
    assert abs(out["energy"].item() - d["E"]) <= 1e-10 * abs(d["E"])
    assert np.abs(out["rho"].cpu().numpy() - rho).max() <= 1e-12 * np.abs(rho).max()
    s.close()
