"""Writes tests/golden/*.json: forces, densities and energies of small seeded
boxes computed by the CPU oracle alone (oracle.forces, the half-list
Newton's-third-law sums of Eq. (1)-(3)), so that tests can compare the CUDA
path with stored oracle values and the oracle with its own earlier output.

Run from the repository root: python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import pathlib
import sys

ROOT = pathlib.Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1212_6332_gb300 import inputs as I  # noqa: E402

HERE = pathlib.Path(__file__).resolve().parent

# (file stem, potential, fcc repeats, lattice constant, temperature, seed)
CASES = [
    ("rgl_cu_4x4x4_300K", I.RGL_CU, 4, I.A_CU, 300.0, 4401),
    ("sc_cu_5x5x5_1200K", I.SC_CU, 5, I.A_CU, 1200.0, 4402),
]


def case_record(name, spec, n, a, temp, seed) -> dict:
    bx = I.perturbed_fcc(n, a, temp, I.MASS_CU, seed=seed)
    out = O.forces(O.Potential(spec), bx.x, bx.box)
    return {
        "what": "oracle.forces (half-list sums of Eq. 1-3, float64) on inputs.perturbed_fcc",
        "potential": spec, "repeats": n, "lattice": a, "temperature_K": temp, "seed": seed,
        "box": bx.box.tolist(), "x": bx.x.tolist(),
        "E": float(out["E"]), "rho": np.asarray(out["rho"]).tolist(), "f": np.asarray(out["f"]).tolist(),
    }


def main() -> None:
    for case in CASES:
        rec = case_record(*case)
        (HERE / f"{case[0]}.json").write_text(json.dumps(rec, indent=0) + "\n")
        print(f"wrote {case[0]}.json: {len(rec['x'])} atoms, E = {rec['E']:.12f} eV")


if __name__ == "__main__":
    main()
