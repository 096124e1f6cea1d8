"""Seeded synthetic inputs: fcc lattices, perturbations, Maxwell-Boltzmann
velocities, strains and batches of uneven boxes.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark. It holds no arithmetic of the many-body method itself (no
potential, neighbour search, force or integrator): it only draws the inputs
that both sides consume, so both see bit-identical arrays.

Random numbers come from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as
a counter-based generator: the k-th draw of stream ``seed`` is
``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15)``, so any slice of a stream can
be drawn independently and vectorised in numpy.

Units: Angstrom, eV, fs, atomic mass units (u), kelvin.
"""
from __future__ import annotations

import dataclasses

import numpy as np

KB_EV_PER_K = 8.617333262e-5          # Boltzmann constant, eV/K (CODATA 2018)
MVV_EV = 103.642696527               # 1 u * (A/fs)^2 in eV

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA)


def derive_seed(base: int, index: int) -> int:
    """Seed of sub-stream ``index`` (one box, one configuration)."""
    return int(splitmix64((base + index) & 0xFFFFFFFFFFFFFFFF, 1)[0])


def uniform(seed: int, count: int, start: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller, two uniforms per normal."""
    u = uniform(seed, 2 * count, 2 * start)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def wrap(x: np.ndarray, box) -> np.ndarray:
    """Maps coordinates into [0, L) per axis: x - L*floor(x/L), one addition
    of L if rounding left it negative, then one subtraction of L if it is L."""
    box = np.asarray(box, dtype=np.float64)
    y = x - box * np.floor(x / box)
    y = np.where(y < 0.0, y + box, y)
    return np.where(y >= box, y - box, y)


def fcc_lattice(n: int, a: float, ny: int | None = None, nz: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Ideal fcc sites of n x ny x nz conventional cells (4 atoms each).

    Atom index = ((ix * ny + iy) * nz + iz) * 4 + b, basis b in the order
    (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2). Returns (x [N,3], box [3]).
    """
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    x = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    box = np.array([n * a, ny * a, nz * a], dtype=np.float64)
    return x, box


def maxwell_velocities(n_atoms: int, temperature: float, mass: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/fs) with zero net momentum, rescaled
    so that sum(m v^2) / ((3N-3) kB) equals ``temperature`` exactly."""
    if temperature <= 0.0 or n_atoms < 2:
        return np.zeros((n_atoms, 3))
    sigma = np.sqrt(KB_EV_PER_K * temperature / (mass * MVV_EV))
    v = normal(seed, 3 * n_atoms).reshape(n_atoms, 3) * sigma
    v -= v.mean(axis=0)
    mv2 = mass * MVV_EV * np.sum(v * v)
    target = (3 * n_atoms - 3) * KB_EV_PER_K * temperature
    return v * np.sqrt(target / mv2)


@dataclasses.dataclass
class Box:
    """One periodic box of atoms: wrapped positions, velocities, lengths."""
    x: np.ndarray        # [N, 3] float64, wrapped into [0, L)
    v: np.ndarray        # [N, 3] float64, A/fs
    box: np.ndarray      # [3] float64
    seed: int

    @property
    def n(self) -> int:
        return self.x.shape[0]


def perturbed_fcc(n: int, a: float, temperature: float, mass: float, seed: int,
                  amplitude: float = 0.05) -> Box:
    """fcc box with each coordinate displaced by U(-amplitude, amplitude),
    wrapped, and Maxwell-Boltzmann velocities at ``temperature``.

    Stream layout for ``seed``: sub-stream 0 draws the displacements,
    sub-stream 1 the velocities.
    """
    x, box = fcc_lattice(n, a)
    if amplitude > 0.0:
        u = uniform(derive_seed(seed, 0), x.size).reshape(x.shape)
        x = x + (2.0 * u - 1.0) * amplitude
    x = wrap(x, box)
    v = maxwell_velocities(x.shape[0], temperature, mass, derive_seed(seed, 1))
    return Box(x=x, v=v, box=box, seed=seed)


def strained_fcc(n: int, a: float, seed: int, strain: float = 0.02, sigma: float = 0.1) -> Box:
    """fcc box with an isotropic strain s ~ U(1-strain, 1+strain) applied to
    box and sites, then N(0, sigma^2) displacements per coordinate, wrapped.
    Velocities are zero (configurations for potential fitting)."""
    s = 1.0 - strain + 2.0 * strain * uniform(derive_seed(seed, 0), 1)[0]
    x, box = fcc_lattice(n, a * s)
    x = x + sigma * normal(derive_seed(seed, 1), x.size).reshape(x.shape)
    x = wrap(x, box)
    return Box(x=x, v=np.zeros_like(x), box=box, seed=seed)


@dataclasses.dataclass
class Batch:
    """Many independent periodic boxes stored back to back."""
    x: np.ndarray              # [sum N_b, 3]
    v: np.ndarray              # [sum N_b, 3]
    atom_offsets: np.ndarray   # [B+1] int64
    box: np.ndarray            # [B, 3]
    n_cells: np.ndarray        # [B] fcc repeats per box
    temperature: np.ndarray    # [B]

    @property
    def n_boxes(self) -> int:
        return self.box.shape[0]


def batch_of_boxes(n_boxes: int, a: float, mass: float, seed: int, n_lo: int = 3, n_hi: int = 10,
                   t_lo: float = 300.0, t_hi: float = 1500.0, amplitude: float = 0.05) -> Batch:
    """``n_boxes`` fcc boxes with n ~ U{n_lo..n_hi} repeats and
    T ~ U(t_lo, t_hi); box b is ``perturbed_fcc`` with seed derive_seed(seed, b+2)."""
    u = uniform(derive_seed(seed, 0), n_boxes)
    ns = n_lo + np.minimum((u * (n_hi - n_lo + 1)).astype(np.int64), n_hi - n_lo)
    temps = t_lo + (t_hi - t_lo) * uniform(derive_seed(seed, 1), n_boxes)
    xs, vs, boxes = [], [], []
    for b in range(n_boxes):
        bx = perturbed_fcc(int(ns[b]), a, float(temps[b]), mass, derive_seed(seed, b + 2), amplitude)
        xs.append(bx.x)
        vs.append(bx.v)
        boxes.append(bx.box)
    counts = np.array([x.shape[0] for x in xs], dtype=np.int64)
    offs = np.zeros(n_boxes + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    return Batch(x=np.concatenate(xs), v=np.concatenate(vs), atom_offsets=offs,
                 box=np.stack(boxes), n_cells=ns, temperature=temps)


# Potential parameter sets of the paper's workloads (second-moment tight
# binding after Cleri and Rosato; Sutton-Chen). Plain data, no arithmetic.
RGL_CU = dict(kind="rgl", A=0.0855, xi=1.224, p=10.960, q=2.278, r0=2.5562, r_taper=4.5, r_cut=5.0)
RGL_NI = dict(kind="rgl", A=0.0376, xi=1.070, p=16.999, q=1.189, r0=2.4911, r_taper=4.3, r_cut=4.8)
SC_CU = dict(kind="sc", eps=0.012382, c=39.432, a=3.61, n=9.0, m=6.0, r_taper=6.92, r_cut=7.22)
MASS_CU = 63.546
MASS_NI = 58.6934
A_CU = 3.615
A_NI = 3.523
