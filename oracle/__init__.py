"""CPU FP64 oracle for the many-body MD hot path (test infrastructure only).

A ctypes wrapper around ``md_oracle.c``. Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import this package; the CUDA library
and its Python binding never do, and share no code with it.

Every function here takes numpy float64 arrays in the caller's atom order:
positions ``x`` [N, 3] (wrapped into [0, L)), box lengths ``box`` [3].
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_LIBDIR = _HERE / "_lib"
_SO = _LIBDIR / "libmd_oracle.so"

KIND = {"rgl": 0, "sc": 1, "spline": 2}
RGL_ORDER = ("A", "xi", "p", "q", "r0")
SC_ORDER = ("eps", "c", "a", "n", "m")


def build(force: bool = False) -> pathlib.Path:
    """Compiles the oracle with gcc: -O2, no fast-math, no FMA contraction
    (the neighbour-list distance test must round after every operation)."""
    src = _HERE / "md_oracle.c"
    if not force and _SO.exists() and _SO.stat().st_mtime >= src.stat().st_mtime:
        return _SO
    _LIBDIR.mkdir(exist_ok=True)
    tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           str(src), "-o", str(tmp), "-lm"]
    # OpenMP serves only the all-cores timing (orc_set_threads > 1); without
    # it the library builds serial and reports one thread
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.orc_pot_new.restype = vp
    lib.orc_pot_new.argtypes = [i32, _D, dbl, dbl, i32, i32, i32, _D, dbl, dbl, dbl, dbl]
    lib.orc_pot_free.argtypes = [vp]
    lib.orc_pot_new_alloy.restype = vp
    lib.orc_pot_new_alloy.argtypes = [i32, i32, i32, _D, dbl, dbl, dbl, dbl]
    lib.orc_pot_set_types.argtypes = [vp, _I]
    lib.orc_pot_eval.argtypes = [vp, i32, _D, _D, _D, _D, _D]
    lib.orc_embed_eval.argtypes = [vp, i32, _D, _D, _D, _D]
    lib.orc_wrap.argtypes = [i32, _D, _D]
    lib.orc_pairs_brute.restype = i64
    lib.orc_pairs_brute.argtypes = [i32, _D, _D, dbl, _I, _I, i64]
    lib.orc_pairs_cells.restype = i64
    lib.orc_pairs_cells.argtypes = [i32, _D, _D, dbl, _I, _I, i64]
    lib.orc_forces_brute.restype = dbl
    lib.orc_forces_brute.argtypes = [vp, i32, _D, _D, _D, _D, _D]
    lib.orc_forces_pairs.restype = dbl
    lib.orc_forces_pairs.argtypes = [vp, i32, _D, _D, i64, _I, _I, _D, _D, _D, _D]
    lib.orc_md_run.restype = i64
    lib.orc_md_run.argtypes = [vp, i32, _D, _D, _D, dbl, dbl, dbl, i32, _D, dbl, dbl, dbl, dbl, dbl, _D]
    lib.orc_virial_pairs.restype = dbl
    lib.orc_virial_pairs.argtypes = [vp, i32, _D, _D, i64, _I, _I]
    lib.orc_param_deriv.restype = dbl
    lib.orc_param_deriv.argtypes = [vp, i32, i32, _D, _D, i64, _I, _I, _D]
    lib.orc_param_grad.argtypes = [vp, i32, i32, _D, _D, i64, _I, _I, _D, dbl, _D]
    lib.orc_set_threads.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    lib.orc_max_threads.restype = i32
    lib.orc_pairs_cells_par.restype = i64
    lib.orc_pairs_cells_par.argtypes = [i32, _D, _D, dbl, _I, _I, i64, i32]
    lib.orc_forces_pairs_par.restype = dbl
    lib.orc_forces_pairs_par.argtypes = [vp, i32, _D, _D, i64, _I, _I, _D, _D, _D, _D, i32]
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Potential:
    """Oracle-side potential. ``spec`` is a dict like
    ``{"kind": "rgl", "A":..., "xi":..., "p":..., "q":..., "r0":..., "r_taper":..., "r_cut":...}``,
    ``{"kind": "sc", "eps", "c", "a", "n", "m", "r_taper", "r_cut"}`` or
    ``{"kind": "spline", "phi": knots, "f": knots, "F": knots, "r_lo", "r_hi", "rho_lo", "rho_hi"}`` or,
    for several species, ``{"kind": "alloy", "n_types": T, "phi": [V^(ab) knots per type pair],
    "f": [rho^(ab) knots per type pair], "F": [F^(a) knots per type], "r_lo", "r_hi", "rho_lo",
    "rho_hi"}`` with the type pairs a <= b in row-major order ((0,0), (0,1), ..., (1,1), ...)."""

    def __init__(self, spec: dict):
        lib = _load()
        self.spec = dict(spec)
        kind = spec["kind"]
        prm = np.zeros(8)
        knots = np.zeros(1)
        n_phi = n_f = n_F = 0
        r_lo = r_hi = rho_lo = rho_hi = 0.0
        r_taper = float(spec.get("r_taper", 0.0))
        r_cut = float(spec.get("r_cut", 0.0))
        if kind == "rgl":
            prm[:5] = [spec[k] for k in RGL_ORDER]
            self.n_param = 5
        elif kind == "sc":
            prm[:5] = [spec[k] for k in SC_ORDER]
            self.n_param = 5
        elif kind == "spline":
            phi, f, F = (_f64(spec[k]) for k in ("phi", "f", "F"))
            n_phi, n_f, n_F = len(phi), len(f), len(F)
            knots = np.concatenate([phi, f, F])
            r_lo, r_hi = float(spec["r_lo"]), float(spec["r_hi"])
            rho_lo, rho_hi = float(spec["rho_lo"]), float(spec["rho_hi"])
            r_taper = r_cut = r_hi
            self.n_param = n_phi + n_f + n_F
        elif kind == "alloy":
            T = int(spec["n_types"])
            phi = [_f64(a) for a in spec["phi"]]
            f = [_f64(a) for a in spec["f"]]
            F = [_f64(a) for a in spec["F"]]
            if len(phi) != T * (T + 1) // 2 or len(f) != len(phi) or len(F) != T:
                raise ValueError("alloy: T(T+1)/2 pair tables and T embedding tables")
            knots = np.concatenate(phi + f + F)
            r_lo, r_hi = float(spec["r_lo"]), float(spec["r_hi"])
            rho_lo, rho_hi = float(spec["rho_lo"]), float(spec["rho_hi"])
            r_cut = r_hi
            self.n_param = knots.size
            self.r_cut = r_cut
            self.n_types = T
            self._prm, self._knots = prm, knots
            self._h = lib.orc_pot_new_alloy(T, len(phi[0]), len(F[0]), _dp(knots), r_lo, r_hi, rho_lo, rho_hi)
            return
        else:
            raise ValueError(kind)
        self.r_cut = r_cut
        self.n_types = 1
        self._prm, self._knots = prm, knots
        self._h = lib.orc_pot_new(KIND[kind], _dp(prm), r_taper, r_cut, n_phi, n_f, n_F, _dp(knots),
                                  r_lo, r_hi, rho_lo, rho_hi)

    def use_types(self, types):
        """Per-atom species for the following calls (None: all species 0)."""
        if types is None:
            self._types = None
            _load().orc_pot_set_types(self._h, None)
            return
        self._types = np.ascontiguousarray(types, dtype=np.int32)
        _load().orc_pot_set_types(self._h, self._types.ctypes.data_as(_I))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_pot_free(self._h)
            self._h = None

    def pair(self, r) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        """(V, V', rho, rho') at distances r."""
        r = _f64(np.atleast_1d(r))
        out = [np.empty_like(r) for _ in range(4)]
        _load().orc_pot_eval(self._h, r.size, _dp(r), *(_dp(o) for o in out))
        return tuple(out)

    def embed(self, rho) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(F, F', F'') at densities rho."""
        rho = _f64(np.atleast_1d(rho))
        out = [np.empty_like(rho) for _ in range(3)]
        _load().orc_embed_eval(self._h, rho.size, _dp(rho), *(_dp(o) for o in out))
        return tuple(out)


def wrap(x, box) -> np.ndarray:
    x = _f64(x).copy()
    box = _f64(box)
    _load().orc_wrap(x.shape[0], _dp(x), _dp(box))
    return x


def set_threads(t: int) -> int:
    """Threads for md_run's pair list and force sums (1 = the plain serial
    functions, the default); returns the count in effect (1 when the
    library was built without OpenMP)."""
    return int(_load().orc_set_threads(int(t)))


def max_threads() -> int:
    """Threads OpenMP would use by default (the host's cores), 1 without OpenMP."""
    return int(_load().orc_max_threads())


def pairs(x, box, rl: float, method: str = "cells", threads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Half list (i < j) of pairs with minimum-image r^2 < rl^2. threads > 0
    with method "cells" uses the all-cores form (the same list)."""
    lib = _load()
    x, box = _f64(x), _f64(box)
    n = x.shape[0]
    if method == "cells" and threads > 0:
        def fn(*a):
            return lib.orc_pairs_cells_par(*a, int(threads))
    else:
        fn = lib.orc_pairs_cells if method == "cells" else lib.orc_pairs_brute
    cap = max(64, n * 80)
    while True:
        pi = np.empty(cap, dtype=np.int32)
        pj = np.empty(cap, dtype=np.int32)
        np_ = fn(n, _dp(x), _dp(box), float(rl), _ip(pi), _ip(pj), cap)
        if np_ <= cap:
            return pi[:np_].copy(), pj[:np_].copy()
        cap = int(np_)


def forces(pot: Potential, x, box, skin: float = 0.0, method: str = "pairs", types=None, threads: int = 0) -> dict:
    """Energies and forces of Eq. (1)-(3). method "pairs" uses the half list
    within r_cut + skin and Newton's third law; "brute" the O(N^2) double
    sums. types: per-atom species for an alloy potential. threads > 0 runs
    the half-list sums in their all-cores form."""
    lib = _load()
    pot.use_types(types)
    x, box = _f64(x), _f64(box)
    n = x.shape[0]
    rho = np.zeros(n)
    e = np.zeros(n)
    f = np.zeros((n, 3))
    if method == "brute":
        E = lib.orc_forces_brute(pot._h, n, _dp(x), _dp(box), _dp(rho), _dp(e), _dp(f))
        Fp = pot.embed(rho)[1] if n else np.zeros(0)
        return dict(E=E, rho=rho, Fp=Fp, e_atom=e, f=f)
    pi, pj = pairs(x, box, pot.r_cut + skin, threads=threads)
    Fp = np.zeros(n)
    if threads > 0:
        E = lib.orc_forces_pairs_par(pot._h, n, _dp(x), _dp(box), pi.size, _ip(pi), _ip(pj), _dp(rho), _dp(Fp),
                                     _dp(e), _dp(f), int(threads))
    else:
        E = lib.orc_forces_pairs(pot._h, n, _dp(x), _dp(box), pi.size, _ip(pi), _ip(pj), _dp(rho), _dp(Fp),
                                 _dp(e), _dp(f))
    return dict(E=E, rho=rho, Fp=Fp, e_atom=e, f=f)


def md_run(pot: Potential, x, v, box, mass: float, dt: float, skin: float, n_steps: int,
           tau_T: float = 0.0, T_e: float = 0.0, tau_p: float = 0.0, P0: float = 0.0,
           beta: float = 0.0, types=None, want_pressure: bool = False) -> dict:
    """Velocity-Verlet trajectory; returns final x, v, box, per-step thermo
    rows (KE, PE, E_tot, T), per-step pressures (Eq. 6, eV/A^3; when
    want_pressure or tau_p > 0, else None) and the number of list rebuilds. With tau_T > 0 the electron-phonon friction of
    Eq. (4) couples every atom to the electronic temperature T_e (K) with
    time constant tau_T (fs); with tau_p > 0 the Berendsen coupling of
    Eq. (5) scales coordinates and box towards the pressure P0 (eV/A^3)
    with compressibility beta (A^3/eV)."""
    lib = _load()
    pot.use_types(types)
    x, v, box = _f64(x).copy(), _f64(v).copy(), _f64(box).copy()
    thermo = np.zeros((n_steps + 1, 4))
    # per-step pressures only when asked for or coupled (each costs a virial pass)
    press = np.zeros(n_steps + 1) if (want_pressure or tau_p > 0.0) else None
    nreb = lib.orc_md_run(pot._h, x.shape[0], _dp(x), _dp(v), _dp(box), float(mass), float(dt), float(skin),
                          int(n_steps), _dp(thermo), float(tau_T), float(T_e), float(tau_p), float(P0),
                          float(beta), _dp(press) if press is not None else None)
    return dict(x=x, v=v, box=box, thermo=thermo, pressure=press, n_rebuild=int(nreb))


def virial(pot: Potential, x, box, types=None) -> float:
    """Pair virial W = sum_i f_i . r_i of the forces of Eq. (3) (eV), the
    interaction part of the pressure of Eq. (6)."""
    lib = _load()
    pot.use_types(types)
    x, box = _f64(x), _f64(box)
    pi, pj = pairs(x, box, pot.r_cut)
    return lib.orc_virial_pairs(pot._h, x.shape[0], _dp(x), _dp(box), pi.size, _ip(pi), _ip(pj))


def param_deriv(pot: Potential, which: int, x, box, types=None) -> tuple[float, np.ndarray]:
    """(dE/dtheta, dF/dtheta [N,3]) for parameter index ``which`` (for an
    alloy: the knot index in the order V pair tables, rho pair tables, F
    tables)."""
    lib = _load()
    pot.use_types(types)
    x, box = _f64(x), _f64(box)
    pi, pj = pairs(x, box, pot.r_cut)
    dF = np.zeros((x.shape[0], 3))
    dE = lib.orc_param_deriv(pot._h, int(which), x.shape[0], _dp(x), _dp(box), pi.size, _ip(pi), _ip(pj),
                             _dp(dF))
    return dE, dF


def param_grad(pot: Potential, x, box, gF, gE: float, grad: np.ndarray | None = None, types=None) -> np.ndarray:
    """Accumulates sum_i gF_i . dF_i/dtheta + gE dE/dtheta into ``grad``."""
    lib = _load()
    pot.use_types(types)
    x, box, gF = _f64(x), _f64(box), _f64(gF)
    if grad is None:
        grad = np.zeros(pot.n_param)
    pi, pj = pairs(x, box, pot.r_cut)
    lib.orc_param_grad(pot._h, pot.n_param, x.shape[0], _dp(x), _dp(box), pi.size, _ip(pi), _ip(pj), _dp(gF),
                       float(gE), _dp(grad))
    return grad


def full_neighbor_lists(n: int, pi: np.ndarray, pj: np.ndarray) -> list[np.ndarray]:
    """Per-atom sorted neighbour sets (both directions) from a half list."""
    a = np.concatenate([pi, pj])
    b = np.concatenate([pj, pi])
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    starts = np.searchsorted(a, np.arange(n + 1))
    return [b[starts[i]:starts[i + 1]] for i in range(n)]


def tabulate_spline(spec: dict, n_knots: int = 200, r_lo: float = 1.5, r_hi: float = 5.0,
                    rho_hi: float | None = None) -> dict:
    """Knot values of a spline model tabulated from an analytic potential:
    V and rho on ``n_knots`` uniform knots over [r_lo, r_hi], F on
    ``n_knots`` uniform knots over [0, rho_hi] (default twice the perfect
    fcc density is supplied by the caller)."""
    pot = Potential(spec)
    r = np.linspace(r_lo, r_hi, n_knots)
    V, _, rho, _ = pot.pair(r)
    rg = np.linspace(0.0, rho_hi, n_knots)
    F = pot.embed(rg)[0]
    return dict(kind="spline", phi=V, f=rho, F=F, r_lo=r_lo, r_hi=r_hi, rho_lo=0.0, rho_hi=rho_hi)
