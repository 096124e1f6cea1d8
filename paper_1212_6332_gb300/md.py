"""Python binding of libmd.so (include/md.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors and numpy arrays into pointers, picks the current torch stream and
turns status codes into exceptions. There is no CPU fallback: if libmd.so is
missing or fails to load, importing the handle raises.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

_PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libmd.so"

FP64, MIXED = 0, 1
POT_RGL, POT_SC, POT_SPLINE = 0, 1, 2
SCHED_AUTO, SCHED_BOX, SCHED_TILE = 0, 1, 2
STATUS = {0: "MD_OK", 1: "MD_ERR_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_NOMEM", 4: "MD_ERR_NEIGH_OVERFLOW",
          5: "MD_ERR_NONFINITE", 6: "MD_ERR_TIMEOUT", 7: "MD_ERR_UNSUPPORTED"}

# every symbol include/md.h declares
SYMBOLS = ("md_create", "md_destroy", "md_set_state", "md_get_state", "md_build_neighbors", "md_get_neighbors",
           "md_max_count", "md_compute_forces", "md_get_forces", "md_step", "md_get_thermo", "md_batch_create",
           "md_batch_destroy", "md_batch_set_state", "md_batch_get_state", "md_batch_compute_forces",
           "md_batch_step", "md_batch_set_potential", "md_set_thermostat", "md_set_newton3", "md_set_types", "md_pressure", "md_set_barostat", "md_get_box", "md_param_grad", "md_num_params", "md_status_string",
           "md_last_error", "md_profile_start", "md_profile_read",
           "md_eval_math", "md_forces_noalloc", "md_batch_thermo",
           "md_batch_schedule", "md_fma_probe", "md_set_deferred_status", "md_sync")
NOALLOC_MAX_ATOMS = 16384
PHASES = ("kick_drift", "rebuild", "pairs", "density", "force", "other", "grad")


class MDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 8), ("r_taper", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("knots", ctypes.POINTER(ctypes.c_double)), ("n_phi", ctypes.c_int),
                ("n_f", ctypes.c_int), ("n_F", ctypes.c_int), ("r_lo", ctypes.c_double), ("r_hi", ctypes.c_double),
                ("rho_lo", ctypes.c_double), ("rho_hi", ctypes.c_double), ("n_types", ctypes.c_int)]


class Config(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("skin", ctypes.c_double), ("dt", ctypes.c_double),
                ("mass", ctypes.c_double), ("precision", ctypes.c_int), ("max_neighbors", ctypes.c_int)]


class Thermo(ctypes.Structure):
    _fields_ = [("ke", ctypes.c_double), ("pe", ctypes.c_double), ("etot", ctypes.c_double),
                ("temperature", ctypes.c_double), ("max_disp", ctypes.c_double), ("n_rebuild", ctypes.c_int64),
                ("step", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double * len(PHASES)), ("timed", ctypes.c_int64 * len(PHASES))]


_lib = None


def load(path: str | pathlib.Path | None = None) -> ctypes.CDLL:
    """Loads libmd.so (raises OSError if it is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = pathlib.Path(path) if path else LIB_PATH
    if not p.exists():
        raise OSError(f"{p} is missing: build it with paper_1212_6332_gb300.build.build()")
    lib = ctypes.CDLL(str(p))
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "md_create": [P(Config), P(Potential), i64, P(vp)],
        "md_destroy": [vp],
        "md_set_state": [vp, dp, dp, vp],
        "md_get_state": [vp, dp, dp, vp],
        "md_build_neighbors": [vp, vp],
        "md_get_neighbors": [vp, dp, dp, ctypes.c_int32, vp],
        "md_max_count": [vp, P(ctypes.c_int32)],
        "md_compute_forces": [vp, dp, dp, dp, dp, dp, vp],
        "md_get_forces": [vp, dp, dp, dp, vp],
        "md_step": [vp, i32, P(Thermo), dp, i32, vp],
        "md_get_thermo": [vp, P(Thermo), vp],
        "md_batch_create": [P(Config), P(Potential), i32, dp, dp, P(vp)],
        "md_batch_destroy": [vp],
        "md_batch_set_state": [vp, dp, dp, vp],
        "md_batch_get_state": [vp, dp, dp, vp],
        "md_batch_compute_forces": [vp, dp, dp, dp, vp],
        "md_batch_step": [vp, i32, i32, i32, dp, vp],
        "md_batch_set_potential": [vp, P(Potential), vp],
        "md_set_thermostat": [vp, ctypes.c_double, ctypes.c_double],
        "md_set_newton3": [vp, ctypes.c_int],
        "md_set_deferred_status": [vp, ctypes.c_int],
        "md_sync": [vp, vp],
        "md_set_types": [vp, vp, vp],
        "md_pressure": [vp, vp, vp],
        "md_set_barostat": [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double],
        "md_get_box": [vp, vp, vp],
        "md_param_grad": [vp, dp, dp, dp, vp],
        "md_num_params": [vp],
        "md_status_string": [i32],
        "md_last_error": [vp],
        "md_profile_start": [vp, i32],
        "md_profile_read": [vp, P(Profile)],
        "md_eval_math": [vp, i32, dp, i64, dp, vp],
        "md_forces_noalloc": [P(Potential), dp, i64, dp, dp, dp, dp, vp],
        "md_batch_thermo": [vp, dp, vp],
        "md_batch_schedule": [vp, P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double)],
        "md_fma_probe": [i32, i64, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int), vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.md_status_string.restype = ctypes.c_char_p
    lib.md_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = lib
    return lib


def potential_struct(spec: dict) -> tuple[Potential, object]:
    """md_potential from a dict (see paper_1212_6332_gb300.inputs for the keys).
    Returns the struct and an object that keeps the knot array alive."""
    P = Potential()
    keep = None
    kind = spec["kind"]
    if kind == "rgl":
        P.kind = POT_RGL
        vals = [spec[k] for k in ("A", "xi", "p", "q", "r0")]
    elif kind == "sc":
        P.kind = POT_SC
        vals = [spec[k] for k in ("eps", "c", "a", "n", "m")]
    elif kind == "alloy":
        # several species: V^(ab), rho^(ab) per type pair (row-major upper
        # triangle), F^(a) per type, on shared grids
        P.kind = POT_SPLINE
        vals = []
        T = int(spec["n_types"])
        tabs = [np.asarray(a, dtype=np.float64) for key in ("phi", "f", "F") for a in spec[key]]
        if len(spec["phi"]) != T * (T + 1) // 2 or len(spec["f"]) != len(spec["phi"]) or len(spec["F"]) != T:
            raise ValueError("alloy: T(T+1)/2 pair tables and T embedding tables")
        knots = np.ascontiguousarray(np.concatenate(tabs))
        keep = knots
        P.knots = knots.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        P.n_phi, P.n_f, P.n_F = len(spec["phi"][0]), len(spec["f"][0]), len(spec["F"][0])
        P.r_lo, P.r_hi = float(spec["r_lo"]), float(spec["r_hi"])
        P.rho_lo, P.rho_hi = float(spec["rho_lo"]), float(spec["rho_hi"])
        P.n_types = T
    elif kind == "spline":
        P.kind = POT_SPLINE
        vals = []
        knots = np.ascontiguousarray(np.concatenate([np.asarray(spec[k], dtype=np.float64)
                                                     for k in ("phi", "f", "F")]))
        keep = knots
        P.knots = knots.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        P.n_phi, P.n_f, P.n_F = len(spec["phi"]), len(spec["f"]), len(spec["F"])
        P.r_lo, P.r_hi = float(spec["r_lo"]), float(spec["r_hi"])
        P.rho_lo, P.rho_hi = float(spec["rho_lo"]), float(spec["rho_hi"])
    else:
        raise ValueError(f"unknown potential kind {kind!r}")
    for k, v in enumerate(vals):
        P.p[k] = float(v)
    P.r_taper = float(spec.get("r_taper", spec.get("r_hi", 0.0)))
    P.r_cut = float(spec.get("r_cut", spec.get("r_hi", 0.0)))
    return P, keep


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a):
    """Pointer of a torch tensor (device or host) or numpy array (host); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 and a.dtype != np.int32:
            raise TypeError("arrays must be float64 (or int32 for lists)")
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(a.data_ptr())


class System:
    """A single periodic box or a batch of independent boxes on one GPU.

    Single box: ``System(pot, box=[Lx, Ly, Lz], n_atoms=N, ...)``.
    Batch:      ``System(pot, boxes=[[Lx, Ly, Lz], ...], atom_offsets=[0, n0, n0+n1, ...], ...)``.
    Arrays are [N, 3] float64 in the caller's atom order; torch CUDA tensors
    are passed by device pointer, numpy arrays and CPU tensors by host pointer.
    """

    def __init__(self, potential: dict, *, box=None, n_atoms: int | None = None, boxes=None, atom_offsets=None,
                 skin: float = 0.3, dt: float = 1.0, mass: float = 63.546, precision: str = "fp64",
                 max_neighbors: int = 0):
        self.lib = load()
        self._h = ctypes.c_void_p()
        cfg = Config()
        cfg.skin, cfg.dt, cfg.mass = float(skin), float(dt), float(mass)
        cfg.precision = {"fp64": FP64, "mixed": MIXED}[precision]
        cfg.max_neighbors = int(max_neighbors)
        self.precision = precision
        pot, self._keep = potential_struct(potential)
        if boxes is None:
            cfg.box[:] = [float(b) for b in box]
            self.n_boxes = 1
            self.n = int(n_atoms)
            self.boxes = np.asarray([box], dtype=np.float64).reshape(1, 3)
            self.atom_offsets = np.array([0, self.n], dtype=np.int64)
            rc = self.lib.md_create(ctypes.byref(cfg), ctypes.byref(pot), self.n, ctypes.byref(self._h))
        else:
            self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
            self.atom_offsets = np.ascontiguousarray(atom_offsets, dtype=np.int64)
            self.n_boxes = self.boxes.shape[0]
            self.n = int(self.atom_offsets[-1])
            rc = self.lib.md_batch_create(ctypes.byref(cfg), ctypes.byref(pot), self.n_boxes,
                                          ctypes.c_void_p(self.atom_offsets.ctypes.data),
                                          ctypes.c_void_p(self.boxes.ctypes.data), ctypes.byref(self._h))
        if rc != 0:
            raise MDError(rc, self.lib.md_last_error(None).decode())
        self.potential = dict(potential)

    # ------------------------------------------------------------ plumbing
    def _check(self, rc: int):
        if rc != 0:
            raise MDError(rc, self.lib.md_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.md_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape, dtype=None):
        torch = _torch()
        return torch.empty(*shape, dtype=dtype or torch.float64, device="cuda")

    # ------------------------------------------------------------ state
    def set_state(self, x, v=None):
        self._check(self.lib.md_set_state(self._h, _ptr(x), _ptr(v), _stream()))

    def get_state(self, x_out=None, v_out=None):
        x = x_out if x_out is not None else self._empty(self.n, 3)
        v = v_out if v_out is not None else self._empty(self.n, 3)
        self._check(self.lib.md_get_state(self._h, _ptr(x), _ptr(v), _stream()))
        return x, v

    def compute_forces(self, x, f=None, e_atom=None, rho=None, energy=None):
        """Sets positions to x and returns forces, per-atom energies, densities and E_T."""
        f = f if f is not None else self._empty(self.n, 3)
        e_atom = e_atom if e_atom is not None else self._empty(self.n)
        rho = rho if rho is not None else self._empty(self.n)
        energy = energy if energy is not None else self._empty(1)
        self._check(self.lib.md_compute_forces(self._h, _ptr(x), _ptr(f), _ptr(e_atom), _ptr(rho), _ptr(energy),
                                               _stream()))
        return dict(f=f, e_atom=e_atom, rho=rho, energy=energy)

    def get_forces(self, f: bool = True, e_atom: bool = True, rho: bool = True):
        """Forces, per-atom energies and densities of the current state (the
        ones not asked for are not copied)."""
        fo = self._empty(self.n, 3) if f else None
        e = self._empty(self.n) if e_atom else None
        r = self._empty(self.n) if rho else None
        self._check(self.lib.md_get_forces(self._h, _ptr(fo), _ptr(e), _ptr(r), _stream()))
        return dict(f=fo, e_atom=e, rho=r)

    def build_neighbors(self):
        self._check(self.lib.md_build_neighbors(self._h, _stream()))

    def max_count(self) -> int:
        out = ctypes.c_int32()
        self._check(self.lib.md_max_count(self._h, ctypes.byref(out)))
        return out.value

    def neighbors(self):
        """(nn [N], nl [N, ld]) int32 CUDA tensors in caller ids."""
        torch = _torch()
        ld = max(1, self.max_count())
        nn = torch.zeros(self.n, dtype=torch.int32, device="cuda")
        nl = torch.full((self.n, ld), -1, dtype=torch.int32, device="cuda")
        self._check(self.lib.md_get_neighbors(self._h, _ptr(nn), _ptr(nl), ld, _stream()))
        return nn, nl

    # ------------------------------------------------------------ dynamics
    def step(self, n: int, history: bool = False, use_graph: bool = False):
        th = Thermo()
        hist = self._empty(max(n, 1), 4) if history else None
        self._check(self.lib.md_step(self._h, int(n), ctypes.byref(th), _ptr(hist), int(use_graph), _stream()))
        out = th.as_dict()
        if history:
            out["history"] = hist[:n]
        return out

    def thermo(self) -> dict:
        th = Thermo()
        self._check(self.lib.md_get_thermo(self._h, ctypes.byref(th), _stream()))
        return th.as_dict()

    # ------------------------------------------------------------ batches
    def batch_compute_forces(self, x, f=None, e_box=None):
        f = f if f is not None else self._empty(self.n, 3)
        e_box = e_box if e_box is not None else self._empty(self.n_boxes)
        self._check(self.lib.md_batch_compute_forces(self._h, _ptr(x), _ptr(f), _ptr(e_box), _stream()))
        return f, e_box

    def batch_step(self, n: int, schedule: str = "auto", use_graph: bool = False, per_box: bool = True):
        sched = {"auto": SCHED_AUTO, "box": SCHED_BOX, "tile": SCHED_TILE}[schedule]
        tb = self._empty(self.n_boxes, 4) if per_box else None
        self._check(self.lib.md_batch_step(self._h, int(n), sched, int(use_graph), _ptr(tb), _stream()))
        return tb

    def schedule(self) -> dict:
        """The autotuner's pick ("tile", "box" or None) and its timings (ms/step)."""
        c, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.md_batch_schedule(self._h, ctypes.byref(c), ctypes.byref(a), ctypes.byref(b)))
        return dict(choice={0: None, SCHED_BOX: "box", SCHED_TILE: "tile"}[c.value], ms_tile=a.value,
                    ms_box=b.value)

    def batch_thermo(self):
        """[n_boxes, 4] (ke, pe, etot, T) of the current state (CUDA tensor)."""
        tb = self._empty(self.n_boxes, 4)
        self._check(self.lib.md_batch_thermo(self._h, _ptr(tb), _stream()))
        return tb

    def set_potential(self, spec: dict):
        pot, keep = potential_struct(spec)
        self._check(self.lib.md_batch_set_potential(self._h, ctypes.byref(pot), _stream()))
        self._keep = keep
        self.potential = dict(spec)

    def set_types(self, types):
        """Species of every atom in caller order (numpy array or CUDA
        tensor of int32), for a potential with several species."""
        import numpy as np
        if hasattr(types, "data_ptr"):
            t = types.to(dtype=__import__("torch").int32).contiguous()
            self._check(self.lib.md_set_types(self._h, ctypes.c_void_p(t.data_ptr()), _stream()))
        else:
            t = np.ascontiguousarray(types, dtype=np.int32)
            self._check(self.lib.md_set_types(self._h, t.ctypes.data_as(ctypes.c_void_p), _stream()))

    def pressure(self):
        """Instantaneous pressure of Eq. (6) of every box (eV/A^3), a device
        tensor of one value per box."""
        out = self._empty(self.n_boxes)
        self._check(self.lib.md_pressure(self._h, _ptr(out), _stream()))
        return out

    def set_barostat(self, P0: float, tau_p: float, beta: float):
        """Berendsen coupling of Eq. (5) towards P0 (eV/A^3) with time
        constant tau_p (fs) and compressibility beta (A^3/eV); tau_p <= 0
        turns it off."""
        self._check(self.lib.md_set_barostat(self._h, float(P0), float(tau_p), float(beta)))

    def box(self):
        """Current box lengths, [n_boxes][3] numpy array (A)."""
        import numpy as np
        out = np.zeros((self.n_boxes, 3))
        self._check(self.lib.md_get_box(self._h, out.ctypes.data_as(ctypes.c_void_p), _stream()))
        return out

    def set_thermostat(self, T_e: float, tau_T: float):
        """Electron-phonon friction of Eq. (4) towards T_e (K) with time
        constant tau_T (fs) in the following steps; tau_T <= 0 turns it off."""
        self._check(self.lib.md_set_thermostat(self._h, float(T_e), float(tau_T)))

    def set_deferred_status(self, on: bool = True):
        """md_set_deferred_status: get_forces, batch_thermo, set_potential and
        param_grad return without waiting for the device status word; a
        condition their kernels raise is reported by the next call that
        waits (sync(), step(), get_state(), ...)."""
        self._check(self.lib.md_set_deferred_status(self._h, int(bool(on))))

    def sync(self):
        """md_sync: waits for the stream and raises MDError for a pending
        device condition."""
        self._check(self.lib.md_sync(self._h, _stream()))

    def set_newton3(self, on: bool = True):
        """Float64 density and force sums over the upper half of each list
        with Newton's third law (atomic partner updates; agrees with the
        default full-list sums to rounding, not bit for bit)."""
        self._check(self.lib.md_set_newton3(self._h, int(bool(on))))

    @property
    def n_params(self) -> int:
        return self.lib.md_num_params(self._h)

    def profile_start(self, timing: bool = False):
        self._check(self.lib.md_profile_start(self._h, int(timing)))

    def profile_read(self) -> dict:
        p = Profile()
        self._check(self.lib.md_profile_read(self._h, ctypes.byref(p)))
        return dict(launches=p.launches, ms={PHASES[k]: p.ms[k] for k in range(len(PHASES))},
                    timed={PHASES[k]: p.timed[k] for k in range(len(PHASES))})

    def eval_math(self, fn: str, x):
        """The library's float64 functions on a CUDA tensor: fn in
        {"exp", "exp_ref", "rsqrt", "rsqrt_ref", "rsqrt_int", "sqrt_int"}."""
        code = {"exp": 0, "exp_ref": 1, "rsqrt": 2, "rsqrt_ref": 3, "rsqrt_int": 4, "sqrt_int": 5}[fn]
        x = x.contiguous()
        out = self._empty(x.numel())
        self._check(self.lib.md_eval_math(self._h, code, _ptr(x), x.numel(), _ptr(out), _stream()))
        return out

    def param_grad(self, g_f, g_e, grad=None):
        grad = grad if grad is not None else self._empty(self.n_params)
        self._check(self.lib.md_param_grad(self._h, _ptr(g_f), _ptr(g_e), _ptr(grad), _stream()))
        return grad


def fma_probe(precision: str = "fp64", iters: int = 1024) -> dict:
    """md_fma_probe: the device's measured FMA rate (flop/s), the launch time
    (ms) and the multiprocessor count, on the current stream."""
    lib = load()
    fl, ms, n_sm = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    rc = lib.md_fma_probe({"fp64": 0, "fp32": 1}[precision], int(iters), ctypes.byref(fl), ctypes.byref(ms),
                          ctypes.byref(n_sm), _stream())
    if rc != 0:
        raise MDError(rc, "md_fma_probe failed")
    return dict(flops=fl.value, ms=ms.value, n_sm=n_sm.value, iters=int(iters))


def forces_noalloc(potential: dict, box, x, f=None, e_atom=None, e_total=None):
    """md_forces_noalloc: forces of one small box (at most NOALLOC_MAX_ATOMS
    atoms) with no device allocation inside the library. x is a [n, 3]
    float64 CUDA tensor; outputs are CUDA tensors (allocated here by torch
    unless given)."""
    torch = _torch()
    lib = load()
    n = x.shape[0]
    f = f if f is not None else torch.empty((n, 3), dtype=torch.float64, device=x.device)
    e_atom = e_atom if e_atom is not None else torch.empty(n, dtype=torch.float64, device=x.device)
    e_total = e_total if e_total is not None else torch.empty(1, dtype=torch.float64, device=x.device)
    pot, keep = potential_struct(potential)
    b = np.ascontiguousarray(box, dtype=np.float64)
    rc = lib.md_forces_noalloc(ctypes.byref(pot), ctypes.c_void_p(b.ctypes.data), n, _ptr(x), _ptr(f),
                               _ptr(e_atom), _ptr(e_total), _stream())
    if rc != 0:
        raise MDError(rc, "md_forces_noalloc failed")
    return dict(f=f, e_atom=e_atom, energy=e_total)
