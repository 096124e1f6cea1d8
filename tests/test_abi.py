"""The C-ABI library builds, loads and exports every symbol include/md.h
declares; argument errors are rejected on the host before any CUDA call (so
these run without a GPU)."""
import ctypes
import pathlib
import re

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_1212_6332_gb300 import build
    build.build()
    from paper_1212_6332_gb300 import md
    return md.load()


def declared_symbols():
    text = (ROOT / "include" / "md.h").read_text()
    return sorted(set(re.findall(r"^MD_API\s+[\w\s\*]+?\b(md_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("md_create", "md_build_neighbors", "md_compute_forces", "md_step", "md_batch_step",
                     "md_param_grad"):
        assert required in names


CITATION = re.compile(r"(Sec\.|Eq\.|Eqs\.|Fig\.|Table\s+\d)|no counterpart in\s+(the\s+)?paper|paper has no counterpart", re.S | re.I)


def declaration_comments():
    """(name, comment) for every MD_API declaration: the comment is the last
    block comment that starts a line before it (one comment may introduce
    several declarations that follow it)."""
    text = (ROOT / "include" / "md.h").read_text()
    out = []
    last_comment = ""
    for m in re.finditer(r"^/\*.*?\*/|^MD_API\s+[\w\s\*]+?\b(md_\w+)\s*\(", text, flags=re.M | re.S):
        if m.group(0).startswith("/*"):
            last_comment = re.sub(r"\s*\n\s*\*(?!/)\s?", " ", m.group(0))
        else:
            out.append((m.group(1), last_comment))
    return out


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    decls = declaration_comments()
    assert {n for n, _ in decls} == set(declared_symbols())
    missing = [n for n, c in decls if not CITATION.search(c)]
    assert not missing, f"declarations without a passage or 'no counterpart in the paper': {missing}"


def test_library_exports_every_declared_symbol(lib):
    from paper_1212_6332_gb300 import md
    names = declared_symbols()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(md.SYMBOLS) == names


def test_status_strings(lib):
    assert lib.md_status_string(0) == b"ok"
    assert lib.md_status_string(4) == b"neighbour list overflow"
    assert lib.md_status_string(99) == b"unknown status"


def _create(lib, box, skin=0.3, pot_over=None, n=10, **cfg_over):
    from paper_1212_6332_gb300 import inputs as I
    from paper_1212_6332_gb300 import md
    spec = dict(I.RGL_CU)
    spec.update(pot_over or {})
    pot, keep = md.potential_struct(spec)
    cfg = md.Config()
    cfg.box[:] = box
    cfg.skin, cfg.dt, cfg.mass = skin, 1.0, I.MASS_CU
    for k, v in cfg_over.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = lib.md_create(ctypes.byref(cfg), ctypes.byref(pot), n, ctypes.byref(h))
    return rc, lib.md_last_error(None).decode()


def test_box_below_twice_the_list_radius_is_rejected(lib):
    rc, msg = _create(lib, [10.0, 10.0, 10.0])  # r_cut + skin = 5.3 >= L/2 = 5
    assert rc == 1 and "half of every box length" in msg


@pytest.mark.parametrize("over,cfg,needle", [
    ({"r0": 0.0}, {}, "r0"),
    ({"r_cut": float("nan")}, {}, "r_cut"),
    ({}, {"mass": 0.0}, "mass"),
    ({}, {"precision": 7}, "precision"),
    ({}, {"max_neighbors": -1}, "max_neighbors"),
    ({}, {"skin": -0.1}, "skin"),
])
def test_invalid_arguments_are_rejected(lib, over, cfg, needle):
    rc, msg = _create(lib, [30.0, 30.0, 30.0], pot_over=over, **cfg)
    assert rc == 1 and needle in msg


def test_negative_atom_count_and_null_handles(lib):
    rc, msg = _create(lib, [30.0, 30.0, 30.0], n=-1)
    assert rc == 1
    assert lib.md_destroy(None) == 1
    assert lib.md_step(None, 1, None, None, 0, None) == 1
    assert lib.md_num_params(None) == -1
    assert lib.md_set_thermostat(None, 300.0, 100.0) == 1
    assert lib.md_set_barostat(None, 0.0, 100.0, 1.0) == 1
    assert lib.md_pressure(None, None, None) == 1
    assert lib.md_get_box(None, None, None) == 1
    assert lib.md_set_types(None, None, None) == 1
    assert lib.md_set_newton3(None, 1) == 1


def test_batch_offsets_must_not_decrease(lib):
    import numpy as np
    from paper_1212_6332_gb300 import inputs as I
    from paper_1212_6332_gb300 import md
    pot, keep = md.potential_struct(I.RGL_CU)
    cfg = md.Config()
    cfg.skin, cfg.dt, cfg.mass = 0.3, 1.0, I.MASS_CU
    offs = np.array([0, 10, 5], dtype=np.int64)
    boxes = np.full((2, 3), 30.0)
    h = ctypes.c_void_p()
    rc = lib.md_batch_create(ctypes.byref(cfg), ctypes.byref(pot), 2, ctypes.c_void_p(offs.ctypes.data),
                             ctypes.c_void_p(boxes.ctypes.data), ctypes.byref(h))
    assert rc == 1 and "decrease" in lib.md_last_error(None).decode()


def test_fma_probe_rejects_bad_arguments_before_any_cuda_call(lib):
    d, m, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    assert lib.md_fma_probe(2, 16, ctypes.byref(d), ctypes.byref(m), ctypes.byref(n), None) == 1
    assert lib.md_fma_probe(0, 0, ctypes.byref(d), ctypes.byref(m), ctypes.byref(n), None) == 1
    assert lib.md_fma_probe(1, 16, None, ctypes.byref(m), ctypes.byref(n), None) == 1
