"""The C-ABI library loads and exports every entry point include/lbsph.h declares;
host-only entry points behave (no GPU compute is issued here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2403_05443_gb300 import build as B
from paper_2403_05443_gb300 import lbsph as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_python_binding_has_the_same_names():
    from paper_2403_05443_gb300 import surrogate as SU
    for n in _declared():
        assert hasattr(L, n) or hasattr(SU, n), n


def test_abi_version_and_status_strings():
    assert L.lb_abi_version() == 5
    assert L.lb_status_string(0) == "ok"
    assert L.lb_status_string(1) == "invalid argument"
    assert L.lb_status_string(99) == "unknown status"


def test_lattice_table_is_d3q19():
    """Same velocity set and weights as the oracle's (compared as vectors: the two
    sides use different direction orders)."""
    from oracle import oracle as O
    c, w = L.lb_lattice()
    co, wo = O.lattice()
    mine = {tuple(v): wi for v, wi in zip(c.tolist(), w)}
    theirs = {tuple(v): wi for v, wi in zip(co.tolist(), wo)}
    assert mine == theirs
    # opposite directions are adjacent pairs (1,2), (3,4), ...
    for i in range(1, 19, 2):
        assert (c[i] == -c[i + 1]).all()


def test_lattice_tables_of_both_lattices():
    """lb_lattice_q(27) against the oracle's D3Q27 (as vectors), its first 19
    directions are the D3Q19 table in the same order, opposite directions are
    adjacent pairs; other lattices are refused."""
    from oracle import oracle as O
    c19, w19 = L.lb_lattice()
    c, w = L.lb_lattice_q(19)
    assert (c == c19).all() and (w == w19).all()
    c, w = L.lb_lattice_q(27)
    co, wo = O.lattice(27)
    assert {tuple(v): wi for v, wi in zip(c.tolist(), w)} == {tuple(v): wi for v, wi in zip(co.tolist(), wo)}
    assert (c[:19] == c19).all()
    for i in range(1, 27, 2):
        assert (c[i] == -c[i + 1]).all()
    with pytest.raises(L.LBError):
        L.lb_lattice_q(15)


def test_create_rejects_bad_d3q27_options_without_touching_the_gpu():
    """D3Q27 takes FP32 storage and periodic boxes; an unknown lattice or
    collision is refused."""
    b = {"nx": 32, "ny": 32, "nz": 32, "tau": 1.0}
    for kw in ({"lattice": 27, "precision": L.LB_BF16}, {"lattice": 27, "precision": L.LB_FP16},
               {"lattice": 27, "collision": 2}, {"lattice": 21}):
        opt = L.Options()
        opt.max_semi, opt.max_particles = 8, 4
        for k, v in kw.items():
            setattr(opt, k, v)
        with pytest.raises(L.LBError) as e:
            L.lb_create([b], opt)
        assert e.value.status == 1


def test_create_rejects_bad_boxes_without_touching_the_gpu():
    opt = L.Options()
    opt.max_semi, opt.max_particles = 8, 4
    for bad in ({"nx": 30, "ny": 32, "nz": 32, "tau": 1.0},     # nx not a multiple of 4
                {"nx": 32, "ny": 32, "nz": 32, "tau": 0.5},     # tau must exceed 1/2
                {"nx": 32, "ny": 2, "nz": 32, "tau": 1.0},
                {"nx": 32, "ny": 32, "nz": 32, "tau": 1.0, "rho0": 0.0}):
        with pytest.raises(L.LBError) as e:
            L.lb_create([bad], opt)
        assert e.value.status == 1
    with pytest.raises(L.LBError):
        L.lb_create([], opt)


def test_header_record_layout():
    text = open(os.path.join(ROOT, "include", "lbsph.h")).read()
    assert "#define LB_RECORD_DOUBLES 25" in text
    assert L.LB_RECORD_DOUBLES == 25
