"""The C-ABI library loads and exports every entry point include/comet.h
declares; host-only helpers behave (no GPU needed)."""
import os
import re

import pytest

import paper_2609_21803_gb300 as P
from oracle import search as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(comet_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2609_21803_gb300 import build as B
    B.build()
    return P.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "comet_eval_modes" in names and "comet_problem_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(P.EXPORTS) >= names


def test_default_opts(lib):
    o = P.comet_default_opts()
    assert o.max_iters == 300 and o.ref_iters == 1500
    assert o.eps_feas == 1e-5 and o.merit_mu == 100.0


def test_mode_code_matches_oracle_definition(lib):
    for s in [(0,), (11, 3), (4, 4, 7, 1), tuple(range(12)) + (0, 1, 2, 3)]:
        assert P.comet_mode_code(s) == S.encode(s, 12)
    assert P.comet_mode_code((12,)) == 0          # mode out of range
    # the 13-mode pushing alphabet (free motion = 12)
    for s in [(12,), (12, 0, 12, 9), (12, 3, 6, 12, 0)]:
        assert P.comet_mode_code(s, 13) == S.encode(s, 13)


def test_struct_layouts():
    import ctypes
    assert ctypes.sizeof(P.ModeSeq) == 40
    assert ctypes.sizeof(P.PlanOpts) == 4 * 4 + 8 + 4 * 4
    assert ctypes.sizeof(P.InstanceDesc) == 4 * 4 + 8 * 16
    assert ctypes.sizeof(P.SolverOpts) == 2 * 4 + 10 * 8 + 2 * 4 + 8
