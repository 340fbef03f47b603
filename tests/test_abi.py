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


def test_headers_compile_as_c_and_a_c_program_drives_the_host_entry_points(lib, tmp_path):
    # the boundary is a C ABI: the public headers compile as strict C11 and a
    # C program linked against the library runs its host-only entry points
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include "comet.h"
#include "comet_proposal.h"
#include "comet_mcts.h"
int main(void) {
    comet_mode_seq q = {0};
    q.len = 2; q.modes[0] = 11; q.modes[1] = 3;
    comet_mcts_opts o;
    comet_mcts* t = NULL;
    comet_mode_seq pool[64];
    float cost[64], viol[64];
    int64_t n = 0, total = 0;
    comet_mcts_stats st;
    if (comet_mcts_default_opts(&o) != COMET_OK) return 2;
    o.n_modes = 3; o.l_max = 3; o.seed = 5;
    if (comet_mcts_create(&o, &t) != COMET_OK) return 3;
    for (;;) {
        if (comet_mcts_ask(t, 0, 8, pool, &n) != COMET_OK) return 4;
        if (n == 0) break;
        for (int64_t i = 0; i < n; ++i) { cost[i] = 1.0f + (float)pool[i].len; viol[i] = 0.0f; }
        if (comet_mcts_tell(t, cost, viol, n) != COMET_OK) return 5;
        total += n;
    }
    comet_mcts_get_stats(t, &st);
    printf("%llu %lld %lld %d\n", (unsigned long long)comet_mode_code(&q, 12), (long long)total,
           (long long)st.evaluations, st.exhausted);
    comet_mcts_destroy(t);
    return comet_mcts_ask(NULL, 0, 1, pool, &n) == COMET_ERR_INVALID_ARG ? 0 : 6;
}
""")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(P.lib_path())
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src), "-o", str(exe),
                    "-L", libdir, "-lcomet", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    # every order of 1..3 segments over 3 modes (3 + 9 + 27) is evaluated once
    assert out == [str(S.encode((11, 3), 12)), "39", "39", "1"]
