"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; host-only argument checks work without a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(gcmg_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1111_0983_gb300 import build, gcmg
    build.build()
    return gcmg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_host_only(lib):
    from paper_1111_0983_gb300 import gcmg
    p = gcmg.default_params(2, 4097, 33)
    assert (p.nu1, p.nu2, p.lam, p.gamma) == (2, 1, 5, 1)
    assert p.delta_over_h == 3.0 and p.c_dirichlet == 0.9 and p.rtol == 1e-10


def test_create_rejects_bad_arguments_without_gpu(lib):
    from paper_1111_0983_gb300 import gcmg
    h = C.c_void_p()
    p = gcmg.default_params(2, 65, 17)
    assert lib.gcmg_create(C.byref(p), None, None, C.byref(h)) == gcmg.GCMG_E_ARG
    assert lib.gcmg_create(None, None, None, C.byref(h)) == gcmg.GCMG_E_ARG
    assert lib.gcmg_create(C.byref(p), None, None, None) == gcmg.GCMG_E_ARG
    assert not h.value
    assert lib.gcmg_num_levels(None) == 0
    assert lib.gcmg_last_error(None) == b"null context"


def test_oracle_builds_separately():
    import oracle
    path = oracle.build()
    assert os.path.exists(path) and "oracle" in os.path.basename(path)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of gcmg_params, gcmg_stats and gcmg_grid have the
    sizes and field offsets the C compiler gives the header's structs."""
    import subprocess
    from paper_1111_0983_gb300 import gcmg
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gcmg.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gcmg_params), sizeof(gcmg_stats), '
                   'sizeof(gcmg_grid), offsetof(gcmg_params, h), offsetof(gcmg_params, diverge_cycles), '
                   'offsetof(gcmg_stats, diverged)); return 0; }\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(gcmg.Params), C.sizeof(gcmg.Stats), C.sizeof(gcmg.Grid), gcmg.Params.h.offset,
            gcmg.Params.diverge_cycles.offset, gcmg.Stats.diverged.offset]
    assert got == want


def test_grid_and_divergence_defaults(lib):
    from paper_1111_0983_gb300 import gcmg
    p = gcmg.default_params(3, 513, 17)
    assert p.h == 0.0 and list(p.origin) == [-1.0, -1.0, -1.0] and p.diverge_cycles == 3


def test_create_grid_rejects_bad_grids_without_gpu(lib):
    from paper_1111_0983_gb300 import gcmg
    p = gcmg.default_params(2, 65, 17)
    h = C.c_void_p()
    g = gcmg.Grid()
    g.dim, g.h = 2, 0.03125
    g.n[0], g.n[1], g.n[2] = 65, 33, 1             # unequal axes
    dummy = C.c_void_p(16)                          # never dereferenced: the grid is rejected first
    assert lib.gcmg_create_grid(C.byref(g), dummy, C.byref(p), None, C.byref(h)) == gcmg.GCMG_E_ARG
    g.n[1], g.h = 65, -1.0                          # negative spacing
    assert lib.gcmg_create_grid(C.byref(g), dummy, C.byref(p), None, C.byref(h)) == gcmg.GCMG_E_ARG
    assert not h.value
    assert lib.gcmg_set_bc_types_from_mask(None, None) == gcmg.GCMG_E_ARG
    assert lib.gcmg_residual(None, None, None, None) == gcmg.GCMG_E_ARG


def test_set_max_cycles_rejects_bad_arguments_without_gpu(lib):
    from paper_1111_0983_gb300 import gcmg
    assert lib.gcmg_set_max_cycles(None, 5) == gcmg.GCMG_E_ARG
