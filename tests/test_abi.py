"""Host-side checks of the C ABI: the library builds and loads, exports every
symbol that include/*.h declares, and rejects invalid arguments before any GPU
work (no compute call is made here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_12872_gb300 import build, dpt
    build.build()
    return dpt.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"DPT_API\s+[\w\s\*]*?\b(dpt_\w+)\s*\(", open(h).read()):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dpt_solve_full" in names
    for nm in names:
        assert hasattr(lib, nm), nm


def test_defaults_and_status_strings(lib):
    from paper_2002_12872_gb300 import dpt
    o = dpt.options()
    assert o.tol == 1e-12 and o.max_iter == 200 and o.prec == 1 and o.max_slices == 3
    assert o.cta_pair == 1
    assert dpt.status_string(-2) == "DPT_ERR_DEGENERATE"
    assert dpt.status_string(0) == "DPT_OK"


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2002_12872_gb300 import dpt
    info = dpt.Info()
    th = np.zeros(4)
    d = np.zeros((4, 4), order="F")
    A = np.zeros((4, 4), order="F")
    E = np.zeros(4)
    p = lambda a: a.ctypes.data
    o = dpt.options()
    # n < 1
    assert lib.dpt_solve_full(0, 0, p(th), p(d), 4, 0.1, ctypes.byref(o), p(A), 4, p(E),
                              ctypes.byref(info), None) == -1
    # ld_delta < n
    assert lib.dpt_solve_full(4, 0, p(th), p(d), 3, 0.1, ctypes.byref(o), p(A), 4, p(E),
                              ctypes.byref(info), None) == -1
    # null pointers
    assert lib.dpt_solve_full(4, 0, None, p(d), 4, 0.1, ctypes.byref(o), p(A), 4, p(E),
                              ctypes.byref(info), None) == -1
    # bad option values
    o2 = dpt.options(max_slices=4)
    assert lib.dpt_solve_full(4, 0, p(th), p(d), 4, 0.1, ctypes.byref(o2), p(A), 4, p(E),
                              ctypes.byref(info), None) == -1
    assert info.status == -1
    # dense dominant form: n < 1, ld_delta < n, nstar >= n, non-finite lambda
    z = np.zeros(4)
    Eo = np.zeros(1)
    dd = lib.dpt_solve_dominant_dense
    assert dd(0, p(th), p(d), 4, -1, 0.1, ctypes.byref(o), p(z), p(Eo),
              ctypes.byref(info), None) == -1
    assert dd(4, p(th), p(d), 3, -1, 0.1, ctypes.byref(o), p(z), p(Eo),
              ctypes.byref(info), None) == -1
    assert dd(4, p(th), p(d), 4, 4, 0.1, ctypes.byref(o), p(z), p(Eo),
              ctypes.byref(info), None) == -1
    assert dd(4, p(th), p(d), 4, -1, float("nan"), ctypes.byref(o), p(z), p(Eo),
              ctypes.byref(info), None) == -1
    assert info.status == -1 and info.nstar == -1
    # plain FP64 beyond 65535: refused before any work
    o64 = dpt.options(prec="fp64")
    assert lib.dpt_solve_full(70000, 0, p(th), p(d), 70000, 0.1, ctypes.byref(o64), p(A), 70000,
                              p(E), ctypes.byref(info), None) == -9
    # homotopy: stages outside 1..1024, n < 1, ld_a < n
    hs = lib.dpt_solve_homotopy
    for args in ((4, 0), (4, 1025), (0, 2)):
        nn, Q = args
        assert hs(nn, p(th), p(d), 4, 0.1, Q, ctypes.byref(o), p(A), 4, p(E),
                  ctypes.byref(info), None) == -1
    assert hs(4, p(th), p(d), 4, 0.1, 2, ctypes.byref(o), p(A), 3, p(E),
              ctypes.byref(info), None) == -1


def test_tuner_arguments_rejected_without_gpu(lib):
    """dpt_tune_batched validates like dpt_solve_batched and stops at the first
    argument error, before any CUDA call."""
    from paper_2002_12872_gb300 import dpt
    th, d, A, E = np.zeros(4), np.zeros((4, 4), order="F"), np.zeros((4, 4), order="F"), np.zeros(4)
    P = ctypes.c_void_p
    n = (ctypes.c_int64 * 1)(4)
    ths, ds, As, Es = ((P * 1)(x.ctypes.data) for x in (th, d, A, E))
    ld = (ctypes.c_int64 * 1)(4)
    lam = (ctypes.c_double * 1)(0.1)
    o = dpt.options()
    best = ctypes.c_int32(7)
    ms = (ctypes.c_double * 3)(5.0, 5.0, 5.0)
    tb = lib.dpt_tune_batched
    assert tb(0, 0, n, ths, ds, ld, lam, ctypes.byref(o), As, ld, Es, ctypes.byref(best), ms,
              None) == -1
    assert tb(1, 0, n, ths, ds, ld, lam, ctypes.byref(o), As, ld, Es, None, ms, None) == -1
    n0 = (ctypes.c_int64 * 1)(0)
    assert tb(1, 0, n0, ths, ds, ld, lam, ctypes.byref(o), As, ld, Es, ctypes.byref(best), ms,
              None) == -1
    assert best.value == 0 and ms[0] == -1.0


def test_selftest_and_server_arguments_rejected_without_gpu(lib):
    from paper_2002_12872_gb300 import dpt
    assert lib.dpt_selftest_bounded_wait(0.0, None) == -1
    assert lib.dpt_selftest_bounded_wait(10.0, None) == -1
    cfg = dpt.ServerCfg()
    lib.dpt_server_cfg_default(ctypes.byref(cfg))
    assert cfg.max_active == 64 and cfg.max_queue == 65536 and cfg.opt.tol == 1e-12
    h = ctypes.c_void_p()
    bad = dpt.ServerCfg()
    lib.dpt_server_cfg_default(ctypes.byref(bad))
    bad.max_active = 0
    assert lib.dpt_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.max_active = 8
    bad.opt.prec = 0                       # the server runs the mixed path only
    assert lib.dpt_server_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert lib.dpt_submit(None, None, None) == -1
    assert lib.dpt_poll(None, 1, None) == -1
    assert lib.dpt_server_destroy(None) == -1


def test_workspace_bytes_without_gpu(lib):
    """dpt_workspace_bytes is host arithmetic over the solves' carve layouts: about
    30 B per element for the mixed real solve (room for three FP16 slices 6,
    float-float A and its copy 16, FP16 increments 4, remainder 4), 3 n^2 doubles per
    real component for
    the FP64 map, and -1 outside its domain."""
    from paper_2002_12872_gb300 import dpt
    for n in (256, 4096, 8192):
        nn = float(n) * n
        assert 30.0 <= dpt.workspace_bytes(n) / nn <= 30.5
        assert 24.0 <= dpt.workspace_bytes(n, prec="fp64") / nn <= 24.2
        assert 48.0 <= dpt.workspace_bytes(n, True, "fp64") / nn <= 48.2
        # complex mixed: staging copies of Delta and A (32 B) plus the grouped solve
        assert 100.0 <= dpt.workspace_bytes(n, True) / nn <= 110.0
    sizes = [dpt.workspace_bytes(n) for n in (1, 100, 1000, 5000)]
    assert sizes == sorted(sizes) and sizes[0] > 0
    assert lib.dpt_workspace_bytes(0, 0, 1) == -1
    assert lib.dpt_workspace_bytes((1 << 20) + 1, 0, 1) == -1
    assert lib.dpt_workspace_bytes(16, 7, 1) == -1
    assert lib.dpt_workspace_bytes(16, 0, 9) == -1


# ctypes mirrors of the header's structs (field names as in C but for `lambda`, a
# Python keyword)
_STRUCTS = [("Options", "dpt_options"), ("Info", "dpt_info"), ("ServerCfg", "dpt_server_cfg"),
            ("Problem", "dpt_problem"), ("ServerStats", "dpt_server_stats")]
_RENAME = {("Problem", "lam"): "lambda"}


def test_struct_layouts_match_the_header(tmp_path):
    """Every field of the binding's ctypes structs sits at the offset a C compiler
    gives it from include/dpt.h, and the sizes agree (a mismatch would make the
    library write past the binding's buffers)."""
    import shutil
    import subprocess
    from paper_2002_12872_gb300 import dpt
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpt.h"', 'int main(void) {']
    for py, c in _STRUCTS:
        lines.append(f'  printf("{py} . %zu\\n", sizeof({c}));')
        for f, _ in getattr(dpt, py)._fields_:
            cf = _RENAME.get((py, f), f)
            lines.append(f'  printf("{py} {f} %zu\\n", offsetof({c}, {cf}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(v) for a, b, v in (ln.split() for ln in out if ln.strip())}
    for py, _ in _STRUCTS:
        cls = getattr(dpt, py)
        assert got[(py, ".")] == ctypes.sizeof(cls), py
        for f, _ in cls._fields_:
            assert got[(py, f)] == getattr(cls, f).offset, (py, f)
