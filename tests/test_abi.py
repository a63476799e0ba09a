"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tsfem.h and include/tsfem3.h declare (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols(header="tsfem.h", prefix="tsf_"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2103_17040_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    decl = _declared_symbols() + _declared_symbols("tsfem3.h", "tsf3_")
    assert len(decl) >= 30
    missing = [s for s in decl if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_mirrors_header():
    import paper_2103_17040_gb300 as T
    decl = _declared_symbols()
    assert sorted(T.EXPORTS) == decl
    decl3 = _declared_symbols("tsfem3.h", "tsf3_")
    assert sorted(T.EXPORTS3) == decl3
    for s in decl + decl3:
        assert callable(getattr(T, s)), s


def test_host_only_calls_without_device():
    """Calls that touch no device: version and default options."""
    import paper_2103_17040_gb300 as T
    T.load_library()
    assert T.tsf_version() >= 100
    o = T.tsf_default_options()
    assert o.precision == T.TSF_MIXED and o.cg_tol == 1e-8 and o.use_graph == 1


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2103_17040_gb300.binding as b
    saved = b._lib
    try:
        b._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            b.load_library(str(tmp_path / "missing.so"))
    finally:
        b._lib = saved


def test_options_struct_layout_matches_header():
    """ctypes layouts of tsf_options / tsf_stats match the C compiler's."""
    import subprocess
    import paper_2103_17040_gb300 as T
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "tsfem3.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(tsf_options), offsetof(tsf_options, cuda_stream),
         offsetof(tsf_options, coupling), sizeof(tsf_stats), offsetof(tsf_stats, coupling_change),
         offsetof(tsf_stats, steps), sizeof(tsf3_stats), offsetof(tsf3_stats, tiling),
         offsetof(tsf3_stats, total_ms), offsetof(tsf3_stats, band_rhs));
  return 0;
}'''
    src = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"tsf_layout_{os.getpid()}.c")
    exe = src[:-2]
    open(src, "w").write(prog)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    os.remove(src)
    os.remove(exe)
    exp = [ctypes.sizeof(T.tsf_options), T.tsf_options.cuda_stream.offset, T.tsf_options.coupling.offset,
           ctypes.sizeof(T.tsf_stats), T.tsf_stats.coupling_change.offset, T.tsf_stats.steps.offset,
           ctypes.sizeof(T.tsf3_stats), T.tsf3_stats.tiling.offset, T.tsf3_stats.total_ms.offset,
           T.tsf3_stats.band_rhs.offset]
    assert [int(x) for x in out] == exp
