"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/ftsp2.h declares, and the ctypes struct layouts
match the C compiler's."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ftsp2.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(ftsp2_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ftsp2_rescale", "ftsp2_density", "ftsp2_entropy", "ftsp2_train_coeffs"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = built.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    from paper_2605_08523_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings(built):
    for code in range(0, -9, -1):
        assert built.status_string(code) != "unknown status"


def test_struct_layouts_match_c(tmp_path):
    from paper_2605_08523_gb300 import _lib
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "ftsp2.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(ftsp2_instance), offsetof(ftsp2_instance, offset),
         offsetof(ftsp2_instance, mu), offsetof(ftsp2_instance, kT));
  printf("%zu %zu %zu %zu %zu\\n", sizeof(ftsp2_table), offsetof(ftsp2_table, beta0),
         offsetof(ftsp2_table, theta), offsetof(ftsp2_table, theta_entropy), offsetof(ftsp2_table, family));
  printf("%zu %zu %zu %zu\\n", sizeof(ftsp2_rescale_rec), offsetof(ftsp2_rescale_rec, flip),
         offsetof(ftsp2_rescale_rec, status), offsetof(ftsp2_rescale_rec, valid));
  printf("%zu %zu %zu %zu\\n", sizeof(ftsp2_train_report), offsetof(ftsp2_train_report, cost0),
         offsetof(ftsp2_train_report, max_err), offsetof(ftsp2_train_report, lambda));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    I, T, R, P = _lib.Instance, _lib.Table, _lib.RescaleRec, _lib.TrainReport
    assert out[0].split() == [str(v) for v in (C.sizeof(I), I.offset.offset, I.mu.offset, I.kT.offset)]
    assert out[1].split() == [str(v) for v in (C.sizeof(T), T.beta0.offset, T.theta.offset, T.theta_entropy.offset,
                                                T.family.offset)]
    assert out[2].split() == [str(v) for v in (C.sizeof(R), R.flip.offset, R.status.offset, R.valid.offset)]
    assert out[3].split() == [str(v) for v in (C.sizeof(P), P.cost0.offset, P.max_err.offset, P.lam.offset)]


def test_builtin_table_matches_oracle_copy():
    # The library and the oracle each carry their own copy of the printed
    # Appendix A table; they must agree digit for digit.
    from oracle import tables
    src = open(os.path.join(ROOT, "paper_2605_08523_gb300", "csrc", "ftsp2_api.cu")).read()
    block = src[src.index("kPrinted[26][4]"):]
    block = block[:block.index("};")]
    nums = [float(v) for v in re.findall(r"[-+]\d\.\d+e[-+]\d+", block)]
    flat = [v for row in tables.PRINTED_B1500 for v in row]
    assert nums == flat


def test_product_path_fails_loudly_without_library(tmp_path):
    # A copy of the binding pointed at a missing library must raise, not fall back.
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2605_08523_gb300 import _lib\n"
            "_lib.LIB_PATH = '/nonexistent/libftsp2.so'\n"
            "_lib._lib = None\n"
            "try:\n    _lib.lib()\nexcept RuntimeError as e:\n    print('raised')\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "raised" in out.stdout


def test_flag_constants_match_header():
    from paper_2605_08523_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "ftsp2.h")).read()
    defs = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define FTSP2_(\w+)\s+(0x[0-9a-fA-F]+|\d+)", src)}
    for name in ("SYNC", "CLAMP", "REFINE1", "REFINE2", "PAIR_TILES", "SINGLE_TILES", "LANCZOS", "MIN_LAYERS",
                 "REFINE_TC", "EPI_DEFERRED", "EPI_INLINE", "FULL_OPERANDS", "LAYER_LAUNCHES", "TARGET_FERMI",
                 "TARGET_ENTROPY"):
        assert defs[name] == getattr(_lib, name), name
    # flags are distinct bits
    bits = [defs[n] for n in ("SYNC", "CLAMP", "REFINE1", "REFINE2", "PAIR_TILES", "SINGLE_TILES", "LANCZOS", "MIN_LAYERS",
                              "REFINE_TC", "EPI_DEFERRED", "EPI_INLINE", "FULL_OPERANDS", "LAYER_LAUNCHES")]
    assert all(b & (b - 1) == 0 for b in bits) and len(set(bits)) == len(bits)


def test_kernel_code_hash_ignores_comments():
    # bench.kernel_sha keys the measured DRAM traffic of the layer kernel: it
    # hashes code only, so comment edits keep a capture valid and code edits
    # do not
    import bench
    src = 'int f() { // a comment\n  /* block\n comment */ return g("//x", \'/\'); }\n'
    code = bench._code_only(src)
    assert "comment" not in code and '"//x"' in code and "'/'" in code
    assert bench._code_only(src.replace("a comment", "another remark")) == code
    assert bench._code_only(src.replace("return", "return 1 +")) != code


def test_model_set_arguments_checked_on_the_host(built):
    # invalid tables are refused before any device call (works without a GPU)
    from paper_2605_08523_gb300 import _lib
    L = built.lib()
    th = (C.c_double * (4 * 65))(*([0.5] * (4 * 65)))

    def create(L_, family, beta0=100.0, mu0=1.0 / 3.0):
        t = (_lib.Table * 1)()
        t[0].L, t[0].L_entropy, t[0].beta0, t[0].mu0, t[0].alpha = L_, 0, beta0, mu0, 0.84
        t[0].theta = C.cast(th, C.POINTER(C.c_double))
        t[0].theta_entropy = None
        t[0].family = family
        h = C.c_void_p()
        return L.ftsp2_model_set_create(t, 1, C.byref(h))

    E_ARG = -1
    assert create(16, 7) == E_ARG                  # unknown family
    assert create(64, 1) == E_ARG                  # Skip-SP2 tables carry an output row: at most 63 layers
    assert create(65, 0) == E_ARG                  # Eq. mlsp2: at most 64 layers
    assert create(0, 0) == E_ARG
    assert create(16, 1, beta0=-1.0) == E_ARG
    assert create(16, 0, mu0=1.0) == E_ARG


def test_wait_limit_arguments(built):
    # host-side checks only: the limit is a process-wide setting read at each call
    default = built.wait_limit_ns()
    assert default == 4_000_000_000
    with pytest.raises(built.Ftsp2Error):
        built.set_wait_limit_ns(10)
    with pytest.raises(built.Ftsp2Error):
        built.set_wait_limit_ns(10 ** 11)
    built.set_wait_limit_ns(1_000_000)
    assert built.wait_limit_ns() == 1_000_000
    built.set_wait_limit_ns(default)
    with pytest.raises(built.Ftsp2Error):
        built.debug_stall_layer(-2)
    with pytest.raises(built.Ftsp2Error):
        built.debug_stall_layer(64)
    built.debug_stall_layer(-1)
