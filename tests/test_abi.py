"""The C-ABI library loads and exports every symbol include/*.h declares, and
argument validation rejects bad calls before any launch (no GPU needed)."""
from __future__ import annotations

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
        names.update(re.findall(r"\b(pg_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2207_01834_gb300.build import build
    from paper_2207_01834_gb300 import _lib

    build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"pg_tree_build", "pg_knn", "pg_bdl_insert", "pg_bdl_erase", "pg_knn_backward"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_symbol(lib):
    from paper_2207_01834_gb300 import _lib

    assert _declared() == set(_lib.SIGNATURES)


def test_version_and_counters(lib):
    assert b"sm_103a" in lib.pg_version()
    assert lib.pg_launch_count() >= 0


def _status(lib, name, *args):
    return getattr(lib, name)(*args)


def test_invalid_arguments_rejected_without_launch(lib):
    out = C.c_void_p()
    fake = C.c_void_p(0x1000)   # never dereferenced: validation fails first
    before = lib.pg_launch_count()
    assert _status(lib, "pg_tree_build", fake, 10, 0, 16, None, C.byref(out)) == 1        # dim 0
    assert _status(lib, "pg_tree_build", fake, 10, 17, 16, None, C.byref(out)) == 1       # dim 17
    assert _status(lib, "pg_tree_build", fake, -1, 3, 16, None, C.byref(out)) == 1        # n < 0
    assert _status(lib, "pg_tree_build", fake, 1 << 31, 3, 16, None, C.byref(out)) == 1   # n >= 2^31
    assert _status(lib, "pg_tree_build", fake, 10, 3, 0, None, C.byref(out)) == 1         # leaf 0
    assert _status(lib, "pg_tree_build", fake, 10, 3, 257, None, C.byref(out)) == 1       # leaf > 256
    assert _status(lib, "pg_tree_build", None, 10, 3, 16, None, C.byref(out)) == 1        # NULL points
    assert _status(lib, "pg_tree_build", fake, 10, 3, 16, None, None) == 1                # NULL out
    assert b"leaf_size" in lib.pg_last_error() or b"out" in lib.pg_last_error()
    assert _status(lib, "pg_knn", None, fake, 10, 5, fake, fake, None) == 1              # NULL tree
    assert _status(lib, "pg_bdl_create", 0, 64, 16, None, C.byref(out)) == 1             # dim 0
    assert _status(lib, "pg_bdl_create", 3, 0, 16, None, C.byref(out)) == 1             # X = 0
    assert _status(lib, "pg_knn_backward", fake, 10, fake, 10, 3, 0, fake, fake, fake, fake, None) == 1  # k=0
    total = C.c_int64()
    assert _status(lib, "pg_range", None, fake, 10, C.c_float(0.1), 0, None, fake, C.byref(total), None) == 1
    assert _status(lib, "pg_range_fill", None, fake, 10, C.c_float(0.1), fake, 10, fake, None) == 1  # NULL tree
    assert _status(lib, "pg_knn_graph", None, 5, 0, None, C.byref(total), None) == 1                # NULL tree
    assert lib.pg_launch_count() == before


def test_injected_allocation_failure_is_reported_before_any_cuda_call(lib):
    """The allocation fault hook (host side): the next device allocation fails
    with PG_ENOMEM, reported through the status and the error text; the tree
    build's first allocation comes before any CUDA call, so no GPU is needed."""
    out = C.c_void_p()
    fake = C.c_void_p(0x1000)   # never dereferenced: the allocation fails first
    before = lib.pg_launch_count()
    assert lib.pg_debug_fail_alloc_after(1) == 0
    try:
        assert _status(lib, "pg_tree_build", fake, 10, 3, 16, None, C.byref(out)) == 2     # PG_ENOMEM
        assert b"injected" in lib.pg_last_error()
        assert out.value is None
    finally:
        lib.pg_debug_fail_alloc_after(0)
    assert lib.pg_launch_count() == before


def test_header_documents_every_entry_point():
    """Each declaration in the header is preceded by a comment."""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        lines = open(h).read().splitlines()
        for i, line in enumerate(lines):
            m = re.match(r"PG_API .*\b(pg_\w+)\(", line)
            if m:
                prev = "\n".join(lines[max(0, i - 30):i])
                assert "*/" in prev, f"{m.group(1)} has no comment"


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_for_c_and_cxx_consumers(tmp_path, lang, std):
    """A plain C or C++ program can include the header and link against the
    library's symbols by name (syntax and type check with the host compiler)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use.c" if lang == "c" else "use.cpp")
    src.write_text('#include "pargeo_gpu.h"\n'
                   "int use(const float *p, long long n) {\n"
                   "    pg_tree *t = 0;\n"
                   "    pg_status s = pg_tree_build(p, n, 3, 16, 0, &t);\n"
                   "    if (s == PG_OK) s = pg_tree_free(t);\n"
                   "    return (int)s;\n"
                   "}\n")
    subprocess.check_call([cc, "-fsyntax-only", std, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src)])


def test_plain_c_program_links_and_calls_the_library(lib, tmp_path):
    """A C program linked against the shared library calls it through the C
    ABI alone: version string, argument validation, thread-local error text
    (no GPU work)."""
    import shutil
    import subprocess

    from paper_2207_01834_gb300.build import LIB

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "main.c"
    src.write_text('#include <stdio.h>\n#include <string.h>\n#include "pargeo_gpu.h"\n'
                   "int main(void) {\n"
                   "    pg_tree *t = 0;\n"
                   "    float p[3] = {0, 0, 0};\n"
                   "    if (!strstr(pg_version(), \"sm_103a\")) return 2;\n"
                   "    if (pg_tree_build(p, 1, 0, 16, 0, &t) != PG_EINVAL || t) return 3;\n"
                   "    if (strlen(pg_last_error()) == 0) return 4;\n"
                   "    puts(pg_last_error());\n"
                   "    return 0;\n"
                   "}\n")
    exe = tmp_path / "main"
    libdir = os.path.dirname(LIB)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-L", libdir, "-lpargeo_gpu", "-Wl,-rpath," + libdir, "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "dim" in r.stdout


def test_error_text_is_per_thread(lib):
    """pg_last_error is thread-local: two threads failing differently at the
    same time each read their own message."""
    import threading

    fake = C.c_void_p(0x1000)
    bad = []

    def worker(dim, leaf, word):
        out = C.c_void_p()
        for _ in range(2000):
            if lib.pg_tree_build(fake, 10, dim, leaf, None, C.byref(out)) != 1 or word not in lib.pg_last_error():
                bad.append(word)
                return

    ts = [threading.Thread(target=worker, args=(0, 16, b"dim")),
          threading.Thread(target=worker, args=(3, 0, b"leaf_size"))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert bad == []



def test_automatic_traversal_choice_without_a_device(lib):
    """PG_KNN_AUTO resolves on the host: the built-in choice is warp per query
    from dimension class 7 with k >= 16 and from class 5 with k > 32,
    postponed leaves otherwise, with the shared-memory heap for k > 16; a
    tune table entry overrides it for its (dimension class, k class, kind)."""
    v = C.c_int(-1)
    for dim, k, all_knn, want in [(3, 10, 1, 3), (5, 16, 0, 3), (7, 15, 0, 3), (7, 16, 0, 4), (9, 64, 1, 4),
                                  (16, 32, 0, 4), (2, 1, 1, 3), (3, 17, 1, 5), (3, 64, 0, 5), (4, 64, 1, 5),
                                  (5, 32, 0, 5), (5, 33, 0, 4), (6, 64, 1, 4)]:
        assert lib.pg_knn_tune_get(dim, k, all_knn, C.byref(v)) == 0
        assert v.value == want, (dim, k, all_knn, v.value)
    try:
        assert lib.pg_knn_tune_set(7, 16, 0, 1) == 0
        lib.pg_knn_tune_get(7, 16, 0, C.byref(v))
        assert v.value == 1
        lib.pg_knn_tune_get(7, 16, 1, C.byref(v))   # the other kind keeps the built-in choice
        assert v.value == 4
    finally:
        lib.pg_knn_tune_set(7, 16, 0, 0)
    assert lib.pg_knn_tune_set(3, 10, 1, 6) != 0     # not a traversal


def test_traversal_constants_match_the_header():
    """The binding's KNN_* numbers are the header's PG_KNN_* values, and every
    traversal the header defines is in KNN_VARIANTS."""
    from paper_2207_01834_gb300 import _lib

    text = open(os.path.join(ROOT, "include", "pargeo_gpu.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define PG_(KNN_\w+)\s+(\d+)", text)}
    assert defs["KNN_AUTO"] == 0 and len(defs) >= 6
    for name, value in defs.items():
        assert getattr(_lib, name) == value, name
    assert sorted(_lib.KNN_VARIANTS) == sorted(v for k, v in defs.items() if k != "KNN_AUTO")
