"""CPU-side checks of the CUDA library: it loads, exports every symbol the
C header declares, and its host-side shape catalogue agrees with the
oracle's (no device calls)."""
import re
import os

import numpy as np
import pytest

from oracle import catalog as cat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def motif():
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def test_exports_every_declared_symbol(motif):
    header = open(os.path.join(ROOT, "include", "motif.h")).read()
    declared = set(re.findall(r"\b(mc_[a-z_0-9]+)\s*\(", header))
    lib = motif.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(motif.EXPORTED)


def test_shape_catalogue_matches_oracle(motif):
    for h in range(1, 9):
        info = motif.shape_info(h)
        shapes = cat.rooted_shapes(h)
        assert motif.num_shapes(h) == len(shapes)
        assert motif.num_unrooted(h) == len(cat.unrooted_shapes(h))
        for i, s in enumerate(shapes):
            assert int(info["code"][i]) == (int(s, 2) if s else 0)
            assert int(info["unrooted"][i]) == cat.unrooted_id(s)
            if h > 1:
                a, b, beta = cat.decompose(s)
                assert int(info["beta"][i]) == beta
                assert int(info["left"][i]) == cat.shape_id(a)
                assert int(info["right"][i]) == cat.shape_id(b)


def test_errors_without_device(motif):
    # argument checks happen before any device work
    st = motif.load().mc_build_tables(None, None, 4, 64, 0, None, None, None)
    assert st == motif.MC_E_INVALID
    assert b"NULL" in motif.load().mc_last_error()


def test_skip_round_programs_match_the_oracle_catalogue():
    # the library's balanced level-k decompositions and a_j (host code)
    # against the oracle's, written independently from Section 3.3.2
    import paper_2009_03052_gb300 as M
    M.load()
    from oracle import catalog as cat
    for k in range(4, 9):
        info = M.skip_round_info(k)
        shapes = cat.rooted_shapes(k)
        for i, s in enumerate(shapes):
            d = cat.balanced_decompose(s, k)
            if d is None:
                assert info["beta"][i] == -1 and info["left"][i] == -1 and info["right"][i] == -1
                continue
            a, b, beta = d
            na, nb = len(a) // 2 + 1, len(b) // 2 + 1
            assert info["beta"][i] == beta, (k, s)
            assert (info["left_size"][i], info["right_size"][i]) == (na, nb), (k, s)
            assert info["left"][i] == cat.rooted_shapes(na).index(a), (k, s)
            assert info["right"][i] == cat.rooted_shapes(nb).index(b), (k, s)
        assert list(info["copies"]) == cat.Catalog(k, skip_round=True).copies_divisor(k)


def test_header_is_plain_c_and_cpp(tmp_path):
    # the boundary is a C ABI: the header compiles as C99 and as C++11
    import os
    import shutil
    import subprocess
    import pytest
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    for cc, std, ext in (("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not installed")
        src = tmp_path / f"t.{ext}"
        src.write_text('#include "motif.h"\nint main(void) { return MC_OK; }\n')
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_autotune_choices_cache_file(motif, tmp_path):
    # the schedule table (host code): choices loaded from a cache file, pinned
    # by mc_autotune_set, appended by the library; unknown schedules refused
    path = tmp_path / "tune.txt"
    n, nnz, maxd = 1_000_000, 19_970_150, 9529
    # key fields: kind k bits h floor(log2 n) floor(2 log2(nnz/n)) floor(log2(maxd+1)) choice
    path.write_text("0 5 64 3 19 8 13 2\n1 5 64 4 19 8 13 1\n")
    motif.autotune(1, str(path))
    assert motif.autotune_choice(0, 5, 64, 3, n, nnz, maxd) == 2
    assert motif.autotune_choice(1, 5, 64, 4, n, nnz, maxd) == 1
    assert motif.autotune_choice(0, 5, 64, 2, n, nnz, maxd) == -1
    # the same degree bucket: another graph of the same shape
    assert motif.autotune_choice(0, 5, 64, 3, n + 1000, nnz + 5000, maxd + 10) == 2
    motif.autotune_set(0, 6, 128, 4, n, nnz, maxd, 2)
    assert motif.autotune_choice(0, 6, 128, 4, n, nnz, maxd) == 2
    with pytest.raises(motif.MotifError):
        motif.autotune_set(1, 6, 128, 4, n, nnz, maxd, 6)   # the merge has schedules 0..5
    with pytest.raises(motif.MotifError):
        motif.autotune(3)
    motif.autotune(1, "")
