"""The C-ABI library builds, loads and exports every symbol include/lingam.h
declares; the binding covers them; no compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lingam.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:lingam_status|const char \*|int32_t)\s*(\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_03772_gb300 import _build
    path = _build.build()
    import paper_2403_03772_gb300 as pkg
    return path, pkg.load(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["lingam_create", "lingam_destroy", "lingam_last_error", "lingam_causal_order",
                 "lingam_fit_adjacency", "varlingam_fit", "lingam_causal_order_batch"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    path, handle = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    for name in _declared():
        assert name in exported, name
        assert getattr(handle, name) is not None


def test_binding_signatures_cover_the_header():
    import paper_2403_03772_gb300 as pkg
    assert set(pkg.SIGNATURES) == set(_declared())


STRUCTS = {"Opts": "lingam_opts", "Stats": "lingam_stats", "Instance": "lingam_instance",
           "Tuning": "lingam_tuning"}


def test_struct_layouts_match_the_header(tmp_path):
    """Size and every field offset of the ctypes mirrors equal the C compiler's
    for the structs of include/lingam.h."""
    import paper_2403_03772_gb300 as pkg
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lingam.h"',
             'int main(void) {']
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(pkg, py)._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        py, field, value = line.split()
        cls = getattr(pkg, py)
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (py, field, got, value)


def test_missing_library_fails_loudly(tmp_path):
    import paper_2403_03772_gb300 as pkg
    saved = pkg._lib
    pkg._lib = None
    try:
        with pytest.raises(ImportError):
            pkg.load(str(tmp_path / "nope.so"))
    finally:
        pkg._lib = saved


def test_create_reports_errors_without_crashing(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _, handle = lib
    h = ctypes.c_void_p()
    code = handle.lingam_create(ctypes.byref(h), 0, None)
    assert code != 0 and not h.value
    assert len(handle.lingam_last_error(None)) > 0


def test_library_has_no_undefined_internal_symbols(lib):
    """Every kernel launcher the library calls is defined in it (a missing
    definition would only show up when the library is loaded on a GPU machine)."""
    path, _ = lib
    out = subprocess.run(["nm", "-D", "--undefined-only", path], capture_output=True, text=True,
                         check=True).stdout
    missing = [line.split()[-1] for line in out.splitlines() if "_ZN2lg" in line]
    assert not missing, missing


def test_pair_tile_info_describes_every_tile(lib):
    import paper_2403_03772_gb300 as pkg
    txt = open(HEADER).read()
    n = int(re.search(r"#define LINGAM_PAIR_TILES (\d+)", txt).group(1))
    assert n == pkg.PAIR_TILES
    for t in range(n):
        g = pkg.lingam_pair_tile_info(t)
        assert 32 * g["wgi"] * g["wgj"] <= 1024
        assert g["groups"] in (1, 2) and g["packed"] in (0, 1) and g["fold"] >= 1
        assert g["stages"] >= 2 and g["wi"] >= 1 and g["wj"] >= 1
        assert g["sub"] in (0, 1, 2, 4)
        # the streamlined block folds on power-of-two chunk counts
        assert g["sub"] == 0 or (g["fold"] & (g["fold"] - 1)) == 0
    for bad in (-1, n):
        with pytest.raises(pkg.LingamError):
            pkg.lingam_pair_tile_info(bad)


def test_shard_ownership_partitions_pairs_symmetrically_and_by_tile(lib):
    """lingam_shard_owner (host, no GPU): every ordered pair has one owner,
    (i, j) and (j, i) the same one, the ranks' shares are within 1 % of equal
    at p = 1000, and every pair-kernel tile lies inside one owner's share."""
    import numpy as np
    import paper_2403_03772_gb300 as pkg
    assert pkg.shard_owner(0, 0, 1, 3) == 0 and pkg.shard_owner(5, 0, 4, 2) == -1
    for p, R in [(40, 2), (100, 3), (257, 5), (1000, 3)]:
        own = np.array([[pkg.shard_owner(i, j, p, R) for j in range(p)] for i in range(p)])
        assert own.min() >= 0 and own.max() < R and np.array_equal(own, own.T)
        if p == 1000:
            off = ~np.eye(p, dtype=bool)
            counts = [int(((own == r) & off).sum()) for r in range(R)]
            assert max(counts) - min(counts) < 0.01 * p * (p - 1) / R
        for t in range(pkg.PAIR_TILES):
            g = pkg.lingam_pair_tile_info(t)
            ti, tj = g["wi"] * g["wgi"], g["wj"] * g["wgj"]
            for a in range(0, p, ti):
                for b in range(0, p, tj):
                    blk = own[a:a + ti, b:b + tj]
                    assert np.all(blk == blk.flat[0])
