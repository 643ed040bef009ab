"""The C-ABI library loads without a GPU and exports every symbol that
include/ttm.h declares; host-only entry points agree with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2408_02398_gb300 import build as B
from paper_2408_02398_gb300 import ttm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "ttm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:ttm|tm)_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = header_functions()
    assert len(names) >= 15
    L = ttm.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(ttm.EXPORTS) == names


def test_status_codes_match_header():
    src = open(os.path.join(ROOT, "include", "ttm.h")).read()
    codes = dict((m[0], int(m[1])) for m in re.findall(r"(TTM_(?:OK|E_[A-Z_]+))\s*=\s*(\d+)", src))
    assert {v: k for k, v in codes.items()} == ttm.STATUS
    common = open(os.path.join(ROOT, "paper_2408_02398_gb300", "csrc", "ttm_common.cuh")).read()
    for name, val in codes.items():
        short = name.replace("TTM_", "")
        assert re.search(r"\b%s\s*=\s*%d\b" % (short, val), common), name


def test_component_counts():
    for n in (2, 4, 6):
        for d in (3, 4):
            assert ttm.ttm_num_components(n, d) == O.num_components(n, d)


def test_default_params():
    p = ttm.params()
    assert p.filter_a == pytest.approx(0.2)   # Sec. 2: a = 1/5
    assert p.order_n == 4 and p.dprime == 3 and p.cube_symmetrize == 1


@pytest.mark.parametrize("cube", [False, True])
def test_rotation_set_equals_oracle_set(cube):
    """The library's quadrature is the same set of rotations as the
    oracle's (written independently; order and quaternion sign may differ)."""
    q_lib = ttm.ttm_rotation_set(40, cube)
    q_or = O.rotation_set(40, cube=cube)
    assert q_lib.shape == q_or.shape
    assert np.allclose(np.linalg.norm(q_lib, axis=1), 1.0)

    def key(q):
        R = O.quat_to_rot(q)
        return tuple(np.round(R.ravel(), 9))

    assert sorted(map(key, q_lib)) == sorted(map(key, q_or))
    if not cube:
        assert np.allclose(q_lib, q_or, atol=1e-14)


def test_rotation_set_rejects_bad_args():
    L = ttm.lib()
    assert L.ttm_rotation_set(0, 1, None) == 1
    assert L.ttm_rotation_set(4, 1, None) == 1


# ------------------------------------------- block processing, host logic --

@pytest.mark.parametrize("Z,tz,slab", [(40, 12, 5), (40, 12, 29), (40, 12, 100), (37, 11, 4), (12, 12, 3),
                                       (64, 16, 1)])
def test_slab_ranges_partition_and_halos(Z, tz, slab):
    """Sec. 3.4 block processing: the output planes of the slabs partition
    the valid planes; each slab's map planes are its output planes plus one
    valid neighbour plane each side; its input covers every map plane's
    template window and one filter plane beyond it (or reaches the tomogram
    edge)."""
    r = ttm.ttm_slab_ranges(Z, tz, slab)
    cz = tz // 2
    vz0, vz1 = cz, Z - (tz - cz) + 1
    assert len(r) == -(-(vz1 - vz0) // slab)
    covered = []
    for o0, o1, m0, m1, i0, i1 in r:
        covered += list(range(o0, o1))
        assert m0 == max(vz0, o0 - 1) and m1 == min(vz1, o1 + 1)
        lo = m0 - cz                       # first plane of the first window
        hi = (m1 - 1) + (tz - 1 - cz)      # last plane of the last window
        assert i0 == 0 or i0 <= lo - 1
        assert i1 == Z or i1 >= hi + 2
        assert 0 <= i0 < i1 <= Z and i1 - i0 >= tz
    assert covered == list(range(vz0, vz1))
    assert ttm.lib().ttm_slab_ranges(Z, Z + 1, slab, None, 0) == -1


def test_merge_peaks_matches_greedy_definition():
    rng = np.random.default_rng(12)
    shape = (20, 30, 40)
    n = 3000
    idx = rng.choice(int(np.prod(shape)), n, replace=False).astype(np.int64)
    val = np.round(rng.normal(size=n), 2).astype(np.float32)   # many equal values: the index breaks ties
    got_i, got_v = ttm.ttm_merge_peaks(idx, val, shape, 60, 4.5)
    order = sorted(range(n), key=lambda k: (-float(val[k]), int(idx[k])))
    zyx = np.stack(np.unravel_index(idx, shape), axis=1).astype(float)
    acc = []
    for k in order:
        if len(acc) == 60:
            break
        if all(np.sum((zyx[k] - zyx[a]) ** 2) >= 4.5 ** 2 for a in acc):
            acc.append(k)
    assert list(got_i) == [int(idx[k]) for k in acc]
    assert np.array_equal(got_v, val[acc])
    assert len(ttm.ttm_merge_peaks(idx[:0], val[:0], shape, 10, 3.0)[0]) == 0


C_MAIN = r"""
#include "ttm.h"
#include <stdio.h>
int main(void)
{
    int rows[6 * 8];
    int n = ttm_slab_ranges(40, 12, 5, rows, 8);
    int64_t idx[2] = {5, 100};
    float val[2] = {1.0f, 2.0f};
    int64_t oi[2];
    float ov[2];
    int m = ttm_merge_peaks(2, idx, val, 10, 10, 10, 2, 1.0, oi, ov);
    printf("%d %d %lld %d\n", n, m, (long long)oi[0], ttm_num_components(4, 4));
    return 0;
}
"""


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """include/ttm.h compiles as strict C99 and as C++17, and a C program
    that calls the host-only entry points links against libttm.so."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    hdr = os.path.join(inc, "ttm.h")
    for cmd in ([gcc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", hdr],
                [shutil.which("g++") or "g++", "-fsyntax-only", "-x", "c++", "-std=c++17", "-Wall", "-Werror", hdr]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    src = tmp_path / "main.c"
    src.write_text(C_MAIN)
    lib_dir = os.path.join(ROOT, "paper_2408_02398_gb300")
    exe = tmp_path / "main"
    r = subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-L", lib_dir, "-lttm", "-Wl,-rpath," + lib_dir,
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["6", "2", "100", "35"]   # 29 valid planes in slabs of 5
