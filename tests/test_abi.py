"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every entry point include/dm.h declares, validates arguments before
touching the device, and its tuner seed follows the paper's formulas."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1505_06864_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dm():
    B.build()
    from paper_1505_06864_gb300 import dm as D
    return D


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(dm_\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported(dm):
    names = declared_functions()
    assert "dm_plan" in names and "dm_solve" in names and len(names) >= 10
    L = ctypes.CDLL(B.LIB)
    for n in names:
        assert hasattr(L, n), n
    # the binding exposes the same names
    for n in names:
        assert hasattr(dm, n), n


def test_invalid_arguments_rejected_without_gpu(dm):
    bad = [dict(N=0, m=4, nrhs=1), dict(N=10, m=0, nrhs=1), dict(N=10, m=4, nrhs=0),
           dict(N=10, m=600, nrhs=1), dict(N=10, m=4, nrhs=65), dict(N=9, m=4, nrhs=1, P=6),
           dict(N=4, m=2, nrhs=1, P=3), dict(N=10, m=4, nrhs=1, P=-1)]
    for kw in bad:
        with pytest.raises(dm.DMError) as e:
            dm.dm_plan(precision=dm.DM_FP64, **kw)
        assert e.value.code == dm.DM_EINVAL, kw
    with pytest.raises(dm.DMError) as e:
        dm.dm_plan(10, 4, 1, 2, 1, precision=9)
    assert e.value.code == dm.DM_EINVAL
    assert dm.dm_last_error()


def test_tuner_seed_is_paper_optimum(dm):
    from oracle import dm_oracle as o
    for N, m, r in [(2048, 256, 1), (4096, 128, 8), (64, 16, 1), (3071, 400, 1), (5, 3, 1)]:
        P, levels, P2 = dm.dm_plan_tune(N, m, r)
        ref = min(max(1, round(o.p_opt_mp(N, m, r))), (N + 1) // 2)
        assert P == ref
        if P >= 21:
            assert P2 == o.supp_partitions(P - 1, P, r, m)
            assert levels == (3 if P2 >= 8 else 2)
        else:
            assert levels == 1
    # explicit choices pass through; P2 follows Eq. (SuppMatrM) or its boundary P/3
    assert dm.dm_plan_tune(2048, 256, 1, P=64, levels=2) == (64, 2, o_supp(64, 1, 256))
    assert dm.dm_plan_tune(2048, 256, 1, P=16, levels=2)[2] == round(16 / 3)
    assert dm.dm_plan_tune(2048, 256, 1, P=4, levels=1) == (4, 1, 1)
    assert dm.dm_plan_tune(64, 16, 1, P=1, levels=3) == (1, 1, 1)


def o_supp(P, r, m):
    from oracle import dm_oracle as o
    return o.supp_partitions(P - 1, P, r, m)


def test_partition_sizes_match_oracle(dm):
    from oracle import dm_oracle as o
    for N, P, m, r in [(2048, 64, 256, 1), (3071, 64, 400, 1), (100, 5, 8, 1), (20, 9, 4, 2), (10, 2, 3, 1),
                       (40, 13, 5, 5), (1, 1, 4, 1)]:
        assert dm.dm_partition_sizes(N, m, r, P) == o.partition_plan(N, P)[1]
        assert dm.dm_partition_sizes(N, m, r, P, dm.DM_PLAN_EQUAL_TIME) == \
            o.partition_lengths_equal_time(N, P, m, r)


def test_plan_flags_checked_without_gpu(dm):
    """The kernel-variant flags are accepted by the host-side partitioner (they
    do not change the partition); an unknown bit is refused before any device
    call, by dm_plan_ex and by dm_partition_sizes."""
    base = dm.dm_partition_sizes(100, 8, 1, 5)
    for fl in (dm.DM_PLAN_FP64_FMA, dm.DM_PLAN_FP64_INV_COLUMN, dm.DM_PLAN_FP64_FMA | dm.DM_PLAN_FP64_INV_COLUMN):
        assert dm.dm_partition_sizes(100, 8, 1, 5, fl) == base
    for fl in (8, 16, 1 << 30):
        with pytest.raises(dm.DMError) as e:
            dm.dm_partition_sizes(100, 8, 1, 5, fl)
        assert e.value.code == dm.DM_EINVAL
        with pytest.raises(dm.DMError) as e:
            dm.dm_plan_ex(100, 8, 1, 5, 1, dm.DM_FP64, fl)
        assert e.value.code == dm.DM_EINVAL and "flags" in dm.dm_last_error()
    with pytest.raises(dm.DMError) as e:
        dm.dm_autotune_ex(100, 8, 1, 9)
    assert e.value.code == dm.DM_EINVAL


def test_tuner_cache_file_read_without_gpu(dm, tmp_path):
    """The tuner's cache file: seven-field lines (no flags column) and
    eight-field lines load; lines that do not describe a valid plan are
    skipped; dm_tuned reports the stored choice with no device work.  A fresh
    process, since the file is read once per process at the first lookup."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    cache.write_text("300 32 2 0 7 2 12.5\n"            # seven fields: flags 0
                     "2048 256 1 0 64 3 80.1 4\n"       # the column-by-column inverse
                     "1000 64 4 3 40 2 9.0 2\n"         # bf16x3, FP64-pipe products
                     "100 8 1 0 80 1 3.0 0\n"           # P too large for N: skipped
                     "100 8 2 9 5 1 3.0 0\n"            # unknown precision: skipped
                     "100 8 3 0 5 1 3.0 64\n"           # unknown flag: skipped
                     "100 600 1 0 5 1 3.0 0\n"          # m above the limit: skipped
                     "not a line\n")
    code = (
        "from paper_1505_06864_gb300 import dm\n"
        "assert dm.dm_tuned(300, 32, 2, 'fp64') == (7, 2, 0)\n"
        "assert dm.dm_tuned(2048, 256, 1, 'fp64') == (64, 3, dm.DM_PLAN_FP64_INV_COLUMN)\n"
        "assert dm.dm_tuned(1000, 64, 4, 'bf16x3') == (40, 2, dm.DM_PLAN_FP64_FMA)\n"
        "for args in [(100, 8, 1, 'fp64'), (100, 8, 3, 'fp64'), (100, 600, 1, 'fp64'), (300, 32, 2, 'fp32')]:\n"
        "    try:\n"
        "        dm.dm_tuned(*args)\n"
        "        raise SystemExit('stored: %r' % (args,))\n"
        "    except dm.DMError as e:\n"
        "        assert e.code == dm.DM_EINVAL and 'no measured choice' in dm.dm_last_error()\n"
        "print('ok')\n")
    env = dict(os.environ, DM_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_serving_arguments_checked_without_gpu(dm):
    """Budget and narrow-request arguments are checked before any device work
    (the server starts no worker for them)."""
    for bad in (-1.0, float("nan"), 1e9):
        with pytest.raises(dm.DMError) as e:
            dm.dm_serve_budget(bad)
        assert e.value.code == dm.DM_EINVAL
    dm.dm_serve_budget(0.0)
    with pytest.raises(dm.DMError) as e:
        dm.dm_submit_cols(None, np.zeros(4), np.zeros(4), 1)
    assert e.value.code == dm.DM_EINVAL
    st = dm.dm_serve_stats()
    assert set(st) == {"admitted", "refused", "runs", "merged"} and all(v >= 0 for v in st.values())


def test_noalloc_refuses_host_arrays_before_the_call(dm):
    """dm_solve_noalloc takes device memory only: numpy arrays are refused by
    the binding with DM_EINVAL and nothing reaches the library."""
    import numpy as np
    A = np.zeros((4, 2, 2))
    v = np.zeros((4, 2, 1))
    with pytest.raises(dm.DMError) as e:
        dm.dm_solve_noalloc(4, 2, 1, 1, A, A, A, v, v.copy())
    assert e.value.code == dm.DM_EINVAL and "CUDA tensor" in str(e.value)


def test_dm_inside_arguments_rejected_without_gpu(dm):
    """dm_plan_inside validates M, J and the subsystem lengths before it
    touches the device."""
    for args in [(20, 4, 1, 4, 5, 1), (20, 4, 1, 2, 1, 1), (20, 4, 1, 0, 2, 1), (20, 4, 1, 2, 2, 3),
                 (5, 4, 1, 4, 2, 1)]:
        with pytest.raises(dm.DMError) as e:
            dm.dm_plan_inside(*args)
        assert e.value.code == dm.DM_EINVAL, args


def test_complex_plan_limits_without_gpu(dm):
    for args in [(10, 300, 1, 2, 1, "fp64"), (10, 200, 1, 2, 1, "bf16x3"), (10, 0, 1, 2, 1, "fp64")]:
        with pytest.raises(dm.DMError) as e:
            dm.dm_plan_complex(*args)
        assert e.value.code == dm.DM_EINVAL, args
