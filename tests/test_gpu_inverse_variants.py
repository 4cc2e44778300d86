"""The three float32 block inverses (column-by-column cluster, panel-blocked,
register-resident) against the oracle, each forced through DM_INV_KERNEL in
a child process (the choice is read once per process).  Shapes cover one
CTA and clusters, ragged panels (m = 5, 40, 100) and the register tile
limit (m = 128, and m = 200 where the register variant hands over to the
column kernel)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import dm_oracle as o
from paper_1505_06864_gb300 import workloads as w

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(9, 5, 1, 2, 1), (97, 40, 3, 7, 2), (60, 100, 2, 6, 1), (40, 128, 8, 8, 1), (21, 200, 2, 4, 1)]

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1505_06864_gb300 import build, dm, workloads as w
build.build()
out = []
for N, m, r, P, lv in json.loads(sys.argv[2]):
    s = w.dominant_system(N, m, r, 23 + m)
    plan = dm.dm_plan(N, m, r, P, lv, "fp32")
    dm.dm_factor(plan, s.A, s.B, s.C)
    x = np.zeros_like(s.b)
    dm.dm_solve(plan, s.b, x)
    q = dm.dm_plan_query(plan)
    dm.dm_destroy(plan)
    np.save(sys.argv[3] + "_%d.npy" % len(out), x)
    out.append({"P2": q["P2"], "iters": q["last_iters"], "corr": q["last_correction"]})
print(json.dumps(out))
"""


@pytest.mark.parametrize("variant", ["column", "panel", "reg"])
def test_float32_inverse_variants(tmp_path, variant):
    env = dict(os.environ, DM_INV_KERNEL=variant)
    stem = str(tmp_path / variant)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(SHAPES), stem], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    for k, (N, m, nr, P, lv) in enumerate(SHAPES):
        s = w.dominant_system(N, m, nr, 23 + m)
        x = np.load(stem + "_%d.npy" % k)
        P2 = info[k]["P2"]
        xref = o.dm(s.A, s.B, s.C, s.b, P, levels=lv, P2=P2 if P2 > 1 else None)
        scale = np.max(np.abs(xref), axis=(0, 1))
        assert np.all(np.max(np.abs(x - xref), axis=(0, 1)) <= 1e-10 * scale), (variant, N, m)
        assert info[k]["corr"] <= 1e-12
