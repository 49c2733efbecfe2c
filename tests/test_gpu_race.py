"""Race detection by schedule: the same inputs run with the grids of the
persistent and grid-stride kernels divided by 1, 3 and 7
(PICASSO_GRID_DIVISOR, read when the library loads, so each divisor runs in
its own process).  Every output is defined independently of the schedule,
so conflict CSRs (both forms), colorings (static order with the small-round
engine, dynamic order) and a run of wide strings must agree bit for bit; a
race in a count, fill or coloring order would show as a difference."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, '.')
from paper_2401_06713_b300 import build, picasso, synth
build.build()

def h(*arrays):
    m = hashlib.sha256()
    for a in arrays:
        m.update(np.ascontiguousarray(a.cpu().numpy()).tobytes())
    return m.hexdigest()

out = {}
chars = synth.pauli_weighted(30000, 64, 0.25, seed=11)
xz = picasso.pack(torch.from_numpy(chars).cuda())
for form in ("earlier", "full"):
    with picasso.Picasso(xz, 64, seed=11, palette=(1, 16), alpha=1.5, csr=form) as p:
        p.assign_lists(*p.round_params())
        p.build_conflicts()
        out["csr_" + form] = h(*p.csr())
with picasso.Picasso(xz, 64, seed=11, palette=(1, 16), alpha=1.5) as p:
    c, r = p.run()
    out["run"] = h(c)
    out["small_rounds"] = p.stats()["small_rounds"]
with picasso.Picasso(xz, 64, seed=11, palette=(1, 16), alpha=1.5, color="dynamic") as p:
    c, r = p.run()
    out["dynamic"] = h(c)
wide = synth.pauli_weighted(8000, 100, 0.1, seed=12)
with picasso.Picasso(picasso.pack(torch.from_numpy(wide).cuda()), 100, seed=12) as p:
    c, r = p.run()
    out["wide"] = h(c)
print(json.dumps(out))
"""


def _run(divisor):
    env = dict(os.environ, PICASSO_GRID_DIVISOR=str(divisor))
    res = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_outputs_do_not_depend_on_the_grid():
    base = _run(1)
    assert base["small_rounds"] > 0  # the engine ran too
    for d in (3, 7):
        assert _run(d) == base, d
