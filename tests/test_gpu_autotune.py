"""The autotuner's pruning by runtime bound (wave_plan_bound, wave_autotune_stats).

Candidates whose bound exceeds the best time measured so far are not timed.
The bound assumes perfect scheduling, so a pruned candidate cannot have been
faster: the plan chosen with pruning must run as fast as the plan chosen
without it (WAVE_TUNE_NOPRUNE=1, in a separate process so that neither run
sees the other's cached plan), within run-to-run noise.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, %(root)r)
import numpy as np, torch
from paper_1806_08299_gb300 import inputs, wave
p = inputs.c3(space_order=%(so)d, nt=4, n=%(n)r)
grid = wave.Grid(p.n, p.h, p.dt, p.nt, p.space_order)
tm, td, tq = (torch.from_numpy(a).cuda() for a in (p.m, p.damp, p.src_q))
wave.fwd(grid, tm, td, p.src_xyz, tq, None, tuning=wave.Tuning(time_tile=0))
print(json.dumps(dict(plan=wave.describe_plan(grid, wave.Tuning(time_tile=0)),
                      stats=wave.autotune_stats())))
"""


def _tuning(wavelib, pl):
    return wavelib.Tuning(time_tile=pl["time_tile"], tile_y=pl["tile_y"], tile_x=pl["tile_x"],
                          vec=pl["vec"], tile_z=pl["tile_z"], kernel=pl["kernel"], rows=pl["rows"],
                          flags=wavelib.WAVE_TIME_SWEEPS)


@pytest.mark.parametrize("so", [16, 4])
def test_pruned_autotune_keeps_the_fastest_plan(wavelib, cuda, so):
    import torch
    n = (384, 384, 256)  # five fields exceed twice L2, so the DRAM term of the bound applies
    env = dict(os.environ)
    env.pop("WAVE_TUNE_CACHE", None)
    out = {}
    for noprune in (False, True):
        e = dict(env)
        if noprune:
            e["WAVE_TUNE_NOPRUNE"] = "1"
        r = subprocess.run([sys.executable, "-c", CHILD % dict(root=ROOT, so=so, n=n)], env=e,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out[noprune] = json.loads(r.stdout.strip().splitlines()[-1])
    cand, pruned = out[False]["stats"]
    assert out[True]["stats"] == [cand, 0]
    assert 0 < pruned < cand  # something was pruned, and something timed
    # both plans on this process's GPU, alternately, best of three
    p = inputs.c3(space_order=so, nt=12, n=n)
    grid = wavelib.Grid(p.n, p.h, p.dt, p.nt, p.space_order)
    tm, td, tq = (torch.from_numpy(a).to(cuda) for a in (p.m, p.damp, p.src_q))
    best = {False: np.inf, True: np.inf}
    for _ in range(3):
        for k in (False, True):
            wavelib.fwd(grid, tm, td, p.src_xyz, tq, None, tuning=_tuning(wavelib, out[k]["plan"]))
            ms, _, steps = wavelib.sweep_stats()
            best[k] = min(best[k], ms / steps)
    torch.cuda.synchronize()
    assert best[False] <= 1.03 * best[True], (out, best)
