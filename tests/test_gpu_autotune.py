"""Autotuner on the GPU: it runs end to end, and the launch shapes it chooses
among change the forces only by FP32 summation order."""
import math

import numpy as np
import pytest

from paper_2006_14952_gb300 import autotune as A
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def forces(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(pm_grid=32, theta=0.4, order=4, **kw)
    s.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
    a = s.short_range_forces().cpu().numpy().astype(np.float64)
    return a


def test_every_tile_setting_gives_the_same_forces():
    pos, mass = W.nfw_clustered(40000, 40, 0.7, 51)
    ref = forces(pos, mass)
    for knob, (values, _) in A.KNOBS.items():
        for v in values:
            a = forces(pos, mass, **{knob: v})
            err = math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())
            assert err < 1e-6, (knob, v, err)


def test_tune_runs_and_caches(tmp_path):
    import torch

    pos, mass = W.nfw_clustered(30000, 30, 0.7, 52)
    params = dict(pm_grid=32, theta=0.4, order=4)
    best, trials = A.tune(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), params, reps=1)
    for k, (values, _) in A.KNOBS.items():
        assert best[k] in values
        assert set(trials[k]) == set(values) and all(t > 0 for t in trials[k].values())
    path = str(tmp_path / "c.json")
    key = A.cache_key(torch.cuda.get_device_name(0), "test", params)
    A.save(path, key, best, trials)
    assert A.lookup(path, key) == best
