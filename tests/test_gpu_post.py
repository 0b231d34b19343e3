"""Pipelined cavity read-out (mmcq_post_cavity / mmcq_take_cavity): each take
returns what the synchronous read-out gives at the posted point, in order, with
steps enqueued in between; the slot ring's limits are errors."""
import math

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _sim(batch):
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sim = pkg.Sim(16, 8, 2, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01, batch=batch)
    for b in range(batch):
        sim.set_m(synthetic.tilted_m(16 * 8 * 2, synthetic.derive_seed(30, b), 0.3), inst=b)
        sim.set_bias((0.05, 0.0, 0.01 * b), inst=b)
        sim.set_cavity(2 * math.pi * (7e9 + 1e8 * b), 2 * math.pi * 20e6, 2 * math.pi * 300e6, inst=b)
    return sim, pkg


@pytest.mark.parametrize("kind", [0, 1], ids=["rk4", "dp45"])
def test_posted_readout_matches_synchronous(kind):
    require_gpu()
    sim, pkg = _sim(3)
    sim.set_integrator(kind, 1e-5, 0)
    sim.step(5, 1e-13)
    sim.post_cavity()
    got = sim.take_cavity()
    ref = sim.cavity(-1)
    for g, r in zip(got, ref):
        for k in r:
            assert g[k] == r[k], (k, g[k], r[k])
    sim.close()


def test_posted_readouts_come_in_order_while_steps_run():
    require_gpu()
    sim, pkg = _sim(2)
    sim.set_integrator(0, 1e-6, 0)
    seen = []
    sim.step(1, 1e-13)
    sim.post_cavity()
    for _ in range(6):
        sim.step(1, 1e-13)
        sim.post_cavity()
        seen.append(sim.take_cavity())
    seen.append(sim.take_cavity())
    acc = [s[0]["accepted"] for s in seen]
    assert acc == list(range(1, 8))
    ref = sim.cavity(-1)
    for g, r in zip(seen[-1], ref):
        assert g["re_alpha"] == r["re_alpha"] and g["t"] == r["t"]
    sim.close()


def test_slot_ring_limits():
    require_gpu()
    sim, pkg = _sim(1)
    with pytest.raises(RuntimeError, match="MMCQ_ERR_STATE"):
        sim.take_cavity()
    for _ in range(pkg.MMCQ_POST_SLOTS):
        sim.post_cavity()
    with pytest.raises(RuntimeError, match="MMCQ_ERR_STATE"):
        sim.post_cavity()
    for _ in range(pkg.MMCQ_POST_SLOTS):
        sim.take_cavity()
    sim.post_cavity()
    sim.take_cavity()
    sim.close()
