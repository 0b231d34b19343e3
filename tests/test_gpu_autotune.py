"""The launch-parameter autotuner (mmcq_autotune): every plan it can choose
computes the oracle's field, the chosen plan is in use for stepping, and the
choice is cached per shape.

For each grid, every candidate of every knob (rows per x-pass block, groups
per block of each column pass, split or one-thread z pass, pipelined or
per-row x inverse, one or two blocks per half of the split y passes) is
applied with mmcq_set_tuning and its demag field is compared with the
oracle's at the tolerance of the field tests (2e-6 of the largest field).
The split y passes do the same arithmetic in either form, so their field is
also compared bit for bit.  Then mmcq_autotune picks a plan, each knob of which must
take one of those values, no slower than the fixed rules by its own timing;
a plan off the rules must step a trajectory that matches the oracle.
"""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu

GRIDS = [
    (32, 32, 1, 4e-9),       # 2-D convolution
    (64, 64, 2, 4e-9),       # 3-D, pz = 4 (batched-map members)
    (128, 128, 2, 4e-9),
    (64, 24, 16, 5e-9),      # pz = 32: split or one-thread z
    (48, 40, 8, 4e-9),       # pz = 16: one-thread or split z
    (1024, 4, 2, 4e-9),      # rows of L = 1024: pipelined or per-row x inverse
    (8, 520, 2, 4e-9),       # y padding 2048: split y passes, one or two blocks per half
]


def _candidates(plan):
    """The rule plan and every single-knob variant of it the tuner may time."""
    out = [dict(plan)]
    r = plan["x_rows"]
    for R in (r // 2, r // 4):
        if R >= 1:
            out.append(dict(plan, x_rows=R))
    for k in range(4):
        g = 1
        while g < plan["col_groups"][k]:
            cg = list(plan["col_groups"])
            cg[k] = g
            out.append(dict(plan, col_groups=cg))
            g *= 2
    if plan["z_split"] in (0, 1):
        out.append(dict(plan, z_split=1 - plan["z_split"]))
    if plan["x_pipe"] == 1:
        out.append(dict(plan, x_pipe=0))
    for k in range(2):
        if plan["y_split"][k] in (0, 1):
            ys = list(plan["y_split"])
            ys[k] = 1 - ys[k]
            out.append(dict(plan, y_split=ys))
    return out


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g[:3])))
def test_every_candidate_plan_matches_oracle(grid):
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    nx, ny, nz, d = grid
    n = nx * ny * nz
    sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.01, batch=2)
    m = synthetic.random_m(n, 4000 + n)
    sim.set_m(m)
    ref = o.demag(sim.get_m().astype(np.float64))
    scale = np.abs(ref).max()
    sim.set_tuning(None)
    rule = sim.tuning()
    cands = _candidates(rule)
    fields = []
    for plan in cands:
        sim.set_tuning(plan)
        assert sim.tuning()["x_rows"] == plan["x_rows"]
        assert sim.tuning()["y_split"] == plan["y_split"]
        got = sim.eval_field(pkg.MMCQ_TERM_DEMAG, inst=1)
        fields.append((plan, got))
        err = np.abs(got.astype(np.float64) - ref).max()
        assert err <= 2e-6 * scale, (plan, err, scale)
    for plan, got in fields[1:]:
        if plan["y_split"] != rule["y_split"] and all(plan[k] == rule[k] for k in rule if k != "y_split"):
            assert np.array_equal(got, fields[0][1]), plan
    sim.set_tuning(None)
    chosen = sim.autotune(reps=3)
    print(f"{nx}x{ny}x{nz}: {len(cands)} candidates; chosen {chosen}")
    assert chosen["eval_ms"] <= chosen["rule_ms"]
    assert chosen["candidates"] >= len(cands)
    now = sim.tuning()
    for k in ("x_rows", "col_groups", "z_split", "x_pipe", "y_split"):
        assert now[k] == chosen[k]
    # the tuner moves one knob at a time, so its choice combines knob values
    # that each appear among the candidates checked above
    for k in ("x_rows", "z_split", "x_pipe"):
        assert chosen[k] in {c[k] for c in cands}, k
    for j in range(4):
        assert chosen["col_groups"][j] in {c["col_groups"][j] for c in cands}, j
    for j in range(2):
        assert chosen["y_split"][j] in {c["y_split"][j] for c in cands}, j
    sim.set_tuning(chosen)
    got = sim.eval_field(pkg.MMCQ_TERM_DEMAG, inst=1).astype(np.float64)
    assert np.abs(got - ref).max() <= 2e-6 * scale
    sim.close()


def test_tuned_plan_steps_the_oracle_trajectory_and_is_cached():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    nx, ny, nz, d = 64, 24, 16, 5e-9
    n = nx * ny * nz
    sim, o = make_pair(nx, ny, nz, d, 1.4e5, 3.65e-12, 1e-3, Ku=1e3)
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(70, 1), 0.2)
    for x in (sim, o):
        x.set_bias((0.1, 0.0, 0.0))
        x.set_cavity(2 * math.pi * 4.5e9, 2 * math.pi * 1e7, 2 * math.pi * 200e6)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    # a plan off the rules on every knob that has a choice, so that stepping
    # runs launch shapes other than the defaults
    sim.set_tuning(None)
    plan = sim.tuning()
    plan["x_rows"] = max(1, plan["x_rows"] // 2)
    plan["col_groups"] = [1 if g else 0 for g in plan["col_groups"]]
    if plan["z_split"] == 1:
        plan["z_split"] = 0
    sim.set_tuning(plan)
    sim.set_integrator(pkg.MMCQ_DP45, 1e-6, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.DP45, 1e-6, oracle.CAV_E)
    sim.step(8, 1e-13)
    o.replay(sim.dt_history())
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    # the tuner times real stages but puts the instance states back: stepping
    # on from here continues the same trajectory
    first = sim.autotune(reps=3)
    done = len(sim.dt_history())
    sim.step(4, 0.0)
    o.replay(sim.dt_history()[done:])
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    # a second handle of the same shape takes the tuner's choice from the cache
    other = pkg.Sim(nx, ny, nz, d, d, d, 1.4e5, 3.65e-12, 1e-3, Ku=1e3)
    again = other.autotune(reps=3)
    assert again["candidates"] == 0
    for k in ("x_rows", "col_groups", "z_split", "x_pipe", "y_split"):
        assert again[k] == first[k]
    # a plan that is not one of this grid's choices is refused, nothing changes
    bad = dict(first, x_rows=first["x_rows"] * 4 + 1)
    with pytest.raises(pkg.MMCQError) as e:
        other.set_tuning(bad)
    assert e.value.code == pkg.MMCQ_ERR_ARG
    assert other.tuning()["x_rows"] == first["x_rows"]
    other.close()
    sim.close()


def test_split_y_halves_per_block_step_the_oracle_trajectory():
    """Dormand-Prince on a grid whose y passes run the split kernel, with each
    half in a block of its own (the inverse's pairs exchanging through
    cluster shared memory): the trajectory is the one-block form's, bit for
    bit, and the oracle's."""
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    nx, ny, nz, d = 8, 520, 2, 4e-9
    n = nx * ny * nz
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(71, 1), 0.3)
    runs = []
    for ys in ([0, 0], [1, 1]):
        sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.01)
        sim.set_tuning(None)
        plan = sim.tuning()
        assert plan["y_split"] in ([0, 0], [1, 1], [0, 1], [1, 0])
        sim.set_tuning(dict(plan, y_split=ys))
        for x in (sim, o):
            x.set_bias((0.05, 0.02, 0.0))
            x.set_cavity(2 * math.pi * 8e9, 2 * math.pi * 1e7, 2 * math.pi * 2e8)
        sim.set_m(m0)
        o.set_m(m0.astype(np.float64))
        sim.set_integrator(pkg.MMCQ_DP45, 1e-6, pkg.MMCQ_CAVITY_E)
        o.set_integrator(oracle.DP45, 1e-6, oracle.CAV_E)
        sim.step(6, 1e-13)
        o.replay(sim.dt_history())
        m = sim.get_m()
        assert np.abs(m.astype(np.float64) - o.get_m()).max() <= 1e-5
        runs.append((m, sim.dt_history()))
        sim.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
