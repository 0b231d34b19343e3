"""Handle groups (mmcq_group_*): several handles of different grids stepped
together as one CUDA graph.  The graph replays exactly the kernels a direct
mmcq_step would enqueue, so a grouped run must equal the same handles stepped
one by one bit for bit (RK4 and DP45, both cavity modes, with a remainder
after the last full chunk, across a re-capture after an integrator change).
One member is also checked against the oracle."""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

# the batched anticrossing map's grid family at reduced size
SHAPES = [(32, 32, 1, 2), (16, 16, 2, 3), (24, 8, 4, 2)]


def _handles(pkg, synthetic, kind, mode):
    out = []
    for k, (nx, ny, nz, nb) in enumerate(SHAPES):
        sim = pkg.Sim(nx, ny, nz, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01, batch=nb)
        n = nx * ny * nz
        for b in range(nb):
            sim.set_m(synthetic.tilted_m(n, synthetic.derive_seed(50, k, b), 0.05), inst=b)
            sim.set_bias((0.02 + 0.03 * b, 0.0, 0.0), inst=b)
            sim.set_cavity(2 * np.pi * (4e9 + 1e9 * k), 2 * np.pi * 1e7, 2 * np.pi * 1e8, inst=b)
        sim.set_integrator(kind, 1e-6, mode)
        out.append(sim)
    return out


def _state(sims):
    return [([s.get_m(b) for b in range(s.batch)], s.cavity(-1)) for s in sims]


def _same(a, b):
    for (ma, ca), (mb, cb) in zip(a, b):
        for x, y in zip(ma, mb):
            assert np.array_equal(x, y)
        for p, q in zip(ca, cb):
            for key in ("t", "re_alpha", "im_alpha", "S", "C", "dt", "accepted", "rejected"):
                assert p[key] == q[key], key


@pytest.mark.parametrize("kind,mode,n,dt", [(0, 0, 37, 5e-14), (0, 1, 20, 5e-14), (1, 0, 23, 1e-13), (1, 1, 17, 1e-13)],
                         ids=["rk4-E", "rk4-P", "dp45-E", "dp45-P"])
def test_group_equals_direct_steps(kind, mode, n, dt):
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    direct = _handles(pkg, synthetic, kind, mode)
    for s in direct:
        s.step(n, dt)
    grouped = _handles(pkg, synthetic, kind, mode)
    g = pkg.Group(grouped, chunk=8)
    g.step(n, dt)
    assert g.replays() == n // 8
    _same(_state(direct), _state(grouped))
    for a, b in zip(direct, grouped):
        assert a.launch_count() == b.launch_count()
    # a second call replays the same graph; a changed integrator re-captures
    for s in direct:
        s.step(9, 0.0 if kind else dt)
    g.step(9, 0.0 if kind else dt)
    for s in direct + grouped:
        s.set_integrator(1 - kind, 1e-6, mode)
    dt2 = 1e-13 if kind == 0 else 5e-14
    for s in direct:
        s.step(16, dt2)
    g.step(16, dt2)
    _same(_state(direct), _state(grouped))
    g.close()
    for s in direct + grouped:
        s.close()


def test_group_member_matches_oracle():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sims = _handles(pkg, synthetic, 0, 0)
    g = pkg.Group(sims, chunk=10)
    g.step(40, 5e-14)
    nx, ny, nz, nb = SHAPES[1]
    for b in range(nb):
        o = oracle.Oracle(nx, ny, nz, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
        o.set_m(synthetic.tilted_m(nx * ny * nz, synthetic.derive_seed(50, 1, b), 0.05).astype(np.float64))
        o.set_bias((0.02 + 0.03 * b, 0.0, 0.0))
        o.set_cavity(2 * np.pi * 5e9, 2 * np.pi * 1e7, 2 * np.pi * 1e8)
        o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
        o.step(40, 5e-14)
        assert np.abs(sims[1].get_m(b).astype(np.float64) - o.get_m()).max() <= 1e-5
    g.close()


def test_group_arguments():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sims = _handles(pkg, synthetic, 0, 0)
    with pytest.raises(pkg.MMCQError):
        pkg.Group([sims[0], sims[0]])
    with pytest.raises(pkg.MMCQError):
        pkg.Group(sims, chunk=0)
    g = pkg.Group(sims)
    with pytest.raises(pkg.MMCQError):
        g.step(3, 0.0)                     # RK4 needs dt > 0
    g.close()
