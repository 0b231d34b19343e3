"""Parity at the full workload sizes, in the launch configuration bench.py times.

The trajectories of the full-size workloads over long horizons are in
test_gpu_horizon.py; this file checks the field itself where the oracle's own
FFT is not used:

* Large CPW-like film (1024x1024x8, 8.4 M cells, Lorentzian coupling profile):
  the demag field at sampled cells by the direct sum (each sample a sum over
  all 8.4 M cells, no FFT on either side of the comparison), and the local
  terms at the same cells in closed form; the field of every launch plan of
  the split y passes equal to the default one, bit for bit.
"""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_large_cpw_fields_at_sampled_cells():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    w = synthetic.large_cpw()
    I = w.instances[0]
    n = I.n
    sim = pkg.Sim(I.nx, I.ny, I.nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha)
    m0 = synthetic.tilted_m(n, I.seed, 0.3)
    sim.set_m(m0)
    sim.set_bias(I.bias)
    prof = I.coupling_profile()
    sim.set_cavity(I.omega_c, I.kappa, I.g, profile=prof)
    x0 = 2.0
    sim.set_cavity_init(x0, 0.0)
    m = sim.get_m().astype(np.float64)
    Bd = sim.eval_field(pkg.MMCQ_TERM_DEMAG).astype(np.float64)
    Bt = sim.eval_field(pkg.MMCQ_TERM_ALL).astype(np.float64)
    # sampled cells: corners, edges, centre and seeded interior points
    rng = np.random.default_rng(5)
    nx, ny, nz = I.nx, I.ny, I.nz
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, ny // 2, nz // 2), (0, ny - 1, 3), (nx - 1, 0, 4)]
    pts += [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))) for _ in range(7)]
    cells = np.array([(z * ny + y) * nx + x for x, y, z in pts])
    o = oracle.Oracle(nx, ny, nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha, demag=oracle.DEMAG_NONE)
    ref = o.demag_at(m, cells)
    scale = np.abs(ref).max()
    err = np.abs(Bd[cells] - ref).max()
    print(f"demag at {len(cells)} cells: max err {err:.3e} T of {scale:.3e} T")
    assert err <= 2e-6 * scale
    # local terms (exchange, bias, cavity x0 * B_rms) from the oracle's own
    # definitions on the full grid (O(N) each), added to the sampled demag
    local = oracle.Oracle(nx, ny, nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha, demag=oracle.DEMAG_NONE)
    local.set_bias(I.bias)
    local.set_cavity(I.omega_c, I.kappa, I.g, profile=prof.astype(np.float64))
    Bl = local.field(m, Gamma=x0)[cells]
    expect = ref + Bl
    err_t = np.abs(Bt[cells] - expect).max()
    print(f"total field at sampled cells: max err {err_t:.3e} T of {np.abs(expect).max():.3e} T")
    assert err_t <= 2e-6 * scale + 2e-6 * np.abs(Bl).max()
    # every launch plan of this grid's split y passes (one block for both
    # halves, or a block per half with the inverse's pairs exchanging through
    # cluster shared memory) gives the same field, bit for bit
    sim.set_tuning(None)
    rule = sim.tuning()
    assert rule["y_split"] != [-1, -1]
    fields = {}
    for ys in ([0, 0], [1, 0], [0, 1], [1, 1]):
        sim.set_tuning(dict(rule, y_split=ys))
        fields[tuple(ys)] = sim.eval_field(pkg.MMCQ_TERM_DEMAG)
    sim.set_tuning(None)
    base = fields[(0, 0)]
    assert np.array_equal(base.astype(np.float64), Bd)
    for ys, f in fields.items():
        assert np.array_equal(f, base), ys
    sim.close()
