"""The coupling sum X = V_c sum_i Ms_i m_i . B_rms,i (Eq. gammafinal) as the
stage kernel reduces it, against the oracle's FP64 sum on the GPU's own m.

The value the stage kernel hands to the cavity update is read back without a
dedicated hook: in P-mode, one accepted RK4 step from empty accumulators adds
C = e^{kappa t} cos(omega_c t) X dt (Eq. Cdiscrete, t = t_cav = dt after the
step), with X taken at the accepted, renormalised m; so X = C / (e^{kappa t}
cos(omega_c t) dt) in FP64 on the host.

Tolerance: each cell's product Ms (m . B_rms) is formed in FP32 (a few
roundings, relative 2^-22 of the largest partial) and the sum is FP64, so the
error is below 1e-7 of sum_i |Ms_i m_i . B_rms,i| for any grid of more than a
handful of cells, whatever the cancellation in X itself.  The read-out X of
mmcq_get_cavity (FP64 products) is held to 1e-12 of the same scale.
"""
import math

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _check(sim, o, wc, kappa, dt, label):
    import paper_2410_00966_gb300 as pkg
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_P)
    sim.reset_cavity()
    sim.step(1, dt)
    c = sim.cavity()
    t = c["t_cav"]
    assert t == pytest.approx(dt, rel=1e-15)
    x_stage = c["C"] / (math.exp(kappa * t) * math.cos(wc * t) * dt)
    m = sim.get_m().astype(np.float64)
    x_or = o.cavity_X(m)
    brms = o.get_brms()
    terms = np.einsum("ij,ij->i", m, brms)
    scale = abs(o.vc) * float(np.sum(np.abs(terms * o.ms_values)))
    print(f"{label}: X stage {x_stage:.12e}, read-out {c['X']:.12e}, oracle {x_or:.12e}; "
          f"scale sum|terms| {scale:.3e}; stage error {abs(x_stage - x_or) / scale:.2e}, "
          f"read-out error {abs(c['X'] - x_or) / scale:.2e} of the scale")
    assert abs(x_stage - x_or) <= 1e-7 * scale
    assert abs(c["X"] - x_or) <= 1e-12 * scale


class _OracleX:
    """The oracle's coupling sum on a handle without the demag kernel."""

    def __init__(self, nx, ny, nz, d, Ms, ms_map):
        import oracle
        self.o = oracle.Oracle(nx, ny, nz, d, d, d, Ms, 1.3e-11, 0.01, demag=oracle.DEMAG_NONE)
        self.ms_values = np.full(nx * ny * nz, Ms) if ms_map is None else ms_map.astype(np.float64)
        if ms_map is not None:
            self.o.set_ms(self.ms_values)
        self.vc = d ** 3

    def set_cavity(self, *a, **k):
        self.o.set_cavity(*a, **k)

    def cavity_X(self, m):
        return self.o.cavity_X(m)

    def get_brms(self):
        return self.o.get_brms()


def test_stage_coupling_sum_with_cancellation():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    nx, ny, nz, d = 40, 24, 6, 4e-9
    n = nx * ny * nz
    ms = synthetic.disk_ms(nx, ny, nz, d, d, 140e-9, 8e5) * synthetic.uniform_ms_map(n, 11, 0.9, 1.1)
    ms = ms.astype(np.float32)
    m0 = synthetic.random_m(n, synthetic.derive_seed(90, 1))      # directions all over the sphere
    rng = np.random.default_rng(91)
    brms = (rng.normal(size=(n, 3)) * 1e-6).astype(np.float32)   # signs of both kinds: X cancels
    wc, kappa, dt = 2 * math.pi * 6e9, 2 * math.pi * 1e7, 1e-13
    sim = pkg.Sim(nx, ny, nz, d, d, d, 8e5, 1.3e-11, 0.01)
    sim.set_ms_map(ms)
    sim.set_m(m0)
    sim.set_bias((0.02, 0.01, 0.0))
    sim.set_cavity(wc, kappa, profile=brms, profile_is_brms=True)
    o = _OracleX(nx, ny, nz, d, 8e5, ms)
    o.set_cavity(wc, kappa, profile=brms.astype(np.float64), profile_is_brms=True)
    _check(sim, o, wc, kappa, dt, "random directions, random B_rms")
    sim.close()


def test_stage_coupling_sum_largest_grid():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    w = synthetic.large_cpw()
    I = w.instances[0]
    sim = pkg.Sim(I.nx, I.ny, I.nz, I.d, I.d, I.d, I.Ms, I.Aex, I.alpha)
    sim.set_m(I.m0())
    sim.set_bias(I.bias)
    prof = I.coupling_profile()
    sim.set_cavity(I.omega_c, I.kappa, I.g, profile=prof)
    o = _OracleX(I.nx, I.ny, I.nz, I.d, I.Ms, None)
    o.set_cavity(I.omega_c, I.kappa, I.g, profile=prof.astype(np.float64))
    _check(sim, o, I.omega_c, I.kappa, 1e-13, "1024x1024x8, Lorentzian profile along y")
    sim.close()
