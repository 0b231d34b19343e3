"""The GPU demag tensor pinned to closed forms, independently of the oracle.

* One cell: a uniformly magnetised prism cell feels B = -mu0 Ms N m with N its
  own (self) demagnetising tensor, which for a rectangular prism is diagonal
  with Aharoni's (1998) closed-form factors.  Several aspect ratios, m along
  each axis.
* A whole prism of cells, uniformly magnetised: the demag field averaged over
  its cells is -mu0 Ms N_prism m, N_prism the prism's own Aharoni factors (the
  sum of the Newell cell-pair tensors over a prism is the prism's tensor).  The
  prisms stay within 16 cell edges, where the GPU tensor is the cell-averaged
  Newell form, so the identity is exact up to the FP32 field.
The closed form comes from oracle.aharoni_dz, a transcription of Aharoni's
formula pinned in the oracle tests against whole-cube and thin-film limits.
"""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi


def _aharoni(oracle, Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return np.array([oracle.aharoni_dz(b, c, a), oracle.aharoni_dz(c, a, b), oracle.aharoni_dz(a, b, c)])


@pytest.mark.parametrize("d", [(4e-9, 4e-9, 4e-9), (6e-9, 4e-9, 2e-9), (2e-9, 5e-9, 9e-9), (5e-9, 5e-9, 1e-9)])
def test_self_demag_factors(d):
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    Ms = 8e5
    sim = pkg.Sim(1, 1, 1, *d, Ms, 1.3e-11, 0.01)
    N = _aharoni(oracle, *d)
    for axis in range(3):
        m = np.zeros((1, 3), np.float32)
        m[0, axis] = 1.0
        sim.set_m(m)
        B = sim.eval_field(pkg.MMCQ_TERM_DEMAG).astype(np.float64)[0]
        expect = np.zeros(3)
        expect[axis] = -MU0 * Ms * N[axis]
        assert np.abs(B - expect).max() <= 2e-6 * MU0 * Ms, (axis, B, expect)
    assert abs(N.sum() - 1.0) < 1e-12
    sim.close()


@pytest.mark.parametrize("shape,d", [((10, 6, 3), (4e-9, 4e-9, 4e-9)), ((7, 12, 2), (3e-9, 5e-9, 2e-9)),
                                     ((16, 1, 4), (2e-9, 6e-9, 3e-9))])
def test_prism_average_demag_factors(shape, d):
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    nx, ny, nz = shape
    n = nx * ny * nz
    Ms = 8e5
    sim = pkg.Sim(nx, ny, nz, *d, Ms, 1.3e-11, 0.01)
    N = _aharoni(oracle, nx * d[0], ny * d[1], nz * d[2])
    for axis in range(3):
        m = np.zeros((n, 3), np.float32)
        m[:, axis] = 1.0
        sim.set_m(m)
        B = sim.eval_field(pkg.MMCQ_TERM_DEMAG).astype(np.float64).mean(0)
        expect = np.zeros(3)
        expect[axis] = -MU0 * Ms * N[axis]
        print(f"{shape}: axis {axis}: <B> {B}, Aharoni {expect}")
        assert np.abs(B - expect).max() <= 2e-6 * MU0 * Ms, (axis, B, expect)
    sim.close()
