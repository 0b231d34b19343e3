"""GPU effective-field terms vs the FP64 oracle, term by term (Sec. 2.1 field
list, Eq. bcav), on ragged, masked, 2-D and 3-D grids.

Tolerance: the FP32 pipeline (FP32 kernel spectrum, FP32 FFTs of length up to
P) is accurate to ~ log2(P) * 2^-24 relative to the largest field; 2e-6 of the
term's maximum is used for every term, which is ~20x that estimate and far
below anything that matters at max|dm| <= 1e-5."""
import math

import numpy as np
import pytest

from gpu_common import f32, make_pair, require_gpu

pytestmark = pytest.mark.gpu

GRIDS = [
    (32, 32, 1, (4e-9, 4e-9, 4e-9)),
    (13, 7, 1, (3e-9, 4e-9, 5e-9)),
    (10, 6, 3, (4e-9, 4e-9, 3e-9)),
    (1, 1, 1, (4e-9, 4e-9, 4e-9)),
    (16, 1, 1, (2e-9, 2e-9, 2e-9)),
    (1, 9, 1, (2e-9, 3e-9, 2e-9)),
    (1, 1, 6, (2e-9, 2e-9, 2e-9)),
    (9, 1, 5, (5e-9, 5e-9, 5e-9)),
    (33, 17, 4, (4e-9, 4e-9, 4e-9)),
    (64, 40, 2, (4e-9, 4e-9, 4e-9)),
    (20, 12, 16, (5e-9, 5e-9, 5e-9)),
    (24, 20, 9, (4e-9, 4e-9, 3e-9)),
    (6, 5, 17, (4e-9, 4e-9, 4e-9)),
    (4, 600, 2, (4e-9, 3e-9, 4e-9)),
    # rows of 256 / 512 / 1024 cells in whole blocks: the compile-time shapes of
    # the x passes; 256 x 40 x 16 also takes the fixed y (P = 128) and z
    # (pz = 32, 4 ky per block) shapes
    (256, 40, 16, (5e-9, 5e-9, 5e-9)),
    # pz = 32 with one ky column: the one-thread z pass (k_zconv<32>)
    (12, 1, 12, (4e-9, 4e-9, 4e-9)),
    (512, 8, 2, (4e-9, 4e-9, 4e-9)),
    (1024, 2, 2, (4e-9, 4e-9, 4e-9)),
]


def _inputs(n, seed, mask_frac=0.15):
    import synthetic
    m = synthetic.random_m(n, seed)
    u = synthetic.uniform(seed + 1, np.arange(n, dtype=np.uint64))
    ms = np.where(u < mask_frac, 0.0, 6e5 + 4e5 * u).astype(np.float32)
    if n == 1:
        ms[:] = 8e5
    return m, ms


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g[:3])))
def test_field_terms_match_oracle(grid):
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    nx, ny, nz, d = grid
    n = nx * ny * nz
    sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.02, Ku=4e4, axis=(0.3, -0.5, 0.8))
    m, ms = _inputs(n, 1000 + n)
    sim.set_ms_map(ms)
    o.set_ms(ms.astype(np.float64))
    sim.set_m(m)
    o.set_m(m.astype(np.float64))
    m_gpu = sim.get_m().astype(np.float64)
    mo = o.get_m()
    assert np.abs(m_gpu - mo).max() < 1e-7
    bias = (0.031, -0.02, 0.05)
    sim.set_bias(bias)
    o.set_bias(bias)
    prof = np.stack([np.linspace(-1, 1, n), np.cos(np.arange(n)), 0.5 * np.ones(n)], 1).astype(np.float32)
    sim.set_cavity(2 * math.pi * 5e9, 1e7, 2 * math.pi * 300e6, profile=prof)
    o.set_cavity(2 * math.pi * 5e9, 1e7, 2 * math.pi * 300e6, profile=prof.astype(np.float64))
    x0 = 3.0
    sim.set_cavity_init(x0, 1.0)
    o.set_cavity_init(x0, 1.0)
    # oracle terms at the GPU's (float32) state, which is what the GPU sees
    Bd = o.demag(m_gpu)
    Bx = o.exchange(m_gpu)
    Ba = o.anis(m_gpu)
    Bfull = o.field(m_gpu, Gamma=x0)
    brms = o.get_brms()
    Bz = np.where((ms > 0)[:, None], np.asarray(bias)[None, :], 0.0)
    Bc = np.where((ms > 0)[:, None], brms * x0, 0.0)
    checks = [
        (pkg.MMCQ_TERM_DEMAG, Bd),
        (pkg.MMCQ_TERM_EXCHANGE, Bx),
        (pkg.MMCQ_TERM_ANIS, Ba),
        (pkg.MMCQ_TERM_ZEEMAN, Bz),
        (pkg.MMCQ_TERM_CAVITY, Bc),
    ]
    for term, ref in checks:
        got = sim.eval_field(term).astype(np.float64)
        scale = max(np.abs(ref).max(), 1e-30)
        err = np.abs(got - ref).max()
        assert err <= 2e-6 * scale, (term, err, scale)
    got = sim.eval_field(pkg.MMCQ_TERM_ALL).astype(np.float64)
    # empty cells carry only the demag field on the GPU (their torque is 0);
    # on magnetic cells the total is the oracle's total field
    ref = Bd + Bx + Ba + Bz + Bc
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 2e-6 * scale
    mag = ms > 0
    assert np.abs(got[mag] - Bfull[mag]).max() <= 2e-6 * scale
    sim.close()
