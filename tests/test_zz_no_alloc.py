"""The allocation-free coupling sum (mmcq_coupling_sum_noalloc).

Some callers cannot allocate device memory: code that runs inside a host
framework whose memory pool owns the GPU, or a latency-bound loop that cannot
pay for cudaMalloc's device-wide synchronisation.  For them the library offers
one entry point whose scratch lives in a fixed static device array.  This test
calls it through the C ABI on device arrays and checks, on two calls in a row,
that it returns the same FP64 coupling sum X as the handle-based read-out
(mmcq_get_cavity) and as an FP64 numpy sum of the very same float32 arrays
(several chunks of cells, so that the last-block finish over the chunk
partials runs, and a case whose terms cancel), and that an oversized request
is refused on the host.

The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import ctypes
import math

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_coupling_sum_matches_handle_readout():
    require_gpu()
    import torch

    import paper_2410_00966_gb300 as pkg
    import synthetic

    nx, ny, nz, d = 24, 20, 3, 4e-9
    n = nx * ny * nz
    sim = pkg.Sim(nx, ny, nz, d, d, d, 8e5, 1.3e-11, 0.01)
    ms = synthetic.disk_ms(nx, ny, nz, d, d, 80e-9, 8e5)
    sim.set_ms_map(ms)
    sim.set_m(synthetic.tilted_m(n, synthetic.derive_seed(77, 0), 0.6))
    # B_rms in tesla with a component along m (no cancellation in the sum)
    brms = (1e-6 * np.stack([np.linspace(0.5, 1.5, n), 0.3 * np.ones(n), np.zeros(n)], 1)).astype(np.float32)
    sim.set_cavity(2 * math.pi * 6e9, 2 * math.pi * 10e6, profile=brms, profile_is_brms=True)
    sim.step(20, 1e-13)
    x_ref = sim.cavity()["X"]

    dev = torch.device("cuda", 0)
    m_dev = torch.empty((n, 3), dtype=torch.float32, device=dev)
    sim.get_m(0, out=m_dev)
    ms_dev = torch.from_numpy(ms).to(dev)
    brms_dev = torch.from_numpy(brms).to(dev)
    torch.cuda.synchronize()
    lib = pkg.lib()
    vc = d ** 3
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    outs = []
    for _ in range(2):
        out = ctypes.c_double(0.0)
        rc = lib.mmcq_coupling_sum_noalloc(ctypes.c_void_p(m_dev.data_ptr()), ctypes.c_void_p(ms_dev.data_ptr()),
                                           ctypes.c_void_p(brms_dev.data_ptr()), n, vc, ctypes.byref(out), stream)
        assert rc == pkg.MMCQ_OK
        outs.append(out.value)
    assert x_ref != 0.0
    for x in outs:
        assert abs(x - x_ref) <= 1e-9 * abs(x_ref), (x, x_ref)
    assert outs[0] == outs[1]

    # beyond the static scratch: refused on the host with a clear code
    big = 4096 * 4096 + 1
    out = ctypes.c_double(0.0)
    rc = lib.mmcq_coupling_sum_noalloc(ctypes.c_void_p(m_dev.data_ptr()), ctypes.c_void_p(ms_dev.data_ptr()),
                                       ctypes.c_void_p(brms_dev.data_ptr()), big, vc, ctypes.byref(out), stream)
    assert rc == pkg.MMCQ_ERR_UNSUPPORTED
    sim.close()


def _noalloc(lib, pkg, m_dev, ms_dev, brms_dev, n, vc, stream):
    out = ctypes.c_double(0.0)
    rc = lib.mmcq_coupling_sum_noalloc(ctypes.c_void_p(m_dev.data_ptr()), ctypes.c_void_p(ms_dev.data_ptr()),
                                       ctypes.c_void_p(brms_dev.data_ptr()), n, vc, ctypes.byref(out), stream)
    assert rc == pkg.MMCQ_OK
    return out.value


@pytest.mark.parametrize("n,cancel", [(3 * 4096 + 123, False), (5 * 4096 + 7, True), (1, False)])
def test_noalloc_coupling_sum_matches_fp64_numpy(n, cancel):
    """Several 4096-cell chunks (the chunk partials are added by the last block
    to finish), against an FP64 sum of the same float32 arrays done by numpy."""
    require_gpu()
    import torch

    import paper_2410_00966_gb300 as pkg

    rng = np.random.default_rng(20241001 + n)
    m = rng.normal(size=(n, 3)).astype(np.float32)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    m = m.astype(np.float32)
    ms = rng.uniform(7.5e5, 8.5e5, n).astype(np.float32)
    ms[rng.random(n) < 0.1] = 0.0
    if cancel:
        # B_rms along y, m with a y component of either sign: the terms cancel
        brms = np.zeros((n, 3), np.float32)
        brms[:, 1] = 1e-6
    else:
        brms = (1e-6 * rng.uniform(0.2, 1.0, (n, 3))).astype(np.float32)
    vc = (4e-9) ** 3
    terms = ms.astype(np.float64) * np.einsum("ij,ij->i", m.astype(np.float64), brms.astype(np.float64))
    x_np = vc * float(np.sum(terms))
    scale = vc * float(np.sum(np.abs(terms)))

    dev = torch.device("cuda", 0)
    m_dev = torch.from_numpy(m).to(dev)
    ms_dev = torch.from_numpy(ms).to(dev)
    brms_dev = torch.from_numpy(brms).to(dev)
    torch.cuda.synchronize()
    lib = pkg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    outs = [_noalloc(lib, pkg, m_dev, ms_dev, brms_dev, n, vc, stream) for _ in range(2)]
    assert outs[0] == outs[1]
    for x in outs:
        # only the order of the FP64 additions differs
        assert abs(x - x_np) <= 1e-13 * scale, (x, x_np, scale)
