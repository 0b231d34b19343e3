"""Helpers shared by the GPU parity tests: build, skip without a GPU, and
set up the CUDA library and the oracle on identical seeded inputs."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00966_gb300 import build
    build.build()
    import oracle
    oracle.build()


def make_pair(nx, ny, nz, d, Ms, Aex, alpha, Ku=0.0, axis=(1.0, 0.0, 0.0), batch=1, demag=None):
    import oracle
    import paper_2410_00966_gb300 as pkg
    if isinstance(d, (int, float)):
        d = (d, d, d)
    sim = pkg.Sim(nx, ny, nz, *d, Ms, Aex, alpha, Ku=Ku, axis=axis, batch=batch)
    o = oracle.Oracle(nx, ny, nz, *d, Ms, Aex, alpha, Ku=Ku, axis=axis,
                      demag=oracle.DEMAG_FFT if demag is None else demag)
    return sim, o


def f32(a):
    return np.asarray(a, dtype=np.float32)
