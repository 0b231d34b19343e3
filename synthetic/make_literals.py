"""Write synthetic/workload_literals.json: the uniform-mode (Kittel) frequencies
that the workloads use as cavity frequencies.

Calls only the oracle: the demagnetising factors of each whole sample are the
oracle's Aharoni (1998) prism factors, which equal the average of the
cell-pair demag tensor over the sample.  Kittel's formula for a bias B and a
uniaxial anisotropy field 2Ku/Ms along x:
    omega = gamma sqrt((B + Bk + (Ny - Nx) mu0 Ms)(B + Bk + (Nz - Nx) mu0 Ms)).

Run:  python synthetic/make_literals.py
"""
import json
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402


def prism_factors(Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return (oracle.aharoni_dz(b, c, a), oracle.aharoni_dz(c, a, b), oracle.aharoni_dz(a, b, c))


def kittel_x(B, Ms, Ku, L):
    Nx, Ny, Nz = prism_factors(*L)
    Bk = 2 * Ku / Ms
    return oracle.GAMMA_LL * math.sqrt((B + Bk + (Ny - Nx) * oracle.MU0 * Ms) *
                                       (B + Bk + (Nz - Nx) * oracle.MU0 * Ms))


def main():
    out = {
        "film_32_omega_kittel": kittel_x(0.05, 8e5, 0.0, (32 * 4e-9, 32 * 4e-9, 4e-9)),
        "yig_wire_omega_kittel": kittel_x(0.1, 1.4e5, 1e3, (256 * 5e-9, 64 * 5e-9, 16 * 5e-9)),
        "large_cpw_omega_kittel": kittel_x(0.03, 8e5, 0.0, (1024 * 4e-9, 1024 * 4e-9, 8 * 4e-9)),
        "_source": "synthetic/make_literals.py (oracle Aharoni prism factors + Kittel formula)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_literals.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    for k, v in out.items():
        if not k.startswith("_"):
            print(k, v, v / 2 / math.pi / 1e9, "GHz")


if __name__ == "__main__":
    main()
