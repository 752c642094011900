"""Inhomogeneous coupling on the GPU (bz_transport_x, bz_inhom_step) against the oracle
(`oracle.inhom`: free streaming through full 3D grid values, RK4 collision per cell).

Bars: free streaming in FP64, relative L-infinity 1e-12 of max|f| (c128 cells), 1e-6 for c64
cells; the drifting density wave against its closed form to 1e-12; Strang steps (FP32
collisions) to relative L-infinity 1e-5 of the change of f.
"""
import math

import numpy as np
import pytest

import bz_inputs as bi
from oracle import inhom, kernels, spectral

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__._libbuild().build()
    import paper_2004_11239_gb300 as m
    return m


@pytest.mark.parametrize("N,nx,dtype", [(8, 8, "c128"), (16, 24, "c128"), (24, 16, "c128"), (32, 32, "c128"),
                                        (16, 8, "c64")])
def test_transport_matches_oracle(bz, N, nx, dtype):
    L, Lx, t = 6.0, 3.0, 0.37
    f0 = bi.inhom_cells(N, L, nx, Lx)
    td = torch.complex128 if dtype == "c128" else torch.complex64
    fd = torch.from_numpy(f0).to("cuda", dtype=td)
    bz.bz_transport_x(N, L, nx, Lx, fd, t)
    torch.cuda.synchronize()
    got = fd.cpu().numpy().astype(np.complex128)
    ref = inhom.transport(f0, L, Lx, t)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"transport N={N} nx={nx} {dtype}: rel_Linf={err:.2e}")
    assert err <= (1e-12 if dtype == "c128" else 1e-6)


def test_transport_density_wave_closed_form_and_reversal(bz):
    N, L, nx, Lx, eps, u, T = 32, 6.0, 8, 4.0, 0.3, 0.7, 0.5
    f0 = bi.drifting_wave_samples(N, L, nx, Lx, eps, u, T)
    fd = torch.from_numpy(f0).cuda()
    x = np.arange(nx) * Lx / nx
    t = 1.1
    bz.bz_transport_x(N, L, nx, Lx, fd, t)
    torch.cuda.synchronize()
    rho = inhom.density(fd.cpu().numpy(), L)
    exact = 1 + eps * math.exp(-(2 * math.pi * t / Lx) ** 2 * T / 2) * np.cos(2 * math.pi * (x - u * t) / Lx)
    assert np.max(np.abs(rho - exact)) < 1e-12
    bz.bz_transport_x(N, L, nx, Lx, fd, -t)
    torch.cuda.synchronize()
    assert np.max(np.abs(fd.cpu().numpy() - f0)) < 1e-12 * np.max(np.abs(f0))


@pytest.mark.parametrize("real", [False, True])
def test_inhom_strang_steps_match_oracle(bz, real):
    N, L, nx, Lx, dt, steps = 8, 6.0, 8, 3.0, 0.1, 2
    R = bi.R_from_L(L)
    f0 = bi.inhom_cells(N, L, nx, Lx)
    plan = bz.bz_plan_create_ex(N, L, R, 0.0, 0.5, 2, 12, data=bz.BZ_DATA_REAL if real else bz.BZ_DATA_COMPLEX)
    batch = bz.bz_batch_create(plan, nx, 0)
    fd = torch.from_numpy(f0).cuda()
    bz.bz_inhom_step(batch, nx, Lx, fd, dt, steps)
    torch.cuda.synchronize()
    got = fd.cpu().numpy()
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    ref = inhom.strang(op, f0, Lx, dt, steps, real=real)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref - f0)))
    coll = float(np.max(np.abs(ref - inhom.transport(f0, L, Lx, dt * steps))) / np.max(np.abs(ref - f0)))
    print(f"inhom Strang N={N} nx={nx} {steps} steps ({'real' if real else 'complex'} form): rel_Linf of the change={err:.2e} "
          f"(collision share of the change {coll:.2f})")
    assert err <= 1e-5
    mass0, mass1 = inhom.density(f0, L).sum(), inhom.density(got, L).sum()
    assert abs(mass1 - mass0) < 1e-12 * abs(mass0)                    # streaming and Q keep the mass
    with pytest.raises(bz.BzError):                                   # more cells than slots
        bz.bz_inhom_step(batch, nx + 8, Lx, torch.zeros((nx + 8) * N ** 3, dtype=torch.complex128).cuda(), dt, 1)
    batch.close()
    plan.close()
