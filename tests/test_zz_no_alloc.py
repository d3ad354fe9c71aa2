"""The allocation-free diagnostics entry point against the context's own.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, or monitoring hooks that must not trigger an allocation's device
synchronisation); it reduces fields the caller holds, with a fixed scratch
array inside the library.  Checked through the C-ABI on two calls in a row,
against vefd_diagnostics on the same state, within the tolerances of the
diagnostics parity test.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _fields(lat, vefd):
    return {f: lat.read(f, device=True) for f in (vefd.RHO_A, vefd.RHO_B, vefd.U, vefd.C)}


def _compare(ref, got):
    assert abs(got[0] / ref[0] - 1) < 1e-6 and abs(got[1] / ref[1] - 1) < 1e-6
    scale = 1e-6 * ref[0]
    assert np.allclose(got[2:5], ref[2:5], rtol=1e-5, atol=scale)
    assert np.allclose(got[5:9], ref[5:9], rtol=1e-5, atol=1e-9)
    assert abs(got[9] - ref[9]) <= 2 and abs(got[14] - ref[14]) <= 2
    assert abs(got[10] - ref[10]) < 1e-3 and abs(got[11] - ref[11]) < 1e-3
    assert np.allclose(got[12:14], ref[12:14], atol=1e-2)
    assert np.isclose(got[15], ref[15], rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("lattice", ["d3q19", "d2q9"])
def test_noalloc_diagnostics_match_context(lattice):
    import torch

    from paper_1406_2686_gb300 import vefd

    if lattice == "d3q19":
        nx, ny, nz = 48, 32, 40
        lat = vefd.Lattice(lattice=vefd.D3Q19, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=0.21,
                           eta_B=0.35)
        lat.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, 8.0, 2.0, 0.1, 5.0, 3, 1e-3)
    else:
        nx, ny, nz = 96, 48, 1
        lat = vefd.Lattice(lattice=vefd.D2Q9, nx=nx, ny=ny, nz=1, ncomp=2, walls=1, G=1.5, eta_A=0.21, eta_B=0.35)
        lat.init_droplet((nx - 1) / 2, (ny - 1) / 2, 0.0, 10.0, 2.0, 0.1, 5.0, 3, 1e-3)
    L2 = 100.0
    lat.set_wall_shear(0.03)
    lat.set_fenep(50.0, 0.14, L2, 1e-3, 1, 1)
    stream = lat.stream.cuda_stream
    for call in range(2):
        lat.step(40)
        ref = lat.diagnostics()
        f = _fields(lat, vefd)
        torch.cuda.synchronize()
        got = vefd.vefd_diagnostics_noalloc(lat.cfg.lattice, nx, ny, nz, 2, L2, f[vefd.RHO_A].data_ptr(),
                                            f[vefd.RHO_B].data_ptr(), f[vefd.U].data_ptr(), f[vefd.C].data_ptr(),
                                            stream)
        _compare(ref, got)
    lat.close()


@pytest.mark.slow
def test_noalloc_at_capacity():
    """Exactly at the documented capacity, 256 x 128 x 256 = 8,388,608 nodes
    (4096 reduction blocks: every partial row of the scratch array is used
    and the result row follows the last one), two calls in a row agree with
    the context's own diagnostics of the same state."""
    import torch

    from paper_1406_2686_gb300 import vefd

    nx, ny, nz = 256, 128, 256
    L2 = 100.0
    lat = vefd.Lattice(lattice=vefd.D3Q19, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=0.21, eta_B=0.35)
    lat.set_wall_shear(0.02)
    lat.set_fenep(100.0, 0.14, L2, 1e-3, 1, 1)
    lat.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, 32.0, 2.0, 0.1, 5.0, 5, 1e-3)
    stream = lat.stream.cuda_stream
    for call in range(2):
        lat.step(4)
        ref = lat.diagnostics()
        f = _fields(lat, vefd)
        torch.cuda.synchronize()
        got = vefd.vefd_diagnostics_noalloc(1, nx, ny, nz, 2, L2, f[vefd.RHO_A].data_ptr(), f[vefd.RHO_B].data_ptr(),
                                            f[vefd.U].data_ptr(), f[vefd.C].data_ptr(), stream)
        _compare(ref, got)
        del f
    lat.close()


def test_noalloc_concurrent_host_threads():
    """Eight host threads call the entry point at the same time, each on its
    own stream, over four different lattices.  The calls share the one
    scratch array, so the library serialises them; every call returns exactly
    (bit for bit) what a lone call on the same fields returned."""
    import threading

    import torch

    from paper_1406_2686_gb300 import vefd

    L2 = 100.0
    cases = []
    for i, (nx, ny, nz) in enumerate([(48, 32, 40), (64, 32, 32), (40, 24, 56), (96, 64, 48)]):
        lat = vefd.Lattice(lattice=vefd.D3Q19, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=0.21,
                           eta_B=0.35)
        lat.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, 6.0 + 2 * i, 2.0, 0.1, 5.0, 3, 1e-3)
        lat.set_wall_shear(0.02 + 0.01 * i)
        lat.set_fenep(50.0, 0.14, L2, 1e-3, 1, 1)
        lat.step(30 + 10 * i)
        f = _fields(lat, vefd)
        torch.cuda.synchronize()
        cases.append(((nx, ny, nz), f, lat))
    s0 = torch.cuda.Stream()

    def call(case, stream):
        (nx, ny, nz), f, _ = case
        return vefd.vefd_diagnostics_noalloc(vefd.D3Q19, nx, ny, nz, 2, L2, f[vefd.RHO_A].data_ptr(),
                                             f[vefd.RHO_B].data_ptr(), f[vefd.U].data_ptr(), f[vefd.C].data_ptr(),
                                             stream.cuda_stream)

    alone = [np.array(call(c, s0)) for c in cases]
    results, errors = {}, []
    start = threading.Barrier(8)

    def worker(t):
        try:
            stream = torch.cuda.Stream()
            start.wait()
            got = [np.array(call(cases[(t + r) % 4], stream)) for r in range(24)]
            results[t] = got
        except Exception as e:  # reported below, on the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    assert not errors, errors
    assert len(results) == 8
    for t, got in results.items():
        for r, v in enumerate(got):
            assert np.array_equal(v, alone[(t + r) % 4]), (t, r)
    for _, _, lat in cases:
        lat.close()
