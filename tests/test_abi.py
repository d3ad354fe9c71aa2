"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/vefd.h, and validates arguments on the host (no GPU
calls are made here)."""
import ctypes
import os
import re

import pytest

from paper_1406_2686_gb300 import build_lib, vefd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vefd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vefd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return vefd.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(vefd.EXPORTS) == names


def test_network_kernels_are_exported(lib):
    """Every entry point of include/vefd_nn.h (the warm-start network) is
    exported and bound; arguments are checked on the host."""
    from paper_1406_2686_gb300 import nn
    src = open(os.path.join(ROOT, "include", "vefd_nn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(vefd_nn_[a-z_0-9]+)\s*\(", src)))
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(nn.NN_EXPORTS) == names
    L = nn.L()
    # K not a multiple of 8, NULL operands: refused before any launch
    assert L.vefd_nn_gemm_bf16(None, 8, None, 8, None, 8, 128, 16, 16, 0, None, None) == nn.ERR_ARG
    assert L.vefd_nn_im2col3d(None, 1, 8, 8, 8, 4, 1, 112, None, None, None) == nn.ERR_ARG
    assert L.vefd_nn_adam(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == nn.ERR_ARG


def test_build_targets_sm_103a():
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cfg(**kw):
    d = dict(lattice=vefd.D3Q19, nx=8, ny=6, nz=4, ncomp=2, walls=1, G=1.5, eta_A=0.2, eta_B=0.3, delta=0.1,
             external_memory=1)
    d.update(kw)
    return vefd.vefd_config(**d)


def test_required_bytes_matches_layout(lib):
    cfg = _cfg()
    n = vefd.vefd_required_bytes(cfg)
    N = 8 * 6 * 4
    # two population buffers, densities, velocity, C twice, AB2 history, debug planes
    assert n >= 4 * N * (2 * 2 * 19 + 2 + 3 + 3 * 6 + 10)
    assert n % 256 == 0


@pytest.mark.parametrize("bad", [dict(lattice=7), dict(nx=0), dict(lattice=vefd.D2Q9, nz=2), dict(ny=2),
                                 dict(ncomp=3), dict(eta_A=0.0), dict(delta=-1.0), dict(G=float("nan"))])
def test_create_rejects_bad_config(lib, bad):
    cfg = _cfg(**bad)
    h = ctypes.c_void_p()
    st = lib.vefd_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == vefd.ERR_ARG and not h.value


def test_parameter_validation_on_host(lib):
    cfg = _cfg()
    ctx = vefd.vefd_create(cfg, 0)
    try:
        assert lib.vefd_set_wall_shear(ctx, 0.2) == vefd.ERR_ARG
        assert "Mach" in vefd.vefd_last_error(ctx)
        assert lib.vefd_set_wall_shear(ctx, 0.05) == vefd.OK
        assert lib.vefd_set_fenep(ctx, -1.0, 0.1, 100.0, 0.0, 0, 1) == vefd.ERR_ARG
        assert lib.vefd_set_fenep(ctx, 10.0, 0.1, 2.0, 0.0, 0, 1) == vefd.ERR_ARG
        assert lib.vefd_set_fenep(ctx, 10.0, 0.1, 100.0, 0.2, 0, 1) == vefd.ERR_ARG  # kappa >= 1/6 in 3D
        assert lib.vefd_set_fenep(ctx, 10.0, 0.1, 100.0, 0.0, 2, 1) == vefd.ERR_ARG
        assert lib.vefd_set_fenep(ctx, 10.0, 0.1, 100.0, 1e-3, 1, 1) == vefd.OK
        assert lib.vefd_set_body_force(ctx, float("inf"), 0.0, 0.0) == vefd.ERR_ARG
        # nothing is bound yet: stepping and reading are refused, not attempted
        assert lib.vefd_step(ctx, 1) == vefd.ERR_STATE
        assert lib.vefd_bind_device_memory(ctx, ctypes.c_void_p(0x1001), 1 << 30) == vefd.ERR_ARG  # misaligned
        assert lib.vefd_bind_device_memory(ctx, ctypes.c_void_p(0x1000), 16) == vefd.ERR_ARG  # too small
        sz = ctypes.c_size_t()
        assert lib.vefd_field_bytes(ctx, vefd.POPS, ctypes.byref(sz)) == vefd.OK and sz.value == 4 * 2 * 19 * 192
        assert lib.vefd_field_bytes(ctx, vefd.C, ctypes.byref(sz)) == vefd.OK and sz.value == 4 * 6 * 192
        assert lib.vefd_field_bytes(ctx, 99, ctypes.byref(sz)) == vefd.ERR_ARG
        n = ctypes.c_int()
        assert lib.vefd_kernels_per_step(ctx, ctypes.byref(n)) == vefd.OK and n.value == 2
    finally:
        vefd.vefd_destroy(ctx)


def test_step_graph_and_ensemble_argument_checks(lib):
    """The step-graph, wait self-test and ensemble configuration calls check
    their arguments on the host before touching the device."""
    cfg = _cfg()
    ctx = vefd.vefd_create(cfg, 0)
    try:
        for slabs, chunk in ((-2, 256), (65, 256), (8, 3), (8, 0)):
            assert lib.vefd_set_step_graph(ctx, slabs, chunk) == vefd.ERR_ARG
        for slabs in (-1, 0, 1, 2, 8):
            assert lib.vefd_set_step_graph(ctx, slabs, 64) == vefd.OK
        assert lib.vefd_prepare_step_graph(ctx) == vefd.ERR_STATE  # nothing bound
        assert lib.vefd_prepare_steps(ctx, 20) == vefd.ERR_STATE
        assert lib.vefd_wait_selftest(ctx, 2) == vefd.ERR_ARG
        assert lib.vefd_wait_selftest(ctx, 0) == vefd.ERR_STATE
    finally:
        vefd.vefd_destroy(ctx)
    assert lib.vefd_set_step_graph(None, 8, 64) == vefd.ERR_ARG
    assert lib.vefd_prepare_step_graph(None) == vefd.ERR_ARG
    assert lib.vefd_prepare_steps(None, 20) == vefd.ERR_ARG
    assert lib.vefd_ensemble_set_batched(None, 1) == vefd.ERR_ARG
    assert lib.vefd_ensemble_set_config(None, 1, 0) == vefd.ERR_ARG
    assert lib.vefd_ensemble_autotune(None, 64, 32, None) == vefd.ERR_ARG
    assert lib.vefd_ensemble_is_batched(None) == 0
    assert lib.vefd_ensemble_set_groups(None, 2) == vefd.ERR_ARG
    assert lib.vefd_ensemble_set_tile(None, 1) == vefd.ERR_ARG
    assert lib.vefd_ensemble_get_tile(None, ctypes.byref(ctypes.c_int())) == vefd.ERR_ARG
    g = ctypes.c_int()
    assert lib.vefd_ensemble_get_groups(None, ctypes.byref(g)) == vefd.ERR_ARG
    b, z = ctypes.c_int(), ctypes.c_int()
    assert lib.vefd_ensemble_get_config(None, ctypes.byref(b), ctypes.byref(z)) == vefd.ERR_ARG


def test_d2q9_field_sizes(lib):
    cfg = _cfg(lattice=vefd.D2Q9, nz=1, ncomp=1)
    ctx = vefd.vefd_create(cfg, 0)
    try:
        assert vefd.vefd_field_bytes(ctx, vefd.POPS) == 4 * 9 * 48
        assert vefd.vefd_field_bytes(ctx, vefd.U) == 4 * 2 * 48
        assert vefd.vefd_field_bytes(ctx, vefd.C) == 4 * 4 * 48
    finally:
        vefd.vefd_destroy(ctx)


_NOALLOC_ARGS = r"""
import ctypes, sys
sys.path.insert(0, %r)
from paper_1406_2686_gb300 import vefd
lib = vefd.load(build_if_missing=False)
out = (ctypes.c_double * 16)()
p = ctypes.c_void_p(256)  # never dereferenced: every case is refused on the host
cases = [
    (1, 257, 128, 256, 2, 100.0, p, p, p, p),  # one x-row beyond the 8,388,608-node scratch capacity
    (1, 4096, 4096, 4096, 2, 100.0, p, p, p, p),
    (0, 8, 8, 2, 1, 100.0, p, None, p, p),     # D2Q9 needs nz == 1
    (1, 8, 8, 8, 2, 100.0, p, None, p, p),     # two components need rho_B
    (1, 8, 8, 8, 1, 2.0, p, None, p, p),       # L^2 must exceed 3
    (2, 8, 8, 8, 1, 100.0, p, None, p, p),     # unknown lattice
    (1, 0, 8, 8, 1, 100.0, p, None, p, p),     # empty lattice
    (1, 8, 8, 8, 3, 100.0, p, p, p, p),        # three components
    (1, 8, 8, 8, 1, 100.0, None, None, p, p),  # NULL input
]
print(",".join(str(lib.vefd_diagnostics_noalloc(*c, None, out)) for c in cases))
print(lib.vefd_diagnostics_noalloc(1, 8, 8, 8, 1, 100.0, p, None, p, p, None, None))
"""


def test_noalloc_argument_checks_without_a_device(lib):
    """The allocation-free diagnostics refuse bad sizes, the oversize lattice
    and NULL inputs on the host, before any CUDA call: run with no visible
    device, so that a check that let a case through would answer
    VEFD_ERR_CUDA (no device) rather than launch on placeholder pointers."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _NOALLOC_ARGS % root], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    codes, null_out = r.stdout.split()
    assert codes.split(",") == [str(vefd.ERR_ARG)] * 9, codes
    assert int(null_out) == vefd.ERR_ARG


def test_lattice_size_limit(lib):
    """One lattice holds at most 2^31 / 40 nodes (32-bit plane offsets): the
    largest admitted size is sized, one node more is refused, with and
    without walls (the check needs no device)."""
    limit = (1 << 31) // 40
    assert limit == 53687091
    assert vefd.vefd_required_bytes(_cfg(nx=limit, ny=1, nz=1, lattice=vefd.D2Q9, walls=0)) > 0
    with pytest.raises(vefd.VefdError):
        vefd.vefd_required_bytes(_cfg(nx=limit + 1, ny=1, nz=1, lattice=vefd.D2Q9, walls=0))
    # 512 x 256 x 409 = 53,608,448 nodes fit; 512 x 256 x 410 = 53,739,520 do not
    assert vefd.vefd_required_bytes(_cfg(nx=512, ny=256, nz=409)) > 0
    with pytest.raises(vefd.VefdError):
        vefd.vefd_required_bytes(_cfg(nx=512, ny=256, nz=410))
