"""Host-side logic of the benchmark (no GPU): the ensemble parameter sweep
draws deterministic set-ups inside the stated ranges, and the headline
workload's parameters follow from Ca = 0.1 and De = 1."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ensemble_sweep_ranges_and_determinism():
    a, dropped = bench.ensemble_setups(screen=0)
    b, _ = bench.ensemble_setups(screen=0)
    assert dropped == 0 and len(a) == 64
    assert [(s.dims, s.Ca, s.De, s.conf, s.lam, s.phase) for s in a] == \
        [(s.dims, s.Ca, s.De, s.conf, s.lam, s.phase) for s in b]
    for s in a:
        nx, ny, nz = s.dims
        assert nx in (32, 64, 96) and 32 <= ny <= 96 and 32 <= nz <= 96 and ny % 8 == 0 and nz % 8 == 0
        assert 0.05 <= s.Ca <= 0.3 and 0.1 <= s.De <= 4.0 and 0.3 <= s.conf <= 0.8 and 0.5 <= s.lam <= 2.0
        assert s.phase in (-1, 1)
        assert 2.0 * s.R <= 0.8 * min(nx, nz) + 1e-12 and s.u_wall <= 0.08
        assert math.isclose(s.R, s.conf * ny / 2.0)
    # the sweep covers both phases and a spread of every parameter
    assert {s.phase for s in a} == {-1, 1}
    assert max(s.conf for s in a) - min(s.conf for s in a) > 0.3
    assert max(s.De for s in a) / min(s.De for s in a) > 10.0


def test_small_ensemble_and_headline_setup():
    small = bench.small_setups()
    assert len(small) == 256 and all(s.dims == (32, 16, 16) for s in small)
    S = bench.Setup("droplet128", "fp32")
    assert (S.NX, S.NY, S.NZ, S.R) == (128, 64, 128, 16.0)
    assert S.step_bytes == 400 and S.pop_bytes == 304
    assert math.isclose(S.u_wall, S.gdot * S.NY / 2.0)
    assert bench.Setup("droplet128", "fp16").step_bytes == 256


@pytest.mark.parametrize("name", ["lattice_collide_stream", "densities_fenep_fd"])
def test_recorded_traffic_matches_sources_or_is_null(name):
    """The committed DRAM traffic is reported only for the step-kernel
    sources and the kernel choice it was captured on."""
    import json
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[name]
    got = bench.recorded_traffic(name)
    if rec["kernel_sha"] == bench.kernel_source_hash():
        assert got == rec["dram_bytes_read"] + rec["dram_bytes_write"] == rec["dram_bytes_per_launch"]
        assert bench.recorded_traffic(name, rec["kernel_config"]) == got
        assert bench.recorded_traffic(name, [rec["kernel_config"][0] + 1, rec["kernel_config"][1]]) is None
    else:
        assert got is None


def test_kernel_source_hash_covers_the_step_kernels():
    """Every local include of the step kernels' translation units is in the
    hashed set, so a change to any of them invalidates the traffic record."""
    import re
    csrc = os.path.join(ROOT, "paper_1406_2686_gb300", "csrc")
    todo, seen = ["lbm_kernels.cu", "fd_kernels.cu"], set()
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        todo += re.findall(r'#include "([^"]+)"', open(os.path.join(csrc, f)).read())
    assert seen == set(bench.STEP_KERNEL_SOURCES)
