"""The stored FP64 oracle samples of the 256 x 128 x 256 droplet (written by
oracle/make_droplet256_reference.py, which runs only the oracle) against the
sources they were written from: the oracle's source hash, the parameters of
the set-up and the shapes of the stored planes.  A change to the oracle makes
the samples stale; this test then fails until they are written again."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))

import make_droplet256_reference as ref  # noqa: E402

SAMPLES = [os.path.join(ROOT, "tests", "golden", "droplet256_fp64_%d.npz" % n) for n in (2000, 5000)]


@pytest.mark.parametrize("path", SAMPLES, ids=["2000_steps", "5000_steps"])
def test_sample_matches_oracle_sources(path):
    assert os.path.exists(path), path
    z = np.load(path)
    meta = json.loads(str(z["meta"]))
    assert meta["oracle_sha"] == ref.source_sha()
    assert meta["seed"] == ref.SEED
    assert str(meta["steps"]) in os.path.basename(path)
    for k, v in ref.droplet_params().items():
        assert meta["params"][k] == pytest.approx(v, rel=1e-12, abs=0), k
    nx, ny, nz = ref.NX, ref.NY, ref.NZ
    assert z["zplane"].shape == (11, ny, nx) and z["yplane"].shape == (11, nz, nx)
    assert z["zplane"].dtype == np.float64 and np.all(np.isfinite(z["zplane"])) and np.all(np.isfinite(z["yplane"]))
    assert z["diag"].shape == (16,) and 0.0 < z["diag"][10] < 1.0   # the deformation D
    # the stored densities are those of a droplet: A-rich inside, B-rich outside
    rA = z["zplane"][0]
    assert rA[ny // 2, nx // 2] > 1.5 and rA[0, 0] < 0.5
