"""The bounds-checked debug library (GPU required).

compute-sanitizer is not available on this machine; instead the library is
built a second time with VEFD_BOUNDS_CHECK, where every neighbour index the
step kernels compute (pushes, density and stress gathers, the FENE-P
stencil) is checked against the lattice before the access.  Run in a child
process on the odd and ragged shapes of the parity variants and the lattices
of whole tiles that admit partial densities (post mode 3), every kernel
choice they admit, the step graph and a batched ensemble: no index leaves
the lattice (guard bit VEFD_ST_BOUNDS stays clear), and the checked build
still matches the oracle after three steps.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
import numpy as np
from paper_1406_2686_gb300 import build_lib, vefd
from pairs import Pair, rel_l2
from test_parity_gpu import PARTS_CASES, VARIANTS
from test_ensemble_gpu import BATCH_BOXES, make
L = vefd.load()
assert L._name == build_lib.LIB_DEBUG, L._name
out = {"cases": 0, "bounds": [], "parity": []}
cases = sorted(VARIANTS.items()) + sorted(("parts_" + k, v) for k, v in PARTS_CASES.items())
for name, v in cases:
    P = Pair(**v)
    P.init_random(seed=5)
    P.step(3)
    bits = P.g.status()
    out["cases"] += 1
    if bits & vefd.ST_BOUNDS:
        out["bounds"].append(name)
    g, o = P.both("pops")
    if rel_l2(g, o) > 1e-6 or bits:
        out["parity"].append([name, rel_l2(g, o), bits])
    for tile in range(6):
        for post in range(4):
            Q = Pair(**v)
            try:
                Q.g.set_kernel_config(tile, post)
            except vefd.VefdError:
                continue
            Q.init_random(seed=5)
            for slabs in (0, 2):
                try:
                    Q.g.set_step_graph(slabs, 4)
                except vefd.VefdError:
                    continue
                Q.g.step(9)
            out["cases"] += 1
            if Q.g.status() & vefd.ST_BOUNDS:
                out["bounds"].append([name, tile, post])
ens = [make(b, seed=40 + i) for i, b in enumerate(BATCH_BOXES)]
E = vefd.Ensemble(ens)
for tile in (0, 1):
    E.set_tile(tile)
    E.step(17, chunk=4)
    out["cases"] += 1
    if any(L_.status() & vefd.ST_BOUNDS for L_ in ens):
        out["bounds"].append(["ensemble", tile])
print(json.dumps(out))
"""


def test_bounds_checked_library_on_odd_shapes():
    from paper_1406_2686_gb300 import build_lib
    build_lib.build(debug=True)
    env = dict(os.environ, VEFD_DEBUG_LIB="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}],
                       env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print("bounds-checked cases:", out["cases"])
    assert out["cases"] > 100
    assert out["bounds"] == [], out["bounds"]
    assert out["parity"] == [], out["parity"]
