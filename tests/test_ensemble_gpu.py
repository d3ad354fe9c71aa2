"""Kernel choices, the autotuner and ensembles of lattices (GPU required).

Every kernel choice runs the method's arithmetic (Sec. 2.1 collide-stream,
Sec. 2.2 FENE-P update) in the same order, and an ensemble only changes how
the launches of independent lattices are issued; so all comparisons here are
bit for bit against plain stepping of one lattice.
"""
import numpy as np
import pytest

from paper_1406_2686_gb300 import inputs

pytestmark = pytest.mark.gpu

BOXES = [
    dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=1),
    dict(lattice=1, nx=36, ny=10, nz=7, ncomp=2, walls=1, G=1.5, u_wall=-0.02, eta_p=0.1, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=-1),
    dict(lattice=1, nx=32, ny=8, nz=5, ncomp=1, walls=0, eta_p=0.1, tau_p=20.0, L2=50.0, kappa=0.02,
         fext=(1e-5, -1e-5, 0.0)),
    dict(lattice=0, nx=64, ny=13, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=30.0, L2=40.0, kappa=0.01, phase=-1),
    dict(lattice=1, nx=32, ny=8, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.15, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=1, coupling=1),
    dict(lattice=1, nx=9, ny=10, nz=11, ncomp=1, walls=0, fext=(3e-5, 1e-5, -2e-5), eta_p=0.2, tau_p=20.0,
         L2=30.0, kappa=0.03),
    dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=1, precision=1),
]


def make(box, seed):
    from paper_1406_2686_gb300 import vefd
    p = dict(box)
    lat = p.pop("lattice")
    nz = p.pop("nz", 1) if lat == 1 else 1
    L = vefd.Lattice(lattice=lat, nx=p["nx"], ny=p["ny"], nz=nz, ncomp=p["ncomp"], walls=p["walls"],
                     G=p.get("G", 0.0), eta_A=0.2, eta_B=0.3, delta=0.1, precision=p.get("precision", 0))
    L.set_wall_shear(p.get("u_wall", 0.0))
    L.set_body_force(*p.get("fext", (0.0, 0.0, 0.0)))
    L.set_fenep(p["tau_p"], p["eta_p"], p["L2"], p.get("kappa", 0.0), p.get("phase", 0), 1)
    L.set_polymer_coupling(p.get("coupling", 0))
    ndim, nc = (3, 6) if lat == 1 else (2, 4)
    rA, rB, u, C = inputs.random_state(p["nx"], p["ny"], nz, ndim, p["ncomp"], nc, seed=seed)
    L.init_fields(*[inputs.to_f32_exact(a) for a in (rA, rB, u, C)])
    return L


def state(L):
    from paper_1406_2686_gb300 import vefd
    return L.read(vefd.POPS), L.read(vefd.C), L.read(vefd.RPREV)


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(state(a), state(b)))


@pytest.mark.parametrize("k", [0, 3, 4])
def test_kernel_choices_bit_identical(k):
    """Tiles 0-2 with the tiled (1) or z-marching (2) densities pass give the
    same bits.  The persistent tiles (3-5) are compiled separately and may
    contract multiply-adds differently, and the column march with fused
    densities (0) sums each new density in another order: both agree to FP32
    rounding."""
    ref = make(BOXES[k], seed=11)
    ref.set_kernel_config(0, 1)
    ref.step(5)
    seen = set()
    for post in (1, 2):
        for tile in range(6):
            L = make(BOXES[k], seed=11)
            L.set_kernel_config(tile, post)
            seen.add(L.kernel_config())
            L.step(5)
            if tile < 3:
                assert same(L, ref), (tile, post, L.kernel_config())
            else:
                for a, r in zip(state(L), state(ref)):
                    assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r), (tile, post)
            assert L.status() == 0
    F = make(BOXES[k], seed=11)
    F.set_kernel_config(0, 0)
    F.step(5)
    for a, r in zip(state(F), state(ref)):
        assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r)
    assert F.status() == 0
    # these 3-D boxes admit all three tiles (and their persistent forms); the
    # 64 x 13 D2Q9 box is too low for 32 x 16
    assert {t for t, _ in seen} == ({0, 1, 2, 3, 4, 5} if BOXES[k]["lattice"] == 1 else {0, 1, 3, 4})


def test_kernel_config_reports_and_rejects():
    from paper_1406_2686_gb300 import vefd
    L = make(BOXES[0], seed=1)
    assert L.kernel_config() == (0, 2)  # 64 x 16 x 6: default tiles + z-marching pass
    L.set_kernel_config(0, 0)
    assert L.kernel_config() == (0, 0)  # and it admits the column march
    L.set_kernel_config(2, 1)
    assert L.kernel_config() == (2, 1)
    L.set_kernel_config(4, 2)
    assert L.kernel_config() == (4, 2)
    # partial densities: tiles 32 x 4 x 2 and 32 x 2 x 4 only, else the z-marching pass
    L.set_kernel_config(0, 3)
    assert L.kernel_config() == (0, 3)
    L.set_kernel_config(1, 3)
    assert L.kernel_config() == (1, 2)  # NZ = 6 is no multiple of the 32 x 2 x 4 tile's 4 planes
    W = make(dict(BOXES[0], nz=8), seed=1)
    W.set_kernel_config(1, 3)
    assert W.kernel_config() == (1, 3)
    L.set_kernel_config(2, 3)
    assert L.kernel_config() == (2, 2)
    L.set_kernel_config(3, 3)
    assert L.kernel_config() == (3, 2)
    T = make(BOXES[1], seed=1)  # 36 x 10 x 7: tiles fit, the column does not
    assert T.kernel_config() == (0, 1)
    T.set_kernel_config(0, 3)
    assert T.kernel_config() == (0, 1)
    S = make(BOXES[5], seed=1)  # 9 x 10 x 11: no staged tile fits
    assert S.kernel_config() == (-1, -1)
    for bad in ((6, 0), (-1, 0), (0, 4)):
        with pytest.raises(vefd.VefdError) as ei:
            L.set_kernel_config(*bad)
        assert ei.value.status == vefd.ERR_ARG


def test_autotune_leaves_state_and_picks_fastest():
    L = make(BOXES[0], seed=4)
    R = make(BOXES[0], seed=4)
    L.step(3)
    R.step(3)
    times = L.autotune(steps=20)
    assert len(times) == 18
    measured = [(t, i) for i, t in enumerate(times) if t >= 0]
    assert len(measured) >= 13  # 1 fused + 6 tiled + 6 z-marching
    best = min(measured)[1]
    assert L.kernel_config() == (best % 6, best // 6)
    assert L.steps_done == 3
    assert same(L, R)
    R.set_kernel_config(*L.kernel_config())
    L.step(4)
    R.step(4)
    assert same(L, R)


def test_ensemble_matches_single_lattices():
    """Seven uneven boxes (D3Q19/D2Q9, one/two components, both feedback
    couplings, FP32/FP16 storage) stepped as one graph equal each box stepped
    alone, across the Euler start, graph replays, an odd remainder, a
    parameter change and a kernel-choice change."""
    from paper_1406_2686_gb300 import vefd
    ens_members = [make(b, seed=20 + i) for i, b in enumerate(BOXES)]
    alone = [make(b, seed=20 + i) for i, b in enumerate(BOXES)]
    E = vefd.Ensemble(ens_members)
    E.step(37, chunk=8)             # 1 eager start, 4 replays, 4 eager steps
    for L in alone:
        L.step(37)
    for a, b in zip(ens_members, alone):
        assert a.steps_done == 37
        assert same(a, b)
    E.step(1, chunk=8)              # odd parity afterwards
    E.step(16, chunk=8)             # re-captured for the other parity
    ens_members[0].set_wall_shear(0.01)
    ens_members[2].set_kernel_config(4, 1)
    E.step(20, chunk=4)             # re-captured for the new parameters
    for L in alone:
        L.step(17)
    alone[0].set_wall_shear(0.01)
    alone[2].set_kernel_config(4, 1)
    for L in alone:
        L.step(20)
    for a, b in zip(ens_members, alone):
        assert a.steps_done == 74 == b.steps_done
        assert same(a, b)
        assert a.status() == 0
    E.close()


def test_ensemble_errors():
    from paper_1406_2686_gb300 import vefd
    A = make(BOXES[2], seed=1)
    with pytest.raises(vefd.VefdError):
        vefd.Ensemble([A, A])
    E = vefd.Ensemble([A])
    for chunk in (0, 3, -2):
        with pytest.raises(vefd.VefdError) as ei:
            E.step(4, chunk=chunk)
        assert ei.value.status == vefd.ERR_ARG
    E.step(0)
    assert A.steps_done == 0
    E.close()


# D3Q19 boxes that admit the batched launches (NX % 32 == 0, NY % 8 == 0):
# uneven sizes, an odd NZ (a half-empty last lattice tile), walls on and off,
# both feedback couplings, and a box only one lattice tile deep (NZ 2)
BATCH_BOXES = [
    dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=1),
    dict(lattice=1, nx=32, ny=8, nz=5, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=20.0, L2=50.0, kappa=0.02,
         fext=(1e-5, -1e-5, 0.0), phase=-1),
    dict(lattice=1, nx=96, ny=24, nz=9, ncomp=2, walls=1, G=1.5, u_wall=-0.02, eta_p=0.15, tau_p=20.0, L2=50.0,
         kappa=0.01, phase=1, coupling=1),
    dict(lattice=1, nx=32, ny=16, nz=2, ncomp=2, walls=1, G=1.5, u_wall=0.01, eta_p=0.1, tau_p=25.0, L2=40.0,
         kappa=0.01, phase=-1),
    dict(lattice=1, nx=32, ny=8, nz=12, ncomp=2, walls=1, G=1.2, u_wall=0.02, eta_p=0.1, tau_p=20.0, L2=60.0,
         kappa=0.0, phase=1),
]


def close_state(a, b, rel=1e-6):
    """Populations and C within `rel` (relative L2); the AB2 history R, the
    FENE-P right-hand side, is a difference of nearly cancelling terms and is
    allowed 20 times more."""
    return all(np.linalg.norm(x - y) <= r * np.linalg.norm(y)
               for x, y, r in zip(state(a), state(b), (rel, rel, 20 * rel)))


def _batched_vs_alone(boxes, prep, steps=(23, 1, 16)):
    """Steps an ensemble of `boxes` (after prep(L)) with batched launches and
    the same boxes alone; returns both lists."""
    from paper_1406_2686_gb300 import vefd
    ens = [make(b, seed=40 + i) for i, b in enumerate(boxes)]
    alone = [make(b, seed=40 + i) for i, b in enumerate(boxes)]
    for L in ens + alone:
        prep(L)
    E = vefd.Ensemble(ens)
    for seg, n in enumerate(steps):
        E.step(n, chunk=4)
        if n >= 8:
            assert E.batched
        for L in alone:
            L.step(n)
        for k, (a, r) in enumerate(zip(ens, alone)):
            assert close_state(a, r, 1e-3 if a.cfg.precision else 1e-6), (seg, k)
    E.close()
    return ens, alone


def test_batched_ensemble_matches_single_lattices():
    """Two launches per step over all boxes' tiles give each box's own step:
    the same arithmetic as the per-lattice kernels (separately compiled, so
    multiply-add contraction may differ in the last ulp), across the Euler
    start, replays of both parities and an odd remainder."""
    ens, alone = _batched_vs_alone(BATCH_BOXES, lambda L: None)
    for a, b in zip(ens, alone):
        assert a.steps_done == b.steps_done == 40
        assert close_state(a, b)
        assert a.status() == 0


@pytest.mark.parametrize("variant", ["fp32", "fp16", "mrt_chol"])
def test_batched_ensemble_tile_32x8x1(variant):
    """Batched launches with 32 x 8 x 1 lattice tiles give each box's own step
    (FP32 rounding), across the Euler start, replays of both parities and an
    odd remainder, and agree with the 32 x 4 x 2 tiles to the same rounding."""
    from paper_1406_2686_gb300 import vefd
    boxes = [dict(b) for b in BATCH_BOXES]
    prep = lambda L: None
    if variant == "fp16":
        for b in boxes:
            b["precision"] = 1
    elif variant == "mrt_chol":
        def prep(L):
            L.set_collision(1)
            L.set_conformation_update(1)
    rel = 1e-3 if variant == "fp16" else 1e-6
    ens = [make(b, seed=80 + i) for i, b in enumerate(boxes)]
    ref = [make(b, seed=80 + i) for i, b in enumerate(boxes)]
    alone = [make(b, seed=80 + i) for i, b in enumerate(boxes)]
    for L in ens + ref + alone:
        prep(L)
    E, R = vefd.Ensemble(ens), vefd.Ensemble(ref)
    E.set_tile(1)
    assert E.tile == 1 and R.tile == 0
    for n in (23, 1, 16):
        E.step(n, chunk=4)
        R.step(n, chunk=4)
        for L in alone:
            L.step(n)
    assert E.batched and R.batched
    for a, r, c in zip(ens, ref, alone):
        assert close_state(a, c, rel) and close_state(a, r, rel)
        assert a.status() == 0
    with pytest.raises(vefd.VefdError) as ei:
        E.set_tile(2)
    assert ei.value.status == vefd.ERR_ARG
    E.close()
    R.close()


@pytest.mark.parametrize("groups", [1, 2, 4, 9])
def test_batched_ensemble_group_counts_bit_identical(groups):
    """The group count only changes which graph branch a member's tiles are
    launched in: 1, 2, 4 and more groups than members (clamped to one member
    per group) give the default count's bits, and the same state as each box
    stepped alone to FP32 rounding."""
    from paper_1406_2686_gb300 import vefd
    ref = [make(b, seed=60 + i) for i, b in enumerate(BATCH_BOXES)]
    got = [make(b, seed=60 + i) for i, b in enumerate(BATCH_BOXES)]
    alone = [make(b, seed=60 + i) for i, b in enumerate(BATCH_BOXES)]
    R, G = vefd.Ensemble(ref), vefd.Ensemble(got)
    assert R.groups == 0
    G.set_groups(groups)
    assert G.groups == groups
    for n in (23, 1, 16):
        R.step(n, chunk=4)
        G.step(n, chunk=4)
        for L in alone:
            L.step(n)
    assert G.batched and R.batched
    for a, b, c in zip(got, ref, alone):
        assert same(a, b)
        assert close_state(a, c)
    with pytest.raises(vefd.VefdError) as ei:
        G.set_groups(65)
    assert ei.value.status == vefd.ERR_ARG
    R.close()
    G.close()


@pytest.mark.parametrize("variant", ["fp16", "mrt_chol", "one_component"])
def test_batched_ensemble_variants(variant):
    """The batched kernels for 16-bit storage, the moment-space collision with
    the log-Cholesky conformation update, and one-component boxes."""
    boxes = [dict(b) for b in BATCH_BOXES[:3]]
    prep = lambda L: None
    if variant == "fp16":
        for b in boxes:
            b["precision"] = 1
    elif variant == "mrt_chol":
        def prep(L):
            L.set_collision(1)
            L.set_conformation_update(1)
    else:
        for b in boxes:
            b.update(ncomp=1, G=0.0, phase=0)
    ens, alone = _batched_vs_alone(boxes, prep)
    for a, b in zip(ens, alone):
        assert close_state(a, b, 1e-6 if variant != "fp16" else 1e-3)
        assert a.status() == 0


def test_batched_ensemble_selection():
    """Batched launches only where every member allows them; otherwise (and on
    request) one graph branch per member, bit for bit equal to stepping alone."""
    from paper_1406_2686_gb300 import vefd
    A = make(BATCH_BOXES[0], seed=3)
    B = make(BATCH_BOXES[4], seed=4)
    E = vefd.Ensemble([A, B])
    E.step(9, chunk=4)
    assert E.batched
    E.set_batched(False)
    E.step(8, chunk=4)
    assert not E.batched
    E.set_batched(True)
    E.step(8, chunk=4)
    assert E.batched
    B.set_kernel_config(0, 1)  # tiled densities pass: not batchable
    E.step(8, chunk=4)
    assert not E.batched
    E.close()
    # branch mode is bit-identical
    C = make(BATCH_BOXES[0], seed=5)
    D = make(BATCH_BOXES[0], seed=5)
    E = vefd.Ensemble([C])
    E.set_batched(False)
    E.step(13, chunk=4)
    D.step(13)
    assert same(C, D)
    E.close()
    with pytest.raises(vefd.VefdError):
        vefd.vefd_ensemble_set_batched(None, 1)


def test_batched_ensemble_many_members():
    """Forty boxes, two launches per step, each equal to the box stepped alone."""
    from paper_1406_2686_gb300 import vefd
    boxes = []
    for i in range(40):
        b = dict(BATCH_BOXES[i % 5])
        boxes.append(b)
    ens = [make(b, seed=100 + i) for i, b in enumerate(boxes)]
    alone = [make(b, seed=100 + i) for i, b in enumerate(boxes)]
    E = vefd.Ensemble(ens)
    E.step(17, chunk=8)
    assert E.batched
    for L in alone:
        L.step(17)
    for a, b in zip(ens, alone):
        assert close_state(a, b)
        assert a.status() == 0
    E.close()


def test_ensemble_config_and_autotune():
    """The ensemble's own autotuner times graph branches and batched launches
    with two lattice tiles and three z-segment lengths of the densities pass,
    keeps the fastest, and its timed steps are ordinary steps (results as
    stepping alone); an ensemble the batched kernels cannot take only times
    the branches."""
    from paper_1406_2686_gb300 import vefd
    boxes = BATCH_BOXES[:3]
    ens = [make(b, seed=60 + i) for i, b in enumerate(boxes)]
    alone = [make(b, seed=60 + i) for i, b in enumerate(boxes)]
    E = vefd.Ensemble(ens)
    assert E.config == (1, 0)
    E.set_config(True, 3)
    assert E.config == (1, 3)
    E.step(9, chunk=4)                      # 1 eager start, 2 replays with 3-plane segments
    assert E.batched
    times = E.autotune(steps=8, chunk=4)    # 7 x (8 + 4) steps
    assert len(times) == 7 and all(t > 0 for t in times)
    best = int(np.argmin(times))
    b, z = E.config
    assert b == (0 if best == 0 else 1)
    if best > 0:
        assert E.tile == (0 if best < 4 else 1)
    E.step(8, chunk=4)
    total = 9 + 7 * 12 + 8
    for L in alone:
        L.step(total)
    for a, r in zip(ens, alone):
        assert a.steps_done == total
        assert close_state(a, r)
        assert a.status() == 0
    for bad in ((2, 0), (1, -1)):
        with pytest.raises(vefd.VefdError) as ei:
            vefd.vefd_ensemble_set_config(E.ens, *bad)
        assert ei.value.status == vefd.ERR_ARG
    with pytest.raises(vefd.VefdError) as ei:
        E.autotune(steps=6, chunk=4)
    assert ei.value.status == vefd.ERR_ARG
    E.close()
    # a D2Q9 member: no batched launches, only the branches are timed
    F = vefd.Ensemble([make(BOXES[3], seed=5), make(BATCH_BOXES[0], seed=6)])
    times = F.autotune(steps=4, chunk=2)
    assert times[0] > 0 and times[1:] == [-1.0] * 6
    assert F.config[0] == 0
    F.close()


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("case", ["walls", "periodic", "fp16"])
def test_partial_densities_step_graph_bit_identical(case, tile):
    """Post mode 3 (partial densities written by the lattice kernel, completed
    by the z-marching pass) in the pipelined y-slab step graph: bit-identical
    to its own eager launch pairs, over graph replays and odd remainders (a
    slab's tiles push partial sums into the neighbouring slabs' rows, which
    the graph edges order)."""
    box = {"walls": dict(BATCH_BOXES[0], ny=32, nz=8),
           "periodic": dict(BATCH_BOXES[1], ny=32, nz=8),
           "fp16": dict(BATCH_BOXES[0], ny=32, nz=8, precision=1)}[case]
    G = make(box, seed=81)
    R = make(box, seed=81)
    for L in (G, R):
        L.set_kernel_config(tile, 3)
        assert L.kernel_config() == (tile, 3)
    R.set_step_graph(0)
    G.set_step_graph(4, 8)
    assert G.step_graph == (4, 8, True)
    for n in (9, 8, 3, 16, 5):
        G.step(n)
        R.step(n)
        assert same(G, R), n
    assert G.status() == 0 and R.status() == 0


@pytest.mark.parametrize("case", ["walls", "periodic", "equilibrium_coupling", "fp16"])
def test_step_graph_bit_identical(case):
    """The pipelined y-slab step graph (each slab's lattice kernel and
    densities/FENE-P pass a node waiting only for its neighbouring slabs) runs
    the eager step's kernels on row ranges: bit-identical results, across the
    Euler start, replays of both parities, remainder graphs of many sizes
    (more than the four a context keeps) and odd last steps."""
    from paper_1406_2686_gb300 import vefd
    box = {"walls": dict(BATCH_BOXES[0], ny=32),
           "periodic": dict(BATCH_BOXES[1], ny=16, nz=6),
           "equilibrium_coupling": dict(BATCH_BOXES[2], ny=32),
           "fp16": dict(BATCH_BOXES[0], ny=32, precision=1)}[case]
    for slabs in ((2, 4) if box["ny"] == 32 else (2,)):
        G = make(box, seed=71)
        R = make(box, seed=71)
        R.set_step_graph(0)                # eager launch pairs
        assert R.step_graph[2] is False
        G.set_step_graph(slabs, 8)
        assert G.step_graph == (slabs, 8, True)
        calls = (11, 1, 8, 5, 9, 20, 2, 3, 6, 14, 7, 22)
        for k, n in enumerate(calls):
            G.step(n)
            R.step(n)
            assert same(G, R), (slabs, n)
            if k % 2:
                G.prepare_step_graph()     # captures (or keeps) the graph, takes no step
            else:
                G.prepare_steps(calls[(k + 1) % len(calls)])
            assert same(G, R)
        assert G.status() == 0 and G.steps_done == sum(calls)
        G.set_wall_shear(0.005)            # a parameter change re-captures
        R.set_wall_shear(0.005)
        G.step(8)
        R.step(8)
        assert same(G, R)
    # the automatic choice: 8 slabs for NY a multiple of 64, 4 for 32, when
    # every slab holds at least 100,000 nodes; else the whole-lattice form
    assert make(dict(box, nx=128, ny=64, nz=100), seed=1).step_graph == (8, 256, True)   # 102,400 per slab
    assert make(dict(box, nx=128, ny=64, nz=96), seed=1).step_graph == (1, 256, True)    # 98,304 per slab
    assert make(dict(box, nx=128, ny=32, nz=100), seed=1).step_graph == (4, 256, True)
    assert make(dict(box, ny=64), seed=1).step_graph == (1, 256, True)
    assert make(dict(box, ny=16), seed=1).step_graph == (1, 256, True)
    # shapes or choices the graph cannot take step eagerly
    H = make(box, seed=72)
    H.set_step_graph(3, 4)                 # NY not a multiple of 8 * 3
    assert H.step_graph[2] is False
    H.set_step_graph(2, 4)
    H.set_kernel_config(3, 2)              # persistent tile
    assert H.step_graph[2] is False
    for bad in ((65, 4), (2, 3), (-2, 4)):
        with pytest.raises(vefd.VefdError) as ei:
            H.set_step_graph(*bad)
        assert ei.value.status == vefd.ERR_ARG


@pytest.mark.parametrize("k", [0, 3, 4])
@pytest.mark.parametrize("config", [None, (0, 0), (3, 1)])
def test_whole_lattice_graph_bit_identical(k, config):
    """The whole-lattice step graph (eager launch pairs replayed as one graph)
    for lattices and kernel choices the slab split does not take (D2Q9, a
    coupling variant, the column march with fused densities, a persistent
    tile with the tiled pass) gives the eager step's bits across the Euler
    start, replays, parity realignment and eager remainders."""
    box = BOXES[k]
    G = make(box, seed=81)
    R = make(box, seed=81)
    if config is not None:
        G.set_kernel_config(*config)
        R.set_kernel_config(*config)
    R.set_step_graph(0)
    G.set_step_graph(1, 4)
    assert G.step_graph == (1, 4, True)
    for n in (11, 1, 8, 5, 9, 2, 6, 3):
        G.step(n)
        R.step(n)
        assert same(G, R), (n, G.kernel_config())
    assert G.status() == 0 and G.steps_done == 45

