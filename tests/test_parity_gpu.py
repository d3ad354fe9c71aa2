"""Parity of the CUDA library with the FP64 oracle (GPU required).

Tolerances follow from FP32 storage: one step moves populations and C by
rounding of ~6e-8 relative, so stage-wise comparisons use 1e-5 relative L2;
after 2000 steps the contract is 1e-5 relative L2 in u and C and 1e-6
relative total-mass drift.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from paper_1406_2686_gb300 import inputs

from pairs import Pair, dev_rel_l2, max_abs, rel_l2

pytestmark = pytest.mark.gpu

VARIANTS = {
    "d2q9_1c_walls": dict(lattice=0, nx=37, ny=13, ncomp=1, walls=1, u_wall=0.03, fext=(2e-5, -1e-5, 0.0),
                          eta_p=0.05, tau_p=40.0, L2=50.0, kappa=0.02, phase=0),
    "d2q9_2c_periodic": dict(lattice=0, nx=33, ny=20, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=30.0, L2=40.0,
                             kappa=0.01, phase=1),
    "d2q9_2c_walls_matrix": dict(lattice=0, nx=24, ny=17, ncomp=2, walls=1, G=1.2, u_wall=-0.02, eta_p=0.08,
                                 tau_p=25.0, L2=60.0, kappa=0.0, phase=-1),
    "d3q19_2c_walls": dict(lattice=1, nx=35, ny=7, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.04, eta_p=0.12,
                           tau_p=50.0, L2=100.0, kappa=1e-3, phase=1, fext=(1e-5, 0.0, 2e-6)),
    "d3q19_1c_periodic": dict(lattice=1, nx=9, ny=10, nz=11, ncomp=1, walls=0, fext=(3e-5, 1e-5, -2e-5),
                              eta_p=0.2, tau_p=20.0, L2=30.0, kappa=0.03),
    "d3q19_2c_nx1": dict(lattice=1, nx=1, ny=5, nz=3, ncomp=2, walls=1, G=1.4, u_wall=0.02, eta_p=0.1,
                         tau_p=15.0, L2=40.0, phase=1),
    "d3q19_2c_nz1": dict(lattice=1, nx=40, ny=9, nz=1, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1,
                         tau_p=15.0, L2=40.0, phase=-1, kappa=0.01),
    # shapes taken by the TMA-staged lattice kernel (rows of 16-byte multiples),
    # with ragged last tiles in y and z
    "d3q19_2c_tma_ragged": dict(lattice=1, nx=36, ny=10, nz=7, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1,
                                tau_p=20.0, L2=50.0, kappa=0.01, phase=1, fext=(0.0, 0.0, 1e-5)),
    "d3q19_1c_tma_one_tile": dict(lattice=1, nx=32, ny=4, nz=2, ncomp=1, walls=0, eta_p=0.1, tau_p=20.0, L2=50.0,
                                  fext=(1e-5, 0.0, 0.0)),
    "d2q9_2c_tma_periodic": dict(lattice=0, nx=64, ny=13, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=30.0, L2=40.0,
                                 kappa=0.01, phase=-1),
    "d2q9_1c_tma_walls": dict(lattice=0, nx=44, ny=9, ncomp=1, walls=1, u_wall=0.02, eta_p=0.05, tau_p=40.0,
                              L2=50.0, kappa=0.02, fext=(1e-5, 0.0, 0.0)),
    # shapes taken by the z-marching densities/FD pass (NX % 32 == 0, NY % 8 == 0);
    # the last one splits z into segments of two planes
    "d3q19_2c_zm_walls": dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1,
                              tau_p=20.0, L2=50.0, kappa=0.01, phase=1),
    "d3q19_1c_zm_periodic": dict(lattice=1, nx=32, ny=8, nz=5, ncomp=1, walls=0, eta_p=0.1, tau_p=20.0, L2=50.0,
                                 kappa=0.02, fext=(1e-5, -1e-5, 0.0)),
    "d3q19_2c_zm_segments": dict(lattice=1, nx=256, ny=40, nz=8, ncomp=2, walls=1, G=1.5, u_wall=0.02, eta_p=0.1,
                                 tau_p=20.0, L2=50.0, kappa=0.01, phase=-1),
    # several columns in x and y and several z-segments (periodic y, NX = 96)
    "d3q19_2c_fused_wide": dict(lattice=1, nx=96, ny=24, nz=12, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=20.0,
                                L2=50.0, kappa=0.01, phase=1, fext=(1e-5, 0.0, -1e-5)),
    # polymer stress in the equilibrium (Eq. MODEtransformation) instead of a body force
    "d3q19_2c_eqcoupling": dict(lattice=1, nx=32, ny=8, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.15,
                                tau_p=20.0, L2=50.0, kappa=0.01, phase=1, coupling=1),
    "d2q9_1c_eqcoupling": dict(lattice=0, nx=37, ny=13, ncomp=1, walls=1, u_wall=0.03, eta_p=0.1, tau_p=30.0,
                               L2=50.0, kappa=0.01, coupling=1),
    # moment-space collision with the paper's relaxation times (Sec. 2), on the
    # register, TMA and z-marching paths
    "d3q19_2c_mrt_walls": dict(lattice=1, nx=35, ny=7, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.04, eta_p=0.12,
                               tau_p=50.0, L2=100.0, kappa=1e-3, phase=1, fext=(1e-5, 0.0, 2e-6), collision=1),
    "d3q19_2c_mrt_zm": dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1,
                            tau_p=20.0, L2=50.0, kappa=0.01, phase=-1, collision=1),
    "d2q9_2c_mrt_tma": dict(lattice=0, nx=64, ny=13, ncomp=2, walls=0, G=1.5, eta_p=0.1, tau_p=30.0, L2=40.0,
                            kappa=0.01, phase=-1, collision=1),
    "d2q9_1c_mrt_walls": dict(lattice=0, nx=37, ny=13, ncomp=1, walls=1, u_wall=0.03, fext=(2e-5, -1e-5, 0.0),
                              eta_p=0.05, tau_p=40.0, L2=50.0, kappa=0.02, collision=1),
    # Cholesky scheme for the conformation tensor (Sec. 2)
    "d3q19_2c_chol_zm": dict(lattice=1, nx=64, ny=16, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.1,
                             tau_p=20.0, L2=50.0, kappa=0.01, phase=1, chol=1),
    "d2q9_1c_chol_walls": dict(lattice=0, nx=37, ny=13, ncomp=1, walls=1, u_wall=0.03, fext=(2e-5, -1e-5, 0.0),
                               eta_p=0.05, tau_p=40.0, L2=50.0, kappa=0.02, chol=1),
    "d3q19_1c_chol_tma": dict(lattice=1, nx=36, ny=10, nz=7, ncomp=1, walls=1, u_wall=0.03, eta_p=0.1, tau_p=20.0,
                              L2=50.0, kappa=0.01, chol=1),
    # the paper's combination: moment space, stress in the equilibrium, Cholesky
    "d3q19_2c_paper": dict(lattice=1, nx=32, ny=8, nz=6, ncomp=2, walls=1, G=1.5, u_wall=0.03, eta_p=0.15,
                           tau_p=20.0, L2=50.0, kappa=0.01, phase=1, coupling=1, collision=1, chol=1),
}


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(0)


# Deformation tolerances after many steps.  C and sigma_P are compared both
# whole (the contract) and as departures from the identity, which is the
# polymer deformation itself: ||C - I|| is 5-50 times smaller than ||C|| in
# these set-ups, so the same absolute FP32 error weighs that much more.
DEV_TOL = 1e-4


def check_deformation(P, label=""):
    """Relative L2 of C - I and sigma_P - I against the oracle; returns both."""
    eC = dev_rel_l2(*P.both("C"))
    eS = dev_rel_l2(*P.both("sigma"))
    print("%s C: %.2e  C - I: %.2e  sigma_P - I: %.2e" % (label, rel_l2(*P.both("C")), eC, eS))
    assert eC < DEV_TOL, ("C - I", eC)
    assert eS < DEV_TOL, ("sigma_P - I", eS)
    return eC, eS


def check_diagnostics(P, dg=None, do=None, rtol=1e-5):
    """All 16 diagnostics of the library (vefd_diagnostics) against the
    oracle's on the same state (Sec. 4.1 measures and conservation sums):
      0-1 masses to 1e-6 relative; 2-4 momentum to rtol of M max|u|;
      5, 6, 15 (<sigma_xy>, <N_1>, <tr sigma_P> - 3) to rtol of the mean
      magnitude of the summed quantity; 7, 8 (max tr C / L^2, max |u|) to
      rtol and 10 rtol; the indicator phi > 0 (area 9, D 10, theta 11,
      centroid 12-13, volume 14) exactly when no node has |phi| below 1e-4,
      else within what the ambiguous nodes can change."""
    dg = P.g.diagnostics() if dg is None else dg
    do = P.o.diagnostics() if do is None else do
    assert abs(dg[0] / do[0] - 1) < 1e-6
    if P.p["ncomp"] == 2:
        assert abs(dg[1] / do[1] - 1) < 1e-6
    mass = do[0] + do[1]
    for k in (2, 3, 4):
        assert abs(dg[k] - do[k]) <= rtol * mass * do[8] + 1e-12, (k, dg[k], do[k])
    sig = P.o.read(oracle.F_SIGMA_P)
    nc = sig.shape[0]
    yy = 3 if nc == 6 else 2
    tr = sig[0] + sig[yy] + sig[nc - 1]
    scale = {5: np.mean(np.abs(sig[1])), 6: np.mean(np.abs(sig[0] - sig[yy])), 15: np.mean(np.abs(tr - 3.0))}
    for k, sc in scale.items():
        assert abs(dg[k] - do[k]) <= rtol * max(sc, abs(do[k])) + 1e-12, (k, dg[k], do[k], sc)
    assert abs(dg[7] / do[7] - 1) < rtol, (7, dg[7], do[7])
    if do[8] > 0:
        assert abs(dg[8] / do[8] - 1) < 10 * rtol, (8, dg[8], do[8])
    else:
        assert dg[8] == 0.0
    phi = P.o.read(oracle.F_PHI) if P.p["ncomp"] == 2 else np.ones((P.o.nz, P.o.ny, P.o.nx))
    amb = np.abs(phi) < 1e-4
    n_plane = int(np.count_nonzero(amb[P.o.nz // 2]))
    n_all = int(np.count_nonzero(amb))
    assert abs(dg[9] - do[9]) <= n_plane and abs(dg[14] - do[14]) <= n_all, (dg[9], do[9], dg[14], do[14])
    if n_plane == 0:
        assert np.allclose(dg[10:14], do[10:14], rtol=1e-9, atol=1e-9), (dg[10:14], do[10:14])
    else:
        area = max(do[9], 1.0)
        assert abs(dg[10] - do[10]) <= 4.0 * n_plane / area
        assert abs(dg[12] - do[12]) <= P.o.nx * n_plane / area and abs(dg[13] - do[13]) <= P.o.ny * n_plane / area


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_stagewise_derived_fields(name):
    """Moments, Shan-Chen force, polymer force, velocity and relaxation time
    of one seeded state agree with the oracle before any step."""
    P = Pair(**VARIANTS[name])
    P.init_random(seed=3)
    for fld, tol in (("rhoA", 1e-6), ("phi", 1e-6), ("u", 1e-5), ("tau", 1e-6), ("gA", 1e-5), ("gB", 1e-5),
                     ("Fp", 1e-5), ("sigma", 1e-6), ("C", 1e-6)):
        if fld in ("gA", "gB", "phi") and P.p["ncomp"] == 1:
            continue
        g, o = P.both(fld)
        assert rel_l2(g, o) < tol, (fld, rel_l2(g, o))


@pytest.mark.parametrize("name", sorted(VARIANTS))
@pytest.mark.parametrize("nsteps", [1, 3])
def test_steps_match_oracle(name, nsteps):
    """Populations, u, C and the AB2 history after 1 and 3 full steps
    (the first is forward Euler, the rest AB2)."""
    P = Pair(**VARIANTS[name])
    P.init_random(seed=5)
    P.step(nsteps)
    for fld, tol in (("pops", 1e-6), ("u", 1e-5), ("C", 1e-6), ("R", 1e-5)):
        g, o = P.both(fld)
        assert rel_l2(g, o) < tol, (fld, rel_l2(g, o))
    assert P.g.status() == 0 and P.o.status == 0


@pytest.mark.parametrize("name", ["d3q19_2c_tma_ragged", "d2q9_2c_tma_periodic", "d2q9_1c_tma_walls",
                                  "d3q19_2c_zm_walls", "d3q19_1c_zm_periodic", "d3q19_2c_zm_segments",
                                  "d3q19_2c_mrt_zm", "d2q9_2c_mrt_tma", "d3q19_2c_chol_zm", "d3q19_2c_paper"])
def test_tma_and_register_kernels_agree(name, monkeypatch):
    """The TMA-staged kernels (lattice; densities/FD pass, z-marching where the
    shape allows) and the register-only kernels run the same arithmetic in the
    same order: populations and C agree bit for bit (to FP32 rounding for the
    moment-space collision)."""
    from paper_1406_2686_gb300 import vefd
    from pairs import Pair
    P = Pair(**VARIANTS[name])
    P.g.set_kernel_config(0, 2)  # tiled lattice kernel + z-marching pass where the shape allows
    P.init_random(seed=8)
    monkeypatch.setenv("VEFD_NO_TMA", "1")
    Q = Pair(**VARIANTS[name])
    monkeypatch.delenv("VEFD_NO_TMA")
    Q.init_random(seed=8)
    P.g.step(4)
    Q.g.step(4)
    if VARIANTS[name].get("collision", 0) == 0:
        assert np.array_equal(P.g.read(vefd.POPS), Q.g.read(vefd.POPS))
        assert np.array_equal(P.g.read(vefd.C), Q.g.read(vefd.C))
    else:
        # the moment-space kernels are separate instantiations whose multiply-adds
        # the compiler may contract differently: agreement to FP32 rounding
        for f in (vefd.POPS, vefd.C):
            a, r = P.g.read(f), Q.g.read(f)
            assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r)


@pytest.mark.parametrize("seg", ["", "3", "5"])
@pytest.mark.parametrize("name", ["d3q19_2c_zm_walls", "d3q19_1c_zm_periodic", "d3q19_2c_zm_segments",
                                  "d3q19_2c_mrt_zm", "d3q19_2c_chol_zm", "d3q19_2c_paper", "d3q19_2c_fused_wide"])
def test_fused_densities_agree(name, seg, monkeypatch):
    """The column-marching lattice kernel with fused densities stores the same
    populations as the tiled kernel up to the order in which each node's new
    density is summed: after 4 steps populations and C agree to FP32 rounding,
    and the densities of the first step agree to a few ulps.  Run with the
    default z-segments (one plane each at these sizes) and with segments of 3
    and 5 planes, so populations both cross and stay inside segments."""
    from paper_1406_2686_gb300 import vefd
    if seg:
        monkeypatch.setenv("VEFD_ZM_SEGMENT", seg)
    P = Pair(**VARIANTS[name])
    P.g.set_kernel_config(0, 0)
    P.init_random(seed=8)
    Q = Pair(**VARIANTS[name])
    Q.g.set_kernel_config(0, 2)
    Q.init_random(seed=8)
    assert P.g.kernel_config()[1] == 0 and Q.g.kernel_config()[1] == 2
    P.g.step(1)
    Q.g.step(1)
    for f in (vefd.RHO_A, vefd.POPS):
        a, r = P.g.read(f), Q.g.read(f)
        assert np.max(np.abs(a - r)) <= 4e-7 * max(1.0, np.max(np.abs(r))), f
    P.g.step(3)
    Q.g.step(3)
    for f in (vefd.POPS, vefd.C, vefd.U):
        a, r = P.g.read(f), Q.g.read(f)
        assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r), f
    assert P.g.status() == 0


# lattices of whole 32 x 4 x 2 (and, where NZ allows, 32 x 2 x 4) tiles for
# the partial-density kernel choice (post mode 3)
PARTS_CASES = {
    "walls": dict(VARIANTS["d3q19_2c_zm_walls"], nz=8),
    "periodic_wide": dict(VARIANTS["d3q19_2c_fused_wide"]),
    "one_component": dict(VARIANTS["d3q19_1c_zm_periodic"], nz=8),
    "one_tile_in_x": dict(VARIANTS["d3q19_2c_eqcoupling"], nz=8),
    "mrt": dict(VARIANTS["d3q19_2c_mrt_zm"], nz=8),
    "chol": dict(VARIANTS["d3q19_2c_chol_zm"], nz=8),
    "paper": dict(VARIANTS["d3q19_2c_paper"], nz=8),
}


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("name", sorted(PARTS_CASES))
def test_partial_densities_agree(name, tile):
    """Post mode 3: the tiled lattice kernel sums the new populations that stay
    in its tile and writes what it pushes across each face and edge as partial
    sums; the z-marching pass completes the densities from those instead of
    reading the populations back.  Against post mode 2 (the same tile, the
    pass summing the staged populations) only the order of each density's sum
    differs: after one step the densities agree to a few ulps and the
    populations to FP32 rounding, after four steps populations, C and u agree
    to FP32 rounding."""
    from paper_1406_2686_gb300 import vefd
    P = Pair(**PARTS_CASES[name])
    P.g.set_kernel_config(tile, 3)
    P.init_random(seed=9)
    Q = Pair(**PARTS_CASES[name])
    Q.g.set_kernel_config(tile, 2)
    Q.init_random(seed=9)
    assert P.g.kernel_config() == (tile, 3), P.g.kernel_config()
    assert Q.g.kernel_config() == (tile, 2)
    P.g.step(1)
    Q.g.step(1)
    for f in (vefd.RHO_A, vefd.POPS):
        a, r = P.g.read(f), Q.g.read(f)
        assert np.max(np.abs(a - r)) <= 4e-7 * max(1.0, np.max(np.abs(r))), f
    P.g.step(3)
    Q.g.step(3)
    for f in (vefd.POPS, vefd.C, vefd.U, vefd.RHO_A):
        a, r = P.g.read(f), Q.g.read(f)
        assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r), f
    assert P.g.status() == 0 and Q.g.status() == 0


@pytest.mark.parametrize("tile", [0, 1])
def test_droplet_2000_steps_partial_densities(tile):
    """Post mode 3 on the droplet (64 x 24 x 40, R = 6): the 1e-5 contract in
    u and C after 2000 steps, mass drift within 1e-6 and the oracle's
    diagnostics."""
    P = _droplet_pair(64, 24, 40, 6.0)
    P.g.set_kernel_config(tile, 3)
    assert P.g.kernel_config() == (tile, 3)
    m0 = P.g.diagnostics()[:2]
    P.step(2000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    check_deformation(P, "droplet 2000 partial densities")
    m1 = P.g.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6)
    check_diagnostics(P)
    assert P.g.status() == 0


def test_config1_couette_2000_steps():
    """D2Q9 single-component FENE-P Couette, 64 x 32, walls +-0.01, tau = 1,
    lambda = 1000 steps, eta_P/(eta_s + eta_P) = 0.4, L^2 = 100, C = I:
    after 2000 steps, relative L2 of u and C within 1e-5 of the oracle and
    total mass drift within 1e-6."""
    eta_s = 1.0 / 6.0
    P = Pair(lattice=0, nx=64, ny=32, ncomp=1, walls=1, eta_A=eta_s, eta_B=eta_s, u_wall=0.01, tau_p=1000.0,
             eta_p=eta_s * 0.4 / 0.6, L2=100.0, kappa=0.0)
    P.init(np.ones((1, 32, 64)))
    m0 = P.g.diagnostics()[0]
    P.step(2000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    eC, eS = check_deformation(P, "couette 2000")
    assert eC < 1e-5 and eS < 1e-5
    assert abs(P.g.diagnostics()[0] / m0 - 1) < 1e-6
    check_diagnostics(P)


def test_config1_couette_20000_steps():
    """The same Couette set-up over the full 20000 steps (20 relaxation times
    of the polymer, close to the steady state): u and C within 1e-5 relative
    L2 of the oracle, C - I and sigma_P - I too, the mass within 1e-6, all 16
    diagnostics as the oracle's, and the velocity profile the linear Couette
    profile between the walls (halfway bounce-back, walls at y = -1/2 and
    NY - 1/2).  Near steady state the AB2 increment of C falls below half an
    ulp of C - I; the library carries that rounding error into the next
    increment (compensated update), so C keeps converging."""
    eta_s = 1.0 / 6.0
    P = Pair(lattice=0, nx=64, ny=32, ncomp=1, walls=1, eta_A=eta_s, eta_B=eta_s, u_wall=0.01, tau_p=1000.0,
             eta_p=eta_s * 0.4 / 0.6, L2=100.0, kappa=0.0)
    P.init(np.ones((1, 32, 64)))
    m0 = P.g.diagnostics()[0]
    P.step(20000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        print("couette 20000 %s: %.2e" % (fld, rel_l2(g, o)))
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    eC, eS = check_deformation(P, "couette 20000")
    assert eC < 1e-5 and eS < 1e-5
    assert abs(P.g.diagnostics()[0] / m0 - 1) < 1e-6
    check_diagnostics(P)
    ux = P.both("u")[0][0].mean(axis=-1).ravel()  # x-averaged u_x(y)
    y = np.arange(32) + 0.5
    lin = 0.01 - 2 * 0.01 * y / 32.0            # +u_wall at y = -1/2, -u_wall at y = NY - 1/2
    assert np.max(np.abs(ux - lin)) < 1e-6


def _droplet_pair(nx, ny, nz, R, seed=1, **kw):
    """Confined droplet set-up (D3Q19, 2 components, G = 1.5, rho 2.0 / 0.1,
    width 5, phi noise 1e-3, viscoelastic droplet, L^2 = 100) scaled to the
    box: tau_B = 1 at rho = 2.1, eta_A = 0.6 eta_B, eta_P = 0.4 eta_B,
    Ca = 0.1 and De = 1 with sigma = 0.09."""
    etaB = 2.1 / 3.0 * 0.5
    etaA, etaP, sigma = 0.6 * etaB, 0.4 * etaB, 0.09
    gdot = 0.1 * sigma / (R * etaB)
    taup = 1.0 * R * etaB / sigma * etaB / etaP
    p = dict(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=etaA, eta_B=etaB, u_wall=gdot * ny / 2,
             tau_p=taup, eta_p=etaP, L2=100.0, kappa=1e-3, phase=1)
    p.update(kw)
    P = Pair(**p)
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=R, seed=seed, noise=1e-3)
    P.init(rA, rB)
    return P


def test_droplet_2000_steps():
    """Scaled confined viscoelastic droplet (40 x 24 x 40, R = 6, 2R/H = 0.5):
    after 2000 steps the relative L2 error of u and C is within 1e-5 and the
    per-component mass drift within 1e-6."""
    P = _droplet_pair(40, 24, 40, 6.0)
    m0 = P.g.diagnostics()[:2]
    P.step(2000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    check_deformation(P, "droplet 2000")
    m1 = P.g.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6)
    check_diagnostics(P)
    assert P.g.status() == 0


def test_droplet_2000_steps_column_march():
    """The column-marching lattice kernel with partial densities and the
    densities pass that completes them (kernel choice post mode 0) on the
    droplet (64 x 24 x 40, R = 6): the same 1e-5 contract after 2000 steps,
    mass drift within 1e-6 and the diagnostics of the oracle."""
    P = _droplet_pair(64, 24, 40, 6.0)
    P.g.set_kernel_config(0, 0)
    assert P.g.kernel_config() == (0, 0)
    m0 = P.g.diagnostics()[:2]
    P.step(2000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    check_deformation(P, "droplet 2000 column march")
    m1 = P.g.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6)
    check_diagnostics(P)
    assert P.g.status() == 0


@pytest.mark.parametrize("variant", [dict(collision=1), dict(chol=1), dict(collision=1, coupling=1, chol=1)],
                         ids=["mrt", "chol", "paper"])
def test_droplet_2000_steps_variants(variant):
    """The scaled droplet with the paper-faithful variants of Sec. 2 (moment
    space collision, Cholesky scheme, stress in the equilibrium): same 1e-5
    relative L2 contract after 2000 steps and mass drift within 1e-6."""
    P = _droplet_pair(40, 24, 40, 6.0, **variant)
    m0 = P.g.diagnostics()[:2]
    P.step(2000)
    for fld in ("u", "C"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < 1e-5, (fld, rel_l2(g, o))
    check_deformation(P, "droplet 2000 %r" % (variant,))
    m1 = P.g.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6)
    # The Cholesky scheme (Sec. 2) advances the factor of sigma_P and rebuilds
    # C from it every step; the state is the stored C, rounded to FP32 each
    # step with no carry of the rounding error (the direct scheme carries it in
    # the AB2 history), so C - I is about ten times less accurate (1.4e-5 at
    # 2000 steps) and the stress averages are held to 3e-5.
    check_diagnostics(P, rtol=3e-5 if variant.get("chol") else 1e-5)
    assert P.g.status() == 0


def test_full_size_droplet_sampled_step():
    """Full 128 x 64 x 128 confined droplet in the benchmark's launch
    configuration (the pipelined 8-slab step graph, 256-step chunks): after
    600 GPU steps (two graph replays among them) the state is loaded into the
    oracle and both take one more step; every node agrees (one FP32 step),
    mass is conserved over the run, and the diagnostics agree."""
    P = _droplet_pair(128, 64, 128, 16.0)
    assert P.g.step_graph == (8, 256, True)
    m0 = P.g.diagnostics()[:2]
    P.g.step(600)
    m1 = P.g.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1) < 1e-6)
    from paper_1406_2686_gb300 import vefd
    P.o.write(oracle.F_POPS, P.g.read(vefd.POPS).astype(np.float64))
    P.o.write(oracle.F_C, P.g.read(vefd.C).astype(np.float64))
    P.o.write(oracle.F_RPREV, P.g.read(vefd.RPREV).astype(np.float64))
    # the oracle's diagnostics of the library's own state: every value agrees
    check_diagnostics(P)
    P.step(1)
    for fld, tol in (("pops", 1e-6), ("u", 1e-5), ("C", 1e-6)):
        g, o = P.both(fld)
        assert rel_l2(g, o) < tol, (fld, rel_l2(g, o))
    assert dev_rel_l2(*P.both("C")) < 1e-5 and dev_rel_l2(*P.both("sigma")) < 1e-5
    check_diagnostics(P)


def test_config1_closed_form_20000_steps():
    """The GPU path alone reaches the steady-shear closed form of Sec. 3.1
    (Eqs. lindner and lindner2, Lambda = -0.625, L^2 = 100) after 20000 steps
    = 20 tau_P: every component of C within 1e-5 relative of the closed form
    at every node (C - I within 1e-5 relative L2), <sigma_P,xy> = -S and
    <N_1> = N within 1e-5 relative, and the profile the exact Couette line."""
    from paper_1406_2686_gb300 import vefd
    eta_s = 1.0 / 6.0
    g = vefd.Lattice(lattice=0, nx=64, ny=32, nz=1, ncomp=1, walls=1, eta_A=eta_s, eta_B=eta_s)
    g.set_wall_shear(0.01)
    g.set_fenep(1000.0, eta_s * 0.4 / 0.6, 100.0, 0.0, 0, 1)
    g.init_fields(np.ones((1, 32, 64), np.float32))
    g.step(20000)
    C = g.read(vefd.C).astype(np.float64)
    Cex, Z = cf.shear_conformation(-0.625, 100.0)
    ex = np.array([Cex[kk] for kk in (0, 1, 3, 5)])
    for k in range(4):
        err = np.max(np.abs(C[k] - ex[k]))
        print("closed form C[%d]: max rel %.2e" % (k, err / abs(ex[k])))
        assert err <= 1e-5 * abs(ex[k]), (k, err)
    full = np.broadcast_to(ex[:, None, None, None], C.shape)
    assert dev_rel_l2(C, full) < 1e-5
    u = g.read(vefd.U)[0].astype(np.float64)
    assert np.max(np.abs(u - cf.couette_profile(32, 0.01)[None, :, None])) < 2e-7
    d = g.diagnostics()
    S, N = cf.shear_S(0.625, 100.0), cf.shear_N(0.625, 100.0)
    assert abs(d[5] + S) < 1e-5 * S and abs(d[6] - N) < 1e-5 * N and abs(d[15] - N) < 1e-5 * N
    assert abs(d[7] - (ex[0] + ex[2] + ex[3]) / 100.0) < 1e-5 * d[7]


def test_guards_flag_instability():
    """The device guard word reports a NaN and tr C >= L^2 written into C, and
    |u| above the Mach limit (the failure is made on the host side, through
    the field interface; no kernel faults)."""
    from paper_1406_2686_gb300 import vefd
    P = Pair(lattice=1, nx=8, ny=6, nz=4, ncomp=1, walls=1, eta_p=0.1, tau_p=10.0, L2=20.0)
    P.init(np.ones((4, 6, 8)))
    P.g.step(2)
    assert P.g.status() == 0
    C = P.g.read(vefd.C)
    C[0, 1, 2, 3] = np.nan
    P.g.write(vefd.C, C)
    P.g.step(1)
    assert P.g.status() & vefd.ST_NAN
    P.g.init_fields(np.ones((4, 6, 8), np.float32))
    C = P.g.read(vefd.C)
    C[0, 2, 2, 2] = 19.0  # tr C = 21 > L^2 = 20
    P.g.write(vefd.C, C)
    P.g.step(1)
    assert P.g.status() & vefd.ST_TRACE
    with pytest.raises(vefd.VefdError) as ei:
        vefd._check(P.g.ctx, vefd.load().vefd_diagnostics(P.g.ctx, None))
    assert ei.value.status == vefd.ERR_ARG
    u = np.zeros((3, 4, 6, 8), np.float32)
    u[0, 1, 1, 1] = 0.35
    P.g.init_fields(np.ones((4, 6, 8), np.float32), None, u)
    P.g.step(1)
    assert P.g.status() & vefd.ST_MACH
    P.g.clear_status()
    assert P.g.status() == 0


def test_bounded_wait_reports_timeout():
    """A device wait that nothing completes runs out of its clock64 budget,
    sets the timeout bit and returns (no hang, no fault); the host reads
    VEFD_ERR_TIMEOUT, clears the word, and the context keeps stepping with
    the same results as an untouched one."""
    from paper_1406_2686_gb300 import vefd
    P = Pair(lattice=1, nx=32, ny=8, nz=4, ncomp=1, walls=1, eta_p=0.1, tau_p=10.0, L2=20.0)
    P.init(np.ones((4, 8, 32)))
    Q = Pair(lattice=1, nx=32, ny=8, nz=4, ncomp=1, walls=1, eta_p=0.1, tau_p=10.0, L2=20.0)
    Q.init(np.ones((4, 8, 32)))
    P.g.wait_selftest(True)
    assert P.g.status() == 0
    P.g.wait_selftest(False)
    bits = ctypes.c_uint32()
    assert vefd.load().vefd_get_status(P.g.ctx, ctypes.byref(bits)) == vefd.ERR_TIMEOUT
    assert bits.value == vefd.ST_TIMEOUT
    P.g.clear_status()
    P.g.step(3)
    Q.g.step(3)
    assert P.g.status() == 0
    assert np.array_equal(P.g.read(vefd.POPS), Q.g.read(vefd.POPS))
    with pytest.raises(vefd.VefdError) as ei:
        vefd.vefd_wait_selftest(P.g.ctx, 2)
    assert ei.value.status == vefd.ERR_ARG


@pytest.mark.parametrize("variant", [dict(), dict(collision=1, coupling=1, chol=1)], ids=["default", "paper"])
def test_checkpoint_restore_bit_identical(tmp_path, variant):
    """A restored context continues bit-identically (the collision, coupling
    and conformation scheme are part of the checkpoint)."""
    from paper_1406_2686_gb300 import vefd
    P = _droplet_pair(24, 16, 20, 4.0, **variant)
    P.g.step(7)
    path = str(tmp_path / "ck.bin")
    P.g.checkpoint(path)
    P.g.step(9)
    a_pops, a_C, a_R = P.g.read(vefd.POPS), P.g.read(vefd.C), P.g.read(vefd.RPREV)
    g2 = vefd.Lattice(lattice=1, nx=24, ny=16, nz=20, ncomp=2, walls=1, G=0.0, eta_A=1.0, eta_B=1.0)
    g2.restore(path)
    assert g2.steps_done == 7
    g2.step(9)
    assert np.array_equal(g2.read(vefd.POPS), a_pops)
    assert np.array_equal(g2.read(vefd.C), a_C)
    assert np.array_equal(g2.read(vefd.RPREV), a_R)


def test_init_droplet_matches_generator():
    """The library's droplet initialiser reproduces the seeded generator
    (same profile and the same SplitMix64 counter stream)."""
    from paper_1406_2686_gb300 import vefd
    nx, ny, nz = 30, 20, 26
    g = vefd.Lattice(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=0.2, eta_B=0.3)
    g.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, 6.0, 2.0, 0.1, 5.0, 11, 1e-3)
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=6.0, seed=11, noise=1e-3)
    assert np.max(np.abs(g.read(vefd.RHO_A) - rA)) < 2e-6
    assert np.max(np.abs(g.read(vefd.RHO_B) - rB)) < 2e-6


def test_device_pointer_io_roundtrip():
    """Fields read to and written from device memory (torch tensors) match the
    host path."""
    import torch
    from paper_1406_2686_gb300 import vefd
    P = Pair(lattice=1, nx=10, ny=6, nz=4, ncomp=2, walls=1)
    P.init_random(seed=9)
    P.g.step(2)
    for f in (vefd.POPS, vefd.C, vefd.U, vefd.PHI):
        assert np.array_equal(P.g.read(f, device=True).cpu().numpy(), P.g.read(f))
    C = P.g.read(vefd.C, device=True) * 1.0
    C[0] += 0.01
    P.g.write(vefd.C, C)
    assert np.allclose(P.g.read(vefd.C), C.cpu().numpy())
    torch.cuda.synchronize()


def test_empty_step_and_errors():
    from paper_1406_2686_gb300 import vefd
    P = Pair(lattice=0, nx=8, ny=5, ncomp=1)
    P.init_random(seed=2)
    before = P.g.read(vefd.POPS)
    P.g.step(0)
    assert np.array_equal(before, P.g.read(vefd.POPS))
    with pytest.raises(vefd.VefdError):
        P.g.step(-1)
    with pytest.raises(ValueError):
        P.g.write(vefd.C, np.zeros(3, np.float32))
    # densities that are not finite or are negative are refused on the
    # device-side check, and the context must be initialised again
    for bad in (np.nan, -0.5, np.inf):
        rho = np.ones((1, 5, 8), np.float32)
        rho[0, 2, 3] = bad
        with pytest.raises(vefd.VefdError) as ei:
            P.g.init_fields(rho)
        assert ei.value.status == vefd.ERR_ARG
        with pytest.raises(vefd.VefdError) as ei:
            P.g.step(1)
        assert ei.value.status == vefd.ERR_STATE
    P.g.init_fields(np.ones((1, 5, 8), np.float32))
    P.g.step(2)
    assert P.g.status() == 0


# --- 16-bit population storage (FP16 / BF16 deviations, FP32 arithmetic) -----

PREC_TOL = {  # relative L2 after 3 steps from a random state
    1: dict(pops=2e-4, u=3e-3, C=2e-5, R=3e-3),
    2: dict(pops=2e-3, u=3e-2, C=2e-4, R=3e-2),
}


REF256_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
REF256 = os.path.join(REF256_DIR, "droplet256_fp64_5000.npz")
REF256_2000 = os.path.join(REF256_DIR, "droplet256_fp64_2000.npz")

# Unit roundoff of the population storage types (FP32, FP16, BF16).
UNIT_ROUNDOFF = {0: 2.0 ** -24, 1: 2.0 ** -11, 2: 2.0 ** -8}


def _droplet256_vs_oracle(path, prec, steps):
    """The 256 x 128 x 256 droplet (R = 32, 2R/H = 0.5, the benchmark droplet
    scaled) with the given population storage, `steps` steps from the seeded
    state that oracle/make_droplet256_reference.py stored the FP64 oracle's
    run of: relative L2 over the planes z = NZ/2 and y = NY/2 of rho_A,
    rho_B, u, C and C - I, the error of the deformation D of the shear plane,
    and the component mass drift.  Returns (errors, D, the oracle's D)."""
    import json

    from paper_1406_2686_gb300 import vefd
    ref = np.load(path)
    meta = json.loads(str(ref["meta"]))
    nx, ny, nz, R = 256, 128, 256, 32.0
    etaB = 2.1 / 3.0 * 0.5
    p = dict(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=0.6 * etaB, eta_B=etaB,
             u_wall=0.1 * 0.09 / (R * etaB) * ny / 2, tau_p=R * etaB / 0.09 * etaB / (0.4 * etaB), eta_p=0.4 * etaB,
             L2=100.0, kappa=1e-3, phase=1)
    for k, v in p.items():
        assert abs(meta["params"][k] - v) <= 1e-12 * max(1.0, abs(v)), (k, meta["params"][k], v)
    assert meta["steps"] == steps
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=R, seed=meta["seed"], noise=1e-3)
    rA, rB = inputs.to_f32_exact(rA), inputs.to_f32_exact(rB)
    zref, yref = ref["zplane"], ref["yplane"]
    rows = {"rhoA": slice(0, 1), "rhoB": slice(1, 2), "u": slice(2, 5), "C": slice(5, 11)}
    eye = np.array([1, 0, 0, 1, 0, 1.0])[:, None, None]
    g = vefd.Lattice(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=p["G"], eta_A=p["eta_A"],
                     eta_B=p["eta_B"], delta=0.1, precision=prec)
    g.set_wall_shear(p["u_wall"])
    g.set_fenep(p["tau_p"], p["eta_p"], p["L2"], p["kappa"], p["phase"], 1)
    g.init_fields(rA, rB)
    m0 = g.diagnostics()[:2]
    g.step(steps)
    full = np.concatenate([g.read(vefd.RHO_A)[None], g.read(vefd.RHO_B)[None], g.read(vefd.U),
                           g.read(vefd.C)]).astype(np.float64)
    d = g.diagnostics()
    assert g.status() == 0
    g.close()
    zg, yg = full[:, nz // 2], full[:, :, ny // 2]
    err = {}
    for name, sl in rows.items():
        a = np.concatenate([zg[sl].ravel(), yg[sl].ravel()])
        b = np.concatenate([zref[sl].ravel(), yref[sl].ravel()])
        err[name] = rel_l2(a, b)
    cg = np.concatenate([(zg[5:11] - eye).ravel(), (yg[5:11] - eye).ravel()])
    co = np.concatenate([(zref[5:11] - eye).ravel(), (yref[5:11] - eye).ravel()])
    err["CmI"] = rel_l2(cg, co)
    err["D"] = abs(d[10] - ref["diag"][10]) / ref["diag"][10]
    err["mass"] = float(np.max(np.abs(d[:2] / m0 - 1)))
    return err, d[10], ref["diag"][10]


def _print_table(title, table):
    print("\n" + title)
    print("storage  " + "  ".join("%8s" % k for k in ("rhoA", "rhoB", "u", "C", "C-I", "D", "mass")) + "   D")
    for name, e, dval in table:
        print("%-8s " % name + "  ".join("%8.2e" % e[k] for k in ("rhoA", "rhoB", "u", "C", "CmI", "D", "mass"))
              + "   %.5f" % dval)


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(REF256_2000), reason="FP64 reference sample not generated")
def test_full_geometry_fp32_2000_steps_vs_oracle(capsys):
    """The parity contract on the storage-precision geometry: FP32 after 2000
    steps of the 256 x 128 x 256 droplet within 1e-5 relative L2 of the FP64
    oracle in u and C (C - I, the polymer deformation itself, within 1e-4)
    and mass drift within 1e-6.  FP16 and BF16 storage are reported beside it
    and held to mass conservation only: their error bounds belong to the
    5000-step study, and at 2000 steps the droplet is still deforming (D is
    0.053 against 0.134), so the relative error of D is inflated there (FP16:
    5.4 % of 0.053, the same absolute error as 3.3 % of 0.134)."""
    table = []
    for prec in (0, 1, 2):
        e, dval, dref = _droplet256_vs_oracle(REF256_2000, prec, 2000)
        table.append((("fp32", "fp16", "bf16")[prec], e, dval))
    with capsys.disabled():
        _print_table("vs FP64 oracle after 2000 steps, 256x128x256 (oracle D = %.5f)" % dref, table)
    e = table[0][1]
    assert e["u"] < 1e-5 and e["C"] < 1e-5, e
    assert e["CmI"] < 1e-4 and e["rhoA"] < 1e-4 and e["rhoB"] < 1e-4, e
    assert e["D"] < 1e-4 and e["mass"] < 1e-6, e
    for prec in (1, 2):
        name, e, _ = table[prec]
        assert e["mass"] < 1e-6, (name, e["mass"])


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(REF256), reason="FP64 reference sample not generated")
def test_precision_full_geometry_vs_oracle(capsys):
    """The storage-precision study: FP32, FP16 and BF16 population storage,
    each after 5000 steps of the 256 x 128 x 256 droplet, against the FP64
    oracle's run of the same seeded state, per field.

    Bounds.  FP32: the contract holds u and C to 1e-5 after 2000 steps; the
    rounding of every further step adds to the error, at most in proportion
    to the step count without amplification, so after 5000 steps u and C are
    held to 5000/2000 x 1e-5 = 2.5e-5 (the fields rho and C - I, whose norms
    are set by the interface and by the small polymer deformation, to 1e-4).
    FP16 and BF16: no contract fixes their accuracy; the study states it.
    Their bounds guard against regressions: every field, C - I and D within
    100 times the unit roundoff of the storage type (2^-11 and 2^-8).  The
    first measurement put both formats at 10 to 80 times their unit roundoff
    in every field, the same scaling for both, which is what storage
    rounding (and not a defect of one conversion) produces; the factor 100
    was chosen after that measurement.  Every variant conserves mass to
    1e-6."""
    table = []
    for prec in (0, 1, 2):
        e, dval, dref = _droplet256_vs_oracle(REF256, prec, 5000)
        table.append((("fp32", "fp16", "bf16")[prec], e, dval))
    with capsys.disabled():
        _print_table("vs FP64 oracle after 5000 steps, 256x128x256 (oracle D = %.5f)" % dref, table)
    for prec, (name, e, _) in enumerate(table):
        if prec == 0:
            bound = {"u": 2.5e-5, "C": 2.5e-5, "rhoA": 1e-4, "rhoB": 1e-4, "CmI": 1e-4, "D": 1e-4}
        else:
            b = 100.0 * UNIT_ROUNDOFF[prec]
            bound = {k: b for k in ("rhoA", "rhoB", "u", "C", "CmI", "D")}
        for k, v in bound.items():
            assert e[k] < v, (name, k, e[k], v)
        assert e["mass"] < 1e-6, (name, e["mass"])


class PrecPair(Pair):
    def __init__(self, precision, **kw):
        from paper_1406_2686_gb300 import vefd
        super().__init__(**kw)
        p = self.p
        self.g.close()
        self.g = vefd.Lattice(lattice=p["lattice"], nx=p["nx"], ny=p["ny"], nz=p["nz"], ncomp=p["ncomp"],
                              walls=p["walls"], G=p["G"], eta_A=p["eta_A"], eta_B=p["eta_B"], delta=p["delta"],
                              precision=precision)
        self.g.set_wall_shear(p["u_wall"])
        self.g.set_body_force(*p["fext"])
        self.g.set_fenep(p["tau_p"], p["eta_p"], p["L2"], p["kappa"], p["phase"], p["fd_on"])
        self.g.set_polymer_coupling(p["coupling"])


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", ["d3q19_2c_walls", "d3q19_2c_zm_walls", "d3q19_2c_tma_ragged", "d2q9_2c_tma_periodic",
                                  "d2q9_1c_walls"])
def test_16bit_storage_steps(precision, name):
    """16-bit deviation storage follows the oracle within the storage
    rounding, and the FP32 rest population keeps every component's mass to
    FP32 rounding."""
    P = PrecPair(precision, **VARIANTS[name])
    P.init_random(seed=6)
    m0 = P.g.diagnostics()[:2]
    P.step(3)
    tol = PREC_TOL[precision]
    for fld in ("pops", "u", "C", "R"):
        g, o = P.both(fld)
        assert rel_l2(g, o) < tol[fld], (fld, rel_l2(g, o))
    m1 = P.g.diagnostics()[:2]
    k = 2 if P.p["ncomp"] == 2 else 1
    assert np.all(np.abs(m1[:k] / m0[:k] - 1) < 1e-6)


@pytest.mark.parametrize("name", ["d3q19_2c_zm_walls", "d2q9_2c_tma_periodic"])
def test_16bit_tma_and_register_agree(name, monkeypatch):
    """The staged and register-only kernels agree bit for bit in FP16 storage too."""
    from paper_1406_2686_gb300 import vefd
    P = PrecPair(1, **VARIANTS[name])
    P.init_random(seed=8)
    monkeypatch.setenv("VEFD_NO_TMA", "1")
    Q = PrecPair(1, **VARIANTS[name])
    monkeypatch.delenv("VEFD_NO_TMA")
    Q.init_random(seed=8)
    P.g.step(4)
    Q.g.step(4)
    if VARIANTS[name].get("collision", 0) == 0:
        assert np.array_equal(P.g.read(vefd.POPS), Q.g.read(vefd.POPS))
        assert np.array_equal(P.g.read(vefd.C), Q.g.read(vefd.C))
    else:
        # the moment-space kernels are separate instantiations whose multiply-adds
        # the compiler may contract differently: agreement to FP32 rounding
        for f in (vefd.POPS, vefd.C):
            a, r = P.g.read(f), Q.g.read(f)
            assert np.linalg.norm(a - r) <= 1e-6 * np.linalg.norm(r)


def test_precision_error_report(capsys):
    """Per-field error of FP32, FP16 and BF16 population storage against the
    FP64 oracle after 5000 steps of the confined viscoelastic droplet
    (64 x 32 x 64, R = 8, 2R/H = 0.5, the benchmark's parameters scaled).
    FP32 meets the 1e-5 bar; the 16-bit variants are reported with bounds
    from their storage precision, and every variant conserves mass."""
    from paper_1406_2686_gb300 import vefd
    P = _droplet_pair(64, 32, 64, 8.0)
    P.o.step(5000)
    ref = {k: P.o.read(oracle_f) for k, oracle_f in (("rhoA", oracle.F_RHO_A), ("rhoB", oracle.F_RHO_B),
                                                     ("phi", oracle.F_PHI), ("u", oracle.F_U), ("C", oracle.F_C))}
    bounds = {0: dict(rhoA=1e-4, rhoB=1e-5, phi=1e-5, u=1e-5, C=1e-5),
              1: dict(rhoA=2e-2, rhoB=5e-3, phi=5e-3, u=5e-3, C=2e-3),
              2: dict(rhoA=3e-1, rhoB=5e-2, phi=1e-1, u=5e-2, C=5e-2)}
    rows = []
    rA, rB = inputs.droplet_fields(64, 32, 64, R=8.0, seed=1, noise=1e-3)
    for prec in (0, 1, 2):
        G = PrecPair(prec, **P.p)
        G.g.init_fields(inputs.to_f32_exact(rA), inputs.to_f32_exact(rB))
        m0 = G.g.diagnostics()[:2]
        G.g.step(5000)
        errs = {}
        for k, f in (("rhoA", vefd.RHO_A), ("rhoB", vefd.RHO_B), ("phi", vefd.PHI), ("u", vefd.U), ("C", vefd.C)):
            errs[k] = rel_l2(G.g.read(f).astype(np.float64), ref[k])
            assert errs[k] < bounds[prec][k], (prec, k, errs[k])
        m1 = G.g.diagnostics()[:2]
        errs["mass"] = float(np.max(np.abs(m1 / m0 - 1)))
        assert errs["mass"] < 1e-6
        rows.append((("fp32", "fp16", "bf16")[prec], errs))
        G.g.close()
    with capsys.disabled():
        print("\nstorage  " + "  ".join("%8s" % k for k in ("rhoA", "rhoB", "phi", "u", "C", "mass")))
        for name, e in rows:
            print("%-8s " % name + "  ".join("%8.2e" % e[k] for k in ("rhoA", "rhoB", "phi", "u", "C", "mass")))


def _sheared_newtonian_droplet(nx, ny, nz, R, eta):
    """A Newtonian droplet of viscosity ratio 1 (both phases eta) in the
    confined shear flow of Sec. 4.1.  The droplet first relaxes at rest
    (3000 (R/16)^2 steps); its surface tension follows from the Laplace law,
    sigma = R (P_in - P_out) / 2 with the bulk pressure of Eq. PTexpanded and R
    from the droplet volume.  The sheared run starts from that relaxed state
    with the Couette profile imposed (the channel's own spin-up, H^2 / nu
    steps, would let the droplet dissolve noticeably into the matrix
    meanwhile), at the wall speed that sets Ca = 0.1 for the measured sigma,
    for 100 emulsion times.  Returns the D samples (every 5 emulsion times),
    the mean and spread of the last 8, the droplet radius and capillary number
    then, and the droplet Reynolds number rho gdot R^2 / eta."""
    from paper_1406_2686_gb300 import vefd

    def lattice():
        g = vefd.Lattice(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=eta, eta_B=eta)
        g.set_fenep(100.0, 0.0, 100.0, 0.0, 0, 0)
        return g

    rest = lattice()
    rest.init_droplet((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, R, 2.0, 0.1, 5.0, 3, 0.0)
    rest.step(int(3000 * (R / 16.0) ** 2))
    rA, rB = rest.read(vefd.RHO_A), rest.read(vefd.RHO_B)
    d = rest.diagnostics()
    rest.close()
    p = cf.bulk_pressure(rA.astype(np.float64), rB.astype(np.float64), 1.5)
    c = (nz // 2, ny // 2, nx // 2)
    p_in = float(np.mean(p[c[0] - 2:c[0] + 2, c[1] - 2:c[1] + 2, c[2] - 2:c[2] + 2]))
    p_out = float(np.mean(p[:6, ny // 2 - 2:ny // 2 + 2, :6]))
    R_eff = (3.0 * d[14] / (4.0 * math.pi)) ** (1.0 / 3.0)
    sigma = 0.5 * R_eff * (p_in - p_out)
    gdot = 0.1 * sigma / (R_eff * eta)
    tau_em = R_eff * eta / sigma
    g = lattice()
    u_wall = gdot * ny / 2
    u = np.zeros((3, nz, ny, nx), np.float32)
    u[0] = cf.couette_profile(ny, u_wall)[None, :, None]
    g.set_wall_shear(u_wall)
    g.init_fields(rA, rB, u)
    hist, vol = [], []
    for _ in range(20):
        g.step(int(5 * tau_em))
        dg = g.diagnostics()
        hist.append(dg[10])
        vol.append(dg[14])
    assert g.status() == 0
    g.close()
    last = np.array(hist[-8:])
    R_end = (3.0 * float(np.mean(vol[-8:])) / (4.0 * math.pi)) ** (1.0 / 3.0)
    return dict(hist=hist, D=float(last.mean()), D_std=float(last.std()), sigma=sigma, R=R_eff, R_end=R_end,
                Ca_end=gdot * R_end * eta / sigma, tau_em=tau_em, Re=2.1 * gdot * R_eff ** 2 / eta)


def _report_droplet(r, D_sh, capsys):
    with capsys.disabled():
        print("\nLaplace: sigma %.4f (R %.2f, tau_em %.0f steps, Re %.2f); D every 5 tau_em %s; D %.4f +- %.4f; "
              "R_end %.2f, Ca_end %.4f; Shapira-Haber %.4f, Taylor %.4f"
              % (r["sigma"], r["R"], r["tau_em"], r["Re"], " ".join("%.4f" % v for v in r["hist"]), r["D"],
                 r["D_std"], r["R_end"], r["Ca_end"], D_sh, cf.taylor_D(r["Ca_end"], 1.0)))


@pytest.mark.slow
def test_newtonian_droplet_deformation_shapira_haber(capsys):
    """Physics check of the whole GPU path (not parity) at the benchmark's
    viscosity (tau = 1 at rho = 2.1, eta = 0.35) and geometry (R = 16,
    2R/H = 0.5): the steady deformation of the shear plane exceeds Taylor's
    unconfined value and lies within 30 % of the confined prediction of
    Shapira and Haber quoted in Sec. 4.1 (D = 0.1264 at Ca = 0.1, lambda = 1,
    R/H = 0.25), evaluated at the droplet's size then.  Measured: D = 0.150
    against 0.120.  The theory assumes Stokes flow; here the droplet Reynolds
    number rho gdot R^2 / eta is 2.7, and inertia raises D (at R = 24 and 32,
    Re 3.8 and 5.0, D = 0.151 and 0.164).  The bound catches a wrong shear
    direction, a missing or doubled force term or a wrong viscosity; the
    Stokes-regime test below holds D to 10 %."""
    r = _sheared_newtonian_droplet(128, 64, 128, 16.0, 2.1 / 3.0 * 0.5)
    D_sh = cf.shapira_haber_D(r["Ca_end"], 1.0, r["R_end"] / 64)
    _report_droplet(r, D_sh, capsys)
    assert r["D_std"] < 0.03 * r["D"]                   # steady up to the pixel noise
    assert abs(r["D"] / D_sh - 1) < 0.30, (r["D"], D_sh)
    assert r["D"] > cf.taylor_D(r["Ca_end"], 1.0)


@pytest.mark.slow
def test_newtonian_droplet_deformation_stokes_regime(capsys):
    """The same check where the theory applies: Shapira and Haber (and Taylor)
    assume Stokes flow, so the viscosity is doubled (tau = 1.5, eta = 0.7),
    which cuts the droplet Reynolds number by four, and the droplet is resolved
    by 24 nodes (192 x 96 x 192, 2R/H = 0.5): Re = 0.96.  The steady
    deformation lies within 10 % of Shapira-Haber (the agreement the paper's
    Fig. 5 reports for the Newtonian case).  Measured: D = 0.1181 against
    0.1158 (+2 %); at R = 16 (Re 0.67) 0.1126 against 0.1118.  Raising tau
    further lowers Re but also raises the Shan-Chen interdiffusion (mobility
    tau - 1/2): over the longer runs the droplet dissolves (R 15.1 -> 12.7 at
    tau = 3) and D falls below the prediction (-8 % at tau = 2, -21 % at
    tau = 3)."""
    r = _sheared_newtonian_droplet(192, 96, 192, 24.0, 2.1 / 3.0 * 1.0)
    D_sh = cf.shapira_haber_D(r["Ca_end"], 1.0, r["R_end"] / 96)
    _report_droplet(r, D_sh, capsys)
    assert r["Re"] < 1.0
    assert r["D_std"] < 0.03 * r["D"]
    assert abs(r["D"] / D_sh - 1) < 0.10, (r["D"], D_sh)
    assert r["D"] > cf.taylor_D(r["Ca_end"], 1.0)


def test_diagnostics_log_csv(tmp_path):
    """The diagnostics log: rows before the first step and every `every`
    steps, the 16 values of vefd_diagnostics and the mass drift per row, as
    CSV; a guard bit set during the run stops it with ERR_UNSTABLE after
    writing the rows so far."""
    import csv

    from paper_1406_2686_gb300 import monitor, vefd
    P = _droplet_pair(24, 16, 20, 4.0)
    path = str(tmp_path / "diag.csv")
    rows = monitor.run_logged(P.g, 45, 10, path)
    assert [r[0] for r in rows] == [0, 10, 20, 30, 40, 45]
    with open(path) as fh:
        got = list(csv.reader(fh))
    assert got[0] == monitor.COLUMNS and len(got) == 7
    P.o.step(45)
    do = P.o.diagnostics()
    last = np.array([float(v) for v in got[-1][1:17]])
    assert abs(last[0] / do[0] - 1) < 1e-6 and abs(last[10] - do[10]) < 1e-3
    assert max(float(r[-1]) for r in got[1:]) < 1e-6
    C = P.g.read(vefd.C)
    C[0, 3, 4, 5] = np.nan
    P.g.write(vefd.C, C)
    with pytest.raises(vefd.VefdError) as ei:
        monitor.run_logged(P.g, 30, 10, path)
    assert ei.value.status == vefd.ERR_UNSTABLE
    with open(path) as fh:
        assert len(list(csv.reader(fh))) == 3  # header, the starting row and the row that saw the bit
