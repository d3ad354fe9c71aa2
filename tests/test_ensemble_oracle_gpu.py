"""Ensemble members against the FP64 oracle (GPU required).

An ensemble only changes how the launches of independent lattices are issued
(batched launches over the tiles of all members, or one graph branch per
member), so every member must follow the method of Sec. 2 exactly as a
lattice stepped alone does.  Here each member of an uneven ensemble of
confined droplets (both viscoelastic phases, Sec. 4 set-ups) is stepped 500
times through vefd_ensemble_step and compared with its own oracle run: u and
C within the 1e-5 relative L2 contract for FP32 storage (C - I and
sigma_P - I within the deformation bound of the parity tests), the 16-bit
member within its storage bounds, and every member's component masses
within 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_1406_2686_gb300 import inputs

from pairs import dev_rel_l2, rel_l2

pytestmark = pytest.mark.gpu

STEPS = 500
ETA_B = 2.1 / 3.0 * 0.5
# (nx, ny, nz, R, phase, u_wall, tau_p): rows of whole 32 x 8 columns, so
# every member can take the batched launches
MEMBERS = [
    (64, 16, 12, 5.0, +1, 0.020, 60.0),
    (32, 24, 10, 6.0, -1, -0.015, 80.0),
    (96, 8, 6, 3.0, +1, 0.010, 40.0),
    (32, 16, 16, 5.0, -1, 0.025, 50.0),
]
FP16_MEMBERS = [
    (64, 16, 8, 4.0, +1, 0.020, 60.0),
    (32, 8, 12, 3.0, -1, 0.015, 40.0),
]
# FP32: the 2000-step contract; the deformation as in the parity tests.
# FP16: the bounds of the 5000-step storage-precision report (Sec. 2 storage
# of population deviations in 16 bits; C is FP32).
TOL = {0: dict(u=1e-5, C=1e-5, dev=1e-4), 1: dict(u=5e-3, C=2e-3, dev=2e-2)}


def params(m, lattice=1):
    nx, ny, nz, R, phase, uw, taup = m
    return dict(lattice=lattice, nx=nx, ny=ny, nz=nz if lattice == 1 else 1, ncomp=2, walls=1, G=1.5,
                eta_A=0.6 * ETA_B, eta_B=ETA_B, delta=0.1, u_wall=uw, tau_p=taup, eta_p=0.4 * ETA_B, L2=100.0,
                kappa=1e-3, phase=phase)


def fields(m, seed, lattice=1):
    nx, ny, nz, R = m[:4]
    nz = nz if lattice == 1 else 1
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=R, seed=seed, noise=1e-3)
    return inputs.to_f32_exact(rA), inputs.to_f32_exact(rB)


def lattice_of(p, rA, rB, precision=0):
    from paper_1406_2686_gb300 import vefd
    L = vefd.Lattice(lattice=p["lattice"], nx=p["nx"], ny=p["ny"], nz=p["nz"], ncomp=2, walls=1, G=p["G"],
                     eta_A=p["eta_A"], eta_B=p["eta_B"], delta=p["delta"], precision=precision)
    L.set_wall_shear(p["u_wall"])
    L.set_fenep(p["tau_p"], p["eta_p"], p["L2"], p["kappa"], p["phase"], 1)
    L.init_fields(rA, rB)
    return L


def oracle_run(p, rA, rB):
    o = oracle.Oracle(**p)
    o.init_fields(rA, rB)
    o.step(STEPS)
    return o


def compare(L, o, precision, label):
    from paper_1406_2686_gb300 import vefd
    tol = TOL[precision]
    got = {}
    for name, gf, of in (("u", vefd.U, oracle.F_U), ("C", vefd.C, oracle.F_C)):
        got[name] = rel_l2(L.read(gf).astype(np.float64), o.read(of))
    got["C-I"] = dev_rel_l2(L.read(vefd.C).astype(np.float64), o.read(oracle.F_C))
    got["sigma-I"] = dev_rel_l2(L.read(vefd.SIGMA_P).astype(np.float64), o.read(oracle.F_SIGMA_P))
    print("%s: u %.2e  C %.2e  C-I %.2e  sigma-I %.2e" % (label, got["u"], got["C"], got["C-I"], got["sigma-I"]))
    assert got["u"] < tol["u"] and got["C"] < tol["C"], (label, got)
    assert got["C-I"] < tol["dev"] and got["sigma-I"] < tol["dev"], (label, got)
    dg, do = L.diagnostics(), o.diagnostics()
    assert abs(dg[0] / do[0] - 1) < 1e-6 and abs(dg[1] / do[1] - 1) < 1e-6, (label, dg[:2], do[:2])
    assert L.status() == 0


def run_ensemble(members, batched, chunk, precision=0, extra=()):
    """Ensemble of `members` (+ `extra` (lattice, member) pairs stepped as
    graph branches only) stepped STEPS times; each compared with its oracle."""
    from paper_1406_2686_gb300 import vefd
    oracle.set_threads(0)
    setups = [(1, m) for m in members] + list(extra)
    lats, orcs, precs = [], [], []
    for k, (lat, m) in enumerate(setups):
        p = params(m, lat)
        rA, rB = fields(m, seed=100 + k, lattice=lat)
        prec = precision if lat == 1 else 0
        lats.append(lattice_of(p, rA, rB, prec))
        orcs.append(oracle_run(p, rA, rB))
        precs.append(prec)
    E = vefd.Ensemble(lats)
    E.set_batched(batched)
    E.step(STEPS - 13, chunk=chunk)   # Euler start, replays, eager remainder
    E.step(13, chunk=chunk)           # the other ping-pong parity
    assert E.batched == batched
    for k, (L, o) in enumerate(zip(lats, orcs)):
        assert L.steps_done == STEPS
        compare(L, o, precs[k], "%s member %d %r" % ("batched" if batched else "branches", k, setups[k]))
    E.close()
    for L in lats:
        L.close()


def test_batched_ensemble_members_match_oracle():
    """Four uneven FP32 boxes (both viscoelastic phases, opposite wall
    directions) in batched launches."""
    run_ensemble(MEMBERS, batched=True, chunk=32)


def test_batched_fp16_ensemble_members_match_oracle():
    """Two FP16-storage boxes in batched launches (the batched kernels take
    one storage type per ensemble)."""
    run_ensemble(FP16_MEMBERS, batched=True, chunk=16, precision=1)


def test_graph_branch_ensemble_members_match_oracle():
    """Graph branches: the FP32 boxes, an FP16 box and a D2Q9 droplet in one
    ensemble, each member one branch of the replayed graph."""
    extra = [(0, (96, 32, 1, 8.0, +1, 0.02, 50.0))]
    run_ensemble(MEMBERS[:3], batched=False, chunk=16, extra=extra)
    run_ensemble(FP16_MEMBERS[:1], batched=False, chunk=16, precision=1)
