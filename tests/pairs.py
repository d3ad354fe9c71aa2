"""Paired set-up of the CUDA library and the oracle on identical inputs.

Inputs are generated in FP64, rounded to FP32 (the library's storage
precision) and the rounded values are given to both sides, so the two start
from the same state.
"""
import numpy as np

import oracle
from paper_1406_2686_gb300 import inputs

OR_FIELD = {"rhoA": oracle.F_RHO_A, "rhoB": oracle.F_RHO_B, "phi": oracle.F_PHI, "u": oracle.F_U,
            "C": oracle.F_C, "sigma": oracle.F_SIGMA_P, "pops": oracle.F_POPS, "R": oracle.F_RPREV,
            "gA": oracle.F_G_A, "gB": oracle.F_G_B, "Fp": oracle.F_F_P, "tau": oracle.F_TAU}


def gpu_fields():
    from paper_1406_2686_gb300 import vefd
    return {"rhoA": vefd.RHO_A, "rhoB": vefd.RHO_B, "phi": vefd.PHI, "u": vefd.U, "C": vefd.C,
            "sigma": vefd.SIGMA_P, "pops": vefd.POPS, "R": vefd.RPREV, "gA": vefd.G_A, "gB": vefd.G_B,
            "Fp": vefd.F_P, "tau": vefd.TAU}


PARAM_DEFAULTS = dict(lattice=1, nx=8, ny=6, nz=5, ncomp=2, walls=1, G=1.5, eta_A=0.2, eta_B=0.3, delta=0.1,
                      u_wall=0.0, fext=(0.0, 0.0, 0.0), tau_p=100.0, eta_p=0.0, L2=100.0, kappa=0.0, phase=0,
                      fd_on=1, coupling=0, collision=0, chol=0)


class Pair:
    def __init__(self, **kw):
        from paper_1406_2686_gb300 import vefd
        p = dict(PARAM_DEFAULTS)
        p.update(kw)
        if p["lattice"] == 0:
            p["nz"] = 1
        self.p = p
        self.o = oracle.Oracle(**p)
        self.g = vefd.Lattice(lattice=p["lattice"], nx=p["nx"], ny=p["ny"], nz=p["nz"], ncomp=p["ncomp"],
                              walls=p["walls"], G=p["G"], eta_A=p["eta_A"], eta_B=p["eta_B"], delta=p["delta"])
        self.g.set_wall_shear(p["u_wall"])
        self.g.set_body_force(*p["fext"])
        self.g.set_fenep(p["tau_p"], p["eta_p"], p["L2"], p["kappa"], p["phase"], p["fd_on"])
        self.g.set_polymer_coupling(p["coupling"])
        self.g.set_collision(p["collision"])
        self.g.set_conformation_update(p["chol"])
        self.gf = gpu_fields()

    def init(self, rhoA, rhoB=None, u=None, C=None):
        r = [inputs.to_f32_exact(a) for a in (rhoA, rhoB, u, C)]
        self.o.init_fields(*r)
        self.g.init_fields(*r)

    def init_random(self, seed=1, **kw):
        p = self.p
        ndim = 3 if p["lattice"] == 1 else 2
        nc = 6 if p["lattice"] == 1 else 4
        rA, rB, u, C = inputs.random_state(p["nx"], p["ny"], p["nz"], ndim, p["ncomp"], nc, seed=seed, **kw)
        self.init(rA, rB, u, C)

    def step(self, n):
        self.o.step(n)
        self.g.step(n)

    def both(self, name):
        return self.g.read(self.gf[name]).astype(np.float64), self.o.read(OR_FIELD[name])


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))


def identity_rows(nc):
    """1 on the diagonal components of a stored tensor (xx xy xz yy yz zz, or
    xx xy yy zz for D2Q9), 0 elsewhere."""
    return np.array([1, 0, 0, 1, 0, 1.0]) if nc == 6 else np.array([1, 0, 1, 1.0])


def dev_rel_l2(a, b):
    """Relative L2 of the departure from the identity of two tensor fields
    shaped (nc, ...): ||(a - I) - (b - I)|| / ||b - I||.  The identity
    dominates ||C||, so this is the measure of the polymer deformation."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    eye = identity_rows(a.shape[0]).reshape((-1,) + (1,) * (a.ndim - 1))
    return rel_l2(a - eye, b - eye)
