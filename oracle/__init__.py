"""FP64 CPU oracle of the hybrid LBM / FD viscoelastic step.

TEST INFRASTRUCTURE ONLY.  This package restates the method of Gupta,
Sbragaglia & Scagliarini (Sec. 2 and the closed forms of Sec. 3) plainly and
slowly, to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It imports nothing
from the CUDA package and the CUDA package imports nothing from it.

``Oracle`` wraps the C implementation in ``oracle.c`` (loaded with ctypes);
``closed_forms`` holds the analytic results the oracle is pinned against.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

D2Q9, D3Q19 = 0, 1
F_RHO_A, F_RHO_B, F_PHI, F_U, F_C, F_SIGMA_P, F_POPS, F_RPREV = range(8)
F_G_A, F_G_B, F_F_P, F_TAU = 8, 9, 10, 11
ST_NAN, ST_TRACE, ST_MACH, ST_RHO = 1, 2, 4, 8


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("ncomp", ctypes.c_int), ("walls", ctypes.c_int),
        ("G", ctypes.c_double), ("eta_A", ctypes.c_double), ("eta_B", ctypes.c_double),
        ("delta", ctypes.c_double), ("u_wall", ctypes.c_double), ("fext", ctypes.c_double * 3),
        ("tau_p", ctypes.c_double), ("eta_p", ctypes.c_double), ("L2", ctypes.c_double),
        ("kappa", ctypes.c_double), ("phase", ctypes.c_int), ("fd_on", ctypes.c_int), ("coupling", ctypes.c_int),
        ("collision", ctypes.c_int), ("tau_M", ctypes.c_double), ("tau_g", ctypes.c_double), ("chol", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_num_c.argtypes = [vp]
        L.orc_q.argtypes = [vp]
        L.orc_init_fields.argtypes = [vp, dp, dp, dp, dp]
        L.orc_set_params.argtypes = [vp, ctypes.POINTER(OrcParams)]
        L.orc_step.argtypes = [vp, ctypes.c_long]
        L.orc_write_field.argtypes = [vp, ctypes.c_int, dp]
        L.orc_read_field.argtypes = [vp, ctypes.c_int, dp]
        L.orc_set_have_prev.argtypes = [vp, ctypes.c_int]
        L.orc_status.restype = ctypes.c_uint
        L.orc_status.argtypes = [vp]
        L.orc_steps_done.restype = ctypes.c_long
        L.orc_steps_done.argtypes = [vp]
        L.orc_diagnostics.argtypes = [vp, dp]
        L.orc_lattice.argtypes = [ctypes.c_int, ip, dp]
        L.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_source.argtypes = [ctypes.c_int, dp, dp, dp]
        L.orc_fenep_point.argtypes = [dp, dp, ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_long]
        L.orc_fenep_point_form.argtypes = [dp, dp, ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                           ctypes.c_int]
        L.orc_chol_rates.argtypes = [dp, dp, ctypes.c_double, dp, dp]
        L.orc_chol_to_C.argtypes = [dp, ctypes.c_double, dp]
        L.orc_mrt_basis.argtypes = [ctypes.c_int, dp, ip]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


DEFAULTS = dict(lattice=D2Q9, nx=8, ny=8, nz=1, ncomp=1, walls=1, G=0.0, eta_A=1.0 / 6.0,
                eta_B=1.0 / 6.0, delta=0.1, u_wall=0.0, fext=(0.0, 0.0, 0.0), tau_p=1000.0,
                eta_p=0.0, L2=100.0, kappa=0.0, phase=0, fd_on=1, coupling=0, collision=0, tau_M=1.0,
                tau_g=1.0, chol=0)


def make_params(**kw):
    d = dict(DEFAULTS)
    for k in kw:
        if k not in d:
            raise KeyError(k)
    d.update(kw)
    p = OrcParams()
    for k, v in d.items():
        if k == "fext":
            p.fext = (ctypes.c_double * 3)(*[float(t) for t in v])
        else:
            setattr(p, k, type(getattr(p, k))(v))
    return p, d


class Oracle:
    """One lattice of the FP64 oracle.  Fields are numpy arrays shaped
    (comp, nz, ny, nx) (comp dropped for scalars)."""

    def __init__(self, **kw):
        self.params, self.cfg = make_params(**kw)
        self._s = lib().orc_create(ctypes.byref(self.params))
        if not self._s:
            raise ValueError("oracle rejected parameters: %r" % (self.cfg,))
        self.nx, self.ny, self.nz = self.cfg["nx"], self.cfg["ny"], self.cfg["nz"]
        self.N = self.nx * self.ny * self.nz
        self.Q = lib().orc_q(self._s)
        self.nc = lib().orc_num_c(self._s)
        self.ndim = 3 if self.cfg["lattice"] == D3Q19 else 2

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            lib().orc_destroy(s)
            self._s = None

    def set_params(self, **kw):
        cfg = dict(self.cfg)
        cfg.update(kw)
        p, d = make_params(**cfg)
        if lib().orc_set_params(self._s, ctypes.byref(p)) != 0:
            raise ValueError("bad parameters")
        self.params, self.cfg = p, d

    def _shape(self, ncomp):
        return (ncomp, self.nz, self.ny, self.nx) if ncomp > 1 else (self.nz, self.ny, self.nx)

    def init_fields(self, rhoA, rhoB=None, u=None, C=None):
        rA = _f64(rhoA).reshape(-1)
        rB = _f64(rhoB).reshape(-1) if rhoB is not None else None
        uu = _f64(u).reshape(-1) if u is not None else None
        CC = _f64(C).reshape(-1) if C is not None else None
        rc = lib().orc_init_fields(self._s, _dptr(rA), _dptr(rB) if rB is not None else None,
                                   _dptr(uu) if uu is not None else None,
                                   _dptr(CC) if CC is not None else None)
        if rc != 0:
            raise ValueError("init_fields failed")

    def step(self, n=1):
        if lib().orc_step(self._s, int(n)) != 0:
            raise RuntimeError("oracle step failed")

    def _ncomp_of(self, field):
        if field in (F_RHO_A, F_RHO_B, F_PHI, F_TAU):
            return 1
        if field in (F_U, F_G_A, F_G_B, F_F_P):
            return self.ndim
        if field in (F_C, F_SIGMA_P, F_RPREV):
            return self.nc
        if field == F_POPS:
            return self.cfg["ncomp"] * self.Q
        raise ValueError(field)

    def read(self, field):
        nc = self._ncomp_of(field)
        out = np.empty(nc * self.N, dtype=np.float64)
        if lib().orc_read_field(self._s, field, _dptr(out)) != 0:
            raise RuntimeError("read_field failed")
        return out.reshape(self._shape(nc))

    def write(self, field, arr):
        a = _f64(arr).reshape(-1)
        if a.size != self._ncomp_of(field) * self.N:
            raise ValueError("size mismatch")
        if lib().orc_write_field(self._s, field, _dptr(a)) != 0:
            raise RuntimeError("write_field failed")

    def set_have_prev(self, hp):
        lib().orc_set_have_prev(self._s, int(hp))

    @property
    def status(self):
        return int(lib().orc_status(self._s))

    @property
    def steps_done(self):
        return int(lib().orc_steps_done(self._s))

    def diagnostics(self):
        out = np.zeros(16, dtype=np.float64)
        lib().orc_diagnostics(self._s, _dptr(out))
        return out


def set_threads(n=0):
    """OpenMP threads for the oracle's node loops; returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def lattice(lat):
    Q = 19 if lat == D3Q19 else 9
    c = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    lib().orc_lattice(lat, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(w))
    return c.reshape(Q, 3), w


def equilibrium(lat, rho, u):
    Q = 19 if lat == D3Q19 else 9
    uu = _f64(u)
    out = np.zeros(Q)
    lib().orc_equilibrium(lat, float(rho), _dptr(uu), _dptr(out))
    return out


def source(lat, u, F):
    Q = 19 if lat == D3Q19 else 9
    uu, FF = _f64(u), _f64(F)
    out = np.zeros(Q)
    lib().orc_source(lat, _dptr(uu), _dptr(FF), _dptr(out))
    return out


def fenep_point(C, gradu, tau_p, L2, nsteps, Rprev=None, have_prev=False, chol=0):
    """Advance a uniform conformation tensor C (6 comps xx xy xz yy yz zz)
    under a prescribed velocity gradient gradu[i][j] = d_i u_j (chol 1: the
    Cholesky scheme on sigma_P; the history then holds log-Cholesky rates)."""
    CC = _f64(C).copy()
    R = _f64(Rprev).copy() if Rprev is not None else np.zeros(6)
    hp = ctypes.c_int(1 if have_prev else 0)
    g = _f64(gradu).reshape(-1)
    lib().orc_fenep_point_form(_dptr(CC), _dptr(R), ctypes.byref(hp), _dptr(g), float(tau_p), float(L2),
                               int(nsteps), int(chol))
    return CC, R, bool(hp.value)


def chol_rates(C, Cdot, L2):
    """(lam, lam_dot): log-Cholesky variables of sigma_P = f(r_P) C and their
    rates for a given dC/dt (6 comps xx xy xz yy yz zz each)."""
    CC, Cd = _f64(C).copy(), _f64(Cdot).copy()
    lam, rl = np.zeros(6), np.zeros(6)
    lib().orc_chol_rates(_dptr(CC), _dptr(Cd), float(L2), _dptr(lam), _dptr(rl))
    return lam, rl


def chol_to_C(lam, L2):
    out = np.zeros(6)
    lib().orc_chol_to_C(_dptr(_f64(lam).copy()), float(L2), _dptr(out))
    return out


def mrt_basis(lat):
    """(M, kind): the MRT moment basis, M[k, a] for row k and direction a, and
    each row's relaxation kind (0 density, 1 bulk, 2 momentum, 3 shear, 4 other)."""
    Q = 19 if lat == D3Q19 else 9
    M = np.zeros(Q * Q)
    kind = np.zeros(Q, dtype=np.int32)
    lib().orc_mrt_basis(lat, _dptr(M), kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return M.reshape(Q, Q), kind
