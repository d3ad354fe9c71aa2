"""Pins of the oracle's two paper-faithful variants of Sec. 2.

Moment-space (MRT) collision: the paper relaxes each component in the
orthogonal moment basis of Premnath & Abraham (the polynomial rows of
d'Humieres et al. for D3Q19; Lallemand & Luo's for D2Q9), with the
transport coefficients of Eq. TRANSPORTCOEFF: mobility mu = tau_M - 1/2,
shear viscosity rho c_s^2 (tau_s - 1/2), tau_b = tau_s, non-hydrodynamic
modes at unit relaxation time.

Cholesky scheme: sigma_P = f(r_P) C = L L^T, evolved through ln l_ii and
l_ij (Sec. 2, after Vaithianathan & Collins and Perlekar et al.).

Every pin checks the oracle against something other than its own formula:
textbook row norms, exact reduction to the single-relaxation-time form, the
diffusion and viscosity the paper's Eq. TRANSPORTCOEFF predicts, conservation,
a finite-difference derivative, closed-form steady states and the
second-order agreement of two discretisations of the same equation.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf

CS2 = 1.0 / 3.0

# textbook squared row norms of the orthogonal moment bases
NORMS = {oracle.D3Q19: [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8],
         oracle.D2Q9: [9, 36, 36, 6, 12, 6, 12, 4, 4]}


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mrt_basis(lat):
    """Rows are integer, mutually orthogonal, with the published squared
    norms; the conserved density row is all ones and the momentum rows are
    c_x, c_y (, c_z)."""
    M, kind = oracle.mrt_basis(lat)
    c, _ = oracle.lattice(lat)
    G = M @ M.T
    assert np.array_equal(M, np.round(M))
    assert np.allclose(G, np.diag(NORMS[lat]), atol=0)
    assert np.all(M[0] == 1) and kind[0] == 0
    mom = [k for k in range(len(kind)) if kind[k] == 2]
    assert len(mom) == (3 if lat == oracle.D3Q19 else 2)
    for d, k in enumerate(mom):
        assert np.array_equal(M[k], c[:, d])
    nshear = 5 if lat == oracle.D3Q19 else 2
    assert list(kind).count(3) == nshear and list(kind).count(1) == 1


def _uniform_tau_state(lat, seed):
    """Two components with rho_A + rho_B = 2 everywhere and equal viscosities:
    the local tau is the same at every node."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (6, 5, 4) if lat == oracle.D3Q19 else (7, 6, 1)
    r = 0.1 * rng.uniform(-1, 1, (nz, ny, nx))
    ndim = 3 if lat == oracle.D3Q19 else 2
    u = 0.03 * rng.uniform(-1, 1, (ndim, nz, ny, nx))
    nc = 6 if lat == oracle.D3Q19 else 4
    C = np.zeros((nc, nz, ny, nx))
    diag = (0, 3, 5) if nc == 6 else (0, 2, 3)
    for k in range(nc):
        C[k] = (1.0 if k in diag else 0.0) + 0.1 * rng.uniform(-1, 1, (nz, ny, nx))
    return dict(nx=nx, ny=ny, nz=nz), 1.0 + r, 1.0 - r, u, C


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
@pytest.mark.parametrize("coupling", [0, 1])
def test_mrt_with_equal_rates_is_bgk(lat, coupling):
    """With every moment relaxed at the one time tau (tau_M = tau_g = tau),
    Eq. (LB) in moment space is the single-relaxation-time step exactly."""
    dims, rA, rB, u, C = _uniform_tau_state(lat, 4)
    eta = 0.2
    tau = 0.5 + eta / (2.0 * CS2)  # rho = 2
    kw = dict(lattice=lat, ncomp=2, walls=1, G=1.2, eta_A=eta, eta_B=eta, u_wall=0.02, tau_p=30.0, eta_p=0.1,
              L2=40.0, kappa=0.01, phase=1, coupling=coupling, **dims)
    a = oracle.Oracle(collision=0, **kw)
    b = oracle.Oracle(collision=1, tau_M=tau, tau_g=tau, **kw)
    for o in (a, b):
        o.init_fields(rA, rB, u, C)
        o.step(1)
    pa, pb = a.read(oracle.F_POPS), b.read(oracle.F_POPS)
    assert np.max(np.abs(pa - pb)) < 1e-13
    # a different non-hydrodynamic rate changes the result (the basis is used)
    c = oracle.Oracle(collision=1, tau_M=tau, tau_g=1.0, **kw)
    c.init_fields(rA, rB, u, C)
    c.step(1)
    assert np.max(np.abs(c.read(oracle.F_POPS) - pa)) > 1e-8


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mrt_one_component_ignores_tau_M(lat):
    """One component: the momentum moment's non-equilibrium part is exactly
    -F/2 (Eq. equilibrium:vel), so its relaxation time cancels against the
    (1 - 1/(2 tau_M)) source; results do not depend on tau_M."""
    dims, rA, _, u, C = _uniform_tau_state(lat, 6)
    kw = dict(lattice=lat, ncomp=1, walls=1, eta_A=0.15, eta_B=0.15, u_wall=0.02, fext=(1e-5, -2e-5, 0.0),
              tau_p=30.0, eta_p=0.2, L2=40.0, kappa=0.01, collision=1, **dims)
    outs = []
    for tM in (1.0, 0.7, 1.6):
        o = oracle.Oracle(tau_M=tM, **kw)
        o.init_fields(rA, None, u, C)
        o.step(6)
        outs.append(o.read(oracle.F_POPS))
    assert np.max(np.abs(outs[1] - outs[0])) < 1e-12
    assert np.max(np.abs(outs[2] - outs[0])) < 1e-12


@pytest.mark.parametrize("tau_M", [0.8, 1.0, 1.5])
def test_mrt_interdiffusion_mobility(tau_M):
    """Two ideal components (G = 0): a small concentration wave decays at
    D k^2 with D = c_s^2 mu and mu = tau_M - 1/2 (Eq. TRANSPORTCOEFF),
    whatever the shear relaxation time."""
    nx = 64
    k = 2 * math.pi / nx
    x = np.arange(nx)
    wave = np.cos(k * x)
    rA = np.broadcast_to(1 + 0.01 * wave, (1, 2, nx))
    rB = np.broadcast_to(1 - 0.01 * wave, (1, 2, nx))
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=2, ncomp=2, walls=0, G=0.0, eta_A=0.2, eta_B=0.2, fd_on=0,
                      collision=1, tau_M=tau_M, tau_g=1.0)
    o.init_fields(rA, rB)
    amps = []
    for _ in range(6):
        o.step(200)
        a = o.read(oracle.F_RHO_A)[0, 0]
        amps.append(np.dot(a - a.mean(), wave) / np.dot(wave, wave))
    rate = -np.polyfit(np.arange(6) * 200.0, np.log(amps), 1)[0]
    assert abs(rate / (CS2 * (tau_M - 0.5) * k * k) - 1.0) < 5e-3


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mrt_shear_wave_viscosity(lat):
    """A transverse shear wave decays at nu k^2 with rho c_s^2 (tau_s - 1/2)
    = eta (Eqs. TRANSPORTCOEFF, smoothingvisco) when the other modes relax
    with the paper's unit times."""
    ny = 48
    nx, nz = (2, 2) if lat == oracle.D3Q19 else (2, 1)
    k = 2 * math.pi / ny
    y = np.arange(ny)
    ndim = 3 if lat == oracle.D3Q19 else 2
    u0 = np.zeros((ndim, nz, ny, nx))
    u0[0] = 1e-3 * np.sin(k * y)[None, :, None]
    eta, rho = 0.1, 1.3
    o = oracle.Oracle(lattice=lat, nx=nx, ny=ny, nz=nz, ncomp=1, walls=0, eta_A=eta, eta_B=eta, fd_on=0,
                      collision=1)
    o.init_fields(np.full((nz, ny, nx), rho), None, u0)
    amps = []
    for _ in range(6):
        o.step(100)
        u = o.read(oracle.F_U)[0, 0, :, 0]
        amps.append(np.dot(u, np.sin(k * y)) / np.dot(np.sin(k * y), np.sin(k * y)))
    rate = -np.polyfit(np.arange(6) * 100.0, np.log(amps), 1)[0]
    assert abs(rate / (eta / rho * k * k) - 1.0) < 5e-3


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mrt_conservation(lat):
    """Component masses are exact and, in a periodic box, total momentum
    grows by N F_ext per step (the moment relaxation conserves the density
    rows; the momentum rows exchange momentum between components only)."""
    nx, ny, nz = (12, 10, 8) if lat == oracle.D3Q19 else (12, 10, 1)
    from paper_1406_2686_gb300 import inputs
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=3.0, width=3.0, seed=5)
    F = np.array([2e-6, -1e-6, 5e-7 if lat == oracle.D3Q19 else 0.0])
    o = oracle.Oracle(lattice=lat, nx=nx, ny=ny, nz=nz, ncomp=2, walls=0, G=1.5, eta_A=0.2, eta_B=0.3, fext=F,
                      tau_p=50.0, eta_p=0.1, L2=50.0, kappa=1e-2, phase=1, collision=1)
    o.init_fields(rA, rB)
    d0 = o.diagnostics()
    o.step(40)
    d1 = o.diagnostics()
    assert abs(d1[0] - d0[0]) < 1e-12 * d0[0] and abs(d1[1] - d0[1]) < 1e-12 * d0[1]
    assert np.allclose(d1[2:5] - d0[2:5], 40 * o.N * F, rtol=1e-9, atol=1e-12)


# --- Cholesky scheme --------------------------------------------------------

def _full(v):
    return np.array([[v[0], v[1], v[2]], [v[1], v[3], v[4]], [v[2], v[4], v[5]]])


def _sigma(C, L2):
    return (L2 - 3.0) / (L2 - (C[0] + C[3] + C[5])) * C


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_chol_rates_identity(seed):
    """For the log-Cholesky variables of sigma_P = f C and their rates:
    C is recovered exactly, and dL/dt L^T + L dL/dt^T equals the derivative
    of sigma_P(C) = f(tr C) C along dC/dt (central finite difference)."""
    rng = np.random.default_rng(seed)
    L2 = 30.0
    A = rng.normal(size=(3, 3))
    Cm = np.eye(3) + 0.3 * A @ A.T
    C = np.array([Cm[0, 0], Cm[0, 1], Cm[0, 2], Cm[1, 1], Cm[1, 2], Cm[2, 2]])
    Cd = rng.normal(size=6)
    lam, rl = oracle.chol_rates(C, Cd, L2)
    assert np.max(np.abs(oracle.chol_to_C(lam, L2) - C)) < 1e-13
    slot = {(0, 0): 0, (1, 0): 1, (2, 0): 2, (1, 1): 3, (2, 1): 4, (2, 2): 5}
    L, Ld = np.zeros((3, 3)), np.zeros((3, 3))
    for (i, j), k in slot.items():
        if i == j:
            L[i, i] = math.exp(lam[k])
            Ld[i, i] = rl[k] * L[i, i]
        else:
            L[i, j], Ld[i, j] = lam[k], rl[k]
    eps = 1e-6
    sd = _full((_sigma(C + eps * Cd, L2) - _sigma(C - eps * Cd, L2)) / (2 * eps))
    assert np.max(np.abs(Ld @ L.T + L @ Ld.T - sd)) < 1e-8 * np.max(np.abs(sd))
    assert np.allclose(L @ L.T, _full(_sigma(C, L2)), rtol=1e-13, atol=1e-13)


def _shear_g(gdot):
    g = np.zeros((3, 3))
    g[1, 0] = gdot
    return g


@pytest.mark.parametrize("Lam,L2", [(0.625, 100.0), (5.0, 1e4), (30.0, 100.0)])
def test_chol_steady_shear(Lam, L2):
    """The Cholesky scheme has the steady shear state of Eqs. (lindner),
    (lindner2) as its fixed point."""
    taup = 200.0
    C, _, _ = oracle.fenep_point(np.array([1, 0, 0, 1, 0, 1.0]), _shear_g(Lam / taup), taup, L2, int(60 * taup),
                                 chol=1)
    Cex, _ = cf.shear_conformation(Lam, L2)
    assert np.allclose(C, Cex, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("L2", [10.0, 100.0])
def test_chol_steady_elongation(L2):
    """Steady uniaxial elongation of the Cholesky scheme solves Eq. (el8)."""
    taup = 4000.0
    for Lam_e in (0.05, 0.8, 20.0):
        ed = Lam_e / taup
        C, _, _ = oracle.fenep_point(np.array([1, 0, 0, 1, 0, 1.0]), np.diag([-ed / 2, -ed / 2, ed]), taup, L2,
                                     int(80 * taup), chol=1)
        sig = _sigma(C, L2)
        assert abs(cf.elong_Lambda_e(sig[5] - sig[0], L2) - Lam_e) < 1e-7 * max(1.0, Lam_e)


def test_chol_second_order_agreement():
    """The Cholesky and direct schemes are two AB2 discretisations of the same
    equation: along a shear start-up their difference falls as (dt/tau_P)^2."""
    diffs = []
    for taup in (100.0, 400.0):
        g = _shear_g(2.0 / taup)
        a = b = np.array([1, 0, 0, 1, 0, 1.0])
        Ra, Rb = np.zeros(6), np.zeros(6)
        ha = hb = False
        err = 0.0
        for _ in range(int(5 * taup)):
            a, Ra, ha = oracle.fenep_point(a, g, taup, 100.0, 1, Ra, ha, chol=0)
            b, Rb, hb = oracle.fenep_point(b, g, taup, 100.0, 1, Rb, hb, chol=1)
            err = max(err, np.max(np.abs(a - b)) / np.max(np.abs(a)))
        diffs.append(err)
    assert diffs[0] < 1e-3
    assert 12.0 < diffs[0] / diffs[1] < 20.0


@pytest.mark.parametrize("case", [("elong", 10.0, 20.0, 0.14), ("elong", 100.0, 100.0, 0.08),
                                  ("shear", 100.0, 10.0, 1.0)])
def test_chol_keeps_spd(case):
    """Strong flows at coarse time steps: the direct AB2 update on C loses
    positive definiteness or crosses tr C = L^2, while the Cholesky scheme
    keeps C SPD with tr C < L^2 at every step (Sec. 2)."""
    kind, L2, taup, rate = case
    g = np.diag([-rate / 2, -rate / 2, rate]) if kind == "elong" else _shear_g(rate)

    def first_violation(chol):
        C, R, hp = np.array([1, 0, 0, 1, 0, 1.0]), np.zeros(6), False
        for n in range(800):
            C, R, hp = oracle.fenep_point(C, g, taup, L2, 1, R, hp, chol=chol)
            if not np.all(np.isfinite(C)):
                return n
            if C[0] + C[3] + C[5] >= L2 or np.linalg.eigvalsh(_full(C)).min() <= 0:
                return n
        return None

    assert first_violation(0) is not None
    assert first_violation(1) is None


@pytest.mark.slow
def test_chol_couette_closed_form():
    """FENE-P Couette with feedback under the Cholesky scheme reaches the same
    closed-form steady state as the direct scheme (Sec. 3.1)."""
    ny, U = 16, 0.02
    gdot = 2 * U / ny
    taup = 0.625 / gdot
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=4, ny=ny, eta_A=1 / 6, eta_B=1 / 6, u_wall=U, tau_p=taup,
                      eta_p=1 / 9, L2=100.0, chol=1, collision=1)
    o.init_fields(np.ones((1, ny, 4)))
    o.step(int(25 * taup))
    Cex, _ = cf.shear_conformation(-0.625, 100.0)
    C = o.read(oracle.F_C)
    for k, kk in enumerate((0, 1, 3, 5)):
        assert np.max(np.abs(C[k] - Cex[kk])) < 1e-6 * max(1, abs(Cex[kk]))
    u = o.read(oracle.F_U)[0]
    assert np.max(np.abs(u - cf.couette_profile(ny, U)[None, :, None])) < 1e-9
