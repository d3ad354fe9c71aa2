"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types an oracle
formula: they check moment identities, closed-form solutions, conservation
laws and exact discrete solutions, chosen so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf

CS2 = 1.0 / 3.0


# --- lattice tables and single-node formulas (Sec. 2) ----------------------

@pytest.mark.parametrize("lat,Q", [(oracle.D2Q9, 9), (oracle.D3Q19, 19)])
def test_lattice_isotropy(lat, Q):
    """Weights sum to 1; odd moments vanish; second moment c_s^2 I with
    c_s^2 = 1/3 (Sec. 2); fourth moment c_s^4 (d_ij d_kl + d_ik d_jl + d_il d_jk)."""
    c, w = oracle.lattice(lat)
    assert c.shape == (Q, 3)
    D = 3 if lat == oracle.D3Q19 else 2
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("a,ai->i", w, c), 0.0, atol=1e-16)
    M2 = np.einsum("a,ai,aj->ij", w, c, c)
    assert np.allclose(M2[:D, :D], CS2 * np.eye(D), atol=1e-15)
    M3 = np.einsum("a,ai,aj,ak->ijk", w, c, c, c)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c)[:D, :D, :D, :D]
    d = np.eye(D)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    assert np.allclose(M4, iso, atol=1e-15)
    # D3Q19 weight classes of Sec. 2: 1/3, 1/18 (speeds 1), 1/36 (speeds sqrt 2)
    speed2 = (c ** 2).sum(1)
    if lat == oracle.D3Q19:
        assert np.allclose(w[speed2 == 0], 1 / 3) and np.allclose(w[speed2 == 1], 1 / 18)
        assert np.allclose(w[speed2 == 2], 1 / 36)
        assert (speed2 == 1).sum() == 6 and (speed2 == 2).sum() == 12
    # opposite pairs: a and its partner (odd a -> a+1) have c -> -c
    for a in range(1, Q, 2):
        assert np.array_equal(c[a], -c[a + 1])


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_equilibrium_moments(lat):
    """Sum E = rho, sum c E = rho u, sum c c E = rho (c_s^2 I + u u) for the
    equilibrium of Sec. 2."""
    rng = np.random.default_rng(3)
    c, _ = oracle.lattice(lat)
    D = 3 if lat == oracle.D3Q19 else 2
    for _ in range(5):
        rho = rng.uniform(0.1, 2.0)
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.1, 0.1, D)
        E = oracle.equilibrium(lat, rho, u)
        assert abs(E.sum() - rho) < 1e-14
        assert np.allclose(c.T @ E, rho * u, atol=1e-15)
        P = np.einsum("a,ai,aj->ij", E, c, c)[:D, :D]
        assert np.allclose(P, rho * (CS2 * np.eye(D) + np.outer(u[:D], u[:D])), atol=1e-14)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_source_moments(lat):
    """The forcing source of Sec. 2 has zero mass, momentum F and second
    moment u F + F u (the moments it is built to have)."""
    rng = np.random.default_rng(4)
    c, _ = oracle.lattice(lat)
    D = 3 if lat == oracle.D3Q19 else 2
    for _ in range(5):
        u = np.zeros(3)
        F = np.zeros(3)
        u[:D] = rng.uniform(-0.1, 0.1, D)
        F[:D] = rng.uniform(-1e-3, 1e-3, D)
        S = oracle.source(lat, u, F)
        assert abs(S.sum()) < 1e-17
        assert np.allclose(c.T @ S, F, atol=1e-17)
        M2 = np.einsum("a,ai,aj->ij", S, c, c)[:D, :D]
        assert np.allclose(M2, np.outer(u[:D], F[:D]) + np.outer(F[:D], u[:D]), atol=1e-17)


# --- channel flows (Sec. 3.1 set-up) ---------------------------------------

@pytest.mark.parametrize("lat,nz", [(oracle.D2Q9, 1), (oracle.D3Q19, 2)])
def test_couette_newtonian_exact(lat, nz):
    """Moving walls with the bounce-back rule: the steady profile is the exact
    line u_x = U (NY - 1 - 2y)/NY with +U at the lower wall (Sec. 3.1)."""
    ny, U = 12, 0.02
    o = oracle.Oracle(lattice=lat, nx=3, ny=ny, nz=nz, eta_A=0.1, eta_B=0.1, u_wall=U, fd_on=0)
    o.init_fields(np.ones((nz, ny, 3)))
    o.step(4000)
    u = o.read(oracle.F_U)
    ex = cf.couette_profile(ny, U)
    assert np.max(np.abs(u[0] - ex[None, :, None])) < 1e-12 * 1e2
    assert np.max(np.abs(u[1])) < 1e-13
    assert u[0, 0, 0, 0] > 0  # lower wall moves in +x


def test_poiseuille_curvature_and_slip():
    """Body-force channel flow: the bulk second difference equals -F/eta
    (eta = rho c_s^2 (tau - 1/2), Eq. TRANSPORTCOEFF), and the profile is
    exact at tau = 1/2 + sqrt(3)/4 and otherwise offset by the textbook
    half-way bounce-back slip F (16 (tau-1/2)^2 - 3) / (24 nu)
    (He, Zou, Luo & Dembo 1997)."""
    H, F = 16, 1e-6
    for tau in (0.5 + math.sqrt(3.0) / 4.0, 0.8, 1.3):
        eta = (tau - 0.5) / 3.0
        o = oracle.Oracle(lattice=oracle.D2Q9, nx=2, ny=H, eta_A=eta, eta_B=eta, fext=(F, 0, 0), fd_on=0)
        o.init_fields(np.ones((1, H, 2)))
        o.step(int(12 * H * H / eta))
        u = o.read(oracle.F_U)[0, 0, :, 0]
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        assert np.allclose(d2, -F / eta, rtol=1e-7)
        slip = F * (16 * (tau - 0.5) ** 2 - 3.0) / (24.0 * eta)
        ex = cf.poiseuille_profile(H, F, eta) + slip
        assert np.max(np.abs(u - ex)) < 1e-6 * ex.max()


@pytest.mark.parametrize("rho,comp", [(1.0, "A"), (2.0, "A"), (1.5, "B")])
def test_shear_wave_viscosity(rho, comp):
    """A transverse shear wave decays at nu k^2 with nu = eta/rho and
    rho c_s^2 (tau - 1/2) = eta_A f_+ + eta_B f_- (Eqs. TRANSPORTCOEFF,
    smoothingvisco): a pure-A fluid (phi = 1) takes eta_A, pure-B takes eta_B."""
    ny, nx = 48, 2
    etaA, etaB = 0.05, 0.2
    k = 2 * math.pi / ny
    y = np.arange(ny)
    u0 = np.zeros((2, 1, ny, nx))
    u0[0, 0] = 1e-3 * np.sin(k * y)[:, None]
    r = np.full((1, ny, nx), rho)
    zero = np.zeros_like(r)
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, ncomp=2, walls=0, G=0.0, eta_A=etaA, eta_B=etaB, fd_on=0)
    if comp == "A":
        o.init_fields(r, zero, u0)
        eta = etaA
    else:
        o.init_fields(zero, r, u0)
        eta = etaB
    amps = []
    for _ in range(6):
        o.step(100)
        u = o.read(oracle.F_U)[0, 0, :, 0]
        amps.append(np.dot(u, np.sin(k * y)) / np.dot(np.sin(k * y), np.sin(k * y)))
    rate = -np.polyfit(np.arange(6) * 100.0, np.log(amps), 1)[0]
    nu = eta / rho
    assert abs(rate / (nu * k * k) - 1.0) < 5e-3


# --- conservation laws --------------------------------------------------------

def _droplet_oracle(lat, walls, fext=(0, 0, 0), n=(12, 10, 8)):
    nx, ny, nz = n if lat == oracle.D3Q19 else (n[0], n[1], 1)
    from paper_1406_2686_gb300 import inputs
    rA, rB = inputs.droplet_fields(nx, ny, nz, R=3.0, width=3.0, seed=5)
    o = oracle.Oracle(lattice=lat, nx=nx, ny=ny, nz=nz, ncomp=2, walls=walls, G=1.5, eta_A=0.2, eta_B=0.3,
                      u_wall=0.02 if walls else 0.0, fext=fext, tau_p=50.0, eta_p=0.1, L2=50.0, kappa=1e-2,
                      phase=1)
    o.init_fields(rA, rB)
    return o


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_mass_conservation(lat):
    """Per-component mass is exactly conserved: the source has no zeroth
    moment (Sec. 2) and bounce-back returns every population."""
    o = _droplet_oracle(lat, walls=1)
    m0 = o.diagnostics()[:2]
    o.step(60)
    m1 = o.diagnostics()[:2]
    assert np.all(np.abs(m1 / m0 - 1.0) < 1e-13)
    assert o.status == 0


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_momentum_periodic(lat):
    """In a fully periodic box the Shan-Chen pair forces (Eq. SCforce) and the
    central-difference polymer divergence sum to zero, so total momentum
    grows by exactly N F_ext per step (the forcing adds F, Eq. LB)."""
    F = np.array([2e-6, -1e-6, 5e-7])
    if lat == oracle.D2Q9:
        F[2] = 0.0
    o = _droplet_oracle(lat, walls=0, fext=F)
    N = o.N
    p0 = o.diagnostics()[2:5]
    o.step(40)
    p1 = o.diagnostics()[2:5]
    assert np.allclose(p1 - p0, 40 * N * F, rtol=1e-9, atol=1e-12)


# --- Shan-Chen force (Eq. SCforce and its Taylor expansion) ---------------

@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_sc_force_taylor(lat):
    """For rho_B cubic along x, the lattice sum of Eq. (SCforce) equals its
    Taylor expansion exactly: g_A = -G rho_A (c_s^2 d_x rho_B + c_s^4/2 d_x^3
    rho_B) x (the expansion below Eq. PTexpanded; higher terms vanish)."""
    nx, ny = 24, 4
    nz = 3 if lat == oracle.D3Q19 else 1
    G = 1.3
    x = np.arange(nx, dtype=np.float64)
    xc = x - nx / 2
    rb = 1.0 + 1e-2 * xc + 2e-4 * xc ** 2 + 1e-5 * xc ** 3
    rB = np.broadcast_to(rb, (nz, ny, nx)).copy()
    rA = np.broadcast_to(0.5 + 0.01 * np.arange(ny)[:, None], (nz, ny, nx)).copy()
    o = oracle.Oracle(lattice=lat, nx=nx, ny=ny, nz=nz, ncomp=2, walls=0, G=G, fd_on=0)
    o.init_fields(rA, rB)
    g = o.read(oracle.F_G_A)
    d1 = 1e-2 + 4e-4 * xc + 3e-5 * xc ** 2
    d3 = 6e-5
    ex = -G * rA[..., :] * (CS2 * d1 + 0.5 * CS2 ** 2 * d3)
    inner = slice(2, nx - 2)
    assert np.allclose(g[0][..., inner], ex[..., inner], rtol=1e-12, atol=1e-16)
    assert np.max(np.abs(g[1])) < 1e-15
    # walls: the density seen across a wall is the adjacent row (zero normal gradient)
    o2 = oracle.Oracle(lattice=lat, nx=4, ny=6, nz=nz, ncomp=2, walls=1, G=G, fd_on=0)
    rAy = np.broadcast_to((1.0 + 0.1 * np.arange(6))[:, None], (nz, 6, 4)).copy()
    o2.init_fields(rAy, rAy)
    gy = o2.read(oracle.F_G_A)[1][0, :, 0]
    c, w = oracle.lattice(lat)
    s1 = w[c[:, 1] == 1].sum()  # weight of links pointing +y
    # row 0: the -y links see row 0 itself, the +y links row 1: sum = s1 (r1 - r0)
    assert abs(gy[0] - (-G * rAy[0, 0, 0] * s1 * (rAy[0, 1, 0] - rAy[0, 0, 0]))) < 1e-14
    assert abs(gy[-1] - (-G * rAy[0, -1, 0] * s1 * (rAy[0, -1, 0] - rAy[0, -2, 0]))) < 1e-14


# --- polymer feedback force ----------------------------------------------

def test_polymer_force_divergence():
    """F_p = (eta_P/tau_P) div(f C - I): for C = I + eps sin(k y) (e_x e_y + e_y e_x)
    (trace 3, so f = 1) the x-force is the exact central difference
    (eta_P/tau_P) eps sin(k) cos(k y), and there is no y-force (Eq. NS)."""
    ny, nx = 16, 3
    eps, etap, taup = 0.05, 0.3, 20.0
    k = 2 * math.pi / ny
    y = np.arange(ny)
    C = np.zeros((4, 1, ny, nx))
    C[0] = C[2] = C[3] = 1.0
    C[1] = eps * np.sin(k * y)[None, :, None]
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, walls=0, eta_p=etap, tau_p=taup, L2=30.0)
    o.init_fields(np.ones((1, ny, nx)), C=C)
    Fp = o.read(oracle.F_F_P)
    ex = etap / taup * eps * math.sin(k) * np.cos(k * y)
    assert np.allclose(Fp[0, 0, :, 0], ex, atol=1e-16)
    assert np.max(np.abs(Fp[1])) < 1e-17
    # diagonal stretch along x: the force follows d_x of sigma_P,xx = f C_xx
    C2 = np.zeros((4, 1, ny, nx))
    C2[2] = C2[3] = 1.0
    C2[0] = 1.0
    o.init_fields(np.ones((1, ny, nx)), C=C2)
    assert np.max(np.abs(o.read(oracle.F_F_P))) < 1e-17  # C = I: no feedback at rest


def test_polymer_force_phase_modulation():
    """The feedback is modulated by f_+(phi) (droplet phase) or f_-(phi)
    (matrix phase), f_+ + f_- = 1 (Sec. 2, last equation)."""
    ny, nx = 16, 3
    k = 2 * math.pi / ny
    y = np.arange(ny)
    C = np.zeros((4, 1, ny, nx))
    C[0] = C[2] = C[3] = 1.0
    C[1] = 0.05 * np.sin(k * y)[None, :, None]
    rA = np.broadcast_to((1.0 + 0.8 * np.cos(k * y))[:, None], (1, ny, nx)).copy()
    rB = 2.0 - rA
    forces = {}
    for ph in (-1, 0, 1):
        o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, ncomp=2, walls=0, eta_p=0.3, tau_p=20.0,
                          L2=30.0, phase=ph, delta=0.1)
        o.init_fields(rA, rB, C=C)
        forces[ph] = o.read(oracle.F_F_P)
    assert np.allclose(forces[1] + forces[-1], forces[0], atol=1e-17)
    # the droplet phase (phi > 0 where rho_A > rho_B) carries the f_+ feedback
    phi = ((rA - rB) / 2.0)[0, :, 0]
    deep_b = (phi < -0.5) & (np.roll(phi, 1) < -0.5) & (np.roll(phi, -1) < -0.5)
    assert deep_b.sum() >= 3
    assert np.max(np.abs(forces[1][0, 0, deep_b, 0])) < 1e-3 * np.max(np.abs(forces[0]))
    assert np.max(np.abs(forces[-1][0, 0, deep_b, 0] - forces[0][0, 0, deep_b, 0])) < 1e-3 * np.max(np.abs(forces[0]))


# --- FENE-P constitutive equation (Sec. 3) --------------------------------

def _shear_gradu(gdot):
    g = np.zeros((3, 3))
    g[1, 0] = gdot  # d_y u_x
    return g


@pytest.mark.parametrize("Lam,L2", [(0.625, 100.0), (5.0, 1e4), (30.0, 100.0), (0.2, 10.0)])
def test_fenep_steady_shear(Lam, L2):
    """Steady shear: S and N from Eqs. (lindner), (lindner2), sigma_P,yy =
    sigma_P,zz = 1 (Eq. steadyshear)."""
    taup = 200.0
    C0 = np.array([1, 0, 0, 1, 0, 1.0])
    C, R, hp = oracle.fenep_point(C0, _shear_gradu(Lam / taup), taup, L2, int(60 * taup))
    Cex, Z = cf.shear_conformation(Lam, L2)
    assert np.allclose(C, Cex, rtol=1e-9, atol=1e-12)
    f = (L2 - 3) / (L2 - (C[0] + C[3] + C[5]))
    sig = f * C
    assert abs(sig[1] - cf.shear_S(Lam, L2)) < 1e-9 * abs(cf.shear_S(Lam, L2))
    assert abs(sig[0] - 1 - cf.shear_N(Lam, L2)) < 1e-9 * cf.shear_N(Lam, L2)
    assert abs(sig[3] - 1) < 1e-10 and abs(sig[5] - 1) < 1e-10


def test_oldroyd_b_limit():
    """L^2 -> infinity: S -> Lambda and N -> 2 Lambda^2 (Sec. 3.1)."""
    taup, Lam = 100.0, 0.7
    C, _, _ = oracle.fenep_point(np.array([1, 0, 0, 1, 0, 1.0]), _shear_gradu(Lam / taup), taup, 1e10, 6000)
    assert abs(C[1] - Lam) < 1e-7 and abs(C[0] - 1 - 2 * Lam * Lam) < 1e-7


@pytest.mark.parametrize("L2", [10.0, 100.0, 1e4])
def test_fenep_steady_elongation(L2):
    """Steady uniaxial elongation: the steady D = sigma_zz - sigma_xx solves
    Eq. (el8) with the (+) root below D = L^2 - 3 and the (-) root above;
    D/Lambda_e -> 3 at small rate and -> 2 L^2 at large rate (Eq. dimensionalelong)."""
    taup = 4000.0
    seen_branch = set()
    for Lam_e in (1e-3, 0.05, 0.3, 0.8, 2.0, 20.0):
        ed = Lam_e / taup
        g = np.diag([-ed / 2, -ed / 2, ed])
        C, _, _ = oracle.fenep_point(np.array([1, 0, 0, 1, 0, 1.0]), g, taup, L2, int(80 * taup))
        f = (L2 - 3) / (L2 - (C[0] + C[3] + C[5]))
        sig = f * C
        D = sig[5] - sig[0]
        assert abs(sig[0] - sig[3]) < 1e-12
        assert abs(cf.elong_Lambda_e(D, L2) - Lam_e) < 1e-7 * max(1.0, Lam_e)
        T = sig[0] + sig[3] + sig[5] - 3
        assert abs(T - cf.elong_T_from_D(D, Lam_e, L2)) < 1e-7 * max(1.0, T)
        seen_branch.add(D < L2 - 3)
        if Lam_e == 1e-3:
            assert abs(D / Lam_e - 3.0) < 1e-2
        if Lam_e == 20.0:
            assert abs(D / Lam_e / (2 * L2) - 1.0) < 0.08
    assert seen_branch == {True, False}


def test_saos_moduli():
    """Oscillatory shear in the Oldroyd-B limit: S(t)/gamma0 = eta' cos(wt) +
    eta'' sin(wt) after transients, with G'' = w eta' and G' = w eta''
    matching Eq. (modulipred)."""
    taup, L2, g0 = 200.0, 1e12, 1e-5
    for wt in (0.3, 1.0, 3.0):
        w = wt / taup
        C = np.array([1, 0, 0, 1, 0, 1.0])
        R = np.zeros(6)
        hp = False
        ts, Ss = [], []
        nper = int(round(2 * math.pi / w))
        total = 12 * nper + int(10 * taup)
        for n in range(total):
            C, R, hp = oracle.fenep_point(C, _shear_gradu(g0 * math.cos(w * n)), taup, L2, 1, R, hp)
            if n >= total - 2 * nper:
                ts.append(n + 1)
                Ss.append(C[1])
        ts = np.array(ts, dtype=float)
        A = np.stack([np.cos(w * ts), np.sin(w * ts)], 1)
        (a, b), *_ = np.linalg.lstsq(A, np.array(Ss) / g0, rcond=None)
        Gpp, Gp = cf.saos_moduli(w, taup)
        # the explicit update lags the prescribed rate by half a step
        assert abs(w * a / Gpp - 1) < 5e-3 and abs(w * b / Gp - 1) < 5e-3


def test_cessation_relaxation():
    """Shear inception to steady state, then cessation, with the set-up of
    Sec. 3.4 (2 U_w/H = 1e-3, tau_P = 1e4, L^2 = 4.1): T(t) follows
    Eq. (timeunclosed), S/S0 follows Eq. (relax), and the area under S gives
    N0 = 2 gamma_dot integral S dt (Eq. graal).  The residual is the first-order
    start-up error of AB2 across the jump in the rate (~ Delta t / tau_P)."""
    taup, L2, gdot = 1e4, 4.1, 1e-3
    C = np.array([1, 0, 0, 1, 0, 1.0])
    C, R, hp = oracle.fenep_point(C, _shear_gradu(gdot), taup, L2, int(12 * taup))
    f = lambda C: (L2 - 3) / (L2 - (C[0] + C[3] + C[5]))
    sig0 = f(C) * C
    T0, S0, N0 = sig0[0] + sig0[3] + sig0[5] - 3, sig0[1], sig0[0] - sig0[3]
    assert abs(S0 - cf.shear_S(10.0, L2)) < 1e-8 and abs(N0 - cf.shear_N(10.0, L2)) < 1e-7
    area = 0.5 * S0
    zero = np.zeros((3, 3))
    done = 0
    for t_tilde in (0.05, 0.2, 0.5, 1.0):
        while done < int(round(t_tilde * taup)):
            C, R, hp = oracle.fenep_point(C, zero, taup, L2, 1, R, hp)
            area += (f(C) * C)[1]
            done += 1
        sig = f(C) * C
        T = sig[0] + sig[3] + sig[5] - 3
        Tex = cf.cessation_T(T0, L2, t_tilde)
        assert abs(T / Tex - 1) < 1e-3
        assert abs(sig[1] / S0 / cf.cessation_S_ratio(T, T0, L2) - 1) < 1e-6
    # remaining tail of the integral: S decays like exp(-t~ (L^2 - 3)/L^2) once T is small
    for _ in range(int(30 * taup) // 1000):
        for _ in range(1000):
            C, R, hp = oracle.fenep_point(C, zero, taup, L2, 1, R, hp)
            area += (f(C) * C)[1]
    assert abs(N0 - 2 * gdot * area) < 1e-3 * N0


@pytest.mark.slow
def test_couette_fenep_closed_form():
    """FENE-P Couette with feedback (the D2Q9 64x32 set-up, shortened in
    tau_P to keep the CPU run short at the same Lambda = -0.625, L^2 = 100):
    the profile stays linear and C reaches the closed-form steady state
    (Sec. 3.1), including the wall rows (linear-extrapolation ghosts)."""
    ny, U = 16, 0.02
    gdot = 2 * U / ny
    taup = 0.625 / gdot
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=4, ny=ny, eta_A=1 / 6, eta_B=1 / 6, u_wall=U, tau_p=taup,
                      eta_p=1 / 9, L2=100.0)
    o.init_fields(np.ones((1, ny, 4)))
    o.step(int(25 * taup))
    Cex, _ = cf.shear_conformation(-0.625, 100.0)
    C = o.read(oracle.F_C)
    for k, kk in enumerate((0, 1, 3, 5)):
        assert np.max(np.abs(C[k] - Cex[kk])) < 1e-6 * max(1, abs(Cex[kk]))
    u = o.read(oracle.F_U)[0]
    assert np.max(np.abs(u - cf.couette_profile(ny, U)[None, :, None])) < 1e-9
    # the diagnostics of that steady state (Sec. 3.1, Eqs. lindner, lindner2 and N2S)
    _check_couette_diagnostics(o.diagnostics(), 4, ny, U)


def _check_couette_diagnostics(d, nx, ny, U):
    """Diagnostics of a one-component steady FENE-P Couette flow at
    Lambda = tau_P gamma_dot = -0.625, L^2 = 100 (the lower wall moves at +U):
      5  <sigma_P,xy> = -S(0.625, 100)           (shear stress, sign of gamma_dot)
      6  <sigma_P,xx - sigma_P,yy> = N(0.625, 100) (first normal stress difference)
      15 <tr sigma_P> - 3 = N                      (sigma_yy = sigma_zz = 1)
      7  max tr C / L^2 = tr C of the closed form / L^2
      8  max |u| = U (NY - 1) / NY                 (the rows next to the walls)
      0  mass = NX NY; 2-4 momentum = 0 (antisymmetric profile)
      one component, phi = 1 everywhere: the indicator fills the NX x NY
      rectangle, so area 9 = volume 14 = NX NY, the centroid 12, 13 is
      ((NX - 1)/2, (NY - 1)/2), the second moments are (n^2 - 1)/12 and
      theta 11 is pi/2 for the taller side along y, D 10 = (a - b)/(a + b)
      with a, b the square roots of those moments."""
    S, N = cf.shear_S(0.625, 100.0), cf.shear_N(0.625, 100.0)
    Cex, _ = cf.shear_conformation(-0.625, 100.0)
    assert abs(d[5] - (-S)) < 1e-6 * S
    assert abs(d[6] - N) < 1e-6 * N
    assert abs(d[15] - N) < 1e-6 * N
    assert abs(d[7] - (Cex[0] + Cex[3] + Cex[5]) / 100.0) < 1e-8
    assert abs(d[8] - U * (ny - 1) / ny) < 1e-9
    assert abs(d[0] - nx * ny) < 1e-9 and abs(d[1]) == 0.0
    assert np.max(np.abs(d[2:5])) < 1e-10
    assert d[9] == nx * ny and d[14] == nx * ny
    assert abs(d[12] - (nx - 1) / 2) < 1e-12 and abs(d[13] - (ny - 1) / 2) < 1e-12
    ia, ib = math.sqrt((ny * ny - 1) / 12.0), math.sqrt((nx * nx - 1) / 12.0)
    assert abs(d[10] - (ia - ib) / (ia + ib)) < 1e-12
    assert abs(d[11] - math.pi / 2) < 1e-12


def test_couette_diagnostics_signs():
    """The diagnostic pins above catch a transposed or sign-flipped stress
    average: the same Couette flow with the walls reversed (Lambda = +0.625)
    flips <sigma_P,xy> and keeps <N_1> (Eq. N2S: N = 2 S^2 is even in S)."""
    ny, U = 8, 0.02
    gdot = 2 * U / ny
    taup = 0.625 / gdot
    for sign in (+1, -1):
        o = oracle.Oracle(lattice=oracle.D2Q9, nx=2, ny=ny, eta_A=1 / 6, eta_B=1 / 6, u_wall=sign * U, tau_p=taup,
                          eta_p=1 / 9, L2=100.0)
        o.init_fields(np.ones((1, ny, 2)))
        o.step(int(25 * taup))
        d = o.diagnostics()
        S, N = cf.shear_S(0.625, 100.0), cf.shear_N(0.625, 100.0)
        assert abs(d[5] + sign * S) < 1e-6 * S
        assert abs(d[6] - N) < 1e-6 * N and abs(d[15] - N) < 1e-6 * N
        assert abs(d[8] - U * (ny - 1) / ny) < 1e-9


def test_fenep_at_rest_and_symmetry():
    """C = I at rest is an exact fixed point (f(3) = 1); a uniform C relaxes
    with no spatial coupling."""
    o = oracle.Oracle(lattice=oracle.D3Q19, nx=4, ny=5, nz=3, tau_p=10.0, eta_p=0.5, L2=20.0, kappa=0.05)
    o.init_fields(np.ones((3, 5, 4)))
    o.step(5)
    C = o.read(oracle.F_C)
    ident = np.array([1, 0, 0, 1, 0, 1.0])
    assert np.max(np.abs(C - ident[:, None, None, None])) == 0.0


def test_advection_diffusion_mode():
    """A Fourier mode of C advected by a uniform u and diffused by kappa
    evolves by the exact amplification of central differences under
    forward-Euler-then-AB2: eigenvalue lambda = -i U sin(k) - 2 kappa (1 - cos k)
    - f/tau_P for the deviation (Eq. FENE with the artificial diffusivity)."""
    nx, ny = 16, 3
    U, kappa, taup, L2 = 0.05, 0.02, 1e12, 1e12
    k = 2 * math.pi / nx
    x = np.arange(nx)
    eps = 1e-3
    C = np.zeros((4, 1, ny, nx))
    C[0] = C[2] = C[3] = 1.0
    C[1] = eps * np.cos(k * x)[None, None, :]
    u = np.zeros((2, 1, ny, nx))
    u[0] = U
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, walls=0, eta_A=0.1, eta_B=0.1, tau_p=taup, L2=L2,
                      kappa=kappa, eta_p=0.0)
    o.init_fields(np.ones((1, ny, nx)), u=u, C=C)
    nsteps = 50
    o.step(nsteps)
    lam = -1j * U * math.sin(k) - 2 * kappa * (1 - math.cos(k)) - 1.0 / taup
    # AB2 recurrence a_{n+1} = a_n + lam (3/2 a_n - 1/2 a_{n-1}), a_1 = (1 + lam) a_0
    a0, a1 = 1.0 + 0j, 1.0 + lam
    for _ in range(nsteps - 1):
        a0, a1 = a1, a1 + lam * (1.5 * a1 - 0.5 * a0)
    ex = eps * np.real(a1 * np.exp(1j * k * x))
    Cxy = o.read(oracle.F_C)[1, 0, 1, :]
    assert np.allclose(Cxy, ex, atol=1e-12)


def test_deformation_diagnostic_ellipse():
    """D = (a-b)/(a+b) and the orientation angle of Sec. 4.1 for a prescribed
    elliptic droplet in the shear plane."""
    nx, ny = 96, 80
    a, b, th = 22.0, 14.0, math.pi / 5
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xc, yc = x - 47.5, y - 39.5
    xr = xc * math.cos(th) + yc * math.sin(th)
    yr = -xc * math.sin(th) + yc * math.cos(th)
    inside = (xr / a) ** 2 + (yr / b) ** 2 < 1
    rA = np.where(inside, 2.0, 0.1)[None]
    rB = 2.1 - rA
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, ncomp=2, G=0.0)
    o.init_fields(rA, rB)
    d = o.diagnostics()
    assert abs(d[10] - (a - b) / (a + b)) < 0.01
    assert abs(d[11] - th) < 0.01
    assert abs(d[9] - math.pi * a * b) / (math.pi * a * b) < 0.02
    # centroid of the ellipse and, for D2Q9, volume = area of the one plane
    assert abs(d[12] - 47.5) < 0.05 and abs(d[13] - 39.5) < 0.05
    assert d[14] == d[9] == np.count_nonzero(inside)
    # at rest with C = I: no stress, no motion
    assert d[5] == 0.0 and d[6] == 0.0 and d[15] == 0.0 and d[8] == 0.0
    assert abs(d[7] - 3.0 / o.cfg["L2"]) < 1e-15


def test_deformation_diagnostic_sphere_and_angle_range():
    """3-D indicator: a sphere of radius r at an off-centre point gives the
    volume (4/3) pi r^3 (14), the disc of its mid-plane z = NZ/2 (9, the
    plane of Sec. 4.1's D), D = 0 and the centroid of the sphere.  An
    ellipse rotated by -pi/5 returns theta = -pi/5 (11 lies in (-pi/2, pi/2])."""
    nx, ny, nz, r = 40, 36, 32, 9.0
    c = (21.3, 17.0, 16.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 < r * r
    rA = np.where(inside, 2.0, 0.1)
    o = oracle.Oracle(lattice=oracle.D3Q19, nx=nx, ny=ny, nz=nz, ncomp=2, G=0.0)
    o.init_fields(rA, 2.1 - rA)
    d = o.diagnostics()
    assert abs(d[14] - 4.0 / 3.0 * math.pi * r ** 3) / d[14] < 0.02
    assert d[14] == np.count_nonzero(inside) and d[9] == np.count_nonzero(inside[nz // 2])
    assert abs(d[9] - math.pi * r * r) / d[9] < 0.03
    assert d[10] < 0.02
    assert abs(d[12] - c[0]) < 0.1 and abs(d[13] - c[1]) < 1e-9
    nx, ny = 96, 80
    a, b, th = 22.0, 14.0, -math.pi / 5
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xc, yc = x - 47.5, y - 39.5
    xr = xc * math.cos(th) + yc * math.sin(th)
    yr = -xc * math.sin(th) + yc * math.cos(th)
    rA = np.where((xr / a) ** 2 + (yr / b) ** 2 < 1, 2.0, 0.1)[None]
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, ncomp=2, G=0.0)
    o.init_fields(rA, 2.1 - rA)
    d = o.diagnostics()
    assert abs(d[11] - th) < 0.01 and abs(d[10] - (a - b) / (a + b)) < 0.01


def _golden():
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


@pytest.mark.slow
def test_laplace_law_shan_chen():
    """Shan-Chen droplets at G = 1.5, rho_tot = 2.1 (Sec. 4.1): the bulk
    pressure jump P_b = c_s^2 rho + c_s^2 G rho_A rho_B (Eq. PTexpanded) is
    linear in 1/R (2D Laplace law), with a surface tension near the printed
    0.09 and bulk densities near 2.0 / 0.1.  The paper's numbers come from
    3D MRT runs, so the agreement asked for is ~20%, not parity."""
    from paper_1406_2686_gb300 import inputs
    gold = _golden()
    n, G = 64, gold["G_droplet"]
    Rs, dps, inner = [], [], []
    for R in (8, 11, 14, 17):
        rA, rB = inputs.droplet_fields(n, n, 1, R=R, width=5.0, noise=0.0)
        o = oracle.Oracle(lattice=oracle.D2Q9, nx=n, ny=n, ncomp=2, walls=0, G=G, eta_A=0.35, eta_B=0.35, fd_on=0)
        o.init_fields(rA, rB)
        o.step(3000)
        A, B = o.read(oracle.F_RHO_A)[0], o.read(oracle.F_RHO_B)[0]
        c = n // 2
        dps.append(cf.bulk_pressure(A[c, c], B[c, c], G) - cf.bulk_pressure(A[0, 0], B[0, 0], G))
        Rs.append(R)
        inner.append((A[c, c], B[c, c]))
        assert o.status == 0
    Rs, dps = np.array(Rs, float), np.array(dps)
    slope, icpt = np.polyfit(1.0 / Rs, dps, 1)
    fit = slope / Rs + icpt
    assert np.max(np.abs(fit - dps)) < 0.02 * dps.max()
    assert abs(icpt) < 0.1 * dps.min()
    assert abs(slope / gold["sigma_AB_G1.5"] - 1.0) < 0.2
    assert gold["sigma_AB_min"] < slope < gold["sigma_AB_max"]
    for a, b in inner:
        assert abs(a / gold["rho_A_rich_A"] - 1.0) < 0.1
        assert abs(b / gold["rho_A_rich_B"] - 1.0) < 0.2


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("etas,etap,taup", [(0.1, 0.05, 30.0), (0.1, 0.1, 10.0)])
def test_viscoelastic_shear_wave_dispersion(coupling, etas, etap, taup):
    """A small transverse wave in an Oldroyd-B fluid (L^2 -> infinity) decays
    at the slow root s of rho s (1 + tau_P s) + k^2 (eta_s (1 + tau_P s) + eta_P)
    = 0, from the linearised Eqs. NS and FENE (tau_P dS/dt + S = tau_P du_x/dy,
    feedback (eta_P/tau_P) dS/dy).  Holds for the body-force feedback and for
    the equilibrium-stress feedback of Eq. MODEtransformation; the Newtonian
    rate k^2 (eta_s + eta_P) differs by ~1.5 % and is excluded."""
    ny, nx = 64, 2
    k = 2 * math.pi / ny
    y = np.arange(ny)
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=nx, ny=ny, walls=0, eta_A=etas, eta_B=etas, eta_p=etap, tau_p=taup,
                      L2=1e10, coupling=coupling)
    u0 = np.zeros((2, 1, ny, nx))
    u0[0, 0] = 1e-4 * np.sin(k * y)[:, None]
    o.init_fields(np.ones((1, ny, nx)), u=u0)
    ts, amps = [], []
    for t in range(0, 3000, 100):
        if t:
            o.step(100)
        u = o.read(oracle.F_U)[0, 0, :, 0]
        ts.append(t)
        amps.append(np.dot(u, np.sin(k * y)) / np.dot(np.sin(k * y), np.sin(k * y)))
    ts, amps = np.array(ts, float), np.array(amps)
    sel = ts >= 1000
    rate = -np.polyfit(ts[sel], np.log(np.abs(amps[sel])), 1)[0]
    a, b, c = taup, 1 + k * k * etas * taup, k * k * (etas + etap)
    slow = -(-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
    newt = k * k * (etas + etap)
    assert abs(rate / slow - 1) < 4e-3
    assert abs(rate / newt - 1) > 8e-3


@pytest.mark.slow
def test_couette_fenep_equilibrium_coupling():
    """With the polymer stress in the equilibrium (Eq. MODEtransformation)
    the FENE-P Couette flow reaches the same steady-shear closed form."""
    ny, U = 16, 0.02
    gdot = 2 * U / ny
    taup = 0.625 / gdot
    o = oracle.Oracle(lattice=oracle.D2Q9, nx=4, ny=ny, eta_A=1 / 6, eta_B=1 / 6, u_wall=U, tau_p=taup,
                      eta_p=1 / 9, L2=100.0, coupling=1)
    o.init_fields(np.ones((1, ny, 4)))
    o.step(int(25 * taup))
    Cex, _ = cf.shear_conformation(-0.625, 100.0)
    C = o.read(oracle.F_C)
    for k, kk in enumerate((0, 1, 3, 5)):
        assert np.max(np.abs(C[k] - Cex[kk])) < 1e-6 * max(1, abs(Cex[kk]))
    u = o.read(oracle.F_U)[0]
    assert np.max(np.abs(u - cf.couette_profile(ny, U)[None, :, None])) < 1e-9
