"""Analytic results of Gupta, Sbragaglia & Scagliarini that pin the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Every function below
restates one closed form of the paper (or a textbook lattice-Boltzmann result
named in its docstring); none of them calls the oracle.

Notation follows the paper: Lambda = tau_P * shear rate, S = sigma_P,xy,
N = sigma_P,xx - 1, T = tr sigma_P - 3, D = sigma_P,zz - sigma_P,xx,
Lambda_e = tau_P * elongation rate, sigma_P = f(r_P) C.
"""
import math

import numpy as np

CS2 = 1.0 / 3.0


# --- steady shear (Sec. 3.1) ---------------------------------------------

def shear_S(Lam, L2):
    """Polymer shear stress S(Lambda, L), Eq. (lindner): the real root of the
    cubic 2 S^3 / L^2 + S - Lambda = 0 (Eq. cubic)."""
    a = L2 / 6.0
    return 2.0 * math.sqrt(a) * math.sinh(math.asinh(Lam * L2 / 4.0 * a ** -1.5) / 3.0)


def shear_N(Lam, L2):
    """First normal stress difference N(Lambda, L), Eq. (lindner2); N = 2 S^2 (Eq. N2S)."""
    a = L2 / 6.0
    return 8.0 * a * math.sinh(math.asinh(Lam * L2 / 4.0 * a ** -1.5) / 3.0) ** 2


def shear_conformation(Lam, L2):
    """Steady conformation tensor for u_x = gamma_dot * y (Sec. 3.1):
    sigma_P,yy = sigma_P,zz = 1, sigma_P,xx = 1 + N, sigma_P,xy = S, and
    C = sigma_P / Z with Z = (L^2 - 3 + tr sigma_P) / L^2 (Eq. FENErevised).
    Returns (C in order xx xy xz yy yz zz, Z).  Lambda may be negative
    (the shear stress takes the sign of the shear rate)."""
    S = math.copysign(shear_S(abs(Lam), L2), Lam)
    N = shear_N(abs(Lam), L2)
    sig = np.array([1.0 + N, S, 0.0, 1.0, 0.0, 1.0])
    Z = (L2 - 3.0 + sig[0] + sig[3] + sig[5]) / L2
    return sig / Z, Z


# --- steady elongation (Sec. 3.2) ----------------------------------------

def elong_P(D, L2):
    """Coefficients P1, P2, P3 of the quadratic in Lambda_e, Eq. (el9)."""
    P1 = 2.0 * D * L2
    P2 = -4.0 * D * D + (L2 - D - 3.0) * (D + 3.0)
    P3 = 2.0 * D ** 3 / L2 - (L2 - D - 3.0) * D
    return P1, P2, P3


def elong_Lambda_e(D, L2):
    """Dimensionless elongation rate for a given D, Eq. (el8), taking the
    (+) root below the branch point D = L^2 - 3 and the (-) root above it."""
    P1, P2, P3 = elong_P(D, L2)
    disc = max(P2 * P2 - 4.0 * P1 * P3, 0.0)
    sign = 1.0 if D < L2 - 3.0 else -1.0
    return (-P2 + sign * math.sqrt(disc)) / (2.0 * P1)


def elong_D(Lam_e, L2):
    """Invert Eq. (el8) for D by bisection on the monotone branch."""
    lo, hi = 0.0, 1.0
    while elong_Lambda_e(hi, L2) < Lam_e:
        hi *= 2.0
        if hi > 1e12:
            raise ValueError("no root")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid == 0.0 or elong_Lambda_e(mid, L2) < Lam_e:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def elong_T_from_D(D, Lam_e, L2):
    """T from the first equation of the elongation system (Sec. 3.2):
    (L^2 + T) T / L^2 = 2 Lambda_e D, the positive root."""
    # T^2 + L^2 T - 2 Lambda_e D L^2 = 0
    return 0.5 * (-L2 + math.sqrt(L2 * L2 + 8.0 * Lam_e * D * L2))


# --- small-amplitude oscillatory shear (Sec. 3.3) ------------------------

def saos_moduli(omega, tau_p):
    """Dimensionless loss and storage moduli (G'', G'), Eq. (modulipred),
    reading the garbled exponent as (omega tau_P)^2."""
    wt = omega * tau_p
    return wt / (1.0 + wt * wt), wt * wt / (1.0 + wt * wt)


# --- cessation of steady shear (Sec. 3.4) --------------------------------

def cessation_T(T0, L2, t_tilde, nsub=20000):
    """T(t~) after cessation from RK4 integration of Eq. (timeunclosed),
    dT/dt~ = T (L^2 + T)^2 / (L^2 (3 - L^2)); t~ = (t - t0)/tau_P."""
    def rhs(T):
        return T * (L2 + T) ** 2 / (L2 * (3.0 - L2))
    T = float(T0)
    if t_tilde <= 0:
        return T
    h = t_tilde / nsub
    for _ in range(nsub):
        k1 = rhs(T)
        k2 = rhs(T + 0.5 * h * k1)
        k3 = rhs(T + 0.5 * h * k2)
        k4 = rhs(T + h * k3)
        T += h * (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
    return T


def cessation_S_ratio(T, T0, L2):
    """S(t)/S_0 as a function of T(t), Eq. (relax)."""
    e = (L2 - 3.0) / L2
    return (T / T0) ** e * ((L2 + T) / (L2 + T0)) ** (1.0 - e)


# --- droplet deformation (Sec. 4.1) --------------------------------------

def taylor_D(Ca, lam):
    """Taylor's small-deformation result, Eq. (deformation)."""
    return (19.0 * lam + 16.0) / (16.0 * lam + 16.0) * Ca


def shapira_haber_D(Ca, lam, R_over_H, Csh=5.6996):
    """Confinement-corrected deformation of Shapira & Haber (Sec. 4.1), with
    the mid-gap coefficient C_sh = 5.6996 the paper quotes."""
    return taylor_D(Ca, lam) * (1.0 + Csh * (2.5 * lam + 1.0) / (lam + 1.0) * R_over_H ** 3)


# --- Shan-Chen bulk pressure (Sec. 2) -------------------------------------

def bulk_pressure(rhoA, rhoB, G):
    """P_b = c_s^2 (rho_A + rho_B) + c_s^2 G rho_A rho_B, from Eq. (PTexpanded)."""
    return CS2 * (rhoA + rhoB) + CS2 * G * rhoA * rhoB


# --- textbook lattice-Boltzmann channel flows ----------------------------

def couette_profile(ny, u_wall):
    """Plane Couette flow between half-way walls at y = -1/2 (velocity +U)
    and y = NY - 1/2 (velocity -U): u_x(y) = U (NY - 1 - 2 y) / NY."""
    y = np.arange(ny, dtype=np.float64)
    return u_wall * (ny - 1 - 2 * y) / ny


def poiseuille_profile(ny, F, eta):
    """Body-force driven channel flow between walls at y = -1/2 and
    y = NY - 1/2: u_x(y) = F / (2 eta) (y + 1/2)(NY - 1/2 - y)."""
    y = np.arange(ny, dtype=np.float64)
    return F / (2.0 * eta) * (y + 0.5) * (ny - 0.5 - y)


def shear_wave_rate(tau, k):
    """Continuum decay rate nu k^2 of a transverse shear wave, nu = c_s^2 (tau - 1/2)
    (Eq. TRANSPORTCOEFF with eta = rho nu)."""
    return CS2 * (tau - 0.5) * k * k
