"""The closed forms used as pins, checked against the equations they solve."""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf


@pytest.mark.parametrize("Lam,L2", [(0.625, 100.0), (1e-3, 100.0), (50.0, 1e4), (10.0, 4.1)])
def test_lindner_solves_cubic(Lam, L2):
    """Eq. (lindner) is the real root of Eq. (cubic); Eq. (lindner2) is 2 S^2
    (Eq. N2S); and (S, N) satisfy the system Eq. (EQNS)."""
    S, N = cf.shear_S(Lam, L2), cf.shear_N(Lam, L2)
    assert abs(2 * S ** 3 / L2 + S - Lam) < 1e-12 * max(1, Lam)
    assert abs(N - 2 * S * S) < 1e-12 * max(1, N)
    assert abs((1 + N / L2) * N - 2 * Lam * S) < 1e-10 * max(1, N)
    assert abs((1 + N / L2) * S - Lam) < 1e-12 * max(1, Lam)


def test_config1_values():
    """D2Q9 Couette set-up: H = 32, U_w = 0.01, tau_P = 1000 -> Lambda = 0.625, L^2 = 100."""
    S, N = cf.shear_S(0.625, 100.0), cf.shear_N(0.625, 100.0)
    assert abs(S - 0.620228175) < 2e-9 and abs(N - 0.769365979) < 2e-9
    C, Z = cf.shear_conformation(0.625, 100.0)
    assert abs(Z - 1.007693660) < 2e-9
    assert abs(C[1] - 0.615492783) < 2e-9 and abs(C[0] - 1.755857013) < 2e-9 and abs(C[3] - 0.992365081) < 2e-9


@pytest.mark.parametrize("L2", [10.0, 100.0, 1e4])
def test_elongation_quadratic(L2):
    """Eq. (el8) roots satisfy the quadratic Eq. (el7) and, with T from the
    first equation of the system, the second equation too; D/Lambda_e -> 3
    for small D (Eq. dimensionalelong)."""
    for D in (1e-3, 0.5, 0.5 * (L2 - 3), 2 * L2, 30 * L2):
        Le = cf.elong_Lambda_e(D, L2)
        P1, P2, P3 = cf.elong_P(D, L2)
        assert abs(P1 * Le * Le + P2 * Le + P3) < 1e-9 * max(1, abs(P3), abs(P2 * Le))
        T = cf.elong_T_from_D(D, Le, L2)
        assert abs(-(L2 + T) / L2 * D + Le * (D + T) + 3 * Le) < 1e-8 * max(1, D)
    assert abs(1e-3 / cf.elong_Lambda_e(1e-3, L2) - 3.0) < 1e-2
    D = cf.elong_D(0.3, L2)
    assert abs(cf.elong_Lambda_e(D, L2) - 0.3) < 1e-10


def test_saos_limits():
    """G'' -> w tau, G' -> (w tau)^2 at small w tau; G' -> 1, G'' -> 0 at large."""
    Gpp, Gp = cf.saos_moduli(1e-4, 10.0)
    assert abs(Gpp / 1e-3 - 1) < 1e-5 and abs(Gp / 1e-6 - 1) < 1e-5
    Gpp, Gp = cf.saos_moduli(1e3, 10.0)
    assert abs(Gp - 1) < 1e-7 and Gpp < 1e-3


def test_cessation_oldroyd_limit():
    """Eq. (timeunclosed) reduces to T0 exp(-t~) for L^2 >> 1, and Eq. (relax) to
    S/S0 = T/T0."""
    assert abs(cf.cessation_T(2.0, 1e9, 1.0, nsub=2000) / (2 * math.exp(-1)) - 1) < 1e-7
    assert abs(cf.cessation_S_ratio(0.5, 2.0, 1e12) - 0.25) < 1e-9


def test_taylor_and_confinement():
    """Taylor's law at lambda = 1 is 35/32 Ca; the confinement correction uses
    C_sh = 5.6996 at mid-gap (Sec. 4.1)."""
    assert abs(cf.taylor_D(0.1, 1.0) - 0.109375) < 1e-12
    ex = 0.109375 * (1 + 5.6996 * 3.5 / 2 * 0.25 ** 3)
    assert abs(cf.shapira_haber_D(0.1, 1.0, 0.25) - ex) < 1e-12


def test_couette_profile_walls():
    u = cf.couette_profile(4, 1.0)
    # half-way walls at -1/2 (velocity +1) and 3.5 (velocity -1): linear through the nodes
    assert np.allclose(u, [0.75, 0.25, -0.25, -0.75])
