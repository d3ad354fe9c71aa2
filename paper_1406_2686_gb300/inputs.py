"""Seeded synthetic inputs shared by the CUDA path and the oracle.

Holds none of the method's arithmetic: only initial density/velocity/
conformation fields.  Random numbers come from SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
evaluated counter-style: draw i of stream `seed` is mix(seed + (i+1)*gamma).
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, index):
    """SplitMix64 output for counters `index` (uint64 array) of stream `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed, n):
    """n uniform draws in [-1, 1) with 53-bit resolution."""
    u = (splitmix64(seed, np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    return u * (2.0 ** -52) - 1.0


def droplet_fields(nx, ny, nz, R, rho_in=2.0, rho_out=0.1, width=5.0, center=None, seed=1,
                   noise=1e-3):
    """Two-component droplet initial densities (rho_A, rho_B), shape (nz, ny, nx).

    rho_A = rho_out + (rho_in - rho_out) (1 + tanh(2 (R - r) / width)) / 2,
    rho_B mirrored so that rho_A + rho_B = rho_in + rho_out, plus an order-
    parameter perturbation phi += noise * U[-1, 1) per node at fixed total
    density.  Distances are measured from `center` (default: box centre,
    (n-1)/2 per axis; for nz == 1 the z-offset is zero)."""
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    rA = rho_out + (rho_in - rho_out) * 0.5 * (1.0 + np.tanh(2.0 * (R - r) / width))
    tot = rho_in + rho_out
    rB = tot - rA
    if noise:
        dphi = noise * uniform_pm1(seed, nx * ny * nz).reshape(nz, ny, nx)
        rA = rA + 0.5 * tot * dphi
        rB = rB - 0.5 * tot * dphi
    return rA, rB


def random_state(nx, ny, nz, ndim, ncomp, nc, seed=1, rho0=(1.0, 1.0), drho=0.05, uamp=0.02,
                 camp=0.2):
    """Generic smooth-plus-noise state for stage-wise parity: per-component
    densities rho0[s] (1 + drho U), velocity uamp U per component, and an SPD
    conformation tensor C = I + camp * sym(noise) (diagonal kept > 1 - camp).
    Returns (rhoA, rhoB or None, u (ndim, nz, ny, nx), C (nc, nz, ny, nx))."""
    n = nx * ny * nz
    shp = (nz, ny, nx)
    k = 0

    def draw():
        nonlocal k
        k += 1
        return uniform_pm1(seed * 1000003 + k, n).reshape(shp)

    rA = rho0[0] * (1.0 + drho * draw())
    rB = rho0[1] * (1.0 + drho * draw()) if ncomp == 2 else None
    u = np.stack([uamp * draw() for _ in range(ndim)])
    if nc == 6:
        comps = ["xx", "xy", "xz", "yy", "yz", "zz"]
    else:
        comps = ["xx", "xy", "yy", "zz"]
    C = []
    for name in comps:
        if name[0] == name[1]:
            C.append(1.0 + 0.5 * camp * (1.0 + draw()))
        else:
            C.append(0.25 * camp * draw())
    return rA, rB, u, np.stack(C)


def to_f32_exact(a):
    """Round to FP32 and return as FP64, so both sides start from the same values."""
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)
