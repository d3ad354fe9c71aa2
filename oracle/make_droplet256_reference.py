"""Write the FP64 reference sample of the 256 x 128 x 256 confined droplet.

TEST INFRASTRUCTURE ONLY: runs the oracle (and the seeded input generator),
nothing else, and stores what the storage-precision test compares with.

Set-up (Sec. 4, the confined viscoelastic droplet, scaled to R = 32 so that
2R/H = 0.5 with H = NY = 128): D3Q19, two components, G = 1.5, droplet
densities 2.0 / 0.1 with interface width 5 and phi noise 1e-3 (SplitMix64
seed 1), tau_B = 1 at rho = 2.1 (eta_B = 0.35), eta_A = 0.6 eta_B,
eta_P = 0.4 eta_B in the droplet phase, Ca = 0.1 and De = 1 with
sigma = 0.09, L^2 = 100, kappa = 1e-3.  Initial densities are rounded to FP32
(the library's storage) before the oracle gets them, as in the tests.

The oracle steps 5000 times (about 3 s per step on 8 x86 cores) and the
script stores, in FP64:
  - the plane z = NZ/2 (the shear plane through the droplet centre) and the
    plane y = NY/2 (the mid-gap plane) of rho_A, rho_B, u (3) and C (6);
  - the oracle's 16 diagnostics (D at index 10);
  - the parameters, the seed, the step count and the SHA-256 of oracle.c.

Usage: python oracle/make_droplet256_reference.py [--steps 5000] [--out PATH]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1406_2686_gb300 import inputs  # noqa: E402

DEFAULT_OUT = os.path.join(ROOT, "tests", "golden", "droplet256_fp64_5000.npz")
NX, NY, NZ, R, SEED = 256, 128, 256, 32.0, 1


def droplet_params(nx=NX, ny=NY, nz=NZ, R=R):
    """Parameters of the confined droplet (Sec. 4 set-up, Eq. DeborahOLDROYD for
    tau_P, the capillary number for the wall speed)."""
    etaB = 2.1 / 3.0 * 0.5
    etaA, etaP, sigma = 0.6 * etaB, 0.4 * etaB, 0.09
    gdot = 0.1 * sigma / (R * etaB)
    taup = 1.0 * R * etaB / sigma * etaB / etaP
    return dict(lattice=1, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=etaA, eta_B=etaB,
                u_wall=gdot * ny / 2, tau_p=taup, eta_p=etaP, L2=100.0, kappa=1e-3, phase=1)


def source_sha():
    h = hashlib.sha256()
    for name in ("oracle.c", "oracle.h"):
        with open(os.path.join(HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def planes(o):
    """Mid-z and mid-y planes of rho_A, rho_B, u and C, stacked as
    (11, NY, NX) and (11, NZ, NX): rows rho_A, rho_B, u_x, u_y, u_z, C_xx,
    C_xy, C_xz, C_yy, C_yz, C_zz."""
    rA, rB = o.read(oracle.F_RHO_A), o.read(oracle.F_RHO_B)
    u, C = o.read(oracle.F_U), o.read(oracle.F_C)
    full = np.concatenate([rA[None], rB[None], u, C])
    return full[:, o.nz // 2, :, :].copy(), full[:, :, o.ny // 2, :].copy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--nz", type=int, default=NZ)
    ap.add_argument("--R", type=float, default=R)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    p = droplet_params(a.nx, a.ny, a.nz, a.R)
    sha = source_sha()  # the library loaded below is built from these sources
    nthreads = oracle.set_threads(a.threads)
    o = oracle.Oracle(**p)
    rA, rB = inputs.droplet_fields(a.nx, a.ny, a.nz, R=a.R, seed=SEED, noise=1e-3)
    o.init_fields(inputs.to_f32_exact(rA), inputs.to_f32_exact(rB))
    diag0 = o.diagnostics()
    t0 = time.time()
    done = 0
    while done < a.steps:
        n = min(100, a.steps - done)
        o.step(n)
        done += n
        el = time.time() - t0
        print("step %d  %.1f s  (%.2f s/step, %d threads)" % (done, el, el / done, nthreads), flush=True)
    if o.status != 0:
        raise RuntimeError("oracle guard bits set: %d" % o.status)
    zplane, yplane = planes(o)
    meta = dict(params=p, seed=SEED, steps=a.steps, oracle_sha=sha, threads=nthreads,
                seconds=time.time() - t0, rows=["rhoA", "rhoB", "ux", "uy", "uz", "Cxx", "Cxy", "Cxz", "Cyy",
                                                  "Cyz", "Czz"])
    tmp = a.out + ".tmp.npz"
    np.savez_compressed(tmp, zplane=zplane, yplane=yplane, diag=o.diagnostics(), diag0=diag0,
                        meta=np.array(json.dumps(meta)))
    os.replace(tmp, a.out)
    print("wrote", a.out, json.dumps(meta))


if __name__ == "__main__":
    main()
