"""Learned warm start of confined-droplet runs (no counterpart in the paper).

A 3-D convolutional U-Net (``nn.UNet``; every convolution, gradient and
optimizer step runs in this package's CUDA kernels, the products on the
tcgen05 tensor cores) maps a set-up -- the initial droplet phase field, the
wall-normal coordinate and five scalars (capillary number Ca, Deborah number
De, confinement 2R/H, viscosity ratio lambda, viscoelastic droplet or matrix)
-- to the near-steady fields phi, u and C of the sheared droplet.  Its
training data are steady states the lattice-Boltzmann / FENE-P step itself
produces (Sec. 4 set-ups in a 64^3 box).  A warm run starts the same step
from the predicted fields; the step alone decides the steady state, and the
gain is the time the run needs to get there.

Steady state (the stopping rule of both runs): the deformation D = (a - b) /
(a + b) of the droplet in the shear plane z = N/2, from the second moments of
the smooth indicator w = clip((1 + phi / 0.9) / 2, 0, 1), changes by less than
`tol` over each of several consecutive emulsion times tau_em = R eta_M / sigma.
"""
import math
import time

import numpy as np

from . import inputs, nn, vefd

RHO_IN, RHO_OUT = 2.0, 0.1
RHO_TOT = RHO_IN + RHO_OUT
SIGMA = 0.09             # surface tension at G = 1.5 (Sec. 4.1)
ETA_REF = RHO_TOT / 3.0 * 0.5   # viscosity of tau = 1 at rho = 2.1
L2 = 100.0
KAPPA = 1e-3
N_IN, N_OUT = 8, 16      # network channels (padded to multiples of 8)
N_FIELDS = 10            # phi, u (3), C - I (6)


def _uniform(seed, idx):
    z = inputs.splitmix64(seed, np.asarray(idx, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Setup:
    """One sheared-droplet set-up in an N^3 box, or an nx x ny x nz box when
    dims is given (walls in y; the wall distance H = ny sets R and U).

    Viscoelastic droplet (phase +1): Newtonian matrix eta_B = eta_ref, droplet
    total viscosity lambda eta_B split 60/40 between solvent eta_A and polymer
    eta_P.  Viscoelastic matrix (phase -1): matrix total eta_ref split 60/40
    (eta_B, eta_P), droplet eta_A = lambda eta_ref.  Then with the matrix
    total viscosity eta_M: shear rate Ca sigma / (R eta_M), wall speed
    U = rate N / 2, tau_P = De tau_em eta_M / eta_P, tau_em = R eta_M / sigma."""

    def __init__(self, Ca, De, conf, lam, phase, N=64, dims=None):
        self.Ca, self.De, self.conf, self.lam, self.phase, self.N = Ca, De, conf, lam, int(phase), N
        self.dims = tuple(dims) if dims is not None else (N, N, N)
        H = self.dims[1]
        self.R = conf * H / 2.0
        if self.phase > 0:
            self.eta_B = ETA_REF
            tot = lam * ETA_REF
            self.eta_A, self.eta_P = 0.6 * tot, 0.4 * tot
            self.eta_M = ETA_REF
        else:
            self.eta_B, self.eta_P = 0.6 * ETA_REF, 0.4 * ETA_REF
            self.eta_A = lam * ETA_REF
            self.eta_M = ETA_REF
        self.gdot = Ca * SIGMA / (self.R * self.eta_M)
        self.u_wall = self.gdot * H / 2.0
        self.tau_em = self.R * self.eta_M / SIGMA
        self.tau_p = De * self.tau_em * self.eta_M / self.eta_P

    def scalars(self):
        """The five set-up scalars scaled to about [-1, 1]."""
        return np.array([(self.Ca - 0.175) / 0.125, (math.log(self.De) - math.log(0.632)) / 1.84,
                         (self.conf - 0.475) / 0.125, math.log2(self.lam), float(self.phase)])

    def lattice(self):
        nx, ny, nz = self.dims
        lat = vefd.Lattice(lattice=vefd.D3Q19, nx=nx, ny=ny, nz=nz, ncomp=2, walls=1, G=1.5, eta_A=self.eta_A,
                           eta_B=self.eta_B, delta=0.1)
        lat.set_wall_shear(self.u_wall)
        lat.set_fenep(self.tau_p, self.eta_P, L2, KAPPA, self.phase, 1)
        return lat

    def cold(self, seed=1):
        lat = self.lattice()
        nx, ny, nz = self.dims
        lat.init_droplet((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0, self.R, RHO_IN, RHO_OUT, 5.0, seed, 1e-3)
        return lat


def sample_setups(n, seed=11, umax=0.08, N=64):
    """n set-ups with Ca in [0.05, 0.3], De in [0.1, 4] (log-uniform),
    2R/H in [0.35, 0.6], lambda in [0.5, 2] (log-uniform) and the viscoelastic
    phase, drawn from SplitMix64(seed); draws whose wall speed would exceed
    umax (too high a Mach number in a 64^3 box) are skipped."""
    out, k = [], 0
    while len(out) < n:
        u = _uniform(seed, np.arange(5 * k, 5 * k + 5))
        k += 1
        s = Setup(0.05 + 0.25 * u[0], math.exp(math.log(0.1) + u[1] * math.log(40.0)), 0.35 + 0.25 * u[2],
                  2.0 ** (2.0 * u[3] - 1.0), 1 if u[4] < 0.5 else -1, N)
        if s.u_wall <= umax:
            out.append(s)
    return out


def deformation(phi_plane):
    """D = (a - b)/(a + b) of the smooth indicator in one x-y plane [ny, nx]."""
    w = np.clip(0.5 * (1.0 + phi_plane / 0.9), 0.0, 1.0)
    ny, nx = w.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    ixx = (w * (x - cx) ** 2).sum() / m
    iyy = (w * (y - cy) ** 2).sum() / m
    ixy = (w * (x - cx) * (y - cy)).sum() / m
    tr, det = ixx + iyy, ixx * iyy - ixy * ixy
    disc = math.sqrt(max(0.25 * tr * tr - det, 0.0))
    a, b = math.sqrt(0.5 * tr + disc), math.sqrt(max(0.5 * tr - disc, 0.0))
    return (a - b) / (a + b)


STEP_QUANTUM = 50  # the check interval of the steady rule is a multiple of this


def check_interval(setup):
    """Steps between two checks of the steady rule: the emulsion time, rounded
    to a multiple of STEP_QUANTUM (at least one quantum)."""
    return STEP_QUANTUM * max(1, int(round(setup.tau_em / STEP_QUANTUM)))


def deformation_device(phi_plane):
    """deformation() of a device tensor [ny, nx] (FP64 moments on the device)."""
    import torch
    w = torch.clamp(0.5 * (1.0 + phi_plane.double() / 0.9), 0.0, 1.0)
    ny, nx = w.shape
    y = torch.arange(ny, device=w.device, dtype=torch.float64)[:, None]
    x = torch.arange(nx, device=w.device, dtype=torch.float64)[None, :]
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    ixx = (w * (x - cx) ** 2).sum() / m
    iyy = (w * (y - cy) ** 2).sum() / m
    ixy = (w * (x - cx) * (y - cy)).sum() / m
    tr, det = ixx + iyy, ixx * iyy - ixy * ixy
    disc = torch.sqrt(torch.clamp(0.25 * tr * tr - det, min=0.0))
    a, b = torch.sqrt(0.5 * tr + disc), torch.sqrt(torch.clamp(0.5 * tr - disc, min=0.0))
    return float((a - b) / (a + b))


def run_to_steady(setup, lat, tol=1e-5, max_steps=80000, hold=5):
    """Steps `lat` in chunks of about one emulsion time (check_interval) until
    D has changed by less than tol in each of `hold` consecutive chunks (a
    single quiet chunk can be the turning point of an overshoot).  Returns
    (steps, D, seconds, converged)."""
    import torch
    chunk = check_interval(setup)
    zc = setup.N // 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, d_prev, quiet, converged = 0, None, 0, False
    while steps < max_steps:
        lat.step(chunk)
        steps += chunk
        d = deformation(lat.read(vefd.PHI)[zc])
        quiet = quiet + 1 if (d_prev is not None and abs(d - d_prev) < tol) else 0
        d_prev = d
        if quiet >= hold:
            converged = True
            break
    torch.cuda.synchronize()
    return steps, d, time.perf_counter() - t0, converged


def fields(lat):
    """(phi [N,N,N], u [3,N,N,N], C [6,N,N,N]) of a lattice on the host."""
    return lat.read(vefd.PHI), lat.read(vefd.U), lat.read(vefd.C)


def net_input(setup, phi0):
    """[N, N, N, 8] channels: initial phi, wall-normal coordinate, the five scalars, 0."""
    N = setup.N
    x = np.zeros((N, N, N, N_IN), dtype=np.float32)
    x[..., 0] = phi0
    x[..., 1] = (np.arange(N, dtype=np.float32)[None, :, None] - (N - 1) / 2.0) / (N / 2.0)
    x[..., 2:7] = setup.scalars().astype(np.float32)
    return x


C_SCALE = 2.0  # typical size of C - I at steady state


def net_target(setup, phi0, phi, u, C):
    """[N, N, N, 16]: phi - phi0, u / U_wall, (C - I) / C_SCALE, zero padding."""
    N = setup.N
    t = np.zeros((N, N, N, N_OUT), dtype=np.float32)
    t[..., 0] = phi - phi0
    for k in range(3):
        t[..., 1 + k] = u[k] / setup.u_wall
    eye = (0, 3, 5)
    for k in range(6):
        t[..., 4 + k] = (C[k] - (1.0 if k in eye else 0.0)) / C_SCALE
    return t


def make_dataset(setups, tol=1e-5, max_steps=80000, log=None):
    """Runs every set-up from rest to its steady state; returns the network
    inputs and targets and the cold-run records."""
    X, Y, rec = [], [], []
    for i, s in enumerate(setups):
        lat = s.cold(seed=100 + i)
        phi0 = lat.read(vefd.PHI)
        steps, d, sec, conv = run_to_steady(s, lat, tol, max_steps)
        phi, u, C = fields(lat)
        X.append(net_input(s, phi0))
        Y.append(net_target(s, phi0, phi, u, C))
        rec.append(dict(steps=steps, D=d, seconds=sec, converged=conv))
        if log:
            log("sample %d: Ca %.3f De %.2f 2R/H %.2f lambda %.2f phase %+d -> %d steps, D %.4f%s" %
                (i, s.Ca, s.De, s.conf, s.lam, s.phase, steps, d, "" if conv else " (cap)"))
        lat.close()
    return np.stack(X), np.stack(Y), rec


def make_dataset_ensemble(setups, tol=1e-5, max_steps=80000, group=32, hold=5, seed0=100, log=None):
    """make_dataset with the set-ups stepped together as ensembles of up to
    `group` lattices (vefd.Ensemble: one replayed graph per STEP_QUANTUM steps
    for all of them).  Each member follows the steady rule of run_to_steady on
    its own check interval; converged members (and those at max_steps) leave,
    and the next set-ups join.  Same seeds and the same fields as
    make_dataset up to the floating-point order of the ensemble kernels."""
    import torch
    n = len(setups)
    X, Y = [None] * n, [None] * n
    rec = [None] * n
    pending = list(range(n))
    active = []  # [index, lattice, phi0, steps, d_prev, quiet]
    t0 = time.perf_counter()
    E = None
    while pending or active:
        changed = False
        while pending and len(active) < group:
            i = pending.pop(0)
            lat = setups[i].cold(seed=seed0 + i)
            active.append([i, lat, lat.read(vefd.PHI), 0, None, 0])
            changed = True
        if changed or E is None:
            if E is not None:
                E.close()
            E = vefd.Ensemble([a[1] for a in active])
        E.step(STEP_QUANTUM, chunk=STEP_QUANTUM)
        done = []
        for a in active:
            i, lat = a[0], a[1]
            s = setups[i]
            a[3] += STEP_QUANTUM
            if a[3] % check_interval(s):
                continue
            d = deformation_device(lat.read(vefd.PHI, device=True)[s.dims[2] // 2])
            a[5] = a[5] + 1 if (a[4] is not None and abs(d - a[4]) < tol) else 0
            a[4] = d
            if a[5] >= hold or a[3] >= max_steps:
                phi, u, C = fields(lat)
                X[i] = net_input(s, a[2])
                Y[i] = net_target(s, a[2], phi, u, C)
                rec[i] = dict(steps=a[3], D=d, seconds=None, converged=a[5] >= hold)
                done.append(a)
                if log:
                    log("sample %d: Ca %.3f De %.2f 2R/H %.2f lambda %.2f phase %+d -> %d steps, D %.4f%s" %
                        (i, s.Ca, s.De, s.conf, s.lam, s.phase, a[3], d, "" if a[5] >= hold else " (cap)"))
        if done:
            E.close()
            E = None
            for a in done:
                active.remove(a)
                a[1].close()
    if E is not None:
        E.close()
    torch.cuda.synchronize()
    if log:
        log("ensemble dataset: %d set-ups in %.1f s" % (n, time.perf_counter() - t0))
    return np.stack(X), np.stack(Y), rec


def train(net, X, Y, epochs=30, lr=1e-3, seed=0, log=None, warmup=1):
    """Adam on the mean squared error of the normalised targets, one sample per
    step, the learning rate decaying geometrically to lr / 10 over the epochs;
    over the first `warmup` epochs it also ramps linearly from lr / 10, so that
    the first steps at full rate cannot switch off whole layers of units."""
    import torch
    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    rng = np.random.default_rng(seed)
    losses = []
    k = 0
    for ep in range(epochs):
        tot = torch.zeros(8, device="cuda")
        lr_ep = lr * 0.1 ** (ep / max(1, epochs - 1))
        for i in rng.permutation(n):
            ramp = min(1.0, 0.1 + 0.9 * k / max(1, warmup * n)) if warmup > 0 else 1.0
            k += 1
            out = net.forward(Xd[i:i + 1].contiguous())
            parts, grad = nn.mse(out, Yd[i:i + 1].contiguous())
            net.backward(grad)
            net.adam_step(lr=lr_ep * ramp)
            tot += parts
        losses.append(float(tot.sum()) / (n * Y[0].size))
        if log and (ep % 5 == 4 or ep == epochs - 1):
            log("epoch %d: loss %.4e" % (ep + 1, losses[-1]))
    return losses


def warm_lattice(net, setup, phi0_dev, blend=1.0):
    """A lattice started from the network's prediction, built on the device:
    input assembly (host, cheap), network, field conversion, init_fields.
    The predicted increments over the cold start (phi - phi0, u, C - I) are
    scaled by `blend` (1: the prediction, 0: the cold start).  Each
    component's density field is rescaled to the set-up's mass (that of the
    initial droplet): the step conserves the masses, so they, not the
    prediction, decide the droplet size."""
    import torch
    phi0 = phi0_dev.cpu().numpy()
    x = torch.from_numpy(net_input(setup, phi0)[None]).cuda().contiguous()
    out = net.forward(x)[0]
    if blend != 1.0:
        nn.scale(out, blend)
    rA, rB, u, C = nn.to_fields(out, phi0_dev, setup.u_wall, C_SCALE, RHO_TOT, L2)
    mA = 0.5 * RHO_TOT * float(np.sum(1.0 + phi0.astype(np.float64)))
    mB = 0.5 * RHO_TOT * float(np.sum(1.0 - phi0.astype(np.float64)))
    nn.scale(rA, mA / nn.total(rA))
    nn.scale(rB, mB / nn.total(rB))
    lat = setup.lattice()
    lat.init_fields(rA, rB, u, C)
    return lat


def evaluate(net, setups, tol=1e-5, max_steps=80000, log=None, blend=1.0):
    """Cold and warm runs of every set-up to steady state; per set-up the
    steps, seconds (warm: including the network prediction) and D of both
    (`blend` as in warm_lattice)."""
    import torch
    res = []
    for i, s in enumerate(setups):
        cold = s.cold(seed=500 + i)
        phi0 = cold.read(vefd.PHI, device=True).clone()
        c_steps, c_d, c_sec, c_conv = run_to_steady(s, cold, tol, max_steps)
        cold.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        warm = warm_lattice(net, s, phi0, blend)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        w_steps, w_d, w_sec, w_conv = run_to_steady(s, warm, tol, max_steps)
        warm.close()
        r = dict(cold_steps=c_steps, cold_seconds=c_sec, cold_D=c_d, cold_converged=c_conv, warm_steps=w_steps,
                 warm_seconds=w_sec + t_pred, predict_seconds=t_pred, warm_D=w_d, warm_converged=w_conv,
                 D_rel_err=abs(w_d - c_d) / max(abs(c_d), 1e-12))
        res.append(r)
        if log:
            log("eval %d (Ca %.3f De %.2f 2R/H %.2f lambda %.2f phase %+d): cold %d steps %.2fs D %.4f | "
                "warm %d steps %.2fs D %.4f | dD/D %.2e" % (i, s.Ca, s.De, s.conf, s.lam, s.phase, c_steps, c_sec, c_d,
                                                           w_steps, r["warm_seconds"], w_d, r["D_rel_err"]))
    return res
