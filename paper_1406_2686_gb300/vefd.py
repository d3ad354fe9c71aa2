"""Thin ctypes binding of libvefd (C-ABI in ``include/vefd.h``).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libvefd.so``.  The module-level functions carry the C names;
``Lattice`` is a convenience wrapper that keeps its device memory in a torch
tensor and runs on torch's current CUDA stream.  There is no CPU fallback:
if the library or a GPU is missing, calls raise.
"""
import ctypes
import os

import numpy as np

from . import build_lib

D2Q9, D3Q19 = 0, 1
FP32, FP16, BF16 = 0, 1, 2
RHO_A, RHO_B, PHI, U, C, SIGMA_P, POPS, RPREV, G_A, G_B, F_P, TAU = range(12)
OK, ERR_ARG, ERR_CUDA, ERR_UNSTABLE, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5
ST_NAN, ST_TRACE, ST_MACH, ST_RHO, ST_TIMEOUT, ST_BOUNDS = 1, 2, 4, 8, 16, 32


class VefdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("vefd status %d: %s" % (status, msg))
        self.status = status


class vefd_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("ncomp", ctypes.c_int), ("walls", ctypes.c_int),
        ("G", ctypes.c_double), ("eta_A", ctypes.c_double), ("eta_B", ctypes.c_double),
        ("delta", ctypes.c_double), ("external_memory", ctypes.c_int), ("precision", ctypes.c_int),
    ]


EXPORTS = [
    "vefd_create", "vefd_required_bytes", "vefd_bind_device_memory", "vefd_destroy", "vefd_set_stream",
    "vefd_set_wall_shear", "vefd_set_body_force", "vefd_set_fenep", "vefd_init_fields", "vefd_init_droplet",
    "vefd_write_field", "vefd_step", "vefd_read_field", "vefd_field_bytes", "vefd_diagnostics",
    "vefd_get_status", "vefd_clear_status", "vefd_steps_done", "vefd_checkpoint", "vefd_restore",
    "vefd_last_error", "vefd_kernels_per_step", "vefd_profile_kernels", "vefd_kernel_times",
    "vefd_diagnostics_noalloc", "vefd_set_polymer_coupling", "vefd_set_kernel_config", "vefd_get_kernel_config",
    "vefd_autotune", "vefd_ensemble_create", "vefd_ensemble_step", "vefd_ensemble_last_error",
    "vefd_ensemble_destroy", "vefd_wait_selftest", "vefd_ensemble_set_batched", "vefd_ensemble_set_config",
    "vefd_ensemble_get_config", "vefd_ensemble_autotune", "vefd_set_step_graph", "vefd_get_step_graph",
    "vefd_prepare_step_graph", "vefd_ensemble_is_batched", "vefd_set_collision", "vefd_set_conformation_update",
    "vefd_prepare_steps", "vefd_ensemble_set_groups", "vefd_ensemble_get_groups", "vefd_ensemble_set_tile",
    "vefd_ensemble_get_tile",
]

_lib = None


def library_path():
    return build_lib.LIB


def load(build_if_missing=True):
    """Load libvefd.so (building it in-tree when absent and nvcc is present).
    With VEFD_DEBUG_LIB=1 in the environment the bounds-checked debug library
    is loaded instead (guard bit ST_BOUNDS)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("VEFD_DEBUG_LIB") == "1"
    path = build_lib.LIB_DEBUG if debug else build_lib.LIB
    if not os.path.exists(path) or not build_lib.up_to_date(debug):
        if not build_if_missing:
            raise OSError("libvefd.so is not built: run __graft_entry__.build()")
        build_lib.build(debug=debug)
    L = ctypes.CDLL(path)
    vp, sz, i64, dbl, cint = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    pcfg = ctypes.POINTER(vefd_config)
    sigs = {
        "vefd_create": [pcfg, vp, ctypes.POINTER(vp)],
        "vefd_required_bytes": [pcfg, ctypes.POINTER(sz)],
        "vefd_bind_device_memory": [vp, vp, sz],
        "vefd_set_stream": [vp, vp],
        "vefd_set_wall_shear": [vp, dbl],
        "vefd_set_body_force": [vp, dbl, dbl, dbl],
        "vefd_set_fenep": [vp, dbl, dbl, dbl, dbl, cint, cint],
        "vefd_init_fields": [vp, vp, vp, vp, vp, cint],
        "vefd_init_droplet": [vp, dbl, dbl, dbl, dbl, dbl, dbl, dbl, ctypes.c_uint64, dbl],
        "vefd_write_field": [vp, cint, vp, sz, cint],
        "vefd_step": [vp, i64],
        "vefd_read_field": [vp, cint, vp, sz, cint],
        "vefd_field_bytes": [vp, cint, ctypes.POINTER(sz)],
        "vefd_diagnostics": [vp, ctypes.POINTER(dbl)],
        "vefd_get_status": [vp, ctypes.POINTER(ctypes.c_uint32)],
        "vefd_clear_status": [vp],
        "vefd_steps_done": [vp, ctypes.POINTER(i64)],
        "vefd_checkpoint": [vp, ctypes.c_char_p],
        "vefd_restore": [vp, ctypes.c_char_p],
        "vefd_kernels_per_step": [vp, ctypes.POINTER(cint)],
        "vefd_profile_kernels": [vp, cint],
        "vefd_kernel_times": [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)],
        "vefd_diagnostics_noalloc": [cint, cint, cint, cint, cint, dbl, vp, vp, vp, vp, vp, ctypes.POINTER(dbl)],
        "vefd_set_polymer_coupling": [vp, cint],
        "vefd_set_kernel_config": [vp, cint, cint],
        "vefd_set_collision": [vp, cint],
        "vefd_set_conformation_update": [vp, cint],
        "vefd_get_kernel_config": [vp, ctypes.POINTER(cint), ctypes.POINTER(cint)],
        "vefd_autotune": [vp, cint, ctypes.POINTER(dbl)],
        "vefd_ensemble_create": [ctypes.POINTER(vp), cint, vp, ctypes.POINTER(vp)],
        "vefd_ensemble_step": [vp, i64, i64],
        "vefd_ensemble_set_batched": [vp, cint],
        "vefd_wait_selftest": [vp, cint],
        "vefd_ensemble_set_config": [vp, cint, cint],
        "vefd_ensemble_get_config": [vp, ctypes.POINTER(cint), ctypes.POINTER(cint)],
        "vefd_ensemble_autotune": [vp, i64, i64, ctypes.POINTER(dbl)],
        "vefd_set_step_graph": [vp, cint, cint],
        "vefd_prepare_step_graph": [vp],
        "vefd_prepare_steps": [vp, i64],
        "vefd_ensemble_set_groups": [vp, cint],
        "vefd_ensemble_set_tile": [vp, cint],
        "vefd_ensemble_get_tile": [vp, ctypes.POINTER(cint)],
        "vefd_ensemble_get_groups": [vp, ctypes.POINTER(cint)],
        "vefd_get_step_graph": [vp, ctypes.POINTER(cint), ctypes.POINTER(cint), ctypes.POINTER(cint)],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = cint
    L.vefd_destroy.argtypes = [vp]
    L.vefd_destroy.restype = None
    L.vefd_last_error.argtypes = [vp]
    L.vefd_last_error.restype = ctypes.c_char_p
    L.vefd_ensemble_is_batched.argtypes = [vp]
    L.vefd_ensemble_is_batched.restype = cint
    L.vefd_ensemble_destroy.argtypes = [vp]
    L.vefd_ensemble_destroy.restype = None
    L.vefd_ensemble_last_error.argtypes = [vp]
    L.vefd_ensemble_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


# --- C names, argument marshalling only ------------------------------------

def _check(ctx, st):
    if st != OK:
        msg = load().vefd_last_error(ctx) if ctx else b""
        raise VefdError(st, (msg or b"").decode())
    return st


def vefd_required_bytes(cfg):
    n = ctypes.c_size_t()
    _check(None, load().vefd_required_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def vefd_create(cfg, stream=0):
    h = ctypes.c_void_p()
    _check(None, load().vefd_create(ctypes.byref(cfg), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def vefd_bind_device_memory(ctx, ptr, nbytes):
    return _check(ctx, load().vefd_bind_device_memory(ctx, ctypes.c_void_p(ptr), nbytes))


def vefd_destroy(ctx):
    load().vefd_destroy(ctx)


def vefd_set_stream(ctx, stream):
    return _check(ctx, load().vefd_set_stream(ctx, ctypes.c_void_p(stream)))


def vefd_set_wall_shear(ctx, u_wall):
    return _check(ctx, load().vefd_set_wall_shear(ctx, float(u_wall)))


def vefd_set_body_force(ctx, fx, fy, fz):
    return _check(ctx, load().vefd_set_body_force(ctx, float(fx), float(fy), float(fz)))


def vefd_set_fenep(ctx, tau_p, eta_p, L2, kappa, phase, fd_on=1):
    return _check(ctx, load().vefd_set_fenep(ctx, float(tau_p), float(eta_p), float(L2), float(kappa), int(phase),
                                             int(fd_on)))


def vefd_set_polymer_coupling(ctx, mode):
    return _check(ctx, load().vefd_set_polymer_coupling(ctx, int(mode)))


def vefd_init_fields(ctx, rhoA, rhoB, u, C0, on_device):
    return _check(ctx, load().vefd_init_fields(ctx, rhoA, rhoB, u, C0, int(on_device)))


def vefd_init_droplet(ctx, cx, cy, cz, R, rho_in, rho_out, width, seed, phi_amp):
    return _check(ctx, load().vefd_init_droplet(ctx, cx, cy, cz, R, rho_in, rho_out, width, seed, phi_amp))


def vefd_write_field(ctx, field, src, nbytes, on_device):
    return _check(ctx, load().vefd_write_field(ctx, int(field), ctypes.c_void_p(src), nbytes, int(on_device)))


def vefd_step(ctx, nsteps):
    return _check(ctx, load().vefd_step(ctx, int(nsteps)))


def vefd_read_field(ctx, field, dst, nbytes, on_device):
    return _check(ctx, load().vefd_read_field(ctx, int(field), ctypes.c_void_p(dst), nbytes, int(on_device)))


def vefd_field_bytes(ctx, field):
    n = ctypes.c_size_t()
    _check(ctx, load().vefd_field_bytes(ctx, int(field), ctypes.byref(n)))
    return n.value


def vefd_diagnostics(ctx):
    out = (ctypes.c_double * 16)()
    _check(ctx, load().vefd_diagnostics(ctx, out))
    return np.array(out[:], dtype=np.float64)


def vefd_get_status(ctx):
    """Returns the guard bits (0 when stable); never raises on instability."""
    bits = ctypes.c_uint32()
    st = load().vefd_get_status(ctx, ctypes.byref(bits))
    if st not in (OK, ERR_UNSTABLE, ERR_TIMEOUT):
        _check(ctx, st)
    return int(bits.value)


def vefd_set_step_graph(ctx, slabs, chunk=256):
    return _check(ctx, load().vefd_set_step_graph(ctx, int(slabs), int(chunk)))


def vefd_prepare_step_graph(ctx):
    return _check(ctx, load().vefd_prepare_step_graph(ctx))


def vefd_prepare_steps(ctx, nsteps):
    return _check(ctx, load().vefd_prepare_steps(ctx, int(nsteps)))


def vefd_get_step_graph(ctx):
    s, c, a = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().vefd_get_step_graph(ctx, ctypes.byref(s), ctypes.byref(c), ctypes.byref(a)))
    return s.value, c.value, bool(a.value)


def vefd_wait_selftest(ctx, arrive):
    return _check(ctx, load().vefd_wait_selftest(ctx, int(arrive)))


def vefd_clear_status(ctx):
    return _check(ctx, load().vefd_clear_status(ctx))


def vefd_steps_done(ctx):
    n = ctypes.c_int64()
    _check(ctx, load().vefd_steps_done(ctx, ctypes.byref(n)))
    return n.value


def vefd_checkpoint(ctx, path):
    return _check(ctx, load().vefd_checkpoint(ctx, os.fsencode(path)))


def vefd_restore(ctx, path):
    return _check(ctx, load().vefd_restore(ctx, os.fsencode(path)))


def vefd_last_error(ctx):
    return (load().vefd_last_error(ctx) or b"").decode()


def vefd_kernels_per_step(ctx):
    n = ctypes.c_int()
    _check(ctx, load().vefd_kernels_per_step(ctx, ctypes.byref(n)))
    return n.value


def vefd_profile_kernels(ctx, on):
    return _check(ctx, load().vefd_profile_kernels(ctx, int(on)))


def vefd_kernel_times(ctx):
    """(ms[3], launches[3]) per kernel class: moments, lattice, FENE-P."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(ctx, load().vefd_kernel_times(ctx, ms, n))
    return list(ms), list(n)


def vefd_diagnostics_noalloc(lattice, nx, ny, nz, ncomp, L2, rho_A, rho_B, u, C, stream=0):
    """Allocation-free diagnostics of device fields (pointers as ints)."""
    out = (ctypes.c_double * 16)()
    st = load().vefd_diagnostics_noalloc(int(lattice), int(nx), int(ny), int(nz), int(ncomp), float(L2),
                                         ctypes.c_void_p(rho_A), ctypes.c_void_p(rho_B) if rho_B else None,
                                         ctypes.c_void_p(u), ctypes.c_void_p(C), ctypes.c_void_p(stream), out)
    _check(None, st)
    return np.array(out[:], dtype=np.float64)


def vefd_set_collision(ctx, model):
    return _check(ctx, load().vefd_set_collision(ctx, int(model)))


def vefd_set_conformation_update(ctx, scheme):
    return _check(ctx, load().vefd_set_conformation_update(ctx, int(scheme)))


def vefd_set_kernel_config(ctx, lattice_tile, post_mode):
    return _check(ctx, load().vefd_set_kernel_config(ctx, int(lattice_tile), int(post_mode)))


def vefd_get_kernel_config(ctx):
    """(lattice_tile, post_mode) in effect; -1 means the unstaged kernels."""
    t, m = ctypes.c_int(), ctypes.c_int()
    _check(ctx, load().vefd_get_kernel_config(ctx, ctypes.byref(t), ctypes.byref(m)))
    return t.value, m.value


def vefd_autotune(ctx, steps):
    """Times the admitted kernel choices and applies the fastest; returns the
    eighteen times in ms (index post_mode * 6 + lattice_tile, -1 when not admitted)."""
    out = (ctypes.c_double * 18)()
    _check(ctx, load().vefd_autotune(ctx, int(steps), out))
    return list(out)


def _ens_check(ens, st):
    if st != OK:
        msg = load().vefd_ensemble_last_error(ens) if ens else b""
        raise VefdError(st, (msg or b"").decode())
    return st


def vefd_ensemble_create(ctxs, stream=0):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    h = ctypes.c_void_p()
    _ens_check(None, load().vefd_ensemble_create(arr, len(ctxs), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def vefd_ensemble_step(ens, nsteps, chunk=32):
    return _ens_check(ens, load().vefd_ensemble_step(ens, int(nsteps), int(chunk)))


def vefd_ensemble_set_batched(ens, on):
    return _ens_check(ens, load().vefd_ensemble_set_batched(ens, int(on)))


def vefd_ensemble_set_config(ens, batched, post_segment=0):
    return _ens_check(ens, load().vefd_ensemble_set_config(ens, int(batched), int(post_segment)))


def vefd_ensemble_get_config(ens):
    b, z = ctypes.c_int(), ctypes.c_int()
    _ens_check(ens, load().vefd_ensemble_get_config(ens, ctypes.byref(b), ctypes.byref(z)))
    return b.value, z.value


def vefd_ensemble_set_tile(ens, tile):
    return _ens_check(ens, load().vefd_ensemble_set_tile(ens, int(tile)))


def vefd_ensemble_get_tile(ens):
    t = ctypes.c_int()
    _ens_check(ens, load().vefd_ensemble_get_tile(ens, ctypes.byref(t)))
    return t.value


def vefd_ensemble_set_groups(ens, groups):
    return _ens_check(ens, load().vefd_ensemble_set_groups(ens, int(groups)))


def vefd_ensemble_get_groups(ens):
    g = ctypes.c_int()
    _ens_check(ens, load().vefd_ensemble_get_groups(ens, ctypes.byref(g)))
    return g.value


def vefd_ensemble_autotune(ens, steps=64, chunk=32):
    t = (ctypes.c_double * 7)()
    _ens_check(ens, load().vefd_ensemble_autotune(ens, int(steps), int(chunk), t))
    return [float(v) for v in t]


def vefd_ensemble_is_batched(ens):
    return bool(load().vefd_ensemble_is_batched(ens))


def vefd_ensemble_last_error(ens):
    return (load().vefd_ensemble_last_error(ens) or b"").decode()


def vefd_ensemble_destroy(ens):
    load().vefd_ensemble_destroy(ens)


# --- convenience wrapper -----------------------------------------------------

def _np_ptr(a):
    return a.ctypes.data if a is not None else None


class Lattice:
    """A lattice whose device memory is a torch tensor bound to the library.

    Fields are exchanged as numpy arrays (host) or torch CUDA tensors (device),
    shaped (comp, nz, ny, nx) (comp dropped for scalar fields), FP32.
    """

    def __init__(self, lattice=D3Q19, nx=16, ny=16, nz=16, ncomp=2, walls=1, G=0.0, eta_A=1.0 / 6.0,
                 eta_B=1.0 / 6.0, delta=0.1, device="cuda", stream=None, precision=FP32):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("vefd needs a CUDA device")
        load()
        self.torch = torch
        self.cfg = vefd_config(lattice, nx, ny, nz, ncomp, walls, G, eta_A, eta_B, delta, 1, precision)
        self.nx, self.ny, self.nz, self.ncomp = nx, ny, nz, ncomp
        self.N = nx * ny * nz
        self.D = 3 if lattice == D3Q19 else 2
        self.NC = 6 if lattice == D3Q19 else 4
        self.Q = 19 if lattice == D3Q19 else 9
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = vefd_required_bytes(self.cfg)
        self.mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.mem.data_ptr()
        self._aligned = (base + 255) & ~255
        self.ctx = vefd_create(self.cfg, self.stream.cuda_stream)
        vefd_bind_device_memory(self.ctx, self._aligned, nbytes)

    def close(self):
        if getattr(self, "ctx", None):
            vefd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def planes(self, field):
        return vefd_field_bytes(self.ctx, field) // (4 * self.N)

    def shape(self, field):
        p = self.planes(field)
        return (p, self.nz, self.ny, self.nx) if p > 1 else (self.nz, self.ny, self.nx)

    def set_wall_shear(self, u):
        vefd_set_wall_shear(self.ctx, u)

    def set_body_force(self, fx, fy=0.0, fz=0.0):
        vefd_set_body_force(self.ctx, fx, fy, fz)

    def set_fenep(self, tau_p, eta_p, L2, kappa=0.0, phase=0, fd_on=1):
        vefd_set_fenep(self.ctx, tau_p, eta_p, L2, kappa, phase, fd_on)

    def set_polymer_coupling(self, mode):
        vefd_set_polymer_coupling(self.ctx, mode)

    def set_collision(self, model):
        vefd_set_collision(self.ctx, model)

    def set_conformation_update(self, scheme):
        vefd_set_conformation_update(self.ctx, scheme)

    def init_fields(self, rhoA, rhoB=None, u=None, C=None):
        t = self.torch
        if isinstance(rhoA, t.Tensor):
            args = [x.contiguous().float() if x is not None else None for x in (rhoA, rhoB, u, C)]
            ptrs = [x.data_ptr() if x is not None else None for x in args]
            vefd_init_fields(self.ctx, *[ctypes.c_void_p(p) if p else None for p in ptrs], 1)
        else:
            args = [np.ascontiguousarray(x, dtype=np.float32) if x is not None else None for x in (rhoA, rhoB, u, C)]
            vefd_init_fields(self.ctx, *[ctypes.c_void_p(_np_ptr(x)) if x is not None else None for x in args], 0)

    def init_droplet(self, cx, cy, cz, R, rho_in=2.0, rho_out=0.1, width=5.0, seed=1, phi_amp=1e-3):
        vefd_init_droplet(self.ctx, cx, cy, cz, R, rho_in, rho_out, width, seed, phi_amp)

    def step(self, n=1):
        vefd_step(self.ctx, n)

    def read(self, field, device=False):
        nbytes = vefd_field_bytes(self.ctx, field)
        if device:
            out = self.torch.empty(self.shape(field), dtype=self.torch.float32, device="cuda")
            vefd_read_field(self.ctx, field, out.data_ptr(), nbytes, 1)
            return out
        out = np.empty(self.shape(field), dtype=np.float32)
        vefd_read_field(self.ctx, field, out.ctypes.data, nbytes, 0)
        return out

    def write(self, field, arr):
        nbytes = vefd_field_bytes(self.ctx, field)
        t = self.torch
        if isinstance(arr, t.Tensor):
            a = arr.contiguous().float()
            if a.numel() * 4 != nbytes:
                raise ValueError("size mismatch")
            vefd_write_field(self.ctx, field, a.data_ptr(), nbytes, 1)
        else:
            a = np.ascontiguousarray(arr, dtype=np.float32)
            if a.nbytes != nbytes:
                raise ValueError("size mismatch")
            vefd_write_field(self.ctx, field, a.ctypes.data, nbytes, 0)

    def diagnostics(self):
        return vefd_diagnostics(self.ctx)

    def status(self):
        return vefd_get_status(self.ctx)

    def set_step_graph(self, slabs, chunk=256):
        """Pipelined y-slab step graph (slabs >= 2; 0 off; -1 automatic)."""
        vefd_set_step_graph(self.ctx, slabs, chunk)

    def prepare_step_graph(self):
        """Capture the step graph now (no step taken) so that the next long
        step call only replays it."""
        vefd_prepare_step_graph(self.ctx)

    def prepare_steps(self, nsteps):
        """Capture every graph a later step(nsteps) call replays (no step taken)."""
        vefd_prepare_steps(self.ctx, nsteps)

    @property
    def step_graph(self):
        """(slabs, chunk, active)."""
        return vefd_get_step_graph(self.ctx)

    def wait_selftest(self, arrive):
        """One bounded device wait that completes (arrive=True) or runs out
        and sets ST_TIMEOUT (arrive=False); no fault either way."""
        vefd_wait_selftest(self.ctx, 1 if arrive else 0)

    def clear_status(self):
        vefd_clear_status(self.ctx)

    @property
    def steps_done(self):
        return vefd_steps_done(self.ctx)

    def checkpoint(self, path):
        vefd_checkpoint(self.ctx, path)

    def restore(self, path):
        vefd_restore(self.ctx, path)

    def kernels_per_step(self):
        return vefd_kernels_per_step(self.ctx)

    def profile_kernels(self, on=True):
        vefd_profile_kernels(self.ctx, on)

    def kernel_times(self):
        return vefd_kernel_times(self.ctx)

    def set_kernel_config(self, lattice_tile, post_mode=2):
        """Staged tile (0-5) and densities/FENE-P pass (0 column march with fused
        densities, 1 tiled pass, 2 z-marching pass (the default), 3 partial
        densities from the tiled lattice kernel); shapes that do not admit a
        choice fall back as vefd_set_kernel_config documents."""
        vefd_set_kernel_config(self.ctx, lattice_tile, post_mode)

    def kernel_config(self):
        return vefd_get_kernel_config(self.ctx)

    def autotune(self, steps=50):
        return vefd_autotune(self.ctx, steps)


class Ensemble:
    """Independent lattices stepped together as one replayed CUDA graph: two
    batched launches per step over all members when they allow it, else one
    concurrent branch per lattice.  Holds references to its members."""

    def __init__(self, lattices, stream=None):
        import torch
        self.members = list(lattices)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.ens = vefd_ensemble_create([m.ctx for m in self.members], s.cuda_stream)

    def step(self, n, chunk=32):
        vefd_ensemble_step(self.ens, n, chunk)

    def set_batched(self, on):
        """One launch per kernel phase over all members (default), or one
        graph branch per member."""
        vefd_ensemble_set_batched(self.ens, 1 if on else 0)

    @property
    def batched(self):
        """True when the captured graph uses the batched launches."""
        return vefd_ensemble_is_batched(self.ens)

    def set_config(self, batched, post_segment=0):
        vefd_ensemble_set_config(self.ens, 1 if batched else 0, post_segment)

    @property
    def config(self):
        """(batched, post z-segment) requested for the replays."""
        return vefd_ensemble_get_config(self.ens)

    def set_tile(self, tile):
        """Lattice tiles of the batched launches: 0 32 x 4 x 2, 1 32 x 8 x 1."""
        vefd_ensemble_set_tile(self.ens, tile)

    @property
    def tile(self):
        return vefd_ensemble_get_tile(self.ens)

    def set_groups(self, groups):
        """Group count of the batched launches (0: automatic, 4)."""
        vefd_ensemble_set_groups(self.ens, groups)

    @property
    def groups(self):
        return vefd_ensemble_get_groups(self.ens)

    def autotune(self, steps=64, chunk=32):
        """Times graph branches and batched launches with three z-segments,
        keeps the fastest; the timed steps advance every member."""
        return vefd_ensemble_autotune(self.ens, steps, chunk)

    def close(self):
        if getattr(self, "ens", None):
            vefd_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
