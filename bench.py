#!/usr/bin/env python
"""Throughput of the hybrid LBM / FENE-P step on GB300 (one JSON line).

Workload (default): the D3Q19 two-component Shan-Chen FENE-P confined droplet,
128 x 128 x 64 with the 64 axis wall-normal (NX = 128, NY = 64, NZ = 128),
droplet R = 16 at the box centre, G = 1.5, rho 2.0 / 0.1, interface width 5,
phi noise 1e-3 (SplitMix64 seed 1), viscoelastic droplet (f_+ feedback),
L^2 = 100, De = 1, Ca = 0.1 (sigma = 0.09), tau_B = 1 at rho = 2.1,
eta_A = 0.6 eta_B, eta_P = 0.4 eta_B, kappa = 1e-3.  FP32 populations and C.

One bench step = one time step of the whole hot path over the lattice.
`value` is MLUPS (1e6 node updates per second) summed over ranks, timed with
CUDA events on the library's stream over exactly --steps steps after
--warmup untimed steps.  The populations (152 MB per buffer) exceed the 129 MB
L2, so no flush is needed between steps.

--workload droplet256 runs the 256 x 256 x 128 precision-variant geometry and
--precision fp16|bf16 stores the moving population deviations in 16 bits;
the default FP32 run also times both 16-bit variants ("variants").

--impl reference times the FP64 CPU oracle (the only other place this file
runs oracle code) on a bounded slab of the same workload.
Multi-GPU (torchrun): every rank runs its own replica (weak scaling, no
collective on the data path); the max time over ranks is reported.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (NX, NY wall-normal, NZ, droplet radius); 2R/H = 0.5 in both
    "droplet128": (128, 64, 128, 16.0),
    "droplet256": (256, 128, 256, 32.0),
}
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
ETA_B = 2.1 / 3.0 * 0.5
ETA_A, ETA_P, SIGMA = 0.6 * ETA_B, 0.4 * ETA_B, 0.09


class Setup:
    """Droplet workload geometry and the parameters that follow from Ca = 0.1
    and De = 1 (tau_B = 1 at rho = 2.1, eta_A = 0.6 eta_B, eta_P = 0.4 eta_B)."""

    def __init__(self, workload="droplet128", precision="fp32"):
        self.name = workload
        self.NX, self.NY, self.NZ, self.R = WORKLOADS[workload]
        self.prec_name = precision
        self.prec = PRECISIONS[precision]
        self.gdot = 0.1 * SIGMA / (self.R * ETA_B)
        self.u_wall = self.gdot * self.NY / 2.0
        self.tau_p = 1.0 * self.R * ETA_B / SIGMA * ETA_B / ETA_P
        self.N = self.NX * self.NY * self.NZ
        store = {"fp32": "FP32", "fp16": "FP16", "bf16": "BF16"}[precision]
        self.text = ("D3Q19 two-component Shan-Chen FENE-P confined droplet R=%d, %dx%dx%d (NX=%d, NY=%d wall-normal, "
                     "NZ=%d), G=1.5, L2=100, De=1, Ca=0.1, %s population deviations, FP32 C"
                     % (self.R, self.NX, self.NZ, self.NY, self.NX, self.NY, self.NZ, store))
        # algorithmic bytes per node update (each value read and written once per step):
        # populations (moving ones in the storage type, rest in FP32) + C + AB2 history
        pbytes = 2 * 18 * (4 if self.prec == 0 else 2) * 2 + 2 * 4 * 2
        self.pop_bytes = pbytes
        self.step_bytes = pbytes + 6 * 4 * 2 + 6 * 4 * 2   # 400 for FP32, 256 for 16-bit
        # the same count with every population (the rest one too) in the storage
        # type: 400 for FP32, 248 for 16-bit storage
        self.step_bytes_all_stored = 2 * 19 * (4 if self.prec == 0 else 2) * 2 + 6 * 4 * 2 * 2
KERNEL_NAMES = ["moments", "lattice_collide_stream", "densities_fenep_fd"]


def kernel_algo_bytes(setup, name):
    """Algorithmic bytes per node of each kernel class of the two-kernel step."""
    if name == "lattice_collide_stream":
        return setup.pop_bytes                  # populations read + written
    if name == "densities_fenep_fd":
        return 6 * 4 * 2 + 6 * 4 * 2            # C and AB2 history (the population re-read is overhead)
    return 0                                    # initial densities only
MLUPS = "MLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="droplet128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--no-variants", action="store_true", help="skip the 16-bit storage variant timings")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-lattice ensemble timing")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default kernel tiles")
    ap.add_argument("--no-warmstart", action="store_true",
                    help="skip the bounded warm-start measurement (48 training set-ups, 40 epochs, 8 held out)")
    ap.add_argument("--step-graph", type=int, default=-1,
                    help="slabs of the pipelined step graph (-1 automatic, 0 eager launch pairs)")
    ap.add_argument("--kernel-config", default="",
                    help="lattice_tile,post_mode kernel choice for the timed lattice (default: the library default)")
    ap.add_argument("--profile-region", action="store_true",
                    help="only run --warmup steps, prepare the graphs of --steps steps and bracket that one call "
                         "with cudaProfilerStart/Stop (for ncu --profile-from-start off); prints no JSON line")
    ap.add_argument("--warmstart", action="store_true",
                    help="measure time to steady deformation, warm start from the trained network vs cold start")
    ap.add_argument("--ws-train", type=int, default=128, help="training set-ups for --warmstart")
    ap.add_argument("--ws-eval", type=int, default=12, help="held-out set-ups for --warmstart")
    ap.add_argument("--ws-epochs", type=int, default=60)
    ap.add_argument("--ws-lr", type=float, default=5e-4)
    ap.add_argument("--ws-blend", type=float, default=0.5,
                    help="scale of the predicted increments over the cold start (1: the prediction as it is)")
    ap.add_argument("--ws-channels", default="16,32,80,152",
                    help="U-Net channels per level (multiples of 8; 16,32,80,152 = 2.07 M parameters)")
    ap.add_argument("--ws-tol", type=float, default=2e-6)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def _hash_sources(names):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1406_2686_gb300", "csrc")
    for f in sorted(names):
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def source_hash():
    """Hash of every CUDA source of the library."""
    csrc = os.path.join(ROOT, "paper_1406_2686_gb300", "csrc")
    return _hash_sources([f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh"))])


# the translation units and headers the two step kernels (and their launch
# shapes) are built from
STEP_KERNEL_SOURCES = ("vefd_internal.cuh", "lbm_impl.cuh", "lbm_kernels.cu", "fd_kernels.cu")


def kernel_source_hash():
    """Hash of the step kernels' sources: a recorded ncu traffic figure holds
    while these are unchanged, whatever else in the library changes."""
    return _hash_sources(STEP_KERNEL_SOURCES)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel, kernel_config=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current step-kernel sources (and, when given, the same kernel
    choice)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("kernel_sha") != kernel_source_hash():
        return None
    if kernel_config is not None and list(e.get("kernel_config", [])) != list(kernel_config):
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = []
        smax = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# the paper-faithful choices of Sec. 2 (reported beside the headline)
PAPER_MODEL = dict(collision=1, coupling=1, chol=1)


def make_lattice(S, model=None):
    from paper_1406_2686_gb300 import vefd
    lat = vefd.Lattice(lattice=vefd.D3Q19, nx=S.NX, ny=S.NY, nz=S.NZ, ncomp=2, walls=1, G=1.5, eta_A=ETA_A,
                       eta_B=ETA_B, delta=0.1, precision=S.prec)
    lat.set_wall_shear(S.u_wall)
    lat.set_fenep(S.tau_p, ETA_P, 100.0, 1e-3, 1, 1)
    m = model or {}
    lat.set_collision(m.get("collision", 0))
    lat.set_polymer_coupling(m.get("coupling", 0))
    lat.set_conformation_update(m.get("chol", 0))
    lat.init_droplet((S.NX - 1) / 2.0, (S.NY - 1) / 2.0, (S.NZ - 1) / 2.0, S.R, 2.0, 0.1, 5.0, 1, 1e-3)
    return lat


def droplet_host_fields(S, torch):
    from paper_1406_2686_gb300 import inputs
    rA, rB = inputs.droplet_fields(S.NX, S.NY, S.NZ, R=S.R, seed=1, noise=1e-3)
    a = torch.from_numpy(rA.astype("float32")).pin_memory()
    b = torch.from_numpy(rB.astype("float32")).pin_memory()
    return a, b


def run_e2e(S, lat, torch, steps):
    """End to end through the C-ABI with pinned host buffers: upload the initial
    densities, run `steps` steps, read phi, u and C back to the host and take
    the FP64 diagnostics; wall-clock time around all of it."""
    import ctypes

    from paper_1406_2686_gb300 import vefd
    rA, rB = droplet_host_fields(S, torch)
    outs = {f: torch.empty(vefd.vefd_field_bytes(lat.ctx, f) // 4, dtype=torch.float32).pin_memory()
            for f in (vefd.PHI, vefd.U, vefd.C)}
    h2d = rA.numel() * 4 + rB.numel() * 4
    d2h = sum(t.numel() * 4 for t in outs.values()) + 16 * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vefd.vefd_init_fields(lat.ctx, ctypes.c_void_p(rA.data_ptr()), ctypes.c_void_p(rB.data_ptr()), None, None, 0)
    lat.step(steps)
    for f, t in outs.items():
        vefd.vefd_read_field(lat.ctx, f, t.data_ptr(), t.numel() * 4, 0)
    lat.diagnostics()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dt, h2d, d2h


def cpu_baseline(S, budget_s=15.0):
    """The FP64 oracle as it stands, on the host cores, on the same droplet
    lattice: as many steps as fit in the budget (at least two)."""
    import oracle
    from paper_1406_2686_gb300 import inputs
    cores = oracle.set_threads(0)
    NX, NY, NZ = S.NX, S.NY, S.NZ
    rA, rB = inputs.droplet_fields(NX, NY, NZ, R=S.R, seed=1, noise=1e-3)
    o = oracle.Oracle(lattice=1, nx=NX, ny=NY, nz=NZ, ncomp=2, walls=1, G=1.5, eta_A=ETA_A, eta_B=ETA_B,
                      delta=0.1, u_wall=S.u_wall, tau_p=S.tau_p, eta_p=ETA_P, L2=100.0, kappa=1e-3, phase=1)
    o.init_fields(inputs.to_f32_exact(rA), inputs.to_f32_exact(rB))
    o.step(1)
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step(1)
        n += 1
        dt = time.perf_counter() - t0
        if n >= 2 and dt > budget_s:
            break
    N = NX * NY * NZ
    return {"value": N * n / dt / 1e6, "unit": MLUPS, "cores": cores, "kind": "oracle",
            "sample": "%d steps of the full %dx%dx%d droplet lattice (FP64, OpenMP over nodes)" % (n, NX, NY, NZ)}


def replica_throughput(elapsed_ms, nodes_per_rank, steps, device="cpu"):
    """Whole-job MLUPS of independent replicas: every rank advanced
    `nodes_per_rank` nodes for `steps` steps; the job time is the slowest
    rank's (max over ranks).  Returns (max elapsed ms, MLUPS)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = float(elapsed_ms)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, nodes_per_rank * steps * world / (ms / 1e3) / 1e6


def time_variant(S, steps, warmup, model=None, kernel_config=None):
    """MLUPS of one storage, model or kernel-choice variant on the same workload (events on the library stream)."""
    import torch
    lat = make_lattice(S, model)
    if kernel_config is not None:
        lat.set_kernel_config(*kernel_config)
    lat.step(warmup)
    lat.prepare_steps(steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    peak, _ = measured_peak()
    bw = S.step_bytes * S.N / (ms / steps / 1e3) / 1e9
    bw_all = S.step_bytes_all_stored * S.N / (ms / steps / 1e3) / 1e9
    out = {"value": round(S.N * steps / (ms / 1e3) / 1e6, 1), "unit": MLUPS, "ms_per_step": round(ms / steps, 5),
           "step_roofline": {"achieved": round(bw, 1), "frac": round(bw / peak, 4),
                             "algorithmic_bytes_per_node": S.step_bytes,
                             "frac_all_populations_stored": round(bw_all / peak, 4),
                             "bytes_per_node_all_populations_stored": S.step_bytes_all_stored},
           "status_bits": lat.status(),
           "kernel_config": list(lat.kernel_config()), "step_graph": list(lat.step_graph)}
    lat.close()
    return out


def measured_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except Exception:
        return 1900.0, "fallback"


def time_nn_gemm(reps=20):
    """TFLOP/s of the warm-start network's tensor-core GEMM (vefd_nn_gemm_bf16:
    TMA-fed 4-stage ring, tcgen05 BF16 MMAs with FP32 accumulation in tensor
    memory): a square 8192^3 product, and the shape of a 16 -> 32 channel
    3x3x3 convolution on the 64^3 input (im2col: M = 262144 voxels, N = 32,
    K = 27 * 16 = 432 padded to 432) whose operands stream from HBM.
    Events on the current stream around `reps` back-to-back launches."""
    import torch

    from paper_1406_2686_gb300 import nn
    peak, src = measured_bf16_peak()
    out = {"peak_tflops": peak, "peak_source": src}
    for name, (M, N, K) in (("square_8192", (8192, 8192, 8192)), ("conv_64cube_16to32", (262144, 32, 432))):
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(3):
            nn.gemm(A, B, C=C, status=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            nn.gemm(A, B, C=C, status=st)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tf = 2.0 * M * N * K / (ms / 1e3) / 1e12
        # spot check against a plain torch matmul of the same BF16 operands
        rows = torch.arange(0, M, max(1, M // 64), device="cuda")
        ref = (A[rows].float() @ B.float().T)
        err = float((C[rows] - ref).abs().max() / ref.abs().max().clamp_min(1e-30))
        out[name] = {"M": M, "N": N, "K": K, "ms": round(ms, 4), "tflops": round(tf, 1), "frac": round(tf / peak, 4),
                     "hbm_gbs": round((M * K * 2 + N * K * 2 + M * N * 4) / (ms / 1e3) / 1e9, 1),
                     "max_rel_err_vs_fp32_matmul": err, "status": int(st.item())}
        del A, B, C
    return out


def time_d2q9_couette(big_steps=1000, warmup=100):
    """The single-component D2Q9 FENE-P Couette set-up (tau = 1, walls +-0.01,
    tau_P = 1000, eta_P / (eta_s + eta_P) = 0.4, L^2 = 100, C = I): the wall
    time of its 20000 steps on the 64 x 32 lattice (2048 nodes, so launch-
    latency bound), and MLUPS on a scaled 4096 x 2048 lattice, where the
    algorithmic bytes are 136 per node update (18 populations, 4 C
    components and 4 history components, each read and written once)."""
    import numpy as np
    import torch

    from paper_1406_2686_gb300 import vefd
    eta_s = 1.0 / 6.0
    peak, _ = measured_peak()

    def lattice(nx, ny):
        L = vefd.Lattice(lattice=vefd.D2Q9, nx=nx, ny=ny, nz=1, ncomp=1, walls=1, eta_A=eta_s, eta_B=eta_s)
        L.set_wall_shear(0.01)
        L.set_fenep(1000.0, eta_s * 0.4 / 0.6, 100.0, 0.0, 0, 1)
        L.init_fields(np.ones((1, ny, nx), np.float32))
        return L

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    small = lattice(64, 32)
    small.step(1)
    small.prepare_step_graph()  # the whole-lattice graph, captured outside the timed region
    torch.cuda.synchronize()
    e0.record(small.stream)
    small.step(20000)
    e1.record(small.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["64x32_20000_steps"] = {"ms": round(ms, 2), "us_per_step": round(ms / 20000 * 1e3, 2),
                                "step_graph": list(small.step_graph), "status_bits": small.status()}
    small.close()
    big = lattice(4096, 2048)
    big.step(warmup)
    big.prepare_step_graph()
    torch.cuda.synchronize()
    e0.record(big.stream)
    big.step(big_steps)
    e1.record(big.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n = 4096 * 2048
    bw = 136 * n / (ms / big_steps / 1e3) / 1e9
    out["4096x2048"] = {"value": round(n * big_steps / (ms / 1e3) / 1e6, 1), "unit": MLUPS, "steps": big_steps,
                        "step_roofline": {"achieved": round(bw, 1), "frac": round(bw / peak, 4),
                                          "algorithmic_bytes_per_node": 136}, "status_bits": big.status()}
    big.close()
    return out


def ensemble_setups(n=64, seed=7, umax=0.08, screen=100):
    """n uneven sheared-droplet boxes sweeping the set-up: NX in {32, 64, 96},
    NY and NZ in {32, 40, ..., 96}; Ca in [0.05, 0.3], De in [0.1, 4]
    (log-uniform), 2R/H in [0.3, 0.8], viscosity ratio in [0.5, 2]
    (log-uniform), droplet or matrix viscoelastic; all drawn from
    SplitMix64(seed).  Draws whose droplet does not fit the box (2R above 0.8
    of NX or NZ) or whose wall speed would exceed umax are skipped, and so
    are draws whose start-up transient trips a guard (|u| > 0.3 from the
    sharp initial interface) within `screen` steps (0: no screening, no GPU
    needed).  Returns (set-ups, number screened out)."""
    import math

    from paper_1406_2686_gb300 import inputs
    from paper_1406_2686_gb300 import warmstart as ws
    out, k, dropped = [], 0, 0
    while len(out) < n:
        r = [int(inputs.splitmix64(seed, 8 * k + j)) for j in range(3)]
        u = [inputs.splitmix64(seed, 8 * k + 3 + j) / 2.0 ** 64 for j in range(5)]
        k += 1
        dims = (32 * (1 + r[0] % 3), 8 * (4 + r[1] % 9), 8 * (4 + r[2] % 9))
        s = ws.Setup(0.05 + 0.25 * u[0], math.exp(math.log(0.1) + u[1] * math.log(40.0)), 0.3 + 0.5 * u[2],
                     2.0 ** (2.0 * u[3] - 1.0), 1 if u[4] < 0.5 else -1, dims=dims)
        s.seed = k
        if not (2.0 * s.R <= 0.8 * min(dims[0], dims[2]) and s.u_wall <= umax):
            continue
        if screen:
            L = s.cold(seed=s.seed)
            L.step(screen)
            bad = L.status() != 0
            L.close()
            if bad:
                dropped += 1
                continue
        out.append(s)
    return out, dropped


def small_setups(n=256):
    """n small sheared-droplet boxes, 32 x 16 x 16 (8192 nodes each), one set-up."""
    from paper_1406_2686_gb300 import warmstart as ws
    s = ws.Setup(0.1, 1.0, 0.5, 1.0, 1, dims=(32, 16, 16))
    s.seed = 1
    return [s] * n


def time_ensemble(steps, warmup, chunk=32, setups=None, label=None):
    """Many independent sheared-droplet lattices: stepped one after another on
    one stream (plain vefd_step per lattice) versus as one ensemble, either one
    CUDA graph with a concurrent branch per lattice or two batched launches per
    step over the tiles of all lattices.  Same lattices, same steps; MLUPS of
    each."""
    import torch

    from paper_1406_2686_gb300 import vefd
    screened = 0
    if setups is None:
        setups, screened = ensemble_setups()
        label = ("64 D3Q19 two-component sheared droplets, NX in {32,64,96}, NY, NZ in {32,...,96} step 8; "
                 "Ca in [0.05,0.3], De in [0.1,4], 2R/H in [0.3,0.8], lambda in [0.5,2], either phase "
                 "viscoelastic (SplitMix64 seed 7); draws whose start-up transient trips a guard within 100 "
                 "steps are replaced")

    def build():
        return [s.cold(seed=s.seed) for s in setups]

    nodes = sum(a * b * c for a, b, c in (s.dims for s in setups))
    stream = torch.cuda.current_stream()
    out = {"lattices": len(setups), "nodes": nodes, "steps": steps, "chunk": chunk, "boxes": label,
           "screened_out": screened}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lats = build()
    for L in lats:
        L.step(warmup + chunk)  # the same steps the ensembles take before their timed region
        L.prepare_steps(steps)  # every graph the timed step(steps) replays
    torch.cuda.synchronize()
    e0.record(stream)
    for L in lats:
        L.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["one_stream"] = {"value": round(nodes * steps / (ms / 1e3) / 1e6, 1), "unit": MLUPS, "ms": round(ms, 3)}
    import numpy as np
    seq_state = [L.read(vefd.C) for L in lats[:2]]
    for L in lats:
        L.close()
    status = 0
    for key, batched in (("graph", False), ("batched", True)):
        lats = build()
        E = vefd.Ensemble(lats, stream)
        E.set_batched(batched)
        E.step(warmup, chunk)
        E.step(chunk, chunk)  # captures the ensemble's chunk graph before the timed region
        torch.cuda.synchronize()
        e0.record(stream)
        E.step(steps, chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[key] = {"value": round(nodes * steps / (ms / 1e3) / 1e6, 1), "unit": MLUPS, "ms": round(ms, 3),
                    "launches_per_step": 2 * min(4, len(setups)) if E.batched else 2 * len(setups)}
        got = [L.read(vefd.C) for L in lats[:2]]
        out[key]["bit_identical"] = all(np.array_equal(a, g) for a, g in zip(seq_state, got))
        out[key]["max_rel_diff"] = float(max(np.linalg.norm(g - a) / np.linalg.norm(a) for a, g in zip(seq_state, got)))
        status |= max(L.status() for L in lats)
        E.close()
        for L in lats:
            L.close()
    out["status_bits"] = status
    return out


def run_ours(args):
    import torch

    from paper_1406_2686_gb300 import vefd

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vefd.load(build_if_missing=True)
    S = Setup(args.workload, args.precision)
    NX, NY, NZ = S.NX, S.NY, S.NZ
    lat = make_lattice(S)
    lat.set_step_graph(args.step_graph)
    if args.kernel_config:
        lat.set_kernel_config(*[int(v) for v in args.kernel_config.split(",")])
    stream = lat.stream
    K, W = args.steps, args.warmup
    tune = None
    if not args.no_autotune:
        # every kernel choice timed on a scratch lattice of this configuration
        # (results are bit-identical across choices); reported, not applied:
        # the headline runs the default choice that the committed ncu traffic
        # figures were taken on
        default_config = lat.kernel_config()
        times = lat.autotune(steps=50)
        tune = {"fastest": list(lat.kernel_config()), "ms_per_50_steps": [round(t, 3) for t in times],
                "index": "post_mode * 6 + lattice_tile; -1 = not admitted", "applied": False}
        lat.set_kernel_config(*default_config)
    timed_config = list(lat.kernel_config())
    with torch.cuda.stream(stream):
        lat.step(W)
        lat.prepare_steps(K)  # capture every graph step(K) replays, outside the timed region (no step is taken)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    # launches in the timed region: steps replayed by the step graph (whole
    # chunks and one graph of the even remainder; two launches per slab and
    # step), the rest (an odd last step) one lattice kernel and one pass
    slabs, chunk, active = lat.step_graph
    graph_steps = (K // chunk) * chunk + ((K % chunk) & ~1) if active else 0
    launches = int(graph_steps * lat.kernels_per_step() * max(slabs, 1) + (K - graph_steps) * lat.kernels_per_step())
    step_graph = {"slabs": slabs, "chunk": chunk, "active": active, "graph_steps": graph_steps}
    # per-kernel durations: the same K steps again with an event pair around
    # every launch (on the library's stream, one launch pair per step: kernel
    # timing turns the step graph off), kept out of the headline timing
    lat.profile_kernels(True)
    lat.step(K)
    kms, klaunch = lat.kernel_times()
    lat.profile_kernels(False)
    status = lat.status()
    N = NX * NY * NZ
    ms, value = replica_throughput(ms, N, K, device="cuda")
    peak, peak_kind = measured_peak()
    # dominant kernel and its roofline
    dom = max(range(3), key=lambda k: kms[k])
    dname = KERNEL_NAMES[dom]
    avg_s = kms[dom] / max(klaunch[dom], 1) / 1e3
    algo = kernel_algo_bytes(S, dname) * N
    achieved = algo / avg_s / 1e9
    traffic = recorded_traffic(dname, timed_config) if (S.name, S.prec) == ("droplet128", 0) else None
    roof = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "algorithmic_bytes_per_launch": algo,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind}
    step_achieved = S.step_bytes * N / (ms / K / 1e3) / 1e9
    kernels = {KERNEL_NAMES[k]: {"launches": klaunch[k], "ms_total": round(kms[k], 3),
                                 "share": round(kms[k] / max(sum(kms), 1e-12), 4)} for k in range(3)}
    e2e = None
    if not args.no_e2e:
        # one untimed pass captures the graphs the timed pass replays (the
        # state after the upload is the same both times)
        run_e2e(S, lat, torch, K)
        # a 20-step call is a few milliseconds of host wall clock: report the
        # median of five whole passes and their spread
        dts = []
        for _ in range(5):
            dt, h2d, d2h = run_e2e(S, lat, torch, K)
            dts.append(dt)
        dt = sorted(dts)[len(dts) // 2]
        _, e2e_val = replica_throughput(dt * 1e3, N, K, device="cuda")
        e2e = {"value": round(e2e_val, 1), "unit": MLUPS, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K, "passes_ms": [round(x * 1e3, 3) for x in dts],
               "what": "init from pinned host densities + %d steps + phi/u/C read to pinned host + diagnostics; "
                       "median of 5 passes" % K}
    line = {
        "metric": "MLUPS & % HBM roofline", "value": round(value, 1), "unit": MLUPS, "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(ms / K, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": S.text, "nodes": N, "global_nodes": N * world, "population_storage": S.prec_name,
                   "l2": "inputs larger than L2 (152 MB per population buffer > 129 MB), no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "step_roofline": {"achieved": round(step_achieved, 1), "peak": peak, "unit": "GB/s",
                          "frac": round(step_achieved / peak, 4),
                          "algorithmic_bytes_per_node": S.step_bytes},
        "kernels": kernels, "gpu_launches": launches, "step_graph": step_graph, "clocks": clk, "e2e": e2e,
        "autotune": tune, "kernel_config": timed_config,
        "status_bits": status, "source_sha": source_hash(), "kernel_sha": kernel_source_hash(),
    }
    lat.close()
    if not args.no_variants and S.prec == 0:
        # NEXT-1 storage variants of the same workload, reported beside the FP32 headline
        vsteps = max(200, K // 5)
        line["variants"] = {pn: time_variant(Setup(S.name, pn), vsteps, min(W, 50)) for pn in ("fp16", "bf16")}
        for name, model in (("mrt", dict(collision=1)), ("cholesky", dict(chol=1)), ("paper_sec2", PAPER_MODEL)):
            line["variants"][name] = time_variant(S, vsteps, min(W, 50), model)
        # the column-marching lattice kernel with partial densities (post mode 0)
        line["variants"]["fused_densities"] = time_variant(S, vsteps, min(W, 50), kernel_config=(0, 0))
        line["variants"]["d2q9_couette"] = time_d2q9_couette()
        line["nn_gemm"] = time_nn_gemm()
        line["variants"]["note"] = ("fp16/bf16: 16-bit moving-population deviations, FP32 rest population, FP32 arithmetic "
                                    "and C; mrt: moment-space collision with the paper's relaxation times; cholesky: "
                                    "log-Cholesky conformation update; paper_sec2: both plus the polymer stress in the "
                                    "equilibrium; %d steps each; d2q9_couette: the one-component D2Q9 Couette "
                                    "set-up, 20000 steps at 64 x 32 (time) and MLUPS at 4096 x 2048" % vsteps)
    if not args.no_warmstart and S.prec == 0:
        # bounded form of --warmstart: 48 training set-ups, 40 epochs, 8 held out
        line["warmstart"] = warmstart_measure(48, 8, 40, args.ws_lr, args.ws_tol,
                                              tuple(int(v) for v in args.ws_channels.split(",")), args.ws_blend)
    if not args.no_ensemble and S.prec == 0:
        line["ensemble"] = time_ensemble(max(100, K // 20), min(W, 20))
        line["ensemble_small"] = time_ensemble(max(100, K // 20), min(W, 20), setups=small_setups(),
                                               label="256 D3Q19 two-component sheared droplets, 32 x 16 x 16 each")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(S)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def warmstart_measure(n_train, n_eval, epochs, lr, tol, channels=(16, 32, 80, 152), blend=0.5, log=None):
    """Time to steady deformation of held-out droplet set-ups, cold start
    versus a start from the trained network's prediction: data from the
    method's own steady states, training and prediction on this package's
    kernels, then both runs to the same steady rule.  Returns the result dict."""
    import numpy as np
    import torch

    from paper_1406_2686_gb300 import nn, warmstart as ws
    t0 = time.perf_counter()
    train_setups = ws.sample_setups(n_train, seed=11)
    eval_setups = ws.sample_setups(n_eval, seed=29)
    X, Y, rec = ws.make_dataset(train_setups, tol=tol, log=log)
    t_data = time.perf_counter() - t0
    net = nn.UNet(ws.N_IN, ws.N_OUT, seed=0, channels=tuple(channels))
    t1 = time.perf_counter()
    losses = ws.train(net, X, Y, epochs=epochs, lr=lr, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    res = ws.evaluate(net, eval_setups, tol=tol, log=log, blend=blend)
    cold = np.array([r["cold_seconds"] for r in res])
    warm = np.array([r["warm_seconds"] for r in res])
    derr = np.array([r["D_rel_err"] for r in res])
    speed = cold / warm
    within = derr <= 0.01
    return {
        "metric": "time-to-steady deformation, warm-start vs plain", "value": round(float(np.median(speed)), 3),
        "unit": "x (cold / warm wall time, median over held-out set-ups)", "higher_is_better": True,
        "median_speedup_within_1pct": round(float(np.median(speed[within])), 3) if within.any() else None,
        "config": {"box": "64^3 D3Q19 two-component droplet, walls in y", "train_setups": len(train_setups),
                   "eval_setups": len(eval_setups), "steady_rule": "|dD| < %g per tau_em over 5 consecutive tau_em "
                   "(mid-plane, smooth indicator)" % tol, "network": "3-D U-Net, %d parameters, BF16 tcgen05 GEMMs, "
                   "FP32 accumulate" % net.n_params(), "channels": list(channels), "epochs": epochs, "lr": lr,
                   "blend": blend,
                   "lr_schedule": "linear ramp from lr/10 over the first epoch, then geometric decay to lr/10"},
        "steps": {"cold_median": int(np.median([r["cold_steps"] for r in res])),
                  "warm_median": int(np.median([r["warm_steps"] for r in res]))},
        "seconds": {"cold_median": round(float(np.median(cold)), 4), "warm_median": round(float(np.median(warm)), 4),
                    "predict_median": round(float(np.median([r["predict_seconds"] for r in res])), 4),
                    "dataset": round(t_data, 2), "training": round(t_train, 2)},
        "D_rel_err": {"median": float(np.median(derr)), "max": float(np.max(derr)),
                      "within_1pct": int(np.sum(within))},
        "speedup_per_setup": [round(float(v), 3) for v in speed], "loss_first_last": [losses[0], losses[-1]],
        "all_converged": bool(all(r["cold_converged"] and r["warm_converged"] for r in res)),
        "status": net.status(),
    }


def run_warmstart(args):
    """The warm-start measurement alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    chans = tuple(int(v) for v in args.ws_channels.split(","))
    line = warmstart_measure(args.ws_train, args.ws_eval, args.ws_epochs, args.ws_lr, args.ws_tol, chans,
                             args.ws_blend, log=log)
    line.update({"n_gpus": 1, "data": "synthetic (steady states generated by the lattice-Boltzmann/FENE-P step)"})
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1406_2686_gb300 import inputs
    cores = oracle.set_threads(0)
    K, W = args.steps, args.warmup
    S = Setup(args.workload, "fp32")
    NX, NY, NZ = S.NX, S.NY, S.NZ

    def make(nz_s):
        rA, rB = inputs.droplet_fields(NX, NY, nz_s, R=S.R, seed=1, noise=1e-3,
                                       center=((NX - 1) / 2.0, (NY - 1) / 2.0, (nz_s - 1) / 2.0))
        o = oracle.Oracle(lattice=1, nx=NX, ny=NY, nz=nz_s, ncomp=2, walls=1, G=1.5, eta_A=ETA_A, eta_B=ETA_B,
                          delta=0.1, u_wall=S.u_wall, tau_p=S.tau_p, eta_p=ETA_P, L2=100.0, kappa=1e-3, phase=1)
        o.init_fields(inputs.to_f32_exact(rA), inputs.to_f32_exact(rB))
        return o

    probe = make(4)
    t0 = time.perf_counter()
    probe.step(2)
    per_node = (time.perf_counter() - t0) / (2 * NX * NY * 4)
    budget = 150.0
    nz_s = int(budget / max(K + W, 1) / per_node / (NX * NY))
    nz_s = max(2, min(NZ, nz_s))
    o = make(nz_s)
    o.step(W)
    t0 = time.perf_counter()
    o.step(K)
    dt = time.perf_counter() - t0
    n = NX * NY * nz_s
    value = n * K / dt / 1e6
    sample = "each step: one FP64 oracle time step of a %dx%dx%d slab of the droplet workload" % (NX, NY, nz_s)
    line = {
        "metric": "MLUPS & % HBM roofline", "value": round(value, 3), "unit": MLUPS, "impl": "reference",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": round(dt / K * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": S.text, "nodes": NX * NY * NZ, "sample_nodes": n},
        "cpu_baseline": {"value": round(value, 3), "unit": MLUPS, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": MLUPS, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_region(args):
    """The headline workload's K-step call alone between cudaProfilerStart and
    cudaProfilerStop: with `ncu --profile-from-start off --graph-profiling
    graph` the replayed step graph is measured as one workload, its slabs
    running concurrently as in the timed region."""
    import torch

    from paper_1406_2686_gb300 import vefd
    torch.cuda.set_device(0)
    vefd.load(build_if_missing=True)
    S = Setup(args.workload, args.precision)
    lat = make_lattice(S)
    lat.set_step_graph(args.step_graph)
    if args.kernel_config:
        lat.set_kernel_config(*[int(v) for v in args.kernel_config.split(",")])
    lat.step(args.warmup)
    lat.prepare_steps(args.steps)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    lat.step(args.steps)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print("profiled %d steps, step graph %r, kernel choice %r, status %d"
          % (args.steps, lat.step_graph, lat.kernel_config(), lat.status()), file=sys.stderr)
    lat.close()


def main():
    args = parse()
    if args.profile_region:
        run_profile_region(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.warmstart:
        run_warmstart(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
