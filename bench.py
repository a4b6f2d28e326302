"""Benchmark: slab factor+solve of the 3-D variable-coefficient diffusion workload.

Workload (one "step" = the whole hot path): -div(kappa grad u) = f on the unit cube, n = 96
(95^3 = 857,375 unknowns), slab spacing b = 8 (11 interfaces of 9025 unknowns), kappa = exp(g)
with g a seeded 8-mode Fourier field of unit variance, 16 right-hand sides f ~ N(0,1); FP32 factor
(3-D slab elimination, T assembly and Stage 2 on the tensor cores in FP32-accurate products, the
elimination order chosen by the library's cost model) followed by the solve with FP64
stencil-residual refinement until max relres <= 1e-10.  Inputs are resident in HBM when the timed
region starts; every step streams tens of GB of factors (far more than the 129 MB L2), so no
explicit L2 flush is needed.  --workload selects the other workloads (2-D diffusion n = 2048,
2-D Helmholtz n = 4096, the batched adjoint as CUDA graphs, the J_0 benchmark).

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve s at 1e-10 rel. residual vs plain FP64 GPU; dense TFLOP/s % of peak"


# ---------------------------------------------------------------- replicas (one process per GPU)
# The method's multi-GPU form here is replicas: under torchrun every rank factors and solves its
# own copy of the workload on its own GPU (no exchange on the data path); the timed region is
# bracketed by barriers and the slowest rank's time is reported, by rank 0 alone.
def dist_env():
    """(rank, local_rank, world_size) from the launcher's environment; (0, 0, 1) without one."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def dist_init(backend: str) -> None:
    """Join the process group when more than one rank runs (env:// rendezvous)."""
    import torch.distributed as dist
    if dist_env()[2] > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, init_method="env://")


def _dist_on() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def dist_barrier() -> None:
    if _dist_on():
        import torch.distributed as dist
        dist.barrier()


def dist_max(x: float) -> float:
    """Largest value of x over the ranks (x itself with one rank)."""
    if not _dist_on():
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


HOST_NUMA = {"node": None, "cpus": None}
_FULL_AFFINITY = None


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if part:
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_host_to_gpu(index):
    """Run this process on the CPUs of the GPU's NUMA node (from sysfs), so that the pinned host
    buffers allocated afterwards sit next to the GPU; restore_host_affinity() undoes it.  Records the
    node in HOST_NUMA; leaves everything as it is where the node is unknown."""
    global _FULL_AFFINITY
    import torch
    try:
        pr = torch.cuda.get_device_properties(index)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as fh:
            node = int(fh.read())
        if node < 0:
            return
        with open(f"/sys/devices/system/node/node{node}/cpulist") as fh:
            full = os.sched_getaffinity(0)
            cpus = _cpulist(fh.read()) & full
        if not cpus:
            return
        _FULL_AFFINITY = full
        os.sched_setaffinity(0, cpus)
        HOST_NUMA.update(node=node, cpus=len(cpus))
    except (OSError, ValueError, AttributeError):
        return


def restore_host_affinity():
    if _FULL_AFFINITY:
        os.sched_setaffinity(0, _FULL_AFFINITY)


def rank_device():
    """This rank's GPU (cuda:LOCAL_RANK), made current, with the process group joined; the host
    thread moves to the GPU's NUMA node (bind_host_to_gpu)."""
    import torch
    dev = torch.device("cuda", dist_env()[1])
    torch.cuda.set_device(dev)
    dist_init("nccl")
    bind_host_to_gpu(dev.index)
    return dev
WORKLOAD = dict(workload="2D var-coef diffusion n=2048 b=32 k=64 (kappa=exp(16-mode field), f~N(0,1)), "
                         "FP32 factor + FP64 refinement to 1e-10",
                n=2048, b=32, k=64, rtol=1e-10, kind="diffusion")
DIFFUSION3D = dict(workload="3D var-coef diffusion n=96 b=8 k=16 (kappa=exp(8-mode 3-D field), f~N(0,1)), "
                            "FP32 factor + FP64 refinement to 1e-10",
                   n=96, b=8, k=16, rtol=1e-10, kind="diffusion3d")
HELMHOLTZ = dict(workload="2D Helmholtz n=4096 b=32 k=1 (c=1+0.3 r, 8-mode field, 10 points per wavelength, "
                          "point source), pivoted factor + FP64 refinement to 1e-10",
                 n=4096, b=32, k=1, rtol=1e-10, kind="helmholtz")
SMS = 152
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.samples = []
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                                           f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = sorted(x for x in (num(s[0]) for s in self.samples) if x is not None)
        mx = [x for x in (num(s[1]) for s in self.samples) if x is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------------------- algorithmic work model
def tree_nodes(s):
    """(c, k, w) of every node of the ruler tree over rows 1..s."""
    out = []
    k = 0
    while (1 << k) <= s:
        p = 1 << k
        c = p
        while c <= s:
            lo, hi = c - p + 1, min(s, c + p - 1)
            out.append((c, k, hi - lo + 1))
            c += 2 * p
        k += 1
    return out


def oddeven_levels(NI):
    """(nb, nc) per level of the odd-even order: blocks eliminated, and those with a right neighbour."""
    out, step = [], 1
    while step < NI:
        nrem = (NI - 1) // step + 1
        if nrem < 2:
            break
        out.append((nrem // 2, (nrem - 1) // 2))
        step *= 2
    return out


def work_model_3d(n, b, k, passes, stage2):
    """Algorithmic flops per kernel class for the 3-D path (dense per-node tree along z).

    Stage 1 (the slab elimination, slab_* classes and assemble_T) and Stage 2 (panel, trailing,
    schur_update) are counted apart, as the library times them apart."""
    s = n - 1
    m = b - 1
    M = m * s
    Mp = (M + 63) // 64 * 64
    si = s * s
    sp = (si + 63) // 64 * 64
    NS, NI = n // b, n // b - 1
    W = {k_: 0.0 for k_ in ("tree_factor", "assemble_T", "panel", "trailing", "schur_update", "sweep_products",
                            "tree_up", "tree_down", "stencil", "slab_panel", "slab_trailing", "slab_schur")}
    for (c, kk, w) in tree_nodes(s):
        wl = w * s
        wmax = min(s, (1 << (kk + 1)) - 1)
        wsp = (wmax * s + 63) // 64 * 64
        ident0 = 3 * Mp + 2 * wsp
        for kb in range(Mp // 64):                     # batched tall Cholesky of [S; B^T; I]
            rows = ident0 + (kb + 1) * 64
            W["slab_panel"] += NS * (rows // 64 - kb - 1) * (2 * 64 ** 3 + 2 * 64 ** 3 / 3)
            c0 = (kb + 1) * 64
            if c0 < Mp:
                nn = Mp - c0
                W["slab_trailing"] += NS * 2 * 64 * (nn * (nn + 1) / 2 + (rows - Mp) * nn)
        W["slab_schur"] += NS * (2.0 * (2 * Mp) ** 2 * Mp + 2 * 2.0 * 2 * Mp * wl * Mp)
        W["assemble_T"] += NS * 3 * 2.0 * wl * wl * Mp
        W["tree_up"] += passes * NS * k * (2.0 * Mp * Mp + 2.0 * 2 * Mp * Mp + 2.0 * 2 * wsp * Mp)
        W["tree_down"] += passes * NS * k * (2.0 * Mp * 2 * Mp + 2.0 * Mp * 2 * wsp + 2.0 * Mp * Mp)
    W2 = work_model_stage2(sp, NI, k, passes, stage2)
    for key in ("panel", "trailing", "schur_update", "sweep_products"):
        W[key] += W2[key]
    W["stencil"] = passes * 24.0 * s ** 3 * k
    return W


def alg1_cholesky_flops(si, NI):
    """Algorithm 1 in Cholesky form on the unpadded interface blocks (s = si): per interface the
    Cholesky of S_j (s^3/3), Y_j = L_j^-1 T_{j,j+1} (s^3) and S_{j+1} = T_{j+1,j+1} - Y_j^T Y_j (s^3):
    N_I s^3/3 + (N_I - 1) 2 s^3.  The odd-even order performs about 4x these flops."""
    return NI * si ** 3 / 3.0 + (NI - 1) * 2.0 * si ** 3


def work_model_stage2(sp, NI, k, passes, stage2):
    """Stage-2 (SPD) flops: tall Cholesky panels and trailing updates, Schur updates, solve products."""
    W = {"panel": 0.0, "trailing": 0.0}
    for j in range(NI):
        lt0 = sp if stage2 == "oddeven" else (2 if j < NI - 1 else 1) * sp
        for kb in range(sp // 64):
            rows = lt0 + (kb + 1) * 64
            W["panel"] += (rows // 64 - kb - 1) * (2 * 64 ** 3 + 2 * 64 ** 3 / 3)
            c0 = (kb + 1) * 64
            if c0 < sp:
                nn = sp - c0
                W["trailing"] += 2 * 64 * (nn * (nn + 1) / 2 + (rows - sp) * nn)
    if stage2 == "oddeven":
        lv = oddeven_levels(NI)
        nb, nc = sum(x for x, _ in lv), sum(y for _, y in lv)
        W["schur_update"] = nb * (2.0 * sp ** 3 + sp * sp * (sp + 1.0)) + nc * (4.0 * sp ** 3 + sp * sp * (sp + 1.0))
        W["sweep_products"] = passes * (4 * nb + 2 * nc + 2) * 2.0 * sp * sp * k
    else:
        W["schur_update"] = (NI - 1) * sp * sp * (sp + 1.0)
        W["sweep_products"] = passes * (4 * NI - 2) * 2.0 * sp * sp * k
    return W


def work_model(n, b, k, passes, stage2="sweep", kind="diffusion"):
    """Algorithmic flops (or bytes) per kernel class for one factor + `passes` solve passes.

    Explicit inverse factors (L^{-1}, L^{-T}) are stored and applied as dense blocks, so
    their products count as dense (2 s^3 per s x s x s product; s(s+1)s for a lower-half update)."""
    if kind == "diffusion3d":
        return work_model_3d(n, b, k, passes, stage2)
    s = n - 1
    sp = (s + 63) // 64 * 64
    m = b - 1
    NS, NI = n // b, n // b - 1
    nodes = tree_nodes(s)
    W = {}
    # Stage 1 tree factor: per node Cholesky + inverse (2/3 m^3), Z = Li B (m^2 * 2m), R update (2m)^2 m,
    # interface columns 2w: z = Li b (m^2), two m x m products (2 m^2)
    W["tree_factor"] = NS * sum(2 * (2 * m ** 3 / 3 + 2 * m ** 3 + 4 * m ** 3 + 2 * w * 3 * m * m)
                                for (_, _, w) in nodes)
    W["assemble_T"] = 4.0 * sp * sp * (2 * NI - 1)                      # bytes of T written (FP32)
    # Stage 2: panel CTAs (Cholesky+inverse 2/3 * 64^3 + product 2 * 64^3), trailing products, Schur update
    pan = trail = 0.0
    for j in range(NI):
        lt0 = sp if stage2 == "oddeven" else (2 if j < NI - 1 else 1) * sp
        for kb in range(sp // 64):
            rows = lt0 + (kb + 1) * 64
            nrt = rows // 64 - kb - 1
            pan += nrt * (2 * 64 ** 3 + 2 * 64 ** 3 / 3)
            c0 = (kb + 1) * 64
            if c0 < sp:
                nn = sp - c0
                trail += 2 * 64 * (nn * (nn + 1) / 2 + (rows - sp) * nn)
    W["panel"] = pan
    W["trailing"] = trail
    if kind == "helmholtz":
        # blocked Gauss-Jordan of [S | T | I] over [T | T]: rank-64 updates of the top and bottom rows
        pan = trail = 0.0
        for j in range(NI):
            wt = (3 if j < NI - 1 else 2) * sp
            for kb in range(sp // 64):
                c0 = 64 * kb
                trail += 2.0 * sp * (wt - c0 - 64) * 64
                if j < NI - 1:
                    trail += 2.0 * sp * (2 * sp - c0 - 64) * 64
                pan += 2.0 * 64 * 64 * (wt - c0 - 64) + 2.0 * 64 ** 3
        W["panel"] = pan
        W["trailing"] = trail
        W["schur_update"] = 0.0
        W["sweep_products"] = passes * (3 * NI - 2) * 2.0 * sp * sp * k
        W["tree_up"] = passes * NS * k * sum(2 * (m * m + 2 * m * m + 2 * w * m) for (_, _, w) in nodes)
        W["tree_down"] = passes * NS * k * sum(2 * (2 * m * m + 2 * w * m) for (_, _, w) in nodes)
        W["stencil"] = passes * 24.0 * s * s * k
        W["tree_factor"] = NS * sum(2 * (2 * m ** 3 + 2 * m ** 3 + 4 * m ** 3 + 2 * w * 3 * m * m)
                                    for (_, _, w) in nodes)
        return W
    if stage2 == "oddeven":
        lv = oddeven_levels(NI)
        nb, nc = sum(x for x, _ in lv), sum(y for _, y in lv)
        W["schur_update"] = nb * (2.0 * sp ** 3 + sp * sp * (sp + 1.0)) + nc * (4.0 * sp ** 3 + sp * sp * (sp + 1.0))
        W["sweep_products"] = passes * (4 * nb + 2 * nc + 2) * 2.0 * sp * sp * k
    else:
        W["schur_update"] = (NI - 1) * sp * sp * (sp + 1.0)
        W["sweep_products"] = passes * (4 * NI - 2) * 2.0 * sp * sp * k
    # tree passes: compulsory HBM bytes only (a lower bound of the traffic): per node the FP32 factor
    # blocks L^-1 and Z_tb (3 m^2) and the interface columns Z_I (2 w m) once; per pass the up pass reads
    # the FP64 load of the slab interiors and writes y (m k FP32 per node), the down pass reads y and
    # writes the FP64 solution of the slab interiors -- and reads it too in the refinement passes, which
    # accumulate.  Intermediate condensed vectors and the interface values are left out (they may stay
    # in L2).
    nn = NS * len(nodes)
    fac = NS * sum(4 * 3 * m * m + 4 * 2 * w * m for (_, _, w) in nodes)
    uint = 8.0 * NS * s * m * k                                          # FP64 interior vector, one pass
    W["tree_up"] = passes * (fac + uint + 4.0 * nn * m * k)
    W["tree_down"] = passes * (fac + 4.0 * nn * m * k + uint) + (passes - 1) * uint
    W["stencil"] = passes * 24.0 * s * s * k                            # bytes: read u, f; write r (FP64)
    return W


BOUND = {"tree_factor": "alu", "assemble_T": "hbm", "panel": "alu", "trailing": "tensor",
         "schur_update": "tensor", "sweep_products": "tensor", "tree_up": "hbm", "tree_down": "hbm",
         "stencil": "hbm"}


BOUND3 = dict(BOUND, assemble_T="tensor", tree_up="tensor", tree_down="tensor", slab_panel="alu",
              slab_trailing="tensor", slab_schur="tensor")

# Measured DRAM bytes per pass (dram__bytes_read.sum + dram__bytes_write.sum summed over the 11
# height launches of one pass; one ncu capture of the 2-D diffusion workload, n = 2048, b = 32, k = 64,
# NVTX range profiled_step): the down pass moves more in the refinement passes, which read the FP64
# solution they accumulate into.  Other n at the same b and k scale with the node count, (n / 2048)^2.
TRAFFIC = {
    "tree_down": {"first": 6.997e9, "refine": 8.872e9, "n": 2048, "launches": 11,
                  "from": "ncu, n=2048: 6.997 GB first pass, 8.872 GB refinement pass, 11 launches each"},
    "tree_up": {"first": 10.246e9, "refine": 10.242e9, "n": 2048, "launches": 11,
                "from": "ncu, n=2048: 10.246 GB first pass, 10.242 GB refinement pass, 11 launches each"},
}
# How each tensor-core class multiplies (set per run in run_gpu): "f16x3" three FP16 MMAs of
# row-scaled hi/lo splits per algorithmic FP32 flop (the FP32 factor's Schur and trailing
# products), "tf32x3" three TF32 MMAs (3xTF32), "tf32" one TF32 MMA.
MMA_MODE = {}


def roofline_for(cls, ms, count, work, peaks, clocks, bounds=None):
    bound = (bounds or BOUND).get(cls, "alu")
    t = ms * 1e-3
    if bound == "hbm":
        achieved = work[cls] / t / 1e9
        peak = peaks.get("hbm_gbs", 6801.0)
        unit, src = "GB/s", "measured copy bandwidth (MEASURED_PEAKS.json)"
    elif bound == "tensor":
        achieved = work[cls] / t / 1e12
        bf16 = peaks.get("bf16_tflops", 1891.8)
        mode = MMA_MODE.get(cls, "tf32x3")
        if mode == "f16x3":
            peak = bf16
            src = ("measured bf16 dense (= fp16 dense rate); algorithmic FP32 flops, three FP16 MMAs of "
                   "row-scaled hi/lo splits per flop")
        else:
            peak = bf16 * 1.1 / 2.25
            src = ("measured bf16 dense x 1.1/2.25 (tf32 nominal ratio); algorithmic FP32 flops, "
                   + ("three TF32 MMAs per flop (3xTF32)" if mode == "tf32x3" else "one TF32 MMA per flop"))
        unit = "TFLOP/s"
    else:
        mhz = peaks.get("sm_max_mhz", 2070.0)
        achieved = work[cls] / t / 1e12
        peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        unit, src = "TFLOP/s", f"FP32 FMA issue rate {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {mhz:.0f} MHz"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": None, "kernel": cls, "launches": count, "avg_launch_us": ms * 1e3 / max(count, 1),
            "peak_source": src}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2211_07572_gb300 import inputs
    from paper_2211_07572_gb300.solver import SlabSolver

    W = dict({"helmholtz4096": HELMHOLTZ, "diffusion2048": WORKLOAD}.get(args.workload, DIFFUSION3D))
    helm = W["kind"] == "helmholtz"
    dim = 3 if W["kind"] == "diffusion3d" else 2
    if args.n:
        W.update(n=args.n, b=args.b or W["b"], k=args.k or W["k"])
        W["workload"] = (f"2D Helmholtz n={W['n']} b={W['b']} point source" if helm else
                         f"{'3D' if W['kind'] == 'diffusion3d' else '2D'} var-coef diffusion n={W['n']} b={W['b']} "
                         f"k={W['k']}")
    n, b, k = W["n"], W["b"], W["k"]
    dev = rank_device()
    rank, _, world = dist_env()
    if helm:
        p = inputs.helmholtz(n, b, dim=2, n_modes=8, field_seed=3)
        coeff = dict(kind=inputs.HELMHOLTZ, c=torch.from_numpy(p.c).to(dev), omega=p.omega)
        f_host = torch.from_numpy(np.ascontiguousarray(p.f[:k])).pin_memory()
    elif dim == 3:
        p = inputs.diffusion(n, b, k=0, dim=3, n_modes=8, field_seed=4, rhs_seed=104)
        coeff = dict(kind=inputs.DIFFUSION, kappa=torch.from_numpy(p.kappa).to(dev))
        f_host = torch.from_numpy(inputs.normal_rhs(3, n, k, 104)).pin_memory()
    else:
        p = inputs.diffusion(n, b, k=0, n_modes=16, field_seed=2, rhs_seed=102)
        coeff = dict(kind=inputs.DIFFUSION, kappa=torch.from_numpy(p.kappa).to(dev))
        f_host = torch.from_numpy(inputs.normal_rhs(2, n, k, 102)).pin_memory()
    f = f_host.to(dev)
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream(dev)
    prec = args.precision

    NI = n // b - 1
    MMA_MODE.clear()
    if prec == "tf32":
        MMA_MODE.update(schur_update="tf32", trailing="tf32", assemble_T="tf32", slab_trailing="tf32",
                        slab_schur="tf32")                     # factor products
    elif prec == "fp32" and not helm:
        MMA_MODE.update(schur_update="f16x3", trailing="f16x3", slab_trailing="f16x3", slab_schur="f16x3")
        if dim == 3:
            MMA_MODE["assemble_T"] = "f16x3"                    # 3-D T assembly products
    stage2 = "sweep" if helm else args.stage2          # "auto": the library's own choice (read back below)

    def solver(precision, **kw):
        kk = dict(coeff)
        kind = kk.pop("kind")
        return SlabSolver(dim, n, b, kind, precision=precision, stream=stream, device=dev, **kk, **kw)

    W["krylov"] = args.krylov

    iprec = None if args.interface == "default" else args.interface
    W["interface"] = args.interface

    def make():
        return solver(prec, rtol=W["rtol"], max_refine=40, stage2=stage2, krylov=args.krylov,
                      interface_precision=iprec)

    def step(f_in, u_out, counts=None, orders=None):
        s = make()
        if orders is not None:
            orders.append(s.stage2_order)               # the order the factor used ("auto" resolved)
        _, rel, it = s.solve(f_in, u_out, allow_noconv=True)
        if counts is not None:
            counts.append(sum(s.profile_read()[1].values()))
        s.close()
        return rel, it

    orders = []
    if args.once:
        # warm-up steps first (the tuner decides during them), then the step a profiler looks at, inside
        # the NVTX range "profiled_step" (ncu --nvtx --nvtx-include "profiled_step/")
        for _ in range(args.once_warmup):
            step(f, u)
        torch.cuda.synchronize()
        cnt = []
        torch.cuda.nvtx.range_push("profiled_step")
        rel, it = step(f, u, cnt, orders)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        W["stage2"] = orders[0]
        if rank == 0:
            print(json.dumps({"once": True, "config": W, "max_relres": float(np.max(rel)), "refine_steps": it,
                              "gpu_launches": cnt[0]}))
        return
    for _ in range(max(args.warmup, 1)):
        rel, it = step(f, u, orders=orders)
    stage2 = orders[0]
    W["stage2"] = stage2
    sampler = ClockSampler()
    sampler.start()
    dist_barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rels, its, launches = [], [], []
    for _ in range(args.steps):
        rel, it = step(f, u, launches)
        rels.append(float(np.max(rel)))
        its.append(it)
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    ms = dist_max(e0.elapsed_time(e1) / args.steps)
    # end to end through the public API with host buffers: H2D of f and D2H of u inside the region,
    # all on the compute stream: the load's copy, the factor and solve, the solution's copy, then the
    # handle is released.  (Overlapping the copy with the factor measured slower: the factor's device
    # allocations stall a copy in flight, 2.1 GB took 131 ms instead of 10 ms.)  Device staging buffers
    # for the load and the solution are allocated once, outside the region.
    u_host = torch.empty_like(f_host).pin_memory()
    fd = torch.empty_like(f)
    ud = torch.empty_like(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne2e = max(1, args.steps)
    parts = {"h2d_ms": [], "device_ms": [], "d2h_ms": [], "step_ms": []}
    for _ in range(ne2e):
        ts = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        fd.copy_(f_host, non_blocking=True)
        ev[1].record(stream)
        s_e2e = make()
        s_e2e.solve(fd, ud, allow_noconv=True)
        ev[2].record(stream)
        u_host.copy_(ud, non_blocking=True)
        ev[3].record(stream)
        s_e2e.close()
        torch.cuda.synchronize()
        parts["step_ms"].append((time.perf_counter() - ts) * 1e3)
        parts["h2d_ms"].append(ev[0].elapsed_time(ev[1]))
        parts["device_ms"].append(ev[1].elapsed_time(ev[2]))
        parts["d2h_ms"].append(ev[2].elapsed_time(ev[3]))
    e2e_s = dist_max((time.perf_counter() - t0) / ne2e)
    e2e_parts = {k: float(np.median(v)) for k, v in parts.items()}
    e2e_parts["host_ms"] = e2e_parts["step_ms"] - e2e_parts["h2d_ms"] - e2e_parts["device_ms"] - e2e_parts["d2h_ms"]
    e2e_parts["step_ms_spread"] = [float(min(parts["step_ms"])), float(max(parts["step_ms"]))]
    e2e_parts["note"] = ("medians per step on the compute stream: H2D of the loads; device = factor + solve (handle "
                         "setup and the refinement's host decisions included); D2H of the solution; host = the rest "
                         "of the wall time (releasing the handle)")
    sampler.stop()
    clocks = sampler.summary()

    # phase split from one plain step (events on the launch stream only), then per-kernel-class
    # device time from one profiled step (an event pair around every launch)
    t_f0 = torch.cuda.Event(enable_timing=True)
    t_fac = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_f0.record(stream)
    s = make()
    t_fac.record(stream)
    s.solve(f, u, allow_noconv=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    s.close()
    factor_ms = t_f0.elapsed_time(t_fac)
    solve_ms = t_fac.elapsed_time(t_end)
    s = solver(prec, rtol=W["rtol"], max_refine=40, profile=True, stage2=stage2, krylov=args.krylov,
               interface_precision=iprec)
    _, rel1, it1 = s.solve(f, u, allow_noconv=True)
    torch.cuda.synchronize()
    cls_ms, cls_cnt = s.profile_read()
    s.close()
    passes = it1 + 1
    work = work_model(n, b, k, passes, stage2, W["kind"])
    peaks = _peaks()
    bmap = BOUND3 if dim == 3 else BOUND
    dom = max((c for c in cls_ms if c in bmap and work.get(c, 0) > 0), key=lambda c: cls_ms[c])
    roof = roofline_for(dom, cls_ms[dom], cls_cnt[dom], work, peaks, clocks, bmap)
    if W["kind"] == "diffusion" and (b, k) == (32, 64) and dom in TRAFFIC and prec == "fp32":
        tr = TRAFFIC[dom]
        scale = (n / tr["n"]) ** 2                                      # nodes of the tree at fixed b
        per_pass = (tr["first"] + (passes - 1) * tr["refine"]) / passes * scale
        roof["traffic"] = per_pass / tr["launches"]
        roof["traffic_source"] = (tr["from"] + f"; mean over {passes} passes" +
                                  (f", x{scale:.2f} nodes at n={n}" if n != tr["n"] else "") +
                                  f", per tree launch ({tr['launches']} a pass)")
        roof["traffic_achieved"] = per_pass * passes / (cls_ms[dom] * 1e-3) / 1e9
        roof["traffic_frac"] = roof["traffic_achieved"] / roof["peak"]
    dense_cls = ("trailing", "schur_update", "sweep_products") + (
        ("assemble_T", "tree_up", "tree_down", "slab_trailing", "slab_schur") if dim == 3 else ())
    dense = {c: roofline_for(c, cls_ms[c], cls_cnt[c], work, peaks, clocks, bmap)
             for c in dense_cls if cls_ms.get(c, 0) > 0}
    # Stage 2 against the algorithmic count of Algorithm 1 in Cholesky form on the unpadded blocks, over
    # the measured time of every Stage-2 factor class (panels, trailing and Schur updates)
    si = (n - 1) ** (dim - 1)
    s2_ms = sum(cls_ms.get(c, 0.0) for c in ("panel", "trailing", "schur_update"))
    if s2_ms > 0 and not helm:
        a1 = alg1_cholesky_flops(si, NI)
        pk = peaks.get("bf16_tflops", 1891.8) * (1.0 if MMA_MODE.get("schur_update") == "f16x3" else 1.1 / 2.25)
        dense["stage2_alg1"] = {
            "bound": "tensor", "achieved": a1 / (s2_ms * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
            "frac": a1 / (s2_ms * 1e-3) / 1e12 / pk, "traffic": None, "ms": s2_ms, "flops": a1,
            "count": "Algorithm 1 in Cholesky form, unpadded s = (n-1)^(d-1): N_I s^3/3 + (N_I-1) 2 s^3",
            "order": stage2, "order_flops": work["panel"] + work["trailing"] + work["schur_update"],
            "peak_source": "measured bf16 dense (= fp16 dense rate)" if pk == peaks.get("bf16_tflops", 1891.8)
                           else "measured bf16 dense x 1.1/2.25 (tf32 nominal ratio)"}
    line = {
        "metric": METRIC,
        "value": ms / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32 factor (FP32-accurate tensor products: three FP16 products of row-scaled hi/lo "
                          "splits in the factor, 3xTF32 in the solve) / f64 residual+refinement",
                  "tf32": "f32 factor (single-pass TF32 tensor products) / f64 residual+refinement",
                  "fp64": "f64"}[prec] + ("" if iprec is None else f"; interface {iprec}"
                                            + (" (FP64-accurate tensor-core products)" if iprec == "fp64tc" else "")),
        "data": "synthetic",
        "config": dict(W, precision=prec, autotune=bool(args.autotune),
                       l2="every step streams > 10 GB (>> 129 MB L2); no explicit flush"),
        "max_relres": max(rels),
        "refine_steps": its,
        "phase_ms": {"factor": factor_ms, "solve_refine": solve_ms},
        "kernel_ms": {c: round(v, 3) for c, v in cls_ms.items()},
        "kernel_launches": cls_cnt,
        "roofline": roof,
        "dense_rooflines": dense,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(f_host.numel() * 8),
                "d2h_bytes_per_step": int(u_host.numel() * 8), "breakdown": e2e_parts},
        "gpu_launches": int(np.mean(launches)) if launches else None,
        "clocks": clocks,
    }
    if args.fp64_comparator and (prec != "fp64" or iprec is not None):
        line["fp64_gpu"] = fp64_comparator(
            lambda: solver("fp64", rtol=W["rtol"], max_refine=40, interface_precision="fp64"), f)
        line["fp64_gpu"]["mixed_speedup"] = line["fp64_gpu"]["value"] / line["value"]
    if world > 1:
        line["config"]["parallelism"] = f"replicas{world}"     # one problem per GPU, no data exchange
    if rank != 0:
        return
    line["config"]["host_numa"] = dict(HOST_NUMA)
    restore_host_affinity()                                  # the CPU baseline uses every core
    if args.cpu_baseline and world == 1:
        rungs = ((256, 1),) if helm else (((32, 3), (48, 1)) if dim == 3 else ((512, 3),))
        line["cpu_baseline"] = cpu_baseline(n, b, k, kind=W["kind"], rungs=rungs)
    print(json.dumps(line))


def fp64_comparator(make64, f):
    """Plain FP64 GPU path: same algorithm, all FP64, to the same relative residual.  One pass meets
    it for the diffusion workloads; the near-resonant Helmholtz cavity needs a few FP64 refinement
    passes (its FP64 factor alone leaves a relative residual of a few percent)."""
    import numpy as np
    import torch
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    steps = []

    def one():
        s = make64()
        _, rel, it = s.solve(f, u)
        s.close()
        steps.append(it)
        return rel

    one()                                                    # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rel = one()
    e1.record(stream)
    torch.cuda.synchronize()
    return {"value": e0.elapsed_time(e1) / 1e3, "unit": "s", "max_relres": float(np.max(rel)),
            "refine_steps": steps[-1],
            "path": "FP64 factor and solve on the same kernels (SIMT FP64), refined in FP64 to the same "
                    "relative residual (0 steps: one pass)"}


def cpu_sample(n_full, b, k, n_sample, kind="diffusion"):
    """One oracle run (banded LU, FP64) on a bounded sample of the workload: n = n_sample, same b and
    k loads, extrapolated to n_full by the banded-LU cost model (factor ~ N w^2, solve ~ k N w with
    N = n^d, w = n^(d-1)).  The Helmholtz sample keeps 10 points per wavelength and pivots.  The
    convection sample pivots and, like that workload's step, also factors A^T and solves the adjoint
    system (load 2 (u - u_t))."""
    import oracle
    from paper_2211_07572_gb300 import inputs
    oracle.build()
    dim = 3 if kind == "diffusion3d" else 2
    if kind == "helmholtz":
        p = inputs.helmholtz(n_sample, b, dim=2, n_modes=8, field_seed=3)
    elif kind == "convection":
        p = inputs.convection(n_sample, b, k)
    elif dim == 3:
        p = inputs.diffusion(n_sample, b, k=k, dim=3, n_modes=8, field_seed=4, rhs_seed=104)
    else:
        p = inputs.diffusion(n_sample, b, k=k, n_modes=16, field_seed=2, rhs_seed=102)
    piv = kind in ("helmholtz", "convection")
    w = (n_sample - 1) ** (dim - 1)
    t0 = time.perf_counter()
    A = oracle.assemble_problem(p)
    lu = oracle.BandLU(A, w, pivot=piv)
    lut = oracle.BandLU(A.transpose(), w, pivot=piv) if kind == "convection" else None
    t1 = time.perf_counter()
    u = lu.solve(p.f)
    if lut is not None:
        lut.solve(2.0 * (u - inputs.normal_rhs(2, n_sample, p.f.shape[0], 107)))
    t2 = time.perf_counter()
    rr = float(oracle.relres(A, u, p.f).max())
    scale = n_full / n_sample
    est = (t1 - t0) * scale ** (3 * dim - 2) + (t2 - t1) * scale ** (2 * dim - 1)
    return {"n": n_sample, "factor_s": t1 - t0, "solve_s": t2 - t1, "relres": rr, "est": est, "dim": dim,
            "cores": oracle.threads()}


def cpu_baseline(n_full, b, k, kind="diffusion", rungs=((512, 3),)):
    """The oracle timed on a ladder of bounded samples (n, repeats); the value is the median
    extrapolation of the largest rung, the spread of its repeats and the exponent the rungs show
    between them are reported beside it."""
    import statistics
    res = {}
    for n_s, rep in rungs:
        res[n_s] = [cpu_sample(n_full, b, k, n_s, kind) for _ in range(rep)]
    top = max(res)
    ests = [r["est"] for r in res[top]]
    dim = res[top][0]["dim"]
    parts = []
    for n_s in sorted(res):
        rs = res[n_s]
        parts.append(f"n={n_s}: factor {', '.join(f'{r['factor_s']:.2f}' for r in rs)} s, solve "
                     f"{statistics.median(r['solve_s'] for r in rs):.2f} s, relres {max(r['relres'] for r in rs):.1e}")
    lo = min(res)
    expo = ""
    if lo != top:
        f_lo = statistics.median(r["factor_s"] for r in res[lo])
        f_hi = statistics.median(r["factor_s"] for r in res[top])
        import math
        expo = f"; measured factor exponent n={lo}->{top}: {math.log(f_hi / f_lo) / math.log(top / lo):.2f}"
    return {"value": statistics.median(ests), "unit": "s", "cores": res[top][0]["cores"], "kind": "oracle",
            "spread": [min(ests), max(ests)],
            "sample": f"banded LU FP64 (b={b}, k={k}) on a ladder -- " + "; ".join(parts) +
                      f"; value = median over the n={top} repeats extrapolated to n={n_full} by n^{3 * dim - 2} "
                      f"(factor) and k n^{2 * dim - 1} (solve), spread {min(ests):.0f}-{max(ests):.0f} s" + expo}


def run_adjoint_batch(args):
    """Batched adjoint workload: 256 independent 2-D diffusion problems, n in {256, ..., 1024}, b = 16;
    per step every problem is factored, solved, its loss ||u - u_t||^2 formed and dL/dkappa computed by
    the adjoint solve.  Default: the CUDA-graph batch (slab_batch: everything allocated once, one graph
    launch per wave of problems); --no-graph: the stream-per-problem path (slab_factor_batched ...)."""
    import numpy as np
    import torch

    from paper_2211_07572_gb300 import inputs
    from paper_2211_07572_gb300.solver import GraphBatch, batched_adjoint_gradients
    dev = rank_device()
    rank, _, world = dist_env()
    sizes = inputs.adjoint_batch_sizes()
    count = args.count or len(sizes)
    sizes = [int(n) for n in sizes[:count]]
    data = [inputs.adjoint_instance(i, n) for i, n in enumerate(sizes)]
    prec = args.precision
    stream = torch.cuda.current_stream(dev)
    line_extra = {}
    if args.graph:
        t0 = time.perf_counter()
        gb = GraphBatch(sizes, b=16, precision=prec, rtol=1e-12, steps=args.graph_steps, wave=args.wave,
                        branches=args.branches)
        t_create = time.perf_counter() - t0
        host = []                                      # pinned host copies of every input
        for i, d in enumerate(data):
            hk = torch.from_numpy(d["kappa"]).pin_memory()
            hf = torch.from_numpy(d["f"]).pin_memory()
            ht = torch.from_numpy(d["u_target"]).pin_memory()
            host.append((hk, hf, ht))
            gb.set_inputs(i, hk.to(dev), hf.to(dev), ht.to(dev))
        torch.cuda.synchronize()

        def step():
            gb.run(stream)
            return gb.results()

        for _ in range(args.warmup):
            L, ru, rl = step()
        sampler = ClockSampler()
        sampler.start()
        dist_barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        worst = 0.0
        for _ in range(args.steps):
            L, ru, rl = step()
            worst = max(worst, float(ru.max()), float(rl.max()))
        e1.record(stream)
        torch.cuda.synchronize()
        dist_barrier()
        sec = dist_max(e0.elapsed_time(e1) / 1e3 / args.steps)
        # end to end: inputs from pinned host memory into the batch's buffers, every gradient back
        grads_host = [torch.empty((n + 1, n + 1), dtype=torch.float64).pin_memory() for n in sizes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for i, (hk, hf, ht) in enumerate(host):
                k_, f_, t_ = gb.inputs(i)
                k_.copy_(hk.view_as(k_), non_blocking=True)
                f_.copy_(hf.view_as(f_), non_blocking=True)
                t_.copy_(ht.view_as(t_), non_blocking=True)
            gb.run(stream)
            for i in range(count):
                grads_host[i].copy_(gb.outputs(i)[2], non_blocking=True)
            gb.results()
            torch.cuda.synchronize()
        e2e = dist_max((time.perf_counter() - t0) / args.steps)
        sampler.stop()
        h2d = sum(int(a.numel() + b_.numel() + c.numel()) * 8 for a, b_, c in host)
        d2h = sum(int(g.numel()) * 8 for g in grads_host)
        line_extra = {"e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                      "max_relres": worst, "graph": {"create_s": t_create, "device_bytes": gb.device_bytes,
                                                     "waves": (count + (args.wave or count) - 1) // (args.wave or count),
                                                     "branches": args.branches, "refine_steps": args.graph_steps}}
        losses = L
        gb.close()
        timing = "CUDA events around the graph launches and the results read (device-resident inputs)"
    else:
        probs, fs, uts = [], [], []
        for d, n in zip(data, sizes):
            probs.append(dict(dim=2, n=int(n), b=16, kind=inputs.DIFFUSION, kappa=d["kappa"]))
            fs.append(torch.from_numpy(d["f"]).to(dev))
            uts.append(torch.from_numpy(d["u_target"]).to(dev))

        def step(precision=prec):
            return batched_adjoint_gradients(probs, fs, uts, wave=args.wave or 32, workers=8, precision=precision)

        for _ in range(args.warmup):
            step()
        sampler = ClockSampler()
        sampler.start()
        dist_barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            losses, grads = step()
        torch.cuda.synchronize()
        dist_barrier()
        sec = dist_max((time.perf_counter() - t0) / args.steps)
        sampler.stop()
        timing = "host clock around device-synchronised steps (problems run on their own streams)"
    line = {
        "metric": "batched adjoint: factor+solve+adjoint+gradient s per batch",
        "value": sec, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32 factor (FP32-accurate tensor products) / f64 residual+refinement" if prec == "fp32"
                  else prec),
        "data": "synthetic",
        "config": {"workload": f"batched adjoint {count} x 2D diffusion n in {{256..1024}} b=16, L=||u-u_t||^2",
                   "count": count, "wave": args.wave, "precision": prec, "graph": bool(args.graph),
                   "timing": timing},
        "instances_per_s": count / sec,
        "mean_loss": float(np.mean(losses)),
        "clocks": sampler.summary(),
    }
    line.update(line_extra)
    if args.fp64_comparator and prec != "fp64" and not args.graph:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step("fp64")
        torch.cuda.synchronize()
        line["fp64_gpu"] = {"value": time.perf_counter() - t0, "unit": "s", "path": "same batch, FP64 factor"}
    if world > 1:
        line["config"]["parallelism"] = f"replicas{world}"
    if rank == 0:
        print(json.dumps(line))


def run_j0(args):
    """Second workload: constant-coefficient Helmholtz with Dirichlet data J_0(k |x - (-0.1, 0.5)|),
    n = 1024, b = 32, k = 27.1 (the first row of the paper's second-order FD table, Sec. 6.2).  A step
    is: factor, move the boundary data into the load (slab_boundary_lift), solve with refinement."""
    import numpy as np
    import torch

    from paper_2211_07572_gb300 import inputs
    from paper_2211_07572_gb300.solver import SlabSolver
    dev = rank_device()
    rank, _, world = dist_env()
    n, b = args.n or 1024, args.b or 32
    d = inputs.bessel_j0(n, b)
    p = d["problem"]
    c = torch.from_numpy(p.c).to(dev)
    g_host = torch.from_numpy(d["g"]).pin_memory()
    g = g_host.to(dev)
    prec = args.precision
    stream = torch.cuda.current_stream(dev)

    def step(gd, counts=None):
        s = SlabSolver(2, n, b, p.kind, c=c, omega=p.omega, precision=prec, rtol=1e-10, max_refine=40,
                       stream=stream, device=dev)
        fd = s.boundary_lift(gd)
        u, rel, it = s.solve(fd, allow_noconv=True)
        if counts is not None:
            counts.append(sum(s.profile_read()[1].values()))
        s.close()
        return u, rel, it

    for _ in range(args.warmup):
        step(g)
    sampler = ClockSampler()
    sampler.start()
    dist_barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches, its, rels = [], [], []
    for _ in range(args.steps):
        u, rel, it = step(g, launches)
        its.append(it)
        rels.append(float(np.max(rel)))
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    ms = dist_max(e0.elapsed_time(e1) / args.steps)
    # end to end: boundary data from pinned host memory, solution back to pinned host memory
    u_host = torch.empty((1, (n - 1) ** 2), dtype=torch.float64).pin_memory()
    gd = torch.empty_like(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gd.copy_(g_host, non_blocking=True)
        u, _, _ = step(gd)
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e = dist_max((time.perf_counter() - t0) / args.steps)
    sampler.stop()
    err = float(np.linalg.norm(u_host.numpy() - d["u_true"]) / np.linalg.norm(d["u_true"]))
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32 slab trees, f64 interface, f64 refinement"}.get(prec, prec),
        "data": "synthetic",
        "config": {"workload": f"2D constant-coefficient Helmholtz n={n} b={b} wavenumber 27.1, Dirichlet data "
                               "J_0(k|x-(-0.1,0.5)|), zero load", "n": n, "b": b, "precision": prec,
                   "l2": "every step streams > 1 GB (>> 129 MB L2); no explicit flush"},
        "max_relres": max(rels), "refine_steps": its, "relerr_true": err,
        "paper_relerr_true_N1M": 1.8e-3,
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(g_host.numel() * 8),
                "d2h_bytes_per_step": int(u_host.numel() * 8)},
        "gpu_launches": launches[-1] if launches else None,
        "clocks": sampler.summary(),
    }))


def run_reference(args):
    """The reference arm: the oracle (banded LU) timed as it stands on the host cores, each step one
    bounded sample of the default workload (3-D diffusion, n = ref_n) extrapolated to n = 96."""
    W = DIFFUSION3D
    n, b, k = W["n"], W["b"], W["k"]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        cpu_sample(n, b, k, 16, kind=W["kind"])
    for _ in range(args.steps):
        vals.append(cpu_sample(n, b, k, args.ref_n, kind=W["kind"]))
    import statistics
    ests = [x["est"] for x in vals]
    v = statistics.mean(ests)
    cb = {"value": v, "unit": "s", "cores": vals[0]["cores"], "kind": "oracle", "spread": [min(ests), max(ests)],
          "sample": f"banded LU FP64 at n={args.ref_n} (b={b}, k={k}) per step, factor "
                    f"{statistics.median(x['factor_s'] for x in vals):.2f} s median; extrapolated to n={n} by n^7 "
                    f"(factor) and k n^5 (solve)"}
    print(json.dumps({
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": dict(W, impl="CPU oracle banded LU, extrapolated from a bounded sample"),
        "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t0}))


def run_convection(args):
    """Nonsymmetric workload: 2-D convection-diffusion -div(kappa grad u) + beta.grad u = f, n = 2048,
    b = 32, 16 loads, kappa = exp(16-mode field), |beta| <= 20 (8-mode fields).  A step is: factor, solve
    with refinement to 1e-10, the adjoint solve A^T lambda = 2 (u - u_t) on the same factors (every
    phase transposed) refined to 1e-10, and the gradient dL/dkappa of L = ||u - u_t||^2."""
    import numpy as np
    import torch

    from paper_2211_07572_gb300 import inputs
    from paper_2211_07572_gb300.solver import SlabSolver
    dev = rank_device()
    rank, _, world = dist_env()
    n, b, k = args.n or 2048, args.b or 32, args.k or 16
    p = inputs.convection(n, b, k)
    kappa = torch.from_numpy(p.kappa).to(dev)
    beta = torch.from_numpy(p.beta).to(dev)
    f_host = torch.from_numpy(p.f).pin_memory()
    ut_host = torch.from_numpy(inputs.normal_rhs(2, n, k, 107)).pin_memory()
    f, ut = f_host.to(dev), ut_host.to(dev)
    stream = torch.cuda.current_stream(dev)

    def step(fd, utd, prec=args.precision, counts=None, pivot=args.pivot, profile=False, split=None):
        s = SlabSolver(2, n, b, inputs.CONVECTION, kappa=kappa, beta=beta, precision=prec, rtol=1e-10,
                       max_refine=40, stream=stream, device=dev, pivot=pivot, profile=profile)
        if split is not None:
            split[1].record(stream)
        u, rel, it = s.solve(fd, allow_noconv=True)
        if split is not None:
            split[2].record(stream)
        lam, g = s.adjoint(2 * (u - utd), u, allow_noconv=True)
        if split is not None:
            split[3].record(stream)
        if counts is not None:
            counts.append(sum(s.profile_read()[1].values()))
        if profile:
            cls_ms, cls_cnt = s.profile_read()
            s.close()
            return cls_ms, cls_cnt
        s.close()
        return u, lam, g, rel, it

    for _ in range(args.warmup):
        step(f, ut)
    sampler = ClockSampler()
    sampler.start()
    dist_barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches, its, rels = [], [], []
    for _ in range(args.steps):
        u, lam, g, rel, it = step(f, ut, counts=launches)
        its.append(it)
        rels.append(float(np.max(rel)))
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    ms = dist_max(e0.elapsed_time(e1) / args.steps)
    # adjoint accuracy: relative residual of A^T lambda = 2 (u - u_t) in FP64
    s = SlabSolver(2, n, b, inputs.CONVECTION, kappa=kappa, beta=beta, precision=args.precision, stream=stream,
                   device=dev)
    rhs = 2 * (u - ut)
    adj_rel = float(((rhs - s.apply_transpose(lam)).norm(dim=1) / rhs.norm(dim=1)).max())
    s.close()
    # end to end: loads and targets from pinned host memory, u and the gradient back
    u_host = torch.empty_like(f_host).pin_memory()
    g_host = torch.empty((n + 1, n + 1), dtype=torch.float64).pin_memory()
    fd, utd = torch.empty_like(f), torch.empty_like(ut)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fd.copy_(f_host, non_blocking=True)
        utd.copy_(ut_host, non_blocking=True)
        u, lam, g, _, _ = step(fd, utd)
        u_host.copy_(u, non_blocking=True)
        g_host.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
    e2e = dist_max((time.perf_counter() - t0) / args.steps)
    sampler.stop()
    # one step split into factor / solve / adjoint + gradient, and one with every launch timed by class
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    step(f, ut, split=ev)
    torch.cuda.synchronize()
    phases = {"factor": ev[0].elapsed_time(ev[1]), "solve": ev[1].elapsed_time(ev[2]),
              "adjoint_and_gradient": ev[2].elapsed_time(ev[3])}
    cls_ms, cls_cnt = step(f, ut, profile=True)
    other_pivot = "local" if args.pivot == "tournament" else "tournament"
    torch.cuda.synchronize()
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    _, _, _, rel_v, it_v = step(f, ut, pivot=other_pivot)
    v1.record(stream)
    torch.cuda.synchronize()
    variant = {"pivot": other_pivot, "ms_per_step": v0.elapsed_time(v1), "max_relres": float(np.max(rel_v)),
               "refine_steps": it_v}
    fp64 = None
    if args.fp64_comparator:
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        step(f, ut, prec="fp64")
        a1.record(stream)
        torch.cuda.synchronize()
        fp64 = dist_max(a0.elapsed_time(a1)) / 1e3
    if rank != 0:
        return
    cpu = None
    if args.cpu_baseline and world == 1:
        restore_host_affinity()                                  # the CPU baseline uses every core
        cpu = cpu_baseline(n, b, k, kind="convection", rungs=((128, 2), (256, 2)))
    print(json.dumps({
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32 factor (slab trees, interface), f64 residual + refinement"}.get(args.precision,
                                                                                               args.precision),
        "data": "synthetic",
        "config": {"workload": f"2D convection-diffusion n={n} b={b} k={k} (kappa=exp(16-mode field), "
                               "|beta|<=20 8-mode fields, f~N(0,1)); step = factor + solve + transposed adjoint "
                               "solve + dL/dkappa", "n": n, "b": b, "k": k, "precision": args.precision,
                   "pivot": args.pivot,
                   "l2": "every step streams > 1 GB (>> 129 MB L2); no explicit flush"},
        "max_relres": max(rels), "refine_steps": its, "adjoint_max_relres": adj_rel, "pivot": args.pivot,
        "phases_ms": phases, "classes_ms": {c: round(v, 3) for c, v in cls_ms.items() if v > 0},
        "classes_launches": {c: v for c, v in cls_cnt.items() if v > 0}, "other_pivot": variant,
        "fp64_gpu": {"value": fp64, "unit": "s"} if fp64 is not None else None,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(2 * f_host.numel() * 8),
                "d2h_bytes_per_step": int(u_host.numel() * 8 + g_host.numel() * 8)},
        "gpu_launches": launches[-1] if launches else None,
        "clocks": sampler.summary(),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "tf32"],
                    help="factor precision (default fp32; helmholtz4096: fp64 slab trees with the FP64-accurate "
                         "tensor-core interface, since an FP32 factor does not converge at 10 points per wavelength "
                         "and n >= 512)")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--b", type=int, default=0)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--ref-n", type=int, default=32, help="reference arm: oracle sample size (3-D)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-fp64", dest="fp64_comparator", action="store_false")
    ap.add_argument("--once", action="store_true",
                    help="warm-up steps, then one step in the NVTX range profiled_step (for profilers)")
    ap.add_argument("--once-warmup", type=int, default=3, help="--once: warm-up steps before the profiled one")
    ap.add_argument("--count", type=int, default=0, help="adjoint256: number of problems (0: all 256)")
    ap.add_argument("--wave", type=int, default=64, help="adjoint256: problems per wave (graph: per graph)")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="adjoint256: stream-per-problem path instead of the CUDA-graph batch")
    ap.add_argument("--graph-steps", type=int, default=4, help="adjoint256 graph: refinement passes per solve")
    ap.add_argument("--branches", type=int, default=32, help="adjoint256 graph: parallel branches per wave")
    ap.add_argument("--workload", default="diffusion3d96",
                    choices=["diffusion2048", "helmholtz4096", "diffusion3d96", "adjoint256", "helmholtzj0",
                             "convection2048"],
                    help="diffusion3d96: the default bench line (3-D diffusion n=96, b=8, k=16); diffusion2048, "
                         "helmholtz4096, adjoint256, helmholtzj0, convection2048: the other workloads")
    ap.add_argument("--krylov", type=int, default=0, help="0: plain refinement; m: FP64 GMRES(m) refinement")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the fixed size heuristic for the factor products instead of the online tuner "
                         "(which decides during the warm-up steps)")
    ap.add_argument("--interface", default="default", choices=["default", "fp32", "fp64", "fp64tc", "tf32"],
                    help="precision of the interface system (fp64tc: FP64-accurate tensor-core products)")
    ap.add_argument("--pivot", default="tournament", choices=["tournament", "local"],
                    help="convection2048: row choice of the Gauss-Jordan interface elimination")
    ap.add_argument("--stage2", default="auto", choices=["auto", "sweep", "oddeven"],
                    help="elimination order of T (auto: odd-even for 4 or more interfaces)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp32"
        if args.workload == "helmholtz4096":
            args.precision = "fp64"
            if args.interface == "default":
                args.interface = "fp64tc"
    if args.gpus != dist_env()[2] and dist_env()[2] > 1:
        raise SystemExit(f"--gpus {args.gpus} but the launcher started {dist_env()[2]} ranks")
    if args.impl != "reference":
        from paper_2211_07572_gb300 import _lib
        _lib.load().slab_autotune(1 if args.autotune else 0)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint256":
        run_adjoint_batch(args)
    elif args.workload == "helmholtzj0":
        run_j0(args)
    elif args.workload == "convection2048":
        run_convection(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
