#!/usr/bin/env python3
"""Benchmark of the B300 TDA-BSE hot path (one JSON line on rank 0).

A step is one pass of the whole path over the split-precision-at-scale workload (2-atom
diamond-like cell, 13 NAOs and 75 ABFs per atom, 4x4x4 coarse / 12x12x12 dense mesh,
Nv = Nc = 4, H dimension 27648):
  (a) W(q) interpolation, (b) per-k projection stage, (b+c) assembly of H, the dipole
  vector, and (d) a 500-step Haydock spectrum for 3 polarisations on 1001 frequencies.
value = H elements (dim^2) per second of whole step; the assembly-only rate, the FP64
GPU path, the accuracy against the FP64 path and the stage breakdown are extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision bf16x3|bf16x2|bf16x1|tf32x2|fp64]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_BSE elements/s (split-prec TC vs FP64 GPU) at ≤1 meV lowest-exciton error"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per 128x128 tile of the current
# Hermitian matvec kernel, from one ncu capture of the 16000-dim case (7875 tiles):
# 1.032827 GB read (the tiles themselves) + 45.72 MB written (the partial slots).
MV_DRAM_BYTES_PER_TILE = (1.032827e9 + 45.723136e6) / 7875
# DRAM bytes per transfer q of the split assembly's two slab kernels, from ncu captures of one
# 20-q slab of the 16000-dim case (10^3 k-points, N_aux 150, Nv = Nc = 4): the projections
# (313.4 MB read, 922.3 MB written: the M_vv bf16 pieces and M_cc) and the fused direct term
# in its column-half form (1078.0 MB read, 71.3 MB written).  Both grow in proportion to the
# k-points per q.
ASM_DRAM_BYTES_PER_Q_MESH10 = ((313.358848e6 + 922.320640e6) + (1077.953e6 + 71.327744e6)) / 20
UNIT = "H elements/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--haydock-steps", type=int, default=500)
    ap.add_argument("--n-omega", type=int, default=1001)
    ap.add_argument("--eta", type=float, default=0.1)
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip the FP64 GPU comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--small", action="store_true", help="tiny workload (for profiling captures)")
    ap.add_argument("--mesh", type=int, default=0, help="override the dense mesh N x N x N (profiling captures)")
    ap.add_argument("--no-full-bse", action="store_true", help="skip the full-BSE (coupling block) report")
    ap.add_argument("--full-bse-only", action="store_true",
                    help="print only the full-BSE report (for profiling captures of its kernels)")
    ap.add_argument("--no-matfree", action="store_true", help="skip the matrix-free spectrum report")
    ap.add_argument("--no-finite-q", action="store_true",
                    help="skip the finite exciton momentum H(Q) assembly report")
    ap.add_argument("--batch16", action="store_true",
                    help="add the 16-uneven-crystal batch (one CUDA graph) report under 'batched_uneven'")
    return ap.parse_args()


# Nominal dense tensor rates of the part (B300: tf32 1.1, bf16 2.25 PFLOP/s): a tf32 contraction
# takes the measured bf16 peak times their ratio.
TF32_PER_BF16 = 1.1 / 2.25
PIECE_PRODUCTS = {"bf16x3": 6, "bf16x2": 3, "bf16x1": 1, "tf32x2": 3}


def tensor_peak(pk, precision, key="bf16_tflops_sustained"):
    return pk[key] * (TF32_PER_BF16 if precision == "tf32x2" else 1.0)


def tf32x2_report(inp, d, spec, ctx, H64, w_d, prof, pk, args):
    """The same workload assembled with two tf32 pieces per operand (BSE_TF32X2: 3 kind::tf32
    products instead of bf16x3's 6 bf16 ones): assembly time, the M_vv W(q) kernel's tensor
    rate against bf16x3's, and its errors against the FP64 GPU path (outside the timed region)."""
    import torch
    from paper_2607_05853_b300.api import BSE
    st = torch.cuda.current_stream()
    dim2 = float(ctx.dim) ** 2
    c3 = BSE.from_inputs(inp, precision="tf32x2")
    H3 = torch.empty((ctx.dim, ctx.dim), dtype=torch.complex64, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):                      # the first pass warms up
        if rep == 1:
            c3.profile(True)
        a.record(st)
        c3.interp_W(d["W_R"], d["V0"])
        c3.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        c3.assemble(H3)
        b.record(st)
        c3.sync()
    tf_ms = a.elapsed_time(b)
    g1_tf, _ = c3.profile_read("g1")
    ex_tf, _ = c3.profile_read("exch")
    c3.profile(False)
    diff = H3.to(torch.complex128) - H64
    dmax = diff.abs().max().item()
    del diff
    w_t, r_t = c3.lowest(H3, 10, 300)
    c3.sync()
    nk, naux, nv = spec.n_k, spec.n_aux, spec.nv
    nq_half = (nk + sum(1 for q in range(nk) if _self_conj(q, spec.dense))) // 2
    g1_mac = 8.0 * nq_half * nk * nv * nv * naux * naux
    per = max(1, args.steps)
    g1_bf = prof["g1"][0] / per
    tf_peak, bf_peak = tensor_peak(pk, "tf32x2"), tensor_peak(pk, "bf16x3")
    out = {"assembly_ms": tf_ms, "elements_per_s": dim2 / (tf_ms / 1000.0),
           "g1_ms": g1_tf, "g1_ms_bf16x3": g1_bf, "exchange_ms": ex_tf,
           "g1_tensor_tflops": g1_mac * 3 / (g1_tf * 1e-3) / 1e12,
           "g1_tensor_frac": g1_mac * 3 / (g1_tf * 1e-3) / 1e12 / tf_peak,
           "g1_tensor_tflops_bf16x3": g1_mac * 6 / (g1_bf * 1e-3) / 1e12,
           "g1_tensor_frac_bf16x3": g1_mac * 6 / (g1_bf * 1e-3) / 1e12 / bf_peak,
           "tensor_peak_tf32": tf_peak,
           "peak_source": pk["source"] + " (sustained bf16 x nominal tf32/bf16 ratio 1.1/2.25)",
           "max_abs_dH_eV": dmax, "lowest10_abs_err_meV": (1000.0 * (w_t - w_d).abs()).tolist(),
           "note": "the bench workload with two tf32 pieces per FP32 operand (3 kind::tf32 products) instead of "
                   "bf16x3 (6 bf16 products); g1 = the M_vv W(q) kernel (fused with the second contraction "
                   "where N_aux <= 160); errors against the FP64 GPU path"}
    del H3
    c3.close()
    return out


def workload(small, mesh=0):
    import dataclasses
    from synth import config_spec
    spec = config_spec(0 if small else 2)
    if mesh:
        spec = dataclasses.replace(spec, dense=(mesh, mesh, mesh), name=f"{spec.name}-mesh{mesh}")
    return spec


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "source": "fallback"}


# ------------------------------------------------------------------------------ oracle leg
def cpu_baseline(inp, seconds, rng_seed=5):
    """The FP64 oracle, as it stands, on a bounded sample of H blocks of the same workload."""
    import oracle as O
    orc = O.BSEOracle(inp)
    rng = np.random.default_rng(rng_seed)
    nk = orc.nk
    k1s = rng.integers(0, nk, 4)
    n = 0
    t0, c0 = time.perf_counter(), time.process_time()
    while time.perf_counter() - t0 < seconds:
        k1 = int(k1s[n % 4])
        k2 = int(rng.integers(0, nk))
        orc.block(k1, k2)
        n += 1
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    try:
        import threadpoolctl
        pool = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or 1
    except Exception:
        pool = None
    used = cpu / dt if dt > 0 else 1.0      # threads actually busy on average (process CPU time / wall time)
    elems = n * orc.nvc * orc.nvc
    return {"value": elems / dt, "unit": UNIT, "cores": max(1, int(round(used))), "kind": "oracle",
            "host_cores": os.cpu_count(), "blas_pool_threads": pool, "threads_busy_avg": round(used, 2),
            "sample": f"{n} H blocks ({elems} elements) of the 27648-dim workload, W(q) and C(k) "
                      f"memoised per block as the oracle does, {dt:.1f} s on host cores (assembly only: "
                      f"the GPU line's value also includes the spectrum)"}


def _qplus(mesh):
    """One of each q / -q pair of the mesh (self-conjugate q once): the transfers the assembly
    computes."""
    n1, n2, n3 = (int(x) for x in mesh)
    seen, out = set(), []
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                q = (a, b, c)
                if q in seen:
                    continue
                mq = ((n1 - a) % n1, (n2 - b) % n2, (n3 - c) % n3)
                seen.add(q)
                seen.add(mq)
                out.append(q)
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks, returned on every rank (the job's wall time is that of
    its slowest rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, units_per_step: float, t_max_ms: float) -> float:
    """Whole-job rate: every rank processes units_per_step per step (weak scaling)."""
    return world * steps * units_per_step / (t_max_ms / 1000.0)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import make_inputs
    spec = workload(args.small, args.mesh)
    inp = make_inputs(spec)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(inp, min(per_step, 5.0))
    vals = [cpu_baseline(inp, per_step, rng_seed=100 + s) for s in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    cb = dict(vals[0])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * spec.dim ** 2 / v,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator, shapes of the paper's Si/MgO workloads)",
           "config": {"workload": spec.name, "dim": spec.dim, "n_k": spec.n_k, "n_aux": spec.n_aux,
                      "n_ao": spec.n_ao, "nv": spec.nv, "nc": spec.nc},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------------------ our path
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    from paper_2607_05853_b300.api import BSE, launch_count
    from synth import make_inputs

    spec = workload(args.small, args.mesh)
    dev = torch.device("cuda", local)
    if args.full_bse_only:
        omega = torch.linspace(0.0, 10.0, args.n_omega, dtype=torch.float64, device=dev)
        dim = spec.n_k * spec.nv * spec.nc
        print(json.dumps({"full_bse": full_bse_report(spec, args, dev, min(args.haydock_steps, 2 * dim), omega,
                                                      peaks())}))
        return
    inp = make_inputs(spec)

    def h2d(x, dt):
        return torch.from_numpy(np.ascontiguousarray(x, dt)).pin_memory()

    host = {k: h2d(inp[k], np.float64) for k in ("W_R", "V0", "C_R", "e_qp", "e_ks")}
    host.update({k: h2d(inp[k], np.complex128) for k in ("c_k", "vel")})
    d = {k: v.to(dev) for k, v in host.items()}
    ctx = BSE.from_inputs(inp, precision=args.precision)
    H = torch.empty((ctx.dim, ctx.dim), dtype=ctx.h_dtype, device=dev)
    u = torch.empty((3, ctx.dim), dtype=torch.complex128, device=dev)
    omega = torch.linspace(0.0, 10.0, args.n_omega, dtype=torch.float64, device=dev)
    eps2 = torch.empty(args.n_omega, dtype=torch.float64, device=dev)
    pref = 4.0 * np.pi ** 2 / (3.0 * spec.n_k * float(inp["volume"]))
    nsteps = min(args.haydock_steps, ctx.dim)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()

    def step(dd=d):
        ctx.interp_W(dd["W_R"], dd["V0"])
        ctx.project_pairs(dd["C_R"], dd["c_k"], dd["e_qp"])
        ctx.assemble(H)
        ctx.dipole_vector(dd["vel"], dd["e_ks"], u)
        ctx.spectrum(H, u, nsteps, omega, args.eta, pref, eps2)

    for _ in range(args.warmup):
        step()
    ctx.sync()

    # ---- timed region: K steps, L2 flushed between steps (outside the events) ----------
    ctx.profile(True)
    launches0 = launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sub = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(st)
            ctx.interp_W(d["W_R"], d["V0"])
            ctx.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
            sub[i][0].record(st)
            ctx.assemble(H)
            sub[i][1].record(st)
            ctx.dipole_vector(d["vel"], d["e_ks"], u)
            ctx.spectrum(H, u, nsteps, omega, args.eta, pref, eps2)
            ev[i][1].record(st)
        torch.cuda.synchronize()
    launches = launch_count() - launches0
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    pre_ms = [ev[i][0].elapsed_time(sub[i][0]) for i in range(args.steps)]
    asm_ms = [sub[i][0].elapsed_time(sub[i][1]) for i in range(args.steps)]
    spec_ms = [sub[i][1].elapsed_time(ev[i][1]) for i in range(args.steps)]
    prof = {k: ctx.profile_read(k) for k in ("interp", "half", "project", "g1", "g2", "exch", "matvec", "reorth")}
    ctx.profile(False)
    t_total = sum(step_ms)
    if world > 1:
        t_total = max_over_ranks(t_total, dist, dev)
    dim2 = float(ctx.dim) ** 2
    value = job_throughput(world, args.steps, dim2, t_total)
    asm_rate = dim2 / (statistics.mean([p + a for p, a in zip(pre_ms, asm_ms)]) / 1000.0)

    # ---- end to end: host inputs -> device -> path -> eps2 back to host ----------------
    h_out = torch.empty(args.n_omega, dtype=torch.float64).pin_memory()
    in_bytes = sum(v.numel() * v.element_size() for v in host.values())
    e2e_ms = []
    for i in range(max(1, min(args.steps, 2))):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        dd = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        step(dd)
        h_out.copy_(eps2, non_blocking=True)
        b.record(st)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e = {"value": dim2 / (statistics.mean(e2e_ms) / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
           "d2h_bytes_per_step": int(h_out.numel() * 8)}

    # ---- roofline of the dominant kernel ----------------------------------------------------
    pk = peaks()
    top = max(prof, key=lambda k: prof[k][0])
    ms, n = prof[top]
    per_launch_ms = ms / max(n, 1)
    h_elem = 16 if args.precision == "fp64" else 8
    nk, naux, nv, nc = spec.n_k, spec.n_aux, spec.nv, spec.nc
    if top == "matvec":
        if args.precision == "fp64" or ctx.dim % 2:
            alg = dim2 * h_elem + 3 * ctx.dim * 16 * 2
            roof_note = "Lanczos matvec (full read): algorithmic bytes = dim^2 x H element + 3 vectors in/out"
        else:
            HT = 128
            nbt = (ctx.dim + HT - 1) // HT
            ntiles = nbt * (nbt + 1) // 2
            alg = ntiles * HT * HT * h_elem
            roof_note = ("Lanczos matvec k_hmv_tma, Hermitian half read: algorithmic bytes = the upper-triangle "
                         "128x128 tiles of the complex64 H (the only part the method must read), per launch; "
                         "traffic = DRAM read+write bytes per tile from an ncu capture of the 16000-dim case "
                         "(7875 tiles) times this launch's tile count")
        roof = {"bound": "hbm", "achieved": alg / (per_launch_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
        if args.precision != "fp64" and ctx.dim % 2 == 0:
            roof["traffic"] = MV_DRAM_BYTES_PER_TILE * ntiles
    elif top == "g1" and args.precision != "fp64":
        pieces = PIECE_PRODUCTS[args.precision]
        alg = 8.0 * nk * nv * nv * naux * naux * pieces * (ctx_slab_q(ctx, spec))
        roof = {"bound": "tensor", "achieved": alg / (per_launch_ms * 1e-3) / 1e12,
                "peak": tensor_peak(pk, args.precision), "unit": "TFLOP/s"}
        roof_note = "M_vv W(q): executed tensor flops (8 N_k Nv^2 Naux^2 x split products) per launch"
    else:
        alg = None
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s"}
        roof_note = f"dominant kernel {top}"
    if roof.get("achieved") is not None and roof.get("peak"):
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        roof["frac"] = None
    roof.setdefault("traffic", None)
    roof["kernel"] = top
    # tensor-pipe fraction of the split-precision assembly GEMMs (executed bf16 products:
    # 8 real flops per complex MAC x the kept piece products; M_vv W(q) over the unique q of
    # each q/-q pair, the exchange over the full square)
    tensor = None
    if args.precision != "fp64":
        pieces = PIECE_PRODUCTS[args.precision]
        nq_half = (nk + sum(1 for q in range(nk) if _self_conj(q, spec.dense))) // 2
        g1_flops = 8.0 * nq_half * nk * nv * nv * naux * naux * pieces
        ex_flops = 8.0 * float(ctx.dim) ** 2 * naux * pieces
        g1_ms, g1_n = prof["g1"]
        g2_ms, g2_n = prof["g2"]
        ex_ms, ex_n = prof["exch"]
        if g1_n and ex_n:
            per = max(1, args.steps)
            a_g1 = g1_flops / ((g1_ms / per) * 1e-3) / 1e12
            a_ex = ex_flops / ((ex_ms / per) * 1e-3) / 1e12
            asm_s = statistics.mean([p + a for p, a in zip(pre_ms, asm_ms)]) * 1e-3
            sus = tensor_peak(pk, args.precision)
            fused = g2_n == 0
            tensor = {"bound": "tensor", "unit": "TFLOP/s", "peak": sus,
                      "peak_source": pk["source"] + (" (sustained bf16 x nominal tf32/bf16 ratio 1.1/2.25)"
                                                     if args.precision == "tf32x2" else " (sustained bf16)"),
                      "g1_achieved": a_g1, "g1_frac": a_g1 / sus,
                      "exchange_achieved": a_ex, "exchange_frac": a_ex / sus,
                      "assembly_achieved": (g1_flops + ex_flops) / asm_s / 1e12,
                      "assembly_frac": (g1_flops + ex_flops) / asm_s / 1e12 / sus,
                      "direct_fused": fused,
                      "note": "executed tensor flops per step = 8 x complex MACs x piece products; g1 = the M_vv W(q) "
                              "GEMM" + (" fused with the second contraction T M_cc^T and the H update (its time "
                                        "includes that CUDA-core epilogue)" if fused else "") +
                              "; assembly = per-k stage + projections + every GEMM, with the tensor-core flops of "
                              "M_vv W(q) and the exchange"}
    roof["peak_source"] = pk["source"]
    roof["note"] = roof_note

    # ---- FP64 GPU comparison and accuracy (outside the timed region) ----------------------
    extra = {}
    if not args.no_fp64_compare and args.precision != "fp64":
        ref = BSE.from_inputs(inp, precision="fp64")
        H64 = torch.empty((ctx.dim, ctx.dim), dtype=torch.complex128, device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ref.interp_W(d["W_R"], d["V0"])
        ref.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        ref.assemble(H64)
        b.record(st)
        ref.sync()
        fp64_ms = a.elapsed_time(b)
        dH = (H.to(torch.complex128) - H64).abs().max().item()
        fro = torch.linalg.matrix_norm(H.to(torch.complex128) - H64).item()
        w_s, r_s = ctx.lowest(H, 10, 300)
        w_d, r_d = ref.lowest(H64, 10, 300)
        ref.sync()
        eps64 = torch.empty_like(eps2)
        u64 = ref.dipole_vector(d["vel"], d["e_ks"])
        ref.spectrum(H64, u64, nsteps, omega, args.eta, pref, eps64)
        ref.sync()
        l2 = (torch.linalg.norm(eps2 - eps64) / torch.linalg.norm(eps64)).item()
        extra["fp64_gpu"] = {"assembly_ms": fp64_ms, "elements_per_s": dim2 / (fp64_ms / 1000.0),
                             "speedup_split_over_fp64": (dim2 / (fp64_ms / 1000.0)) and asm_rate / (dim2 / (fp64_ms / 1000.0))}
        extra["accuracy_vs_fp64"] = {"max_abs_dH_eV": dH, "frobenius_dH_eV": fro,
                                     "lowest10_abs_err_meV": (1000.0 * (w_s - w_d).abs()).tolist(),
                                     "lowest10_eV": w_d.tolist(), "ritz_resid_max_eV": float(max(r_s.max(), r_d.max())),
                                     "spectrum_rel_L2": l2}
        # the same split assembly with H stored complex128 (bse_params.h_complex128)
        c2 = BSE.from_inputs(inp, precision=args.precision, h_complex128=True)
        H2 = torch.empty((ctx.dim, ctx.dim), dtype=torch.complex128, device=dev)
        for rep in range(2):                      # the first pass warms up
            a.record(st)
            c2.interp_W(d["W_R"], d["V0"])
            c2.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
            c2.assemble(H2)
            b.record(st)
            c2.sync()
        c128_ms = a.elapsed_time(b)
        diff = H2 - H64
        dmax = diff.abs().max().item()
        ddiag = diff.diagonal().abs().max().item()
        w_c, r_c = c2.lowest(H2, 10, 300)
        c2.profile(True)
        eps_c = torch.empty_like(eps2)
        n_mv = 20
        c2.spectrum(H2, u64, n_mv, omega, args.eta, pref, eps_c)
        mv_ms, mv_n = c2.profile_read("matvec")
        c2.profile(False)
        c2.sync()
        mv_per = mv_ms / max(mv_n, 1)
        extra["split_h_complex128"] = {
            "assembly_ms": c128_ms, "elements_per_s": dim2 / (c128_ms / 1000.0),
            "max_abs_dH_eV": dmax, "max_abs_dH_diagonal_eV": ddiag,
            "lowest10_abs_err_meV": (1000.0 * (w_c - w_d).abs()).tolist(),
            "matvec_ms_per_step": mv_per,
            "matvec_roofline": {"bound": "hbm", "achieved": dim2 * 16 / (mv_per * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                                "unit": "GB/s", "frac": dim2 * 16 / (mv_per * 1e-3) / 1e9 / pk["hbm_gbs"]},
            "note": "bf16x3 assembly with H stored complex128 (diagonal E_c - E_v exact in FP64); its spectrum "
                    "reads the full complex128 H with the FP64 path's product (n_pol vectors per read), timed "
                    f"over {n_mv} Lanczos steps; errors against the FP64 GPU path"}
        del H2, diff
        c2.close()
        if args.precision == "bf16x3":
            extra["split_tf32x2"] = tf32x2_report(inp, d, spec, ctx, H64, w_d, prof, pk, args)
        del H64
        ref.close()

    # ---- finite exciton momentum (outside the timed region): H(Q) on the same workload -------
    if not args.no_finite_q:
        VR = torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).to(dev)
        per_q = []
        n1 = int(spec.dense[0])
        for i, Q in enumerate(((1, 0, 0), (1, 0, 0), (n1 // 2, 0, 0), (1, 1, 0))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ctx.set_momentum(Q, VR)
            ctx.interp_W(d["W_R"], None)
            ctx.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
            ctx.assemble(H)
            b.record(st)
            ctx.sync()
            if i == 0:
                continue                    # first use of the shifted kernels: warm-up
            w_q, r_q = ctx.lowest(H, 1, 300)
            ctx.sync()
            ms = a.elapsed_time(b)
            per_q.append({"Q": list(Q), "assembly_ms": ms, "elements_per_s": dim2 / (ms / 1000.0),
                          "lowest_exciton_eV": w_q.item()})
        ctx.set_momentum((0, 0, 0), None)
        extra["finite_momentum"] = {
            "precision": args.precision, "per_Q": per_q,
            "q0_assembly_ms": statistics.mean([p + a for p, a in zip(pre_ms, asm_ms)]),
            "note": "H(Q) = bse_set_momentum + interp_W + project_pairs + assemble (conduction bands at k+Q, "
                    "exchange with sum_R w_R Vbar(R) e^{+iQ.R}), Q in dense-mesh steps; outside the timed region"}

    # ---- matrix-free spectrum (outside the timed region): H never stored --------------------
    if not args.no_matfree and args.precision != "fp64":
        mf_steps = 12
        ab_s = torch.zeros((3, 3, mf_steps), dtype=torch.float64, device=dev)
        ab_m = torch.zeros_like(ab_s)
        e_s = torch.empty_like(eps2)
        e_m = torch.empty_like(eps2)
        ctx.interp_W(d["W_R"], d["V0"])
        ctx.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        ctx.assemble(H)
        u_m = ctx.dipole_vector(d["vel"], d["e_ks"])
        evm = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ctx.spectrum_matfree(u_m, 2, omega, args.eta, pref, e_m)      # warm-up (workspace)
        ctx.sync()
        evm[0].record(st)
        ctx.spectrum(H, u_m, mf_steps, omega, args.eta, pref, e_s, ab_s)
        evm[1].record(st)
        ctx.spectrum_matfree(u_m, mf_steps, omega, args.eta, pref, e_m, ab_m)
        evm[2].record(st)
        ctx.sync()
        a_s, a_m = ab_s[:, :2].cpu().numpy(), ab_m[:, :2].cpu().numpy()
        el = 8
        extra["matrix_free"] = {
            "steps": mf_steps, "stored_ms_per_step": evm[0].elapsed_time(evm[1]) / mf_steps,
            "matfree_ms_per_step": evm[1].elapsed_time(evm[2]) / mf_steps,
            "assembly_ms": statistics.mean(asm_ms),
            "H_bytes": int(ctx.dim) ** 2 * el,
            "lanczos_coeff_max_rel_diff": float(np.abs(a_s - a_m).max() / np.abs(a_s).max()),
            "eps2_rel_L2_diff": (torch.linalg.norm(e_s - e_m) / torch.linalg.norm(e_s)).item(),
            "note": "each matrix-free product recomputes the direct term slab by slab (projections, M_vv W(q) "
                    "on tensor cores, blocks applied as formed) plus the exchange and diagonal; memory is the "
                    "slab workspace instead of H"}

    # ---- full BSE (outside the timed region): coupling block, paired spectrum, lowest Omega ----
    if not args.no_full_bse:
        from paper_2607_05853_b300.api import BseError
        try:
            extra["full_bse"] = full_bse_report(spec, args, dev, nsteps, omega, pk)
        except BseError as e:          # e.g. an indefinite [[A, B], [B*, A*]]: report, keep the line
            extra["full_bse"] = {"error": str(e)}

    clocks = clk.summary()
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64"}.get(args.precision, f"{args.precision} (assembly: {'tf32' if args.precision == 'tf32x2' else 'bf16'}-piece tensor-core GEMMs with f32 "
                                                     "accumulation, f32 projections, f64 phases and diagonal; H "
                                                     "stored complex64; Lanczos: f64 recursion and basis, f32 "
                                                     "products on the complex64 H with compensated sums)"),
        "data": "synthetic (seeded generator, shapes of the paper's Si/MgO workloads)",
        "config": {"workload": spec.name, "dim": ctx.dim, "n_k": spec.n_k, "mesh": list(spec.dense),
                   "n_aux": spec.n_aux, "n_ao": spec.n_ao, "nv": nv, "nc": nc, "haydock_steps": nsteps,
                   "n_pol": 3, "n_omega": args.n_omega, "precision": args.precision,
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
        "stages_ms": {"interp+per_k": statistics.mean(pre_ms), "assemble": statistics.mean(asm_ms),
                      "dipole+spectrum": statistics.mean(spec_ms)},
        "value_note": "value = dim^2 / (one whole hot-path step: W(q) interpolation, pair projections, assembly, "
                      "dipole vector and the 3-polarisation Haydock spectrum); the assembly-only rate "
                      "(interp + project + assemble) is assembly_elements_per_s",
        "assembly_elements_per_s": asm_rate,
        "assembly_dram_bytes_est": (
            {"slab_kernels": ASM_DRAM_BYTES_PER_Q_MESH10 * (spec.n_k / 1000.0) * len(_qplus(spec.dense)),
             "H_bytes": float(ctx.dim) ** 2 * (16 if args.precision == "fp64" else 8),
             "note": "projections + fused direct term: DRAM bytes per q from ncu on the 16000-dim case, "
                     "scaled by k-points per q and the unique q of this mesh (the exchange GEMM's H write "
                     "and the per-k stage come on top); H_bytes is what the assembly must write"}
            if args.precision != "fp64" and spec.n_aux <= 160 else None),
        "spectrum_throughput": {"haydock_steps_per_s": nsteps / (statistics.mean(spec_ms) / 1000.0),
                                "matvec_GBps": roof.get("achieved") if top == "matvec" else None},
        "kernels_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]},
        "roofline": roof, "tensor_roofline": tensor, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
    }
    result.update(extra)
    if args.batch16:
        del H
        torch.cuda.empty_cache()
        result["batched_uneven"] = batch16_report(world=world, rank=rank, dist=dist if world > 1 else None)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(inp, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def full_bse_report(spec, args, dev, nsteps, omega, pk):
    """Full BSE on the same geometry with the W scale halved (the synthetic inputs need it for
    [[A, B], [B*, A*]] to be positive definite): A and B assembled, the 3-polarisation
    full-BSE spectrum (Lanczos in the M inner product, nsteps steps) next to the TDA one, the
    lowest paired excitations; per-kernel times from the library's event profile."""
    import torch
    from paper_2607_05853_b300.api import BSE
    from synth import full_bse_spec, make_inputs
    fspec = full_bse_spec(spec)
    inp = make_inputs(fspec)
    d = {k: torch.from_numpy(np.ascontiguousarray(inp[k], np.float64)).to(dev)
         for k in ("W_R", "V0", "C_R", "e_qp", "e_ks")}
    d.update({k: torch.from_numpy(np.ascontiguousarray(inp[k], np.complex128)).to(dev) for k in ("c_k", "vel")})
    ctx = BSE.from_inputs(inp, precision=args.precision)
    A = torch.empty((ctx.dim, ctx.dim), dtype=ctx.h_dtype, device=dev)
    B = torch.empty_like(A)
    pref = 4.0 * np.pi ** 2 / (3.0 * fspec.n_k * float(inp["volume"]))
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    eps_f = torch.empty(omega.numel(), dtype=torch.float64, device=dev)
    eps_t = torch.empty_like(eps_f)
    for rep in range(2):                    # the first pass warms up (allocations, tensor maps)
        ctx.sync()
        ev[0].record(st)
        ctx.interp_W(d["W_R"], d["V0"])
        ctx.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        ctx.assemble(A)
        u = ctx.dipole_vector(d["vel"], d["e_ks"])
        ctx.profile(rep == 1)               # per-kernel times of B's assembly and the full spectrum only
        ev[1].record(st)
        ctx.assemble_coupling(B)
        ev[2].record(st)
        ctx.spectrum_full(A, B, u, nsteps, omega, args.eta, pref, eps_f)
        ev[3].record(st)
        if rep == 1:
            prof_f = {k: ctx.profile_read(k) for k in ("matvec", "reorth", "project", "g1", "g2", "exch")}
        ctx.profile(False)
        ctx.spectrum(A, u, nsteps, omega, args.eta, pref, eps_t)
        ev[4].record(st)
        w_f, r_f = ctx.lowest_full(A, B, 10, 400)
        ev[5].record(st)
        ctx.sync()
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]
    # algorithmic bytes of one step's product M r: the upper-triangle 128 x 128 tiles of A and
    # of B (both Hermitian/symmetric), once each; the product time per step from the profile
    el = 16 if args.precision == "fp64" else 8
    mv_ms, mv_n = prof_f["matvec"]
    nbt = (ctx.dim + 127) // 128
    alg = 2.0 * (nbt * (nbt + 1) // 2) * 128 * 128 * el
    per_step_ms = mv_ms / (nsteps + 1)
    achieved = alg / (per_step_ms * 1e-3) / 1e9 if mv_n else None
    out = {
        "workload": fspec.name, "dim": ctx.dim, "w_scale": fspec.s_W, "haydock_steps": nsteps,
        "per_k_and_A_ms": ms[0], "assemble_B_ms": ms[1], "spectrum_full_ms": ms[2], "spectrum_tda_ms": ms[3],
        "lowest_full_ms": ms[4],
        "lowest_full_eV": w_f.tolist(), "lowest_full_resid_eV": r_f.tolist(),
        "eps2_full_vs_tda_rel_L2": (torch.linalg.norm(eps_f - eps_t) / torch.linalg.norm(eps_t)).item(),
        "kernels_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof_f.items() if v[1]},
        "product_roofline": {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": pk["hbm_gbs"],
                             "frac": achieved / pk["hbm_gbs"] if achieved else None,
                             "per_step_ms": per_step_ms, "launches_per_step": mv_n / (nsteps + 1),
                             "note": "product M r per Lanczos step: algorithmic bytes = the upper-triangle tiles "
                                     "of A and of B once each; the half-read kernel runs twice per step (A on "
                                     "(x, conj y), B on (y, conj x), 2 x 3 polarisation vectors each), so each "
                                     "matrix half is read once"},
    }
    del A, B
    ctx.close()
    torch.cuda.empty_cache()
    return out


def ctx_slab_q(ctx, spec):
    return 1


def _self_conj(q, dense):
    """q == -q on the mesh (every coordinate 0 or N/2)."""
    n1, n2, n3 = dense
    m = (q // (n2 * n3), (q // n3) % n2, q % n3)
    return all((2 * mi) % ni == 0 for mi, ni in zip(m, (n1, n2, n3)))


def batch16_report(precision="bf16x3", world=1, rank=0, dist=None):
    """16 seeded crystals of uneven size assembled as one CUDA graph: per-system throughput
    inside the batch, the isolated throughput of each system, aggregate speedup over running
    them one after another, and Jain's fairness index of (batched / isolated) throughput.
    Under torchrun the systems are sharded across the ranks (longest-processing-time-first,
    paper_2607_05853_b300.shard), each rank running its own batch graph; the report then
    gathers every rank's systems (metadata only) and the job time is the slowest rank's."""
    import torch
    from paper_2607_05853_b300.api import BSE, batch_assemble, batch_release
    from paper_2607_05853_b300.shard import assembly_work, assign_systems
    from synth import batched_specs, make_inputs
    specs = batched_specs(16)
    mine = assign_systems([assembly_work(sp.n_k, sp.n_aux, sp.nv, sp.nc) for sp in specs], world)[rank]
    systems, Hs, dims, tiles = [], [], [], []
    for sp in [specs[i] for i in mine]:
        inp = make_inputs(sp)
        b = BSE.from_inputs(inp, precision=precision)
        d = {k: torch.from_numpy(np.ascontiguousarray(inp[k])).cuda() for k in ("W_R", "V0", "C_R", "e_qp", "c_k")}
        b.interp_W(d["W_R"], d["V0"])
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        tiles.append(b.autotune())
        systems.append(b)
        Hs.append(torch.empty((b.dim, b.dim), dtype=b.h_dtype, device="cuda"))
        dims.append(b.dim)
        del d
    st = torch.cuda.current_stream()
    iso = []
    for b, H in zip(systems, Hs):
        b.assemble(H)  # warm
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        b.assemble(H)
        e.record(st)
        torch.cuda.synchronize()
        iso.append(a.elapsed_time(e))
    el = [float(dm) ** 2 for dm in dims]
    out = {"systems": 16, "ranks": world, "precision": precision, "serial_ms": sum(iso),
           "serial_elements_per_s": sum(el) / (sum(iso) / 1e3)}
    for schedule in ("worklist", "chains"):
        batch_assemble(systems, Hs, schedule=schedule)  # build + first replay
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        batch_assemble(systems, Hs, schedule=schedule)
        e.record(st)
        torch.cuda.synchronize()
        t_batch = a.elapsed_time(e)
        stamps = batch_assemble(systems, Hs, stamps=True, schedule=schedule)
        done_ms = [x / 1e6 for x in stamps]
        rows = list(zip(dims, tiles, iso, done_ms))
        if dist is not None:       # gather the ranks' per-system results (reporting only)
            parts = [None] * world
            dist.all_gather_object(parts, (t_batch, rows))
            t_batch = max(p[0] for p in parts)
            rows = [r for p in parts for r in p[1]]
        x = [t_i / max(c_i, 1e-9) for _, _, t_i, c_i in rows]   # batched / isolated throughput
        jain = sum(x) ** 2 / (len(x) * sum(v * v for v in x))
        elr = [float(r[0]) ** 2 for r in rows]
        res = {"graph_ms": t_batch, "aggregate_elements_per_s": sum(elr) / (t_batch / 1e3),
               "batch_speedup_over_serial": sum(r[2] for r in rows) / t_batch, "jain_fairness": jain,
               "per_system": [{"dim": dm, "tile": tl, "isolated_ms": round(ti, 3), "done_in_batch_ms": round(c, 3),
                               "elements_per_s_isolated": float(dm) ** 2 / (ti / 1e3)}
                              for dm, tl, ti, c in rows]}
        if schedule == "worklist":
            out["serial_ms"] = sum(r[2] for r in rows)
            out["serial_elements_per_s"] = sum(elr) / (out["serial_ms"] / 1e3)
            out.update(res)
            out["schedule"] = "worklist: grouped tensor-core launches over the (system, q-slab, tile) work list"
        else:
            out["chains"] = res
    batch_release()
    for b in systems:
        b.close()
    return out


if __name__ == "__main__":
    main()
