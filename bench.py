#!/usr/bin/env python
"""Schwarz-coupled element-updates/s of one O-SAM controller step on a GB300.

Workload (N=1 line): the FOM / OpInf hybrid -- subdomain A a 40x40x80 Neo-Hookean hex8 FOM, subdomain
B (mirror 40x40x80 mesh, 2-layer overlap) a quadratic OpInf ROM of rank 64 fitted (Tikhonov
lambda = 1e-6) by the library's opinf_fit on 500 snapshots of a seeded FOM-FOM training run of the same
geometry; explicit central difference dt = 1e-6 s, controller steps of 20 substeps, relative tolerance
1e-12, at most 64 Schwarz iterations.  A bench "step" is one controller step (every Schwarz
iteration: FOM substeps, ROM substeps, overlap transfers, convergence check).

value   = FOM element-updates executed in the timed steps / device time of those steps, each step one
          launch of the library's captured controller-step graph (its default path), CUDA events on the
          library's stream; L2 flushed between steps by a 256 MiB write outside the timing.
e2e     = the same metric through the public API with host buffers: every step sets the FOM and ROM
          states from pinned host memory, runs schwarz_step (its default, graph-captured path) and reads
          the states back; wall-clock time on the host.
roofline= the Neo-Hookean FP64 internal-force kernel (the dominant kernel): algorithmic FP64 flops of
          its launches / their CUDA-event time, from a second timed pass of the same steps driven from
          the host with events around every force launch, against the FP64 peak.
variants= both force precisions (native FP64; double-float on the FP32 pipes), each timed as the
          graph-captured step and in the host-driven profiling loop, with its own roofline.
batched_vs_plain = 256 FOM / OpInf(r=32) samples advanced by one batched context vs one context per
          sample (ROMs fitted per sample from batched training runs, untimed).
--impl reference times the CPU oracle on a bounded sample of the same workload.
Multi-GPU: replicas only (the coupled step does not shard); each rank runs the workload on its GPU.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Schwarz-coupled element-updates/sec on 1 GB300"
UNIT = "element-updates/s"
# FP64 flops of one Neo-Hookean element evaluation in the sum-factorised kernel (FMA = 2 flops,
# each of the 8 cube roots counted as one flop): edge scaling 24 + differences 36 + interpolation to
# the Gauss points 180 + 8 x 90 constitutive + 36 accumulation + 180 transposed interpolation +
# 48 nodal accumulation + 8.
FLOPS_PER_NH_ELEMENT = 1232
# FP64 nominal figure of the recipe for the GB300 (1.25 TFLOP/s); the rooflines divide by the FP64
# peak measured on the GPU itself (measure_fp64_peak) and give the fraction of this one beside it
FP64_NOMINAL_TFLOPS = 1.25
# double-float force: FP32-pipe thread-instructions per Neo-Hookean element (ncu smsp__inst_executed
# x 32 / elements of the phased kernel) and the FP32 issue peak (152 SMs x 128 lanes x 2.07 GHz)
F32X2_INST_PER_NH_ELEMENT = 12012
FP32_ISSUE_PEAK_TINST = 152 * 128 * 2.07e9 / 1e12
# DRAM traffic of one force launch of the bench workload (ncu dram__bytes_read.sum + write.sum),
# valid only for the kernel source and variant (tiled or not) it was captured on.
FORCE_TRAFFIC = {"source_sha256": "5329782da603ec0d213b49ef60d6836089a9f41f0ba6bc0fa18cff46cede7c3d",
                 "bytes_per_launch": 3.567616e6, "tiled": True, "register_cap": 0}
# the same for the Neo-Hookean tangent-action kernel of the implicit block (sources TANGENT_SOURCES)
# bytes one tangent launch must move per element: the stored linearisation (22 doubles x 8 Gauss
# points) + p at 8 nodes / 8 elements per node (24 B); the element buffer stays in L2
TANGENT_BYTES_PER_ELEMENT = 22 * 8 * 8 + 24
TANGENT_TRAFFIC = {"source_sha256": "cd475f28af922fbeaa85abd62d838d03451fea6f47a72d3046ce0d821fae63fc",
                   "bytes_per_launch": 1.947856e8}


STATE_BYTES_PER_NODE_UPDATE = 152
# FP64 flops of one Neo-Hookean element tangent action K(u) p of the implicit Newton-CG (FMA = 2
# flops), from the Gauss-point linearisation stored with the Newton residual's force: scaling of p
# 24 + differences of p 36 + their interpolation to the Gauss points 180 + 8 x 166 (cof : G and F : G
# 36, derivative of the cofactor 63, scalar chain 4, dP 63) + 36 accumulation + 180 transposed
# interpolation + 48 nodal accumulation.
TANGENT_FLOPS_PER_NH_ELEMENT = 1832
# bytes the FP32 tangent kernel must move per element: the FP32 linearisation (22 floats x 8 Gauss
# points) from HBM, p at 8 nodes / 8 elements per node (24 B), the FP32 element buffer out (24 floats)
TANGENT32_BYTES_PER_ELEMENT = 22 * 8 * 4 + 24 + 24 * 4
# DRAM traffic of one FP32-tangent launch (ncu, same sources as TANGENT_TRAFFIC)
TANGENT32_TRAFFIC = {"source_sha256": "cd475f28af922fbeaa85abd62d838d03451fea6f47a72d3046ce0d821fae63fc",
                     "bytes_per_launch": 9.375027e7}
# FP64 flops of one Saint Venant-Kirchhoff element force: the 504 flops of the sum factorisation
# around the constitutive law (as for Neo-Hookean) + 8 x 115 (Green-Lagrange strain 48, S 13, P = F S 54)
FLOPS_PER_SVK_ELEMENT = 1424


# the measured FP64 peak of this run (set by measure_fp64_peak before any roofline is formed)
FP64_PEAK = [FP64_NOMINAL_TFLOPS]
FP64_PEAK_KIND = ["of nominal: the recipe's 1.25 TFLOP/s (FP64 probes skipped)"]


def measure_fp64_peak(osam, local, repeats=10):
    """The FP64 roofline denominator measured on this GPU: the best of `repeats` launches (~20 ms
    each) of the library's FMA probe and of its FP64 tensor-core (mma.sync m8n8k4) probe, with the SM
    clock sampled during them; the interleaved probe shows whether the two share one unit."""
    clocks = ClockSampler(local)
    clocks.start()
    fma, _ = osam.fp64_probe(0, repeats, local)
    mma, _ = osam.fp64_probe(1, repeats, local)
    mix, _ = osam.fp64_probe(2, max(2, repeats // 2), local)
    # the per-warp latency floor of the element kernels on small meshes (one block on one SM)
    issue = {f"{w}_warps_{l}_lanes": osam.fp64_issue_probe(w, l, local) for w, l in ((1, 32), (1, 8), (4, 32), (8, 32))}
    clk = clocks.stop()
    best = float(max(fma.max(), mma.max()))
    FP64_PEAK[0] = best
    FP64_PEAK_KIND[0] = "of measured: FP64 peak of this GPU (fp64_peak block)"
    return {"tflops": best, "unit": "TFLOP/s", "repeats": repeats,
            "fma_best": float(fma.max()), "fma_median": float(np.median(fma)),
            "mma_best": float(mma.max()), "mma_median": float(np.median(mma)),
            "fma_plus_mma_interleaved_best": float(mix.max()),
            "issue_ns_per_warp_instruction": issue,
            "sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "clock_reasons": clk["reasons"],
            "nominal_tflops": FP64_NOMINAL_TFLOPS,
            "kind": "measured: best of the FP64 FMA and FP64 tensor-core probes (osam_fp64_probe)"}


def host_cpu():
    """CPU model and logical core count of the host the oracle legs run on."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
        if model is None:   # Arm hosts: implementer / part numbers only
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model, "nproc": os.cpu_count()}


def measured_hbm_gbs():
    """(HBM copy bandwidth in GB/s, where it comes from): the measured figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback (6.8 TB/s)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=90)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="osam", choices=["osam", "reference"])
    ap.add_argument("--n", type=int, default=40)
    ap.add_argument("--nz", type=int, default=80)
    ap.add_argument("--rank", type=int, default=64)
    ap.add_argument("--snapshots", type=int, default=500)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32x2"],
                    help="f64: native FP64 force; f32x2: double-float force on the FP32 pipes (FP64 state)")
    ap.add_argument("--scatter", default="auto", choices=["auto", "gather", "atomic", "tiled", "lowreg", "tiled_lowreg"],
                    help="force-kernel configuration (auto: the library's autotuner); fixed choices make ncu "
                         "captures reproducible")
    ap.add_argument("--batched-samples", type=int, default=256)
    ap.add_argument("--batched-snapshots", type=int, default=100)
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--batched-plain-steps", type=int, default=0,
                    help="timed steps of the one-context-per-sample arm (0: as many as the batched arm)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain parameter sweep")
    ap.add_argument("--no-large", action="store_true", help="skip the large FOM-OpInf-FOM chain")
    ap.add_argument("--fp64-peak-repeats", type=int, default=10,
                    help="launches per FP64 probe for the roofline denominator (0: skip the probes and divide by "
                         "the nominal 1.25 TFLOP/s, for profiling runs)")
    ap.add_argument("--large-only", action="store_true", help="run only the large-chain block (profiling runs)")
    ap.add_argument("--fit-only", action="store_true",
                    help="profiling entry: one opinf_fit of seeded synthetic snapshots of the headline size "
                         "(--snapshots x 403,440 free dofs, 5,043 Schwarz dofs, rank --rank), no training run")
    ap.add_argument("--large-n", type=int, default=96)
    ap.add_argument("--large-nz", type=int, default=192)
    ap.add_argument("--large-rank", type=int, default=128)
    ap.add_argument("--large-snapshots", type=int, default=500)
    ap.add_argument("--large-steps", type=int, default=5)
    ap.add_argument("--no-implicit", action="store_true", help="skip the implicit-FOM measurement")
    ap.add_argument("--implicit-only", action="store_true",
                    help="run only the implicit-FOM block (stand-in ROM operators): profiling runs")
    ap.add_argument("--fom-only", action="store_true",
                    help="FOM-FOM coupling of the same geometry (no ROM, no training): profiling runs")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def source_sha(files=("step_kernels.cu", "hex8_math.cuh", "trace_item.cuh", "fp_bits.cuh")):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2511_20687_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


TANGENT_SOURCES = ("tangent_kernels.cu", "hex8_math.cuh", "nh_tangent.cuh", "fp_bits.cuh")


# ---------------------------------------------------------------------------------------------
# workload construction
# ---------------------------------------------------------------------------------------------
def rom_dof_masks(sd):
    """Free and Schwarz dof masks of the top subdomain of a two-subdomain bar (Schwarz face z = 0)."""
    _, _, kk = sd.node_grid()
    schwarz = kk == 0
    clamped = np.repeat(sd.dirichlet, 3).reshape(-1, 3) > 0
    free = (~clamped & ~schwarz[:, None]).reshape(-1)
    return free, np.repeat(schwarz, 3)


def train_rom(W, osam, args, device, log, material="nh", rank=None, cubic=False, snapshots=None):
    """Seeded FOM-FOM training run (snapshot every 4th step) and GPU OpInf fit of subdomain B."""
    rank = rank or args.rank
    n_snap = snapshots or args.snapshots
    rng = np.random.default_rng(W.SEED_BASE + 1)
    amp = float(rng.uniform(0.5e-3, 1.0e-3))
    nu = 0.3 if material == "svk" else 0.25
    spec = W.bar_chain("train", args.n, [args.nz, args.nz], ["fom", "fom"], material, 1e9, nu, 1000.0, amp, 1e-6, 4)
    prob = osam.Problem(spec, device=device)
    free, sdof = rom_dof_masks(spec.subdomains[1])
    U = np.empty((n_snap, int(free.sum())))
    A = np.empty_like(U)
    S = np.empty((n_snap, int(sdof.sum())))
    t0 = time.time()
    v0 = None
    for k in range(n_snap):
        prob.step()
        u, v, a = prob.state(1, fields=(0, 1, 2) if k == 0 else (0, 2))
        U[k] = u.reshape(-1)[free]
        A[k] = a.reshape(-1)[free]
        S[k] = u.reshape(-1)[sdof]
        if k == 0:
            v0 = v.reshape(-1)[free].copy()
    prob.close()
    log(f"training run ({material}): {n_snap} controller steps of 4 substeps in {time.time() - t0:.1f}s "
        f"(amplitude {amp:.3e})")
    t0 = time.time()
    ops = osam.opinf_fit(U, A, S, r=rank, lam=1e-6, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, device=device,
                         cubic=cubic)
    fit_s = time.time() - t0
    log(f"opinf_fit: r={rank} r_s={ops['r_s']}{' cubic' if cubic else ''} in {fit_s:.1f}s")
    fit = {"gpu_seconds": fit_s, "r": rank, "r_s": int(ops["r_s"]), "n_snap": n_snap,
           "n_dof": int(U.shape[1]), "n_sdof": int(S.shape[1]), "training": (U, A, S, v0)}
    keys = ("Phi", "Phi_S", "K", "H", "B", "c") + (("C",) if cubic else ())
    return {k: ops[k] for k in keys}, fit


def train_batched_roms(W, osam, torch, specs_ff, snapshots, r, device, log, chunk=32):
    """Per-sample OpInf ROMs of subdomain B: FOM-FOM training runs of the samples advanced together
    as batches (controller steps of 4 substeps, one snapshot per step, double-float force), snapshots
    gathered on the device, then one GPU opinf_fit per sample."""
    dev = f"cuda:{device}"
    ops, ranks = [], []
    t0 = time.time()
    for c0 in range(0, len(specs_ff), chunk):
        group = specs_ff[c0:c0 + chunk]
        for sp in group:
            sp.n_substeps = 4
        batch = osam.Batch(group, precision=osam.F32X2_FORCE, device=device)
        idx = []
        for sp in group:
            f, sd = rom_dof_masks(sp.subdomains[1])
            idx.append((torch.from_numpy(np.flatnonzero(f)).to(dev), torch.from_numpy(np.flatnonzero(sd)).to(dev)))
        max_nn = max(sp.subdomains[1].n_nodes for sp in group)
        bu = torch.empty((max_nn, 3), dtype=torch.float64, device=dev)
        ba = torch.empty((max_nn, 3), dtype=torch.float64, device=dev)
        U = [torch.empty((snapshots, fi.numel()), dtype=torch.float64, device=dev) for fi, _ in idx]
        A = [torch.empty_like(x) for x in U]
        S = [torch.empty((snapshots, si.numel()), dtype=torch.float64, device=dev) for _, si in idx]
        for k in range(snapshots):
            batch.step()
            for i, (fi, si) in enumerate(idx):
                nn = group[i].subdomains[1].n_nodes
                ub, ab = bu[:nn], ba[:nn]
                batch.state(1, out=(ub, None, ab), inst=i)
                uf, af = ub.reshape(-1), ab.reshape(-1)
                U[i][k] = uf[fi]
                A[i][k] = af[fi]
                S[i][k] = uf[si]
        batch.close()
        torch.cuda.synchronize()
        for i in range(len(group)):
            # a short training run can have a numerical rank below r: take the largest of r, 3r/4, r/2, ...
            for rr in (r, 3 * r // 4, r // 2, r // 4):
                try:
                    o = osam.opinf_fit(U[i], A[i], S[i], r=rr, lam=1e-6, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64,
                                       device=device)
                    break
                except osam.OsamError:
                    if rr == r // 4:
                        raise
            ranks.append(rr)
            ops.append({1: {k: o[k] for k in ("Phi", "Phi_S", "K", "H", "B", "c")}})
        del U, A, S
    log(f"batched training: {len(specs_ff)} samples x {snapshots} snapshots, r={r} ({sum(x == r for x in ranks)} "
        f"samples at full rank), in {time.time() - t0:.1f}s")
    return ops, ranks


def measure_batched(W, osam, torch, flush, args, device, log, rank=0, world=1):
    """Batched vs plain on the parameter-sweep workload: the same samples (FOM / OpInf pairs) advanced
    by one batched context (graph-captured step) and by one context per sample, run one after another.
    Under torchrun the samples are sharded over the ranks by element count (shard_samples): each rank
    trains and advances its own, with no exchange on the data path; the per-instance reports are
    gathered at the end, time is the maximum over ranks and the element-updates the sum."""
    import torch.distributed as dist
    multi = world > 1

    def barrier():
        if multi:
            dist.barrier()

    specs_all = W.batched_samples(n_samples=args.batched_samples, rom=True)
    ff_all = W.batched_samples(n_samples=args.batched_samples, rom=False)
    mine = shard_samples([sp.subdomains[0].n_elements for sp in specs_all], world)[rank]
    specs = [specs_all[i] for i in mine]
    ops, ranks = train_batched_roms(W, osam, torch, [ff_all[i] for i in mine], args.batched_snapshots, 32, device,
                                    log)
    batch = osam.Batch(specs, rom_ops=ops, device=device)
    for _ in range(3):
        batch.step()
    torch.cuda.synchronize()
    dev_ms, upd, wall, its = 0.0, 0, 0.0, []
    per_inst = {i: [] for i in mine}
    for _ in range(args.batched_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        per, tot = batch.step()
        torch.cuda.synchronize()
        barrier()
        wall += time.perf_counter() - t0
        dev_ms += tot["elapsed_ms"]
        upd += tot["element_updates"]
        its += [p["iterations"] for p in per]
        for i, p in zip(mine, per):
            per_inst[i].append((p["status"], p["iterations"]))
    tuning = batch.tuning()
    # the batched force kernel's roofline: one more step driven from the host with CUDA events around
    # every force launch
    batch.profile(True)
    batch.set_graph(False)
    _, prof_tot = batch.step()
    bprof = batch.profile_read()
    batch.profile(False)
    batch.close()
    bach_force = FLOPS_PER_NH_ELEMENT * bprof["force_elements"] / (bprof["force_ms"] * 1e-3) / 1e12
    # the same samples with the tiled force kernel forced (the autotuner's choice is timed against it)
    tb = osam.Batch(specs, rom_ops=ops, device=device, scatter=osam.SCATTER_GATHER_TILED)
    tb.step()
    t_ms, t_upd = 0.0, 0
    for _ in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        _, tt = tb.step()
        t_ms += tt["elapsed_ms"]
        t_upd += tt["element_updates"]
    tb.close()
    singles = [osam.Problem(sp, rom_ops=o, device=device) for sp, o in zip(specs, ops)]
    for p in singles:
        p.step()
    torch.cuda.synchronize()
    p_ms, p_upd, p_wall = 0.0, 0, 0.0
    plain_steps = args.batched_plain_steps or args.batched_steps
    for _ in range(plain_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for p in singles:
            r = p.step()
            p_ms += r["elapsed_ms"]
            p_upd += r["element_updates"]
        torch.cuda.synchronize()
        barrier()
        p_wall += time.perf_counter() - t0
    for p in singles:
        p.close()
    reports = gather_reports(per_inst)
    (wall_ms, upd_all), (dev_max, _), (p_wall_ms, p_upd_all), (p_dev, _), (t_dev, t_upd_all) = combine_ranks(
        [(wall * 1e3, upd), (dev_ms, upd), (p_wall * 1e3, p_upd), (p_ms, p_upd), (t_ms, t_upd)], f"cuda:{device}")
    n_el = sum(sp.subdomains[0].n_elements for sp in specs_all)
    all_its = [it for v in reports.values() for _, it in v]
    out = {"workload": f"{len(specs_all)} FOM / OpInf(r=32) pairs, n x n x 2n Neo-Hookean FOM, n ~ U{{8..32}}, "
                       f"{n_el} FOM elements in total, ROMs fitted on {args.batched_snapshots} snapshots each",
           "rom_ranks": {"32": sum(x == 32 for x in ranks), "below_32": sum(x < 32 for x in ranks)},
           "steps": args.batched_steps, "value": upd_all / (wall_ms * 1e-3),
           "value_device": upd_all / (dev_max * 1e-3),
           "plain_steps": plain_steps, "plain_value": p_upd_all / (p_wall_ms * 1e-3),
           "plain_value_device": p_upd_all / (p_dev * 1e-3),
           "speedup": (upd_all / wall_ms) / (p_upd_all / p_wall_ms),
           "mean_iterations": float(np.mean(all_its)), "max_iterations": int(max(all_its)), "unit": UNIT,
           "instances_reported": len(reports), "ranks": world,
           "scaling": "strong (the 256 samples are split over the ranks)" if multi else None,
           "tuning": tuning, "timing": "host wall clock around each synchronous step call (value) and the "
                                       "library's CUDA events (value_device); L2 flushed between steps; "
                                       "under torchrun a barrier on both sides and the maximum over ranks",
           "roofline": {"bound": "alu", "kernel": "batched internal force (Neo-Hookean, %s)" %
                        ("tiled" if tuning.get("tiled") else "%d-thread blocks" % tuning["element_block"]),
                        "achieved": bach_force, "peak": FP64_PEAK[0], "unit": "TFLOP/s",
                        "frac": bach_force / FP64_PEAK[0], "flops_per_element": FLOPS_PER_NH_ELEMENT,
                        "force_ms_per_launch": bprof["force_ms"] / max(1, bprof["force_launches"]),
                        "elements_per_launch": bprof["force_elements"] // max(1, bprof["force_launches"]),
                        "force_launches_per_step": bprof["force_launches"],
                        "force_time_share": bprof["force_ms"] / prof_tot["elapsed_ms"],
                        "kernel_launches_per_step": bprof["kernel_launches"],
                        "peak_kind": FP64_PEAK_KIND[0]},
           "tiled_forced": {"value_device": t_upd_all / (t_dev * 1e-3), "steps": 2,
                            "note": "the same samples with the 8x4x4-tile force kernel forced (n x n x 2n "
                                    "meshes, n in 8..32, leave partial tiles on most instances)"}}
    if rank == 0:
        # the oracle on a bounded sample of the same sweep: two samples of this rank, one controller step
        # of one Schwarz iteration each, their fitted ROMs
        from oracle import oracle as O
        o_upd, o_s = 0, 0.0
        for sp, o in list(zip(specs, ops))[:2]:
            sp.max_iters = 1
            ref = O.Problem(sp, rom_ops=o)
            t0 = time.process_time()
            ref.step()
            o_s += time.process_time() - t0
            o_upd += sp.n_substeps * sp.subdomains[0].n_elements
        out.update({"oracle_value": o_upd / o_s, "oracle_cores": 1,
                    "oracle_sample": f"two samples, one controller step of one Schwarz iteration each, {o_s:.1f} s CPU"})
    return out


def measure_fit(fit_info, log):
    """opinf_fit on the GPU (timed during training, host snapshot matrices in, operators out) against
    the oracle's numpy fit of the same snapshots with the same r and r_s."""
    from oracle import fit as OF
    U, A, S, _ = fit_info["training"]
    t0 = time.perf_counter()
    OF.opinf_fit(U.T, A.T, S.T, r=fit_info["r"], lam=1e-6, r_s=fit_info["r_s"])
    cpu = time.perf_counter() - t0
    log(f"oracle fit: {cpu:.1f}s")
    one = fit_one_thread_sample(fit_info, log)
    gemm = fit_gemm_roofline(U, A, S, fit_info["r"], fit_info["r_s"], log)
    return {**{k: v for k, v in fit_info.items() if k != "training"}, "unit": "s", "higher_is_better": False,
            "oracle_seconds": cpu,
            "oracle_threads": os.cpu_count(), "oracle_kind": "oracle/fit.py (numpy SVD and solve, threaded BLAS)",
            "speedup_vs_oracle": cpu / fit_info["gpu_seconds"], "one_thread_sample": one, "gemm": gemm,
            "roofline": gemm["roofline"]}


def fit_gemm_roofline(U, A, S, r, rs, log, device=0):
    """The fit from device arrays with the library's GEMM accounting on (CUDA events around every
    contraction): FP64 flops of its GEMMs / their event time against the measured FP64 peak."""
    import torch
    from paper_2511_20687_gb300 import osam
    dev = f"cuda:{device}"
    Ud, Ad, Sd = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (U, A, S))
    osam.opinf_fit(Ud, Ad, Sd, r=r, lam=1e-6, r_s=rs, device=device)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    osam.opinf_fit(Ud, Ad, Sd, r=r, lam=1e-6, r_s=rs, device=device)
    plain_s = time.perf_counter() - t0
    osam.fit_profile(True)
    osam.opinf_fit(Ud, Ad, Sd, r=r, lam=1e-6, r_s=rs, device=device)
    prof = osam.fit_profile(False)
    achieved = prof["gemm_flops"] / (prof["gemm_ms"] * 1e-3) / 1e12
    log(f"fit GEMMs: {prof['gemm_launches']} products, {prof['gemm_flops'] / 1e9:.0f} GFLOP in {prof['gemm_ms']:.1f} ms "
        f"= {achieved:.3f} TFLOP/s; device-input fit {plain_s:.2f} s")
    del Ud, Ad, Sd
    torch.cuda.empty_cache()
    return {"device_input_seconds": plain_s, "gemm_ms": prof["gemm_ms"], "gemm_flops": prof["gemm_flops"],
            "gemm_launches": prof["gemm_launches"], "gemm_share_of_fit": prof["gemm_ms"] * 1e-3 / plain_s,
            "roofline": {"bound": "alu", "kernel": "k_gemm_mma (+ k_gemm_reduce), FP64 tensor-core mma.sync m8n8k4", "achieved": achieved,
                         "peak": FP64_PEAK[0], "unit": "TFLOP/s", "frac": achieved / FP64_PEAK[0],
                         "peak_kind": FP64_PEAK_KIND[0],
                         "timing": "library CUDA events around every GEMM of one device-input fit "
                                   "(osam_fit_profile)"}}


def fit_one_thread_sample(fit_info, log, n_snap=100):
    """The fit on a bounded sample (the first n_snap snapshots, same r and r_s): the GPU from host
    arrays, the oracle's numpy fit in a child process with one BLAS thread (the other oracle figures
    are one core too)."""
    from paper_2511_20687_gb300 import osam
    U, A, S, _ = fit_info["training"]
    U, A, S = (np.ascontiguousarray(x[:n_snap]) for x in (U, A, S))
    r, rs = fit_info["r"], fit_info["r_s"]
    t0 = time.perf_counter()
    osam.opinf_fit(U, A, S, r=r, lam=1e-6, r_s=rs)
    gpu_s = time.perf_counter() - t0
    with tempfile.TemporaryDirectory() as d:
        for name, x in (("U", U), ("A", A), ("S", S)):
            np.save(os.path.join(d, name + ".npy"), x)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import os, sys, time, numpy as np\n"
                f"sys.path.insert(0, {ROOT!r})\n"
                "from oracle import fit as OF\n"
                f"U, A, S = (np.load(os.path.join({d!r}, n + '.npy')) for n in 'UAS')\n"
                "t0 = time.process_time()\n"
                f"OF.opinf_fit(U.T, A.T, S.T, r={r}, lam=1e-6, r_s={rs})\n"
                "print(time.process_time() - t0)\n")
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    cpu_s = float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    log(f"fit sample ({n_snap} snapshots): GPU {gpu_s:.2f}s, oracle on one thread {cpu_s}s")
    return {"n_snap": n_snap, "gpu_seconds": gpu_s, "oracle_seconds": cpu_s, "oracle_threads": 1,
            "speedup_vs_oracle": (cpu_s / gpu_s) if cpu_s else None,
            "note": "GPU from host arrays; oracle in a child process with OMP/OPENBLAS/MKL_NUM_THREADS=1"}


def measure_select(osam, fit_info, local, log, sample_snaps=100, sample_r=32):
    """Schwarz-aware regularisation selection (Algorithm 3, 11 candidates 1e-10 .. 1, rollouts with the
    online step 1e-6 s and 4 steps between snapshots): the GPU on the whole headline training set, and
    GPU and oracle on a bounded sample of it (first snapshots, smaller rank)."""
    from oracle import fit as OF
    U, A, S, v0 = fit_info["training"]
    lams = OF.lambda_grid()
    t0 = time.perf_counter()
    full = osam.opinf_select(U, A, S, v0, r=fit_info["r"], lambdas=lams, dt=1e-6, substeps=4, r_s=fit_info["r_s"],
                             device=local)
    gpu_full = time.perf_counter() - t0
    Us, As, Ss = U[:sample_snaps], A[:sample_snaps], S[:sample_snaps]
    t0 = time.perf_counter()
    gs = osam.opinf_select(Us, As, Ss, v0, r=sample_r, lambdas=lams, dt=1e-6, substeps=4, device=local)
    gpu_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oe, ob, _ = OF.select_lambda(Us.T, As.T, Ss.T, v0, r=sample_r, lambdas=lams, dt=1e-6, k=4, r_s=gs["r_s"])
    cpu_s = time.perf_counter() - t0
    fin = np.isfinite(oe)
    agree = bool(gs["best"] == ob) and bool(np.all(np.abs(gs["errors"][fin] - oe[fin]) <= 1e-6 * oe[fin] + 1e-9))
    log(f"opinf_select: GPU {gpu_full:.1f}s (full), sample GPU {gpu_s:.1f}s vs oracle {cpu_s:.1f}s")
    return {"candidates": [float(x) for x in lams], "unit": "s", "higher_is_better": False,
            "gpu_seconds": gpu_full, "errors": [float(x) for x in full["errors"]], "selected_lambda": full["lambda"],
            "workload": f"{fit_info['n_snap']} snapshots x {fit_info['n_dof']} free dofs, r={fit_info['r']}, "
                        f"r_s={fit_info['r_s']}, 11 rollouts of {4 * (fit_info['n_snap'] - 1)} steps",
            "sample": f"first {sample_snaps} snapshots, r={sample_r}, r_s={gs['r_s']}, 11 candidates",
            "sample_gpu_seconds": gpu_s, "sample_oracle_seconds": cpu_s, "oracle_threads": os.cpu_count(),
            "sample_speedup_vs_oracle": cpu_s / gpu_s, "sample_agrees_with_oracle": agree}


def measure_adjoint(W, osam, local, log, oracle_steps=40):
    """Checkpointed adjoint of the 20x20x40 Neo-Hookean bar (1000 steps, checkpoints every 50): J and its
    gradients w.r.t. u0, v0, lambda_e, mu_e on the GPU, against the oracle's adjoint of the same bar on
    a bounded number of steps."""
    from oracle import oracle as O
    p, w = W.adjoint_bar()
    sd = p.subdomains[0]
    n = p.info["n_steps"]
    args = (sd.dims, sd.h, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, sd.u0, None, p.dt, n, w)
    osam.adjoint(*args, checkpoint_every=50, device=local)  # warm-up
    reps = [osam.adjoint(*args, checkpoint_every=50, device=local)["elapsed_ms"] for _ in range(3)]
    gpu_ms = min(reps)
    t0 = time.process_time()
    O.adjoint(sd.dims, sd.h, sd.origin, "nh", sd.lam_e, sd.mu_e, sd.rho, sd.dirichlet, sd.u0, None, p.dt,
              oracle_steps, w)
    cpu_s = time.process_time() - t0
    ne = sd.n_elements
    gpu_rate = ne * n / (gpu_ms * 1e-3)
    cpu_rate = ne * oracle_steps / cpu_s
    log(f"adjoint: GPU {gpu_ms:.1f} ms for {n} steps, oracle {cpu_s:.1f}s for {oracle_steps} steps")
    return {"workload": f"adjoint_bar {sd.dims[0]}x{sd.dims[1]}x{sd.dims[2]} Neo-Hookean, per-element Lame "
                        f"parameters, {n} steps, checkpoints every 50",
            "unit": "element-steps/s (forward + reverse)", "value": gpu_rate, "ms": gpu_ms,
            "oracle_value": cpu_rate, "oracle_cores": 1,
            "oracle_sample": f"the same bar, {oracle_steps} steps, {cpu_s:.1f} s CPU", "speedup_vs_oracle": gpu_rate / cpu_rate,
            "timing": "library CUDA events around the whole adjoint call (best of 3 after a warm-up)"}


def measure_implicit(W, osam, torch, flush, rom_ops, args, local, log, steps=2, oracle_dims=(4, 4, 8),
                     max_iters=None, warmup=1):
    """Implicit Newmark FOM (beta = 1/4, gamma = 1/2; Newton with mass-preconditioned matrix-free CG)
    in the headline hybrid: the same 40x40x80 Neo-Hookean FOM and fitted ROM, the FOM integrated
    implicitly at the same dt (host-driven steps, no graph).  Metric as the headline (FOM
    element-updates/s) plus Newton / CG counts and the tangent-action kernel's FP64 roofline; the
    oracle (dense assembled tangent, Cholesky) and the GPU on a bounded sample: a small implicit
    Neo-Hookean bar."""
    from oracle import oracle as O
    spec = hybrid_spec(W, args)
    spec.subdomains[0].integrator = "implicit"
    if max_iters:
        spec.max_iters = max_iters

    def run(precision):
        tag = "implicit_tangent32" if precision == osam.FP64_TANGENT32 else "implicit_f64"
        prob = osam.Problem(spec, rom_ops=rom_ops, device=local, precision=precision)
        for _ in range(warmup):
            prob.step()
        # the library's default path (the controller step as one graph, Newton and CG as device-side
        # WHILE loops); then the host-driven loop with CUDA events around every tangent launch
        prob.profile(False)
        total_ms, upd, its = 0.0, 0, []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            r = prob.step()
            total_ms += r["elapsed_ms"]
            upd += r["element_updates"]
            its.append(r["iterations"])
        prob.profile(True)
        p_ms, p_its = 0.0, []
        torch.cuda.nvtx.range_push(tag + "_host")
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            r = prob.step()
            p_ms += r["elapsed_ms"]
            p_its.append(r["iterations"])
        torch.cuda.nvtx.range_pop()
        ip = prob.implicit_profile()
        prof = prob.profile_read()
        prob.profile(False)
        prob.close()
        return total_ms, upd, its, p_ms, p_its, ip, prof

    total_ms, upd, its, p_ms, p_its, ip, prof = run(osam.FP64)
    ne = spec.subdomains[0].n_elements
    substeps = 20 * sum(p_its)
    achieved = TANGENT_FLOPS_PER_NH_ELEMENT * ip["tangent_elements"] / (ip["tangent_ms"] * 1e-3) / 1e12
    # the same with the Neo-Hookean Newton tangent in FP32 (OSAM_FP64_TANGENT32): residual, Newton test
    # and CG vectors in FP64; its tangent kernel moves the FP32 linearisation (704 B per element), reads
    # p and writes the FP32 element buffer (96 B per element, L2-resident) -- an HBM-bound kernel
    t_ms, t_upd, t_its, tp_ms, tp_its, tip, _ = run(osam.FP64_TANGENT32)
    t_sub = 20 * sum(tp_its)
    t_launch_ms = tip["tangent_ms"] / max(1, tip["tangent_launches"])
    t_bytes = ne * TANGENT32_BYTES_PER_ELEMENT
    hbm_peak, hbm_kind = measured_hbm_gbs()
    t_gbs = t_bytes / (t_launch_ms * 1e-3) / 1e9 if t_launch_ms > 0 else None
    fp32_tangent = {
        "value": t_upd / (t_ms * 1e-3), "ms_per_step": t_ms / steps, "mean_iterations": float(np.mean(t_its)),
        "newton_per_substep": tip["newton_steps"] / max(1, t_sub),
        "cg_per_newton": tip["cg_iterations"] / max(1, tip["newton_steps"]),
        "ms_per_step_host_loop": tp_ms / steps,
        "tangent_time_share": tip["tangent_ms"] / tp_ms if tp_ms else None,
        "roofline": {"bound": "hbm", "kernel": "k_tangent_lin32_b (Neo-Hookean, FP32)",
                     "achieved": t_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": t_gbs / hbm_peak if (t_gbs and hbm_peak) else None, "peak_kind": hbm_kind,
                     "algorithmic_bytes_per_launch": t_bytes, "ms_per_launch": t_launch_ms,
                     "traffic": (TANGENT32_TRAFFIC["bytes_per_launch"]
                                 if TANGENT32_TRAFFIC["source_sha256"] == source_sha(TANGENT_SOURCES) else None)},
        "speedup_vs_fp64_tangent": (t_upd / t_ms) / (upd / total_ms),
        "parity": "1e-9 relative L2 vs the oracle, 1e-10 vs the FP64 tangent (tests/test_gpu_implicit.py)"}
    log(f"implicit, FP32 tangent: {t_ms / steps:.1f} ms/step, {fp32_tangent['newton_per_substep']:.2f} "
        f"Newton/substep, {fp32_tangent['cg_per_newton']:.1f} CG/Newton, tangent {t_launch_ms * 1e3:.1f} us/launch")
    # bounded sample: a small implicit Neo-Hookean bar, 1 controller step of 4 substeps, both sides
    sample = W.single_bar("imp_sample", oracle_dims[0], oracle_dims[2], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 4)
    sample.subdomains[0].integrator = "implicit"
    g = osam.Problem(sample, device=local)
    g.step()
    rg = g.step()
    g.close()
    ref = O.Problem(sample)
    t0 = time.process_time()
    ref.step()
    cpu_s = time.process_time() - t0
    ns = sample.subdomains[0].n_elements * 4
    log(f"implicit: {total_ms / steps:.1f} ms/step, {ip['newton_steps'] / max(1, substeps):.2f} Newton/substep, "
        f"{ip['cg_iterations'] / max(1, ip['newton_steps']):.1f} CG/Newton, tangent {achieved:.3f} TFLOP/s")
    return {"workload": f"fom_opinf_hybrid {args.n}x{args.n}x{args.nz} Neo-Hookean FOM integrated implicitly "
                        f"(Newmark beta=1/4, gamma=1/2) + r={args.rank} OpInf ROM, dt=1e-6, 20 substeps",
            "unit": UNIT, "value": upd / (total_ms * 1e-3), "ms_per_step": total_ms / steps, "steps": steps,
            "mean_iterations": float(np.mean(its)),
            "newton_per_substep": ip["newton_steps"] / max(1, substeps),
            "cg_per_newton": ip["cg_iterations"] / max(1, ip["newton_steps"]),
            "ms_per_step_host_loop": p_ms / steps,
            "tangent_time_share": ip["tangent_ms"] / p_ms if p_ms else None,
            "roofline": {"bound": "alu", "kernel": "k_tangent_lin_b (Neo-Hookean)", "achieved": achieved,
                         "peak": FP64_PEAK[0], "unit": "TFLOP/s", "frac": achieved / FP64_PEAK[0],
                         "traffic": (TANGENT_TRAFFIC["bytes_per_launch"]
                                     if TANGENT_TRAFFIC["source_sha256"] == source_sha(TANGENT_SOURCES) else None),
                         "algorithmic_bytes_per_launch": ne * TANGENT_BYTES_PER_ELEMENT,
                         "flops_per_element": TANGENT_FLOPS_PER_NH_ELEMENT,
                         "ms_per_launch": ip["tangent_ms"] / max(1, ip["tangent_launches"]),
                         "peak_kind": FP64_PEAK_KIND[0]},
            "timing": "value: library CUDA events around each controller step, each one graph launch with the "
                      "Newton and CG loops as device-side WHILE nodes (L2 flushed between steps); roofline and "
                      "counts: a second pass of the same steps driven from the host with CUDA events around "
                      "every tangent launch",
            "kernel_launches": prof["kernel_launches"],
            "sample": f"implicit Neo-Hookean bar {oracle_dims[0]}x{oracle_dims[1]}x{oracle_dims[2]}, 1 controller "
                      f"step of 4 substeps",
            "sample_gpu_value": ns * rg["iterations"] / (rg["elapsed_ms"] * 1e-3),
            "sample_oracle_value": ns / cpu_s, "oracle_cores": 1,
            "parity": "1e-9 relative L2 vs the oracle (tests/test_gpu_implicit.py)",
            "fp32_tangent": fp32_tangent}


def _timed_steps(prob, torch, flush, steps, warmup):
    for _ in range(warmup):
        prob.step()
    ms, upd, its = 0.0, 0, []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        r = prob.step()
        ms += r["elapsed_ms"]
        upd += r["element_updates"]
        its.append(r["iterations"])
    return ms, upd, its


def _sample_pair(W, osam, spec, rom_ops, local, n_steps=2):
    """The same variant on a small seeded problem, GPU and oracle side by side (element-updates/s of
    the FOM subdomains; oracle on one core)."""
    from oracle import oracle as O
    g = osam.Problem(spec, rom_ops=rom_ops, device=local)
    g.step()
    gms, gupd = 0.0, 0
    for _ in range(n_steps):
        r = g.step()
        gms += r["elapsed_ms"]
        gupd += r["element_updates"]
    g.close()
    ref = O.Problem(spec, rom_ops=rom_ops)
    t0 = time.process_time()
    its = [ref.step()["iterations"] for _ in range(n_steps)]
    cpu = time.process_time() - t0
    upd = sum(it * sum((sd.n_substeps or spec.n_substeps) * sd.n_elements for sd in spec.subdomains
                       if sd.kind == "fom") for it in its)
    return {"sample_gpu_value": gupd / (gms * 1e-3), "sample_oracle_value": upd / cpu, "oracle_cores": 1}


def _small_cubic_rom(W, spec_ff, i, r):
    from oracle import fit as OF
    from oracle import oracle as O
    prob = O.Problem(spec_ff)
    free, sdof = prob.free_dofs(i), prob.schwarz_dofs(i)
    U, A, S = [], [], []
    for _ in range(40):
        prob.step()
        u, _, a = prob.state(i)
        U.append(u.reshape(-1)[free]); A.append(a.reshape(-1)[free]); S.append(u.reshape(-1)[sdof])
    return OF.opinf_fit(np.array(U).T, np.array(A).T, np.array(S).T, r=r, lam=1e-6, r_s=4, cubic=True)


def measure_next_rows(W, osam, torch, flush, rom_ops, args, local, log, steps=5, warmup=2):
    """The headline hybrid under the method's other variants (each a parity-tested path):
    additive sweeps (FOM and ROM concurrently on their own streams), mixed time integrators and steps
    (the FOM implicit with 2 substeps of 10 us per controller step, the ROM explicit with 20 of 1 us,
    coupled through the temporal interpolant), and the Saint Venant-Kirchhoff FOM with a cubic OpInf
    ROM (r = 20, fitted on the GPU from a Saint Venant-Kirchhoff FOM-FOM run).  Metric as the headline,
    plus the controller intervals advanced per second (T = 20 us each)."""
    out = {}
    T = 20e-6
    spec = hybrid_spec(W, args)
    spec.schwarz = "additive"
    prob = osam.Problem(spec, rom_ops=rom_ops, device=local)
    ms, upd, its = _timed_steps(prob, torch, flush, steps, warmup)
    prob.close()
    out["additive"] = {"value": upd / (ms * 1e-3), "ms_per_step": ms / steps, "mean_iterations": float(np.mean(its)),
                       "intervals_per_s": steps / (ms * 1e-3),
                       "workload": "headline hybrid, additive sweeps (FOM and ROM on their own streams)"}
    spec = hybrid_spec(W, args)
    spec.subdomains[0].integrator = "implicit"
    spec.subdomains[0].n_substeps = 2
    prob = osam.Problem(spec, rom_ops=rom_ops, device=local)
    ms, upd, its = _timed_steps(prob, torch, flush, max(2, steps // 2), 1)
    prob.close()
    prob = osam.Problem(spec, rom_ops=rom_ops, device=local, precision=osam.FP64_TANGENT32)
    t_ms, t_upd, t_its = _timed_steps(prob, torch, flush, max(2, steps // 2), 1)
    prob.close()
    n = max(2, steps // 2)
    out["mixed_implicit_explicit"] = {
        "value": upd / (ms * 1e-3), "ms_per_step": ms / n, "mean_iterations": float(np.mean(its)),
        "intervals_per_s": n / (ms * 1e-3),
        "fp32_tangent": {"value": t_upd / (t_ms * 1e-3), "ms_per_step": t_ms / n,
                         "mean_iterations": float(np.mean(t_its)), "intervals_per_s": n / (t_ms * 1e-3)},
        "workload": "headline hybrid, FOM implicit (Newmark 1/4, 1/2) with 2 substeps of 10 us, ROM explicit with "
                    "20 substeps of 1 us, temporal interpolant between them (each controller step one graph launch, "
                    "Newton and CG as device-side loops)"}
    svk_ops, svk_fit = train_rom(W, osam, args, local, log, material="svk", rank=20, cubic=True, snapshots=300)
    spec = W.bar_chain("svk_copinf", args.n, [args.nz, args.nz], ["fom", "rom"], "svk", 1e9, 0.3, 1000.0, 1e-3,
                       1e-6, 20, max_iters=64)
    prob = osam.Problem(spec, rom_ops={1: svk_ops}, device=local)
    ms, upd, its = _timed_steps(prob, torch, flush, steps, warmup)
    p_ms, p_upd, _, prof = timed_pass(prob, torch, flush, 2, profile=True)
    prob.close()
    achieved = FLOPS_PER_SVK_ELEMENT * prof["force_elements"] / (prof["force_ms"] * 1e-3) / 1e12
    out["svk_copinf"] = {
        "value": upd / (ms * 1e-3), "ms_per_step": ms / steps, "mean_iterations": float(np.mean(its)),
        "intervals_per_s": steps / (ms * 1e-3),
        "workload": f"{args.n}x{args.n}x{args.nz} Saint Venant-Kirchhoff FOM + cubic OpInf ROM r=20 "
                    f"(r_s={svk_fit['r_s']}, fitted on {svk_fit['n_snap']} snapshots of an SVK FOM-FOM run)",
        "fit_seconds": svk_fit["gpu_seconds"],
        "roofline": {"bound": "alu", "kernel": "k_force_*<SaintVenantKirchhoff>", "achieved": achieved,
                     "peak": FP64_PEAK[0], "unit": "TFLOP/s", "frac": achieved / FP64_PEAK[0],
                     "flops_per_element": FLOPS_PER_SVK_ELEMENT,
                     "force_ms_per_launch": prof["force_ms"] / max(1, prof["force_launches"])}}
    # oracle beside each variant, on a small bar of the same kind (3x3x[8,8] FOMs, 20 substeps)
    small = W.bar_chain("s_add", 3, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20, max_iters=64)
    small.schwarz = "additive"
    out["additive"].update(_sample_pair(W, osam, small, None, local),
                           sample="3x3x8 + 3x3x8 Neo-Hookean FOM-FOM bar, additive, 2 controller steps")
    small = W.bar_chain("s_mix", 3, [8, 8], ["fom", "fom"], "nh", 1e9, 0.25, 1000.0, 1e-3, 1e-6, 20, max_iters=64)
    small.subdomains[0].integrator = "implicit"
    small.subdomains[0].n_substeps = 2
    out["mixed_implicit_explicit"].update(
        _sample_pair(W, osam, small, None, local),
        sample="3x3x8 + 3x3x8 Neo-Hookean bar, FOM 0 implicit 2 x 10 us, FOM 1 explicit 20 x 1 us, 2 controller steps")
    small_ff = W.bar_chain("s_svkff", 3, [8, 8], ["fom", "fom"], "svk", 1e9, 0.3, 1000.0, 1e-3, 1e-6, 4)
    small = W.bar_chain("s_svk", 3, [8, 8], ["fom", "rom"], "svk", 1e9, 0.3, 1000.0, 1e-3, 1e-6, 20, max_iters=64)
    out["svk_copinf"].update(_sample_pair(W, osam, small, {1: _small_cubic_rom(W, small_ff, 1, 6)}, local),
                             sample="3x3x8 SVK FOM + cubic ROM r=6 (oracle-fitted on 40 snapshots), 2 controller steps")
    for k, v in out.items():
        log(f"{k}: {v['value']:.3e} element-updates/s, {v['ms_per_step']:.2f} ms/step, {v['mean_iterations']:.1f} its; "
            f"sample GPU {v['sample_gpu_value']:.3e} vs oracle {v['sample_oracle_value']:.3e}")
    out["note"] = (f"intervals_per_s: controller intervals of {T * 1e6:.0f} us advanced per second; "
                   "parity: tests/test_gpu_additive.py, test_gpu_mixed_dt.py, test_gpu_svk.py, test_gpu_cubic.py")
    return out


# FP32 FMA peak of the FP32-force variant (152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz)
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def train_large_rom(W, osam, torch, args, device, log):
    """The middle ROM of the large chain: a seeded FOM-FOM-FOM training run of the same geometry
    (controller steps of 4 substeps, one snapshot of the middle subdomain per step, double-float
    force, snapshots kept on the device), then the library's opinf_fit of rank args.large_rank."""
    rng = np.random.default_rng(W.SEED_BASE + 5)
    amp = float(rng.uniform(0.5e-3, 1.0e-3))
    spec = W.large_chain(args.large_n, args.large_nz, rom_middle=False, amplitude=amp, n_substeps=4)
    dev = f"cuda:{device}"
    free, sdof = W.subdomain_dof_masks(spec, 1)
    fi = torch.from_numpy(np.flatnonzero(free)).to(dev)
    si = torch.from_numpy(np.flatnonzero(sdof)).to(dev)
    n_snap = args.large_snapshots
    U = torch.empty((n_snap, fi.numel()), dtype=torch.float64, device=dev)
    A = torch.empty_like(U)
    S = torch.empty((n_snap, si.numel()), dtype=torch.float64, device=dev)
    nn = spec.subdomains[1].n_nodes
    bu = torch.empty((nn, 3), dtype=torch.float64, device=dev)
    ba = torch.empty_like(bu)
    prob = osam.Problem(spec, precision=osam.F32X2_FORCE, device=device)
    t0 = time.time()
    for k in range(n_snap):
        prob.step()
        prob.state(1, out=(bu, None, ba))
        uf, af = bu.reshape(-1), ba.reshape(-1)
        U[k] = uf[fi]
        A[k] = af[fi]
        S[k] = uf[si]
    torch.cuda.synchronize()
    prob.close()
    train_s = time.time() - t0
    t0 = time.time()
    ops = osam.opinf_fit(U, A, S, r=args.large_rank, lam=1e-6, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, device=device)
    fit_s = time.time() - t0
    info = {"training_seconds": train_s, "fit_seconds": fit_s, "n_snap": n_snap, "n_dof": int(fi.numel()),
            "n_sdof": int(si.numel()), "r": args.large_rank, "r_s": int(ops["r_s"]), "amplitude": amp}
    del U, A, S
    torch.cuda.empty_cache()
    log(f"large chain: training run {n_snap} x 4 substeps in {train_s:.1f}s, opinf_fit r={args.large_rank} "
        f"r_s={ops['r_s']} over {info['n_dof']} dofs in {fit_s:.1f}s")
    return {k: ops[k] for k in ("Phi", "Phi_S", "K", "H", "B", "c")}, info


def measure_large(W, osam, torch, flush, args, local, log, warmup=3):
    """The large chain: two n x n x nz Neo-Hookean FOMs with the quadratic OpInf ROM (rank
    args.large_rank, fitted on the GPU from the chain's own FOM-FOM-FOM training run) in the middle,
    dt = 5e-7, controller steps of 20 substeps.  FP64 (the library's default graph-captured steps)
    and the FP32-force variant (FP32 element force, FP64 state), each with its force kernel's
    roofline from a host-driven pass with CUDA events around every force launch.  The FP32-force
    rounding noise keeps the relative criterion above 1e-12, so that variant runs with its iteration
    count fixed to the largest FP64 count (same work per step); beside them the oracle on a bounded
    sample of the same chain."""
    ops, info = train_large_rom(W, osam, torch, args, local, log)
    out = {"workload": f"large_chain {args.large_n}x{args.large_n}x{args.large_nz} Neo-Hookean FOM - quadratic OpInf "
                       f"ROM r={args.large_rank} (r_s={info['r_s']}, fitted on {info['n_snap']} snapshots of "
                       f"{info['n_dof']} free dofs) - FOM, dt=5e-7, 20 substeps per controller step",
           "unit": UNIT, "fit": info}
    max_its = None
    for name, prec in (("f64", osam.FP64), ("fp32_force", osam.FP32_FORCE)):
        spec = W.large_chain(args.large_n, args.large_nz, rom_middle=True)
        if max_its is not None:
            spec.max_iters = max_its
        prob = osam.Problem(spec, rom_ops={1: ops}, device=local, precision=prec)
        ms, upd, its = _timed_steps(prob, torch, flush, args.large_steps, warmup)
        p_ms, p_upd, _, prof = timed_pass(prob, torch, flush, 2, profile=True)
        tuning = prob.tuning()
        prob.close()
        if max_its is None:
            max_its = int(max(its))
        per_launch = prof["force_ms"] / max(1, prof["force_launches"])
        achieved = FLOPS_PER_NH_ELEMENT * prof["force_elements"] / (prof["force_ms"] * 1e-3) / 1e12
        peak = FP64_PEAK[0] if name == "f64" else FP32_FMA_PEAK_TFLOPS
        out[name] = {"value": upd / (ms * 1e-3), "ms_per_step": ms / args.large_steps, "steps": args.large_steps,
                     "warmup": warmup, "mean_iterations": float(np.mean(its)), "max_iterations": int(max(its)),
                     "effective_rate": upd / (ms * 1e-3) / float(np.mean(its)),
                     "value_host_loop": p_upd / (p_ms * 1e-3), "tuning": tuning,
                     "roofline": {"bound": "alu", "kernel": "internal force (Neo-Hookean, %s)" % name,
                                  "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                  "flops_per_element": FLOPS_PER_NH_ELEMENT, "elements_per_launch":
                                  spec.subdomains[0].n_elements, "force_ms_per_launch": per_launch,
                                  "force_time_share": prof["force_ms"] / p_ms,
                                  "peak_kind": (FP64_PEAK_KIND[0] if name == "f64"
                                                else "FP32 FMA: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"),
                                  "frac_of_nominal": (achieved / FP64_NOMINAL_TFLOPS if name == "f64" else None)}}
        if name == "fp32_force":
            out[name]["iterations"] = f"fixed at {max_its} (the largest FP64 count)"
        log(f"large chain [{name}]: {out[name]['value']:.3e} element-updates/s, {ms / args.large_steps:.1f} ms/step, "
            f"{np.mean(its):.1f} its, force {per_launch:.3f} ms/launch = {achieved:.3f} TFLOP/s")
    # oracle on a bounded sample: the same chain, one controller step of one substep and one Schwarz
    # iteration, seeded stand-in ROM operators of the fitted sizes (the set-up is not timed)
    from oracle import oracle as O
    spec = W.large_chain(args.large_n, args.large_nz, rom_middle=True, n_substeps=1)
    spec.max_iters = 1
    free, sdof = W.subdomain_dof_masks(spec, 1)
    stand_in = W.synthetic_rom_operators(int(free.sum()), int(sdof.sum()), args.large_rank, info["r_s"],
                                         W.SEED_BASE + 15)
    ref = O.Problem(spec, rom_ops={1: stand_in})
    t0 = time.process_time()
    ref.step()
    cpu_s = time.process_time() - t0
    cpu_upd = 2 * spec.subdomains[0].n_elements
    out["oracle"] = {"value": cpu_upd / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                     "sample": f"1 controller step of 1 substep x 1 Schwarz iteration of the same chain (stand-in ROM "
                               f"operators of the fitted sizes), {cpu_s:.1f} s CPU"}
    out["parity"] = ("1e-9 (FP64), 1e-5 (FP32 force) relative L2 vs the oracle on a truncated horizon of the full "
                     "chain (tests/test_gpu_fullsize.py)")
    return out


def fit_only(W, osam, torch, args, local, log):
    """One GPU fit of seeded synthetic snapshots shaped like the headline training set: U = low-rank
    signal (decaying mode weights) + noise over the ROM subdomain's free dofs, A and S likewise."""
    dev = f"cuda:{local}"
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.SEED_BASE + 17)
    # the 40x40x80 ROM mesh: 41 x 41 x 81 nodes, the Schwarz face z = 0 excluded from the free dofs
    ns, n_dof, n_sdof = args.snapshots, 3 * 41 * 41 * 80, 3 * 41 * 41
    k = args.rank + 16
    w = torch.pow(0.8, torch.arange(k, dtype=torch.float64, device=dev))
    modes = torch.randn((k, n_dof), generator=gen, dtype=torch.float64, device=dev)
    U = (torch.randn((ns, k), generator=gen, dtype=torch.float64, device=dev) * w) @ modes
    U += 1e-6 * torch.randn((ns, n_dof), generator=gen, dtype=torch.float64, device=dev)
    A = (torch.randn((ns, k), generator=gen, dtype=torch.float64, device=dev) * w) @ modes
    S = torch.randn((ns, n_sdof), generator=gen, dtype=torch.float64, device=dev)
    del modes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    osam.opinf_fit(U, A, S, r=args.rank, lam=1e-6, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, device=local)
    secs = time.perf_counter() - t0
    osam.fit_profile(True)
    osam.opinf_fit(U, A, S, r=args.rank, lam=1e-6, r_s=0, energy_s=1.0 - 1e-6, r_s_max=64, device=local)
    prof = osam.fit_profile(False)
    achieved = prof["gemm_flops"] / (prof["gemm_ms"] * 1e-3) / 1e12
    # Algorithm 3 on the same snapshots (11 candidates, rollouts 4 steps apart): the selection kernels
    # (random snapshots are no dynamical system: every rollout may blow up, which the selection reports)
    t0 = time.perf_counter()
    try:
        best = int(osam.opinf_select(U, A, S, None, args.rank, np.logspace(-10, 0, 11), 1e-6, 4, r_s=0,
                                     energy_s=1.0 - 1e-6, r_s_max=64, device=local)["best"])
    except osam.OsamError as err:
        best = f"none ({err})"
    sel_s = time.perf_counter() - t0
    log(f"fit-only: {ns} x {n_dof}, r={args.rank}: {secs:.2f} s, GEMMs {achieved:.3f} TFLOP/s; selection {sel_s:.2f} s")
    return {"n_snap": ns, "n_dof": n_dof, "r": args.rank, "seconds": secs, **prof, "gemm_tflops": achieved,
            "select_seconds": sel_s, "select_best": best}


def measure_fom_fom_plain(W, osam, local, log, repeats=10):
    """FOM-FOM plain: two 6x6x12 linear-elastic FOMs (global 6x6x22), 200 steps in 10 controller steps
    of 20 substeps, relative tolerance 1e-12, at most 64 Schwarz iterations -- the whole run, repeated,
    as graph-captured controller steps and from the host loop (the latency-bound configuration where
    the graph matters most); beside it the oracle over the whole run on one core."""
    from oracle import oracle as O
    out = {"workload": "fom_fom_plain 2 x 6x6x12 linear elastic, 10 controller steps of 20 substeps (the whole "
                       "200-step run), tol 1e-12, max 64 iterations", "unit": UNIT, "repeats": repeats}
    for mode in ("graph", "host_loop"):
        ms, wall, upd, its = 0.0, 0.0, 0, []
        for rep in range(repeats + 1):          # the first run is a warm-up
            spec = W.fom_fom_plain()
            prob = osam.Problem(spec, device=local)
            prob.set_graph(mode == "graph")
            t0 = time.perf_counter()
            run_ms, run_upd, run_its = 0.0, 0, []
            for _ in range(spec.n_controller_steps):
                r = prob.step()
                run_ms += r["elapsed_ms"]
                run_upd += r["element_updates"]
                run_its.append(r["iterations"])
            run_wall = time.perf_counter() - t0
            prob.close()
            if rep:
                ms += run_ms
                wall += run_wall
                upd += run_upd
                its += run_its
        out[mode] = {"value": upd / (ms * 1e-3), "value_wall": upd / wall, "ms_per_run": ms / repeats,
                     "ms_per_step": ms / (repeats * 10), "mean_iterations": float(np.mean(its)),
                     "max_iterations": int(max(its))}
    spec = W.fom_fom_plain()
    ref = O.Problem(spec)
    t0 = time.process_time()
    o_its = [ref.step()["iterations"] for _ in range(spec.n_controller_steps)]
    cpu_s = time.process_time() - t0
    o_upd = sum(o_its) * spec.n_substeps * sum(sd.n_elements for sd in spec.subdomains)
    out["oracle"] = {"value": o_upd / cpu_s, "seconds_per_run": cpu_s, "cores": 1, "kind": "oracle",
                     "mean_iterations": float(np.mean(o_its)), "sample": "the whole 200-step run"}
    out["timing"] = ("value: the library's CUDA events around every controller step (graph build excluded); "
                     "value_wall: host wall clock around the run's step calls")
    out["parity"] = "1e-9 relative L2 vs the oracle over all 200 steps (tests/test_gpu_parity.py)"
    log(f"fom_fom_plain: graph {out['graph']['value']:.3e}, host loop {out['host_loop']['value']:.3e}, oracle "
        f"{out['oracle']['value']:.3e} element-updates/s; {out['graph']['mean_iterations']:.1f} its")
    return out


def hybrid_spec(W, args):
    return W.fom_opinf_hybrid(args.n, args.nz, rom=True)


# ---------------------------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------------------------
def oracle_sample_problem(W, args, n_substeps):
    """The hybrid workload for the oracle with seeded stand-in ROM operators of the same sizes and one
    Schwarz iteration per controller step (a bounded sample of the same FOM work)."""
    spec = hybrid_spec(W, args)
    spec.n_substeps = n_substeps
    spec.max_iters = 1
    sd = spec.subdomains[1]
    n_sdof = 3 * (args.n + 1) ** 2
    n_free = 3 * sd.n_nodes - n_sdof
    ops = W.synthetic_rom_operators(n_free, n_sdof, args.rank, 32, W.SEED_BASE + 11)
    return spec, {1: ops}


def cpu_oracle_rate(W, args, n_substeps, min_seconds, max_steps=None):
    from oracle import oracle as O
    spec, ops = oracle_sample_problem(W, args, n_substeps)
    prob = O.Problem(spec, rom_ops=ops)
    ne = spec.subdomains[0].n_elements
    steps, elapsed = 0, 0.0
    while elapsed < min_seconds and (max_steps is None or steps < max_steps):
        t0 = time.process_time()
        prob.step()
        elapsed += time.process_time() - t0
        steps += 1
    return steps * n_substeps * ne / elapsed, steps, elapsed


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2511_20687_gb300 import workloads as W
    n_sub = 5
    spec, ops = oracle_sample_problem(W, args, n_sub)
    from oracle import oracle as O
    prob = O.Problem(spec, rom_ops=ops)
    ne = spec.subdomains[0].n_elements
    for _ in range(args.warmup):
        prob.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prob.step()
    dt = time.perf_counter() - t0
    value = args.steps * n_sub * ne / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"fom_opinf_hybrid {args.n}x{args.n}x{args.nz} NH FOM + r={args.rank} OpInf ROM",
                       "sample": f"{n_sub} substeps x 1 Schwarz iteration per step, seeded stand-in ROM operators",
                       "l2": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"{args.steps} controller steps of {n_sub} substeps, 1 Schwarz iteration each"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def combine_ranks(pairs, device):
    """Whole-job figures of replicas: for every (milliseconds, element-updates) pair, the maximum time
    and the summed updates over all ranks (identity on a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [(float(ms), int(u)) for ms, u in pairs]
    ms = torch.tensor([float(p[0]) for p in pairs], dtype=torch.float64, device=device)
    up = torch.tensor([float(p[1]) for p in pairs], dtype=torch.float64, device=device)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(up, op=dist.ReduceOp.SUM)
    return [(float(a), int(b)) for a, b in zip(ms.tolist(), up.tolist())]


def shard_samples(sizes, world):
    """Split samples over `world` ranks by their element counts: largest first, each to the rank with
    the least work so far (ties to the lowest rank); returns each rank's sample indices, ascending."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def gather_reports(mine):
    """Every rank's {sample index: report} gathered on every rank and merged (identity on one
    process); the data-path needs no exchange, this is the sweep's only collective."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dict(mine)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(mine))
    out = {}
    for p in parts:
        out.update(p)
    return out


def timed_pass(prob, torch, flush, steps, profile):
    """`steps` controller steps with CUDA-event timing per step (L2 flushed in between, outside the
    timing).  profile=True brackets every force launch with CUDA events (host-driven iterations)."""
    prob.profile(profile)
    prob.set_graph(not profile)
    torch.cuda.synchronize()
    total_ms, updates, iters = 0.0, 0, []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        r = prob.step()
        total_ms += r["elapsed_ms"]
        updates += r["element_updates"]
        iters.append(r["iterations"])
    torch.cuda.synchronize()
    prof = prob.profile_read()
    prob.profile(False)
    return total_ms, updates, iters, prof


def e2e_pass(prob, torch, steps, rank_r):
    """Same metric through the public API with pinned host buffers: state in, step, state out, on the
    library's default path (graph-captured controller steps; the profiling pass before this one drives
    the steps from the host)."""
    prob.set_graph(True)
    nA = prob.sizes(0)["n_nodes"]
    hu = [torch.empty((nA, 3), dtype=torch.float64).pin_memory() for _ in range(3)]
    hq = [torch.empty(rank_r, dtype=torch.float64).pin_memory() for _ in range(3)]
    prob.state(0, out=tuple(hu))
    q = prob.reduced_state(1)
    for k in range(3):
        hq[k].copy_(torch.from_numpy(q[k]))
    updates = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        prob.set_state(0, hu[0], hu[1], hu[2])
        prob.set_reduced_state(1, hq[0], hq[1], hq[2])
        r = prob.step()
        updates += r["element_updates"]
        prob.state(0, out=tuple(hu))
        out_q = prob.reduced_state(1)
        for k in range(3):
            hq[k].copy_(torch.from_numpy(out_q[k]))
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    io_bytes = 3 * nA * 3 * 8 + 3 * rank_r * 8
    return {"value": updates / secs, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
            "seconds": secs, "updates": updates}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch

    def log(msg):
        if rank == 0:
            print(f"[bench] {msg}", file=sys.stderr, flush=True)

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2511_20687_gb300 import build_lib
    if rank == 0:
        build_lib.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2511_20687_gb300 import osam
    from paper_2511_20687_gb300 import workloads as W

    fit_info = None
    fp64_peak = (measure_fp64_peak(osam, local, args.fp64_peak_repeats) if args.fp64_peak_repeats > 0 else
                 {"tflops": FP64_NOMINAL_TFLOPS, "kind": "nominal (probes skipped)", "fma_best": None,
                  "mma_best": None, "fma_plus_mma_interleaved_best": None, "sm_mhz": None})
    log(f"FP64 peak: {fp64_peak['tflops']:.3f} TFLOP/s ({fp64_peak['kind']}; FMA {fp64_peak['fma_best']}, tensor-core "
        f"MMA {fp64_peak['mma_best']}, interleaved {fp64_peak['fma_plus_mma_interleaved_best']}, {fp64_peak['sm_mhz']} MHz)")
    if args.fit_only:
        print(json.dumps({"fit_only": fit_only(W, osam, torch, args, local, log)}), flush=True)
        return
    if args.large_only:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
        print(json.dumps({"large_chain": measure_large(W, osam, torch, flush, args, local, log),
                          "fp64_peak": fp64_peak}), flush=True)
        return
    if args.implicit_only:
        # profiling entry: the implicit-FOM block alone, with seeded stand-in ROM operators of the
        # fitted model's sizes and at most 3 Schwarz iterations per controller step
        spec, ops = oracle_sample_problem(W, args, 20)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
        res = measure_implicit(W, osam, torch, flush, ops, args, local, log, steps=args.steps, max_iters=3,
                               warmup=args.warmup)
        print(json.dumps({"implicit": res}), flush=True)
        return
    if args.fom_only:
        spec = W.fom_opinf_hybrid(args.n, args.nz, rom=False)
        rom_ops = None
    else:
        hyb_ops, fit_info = train_rom(W, osam, args, local, log)
        rom_ops = {1: hyb_ops}
        spec = hybrid_spec(W, args)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    head_prec = osam.F32X2_FORCE if args.precision == "f32x2" else osam.FP64
    results = {}
    for prec in ([head_prec] + [p for p in (osam.FP64, osam.F32X2_FORCE) if p != head_prec]):
        name = "f32x2" if prec == osam.F32X2_FORCE else "f64"
        scatter = {"auto": osam.SCATTER_AUTO, "gather": osam.SCATTER_GATHER, "atomic": osam.SCATTER_ATOMIC,
                   "tiled": osam.SCATTER_GATHER_TILED, "lowreg": osam.SCATTER_GATHER_LOWREG,
                   "tiled_lowreg": osam.SCATTER_GATHER_TILED_LOWREG}[args.scatter]
        prob = osam.Problem(spec, rom_ops=rom_ops, device=local, precision=prec, scatter=scatter)
        log(f"[{name}] tuning: {prob.tuning()}")
        for _ in range(args.warmup):
            r = prob.step()
        # headline timed region: the library's default path, each controller step one graph launch
        # (Schwarz iterations in a device-side while node), CUDA events around every step
        clocks = ClockSampler(local) if prec == head_prec else None
        if clocks:
            clocks.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.nvtx.range_push("timed" if prec == head_prec else f"timed_{name}")
        total_ms, updates, iters, launches = timed_pass(prob, torch, flush, args.steps, profile=False)
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop() if clocks else None
        # kernel-timing region: the same steps driven from the host with CUDA events around every
        # internal-force launch (the roofline's per-launch durations)
        torch.cuda.nvtx.range_push(f"profiled_{name}")
        p_ms, p_upd, _, prof = timed_pass(prob, torch, flush, args.steps, profile=True)
        torch.cuda.nvtx.range_pop()
        e2e = e2e_pass(prob, torch, args.e2e_steps, args.rank) if (args.e2e_steps > 0 and rom_ops) else None
        (total_ms, updates), (p_ms, p_upd), e2e_pair = combine_ranks(
            [(total_ms, updates), (p_ms, p_upd), (e2e["seconds"] * 1e3, e2e["updates"]) if e2e else (1.0, 0)],
            f"cuda:{local}")
        if e2e:
            e2e["value"] = e2e_pair[1] / (e2e_pair[0] * 1e-3)
            del e2e["seconds"], e2e["updates"]
        n_launch = launches["kernel_launches"]
        if world > 1:   # the whole job's launches, like the whole job's element-updates
            n_launch = combine_ranks([(0.0, n_launch)], f"cuda:{local}")[0][1]
        results[name] = {"total_ms": total_ms, "updates": updates, "iters": iters, "prof": prof, "clk": clk,
                         "launches": n_launch, "prof_total_ms": p_ms,
                         "host_value": p_upd / (p_ms * 1e-3), "host_ms_per_step": p_ms / args.steps, "e2e": e2e,
                         "tuning": prob.tuning()}
        prob.close()
    head = results["f32x2" if head_prec == osam.F32X2_FORCE else "f64"]

    def roofline(res, prec_name):
        prof = res["prof"]
        per_launch = prof["force_ms"] / max(1, prof["force_launches"])
        if prec_name == "f64":
            achieved = FLOPS_PER_NH_ELEMENT * prof["force_elements"] / (prof["force_ms"] * 1e-3) / 1e12
            same = (FORCE_TRAFFIC["source_sha256"] == source_sha()
                    and FORCE_TRAFFIC["tiled"] == bool(res["tuning"].get("tiled"))
                    and FORCE_TRAFFIC.get("register_cap", 0) == res["tuning"].get("register_cap", 0))
            traffic = FORCE_TRAFFIC["bytes_per_launch"] if same else None
            return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK[0], "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK[0], "traffic": traffic,
                    "kernel": (("k_force_tile_occ_b<NeoHookean> (128-register cap)" if res["tuning"].get("register_cap")
                                else "k_force_tile_b<NeoHookean, gather>") if res["tuning"].get("tiled")
                               else "k_force_b<NeoHookean, f64, %s>" % res["tuning"]["scatter"]),
                    "peak_kind": FP64_PEAK_KIND[0],
                    "frac_of_nominal": achieved / FP64_NOMINAL_TFLOPS,
                    "flops_per_element": FLOPS_PER_NH_ELEMENT, "elements_per_launch":
                    prof["force_elements"] // max(1, prof["force_launches"]),
                    "force_ms_per_launch": per_launch,
                    "force_time_share": prof["force_ms"] / res["prof_total_ms"]}
        # double-float force: FP32-pipe instruction issue is the binding unit
        achieved = F32X2_INST_PER_NH_ELEMENT * prof["force_elements"] / (prof["force_ms"] * 1e-3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": FP32_ISSUE_PEAK_TINST, "unit": "Tinst/s (FP32 pipe)",
                "frac": achieved / FP32_ISSUE_PEAK_TINST, "traffic": None, "kernel": "k_force_df2_b<NeoHookean>",
                "peak_kind": "152 SMs x 128 lanes x 2.07 GHz", "fp64_equivalent_tflops":
                FLOPS_PER_NH_ELEMENT * prof["force_elements"] / (prof["force_ms"] * 1e-3) / 1e12,
                "force_ms_per_launch": per_launch, "force_time_share": prof["force_ms"] / res["prof_total_ms"]}

    batched = None
    if not args.no_batched and not args.fom_only:
        batched = measure_batched(W, osam, torch, flush, args, local, log, rank, world)
        log(f"batched: {batched['value']:.3e} vs plain {batched['plain_value']:.3e} ({batched['speedup']:.1f}x)")

    fit_meas = select_meas = adjoint_meas = implicit_meas = None
    if world == 1 and not args.no_cpu_baseline and fit_info is not None:
        fit_meas = measure_fit(fit_info, log)
        select_meas = measure_select(osam, fit_info, local, log)
        adjoint_meas = measure_adjoint(W, osam, local, log)
    plain_meas = None
    if world == 1 and not args.fom_only:
        plain_meas = measure_fom_fom_plain(W, osam, local, log)
    large_meas = None
    if world == 1 and not args.no_large and not args.fom_only:
        large_meas = measure_large(W, osam, torch, flush, args, local, log)
    next_meas = None
    if world == 1 and not args.no_implicit and rom_ops:
        implicit_meas = measure_implicit(W, osam, torch, flush, rom_ops, args, local, log)
        next_meas = measure_next_rows(W, osam, torch, flush, rom_ops, args, local, log)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.fom_only:
        rate, steps, secs = cpu_oracle_rate(W, args, 20, 10.0, max_steps=4)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"{steps} controller step(s) x 1 Schwarz iteration x 20 substeps of the {args.n}x{args.n}x"
                         f"{args.nz} NH FOM + r={args.rank} ROM (seeded stand-in operators), {secs:.1f} s CPU"}

    if rank == 0:
        head_name = "f32x2" if head_prec == osam.F32X2_FORCE else "f64"
        value = head["updates"] / (head["total_ms"] * 1e-3)
        variants = {}
        for name, res in results.items():
            variants[name] = {"value": res["updates"] / (res["total_ms"] * 1e-3),
                              "ms_per_step": res["total_ms"] / args.steps,
                              "value_host_loop": res["host_value"], "ms_per_step_host_loop": res["host_ms_per_step"],
                              "e2e": res["e2e"]["value"] if res["e2e"] else None, "tuning": res["tuning"],
                              "roofline": roofline(res, name),
                              "parity": "1e-9 relative L2 vs the FP64 oracle (tests/test_gpu_parity.py)"}
        clk = head["clk"] or {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        # HBM: the explicit state the method must move per node update (u, v read + write, a read +
        # write, lumped mass read: 96 + 48 + 8 B), times nodes per element of the FOM mesh
        sd0 = spec.subdomains[0]
        bytes_per_update = STATE_BYTES_PER_NODE_UPDATE * sd0.n_nodes / sd0.n_elements
        hbm_peak, hbm_kind = measured_hbm_gbs()
        hbm = {}
        for name, v in variants.items():
            gbs = v["value"] * bytes_per_update / 1e9
            hbm[name] = {"achieved_gbs": gbs, "frac": gbs / hbm_peak if hbm_peak else None}
        hbm = {"algorithmic_bytes_per_element_update": bytes_per_update, "peak_gbs": hbm_peak,
               "peak_kind": hbm_kind, **hbm,
               "note": "the path is bound by the FP64 (or FP32-issue) pipes, not by HBM"}
        mean_it = float(np.mean(head["iters"]))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["total_ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head_name == "f64" else "f32x2",
                "data": "synthetic",
                "config": {"workload": (f"fom_fom {args.n}x{args.n}x{args.nz} x2 Neo-Hookean FOMs" if args.fom_only else
                                        f"fom_opinf_hybrid {args.n}x{args.n}x{args.nz} Neo-Hookean FOM + "
                                        f"r={args.rank} quadratic OpInf ROM (fitted on {args.snapshots} snapshots)"),
                           "dt": 1e-6, "substeps_per_step": 20, "tol_rel": 1e-12, "max_iters": 64,
                           "fom_elements": spec.subdomains[0].n_elements, "parallelism": "replicas",
                           "l2": "flushed between steps (256 MiB write)",
                           "mean_iterations": float(np.mean(head["iters"])), "max_iterations": int(max(head["iters"])),
                           "timing": "value: graph-captured controller steps (the library default; Schwarz "
                                     "iterations in a device-side while node), CUDA events around every step; "
                                     "roofline: a second pass of the same steps driven from the host with CUDA "
                                     "events around every internal-force launch (variants[*].value_host_loop)"},
                "roofline": roofline(head, head_name), "cpu_baseline": cpu, "e2e": head["e2e"],
                "gpu_launches": head["launches"],
                "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
                "variants": variants, "batched_vs_plain": batched, "opinf_fit": fit_meas, "opinf_select": select_meas,
                "adjoint": adjoint_meas, "implicit": implicit_meas, "next_rows": next_meas, "large_chain": large_meas,
                "fom_fom_plain": plain_meas,
                "hbm": hbm, "fp64_peak": fp64_peak,
                "effective_rate": value / mean_it,
                "rom_substeps_per_s": mean_it * 20 * args.steps / (head["total_ms"] * 1e-3) if not args.fom_only else None}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
