"""Benchmark of the GB300 MD ERI library on the class-sweep workload.

One step = every class (la lb|lc ld) with l in {s, p, d} (81 classes), each a
list-form batch of 1e5 contracted quartets (K = 3 per shell, even-tempered
exponents 0.2*3^k, centres in a 12-bohr cube, pairs drawn from 2048 random
pairs per side), all computed by eri_batch in FP64 and stored in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl library|reference]

Prints one JSON line (rank 0).  Under torchrun every rank computes its own
seeded copy of the sweep (weak scaling, no collective on the data path).
``--impl reference`` times the CPU oracle (oracle/, double build) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ERI quartets/s per class, % FP64 peak; fwd+grad vs plain FP64 at 1e-10 abs"
UNIT = "quartets/s"
NQ_PER_CLASS = 100_000
K_PER_SHELL = 3
POOL, NPAIRS = 512, 2048
# FP64 FMA pipe of one GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
L2_BYTES = 129 * 1024 * 1024
WORKLOAD = "class-sweep: 81 classes (l<=2), K=3 per shell, 1e5 quartets/class, FP64"


def classes():
    return synth.all_classes(2)


def sweep(seed, only=None, nq=NQ_PER_CLASS):
    basis, pools = synth.class_sweep_pools(seed=seed, pool=POOL, K=K_PER_SHELL)
    sel = classes() if only is None else [only]
    batches = {c: synth.class_sweep_batch(pools, c, seed=seed, npairs=NPAIRS, nq=nq) for c in sel}
    return basis, batches


# --------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def oracle_sweep_rate(basis, batches, budget_s=18.0, threads=None):
    """Quartets/s of the CPU oracle (double build, as it stands) on the sweep,
    extrapolated from a bounded per-class sample."""
    import oracle
    threads = threads or (os.cpu_count() or 1)
    per_class = budget_s / len(batches)
    total_time, total_q, sampled = 0.0, 0, 0
    for cls, (bra, ket, q) in batches.items():
        qs = synth.quartet_shells(bra, ket, q[:1])
        t0 = time.perf_counter()
        oracle.eri_quartets(basis, qs, prec="d")
        t1 = max(time.perf_counter() - t0, 1e-6)
        n = int(max(threads, min(q.shape[0], per_class * threads / t1)))
        n = min(n, q.shape[0])
        qs = synth.quartet_shells(bra, ket, q[:n])
        t0 = time.perf_counter()
        oracle.eri_quartets(basis, qs, prec="d", threads=threads)
        dt = time.perf_counter() - t0
        total_time += dt / n * q.shape[0]
        total_q += q.shape[0]
        sampled += n
    return total_q / total_time, threads, sampled


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    basis, batches = sweep(0)
    for _ in range(args.warmup):
        oracle_sweep_rate(basis, batches, budget_s=args.ref_budget / 4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, sampled = oracle_sweep_rate(basis, batches, budget_s=args.ref_budget)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(batches) * NQ_PER_CLASS / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "classes": len(batches), "quartets_per_class": NQ_PER_CLASS,
                   "K_per_shell": K_PER_SHELL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sampled} quartets per step spread over all 81 classes, "
                                   f"~{args.ref_budget:.0f} s of CPU work per step, extrapolated to 1e5/class"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ("eri_fwd.cu", "eri_tile.cuh", "eri_device.cuh", "eri_internal.h", "eri_tables.cu")


def kernel_source_sha():
    """First 16 hex digits of the SHA-256 of the forward kernel's sources, concatenated."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2506_12501_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM traffic per launch of the forward kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "fwd_kernel_class_sweep.md")
    try:
        text = open(path).read()
        sha = kernel_source_sha()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch_avg:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != sha:
        return None
    return float(t.group(1))


def reduce_max(value, dist, device):
    """Max over ranks of a per-rank float (the slowest rank sets the job time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, quartets_per_rank_step, steps, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * quartets_per_rank_step * steps / (max_ms / 1e3)


def run_variants(args, eri, dev):
    """The split-precision, adjoint and batched forms, each timed against the
    plain FP64 per-class kernels on the same GPU (bounded sizes; see config)."""
    import torch

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    out = {}
    which = set(args.variants.split(",")) if args.variants else {"split", "adjoint", "batched", "threecentre"}
    # split precision on the high-l workload
    split = {}
    for cls in ([(2, 2, 2, 2), (3, 3, 3, 3), (3, 3, 2, 2)] if "split" in which else []):
        for K, nq in ((1, 100_000), (5, args.split_nq_k5)):
            basis, bra, ket, q = synth.split_batch(cls, K=K, seed=0, nq=nq)
            db = eri.DeviceBasis(basis)
            b = torch.as_tensor(bra, device=dev)
            k = torch.as_tensor(ket, device=dev)
            qq = torch.as_tensor(q, device=dev)
            o64 = torch.empty(eri.out_len(cls, len(bra), len(ket), nq), dtype=torch.float64, device=dev)
            osp = torch.empty_like(o64)
            t64 = timed(lambda: eri.eri_batch(cls, db, b, k, qq, out=o64))
            tsp = timed(lambda: eri.eri_batch(cls, db, b, k, qq, out=osp, precision=eri.ERI_PREC_SPLIT))
            err = float((osp - o64).abs().max())
            split["".join(map(str, cls)) + f"_K{K}"] = {
                "quartets": nq, "fp64_ms": t64, "split_ms": tsp, "speedup": t64 / tsp,
                "fp64_quartets_per_s": nq / (t64 / 1e3), "split_quartets_per_s": nq / (tsp / 1e3),
                "max_abs_err_vs_fp64": err, "max_abs_fp64": float(o64.abs().max())}
            del o64, osp
    if split:
        out["split"] = split
    if "adjoint" in which:
        out["adjoint"] = adjoint_variant(args, eri, dev, timed)
    if "batched" in which:
        out["batched"] = batched_variant(args, eri, dev, timed)
    if "threecentre" in which:
        out["threecentre"] = three_centre_variant(args, eri, dev, timed)
    return out


def three_centre_variant(args, eri, dev, timed):
    """3-centre integrals (x|cd), x a real solid harmonic: uncontracted
    auxiliary shells lx <= 3 against the class-sweep orbital pairs (K = 3),
    1e5 triples per class; the form (side order) each class ran and its FP64
    operation count give GFLOP/s and the fraction of the FP64 peak."""
    import torch
    from paper_2506_12501_gb300 import opcount
    basis, orb, aux = synth.three_centre_pools(seed=0, pool=512)
    db = eri.DeviceBasis(basis)
    per, tot_ms, tot_flops, tot_n = {}, 0.0, 0.0, 0
    for lx in range(4):
        nterms = int(np.count_nonzero(np.abs(eri.solid_harmonics(lx)) > 1e-14))
        for lc, ld in ((0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)):
            x, ket, t = synth.three_centre_batch(orb, aux, (lx, lc, ld), seed=0, nt=args.three_nt)
            xd, kd, td = (torch.as_tensor(v, device=dev) for v in (x, ket, t))
            o = torch.empty(len(t) * (2 * lx + 1) * eri.nc(lc) * eri.nc(ld), dtype=torch.float64, device=dev)
            ms = timed(lambda: eri.eri_batch3(lx, lc, ld, db, xd, kd, td, pure=True, out=o), reps=2)
            sw, _ = eri.eri_last_form()
            f = opcount.sparse_flops3((lx, lc, ld), 1, 9, True, sw, nterms) * len(t)
            per[f"{lx}{lc}{ld}"] = {"ms": ms, "form": "swapped" if sw else "plain",
                                    "triples_per_s": len(t) / (ms / 1e3), "gflops_sparse": f / (ms / 1e3) / 1e9}
            tot_ms += ms
            tot_flops += f
            tot_n += len(t)
    return {"workload": f"x real solid harmonics lx <= 3 (K = 1, exponents 10^U(-1,1)) x orbital pairs l <= 2 "
                        f"(K = 3), 24 classes x {args.three_nt} triples",
            "triples": tot_n, "ms": tot_ms, "triples_per_s": tot_n / (tot_ms / 1e3),
            "gflops_sparse": tot_flops / (tot_ms / 1e3) / 1e9,
            "frac_fp64_peak_sparse": tot_flops / (tot_ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS, "per_class": per}


def adjoint_variant(args, eri, dev, timed):
    """The adjoint on the 16-atom molecule-shaped basis, a sample of every class."""
    import torch
    basis, D, bf_off = synth.adjoint_workload(natom=16, radius=4.4, seed=0)
    pairs, batches = synth.all_unique_quartets(basis)
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees this variant too
    db = eri.DeviceBasis(basis)
    from paper_2506_12501_gb300 import opcount
    tf = tg = 0.0
    gflop = 0.0
    nq_tot = 0
    per = {}
    kern = {eri.PROF_GRAD: 0.0, eri.PROF_PAIR: 0.0, eri.PROF_PREPASS: 0.0}
    for cls, (bra, ket, q) in batches.items():
        q = q[: args.adjoint_nq]
        W = synth.density_weights(cls, bra, ket, q, D, bf_off)
        b = torch.as_tensor(bra, device=dev)
        k = torch.as_tensor(ket, device=dev)
        qq = torch.as_tensor(q, device=dev)
        Wd = torch.as_tensor(W, device=dev)
        o = torch.empty(W.size, dtype=torch.float64, device=dev)
        gc = torch.zeros_like(db.centres)
        ge = torch.zeros_like(db.exps)
        t_f = timed(lambda: eri.eri_batch(cls, db, b, k, qq, out=o), reps=1)
        t_g = timed(lambda: eri.eri_batch_grad(cls, db, b, k, qq, Wd, gc, ge), reps=1)
        gforms = eri.eri_last_grad_forms()
        # the same call once more under the library's launch events: kernel time
        # of the two adjoint launches, of the pair tables and of the prepass
        torch.cuda.synchronize()
        eri.eri_profile_read()
        eri.eri_profile_enable(True)
        eri.eri_batch_grad(cls, db, b, k, qq, Wd, gc, ge)
        torch.cuda.synchronize()
        eri.eri_profile_enable(False)
        for kid, (_, ms) in eri.eri_profile_read().items():
            if kid in kern:
                kern[kid] += ms
        tf += t_f
        tg += t_g
        per["".join(map(str, cls))] = {"quartets": len(q), "fwd_ms": t_f, "grad_ms": t_g,
                                       "grad_forms": "".join("XV"[f] for f in gforms)}
        nq_tot += len(q)
        Ks = basis.shell_K
        kb = (Ks[bra[q[:, 0], 0]] * Ks[bra[q[:, 0], 1]]).astype(np.int64)
        kk = (Ks[ket[q[:, 1], 0]] * Ks[ket[q[:, 1], 1]]).astype(np.int64)
        for (x, y), n in zip(*np.unique(np.stack([kb, kk], 1), axis=0, return_counts=True)):
            gflop += n * opcount.grad_flops(cls, int(x), int(y), gforms)
    torch.cuda.profiler.stop()
    return {"workload": f"16-atom molecule basis, {len(batches)} classes, <= {args.adjoint_nq} "
                        "quartets per class", "quartets": nq_tot, "fwd_ms": tf, "grad_ms": tg,
            "grad_over_fwd": tg / tf, "grad_quartets_per_s": nq_tot / (tg / 1e3),
            "grad_gflops_sparse": gflop / (tg / 1e3) / 1e9,
            "grad_frac_fp64_peak_sparse": gflop / (tg / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
            "grad_kernel_ms": kern[eri.PROF_GRAD], "grad_pair_tables_ms": kern[eri.PROF_PAIR],
            "grad_prepass_ms": kern[eri.PROF_PREPASS],
            "grad_kernel_frac_fp64_peak_sparse": gflop / (kern[eri.PROF_GRAD] / 1e3) / 1e9 / FP64_PEAK_GFLOPS
            if kern[eri.PROF_GRAD] > 0 else None, "per_class": per}


def batched_variant(args, eri, dev, timed):
    """The screened molecule-shaped workload in one persistent graph launch."""
    import torch
    mb = synth.molecule_basis(natom=args.molecule_natom, radius=7.0 * (args.molecule_natom / 64) ** (1 / 3), seed=0)
    mdb = eri.DeviceBasis(mb)
    nbf = int(((mb.shell_l + 1) * (mb.shell_l + 2) // 2).sum())
    rng = np.random.default_rng(2)
    U = rng.uniform(-1, 1, (nbf, nbf))
    Dm = torch.as_tensor(np.triu(U) + np.triu(U, 1).T, device=dev)
    t0 = time.perf_counter()
    plan = eri.Plan(mdb, threshold=1e-12)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    info = plan.info()
    # FP64 operations of the plan's jobs (plain forms, each job's own orientation)
    from paper_2506_12501_gb300 import opcount
    flops = 0.0
    for j in range(info["njobs"]):
        cls, nq, _, _ = plan.job(j)
        kb, kk = plan.job_degrees(j)
        flops += nq * opcount.sparse_flops(cls, kb, kk, form=(False, False))
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.execute(D=Dm, energy=e)  # graph capture outside the profiled region
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed replays
    t_exec = timed(lambda: plan.execute(D=Dm, energy=e), reps=2)
    torch.cuda.profiler.stop()
    J = torch.empty_like(Dm)
    t_j = timed(lambda: plan.coulomb(Dm, J), reps=2)
    K = torch.empty_like(Dm)
    t_jk = timed(lambda: plan.jk(Dm, J=J, K=K), reps=2)
    res = {"workload": f"{args.molecule_natom} atoms (s x3 K=6,3,1, p x2 K=3,1, d K=1), Schwarz 1e-12, "
                       "energy digestion, one persistent graph-captured launch",
           "quartets": info["nquartets"], "jobs": info["njobs"], "work_items": info["nitems"],
           "create_s": t_create, "execute_ms": t_exec,
           "quartets_per_s": info["nquartets"] / (t_exec / 1e3), "energy": float(e.item()),
           "gflops_sparse": flops / (t_exec / 1e3) / 1e9,
           "frac_fp64_peak_sparse": flops / (t_exec / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
           "coulomb_ms": t_j, "coulomb_quartets_per_s": info["nquartets"] / (t_j / 1e3),
           "coulomb_trace_DJ": float((Dm * J).sum().item()),
           "jk_ms": t_jk, "jk_quartets_per_s": info["nquartets"] / (t_jk / 1e3),
           "exchange_trace_DK": float((Dm * K).sum().item()),
           "status": plan.status()}
    plan.destroy()
    return res


def run_library(args):
    import torch
    import torch.distributed as dist

    import paper_2506_12501_gb300 as eri
    from paper_2506_12501_gb300 import opcount

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eri.lib()

    only = tuple(int(x) for x in args.only_class) if args.only_class else None
    prec = eri.ERI_PREC_SPLIT if args.precision == "split" else eri.ERI_PREC_FP64
    basis, batches = sweep(seed=rank, only=only, nq=args.nq)
    nq_class = args.nq
    db = eri.DeviceBasis(basis)
    dev_batches, outs = {}, {}
    for cls, (bra, ket, q) in batches.items():
        dev_batches[cls] = (torch.as_tensor(bra, device=dev), torch.as_tensor(ket, device=dev),
                            torch.as_tensor(q, device=dev))
        outs[cls] = torch.empty(eri.out_len(cls, bra.shape[0], ket.shape[0], q.shape[0]), dtype=torch.float64,
                                device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    dense = {c: opcount.dense_flops(c, K_PER_SHELL ** 2, K_PER_SHELL ** 2) for c in batches}
    stream = torch.cuda.current_stream()
    forms = {}

    def step(timing=None):
        for cls, (b, k, q) in dev_batches.items():
            if timing is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            eri.eri_batch(cls, db, b, k, q, out=outs[cls], precision=prec)
            forms[cls] = eri.eri_last_form()
            if timing is not None:
                e1.record(stream)
                timing[cls].append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the FP64 operations of the form each class runs (chosen during warm-up)
    sparse = {c: opcount.sparse_flops(c, K_PER_SHELL ** 2, K_PER_SHELL ** 2, form=forms[c]) for c in batches}
    eri.eri_profile_read()
    eri.eri_profile_enable(True)
    timing = {c: [] for c in batches}
    step_events = []
    n_launch0 = eri.eri_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees only the timed steps
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the step events)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            step(timing)
            s1.record(stream)
            step_events.append((s0, s1))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        torch.cuda.profiler.stop()
    n_launch = eri.eri_launch_count() - n_launch0
    prof = eri.eri_profile_read()
    eri.eri_profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in step_events]
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = reduce_max(total_ms, dist, dev)
    nq_step = len(batches) * nq_class
    value = job_rate(world, nq_step, args.steps, total_ms)

    per_class = {}
    for cls in batches:
        ms = statistics.median(a.elapsed_time(b) for a, b in timing[cls])
        qps = nq_class / (ms / 1e3)
        per_class["".join(map(str, cls))] = {
            "ms": round(ms, 4), "quartets_per_s": qps,
            "form": ("swapped " if forms[cls][0] else "") + ("hrr" if forms[cls][1] else "plain"),
            "gflops_sparse": sparse[cls] * qps / 1e9, "gflops_dense": dense[cls] * qps / 1e9,
            "frac_fp64_peak_sparse": sparse[cls] * qps / 1e9 / FP64_PEAK_GFLOPS,
            "frac_fp64_peak_dense": dense[cls] * qps / 1e9 / FP64_PEAK_GFLOPS}
    fwd_launches, fwd_ms = prof[eri.PROF_FWD]
    flops_per_step = sum(sparse[c] * nq_class for c in batches)
    dense_per_step = sum(dense[c] * nq_class for c in batches)
    fwd_gflops = flops_per_step * args.steps / (fwd_ms / 1e3) / 1e9 if fwd_ms > 0 else None
    roofline = {"bound": "alu", "kernel": "fwd_kernel", "achieved": fwd_gflops, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": (fwd_gflops / FP64_PEAK_GFLOPS) if fwd_gflops else None,
                "traffic": profile_traffic(),
                "peak_source": "FP64 FMA pipe, 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (unit counts and max clock); "
                               "a DFMA microbenchmark measured 1.20 TFLOP/s at 1.99 GHz",
                "flops_counted": "FP64 operations of the implemented sparse MD sequence (FMA=2)",
                "fwd_launches": fwd_launches, "fwd_ms_per_launch": fwd_ms / max(fwd_launches, 1),
                "gflops_dense_formulation": dense_per_step * args.steps / (fwd_ms / 1e3) / 1e9 if fwd_ms else None,
                "frac_dense_formulation": (dense_per_step * args.steps / (fwd_ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS)
                if fwd_ms else None,
                "other_kernels_ms_per_step": {"pair": prof[eri.PROF_PAIR][1] / args.steps,
                                              "prepass": prof[eri.PROF_PREPASS][1] / args.steps}}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_in = {c: tuple(torch.as_tensor(x).pin_memory() for x in batches[c]) for c in batches}
        host_basis = {k: torch.as_tensor(np.asarray(getattr(basis, k))).pin_memory()
                      for k in ("centres", "shell_atom", "shell_l", "shell_K", "shell_off", "exps", "coefs")}
        host_out = torch.empty(sum(o.numel() for o in outs.values()), dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for v in host_in.values() for t in v) + \
            sum(t.numel() * t.element_size() for t in host_basis.values())
        d2h = host_out.numel() * 8
        # each class's integrals go back to the host on a second stream while
        # the next class computes.  A class's copy is queued only after the
        # next eri_batch call has returned: that call reads a few bytes back
        # (its validation pass), and a read queued behind a large copy on the
        # device-to-host engine would stall it.  The step ends when every
        # copy has landed.
        cstream = torch.cuda.Stream(device=dev)

        def read_back(p):
            cstream.wait_event(p[3])
            with torch.cuda.stream(cstream):
                host_out[p[1]:p[1] + p[2]].copy_(outs[p[0]], non_blocking=True)
        e_ms = []
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for k_, t in host_basis.items():
                getattr(db, k_).copy_(t.reshape(getattr(db, k_).shape), non_blocking=True)
            off = 0
            pending = None
            for cls in batches:
                b, k, q = (d.copy_(h, non_blocking=True) for d, h in zip(dev_batches[cls], host_in[cls]))
                eri.eri_batch(cls, db, b, k, q, out=outs[cls], precision=prec)
                done = torch.cuda.Event()
                done.record(stream)
                if pending is not None:
                    read_back(pending)
                pending = (cls, off, outs[cls].numel(), done)
                off += outs[cls].numel()
            read_back(pending)
            stream.wait_stream(cstream)
            a1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                e_ms.append(a0.elapsed_time(a1))
        e2e = {"value": world * nq_step / (statistics.median(e_ms) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": len(e_ms),
               "step_ms": [round(x, 2) for x in e_ms]}

    variants = None
    if rank == 0 and not args.no_variants and (only is None or args.variants):
        variants = run_variants(args, eri, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sampled = oracle_sweep_rate(basis, batches, budget_s=args.ref_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sampled} quartets over all 81 classes (~{args.ref_budget:.0f} s of CPU work, "
                         f"double build of the oracle on {cores} host threads), extrapolated to 1e5/class"}

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == eri.ERI_PREC_FP64 else "f64+f32x2",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if only is None else f"single class {args.only_class}, {nq_class} quartets",
                       "classes": len(batches), "quartets_per_class": nq_class,
                       "K_per_shell": K_PER_SHELL, "pairs_per_side": NPAIRS, "pool_per_l": POOL,
                       "l2": "flushed between timed steps (256 MiB write); outputs 8 GB/step also exceed L2",
                       "parallelism": f"weak x{world}: each rank its own seeded sweep"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch,
            "clocks": clk.summary(), "wall_s_timed": t_wall, "step_ms": step_ms, "variants": variants,
            "per_class": per_class,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["library", "reference"], default="library")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=18.0, help="seconds of oracle CPU work per reference step")
    ap.add_argument("--only-class", default=None, help="profiling aid: one class, e.g. 2222")
    ap.add_argument("--no-variants", action="store_true", help="skip the split/adjoint/batched measurements")
    ap.add_argument("--variants", default=None, help="comma list of split,adjoint,batched,threecentre (default: all)")
    ap.add_argument("--split-nq-k5", type=int, default=10_000)
    ap.add_argument("--adjoint-nq", type=int, default=20_000)
    ap.add_argument("--molecule-natom", type=int, default=16)
    ap.add_argument("--three-nt", type=int, default=100_000, help="triples per 3-centre class")
    ap.add_argument("--nq", type=int, default=NQ_PER_CLASS, help="quartets per class")
    ap.add_argument("--precision", choices=["fp64", "split"], default="fp64",
                    help="transforms of the timed sweep (profiling aid; the benchmark value is fp64)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_library(args)


if __name__ == "__main__":
    main()
