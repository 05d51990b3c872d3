"""Benchmark of the GB300 MD ERI library.

Headline workload, one step: every class (la lb|lc ld) with l in {s, p, d}
(81 classes), each a list-form batch of 1e5 contracted quartets (K = 3 per
shell, even-tempered exponents 0.2*3^k, centres in a 12-bohr cube, pairs
drawn from 2048 random pairs per side), all computed by eri_batch in FP64
and stored in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl library|reference]
                  [--variants LIST|none] [--detail-out PATH]

Output: detail lines first (one JSON object each, with a "detail" key: the
per-class rates, each measured variant, the arithmetic-throughput probes),
then, LAST, one compact JSON line with the headline metric, the roofline of
the dominant kernel, the CPU baseline, the end-to-end rate and the clocks.
``--detail-out`` also writes every detail object into one JSON file.

Variants, each at its stated size and timed against the plain FP64 per-class
kernel on the same GPU:
  split        (dd|dd), (ff|ff), (ff|dd), K = 1 and 5 per shell, 1e5 quartets
               each, exponents log-uniform in [0.05, 50]: FP64 against FP32
               hi+lo transforms, error of both against the oracle on a sample;
  adjoint      all 1.08e7 unique quartets of 16 atoms (s x3 K=6,3,1, p x2
               K=3,1, d K=1), W = D_ab D_cd: forward and gradient times;
  batched      64 atoms, Schwarz 1e-12, energy digestion in one persistent
               graph-replayed launch (partitioned over ranks under torchrun);
               J and J + K on the 16-atom plan;
  threecentre  (x|cd), x a real solid harmonic, 24 classes x 1e5 triples;
  peaks        FP64 FMA, FP64 MMA and FP32 FMA throughput probes.

Under torchrun every rank computes its own seeded copy of the class sweep
(weak scaling, no collective on the data path); the batched variant splits
one plan's work items over the ranks and all-reduces the energy.
``--impl reference`` times the CPU oracle (oracle/, double build) on a
bounded sample of the class sweep instead.
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
# FP64 FMA pipe of one GB300 from unit counts and the maximum clock:
# 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
L2_BYTES = 129 * 1024 * 1024
WORKLOAD = "class-sweep: 81 classes (l<=2), K=3 per shell, 1e5 quartets/class, FP64"
ALL_VARIANTS = ("peaks", "split", "adjoint", "batched", "threecentre")

DETAILS: list = []


def emit_detail(name, obj, rank=0):
    """Print one detail object (rank 0) and keep it for --detail-out."""
    if rank != 0:
        return
    d = {"detail": name, **obj}
    DETAILS.append(d)
    print(json.dumps(d), flush=True)


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
def oracle_sweep_rate(basis, batches, budget_s=12.0, threads=None):
    """The CPU oracle (double build, as it stands) on a bounded sample of the
    sweep: per class a leading slice of its quartets sized to about
    budget_s / 81 seconds on `threads` host threads.  Returns (rate over the
    sweep's class mix in quartets/s, threads, quartets sampled, seconds spent
    in the timed oracle calls)."""
    import oracle
    threads = threads or (os.cpu_count() or 1)
    per_class = budget_s / len(batches)
    total_time, total_q, sampled, spent = 0.0, 0, 0, 0.0
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
        spent += dt
        total_time += dt / n * q.shape[0]
        total_q += q.shape[0]
        sampled += n
    return total_q / total_time, threads, sampled, spent


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    basis, batches = sweep(0)
    # each step a bounded sample sized so that the whole run takes a few minutes
    budget = args.ref_budget or min(18.0, max(3.0, 150.0 / (args.steps + 0.25 * args.warmup)))
    for _ in range(args.warmup):
        oracle_sweep_rate(basis, batches, budget_s=budget / 4)
    vals, walls = [], []
    sampled = cores = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, cores, sampled, _ = oracle_sweep_rate(basis, batches, budget_s=budget)
        walls.append(time.perf_counter() - t0)
        vals.append(v)
    value = statistics.median(vals)
    full_step_ms = 1e3 * len(batches) * NQ_PER_CLASS / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "classes": len(batches), "quartets_per_class": NQ_PER_CLASS,
                   "K_per_shell": K_PER_SHELL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sampled} quartets per step spread over all 81 classes (~{budget:.1f} s of "
                                   f"oracle work per step on {cores} threads); value = the sweep's class mix at "
                                   f"the sampled per-class rates"},
        "ms_per_step_note": "wall time of one sampled step; the full 8.1e6-quartet step would take "
                            f"{full_step_ms / 1e3:.0f} s at this rate",
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "the oracle reads and writes host memory: no copies"},
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
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw) if pw else None}


KERNEL_SOURCES = ("eri_fwd.cu", "eri_tile.cuh", "eri_device.cuh", "eri_internal.h", "eri_tables.cu")


def kernel_source_sha():
    """First 16 hex digits of the SHA-256 of the forward kernel's sources, concatenated."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2506_12501_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per fwd_kernel launch of the full sweep, from the committed
    ncu summary, if it was taken on the current kernel source (else None).
    The summary holds the one-pass DRAM counters of one full-size step
    (81 launches, 1e5 quartets per class), averaged per launch."""
    path = os.path.join(ROOT, "profiles", "fwd_kernel_class_sweep.md")
    try:
        text = open(path).read()
        sha = kernel_source_sha()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
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


def timed(fn, reps=1, warm=True):
    """Fastest of `reps` CUDA-event timings (ms) of fn on the current stream."""
    import torch
    if warm:
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


def oracle_sample_error(cls, basis, bra, ket, q, outs, n, seed=5):
    """Max |x - oracle| of each list-form output in `outs` on n seeded quartets."""
    import oracle
    nab = synth_nc(cls[0]) * synth_nc(cls[1])
    ncd = synth_nc(cls[2]) * synth_nc(cls[3])
    pick = np.sort(np.random.default_rng(seed).choice(len(q), n, replace=False))
    ref = oracle.eri_quartets(basis, synth.quartet_shells(bra, ket, q[pick]), prec="d",
                              threads=os.cpu_count() or 1).reshape(n, nab * ncd)
    errs = []
    for o in outs:
        got = o.view(nab * ncd, len(q))[:, pick].T.cpu().numpy()
        errs.append(float(np.abs(got - ref).max()))
    return errs, float(np.abs(ref).max())


def synth_nc(l):
    return (l + 1) * (l + 2) // 2


def peaks_variant(eri):
    out = {}
    for name, kind in (("dfma", eri.PEAK_DFMA), ("dmma", eri.PEAK_DMMA), ("ffma", eri.PEAK_FFMA),
                       ("dfma_one_chain_8_warps_per_sm", eri.PEAK_DFMA_ONE_CHAIN)):
        g, mhz = eri.eri_peak_probe(kind)
        out[name] = {"gflops": g, "sm_mhz": mhz}
    out["dfma_per_clk_per_sm"] = out["dfma"]["gflops"] * 1e9 / 2 / (out["dfma"]["sm_mhz"] * 1e6) / 152
    out["dfma_gflops_at_max_clock"] = out["dfma"]["gflops"] * 2070.0 / out["dfma"]["sm_mhz"]
    return out


def split_variant(args, eri, dev):
    """(dd|dd), (ff|ff), (ff|dd) at K = 1 and 5 per shell, 1e5 quartets each:
    FP64 and split-precision transforms, each timed once after a warm-up
    call on a leading slice (form choice and tile tuning), and both compared
    with the oracle on a seeded sample."""
    import torch
    from paper_2506_12501_gb300 import opcount
    res = {}
    for cls in ((2, 2, 2, 2), (3, 3, 3, 3), (3, 3, 2, 2)):
        for K in (1, 5):
            nq = args.split_nq
            basis, bra, ket, q = synth.split_batch(cls, K=K, seed=0, nq=nq)
            db = eri.DeviceBasis(basis)
            b = torch.as_tensor(bra, device=dev)
            k = torch.as_tensor(ket, device=dev)
            qq = torch.as_tensor(q, device=dev)
            warm = qq[: min(nq, 20_000)].contiguous()
            o64 = torch.empty(eri.out_len(cls, len(bra), len(ket), nq), dtype=torch.float64, device=dev)
            osp = torch.empty_like(o64)
            ow = torch.empty(eri.out_len(cls, len(bra), len(ket), warm.shape[0]), dtype=torch.float64, device=dev)
            eri.eri_batch(cls, db, b, k, warm, out=ow)
            torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed calls
            t64 = timed(lambda: eri.eri_batch(cls, db, b, k, qq, out=o64), warm=False)
            torch.cuda.profiler.stop()
            f64form = eri.eri_last_form()
            f64tile = eri.eri_last_tile()
            eri.eri_batch(cls, db, b, k, warm, out=ow, precision=eri.ERI_PREC_SPLIT)
            torch.cuda.profiler.start()
            tsp = timed(lambda: eri.eri_batch(cls, db, b, k, qq, out=osp, precision=eri.ERI_PREC_SPLIT), warm=False)
            torch.cuda.profiler.stop()
            sptile = eri.eri_last_tile()
            spform = eri.eri_last_form()
            del ow
            nsamp = 2 if (cls == (3, 3, 3, 3) and K == 5) else (4 if K == 5 else 16)
            (e64, esp), refmax = oracle_sample_error(cls, basis, bra, ket, q, [o64, osp], nsamp)
            flops = opcount.sparse_flops(cls, K * K, K * K, form=f64form) * nq
            res["".join(map(str, cls)) + f"_K{K}"] = {
                "quartets": nq, "fp64_ms": round(t64, 3), "split_ms": round(tsp, 3), "speedup": t64 / tsp,
                "fp64_form": ("swapped " if f64form[0] else "") + ("hrr" if f64form[1] else "plain"),
                "split_form": "swapped" if spform[0] else "plain",
                "fp64_tile": "TQ{tq} IC{ic} x{threads}".format(**f64tile),
                "split_tile": "TQ{tq} IC{ic} x{threads}".format(**sptile),
                "fp64_quartets_per_s": nq / (t64 / 1e3), "split_quartets_per_s": nq / (tsp / 1e3),
                "fp64_gflops_sparse": flops / (t64 / 1e3) / 1e9,
                "fp64_frac_fp64_peak": flops / (t64 / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
                "max_abs_split_vs_fp64": float((osp - o64).abs().max()),
                "oracle_sample": nsamp, "max_abs_fp64_vs_oracle": e64, "max_abs_split_vs_oracle": esp,
                "max_abs_oracle_sample": refmax}
            del o64, osp
            torch.cuda.empty_cache()
    return {"workload": f"(dd|dd), (ff|ff), (ff|dd); K = 1 and 5 per shell; {args.split_nq} quartets each; "
                        "exponents 10^U(log 0.05, log 50); centres U[0,12]^3", "per_class": res}


def adjoint_variant(args, eri, dev):
    """The adjoint over every unique quartet of the 16-atom molecule-shaped
    basis (1.08e7 quartets, all classes), W = D_ab D_cd: the forward pass and
    the gradient pass timed over all classes, after one warm-up pass."""
    import torch
    from paper_2506_12501_gb300 import opcount
    basis, D, bf_off = synth.adjoint_workload(natom=16, radius=4.4, seed=0)
    pairs, batches = synth.all_unique_quartets(basis)
    db = eri.DeviceBasis(basis)
    data = []
    gflop = fflop = 0.0
    for cls, (bra, ket, q) in batches.items():
        if args.adjoint_only and "".join(map(str, cls)) not in args.adjoint_only.split(","):
            continue
        if args.adjoint_nq:
            q = q[: args.adjoint_nq]
        W = synth.density_weights(cls, bra, ket, q, D, bf_off)
        t = [torch.as_tensor(x, device=dev) for x in (bra, ket, q, W)]
        o = torch.empty(W.size, dtype=torch.float64, device=dev)
        Ks = basis.shell_K
        kb = (Ks[bra[q[:, 0], 0]] * Ks[bra[q[:, 0], 1]]).astype(np.int64)
        kk = (Ks[ket[q[:, 1], 0]] * Ks[ket[q[:, 1], 1]]).astype(np.int64)
        sig = np.unique(np.stack([kb, kk], 1), axis=0, return_counts=True)
        data.append((cls, t, o, sig, len(q)))
    gc = torch.zeros_like(db.centres)
    ge = torch.zeros_like(db.exps)

    def fwd():
        for cls, (b, k, qq, W), o, _, _ in data:
            eri.eri_batch(cls, db, b, k, qq, out=o)

    forms = {}
    ev = {}

    def grad(per=None):
        for cls, (b, k, qq, W), o, _, _ in data:
            if per is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
            eri.eri_batch_grad(cls, db, b, k, qq, W, gc, ge)
            if per is not None:
                e1.record()
                per[cls] = (e0, e1)
            forms[cls] = eri.eri_last_grad_forms()

    def fwd_per(per):
        for cls, (b, k, qq, W), o, _, _ in data:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            eri.eri_batch(cls, db, b, k, qq, out=o)
            e1.record()
            per[cls] = (e0, e1)

    t_f = timed(fwd)
    grad()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed pass
    t_g = timed(grad, warm=False)
    torch.cuda.profiler.stop()
    # per-class times (one more pass of each, events around every call)
    pf, pg = {}, {}
    fwd_per(pf)
    grad(pg)
    torch.cuda.synchronize()
    per_class = {"".join(map(str, c)): {"quartets": n, "fwd_ms": round(pf[c][0].elapsed_time(pf[c][1]), 3),
                                        "grad_ms": round(pg[c][0].elapsed_time(pg[c][1]), 3)}
                 for c, _, _, _, n in data}
    if args.adjoint_schemes:
        # every class once more with one launch forced (either side order) and
        # with two launches forced (either form each); the forms of the
        # timed default pass stay the ones counted below
        forms_default = dict(forms)
        for label, mask in (("grad_one_ms", (1 << eri.ERI_GRAD_X) | (1 << eri.ERI_GRAD_V) | (1 << eri.ERI_GRAD_ONE)),
                            ("grad_two_ms", (1 << eri.ERI_GRAD_X) | (1 << eri.ERI_GRAD_V) | (1 << eri.ERI_GRAD_TWO))):
            prev = eri.eri_set_grad_forms(mask)
            try:
                grad()
                pm = {}
                grad(pm)
                torch.cuda.synchronize()
            finally:
                eri.eri_set_grad_forms(prev)
            for c, _, _, _, _ in data:
                per_class["".join(map(str, c))][label] = round(pm[c][0].elapsed_time(pm[c][1]), 3)
        forms.clear()
        forms.update(forms_default)
    nq_tot = sum(d[4] for d in data)
    for cls, _, _, (keys, counts), _ in data:
        for (x, y), n in zip(keys, counts):
            gflop += n * opcount.grad_flops(cls, int(x), int(y), forms[cls])
            fflop += n * opcount.sparse_flops(cls, int(x), int(y), form=(False, False))
    # kernel time of the adjoint launches, pair tables and prepass (library events)
    torch.cuda.synchronize()
    eri.eri_profile_read()
    eri.eri_profile_enable(True)
    grad()
    torch.cuda.synchronize()
    eri.eri_profile_enable(False)
    prof = eri.eri_profile_read()
    kms = prof[eri.PROF_GRAD][1]
    return {"workload": f"16-atom molecule basis, {len(data)} classes, {nq_tot} unique quartets, "
                        "W = D_ab D_cd", "quartets": nq_tot, "fwd_ms": t_f, "grad_ms": t_g,
            "grad_over_fwd": t_g / t_f, "fwd_quartets_per_s": nq_tot / (t_f / 1e3),
            "grad_quartets_per_s": nq_tot / (t_g / 1e3),
            "grad_gflops_sparse": gflop / (t_g / 1e3) / 1e9,
            "grad_frac_fp64_peak_sparse": gflop / (t_g / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
            "grad_kernel_ms": kms, "grad_pair_tables_ms": prof[eri.PROF_PAIR][1],
            "grad_prepass_ms": prof[eri.PROF_PREPASS][1],
            "grad_kernel_frac_fp64_peak_sparse": gflop / (kms / 1e3) / 1e9 / FP64_PEAK_GFLOPS if kms > 0 else None,
            "fwd_frac_fp64_peak_sparse_plain": fflop / (t_f / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
            "grad_forms": {"".join(map(str, c)): "".join("XVO?S"[f] for f in v) for c, v in forms.items()},
            "per_class": per_class}


def batched_variant(args, eri, dev, world, rank, dist):
    """The screened molecule-shaped workload in one persistent graph launch;
    with several ranks each executes its slice of the plan and the energy is
    all-reduced."""
    import torch
    from paper_2506_12501_gb300 import opcount

    def make(natom):
        mb = synth.molecule_basis(natom=natom, radius=7.0 * (natom / 64) ** (1 / 3), seed=0)
        mdb = eri.DeviceBasis(mb)
        nbf = int(((mb.shell_l + 1) * (mb.shell_l + 2) // 2).sum())
        U = np.random.default_rng(2).uniform(-1, 1, (nbf, nbf))
        Dm = torch.as_tensor(np.triu(U) + np.triu(U, 1).T, device=dev)
        t0 = time.perf_counter()
        plan = eri.Plan(mdb, threshold=1e-12)
        torch.cuda.synchronize()
        return mdb, Dm, plan, time.perf_counter() - t0

    natom = args.molecule_natom
    mdb, Dm, plan, t_create = make(natom)
    info = plan.info()
    if world > 1:
        plan.set_slice(rank, world)
    sl = plan.slice_info()
    flops = 0.0
    for j in range(info["njobs"]):
        cls, nq, _, _ = plan.job(j)
        kb, kk = plan.job_degrees(j)
        flops += nq * opcount.sparse_flops(cls, kb, kk, form=(False, False))
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.execute(D=Dm, energy=e)  # graph capture, outside the timed run
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed replay
    t_exec = timed(lambda: plan.execute(D=Dm, energy=e), warm=False)
    torch.cuda.profiler.stop()
    energy = float(e.item())
    if world > 1:
        t_exec = reduce_max(t_exec, dist, dev)
        et = torch.tensor([energy], dtype=torch.float64, device=dev)
        dist.all_reduce(et)
        energy = float(et.item())
    res = {"workload": f"{natom} atoms (s x3 K=6,3,1, p x2 K=3,1, d K=1), Schwarz 1e-12, energy digestion, "
                       f"one persistent graph-replayed launch" + (f", work items split over {world} ranks + "
                                                                  "one all-reduce" if world > 1 else ""),
           "quartets": info["nquartets"], "jobs": info["njobs"], "work_items": info["nitems"],
           "slice_quartets_rank0": sl["nquartets"], "create_s": t_create, "execute_ms": t_exec,
           "quartets_per_s": info["nquartets"] / (t_exec / 1e3), "energy": energy,
           "gflops_sparse": flops / (t_exec / 1e3) / 1e9,
           "frac_fp64_peak_sparse": flops / (t_exec / 1e3) / 1e9 / FP64_PEAK_GFLOPS / world,
           "status": plan.status()}
    plan.destroy()
    if world == 1:
        # J and J + K, and the energy again, on the 16-atom plan
        mdb, Dm, plan, _ = make(16)
        info16 = plan.info()
        e16 = torch.zeros(1, dtype=torch.float64, device=dev)
        t_e = timed(lambda: plan.execute(D=Dm, energy=e16), reps=3)
        J = torch.empty_like(Dm)
        t_j = timed(lambda: plan.coulomb(Dm, J), reps=3)
        K = torch.empty_like(Dm)
        t_jk = timed(lambda: plan.jk(Dm, J=J, K=K), reps=3)
        res["atoms16"] = {"quartets": info16["nquartets"], "energy_ms": t_e, "coulomb_ms": t_j, "jk_ms": t_jk,
                          "energy_quartets_per_s": info16["nquartets"] / (t_e / 1e3)}
        plan.destroy()
    return res


def three_centre_variant(args, eri, dev):
    """3-centre integrals (x|cd), x a real solid harmonic: uncontracted
    auxiliary shells lx <= 3 against the class-sweep orbital pairs (K = 3),
    1e5 triples per class; the form (side order) each class ran and its FP64
    operation count give GFLOP/s and the fraction of the FP64 peak."""
    import torch
    from paper_2506_12501_gb300 import opcount
    basis, orb, aux = synth.three_centre_pools(seed=0, pool=512)
    db = eri.DeviceBasis(basis)
    tot_ms, tot_flops, tot_n = 0.0, 0.0, 0
    for lx in range(4):
        nterms = int(np.count_nonzero(np.abs(eri.solid_harmonics(lx)) > 1e-14))
        for lc, ld in ((0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)):
            x, ket, t = synth.three_centre_batch(orb, aux, (lx, lc, ld), seed=0, nt=args.three_nt)
            xd, kd, td = (torch.as_tensor(v, device=dev) for v in (x, ket, t))
            o = torch.empty(len(t) * (2 * lx + 1) * eri.nc(lc) * eri.nc(ld), dtype=torch.float64, device=dev)
            ms = timed(lambda: eri.eri_batch3(lx, lc, ld, db, xd, kd, td, pure=True, out=o), reps=2)
            sw, _ = eri.eri_last_form()
            tot_ms += ms
            tot_flops += opcount.sparse_flops3((lx, lc, ld), 1, 9, True, sw, nterms) * len(t)
            tot_n += len(t)
    return {"workload": f"x real solid harmonics lx <= 3 (K = 1, exponents 10^U(-1,1)) x orbital pairs l <= 2 "
                        f"(K = 3), 24 classes x {args.three_nt} triples",
            "triples": tot_n, "ms": tot_ms, "triples_per_s": tot_n / (tot_ms / 1e3),
            "gflops_sparse": tot_flops / (tot_ms / 1e3) / 1e9,
            "frac_fp64_peak_sparse": tot_flops / (tot_ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS}


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
    if only is not None and args.high_l_k:
        # profiling aid: one class of the high-l workload (l up to f, K per shell)
        hb = synth.split_batch(only, K=args.high_l_k, seed=rank, nq=args.nq)
        basis, batches = hb[0], {only: hb[1:]}
    else:
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
    Kps = args.high_l_k if (only is not None and args.high_l_k) else K_PER_SHELL
    dense = {c: opcount.dense_flops(c, Kps ** 2, Kps ** 2) for c in batches}
    stream = torch.cuda.current_stream()
    forms = {}
    tiles = {}

    def step(timing=None):
        for cls, (b, k, q) in dev_batches.items():
            if timing is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            eri.eri_batch(cls, db, b, k, q, out=outs[cls], precision=prec)
            forms[cls] = eri.eri_last_form()
            tiles[cls] = eri.eri_last_tile()
            if timing is not None:
                e1.record(stream)
                timing[cls].append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the FP64 operations of the form each class runs (chosen during warm-up)
    sparse = {c: opcount.sparse_flops(c, Kps ** 2, Kps ** 2, form=forms[c]) for c in batches}
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
            "ms": round(ms, 4), "qps": round(qps),
            "form": ("swapped " if forms[cls][0] else "") + ("hrr" if forms[cls][1] else "plain"),
            "tile": "TQ{tq} IC{ic} x{threads}".format(**tiles[cls]),
            "gflops": round(sparse[cls] * qps / 1e9, 1),
            "frac": round(sparse[cls] * qps / 1e9 / FP64_PEAK_GFLOPS, 4),
            "frac_dense": round(dense[cls] * qps / 1e9 / FP64_PEAK_GFLOPS, 4)}
    emit_detail("per_class", {"note": "qps = quartets/s; gflops and frac from the sparse FP64 count of the form "
                                      "that ran; frac_dense from the dense-GEMM count",
                              "per_class": per_class, "step_ms": [round(x, 3) for x in step_ms]}, rank)
    fwd_launches, fwd_ms = prof[eri.PROF_FWD]
    flops_per_step = sum(sparse[c] * nq_class for c in batches)
    dense_per_step = sum(dense[c] * nq_class for c in batches)
    fwd_gflops = flops_per_step * args.steps / (fwd_ms / 1e3) / 1e9 if fwd_ms > 0 else None
    roofline = {"bound": "alu", "kernel": "fwd_kernel", "achieved": fwd_gflops, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": (fwd_gflops / FP64_PEAK_GFLOPS) if fwd_gflops else None,
                "traffic": profile_traffic(),
                "peak_source": "derived: FP64 FMA pipe, 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                "flops": "sparse FP64 count of the implemented sequence, FMA = 2",
                "ms_per_launch": round(fwd_ms / max(fwd_launches, 1), 4),
                "frac_dense_formulation": round(dense_per_step * args.steps / (fwd_ms / 1e3) / 1e9 /
                                                FP64_PEAK_GFLOPS, 3) if fwd_ms else None}
    emit_detail("roofline_other_kernels", {"pair_ms_per_step": prof[eri.PROF_PAIR][1] / args.steps,
                                           "prepass_ms_per_step": prof[eri.PROF_PREPASS][1] / args.steps,
                                           "fwd_launches": fwd_launches}, rank)

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
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": len(e_ms)}
        emit_detail("e2e", {"step_ms": [round(x, 2) for x in e_ms]}, rank)
        del host_in, host_out

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sampled, spent = oracle_sweep_rate(basis, batches, budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sampled} quartets over all 81 classes ({spent:.0f} s of oracle work, double build, "
                         f"{cores} host threads); value = the sweep's class mix at the sampled per-class rates"}

    # ---- variants (each at its stated size)
    which = ALL_VARIANTS if args.variants is None else tuple(v for v in args.variants.split(",") if v and v != "none")
    summary = {}
    del outs, dev_batches, flush
    torch.cuda.empty_cache()
    if only is None or args.variants:
        if "peaks" in which and rank == 0:
            p = peaks_variant(eri)
            emit_detail("peaks", p, rank)
            summary["dfma_measured_gflops"] = round(p["dfma"]["gflops"], 1)
        if "split" in which and rank == 0 and world == 1:
            s = split_variant(args, eri, dev)
            emit_detail("split", s, rank)
            summary["split_speedup"] = {k: round(v["speedup"], 2) for k, v in s["per_class"].items()}
        if "adjoint" in which and rank == 0 and world == 1:
            a = adjoint_variant(args, eri, dev)
            emit_detail("adjoint", a, rank)
            summary["adjoint"] = {"grad_over_fwd": round(a["grad_over_fwd"], 2),
                                  "grad_frac": round(a["grad_frac_fp64_peak_sparse"], 3),
                                  "grad_qps": round(a["grad_quartets_per_s"])}
        if "batched" in which:
            bv = batched_variant(args, eri, dev, world, rank, dist)
            emit_detail("batched", bv, rank)
            summary["batched"] = {"natom": args.molecule_natom, "qps": round(bv["quartets_per_s"]),
                                  "frac": round(bv["frac_fp64_peak_sparse"], 3)}
        if "threecentre" in which and rank == 0 and world == 1:
            t3 = three_centre_variant(args, eri, dev)
            emit_detail("threecentre", t3, rank)
            summary["threecentre_tps"] = round(t3["triples_per_s"])

    if world > 1:
        dist.barrier()
    if rank == 0:
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                json.dump(DETAILS, f, indent=1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == eri.ERI_PREC_FP64 else "f64+f32x2",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if only is None else
                       f"single class {args.only_class}{' of the high-l workload' if args.high_l_k else ''}, "
                       f"{nq_class} quartets",
                       "classes": len(batches), "quartets_per_class": nq_class, "K_per_shell": Kps,
                       "l2": "flushed between timed steps (256 MiB write); outputs of 8 GB/step exceed L2",
                       "parallelism": f"weak x{world}: each rank its own seeded sweep"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": n_launch,
            "clocks": clk.summary(), "variants": summary,
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
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=None,
                    help="seconds of oracle work per reference step (default: a few minutes in all)")
    ap.add_argument("--only-class", default=None, help="profiling aid: one class, e.g. 2222")
    ap.add_argument("--high-l-k", type=int, default=0,
                    help="profiling aid with --only-class: the high-l workload (exponents 10^U(log 0.05, log 50)) "
                         "with this K per shell instead of the class sweep")
    ap.add_argument("--variants", default=None,
                    help="comma list of " + ",".join(ALL_VARIANTS) + " (default: all; 'none' for none)")
    ap.add_argument("--split-nq", type=int, default=100_000)
    ap.add_argument("--adjoint-nq", type=int, default=0, help="quartets per class of the adjoint (0: all)")
    ap.add_argument("--adjoint-only", default=None, help="profiling aid: comma list of adjoint classes, e.g. 1010")
    ap.add_argument("--adjoint-schemes", action="store_true",
                    help="adjoint variant: also time every class with one launch and with two launches forced")
    ap.add_argument("--molecule-natom", type=int, default=64)
    ap.add_argument("--three-nt", type=int, default=100_000, help="triples per 3-centre class")
    ap.add_argument("--nq", type=int, default=NQ_PER_CLASS, help="quartets per class")
    ap.add_argument("--precision", choices=["fp64", "split"], default="fp64",
                    help="transforms of the timed sweep (profiling aid; the benchmark value is fp64)")
    ap.add_argument("--detail-out", default=None, help="also write every detail object to this JSON file")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_library(args)


if __name__ == "__main__":
    main()
