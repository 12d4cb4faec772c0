#!/usr/bin/env python
"""Benchmark of the GPU arrowhead eigen-solver (one JSON line on rank 0).

Workload: the graded arrowhead of order n = 16384 (|d| = 10^U[-15,0] with random
signs, z = 10^U[-10,0], alpha = 1e3), all n eigenpairs with the full n x n
eigenvector matrix in FP64.  One step = one complete arrow_eig call (reduction,
shift-and-invert solve for every eigenvalue, remedies, vectors).

value      eigenpairs/s of the whole job, inputs resident in HBM, device time of
           exactly K steps (CUDA events on the solve stream), max over ranks.
           Between steps a 512 MiB buffer is written to flush L2 (129 MB).
e2e        the same metric through arrow_eig_host: pinned host d, z in, lambda
           and V (2 GiB) out, copies inside the timed region.
roofline   the eigenvalue kernel (k_eig): algorithmic FP64 flops per launch
           (3 per term per evaluation of the secular function: subtract,
           divide, add, as in Algorithm 3; 3 more per Newton evaluation that
           forms the derivative; 3 per term for the shift choice where it ran
           in FP64; 20 per term for the
           double-double element b, or 3 for a standard-precision b under
           Algorithm 5's gate; 6 per eigenvector component, which k_eig
           writes as soon as each eigenvalue is known) over its event-timed
           duration, against the
           FP64 ALU peak 152 SMs x 4 flop/clk x 2070 MHz.  Also reported: the
           all-FP64 bisection's algorithmic work over the headline form's k_eig
           time (fp64_bisection_equivalent_tflops).
forms      fp32_newton_gated (default headline): two FP32 model steps open
           the search, then the bracketed Newton finish in FP64 (same Pick
           function, bracket and stop test as Algorithm 3), with Algorithm 5's
           gates (b in standard precision unless the spike ratio and K_b ask for
           double-double); Algorithm 1's midpoint test in FP32 with an error
           bound, in FP64 only where the bound leaves its sign open.
           fp64_newton_gated: the same without FP32 (opening and midpoint
           test); fp32_newton / fp64_newton: b always in double-double; fp32:
           FP32 opening bracket then FP64 bisection; fp64: all-FP64 bisection as
           in Algorithm 3.  All six are timed; --form picks the headline.
cpu_baseline  the CPU oracle on a bounded sample of eigenpairs of the same
           matrix, on all host cores.
--impl reference   times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun): each rank solves its own instance (weak scaling, no
collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s at ≤10nε64 rel. err (n=16384, batched); p50/p99 solve latency"
UNIT = "eigenpairs/s"
N_DEFAULT = 16384
# k_check k_rank k_reduce k_post k_eig k_fix_decide k_fix_solve k_place k_vectors
LAUNCHES_PER_STEP = 9
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12


# ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size k_eig
# launch (graded n = 16384, fp32_newton_gated form; a 1-pass capture), with the hash
# of the CUDA sources it was measured on.  The bench reports it as the
# roofline's traffic only while the form, n and sources match.
KEIG_TRAFFIC = {"form": "fp32_newton_gated", "n": 16384,
                "read": 11312296960, "write": 8553951488,
                "src_sha256": "2314eb003cadf94aa5bd37e1455cc8c22230495a9c393ee842b94bd36f7bdd5d"}


def csrc_sha256():
    import hashlib
    d = os.path.join(ROOT, "paper_1302_7203_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        p = os.path.join(d, f)
        if os.path.isfile(p):
            h.update(f.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


# solver forms: (ae_opts.precision, ae_opts.finish, ae_opts.bgate)
FORMS = {"fp32": (1, 0, 0), "fp64": (0, 0, 0), "fp32_newton": (1, 1, 0),
         "fp64_newton": (0, 1, 0), "fp64_newton_gated": (0, 1, 1),
         "fp32_newton_gated": (1, 1, 1)}


def form_opts(arrowhead, form, **kw):
    prec, fin, gate = FORMS[form]
    return arrowhead.default_opts(precision=prec, finish=fin, bgate=gate, **kw)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--form", default="fp32_newton_gated", choices=list(FORMS),
                   help="headline form: fp32_newton_gated = FP32 opening, Algorithm 5's "
                        "precision gates and the bracketed Newton finish in FP64 (default); "
                        "fp64_newton_gated = the same without the FP32 opening; fp64_newton / "
                        "fp32_newton = b always double-double; fp32 = FP32 opening bracket + "
                        "FP64 bisection; fp64 = all-FP64 bisection (Algorithm 3)")
    p.add_argument("--forms", default=",".join(FORMS),
                   help="comma-separated forms to time beside the headline (default: all)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-extras", action="store_true",
                   help="skip the DPR1 / SVD / batched / serving measurements")
    p.add_argument("--serve-requests", type=int, default=120)
    p.add_argument("--batch-only", type=int, default=0, metavar="COUNT",
                   help="profiling aid: run only the batched plan on the first COUNT "
                        "instances of the 4096-instance set (2 warm-up runs, 1 timed) "
                        "and print one line about it")
    return p.parse_args()


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def eig_kernel_flops(n, ncomp, total_iter, fix_iter, n_ddb=None, total_deriv=0, vectors=True,
                     n_mid=None):
    """Algorithmic FP64 flops of one k_eig launch (see module docstring).

    Per term: 3 flops for the shift choice (Algorithm 1's midpoint test) where
    it ran in FP64 (n_mid = the eigenpairs whose test did; None: all of them);
    20 for the double-double b, or 3 (subtract, divide, add) for a standard one
    where Algorithm 5's gate kept it (n_ddb = the eigenpairs it sent to
    double-double; None: all double-double); 3 per FP64 evaluation of the
    secular function (subtract, divide, add, as in Algorithm 3) and 3 more per
    Newton evaluation that also formed the derivative (total_deriv).  vectors:
    6 flops per eigenvector component (Eq. Aeigenvec: 2 subtractions and a
    division; square, add and scale to normalise), which k_eig writes.  Work
    done in FP32 (the opening model steps, the certified midpoint tests) is
    not counted."""
    terms = n - 2                    # each O(n) pass runs over the other poles
    b = 20.0 * ncomp if n_ddb is None else 3.0 * ncomp + 20.0 * n_ddb
    vec = 6.0 * (n - 1) * ncomp if vectors else 0.0
    evals = 3.0 * (total_iter - fix_iter) + 3.0 * total_deriv
    mid = 3.0 * (ncomp if n_mid is None else n_mid)
    return terms * (evals + mid + b) + vec


def form_flops(n, info, form):
    """eig_kernel_flops for a run of `form` from its ae_info counters."""
    prec, _, gate = FORMS[form]
    return eig_kernel_flops(n, info["n_reduced"], info["total_iter"], info["fix_iter"],
                            info["n_ddb"] if gate else None, info["total_deriv"],
                            n_mid=info["n_mid64"] if prec == 1 else None)


def cpu_baseline(d, z, alpha, n, seconds):
    """Time the oracle on a sample; also return its results for an error check."""
    import oracle
    oracle.build_oracle()
    # size the sample from a short calibration run
    ks = np.linspace(0, n - 1, 16).astype(np.int64)
    t0 = time.perf_counter()
    oracle.arrow_eig(d, z, alpha, ks=ks)
    per = (time.perf_counter() - t0) / ks.size
    cnt = int(max(16, min(n, seconds / max(per, 1e-9))))
    ks = np.unique(np.linspace(0, n - 1, cnt).astype(np.int64))
    t0 = time.perf_counter()
    res = oracle.arrow_eig(d, z, alpha, ks=ks)
    dt = time.perf_counter() - t0
    return ({"value": ks.size / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
             "sample": f"{ks.size} of {n} eigenpairs (evenly spaced) with vectors, "
                       f"double-double oracle, {dt:.1f} s"}, ks, res)


def max_err_neps(lam, Vcols, res, n):
    """Max relative error of GPU results vs the oracle sample, in units of n eps64."""
    eps = 2.0 ** -53
    tol = 10 * n * eps
    scale = np.maximum(np.abs(res["lam"]), 4 * res["abserr"] / tol)
    el = np.max(np.abs(lam - res["lam"]) / scale) / (n * eps)
    ev = np.max(np.abs(Vcols - res["V"]) /
                np.maximum(np.abs(res["V"]), np.finfo(float).tiny)) / (n * eps)
    return {"lambda": float(el), "vectors": float(ev), "bound": 10.0}


def timed_device(fn, steps, warmup, stream, flush):
    """Device time (ms per step) of fn() over `steps` runs after `warmup`."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for i in range(steps):
        flush.fill_(i & 0xff)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def extras(arrowhead, W, dev, stream, flush, args):
    """DPR1, SVD, Hermitian and non-symmetric arrowheads (n = 8192), the batched
    set and a serving sweep."""
    import torch
    out = {}
    opts = form_opts(arrowhead, args.form, profile=1)
    n = 8192
    d, u, rho = W.uniform_dpr1(n, seed=3)
    dt, ut = torch.as_tensor(d, device=dev), torch.as_tensor(u, device=dev)
    Q = torch.empty((n, n), dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    info = {}

    def f_dpr1():
        info.update(arrowhead.dpr1_eig(dt, ut, rho, opts=opts, info=True,
                                       out={"lam": lam, "Q": Q}, stream=stream)["info"])
    ms = timed_device(f_dpr1, 3, 1, stream, flush)
    fl = form_flops(n + 1, info, args.form)
    out["dpr1_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"],
                         "frac_fp64": fl / (info["ms_eig"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    d, z, al = W.uniform_tsvd(n, seed=4)
    dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
    U = torch.empty((n, n), dtype=torch.float64, device=dev)

    def f_svd():
        info.update(arrowhead.tri_arrow_svd(dt, zt, al, opts=opts, info=True,
                                            out={"s": lam, "U": U, "V": Q}, stream=stream)["info"])
    ms = timed_device(f_svd, 3, 1, stream, flush)
    fl = form_flops(n, info, args.form)
    out["svd_n8192"] = {"value": n / (ms / 1e3), "unit": "singular triplets/s", "ms_per_step": ms,
                        "k_eig_ms": info["ms_eig"],
                        "frac_fp64": fl / (info["ms_eig"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    # Hermitian arrowhead (Sec. 6.1), complex U
    d, z, al = W.uniform_herm(n, seed=8)
    dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
    del U
    Uc = torch.empty((n, n), dtype=torch.complex128, device=dev)

    def f_herm():
        info.update(arrowhead.herm_arrow_eig(dt, zt, al, opts=opts, info=True,
                                             out={"lam": lam, "U": Uc}, stream=stream)["info"])
    ms = timed_device(f_herm, 3, 1, stream, flush)
    fl = form_flops(n, info, args.form)
    out["herm_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"],
                         "frac_fp64": fl / (info["ms_eig"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    del Uc
    # non-symmetric arrowhead (Remark of Sec. 6.1), right and left vectors
    d, zc, zr, al = W.uniform_nsym(n, seed=10)
    dt, zct, zrt = (torch.as_tensor(x, device=dev) for x in (d, zc, zr))
    Y = torch.empty((n, n), dtype=torch.float64, device=dev)

    def f_nsym():
        info.update(arrowhead.nsym_arrow_eig(dt, zct, zrt, al, opts=opts, info=True,
                                             out={"lam": lam, "X": Q, "Y": Y},
                                             stream=stream)["info"])
    ms = timed_device(f_nsym, 3, 1, stream, flush)
    fl = form_flops(n, info, args.form)
    out["nsym_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"],
                         "frac_fp64": fl / (info["ms_eig"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    del Q, Y
    # batched: 4096 instances, orders log-uniform in [32, 4096], one CUDA-graph plan
    inst = W.uniform_batch(4096, seed=2)
    B = arrowhead.Batch(inst, opts=form_opts(arrowhead, args.form), stream=stream)
    ms = timed_device(lambda: B.run(), 2, 1, stream, flush)
    binfo = B.run(info=True)
    tot_n = int(B.n_off[-1])
    out["batched_4096"] = {"value": tot_n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "instances": len(inst), "eigenpairs": tot_n,
                           "sum_n2": int((B.n.astype(np.int64) ** 2).sum()),
                           "fp64_steps_per_eigenpair": binfo["total_iter"] / tot_n,
                           "team_widths": {str(b): arrowhead.lib().ae_team_width(b)
                                           for b in (32, 64, 128, 256, 512)}}
    B.close()
    del B
    torch.cuda.empty_cache()
    # serving: Poisson arrivals of mixed kinds, orders log-uniform in [64, 16384]
    out["serving"] = serve_sweep(arrowhead, W, dev, args.serve_requests,
                                 form_opts(arrowhead, args.form))
    return out


def serve_sweep(arrowhead, W, dev, count, opts):
    import torch
    res = {}
    for rate in (20.0, 200.0, 2000.0):
        t_arr, kinds, ns = W.serve_stream(rate, count, seed=5)
        reqs = []
        for i, (k, n) in enumerate(zip(kinds, ns)):
            if k == 0:
                d, z, a = W.uniform_arrow(int(n), seed=10_000 + i)
            elif k == 1:
                d, z, a = W.uniform_dpr1(int(n), seed=10_000 + i)
            else:
                d, z, a = W.uniform_tsvd(int(n), seed=10_000 + i)
            reqs.append((int(k), torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev), a))
        srv = arrowhead.Server(budget_bytes=96 << 30, max_inflight=16, queue_cap=1 << 16,
                               opts=opts)
        t0 = time.perf_counter()
        pending = []
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and t_arr[i] <= now:
                k, dt, zt, a = reqs[i]
                tk = srv.submit(k, dt, zt, a, vectors=True)
                if tk is not None:
                    pending.append(tk)
                i += 1
            still = []
            for tk in pending:
                st, _ = srv.poll(tk)
                if st in (arrowhead.REQ_DONE, arrowhead.REQ_ERROR):
                    srv.release(tk)
                else:
                    still.append(tk)
            pending = still
            time.sleep(0.0002)
        st = srv.stats()
        srv.close()
        res[f"{int(rate)}/s"] = {"p50_ms": 1e3 * st["p50_s"], "p99_ms": 1e3 * st["p99_s"],
                                 "eigenpairs_per_s": st["eigenpairs_per_s"],
                                 "completed": st["completed"], "rejected": st["rejected"],
                                 "failed": st["failed"]}
    res["requests_per_rate"] = count
    res["mix"] = "arrow/DPR1/SVD uniform, orders log-uniform [64, 16384], vectors kept on device"
    return res


def workload_config(n, form, world):
    """The `config` of both arms' JSON lines (the reference arm times a sample of
    the same workload, said in its cpu_baseline.sample)."""
    return {"workload": f"graded arrowhead n={n}: all eigenpairs + full V",
            "n": n, "form": form, "l2": "512 MiB write between steps (L2 flush)",
            "parallelism": f"{world} independent instances"}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    from paper_1302_7203_gb300 import workloads as W
    import oracle
    oracle.build_oracle()
    n = args.n
    d, z, alpha = W.graded_arrow(n, seed=1)
    per_step = max(8, int(args.cpu_seconds * 4 / max(args.steps + args.warmup, 1)))
    ks0 = np.linspace(0, n - 1, per_step).astype(np.int64)
    for _ in range(args.warmup):
        oracle.arrow_eig(d, z, alpha, ks=ks0[:8])
    t0 = time.perf_counter()
    for s in range(args.steps):
        ks = np.unique((ks0 + s) % n)
        oracle.arrow_eig(d, z, alpha, ks=ks)
    dt = time.perf_counter() - t0
    done = per_step * args.steps
    val = done / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (double-double oracle)",
            "data": "synthetic",
            "config": workload_config(n, args.form, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} evenly spaced eigenpairs (with vectors) "
                                       f"per step of the {n}; double-double oracle"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_1302_7203_gb300 import arrowhead, build, shard, workloads as W
    build.build()
    torch.cuda.set_device(local)
    if args.batch_only > 0:
        inst = W.uniform_batch(4096, seed=2)[:args.batch_only]
        st = torch.cuda.current_stream()
        B = arrowhead.Batch(inst, opts=form_opts(arrowhead, args.form), stream=st)
        for _ in range(2):
            B.run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        B.run()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"mode": "batch_only", "instances": len(inst),
                          "eigenpairs": int(B.n_off[-1]), "ms": ms,
                          "eigenpairs_per_s": int(B.n_off[-1]) / (ms / 1e3)}), flush=True)
        B.close()
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    d, z, alpha = W.graded_arrow(n, seed=shard.rank_seed(1, rank))
    dev = torch.device("cuda", local)
    dt = torch.as_tensor(d, device=dev)
    zt = torch.as_tensor(z, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(form):
        opts = form_opts(arrowhead, form, profile=1)

        def step():
            return arrowhead.arrow_eig(dt, zt, alpha, opts=opts, info=True,
                                       out={"lam": lam, "V": V}, stream=stream)

        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        infos = []
        with Clocks(local) as clk:
            torch.cuda.synchronize()
            for i in range(args.steps):
                flush.fill_(i & 0xff)                 # evict L2 between steps
                starts[i].record(stream)
                infos.append(step()["info"])
                ends[i].record(stream)
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        total = float(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
        if world > 1:
            total = shard.max_over_ranks(total, device=dev)
        return total, infos, clk

    primary = args.form
    # the other forms first, so lam/V hold the headline form's results at the end
    wanted = [f for f in args.forms.split(",") if f in FORMS]
    runs = {f: timed(f) for f in wanted if f != primary}
    runs[primary] = timed(primary)
    total_ms, infos, clk = runs[primary]
    value = world * n * args.steps / (total_ms / 1e3)
    info = infos[-1]
    eig_ms = float(np.mean([x["ms_eig"] for x in infos]))
    flops = form_flops(n, info, primary)
    achieved = flops / (eig_ms / 1e3) / 1e12
    # the all-FP64 bisection's algorithmic work (its measured step count) over
    # this form's k_eig time: the rate at which the paper's work gets done
    eq = None
    if "fp64" in runs:
        i64 = runs["fp64"][1][-1]
        eq = eig_kernel_flops(n, i64["n_reduced"], i64["total_iter"],
                              i64["fix_iter"]) / (eig_ms / 1e3) / 1e12
    traffic = None
    if (KEIG_TRAFFIC["form"] == primary and KEIG_TRAFFIC["n"] == n
            and KEIG_TRAFFIC["src_sha256"] == csrc_sha256()):
        traffic = KEIG_TRAFFIC["read"] + KEIG_TRAFFIC["write"]
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
            "traffic_note": "bytes per k_eig launch: the per-warp stored (delta_j, "
                            "zeta_j^2/delta_j) pairs (written once per eigenpair, re-read "
                            "by each FP64 evaluation), the staged eigenvector column and "
                            "the n x n V written once",
            "kernel": "k_eig", "kernel_ms": eig_ms,
            "fp64_bisection_equivalent_tflops": eq,
            "peak_note": "FP64 ALU: 152 SMs x 4 flop/clk x 2070 MHz (nominal 1.25 TFLOP/s)"}

    e2e = None
    if not args.no_e2e:
        dh = torch.as_tensor(d).pin_memory()
        zh = torch.as_tensor(z).pin_memory()
        lh = torch.empty(n, dtype=torch.float64).pin_memory()
        Vh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        eopts = form_opts(arrowhead, primary)
        arrowhead.arrow_eig_host(dh, zh, alpha, opts=eopts, out={"lam": lh, "V": Vh},
                                 stream=stream)
        t0 = time.perf_counter()
        ne = max(2, min(args.steps, 3))
        for _ in range(ne):
            arrowhead.arrow_eig_host(dh, zh, alpha, opts=eopts, out={"lam": lh, "V": Vh},
                                     stream=stream)
        te = time.perf_counter() - t0
        if world > 1:
            te = shard.max_over_ranks(te, device=dev)
        e2e = {"value": world * n * ne / te, "unit": UNIT,
               "h2d_bytes_per_step": 2 * (n - 1) * 8, "d2h_bytes_per_step": (n + n * n) * 8}

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, ks, ores = cpu_baseline(d, z, alpha, n, args.cpu_seconds)
        kt = torch.as_tensor(ks, device=dev)
        err = max_err_neps(lam[kt].cpu().numpy(), V[kt].t().cpu().numpy(), ores, n)
    extra = None
    if world == 1 and not args.no_extras:
        del V
        torch.cuda.empty_cache()
        extra = extras(arrowhead, W, dev, stream, flush, args)

    if rank == 0:
        variants = {}
        for form, (tot, inf, _) in runs.items():
            variants[form] = {
                "value": world * n * args.steps / (tot / 1e3), "ms_per_step": tot / args.steps,
                "ms_eig": float(np.mean([x["ms_eig"] for x in inf])),
                "fp64_steps_per_eigenpair": inf[-1]["total_iter"] / n,
                "fp32_fallbacks": inf[-1]["n_fp32_fallback"],
                "b_double_double": inf[-1]["n_ddb"]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(n, primary, world),
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "max_err_neps": err, "variants": variants, "extras": extra,
                "clocks": clk.summary(), "gpu_launches": LAUNCHES_PER_STEP * args.steps,
                "phases_ms": {k: float(np.mean([x[k] for x in infos]))
                              for k in ("ms_reduce", "ms_eig", "ms_fix", "ms_vectors")},
                "solver": {k: info[k] for k in ("n_nearzero", "n_otherpole", "n_dpr1shift",
                                                "n_capped", "max_iter_used", "total_iter",
                                                "fix_iter", "total_deriv", "n_ddb",
                                                "n_mid64", "max_Kb", "max_Knu")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
