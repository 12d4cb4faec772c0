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
           in FP64; 20 per term for the double-double element b, or 3 for a
           standard-precision b under Algorithm 5's gate; 6 per eigenvector
           component, which k_eig writes as soon as each eigenvalue is known)
           over its event-timed duration, against the FP64 FMA throughput
           measured on this GPU at the start of the run (ae_fma_peaks).  Also
           reported: the FP64 instructions the kernel retires per term (from
           the per-pass instruction counts and the solver's counters) and the
           FP64-pipe busy fraction they imply; a mixed FP32 + FP64 roofline
           for the forms that work in FP32 and double-float; and the all-FP64
           bisection's algorithmic work over the headline form's k_eig time.
forms      fp32_newton_gated (default headline): FP32 model steps open the
           search, then the bracketed Newton finish in FP64 (same Pick
           function, bracket and stop test as Algorithm 3), with Algorithm 5's
           gates (b in standard precision unless the spike ratio and K_b ask for
           double-double); Algorithm 1's midpoint test in FP32 with an error
           bound, in FP64 only where the bound leaves its sign open.
           fp64_newton_gated: the same without FP32 (opening and midpoint
           test); fp32_newton / fp64_newton: b always in double-double; fp32:
           FP32 opening bracket then FP64 bisection; fp64: all-FP64 bisection as
           in Algorithm 3.  All six are timed; --form picks the headline.
           Every form's results are compared with the CPU oracle on a sample
           of eigenpairs (max_err_neps, in units of n eps64; the bar is 10);
           parity_ok is false when any form or extra misses it.
cpu_baseline  the CPU oracle on a bounded sample of eigenpairs of the same
           matrix, on all host cores.  --cpu-full also times it end to end on
           the other configurations (median of 3).
extras     the plain method on the n = 1000 uniform arrowhead, DPR1 and
           triangular-arrowhead SVD (n = 8192), Hermitian and non-symmetric
           arrowheads (n = 8192), the 4096-instance batched set, and a serving
           sweep of Poisson request streams, each with its error against the
           oracle.
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
EPS64 = 2.0 ** -53
ERR_BOUND = 10.0            # the acceptance bar, in units of n eps64
# k_check k_rank k_reduce k_post k_eig k_fix_decide k_fix_solve k_place k_vectors
LAUNCHES_PER_STEP = 9
# nominal FP64 rate, for context only (the roofline uses the measured one)
FP64_NOMINAL_TFLOPS = 152 * 4 * 2070e6 / 1e12

# FP64 instructions a term of each O(n) pass of k_eig retires (per lane):
# Algorithm 1's midpoint test in FP64 (difference, reciprocal 3, accumulate);
# pass A with a standard-precision b (difference 1, reciprocal 3, quotient 1,
# sum 1, sum of squares 1, stores' address arithmetic 1); with a double-double
# b (ordered TwoSum 4, reciprocal 3, partial quotients 4, compensated add 6,
# sum of squares 1, misc. 3); an FP64 evaluation of the secular function
# (1 - x delta, reciprocal 3, accumulate), plus 3 when it forms the derivative;
# an eigenvector component (difference 2, reciprocal 3, product, square-sum,
# scale), one difference fewer where the input is sorted and undeflated and
# the pass reads the stored shifted difference (arrowhead, Hermitian and
# non-symmetric kinds).
INSTR_PER_TERM = {"mid": 6, "b_std": 8, "b_dd": 21, "eval": 5, "deriv": 3, "vector": 8,
                  "vector_stored": 7}
# algorithmic FP32 flops a term of an FP32 pass (difference, division, sum and
# the derivative's three) and of a double-float pass (the emulated products,
# reciprocal and compensated sums of the opening model step, counted by the
# FP32 operations they take, a fused multiply-add as 2)
FP32_FLOPS_PER_TERM = {"f32": 6, "df": 45}


# ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size k_eig
# launch (graded n = 16384, fp32_newton_gated form; a 1-pass capture), with the hash
# of the CUDA sources it was measured on.  The bench reports it as the
# roofline's traffic only while the form, n and sources match.
KEIG_TRAFFIC = {"form": "fp32_newton_gated", "n": 16384,
                "read": 15391182336, "write": 8560969728,
                "src_sha256": "9489edb4e9a5e1dee06e85a7d58353c99dcb4c0b624319cdff3c9a6801bf74d8"}


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

SERVE_RATES = (100, 300, 1000, 2000, 5000, 10000, 20000, 50000)


def form_opts(arrowhead, form, **kw):
    prec, fin, gate = FORMS[form]
    return arrowhead.default_opts(precision=prec, finish=fin, bgate=gate, **kw)


def parse(argv=None):
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
    p.add_argument("--no-cpu", action="store_true",
                   help="skip the timed CPU baseline (the parity sample is still solved)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--cpu-full", action="store_true",
                   help="also time the oracle end to end on configs 0, 1, 3a, 3b (median "
                        "of 3) and on a sample of the batched set (minutes)")
    p.add_argument("--parity-sample", type=int, default=256,
                   help="eigenpairs of the benchmark matrix compared with the oracle when "
                        "the CPU baseline is skipped")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the n=1000 / DPR1 / SVD / Hermitian / non-symmetric / batched / "
                        "serving measurements")
    p.add_argument("--serve-requests", type=int, default=2000,
                   help="requests per rate (fewer at rates that would take over 10 s)")
    p.add_argument("--serve-rates", default=",".join(str(r) for r in SERVE_RATES))
    p.add_argument("--split", default="none", choices=["none", "instance", "batch"],
                   help="multi-GPU work division: none = one independent instance per rank "
                        "(weak scaling, the default); instance = the one n x n instance split "
                        "by eigenpair ranges (arrow_eig_part, strong scaling); batch = the "
                        "4096-instance batched set bin-packed on n^2 across ranks (strong "
                        "scaling)")
    p.add_argument("--batch-only", type=int, default=0, metavar="COUNT",
                   help="profiling aid: run only the batched plan on the first COUNT "
                        "instances of the 4096-instance set (2 warm-up runs, 1 timed) "
                        "and print one line about it")
    return p.parse_args(argv)


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


# ---------------------------------------------------------------------------
# roofline accounting (host arithmetic on the solver's counters)
# ---------------------------------------------------------------------------
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


def fp64_instructions(n, info, form, terms=None, stored_diff=False):
    """FP64 lane-instructions the O(n) passes of one k_eig launch retire, from
    INSTR_PER_TERM and the solver's counters (the Newton finish's scalar
    bookkeeping, O(1) per eigenpair, is not included).  `terms`: the terms
    of an O(n) pass (default n - 2); `stored_diff`: the eigenvector pass
    reads the stored shifted differences (sorted, undeflated arrowhead)."""
    prec, _, gate = FORMS[form]
    ncomp = info["n_reduced"]
    t = (n - 2) if terms is None else terms
    c = INSTR_PER_TERM
    mid = c["mid"] * (info["n_mid64"] if prec == 1 else ncomp)
    b = (c["b_std"] * ncomp + c["b_dd"] * info["n_ddb"]) if gate else c["b_dd"] * ncomp
    evals = (c["eval"] * (info["total_iter"] - info["fix_iter"]) +
             c["deriv"] * info["total_deriv"])
    vec = (c["vector_stored"] if stored_diff else c["vector"]) * ncomp * \
        ((n - 1) if terms is None else terms + 1)
    return t * (mid + b + evals) + vec


def remedy_work(info, terms):
    """Algorithmic FP64 flops and FP64 lane-instructions of the remedy solves
    (Remarks 1 and 2), for a roofline over a whole plan whose time includes
    them: a Remark 1 / 2(b) solve forms its rho-denominator in double-double
    (20 flops, INSTR_PER_TERM b_dd a term), a Remark 2(a) solve a standard b
    from the other pole (3 flops, b_std); each remedy's FP64 evaluations
    (fix_iter, 3 flops and `eval` instructions a term) and its rewritten
    eigenvector column (6 flops and `vector` instructions a component)."""
    c = INSTR_PER_TERM
    n_dd = info["n_dpr1shift"] + info["n_nearzero"]
    n_op = info["n_otherpole"]
    flops = terms * (20.0 * n_dd + 3.0 * n_op + 3.0 * info["fix_iter"]) + \
        6.0 * (terms + 1) * (n_dd + n_op)
    instr = terms * (c["b_dd"] * n_dd + c["b_std"] * n_op + c["eval"] * info["fix_iter"]) + \
        c["vector"] * (terms + 1) * (n_dd + n_op)
    return flops, instr


def fp32_flops(n, info, terms=None):
    """Algorithmic FP32 flops of the FP32 and double-float passes (all
    eigenpairs, remedies included)."""
    t = (n - 2) if terms is None else terms
    return t * (FP32_FLOPS_PER_TERM["f32"] * info.get("n_f32_passes", 0) +
                FP32_FLOPS_PER_TERM["df"] * info.get("n_df_passes", 0))


def roofline_numbers(flops64, instr64, flops32, seconds, peaks):
    """frac of the FP64 roofline, the FP64-pipe busy fraction the instruction
    count implies (an FMA lane-instruction is 2 flops of peak), and the mixed
    FP32 + FP64 bound (the pipes run side by side: the slower one bounds)."""
    p64 = peaks["fp64_tflops"] * 1e12
    p32 = peaks["fp32_tflops"] * 1e12
    achieved = flops64 / seconds / 1e12
    t64, t32 = flops64 / p64, flops32 / p32
    return {"achieved": achieved, "frac": achieved / peaks["fp64_tflops"],
            "fp64_instr_per_term": None, "fp64_pipe_busy_implied": instr64 / (p64 / 2) / seconds,
            "mixed": {"fp64_tflop": flops64 / 1e12, "fp32_tflop": flops32 / 1e12,
                      "t_fp64_ms": 1e3 * t64, "t_fp32_ms": 1e3 * t32,
                      "frac": max(t64, t32) / seconds}}


def batch_terms(ns):
    """The terms of an average O(n) pass over a batch's eigenpairs: each of an
    instance's n_i eigenpairs runs its passes over n_i - 2 other poles."""
    ns = np.asarray(ns, dtype=np.float64)
    return float((ns * (ns - 2)).sum() / ns.sum())


# ---------------------------------------------------------------------------
# errors against the oracle
# ---------------------------------------------------------------------------
def max_err_neps(lam, Vcols, res, n):
    """Max relative error of GPU results vs the oracle sample, in units of n
    eps64.  An eigenvalue whose oracle bound exceeds a quarter of the bar is
    compared against that bound and counted in `widened`."""
    tol = ERR_BOUND * n * EPS64
    lam_or = res["lam"]
    absb = res.get("abserr", np.zeros_like(lam_or))
    wid = 4 * absb / tol > np.abs(lam_or)
    scale = np.maximum(np.abs(lam_or), 4 * absb / tol)
    scale = np.where(scale == 0, 1.0, scale)
    el = float(np.max(np.abs(lam - lam_or) / scale) / (n * EPS64)) if lam.size else 0.0
    out = {"lambda": el, "bound": ERR_BOUND, "widened": int(wid.sum()),
           "pairs": int(lam_or.size)}
    if Vcols is not None:
        ref = res["V"]
        ev = np.max(np.abs(Vcols - ref) / np.maximum(np.abs(ref), np.finfo(float).tiny))
        out["vectors"] = float(ev / (n * EPS64))
    return out


def err_ok(e):
    return e is None or (e["lambda"] <= e["bound"] and e.get("vectors", 0.0) <= e["bound"])


def sample_ks(n, count, seed=0):
    """Ends, middle and an even spread of `count` positions."""
    ks = np.concatenate([[0, 1, n // 2, n - 2, n - 1], np.linspace(0, n - 1, count)])
    return np.unique(np.clip(ks.astype(np.int64), 0, n - 1))


def cpu_baseline(d, z, alpha, n, seconds):
    """Time the oracle on a sample; also return its results for an error check."""
    import oracle
    oracle.build_oracle()
    # size the sample from a short calibration run
    ks = np.linspace(0, n - 1, 2 * oracle.threads()).astype(np.int64)
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


def measure_peaks(arrowhead, index, stream):
    """FP64 and FP32 FMA throughput of this GPU (ae_fma_peaks), best of 3 calls,
    with the SM clock sampled meanwhile."""
    best = {"fp64_tflops": 0.0, "fp32_tflops": 0.0}
    with Clocks(index) as clk:
        for _ in range(3):
            p = arrowhead.fma_peaks(stream=stream)
            for k in best:
                best[k] = max(best[k], p[k])
    best["clocks"] = clk.summary()
    best["how"] = ("ae_fma_peaks: a grid filling every SM runs 8 independent FMA chains a "
                   "thread; CUDA-event time, best of 3 x 3 launches")
    return best


# ---------------------------------------------------------------------------
# extras
# ---------------------------------------------------------------------------
def extras(arrowhead, W, dev, stream, flush, args, peaks):
    """Plain method on n = 1000; DPR1, SVD, Hermitian and non-symmetric
    arrowheads (n = 8192); the batched set; a serving sweep.  Each with its
    error against the oracle on sampled columns."""
    import torch
    import oracle
    out = {}
    opts = form_opts(arrowhead, args.form, profile=1)
    info = {}

    def kernel_roof(n, form, ms_eig, terms=None, stored=False):
        fl = form_flops(n, info, form)
        ins = fp64_instructions(n, info, form, terms, stored_diff=stored and
                                info["n_deflated"] == 0)
        r = roofline_numbers(fl, ins, fp32_flops(n, info, terms), ms_eig / 1e3, peaks)
        return {"frac_fp64": r["frac"], "fp64_pipe_busy_implied": r["fp64_pipe_busy_implied"],
                "mixed_frac": r["mixed"]["frac"]}

    # config 0: the plain method (all-FP64 bisection, Algorithm 3 as printed)
    # and the headline form on the n = 1000 uniform arrowhead; full oracle
    n = 1000
    d, z, a = W.uniform_arrow(n, seed=0)
    dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    ref = oracle.arrow_eig(d, z, a)
    res0 = {}
    for form in ("fp64", args.form):
        o = form_opts(arrowhead, form, profile=1)

        def f0():
            info.update(arrowhead.arrow_eig(dt, zt, a, opts=o, info=True,
                                            out={"lam": lam, "V": V}, stream=stream)["info"])
        ms = timed_device(f0, 10, 3, stream, flush)
        e = max_err_neps(lam.cpu().numpy(), V.t().cpu().numpy(), ref, n)
        res0[form] = {"value": n / (ms / 1e3), "ms_per_step": ms, "k_eig_ms": info["ms_eig"],
                      "max_err_neps": e, **kernel_roof(n, form, info["ms_eig"], stored=True)}
    out["uniform_n1000"] = {"unit": UNIT, "forms": res0,
                            "note": "config 0; fp64 = the plain method (Algorithm 3's "
                                    "bisection, b in double-double); errors on all 1000 "
                                    "eigenpairs"}
    del V
    n = 8192
    ks = sample_ks(n, 64)
    kt = torch.as_tensor(ks, device=dev)
    d, u, rho = W.uniform_dpr1(n, seed=3)
    dt, ut = torch.as_tensor(d, device=dev), torch.as_tensor(u, device=dev)
    Q = torch.empty((n, n), dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)

    def f_dpr1():
        info.update(arrowhead.dpr1_eig(dt, ut, rho, opts=opts, info=True,
                                       out={"lam": lam, "Q": Q}, stream=stream)["info"])
    ms = timed_device(f_dpr1, 3, 1, stream, flush)
    r = oracle.dpr1_eig(d, u, rho, ks=ks)
    e = max_err_neps(lam[kt].cpu().numpy(), Q[kt].t().cpu().numpy(),
                     {"lam": r["lam"], "V": r["Q"]}, n)
    out["dpr1_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"], "max_err_neps": e,
                         **kernel_roof(n + 1, args.form, info["ms_eig"])}
    d, z, al = W.uniform_tsvd(n, seed=4)
    dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
    U = torch.empty((n, n), dtype=torch.float64, device=dev)

    def f_svd():
        info.update(arrowhead.tri_arrow_svd(dt, zt, al, opts=opts, info=True,
                                            out={"s": lam, "U": U, "V": Q}, stream=stream)["info"])
    ms = timed_device(f_svd, 3, 1, stream, flush)
    r = oracle.tsvd(d, z, al, ks=ks)
    s = lam[kt].cpu().numpy()
    eV = max_err_neps(s, Q[kt].t().cpu().numpy(), {"lam": r["s"], "V": r["V"]}, n)
    eU = max_err_neps(s, U[kt].t().cpu().numpy(), {"lam": r["s"], "V": r["U"]}, n)
    eV["vectors_U"] = eU["vectors"]
    out["svd_n8192"] = {"value": n / (ms / 1e3), "unit": "singular triplets/s", "ms_per_step": ms,
                        "k_eig_ms": info["ms_eig"], "max_err_neps": eV,
                        **kernel_roof(n, args.form, info["ms_eig"])}
    # Hermitian arrowhead (Sec. 6.1), complex U
    d, z, al = W.uniform_herm(n, seed=8)
    dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
    del U
    Uc = torch.empty((n, n), dtype=torch.complex128, device=dev)

    def f_herm():
        info.update(arrowhead.herm_arrow_eig(dt, zt, al, opts=opts, info=True,
                                             out={"lam": lam, "U": Uc}, stream=stream)["info"])
    ms = timed_device(f_herm, 3, 1, stream, flush)
    r = oracle.herm_eig(d, z, al, ks=ks)
    r["V"] = r["U"]
    e = max_err_neps(lam[kt].cpu().numpy(), Uc[kt].t().cpu().numpy(), r, n)
    out["herm_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"], "max_err_neps": e,
                         **kernel_roof(n, args.form, info["ms_eig"], stored=True)}
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
    r = oracle.nsym_eig(d, zc, zr, al, ks=ks)
    r["V"] = r["X"]
    lk = lam[kt].cpu().numpy()
    e = max_err_neps(lk, Q[kt].t().cpu().numpy(), r, n)
    r["V"] = r["Y"]
    e["vectors_Y"] = max_err_neps(lk, Y[kt].t().cpu().numpy(), r, n)["vectors"]
    out["nsym_n8192"] = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "k_eig_ms": info["ms_eig"], "max_err_neps": e,
                         **kernel_roof(n, args.form, info["ms_eig"], stored=True)}
    del Q, Y
    # batched: 4096 instances, orders log-uniform in [32, 4096], one CUDA-graph plan
    inst = W.uniform_batch(4096, seed=2)
    B = arrowhead.Batch(inst, opts=form_opts(arrowhead, args.form), stream=stream)
    ms = timed_device(lambda: B.run(), 2, 1, stream, flush)
    binfo = B.run(info=True)
    tot_n = int(B.n_off[-1])
    tm = batch_terms(B.n)
    # the flop count of an average pass, over the whole plan's time (the plan's
    # other stages are ~13 % of it, so this understates k_batch_eig's rate)
    ncomp = binfo["n_reduced"]
    b_info = dict(binfo)
    fl = eig_kernel_flops(tm + 2, ncomp, b_info["total_iter"], b_info["fix_iter"],
                          b_info["n_ddb"] if FORMS[args.form][2] else None,
                          b_info["total_deriv"],
                          n_mid=b_info["n_mid64"] if FORMS[args.form][0] == 1 else None)
    ins = fp64_instructions(int(round(tm)) + 2, b_info, args.form, terms=tm)
    # the plan's time includes its remedy stage (about a tenth of this set's
    # eigenpairs): count that work too
    rf, ri = remedy_work(b_info, tm)
    fl += rf
    ins += ri
    rb = roofline_numbers(fl, ins, fp32_flops(0, b_info, terms=tm), ms / 1e3, peaks)
    # errors: 24 instances spread over the orders (the largest included), 24
    # sampled eigenpairs each
    order = np.argsort(B.n, kind="stable")
    pick = np.unique(np.concatenate([order[np.linspace(0, len(inst) - 1, 23).astype(int)],
                                     order[-1:]]))
    worst = {"lambda": 0.0, "vectors": 0.0, "bound": ERR_BOUND, "widened": 0, "pairs": 0}
    for i in pick:
        ni = int(B.n[i])
        ksi = sample_ks(ni, 24)
        di, zi, ai = inst[i]
        ri = oracle.arrow_eig(di, zi, ai, ks=ksi)
        ei = max_err_neps(B.lam(i).cpu().numpy()[ksi], B.V(i).cpu().numpy()[:, ksi], ri, ni)
        for k in ("lambda", "vectors"):
            worst[k] = max(worst[k], ei[k])
        worst["widened"] += ei["widened"]
        worst["pairs"] += ei["pairs"]
    out["batched_4096"] = {"value": tot_n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "instances": len(inst), "eigenpairs": tot_n,
                           "sum_n2": int((B.n.astype(np.int64) ** 2).sum()),
                           "fp64_steps_per_eigenpair": binfo["total_iter"] / tot_n,
                           "roofline": {"bound": "alu", "achieved": rb["achieved"],
                                        "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                                        "frac": rb["frac"],
                                        "fp64_pipe_busy_implied": rb["fp64_pipe_busy_implied"],
                                        "mixed": rb["mixed"],
                                        "note": "algorithmic FP64 flops of all eigenpairs "
                                                "and of the remedy solves (average pass "
                                                "length) over the whole plan's time, against "
                                                "the measured FP64 rate"},
                           "remedies": int(binfo["n_dpr1shift"] + binfo["n_nearzero"] +
                                           binfo["n_otherpole"]),
                           "b_double_double": int(binfo["n_ddb"]),
                           "max_err_neps": {**worst, "instances": int(pick.size)},
                           "team_widths": {str(b): arrowhead.lib().ae_team_width(b)
                                           for b in (32, 64, 128, 256, 512)}}
    B.close()
    del B
    torch.cuda.empty_cache()
    rates = [float(x) for x in args.serve_rates.split(",") if x]
    out["serving"] = serve_sweep(arrowhead, W, dev, args.serve_requests, rates,
                                 form_opts(arrowhead, args.form))
    return out


def serve_requests(W, dev, count, seed=5):
    """The request mix of the serving sweep (the same at every rate): kinds
    uniform over arrowhead / DPR1 / SVD, orders log-uniform in [64, 16384]."""
    import torch
    _, kinds, ns = W.serve_stream(1.0, count, seed=seed)
    reqs = []
    for i, (k, n) in enumerate(zip(kinds, ns)):
        if k == 0:
            d, z, a = W.uniform_arrow(int(n), seed=10_000 + i)
        elif k == 1:
            d, z, a = W.uniform_dpr1(int(n), seed=10_000 + i)
        else:
            d, z, a = W.uniform_tsvd(int(n), seed=10_000 + i)
        reqs.append((int(k), torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev), a,
                     (d, z, a)))
    return reqs


def serve_check(arrowhead, srv, tk, kind, host):
    """Sampled error of a served result against the oracle."""
    import oracle
    d, z, a = host
    res = srv.result(tk)
    lam = res["lam"].cpu().numpy()
    n = lam.size
    ks = sample_ks(n, 16)
    if kind == 0:
        r = oracle.arrow_eig(d, z, a, ks=ks)
    elif kind == 1:
        q = oracle.dpr1_eig(d, z, a, ks=ks)
        r = {"lam": q["lam"], "V": q["Q"]}
    else:
        q = oracle.tsvd(d, z, a, ks=ks)
        r = {"lam": q["s"], "V": q["V"]}
    return max_err_neps(lam[ks], res["V"].cpu().numpy()[:, ks], r, n)


def serve_sweep(arrowhead, W, dev, count, rates, opts):
    """Poisson request streams at each offered rate: goodput, rejections, p50 /
    p99 latency of completed requests, eigenpairs/s.  At least `count`
    requests per rate, or 10 s of arrivals at the low rates."""
    res = {}
    reqs = serve_requests(W, dev, count)
    rng = np.random.default_rng(55)
    checked = {"lambda": 0.0, "vectors": 0.0, "bound": ERR_BOUND, "widened": 0, "pairs": 0,
               "requests": 0}
    for ri, rate in enumerate(rates):
        m = int(min(count, max(50, np.ceil(10.0 * rate))))
        t_arr = np.cumsum(rng.exponential(1.0 / rate, m))
        srv = arrowhead.Server(budget_bytes=96 << 30, max_inflight=16, queue_cap=1 << 16,
                               opts=opts)
        t0 = time.perf_counter()
        pending = []
        i = 0
        rejected = 0
        check_left = 6 if ri == 0 else 0
        keep = []
        while i < m or pending:
            now = time.perf_counter() - t0
            while i < m and t_arr[i] <= now:
                k, dt, zt, a, host = reqs[i]
                tk = srv.submit(k, dt, zt, a, vectors=True)
                if tk is None:
                    rejected += 1
                else:
                    pending.append((tk, k, host))
                i += 1
            still = []
            for tk, k, host in pending:
                st, _ = srv.poll(tk)
                if st in (arrowhead.REQ_DONE, arrowhead.REQ_ERROR):
                    if st == arrowhead.REQ_DONE and check_left > 0 and k == check_left % 3:
                        keep.append((tk, k, host))      # checked after the stream
                        check_left -= 1
                    else:
                        srv.release(tk)
                else:
                    still.append((tk, k, host))
            pending = still
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        st = srv.stats()
        for tk, k, host in keep:
            e = serve_check(arrowhead, srv, tk, k, host)
            for key in ("lambda", "vectors"):
                checked[key] = max(checked[key], e[key])
            checked["widened"] += e["widened"]
            checked["pairs"] += e["pairs"]
            checked["requests"] += 1
            srv.release(tk)
        keep.clear()
        srv.close()
        res[f"{int(rate)}/s"] = {"offered_per_s": rate, "requests": m,
                                 "completed": st["completed"], "rejected": rejected,
                                 "failed": st["failed"], "merged": st["merged"],
                                 "goodput_per_s": st["completed"] / wall,
                                 "p50_ms": 1e3 * st["p50_s"], "p99_ms": 1e3 * st["p99_s"],
                                 "eigenpairs_per_s": st["eigenpairs_per_s"],
                                 "wall_s": wall}
    res["mix"] = ("arrow/DPR1/SVD uniform, orders log-uniform [64, 16384], vectors kept on "
                  "device; the same requests at every rate; 16 streams; runs of arrowheads of "
                  "order <= 1024 at the head of the queue merged into batched passes")
    res["max_err_neps"] = checked
    return res


# ---------------------------------------------------------------------------
# the reference arm and the full CPU baselines
# ---------------------------------------------------------------------------
def workload_config(n, form, world):
    """The `config` of both arms' JSON lines (the reference arm times a sample of
    the same workload, said in its cpu_baseline.sample)."""
    return {"workload": f"graded arrowhead n={n}: all eigenpairs + full V",
            "n": n, "form": form, "l2": "512 MiB write between steps (L2 flush)",
            "parallelism": f"{world} independent instances"}


def reference_per_step(threads):
    """Eigenpairs a reference-arm step solves: four per host thread, so that
    every core has work in every step."""
    return 4 * max(1, int(threads))


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    from paper_1302_7203_gb300 import workloads as W
    import oracle
    oracle.build_oracle()
    n = args.n
    d, z, alpha = W.graded_arrow(n, seed=1)
    per_step = reference_per_step(oracle.threads())
    stride = max(1, n // per_step)
    base = np.arange(per_step, dtype=np.int64) * stride
    for s in range(args.warmup):
        oracle.arrow_eig(d, z, alpha, ks=np.unique((base + 7919 * (s + 1)) % n))
    t0 = time.perf_counter()
    done = 0
    for s in range(args.steps):
        ks = np.unique((base + s) % n)
        oracle.arrow_eig(d, z, alpha, ks=ks)
        done += ks.size
    dt = time.perf_counter() - t0
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


def cpu_full(W):
    """The oracle end to end (all eigenpairs and vectors), median of 3, on
    configs 0, 1, 3a and 3b; config 2 on 64 seeded instances, extrapolated
    to the whole set by sum n^2."""
    import oracle
    oracle.build_oracle()
    out = {"cores": oracle.threads()}

    def med3(fn):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts))
    d, z, a = W.uniform_arrow(1000, seed=0)
    t = med3(lambda: oracle.arrow_eig(d, z, a))
    out["config0_uniform_n1000"] = {"s": t, "eigenpairs_per_s": 1000 / t}
    d, z, a = W.graded_arrow(16384, seed=1)
    t = med3(lambda: oracle.arrow_eig(d, z, a))
    out["config1_graded_n16384"] = {"s": t, "eigenpairs_per_s": 16384 / t}
    d, u, rho = W.uniform_dpr1(8192, seed=3)
    t = med3(lambda: oracle.dpr1_eig(d, u, rho))
    out["config3a_dpr1_n8192"] = {"s": t, "eigenpairs_per_s": 8192 / t}
    d, z, a = W.uniform_tsvd(8192, seed=4)
    t = med3(lambda: oracle.tsvd(d, z, a))
    out["config3b_svd_n8192"] = {"s": t, "eigenpairs_per_s": 8192 / t}
    inst = W.uniform_batch(4096, seed=2)
    ns = np.array([len(x[0]) + 1 for x in inst], dtype=np.float64)
    pick = np.random.default_rng(2).choice(len(inst), 64, replace=False)
    t0 = time.perf_counter()
    for i in pick:
        oracle.arrow_eig(*inst[i])
    t = time.perf_counter() - t0
    scale = (ns ** 2).sum() / (ns[pick] ** 2).sum()
    out["config2_batched_4096"] = {"sample_s": t, "sample_instances": 64,
                                   "extrapolated_s": t * scale,
                                   "eigenpairs_per_s": ns.sum() / (t * scale),
                                   "how": "64 seeded instances, scaled by sum n^2"}
    return out


def run_split(args, arrowhead, W, shard, dev, stream, rank, world, local, peaks):
    """--split instance / batch: the strong-scaling divisions of one workload
    across the ranks; prints the JSON line on rank 0."""
    import torch
    import torch.distributed as dist
    n = args.n
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    opts = form_opts(arrowhead, args.form, profile=1)
    if args.split == "instance":
        d, z, alpha = W.graded_arrow(n, seed=1)
        dt, zt = torch.as_tensor(d, device=dev), torch.as_tensor(z, device=dev)
        pos0, cnt = arrowhead.arrow_eig_part_size(dt, zt, rank, world, stream=stream)
        lam = torch.empty(max(cnt, 1), dtype=torch.float64, device=dev)
        V = torch.empty((max(cnt, 1), n), dtype=torch.float64, device=dev)

        def step():
            return arrowhead.arrow_eig_part(dt, zt, alpha, rank, world, opts=opts, info=True,
                                            out={"lam": lam, "V": V}, stream=stream)
        units = n
        launches = LAUNCHES_PER_STEP + 1          # and k_part
        workload = f"graded arrowhead n={n}: all eigenpairs + full V, split by eigenpair ranges"
    else:
        inst = W.uniform_batch(4096, seed=2)
        sizes = np.array([len(x[0]) + 1 for x in inst])
        mine = shard.pack_instances(sizes, world)[rank]
        B = arrowhead.Batch([inst[i] for i in mine], opts=form_opts(arrowhead, args.form),
                            stream=stream)

        def step():
            B.run()
        units = int(sizes.sum())
        # prep, eigenpairs, remedy decisions and solves, placement, vectors, status
        launches = 7
        workload = "4096 uniform arrowheads, orders log-uniform [32, 4096], bin-packed on n^2"
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    tot = 0.0
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            e.record(stream)
            e.synchronize()
            tot += a.elapsed_time(e)
    if world > 1:
        dist.barrier()
        tot = shard.max_over_ranks(tot, device=dev)
    if rank == 0:
        line = {"metric": METRIC, "value": units * args.steps / (tot / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": tot / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload, "n": n, "form": args.form,
                           "split": args.split, "l2": "512 MiB write between steps (L2 flush)",
                           "parallelism": f"{args.split} split over {world} ranks"},
                "e2e": None, "roofline": None, "cpu_baseline": None,
                "peaks_measured": peaks, "clocks": clk.summary(),
                "gpu_launches": launches * args.steps,
                "note": "multi-GPU division; on this pool measured at one GPU only"}
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
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
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    peaks = measure_peaks(arrowhead, local, stream)
    if args.split != "none":
        run_split(args, arrowhead, W, shard, dev, stream, rank, world, local, peaks)
        if world > 1:
            dist.destroy_process_group()
        return
    d, z, alpha = W.graded_arrow(n, seed=shard.rank_seed(1, rank))

    # the oracle sample every form is compared with (timed as the CPU baseline
    # on rank 0 of a one-GPU run)
    cpu = None
    ks = ores = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, ks, ores = cpu_baseline(d, z, alpha, n, args.cpu_seconds)
    elif rank == 0:
        import oracle
        ks = sample_ks(n, args.parity_sample)
        ores = oracle.arrow_eig(d, z, alpha, ks=ks)

    dt = torch.as_tensor(d, device=dev)
    zt = torch.as_tensor(z, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    kt = torch.as_tensor(ks, device=dev) if ks is not None else None

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
        err = None
        if kt is not None:
            err = max_err_neps(lam[kt].cpu().numpy(), V[kt].t().cpu().numpy(), ores, n)
        return total, infos, clk, err

    primary = args.form
    # the other forms first, so lam/V hold the headline form's results at the end
    wanted = [f for f in args.forms.split(",") if f in FORMS]
    runs = {f: timed(f) for f in wanted if f != primary}
    runs[primary] = timed(primary)
    total_ms, infos, clk, err = runs[primary]
    value = world * n * args.steps / (total_ms / 1e3)
    info = infos[-1]
    eig_ms = float(np.mean([x["ms_eig"] for x in infos]))
    stored = info["n_deflated"] == 0          # sorted input: the graded workload is
    ins = fp64_instructions(n, info, primary, stored_diff=stored)
    rl = roofline_numbers(form_flops(n, info, primary), ins, fp32_flops(n, info), eig_ms / 1e3,
                          peaks)
    rl["fp64_instr_per_term"] = ins / (n - 2) / info["n_reduced"]
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
    roof = {"bound": "alu", "achieved": rl["achieved"], "peak": peaks["fp64_tflops"],
            "unit": "TFLOP/s", "frac": rl["frac"], "traffic": traffic,
            "traffic_note": "bytes per k_eig launch: the per-warp stored (delta_j, "
                            "zeta_j^2/delta_j) pairs (written once per eigenpair, re-read "
                            "by each FP64 evaluation), the staged eigenvector column and "
                            "the n x n V written once",
            "kernel": "k_eig", "kernel_ms": eig_ms,
            "fp64_instr_per_term": rl["fp64_instr_per_term"],
            "fp64_pipe_busy_implied": rl["fp64_pipe_busy_implied"],
            "mixed_fp32_fp64": rl["mixed"],
            "fp64_bisection_equivalent_tflops": eq,
            "peak_note": "measured FP64 FMA throughput of this GPU (ae_fma_peaks, of "
                         f"measured); nominal 152 SMs x 4 flop/clk x 2070 MHz = "
                         f"{FP64_NOMINAL_TFLOPS:.3f} TFLOP/s",
            "peaks_measured": peaks}

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

    extra = None
    if world == 1 and not args.no_extras:
        del V
        torch.cuda.empty_cache()
        extra = extras(arrowhead, W, dev, stream, flush, args, peaks)
    if rank == 0 and args.cpu_full:
        extra = dict(extra or {})
        extra["cpu_full"] = cpu_full(W)

    if rank == 0:
        variants = {}
        for form, (tot, inf, _, er) in runs.items():
            fl = form_flops(n, inf[-1], form)
            me = float(np.mean([x["ms_eig"] for x in inf]))
            variants[form] = {
                "value": world * n * args.steps / (tot / 1e3), "ms_per_step": tot / args.steps,
                "ms_eig": me, "frac_fp64": fl / (me / 1e3) / 1e12 / peaks["fp64_tflops"],
                "fp64_steps_per_eigenpair": inf[-1]["total_iter"] / n,
                "fp32_fallbacks": inf[-1]["n_fp32_fallback"],
                "b_double_double": inf[-1]["n_ddb"], "max_err_neps": er}
        errs = [v["max_err_neps"] for v in variants.values()]
        for v in (extra or {}).values():
            if isinstance(v, dict):
                if "max_err_neps" in v:
                    errs.append(v["max_err_neps"])
                for f in v.get("forms", {}).values():
                    errs.append(f.get("max_err_neps"))
        parity_ok = all(err_ok(e) for e in errs)
        if not parity_ok:
            print("bench: a result misses the 10 n eps64 bar against the oracle "
                  "(parity_ok false)", file=sys.stderr, flush=True)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(n, primary, world),
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "max_err_neps": err, "parity_ok": parity_ok,
                "variants": variants, "extras": extra,
                "clocks": clk.summary(), "gpu_launches": LAUNCHES_PER_STEP * args.steps,
                "phases_ms": {k: float(np.mean([x[k] for x in infos]))
                              for k in ("ms_reduce", "ms_eig", "ms_fix", "ms_vectors")},
                "solver": {k: info[k] for k in ("n_nearzero", "n_otherpole", "n_dpr1shift",
                                                "n_capped", "max_iter_used", "total_iter",
                                                "fix_iter", "total_deriv", "n_ddb",
                                                "n_mid64", "n_f32_passes", "n_df_passes",
                                                "max_Kb", "max_Knu")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
