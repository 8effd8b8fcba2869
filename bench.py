"""Benchmark of the MLCC3 triples hot path (one JSON line on rank 0).

A step is one pass of the whole path on one synthetic system: integral
build, triples residual, right and transpose Jacobian transformations of the
state vectors, the three transition densities and the oscillator strength.
The metric is the algorithmic throughput of the step (the paper's leading
flop counts, Sec. 3: Omega 4, rho 8, sigma 8, D^{0-0} 10, D^{m-0} 10,
D^{0-m} 16, in units of N_V n_v^3 n_o^3) divided by the measured step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triples sweep TFLOP/s & s/Davidson-iter vs FP64 GPU path at 1e-6 error in f"
WORKLOADS = {
    # name: (N_O, N_V, n_o, n_v, N_J, states)
    "guanine_like_small": (20, 200, 12, 60, 600, 1),
    "tiny": (6, 24, 4, 8, 72, 1),
    # a small system with the largest workload's active virtual space (n_v = 150:
    # one batch per tensor-core tile), for kernel captures that must stay small
    "betaine_shape_small": (10, 300, 6, 150, 600, 1),
}
# uneven systems of the batched sweep, (n_o, n_v, N_V), N_O = n_o + 8, N_J = 3 N_V
SWEEP_SYSTEMS = [(8, 40, 120), (11, 60, 216), (14, 80, 312), (18, 100, 408), (21, 120, 504),
                 (24, 140, 600)]
# Leading FLOP counts per state in units of N_V n_v^3 n_o^3 (Sec. 3); D^{0-0} is
# D^{m-0} with the multipliers in place of L (same count)
FLOP_UNITS = {"omega": 4, "rho": 8, "sigma": 8, "D_m0": 10, "D_00": 10, "D_0m": 16}
UNITS_PER_STEP = sum(FLOP_UNITS.values())      # per state
FP64_PEAK_TFLOPS = 1.25                        # nominal GB300 FP64 (ALU bound)


def algorithmic_flops(NO, NV, no, nv, nstates):
    return UNITS_PER_STEP * NV * nv ** 3 * no ** 3 * nstates


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "memory.used")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.first = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # sampling is running before the timed region starts; the rows that
            # arrive from here on fall inside it
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.rows)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = self.rows[self.first:]
        out = {}
        if not rows:  # a timed region shorter than one sampling interval
            rows = self.rows[-1:]
            out["note"] = "no sample inside the timed region; the last one before it"
        sm = [float(r[0]) for r in rows if r[0].replace('.', '', 1).isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace('.', '', 1).isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v == "Active"})
        mem = [float(r[8]) for r in rows if len(r) > 8 and r[8].replace('.', '', 1).isdigit()]
        out.update({"sm_mhz": statistics.median(sm) if sm else None,
                    "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                    "samples": len(self.rows) - self.first})
        if mem:
            out["memory_used_mib_max"] = max(mem)
        return out


# the sources that fix the tensor-core kernel and its launch plans (the DRAM
# traffic figure in profiles/traffic.json is valid while these are unchanged)
TC_SOURCES = ("kernels_tc.cu", "kernels_tc.cuh", "tc_host.cu", "mlcc3_capi.cu", "engine.cuh")


def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2202_08612_gb300", "csrc")
    for fn in TC_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel sources changed since it was captured."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t[kernel]
        return e["bytes_per_launch"] if e.get("source_digest") == source_digest() else None
    except Exception:
        return None


# --------------------------------------------------------------------------------------
def oracle_sample(workload, seed):
    """The oracle on a bounded sample of the workload: the same system with the
    active occupied space cut to n_o = 4 (every stage of the step)."""
    import oracle as O
    from paper_2202_08612_gb300 import synth
    NO, NV, no, nv, NJ, ns = WORKLOADS[workload]
    no_s = min(no, 4)
    s = synth.make_system(NO, NV, no_s, nv, NJ, seed=seed)
    st = synth.make_states(s, 1, seed=seed + 1)
    lam1, lam2 = synth.make_multipliers(s, seed=seed + 2)
    mu = synth.make_dipole(s, seed=seed + 3)
    D00_in = synth.reference_density(s)
    t = time.perf_counter()
    oc = O.make_ctx(s)
    O.triples_omega(oc)
    w = float(st.omega[0])
    O.jacobian_right(oc, w, st.R1[0], O.to_full(oc, st.R2[0]))
    O.jacobian_left(oc, w, st.L1[0], O.to_full(oc, st.L2[0]))
    d00, dm0, d0m = O.transition_densities(oc, w, lam1, O.to_full(oc, lam2), st.R1[0],
                                           O.to_full(oc, st.R2[0]), st.L1[0],
                                           O.to_full(oc, st.L2[0]), D00_in)
    O.oscillator_strength(oc, w, d0m, dm0, mu)
    dt = time.perf_counter() - t
    fl = algorithmic_flops(NO, NV, no_s, nv, 1)
    return fl / dt / 1e12, dt, f"same system with n_o cut to {no_s} (all stages of one step)"


def run_reference(args, rank):
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"the oracle sample is defined for {sorted(WORKLOADS)} only"}), flush=True)
        return
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, sample = oracle_sample(args.workload, 1000 + i)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    NO, NV, no, nv, NJ, ns = WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.workload)},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name(w):
    NO, NV, no, nv, NJ, ns = WORKLOADS[w]
    return f"{w}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}, {ns} state(s)"


# --------------------------------------------------------------------------------------
class Problem:
    def __init__(self, workload, seed, device):
        import torch
        from paper_2202_08612_gb300 import synth
        NO, NV, no, nv, NJ, ns = WORKLOADS[workload]
        self.dims = (NO, NV, no, nv, NJ)
        self.ns = ns
        s = synth.make_system(NO, NV, no, nv, NJ, seed=seed)
        st = synth.make_states(s, ns, seed=seed + 1)
        lam1, lam2 = synth.make_multipliers(s, seed=seed + 2)
        self.host = dict(chol=s.chol, t1=s.t1, eps=s.eps, t2c=s.t2c, t2x=s.t2x, R1=st.R1, R2=st.R2,
                         L1=st.L1, L2=st.L2, lam1=lam1, lam2=lam2, mu=synth.make_dipole(s, seed=seed + 3),
                         D00_in=synth.reference_density(s))
        self.host = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in self.host.items()}
        self.omega = st.omega
        self.dev = {k: torch.from_numpy(v).to(device) for k, v in self.host.items()}
        nmo = NO + NV
        z = lambda shape: torch.zeros(shape, dtype=torch.float64, device=device)
        self.out_dev = dict(o1=z((NV, NO)), o2=z(s.t2c.shape), rho1=z(st.R1.shape), rho2=z(st.R2.shape),
                            sig1=z(st.R1.shape), sig2=z(st.R2.shape), D00=z((nmo, nmo)),
                            Dm0=z((nmo, nmo)), D0m=z((nmo, nmo)))
        self.out_host = {k: np.zeros(tuple(v.shape)) for k, v in self.out_dev.items()}

    def step(self, ctx, x, o):
        """One pass of the whole path; x/o are device tensors or host arrays."""
        ctx.build_integrals(x["chol"], x["t1"], x["eps"], x["t2c"], x["t2x"])
        ctx.triples_omega(o["o1"], o["o2"])
        ctx.jacobian_right(self.omega, x["R1"], x["R2"], o["rho1"], o["rho2"])
        ctx.jacobian_left(self.omega, x["L1"], x["L2"], o["sig1"], o["sig2"])
        fs = []
        for n in range(self.ns):
            w = float(self.omega[n])
            ctx.transition_density(w, x["lam1"], x["lam2"], x["R1"][n], x["R2"][n], x["L1"][n],
                                   x["L2"][n], x["D00_in"], o["D00"], o["Dm0"], o["D0m"])
            fs.append(ctx.oscillator_strength(w, o["D0m"], o["Dm0"], x["mu"]))
        return fs

    def sd_model_part(self, n):
        """<L, D R> of state n with D the orbital-energy differences (the model of the
        singles-doubles Jacobian block that the Rayleigh quotient is given)."""
        from paper_2202_08612_gb300 import synth
        NO, NV, no, nv, NJ = self.dims
        e = self.host["eps"]
        eo, ev = e[:NO], e[NO:]
        d1 = ev[:, None] - eo[None, :]
        d2 = (ev[None, :nv, None, None] + ev[None, None, None, :] - eo[:no, None, None, None]
              - eo[None, None, :, None])
        dims = synth.Dims(NO, NV, no, nv, NJ)
        h = self.host
        return synth.sd_dot(dims, h["L1"][n], h["L2"][n], d1 * h["R1"][n], d2 * h["R2"][n])

    def bytes_io(self):
        i = sum(v.nbytes for v in self.host.values()) + 8 * self.ns
        o = sum(v.nbytes for v in self.out_host.values()) + 8 * self.ns
        return i, o


def job_throughput(ms_local, steps, flops_per_rank_step, world, device=None):
    """Whole-job timing of a weak-scaling run: every rank processed its own
    system for `steps` steps in ms_local milliseconds; the job's time is the
    slowest rank's (an all-reduce MAX when a process group is up, on `device`)
    and its throughput counts the work of all ranks.  Returns (ms per step,
    TFLOP/s)."""
    import torch
    ms_total = ms_local
    if device is not None:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms = ms_total / steps
    return ms, flops_per_rank_step * world / (ms * 1e-3) / 1e12


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2202_08612_gb300 import binding, build
    build.build()
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    NO, NV, no, nv, NJ, ns = WORKLOADS[args.workload]
    prob = Problem(args.workload, 2022 + 17 * rank, device)
    stream = torch.cuda.current_stream(device)
    split = args.precision == "split"
    prec = binding.MLCC3_SPLIT_BF16X3 if split else binding.MLCC3_FP64
    ctx = binding.Context(*prob.dims, precision=prec, stream=stream.cuda_stream)
    apply_params(ctx, args)
    if args.tc_group:
        ctx.set_param("tc_group", args.tc_group)
    if args.tc_wide_bn:
        ctx.set_param("tc_wide_bn", args.tc_wide_bn)
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize(device)

    f_ours = None
    for _ in range(args.warmup):
        f_ours = prob.step(ctx, prob.dev, prob.out_dev)
    ctx.profile(True)
    with ClockSampler(local_rank) as clk:
        barrier()  # every rank's clock sampling is running before any rank starts
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            prob.step(ctx, prob.dev, prob.out_dev)
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    stats = ctx.kernel_stats()
    ctx.profile(False)
    fl = algorithmic_flops(NO, NV, no, nv, ns)
    ms, value = job_throughput(ms_total, args.steps, fl, world, device if dist else None)

    # per-stage time of the Davidson-iteration part (rho + sigma of the state vectors)
    barrier()
    t = time.perf_counter()
    ctx.jacobian_right(prob.omega, prob.dev["R1"], prob.dev["R2"], prob.out_dev["rho1"], prob.out_dev["rho2"])
    ctx.jacobian_left(prob.omega, prob.dev["L1"], prob.dev["L2"], prob.out_dev["sig1"], prob.out_dev["sig2"])
    torch.cuda.synchronize(device)
    s_iter = time.perf_counter() - t

    # end to end through the C ABI with host buffers (staged by the library)
    barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        prob.step(ctx, prob.host, prob.out_host)
    torch.cuda.synchronize(device)
    e2e_s = (time.perf_counter() - t) / args.steps
    bi, bo = prob.bytes_io()
    e2e = {"value": fl * world / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": bo}

    # dominant kernel of the timed region (call-site tags "name:site" aggregated by name)
    agg = {}
    for k, (nl, kms_, kfl_) in stats.items():
        base = k.split(":")[0]
        a = agg.setdefault(base, [0, 0.0, 0.0])
        a[0] += nl
        a[1] += kms_
        a[2] += kfl_
    dom = max(agg.items(), key=lambda kv: kv[1][1])
    name, (launches, kms, kfl) = dom
    alg = kfl / (kms * 1e-3) / 1e12 if kms > 0 else None
    if name.startswith("tc_gemm"):
        pk = peaks().get("bf16_tflops_sustained") or 1700.0
        achieved = 3.0 * alg if alg else None  # three BF16 products per algorithmic product
        roofline = {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": pk,
                    "unit": "TFLOP/s", "frac": achieved / pk if achieved else None,
                    "traffic": traffic_for(name), "achieved_algorithmic": alg,
                    "launches_per_step": launches / args.steps, "share_of_step": kms / ms_total,
                    "peak_note": "measured sustained dense BF16 (MEASURED_PEAKS.json); achieved "
                                 "counts the 3 BF16 products (hi*hi, hi*lo, lo*hi) per product"}
    else:
        roofline = {"kernel": name, "bound": "alu", "achieved": alg, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": alg / FP64_PEAK_TFLOPS if alg else None,
                    "traffic": traffic_for(name), "launches_per_step": launches / args.steps,
                    "share_of_step": kms / ms_total,
                    "peak_note": "nominal GB300 FP64 (FP64 FMA on the SIMT pipes)"}
    gpu_launches = sum(v[0] for v in stats.values())

    # the plain FP64 GPU path on the same system: its throughput and f
    fp64 = None
    if split and not args.no_fp64_compare:
        ctx64 = binding.Context(*prob.dims, precision=binding.MLCC3_FP64, stream=stream.cuda_stream)
        out64 = {k: torch.zeros_like(v) for k, v in prob.out_dev.items()}
        f64 = prob.step(ctx64, prob.dev, out64)
        barrier()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        f64 = prob.step(ctx64, prob.dev, out64)
        e3.record(stream)
        barrier()
        ms64 = e2.elapsed_time(e3)
        # excitation-energy Rayleigh quotient of state 0 in both precisions, with
        # the orbital-energy-difference model of the singles-doubles block
        sd = prob.sd_model_part(0)
        x = prob.dev
        rq = [cx.rayleigh_quotient(float(prob.omega[0]), x["R1"][0], x["R2"][0], x["L1"][0],
                                   x["L2"][0], sd) for cx in (ctx, ctx64)]
        fp64 = {"value": fl / (ms64 * 1e-3) / 1e12, "ms_per_step": ms64,
                "speedup_of_split": ms64 / ms,
                "f_abs_diff": max(abs(a - b) for a, b in zip(f_ours, f64)),
                "f_fp64": f64,
                "omega_rq": {"split": rq[0], "fp64": rq[1], "abs_diff_hartree": abs(rq[0] - rq[1])}}
        ctx64.close()

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu_v, cpu_dt, sample = oracle_sample(args.workload, 77)
            cpu = {"value": cpu_v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": sample, "seconds": cpu_dt}
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16x3" if split else "f64",
                "data": "synthetic",
                "config": {"workload": workload_name(args.workload),
                           "precision": "split bf16x3 / fp32 accumulate / fp64 denominators and reductions"
                           if split else "fp64",
                           "parallelism": f"replicas x{world} (independent systems)",
                           "l2": "inputs larger than L2 (Cholesky vectors "
                                 f"{prob.host['chol'].nbytes / 2**20:.0f} MiB)"},
                "s_per_davidson_iter": s_iter,
                "fp64_gpu_path": fp64, "f": f_ours,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": e2e, "clocks": clk.summary(), "gpu_launches": gpu_launches,
                "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in agg.items()},
                "call_sites": {k: round(v[1] / args.steps, 3) for k, v in
                               sorted(stats.items(), key=lambda kv: -kv[1][1])[:24]},
                "tc_sites": tc_site_fracs(stats, args.steps,
                                          peaks().get("bf16_tflops_sustained") or 1700.0)}
        print(json.dumps(line), flush=True)
    ctx.close()


def run_sweep(args):
    """Batched sweep: right transformations of --vectors trial vectors on each of
    the six uneven systems, one captured graph per sweep (mlcc3_sweep_*), timed
    against the same transformations issued eagerly, system after system."""
    import torch
    from paper_2202_08612_gb300 import binding, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = binding.MLCC3_SPLIT_BF16X3 if args.precision == "split" else binding.MLCC3_FP64
    ctxs, vecs, omegas, flops = [], [], [], 0.0
    for q, (no, nv, NV) in enumerate(SWEEP_SYSTEMS):
        NO, NJ = no + 8, 3 * NV
        sysq = synth.make_system(NO, NV, no, nv, NJ, seed=2022 + q)
        st = synth.make_states(sysq, args.vectors, seed=3022 + q)
        d = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        c = binding.Context(NO, NV, no, nv, NJ, precision=prec)
        c.build_integrals(d(sysq.chol), d(sysq.t1), d(sysq.eps), d(sysq.t2c), d(sysq.t2x))
        R1, R2 = d(st.R1), d(st.R2)
        rho1, rho2 = torch.zeros_like(R1), torch.zeros_like(R2)
        ctxs.append(c)
        vecs.append((R1, R2, rho1, rho2))
        omegas.append(st.omega)
        flops += 8.0 * NV * nv ** 3 * no ** 3 * args.vectors
        del sysq, st
    sw = binding.Sweep(ctxs, tune=True)
    for q, v in enumerate(vecs):
        sw.set_system(q, *v)
    w = np.concatenate(omegas)
    stream = torch.cuda.current_stream(dev)

    def timed(f, n):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n):
            f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / n

    for _ in range(args.warmup):
        sw.run(w)
    with ClockSampler(0) as clk:
        t_graph = timed(lambda: sw.run(w), args.steps)

    def eager():
        for c, (R1, R2, rho1, rho2), om in zip(ctxs, vecs, omegas):
            c.jacobian_right(om, R1, R2, rho1, rho2)
    eager()
    t_eager = timed(eager, max(1, args.steps // 2))
    info = sw.info()
    del stream
    line = {"metric": METRIC, "value": flops / t_graph / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_graph * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if args.precision == "split" else "f64", "data": "synthetic",
            "config": {"workload": "uneven_sweep: 6 systems (n_o,n_v,N_V) " +
                       " ".join(f"({a},{b},{c})" for a, b, c in SWEEP_SYSTEMS) +
                       f", N_O = n_o + 8, N_J = 3 N_V, {args.vectors} trial vectors each",
                       "precision": args.precision},
            "s_per_davidson_iter": t_graph, "eager": {"ms": t_eager * 1e3,
                                                      "tflops": flops / t_eager / 1e12,
                                                      "graph_speedup": t_eager / t_graph},
            "graph": info, "clocks": clk.summary(), "algorithmic_flop_per_sweep": flops}
    print(json.dumps(line), flush=True)
    sw.close()
    for c in ctxs:
        c.close()


# large systems: measured component by component (integral build, Omega, one
# Davidson iteration = rho and sigma of every trial vector, densities of one state)
# name: (N_O, N_V, n_o, n_v, N_J, valence trial vectors)
LARGE = {
    "guanine_like": (40, 500, 20, 120, 1500, 4),
    "betaine_like": (100, 1000, 20, 150, 4000, 2),
}


def device_system(NO, NV, no, nv, NJ, nvec, seed, dev, core, t2_norm=None, cvs_last=0):
    """Seeded synthetic inputs of the large workloads, drawn on the device
    (torch Philox): the distributions of paper_2202_08612_gb300.synth, without
    the host-side generation of a 10-40 GB Cholesky tensor.  t2_norm: the
    molecule-scaled variant (Cholesky scale lowered so that the active doubles
    block has norm at most t2_norm).  cvs_last: the last cvs_last vectors are
    core states (elements without the core orbital 0 removed, omega 10.2 Ha)."""
    import torch
    g = torch.Generator(device=dev).manual_seed(seed)
    f64 = torch.float64
    U = lambda lo, hi, n: lo + (hi - lo) * torch.rand(n, dtype=f64, device=dev, generator=g)
    N = lambda *shape: torch.randn(*shape, dtype=f64, device=dev, generator=g)
    nmo = NO + NV
    eps = torch.cat([U(-1.5, -0.3, NO), U(0.1, 3.0, NV)])
    if core:
        eps[0] = -10.0
    chol = torch.empty((NJ, nmo, nmo), dtype=f64, device=dev)
    for j0 in range(0, NJ, 128):
        b = N(min(128, NJ - j0), nmo, nmo) * 0.05
        chol[j0:j0 + b.shape[0]] = (b + b.transpose(1, 2)) * (0.5 ** 0.5)
        del b
    t1 = N(NV, NO) * 0.01
    Lvo = chol[:, NO:, :NO]                                   # [J][A][I]
    den = (eps[:no, None, None, None] + eps[None, None, :NO, None]
           - eps[NO:NO + nv][None, :, None, None] - eps[NO:][None, None, None, :])
    A = Lvo[:, :nv, :no].permute(2, 1, 0).reshape(no * nv, NJ)
    B = Lvo.permute(0, 2, 1).reshape(NJ, NO * NV)
    t2c = (A @ B).reshape(no, nv, NO, NV) / den               # t^{aD}_{iL} = (ai|DL)/D
    del A, B
    A = Lvo[:, :nv, :].permute(1, 2, 0).reshape(nv * NO, NJ)  # [a][L][J]
    B = Lvo[:, :, :no].reshape(NJ, NV * no)                   # [J][D][i]
    t2x = (A @ B).reshape(nv, NO, NV, no).permute(3, 0, 1, 2).contiguous() / den  # t^{aD}_{Li}
    del A, B, Lvo
    if t2_norm is not None:
        nrm = float(t2c.pow(2).sum().sqrt())
        if nrm > t2_norm:  # amplitudes are quadratic in the Cholesky scale
            f = t2_norm / nrm
            chol *= f ** 0.5
            t2c *= f
            t2x *= f
    R1 = N(nvec, NV, NO)
    R2 = N(nvec, no, nv, NO, NV)
    aa = R2[:, :, :, :no, :nv]
    R2[:, :, :, :no, :nv] = 0.5 * (aa + aa.permute(0, 3, 4, 1, 2))
    for n in range(nvec):
        R1[n] *= (0.95 / R1[n].pow(2).sum()).sqrt()
        R2[n] *= (0.05 / R2[n].pow(2).sum()).sqrt()
    L1 = R1 + 0.3 * N(*R1.shape) * R1.abs().mean()
    L2 = R2 + 0.3 * N(*R2.shape) * R2.abs().mean()
    aa = L2[:, :, :, :no, :nv]
    L2[:, :, :, :no, :nv] = 0.5 * (aa + aa.permute(0, 3, 4, 1, 2))
    omega = (0.3 + 0.3 * torch.rand(nvec, dtype=f64, generator=torch.Generator().manual_seed(seed))).numpy()
    for n in range(nvec - cvs_last, nvec):
        # a core state: only elements that carry the core occupied orbital 0
        for X1, X2 in ((R1, R2), (L1, L2)):
            X1[n][:, 1:] = 0.0
            keep = torch.zeros_like(X2[n], dtype=torch.bool)
            keep[0] = True
            keep[:, :, 0] = True
            X2[n] *= keep
        omega[n] = 10.2
    mu = N(3, nmo, nmo) * 0.1
    mu = 0.5 * (mu + mu.transpose(1, 2))
    D00 = torch.zeros((nmo, nmo), dtype=f64, device=dev)
    D00[range(NO), range(NO)] = 2.0
    return dict(chol=chol, t1=t1, eps=eps, t2c=t2c, t2x=t2x, R1=R1, R2=R2, L1=L1, L2=L2,
                lam1=N(NV, NO) * 0.01, lam2=t2c, mu=mu, D00_in=D00), omega


def run_large(args):
    """Large guanine- or betaine-shaped system in the split precision.  Stage
    "davidson": integral build, Omega, then --steps timed Davidson iterations
    (rho and sigma of all valence trial vectors in one call each, after --warmup
    untimed ones); the roofline line is the tensor-core kernel's share of them.
    Stage "densities": integral build, then the three transition densities and f
    of one state (run_large_densities)."""
    import torch
    from paper_2202_08612_gb300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    NO, NV, no, nv, NJ, nvec = LARGE[args.workload]
    core = args.workload == "betaine_like"
    if args.stage in ("densities", "cvs", "ground"):
        nvec = 1
    x, omega = device_system(NO, NV, no, nv, NJ, nvec, 2022, dev, core)
    cvs = args.stage == "cvs"
    core_mask = None
    if cvs:
        if not core:
            raise SystemExit("the cvs stage needs the core orbital of the betaine_like workload")
        # core-valence separation: the state's vectors keep the elements that carry
        # the core occupied orbital 0, at omega 10.2 Ha (below the core batches'
        # smallest denominator)
        core_mask = np.zeros(NO, dtype=np.uint8)
        core_mask[0] = 1
        for k in ("R", "L"):
            x[k + "1"][:, :, 1:] = 0.0
            keep = torch.zeros_like(x[k + "2"][0], dtype=torch.bool)
            keep[0] = True
            keep[:, :, 0] = True
            x[k + "2"] *= keep
        omega = np.array([10.2])
    stream = torch.cuda.current_stream(dev)
    prec = binding.MLCC3_SPLIT_BF16X3 if args.precision == "split" else binding.MLCC3_FP64
    z = lambda t: torch.zeros_like(t)
    # every output exists before the context sizes its chunks from the free memory
    o1, o2 = z(x["R1"][0]), z(x["t2c"])
    rho1, rho2, sig1, sig2 = z(x["R1"]), z(x["R2"]), z(x["R1"]), z(x["R2"])
    nmo = NO + NV
    D = [torch.zeros((nmo, nmo), dtype=torch.float64, device=dev) for _ in range(3)]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ctx = binding.Context(NO, NV, no, nv, NJ, precision=prec, stream=stream.cuda_stream,
                          core_mask=core_mask)
    # unique batches held per chunk: leaves room for the integral blocks, their
    # split copies and the per-call scratch next to the caller's tensors
    apply_params(ctx, args)
    if args.stage not in ("densities", "ground"):
        ctx.set_param("chunk_blocks", args.chunk_blocks)
    if args.tc_group:
        ctx.set_param("tc_group", args.tc_group)
    if args.tc_wide_bn:
        ctx.set_param("tc_wide_bn", args.tc_wide_bn)
    unit = NV * nv ** 3 * no ** 3

    def timed(f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        f()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ms_build = timed(lambda: ctx.build_integrals(x["chol"], x["t1"], x["eps"], x["t2c"], x["t2x"]))
    del x["chol"]  # the context keeps its own T1-transformed copy
    torch.cuda.empty_cache()
    if args.stage == "densities":
        return run_large_densities(args, ctx, x, omega, D, unit, ms_build, NO, NV, no, nv, NJ,
                                   core, prec == binding.MLCC3_SPLIT_BF16X3)
    if args.stage == "ground":
        return run_large_ground(args, ctx, x, D, unit, ms_build, NO, NV, no, nv, NJ, core,
                                prec == binding.MLCC3_SPLIT_BF16X3, rho1, rho2)
    ms_omega_first = timed(lambda: ctx.triples_omega(o1, o2))
    ms_omega = timed(lambda: ctx.triples_omega(o1, o2))

    def davidson():
        ctx.jacobian_right(omega, x["R1"], x["R2"], rho1, rho2)
        ctx.jacobian_left(omega, x["L1"], x["L2"], sig1, sig2)

    for _ in range(args.warmup):
        davidson()
    ctx.profile(True)
    with ClockSampler(0) as clk:
        ms_it = timed(lambda: [davidson() for _ in range(args.steps)]) / args.steps
    stats = ctx.kernel_stats()
    ctx.profile(False)
    tc = [v for k, v in stats.items() if k.startswith("tc_gemm")]
    tc_ms = sum(v[1] for v in tc) / args.steps
    tc_fl = sum(v[2] for v in tc) / args.steps
    pk = peaks().get("bf16_tflops_sustained") or 1700.0
    alg = tc_fl / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    # CVS: only the triples that carry the core index (n_o^3 - (n_o - 1)^3 of the n_o^3
    # ordered ones) contribute
    rs = float(FLOP_UNITS["rho"] + FLOP_UNITS["sigma"])
    fl_it = rs * NV * nv ** 3 * (no ** 3 - (no - 1) ** 3) * nvec if cvs else rs * unit * nvec
    line = {"metric": METRIC, "value": fl_it / (ms_it * 1e-3) / 1e12, "unit": "TFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_it,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if prec == binding.MLCC3_SPLIT_BF16X3 else "f64",
            "data": "synthetic (device-generated, torch Philox)",
            "config": {"workload": f"{args.workload}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}, "
                                   + ("1 core (CVS) trial vector at omega 10.2 Ha" if cvs else
                                      f"{nvec} valence trial vectors")
                                   + (", core orbital at -10 Ha" if core else ""),
                       "step": "one Davidson iteration: rho and sigma of all trial vectors",
                       "flop_units": "16 N_V n_v^3 (n_o^3 - (n_o-1)^3) (CVS)" if cvs else "16 N_V n_v^3 n_o^3 per vector",
                       "chunk_blocks": args.chunk_blocks,
                       "precision": args.precision},
            "s_per_davidson_iter": ms_it * 1e-3,
            "build_integrals_ms": ms_build,
            "omega": {"ms": ms_omega, "ms_first_call": ms_omega_first,
                      "tflops": FLOP_UNITS["omega"] * unit / (ms_omega * 1e-3) / 1e12},
            "roofline": {"kernel": "tc_gemm_kernel", "bound": "tensor",
                         "achieved": 3.0 * alg if alg else None, "peak": pk, "unit": "TFLOP/s",
                         "frac": 3.0 * alg / pk if alg else None, "achieved_algorithmic": alg,
                         "share_of_step": tc_ms / ms_it,
                         "peak_note": "measured sustained dense BF16 (MEASURED_PEAKS.json); achieved "
                                      "counts the 3 BF16 products per product"},
            "clocks": clk.summary(),
            "hbm_used_gb": (lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info(dev)),
            "call_sites": {k: round(v[1] / args.steps, 3) for k, v in
                           sorted(stats.items(), key=lambda kv: -kv[1][1])[:16]},
            "tc_sites": tc_site_fracs(stats, args.steps, pk)}
    print(json.dumps(line), flush=True)
    ctx.close()


def tc_site_fracs(stats, steps, pk):
    """ms per step and fraction of the BF16 peak (3 products per product) of each
    tensor-core call site."""
    return {k.split(":", 1)[1]: {"ms": round(v[1] / steps, 3),
                                 "frac": round(3.0 * v[2] / (v[1] * 1e-3) / 1e12 / pk, 4) if v[1] > 0 else None}
            for k, v in stats.items() if k.startswith("tc_gemm_kernel:")}


def run_nv_scaling(args):
    """The ρ and σ of one trial vector at fixed active space (N_O=20, n_o=12,
    n_v=60, N_J=600) for N_V = 200, 400, 800: the time is affine in N_V (the
    d-terms scale with N_V, the l-terms, conversions and denominators do not)."""
    import torch
    from paper_2202_08612_gb300 import binding, build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    NO, no, nv, NJ = 20, 12, 60, 600
    pts = []
    for NV in (200, 400, 800):
        x, omega = device_system(NO, NV, no, nv, NJ, 1, 2022, dev, False)
        out = [torch.zeros_like(x[k]) for k in ("R1", "R2", "R1", "R2")]
        ctx = binding.Context(NO, NV, no, nv, NJ, precision=binding.MLCC3_SPLIT_BF16X3,
                              stream=stream.cuda_stream)
        ctx.build_integrals(x["chol"], x["t1"], x["eps"], x["t2c"], x["t2x"])

        def it():
            ctx.jacobian_right(omega, x["R1"], x["R2"], out[0], out[1])
            ctx.jacobian_left(omega, x["L1"], x["L2"], out[2], out[3])
        for _ in range(args.warmup):
            it()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            it()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        rs = FLOP_UNITS["rho"] + FLOP_UNITS["sigma"]
        pts.append({"N_V": NV, "ms": ms, "tflops": rs * NV * nv ** 3 * no ** 3 / (ms * 1e-3) / 1e12})
        ctx.close()
        del x, out
        torch.cuda.empty_cache()
    nvs = np.array([p["N_V"] for p in pts], dtype=float)
    ms = np.array([p["ms"] for p in pts])
    slope, icpt = np.polyfit(nvs, ms, 1)
    resid = float(np.max(np.abs(ms - (slope * nvs + icpt)) / ms))
    print(json.dumps({"metric": METRIC, "value": pts[-1]["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": pts[-1]["ms"],
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "bf16x3", "data": "synthetic (device-generated, torch Philox)",
                      "config": {"workload": "nv_scaling: N_O=20 n_o=12 n_v=60 N_J=600, N_V = 200, 400, "
                                             "800, one trial vector (value: the N_V = 800 point)"},
                      "points": pts, "fit_ms": {"per_N_V": slope, "intercept": icpt,
                                                "max_rel_residual": resid}}), flush=True)


def run_large_ground(args, ctx, x, D, unit, ms_build, NO, NV, no, nv, NJ, core, split, eta1, eta2):
    """The ground-state stages of a large system (the paper's lambda and D^{0-0}
    rows): the multipliers' triples transformation (lambda^T A at omega = 0,
    counted as sigma, 8 N_V n_v^3 n_o^3) and the ground-state density D^{0-0}
    alone (10 N_V n_v^3 n_o^3), each timed after one untimed call."""
    import torch
    dev = x["R1"].device
    stream = torch.cuda.current_stream(dev)
    lam1, lam2 = x["lam1"], x["lam2"]
    e1, e2 = eta1[0], eta2[0]

    def timed(f):
        e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        f()
        e1_.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1_)
    ctx.multiplier_transformation(lam1, lam2, e1, e2)
    ctx.ground_density(lam1, lam2, D[0])
    ctx.profile(True)
    with ClockSampler(0) as clk:
        ms_lam = statistics.median(timed(lambda: ctx.multiplier_transformation(lam1, lam2, e1, e2))
                                   for _ in range(max(1, args.steps)))
        ms_d00 = statistics.median(timed(lambda: ctx.ground_density(lam1, lam2, D[0]))
                                   for _ in range(max(1, args.steps)))
    stats = ctx.kernel_stats()
    ctx.profile(False)
    pk = peaks().get("bf16_tflops_sustained") or 1700.0
    tc = [v for k, v in stats.items() if k.startswith("tc_gemm")]
    tc_ms, tc_fl = sum(v[1] for v in tc), sum(v[2] for v in tc)
    alg = tc_fl / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    fl_lam, fl_d00 = FLOP_UNITS["sigma"] * unit, FLOP_UNITS["D_00"] * unit
    line = {"metric": METRIC, "value": (fl_lam + fl_d00) / ((ms_lam + ms_d00) * 1e-3) / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": ms_lam + ms_d00, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3" if split else "f64",
            "data": "synthetic (device-generated, torch Philox)",
            "config": {"workload": f"{args.workload}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}"
                                   + (", core orbital at -10 Ha" if core else ""),
                       "step": "multiplier transformation (lambda^T A at omega = 0) + D^{0-0}",
                       "flop_units": "8 + 10 N_V n_v^3 n_o^3"},
            "lambda": {"ms": ms_lam, "tflops": fl_lam / (ms_lam * 1e-3) / 1e12},
            "D00": {"ms": ms_d00, "tflops": fl_d00 / (ms_d00 * 1e-3) / 1e12},
            "build_integrals_ms": ms_build,
            "roofline": {"kernel": "tc_gemm_kernel", "bound": "tensor",
                         "achieved": 3.0 * alg if alg else None, "peak": pk, "unit": "TFLOP/s",
                         "frac": 3.0 * alg / pk if alg else None, "achieved_algorithmic": alg,
                         "share_of_step": tc_ms / (max(1, args.steps) * (ms_lam + ms_d00))},
            "clocks": clk.summary(),
            "call_sites": {k: round(v[1] / max(1, args.steps), 3) for k, v in
                           sorted(stats.items(), key=lambda kv: -kv[1][1])[:16]},
            "tc_sites": tc_site_fracs(stats, max(1, args.steps), pk)}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_large_densities(args, ctx, x, omega, D, unit, ms_build, NO, NV, no, nv, NJ, core, split):
    """The three transition densities and f of one state of a large system, in a
    process of their own: the densities hold every batch that touches a range of
    occupied indices (at 100/1000/20/150 about 300 blocks of n_v^3 per array)."""
    import torch
    w = float(omega[0])
    f = []
    dev = x["R1"].device
    stream = torch.cuda.current_stream(dev)

    def run():
        ctx.transition_density(w, x["lam1"], x["lam2"], x["R1"][0], x["R2"][0], x["L1"][0],
                               x["L2"][0], x["D00_in"], *D)
        f.append(ctx.oscillator_strength(w, D[2], D[1], x["mu"]))

    ctx.profile(True)
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    stats = ctx.kernel_stats()
    ctx.profile(False)
    tc = [v for k, v in stats.items() if k.startswith("tc_gemm")]
    tc_ms, tc_fl = sum(v[1] for v in tc), sum(v[2] for v in tc)
    pk = peaks().get("bf16_tflops_sustained") or 1700.0
    alg = tc_fl / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    dens = float(FLOP_UNITS["D_m0"] + FLOP_UNITS["D_00"] + FLOP_UNITS["D_0m"])
    line = {"metric": METRIC, "value": dens * unit / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3" if split else "f64", "data": "synthetic (device-generated, torch Philox)",
            "config": {"workload": f"{args.workload}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}, one state"
                                   + (", core orbital at -10 Ha" if core else ""),
                       "step": "D^{0-0}, D^{m-0}, D^{0-m} and f of one state (first call)",
                       "flop_units": "(10 + 10 + 16) N_V n_v^3 n_o^3"},
            "f": f[0], "build_integrals_ms": ms_build,
            "roofline": {"kernel": "tc_gemm_kernel", "bound": "tensor",
                         "achieved": 3.0 * alg if alg else None, "peak": pk, "unit": "TFLOP/s",
                         "frac": 3.0 * alg / pk if alg else None, "achieved_algorithmic": alg,
                         "share_of_step": tc_ms / ms},
            "clocks": clk.summary(),
            "hbm_used_gb": (lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info(dev)),
            "call_sites": {k: round(v[1], 3) for k, v in
                           sorted(stats.items(), key=lambda kv: -kv[1][1])[:16]},
            "tc_sites": tc_site_fracs(stats, 1, pk)}
    print(json.dumps(line), flush=True)
    ctx.close()


# --------------------------------------------------------------------------------------
# The largest configuration as the default step: one pass of the whole path over
# a betaine-shaped system with a core orbital, two valence states and one core
# (CVS) state.  name: (N_O, N_V, n_o, n_v, N_J, valence states, core states)
WHOLE = {"betaine_like": (100, 1000, 20, 150, 4000, 2, 1)}


def apply_params(ctx, args):
    """The --param KEY=VALUE settings, applied to a timed context."""
    for kv in args.param:
        k, _, v = kv.partition("=")
        ctx.set_param(k.strip(), int(v))


def whole_step_flops(NO, NV, no, nv, nval, ncore):
    """Algorithmic flops of one whole step (the paper's leading counts, Sec. 3):
    Omega once; rho + sigma + D^{m-0} + D^{0-m} per valence state and D^{0-0}
    once for all of them (one densities call; D^{0-0} does not depend on the
    state) (units N_V n_v^3 n_o^3); a core state's rho and sigma with the
    paper's CVS count (8 N_V n_v^3 n_o^2 each), its D^{m-0} and D^{0-m}, which
    read the CVS-restricted L3 and R3, reduced the same way (units
    N_V n_v^3 n_o^2), and the D^{0-0} its own densities call builds, in full."""
    F = FLOP_UNITS
    u3, u2 = NV * nv ** 3 * no ** 3, NV * nv ** 3 * no ** 2
    val = (F["rho"] + F["sigma"] + F["D_m0"] + F["D_0m"]) * u3
    core = (F["rho"] + F["sigma"] + F["D_m0"] + F["D_0m"]) * u2 + F["D_00"] * u3
    return (F["omega"] + (F["D_00"] if nval else 0)) * u3 + nval * val + ncore * core


class WholeProblem:
    """Inputs and outputs of the whole step; `x`/`o` hold device tensors or pinned
    host tensors (the same call sequence either way)."""

    def __init__(self, x, omega, nval, ncore):
        self.x, self.omega, self.nval, self.ncore = x, omega, nval, ncore

    @staticmethod
    def outputs(x, nval, like):
        z = lambda t: like(t)
        NV, NO = x["R1"].shape[1], x["R1"].shape[2]
        nmo = NO + NV
        o = {"o1": z(x["R1"][0]), "o2": z(x["t2c"]),
             "rho1": z(x["R1"][:nval]), "rho2": z(x["R2"][:nval]),
             "sig1": z(x["R1"][:nval]), "sig2": z(x["R2"][:nval]),
             "D00": z(x["mu"][0]), "Dm0": z(x["mu"][:nval]), "D0m": z(x["mu"][:nval])}
        assert o["D00"].shape == (nmo, nmo)
        return o

    def step(self, ctx, x, o, tally=None):
        """Integral build, Omega, then rho and sigma of the valence vectors (one
        call each, skip rule off), the densities and f of each valence state,
        and rho, sigma, densities and f of the core state (skip rule on)."""
        nv_, w = self.nval, self.omega
        t = tally if tally is not None else (lambda *a: None)
        ctx.build_integrals(x["chol"], x["t1"], x["eps"], x["t2c"], x["t2x"])
        t("in", x["chol"], x["t1"], x["eps"], x["t2c"], x["t2x"])
        ctx.triples_omega(o["o1"], o["o2"])
        t("out", o["o1"], o["o2"])
        ctx.set_param("cvs", 0)
        ctx.jacobian_right(w[:nv_], x["R1"][:nv_], x["R2"][:nv_], o["rho1"], o["rho2"])
        ctx.jacobian_left(w[:nv_], x["L1"][:nv_], x["L2"][:nv_], o["sig1"], o["sig2"])
        t("in", x["R1"][:nv_], x["R2"][:nv_], x["L1"][:nv_], x["L2"][:nv_])
        t("out", o["rho1"], o["rho2"], o["sig1"], o["sig2"])
        fs = []
        for sl in (slice(0, nv_), slice(nv_, nv_ + self.ncore)):   # valence, then core states
            m = sl.stop - sl.start
            if m == 0:
                continue
            if sl.start == nv_:
                ctx.set_param("cvs", 1)
                ctx.jacobian_right(w[sl], x["R1"][sl], x["R2"][sl], o["rho1"][:m], o["rho2"][:m])
                ctx.jacobian_left(w[sl], x["L1"][sl], x["L2"][sl], o["sig1"][:m], o["sig2"][:m])
                t("in", x["R1"][sl], x["R2"][sl], x["L1"][sl], x["L2"][sl])
                t("out", o["rho1"][:m], o["rho2"][:m], o["sig1"][:m], o["sig2"][:m])
            # the densities of the group's states in one call (tau, lambda3, D^{0-0} shared)
            ctx.transition_densities(w[sl], x["lam1"], x["lam2"], x["R1"][sl], x["R2"][sl],
                                     x["L1"][sl], x["L2"][sl], x["D00_in"], o["D00"],
                                     o["Dm0"][:m], o["D0m"][:m])
            t("in", x["lam1"], x["lam2"], x["R1"][sl], x["R2"][sl], x["L1"][sl], x["L2"][sl],
              x["D00_in"])
            t("out", o["D00"], o["Dm0"][:m], o["D0m"][:m])
            for k in range(m):
                fs.append(ctx.oscillator_strength(float(w[sl.start + k]), o["D0m"][k], o["Dm0"][k],
                                                  x["mu"]))
                t("in", x["mu"])
        ctx.set_param("cvs", 1)
        return fs


def whole_fp64_comparison(NO, NV, no_s, nv, NJ, nval, ncore, dev, stream):
    """The plain FP64 GPU path against the split path where the FP64 step fits in
    the bench: the workload's shape with the active occupied space cut to
    no_s, molecule-scaled amplitudes (doubles norm 0.3, f of physical size), the
    same state mix.  Reports f with the leading-order CCSD-level densities added,
    the excitation-energy Rayleigh quotient (orbital-energy model of the
    singles-doubles block), normwise errors of every output and both step times."""
    import torch
    from paper_2202_08612_gb300 import binding
    x, omega = device_system(NO, NV, no_s, nv, NJ, nval + ncore, 4044, dev, True, t2_norm=0.3,
                             cvs_last=ncore)
    mask = np.zeros(NO, dtype=np.uint8)
    mask[0] = 1
    prob = WholeProblem(x, omega, nval, ncore)
    res = {}
    for name, prec in (("split", binding.MLCC3_SPLIT_BF16X3), ("fp64", binding.MLCC3_FP64)):
        ctx = binding.Context(NO, NV, no_s, nv, NJ, precision=prec, stream=stream.cuda_stream,
                              core_mask=mask)
        o = WholeProblem.outputs(x, nval, torch.zeros_like)
        prob.step(ctx, x, o)  # warm-up (plans, layouts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.step(ctx, x, o)
        e1.record(stream)
        torch.cuda.synchronize()
        # f of the last state computed (the core state) and of valence state 0 with the
        # leading-order CCSD-level parts: D^{0-m}_{AI} += R^A_I, D^{m-0}_{IA} += L^A_I
        fs = []
        for n in (0, nval):
            ctx.set_param("cvs", 1 if n >= nval else 0)
            D = [torch.zeros_like(o["D00"]) for _ in range(3)]
            ctx.transition_density(float(omega[n]), x["lam1"], x["lam2"], x["R1"][n], x["R2"][n],
                                   x["L1"][n], x["L2"][n], x["D00_in"], *D)
            D[2][NO:, :NO] += x["R1"][n]
            D[1][:NO, NO:] += x["L1"][n].T
            fs.append(ctx.oscillator_strength(float(omega[n]), D[2], D[1], x["mu"]))
        ctx.set_param("cvs", 0)
        e = x["eps"]
        d1 = e[NO:, None] - e[None, :NO]
        d2 = (e[NO:NO + nv][None, :, None, None] + e[NO:][None, None, None, :]
              - e[:no_s, None, None, None] - e[None, None, :NO, None])
        from paper_2202_08612_gb300 import synth
        w_ = torch.from_numpy(synth.block_weights(synth.Dims(NO, NV, no_s, nv, NJ))).to(dev)
        sd = float((x["L1"][0] * d1 * x["R1"][0]).sum() + (w_ * x["L2"][0] * d2 * x["R2"][0]).sum())
        rq = ctx.rayleigh_quotient(float(omega[0]), x["R1"][0], x["R2"][0], x["L1"][0], x["L2"][0], sd)
        res[name] = {"ms": e0.elapsed_time(e1), "f": fs, "rq": rq,
                     "out": {k: v.cpu().numpy() for k, v in o.items()}}
        ctx.close()
        del o
        torch.cuda.empty_cache()
    a, b = res["split"], res["fp64"]

    def nrm(u, v):
        return float(np.abs(u - v).max() / max(np.abs(v).max(), 1e-300))
    errs = {k: nrm(a["out"][k], b["out"][k])
            for k in ("o1", "o2", "rho1", "rho2", "sig1", "sig2", "D00", "Dm0", "D0m")}
    del x
    torch.cuda.empty_cache()
    return {"subset": f"N_O={NO} N_V={NV} n_o={no_s} n_v={nv} N_J={NJ} (the workload with the active "
                      f"occupied space cut to {no_s}), molecule-scaled amplitudes (doubles norm 0.3), "
                      f"{nval} valence + {ncore} core state(s)",
            "ms_per_step": {"split": a["ms"], "fp64": b["ms"]},
            "speedup_of_split": b["ms"] / a["ms"],
            "f": {"split": a["f"], "fp64": b["f"],
                  "abs_diff": max(abs(u - v) for u, v in zip(a["f"], b["f"]))},
            "omega_rq": {"split": a["rq"], "fp64": b["rq"], "abs_diff_hartree": abs(a["rq"] - b["rq"])},
            "normwise_rel_err": errs}


def host_chol_rows(NO, NV, no, nv, NJ, seed):
    """The recipe's Cholesky vectors on the rows the oracle's residual sample
    reads (occupied and active virtual orbitals, all columns), drawn on the host
    (torch CPU generator): symmetric on the held square block, N(0, 0.05^2)."""
    import torch
    g = torch.Generator().manual_seed(seed)
    nmo = NO + NV
    rows = np.concatenate([np.arange(NO), NO + np.arange(nv)])
    data = torch.randn((NJ, len(rows), nmo), dtype=torch.float64, generator=g) * 0.05
    sq = data[:, :, rows]
    data[:, :, rows] = (sq + sq.transpose(1, 2)) * (0.5 ** 0.5)
    return rows, data.numpy()


def oracle_residual_sample(NO, NV, no, nv, NJ, rows, data, eps, t1, t2c, t2x, reps, core=True):
    """The oracle's batched form on a bounded sample of the whole step: the
    ground-state residual stage (tau3 blocks of every ordering, contravariant
    form, back-contraction) of one unique batch i > j > k, `reps` times.  The
    integral blocks it reads are built first and are not timed.  Returns
    (TFLOP/s of the paper's Omega count for the batch's six orderings, seconds
    per repetition, sample text)."""
    from oracle import batched as B
    cr = B.CholRows(rows, data)
    mask = np.zeros(NO, dtype=np.uint8)
    if core:
        mask[0] = 1
    b = B.BCtx(NO, NV, no, nv, eps, cr, t1, t2c, t2x, mask)
    for n in ("vVvo", "Oovo", "ovov", "oOov", "Vvov", "ovOV", "oVOv"):
        b.gn(n)
    S = [(no - 1, no // 2, 1)]
    dts = []
    for _ in range(reps):
        t = time.perf_counter()
        B.triples_omega(b, S)
        dts.append(time.perf_counter() - t)
    dt = statistics.median(dts)
    fl = FLOP_UNITS["omega"] * NV * nv ** 3 * B.n_ordered(S)
    return fl / dt / 1e12, dt, (f"oracle (batched form) ground-state residual stage of one unique "
                                f"batch {S[0]} (its 6 orderings) of the workload, counted with the "
                                f"paper's Omega flops for those orderings; integral blocks built "
                                f"beforehand, untimed")


def run_whole(args, rank, world, local_rank):
    import torch
    from paper_2202_08612_gb300 import binding, build
    build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    NO, NV, no, nv, NJ, nval, ncore = WHOLE[args.workload]
    stream = torch.cuda.current_stream(dev)
    x, omega = device_system(NO, NV, no, nv, NJ, nval + ncore, 2022 + 17 * rank, dev, True,
                             cvs_last=ncore)
    mask = np.zeros(NO, dtype=np.uint8)
    mask[0] = 1
    fl = whole_step_flops(NO, NV, no, nv, nval, ncore)
    # the oracle sample's Cholesky rows, before the device memory fills up
    rows = np.concatenate([np.arange(NO), NO + np.arange(nv)])
    oracle_in = None
    if rank == 0 and not args.no_cpu_baseline:
        oracle_in = {"rows": rows, "data": x["chol"][:, torch.from_numpy(rows).to(dev), :].cpu().numpy(),
                     **{k: x[k].cpu().numpy() for k in ("eps", "t1", "t2c", "t2x")}}
    prob = WholeProblem(x, omega, nval, ncore)
    o = WholeProblem.outputs(x, nval, torch.zeros_like)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ctx = binding.Context(NO, NV, no, nv, NJ, precision=binding.MLCC3_SPLIT_BF16X3,
                          stream=stream.cuda_stream, core_mask=mask)
    ctx.set_param("chunk_blocks", args.chunk_blocks)
    apply_params(ctx, args)
    # the densities' scratch and the Jacobians' do not fit side by side next to
    # the resident inputs: every call frees its own
    ctx.set_param("release_scratch", 1)
    dist = world > 1

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize(device=dev)

    for _ in range(args.warmup):
        f_ours = prob.step(ctx, x, o)
    ctx.profile(True)
    with ClockSampler(local_rank) as clk:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            f_ours = prob.step(ctx, x, o)
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    stats = ctx.kernel_stats()
    ctx.profile(False)
    hbm_used = (lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info(dev))
    ms, value = job_throughput(ms_total, args.steps, fl, world, dev if dist else None)
    # one Davidson iteration of the step on its own: rho and sigma of the valence vectors
    ctx.set_param("cvs", 0)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e2.record(stream)
    ctx.jacobian_right(omega[:nval], x["R1"][:nval], x["R2"][:nval], o["rho1"], o["rho2"])
    ctx.jacobian_left(omega[:nval], x["L1"][:nval], x["L2"][:nval], o["sig1"], o["sig2"])
    e3.record(stream)
    barrier()
    s_iter = e2.elapsed_time(e3) * 1e-3
    ctx.set_param("cvs", 1)

    # end to end through the C ABI with pinned host buffers: every step copies its
    # inputs in and its outputs out inside the timed region
    xh = {k: v.cpu().pin_memory() for k, v in x.items()}
    del x, o
    prob.x = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    oh = WholeProblem.outputs(xh, nval, lambda t: torch.zeros_like(t).pin_memory())
    tally = {"in": 0, "out": 0}

    def count(kind, *arrs):
        tally[kind] += sum(a.numel() * a.element_size() for a in arrs)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    prob.step(ctx, xh, oh)            # host staging buffers exist from here on
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        prob.step(ctx, xh, oh, tally=count)
    torch.cuda.synchronize(device=dev)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    e2e = {"value": fl * world / e2e_s / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": tally["in"] // e2e_steps,
           "d2h_bytes_per_step": tally["out"] // e2e_steps + 8 * (nval + ncore),
           "steps": e2e_steps, "host_buffers": "pinned"}
    ctx.close()
    del xh, oh
    torch.cuda.empty_cache()

    # dominant kernel of the timed region
    agg = {}
    for k, (nl, kms_, kfl_) in stats.items():
        a = agg.setdefault(k.split(":")[0], [0, 0.0, 0.0])
        a[0] += nl
        a[1] += kms_
        a[2] += kfl_
    name, (launches, kms, kfl) = max(agg.items(), key=lambda kv: kv[1][1])
    alg = kfl / (kms * 1e-3) / 1e12 if kms > 0 else None
    pk = peaks().get("bf16_tflops_sustained") or 1700.0
    roofline = {"kernel": name, "bound": "tensor", "achieved": 3.0 * alg if alg else None, "peak": pk,
                "unit": "TFLOP/s", "frac": 3.0 * alg / pk if alg else None,
                "traffic": traffic_for(name), "achieved_algorithmic": alg,
                "launches_per_step": launches / args.steps, "share_of_step": kms / ms_total,
                "peak_note": "measured sustained dense BF16 (MEASURED_PEAKS.json); achieved "
                             "counts the 3 BF16 products (hi*hi, hi*lo, lo*hi) per product; "
                             "flops are the kernel's own products (launch accounting)"}
    gpu_launches = sum(v[0] for v in stats.values())

    fp64 = None
    if rank == 0 and not args.no_fp64_compare:
        fp64 = whole_fp64_comparison(NO, NV, 4, nv, NJ, nval, ncore, dev, stream)

    if rank == 0:
        cpu = None
        if oracle_in is not None:
            v, dt, sample = oracle_residual_sample(NO, NV, no, nv, NJ, oracle_in["rows"],
                                                   oracle_in["data"], oracle_in["eps"],
                                                   oracle_in["t1"], oracle_in["t2c"],
                                                   oracle_in["t2x"], reps=1)
            cpu = {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": sample, "seconds": dt}
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16x3", "data": "synthetic (device-generated, torch Philox)",
                "config": {"workload": f"{args.workload}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}, "
                                       f"core orbital at -10 Ha, {nval} valence + {ncore} core (CVS) "
                                       "state(s)",
                           "step": "integral build, Omega, rho and sigma of the valence vectors, "
                                   "their densities in one call (D^{0-0} once, D^{m-0} and D^{0-m} "
                                   "per state) and f, then rho, sigma, densities and f of the core "
                                   "state",
                           "flop_count": "Omega 4 + D^{0-0} 10 + 42 per valence state "
                                         "(N_V n_v^3 n_o^3); per core state 42 N_V n_v^3 n_o^2 + "
                                         "10 N_V n_v^3 n_o^3 (whole_step_flops)",
                           "algorithmic_flop_per_step": fl,
                           "precision": "split bf16x3 / fp32 accumulate / fp64 denominators and reductions",
                           "parallelism": f"replicas x{world} (independent systems)",
                           "chunk_blocks": args.chunk_blocks,
                           **({"params": list(args.param)} if args.param else {}),
                           "l2": "inputs larger than L2 (Cholesky vectors "
                                 f"{NJ * (NO + NV) ** 2 * 8 / 2**30:.1f} GiB)"},
                "s_per_davidson_iter": s_iter, "fp64_gpu_path": fp64,
                "f_step": {"values": f_ours,
                           "note": "f of the timed step's states from the triples parts of the "
                                   "densities on the configuration's distribution (amplitudes of "
                                   "order 1 at this size, hence not of physical size); the accuracy "
                                   "of f is reported under fp64_gpu_path"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
                "gpu_launches": gpu_launches, "hbm_used_gb": hbm_used,
                "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in agg.items()},
                "call_sites": {k: round(v[1] / args.steps, 3) for k, v in
                               sorted(stats.items(), key=lambda kv: -kv[1][1])[:24]},
                "site_totals": site_totals(stats, args.steps),
                "tc_sites": tc_site_fracs(stats, args.steps, pk)}
        print(json.dumps(line), flush=True)


def site_totals(stats, steps):
    """ms per step of each (kernel, call site) pair, the chunk part of the tag
    dropped (a site runs once per chunk of batches): "kernel:site"."""
    out = {}
    for k, v in stats.items():
        parts = k.split(":")
        key = parts[0] + (":" + parts[-1] if len(parts) > 1 else "")
        out[key] = out.get(key, 0.0) + v[1] / steps
    return {k: round(v, 3) for k, v in sorted(out.items(), key=lambda kv: -kv[1]) if v >= 1.0}


def run_reference_whole(args, rank):
    """The oracle's arm for the whole-step workload: inputs of the workload's shape
    drawn on the host (the rows of the Cholesky vectors the sample reads), the
    integral blocks built once, then `--warmup` + `--steps` samples of the
    ground-state residual stage of one unique batch; the timed samples give the
    value."""
    if rank != 0:
        return
    import torch
    from oracle import batched as B
    NO, NV, no, nv, NJ, nval, ncore = WHOLE[args.workload]
    rows, data = host_chol_rows(NO, NV, no, nv, NJ, 5151)
    g = torch.Generator().manual_seed(5152)
    eps = torch.cat([-1.5 + 1.2 * torch.rand(NO, dtype=torch.float64, generator=g),
                     0.1 + 2.9 * torch.rand(NV, dtype=torch.float64, generator=g)]).numpy()
    eps[0] = -10.0
    t1 = (0.01 * torch.randn(NV, NO, dtype=torch.float64, generator=g)).numpy()
    # MP2-like doubles from the bare integrals: Lov[J][L][D] = L^J_{L, N_O + D}
    Lov = data[:, :NO, NO:]
    eo, ev = eps[:NO], eps[NO:]
    den = (eo[:no, None, None, None] + eo[None, None, :, None]
           - ev[None, :nv, None, None] - ev[None, None, None, :])
    J = data.shape[0]
    A = Lov[:, :no, :nv].transpose(1, 2, 0).reshape(no * nv, J)
    t2c = (A @ Lov.reshape(J, NO * NV)).reshape(no, nv, NO, NV) / den       # (ai|DL) / D
    t2x = np.einsum('JLa,JiD->iaLD', Lov[:, :, :nv], Lov[:, :no, :], optimize=True) / den  # (aL|Di) / D
    mask = np.zeros(NO, dtype=np.uint8)
    mask[0] = 1
    b = B.BCtx(NO, NV, no, nv, eps, B.CholRows(rows, data), t1, t2c, t2x, mask)
    for n in ("vVvo", "Oovo", "ovov", "oOov", "Vvov", "ovOV", "oVOv"):
        b.gn(n)
    S = [(no - 1, no // 2, 1)]
    fl = FLOP_UNITS["omega"] * NV * nv ** 3 * B.n_ordered(S)
    vals = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        B.triples_omega(b, S)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            vals.append(dt)
    dt = statistics.mean(vals)
    value = fl / dt / 1e12
    sample = (f"oracle (batched form) ground-state residual stage of one unique batch {S[0]} "
              f"(its 6 orderings) of the workload per step, counted with the paper's Omega flops "
              f"for those orderings; inputs drawn on the host, integral blocks built once, untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: N_O={NO} N_V={NV} n_o={no} n_v={nv} N_J={NJ}, "
                                   f"core orbital at -10 Ha, {nval} valence + {ncore} core (CVS) state(s)"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fp64emu(args):
    """FP64-accurate products on the tensor cores (mlcc3_fp64emu_gemm, 5 and 6
    digit slices) against cuBLAS DGEMM (the SIMT FP64 rate) on one square
    product of the Cholesky-index size (M = N = K = 4096): TFLOP/s of each and
    the normwise error against DGEMM."""
    import torch
    from paper_2202_08612_gb300 import binding
    dev = torch.device("cuda", 0)
    n = 4096
    g = torch.Generator(device=dev)
    g.manual_seed(2022)
    A = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    fl = 2.0 * n ** 3

    def timed(f, k):
        for _ in range(max(1, args.warmup)):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ref = A @ B.T
    ms_d = timed(lambda: torch.matmul(A, B.T, out=C), args.steps)
    res = {}
    for s in (5, 6):
        ms = timed(lambda: binding.fp64emu_gemm(A, B, C, slices=s), args.steps)
        err = float(torch.linalg.norm(C - ref) / torch.linalg.norm(ref))
        res[s] = {"ms": ms, "tflops": fl / ms / 1e9, "normwise_rel_err_vs_dgemm": err}
    print(json.dumps({"metric": "FP64-accurate GEMM TFLOP/s (tensor-core digit slices vs DGEMM)",
                      "value": res[5]["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "config": {"workload": f"C = A B^T, M = N = K = {n}, FP64 normal entries",
                                 "note": "each call allocates and frees its temporaries"},
                      "slices": {str(k): v for k, v in res.items()},
                      "dgemm": {"ms": ms_d, "tflops": fl / ms_d / 1e9}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="betaine_like",
                    choices=sorted(set(WORKLOADS) | set(WHOLE) | set(LARGE)) + ["uneven_sweep", "nv_scaling", "fp64emu_gemm"])
    ap.add_argument("--vectors", type=int, default=4,
                    help="trial vectors per system of the uneven_sweep workload")
    ap.add_argument("--precision", default="split", choices=("split", "fp64"))
    ap.add_argument("--tc-group", type=int, default=0,
                    help="batches per triples-build tensor-core tile (0: library default)")
    ap.add_argument("--tc-wide-bn", type=int, default=0,
                    help="tile width of the pair contractions wider than 256 columns "
                         "(128, 160 or 256; 0: the library default)")
    ap.add_argument("--chunk-blocks", type=int, default=128,
                    help="large workloads: unique batches held per chunk")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="whole-step workload: steps of the end-to-end (pinned host buffers) run")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle sample (CPU baseline)")
    ap.add_argument("--stage", default=None, choices=("davidson", "densities", "cvs", "ground"),
                    help="large workloads: Davidson iterations (rho, sigma) of the valence "
                         "vectors, the densities and f of one state, the Davidson iteration "
                         "of one core (CVS) state, or the ground-state stages (multiplier "
                         "transformation and D^{0-0})")
    ap.add_argument("--param", action="append", default=[], metavar="KEY=VALUE",
                    help="a context parameter (mlcc3_set_param) for the timed contexts; repeatable")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the untimed FP64-path comparison step")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl")
    if args.impl == "ours" and args.workload == "fp64emu_gemm":
        run_fp64emu(args)
    elif args.impl == "ours" and args.workload == "uneven_sweep":
        run_sweep(args)
    elif args.impl == "ours" and args.workload == "nv_scaling":
        run_nv_scaling(args)
    elif args.impl == "ours" and args.workload in LARGE and (args.stage is not None
                                                             or args.workload not in WHOLE):
        args.stage = args.stage or "davidson"
        run_large(args)
    elif args.impl == "ours" and args.workload in WHOLE:
        run_whole(args, rank, world, local_rank)
    elif args.impl == "reference" and args.workload in WHOLE and args.stage is None:
        run_reference_whole(args, rank)
    elif args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
