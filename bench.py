#!/usr/bin/env python
"""Benchmark of the time-step-targeting Krylov hot path on one GB300.

Workload: the L=32 Hubbard chain superblock (U=4, t=1, half filling, m=400 kept states, one bond
across the central cut; seeded Gaussian-sector twin of a truncated DMRG superblock, complex128),
excited by c^dag on the first right site, advanced with tau=0.05, n_v=4 time targets and n_K=10.

One step = one time step of the hot path: the Krylov advance (n_K Lanczos steps, each a grouped
H psi + FP64 CGS2), the tridiagonal exponential and target assembly, the weighted rho_L of the
ground state and the 4 targets, its eigendecomposition, and two expectation values.
`value` = Krylov steps/s over the whole job (n_K per step); L2 is flushed before every step.
The default arithmetic of H psi is the tensor-core path (bf16 Ozaki slices, --slices 4); the plain
FP64 GPU path is timed beside it on the same workload, with the largest difference of the measured
observables over a 20-step trajectory (vs_fp64_gpu).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64 NumPy) on the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Krylov steps/s & Hψ TFLOP/s vs plain FP64 GPU at ≤1e-8 error; p50/p99 step latency"
UNIT = "Krylov steps/s"
# The bench workloads (synthetic Gaussian-sector twins of truncated DMRG superblocks at the central
# cut, complex128, c^dag excitation on the first right site).  C2 is the headline; C3 and C4 are
# measured beside it.
CONFIGS = {
    "C2": dict(L=32, m=400, U=4.0, t=1.0, nbonds=1, tau=0.05, n_v=4, nk=10, seed_index=1,
               name="1D Hubbard chain L=32 U=4 half filling m=400 superblock (synthetic Gaussian-sector twin), "
                    "c^dag excitation, tau=0.05, n_v=4, n_K=10, complex128"),
    "C3": dict(L=32, m=800, U=8.0, t=1.0, nbonds=2, tau=0.05, n_v=4, nk=10, seed_index=2,
               name="2x16 Hubbard ladder U=8 half filling m=800 superblock (synthetic twin, 2 bonds across the cut), "
                    "c^dag excitation, tau=0.05, n_v=4, n_K=10, complex128"),
    "C4": dict(L=48, m=1000, U=10.0, t=1.0, nbonds=1, tau=0.02, n_v=4, nk=10, seed_index=4,
               name="1D Hubbard chain L=48 U=10 half filling m=1000 superblock (synthetic twin), "
                    "c^dag excitation, tau=0.02, n_v=4, n_K=10, complex128"),
}
WL = CONFIGS["C2"]
WORKLOAD_NAME = WL["name"]
FLUSH_BYTES = 256 << 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes of one tensor-path H psi, from an ncu capture summarised in this file; valid only while the
# kernels, plans and workload generator are byte-identical to those captured (digest below)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_hpsi_ozaki_L32_m400_chain.md")
TRAFFIC_SOURCES = ("paper_1103_5391_gb300/csrc/ozaki.cu", "paper_1103_5391_gb300/csrc/plan.cu",
                   "paper_1103_5391_gb300/csrc/internal.h", "workloads/sectors.py")


def sources_digest():
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def hpsi_traffic():
    """(bytes per H psi, note) from the committed capture, or (None, why not)."""
    try:
        with open(TRAFFIC_FILE) as f:
            text = f.read()
    except OSError:
        return None, "no DRAM capture committed"
    b = re.search(r"^traffic_bytes_per_hpsi: (\d+)$", text, re.M)
    d = re.search(r"^sources_sha256: ([0-9a-f]{64})$", text, re.M)
    if not b or not d:
        return None, "DRAM capture summary unreadable"
    if d.group(1) != sources_digest():
        return None, "kernel or workload sources changed since the DRAM capture"
    return int(b.group(1)), "dram__bytes_read.sum + dram__bytes_write.sum of the 4 launches of one H psi (ncu, " \
                            + os.path.relpath(TRAFFIC_FILE, ROOT) + ")"


def measured_peaks():
    """(peaks dict, source): the measured copy bandwidth and bf16 GEMM rates of this GPU pool, or the
    fallback figures when the measurement file is absent."""
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return {k: float(d[k]) for k in FALLBACK_PEAKS}, "of measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError, TypeError):
        return dict(FALLBACK_PEAKS), "of fallback (no MEASURED_PEAKS.json)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="C2",
                    help="workload of the headline line (C2 by default; C3 and C4 are also measured beside C2)")
    ap.add_argument("--no-other-configs", action="store_true", help="measure the headline workload only")
    ap.add_argument("--batch-jobs", type=int, default=24, help="jobs of the batched-mix measurement (0: skip)")
    ap.add_argument("--oracle-rate", metavar="CONFIG", default=None,
                    help="(internal) time the oracle's step on CONFIG in this process and print one JSON line")
    ap.add_argument("--prec", choices=["ozaki", "fp64"], default="ozaki")
    ap.add_argument("--slices", type=int, default=4)
    ap.add_argument("--serving", action="store_true", help="serving mix instead of the single-workload line")
    ap.add_argument("--jobs", type=int, default=24)
    ap.add_argument("--job-steps", type=int, default=20)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--job-lmax", type=int, default=48, help="serving: largest L of a job (even, >= 16)")
    ap.add_argument("--job-mmax", type=int, default=768, help="serving: largest m of a job (>= 128)")
    ap.add_argument("--gap-ms", type=float, default=20.0, help="serving: mean inter-arrival time")
    ap.add_argument("--max-group", type=int, default=1, help="serving: batch up to this many jobs per group (1: off)")
    ap.add_argument("--batch-window-us", type=int, default=2000, help="serving: how long a job waits for partners")
    ap.add_argument("--profile-hpsi", type=int, default=0, metavar="N",
                    help="only apply H psi N times on the workload (a short run for ncu captures)")
    ap.add_argument("--tile-m", type=int, default=0, choices=[0, 64, 128],
                    help="--profile-hpsi: fix the tile M of the tensor kernel (0: autotuned)")
    ap.add_argument("--thin-dim", type=int, default=None,
                    help="profile mode: products with fewer rows or columns run on the FP64 thin warps (0 = none)")
    ap.add_argument("--precision-errors", action="store_true",
                    help="errors of the tensor path (S = 2..6 slices) against the FP64 path on the L=48 m=1000 chain")
    return ap.parse_args()


def workload(wl=WL):
    from workloads import sectors as S
    return S.make_synthetic(wl["L"], wl["m"], wl["U"], t=wl["t"], nbonds=wl["nbonds"], seed=S.SEED_BASE + wl["seed_index"])


def _pairs(ss, Q):
    ridx = {q: k for k, q in enumerate(ss.rsec)}
    pair = {}
    for qi, q in enumerate(ss.lsec):
        ri = ridx.get((Q[0] - q[0], Q[1] - q[1]))
        if ri is not None:
            pair[qi] = ri
    return pair


def _connection_blocks(ss, pair):
    """(dL_out, dL_in, dR_in, dR_out) of every sector-pair product of the boundary terms (both halves of
    each hopping, both spins, every bond)."""
    out = []
    for b in range(ss.nbonds):
        for s in range(2):
            for A, B in ((ss.cdagL[b][s], ss.cR[b][s]),
                         ({(i, o): 0 for (o, i) in ss.cdagL[b][s]}, {(i, o): 0 for (o, i) in ss.cR[b][s]})):
                for (qo, qi) in A:
                    if qi not in pair or qo not in pair:
                        continue
                    ri, ro = pair[qi], pair[qo]
                    if (ro, ri) not in B:
                        continue
                    out.append((ss.ldim[qo], ss.ldim[qi], ss.rdim[ri], ss.rdim[ro]))
    return out


def algorithmic_hpsi_flops(ss, Q):
    """8 flops per complex MAC, cheaper association per two-sided term, one GEMM per block term."""
    pair = _pairs(ss, Q)
    fl = 0.0
    for qi, ri in pair.items():
        dl, dr = ss.ldim[qi], ss.rdim[ri]
        fl += 8.0 * (dl * dl * dr + dl * dr * dr)
    for a, b_, c, d in _connection_blocks(ss, pair):
        fl += 8.0 * min(b_ * c * d + a * b_ * d, a * b_ * c + a * c * d)
    return fl


def algorithmic_hpsi_bytes(ss, Q):
    """Lower bound of the DRAM bytes of one H psi: read psi and write H psi once (16 D each) and read
    every operator block the product uses once (complex128)."""
    pair = _pairs(ss, Q)
    D = sum(ss.ldim[qi] * ss.rdim[ri] for qi, ri in pair.items())
    ops = sum(ss.ldim[qi] ** 2 + ss.rdim[ri] ** 2 for qi, ri in pair.items())
    ops += sum(a * b_ + c * d for a, b_, c, d in _connection_blocks(ss, pair))
    return 32.0 * D + 16.0 * ops


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = sum(i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas")
        if n:
            return n
    except Exception:
        pass
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count()


class OracleStep:
    """One time step of the CPU oracle on the same workload (FP64 NumPy)."""

    def __init__(self, ss, wl=WL):
        from oracle import blocks as oblocks
        from oracle import density, krylov, superblock
        self.k, self.d, self.s = krylov, density, superblock
        self.ss, self.wl = ss, wl
        self.sb = superblock.Superblock(ss.lsec, ss.ldim, ss.rsec, ss.rdim)
        self.HL, self.HR = oblocks.BlockOp(ss.HL, False), oblocks.BlockOp(ss.HR, False)
        self.conns = []
        for b in range(ss.nbonds):
            for s in range(2):
                A, B = oblocks.BlockOp(ss.cdagL[b][s], True), oblocks.BlockOp(ss.cR[b][s], True)
                self.conns += [(ss.coeff_t, A, B), (-ss.coeff_t, A.dagger(), B.dagger())]
        self.nL, self.nR = oblocks.BlockOp(ss.nL, False), oblocks.BlockOp(ss.nR, False)
        exc = oblocks.BlockOp(ss.cdag_exc, True)
        self.phi = superblock.apply_op(self.sb, None, exc, ss.Q0, ss.psi_gs, ss.Q1)
        self.times = krylov.target_times(wl["tau"], wl["n_v"])
        self.wgs, self.w = density.tst_weights(wl["n_v"])

    def step(self):
        Q = self.ss.Q1
        hf = lambda v: self.s.apply_h(self.sb, self.HL, self.HR, self.conns, Q, v)
        targets, n_used, err = self.k.evolve(hf, self.phi, self.times, self.wl["nk"])
        rho = self.d.rho_left(self.sb, [(self.ss.Q0, self.ss.psi_gs)] + [(Q, t) for t in targets], [self.wgs] + self.w)
        self.d.rho_eig(rho)
        self.s.expect(self.sb, self.nL, None, Q, targets[-1])
        self.s.expect(self.sb, None, self.nR, Q, targets[-1])
        self.phi = targets[-1]
        return n_used


def host_cpu():
    """(logical CPUs this process may run on, CPU model name)."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return n, model or platform.machine()


def oracle_rate(ss, wl, block_s=1.6, reps=5):
    """Best of `reps` blocks (each at least block_s seconds of whole oracle time steps, after one
    warm-up step) in Krylov steps/s; also the steps and seconds of all blocks."""
    st = OracleStep(ss, wl)
    st.step()
    best, ks_all, n_all, t_all = 0.0, 0, 0, 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        ks = n = 0
        while n == 0 or time.perf_counter() - t0 < block_s:
            ks += st.step()
            n += 1
        dt = time.perf_counter() - t0
        best = max(best, ks / dt)
        ks_all, n_all, t_all = ks_all + ks, n_all + n, t_all + dt
    return best, n_all, ks_all, t_all


def oracle_rate_one_core(key):
    """The same measurement in a child process pinned to one CPU with one BLAS thread."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cpu0 = min(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None
    pin = (lambda: os.sched_setaffinity(0, {cpu0})) if cpu0 is not None else None
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate", key], env=env,
                           preexec_fn=pin, capture_output=True, text=True, timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:
        return {"error": f"one-core oracle run failed: {e}"}


def cpu_baseline(ss, key="C2"):
    """The oracle's time step on the host: all cores (BLAS threads = cores) and one core, best of 5."""
    wl = CONFIGS[key]
    ncpu, model = host_cpu()
    best, n, ks, dt = oracle_rate(ss, wl)
    one = oracle_rate_one_core(key)
    return {"value": best, "unit": UNIT, "cores": ncpu, "kind": "oracle", "cpu_model": model, "nproc": ncpu,
            "blas_threads": blas_threads(),
            "one_core": one.get("value"), "one_core_note": one.get("sample", one.get("error")),
            "sample": f"best of 5 blocks (>= 1.6 s each) of whole oracle time steps of the same workload "
                      f"(n_K Krylov steps + rho_L + eig + 2 observables per time step): {n} time steps, {ks} Krylov "
                      f"steps in {dt:.1f} s; FP64 NumPy on {ncpu} host cores ({model})"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.idx = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def config_dict(wl):
    return {"workload": wl["name"], **{k: wl[k] for k in ("L", "m", "U", "t", "nbonds", "tau", "n_v", "nk")}}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    ss = workload()
    st = OracleStep(ss)
    for _ in range(args.warmup):
        st.step()
    times, ks = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ks += st.step()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    val = ks / total
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic", "impl": "reference",
            "config": {**config_dict(WL), "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": host_cpu()[0], "cpu_model": host_cpu()[1],
                             "blas_threads": blas_threads(), "kind": "oracle",
                             "sample": f"{args.steps} oracle time steps ({ks} Krylov steps) after {args.warmup} warm-up"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Runner:
    """Device buffers and one time step of the hot path through the C ABI."""

    def __init__(self, T, problem, ctx, ss, dev, stream, wl=WL):
        import torch
        self.T, self.P, self.ctx, self.ss, self.stream = T, problem, ctx, ss, stream
        c128 = dict(dtype=torch.complex128, device=dev)
        self.Q0, self.Q1 = ss.Q0, ss.Q1
        self.n1 = T.tdmrg_sector_size(ctx, self.Q1)
        self.psi_gs = torch.as_tensor(ss.psi_gs).to(dev)
        self.phi = torch.zeros(self.n1, **c128)
        T.tdmrg_apply_op(ctx, -1, problem.OP_EXC, self.Q0, self.psi_gs, self.Q1, self.phi)   # phi = c^dag_j psi (Eq. b)
        self.phi0 = self.phi.clone()
        self.nv, self.nk = wl["n_v"], wl["nk"]
        self.times = [x * wl["tau"] / (self.nv - 1) for x in range(self.nv)]
        self.targets = [torch.zeros(self.n1, **c128) for _ in range(self.nv - 1)] + [self.phi]   # advance in place
        self.wgs, self.w = T.tdmrg_tst_weights(self.nv)
        self.nr, self.ne = T.tdmrg_rho_size(ctx)
        self.rho = torch.zeros(self.nr, **c128)
        self.evals = torch.zeros(self.ne, dtype=torch.float64, device=dev)
        self.evecs = torch.zeros(self.nr, **c128)
        self.obs = torch.zeros(2, **c128)
        self.aux = torch.cuda.Stream(device=dev)   # observables beside rho_L and its eigendecomposition
        self.cur = stream                          # stream the step is issued on (the capture stream in capture)

    def reset(self):
        self.phi.copy_(self.phi0)

    def capture(self, torch, stream):
        """One time step as a CUDA graph (after a direct step has compiled plans and workspace)."""
        side = torch.cuda.Stream(device=stream.device)
        side.wait_stream(stream)
        self.T.tdmrg_set_stream(self.ctx, side.cuda_stream)
        self.graph = torch.cuda.CUDAGraph()
        self.cur = side
        with torch.cuda.graph(self.graph, stream=side, capture_error_mode="thread_local"):
            self.step()
        self.cur = stream
        self.T.tdmrg_set_stream(self.ctx, stream.cuda_stream)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()

    def step(self):
        """One time step.  The observables only read the evolved state, so they run on a second
        stream beside the eigendecomposition of rho_L (whose Jacobi seed, one CTA per sector, leaves
        most SMs idle); fork and join are events, which a graph capture keeps as dependencies."""
        import torch
        T, c, P = self.T, self.ctx, self.P
        T.tdmrg_evolve(c, self.Q1, self.phi, self.times, self.nk, self.targets)
        T.tdmrg_density_matrix(c, [(self.Q0, self.psi_gs)] + [(self.Q1, t) for t in self.targets], [self.wgs] + self.w,
                               self.rho)
        fork, join = torch.cuda.Event(), torch.cuda.Event()
        fork.record(self.cur)
        self.aux.wait_event(fork)
        T.tdmrg_set_stream(c, self.aux.cuda_stream)
        T.tdmrg_expect(c, P.OP_N, -1, self.Q1, self.phi, self.obs[0:1])
        T.tdmrg_expect(c, -1, P.OP_N, self.Q1, self.phi, self.obs[1:2])
        join.record(self.aux)
        T.tdmrg_set_stream(c, self.cur.cuda_stream)
        T.tdmrg_rho_eig(c, self.rho, self.evals, self.evecs)
        self.cur.wait_event(join)


def replica_value(total_ms, work_units, world_size, device=None):
    """Whole-job throughput of independent replicas: the units all ranks processed divided by the
    slowest rank's timed device time (one all-reduce of a scalar; no data-path collective)."""
    import torch
    if world_size > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world_size * work_units / (total_ms * 1e-3), total_ms


def timed_steps(torch, runner, steps, flush, stream, barrier, graph=False):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record(stream)
        if graph:
            runner.replay()
        else:
            runner.step()
        e1.record(stream)
    barrier()
    return [a.elapsed_time(b) for a, b in ev]


def time_hpsi(torch, T, ctx, Q, x, out, flush, stream, reps=50):
    for _ in range(3):
        T.tdmrg_apply_h(ctx, Q, x, out)
    hev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in hev:
        flush.fill_(1)
        e0.record(stream)
        T.tdmrg_apply_h(ctx, Q, x, out)
        e1.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in hev)


def trajectory(torch, runner, steps):
    """Observables <n_L>, <n_R> after each of `steps` time steps from the initial excitation."""
    runner.reset()
    out = []
    for _ in range(steps):
        runner.step()
        out.append(runner.obs.clone())
    torch.cuda.synchronize()
    return torch.stack(out).cpu().numpy()


def work_decomposition(T, ctx, ss, Q, slices, alg):
    """Executed tensor flops of one H psi against the algorithmic count: the plan's association
    (stage 1 then stage 2 for every two-sided term), the S(S+1)/2 slice products, and the padding of
    sector blocks into MMA tiles."""
    plan = T.tdmrg_hpsi_flops(ctx, Q)
    tensor = T.tdmrg_hpsi_tensor_flops(ctx, Q)
    groups = slices * (slices + 1) / 2
    return {"alg_gflop": alg / 1e9, "plan_gflop": plan / 1e9, "executed_tensor_gflop": tensor / 1e9,
            "executed_over_alg": tensor / alg if alg else None, "association_factor": plan / alg if alg else None,
            "slice_factor": groups, "padding_factor": tensor / (plan * groups) if plan else None}


def measure_config(args, torch, T, problem, key, dev, stream, flush, barrier, steps, headline=False):
    """Steps/s of the tensor path and of the FP64 path on one workload, H psi alone on both, the
    observable difference over a 20-step trajectory, and the roofline of H psi."""
    wl = CONFIGS[key]
    ss = workload(wl)
    res = {"config": config_dict(wl)}
    mixed = args.prec == "ozaki"
    prec = T.TDMRG_OZAKI_BF16 if mixed else T.TDMRG_FP64
    ctx = T.tdmrg_create(device=dev.index, stream=stream.cuda_stream, prec=prec, ozaki_slices=args.slices)
    try:
        problem.load_synthetic(ctx, ss)
        run = Runner(T, problem, ctx, ss, dev, stream, wl)
        run.step()                      # compiles plans, allocates workspace
        l0 = T.tdmrg_launch_count(ctx)
        run.step()
        res["launches_per_step"] = T.tdmrg_launch_count(ctx) - l0
        run.capture(torch, stream)      # the timed step is one CUDA-graph replay of the same launches
        for _ in range(args.warmup):
            run.replay()
        barrier()
        sampler = ClockSampler(dev.index) if headline else None
        if headline:
            time.sleep(0.25)
        step_ms = timed_steps(torch, run, steps, flush, stream, barrier, graph=True)
        if headline:
            res["clocks"] = sampler.stop()
        T.tdmrg_evolve_info(ctx)   # raises if a bounded device wait ran out during the timed steps
        res["step_ms"] = step_ms
        res["value"] = run.nk * len(step_ms) / (sum(step_ms) * 1e-3)
        srt = sorted(step_ms)
        res["step_latency_ms"] = {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]}
        Q1 = run.Q1
        hx = torch.zeros(run.n1, dtype=torch.complex128, device=dev)
        h_ms = time_hpsi(torch, T, ctx, Q1, run.phi0, hx, flush, stream)
        alg = algorithmic_hpsi_flops(ss, Q1)
        alg_bytes = algorithmic_hpsi_bytes(ss, Q1)
        res["D"] = run.n1
        res["hpsi"] = {"ms": h_ms, "alg_tflops": alg / (h_ms * 1e-3) / 1e12, "alg_bytes": alg_bytes}
        if mixed:
            res["hpsi"]["work"] = work_decomposition(T, ctx, ss, Q1, args.slices, alg)
            res["hpsi"]["tuning"] = {"stage%d" % (k + 1): {"tile_m": m, "schedule": "queue" if q == 1 else "static"}
                                     for k, (m, q) in enumerate(T.tdmrg_hpsi_tuning(ctx, Q1))}
        if headline:
            res["run"] = run
            res["ctx"] = ctx
        # the plain FP64 GPU path on the same workload, and the observable difference to it
        if mixed:
            traj_steps = 20
            traj_m = trajectory(torch, run, traj_steps)
            T.tdmrg_set_precision(ctx, T.TDMRG_FP64, 4)
            traj_f = trajectory(torch, run, traj_steps)
            run.reset()
            run.step()
            run.capture(torch, stream)
            for _ in range(2):
                run.replay()
            f_ms = timed_steps(torch, run, min(steps, 40), flush, stream, barrier, graph=True)
            hf_ms = time_hpsi(torch, T, ctx, Q1, run.phi0, hx, flush, stream)
            res["vs_fp64_gpu"] = {"value": run.nk * len(f_ms) / (sum(f_ms) * 1e-3), "unit": UNIT,
                                  "ms_per_step": statistics.mean(f_ms), "hpsi_ms": hf_ms,
                                  "hpsi_tflops": alg / (hf_ms * 1e-3) / 1e12,
                                  "speedup_steps": res["value"] / (run.nk * len(f_ms) / (sum(f_ms) * 1e-3)),
                                  "obs_err": float(np.abs(traj_m - traj_f).max()), "obs_err_steps": traj_steps}
            if headline:
                T.tdmrg_set_precision(ctx, prec, args.slices)   # the e2e leg runs the headline path again
                run.reset()
                run.step()
                run.capture(torch, stream)
    finally:
        if not headline:
            T.tdmrg_destroy(ctx)
    return res


def measure_batched(args, torch, T, problem, dev, stream, flush, barrier, njobs, steps=5, warmup=2):
    """Aggregate Krylov steps/s of a mix of independent jobs (chains and two-leg ladders, L in [16, 48],
    m log-uniform in [128, 512], U in {2, 4, 8}; seeded): a full time step per job (Krylov advance, rho_L
    of the ground state and the targets, its eigendecomposition, two observables), (a) each job on its own
    stream, (b) the advances of all jobs as one segmented advance over their direct sum (one grouped
    product per Lanczos step for every job), the rest per job on its stream."""
    from workloads import sectors as S
    prec = T.TDMRG_OZAKI_BF16 if args.prec == "ozaki" else T.TDMRG_FP64
    rng = np.random.default_rng(1103)
    jobs = []
    for k in range(njobs):
        L = int(rng.choice([16, 24, 32, 40, 48]))
        m = int(np.exp(rng.uniform(np.log(128), np.log(512))))
        nb = 1 if rng.random() < 0.7 else 2
        ss = S.make_synthetic(L, m, float(rng.choice([2.0, 4.0, 8.0])), nbonds=nb, seed=2000 + k)
        ctx = T.tdmrg_create(device=dev.index, stream=stream.cuda_stream, prec=prec, ozaki_slices=args.slices)
        problem.load_synthetic(ctx, ss)
        jobs.append(Runner(T, problem, ctx, ss, dev, stream, WL))
    nv, nk, times = WL["n_v"], WL["nk"], jobs[0].times
    streams = [torch.cuda.Stream(device=dev) for _ in jobs]

    def tail(r, st, targets):   # rho_L, its eigendecomposition and the observables of one job on its stream
        T.tdmrg_set_stream(r.ctx, st.cuda_stream)
        T.tdmrg_density_matrix(r.ctx, [(r.Q0, r.psi_gs)] + [(r.Q1, t) for t in targets], [r.wgs] + r.w, r.rho)
        T.tdmrg_rho_eig(r.ctx, r.rho, r.evals, r.evecs)
        T.tdmrg_expect(r.ctx, problem.OP_N, -1, r.Q1, targets[-1], r.obs[0:1])
        T.tdmrg_expect(r.ctx, -1, problem.OP_N, r.Q1, targets[-1], r.obs[1:2])
        T.tdmrg_set_stream(r.ctx, stream.cuda_stream)

    def step_streams():
        ev = torch.cuda.Event()
        ev.record(stream)
        for r, st in zip(jobs, streams):
            st.wait_event(ev)
            T.tdmrg_set_stream(r.ctx, st.cuda_stream)
            T.tdmrg_evolve(r.ctx, r.Q1, r.phi, r.times, nk, r.targets)
            tail(r, st, r.targets)
        for st in streams:
            stream.wait_stream(st)

    big = T.tdmrg_create(device=dev.index, stream=stream.cuda_stream, prec=prec, ozaki_slices=args.slices)
    Qs, off = T.tdmrg_direct_sum(big, [r.ctx for r in jobs], [r.Q1 for r in jobs])
    bphi = torch.cat([r.phi0 for r in jobs])
    bphi0 = bphi.clone()
    btg = [torch.zeros_like(bphi) for _ in range(nv - 1)] + [bphi]   # advance in place, like the single job
    seg = [off[k + 1] - off[k] for k in range(njobs)]

    Q0s = (Qs[0] - 1, Qs[1])   # the ground states' sector of the sum (every job's excitation is c^dag_up)
    bpsi = torch.cat([r.psi_gs for r in jobs])
    nr, ne = T.tdmrg_rho_size(big)
    brho = torch.zeros(nr, dtype=torch.complex128, device=dev)
    bev = torch.zeros(ne, dtype=torch.float64, device=dev)
    bU = torch.zeros_like(brho)

    def step_batched():
        # one segmented advance, one grouped rho_L (every job normalised apart) and one eigendecomposition over
        # every job's sectors; the observables per job on its own stream beside the eigendecomposition
        T.tdmrg_evolve_segments(big, Qs, bphi, seg, times, nk, btg)
        T.tdmrg_density_matrix(big, [(Q0s, bpsi)] + [(Qs, t) for t in btg], [jobs[0].wgs] + jobs[0].w, brho)
        ev = torch.cuda.Event()
        ev.record(stream)
        for k, (r, st) in enumerate(zip(jobs, streams)):
            st.wait_event(ev)
            T.tdmrg_set_stream(r.ctx, st.cuda_stream)
            last = btg[-1][off[k]: off[k + 1]]
            T.tdmrg_expect(r.ctx, problem.OP_N, -1, r.Q1, last, r.obs[0:1])
            T.tdmrg_expect(r.ctx, -1, problem.OP_N, r.Q1, last, r.obs[1:2])
            T.tdmrg_set_stream(r.ctx, stream.cuda_stream)
        T.tdmrg_rho_eig(big, brho, bev, bU)
        for st in streams:
            stream.wait_stream(st)

    def timed(fn):
        for _ in range(warmup):
            fn()
        barrier()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            barrier()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    for r in jobs:
        r.reset()
    t_streams = timed(step_streams)
    bphi.copy_(bphi0)
    t_batch = timed(step_batched)
    # the same first step both ways: every job's targets agree
    for r in jobs:
        r.reset()
    bphi.copy_(bphi0)
    step_streams()
    step_batched()
    barrier()
    diff = max(float((btg[x][off[k]: off[k + 1]] - jobs[k].targets[x]).abs().max() /
                     jobs[k].targets[x].abs().max()) for k in range(njobs) for x in range(nv))
    ev_diff = float((bev - torch.cat([r.evals for r in jobs])).abs().max())
    T.tdmrg_destroy(big)
    for r in jobs:
        T.tdmrg_destroy(r.ctx)
    return {"jobs": njobs, "D_total": int(off[-1]), "unit": UNIT,
            "value": njobs * nk / (t_batch * 1e-3), "ms_per_step": t_batch,
            "value_streams": njobs * nk / (t_streams * 1e-3), "ms_per_step_streams": t_streams,
            "speedup_vs_streams": t_streams / t_batch, "max_rel_diff_vs_streams": diff,
            "max_eigenvalue_diff_vs_streams": ev_diff,
            "mode": "the jobs' superblocks as one direct sum: one segmented Krylov advance (one grouped product "
                    "per Lanczos step for every job), one grouped rho_L and one eigendecomposition over every "
                    "job's sectors, observables per job; compared with every job's whole step on its own stream"}


def roofline_of(res, mixed, peaks, peak_src, dmma_peak, dfma_peak, traffic=None, traffic_note=None):
    """Roofline of H psi: algorithmic FP64-equivalent flops (cheaper association per term, 8 per complex
    MAC) per H psi over its measured time, against the measured bf16 dense peak (tensor path) or the
    FP64 MMA peak measured live (FP64 path)."""
    h = res["hpsi"]
    alg_tf = h["alg_tflops"]
    if mixed:
        roof = {"bound": "tensor", "achieved": alg_tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "peak_source": "bf16 dense burst " + peak_src,
                "kernel": "H psi on the tensor path (bf16 slicing + tcgen05 GEMM launches of one product)",
                "work": h.get("work")}
        w = h.get("work") or {}
        if w.get("executed_tensor_gflop"):
            roof["executed_tensor_tflops"] = w["executed_tensor_gflop"] * 1e9 / (h["ms"] * 1e-3) / 1e12
            roof["executed_frac"] = roof["executed_tensor_tflops"] / roof["peak"]
    else:
        roof = {"bound": "tensor", "achieved": alg_tf, "peak": dmma_peak, "unit": "TFLOP/s",
                "peak_source": f"FP64 tensor MMA (mma.sync m8n8k4 f64) loop on every SM, measured live by "
                               f"tdmrg_fp64_peak (not in MEASURED_PEAKS.json); DFMA {dfma_peak:.2f} TFLOP/s",
                "kernel": "gemm_f64_kernel (H psi, 2 launches)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["alg_bytes"] = h["alg_bytes"]
    roof["traffic"] = traffic
    roof["traffic_source"] = traffic_note
    roof["traffic_over_alg_bytes"] = traffic / h["alg_bytes"] if traffic else None
    roof["hbm_frac_of_alg_bytes"] = h["alg_bytes"] / (h["ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"]
    return roof


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mixed = args.prec == "ozaki"
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peaks, peak_src = measured_peaks()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    key = args.config
    wl = CONFIGS[key]
    res = measure_config(args, torch, T, problem, key, dev, stream, flush, barrier, args.steps, headline=True)
    run, ctx = res.pop("run"), res.pop("ctx")
    nk = run.nk
    value, total_ms = replica_value(sum(res["step_ms"]), nk * args.steps, ws, dev)
    launches = res["launches_per_step"] * args.steps
    dmma_peak, dfma_peak = T.tdmrg_fp64_peak(local)

    # end to end through the C ABI with host buffers: H2D phi, step, D2H observables + rho_L spectrum
    e2e_steps = max(3, min(args.steps, 50))
    phi_h = run.phi0.cpu().pin_memory()
    obs_h = torch.zeros(2, dtype=torch.complex128).pin_memory()
    ev_h = torch.zeros(run.ne, dtype=torch.float64).pin_memory()
    barrier()
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for e0, e1 in ee:
        flush.fill_(1)
        e0.record(stream)
        run.phi.copy_(phi_h, non_blocking=True)
        run.step()
        obs_h.copy_(run.obs, non_blocking=True)
        ev_h.copy_(run.evals, non_blocking=True)
        e1.record(stream)
    barrier()
    e2e_val, e2e_ms = replica_value(sum(a.elapsed_time(b) for a, b in ee), nk * e2e_steps, ws, dev)
    T.tdmrg_destroy(ctx)

    others = {}
    if rank == 0 and not args.no_other_configs and key == "C2":
        for k2 in ("C3", "C4"):
            r2 = measure_config(args, torch, T, problem, k2, dev, stream, flush, barrier, min(args.steps, 20))
            r2["roofline"] = roofline_of(r2, mixed, peaks, peak_src, dmma_peak, dfma_peak)
            r2.pop("step_ms")
            others[k2] = r2

    batched = None
    if rank == 0 and args.batch_jobs > 0:
        batched = measure_batched(args, torch, T, problem, dev, stream, flush, barrier, args.batch_jobs)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(workload(wl), key)
    if rank == 0:
        traffic, traffic_note = hpsi_traffic() if (mixed and key == "C2") else (None, "no DRAM capture for this path")
        roof = roofline_of(res, mixed, peaks, peak_src, dmma_peak, dfma_peak, traffic, traffic_note)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {**config_dict(wl), "D": res["D"],
                       "prec": f"ozaki-bf16 x{args.slices} slices (tcgen05), FP64 Lanczos/eig" if mixed else "fp64",
                       "l2": f"flushed before every step ({FLUSH_BYTES >> 20} MB write)", "parallelism": "replicas"},
            "step_latency_ms": res["step_latency_ms"],
            "hpsi": res["hpsi"],
            "vs_fp64_gpu": res.get("vs_fp64_gpu"),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * run.n1,
                    "d2h_bytes_per_step": 16 * 2 + 8 * run.ne},
            "gpu_launches": launches,
            "step_mode": "CUDA graph replay of one time step (captured from the direct C-ABI calls; the observables on a second stream beside the eigendecomposition)",
            "clocks": res.get("clocks"),
            "other_configs": others or None,
            "batched_jobs": batched,
            "precision_note": "the tensor path is Ozaki integer slicing (exact bf16 slice products, int64 "
                              "recombination); split-FP32 / 3xTF32 and BF16x3 with FP32 accumulation are not "
                              "built: their FP32 accumulation bounds the error near 1e-7, above the 1e-8 target",
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """Continuous batching: a seeded Poisson stream of time-evolution jobs of mixed geometry and size
    through tdmrg_server_* (admission by HBM footprint, per-job streams, CUDA-graph steps)."""
    import torch
    from paper_1103_5391_gb300 import problem
    from paper_1103_5391_gb300 import tdmrg as T
    from workloads import sectors as S
    torch.cuda.set_device(0)
    rng = np.random.default_rng(S.SEED_BASE + 4)
    jobs, t_gen = [], time.perf_counter()
    for k in range(args.jobs):
        L = int(rng.choice(np.arange(16, args.job_lmax + 2, 2)))
        ladder = bool(rng.integers(2))
        U = float(rng.choice([2.0, 4.0, 8.0]))
        m = int(round(np.exp(rng.uniform(np.log(128), np.log(args.job_mmax)))))
        ss = S.make_synthetic(L, m, U, nbonds=2 if ladder else 1, seed=S.SEED_BASE + 100 + k)
        ctx = T.tdmrg_create(device=0, stream=torch.cuda.current_stream().cuda_stream, prec=T.TDMRG_OZAKI_BF16,
                             ozaki_slices=args.slices)
        problem.load_synthetic(ctx, ss)
        psi = torch.as_tensor(ss.psi_gs).cuda()
        phi = torch.zeros(T.tdmrg_sector_size(ctx, ss.Q1), dtype=torch.complex128, device="cuda")
        T.tdmrg_apply_op(ctx, -1, problem.OP_EXC, ss.Q0, psi, ss.Q1, phi)
        jobs.append(dict(L=L, ladder=ladder, U=U, m=m, ss=ss, ctx=ctx, psi=psi, phi=phi))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    gaps = rng.exponential(args.gap_ms * 1e-3, args.jobs)
    srv = T.tdmrg_server_create(0, 0, args.max_active)
    if args.max_group > 1:
        T.tdmrg_server_set_batching(srv, args.max_group, args.batch_window_us)
    nk, steps = WL["nk"], args.job_steps
    ids, peak_running = [], 0
    t0 = time.perf_counter()
    t_next = t0
    for jb, gap in zip(jobs, gaps):
        t_next += gap
        while time.perf_counter() < t_next:
            peak_running = max(peak_running, T.tdmrg_server_stats(srv)[1])
            time.sleep(0.0005)
        ss = jb["ss"]
        ids.append(T.tdmrg_server_submit(srv, jb["ctx"], ss.Q0, jb["psi"], ss.Q1, jb["phi"], WL["tau"], WL["n_v"], nk, steps,
                                         [(problem.OP_N, -1), (-1, problem.OP_N)]))
    done = {}
    while len(done) < len(ids):
        peak_running = max(peak_running, T.tdmrg_server_stats(srv)[1])
        for jid in ids:
            if jid not in done:
                st, n, obs, ms = T.tdmrg_server_poll(srv, jid, steps, 2)
                if st >= T.TDMRG_JOB_DONE:
                    done[jid] = (st, ms)
        time.sleep(0.001)
    makespan = time.perf_counter() - t0
    groups, grouped = T.tdmrg_server_batch_stats(srv)
    T.tdmrg_server_destroy(srv)
    ms = np.concatenate([done[j][1] for j in ids])
    ok = sum(1 for j in ids if done[j][0] == T.TDMRG_JOB_DONE)
    for jb in jobs:
        T.tdmrg_destroy(jb["ctx"])
    line = {"metric": "serving mix: Krylov steps/s and per-step latency", "value": ok * steps * nk / makespan,
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"Poisson stream of {args.jobs} jobs (mean inter-arrival {args.gap_ms:g} ms), chains and "
                                   f"2-leg ladders L in [16, {args.job_lmax}], U in {{2, 4, 8}}, m log-uniform in "
                                   f"[128, {args.job_mmax}], tau=0.05, "
                                   f"n_v=4, n_K=10, {steps} time steps each, ozaki-bf16 x{args.slices}",
                       "max_active": args.max_active, "max_group": args.max_group,
                       "batch_window_us": args.batch_window_us if args.max_group > 1 else None},
            "groups": groups, "grouped_jobs": grouped,
            "jobs_done": ok, "makespan_s": makespan, "peak_running": peak_running,
            "step_latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                                "mean": float(ms.mean())},
            "host_generation_s": t_gen}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_hpsi(args):
    """N applications of H psi on the bench workload, nothing else: after the plan build (two static
    slicing launches, then 4 timed launches of each tile shape x schedule choice per stage: 4 choices,
    or 2 with --tile-m) every application is slice rows, stage-1 GEMM, slice columns, stage-2 GEMM."""
    import torch
    from paper_1103_5391_gb300 import problem, tdmrg as T
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ss = workload()
    prec = T.TDMRG_OZAKI_BF16 if args.prec == "ozaki" else T.TDMRG_FP64
    ctx = T.tdmrg_create(device=0, stream=stream.cuda_stream, prec=prec, ozaki_slices=args.slices)
    try:
        problem.load_synthetic(ctx, ss)
        if args.thin_dim is not None:
            T.tdmrg_set_thin_dim(ctx, args.thin_dim)
        if args.tile_m:
            T.tdmrg_set_tile_m(ctx, args.tile_m)
        n = T.tdmrg_sector_size(ctx, ss.Q1)
        x = torch.randn(n, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        for _ in range(args.profile_hpsi):
            T.tdmrg_apply_h(ctx, ss.Q1, x, y)
        torch.cuda.synchronize()
    finally:
        T.tdmrg_destroy(ctx)
    print(json.dumps({"profile_hpsi": args.profile_hpsi, "D": n, "prec": args.prec}), flush=True)
    return 0


def run_precision_errors(args):
    """Relative errors of H psi and of one time step's targets on the tensor path with S = 2..6 slices,
    against the FP64 GPU path (itself checked against the oracle in the tests), on the L=48 U=10 m=1000
    chain twin (tau = 0.02, n_v = 4, n_K = 10)."""
    import torch
    from paper_1103_5391_gb300 import problem, tdmrg as T
    from workloads import sectors
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ss = sectors.make_synthetic(48, 1000, 10.0, nbonds=1, seed=sectors.SEED_BASE + 4)
    times = [x * 0.02 / 3 for x in range(4)]
    g = torch.Generator(device="cpu").manual_seed(11)
    res = {}
    for S in (0, 2, 3, 4, 5, 6):   # 0: the FP64 path
        prec = T.TDMRG_FP64 if S == 0 else T.TDMRG_OZAKI_BF16
        ctx = T.tdmrg_create(device=0, stream=stream.cuda_stream, prec=prec, ozaki_slices=S if S else 4)
        try:
            problem.load_synthetic(ctx, ss)
            n = T.tdmrg_sector_size(ctx, ss.Q1)
            if S == 0:
                x = torch.complex(torch.randn(n, generator=g, dtype=torch.float64),
                                  torch.randn(n, generator=g, dtype=torch.float64)).cuda()
                phi = torch.as_tensor(ss.phi).cuda()
            y = torch.zeros_like(x)
            T.tdmrg_apply_h(ctx, ss.Q1, x, y)
            tg = [torch.zeros_like(phi) for _ in times]
            T.tdmrg_evolve(ctx, ss.Q1, phi, times, 10, tg)
            torch.cuda.synchronize()
            if S == 0:
                y0, t0 = y, tg[-1]
            else:
                res[S] = {"hpsi": float((y - y0).abs().max() / y0.abs().max()),
                          "target": float((tg[-1] - t0).abs().max() / t0.abs().max())}
        finally:
            T.tdmrg_destroy(ctx)
    print(json.dumps({"precision_errors": res, "workload": "L=48 U=10 m=1000 chain twin, D = %d" % n,
                      "reference": "FP64 GPU path", "step": "tau = 0.02, n_v = 4, n_K = 10"}), flush=True)
    return 0


def main():
    args = parse()
    if args.oracle_rate:
        wl = CONFIGS[args.oracle_rate]
        best, n, ks, dt = oracle_rate(workload(wl), wl)
        print(json.dumps({"value": best, "sample": f"best of 5 blocks, {n} time steps ({ks} Krylov steps) in {dt:.1f} s "
                                                    f"on one core, one BLAS thread"}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_hpsi > 0:
        return run_profile_hpsi(args)
    if args.precision_errors:
        return run_precision_errors(args)
    if args.serving:
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
