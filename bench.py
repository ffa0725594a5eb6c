#!/usr/bin/env python3
"""Throughput of the batched Parallel-Tempering path (smoothed-cubic 4-body random-laser model).

Workload (one GPU): N = 256 modes, 16 disorder samples x 48 temperatures (geometric 0.25-1.6) x 2
replicas = 1536 chains, FP32 amplitudes/fields with FP64 energies.  One step = one swap interval:
64 sweeps of every chain, the FP64-accumulated resync, 4 measurements (E, Y2, Y4, q histogram) and a
swap pass.  Metric: chain-sweeps/s.  Inputs are synthetic (Gaussian couplings, sigma_J = 1/N, on the
comb graph); the coupling store (16 x 22 MB) is larger than L2, so no flush is needed between steps.

Also reported: the plain FP64 GPU sweep (the paper's design) on the same workload, the roofline of
the sweep kernel, an end-to-end number through host buffers, and the FP64 CPU oracle on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEP_SWEEPS = 64
N_MODES = 256
CPU_SAMPLE_SECONDS = 15.0


# ------------------------------------------------------------------------------------------- accounting
METRIC = "chain-sweeps/s at N=256 vs plain FP64; eff. samples/s learned vs plain PT"


def flops_per_chain_sweep(N: int) -> float:
    """Algorithmic FP32 flops of one sweep (N/2 pair updates) of the pair-factored field evaluation,
    averaged exactly over the pair distribution (j uniform, k uniform among the other modes):
    per pair product z = a_x a_y (6 flops) used by either field, per coupling term acc += J z (4),
    per field row h += conj(a_m) acc (8)."""
    s = np.arange(2 * N - 1)
    m = np.array([max(0, (ss - 1) // 2 - max(0, ss - (N - 1)) + 1) if ss >= 1 else 0 for ss in s])
    K = np.arange(N)
    tot = 0.0
    for j in range(N):
        inj = (s - j >= 0) & (s - j < N) & (s != 2 * j)
        kk = K[K != j]
        ink = (s[None, :] - kk[:, None] >= 0) & (s[None, :] - kk[:, None] < N) & (s[None, :] != 2 * kk[:, None])
        tj = np.where(inj, m - 1, 0)[None, :]
        tk = np.where(ink, m[None, :] - 1, 0)
        both = inj[None, :] & ink
        union = np.where(both, np.where(s[None, :] == j + kk[:, None], m - 1, m), np.where(inj[None, :] | ink, m - 1, 0))
        rows = (tj > 0).sum() * len(kk) + (tk > 0).sum()
        tot += 6.0 * union.sum() + 4.0 * (tj.sum() * len(kk) + tk.sum()) + 8.0 * rows
    return tot / (N * (N - 1)) * (N / 2)


def count_quads(N: int) -> int:
    """|Q| of the N-mode comb: pairs {x<y} grouped by their sum s; every two pairs of one sum make one
    quadruplet."""
    m = np.zeros(2 * N, np.int64)
    for x in range(N):
        for y in range(x + 1, N):
            m[x + y] += 1
    return int((m * (m - 1) // 2).sum())


def survey_flops_per_chain_sweep(N: int) -> float:
    """Algorithmic work of one chain-sweep as the hot-path scope counts it: 4|Q| coupling terms (every term
    is visited by each of its 4 modes once per sweep on average: N/2 pair updates x 2 fields x 4|Q|/N
    terms), 16 FP32 flops each (two complex multiplies, a real scale, an add)."""
    return 16.0 * 4.0 * count_quads(N)


def kernel_code_sha(path):
    """sha1 (12 hex digits) of a CUDA source with its comments and white space removed: the key under which a
    profile's counters stay valid (a comment edit leaves the compiled kernels unchanged)."""
    import hashlib
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha1(src.encode()).hexdigest()[:12]


def profiled_traffic():
    """DRAM bytes per bench sweep launch from the committed ncu summary, or None if the kernel code changed
    since the counters were taken."""
    try:
        txt = open(os.path.join(ROOT, "profiles", "sweep_kernel_n256.md")).read()
        sha = kernel_code_sha(os.path.join(ROOT, "paper_2511_13508_gb300", "csrc", "pt_sweep.cu"))
    except OSError:
        return None
    if ("code sha1 prefix `%s`" % sha) not in txt:
        return None
    for line in txt.splitlines():
        if line.startswith("traffic_bytes_per_bench_launch:"):
            return float(line.split(":")[1])
    return None


def peak_fp32_tflops(sm_count=152, mhz=2070.0):
    """FP32 FMA peak from unit counts: SMs x 128 FP32 lanes x 2 flops x clock (context for the measured one)."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def measure_fp32_peak(reps=3, target_ms=60.0):
    """Measured FP32 fused multiply-add throughput (pt_fma_probe): 8 resident blocks of 256 threads per SM
    (SM count read from the device), each thread 8 independent chains; packed (paired FMA) and scalar
    variants, one warm-up launch each, then `reps` launches timed with CUDA events on one stream; the
    larger rate is the peak.  Returns TFLOP/s and the details."""
    import torch
    import paper_2511_13508_gb300 as pkg
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = int(props.multi_processor_count)
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"sm_count": sms, "blocks": blocks, "threads": threads}
    for packed in (1, 0):
        iters = 2000
        for _ in range(3):  # calibrate the launch to about target_ms
            pkg.fma_probe(packed, blocks, threads, iters, sink.data_ptr(), stream.cuda_stream)
            ev0.record(stream)
            pkg.fma_probe(packed, blocks, threads, iters, sink.data_ptr(), stream.cuda_stream)
            ev1.record(stream)
            stream.synchronize()
            ms = ev0.elapsed_time(ev1)
            iters = max(100, int(iters * target_ms / max(ms, 1e-3)))
        ev0.record(stream)
        for _ in range(reps):
            pkg.fma_probe(packed, blocks, threads, iters, sink.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        stream.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        out["packed" if packed else "scalar"] = blocks * threads * iters * 32.0 * reps / sec / 1e12
        out["iters"] = iters
    out["tflops"] = max(out["packed"], out["scalar"])
    return out


# ------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index=0):
        self.rows, self.proc, self.idx = [], None, gpu_index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows if len(r) >= 8 for n, v in zip(names, r[4:8]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    N, nq, seed, sweeps, temps = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2511_13508_gb300 import workload
    J = workload.couplings(N, nq, seed)
    pt = oracle.OraclePT([N], [J], temps, 1, 17, swap_every=0, measure_every=16, resync_every=64)
    t0 = time.perf_counter()
    pt.sweep(sweeps)
    return sweeps * len(temps), time.perf_counter() - t0


def cpu_oracle_rate(target_seconds=CPU_SAMPLE_SECONDS, workers=None):
    """Oracle chain-sweeps/s on the host cores: independent processes (spawned), each running a few
    N=256 chains of the same workload for a bounded number of sweeps."""
    workers = workers or os.cpu_count() or 1
    import oracle
    nq = len(oracle.enumerate_quads(N_MODES))
    # calibrate: one chain, one sweep
    t_one = _oracle_worker((N_MODES, nq, 301, 1, [0.25]))[1]
    per_worker = max(1, int(target_seconds / max(t_one, 1e-3)))
    temps = [0.25, 1.6]
    sweeps = max(1, per_worker // len(temps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(N_MODES, nq, 301 + i, sweeps, temps) for i in range(workers)])
        wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    return {"value": done / wall, "unit": "chain-sweeps/s", "cores": workers, "kind": "oracle",
            "sample": "%d processes x %d chains (N=256, T=0.25 and 1.6) x %d sweeps, FP64, single-threaded each"
                      % (workers, len(temps), sweeps)}


# ------------------------------------------------------------------------------------------- ranks
def rank_seeds(seeds, rank):
    """Weak scaling: every rank simulates its own disorder samples (seed ranges 1000 apart); samples are
    independent problems, so the data path needs no collective."""
    return [int(s) + 1000 * int(rank) for s in seeds]


def max_over_ranks(value, dist, device="cpu"):
    """The timing rule: the slowest rank's time (all-reduce MAX; identity on one rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / (ms / 1e3)


def _free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_entry(rank, world, port, target, args, init_group, backend):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), LOCAL_WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist = None
    if init_group:
        import torch.distributed as dist
        dist.init_process_group(backend, rank=rank, world_size=world)
    try:
        rc = target(rank, world, dist, *args)
    finally:
        if dist is not None:
            dist.destroy_process_group()
    sys.exit(int(rc or 0))


def spawn_ranks(world, target, args=(), init_group=True, backend="gloo", timeout=3600.0):
    """One process per rank on this node (spawned, so no CUDA state is inherited), each with RANK, LOCAL_RANK,
    WORLD_SIZE and MASTER_ADDR/PORT (127.0.0.1) set as a launcher would, running target(rank, world, dist,
    *args) (dist: the joined process group when init_group, else None and the target joins it).  Returns the
    exit codes in rank order."""
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_entry, args=(r, world, port, target, tuple(args), init_group, backend))
             for r in range(world)]
    for p in procs:
        p.start()
    t0 = time.time()
    for p in procs:
        p.join(timeout=max(1.0, timeout - (time.time() - t0)))
    codes = []
    for p in procs:
        if p.is_alive():
            p.terminate()
            p.join(timeout=10)
            codes.append(-1)
        else:
            codes.append(p.exitcode)
    return codes


def _bench_rank(rank, world, dist, argv):
    """A rank started by `bench.py --gpus N` itself: the same path as under torchrun."""
    return main(argv)


# ------------------------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, dist):
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload

    torch.cuda.set_device(rank % torch.cuda.device_count())
    pkg.build()
    W = workload.workloads()["n256_large"]
    nq = len(pkg.enumerate_quads(N_MODES))
    seeds = rank_seeds(W.seeds, rank)  # weak scaling: every rank its own 16 samples
    Js = [workload.couplings(N_MODES, nq, s) for s in seeds]
    stream = torch.cuda.Stream()
    kw = dict(swap_every=W.swap_every, measure_every=W.measure_every, resync_every=W.resync_every)
    pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 12345 + rank, precision="fp32", stream=stream, **kw)
    chains = pt.n_chains

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        pt.sweep(STEP_SWEEPS)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            pt.sweep(STEP_SWEEPS)
        ev1.record(stream)
        barrier()
    pt.sync()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, dist, device="cuda")
    value = whole_job_rate(chains * STEP_SWEEPS * args.steps, world, ms)

    # ---- sweep kernel alone (roofline): one launch of 64 sweeps without measurement/resync/swap
    pk = pkg.PT(W.Ns, Js, W.temps, W.replicas, 777, precision="fp32", stream=stream, swap_every=0,
                measure_every=0, resync_every=0, use_graphs=False)
    pk.sweep(STEP_SWEEPS)
    pk.sync()
    reps = 3
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        pk.sweep(STEP_SWEEPS)
    ev1.record(stream)
    torch.cuda.synchronize()
    kms = ev0.elapsed_time(ev1) / reps
    fl_exec = flops_per_chain_sweep(N_MODES) * chains * STEP_SWEEPS
    fl = survey_flops_per_chain_sweep(N_MODES) * chains * STEP_SWEEPS
    clocks = clk.summary()
    pk.close()
    probe = measure_fp32_peak()
    peak = probe["tflops"]
    achieved = fl / (kms / 1e3) / 1e12
    achieved_exec = fl_exec / (kms / 1e3) / 1e12

    # ---- plain FP64 GPU sweep (paper's design) on the same workload, bounded sample
    pp = pkg.PT(W.Ns, Js, W.temps, W.replicas, 4242, precision="fp64_plain", stream=stream, **kw)
    pp.sweep(1)
    pp.sync()
    torch.cuda.synchronize()
    ev0.record(stream)
    pp.sweep(2)
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_rate = chains * 2 / (ev0.elapsed_time(ev1) / 1e3)
    pp.close()

    # ---- end to end through host buffers: state in (h2d), one step, observables + state out (d2h)
    a_host, _ = pt.state()
    a_host = np.ascontiguousarray(a_host)
    pt.sync()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 2)
    for _ in range(e2e_steps):
        pt.set_state(a_host)
        pt.sweep(STEP_SWEEPS)
        obs = pt.observables()
        a_host, _ = pt.state()
    wall = time.perf_counter() - t0
    h2d = a_host.size * 8  # FP32 complex amplitudes uploaded
    d2h = sum(v.nbytes for v in obs.values()) + a_host.size * 8 + chains * 8
    e2e = {"value": chains * STEP_SWEEPS * e2e_steps * world / wall, "unit": "chain-sweeps/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    pt.close()
    return dict(value=value, ms=ms, kms=kms, achieved=achieved, achieved_exec=achieved_exec, peak=peak, probe=probe,
                clocks=clocks, plain_rate=plain_rate, e2e=e2e, fl=fl, fl_exec=fl_exec)


def learned_leg(t_min=None, global_every=None, series=4096, burn_in=4096):
    """Effective samples/s at the coldest temperature, learned global move vs plain PT, on the learned-proposal
    workload (N=64, 16 samples x 32 T [0.3,1.6] x 2 replicas; 2^14 training configurations per sample from
    the 8 coldest temperatures; a global move every 8 sweeps).  t_min / global_every move the ladder's cold
    end and the move's period (the colder leg: where plain PT is slow)."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import gain, workload
    W = workload.workloads()["n64_learned"]
    nq = len(pkg.enumerate_quads(W.Ns[0]))
    Js = [workload.couplings(W.Ns[0], nq, s) for s in W.seeds]
    tmin = W.t_min if t_min is None else t_min
    temps = workload.geometric_ladder(tmin, W.t_max, W.n_temps)
    every = W.extra["global_every"] if global_every is None else global_every
    pt = pkg.PT(W.Ns, Js, temps, W.replicas, 4401, precision="fp32", stream=torch.cuda.Stream(),
                swap_every=W.swap_every, measure_every=W.measure_every, resync_every=W.resync_every)
    r = gain.measure(pt, n_cold=W.extra["n_cold"], global_every=every,
                     train_configs=W.extra["train_configs"], train_steps=6000, series=series, burn_in=burn_in)
    pt.close()
    r["workload"] = "N=64 comb, 16 samples x 32 T [%g,%g] x 2 replicas, FP32" % (tmin, W.t_max)
    r["unit"] = "effective samples/s of E (and of q^2) at the coldest T"
    return r


def graph_leg(sweeps=64, plain_sweeps=4):
    """The paper's own graph: random mode frequencies with the matching condition of linewidth
    1/(2(N-1)) (N = 64, 16 samples x 32 T [0.3,1.6] x 2 replicas): the FP32 group kernels and, on a bounded
    sample, the FP64 quadruplet-list path; CUDA events on the library's stream."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    N, S, R = 64, 16, 2
    temps = workload.geometric_ladder(0.3, 1.6, 32)
    graphs = [pkg.fmc_graph(workload.random_frequencies(N, 500 + s)) for s in range(S)]
    Js = [workload.couplings(N, len(g), 600 + s) for s, g in enumerate(graphs)]
    out = {}
    for prec, n in (("fp32", sweeps), ("fp64_plain", plain_sweeps)):
        stream = torch.cuda.Stream()
        pt = pkg.PT([N] * S, Js, temps, R, 31, precision=prec, stream=stream, graphs=graphs,
                    swap_every=64, measure_every=16, resync_every=64)
        pt.sweep(2)
        pt.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pt.sweep(n)
        ev1.record(stream)
        torch.cuda.synchronize()
        out[prec] = pt.n_chains * n / (ev0.elapsed_time(ev1) / 1e3)
        pt.close()
    # a sparse mode-locked graph far beyond the comb's size: N = 2048, 16 quadruplets per mode
    Ns2 = 2048
    sg = [workload.sparse_comb_graph(Ns2, 16, 700 + s) for s in range(S)]
    sJ = [workload.couplings(Ns2, len(g), 800 + s) * Ns2 for s, g in enumerate(sg)]
    stream = torch.cuda.Stream()
    pt = pkg.PT([Ns2] * S, sJ, temps, R, 37, precision="fp32", stream=stream, graphs=sg,
                swap_every=64, measure_every=16, resync_every=64)
    pt.sweep(1)
    pt.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    pt.sweep(4)
    ev1.record(stream)
    torch.cuda.synchronize()
    sparse = pt.n_chains * 4 / (ev0.elapsed_time(ev1) / 1e3)
    pt.close()
    return {"workload": "N=64 random-frequency mode-locked graph (gamma = 1/(2(N-1))), 16 samples x 32 T x 2 "
                        "replicas", "value": out["fp32"], "unit": "chain-sweeps/s", "path": "FP32 group kernels",
            "fp64_plain_value": out["fp64_plain"],
            "quadruplets_per_sample_mean": float(np.mean([len(g) for g in graphs])),
            "sweeps": sweeps, "plain_sweeps": plain_sweeps,
            "sparse_n2048_z16": {"value": sparse, "unit": "chain-sweeps/s", "sweeps": 4,
                                 "workload": "N=2048 sparse comb graph, 16 quadruplets per mode, 16 samples x 32 T "
                                             "x 2 replicas, FP32 group kernels"}}


def workloads_leg(sweeps=64, peak32=None):
    """The other synthetic workloads at 1 GPU, each a PT run with its own swap (64), measurement (16) and
    resync (64) schedule: chain-sweeps/s from CUDA events on the library's stream over `sweeps` sweeps after
    2 warm-up sweeps, and the achieved fraction of the derived peak (FP32, or FP64 for the FP64 path) from
    the same algorithmic flop count as the roofline of the main line.  The ragged batch runs the shape the
    autotuner picks on it."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    Wall = workload.workloads()
    fl_cache = {}
    peak64 = 152 * 2 * 2 * 2070.0 * 1e6 / 1e12  # 2 FP64 FMA per SM per clock (nominal 1.25 TFLOP/s)
    out = {}
    for key, name, prec, tune in (("n16_fp64", "n16_fp64", "fp64", False), ("n64_batched_fp32", "n64_batched", "fp32", False),
                                  ("n64_batched_fp64", "n64_batched", "fp64", False), ("ragged_fp32", "ragged", "fp32", True)):
        W = Wall[name]
        Js = [workload.couplings(n, len(pkg.enumerate_quads(n)), sd) for n, sd in zip(W.Ns, W.seeds)]
        stream = torch.cuda.Stream()
        pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 51, precision=prec, stream=stream, swap_every=64,
                    measure_every=16, resync_every=64)
        shape = pt.autotune() if tune else None
        pt.sweep(2)
        pt.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pt.sweep(sweeps)
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        per_chain = W.replicas * len(W.temps)
        fl = fl_x = 0.0
        for n in W.Ns:
            if n not in fl_cache:
                fl_cache[n] = (survey_flops_per_chain_sweep(n), flops_per_chain_sweep(n))
            fl += fl_cache[n][0] * per_chain * sweeps
            fl_x += fl_cache[n][1] * per_chain * sweeps
        if prec == "fp32":
            peak = peak32 if peak32 else peak_fp32_tflops()
            basis = "measured FP32 FMA peak (pt_fma_probe)" if peak32 else "FP32 unit-count peak at 2070 MHz"
        else:
            peak, basis = peak64, "2 FP64 FMA/SM/clock x 152 SMs x 2070 MHz"
        achieved = fl / sec / 1e12
        out[key] = {"value": pt.n_chains * sweeps / sec, "unit": "chain-sweeps/s", "precision": prec,
                    "chains": pt.n_chains, "N": sorted(set(int(n) for n in W.Ns)), "sweeps": sweeps,
                    "achieved_tflops": achieved, "peak_tflops": peak, "frac": achieved / peak,
                    "frac_executed": fl_x / sec / 1e12 / peak,
                    "flop_count": "16 flops x 4|Q| per chain-sweep (frac); pair-factored executed count (frac_executed)",
                    "peak_basis": basis, "autotuned_shape": list(shape) if shape else None}
        pt.close()
    return out


def _oracle_calibrate(N, nq):
    """Seconds per chain-sweep of the oracle at N (one chain, enough sweeps for about 0.2 s)."""
    sw = 1
    while True:
        _, t = _oracle_worker((N, nq, 301, sw, [0.5]))
        if t > 0.2 or sw > 1 << 16:
            return t / sw
        sw *= 4


def oracle_rate_mixed(Ns, target_seconds=3.0, workers=None):
    """Oracle chain-sweeps/s on the host cores for a workload of mode counts Ns: one spawned process per core,
    process i simulating two chains (T = 0.5 and 1.5) of one sample with N = Ns[i mod len(Ns)] for about
    target_seconds."""
    import oracle
    workers = workers or os.cpu_count() or 1
    Ns = [int(n) for n in Ns]
    nqs = {n: len(oracle.enumerate_quads(n)) for n in set(Ns)}
    cost = {n: _oracle_calibrate(n, nqs[n]) for n in set(Ns)}
    jobs = []
    for i in range(workers):
        n = Ns[i % len(Ns)]
        jobs.append((n, nqs[n], 501 + i, max(1, int(target_seconds / cost[n] / 2)), [0.5, 1.5]))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    return sum(r[0] for r in res) / wall, workers


def baseline_table_leg(main_line):
    """Every synthetic workload on every implementation, for the baseline table: the FP32 J-sharing path
    (64 sweeps with the workload's schedule), the FP64 J-sharing path and the plain FP64 path (the paper's
    design; bounded samples of sweeps), all timed with CUDA events on the library's stream, and the FP64 oracle
    on the host cores (bounded sample).  chain-sweeps/s each."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    Wall = workload.workloads()
    out = {}
    plan = {"n16_fp64": (64, 64, 16), "n64_batched": (64, 8, 2), "ragged": (64, 8, 2), "n256_large": (0, 1, 0),
            "n64_learned": (64, 8, 2)}
    for name, (s32, s64, splain) in plan.items():
        W = Wall[name]
        Js = [workload.couplings(n, len(pkg.enumerate_quads(n)), sd) for n, sd in zip(W.Ns, W.seeds)]
        row = {"N": sorted(set(int(n) for n in W.Ns)), "chains": W.chains}
        for prec, sw in (("fp32", s32), ("fp64", s64), ("fp64_plain", splain)):
            if sw == 0:
                continue
            stream = torch.cuda.Stream()
            pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 71, precision=prec, stream=stream, swap_every=64,
                        measure_every=16, resync_every=64)
            pt.sweep(1)
            pt.sync()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            pt.sweep(sw)
            ev1.record(stream)
            torch.cuda.synchronize()
            row[prec] = pt.n_chains * sw / (ev0.elapsed_time(ev1) / 1e3)
            row[prec + "_sweeps"] = sw
            pt.close()
        if name == "n256_large":
            row["fp32"] = main_line["value"]
            row["fp64_plain"] = main_line["plain_rate"]
        row["oracle"], row["oracle_cores"] = oracle_rate_mixed(W.Ns)
        out[name] = row
    return out


def precision_leg(burn=512, sweeps=4096):
    """FP32 against FP64 on the batched N=64 workload (64 samples x 32 T [0.3,1.6] x 2 replicas; each path's
    default block shape): the same couplings and seeds (common random numbers), `burn` sweeps, then `sweeps`
    sweeps measured every 16.  Per observable the disorder-averaged FP32 - FP64 difference per temperature
    with its paired jackknife error over samples (analysis.paired_difference), summarised over temperatures.
    The FP64 J-sharing path follows the oracle's chain to 1e-9, so it stands for the oracle here."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import analysis, workload
    W = workload.workloads()["n64_batched"]
    nq = len(pkg.enumerate_quads(64))
    Js = [workload.couplings(64, nq, sd) for sd in W.seeds]
    obs, secs = {}, {}
    for prec in ("fp32", "fp64"):
        pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 61, precision=prec, stream=torch.cuda.Stream(),
                    swap_every=64, measure_every=16, resync_every=64)
        t0 = time.perf_counter()
        pt.sweep(burn)
        pt.reset_observables()
        pt.sweep(sweeps)
        obs[prec] = pt.observables()
        secs[prec] = time.perf_counter() - t0
        pt.close()
    d = analysis.paired_difference(obs["fp32"], obs["fp64"], W.temps, 64)
    summ = analysis.difference_summary(d)
    tmin = {k: {"diff": float(v["diff"][0]), "err": float(v["err"][0]), "ref": float(v["ref"][0])}
            for k, v in d.items() if k != "Pq"}
    return {"workload": "n64_batched: N=64 comb, 64 samples x 32 T [0.3,1.6] x 2 replicas",
            "burn": burn, "sweeps": sweeps, "measure_every": 16,
            "reference": "FP64 J-sharing GPU path, same seeds (follows the FP64 oracle's chain to 1e-9)",
            "observables": "E/N, C_V/N, <q^2>, <q^4>, Y2, Y4 per (sample, T); P_J(q) on 20 coarse bins",
            "summary": summ, "at_T_min": tmin, "wall_s": secs}


def ladder_leg():
    """App. A: specific heat on a ladder of fixed Delta T (N = 64 comb, 8 samples x 32 T [0.2,1.6] x 2
    replicas), the ladder T_i = T_{i-1}/(1 - 0.6/sqrt(C_V(T_i))), and the swap acceptance per neighbouring
    pair on it and on a geometric ladder of the same size and end points."""
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import analysis, workload
    N, S, R = 64, 8, 2
    Js = [workload.couplings(N, len(pkg.enumerate_quads(N)), 800 + s) for s in range(S)]

    def rates(temps, sweeps=8192, burn=2048):
        pt = pkg.PT([N] * S, Js, temps, R, 5, precision="fp32", swap_every=16, measure_every=4, resync_every=64)
        pt.sweep(burn)
        pt.reset_observables()
        pt.sweep(sweeps)
        o = pt.observables()
        acc = o["swap_acc"].sum((0, 1)) / np.maximum(o["swap_att"].sum((0, 1)), 1)
        cv, _ = analysis.specific_heat(o, temps)
        pt.close()
        return acc, cv

    Tlin = np.linspace(0.2, 1.6, 32)
    _, cv = rates(Tlin)
    Tad = analysis.adaptive_ladder(Tlin, cv, 0.2, 1.6, 0.6)
    Tgeo = workload.geometric_ladder(0.2, 1.6, len(Tad))
    a_ad, _ = rates(Tad)
    a_geo, _ = rates(Tgeo)
    inner = slice(0, len(Tad) - 2)
    stat = lambda a: {"mean": float(a[inner].mean()), "min": float(a[inner].min()),
                      "rel_spread": float(a[inner].std() / a[inner].mean())}
    return {"workload": "N=64 comb, 8 samples x 2 replicas, C = 0.6, T in [0.2, 1.6]", "n_temps": len(Tad),
            "temps": [round(float(t), 4) for t in Tad], "adaptive": stat(a_ad), "geometric": stat(a_geo)}


def profile_case():
    """Three launches of the sweep kernel (one sweep each) on half the bench workload: 8 samples
    (176 MB of couplings, larger than L2), 768 chains; no measurement, resync or swap."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    pkg.build()
    W = workload.workloads()["n256_large"]
    nq = len(pkg.enumerate_quads(N_MODES))
    Js = [workload.couplings(N_MODES, nq, s) for s in W.seeds[:8]]
    pt = pkg.PT(W.Ns[:8], Js, W.temps, W.replicas, 5, precision="fp32", swap_every=0, measure_every=0,
                resync_every=0, use_graphs=False)
    for _ in range(3):
        pt.sweep(1)
    pt.sync()
    print("profile case done")
    return 0


def profile_small():
    """Small cases for ncu, a few launches each: the batched N=64 workload itself (64 samples x 32 T x 2
    replicas on the FP32 default 32 x 11 blocks: three 1-sweep launches; 26 MB of couplings, held by the L2 as
    in the timed runs), the ragged batch (96 samples, N in {32 .. 128}, 24 T x 2 replicas, default 16 x 11
    blocks: three 1-sweep launches), then on N=256 (8 samples x 48 T x 2 replicas, 199 MB of couplings) one swap interval
    of 16 sweeps with its resync (energy_kernel), measurement (measure_kernel) and swap pass (swap_kernel),
    and the plain FP64 sweep (plain_sweep_kernel, the paper's design) for one sweep on 2 samples of N=64."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    pkg.build()
    Wb = workload.workloads()["n64_batched"]
    nq64 = len(pkg.enumerate_quads(64))
    Js = [workload.couplings(64, nq64, s) for s in Wb.seeds]
    pt = pkg.PT(Wb.Ns, Js, Wb.temps, 2, 5, precision="fp32", chains_per_block=32, consumer_warps=11,
                swap_every=0, measure_every=0, resync_every=0, use_graphs=False)
    for _ in range(3):
        pt.sweep(1)
    pt.sync()
    pt.close()
    Wr = workload.workloads()["ragged"]
    Js = [workload.couplings(n, len(pkg.enumerate_quads(n)), s) for n, s in zip(Wr.Ns, Wr.seeds)]
    pt = pkg.PT(Wr.Ns, Js, Wr.temps, Wr.replicas, 5, precision="fp32", swap_every=0, measure_every=0,
                resync_every=0, use_graphs=False)
    for _ in range(3):
        pt.sweep(1)
    pt.sync()
    pt.close()
    W = workload.workloads()["n256_large"]
    nq = len(pkg.enumerate_quads(N_MODES))
    Js = [workload.couplings(N_MODES, nq, s) for s in W.seeds[:8]]
    pt = pkg.PT(W.Ns[:8], Js, W.temps, W.replicas, 5, precision="fp32", swap_every=16, measure_every=16,
                resync_every=16, use_graphs=False)
    pt.sweep(16)
    pt.sync()
    pt.close()
    pp = pkg.PT([64] * 2, [workload.couplings(64, nq64, s) for s in (1, 2)], Wb.temps, 2, 5,
                precision="fp64_plain", swap_every=0, measure_every=0, resync_every=0, use_graphs=False)
    pp.sweep(1)
    pp.sync()
    pp.close()
    print("profile small done")
    return 0


def profile_global():
    """Eight learned global-move rounds on the learned-proposal workload (N=64, 16 samples x 32 T x 2 replicas,
    8 coldest temperatures, a round every 8 sweeps; untrained network): 64 sweeps.  For the launch list of a
    round."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    pkg.build()
    W = workload.workloads()["n64_learned"]
    nq = len(pkg.enumerate_quads(W.Ns[0]))
    Js = [workload.couplings(W.Ns[0], nq, s) for s in W.seeds]
    pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 4401, precision="fp32", stream=torch.cuda.Stream(),
                swap_every=W.swap_every, measure_every=W.measure_every, resync_every=W.resync_every)
    pt.learn_init(n_cold=W.extra["n_cold"], batch=512, data_per_sample=W.extra["train_configs"], seed=1)
    pt.set_global_every(W.extra["global_every"])
    pt.sweep(64)
    pt.sync()
    pt.close()
    print("profile global done")
    return 0


def profile_graph():
    """The graph legs' FP32 group kernels, a few launches each: the N=64 random-frequency graph (16 samples x
    32 T x 2 replicas, 2 sweeps per launch) and the N=2048 sparse comb graph (z = 16, 1 sweep per launch)."""
    import torch
    import paper_2511_13508_gb300 as pkg
    from paper_2511_13508_gb300 import workload
    pkg.build()
    S, R = 16, 2
    temps = workload.geometric_ladder(0.3, 1.6, 32)
    kw = dict(swap_every=0, measure_every=0, resync_every=0, use_graphs=False)
    graphs = [pkg.fmc_graph(workload.random_frequencies(64, 500 + s)) for s in range(S)]
    Js = [workload.couplings(64, len(g), 600 + s) for s, g in enumerate(graphs)]
    pt = pkg.PT([64] * S, Js, temps, R, 31, precision="fp32", graphs=graphs, **kw)
    for _ in range(3):
        pt.sweep(2)
    pt.sync()
    pt.close()
    sg = [workload.sparse_comb_graph(2048, 16, 700 + s) for s in range(S)]
    sJ = [workload.couplings(2048, len(g), 800 + s) * 2048 for s, g in enumerate(sg)]
    pt = pkg.PT([2048] * S, sJ, temps, R, 37, precision="fp32", graphs=sg, **kw)
    for _ in range(2):
        pt.sweep(1)
    pt.sync()
    pt.close()
    print("profile graph done")
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal ESS comparison")
    ap.add_argument("--no-graph", action="store_true", help="skip the random-frequency graph leg")
    ap.add_argument("--no-ladder", action="store_true", help="skip the adaptive-ladder leg")
    ap.add_argument("--no-workloads", action="store_true", help="skip the leg of the other synthetic workloads")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32-vs-FP64 observable comparison")
    ap.add_argument("--no-table", action="store_true", help="skip the every-workload x every-implementation table")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for ncu: N=256, 8 samples x 48 T x 2 replicas, three 1-sweep launches")
    ap.add_argument("--profile-small", action="store_true",
                    help="small cases for ncu: N=64 on 32 x 11 blocks, the ragged batch on 16 x 11, the N=256 "
                         "resync/measure/swap kernels, the plain FP64 sweep")
    ap.add_argument("--profile-global", action="store_true",
                    help="run eight learned global-move rounds (for the launch list of a round) and exit")
    ap.add_argument("--profile-graph", action="store_true",
                    help="a few launches of the graph kernels (N=64 random graph, N=2048 sparse graph) and exit")
    args = ap.parse_args(argv)
    if args.profile_case:
        return profile_case()
    if args.profile_small:
        return profile_small()
    if args.profile_global:
        return profile_global()
    if args.profile_graph:
        return profile_graph()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start one rank per GPU here (weak scaling, samples sharded by rank_seeds)
        if args.impl == "gb300":
            import torch
            if torch.cuda.device_count() < args.gpus:
                print("bench.py: --gpus %d but %d CUDA devices visible" % (args.gpus, torch.cuda.device_count()),
                      file=sys.stderr)
                return 2
        codes = spawn_ranks(args.gpus, _bench_rank, (list(sys.argv[1:] if argv is None else argv),),
                            init_group=False)
        return 0 if all(c == 0 for c in codes) else 1
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cfg = {"workload": "n256_large: N=256 comb, 16 samples x 48 T [0.25,1.6] x 2 replicas, FP32 fields",
           "samples_per_gpu": 16, "temps": 48, "replicas": 2, "N": N_MODES, "step": "64 sweeps + resync + "
           "4 measurements + swap pass", "l2": "inputs larger than L2 (398 MB blocked coupling store: 16 x 24.9 MB)"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        # the reference arm is the FP64 CPU oracle, bounded per step
        per = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
        for _ in range(args.warmup):
            cpu_oracle_rate(target_seconds=per / 4)
        vals = [cpu_oracle_rate(target_seconds=per) for _ in range(args.steps)]
        v = statistics.mean(x["value"] for x in vals)
        line = {"metric": METRIC, "value": v, "unit": "chain-sweeps/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "impl": "reference",
                "cpu_baseline": {"value": v, "unit": "chain-sweeps/s", "cores": vals[0]["cores"], "kind": "oracle",
                                 "sample": vals[0]["sample"]},
                "e2e": {"value": v, "unit": "chain-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    # CPU baseline first (spawned processes, before the first GPU call)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate()

    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)) % torch.cuda.device_count())
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    r = run_gpu(args, rank, world, dist)
    learned = learned_cold = None
    if rank == 0 and world == 1 and not args.no_learned:
        learned = learned_leg()
        learned_cold = learned_leg(t_min=0.05, global_every=16, series=8192, burn_in=1 << 15)
    graph = None
    if rank == 0 and world == 1 and not args.no_graph:
        graph = graph_leg()
    ladder = None
    if rank == 0 and world == 1 and not args.no_ladder:
        ladder = ladder_leg()
    wl = None
    if rank == 0 and world == 1 and not args.no_workloads:
        wl = workloads_leg(peak32=r["peak"])
    prec = None
    if rank == 0 and world == 1 and not args.no_precision:
        prec = precision_leg()
    table = None
    if rank == 0 and world == 1 and not args.no_table:
        table = baseline_table_leg(r)
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "chain-sweeps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "roofline": {"bound": "alu", "achieved": r["achieved"], "peak": r["peak"], "unit": "TFLOP/s",
                             "frac": r["achieved"] / r["peak"], "traffic": profiled_traffic(),
                             "kernel": "sweep_kernel<float,8,11> (8 chains x 11 field warps + 1 copy warp per block)",
                             "kernel_ms_per_launch": r["kms"],
                             "flop_count": "algorithmic: 16 FP32 flops x 4|Q| coupling terms per chain-sweep "
                                           "(87.9 MFLOP at N=256)",
                             "flops_per_launch": r["fl"], "frac_survey": r["achieved"] / r["peak"],
                             "achieved_executed": r["achieved_exec"], "frac_executed": r["achieved_exec"] / r["peak"],
                             "flops_per_launch_executed": r["fl_exec"],
                             "executed_count": "flops the pair-factored kernel performs: 6 per pair product, 4 per "
                                               "coupling term, 8 per field row (43.3 MFLOP per chain-sweep at N=256)",
                             "peak_basis": "measured: pt_fma_probe, %d blocks x %d threads, packed %.1f / scalar %.1f "
                                           "TFLOP/s (unit-count peak at the nominal 2070 MHz: %.1f)"
                                           % (r["probe"]["blocks"], r["probe"]["threads"], r["probe"]["packed"],
                                              r["probe"]["scalar"], peak_fp32_tflops(r["probe"]["sm_count"]))},
                "cpu_baseline": cpu,
                "e2e": r["e2e"],
                "clocks": r["clocks"],
                # per step (one 64-sweep segment): sweep, renormalisation, resync energy, its part sum, measurement,
                # swap pass, schedule advance
                "gpu_launches": 7 * args.steps,
                "fp64_plain_gpu": {"value": r["plain_rate"], "unit": "chain-sweeps/s",
                                   "speedup_fp32": r["value"] / world / r["plain_rate"]},
                "learned_vs_plain": learned,
                "learned_vs_plain_cold": learned_cold,
                "random_graph": graph,
                "adaptive_ladder": ladder,
                "workloads": wl,
                "precision_error": prec,
                "baseline_table": table}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
