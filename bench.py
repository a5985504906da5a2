"""Benchmark: dof-updates/s of the sparse-tiled DG elastic time step on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config large] [--tile-size 256] [--block 256] [--no-untiled] [--no-cpu]
                    [--no-adjoint] [--no-batched] [--no-multi] [--no-p4]

One step = one full time step of the DG elastic chain (seventeen loops: velocity sub-chain then
stress sub-chain) over the whole mesh.  The default workload is the 1000x500-square mesh of the
300x150 domain (1.0M triangles, P2, FP64, three layers, Ricker source), executed sparse-tiled
with the seed tile size given, fusion scheme {velocity, stress}.  Inputs are resident in HBM and
larger than L2 (no flush needed).  The JSON line carries the tiled throughput (value), the plain
untiled chain on the same GPU, the inspection time, the roofline of the dominant kernel, the
oracle timed on the host cores (cpu_baseline) and an end-to-end number through the C ABI with
host buffers (e2e).  Further keys time the other configurations of the same path: the P4
mesh (p4), the seismogram gradient (adjoint), 64 shots at once (batched) and 16 uneven meshes
as one group (multi).  --impl reference times the oracle itself on the host cores.

Multi-GPU: the workload does not shard in this library; --gpus N runs N independent replicas
(one per rank, launched by torchrun) and reports the sum over ranks / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dof-updates/s per timestep, tiled vs untiled, % HBM roofline; adjoint/fwd time"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x flop/FMA x max SM clock
HBM_FALLBACK_GBS = 6800.0


def max_over_ranks(dist, x, device):
    """The largest value of x over all ranks (x itself when there is no process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Weak scaling: every rank processes units_per_rank units; the job takes the slowest rank's
    time `seconds`."""
    return units_per_rank * world / seconds


def bind_host_to_gpu(dev):
    """Run this process on the CPUs of the GPU's NUMA node, so that page-locked host buffers are
    allocated next to the GPU's host link.  Returns the node, or None when it is unknown (then
    nothing changes)."""
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open("/sys/bus/pci/devices/%s/numa_node" % bus) as f:
            node = int(f.read())
        if node < 0:
            return None
        with open("/sys/devices/system/node/node%d/cpulist" % node) as f:
            cpus = set()
            for part in f.read().strip().split(","):
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return node
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


KERNEL_SOURCES = ("exec.cu", "exec_body.cuh", "dataflow.cuh", "staged.cuh", "passes.cuh", "internal.h")


def source_digest(texts):
    """Hash of C++ sources without comments and blank space: a change to the code changes it, a
    change to a comment does not."""
    import re
    h = hashlib.sha256()
    for src in texts:
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def kernel_hash():
    """source_digest of the executor sources: a committed counter figure counts only for the code
    it was taken on."""
    texts = []
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1708_03183_gb300", "csrc", f)) as fh:
            texts.append(fh.read())
    return source_digest(texts)


def ncu_traffic(kernel, workload, steps, table=None, current=None):
    """DRAM bytes (read + write) of one launch of `kernel` running `steps` time steps, from the
    committed ncu capture (bytes per step of a launch of that kernel on the same workload), if it
    was taken on the current kernel source; otherwise None.  `table` and `current` (the committed
    table and the current source hash) are read from the repository when not given."""
    try:
        if table is None:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
                table = json.load(f)
        e = table[kernel][workload]
        if e.get("source_hash") != (current if current is not None else kernel_hash()):
            return None
        return float(e["bytes_per_step"]) * steps
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons while active."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=2)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for k, n in enumerate(names):
                    if r[4 + k].lower().startswith("active"):
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample_rate(cfg_name, nsteps, scale=4):
    """The oracle on the host cores: `nsteps` time steps of the same workload generator with the
    mesh reduced by `scale` in each direction (single BLAS thread).  Returns dof-updates/s."""
    code = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, %r)
import synth
from oracle.dg import ElasticDG
c = synth.CONFIGS[%r]
cfg = synth.build_config(%r, nx=c["nx"] // %d, ny=c["ny"] // %d, nsteps=%d)
dg = ElasticDG(cfg["mesh"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"])
nc, Np = dg.nc, dg.Np
v, s = np.zeros((nc, 2, Np)), np.zeros((nc, 3, Np))
t = time.perf_counter()
dg.run(v, s, cfg["dt"], %d, cfg["ricker"], cfg["src"])
t = time.perf_counter() - t
print(json.dumps({"t": t, "nc": nc, "Np": Np}))
""" % (ROOT, cfg_name, cfg_name, scale, scale, nsteps, nsteps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return 5 * d["Np"] * d["nc"] * nsteps / d["t"], d


def oracle_all_cores(cfg_name, nsteps, scale=4, procs=None):
    """The oracle on every host core at once: `procs` independent processes (default: every CPU
    of the host), each running `nsteps` steps of the same sample as oracle_sample_rate on one
    core.  The oracle's loops are single-threaded numpy, so replicas are how it uses the host;
    the rate is the sum of the replicas' rates.  Returns (dof-updates/s, processes, seconds)."""
    procs = procs or os.cpu_count() or 1
    code = r"""
import json, os, sys, time
import numpy as np
os.sched_setaffinity(0, range(os.cpu_count()))
sys.path.insert(0, %r)
import synth
from oracle.dg import ElasticDG
c = synth.CONFIGS[%r]
cfg = synth.build_config(%r, nx=c["nx"] // %d, ny=c["ny"] // %d, nsteps=%d)
dg = ElasticDG(cfg["mesh"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"])
nc, Np = dg.nc, dg.Np
v, s = np.zeros((nc, 2, Np)), np.zeros((nc, 3, Np))
sys.stdout.write("ready\n"); sys.stdout.flush()
sys.stdin.readline()
t = time.perf_counter()
dg.run(v, s, cfg["dt"], %d, cfg["ricker"], cfg["src"])
t = time.perf_counter() - t
print(json.dumps({"t": t, "nc": nc, "Np": Np}))
""" % (ROOT, cfg_name, cfg_name, scale, scale, nsteps, nsteps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=env) for _ in range(procs)]
    for q in ps:                    # every replica has built its mesh: start them together
        if q.stdout.readline().strip() != "ready":
            raise RuntimeError(q.stderr.read()[-2000:])
    t0 = time.perf_counter()
    for q in ps:
        q.stdin.write("go\n")
        q.stdin.flush()
    rate = 0.0
    for q in ps:
        out, err = q.communicate(timeout=900)
        if q.returncode != 0:
            raise RuntimeError(err[-2000:])
        d = json.loads(out.strip().splitlines()[-1])
        rate += 5 * d["Np"] * d["nc"] * nsteps / d["t"]
    return rate, procs, time.perf_counter() - t0


def inspector_timing(slt, synth, args, gpu_full_s, scale=4):
    """The GPU inspector against the oracle inspector (Algorithms 1-3 in sequential C on one host
    core, plus its iteration lists; neither side builds local maps, which the library builds only
    when asked for) on the same mesh: the bench workload's generator reduced by `scale` in each
    direction, the bench's tile size, fusion {velocity, stress}, Hilbert renumbering; best of 3 on
    each side (seconds).  The oracle also inspects the bench mesh itself once, against the GPU
    inspection of the bench run (`gpu_full_s`, which also builds the executor plans and the
    dataflow graph)."""
    import torch
    c = synth.CONFIGS[args.config]
    nx, ny = c["nx"] // scale, c["ny"] // scale
    cfg = synth.build_config(args.config, nx=nx, ny=ny, nsteps=1)
    m = cfg["mesh"]
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"], cfg["src"])
    chain = slt.slt_mesh_chain(mesh)
    gpu = float("inf")
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sc = slt.slt_inspect(chain, tile_size=args.tile_size, split=(9,))
        torch.cuda.synchronize()
        gpu = min(gpu, time.perf_counter() - t0)
        del sc
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
import synth
from oracle import inspector as OI
cfg = synth.build_config(%r, nx=%d, ny=%d, nsteps=1)
ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
OI.build()
best = float("inf")
for _ in range(%d):
    t = time.perf_counter()
    for lo, hi in ((0, 9), (9, 17)):
        OI.inspect(ch.sub(lo, hi), %d, renumber=True, xy=xy, with_local_maps=False)
    best = min(best, time.perf_counter() - t)
print(json.dumps({"t": best}))
"""

    def oracle(nx_, ny_, reps):
        out = subprocess.run([sys.executable, "-c", code % (ROOT, args.config, nx_, ny_, reps, args.tile_size)],
                             capture_output=True, text=True, timeout=900)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        return json.loads(out.stdout.strip().splitlines()[-1])["t"]

    orc = oracle(nx, ny, 3)
    orc_full = oracle(c["nx"], c["ny"], 1)
    return {"sample": "%dx%d squares (%d cells), ts %d, fusion {velocity, stress}, Hilbert renumbering; best of 3"
                      % (nx, ny, m["cell2vert"].shape[0], args.tile_size),
            "gpu_s": gpu, "oracle_s": orc, "oracle_cores": 1, "oracle_over_gpu": orc / gpu,
            "gpu_s_bench_mesh": gpu_full_s, "oracle_s_bench_mesh": orc_full,
            "oracle_over_gpu_bench_mesh": orc_full / gpu_full_s}


def run_reference(args, rank):
    """--impl reference: the oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import synth
    c = synth.CONFIGS[args.config]
    scale = 4
    for _ in range(args.warmup):
        oracle_sample_rate(args.config, 1, scale)
    tot_t, tot_units = 0.0, 0.0
    for _ in range(args.steps):
        rate, d = oracle_sample_rate(args.config, 1, scale)
        tot_t += d["t"]
        tot_units += 5 * d["Np"] * d["nc"]
    value = tot_units / tot_t
    sample = "one time step per step of the %dx%d-square mesh (%d cells, P%d) from the same generator" % (
        c["nx"] // scale, c["ny"] // scale, d["nc"], c["p"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "dof-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "sample": sample},
            "cpu_baseline": {"value": value, "unit": "dof-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "dof-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def adjoint_timing(slt, synth, args, barrier):
    """Forward (slt_record_batched) and gradient (slt_adjoint_batched) time on the adjoint
    workload: 448x224 squares (200k cells, P2, layered +-5 % per cell), the 8 shots of the top row
    of the 8x8 source grid in one call (fields with the shots innermost), 50 receivers along the
    top edge, checkpoints every 50 steps, `--adjoint-steps` steps; untiled, and on the tiles of
    a {velocity, stress} schedule (ts `--adjoint-ts`, every operator application of the forward
    run, the segment recompute and the reverse sweep on the dataflow executor).  The forward
    records the receivers after every step, so it runs one step per launch."""
    import numpy as np
    import torch
    n = args.adjoint_steps
    cfg = synth.build_config("adjoint", nsteps=n)
    m = cfg["mesh"]
    nc = m["cell2vert"].shape[0]
    shots = np.array([((i + 0.5) * 300.0 / 8, (7 + 0.5) * 150.0 / 8) for i in range(8)])
    rec = np.stack([(np.arange(50) + 0.5) * 6.0, np.full(50, 149.0)], 1)
    base = synth.layered(m)
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], cfg["p"], *base)
    r = slt.slt_receivers_create(mesh, rec)
    rk = torch.tensor(cfg["ricker"], device="cuda")
    S = len(shots)
    data = torch.zeros((n, S, 50, 2), dtype=torch.float64, device="cuda")
    slt.slt_record_batched(mesh, None, r, shots, rk, cfg["dt"], n, data)   # synthetic data, unperturbed model
    slt.slt_mesh_set_material(mesh, cfg["rho"], cfg["lam"], cfg["mu"])      # perturbed model
    out = {"workload": "448x224 squares (%d cells), P2, %d shots in one call, 50 receivers, %d steps, "
                       "checkpoints every 50" % (nc, S, n)}
    sched = slt.slt_inspect(slt.slt_mesh_chain(mesh), tile_size=args.adjoint_ts, split=(9,))
    for name, sc in (("untiled", None), ("tiled_ts%d" % args.adjoint_ts, sched)):
        tr = torch.zeros_like(data)
        g = torch.zeros((3, nc), dtype=torch.float64, device="cuda")
        barrier()
        t0 = time.perf_counter()
        slt.slt_record_batched(mesh, sc, r, shots, rk, cfg["dt"], n, tr)
        barrier()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        J = slt.slt_adjoint_batched(mesh, sc, r, shots, rk, cfg["dt"], n, data, 50, g)
        barrier()
        t_adj = time.perf_counter() - t0
        out[name] = {"forward_ms_per_step": 1e3 * t_fwd / n, "gradient_ms_per_step": 1e3 * t_adj / n,
                     "adjoint_over_forward": t_adj / t_fwd, "misfit": J,
                     "shot_steps_per_s_gradient": S * n / t_adj}
    out["note"] = ("gradient = forward with checkpoints + segment recompute keeping the operator "
                   "intermediates + reverse sweep; all shots of a step in each launch")
    return out


def batched_timing(slt, synth, args, barrier, keep):
    """Multi-shot form: the 708x354 P2 layered mesh (501k cells) with `--shots` point sources on
    the 8x8 grid x = (i+1/2) 300/8, y = (j+1/2) 150/8 (the first `--shots` of them), shots
    innermost.  The library's autotuner picks among the untiled chain and the dataflow executor
    at each tile size of `--batched-ts` with `--shots-per-cta` shots per tile CTA (3 timed steps
    each); the pick is then timed over `--batched-steps` steps."""
    import numpy as np
    import torch
    S = args.shots
    K = args.batched_steps
    W = 3
    cfg = synth.build_config("large", nx=708, ny=354, nsteps=W + K)
    m = cfg["mesh"]
    nc = m["cell2vert"].shape[0]
    Np = (cfg["p"] + 1) * (cfg["p"] + 2) // 2
    grid = np.array([((i + 0.5) * 300.0 / 8, (j + 0.5) * 150.0 / 8) for j in range(8) for i in range(8)])
    pts = grid[np.arange(S) % 64]
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"], cfg["src"])
    t0 = time.perf_counter()
    best, table = slt.slt_autotune(mesh, list(args.batched_ts), nshots=S, block_threads=(256,),
                                   shots_per_cta=[g for g in args.shots_per_cta if g <= S], steps=3, split=(9,))
    tune_s = time.perf_counter() - t0
    sched = slt.slt_inspect(slt.slt_mesh_chain(mesh), best) if best.tile_size else None
    rk = torch.tensor(cfg["ricker"], device="cuda")
    v = torch.zeros((nc, 2, Np, S), dtype=torch.float64, device="cuda")
    s = torch.zeros((nc, 3, Np, S), dtype=torch.float64, device="cuda")
    slt.slt_execute_batched(mesh, sched, pts, v, s, rk, cfg["dt"], W)
    barrier()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        prof = slt.slt_execute_batched(mesh, sched, pts, v, s, rk[W:], cfg["dt"], K, profile=True)
        barrier()
    ms = prof["chain_ms"] / K
    units = 5 * Np * nc * S
    fl = slt.slt_mesh_cost(mesh)["flops_per_step"] * S
    pick = ("untiled" if not best.tile_size else
            "ts%d, %d shots per CTA" % (best.tile_size, best.shots_per_cta or S))
    keep.update(big_mesh=mesh, big_cfg=cfg, shots=pts, S=S, nc=nc, Np=Np)
    # the volume contraction of this layout on the FP64 tensor instruction against DFMA, at this
    # mesh's size (P2) and at the P4 workload's (250k cells), S shots each
    tensor = {}
    for deg, ncell in ((2, nc), (4, 250000)):
        r = slt.slt_fp64_contraction_probe(deg, ncell, S - S % 8 or 8)
        tensor["p%d" % deg] = {"cells": ncell, "dfma_ms": r["dfma_ms"], "dmma_ms": r["dmma_ms"],
                               "dmma_over_dfma": r["dmma_ms"] / r["dfma_ms"],
                               "useful_tflops_dfma": r["useful_flops"] / (r["dfma_ms"] * 1e-3) / 1e12,
                               "useful_tflops_dmma": r["useful_flops"] / (r["dmma_ms"] * 1e-3) / 1e12,
                               "dmma_useful_fraction": r["useful_flops"] / r["dmma_issued_flops"],
                               "rel_diff": r["rel_diff"]}
    return {"workload": "708x354 squares on 300x150 (%d cells), P2 FP64, layered, %d shots on the 8x8 grid, "
                        "%d steps, fields [cell][comp][node][shot] (%.1f GB)" % (nc, S, K, 5 * Np * nc * S * 8 / 1e9),
            "value": units / (ms * 1e-3), "unit": "dof-updates/s", "best": pick, "ms_per_step": ms,
            "fp64_frac": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, "clocks": clk.summary(),
            "autotune": {"seconds": tune_s, "rows": ["ts %d, renumber %d, %d threads, %d shots per CTA: %.2f ms" % tuple(r)
                                                     for r in table]},
            "fp64_tensor_contraction": tensor}


def multi_timing(slt, synth, args, barrier, keep):
    """Many uneven meshes: 16 meshes with cell counts log-uniform in [20k, 400k] (seed 4), degree
    1 + (i mod 3), each sparse-tiled (ts 256, dataflow executor) and advanced `--multi-steps`
    steps as one group (one combined ready queue per degree) against the same meshes run one
    after another with slt_execute."""
    import torch
    K, W = args.multi_steps, 3
    cfgs = synth.multi_configs(16, nsteps=W + K)
    meshes, scheds, fields = [], [], []
    for c in cfgs:
        m = c["mesh"]
        mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], c["p"], c["rho"], c["lam"], c["mu"], c["src"])
        meshes.append(mesh)
        scheds.append(slt.slt_inspect(slt.slt_mesh_chain(mesh), tile_size=256, split=(9,)))
        nc, Np = m["cell2vert"].shape[0], (c["p"] + 1) * (c["p"] + 2) // 2
        fields.append((torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda"),
                       torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda"),
                       torch.tensor(c["ricker"], device="cuda")))
    units = sum(5 * ((c["p"] + 1) * (c["p"] + 2) // 2) * c["mesh"]["cell2vert"].shape[0] for c in cfgs)
    vs, ss, rs = [list(x) for x in zip(*fields)]
    dts = [c["dt"] for c in cfgs]
    keep.update(meshes=meshes, scheds=scheds, cfgs=cfgs, units_multi=units)
    grp = slt.slt_group_create(meshes, scheds)
    slt.slt_group_execute(grp, vs, ss, rs, dts, W)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    slt.slt_group_execute(grp, vs, ss, [r[W:] for r in rs], dts, K)
    e1.record()
    barrier()
    t_many = e0.elapsed_time(e1)
    e0.record()
    for mesh, sc, (v, s, r), dt in zip(meshes, scheds, fields, dts):
        slt.slt_execute(mesh, sc, v, s, r[W:], dt, K)
    e1.record()
    barrier()
    t_seq = e0.elapsed_time(e1)
    ncs = [c["mesh"]["cell2vert"].shape[0] for c in cfgs]
    return {"workload": "16 meshes, %d..%d cells (%d in all), degrees 1-3, ts 256, %d steps" % (
                min(ncs), max(ncs), sum(ncs), K),
            "value": units * K / (t_many * 1e-3), "unit": "dof-updates/s", "ms_per_step": t_many / K,
            "one_after_another_ms_per_step": t_seq / K, "overlap_speedup": t_seq / t_many}


def one_launch_timing(slt, synth, args, barrier, keep):
    """The whole batched configuration in one persistent launch: the 64 shots of the batched
    block (708x354 P2 mesh, tiled at ts `--batched-ts`[0], all shots of a tile in its CTA) and the
    16 uneven meshes of the multi block (ts 256), all from one ready queue
    (slt_group_create_batched), the step captured once as a CUDA graph and replayed; against the
    same two workloads run one after the other (the 64-shot launch, then the group of meshes)."""
    import torch
    K, W = args.batched_steps, 3
    big, cfgs, meshes, scheds = keep["big_mesh"], keep["cfgs"], keep["meshes"], keep["scheds"]
    S, nc, Np, bcfg = keep["S"], keep["nc"], keep["Np"], keep["big_cfg"]
    ts = args.batched_ts[0]
    bsched = slt.slt_inspect(slt.slt_mesh_chain(big), tile_size=ts, split=(9,))
    grp = slt.slt_group_create_batched([big] + meshes, [bsched] + scheds, [S] + [1] * len(meshes),
                                       [keep["shots"]] + [None] * len(meshes))
    bv = torch.zeros((nc, 2, Np, S), dtype=torch.float64, device="cuda")
    bs = torch.zeros((nc, 3, Np, S), dtype=torch.float64, device="cuda")
    fields = [(torch.zeros((c["mesh"]["cell2vert"].shape[0], 2, (c["p"] + 1) * (c["p"] + 2) // 2),
                           dtype=torch.float64, device="cuda"),
               torch.zeros((c["mesh"]["cell2vert"].shape[0], 3, (c["p"] + 1) * (c["p"] + 2) // 2),
                           dtype=torch.float64, device="cuda")) for c in cfgs]
    vs, ss = [bv] + [f[0] for f in fields], [bs] + [f[1] for f in fields]
    K = min(K, len(bcfg["ricker"]) - W, min(len(c["ricker"]) for c in cfgs) - W)
    brk = torch.tensor(bcfg["ricker"][:W + K], device="cuda")
    rks = [brk] + [torch.tensor(c["ricker"][:W + K], device="cuda") for c in cfgs]
    dts = [bcfg["dt"]] + [c["dt"] for c in cfgs]
    slt.slt_group_execute(grp, vs, ss, rks, dts, W)          # captures the graph (W steps)
    slt.slt_group_execute(grp, vs, ss, rks, dts, W)          # replays it
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    slt.slt_group_execute(grp, vs, ss, [r[W:] for r in rks], dts, K)
    e1.record()
    barrier()
    t_one = e0.elapsed_time(e1)
    # the same work as two launches: the 64 shots alone, then the group of meshes
    grp2 = slt.slt_group_create(meshes, scheds)
    e0.record()
    slt.slt_execute_batched(big, bsched, keep["shots"], bv, bs, brk[W:], bcfg["dt"], K)
    slt.slt_group_execute(grp2, vs[1:], ss[1:], [r[W:] for r in rks[1:]], dts[1:], K)
    e1.record()
    barrier()
    t_two = e0.elapsed_time(e1)
    units = 5 * Np * nc * S + keep["units_multi"]
    return {"workload": "the 64-shot 708x354 P2 mesh (ts %d) and the 16 uneven meshes (ts 256) in one persistent "
                        "launch, graph-captured, %d steps" % (ts, K),
            "value": units * K / (t_one * 1e-3), "unit": "dof-updates/s", "ms_per_step": t_one / K,
            "two_launches_ms_per_step": t_two / K, "graph_replays": slt.slt_group_graph_replays(grp)}


def p4_timing(slt, synth, args, barrier):
    """The high-order configuration: 500x250 squares on 300x150 (250k cells), P4, layered,
    sparse-tiled at ts 256 with 384-thread tiles (the autotuner's pick) against the untiled
    chain, `--p4-steps` steps each."""
    import torch
    K, W = args.p4_steps, 3
    cfg = synth.build_config("p4", nsteps=W + K)
    m = cfg["mesh"]
    nc, Np = m["cell2vert"].shape[0], 15
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], 4, cfg["rho"], cfg["lam"], cfg["mu"], cfg["src"])
    sched = slt.slt_inspect(slt.slt_mesh_chain(mesh), tile_size=256, split=(9,), block_threads=384)
    rk = torch.tensor(cfg["ricker"], device="cuda")
    flops = slt.slt_mesh_cost(mesh)["flops_per_step"]
    out = {"workload": "p4: 500x250 squares on 300x150 (%d cells), DG P4 FP64, layered, %d steps" % (nc, K)}
    for name, sc in (("tiled_ts256_bt384", sched), ("untiled", None)):
        v = torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda")
        s = torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda")
        slt.slt_execute(mesh, sc, v, s, rk, cfg["dt"], W)
        barrier()
        prof = slt.slt_execute_profiled(mesh, sc, v, s, rk[W:], cfg["dt"], K)
        barrier()
        ms = prof["chain_ms"] / K
        out[name] = {"ms_per_step": ms, "value": 5 * Np * nc / (ms * 1e-3),
                     "fp64_frac": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    return out


def fp64_peak(slt, reps=20):
    """The FP64 probe (slt_fp64_peak) `reps` times with nvidia-smi clocks sampled meanwhile: the
    arithmetic roof of this path on the GPU at hand (the driver's measured peaks cover only an
    HBM copy and a bf16 GEMM).  Best of the repetitions, TFLOP/s."""
    runs = []
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(reps):
            runs.append(slt.slt_fp64_peak())
    best = {k: max(r[k] for r in runs) for k in ("dfma_tflops", "dmma_tflops", "mixed_tflops")}
    best["lanes"] = slt.slt_fp64_lane_probe()   # warp instructions per clock per SM
    best["clocks"] = clk.summary()
    best["nominal_dfma_tflops"] = FP64_PEAK_TFLOPS
    best["dfma_per_clk_per_sm"] = best["dfma_tflops"] * 1e12 / 2 / 152 / (best["clocks"]["sm_mhz"] or 2070.0) / 1e6
    return best


def workload_name(args):
    import synth
    c = synth.CONFIGS[args.config]
    sc = getattr(args, "scale", 1)
    nx, ny = c["nx"] // sc, c["ny"] // sc
    return ("%s: %dx%d squares on %gx%g, %d triangles, DG P%d FP64, %s material, Ricker f0=%g, "
            "sparse-tiled ts=%d, fusion {velocity, stress}, %s executor" % (
                args.config, nx, ny, c["Lx"], c["Ly"], 2 * nx * ny, c["p"], c["material"],
                c["f0"], args.tile_size,
                ["dataflow", "colour-phase", "cluster dataflow", "staged dataflow", "pass dataflow"][getattr(args, "executor", 0)]))


def sweep(slt, synth, args):
    """Time executor configurations on one workload: for each entry of --sweep, a warm-up launch
    of 3 steps, then the best of two --steps-step launches (kernel time from
    slt_execute_profiled), with the schedule's dependency-graph figures."""
    import torch
    c0 = synth.CONFIGS[args.config]
    over = {"p": args.degree} if args.degree else {}
    K = args.steps
    cfg = synth.build_config(args.config, nsteps=2 * K + 3, nx=c0["nx"] // args.scale, ny=c0["ny"] // args.scale,
                             **over)
    m = cfg["mesh"]
    nc, p = m["cell2vert"].shape[0], cfg["p"]
    Np = (p + 1) * (p + 2) // 2
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], p, cfg["rho"], cfg["lam"], cfg["mu"], cfg["src"])
    chain = slt.slt_mesh_chain(mesh)
    rk = torch.tensor(cfg["ricker"], device="cuda")
    flops = slt.slt_mesh_cost(mesh)["flops_per_step"]
    split = tuple(int(x) for x in args.split.split(":") if x)
    for entry in args.sweep.split(","):
        out = {"workload": "%s, %d cells, P%d" % (args.config, nc, p), "config": entry}
        try:
            sched = None
            if entry != "untiled":
                f = [int(x) for x in entry.split(":")] + [0, 0]
                sched = slt.slt_inspect(chain, tile_size=f[0], split=split, block_threads=f[1], executor=f[2],
                                        release_order=f[3], cluster_size=f[4])
            v = torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda")
            s = torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda")
            slt.slt_execute(mesh, sched, v, s, rk, cfg["dt"], 3)
            best = min(slt.slt_execute_profiled(mesh, sched, v, s, rk[3 + r * K:], cfg["dt"], K)["chain_ms"] / K
                       for r in range(2))
            out.update(ms_per_step=best, fp64_tflops=flops / (best * 1e-3) / 1e12)
            if sched is not None:
                d = slt.slt_schedule_dataflow_info(sched)
                out.update(node_rounds_per_step=d["nodes_per_step"] / max(d["tiles_in_flight"], 1),
                           critical_path_work_weighted=d["critical_path_items"], tiles_in_flight=d["tiles_in_flight"])
        except slt.SltError as e:
            out["error"] = str(e)
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large")
    ap.add_argument("--tile-size", type=int, default=256)
    ap.add_argument("--executor", type=int, default=0,
                    help="0 dataflow (persistent), 1 colour phases, 2 dataflow with one CTA cluster per tile, "
                         "3 staged dataflow (each tile out of shared memory), 4 dataflow with compacted passes")
    ap.add_argument("--cluster-size", type=int, default=8, help="CTAs per tile cluster (executor 2)")
    ap.add_argument("--block", type=int, default=256, help="threads per tile CTA (128, 256 or 384)")
    ap.add_argument("--no-untiled", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--scale", type=int, default=1, help="divide nx, ny of the workload (small profiling cases)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=1000)
    ap.add_argument("--adjoint-ts", type=int, default=64)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-p4", action="store_true")
    ap.add_argument("--no-cluster", action="store_true")
    ap.add_argument("--no-staged", action="store_true")
    ap.add_argument("--p4-steps", type=int, default=200)
    ap.add_argument("--multi-steps", type=int, default=200)
    ap.add_argument("--shots", type=int, default=64)
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--batched-ts", type=lambda t: [int(x) for x in t.split(",")], default=[16, 32, 64])
    ap.add_argument("--shots-per-cta", type=lambda t: [int(x) for x in t.split(",")], default=[16, 64])
    ap.add_argument("--fp64-peak", action="store_true", help="only measure the FP64 roof (probe + clocks)")
    ap.add_argument("--sweep", default=None,
                    help="only time executor configurations on --config (with --degree): comma-separated "
                         "ts:block:executor[:release_order[:cluster_size]], 'untiled' for the untiled chain; "
                         "--steps steps each, --split for the fusion scheme; one JSON line per configuration")
    ap.add_argument("--degree", type=int, default=0, help="--sweep: override the workload's degree")
    ap.add_argument("--split", default="9", help="--sweep: split points of the fusion scheme, ':'-separated")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()          # one rank compiles; the others wait for the library
    if dist:
        dist.barrier()
    import paper_1708_03183_gb300 as slt
    import synth

    if args.fp64_peak:
        if rank == 0:
            print(json.dumps(fp64_peak(slt)))
        return

    if args.sweep:
        if rank == 0:
            sweep(slt, synth, args)
        return

    c0 = synth.CONFIGS[args.config]
    k_untiled = max(args.steps // 4, 10)
    cfg = synth.build_config(args.config, nsteps=args.warmup + max(args.steps, k_untiled) + args.e2e_steps,
                             nx=c0["nx"] // args.scale, ny=c0["ny"] // args.scale)
    m = cfg["mesh"]
    nc = m["cell2vert"].shape[0]
    p = cfg["p"]
    Np, Nfp = (p + 1) * (p + 2) // 2, p + 1
    stream = torch.cuda.current_stream()
    mesh = slt.slt_mesh_create(m["cell2vert"], m["cellxy"], p, cfg["rho"], cfg["lam"], cfg["mu"], cfg["src"])
    info = slt.slt_mesh_info(mesh)
    chain = slt.slt_mesh_chain(mesh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sched = slt.slt_inspect(chain, tile_size=args.tile_size, split=(9,), executor=args.executor,
                            block_threads=args.block, cluster_size=args.cluster_size)
    inspect_s = time.perf_counter() - t0
    subs = [slt.slt_schedule_info(sched, k) for k in range(2)]
    insp_stages = slt.slt_schedule_inspection_times(sched)
    lanes = slt.slt_schedule_lane_info(sched)

    ricker = torch.tensor(cfg["ricker"], device="cuda")
    units_per_step = 5 * Np * nc

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(schedule, K, W):
        v = torch.zeros((nc, 2, Np), dtype=torch.float64, device="cuda")
        s = torch.zeros((nc, 3, Np), dtype=torch.float64, device="cuda")
        slt.slt_execute(mesh, schedule, v, s, ricker, cfg["dt"], W)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            e0.record(stream)
            prof = slt.slt_execute_profiled(mesh, schedule, v, s, ricker[W:], cfg["dt"], K)
            e1.record(stream)
            barrier()
        ms = max_over_ranks(dist, e0.elapsed_time(e1), "cuda")
        return ms, prof, clk.summary()

    ms, prof, clocks = timed(sched, args.steps, args.warmup)
    value = whole_job_rate(units_per_step * args.steps, world, ms * 1e-3)
    cost = slt.slt_mesh_cost(mesh)   # the library's own count of the work its kernels do
    flops = cost["flops_per_step"]
    kern_s = prof["chain_ms"] * 1e-3
    achieved = flops * args.steps / kern_s / 1e12
    hbm_peak, hbm_kind = peaks()
    probe = slt.slt_fp64_peak()
    kname = ("k_dataflow<%d,%d>", "k_tiled<%d,%d>", "k_dataflow_cluster<%d,%d>", "k_staged<%d,%d>",
             "k_passes<%d,%d>")[args.executor] % (
        p, args.block)
    traffic = ncu_traffic(kname, args.config, args.steps) if args.scale == 1 and args.block == 256 else None
    tiled_bytes = cost["tiled_bytes_per_step"]

    out = {"metric": METRIC, "value": value, "unit": "dof-updates/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(args), "ncell": nc, "degree": p, "tile_size": args.tile_size,
                      "dofs": units_per_step, "l2": "inputs larger than L2 (%.2f GB resident per step)" % (
                          (20 * Np + 33) * nc * 8 / 1e9),
                      "parallelism": "replicas" if world > 1 else "1 GPU",
                      "tiles": [s["ntiles"] for s in subs], "colours": [s["ncolours"] for s in subs],
                      "restarts": [s["restarts"] for s in subs], "inspection_s": inspect_s,
                      "inspection_stages_s": insp_stages,
                      "fp64_lane_efficiency": {"tiled": lanes["dataflow_efficiency"],
                                               "staged_passes": lanes["staged_efficiency"],
                                               "untiled": lanes["untiled_efficiency"],
                                               "how": "slt_schedule_lane_info: FP64 warp-lane instructions "
                                                      "a step needs over those its warps issue"},
                      "executor": ["dataflow", "colour phases", "dataflow, tile clusters of %d CTAs" % args.cluster_size,
                                   "staged dataflow (tiles out of shared memory)",
                                   "dataflow with compacted passes"][args.executor],
                      "block_threads": args.block},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP64_PEAK_TFLOPS,
                        "traffic": traffic, "kernel": kname,
                        "peak_kind": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2070 MHz (nominal unit counts)",
                        "measured_fp64": {"dfma_tflops": probe["dfma_tflops"], "dmma_tflops": probe["dmma_tflops"],
                                          "dfma_and_dmma_tflops": probe["mixed_tflops"],
                                          "how": "slt_fp64_peak: 8 independent DFMA chains per thread / 4 "
                                                 "mma.sync.m8n8k4.f64 accumulators per warp, 8 x 256-thread "
                                                 "blocks per SM, CUDA events"},
                        "frac_of_measured_dfma": achieved / probe["dfma_tflops"],
                        "launch_ms_avg": prof["chain_ms"] / max(prof["chain_launches"], 1),
                        "launches": prof["chain_launches"], "steps_per_launch": args.steps / max(prof["chain_launches"], 1),
                        "flops_per_step": flops},
           "hbm": {"algorithmic_bytes_per_step": tiled_bytes,
                   "achieved_gbs": tiled_bytes * args.steps / kern_s / 1e9, "peak_gbs": hbm_peak,
                   "frac": tiled_bytes * args.steps / kern_s / 1e9 / hbm_peak, "peak_kind": hbm_kind},
           "clocks": clocks,
           "gpu_launches": prof["chain_launches"] + prof["layout_launches"] + prof["setup_launches"]}
    if args.executor != 1:
        # the dependency graph the dataflow executor ran: time per step cannot fall below the
        # longest chain (in node times), and reaches the work bound only when the nodes of a step
        # are many more per tile in flight than that chain is long
        dinfo = slt.slt_schedule_dataflow_info(sched)
        out["dataflow"] = {"nodes_per_step": dinfo["nodes_per_step"], "deps_per_step": dinfo["deps_per_step"],
                           "critical_path_nodes_per_step": dinfo["critical_path_nodes"],
                           "critical_path_work_weighted": dinfo["critical_path_items"],
                           "tiles_in_flight": dinfo["tiles_in_flight"],
                           "node_rounds_per_step": dinfo["nodes_per_step"] / max(dinfo["tiles_in_flight"], 1)}

    if not args.no_cluster and args.executor == 0:
        # the same workload with one thread-block cluster per large tile (fewer boundary cells)
        csched = slt.slt_inspect(chain, tile_size=2048, split=(9,), executor=2, cluster_size=4)
        cms, cprof, cclk = timed(csched, k_untiled, args.warmup)
        ck = cprof["chain_ms"] * 1e-3
        out["cluster"] = {"executor": "dataflow, one 4-CTA cluster per tile, ts 2048",
                          "value": whole_job_rate(units_per_step * k_untiled, world, cms * 1e-3),
                          "ms_per_step": cms / k_untiled, "steps": k_untiled,
                          "roofline_frac_fp64": flops * k_untiled / ck / 1e12 / FP64_PEAK_TFLOPS,
                          "traffic": ncu_traffic("k_dataflow_cluster<2,256>", "large_ts2048_c4", k_untiled)
                          if args.scale == 1 else None,
                          "clocks": cclk}
        del csched

    if not args.no_staged and args.executor == 0:
        # the same workload with every tile run out of shared memory (executor 3): the DRAM bytes
        # it saves, and what its one CTA per SM costs on this FP64-bound part
        ssched = slt.slt_inspect(chain, tile_size=256, split=(9,), executor=3, block_threads=384)
        sms, sprof, sclk = timed(ssched, k_untiled, args.warmup)
        sk = sprof["chain_ms"] * 1e-3
        out["staged"] = {"executor": "staged dataflow, tiles out of shared memory, ts 256, 384 threads",
                         "value": whole_job_rate(units_per_step * k_untiled, world, sms * 1e-3),
                         "ms_per_step": sms / k_untiled, "steps": k_untiled,
                         "roofline_frac_fp64": flops * k_untiled / sk / 1e12 / FP64_PEAK_TFLOPS,
                         "traffic": ncu_traffic("k_staged<2,384>", "large_ts256", k_untiled)
                         if args.scale == 1 else None,
                         "clocks": sclk}
        del ssched

    if not args.no_untiled:
        K = k_untiled
        ums, uprof, uclk = timed(None, K, args.warmup)
        ub = cost["untiled_bytes_per_step"]
        uk = uprof["chain_ms"] * 1e-3
        out["untiled"] = {"value": whole_job_rate(units_per_step * K, world, ums * 1e-3), "ms_per_step": ums / K,
                          "steps": K,
                          "roofline_frac_fp64": flops * K / uk / 1e12 / FP64_PEAK_TFLOPS,
                          "hbm_frac": ub * K / uk / 1e9 / hbm_peak, "algorithmic_bytes_per_step": ub,
                          "launches_per_step": uprof["chain_launches"] / K, "clocks": uclk}

    # end to end through the C ABI with pinned host buffers: every step copies the state in,
    # runs one step and copies the state out
    numa = bind_host_to_gpu(local)
    hv = torch.zeros((nc, 2, Np), dtype=torch.float64).pin_memory()
    hs = torch.zeros((nc, 3, Np), dtype=torch.float64).pin_memory()
    hr = torch.tensor(cfg["ricker"], dtype=torch.float64).pin_memory()
    for n in range(3):
        slt.slt_execute_host(mesh, sched, hv, hs, hr[n:n + 1], cfg["dt"], 1)
    barrier()
    t0 = time.perf_counter()
    for n in range(args.e2e_steps):
        slt.slt_execute_host(mesh, sched, hv, hs, hr[n:n + 1], cfg["dt"], 1)
    barrier()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    out["e2e"] = {"value": whole_job_rate(units_per_step * args.e2e_steps, world, e2e_s), "unit": "dof-updates/s",
                  "h2d_bytes_per_step": 5 * Np * nc * 8 + 8, "d2h_bytes_per_step": 5 * Np * nc * 8,
                  "steps": args.e2e_steps, "host_numa_node": numa}

    if not args.no_p4:
        out["p4"] = p4_timing(slt, synth, args, barrier)
    if not args.no_adjoint:
        out["adjoint"] = adjoint_timing(slt, synth, args, barrier)
    keep = {}
    if not args.no_batched:
        del sched, mesh
        torch.cuda.empty_cache()
        out["batched"] = batched_timing(slt, synth, args, barrier, keep)
    if not args.no_multi:
        torch.cuda.empty_cache()
        out["multi"] = multi_timing(slt, synth, args, barrier, keep)
    if not args.no_batched and not args.no_multi:
        torch.cuda.empty_cache()
        out["batched_one_launch"] = one_launch_timing(slt, synth, args, barrier, keep)

    if rank == 0 and world == 1 and not args.no_cpu:
        rate, d = oracle_sample_rate(args.config, 10)
        out["cpu_baseline"] = {"value": rate, "unit": "dof-updates/s", "cores": 1, "kind": "oracle",
                               "host_nproc": os.cpu_count(),
                               "sample": "10 time steps of the same generator's mesh reduced 4x per direction "
                                         "(%d cells, P%d), single BLAS thread, %.1f s" % (d["nc"], p, d["t"])}
        arate, aprocs, asec = oracle_all_cores(args.config, 10)
        out["cpu_baseline"]["all_cores"] = {
            "value": arate, "unit": "dof-updates/s", "cores": aprocs, "kind": "oracle",
            "sample": "%d independent oracle processes, one per host CPU, each the 1-core sample above; "
                      "sum of their rates, %.1f s wall" % (aprocs, asec)}
        others = {}
        for name, steps, scale in (("tiny", 20, 1), ("p4", 3, 4)):
            r, dd = oracle_sample_rate(name, steps, scale)
            others[name] = {"value": r, "sample": "%d steps, %d cells, P%d" % (steps, dd["nc"], synth.CONFIGS[name]["p"])}
        out["cpu_baseline"]["other_configs"] = others
        out["inspector"] = inspector_timing(slt, synth, args, inspect_s)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
