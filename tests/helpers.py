"""Shared helpers for the GPU tests: seeded workloads, oracle runs, comparisons."""
import functools

import numpy as np

import synth
from oracle import inspector as OI
from oracle.dg import ElasticDG

TOL = 1e-11   # relative L2 per field, FP64 (facet increments may be reordered)


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@functools.lru_cache(maxsize=None)
def workload(name, seed_fields=11, **over):
    """Config + seeded random initial fields (so every term acts from the first step)."""
    cfg = synth.build_config(name, **dict(over))
    nc = cfg["mesh"]["cell2vert"].shape[0]
    Np = (cfg["p"] + 1) * (cfg["p"] + 2) // 2
    rng = np.random.default_rng(seed_fields)
    cfg["v0"] = 1e-3 * rng.standard_normal((nc, 2, Np))
    cfg["s0"] = 1e-3 * rng.standard_normal((nc, 3, Np))
    return cfg


@functools.lru_cache(maxsize=None)
def oracle_run(name, nsteps=None, **over):
    cfg = workload(name, **dict(over))
    dg = ElasticDG(cfg["mesh"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"])
    n = cfg["nsteps"] if nsteps is None else nsteps
    v, s = dg.run(cfg["v0"].copy(), cfg["s0"].copy(), cfg["dt"], n, cfg["ricker"], cfg["src"])
    return v, s


def gpu_mesh(slt, cfg):
    m = cfg["mesh"]
    return slt.slt_mesh_create(m["cell2vert"], m["cellxy"], cfg["p"], cfg["rho"], cfg["lam"], cfg["mu"],
                               cfg["src"])


def gpu_run(slt, cfg, nsteps=None, sched=None, mesh=None):
    import torch
    mesh = mesh or gpu_mesh(slt, cfg)
    n = cfg["nsteps"] if nsteps is None else nsteps
    v = torch.tensor(cfg["v0"], device="cuda")
    s = torch.tensor(cfg["s0"], device="cuda")
    r = torch.tensor(cfg["ricker"], device="cuda")
    slt.slt_execute(mesh, sched, v, s, r, cfg["dt"], n)
    torch.cuda.synchronize()
    return v.cpu().numpy(), s.cpu().numpy()


def compare_schedules(slt, gsched, chain_or, sub_bounds, ts, _offset=(0, 0), **opts):
    """Bit-exact comparison of the GPU schedule with the oracle inspector, sub-chain by sub-chain.
    _offset = (first GPU sub-chain index, loop offset of chain_or in the GPU chain)."""
    for k0, (lo0, hi0) in enumerate(sub_bounds):
        k, lo, hi = k0 + _offset[0], lo0 + _offset[1], hi0 + _offset[1]
        o = OI.inspect(chain_or.sub(lo0, hi0), ts, **opts)
        info = slt.slt_schedule_info(gsched, k)
        assert info["ntiles"] == o["ntiles"] and info["ncolours"] == o["ncolours"], (info, o["ncolours"])
        assert info["restarts"] == o["restarts"] and bool(info["fell_back"]) == o["fell_back"]
        assert info["conflicts"] == o["conflicts"] and info["unprojected"] == o["unprojected"]
        assert np.array_equal(slt.slt_schedule_export(gsched, "rank", k), o["rank"])
        assert np.array_equal(slt.slt_schedule_export(gsched, "colour", k), o["colour"])
        for jj in range(hi - lo):
            j = lo + jj
            assert np.array_equal(slt.slt_schedule_export(gsched, "sigma", j), o["sigma"][jj]), ("sigma", j)
            ptr, its = o["lists"][jj]
            assert np.array_equal(slt.slt_schedule_export(gsched, "list_ptr", j), ptr)
            assert np.array_equal(slt.slt_schedule_export(gsched, "list", j), its)
            for d, lm in enumerate(o["local_maps"][jj]):
                if lm is None:
                    continue
                fp_ptr, fp, lmap = lm
                assert np.array_equal(slt.slt_schedule_export(gsched, "fp_ptr", j, d), fp_ptr)
                assert np.array_equal(slt.slt_schedule_export(gsched, "fp", j, d), fp)
                assert np.array_equal(slt.slt_schedule_export(gsched, "lmap", j, d), lmap)
        for jj, f in enumerate(OI.export_flags(chain_or.sub(lo0, hi0), o["sigma"])):
            assert np.array_equal(slt.slt_schedule_export(gsched, "export", lo + jj), f), ("export", lo + jj)
