"""Parity at the full size of the benchmarked workload (1.0M cells, P2), in the launch
configuration bench.py times (dataflow executor, ts 256, fusion {velocity, stress}): the whole
schedule bit for bit against the oracle inspector, and two time steps of the tiled chain against
the oracle's untiled chain.  Minutes of oracle time: marked slow."""
import numpy as np
import pytest

import synth
from oracle import inspector as OI
from oracle.dg import ElasticDG
from tests.helpers import TOL, rel_l2, gpu_mesh

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TS = 256


@pytest.fixture(scope="module")
def large(lib):
    cfg = synth.build_config("large")
    mesh = gpu_mesh(lib, cfg)
    sched = lib.slt_inspect(lib.slt_mesh_chain(mesh), tile_size=TS, split=(9,))
    return cfg, mesh, sched


def test_fullsize_schedule_bit_exact(lib, large):
    cfg, mesh, sched = large
    ch, xy, _, _ = OI.elastic_chain(cfg["mesh"])
    for k, (lo, hi) in enumerate(((0, 9), (9, 17))):
        o = OI.inspect(ch.sub(lo, hi), TS, renumber=True, xy=xy)
        info = lib.slt_schedule_info(sched, k)
        assert (info["ntiles"], info["ncolours"], info["restarts"]) == (o["ntiles"], o["ncolours"], o["restarts"])
        assert np.array_equal(lib.slt_schedule_export(sched, "rank", k), o["rank"])
        assert np.array_equal(lib.slt_schedule_export(sched, "colour", k), o["colour"])
        for jj in range(hi - lo):
            assert np.array_equal(lib.slt_schedule_export(sched, "sigma", lo + jj), o["sigma"][jj])
            ptr, its = o["lists"][jj]
            assert np.array_equal(lib.slt_schedule_export(sched, "list_ptr", lo + jj), ptr)
            assert np.array_equal(lib.slt_schedule_export(sched, "list", lo + jj), its)


def test_fullsize_tiled_steps_match_oracle(lib, large):
    import torch
    cfg, mesh, sched = large
    nc = cfg["mesh"]["cell2vert"].shape[0]
    rng = np.random.default_rng(17)
    v0 = 1e-3 * rng.standard_normal((nc, 2, 6))
    s0 = 1e-3 * rng.standard_normal((nc, 3, 6))
    v, s = torch.tensor(v0, device="cuda"), torch.tensor(s0, device="cuda")
    lib.slt_execute(mesh, sched, v, s, torch.tensor(cfg["ricker"], device="cuda"), cfg["dt"], 2)
    dg = ElasticDG(cfg["mesh"], 2, cfg["rho"], cfg["lam"], cfg["mu"])
    vo, so = dg.run(v0, s0, cfg["dt"], 2, cfg["ricker"], cfg["src"])
    assert rel_l2(v.cpu().numpy(), vo) < TOL and rel_l2(s.cpu().numpy(), so) < TOL
