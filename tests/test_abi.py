"""The C-ABI library loads, exports every entry point declared in include/slt.h, and rejects
invalid arguments on the host before any GPU work (these calls need no GPU)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def slt():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1708_03183_gb300 as m
    return m


def test_every_declared_symbol_is_exported(slt):
    names = slt.exported_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(slt.lib, n), n


def test_version_reports_sm103(slt):
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    assert slt.lib.slt_version(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 0
    assert c.value == 103


def test_chain_validation_on_host(slt):
    ch = slt.slt_chain_create()
    E = slt.slt_set(ch, 4)
    V = slt.slt_set(ch, 5)
    with pytest.raises(slt.SltError) as e:
        slt.slt_map(ch, E, V, 2, [0, 1, 1, 2, 2, 3, 3, 5])   # 5 is outside the vertex set
    assert e.value.code == -1
    with pytest.raises(slt.SltError):
        slt.slt_map(ch, E, V, 0, [])                          # arity 0
    with pytest.raises(slt.SltError):
        slt.slt_map(ch, E, V, 2, [0, -1, 1, 2, 2, 3, 3, 4])   # negative index
    m = slt.slt_map(ch, E, V, 2, [0, 1, 1, 2, 2, 3, 3, 4])
    with pytest.raises(slt.SltError):
        slt.slt_loop(ch, V, [(m, "i")])                       # map does not start at the loop's set
    with pytest.raises(slt.SltError):
        slt.slt_loop(ch, E, [(m, "x")])                       # unknown mode
    with pytest.raises(slt.SltError):
        slt.slt_loop(ch, E, [(7, "r")])                       # unknown map
    slt.slt_loop(ch, E, [(-1, "r"), (m, "i")])
    assert slt.slt_chain_info(ch) == (2, 1, 1)
    for bad in (dict(tile_size=0), dict(colouring=2), dict(max_rounds=-1), dict(split=(0,)), dict(split=(1,)),
                dict(sub_tile_size=(4, -1)), dict(seed_loop=(1,)), dict(seed_loop=(-1,)), dict(shots_per_cta=-1), dict(executor=3),
                dict(executor=4), dict(executor=5), dict(cluster_size=9), dict(release_order=3), dict(release_order=-1),
                dict(block_threads=512, executor=4)):
        with pytest.raises(slt.SltError) as e:
            slt.slt_inspect(ch, renumber=0, **bad)
        assert e.value.code == -1
    with pytest.raises(slt.SltError):
        slt.slt_inspect(ch, renumber=1)                       # no points on the seed set


def test_probe_validation_on_host(slt):
    # argument checks come before any device call
    for bad in ((0, 100, 8), (5, 100, 8), (2, 0, 8), (2, 100, 12), (2, 100, 0), (2, 100, 264), (4, 1 << 24, 256)):
        with pytest.raises(slt.SltError) as e:
            slt.slt_fp64_contraction_probe(*bad)
        assert e.value.code == -1


def test_mesh_validation_on_host(slt):
    import synth
    m = synth.make_mesh(3, 3, seed=0)
    rho, lam, mu = synth.homogeneous(m)
    cases = [dict(degree=0), dict(degree=5), dict(rho=-rho), dict(cellxy=np.full_like(m["cellxy"], np.nan))]
    for c in cases:
        args = dict(cell2vert=m["cell2vert"], cellxy=m["cellxy"], degree=1, rho=rho, lam=lam, mu=mu)
        args.update(c)
        with pytest.raises(slt.SltError) as e:
            slt.slt_mesh_create(stream=0, **args)
        assert e.value.code == -1
    bad = m["cell2vert"].copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(slt.SltError):
        slt.slt_mesh_create(bad, m["cellxy"], 1, rho, lam, mu, stream=0)
