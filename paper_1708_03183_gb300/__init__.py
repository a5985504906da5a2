"""Python binding of libslt.so: sparse-tiled DG elastic-wave time stepping on GB300.

Argument marshalling only: every step of the inspector and executor runs in the CUDA library.
The functions keep the names of the C entry points (include/slt.h).  Device arrays are torch
CUDA tensors (float64 / int32, contiguous); host arrays are numpy arrays.  Importing this
package loads the in-tree library and raises ImportError if it has not been built
(python paper_1708_03183_gb300/build.py, or __graft_entry__.build()); there is no fallback
implementation.
"""
import ctypes
import os

import numpy as np

from . import build as _build_mod

_LIB_PATH = _build_mod.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError("libslt.so is not built (%s); run python paper_1708_03183_gb300/build.py" % _LIB_PATH)
lib = ctypes.CDLL(_LIB_PATH)

P = ctypes.c_void_p
I32, I64, F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class slt_options(ctypes.Structure):
    _fields_ = [("tile_size", I32), ("colouring", I32), ("renumber", I32), ("max_rounds", I32),
                ("prio_seed", ctypes.c_uint64), ("nsplit", I32), ("split", I32 * 15), ("executor", I32),
                ("wait_spins", I32), ("block_threads", I32), ("sub_tile_size", I32 * 16),
                ("cluster_size", I32), ("shots_per_cta", I32), ("seed_loop", I32 * 16),
                ("release_order", I32)]


_SIGS = {
    "slt_last_error": (ctypes.c_char_p, []),
    "slt_version": (ctypes.c_int, [P, P, P]),
    "slt_chain_create": (ctypes.c_int, [P]),
    "slt_chain_destroy": (ctypes.c_int, [P]),
    "slt_set": (ctypes.c_int, [P, I64, P]),
    "slt_map": (ctypes.c_int, [P, I32, I32, I32, P, P]),
    "slt_loop": (ctypes.c_int, [P, I32, I32, P, P, P]),
    "slt_set_points": (ctypes.c_int, [P, I32, P]),
    "slt_chain_info": (ctypes.c_int, [P, P, P, P]),
    "slt_options_default": (ctypes.c_int, [P]),
    "slt_inspect": (ctypes.c_int, [P, P, P, P]),
    "slt_schedule_destroy": (ctypes.c_int, [P]),
    "slt_schedule_info": (ctypes.c_int, [P, I32, P]),
    "slt_schedule_dataflow_info": (ctypes.c_int, [P, P]),
    "slt_schedule_lane_info": (ctypes.c_int, [P, P]),
    "slt_schedule_inspection_times": (ctypes.c_int, [P, P]),
    "slt_schedule_export": (ctypes.c_int, [P, I32, I32, I32, P, P]),
    "slt_mesh_create": (ctypes.c_int, [P, P, I64, I32, P, P, P, P, P, P]),
    "slt_mesh_destroy": (ctypes.c_int, [P]),
    "slt_mesh_info": (ctypes.c_int, [P, P]),
    "slt_mesh_chain": (ctypes.c_int, [P, P]),
    "slt_mesh_cost": (ctypes.c_int, [P, P]),
    "slt_execute": (ctypes.c_int, [P, P, P, P, P, F64, I64, P]),
    "slt_execute_host": (ctypes.c_int, [P, P, P, P, P, F64, I64, P]),
    "slt_execute_profiled": (ctypes.c_int, [P, P, P, P, P, F64, I64, P, P]),
    "slt_execute_batched": (ctypes.c_int, [P, P, I32, P, P, P, P, F64, I64, P, P]),
    "slt_autotune": (ctypes.c_int, [P, P, I32, P, I32, I32, P, I32, P, I32, I32, P, P, P]),
    "slt_execute_many": (ctypes.c_int, [I32, P, P, P, P, P, P, I64, P]),
    "slt_group_create": (ctypes.c_int, [I32, P, P, P]),
    "slt_group_destroy": (ctypes.c_int, [P]),
    "slt_group_execute": (ctypes.c_int, [P, P, P, P, P, I64, P]),
    "slt_group_create_batched": (ctypes.c_int, [I32, P, P, P, P, P]),
    "slt_group_graph_replays": (ctypes.c_int, [P, P]),
    "slt_apply_operator": (ctypes.c_int, [P, I32, P, P, P]),
    "slt_seed_rank_noalloc": (ctypes.c_int, [P, I64, P, P]),
    "slt_fp64_peak": (ctypes.c_int, [P, P]),
    "slt_fp64_lane_probe": (ctypes.c_int, [P, P]),
    "slt_fp64_contraction_probe": (ctypes.c_int, [I32, I64, I32, P, P]),
    "slt_mesh_set_material": (ctypes.c_int, [P, P, P, P, P]),
    "slt_mesh_set_source": (ctypes.c_int, [P, P, P]),
    "slt_receivers_create": (ctypes.c_int, [P, I32, P, P]),
    "slt_receivers_destroy": (ctypes.c_int, [P]),
    "slt_record": (ctypes.c_int, [P, P, P, P, F64, I64, P, P]),
    "slt_adjoint": (ctypes.c_int, [P, P, P, P, F64, I64, P, I32, P, P, P]),
    "slt_record_batched": (ctypes.c_int, [P, P, P, I32, P, P, F64, I64, P, P]),
    "slt_adjoint_batched": (ctypes.c_int, [P, P, P, I32, P, P, F64, I64, P, I32, P, P, P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype, _f.argtypes = _res, _args

STATUS = {0: "SLT_OK", -1: "SLT_ERR_ARG", -2: "SLT_ERR_OOM", -3: "SLT_ERR_CUDA", -4: "SLT_ERR_TIMEOUT",
          -5: "SLT_ERR_CONFLICT_CAP", -6: "SLT_ERR_UNSUPPORTED", -7: "SLT_ERR_STATE"}


class SltError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def _check(rc):
    if rc != 0:
        raise SltError(rc, lib.slt_last_error().decode(errors="replace"))


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


def _dev(t, dtype_name):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch." + dtype_name):
        raise ValueError("expected a contiguous CUDA %s tensor" % dtype_name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    """A cudaStream_t: the given handle, torch's current stream, or NULL (legacy default)."""
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream)) if int(stream) else None


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(lib, self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chain(_Handle):
    _destroy = "slt_chain_destroy"


class Schedule(_Handle):
    _destroy = "slt_schedule_destroy"


class Mesh(_Handle):
    _destroy = "slt_mesh_destroy"


class Receivers(_Handle):
    _destroy = "slt_receivers_destroy"


# ------------------------------------------------------------------ loop chain
def slt_chain_create():
    h = ctypes.c_void_p()
    _check(lib.slt_chain_create(ctypes.byref(h)))
    return Chain(h)


def slt_set(chain, size):
    i = I32()
    _check(lib.slt_set(chain.ptr, int(size), ctypes.byref(i)))
    return i.value


def slt_map(chain, from_set, to_set, arity, values):
    v, vp = _host(np.asarray(values).ravel(), np.int32)
    i = I32()
    _check(lib.slt_map(chain.ptr, from_set, to_set, arity, vp, ctypes.byref(i)))
    return i.value


def slt_loop(chain, set_id, descs):
    """descs: list of (map id or -1, mode char)."""
    ids, idp = _host([d[0] for d in descs], np.int32)
    modes = ctypes.create_string_buffer("".join(d[1] for d in descs).encode())
    i = I32()
    _check(lib.slt_loop(chain.ptr, set_id, len(descs), idp, modes, ctypes.byref(i)))
    return i.value


def slt_set_points(chain, set_id, xy):
    a, ap = _host(xy, np.float64)
    _check(lib.slt_set_points(chain.ptr, set_id, ap))


def slt_chain_info(chain):
    a, b, c = I32(), I32(), I32()
    _check(lib.slt_chain_info(chain.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


# ------------------------------------------------------------------ inspector
def slt_options_default(**kw):
    o = slt_options()
    _check(lib.slt_options_default(ctypes.byref(o)))
    split = kw.pop("split", ())
    for i, t in enumerate(kw.pop("sub_tile_size", ())):
        o.sub_tile_size[i] = t
    for i, t in enumerate(kw.pop("seed_loop", ())):
        o.seed_loop[i] = t
    for k, v in kw.items():
        setattr(o, k, v)
    o.nsplit = len(split)
    for i, s in enumerate(split):
        o.split[i] = s
    return o


def slt_inspect(chain, opts=None, stream=None, **kw):
    if opts is None:
        opts = slt_options_default(**kw)
    h = ctypes.c_void_p()
    _check(lib.slt_inspect(chain.ptr, ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return Schedule(h)


def slt_schedule_info(sched, sub):
    info = np.zeros(8, dtype=np.int64)
    _check(lib.slt_schedule_info(sched.ptr, sub, ctypes.c_void_p(info.ctypes.data)))
    keys = ["ntiles", "ncolours", "restarts", "fell_back", "conflicts", "unprojected", "first", "nloops"]
    return dict(zip(keys, (int(x) for x in info)))


def slt_schedule_dataflow_info(sched):
    info = np.zeros(6, dtype=np.float64)
    _check(lib.slt_schedule_dataflow_info(sched.ptr, ctypes.c_void_p(info.ctypes.data)))
    keys = ["nodes_per_step", "deps_per_step", "critical_path_nodes", "critical_path_items", "items_per_step",
            "tiles_in_flight"]
    return dict(zip(keys, (float(x) for x in info)))


def slt_schedule_lane_info(sched):
    """FP64 warp-lane instructions of one step: needed, issued by the dataflow executors, by the
    staged executor's passes, by the untiled chain."""
    info = np.zeros(4, dtype=np.float64)
    _check(lib.slt_schedule_lane_info(sched.ptr, ctypes.c_void_p(info.ctypes.data)))
    return dict(needed=float(info[0]), dataflow=float(info[1]), staged=float(info[2]), untiled=float(info[3]),
                dataflow_efficiency=float(info[0] / info[1]), staged_efficiency=float(info[0] / info[2]),
                untiled_efficiency=float(info[0] / info[3]))


def slt_schedule_inspection_times(sched):
    """Seconds of slt_inspect per stage."""
    t = np.zeros(8, dtype=np.float64)
    _check(lib.slt_schedule_inspection_times(sched.ptr, ctypes.c_void_p(t.ctypes.data)))
    return dict(partition=float(t[0]), colour_project_tile=float(t[1]), iteration_lists=float(t[2]),
                executor_plans=float(t[3]), staged_plans=float(t[4]), dataflow_graph=float(t[5]))


EXPORT_KINDS = {"rank": 0, "colour": 1, "sigma": 2, "list_ptr": 3, "list": 4, "fp_ptr": 5, "fp": 6, "lmap": 7,
                "succ_ptr": 8, "succ": 9, "indeg0": 10, "indeg": 11, "fp_stage_ptr": 12, "fp_stage": 13, "export": 14}


def slt_schedule_export(sched, kind, loop, desc=0):
    k = EXPORT_KINDS.get(kind, kind)
    n = I64()
    _check(lib.slt_schedule_export(sched.ptr, k, loop, desc, None, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib.slt_schedule_export(sched.ptr, k, loop, desc, ctypes.c_void_p(out.ctypes.data), ctypes.byref(n)))
    return out[:n.value]


# ------------------------------------------------------------------ mesh and executor
def slt_mesh_create(cell2vert, cellxy, degree, rho, lam, mu, src_xy=None, stream=None):
    c2v, c2vp = _host(cell2vert, np.int32)
    xy, xyp = _host(cellxy, np.float64)
    r, rp = _host(rho, np.float64)
    l, lp = _host(lam, np.float64)
    m, mp = _host(mu, np.float64)
    sp = None
    if src_xy is not None:
        s, sp = _host(src_xy, np.float64)
    h = ctypes.c_void_p()
    _check(lib.slt_mesh_create(c2vp, xyp, c2v.shape[0], degree, rp, lp, mp, sp, _stream(stream), ctypes.byref(h)))
    return Mesh(h)


def slt_mesh_info(mesh):
    info = np.zeros(8, dtype=np.int64)
    _check(lib.slt_mesh_info(mesh.ptr, ctypes.c_void_p(info.ctypes.data)))
    keys = ["ncell", "degree", "Np", "nfi", "nfe", "src_cell", "nloops", "split"]
    return dict(zip(keys, (int(x) for x in info)))


def slt_mesh_cost(mesh):
    c = np.zeros(4, dtype=np.float64)
    _check(lib.slt_mesh_cost(mesh.ptr, ctypes.c_void_p(c.ctypes.data)))
    return dict(flops_per_step=float(c[0]), tiled_bytes_per_step=float(c[1]), untiled_bytes_per_step=float(c[2]),
                nnz_dr_ds=int(c[3]))


def slt_fp64_peak(stream=None):
    """Measured FP64 throughput of this GPU (TFLOP/s): DFMA, DMMA (mma.sync m8n8k4), both at once."""
    o = np.zeros(4, dtype=np.float64)
    _check(lib.slt_fp64_peak(_stream(stream), ctypes.c_void_p(o.ctypes.data)))
    return dict(dfma_tflops=float(o[0]), dmma_tflops=float(o[1]), mixed_tflops=float(o[2]), probe_ms=float(o[3]))


def slt_fp64_lane_probe(stream=None):
    """DFMA warp instructions per clock per SM: 32 lanes, 16 lanes, one warp per SM, four warps per SM."""
    o = np.zeros(4, dtype=np.float64)
    _check(lib.slt_fp64_lane_probe(_stream(stream), ctypes.c_void_p(o.ctypes.data)))
    return dict(full_warps=float(o[0]), half_warps=float(o[1]), one_warp_per_sm=float(o[2]),
                four_warps_per_sm=float(o[3]))


def slt_fp64_contraction_probe(degree, ncell, nshots, stream=None):
    o = np.zeros(6)
    _check(lib.slt_fp64_contraction_probe(int(degree), int(ncell), int(nshots), _stream(stream),
                                          ctypes.c_void_p(o.ctypes.data)))
    return {"dfma_ms": o[0], "dmma_ms": o[1], "rel_diff": o[2], "useful_flops": o[3], "dmma_issued_flops": o[4],
            "nnz": int(o[5])}


def slt_mesh_chain(mesh):
    h = ctypes.c_void_p()
    _check(lib.slt_mesh_chain(mesh.ptr, ctypes.byref(h)))
    return Chain(h)


def _check_fields(mesh, v, sigma, ricker, nsteps, nshots=1):
    info = slt_mesh_info(mesh)
    nv, ns = info["ncell"] * 2 * info["Np"] * nshots, info["ncell"] * 3 * info["Np"] * nshots
    if v.numel() != nv or sigma.numel() != ns:
        raise ValueError("v needs %d and sigma %d float64 values" % (nv, ns))
    if ricker is not None and ricker.numel() < nsteps:
        raise ValueError("the source series is shorter than nsteps")


def slt_execute(mesh, sched, v, sigma, ricker, dt, nsteps, stream=None):
    """v [ncell, 2, Np], sigma [ncell, 3, Np]: CUDA float64 tensors, updated in place;
    ricker: CUDA float64 [nsteps] or None; sched None = plain untiled chain."""
    _check_fields(mesh, v, sigma, ricker, nsteps)
    _check(lib.slt_execute(mesh.ptr, sched.ptr if sched is not None else None, _dev(v, "float64"),
                           _dev(sigma, "float64"), _dev(ricker, "float64"), float(dt), int(nsteps), _stream(stream)))


def slt_execute_profiled(mesh, sched, v, sigma, ricker, dt, nsteps, stream=None):
    """slt_execute with per-launch CUDA-event timing; returns a dict of kernel times."""
    _check_fields(mesh, v, sigma, ricker, nsteps)
    prof = np.zeros(8, dtype=np.float64)
    _check(lib.slt_execute_profiled(mesh.ptr, sched.ptr if sched is not None else None, _dev(v, "float64"),
                                    _dev(sigma, "float64"), _dev(ricker, "float64"), float(dt), int(nsteps),
                                    _stream(stream), ctypes.c_void_p(prof.ctypes.data)))
    return dict(chain_ms=prof[0], chain_launches=int(prof[1]), layout_ms=prof[2], layout_launches=int(prof[3]),
                max_launch_ms=prof[4], min_launch_ms=prof[5], setup_ms=prof[6], setup_launches=int(prof[7]))


def slt_execute_batched(mesh, sched, src_xy, v, sigma, ricker, dt, nsteps, stream=None, profile=False):
    """Many shots at once: src_xy [nshots, 2] (host; None = no sources, then nshots comes from v),
    v [ncell, 2, Np, nshots] and sigma [ncell, 3, Np, nshots] CUDA float64 tensors (shots
    innermost), updated in place.  sched None = untiled.  profile=True returns the kernel times."""
    if src_xy is not None:
        xy, xyp = _host(src_xy, np.float64)
        if xy.ndim != 2 or xy.shape[1] != 2:
            raise ValueError("src_xy must be [nshots, 2]")
        S = xy.shape[0]
    else:
        xyp, S = None, int(v.shape[-1])
    if v.dim() != 4 or v.shape[-1] != S or sigma.dim() != 4 or sigma.shape[-1] != S:
        raise ValueError("v and sigma need the shots as their last dimension (%d)" % S)
    _check_fields(mesh, _np_numel(np.empty(v.numel() // S)), _np_numel(np.empty(sigma.numel() // S)), ricker, nsteps)
    prof = np.zeros(8, dtype=np.float64)
    _check(lib.slt_execute_batched(mesh.ptr, sched.ptr if sched is not None else None, S, xyp, _dev(v, "float64"),
                                   _dev(sigma, "float64"), _dev(ricker, "float64"), float(dt), int(nsteps),
                                   _stream(stream), ctypes.c_void_p(prof.ctypes.data) if profile else None))
    if profile:
        return dict(chain_ms=prof[0], chain_launches=int(prof[1]), layout_ms=prof[2], layout_launches=int(prof[3]),
                    max_launch_ms=prof[4], min_launch_ms=prof[5], setup_ms=prof[6], setup_launches=int(prof[7]))


def _group_args(meshes, vs, sigmas, rickers, dts, nsteps, nshots=None):
    n = len(meshes)
    if not (len(vs) == len(sigmas) == len(rickers) == len(dts) == n):
        raise ValueError("one field pair, source series and dt per mesh")
    for i, (m, v, s_, r) in enumerate(zip(meshes, vs, sigmas, rickers)):
        _check_fields(m, v, s_, r, nsteps, nshots[i] if nshots else 1)
    arr = lambda xs: (ctypes.c_void_p * n)(*xs)
    return (arr([_dev(v, "float64") for v in vs]), arr([_dev(x, "float64") for x in sigmas]),
            arr([_dev(r, "float64") for r in rickers]), (ctypes.c_double * n)(*[float(d) for d in dts]))


class Group(_Handle):
    _destroy = "slt_group_destroy"


def slt_group_create(meshes, scheds):
    """Bind meshes to their schedules (None = untiled) for joint execution."""
    n = len(meshes)
    if len(scheds) != n:
        raise ValueError("one schedule (or None) per mesh")
    arr = lambda xs: (ctypes.c_void_p * n)(*xs)
    h = ctypes.c_void_p()
    _check(lib.slt_group_create(n, arr([m.ptr for m in meshes]), arr([s.ptr if s is not None else None for s in scheds]),
                                ctypes.byref(h)))
    g = Group(h)
    g.meshes = list(meshes)   # keep the members alive as long as the group
    g.scheds = list(scheds)
    return g


def slt_group_create_batched(meshes, scheds, nshots, src_xy):
    """The batched form in one persistent, graph-captured launch: members of any degree 1-3,
    member i with nshots[i] shots (sources src_xy[i] [nshots[i], 2], host, or None)."""
    n = len(meshes)
    if not (len(scheds) == len(nshots) == len(src_xy) == n):
        raise ValueError("one schedule, shot count and source array per mesh")
    arr = lambda xs: (ctypes.c_void_p * n)(*xs)
    keep = [None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 2))
            for x in src_xy]
    for k, x in zip(nshots, keep):
        if x is not None and x.shape[0] != k:
            raise ValueError("src_xy[i] needs nshots[i] points")
    h = ctypes.c_void_p()
    _check(lib.slt_group_create_batched(n, arr([m.ptr for m in meshes]),
                                        arr([s.ptr if s is not None else None for s in scheds]),
                                        (ctypes.c_int32 * n)(*[int(k) for k in nshots]),
                                        arr([None if x is None else x.ctypes.data for x in keep]), ctypes.byref(h)))
    g = Group(h)
    g.meshes = list(meshes)
    g.scheds = list(scheds)
    g.nshots = [int(k) for k in nshots]
    return g


def slt_group_graph_replays(group):
    r = I64()
    _check(lib.slt_group_graph_replays(group.ptr, ctypes.byref(r)))
    return r.value


def slt_group_execute(group, vs, sigmas, rickers, dts, nsteps, stream=None):
    """Advance every mesh of the group; per mesh: v [ncell, 2, Np] and sigma [ncell, 3, Np] CUDA
    float64 tensors updated in place ([ncell, 2, Np, nshots], [ncell, 3, Np, nshots] for a member
    with several shots), ricker (CUDA float64 or None), dt."""
    v, s_, r, d = _group_args(group.meshes, vs, sigmas, rickers, dts, nsteps, getattr(group, "nshots", None))
    _check(lib.slt_group_execute(group.ptr, v, s_, r, d, int(nsteps), _stream(stream)))


def slt_execute_many(meshes, scheds, vs, sigmas, rickers, dts, nsteps, stream=None):
    """One-off joint execution (slt_group_create + slt_group_execute)."""
    n = len(meshes)
    if len(scheds) != n:
        raise ValueError("one schedule (or None) per mesh")
    v, s_, r, d = _group_args(meshes, vs, sigmas, rickers, dts, nsteps)
    arr = lambda xs: (ctypes.c_void_p * n)(*xs)
    _check(lib.slt_execute_many(n, arr([m.ptr for m in meshes]), arr([s.ptr if s is not None else None for s in scheds]),
                                v, s_, r, d, int(nsteps), _stream(stream)))


def slt_autotune(mesh, tile_sizes, nshots=1, shapes=False, block_threads=(256,), shots_per_cta=(), steps=5,
                 base=None, stream=None, **kw):
    """Time the untiled chain and every (tile size, shape, CTA size, shots per CTA) candidate on
    this mesh; returns (best slt_options, table rows (tile_size, renumber, block_threads,
    shots_per_cta, ms/step))."""
    base = base if base is not None else slt_options_default(**kw)
    ts, tsp = _host(np.asarray(tile_sizes, dtype=np.int32), np.int32)
    bt, btp = _host(np.asarray(block_threads, dtype=np.int32), np.int32)
    sg, sgp = _host(np.asarray(shots_per_cta if len(shots_per_cta) else [0], dtype=np.int32), np.int32)
    ng = len(shots_per_cta)
    rows = 1 + len(ts) * (2 if shapes else 1) * len(bt) * (max(ng, 1) if nshots > 1 else 1)
    table = np.zeros((rows, 5), dtype=np.float64)
    best = slt_options()
    _check(lib.slt_autotune(mesh.ptr, ctypes.byref(base), int(nshots), tsp, len(ts), int(bool(shapes)), btp, len(bt),
                            sgp if ng else None, ng, int(steps), _stream(stream), ctypes.byref(best),
                            ctypes.c_void_p(table.ctypes.data)))
    return best, table


def slt_execute_host(mesh, sched, v, sigma, ricker, dt, nsteps, stream=None):
    """Host (numpy or pinned CPU torch) fields, updated in place; returns when done."""
    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("expected a contiguous CPU tensor")
            return ctypes.c_void_p(a.data_ptr())
        if not (a.flags["C_CONTIGUOUS"] and a.dtype == np.float64):
            raise ValueError("expected a C-contiguous float64 array")
        return ctypes.c_void_p(a.ctypes.data)
    _check_fields(mesh, v if hasattr(v, "numel") else _np_numel(v), sigma if hasattr(sigma, "numel") else _np_numel(sigma),
                  None if ricker is None else (ricker if hasattr(ricker, "numel") else _np_numel(ricker)), nsteps)
    _check(lib.slt_execute_host(mesh.ptr, sched.ptr if sched is not None else None, ptr(v), ptr(sigma),
                                ptr(ricker), float(dt), int(nsteps), _stream(stream)))


class _np_numel:
    def __init__(self, a):
        self.n = int(np.asarray(a).size)

    def numel(self):
        return self.n


def slt_apply_operator(mesh, op, x, out, stream=None):
    info = slt_mesh_info(mesh)
    rin, rout = (3, 2) if op == 0 else (2, 3)
    if x.numel() != info["ncell"] * rin * info["Np"] or out.numel() != info["ncell"] * rout * info["Np"]:
        raise ValueError("operator input/output sizes do not match the mesh")
    _check(lib.slt_apply_operator(mesh.ptr, op, _dev(x, "float64"), _dev(out, "float64"), _stream(stream)))


def slt_seed_rank_noalloc(xy, rank, stream=None):
    """Hilbert seed ranks of device points xy [n, 2] (float64) into rank [n] (int32), using only
    the library's fixed device scratch (no allocation; at most 1,048,576 points)."""
    n = rank.numel()
    if xy.numel() != 2 * n:
        raise ValueError("xy must hold two coordinates per rank entry")
    _check(lib.slt_seed_rank_noalloc(_dev(xy, "float64"), n, _dev(rank, "int32"), _stream(stream)))


def slt_mesh_set_material(mesh, rho, lam, mu, stream=None):
    r, rp = _host(rho, np.float64)
    l, lp = _host(lam, np.float64)
    m, mp = _host(mu, np.float64)
    n = slt_mesh_info(mesh)["ncell"]
    if r.size != n or l.size != n or m.size != n:
        raise ValueError("material arrays need one value per cell")
    _check(lib.slt_mesh_set_material(mesh.ptr, rp, lp, mp, _stream(stream)))


def slt_mesh_set_source(mesh, src_xy, stream=None):
    sp = None
    if src_xy is not None:
        s_, sp = _host(src_xy, np.float64)
    _check(lib.slt_mesh_set_source(mesh.ptr, sp, _stream(stream)))


def slt_receivers_create(mesh, xy):
    a, ap = _host(np.asarray(xy).reshape(-1, 2), np.float64)
    h = ctypes.c_void_p()
    _check(lib.slt_receivers_create(mesh.ptr, a.shape[0], ap, ctypes.byref(h)))
    rec = Receivers(h)
    rec.n = a.shape[0]
    rec.mesh = mesh
    return rec


def slt_record(mesh, sched, rec, ricker, dt, nsteps, traces, stream=None):
    """traces: CUDA float64 [nsteps, nrec, 2], written."""
    if traces.numel() != nsteps * rec.n * 2 or (ricker is not None and ricker.numel() < nsteps):
        raise ValueError("traces need nsteps * nrec * 2 values and the source series nsteps")
    _check(lib.slt_record(mesh.ptr, sched.ptr if sched is not None else None, rec.ptr, _dev(ricker, "float64"),
                          float(dt), int(nsteps), _dev(traces, "float64"), _stream(stream)))


def slt_adjoint(mesh, sched, rec, ricker, dt, nsteps, data, checkpoint_every, grad, stream=None):
    """Misfit against data [nsteps, nrec, 2] (CUDA float64) and its gradient written to grad
    [3, ncell] (CUDA float64: d/drho, d/dlambda, d/dmu).  Returns the misfit."""
    n = slt_mesh_info(mesh)["ncell"]
    if data.numel() != nsteps * rec.n * 2 or grad.numel() != 3 * n:
        raise ValueError("data needs nsteps * nrec * 2 values and grad 3 * ncell")
    if ricker is not None and ricker.numel() < nsteps:
        raise ValueError("the source series is shorter than nsteps")
    J = ctypes.c_double()
    _check(lib.slt_adjoint(mesh.ptr, sched.ptr if sched is not None else None, rec.ptr, _dev(ricker, "float64"),
                           float(dt), int(nsteps), _dev(data, "float64"), int(checkpoint_every),
                           _dev(grad, "float64"), ctypes.byref(J), _stream(stream)))
    return J.value


def exported_symbols():
    """Names of the entry points declared in include/slt.h."""
    import re
    hdr = open(os.path.join(_build_mod.ROOT, "include", "slt.h")).read()
    return sorted(set(re.findall(r"\b(slt_[a-z_]+)\s*\(", hdr)))


def slt_record_batched(mesh, sched, rec, src_xy, ricker, dt, nsteps, traces, stream=None):
    """Runs from rest of every shot (src_xy [nshots, 2], host); traces: CUDA float64
    [nsteps, nshots, nrec, 2], written."""
    xy, xyp = _host(np.asarray(src_xy).reshape(-1, 2), np.float64)
    S = xy.shape[0]
    if traces.numel() != nsteps * S * rec.n * 2 or (ricker is not None and ricker.numel() < nsteps):
        raise ValueError("traces need nsteps * nshots * nrec * 2 values and the source series nsteps")
    _check(lib.slt_record_batched(mesh.ptr, sched.ptr if sched is not None else None, rec.ptr, S, xyp,
                                  _dev(ricker, "float64"), float(dt), int(nsteps), _dev(traces, "float64"),
                                  _stream(stream)))


def slt_adjoint_batched(mesh, sched, rec, src_xy, ricker, dt, nsteps, data, checkpoint_every, grad, stream=None):
    """Summed misfit of every shot against data [nsteps, nshots, nrec, 2] (CUDA float64) and its
    gradient written to grad [3, ncell]; returns the misfit."""
    xy, xyp = _host(np.asarray(src_xy).reshape(-1, 2), np.float64)
    S = xy.shape[0]
    n = slt_mesh_info(mesh)["ncell"]
    if data.numel() != nsteps * S * rec.n * 2 or grad.numel() != 3 * n:
        raise ValueError("data needs nsteps * nshots * nrec * 2 values and grad 3 * ncell")
    if ricker is not None and ricker.numel() < nsteps:
        raise ValueError("the source series is shorter than nsteps")
    J = ctypes.c_double()
    _check(lib.slt_adjoint_batched(mesh.ptr, sched.ptr if sched is not None else None, rec.ptr, S, xyp,
                                   _dev(ricker, "float64"), float(dt), int(nsteps), _dev(data, "float64"),
                                   int(checkpoint_every), _dev(grad, "float64"), ctypes.byref(J), _stream(stream)))
    return J.value

