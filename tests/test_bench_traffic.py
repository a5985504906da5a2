"""Host logic of bench.py's roofline traffic: the committed DRAM figures count only while the
executor sources they were taken on are unchanged (comments aside)."""
import json
import os
import shutil

import bench

SOURCES = ("exec.cu", "exec_body.cuh", "dataflow.cuh", "internal.h")


def _copy_tree(tmp_path):
    csrc = tmp_path / "paper_1708_03183_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1708_03183_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    assert h0 == bench.kernel_hash()
    p = csrc / "exec_body.cuh"
    src = p.read_text()
    p.write_text(src.replace("#pragma once", "// a new remark\n/* and a block\n   comment */\n#pragma once", 1))
    assert bench.kernel_hash() == h0
    p.write_text(src.replace("#pragma once", "#pragma once\nconstexpr int kUnused = 1;", 1))
    assert bench.kernel_hash() != h0


def test_traffic_counts_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"bytes_per_step": 4.5e9, "source_hash": bench.kernel_hash()}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k<2,256>": {"large": entry}}))
    assert bench.ncu_traffic("k<2,256>", "large", 200) == 4.5e9 * 200
    assert bench.ncu_traffic("k<2,256>", "other", 200) is None
    assert bench.ncu_traffic("k<3,256>", "large", 200) is None
    entry["source_hash"] = "0" * 16
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k<2,256>": {"large": entry}}))
    assert bench.ncu_traffic("k<2,256>", "large", 200) is None


def test_committed_traffic_entries_are_complete():
    # every committed figure names its source hash and the command that took it; a stale hash only
    # makes bench.py report null, it is not an error
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for kernel, per in d.items():
        for workload, e in per.items():
            assert len(e["source_hash"]) == 16 and e["command"].startswith("ncu "), (kernel, workload)
            assert "--clock-control none" in e["command"]
            assert e["bytes_per_step"] == e["read_bytes_per_step"] + e["write_bytes_per_step"]
