"""Host logic of bench.py's roofline traffic: the committed DRAM figures count only while the
executor sources they were taken on are unchanged (comments aside)."""
import json
import os

import bench


def _sources():
    texts = []
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(bench.ROOT, "paper_1708_03183_gb300", "csrc", f)) as fh:
            texts.append(fh.read())
    return texts


def test_source_digest_ignores_comments_but_not_code():
    texts = _sources()
    h0 = bench.source_digest(texts)
    assert h0 == bench.kernel_hash()
    commented = list(texts)
    commented[1] = commented[1].replace("#pragma once", "// a new remark\n/* and a block\n   comment */\n#pragma once", 1)
    assert commented[1] != texts[1] and bench.source_digest(commented) == h0
    respaced = [t.replace("\n", "\n\n") for t in texts]
    assert bench.source_digest(respaced) == h0
    changed = list(texts)
    changed[1] = changed[1].replace("#pragma once", "#pragma once\nconstexpr int kUnused = 1;", 1)
    assert bench.source_digest(changed) != h0


def test_traffic_counts_only_for_the_source_it_was_taken_on():
    table = {"k<2,256>": {"large": {"bytes_per_step": 4.5e9, "source_hash": "a" * 16}}}
    assert bench.ncu_traffic("k<2,256>", "large", 200, table, "a" * 16) == 4.5e9 * 200
    assert bench.ncu_traffic("k<2,256>", "large", 200, table, "b" * 16) is None
    assert bench.ncu_traffic("k<2,256>", "other", 200, table, "a" * 16) is None
    assert bench.ncu_traffic("k<3,256>", "large", 200, table, "a" * 16) is None


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
