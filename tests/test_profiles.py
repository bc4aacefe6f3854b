"""The committed ncu summaries stay tied to the code they describe: the bench's
roofline quotes the DRAM traffic of profiles/traffic.json only for the kernel
source it was captured on (same sha256), and every summary gives a command that
runs committed files only (no scratch scripts)."""
import hashlib
import json
import os
import re


def test_bench_quotes_traffic_only_for_the_captured_source(repo_root):
    """bench.py's roofline takes the DRAM bytes of the committed capture only while
    the kernel's source still has the hash it had at the capture, else null."""
    import bench

    with open(os.path.join(repo_root, "profiles", "traffic.json")) as f:
        tab = json.load(f)
    assert tab
    for cls, ent in tab.items():
        src = os.path.join(repo_root, ent["source"])
        assert os.path.exists(src), (cls, ent["source"])
        with open(src, "rb") as f:
            same = hashlib.sha256(f.read()).hexdigest() == ent["source_sha256"]
        traffic, why = bench._traffic(cls)
        if same:
            assert traffic == ent["dram_bytes_per_launch"] > 0
        else:
            assert traffic is None and "changed" in why


def test_summaries_give_commands_on_committed_files(repo_root):
    d = os.path.join(repo_root, "profiles")
    mds = [f for f in os.listdir(d) if f.endswith(".md")]
    assert mds
    for name in mds:
        with open(os.path.join(d, name)) as f:
            text = f.read()
        assert "ncu " in text and "--clock-control none" in text, name
        assert "_work" not in text, name
        for script in re.findall(r"python ([\w./-]+\.py)", text):
            assert os.path.exists(os.path.join(repo_root, script)), (name, script)
