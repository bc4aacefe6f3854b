"""The committed ncu summaries stay tied to the code they describe: the DRAM traffic
the bench's roofline quotes (profiles/traffic.json) belongs to the current source
of its kernel (same sha256), and every summary gives a command that runs committed
files only (no scratch scripts)."""
import hashlib
import json
import os
import re


def test_traffic_table_matches_the_kernel_source(repo_root):
    with open(os.path.join(repo_root, "profiles", "traffic.json")) as f:
        tab = json.load(f)
    assert tab
    for cls, ent in tab.items():
        src = os.path.join(repo_root, ent["source"])
        assert os.path.exists(src), (cls, ent["source"])
        with open(src, "rb") as f:
            assert hashlib.sha256(f.read()).hexdigest() == ent["source_sha256"], (
                f"{ent['source']} changed since its ncu capture: take the capture again")
        assert ent["dram_bytes_per_launch"] > 0


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
