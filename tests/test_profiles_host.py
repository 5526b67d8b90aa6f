"""The committed ncu summaries and the traffic figures bench.py reports from
them: every entry of bench.TRAFFIC names a summary that states the same
source hash and the same bytes per launch; a summary's capture commands run
committed files only, each with --clock-control none."""
from __future__ import annotations

import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))


def test_every_traffic_entry_agrees_with_its_summary():
    assert bench.TRAFFIC, "no measured traffic at all"
    for (src_hash, workload), (bytes_per_launch, summary) in bench.TRAFFIC.items():
        assert re.fullmatch(r"[0-9a-f]{16}", src_hash), src_hash
        path = os.path.join(ROOT, summary)
        assert os.path.isfile(path), summary
        text = open(path).read()
        assert src_hash in text, (summary, src_hash)
        # the summary's total per launch, in GB with two decimals
        assert f"total per launch | {bytes_per_launch / 1e9:.2f} GB" in text, (summary, bytes_per_launch)
        # the summary's workload is the bench workload the figure is keyed on
        shape = re.match(r"sweep-(\d+x\d+x\d+)-s([0-9.]+)", workload)
        assert shape is not None, workload
        assert f"sweep {shape.group(1)} at {int(float(shape.group(2)) * 100)}% zeros" in text, (summary, workload)
        assert ("--lazy" in text) == workload.endswith("-lazy"), (summary, workload)


def test_measured_traffic_is_keyed_on_the_current_sources():
    current = bench.kernel_hash()
    for (src_hash, workload), (bytes_per_launch, _) in bench.TRAFFIC.items():
        if src_hash == current:
            assert bench.measured_traffic(workload) == bytes_per_launch
    # a workload without a capture on these sources reports no traffic
    assert bench.measured_traffic("no-such-workload") is None


def test_summaries_give_runnable_commands_on_committed_files():
    names = _summaries()
    assert names
    for name in names:
        text = open(os.path.join(PROFILES, name)).read()
        joined = re.sub(r"\\\n\s*", " ", text)  # continuation lines joined
        # commands are the summary's indented code lines that run ncu
        cmds = [ln.strip() for ln in joined.splitlines() if re.match(r" {4,}(\w+=\S+\s+)*ncu\s", ln)]
        assert cmds, f"{name}: no ncu command"
        for ln in cmds:
            if "<the same" in ln:
                continue  # a repeat of the command above with one option changed
            assert "--clock-control none" in ln, f"{name}: {ln}"
            assert "python bench.py" in ln, f"{name}: {ln}"
        assert "_work" not in text, name
    for f in os.listdir(PROFILES):
        assert f.endswith((".md", ".txt")), f"raw or runnable file under profiles/: {f}"
