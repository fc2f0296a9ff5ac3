"""Host logic of bench.py (no GPU): the ncu counters it takes from the
committed summaries under profiles/, only while they match the kernel
sources they were taken on."""
import os
import shutil

import pytest

import bench

REPO = bench.ROOT


def _tree(tmp_path, key_line, extra=""):
    """A copy of the kernel sources plus one summary file under profiles/."""
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(REPO, rel), dst)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_eval_room20_traffic.txt").write_text(
        "kernel: k_eval, one evaluation\n"
        "command: ncu --set full --clock-control none -k regex:k_eval -o x python bench.py\n"
        + key_line + "dram_bytes_per_evaluation_full_workload: 14035712\n"
        "dram_read_bytes_per_evaluation_timed_step: 2562048\n" + extra)
    return tmp_path


def test_counters_read_when_the_sources_match(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel sources sha256[:16]: PLACEHOLDER\n")
    h = bench._kernel_source_hash()
    p = tmp_path / "profiles" / "k_eval_room20_traffic.txt"
    p.write_text(p.read_text().replace("PLACEHOLDER", h))
    # (the key holds a colon: the value is split off at the first ": ")
    assert bench._profiled_traffic() == 14035712.0
    assert bench._profiled_timed_step_read() == 2562048.0
    assert bench._profiled(key="no_such_key") is None


def test_counters_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel sources sha256[:16]: PLACEHOLDER\n")
    p = tmp_path / "profiles" / "k_eval_room20_traffic.txt"
    p.write_text(p.read_text().replace("PLACEHOLDER", bench._kernel_source_hash()))
    assert bench._profiled_traffic() is not None
    # an edit to any header the kernel includes makes the summary stale
    hdr = tmp_path / "paper_2310_10578_gb300" / "csrc" / "internal.h"
    hdr.write_text(hdr.read_text() + "\n// edited\n")
    assert bench._profiled_traffic() is None
    assert bench._profiled_timed_step_read() is None


def test_missing_summary_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel sources sha256[:16]: 0000000000000000\n")
    (tmp_path / "profiles" / "k_eval_room20_traffic.txt").unlink()
    assert bench._profiled_traffic() is None


@pytest.mark.parametrize("name", ["k_eval_room20_traffic.txt", "k_eval_office_traffic.txt"])
def test_committed_summaries_name_their_sources_and_command(name):
    # each committed summary names the hash it was taken on and the full ncu
    # command (with --clock-control none) that made it
    txt = open(os.path.join(REPO, "profiles", name)).read()
    kv = dict(line.split(": ", 1) for line in txt.splitlines() if ": " in line)
    assert len(kv["kernel sources sha256[:16]"].strip()) == 16
    assert kv["command"].startswith("ncu ") and "--clock-control none" in kv["command"]
