"""Host-side logic of bench.py (no GPU): the clock-sample summary, and the
source hash that ties a committed ncu traffic figure to the kernel code it
was measured on."""
import os
import re
import shutil

import pytest

import bench


def _sampler(tmp_path, lines):
    c = bench.ClockSampler(0)
    c.proc = object()            # as if nvidia-smi had been started
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c


def test_clock_summary_reads_load_reasons_and_memory_clock(tmp_path):
    na = "Not Active"
    c = _sampler(tmp_path, [
        f"345, 2032, 150.0, 0x0, {na}, {na}, {na}, {na}, 3996",      # idle sample before the load
        f"2032, 2032, 900.0, 0x0, {na}, {na}, {na}, {na}, 3996",
        f"1900, 2032, 1100.0, 0x4, {na}, {na}, {na}, Active, 3996",
        f"2032, 2032, 950.0, 0x0, {na}, {na}, {na}, {na}, 3996",
        "garbage line",
    ])
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2032.0          # median of the samples under load (> half the max)
    assert s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["mem_mhz"] == 3996.0


def test_clock_summary_without_memory_column(tmp_path):
    na = "Not Active"
    c = _sampler(tmp_path, [f"2032, 2032, 900.0, 0x0, Active, {na}, {na}, {na}"])
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown"] and "mem_mhz" not in s


def test_code_only_drops_comments_and_blank_lines():
    src = "int a = 1;  // one\n\n   // a comment line\nint b = 2;\n"
    assert bench._code_only(src) == bench._code_only("int a = 1;\nint b = 2;")


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    dst = root / "paper_1801_07986_b300" / "csrc"
    dst.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_1801_07986_b300", "csrc")
    for f in ("pn_kernels.cu", "pn_internal.h"):
        shutil.copy(os.path.join(src, f), dst / f)
    return root, dst


def _hash_at(monkeypatch, root):
    monkeypatch.setattr(bench, "ROOT", str(root))
    return bench.kernel_source_hash("fused_packed")


def test_kernel_hash_ignores_comments_and_unused_tunables(tmp_path, monkeypatch):
    root, dst = _copy_sources(tmp_path)
    h0 = _hash_at(monkeypatch, root)
    k = (dst / "pn_kernels.cu").read_text()
    a, _ = bench._FUSED_REGION
    i = k.index("\n", k.index(a)) + 1                  # the line after the region's first
    (dst / "pn_kernels.cu").write_text(k[:i] + "// an added comment\n\n" + k[i:])
    hdr = (dst / "pn_internal.h").read_text()
    (dst / "pn_internal.h").write_text(hdr + "\nconstexpr int kUnusedByThePairKernel = 3;\n")
    assert _hash_at(monkeypatch, root) == h0


@pytest.mark.parametrize("edit", ["region", "tunable"])
def test_kernel_hash_follows_code_changes(tmp_path, monkeypatch, edit):
    root, dst = _copy_sources(tmp_path)
    h0 = _hash_at(monkeypatch, root)
    if edit == "region":
        k = (dst / "pn_kernels.cu").read_text()
        a, _ = bench._FUSED_REGION
        i = k.index("\n", k.index(a)) + 1
        (dst / "pn_kernels.cu").write_text(k[:i] + "static int pn_probe_value = 1;\n" + k[i:])
    else:
        hdr = (dst / "pn_internal.h").read_text()
        m = re.search(r"constexpr int kPackFlushSources = (\d+);", hdr)   # a tunable the kernel names
        assert m
        (dst / "pn_internal.h").write_text(
            hdr.replace(m.group(0), f"constexpr int kPackFlushSources = {2 * int(m.group(1))};"))
    assert _hash_at(monkeypatch, root) != h0


def test_committed_traffic_is_found_for_its_instantiation_only():
    """The committed 128k ncu summary names the kernel instantiation it was
    captured on; bench.py finds its traffic figure for that instantiation
    (on the current source) and for no other, e.g. the 2-way unrolled one."""
    d = os.path.join(bench.ROOT, "profiles")
    keys = []
    for f in os.listdir(d):
        if f.endswith(".md"):
            keys += re.findall(r"traffic_bytes_per_launch\[fused_packed(<[0-9,]+>)\]",
                               open(os.path.join(d, f)).read())
    assert keys, "no committed traffic figure for the packed kernel"
    inst = keys[0]
    assert bench.profiled_traffic("fused_packed", inst) is not None
    nums = [int(v) for v in inst.strip("<>").split(",")]
    other = nums[:]
    other[1] = 2 if nums[1] == 1 else 1                  # the other unroll
    assert bench.profiled_traffic("fused_packed", "<" + ",".join(map(str, other)) + ">") is None
    assert bench.profiled_traffic("fused_packed") is None  # no instantiation named
