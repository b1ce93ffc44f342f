"""The benchmark's reading of the committed ncu summaries (CPU only).

bench.py takes per-cell instruction counts and DRAM bytes from the
machine-readable lines of profiles/*.md, and only while the summary's kernel
source hash equals the current source's: a figure measured on other code is
never reported.  These checks cover that parsing and gating, and that every
summary bench.py names carries the keys it reads.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SUMMARIES = {
    "assemble_mixed_256x256x128_instmix.md": (bench.KERNEL_SOURCES, ["warp_instructions_per_cell", "dram_bytes_per_cell",
                                                                     "variant"]),
    "jvp_mixed_256x256x128.md": (bench.JVP_SOURCES, ["warp_instructions_per_cell", "dram_bytes_per_cell"]),
    "vjp_mixed_128x128x128.md": (bench.VJP_SOURCES, ["warp_instructions_per_cell", "dram_bytes_per_launch"]),
    "assemble_fp64_256x256x128_ops.md": (bench.FP64_SOURCES, ["fp64_ops_per_cell"]),
    "mesh_mixed_256x256x128_faulted.md": (bench.MESH_SOURCES, ["dram_bytes_per_launch"]),
}


@pytest.mark.parametrize("name", sorted(SUMMARIES))
def test_every_summary_has_the_keys_bench_reads(name):
    path = os.path.join(ROOT, "profiles", name)
    text = open(path).read()
    assert "`kernel_source_sha256_16`:" in text
    for key in SUMMARIES[name][1]:
        assert f"`{key}`:" in text, key
    assert "--clock-control none" in text  # every recipe leaves the clocks alone


def test_figures_are_used_only_for_the_source_they_were_taken_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    current = bench.kernel_source_hash()
    summary = ("# a summary\n\nMachine-readable (read by bench.py):\n"
               "- `kernel_source_sha256_16`: `%s`\n- `dram_bytes_per_cell`: `100.5`\n"
               "- `warp_instructions_per_cell`: `16.0`\n")
    (tmp_path / "profiles" / "now.md").write_text(summary % current)
    (tmp_path / "profiles" / "old.md").write_text(summary % "0123456789abcdef")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    # the source hash is computed from the package sources, not from ROOT's
    monkeypatch.setattr(bench, "kernel_source_hash", lambda sources=None: current)
    vals = bench.profile_values("now.md")
    assert bench.profile_number(vals, "warp_instructions_per_cell") == 16.0
    assert bench.scaled_traffic(vals, 1000) == pytest.approx(100500.0)
    assert bench.profile_values("old.md") == {}
    assert bench.scaled_traffic(bench.profile_values("old.md"), 1000) is None
    assert bench.profile_values("missing.md") == {}
    assert bench.profile_number({}, "anything") is None


def test_source_hash_covers_the_two_cell_march():
    """The headline kernel's hash changes with the two-cell march's source."""
    assert "tpfa_xmarch.cuh" in bench.KERNEL_SOURCES
    assert bench.kernel_source_hash() != bench.kernel_source_hash(bench.FP64_SOURCES)


def test_algorithmic_bytes_of_the_headline_workload():
    """The roofline's numerator on 512 x 512 x 256 with 10 links: reads of
    p, p^n (FP32), m^n (FP64), five owned transmissibilities and depth
    (FP32), 40 B per cell; writes of R and diag64 (FP64) and one FP32 value
    per CSR entry (736,101,376 entries, the pattern's closed form)."""
    n, nnz = 512 * 512 * 256, 736101376
    assert bench.algorithmic_bytes(n, nnz, "mixed") == 40 * n + 16 * n + 4 * nnz == 6702501888
    # c_r != 0 adds the FP32 phi0 read
    assert bench.algorithmic_bytes(n, nnz, "mixed", crk=True) == 6702501888 + 4 * n
    # FP64: every field and value 8 bytes, no separate diagonal
    assert bench.algorithmic_bytes(n, nnz, "fp64") == 72 * n + 8 * n + 8 * nnz


def test_host_info_names_the_cpu(tmp_path):
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU architecture: 8\n"
                   "CPU variant\t: 0x0\nCPU part\t: 0xd4f\nCPU revision\t: 0\n\nprocessor\t: 1\nCPU part\t: 0xd4f\n")
    assert bench.host_info(str(arm))["cpu_model"] == "Arm Neoverse V2 (CPU part 0xd4f)"
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Some CPU @ 2.00GHz\n")
    assert bench.host_info(str(x86))["cpu_model"] == "Some CPU @ 2.00GHz"
    assert bench.host_info(str(tmp_path / "missing"))["cpu_model"]  # falls back to the machine name
    assert bench.host_info()["nproc"] >= 1
