"""Host-side logic of bench.py that feeds its JSON line, without a GPU:
the traffic table lookup (keyed by kernel variant and kernel-source hash),
the HiGHS objective used to cross-check LP solutions, and the parsing of
the clock samples taken during the timed region."""
import os

import numpy as np
import pytest

import bench
from paper_2105_12715_gb300 import lpgen


def test_traffic_lookup_matches_variant_and_hash(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    table = tmp_path / "traffic.md"
    table.write_text("| variant | source hash | bytes |\n|---|---|---|\n"
                     f"| -2 | {h} | 127874304 |\n| 4 | 0123456789abcdef | 5 |\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(table))
    assert bench.measured_traffic(-2) == 127874304.0
    assert bench.measured_traffic(4) is None      # captured with other sources
    assert bench.measured_traffic(2) is None      # no row for the variant
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.measured_traffic(-2) is None


def test_kernel_source_hash_follows_the_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2105_12715_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        (csrc / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.kernel_source_hash()
    (csrc / bench.KERNEL_SOURCES[1]).write_text("// changed\n")
    assert bench.kernel_source_hash() != a


def test_highs_objective_is_the_planted_optimum():
    pytest.importorskip("scipy")
    for d in (lpgen.tiny_standard_form(2), lpgen.adversarial(7)):
        got = bench.highs_objective(d)
        assert got == pytest.approx(d.obj_star, rel=1e-7, abs=1e-7)


def test_clock_samples_of_the_timed_region(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = ["0, 1980, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 960.0, 0x4, Not Active, Active, Not Active, Not Active"]
    with open(s.path, "w") as f:
        f.write(rows[0] + "\n")
    s.mark()                      # one sample before the region
    with open(s.path, "a") as f:
        f.write(rows[1] + "\n" + rows[2] + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc, s.f = Done(), open(os.devnull, "w")
    out = s.stop()
    # the sample just before the region and the two within it
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(s.path)
