"""Host-side logic of bench.py that decides whether a run is kept: the summary of the GPU clocks
sampled during the timed region (median SM clock under load, throttle reasons, power), the
number of the committed ncu summary it may report, and the HBM peak it divides by."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _line(sm, mx=2070, power=800.0, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    return "0, %s, %s, %s, %s, %s, %s, %s, %s" % (sm, mx, power, active, hw, hwt, swt, cap)


def test_median_under_load_ignores_idle_samples():
    lines = [_line(345), _line(2070), _line(2055), _line(2070), _line(400)]
    c = bench.summarize_clocks(lines)
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["samples"] == 5
    assert c["reasons"] == [] and c["power_w_max"] == 800.0


def test_all_idle_samples_still_give_a_median():
    c = bench.summarize_clocks([_line(300), _line(330), _line(360)])
    assert c["sm_mhz"] == 330


def test_throttle_reasons_are_collected():
    lines = [_line(2070), _line(1800, hwt="Active"), _line(1900, cap="Active"), _line(1950, swt="active")]
    c = bench.summarize_clocks(lines)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1925


def test_unparsable_lines_and_missing_power_are_tolerated():
    lines = ["", "garbage", _line("[N/A]"), _line(2070, power="[N/A]"), _line(2040, power=950.5),
             "0, 1, 2"]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 2 and c["sm_mhz"] == 2055 and c["power_w_max"] == 950.5


def test_no_samples():
    c = bench.summarize_clocks([])
    assert c["sm_mhz"] is None and c["samples"] == 0 and c["power_w_max"] is None


def test_profile_with_another_hash_gives_no_traffic(tmp_path, monkeypatch):
    p = tmp_path / "profile.md"
    p.write_text("source_hash: 0123456789abcdef\ntraffic_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "PROFILE", str(p))
    assert bench.profiled_traffic() == (None, "kernel changed since the profile")
    p.write_text("no figures here\n")
    assert bench.profiled_traffic() == (None, "profile without traffic")
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() == (None, "no profile")


def test_peak_falls_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6790.7}')
    assert bench.measured_peaks() == (6790.7, "measured")


def _profile_commands():
    """Every shell command in the fenced blocks of the committed ncu summaries, with backslash
    continuations joined."""
    root = os.path.join(os.path.dirname(bench.__file__), "profiles")
    cmds = []
    for name in sorted(os.listdir(root)):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(root, name)).read()
        for block in text.split("```")[1::2]:
            joined = block.replace("\\\n", " ")
            cmds += [(name, c.strip()) for c in joined.splitlines() if c.strip()]
    return cmds


def test_profile_commands_run_committed_files_with_valid_options():
    import shlex
    cmds = _profile_commands()
    assert cmds
    benched = 0
    for name, c in cmds:
        if c.startswith("ncu "):
            assert "--clock-control none" in c, (name, c)
        if "python bench.py" in c:
            args = bench.make_parser().parse_args(shlex.split(c.split("python bench.py", 1)[1]))
            assert args.warmup >= 3, (name, c)
            benched += 1
        assert "_work/" not in c, (name, c)
    assert benched >= len([n for n in os.listdir(os.path.join(os.path.dirname(bench.__file__), "profiles"))
                           if n.endswith(".md")])
