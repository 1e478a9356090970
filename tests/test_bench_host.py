"""Host logic of bench.py, without a GPU: the clock record taken during the
timed region (median SM clock, maximum, throttle reasons that were active)
and the profile figures, which are used only when the committed ncu summary
was taken on the current kernel source."""
import hashlib

import bench


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(sm, mx, hw="Not Active", thermal="Not Active", swth="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {thermal}, {swth}, {cap}"


def test_clock_record():
    c = bench.Clocks(0)
    c.proc = _DoneProc()
    c.lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2070, 2070),
               "garbage", _line(1500, 2070), _line(2055, 2070)]
    r = c.stop()
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 5}
    c.lines = [_line(1400, 2070, hw="Active", thermal="Active")]
    assert bench.Clocks.stop(c)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_record_without_samples():
    c = bench.Clocks(0)
    assert c.stop() is None                      # nvidia-smi never started
    c.proc = _DoneProc()
    c.lines = ["[N/A]"]
    assert c.stop() is None


def test_profile_figures_follow_the_kernel_source(tmp_path, monkeypatch):
    srcs = []
    for i, text in enumerate((b"kernel a", b"kernel b")):
        p = tmp_path / f"k{i}.cuh"
        p.write_bytes(text)
        srcs.append(str(p))
    h = hashlib.sha256(b"kernel akernel b").hexdigest()[:16]
    summary = tmp_path / "profile.txt"
    summary.write_text(f"kernel: k\nkernel_source_sha256_16: {h}\ndram_bytes_per_launch_scaled: 6096000\n"
                       "thread_instructions_per_event: 411\n  indented: not a key\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", srcs)
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.profile_figures() == (6096000.0, 411.0)
    assert bench.traffic_from_profile() == 6096000.0
    (tmp_path / "k1.cuh").write_bytes(b"kernel b changed")
    assert bench.profile_figures() == (None, None)
