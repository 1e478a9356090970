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
                       "thread_instructions_per_event: 411\narith_ops_per_scattering: 286.4\n"
                       "arith_ops_per_crossing: 181.0\n  indented: not a key\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", srcs)
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.profile_figures() == (6096000.0, 411.0)
    assert bench.traffic_from_profile() == 6096000.0
    v = bench.profile_values()
    assert v["arith_ops_per_scattering"] == 286.4 and v["arith_ops_per_crossing"] == 181.0
    assert "thread_instructions_per_scattering" not in v
    (tmp_path / "k1.cuh").write_bytes(b"kernel b changed")
    assert bench.profile_figures() == (None, None)
    assert bench.profile_values() == {}


def test_ray_cell_count_equals_the_oracle_walk():
    """The closed-form count of the cells each orthographic ray crosses (the
    ray trace's channel-segment throughput) equals the number of
    positive-length segments of the oracle's cell walk, ray by ray summed,
    for oblique and axis-aligned cameras."""
    import math
    import numpy as np
    import oracle
    from oracle import raytrace as RT
    shape = (5, 6, 7)
    npx, npy, fov = 9, 8, 8.0
    for th, ph in [(0.3, 0.7), (1.1, 2.0), (0.0, 0.0), (math.pi / 2, 0.0), (2.5, -1.0)]:
        n, u, v = RT.camera_basis(th, ph)
        C = np.array([shape[2], shape[1], shape[0]]) / 2.0
        pix = fov / npx
        tot = 0
        for iy in range(npy):
            for ix in range(npx):
                P = C + ((ix + 0.5) * pix - 0.5 * fov) * u + ((iy + 0.5) * pix - 0.5 * pix * npy) * v
                _, lens = RT.ray_segments(oracle, shape, (False,) * 3, P, n)
                tot += int((lens > 0).sum())
        assert bench.ray_cells(shape, th, ph, npx, npy, fov) == tot
