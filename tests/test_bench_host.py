"""Host-side logic of bench.py and of the oracle's marshalling, on the CPU: the
packed host ray sets of the end-to-end loop, the 32-object workload, the
oracle timing's extrapolation, the DRAM-traffic record's source check, and
the oracle's refusal of arrays of the wrong size."""

import hashlib
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import importlib
    import sys

    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_packed_sets_round_trip(bench, monkeypatch):
    import torch

    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)  # no CUDA here
    rng = np.random.default_rng(0)

    def batch(n):
        return dict(o=rng.random((n, 3), np.float32), d=rng.random((n, 3), np.float32),
                    is_obj=rng.integers(0, 2, n).astype(np.uint8), uniforms=rng.random((n, 5), np.float32))

    sets = [[batch(7), batch(33), batch(1)] for _ in range(3)]  # objects of different ray counts
    packed = [bench._pack(s) for s in sets]
    layout = packed[0][1]
    assert all(p[1] == layout for p in packed)  # sets of the same shapes share one layout
    assert all(p[0].numel() == packed[0][0].numel() for p in packed)
    assert all(off % 256 == 0 for ent in layout for _, off, _, _ in ent)  # 256-byte aligned arrays
    for (blk, _), s in zip(packed, sets):
        for ent, b in zip(layout, s):
            got = bench._unpack(blk, ent)
            assert set(got) == set(b)
            for k in b:
                assert got[k].dtype == {np.float32: torch.float32, np.uint8: torch.uint8}[b[k].dtype.type]
                np.testing.assert_array_equal(got[k].numpy(), b[k])


def test_batched_workload_specs(bench):
    """The 32 objects: the category table in order, rays 32 round(8 2^(5a)) in 256..8192."""
    specs = bench.batched_specs()
    assert len(specs) == 32
    for i, sp in enumerate(specs):
        assert (sp["log2T"], sp["W"], sp["H"]) == bench.CATEGORY_ARCHS[i % 9]
        assert sp["rays"] % 32 == 0 and 256 <= sp["rays"] <= 8192
    samples, rays = bench.batched_totals(specs)
    assert samples == 48 * rays


def test_oracle_step_extrapolation(bench):
    specs = bench.batched_specs()
    per = {i: (16, 0.5) for i in range(32)}  # every object: 16 rays in 0.5 s
    rays = sum(sp["rays"] for sp in specs)
    assert abs(bench.oracle_step_seconds(per, 1, 2.0) - (rays * 0.5 / 16 + 2.0)) < 1e-9
    assert abs(bench.oracle_step_seconds(per, 4, 2.0) - (rays * 0.5 / 16 / 4 + 2.0)) < 1e-9


def test_traffic_record_follows_its_sources(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    digest = hashlib.sha256(b"kernel v1").hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(
        {"k/fp16": {"dram_bytes_per_launch": 123.0, "sources": ["k.cu"], "sources_sha256": digest}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k/fp16") == 123.0
    assert bench.profiled_traffic("other/fp16") is None
    src.write_text("kernel v2")  # the kernel changed after the capture: no traffic figure
    assert bench.profiled_traffic("k/fp16") is None


def test_oracle_refuses_arrays_of_the_wrong_size(orc):
    from helpers import CFG1, case

    a, theta, grid, rays, u, cr = case(CFG1, 4, 8, 8, seed=3)
    orc.batch(a, theta, grid, rays, 8, 8, u=u, c_rand=cr)  # the right sizes pass
    with pytest.raises(ValueError):
        orc.batch(a, theta, grid, rays, 8, 16, u=u, c_rand=cr)  # u holds 8 per ray, 16 read
    with pytest.raises(ValueError):
        orc.batch(a, theta, grid, rays, 8, 8, u=u, c_rand=cr[:2])
    with pytest.raises(ValueError):
        orc.batch(a, theta[:-1], grid, rays, 8, 8, u=u, c_rand=cr)
    with pytest.raises(ValueError):
        orc.sample_ray(grid, rays["o"][0], rays["d"][0], 8, 16, 1e-4, u[0])


def test_clock_record_window_and_reasons(bench):
    """The clock record keeps the samples inside the timed region, takes their
    median SM clock and names every reason seen; with none inside it falls back
    to the nearest sample."""
    lines = [f"2026/12/04 10:00:00.{ms:03d}, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
             for ms, mhz, cap in [(100, 1900, "Not Active"), (200, 2070, "Active"), (300, 2070, "Not Active"),
                                  (400, 1500, "Not Active")]]
    c = bench.ClockSampler("GPU-test")
    c.rows = c.parse_smi(lines)
    assert [r[3] for r in c.rows] == [[], ["sw_power_cap"], [], []]
    t = [r[0] for r in c.rows]
    c.mark(t[0] + 0.05, t[2] + 0.01)  # the samples at .200 and .300
    rec = c.summary()
    assert rec["samples"] == 2 and rec["sm_mhz"] == 2070.0 and rec["reasons"] == ["sw_power_cap"]
    c.mark(t[3] + 0.01, t[3] + 0.02)  # after the last sample: the nearest one
    rec = c.summary()
    assert rec["samples"] == 1 and rec["sm_mhz"] == 1500.0 and "nearest" in rec["note"]
    assert set(bench.NVML_REASONS.values()) == {"sw_power_cap", "hw_slowdown", "sw_thermal_slowdown",
                                                "hw_thermal_slowdown"}
