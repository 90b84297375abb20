"""Host-side logic of bench.py and of the oracle's marshalling, on the CPU: the
packed host batches of the end-to-end loop, the DRAM-traffic record's source
check, and the oracle's refusal of arrays of the wrong size."""

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


def test_packed_batches_round_trip(bench, monkeypatch):
    import torch

    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)  # no CUDA here
    rng = np.random.default_rng(0)
    batches = [dict(o=rng.random((7, 3), np.float32), d=rng.random((7, 3), np.float32),
                    is_obj=rng.integers(0, 2, 7).astype(np.uint8), uniforms=rng.random((7, 5), np.float32))
               for _ in range(3)]
    blocks, layout = bench._pack_batches(batches)
    assert len(blocks) == 3 and all(b.numel() == blocks[0].numel() for b in blocks)
    assert all(off % 256 == 0 for _, off, _, _ in layout)  # every array starts on a 256-byte boundary
    for blk, b in zip(blocks, batches):
        got = bench._unpack(blk, layout)
        assert set(got) == set(b)
        for k in b:
            assert got[k].dtype == {np.float32: torch.float32, np.uint8: torch.uint8}[b[k].dtype.type]
            np.testing.assert_array_equal(got[k].numpy(), b[k])


def test_packed_batches_reject_a_different_shape(bench, monkeypatch):
    import torch

    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    a = dict(o=np.zeros((4, 3), np.float32))
    b = dict(o=np.zeros((5, 3), np.float32))
    with pytest.raises(AssertionError):
        bench._pack_batches([a, b])


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
