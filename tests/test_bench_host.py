"""Host logic of bench.py that needs no GPU: the digest-keyed ncu traffic record that fills
`roofline.traffic`, and the arena layout of DeviceBatch (markers and masks of a batch packed
at 256-byte aligned offsets, restored and read back as one copy each)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_traffic_record_matches_kernel_name_workload_and_digest(tmp_path, monkeypatch):
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment line naming drain_coop_kernel<u8|u16,8> batch512 feedface 1\n"
        "drain_coop_kernel<u8|u16,8> batch512 0123456789abcdef 29166400000\n"
        "drain_coop_kernel<u8,8> tissue4096 0123456789abcdef 35000000\n"
        "drain_coop_kernel<u8|u16,8> batch512 fedcba9876543210 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda: "0123456789abcdef")
    # the name as bench.py builds it (with a space) matches the record written without spaces
    assert bench._traffic_from_profiles("drain_coop_kernel<u8|u16, 8>", "batch512") == 29166400000.0
    assert bench._traffic_from_profiles("drain_coop_kernel<u8, 8>", "tissue4096") == 35000000.0
    assert bench._traffic_from_profiles("drain_coop_kernel<u8, 8>", "batch512") is None      # other workload
    monkeypatch.setattr(bench, "kernel_digest", lambda: "ffffffffffffffff")
    assert bench._traffic_from_profiles("drain_coop_kernel<u8|u16, 8>", "batch512") is None  # stale sources


def test_traffic_record_absent(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profiles("drain_coop_kernel<u8, 8>", "tissue4096") is None


def test_kernel_digest_covers_every_listed_source():
    import os
    import bench
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, f)), f
    d = bench.kernel_digest()
    assert len(d) == 16 and int(d, 16) >= 0


def test_device_batch_arena_layout_on_cpu():
    import bench
    from paper_1605_00930_gb300 import synth
    rng = np.random.default_rng(7)
    cases = []
    for (H, W, dt) in [(3, 5, np.uint8), (17, 33, np.uint16), (1, 1, np.uint8), (64, 65, np.uint16)]:
        mask = rng.integers(0, 200, (H, W)).astype(dt)
        marker = (mask // 2).astype(dt)
        cases.append(synth.Case(marker, mask, 8, "dilate"))
    db = bench.DeviceBatch(cases, "cpu")
    assert all(o % 256 == 0 for o in db.offs)
    assert db.pixels == sum(c.mask.size for c in cases)
    assert db.alg_bytes == 3 * sum(c.mask.nbytes for c in cases)
    assert db.nbytes >= db.offs[-1] + cases[-1].mask.nbytes
    for (m, I, conn, op), c in zip(db.items, cases):
        assert m.dtype == (torch.uint16 if c.mask.dtype == np.uint16 else torch.uint8)
        assert tuple(m.shape) == c.mask.shape and conn == 8 and op == "dilate"
        np.testing.assert_array_equal(m.numpy(), c.marker)
        np.testing.assert_array_equal(I.numpy(), c.mask)
    # a run writes through the views into the marker arena; restore() brings the markers back
    for m, _, _, _ in db.items:
        m.fill_(9)
    assert all(np.all(o == 9) for o in db.outputs())
    db.restore()
    for o, c in zip(db.outputs(), cases):
        np.testing.assert_array_equal(o, c.marker)


def test_reference_arm_prints_one_json_line(monkeypatch, capsys):
    """`bench.py --impl reference` (the oracle arm, CPU only) on the 512^2 workload: one JSON
    line with the contract's keys, the oracle as its CPU baseline and zero copy bytes."""
    import json
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "noiseblur512",
                                      "--steps", "2", "--warmup", "1"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 2
    assert d["warmup"] == 3   # raised to the minimum of three
    assert d["value"] > 0 and d["config"]["name"] == "noiseblur512" and d["config"]["pixels_per_step"] == 512 * 512
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == bench.host_cores()
    assert "whole workload" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_samples_when_over_budget(monkeypatch):
    """Over its time budget the reference arm times a bounded sample: for a single image the
    first rows of it, stated in the line."""
    import bench
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 1e-4)

    class A:
        workload, steps, warmup = "noiseblur512", 2, 3
    d = bench.run_reference(A, 0, 1)
    assert d["config"]["pixels_per_step"] == 16 * 512   # at least 16 rows of the 512 x 512 image
    assert "first 16 rows" in d["cpu_baseline"]["sample"]
