"""Host logic of bench.py that needs no GPU: the DRAM-traffic record is used
only while the kernel's sources are the ones it was captured on, and each
stage's algorithmic byte count covers what that stage must read and write."""
import json
import os

import bench


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "k.cu"
    src.write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    rec = {"workload": "realistic",
           "stages": {"grid": {"sources": ["k.cu"], "sha": bench.csrc_digest(["k.cu"]),
                               "dram_bytes_per_launch": 123.0}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("grid", "realistic") == 123.0
    assert bench.ncu_traffic("grid", "large") is None          # another workload
    assert bench.ncu_traffic("stolt", "realistic") is None     # no entry
    src.write_text("// kernel source, edited\n")
    assert bench.ncu_traffic("grid", "realistic") is None      # captured on other sources


def test_traffic_record_absent_or_unreadable(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("grid", "realistic") is None
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text("{not json")
    assert bench.ncu_traffic("grid", "realistic") is None


def test_committed_traffic_record_is_well_formed():
    """Every stage entry names its sources (files that exist), a digest and
    a positive byte count."""
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    assert d["workload"] == "realistic" and "command" in d
    for stage, e in d["stages"].items():
        assert e["dram_bytes_per_launch"] > 0, stage
        assert len(e["sha"]) == 16
        for p in e["sources"]:
            assert os.path.isfile(os.path.join(bench.ROOT, p)), p


def test_stage_bytes_add_up():
    """The per-stage algorithmic bytes of the realistic plan: the gridding
    reads s_hat and the records and writes the occupied window; the window
    lies inside the gridding grid; every stage moves at least its output."""
    import synth
    from paper_2305_02064_gb300 import Plan
    scan = synth.custom(nx_pos=12, ny_pos=10, nk=40, layout="awr1443", nx=32, ny=24, nz=8, seed=3)
    plan = Plan.for_scan(scan)
    nb = bench.stage_bytes(plan, scan)
    T, R, P, Nk = scan.echo.shape
    L, nkp = T * R * P, ((Nk + 31) // 32) * 32
    ul, vl = bench.occupied_window(plan, scan)
    assert 0 < ul <= 2 * plan.mx and 0 < vl <= 2 * plan.my
    assert nb["grid"] > L * nkp * 8 + ul * vl * nkp * 8
    assert nb["compensate"] > L * Nk * 8 + L * nkp * 8
    V = scan.grid.nx * scan.grid.ny * scan.grid.nz * 8
    assert nb["ifft_x"] >= V and nb["stolt"] >= plan.mx * plan.my * scan.grid.nz * 8
    assert set(nb) >= {"prep", "compensate", "grid", "fft_x", "fft_y", "stolt", "ifft_y", "ifft_x"}
