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


def _ncu_rows(kernels):
    """An ncu --csv launch list: per launch, duration and DRAM bytes."""
    hdr = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",' \
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    out = ["==PROF== Connected to process 1\n", hdr]
    for i, (k, us, rd, wr) in enumerate(kernels):
        for name, unit, v in (("dram__bytes_read.sum", "Mbyte", rd), ("dram__bytes_write.sum", "Mbyte", wr),
                              ("gpu__time_duration.sum", "usecond", us)):
            out.append(f'"{i}","1","python","h","{k}","1","7","(256, 1, 1)","(1, 1, 1)","0","10.3",'
                       f'"Command line profiler metrics","{name}","{unit}","{v}"\n')
    return "".join(out)


def test_ncu_traffic_writer_takes_the_last_complete_image(tmp_path, monkeypatch):
    image = [("zref_kernel(ZrefArgs)", 10, 0.1, 0.1), ("geometry_kernel(GeomArgs)", 30, 0.2, 0.2),
             ("bin_scatter_kernel(ScatterArgs)", 5, 0.1, 0.1), ("void compensate_kernel<0, 1>(A)", 90, 300, 225),
             ("void spread_kernel<2, 4, 8, 4>(SpreadArgs)", 290, 310, 134),
             ("void column_fft_reg_kernel<512, -1, 1>(ColumnFFT)", 80, 130, 110),
             ("void column_fft_reg_kernel<512, -1, 1>(ColumnFFT)", 67, 110, 115),
             ("void stolt_kernel<128, 8, 17, 2>(StoltArgs)", 92, 100, 28),
             ("void column_fft_reg_kernel<256, 1, 1>(ColumnFFT)", 17, 17, 17),
             ("void column_fft_reg_kernel<256, 1, 1>(ColumnFFT)", 16, 16, 17.5)]
    second = [(k, us, rd * 2, wr) for (k, us, rd, wr) in image]
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text(_ncu_rows(image + second + image[:4]))   # the last image is incomplete
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    for p in set(sum(bench.STAGE_SOURCES.values(), [])) | set(bench.COMMON_SOURCES):
        (tmp_path / p).parent.mkdir(parents=True, exist_ok=True)
        (tmp_path / p).write_text("// " + p)
    d = bench.write_ncu_traffic(str(csv_path), "ncu ... python bench.py")
    assert set(d["stages"]) == set(bench.STAGE_SOURCES)
    assert d["stages"]["grid"]["dram_bytes_per_launch"] == (620 + 134) * 1e6     # from the second image
    assert d["stages"]["ifft_x"]["dram_bytes_per_launch"] == (32 + 17.5) * 1e6
    assert d["stages"]["fft_y"]["us"] == 67
    assert bench.ncu_traffic("grid", "realistic") == (620 + 134) * 1e6


def test_plan_geometry_matches_the_library_plan():
    """The reference arm reports the plan's kernel width and spectral grid
    without loading the library; the rule it restates agrees with the plan."""
    import synth
    from paper_2305_02064_gb300 import Plan
    for kw in ({"nx": 24, "ny": 12, "nz": 10}, {"nx": 64, "ny": 100, "nz": 8}, {"nx": 8, "ny": 8, "nz": 4}):
        scan = synth.custom(nx_pos=4, ny_pos=4, nk=8, **kw)
        for tol in (1e-3, 1e-4, 1e-6):
            g = bench.plan_geometry(scan, tol)
            plan = Plan.for_scan(scan, nufft_tol=tol)
            assert g["kernel_width"] == plan.kernel_width
            assert g["spectral_grid"] == [plan.mx, plan.my]


def test_host_cpu_reports_a_model():
    model, cores = bench.host_cpu()
    assert isinstance(model, str) and model
    assert cores >= 1


def test_reference_arm_samples_track_the_whole_scan():
    """With a step budget below one whole image, the reference arm times a
    smaller sample (fewer frequencies, then fewer positions) and scales it by
    the measured whole / sample ratio: its value stays close to the
    whole-image rate, and the line says what the sample was."""
    import argparse
    args = argparse.Namespace(workload="tiny", compensate=1, steps=6, warmup=1, ref_budget=0.001)
    out = bench.run_reference(args, bench.Dist(want_cuda=False))
    assert out["impl"] == "reference" and out["steps"] == 6
    whole = out["whole_scan_seconds"]
    assert "ratio" in out["cpu_baseline"]["sample"]
    est = out["ms_per_step"] * 1e-3
    assert 0.5 * whole < est < 2.0 * whole, (est, whole)
    assert out["cpu_baseline"]["value"] == out["value"] == out["e2e"]["value"]
