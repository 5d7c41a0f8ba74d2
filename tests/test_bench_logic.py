"""Host arithmetic of the benchmark line (no GPU): the roofline of the dominant kernel (bound
chosen by the ridge point of its arithmetic intensity, achieved work over its event time, the
fraction of the peak) and the clock record taken from nvidia-smi samples."""
import os
import tempfile

import bench


def _prof(ms, launches, work, flops):
    z = {"ms": 0.0, "launches": 0, "work": 0.0}
    return {"pcg_solve": {"ms": ms, "launches": launches, "work": work},
            "pcg_flops": {"ms": 0.0, "launches": 0, "work": flops}, "spmv": dict(z)}


def test_roofline_picks_the_bound_by_the_ridge_point():
    hbm, _ = bench.peaks()
    ridge = bench.FP64_PEAK_TFLOPS * 1e12 / (hbm * 1e9)  # flop per byte
    # 2 GB and 0.3 flop/B above the ridge in 10 launches over 5 ms: FP64-arithmetic bound
    work, flops = 2e9, 2e9 * (ridge * 1.5)
    r = bench.roofline(_prof(5.0, 10, work, flops), "fp64")
    assert r["bound"] == "alu"
    assert abs(r["achieved"] - flops / 5e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - flops / 5e-3 / 1e12 / bench.FP64_PEAK_TFLOPS) < 1e-3
    assert r["bytes_per_launch"] == work / 10 and abs(r["avg_launch_us"] - 500.0) < 1e-9
    # below the ridge, or in mixed precision (FP32 arithmetic is far from its roof): HBM bound
    for prec, fl in (("fp64", 2e9 * ridge * 0.5), ("mixed", flops)):
        r = bench.roofline(_prof(5.0, 10, work, fl), prec)
        assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
        assert abs(r["achieved"] - work / 5e-3 / 1e9) < 0.1
        assert abs(r["frac"] - work / 5e-3 / 1e9 / hbm) < 1e-4
    assert bench.roofline(_prof(0.0, 0, 0.0, 0.0), "fp64") is None


def test_kernel_fractions_divide_each_family_s_bytes_by_its_event_time():
    hbm, _ = bench.peaks()
    z = {"ms": 0.0, "launches": 0, "work": 0.0}
    prof = {k: dict(z) for k in ("spmv", "pcg_vector", "ls_energy", "pcg_flops", "host_idle")}
    prof["pcg_solve"] = {"ms": 100.0, "launches": 4, "work": 3e11}
    prof["elastic"] = {"ms": 20.0, "launches": 2, "work": 1e6}  # tets
    prof["contact"] = {"ms": 5.0, "launches": 2, "work": 2e9}
    prof["assembly"] = dict(z)  # no launch in the window: left out
    prof["ccd"] = {"ms": 1.0, "launches": 5, "work": 1e8}
    prof["broad"] = {"ms": 0.0, "launches": 0, "work": 0.0}
    for prec, per_tet in (("fp64", 940), ("mixed", 628)):
        t = bench.kernel_fractions(prof, prec)
        assert set(t) == {"pcg_solve", "elastic", "contact", "ccd", "peak"}
        assert abs(t["pcg_solve"]["gb_s"] - 3e11 / 0.1 / 1e9) < 0.1
        assert t["elastic"]["bytes"] == 1e6 * per_tet
        assert abs(t["elastic"]["gb_s"] - 1e6 * per_tet / 0.02 / 1e9) < 0.1
        assert abs(t["contact"]["hbm_frac"] - 2e9 / 5e-3 / 1e9 / hbm) < 1e-4
        assert t["ccd"]["launches"] == 5 and t["peak"]["hbm_gbs"] == hbm


def test_clock_record_reports_median_clock_and_active_reasons():
    fd, path = tempfile.mkstemp(suffix=".csv")
    rows = ["0, 1900, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2032, 2032, 1050.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1965, 2032, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s.path = Done(), path
    rec = s.stop()
    assert rec["sm_mhz"] == 1965.0 and rec["sm_max_mhz"] == 2032.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(path)


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun the oracle arm runs and prints on rank 0 alone; any other rank exits 0
    without work and without output."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, cwd=root,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_secondary_legs_past_the_leg_budget_are_skipped_and_errors_are_recorded():
    import time

    calls = []

    def leg(x):
        calls.append(x)
        return {"value": x}

    def broken():
        raise RuntimeError("leg failed")

    now = time.perf_counter()
    assert bench.budgeted(now, 60.0, leg, 3) == {"value": 3}
    skipped = bench.budgeted(now - 100.0, 60.0, leg, 4)
    assert "value" not in skipped and skipped["skipped"].startswith("not started")
    assert calls == [3]
    assert bench.budgeted(now, 60.0, broken) == {"error": "RuntimeError: leg failed"}


def test_cpu_leg_times_the_oracle_on_the_batch_s_small_envs():
    """The CPU baseline leg, on the first 24 envs of the uneven batch from their start state: one
    oracle step per env on a sample of the envs of at most CPU_SAMPLE_MAX_TETS tets, one env per
    host thread, with the host's core count and CPU model in the record."""
    from paper_2503_05020_b300 import scenes as S

    wl = bench.Workload("uneven")
    envs = [wl.build(i) for i in range(24)]
    snap = []
    for e in envs:
        x, v = wl.state_at(e, wl.start)
        snap.append((x, v, wl.start))
    tets = [sum(len(s["tets"]) for s in e["soft"]) for e in envs]
    live = [i for i in range(len(envs)) if i != 1]  # an env stopped in the warm-up is left out
    out = bench.cpu_leg(envs, snap, tets, live, S.scene_params(bench.DT))
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT and out["value"] > 0
    assert 1 <= out["cores"] <= (os.cpu_count() or 1)
    assert out["nproc"] == os.cpu_count() and out["cpu_model"]
    lo, hi = (int(t) for t in out["sample"].split("(tets ")[1].split(";")[0].split("-"))
    assert hi <= bench.CPU_SAMPLE_MAX_TETS and lo >= min(tets[i] for i in live)
