"""Host logic of bench.py on the CPU: the clock record taken during the
timed region (median SM clock and the throttle reasons that reject a run)
and the measured-peak lookup."""
import json
import os

import numpy as np
import pytest

import bench


def row(sm, mx=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 900.5, 0x0000000000000000, %s, %s, %s, %s\n" % (sm, mx, hw, hwt, swt, cap)


def test_clean_run():
    c = bench.ClockSampler.summarize([row(2070), row(2055), row(2070)])
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_reasons_are_collected():
    c = bench.ClockSampler.summarize([row(1800, cap="Active"), row(1500, hwt="Active"),
                                      row(1600, swt="Active"), row(1700, hw="Active")])
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                            "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1650.0


def test_unreadable_rows_are_skipped():
    lines = ["garbage\n", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             row(1990)]
    c = bench.ClockSampler.summarize(lines)
    assert c["samples"] == 1 and c["sm_mhz"] == 1990.0
    assert bench.ClockSampler.summarize(["\n"]) is None


def test_peaks_reads_measured_file():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    v, kind = bench.peaks()
    if os.path.exists(path):
        with open(path) as f:
            assert v == pytest.approx(float(json.load(f)["hbm_gbs"]))
        assert kind == "measured"
    else:
        assert (v, kind) == (6800.0, "fallback")


def test_stop_reads_and_removes_the_record(tmp_path):
    """stop() ends the sampling process, summarises its file and deletes it
    (a stand-in process and file; no nvidia-smi needed)."""
    import subprocess
    import sys
    path = tmp_path / "clocks.csv"
    path.write_text(row(2070) + row(2040, cap="Active"))
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    cs.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(30)"])
    c = cs.stop()
    assert cs.proc.poll() is not None
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert not path.exists()
    assert bench.ClockSampler(0).stop() is None          # never started


def test_l2_and_footprint_fields():
    """The roofline record sets the system's device footprint against the L2
    size: the d=6, N=32768 benchmark system fits in GB300's 129 MB L2 (the
    fused step runs out of L2), the N=2^21 one does not."""
    from paper_2112_12271_gb300 import workloads as W
    l2 = bench.l2_bytes()
    assert l2 is None or l2 > 0
    small = bench.footprint_bytes(W.c1_poly_d6(0))
    large = bench.footprint_bytes(W.c1_poly_d6(0, N=2 ** 21))
    assert small < 129e6 < large


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle, timed on the host) prints
    exactly one JSON line with the keys of the benchmark contract."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == bench.WORKLOAD


def test_algorithmic_bytes_follow_the_stated_formula():
    """Bytes per atom-step of the fused force + VV kernel: 4 Z (list) + 4
    (length) + 4 (diameter) + 16 d (x r/w) + 16 d (v r/w) + 2 b_F d (F w/r):
    at d = 6, Z = 17.5 that is 318 B in mixed precision (b_F = 4) and 366 B
    in FP64 (b_F = 8)."""
    assert bench.alg_bytes_per_atom_step(6, 17.5, 4) == pytest.approx(318.0)
    assert bench.alg_bytes_per_atom_step(6, 17.5, 8) == pytest.approx(366.0)
    # the design's own count is larger: 8-byte entries and three FP32 rows
    assert bench.design_bytes_per_atom_step(6, 17.5) > bench.alg_bytes_per_atom_step(6, 17.5, 4)


def test_threaded_oracle_gives_the_serial_trajectory():
    """The OpenMP build of the oracle (timing only) parallelises per-atom and
    per-subcell loops: the positions and velocities it returns equal the
    serial build's bit for bit (only the E and W sums may round differently)."""
    import oracle
    from paper_2112_12271_gb300 import workloads as W
    s = W.make_system(4, 700, phi=0.4, dist="poly", T=0.05, seed=3)
    a = oracle.md_steps(s.x, s.v, s.sigma, s.L, 60, 0.005)
    oracle.set_threads(4)
    b = oracle.md_steps(s.x, s.v, s.sigma, s.L, 60, 0.005, openmp=True)
    assert a["builds"] == b["builds"] >= 2
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
    assert b["E"] == pytest.approx(a["E"], rel=1e-12)


def test_list_build_kernel_count():
    """The launch count of one list build: seven kernels where the half-stencil
    build adds its list sort (d = 6 at N = 32768, n_cell 4; the paper's model at
    d = 5), six elsewhere (the paper's model at d = 3 and 4; n_cell <= 2)."""
    assert bench.list_build_kernels(6, 32768, 4, 4 ** 6) == 7
    assert bench.list_build_kernels(5, 100000, 6, 6 ** 5) == 7
    assert bench.list_build_kernels(4, 100000, 11, 11 ** 4) == 6
    assert bench.list_build_kernels(3, 100000, 30, 30 ** 3) == 6
    assert bench.list_build_kernels(6, 300, 2, 2 ** 6) == 6
