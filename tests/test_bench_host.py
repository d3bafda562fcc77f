"""Host arithmetic of bench.py's side rooflines (no GPU): shared-memory
wavefronts against the measured or nominal issue rate, DRAM bytes against the
measured or fallback copy bandwidth."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_smem_uses_a_plausible_measured_rate(bench):
    wf = bench.ANNEAL_SMEM_WAVEFRONTS["n120_c8_t21"]
    r = bench.side_rooflines("n120_c8_t21", 1000, 2, 0.5, 152, 2.0e9, 1.5)["smem"]
    assert r["achieved"] == pytest.approx(wf * 1000 / 0.5 / 1e9)
    assert r["peak"] == pytest.approx(152 * 1.5 * 2.0e9 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "measured" in r["peak_basis"]


@pytest.mark.parametrize("rate", [5309.0, 0.0, -3.0])
def test_smem_falls_back_to_one_wavefront_per_clock(bench, rate):
    # an SM issues at most 4 shared loads per clock: a larger (or failed)
    # reading is not used as a peak
    r = bench.side_rooflines("n2000_c16_t33", 10, 1, 1.0, 152, 2.0e9, rate)["smem"]
    assert r["peak"] == pytest.approx(152 * 2.0e9 / 1e9)
    assert "nominal" in r["peak_basis"]


def test_hbm_per_launch_traffic(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.side_rooflines("n2000_c16_t33", 10, 3, 0.6, 152, 0.0, 1.0)
    assert "smem" not in r                      # no clock sample: no shared-memory figure
    # three launches of the captured per-launch traffic in 0.6 s
    assert r["hbm"]["achieved"] == pytest.approx(bench.ANNEAL_TRAFFIC["n2000_c16_t33"] * 3 / 0.6 / 1e9)
    assert r["hbm"]["peak"] == 6800.0 and "fallback" in r["hbm"]["peak_basis"]
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6767.4}))
    r = bench.side_rooflines("n2000_c16_t33", 10, 3, 0.6, 152, 0.0, 1.0)
    assert r["hbm"]["peak"] == 6767.4 and "measured" in r["hbm"]["peak_basis"]


def test_no_capture_no_side_figures(bench):
    assert bench.side_rooflines("batch256", 10, 1, 1.0, 152, 2.0e9, 1.0) == {}


def test_algorithmic_ops_per_evaluation(bench):
    # C (T-1) (2E + 12N) + 3 n_obs, worked by hand: 8*20*(2*581 + 12*120) + 3*4057
    # and 16*32*(2*12113 + 12*2000) + 3*105073 -- the figures the profiles quote
    from paper_2506_19866_gb300 import synth
    assert bench.algorithmic_ops_per_eval(synth.make("n120_c8_t21")) == 428491
    assert bench.algorithmic_ops_per_eval(synth.make("n2000_c16_t33")) == 25006931


def test_protocol_table_from_a_result_file(bench, tmp_path):
    # the F2 table is generated from the --paper-protocol result files
    curve = [{"levels": 55 * (k + 1), "T": 1.0, "seconds": 0.5 * (k + 1), "best": 9 - k,
              "accept_rate": 0.9 - 0.1 * k} for k in range(5)]
    res = {"paper_protocol": [{"network": "mtb_63n_178e", "params": 723, "threads": 32,
                               "iters_per_level": 5000, "levels": 1375, "seconds": 49.3,
                               "final_best": 5, "seconds_to_final_best": 2.5,
                               "evals_per_s": 4.46e6, "curve": curve}]}
    p = tmp_path / "pp.json"
    p.write_text(json.dumps(res))
    rows = bench.protocol_table(str(p)).splitlines()
    assert len(rows) == 3
    assert rows[2] == "| 723 params | 32 | 5000 | 49.3 | 5 | 2.50 | 4.46e+06 | 0.90 / 0.70 / 0.50 |"


def test_alu_roofline_both_denominators(bench):
    # achieved = algorithmic ops per launch / launch time, against the measured
    # issue rate (the target's basis) and the nominal 128 INT32 lanes, both at
    # the sampled SM clock
    r = bench.alu_roofline(4.0e12, 0.5, 152, 2000.0, {"alu": 88.0, "lds": 1.0})
    assert r["achieved"] == pytest.approx(8.0)
    assert r["peak"] == pytest.approx(152 * 88.0 * 2.0e9 / 1e12)
    assert r["frac"] == pytest.approx(8.0 / (152 * 88.0 * 2.0e-3))
    assert r["peak_nominal"] == pytest.approx(152 * 128 * 2.0e9 / 1e12)
    assert r["frac_nominal"] == pytest.approx(8.0 / (152 * 128 * 2.0e-3))
    assert "measured" in r["target_basis"]
    # no clock sample or no measured rate: no fractions, never a made-up peak
    r = bench.alu_roofline(4.0e12, 0.5, 152, None, {"alu": 88.0})
    assert r["peak"] is None and r["frac"] is None and r["frac_nominal"] is None
    r = bench.alu_roofline(4.0e12, 0.5, 152, 2000.0, {})
    assert r["peak"] is None and r["frac"] is None and r["frac_nominal"] is not None
