"""The benchmark's algorithmic-byte accounting (the numerators of its roofline fractions) on the
CPU: the formulas of the per-stage minimal traffic, and the C2 figures they give."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import synth  # noqa: E402


class _Plan:
    def __init__(self, precision, nf):
        self.precision, self.nf = precision, nf

    def nufft_params(self):
        return (7, 16.1, self.nf)


def test_grid_pass_bytes_are_the_visibility_stream_plus_one_grid_read_and_write():
    prob = synth.config_c2()
    M, npair, nf = prob.total_vis, 7, 1024
    sb = bench.stage_bytes(prob, _Plan("fp32", nf))
    assert M == 1_363_257
    assert sb["degrid_spread"] == 20 * M + 2 * 8 * nf * nf * npair == 144_705_652
    sb64 = bench.stage_bytes(prob, _Plan("fp64", nf))
    assert sb64["degrid_spread"] == 40 * M + 2 * 16 * nf * nf * npair


def test_fft_bytes_count_the_packed_passes_once():
    prob = synth.config_c2()
    nb, nf = 512, 1024
    sb = bench.stage_bytes(prob, _Plan("fp32", nf))
    per_pair = 2 * 4 * nb * nb + 8 * nb * nf + 8 * nf * nf  # window + beam, half a row buffer each way, grid
    assert sb["fwd_fft"] == sb["adj_fft"] == 7 * per_pair
    assert sb["assemble_R"] == 2 * 4 * 512 * 512 + 7 * 4 * nb * nb


def test_pairs_without_data_move_nothing():
    prob = synth.small_mosaic(3, n=48, nb=32, nchan=1, npoint=3, ndump=2, n_ant=5)
    prob.pairs[1].uvw = prob.pairs[1].uvw[:0]
    sb = bench.stage_bytes(prob, _Plan("fp32", 64))
    assert sb["fwd_fft"] == 2 * (2 * 4 * 32 * 32 + 8 * 32 * 64 + 8 * 64 * 64)


def test_clock_record_takes_the_median_inside_the_timed_region_and_the_active_reasons():
    """The clocks object of the bench line: median SM clock of the samples taken inside the
    timed region, the maximum clock, and every throttle reason seen active there."""
    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    row = lambda sm, hw, pc: [str(sm), "2032", "900.0", "0x0", hw, "Not Active", "Not Active", pc]
    cs.rows = [(0.5, row(900, "Not Active", "Not Active")),      # before the timed region
               (1.1, row(1900, "Not Active", "Not Active")),
               (1.2, row(1950, "Not Active", "Active")),
               (1.3, row(2000, "Not Active", "Not Active")),
               (5.0, row(700, "Active", "Not Active"))]          # after it
    cs.t_begin, cs.t_end = 1.0, 1.4
    rec = cs.stop()
    assert rec["sm_mhz"] == 1950.0 and rec["sm_max_mhz"] == 2032.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples_in_timed_region"] == 3


def test_reference_arm_line_has_the_contract_keys(monkeypatch):
    """bench.py --impl reference: one JSON object with the contract's keys, its cpu_baseline
    and an e2e object that moves no bytes (the oracle runs on the host). The oracle's timing is
    replaced by a constant here; the arm's own arithmetic on it is what is checked."""
    import argparse
    monkeypatch.setattr(bench, "oracle_rate", lambda prob, nvis=None, seed=0: (1000.0, nvis or 64, (nvis or 64) / 1000.0))
    args = argparse.Namespace(config="c2", steps=4, warmup=3)
    out = bench.run_reference(args, 0, 1)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] == 1000.0 and out["higher_is_better"] is True
    assert out["steps"] == 4 and out["warmup"] == 3 and out["n_gpus"] == 1
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert bench.run_reference(args, 1, 2) is None  # other ranks do no work
