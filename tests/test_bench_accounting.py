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
    # window + beam, half a row buffer each way, the stored half (rows 0 .. nf/2) of the grid
    per_pair = 2 * 4 * nb * nb + 8 * nb * nf + 8 * (nf // 2 + 1) * nf
    assert sb["fwd_fft"] == sb["adj_fft"] == 7 * per_pair
    assert sb["assemble_R"] == 2 * 4 * 512 * 512 + 7 * 4 * nb * nb


def test_pairs_without_data_move_nothing():
    prob = synth.small_mosaic(3, n=48, nb=32, nchan=1, npoint=3, ndump=2, n_ant=5)
    prob.pairs[1].uvw = prob.pairs[1].uvw[:0]
    sb = bench.stage_bytes(prob, _Plan("fp32", 64))
    assert sb["fwd_fft"] == 2 * (2 * 4 * 32 * 32 + 8 * 32 * 64 + 8 * 33 * 64)


class _FakeNVML:
    """Stand-in for pynvml: two GPUs in the machine; the visible one is found by UUID."""
    NVML_CLOCK_SM = 1

    def __init__(self, clocks, reasons):
        self.clocks, self.reasons, self.lookups, self.i = clocks, reasons, [], 0

    def nvmlInit(self):
        pass

    def nvmlDeviceGetHandleByUUID(self, uuid):
        self.lookups.append(("uuid", uuid))
        if uuid != "GPU-1111":
            raise RuntimeError("unknown uuid")
        return "h1"

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        self.lookups.append(("bus", bus))
        return "h-bus"

    def nvmlDeviceGetMaxClockInfo(self, h, which):
        assert h == "h1"
        return 2032

    def nvmlDeviceGetClockInfo(self, h, which):
        assert h == "h1" and which == self.NVML_CLOCK_SM
        v = self.clocks[min(self.i, len(self.clocks) - 1)]
        return v

    def nvmlDeviceGetPowerUsage(self, h):
        return 900_000

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.reasons[min(self.i, len(self.reasons) - 1)]
        self.i += 1
        return v


def test_clock_sampler_finds_the_visible_gpu_by_uuid_and_samples_it():
    """The sampler names the GPU by its UUID (NVML and nvidia-smi indices ignore
    CUDA_VISIBLE_DEVICES) and collects samples from a thread until stop() joins it."""
    import time
    nv = _FakeNVML([1900, 1950, 2000], [0, 0x4, 0])
    cs = bench.ClockSampler("GPU-1111", "00000000:18:00.0", period=0.001, nvml=nv).start()
    cs.mark("t_begin")
    time.sleep(0.05)
    cs.mark("t_end")
    rec = cs.stop()
    assert nv.lookups[0] == ("uuid", "GPU-1111") and all(h != "bus" for h, _ in nv.lookups)
    assert rec["samples_in_timed_region"] >= 3 and rec["sm_max_mhz"] == 2032.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["power_w_max"] == 900.0
    assert not cs.thread.is_alive()


def test_clock_record_takes_the_median_inside_the_timed_region_and_the_active_reasons():
    """The clocks object of the bench line: median SM clock of the samples taken inside the
    timed region, the maximum clock, and every throttle reason seen active there."""
    cs = bench.ClockSampler("GPU-x")
    cs.rows = [(0.5, 900.0, 2032.0, 500.0, 0),          # before the timed region
               (1.1, 1900.0, 2032.0, 900.0, 0),
               (1.2, 1950.0, 2032.0, 950.0, 0x4),       # sw_power_cap
               (1.3, 2000.0, 2032.0, 901.0, 0),
               (5.0, 700.0, 2032.0, 300.0, 0x8)]        # after it (hw_slowdown)
    cs.t_begin, cs.t_end = 1.0, 1.4
    rec = cs.stop()
    assert rec["sm_mhz"] == 1950.0 and rec["sm_max_mhz"] == 2032.0 and rec["sm_mhz_min"] == 1900.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples_in_timed_region"] == 3


def test_clock_sampler_without_nvml_reports_why():
    class _NoGPU(_FakeNVML):
        def nvmlDeviceGetHandleByUUID(self, uuid):
            raise RuntimeError("no such device")

        def nvmlDeviceGetHandleByPciBusId(self, bus):
            raise RuntimeError("no such device")
    cs = bench.ClockSampler("GPU-2", "0:1:0.0", nvml=_NoGPU([], [])).start()
    rec = cs.stop()
    assert rec["samples"] == 0 and "no NVML handle" in rec["error"]


def test_clock_sampler_falls_back_to_nvidia_smi_with_its_own_timestamps(monkeypatch):
    """Without NVML bindings the sampler runs nvidia-smi on the same GPU (by UUID) and places
    each row by nvidia-smi's timestamp, not by when the line reached the reader."""
    import datetime
    import subprocess

    class _NoNVML(_FakeNVML):
        def nvmlInit(self):
            raise RuntimeError("NVML bindings missing")

    calls = []

    def ts(sec):
        return datetime.datetime.fromtimestamp(sec).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]

    class _Proc:
        def __init__(self, cmd, **kw):
            calls.append(cmd)
            self.stdout = iter([f"{ts(100.2)}, 1000, 2032, 300.0, Not Active, Not Active, Not Active, Not Active\n",
                                f"{ts(101.2)}, 1980, 2032, 800.0, Not Active, Not Active, Not Active, Active\n",
                                f"{ts(101.4)}, 2000, 2032, 820.0, Not Active, Not Active, Not Active, Not Active\n",
                                "garbage line\n"])

        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    monkeypatch.setattr(subprocess, "Popen", _Proc)
    cs = bench.ClockSampler("GPU-abcd", "0:1:0.0", nvml=_NoNVML([], [])).start()
    cs.t_begin, cs.t_end = 101.0, 101.5
    rec = cs.stop()
    assert "--id=GPU-abcd" in calls[0] and rec["source"] == "nvidia-smi"
    assert rec["samples"] == 3 and rec["samples_in_timed_region"] == 2
    assert rec["sm_mhz"] == 1990.0 and rec["reasons"] == ["sw_power_cap"]


def test_per_kernel_stage_bytes_add_up_to_the_packed_fft_totals():
    prob = synth.config_c2()
    nb, nf = 512, 1024
    sb = bench.stage_bytes(prob, _Plan("fp32", nf))
    assert sb["fwd_rows"] == 7 * (2 * 4 * nb * nb + 8 * nb * nf // 2)
    # the column passes store and read only rows 0 .. nf/2 of each fine grid
    assert sb["fwd_cols"] == 7 * (8 * nb * nf // 2 + 8 * (nf // 2 + 1) * nf)
    assert sb["adj_cols"] == 7 * (8 * (nf // 2 + 1) * nf + 8 * nb * nf // 2)
    assert sb["clear_G"] == 7 * 8 * (nf // 2 + 1) * nf
    assert sb["adj_rows"] == 7 * (8 * nb * nf // 2 + 2 * 4 * nb * nb)
    assert sb["fwd_rows"] + sb["fwd_cols"] == sb["fwd_fft"] and sb["adj_cols"] + sb["adj_rows"] == sb["adj_fft"]


def test_roofline_takes_the_longest_single_kernel_stage():
    """The concurrent dish-convolution branch and multi-kernel stages are never chosen."""
    prob = synth.config_c2()
    stages = {"fusion_K": 9.0, "fwd_rows": 0.03, "fwd_cols": 0.04, "degrid_spread": 0.1,
              "adj_cols": 0.2, "adj_rows": 0.02, "assemble_R": 5.0, "finalize": 0.01}
    r = bench.roofline_of(prob, _Plan("fp32", 1024), stages, 6500.0, "measured")
    sb = bench.stage_bytes(prob, _Plan("fp32", 1024))
    assert r["stage"] == "adj_cols" and r["bound"] == "hbm" and r["launch_ms"] == 0.2
    assert abs(r["achieved"] - sb["adj_cols"] / 0.2e-3 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / 6500.0) < 1e-4


def test_roofline_names_the_grid_pass_that_ran():
    """The degrid_spread stage is labelled with the item pass the autotuner kept (its decision
    text), the scalar pass when untuned, and k_grid_pass for FP64; a stored traffic record is
    attached only when its stage, kernel and tile match the launch."""
    prob = synth.config_c2()
    stages = {"fwd_rows": 0.03, "fwd_cols": 0.04, "degrid_spread": 0.3, "adj_cols": 0.03,
              "adj_rows": 0.02, "assemble_R": 0.01, "finalize": 0.01}
    tc = "nf=1024 w=7 fp64=0 nslot=7 m2=21 -> tensor-core item pass, tile 64, items of 64"
    cg = "nf=1024 w=7 fp64=0 nslot=7 m2=21 -> scalar item pass, tile 32, items of 16"
    r_tc = bench.roofline_of(prob, _Plan("fp32", 1024), stages, 6500.0, "measured", tc)
    r_cg = bench.roofline_of(prob, _Plan("fp32", 1024), stages, 6500.0, "measured", cg)
    r_un = bench.roofline_of(prob, _Plan("fp32", 1024), stages, 6500.0, "measured")
    r_64 = bench.roofline_of(prob, _Plan("fp64", 1024), stages, 6500.0, "measured", "tile 32, chunk 1024")
    assert r_tc["kernel"].startswith("k_grid_tc ") and r_cg["kernel"].startswith("k_grid_cg ")
    assert r_un["kernel"].startswith("k_grid_cg ") and r_64["kernel"].startswith("k_grid_pass ")
    rec = {"kernel": "k_grid_cg<7, 32>", "stage": "degrid_spread", "tile": "tile 32"}
    assert bench.traffic_applies(rec, r_cg, cg)
    assert not bench.traffic_applies(rec, r_tc, tc)          # another kernel
    assert not bench.traffic_applies(rec, r_cg, cg.replace("tile 32", "tile 64"))  # another tile
    r_fft = bench.roofline_of(prob, _Plan("fp32", 1024), dict(stages, degrid_spread=0.001), 6500.0, "measured", cg)
    assert not bench.traffic_applies(rec, r_fft, cg)        # another stage


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
