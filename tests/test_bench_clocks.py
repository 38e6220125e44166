"""bench.py's clock record: the nvidia-smi samples taken during the timed region are reduced to
the median SM clock under load, the maximum clock and the throttle reasons seen (no GPU)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self):
        return 0


def test_clock_record_from_samples(tmp_path):
    b = _bench()
    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 345, 2032, 180.1, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2032, 2032, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2032, 1099.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2010, 2032, 1050.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbled line\n")
    cs = b.ClockSampler(0)
    cs.proc, cs.path = _Done(), str(path)
    rec = cs.stop()
    # the idle sample (345 MHz) is below half the maximum and left out of the median
    assert rec == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 4}
    assert not path.exists()


def test_clock_record_without_nvidia_smi():
    b = _bench()
    cs = b.ClockSampler(0)
    rec = cs.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
