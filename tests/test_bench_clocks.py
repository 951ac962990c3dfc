"""The bench's clock record on CPU: the rows nvidia-smi prints during the
timed region (csv, no header, no units) are reduced to this GPU's median SM
clock, its maximum clock and the throttle reasons seen Active."""
import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _Thread:
    def join(self, timeout=None):
        pass


def _row(idx, bus, sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"{idx}, {bus}, {sm}, {mx}, 650.00, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def _stop(lines, bus_id):
    s = bench.ClockSampler(bus_id)
    s.proc, s.t, s.lines = _Proc(), _Thread(), list(lines)
    return s.stop()


def test_this_gpus_rows_give_median_clock_and_reasons():
    mine, other = "00000009:01:00.0", "00000018:01:00.0"
    lines = [_row(0, mine, 2070, 2070), _row(1, other, 1200, 2070, hw="Active"),
             _row(0, mine, 2055, 2070, cap="Active"), _row(1, other, 1200, 2070),
             _row(0, mine, 2070, 2070), _row(0, mine, "[N/A]", 2070)]
    # torch reports the bus id with a 4-digit domain
    clk = _stop(lines, "0009:01:00.0")
    assert clk["samples"] == 4
    assert clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]           # the other GPU's hw_slowdown is not ours


def test_every_throttle_reason_is_reported():
    bus = "00000009:01:00.0"
    lines = [_row(0, bus, 1800, 2070, hw="Active"), _row(0, bus, 1700, 2070, hwt="Active"),
             _row(0, bus, 1750, 2070, swt="Active")]
    clk = _stop(lines, bus)
    assert clk["sm_mhz"] == 1750.0
    assert clk["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_no_sampler_or_no_rows_gives_no_record():
    s = bench.ClockSampler(None)
    assert s.stop() is None                              # nvidia-smi never started
    assert _stop(["garbage", ""], None) is None
