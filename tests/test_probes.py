"""The throughput probes that set the solvers' arithmetic ceilings.

dex_measure_ex2_rate times independent 2^x chains on the special-function units
and dex_measure_fp32_rate independent packed-FMA chains on the FP32 pipe.  Each
must return a positive rate no larger than what the device's SM count and clock
allow for its unit (2^x: at most 32 per SM per clock; FP32: at most 256 lane
operations per SM per clock, twice the 128 FP32 lanes, a generous upper bound),
and at least a tenth of a plausible floor, so that a probe that skipped its work
or timed the wrong thing fails.
"""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sm_clock_hz(dev):
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    try:
        import subprocess
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                              str(dev)], capture_output=True, text=True, timeout=30).stdout.strip()
        mhz = float(out.splitlines()[0])
    except Exception:
        mhz = 2100.0
    return sms, mhz * 1e6


def test_probe_rates_within_unit_limits():
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    sms, hz = _sm_clock_hz(0)
    ex2 = api.measure_ex2_rate(ctx)
    fp32 = api.measure_fp32_rate(ctx)
    ctx.check()
    assert 0.1 * 4 * sms * hz < ex2 <= 32 * sms * hz * 1.05
    assert 0.1 * 64 * sms * hz < fp32 <= 256 * sms * hz * 1.05
