"""The issue-rate probe behind the bench's ALU roofline (needs a GB300): the
four pipes' rates come out positive and in the order the hardware fixes
(FP32 FMA at one warp-instruction per clock per scheduler, integer
multiply-add and the special-function unit slower, FP64 far slower), and the
FP32 rate sits below the nominal 4 warp-instructions per clock per SM at the
maximum SM clock."""
import pytest

pytestmark = pytest.mark.gpu


def test_issue_rates_are_ordered_and_bounded():
    import torch
    import paper_2001_11252_gb300 as rg
    ctx = rg.Context(0)
    r = ctx.probe_issue_rates()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 4 * 2.2e9        # above the 2070 MHz maximum SM clock
    print({k: "%.3g" % v for k, v in r.items()})
    assert 0 < r["dfma"] < r["mufu"] < r["imad"] < r["ffma"] < nominal
    assert r["ffma"] > 0.5 * sms * 4 * 1.0e9     # at least half the issue rate at 1 GHz
    assert r["ffma"] / r["dfma"] > 16             # FP64 is a small fraction of FP32 on this part
    ctx.close()
