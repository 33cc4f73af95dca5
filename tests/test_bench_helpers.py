"""Host-side arithmetic of bench.py (no GPU).

The U-Net FLOP count behind the `network` roofline object is checked
against the convolutions the numpy U-Net oracle actually performs on a
small input: each call's input and output tensor shapes give its pixels and
channels, with the real channel counts at the ends (4 input features padded
to 16, one output channel of the 16-channel head)."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import unet_oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("widths,H,W", [((16, 32, 32, 48), 16, 32), ((32, 64, 128, 128), 24, 40)])
def test_unet_flops_match_the_convolutions_the_oracle_runs(widths, H, W, monkeypatch):
    bench = load_bench()
    calls = []
    real_conv = unet_oracle.conv

    def counting_conv(x, Wt, b):
        calls.append((x.shape[0] * x.shape[1], x.shape[2], Wt.shape[0]))
        return real_conv(x, Wt, b)

    monkeypatch.setattr(unet_oracle, "conv", counting_conv)
    rng = np.random.default_rng(3)
    params = rng.standard_normal(unet_oracle.num_params(widths)) * 0.1
    unet_oracle.forward(params, widths, rng.standard_normal((H, W, 4)))
    assert len(calls) == 15
    px, cin, cout = calls[0]
    calls[0] = (px, 4, cout)      # 12 of the 16 input channels are zero padding
    px, cin, cout = calls[-1]
    calls[-1] = (px, cin, 1)      # only output channel 0 is the prediction
    flops = sum(2 * 9 * ci * co * n for n, ci, co in calls)
    assert bench.unet_forward_flops(widths, H, W) == flops


def test_config_names_only_the_workload():
    """Both arms print the same `config` object (built from the workload
    alone); measurement results go to `details`, never into `config`."""
    from paper_2402_17337_gb300 import workloads as W
    bench = load_bench()
    cfg = W.plunge_2048x1024()
    a = bench.workload_config(cfg, 1)
    b = bench.workload_config(W.plunge_2048x1024(), 1)
    assert a == b and a["workload"] == "plunge_2048x1024" and (a["nx"], a["ny"]) == (2048, 1024)
    assert set(a) == {"workload", "nx", "ny", "global_batch", "parallelism", "l2"}
    cases = W.batch64()
    c = bench.batch_config(cases, 2)
    assert c["workload"] == "batch64" and c["cases"] == 64 and c["global_batch"] == 128
    assert c["cells_per_step"] == sum(x.cells for x in cases)
