"""GPU unit rates behind the roofline denominators: the MUFU sin/cos and
FP32 FMA rates of the generic path and the tcgen05 f16 MMA rate of the
separable path, measured on the running device through the C ABI."""
import pytest

import __graft_entry__
from paper_1010_2641_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def test_mufu_and_fma_rates():
    mufu = api.microbench(0)["ops_per_clk_per_sm"]
    fma = api.microbench(2)["ops_per_clk_per_sm"]
    assert 12.0 < mufu < 16.5          # 16 sin/cos per SM per clock
    assert 100.0 < fma < 129.0         # 128 FP32 FMA lanes per SM per clock


def test_tcgen05_f16_rate():
    r = api.microbench(8, iters=20000)
    # dense kind::f16 at M=128 N=256 K=16: 8192 flop per SM per clock
    assert 0.85 * 8192 < r["ops_per_clk_per_sm"] < 1.02 * 8192
    assert r["n_sm"] >= 100
