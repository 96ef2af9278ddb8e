"""bench.py's report arithmetic on a synthetic record (CPU, no GPU).

The roofline figures follow from the stage times by fixed formulas: the S
pass moves 8 m n + 4 r (m + n) bytes; Algorithm 1 does 4 p r flops per
problem-iteration at the mean iteration count over (n - n') column problems
of length m' and (m - m') row problems of length n'; the seed does 6 m'n'k
+ 4 (m' + n') k^2 flops per pass, k = r + max(6, r/4), over the ALM
iterations plus 3 prologue passes.  The dominant stage (longest time) names
the line's roofline, and value is m n over the mean step time.
"""
import types

import numpy as np
import pytest

import bench


@pytest.fixture(scope="module")
def pk():
    from paper_1108_5359_gb300 import build, _abi
    build.build()
    _abi.load()
    import paper_1108_5359_gb300 as pkg
    return pkg


def _record(P, seed_ms, filt_ms, spass_ms, iters_mean, seed_iters):
    return dict(P=P, M32=None, wl="c2_5000_r20", precision="fp32", steps=4,
                warmup=3, t_step=seed_ms + filt_ms + spass_ms,
                step_ms=[seed_ms + filt_ms + spass_ms] * 4,
                stage={"seed": [seed_ms] * 3, "filter": [filt_ms] * 3,
                       "spass": [spass_ms] * 3},
                launches=24, wall=0.1, clocks={}, e2e=None, Lrec=None,
                Sh=None, ws=1, cpu_mode=None, parity={"status": 0},
                info={"filter_iters_max": 30,
                      "filter_iters_mean": iters_mean,
                      "seed_iters": seed_iters, "seed_team": -152})


def test_roofline_arithmetic_of_the_default_line(pk):
    # shapes of the 5000 x 5000 rank-20 workload, without its matrix
    P = types.SimpleNamespace(m=5000, n=5000, r=20, rows=np.arange(200),
                              cols=np.arange(200))
    out = bench.report(pk, _record(P, 2.6, 0.24, 0.037, 19.25, 25))
    m = n = 5000
    r, mp, k = 20, 200, 26
    assert out["value"] == pytest.approx(m * n / (2.877e-3))
    sp = out["stages"]["spass"]
    assert sp["algorithmic_bytes"] == 8 * m * n + 4 * r * (m + n)
    assert sp["achieved"] == pytest.approx(
        (8 * m * n + 4 * r * (m + n)) / 0.037e-3 / 1e9)
    assert sp["frac"] == pytest.approx(sp["achieved"] / sp["peak"])
    fl = out["stages"]["filter"]
    flops = 4.0 * r * ((n - mp) * mp + (m - mp) * mp) * 19.25
    assert fl["achieved"] == pytest.approx(flops / 0.24e-3 / 1e12)
    sd = out["stages"]["seed"]
    seed_flops = (25 + 3) * (6.0 * mp * mp * k + 4.0 * (2 * mp) * k ** 2)
    assert sd["achieved"] == pytest.approx(seed_flops / 2.6e-3 / 1e12)
    assert sd["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    # the seed is the longest stage, so it names the roofline
    assert out["roofline"]["kernel"] == "seed_alm_kernel"
    assert out["roofline"]["frac"] == pytest.approx(sd["frac"])
    assert out["roofline"]["traffic"] == 1119488
    assert out["gpu_launches"] == 24


def test_clock_sampler_covers_the_timed_region(tmp_path, monkeypatch):
    # a stand-in nvidia-smi that prints one sample line every 50 ms (the
    # power cap active): the sampler waits for its first line before the
    # timed region starts, leaves the lines taken before out, and reports
    # the median clock, the maximum and the active reasons
    import os
    import sys
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import sys, time\n"
        "i = 0\n"
        "while True:\n"
        "    sm = 2070 if i else 1200\n"
        "    print(f'0, {sm}, 2070, 900.0, Active, Not Active, Not Active, "
        "Not Active, Active', flush=True)\n"
        "    i += 1\n"
        "    time.sleep(0.05)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep +
                       os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.4)
    out = s.stop()
    assert out is not None and out["samples"] >= 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
