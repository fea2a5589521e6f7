"""The benchmark's algorithmic bookkeeping (the numerators of its roofline fractions),
checked against independent derivations: MACs from the layer shapes of the weight
generator, and FC evaluations from the oracle's own second-slice rule."""

import numpy as np
import pytest

import bench
import oracle
import synth

# positions at which each layer's output is computed (L of the output) and its kernel taps
LAYER_L = {"enc1": 4000, "enc2": 2000, "enc3": 1000, "enc4": 500, "dec3": 1000,
           "dec2": 2000, "dec1": 4000, "final": 4000}
CONVT_LIN = {"up3": 500, "up2": 1000, "up1": 2000}


def unet_macs_from_shapes(c0):
    shapes = synth.layer_shapes(c0)
    total = 0
    for name, L in LAYER_L.items():
        cout, cin, k = shapes[name][0]
        total += L * cout * cin * k
    for name, lin in CONVT_LIN.items():
        cin, cout, k = shapes[name][0]
        total += lin * cin * cout * k            # each input position feeds k = 2 outputs
    return total


@pytest.mark.parametrize("c0", [16, 32])
def test_fp32_kernel_table_macs_equal_the_layer_shapes(c0):
    t = bench.kernel_table("fp32", c0)
    assert sum(v[0] for v in t.values()) == 0                   # no tensor-core work
    assert sum(v[1] for v in t.values()) == unet_macs_from_shapes(c0)


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp8"])
def test_wide_tensor_core_kernel_table_covers_the_wide_macs(form):
    t = bench.kernel_table(form, 32)
    assert sum(v[0] + v[1] for v in t.values()) == unet_macs_from_shapes(32)
    assert {"enc4", "up3", "dec3", "up2", "dec2_up1", "dec1_final"} <= set(t)


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp8"])
def test_tensor_core_kernel_table_covers_the_same_macs(form):
    t = bench.kernel_table(form, 16)
    assert sum(v[0] + v[1] for v in t.values()) == unet_macs_from_shapes(16)
    assert unet_macs_from_shapes(16) == 122_496_000          # 245 MFLOP per event
    # on CUDA cores: enc1 (1 -> 16) and the final conv (16 -> 1), 4000 x 16 x 5 MACs each
    assert sum(v[1] for v in t.values()) == 2 * 4000 * 16 * 5


def test_per_interval_kernel_tables_count_every_sequence():
    """The per-interval layout (§3): 40 sequences of 104 bins per event, each layer at
    104 / 2^k positions per sequence; the final conv gives the 4000 central logits."""
    shapes = synth.layer_shapes(16)
    pos = {"enc1": 104, "enc2": 52, "enc3": 26, "enc4": 13, "dec3": 26, "dec2": 52, "dec1": 104}
    want = sum(40 * L * shapes[n][0][0] * shapes[n][0][1] * shapes[n][0][2] for n, L in pos.items())
    want += 4000 * 16 * 5                                       # final conv, 16 -> 1
    for n, lin in {"up3": 13, "up2": 26, "up1": 52}.items():
        cin, cout, k = shapes[n][0]
        want += 40 * lin * cin * cout * k
    for form in ("fp32", "bf16", "fp16", "fp8"):
        t = bench.kernel_table(form, 16, iv=True)
        assert sum(v[0] + v[1] for v in t.values()) == want, form


def test_dominant_kernel_fraction_from_the_method_flops():
    """dec3_up2 (dec3 1000 x 64 x 640 plus up2 1000 x 64 x 64 MACs per event) at 100 us
    per 1000-event launch: 2 x 45.056e6 x 1000 FLOP / 100 us = 901 TFLOP/s."""
    peaks = {"bf16_tflops": 1949.8, "hbm_gbs": 6785.5, "sm_max_mhz": 2070.0}
    r = bench.roofline_of("dec3_up2", 10, 1.0, "fp16", 1000, 155000, peaks)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 901.12) < 0.01
    assert abs(r["frac"] - 901.12 / 1949.8) < 1e-5
    r8 = bench.roofline_of("dec3_up2", 10, 1.0, "fp8", 1000, 155000, peaks)
    assert abs(r8["frac"] - r["frac"] / 2) < 1e-9             # e4m3 peak = 2 x bf16
    front = bench.roofline_of("front", 1, 0.086, "fp16", 1000, 155000, peaks)
    assert set(front["unit_fracs"]) == {"alu", "sfu", "hbm", "tensor"}
    assert front["bound"] == "latency"                          # no unit near its peak


def test_activation_bytes_scale_with_the_element_size():
    b16 = sum(v[2] for v in bench.kernel_table("bf16").values())
    b8 = sum(v[2] for v in bench.kernel_table("fp8").values())
    # everything but the float32 logits (16 KB read by the tail, written by dec1_final)
    assert b16 - 32000 == 2 * (b8 - 32000)


def test_fc_evaluations_follow_the_oracle_second_slice_rule():
    b = synth.generate_standard(40, 3)
    z = b.features[2]
    for edge in (0.0, 0.5, 1.0):
        want = b.n_tracks
        for zi in z:
            s = oracle.slice_index(zi)[0]
            if s >= 0 and oracle.second_slice(zi, s, edge) >= 0:
                want += 1
        assert bench.fc_evaluations(b, edge) == want
    assert bench.fc_evaluations(b, 0.5) > b.n_tracks


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host cores (no GPU needed)
    and prints one JSON line with the same metric as the GPU arm."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--events", "16"], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "events/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
