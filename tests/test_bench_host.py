"""Host-side accounting of bench.py (no GPU): the flop counts behind the
roofline fractions it reports.

The algorithmic count is the separable FIR over C = 4(K-1) + 2 real channels
(two passes of 2W + 1 taps, 2 flops per multiply-add).  The tensor-core kernel
issues MMAs over 4 channels for every harmonic, with band padding and the split
products, so its issued count can never be below the algorithmic count times
the products per step, and the padding stays bounded.
"""
import math

import pytest

import bench

FORMS = sorted(bench.TC_NSPLIT)


def test_algorithmic_flops_closed_form():
    # K = 1: the n = 0 term only (channels f and 1); W = 0: a single tap
    assert bench.algorithmic_flops_per_pixel(1, 0) == 2 * 2 * 1 * 2
    # the 2048^2 setting sigma_s = 10 (W = 30), K = 17: C = 66 channels
    assert bench.algorithmic_flops_per_pixel(17, 30) == 4 * 61 * 66


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("K", [1, 9, 17])
def test_issued_flops_bound_the_algorithmic_count(form, K):
    px = bench.H * bench.W_IMG
    for W in range(0, 33):
        issued = bench.tc_issued_flops(K, W, form)
        useful = bench.algorithmic_flops_per_pixel(K, W) * px * bench.TC_NSPLIT[form]
        assert issued >= useful, (form, K, W)
        # padding: 16-wide K chunks around a 2W + 1 band, 4 channels where K = 1
        # has 2, computed rows past 128 - 2W; bounded once the band fills a chunk
        if W >= 9:
            assert issued <= 12 * useful, (form, K, W)


def test_issued_flops_follow_the_tile_count():
    """2048^2 at W = 9, single FP16 form (second tensor-core layout): 64 x 19
    tiles of 128 - 2W = 110 output rows (8 waves of 152 CTAs); per tile and
    harmonic 4 channels x 4 row chunks (Wp = 16, 16 + 32 + 9 ext columns -> 64)
    of 128 x 32 x 16 and 8 column chunks of 128 x 128 x 16.  The split forms up
    to W = 32 run the first layout: at W = 30 64 x 32 tiles of 64 rows, 6 row
    chunks, two 32-row column blocks of ceil((32 + 2W) / 16) = 6 chunks each."""
    tiles = math.ceil(2048 / 32) * math.ceil(2048 / 110)
    assert tiles == 1216 == 8 * 152
    per_tile = 4 * 4 * 2 * 128 * 32 * 16 + 8 * 2 * 128 * 128 * 16
    assert bench.tc_layout("tc_fp16_single", 9) == "tc2"
    assert bench.tc_issued_flops(1, 9, "tc_fp16_single") == tiles * per_tile
    assert bench.tc_layout("tc_fp16", 9) == bench.tc_layout("tc_bf16", 30) == "tc1"
    assert bench.tc_layout("tc_fp16", 36) == "tc2"
    tiles1 = 64 * 32
    per_tile1 = 4 * 6 * 2 * 128 * 32 * 16 + 2 * 6 * 2 * 128 * 32 * 16
    assert bench.tc_issued_flops(1, 30, "tc_bf16") == 3 * tiles1 * per_tile1
