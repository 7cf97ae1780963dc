"""The bench's algorithmic counts for the learned guess's roofline, written
out by hand for the two network widths: flops = 2 x 9 x the multiply-adds of
each 3x3 layer; HBM bytes per pixel = the step residual (read m^{n-1} 8 B,
write r 4 B), the packing (read m^{n-1}, the seed, r: 8 + 8 + 4 B; write the
padded BF16 input row: 16 channels = 32 B), then every layer's BF16 input row
and output row once (16 channels = 32 B, 32 channels = 64 B; the last layer
writes one FP32 value)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_network_flops_per_pixel():
    assert bench.cnn_flops_per_pixel((10, 32, 32, 32, 1)) == 18 * (10 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
    assert bench.cnn_flops_per_pixel((10, 32, 32, 32, 1)) == 43200
    assert bench.cnn_flops_per_pixel((10, 16, 16, 1)) == 7776


def test_network_bytes_per_pixel():
    # 12 + 52 + (32 + 64) + (64 + 64) + (64 + 64) + (64 + 4)
    assert bench.cnn_bytes_per_pixel((10, 32, 32, 32, 1)) == 484
    # 12 + 52 + (32 + 32) + (32 + 32) + (32 + 4)
    assert bench.cnn_bytes_per_pixel((10, 16, 16, 1)) == 228
