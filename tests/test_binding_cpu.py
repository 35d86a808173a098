"""The binding's argument checks (no GPU needed): the C library trusts the
buffer sizes it is given, so the binding rejects images and buffers of the
wrong shape, element type, layout or device before any call."""
import numpy as np
import pytest
import torch

from paper_2203_02300_gb300 import binding as B


def test_images_must_be_hwc_uint8_and_contiguous():
    assert B._rgb_dims(np.zeros((4, 6, 3), np.uint8)) == (6, 4)
    assert B._rgb_dims(torch.zeros((4, 6, 3), dtype=torch.uint8)) == (6, 4)
    bad = [np.zeros((4, 6), np.uint8), np.zeros((4, 6, 4), np.uint8), np.zeros((4, 6, 3), np.float32),
           np.zeros((6, 4, 3), np.uint8).transpose(1, 0, 2), torch.zeros((4, 6, 3), dtype=torch.int16),
           torch.zeros((4, 12, 3), dtype=torch.uint8)[:, ::2]]
    for a in bad:
        with pytest.raises(ValueError):
            B._rgb_dims(a)


def test_buffers_must_match_shape_type_layout_and_device():
    out = torch.zeros((4, 6), dtype=torch.int16)
    B._expect("out", out, (4, 6), "int16", out)
    B._expect("out", np.zeros((4, 6), np.int16), (4, 6), "int16")
    cases = [(torch.zeros((4, 5), dtype=torch.int16), "int16"),        # shape
             (torch.zeros((4, 6), dtype=torch.int32), "int16"),        # element type
             (torch.zeros((6, 4), dtype=torch.int16).t(), "int16"),    # layout
             (np.zeros((4, 6), np.float32), "int16")]
    for t, dt in cases:
        with pytest.raises(ValueError):
            B._expect("out", t, (4, 6), dt)
    meta = torch.empty((4, 6), dtype=torch.int16, device="meta")
    with pytest.raises(ValueError):
        B._expect("out", meta, (4, 6), "int16", out)                  # device
