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


def test_tile_candidates_follow_the_block_limits():
    # the autotuner only proposes blocks the library accepts: 0 (automatic)
    # or at least 32 positions, a first-pass block with its 2 x arm_l1 halo
    # within 1024 prefix positions unless it is a whole line of <= 1024, a
    # second-pass block within 512 - 2 x arm_l1 unless it is a whole column
    # of <= 512; each candidate a different block count
    from paper_2203_02300_gb300 import tune
    from paper_2203_02300_gb300.binding import Tile
    for L1 in (34, 40, 3):
        for n in (33, 97, 160, 320, 480, 640, 720, 1080, 1280, 1920, 4000):
            hs = tune.first_pass_candidates(n, L1)
            vs = tune.second_pass_candidates(n, L1)
            assert hs[0] == 0 and vs[0] == 0
            for c in hs[1:]:
                assert 32 <= c < n and c + 2 * L1 <= 1024, (n, L1, c)
            for c in vs[1:]:
                assert 32 <= c <= n and (c == n <= 512 or c <= 512 - 2 * L1), (n, L1, c)
            counts = [-(-n // c) for c in vs[1:]]
            assert len(set(counts)) == len(counts)
            assert len(set(hs)) == len(hs)
    assert Tile.of(None) == Tile() and Tile.of(64) == Tile(64, 0, 0) and Tile.of((32, 96, 120)) == Tile(32, 96, 120)
