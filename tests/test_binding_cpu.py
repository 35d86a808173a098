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


def test_tuner_coordinate_search_and_cache(tmp_path, monkeypatch):
    # the tuner's host logic with a fake timer: the pass width first, then the
    # first pass's blocks, then the second's; a change only when more than 1 %
    # faster; the winner cached per shape and read back
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_02300_gb300 import tune
    from paper_2203_02300_gb300.binding import Tile
    monkeypatch.setenv("DCO_TUNE_CACHE", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "fake GPU")
    W, H, D = 640, 480, 128
    cost = {}

    def ms(t):
        base = {32: 1.0, 64: 0.8, 96: 0.795, 128: 0.7}[t.d_chunk]   # 96: within 1 % of 64 (kept 64); 128 wins
        h = {0: 0.0, 320: -0.05, 224: -0.004, 160: 0.02, 128: 0.03, 96: 0.04}[t.h_chunk]
        v = {0: 0.0, 240: 0.01, 160: -0.03, 120: -0.0301, 96: 0.0, 80: 0.05}[t.v_chunk]
        return base + h + v

    class FakeStereo:
        def match(self, left, right, D, p, out):
            cost["last"] = Tile(p.d_chunk, p.h_chunk, p.v_chunk)

    def fake_time(fn, reps):
        fn()
        return ms(cost["last"])
    monkeypatch.setattr(tune, "_time_call", fake_time)
    left = torch.zeros((H, W, 3), dtype=torch.uint8)
    won = tune.tune_tiles(FakeStereo(), left, left, D)
    # 128 beats 64 by far; h 320 beats 0 by 5 %; v 160 beats 0 by 3 % and
    # 120 is not 1 % better than 160
    assert won == Tile(128, 320, 160)
    assert tune.lookup(W, H, D, "fake GPU") == won
    monkeypatch.setattr(tune, "_time_call", lambda fn, reps: (_ for _ in ()).throw(AssertionError("timed again")))
    assert tune.tune_tiles(FakeStereo(), left, left, D) == won   # from the cache
