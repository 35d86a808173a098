"""Batched matching of many pairs of uneven size, replayed from a CUDA graph.

`dco_stereo_match_batch` runs each stage of the path as one launch over all
pairs (up to 64 pairs per launch, descriptors in the kernel parameters).
`BatchGraph` fixes a set of pair shapes (and, optionally, each pair's tile
choice from the autotuner: pass width and blocks), reserves the workspace, warms the
library up (tables, shared-memory opt-ins), captures the batched call on a
stream into a CUDA graph, and replays it for new inputs copied into its
static device buffers.  Only buffer management and graph bookkeeping live
here; every stage runs in libdco_stereo.so.
"""
from __future__ import annotations

from typing import Optional, Sequence

from .binding import Params, Stereo, Tile


class BatchGraph:
    def __init__(self, stereo: Stereo, shapes: Sequence[tuple[int, int, int]],
                 params: Optional[Params] = None, device: int = 0,
                 tiles: Optional[Sequence] = None):
        import torch
        self.st = stereo
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.params = params
        self.dev = torch.device(f"cuda:{device}")
        self.left = [torch.empty((H, W, 3), dtype=torch.uint8, device=self.dev) for W, H, _ in self.shapes]
        self.right = [torch.empty_like(t) for t in self.left]
        self.out = [torch.empty((H, W), dtype=torch.int16, device=self.dev) for W, H, _ in self.shapes]
        self.stream = torch.cuda.Stream(self.dev)
        for t in self.left + self.right:
            t.zero_()
        # per-pair tiles (e.g. tune.tune_batch); 0 fields = the call's parameters
        self.tiles = [Tile.of(v) for v in (tiles or [None] * len(self.shapes))]
        pairs = [(l, r, D, o, t) for l, r, (_, _, D), o, t
                 in zip(self.left, self.right, self.shapes, self.out, self.tiles)]
        self._pairs = pairs
        # warm-up outside capture: workspace, tables, shared-memory opt-ins
        with torch.cuda.stream(self.stream):
            self.st.match_batch(pairs, self.params)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.st.match_batch(pairs, self.params)
        torch.cuda.synchronize(self.dev)

    def load(self, lefts, rights) -> None:
        """Copy the inputs (device or pinned host tensors) into the graph's buffers."""
        for dst, src in zip(self.left, lefts):
            dst.copy_(src, non_blocking=True)
        for dst, src in zip(self.right, rights):
            dst.copy_(src, non_blocking=True)

    def replay(self):
        """Run the captured batch; returns the static output maps."""
        self.graph.replay()
        return self.out

    def __call__(self, lefts, rights):
        self.load(lefts, rights)
        return self.replay()
