"""Batched serving: V views x E lights rendered by one CUDA-graph launch.

Each view is one rt_render_frame_multi call (its G-buffer lit by all E
environment maps on a shared geometry pass); the V calls are captured once
into a CUDA graph and replayed as a single launch.  Timing events recorded
between the views inside the graph give per-view latencies.  Before capture
the context's launch shape can be picked by the native autotuner (rt_tune) on
the first view (or a slice of it).
"""
from __future__ import annotations

from typing import Dict, List, Optional

import torch

from .binding import Renderer


def _event():
    try:
        return torch.cuda.Event(enable_timing=True, external=True)
    except TypeError:   # older torch: events recorded in a capture are external already
        return torch.cuda.Event(enable_timing=True)


class BatchedServer:
    def __init__(self, renderer: Renderer, gbs: List[Dict[str, torch.Tensor]], envs: torch.Tensor,
                 pixel_offsets: Optional[List[int]] = None):
        self.r = renderer
        self.gbs = gbs
        self.envs = envs
        self.offsets = pixel_offsets or [0] * len(gbs)
        P = gbs[0]["pos"].shape[0]
        self.out = torch.empty(len(gbs), envs.shape[0], P, 4, device=envs.device, dtype=torch.float32)
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.events = []
        self.tuned_ms = None

    def tune(self, pixels: Optional[int] = None) -> float:
        """Pick the launch shape (tile shape, lights per launch, warpgroups) with rt_tune on the first
        view, or on its first `pixels` pixels (the search times 36 shapes twice each); returns the
        best time in ms."""
        gb = self.gbs[0]
        if pixels is not None and pixels < gb["pos"].shape[0]:
            gb = {k: v[:pixels] for k, v in gb.items()}
        self.tuned_ms = self.r.tune(gb, self.envs, self.offsets[0])
        return self.tuned_ms

    def render_eager(self) -> torch.Tensor:
        for v, gb in enumerate(self.gbs):
            self.r.render_frame_multi(gb, self.envs, self.offsets[v], out=self.out[v])
        return self.out

    def capture(self) -> None:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.render_eager()          # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.events = [_event() for _ in range(len(self.gbs) + 1)]
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            for v, gb in enumerate(self.gbs):
                self.events[v].record()
                self.r.render_frame_multi(gb, self.envs, self.offsets[v], out=self.out[v])
            self.events[-1].record()

    def replay(self) -> torch.Tensor:
        assert self.graph is not None, "capture() first"
        self.graph.replay()
        return self.out

    def view_latencies_ms(self) -> List[float]:
        """Per-view times of the last replay (call after synchronising)."""
        return [a.elapsed_time(b) for a, b in zip(self.events[:-1], self.events[1:])]
