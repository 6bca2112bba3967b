"""CUDA-graph capture and replay of library calls (``sg_graph_*``)."""

from __future__ import annotations

import contextlib
import ctypes as C

import torch

from . import _lib
from ._lib import check


class Graph:
    """An executable graph of the library calls enqueued on one stream.

    Usage::

        g = Graph()
        with g.capture(stream):
            sim.rollout(64, ..., stream=stream)
        g.launch(stream)   # replays continue from the device-side counters
    """

    def __init__(self):
        self.L = _lib.load()
        self.handle = C.c_void_p()

    @contextlib.contextmanager
    def capture(self, stream: torch.cuda.Stream):
        s = C.c_void_p(stream.cuda_stream)
        check(self.L.sg_graph_begin(s), "sg_graph_begin")
        ok = False
        try:
            with torch.cuda.stream(stream):
                yield self
            ok = True
        finally:
            h = C.c_void_p()
            rc = self.L.sg_graph_end(s, C.byref(h))
            if ok:
                check(rc, "sg_graph_end")
            self.handle = h

    def launch(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        check(self.L.sg_graph_launch(self.handle, C.c_void_p(s.cuda_stream)), "sg_graph_launch")

    def num_nodes(self) -> int:
        n = C.c_int64()
        check(self.L.sg_graph_num_nodes(self.handle, C.byref(n)), "sg_graph_num_nodes")
        return int(n.value)

    def close(self):
        if self.handle.value:
            self.L.sg_graph_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
