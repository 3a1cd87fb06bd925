"""Template search over an unbounded stream: the Python face of tde_stream_*.

A short template y is searched for in a long signal x that arrives in
chunks (the paper's closing remark on long signals). The library quantizes
every chunk as it arrives (the sign quantizer, b = 1: it is pointwise, so a
chunk quantizes the same alone as inside the whole signal; the rank
quantizer's thresholds are order statistics of the whole signal and cannot be
known from a prefix), keeps the last ny - 1 levels, correlates the template
over the lags where it lies wholly inside (Eq. (1), exact integers) and folds
each chunk's tie-ruled maximum into a device-resident running best. Positions
are global: the template at position k of x is lag tau = -k; ties go to the
earliest position, as in the one-shot argmax, so after each chunk the answer
equals Algorithm 1 on the prefix seen so far. This module only marshals
arguments.
"""
from __future__ import annotations

import ctypes

import torch

from . import tde


class TemplateStream:
    """Running exact search for y (FP32, device) in a stream of FP32 chunks
    (tde_stream_create / tde_stream_push / tde_stream_best)."""

    def __init__(self, ctx, y: torch.Tensor, bits: int = 1, engine: str = "auto",
                 max_chunk: int = 1 << 20, stream=None):
        if bits != 1:
            raise ValueError("streaming needs a pointwise quantizer: bits must be 1 (sign)")
        if y.dtype != torch.float32 or not y.is_cuda or y.dim() != 1 or y.numel() < 1:
            raise ValueError("y must be a non-empty 1-D float32 CUDA tensor")
        self.ctx, self.max_chunk = ctx, int(max_chunk)
        self.y = y.contiguous()
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.tde_stream_create(ctx.handle, self.y.data_ptr(), self.y.numel(), int(bits),
                                            tde._engine(engine), self.max_chunk, tde._stream(stream),
                                            ctypes.byref(h)))
        self.handle = h
        self._out = torch.zeros(2, dtype=torch.int64, device=y.device)
        self.best = None

    def push_async(self, x: torch.Tensor, stream=None):
        """Enqueues the next chunk (asynchronous, no host synchronisation);
        chunks longer than max_chunk are pushed in pieces."""
        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 1:
            raise ValueError("chunks must be 1-D float32 CUDA tensors")
        x = x.contiguous()
        for a in range(0, x.numel(), self.max_chunk):
            piece = x[a: a + self.max_chunk]
            self.ctx.check(self.ctx.lib.tde_stream_push(self.handle, piece.data_ptr(), piece.numel(),
                                                        tde._stream(stream)))

    def read(self, stream=None):
        """The running best (lag, value), or None while fewer than ny samples
        have arrived; waits for `stream`."""
        found = ctypes.c_int(0)
        o = self._out
        self.ctx.check(self.ctx.lib.tde_stream_best(self.handle, o.data_ptr(), o.data_ptr() + 8,
                                                    ctypes.byref(found), tde._stream(stream)))
        if not found.value:
            return None
        self.ctx.sync(stream)
        v = o.cpu()
        return int(v[0]), int(v[1])

    def push(self, x: torch.Tensor, stream=None):
        """Adds the next chunk of x; returns the best (lag, value) so far (None
        while fewer than ny samples have arrived)."""
        self.push_async(x, stream)
        self.best = self.read(stream)
        return self.best

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tde_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
