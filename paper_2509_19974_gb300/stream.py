"""Template search over an unbounded stream (overlap-save over chunks).

A short template y is searched for in a long signal x that arrives in
chunks. Every chunk is quantized as it arrives (the sign quantizer, b = 1: it
is pointwise, so a chunk quantizes the same alone as inside the whole
signal; the rank quantizer's thresholds are order statistics of the whole
signal and cannot be known from a prefix). The last ny - 1 quantized samples
are carried over, the template is correlated through the library against
[carry | chunk] over the lags where it lies wholly inside (Eq. (1), exact
integers), and each chunk's tie-ruled maximum is folded into a running best.

Positions are global: the template at position k of x is lag tau = -k of
c[tau] = sum_n x[n] y[n + tau]. Ties go to the smallest |tau| (the earliest
position), as in the one-shot argmax, so after the last chunk the answer
equals Algorithm 1 on the whole signal over its valid lags.
"""
from __future__ import annotations

import torch


class TemplateStream:
    """Running exact search for y (FP32, device) in a stream of FP32 chunks."""

    def __init__(self, ctx, y: torch.Tensor, bits: int = 1, engine: str = "auto"):
        if bits != 1:
            raise ValueError("streaming needs a pointwise quantizer: bits must be 1 (sign)")
        if y.dtype != torch.float32 or not y.is_cuda or y.dim() != 1 or y.numel() < 1:
            raise ValueError("y must be a non-empty 1-D float32 CUDA tensor")
        self.ctx, self.bits, self.engine = ctx, bits, engine
        self.ny = y.numel()
        self.qy = ctx.quantize(y.contiguous(), bits)
        self.carry = torch.empty(0, dtype=torch.int8, device=y.device)
        self.consumed = 0  # samples of x seen so far
        self.best = None   # (lag, value) over the positions seen so far

    def push(self, x: torch.Tensor):
        """Adds the next chunk of x; returns the best (lag, value) so far (None
        while fewer than ny samples have arrived)."""
        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 1:
            raise ValueError("chunks must be 1-D float32 CUDA tensors")
        if x.numel() == 0:
            return self.best
        q = self.ctx.quantize(x.contiguous(), self.bits)
        buf = torch.cat([self.carry, q]) if self.carry.numel() else q
        base = self.consumed - self.carry.numel()  # position of buf[0] in x
        self.consumed += x.numel()
        nb = buf.numel()
        if nb >= self.ny:
            # template wholly inside buf: tau in [-(nb - ny), 0], position base - tau
            lo = -(nb - self.ny)
            c = self.ctx.xcorr_int(buf, self.qy, self.bits, lo, 0, engine=self.engine,
                                   dtype=torch.int64)
            lt, vt = self.ctx.argmax(c, lo)
            self.ctx.sync()
            cand = (-(base - int(lt.item())), int(vt.item()))
            self.best = cand if self.best is None else _better(cand, self.best)
        keep = min(self.ny - 1, nb)
        self.carry = buf[nb - keep:].clone() if keep else buf[:0]
        return self.best


def _better(a, b):
    """The pair (lag, value) the argmax's order prefers: the larger value,
    then the smaller |lag|, then the smaller lag."""
    (la, va), (lb, vb) = a, b
    if va != vb:
        return a if va > vb else b
    ka, kb = (abs(la), la), (abs(lb), lb)
    return a if ka < kb else b
