"""Sliding-window decoding of long syndrome histories through the C ABI.

Windows of W detector layers start every C layers; window k's graph is the
induced subgraph of the stream graph on its layers (qec_graph_create_window),
with the first C layers as its commit region (every layer for the last window).
For each window the library assembles the window syndromes on the device
(stream bits of its layers XOR the previous window's carry) and decodes them,
XOR-accumulating the committed observable; the committed edges leaving the
region flip detectors of the next window (qec_decode_window_batch,
qec_window_assemble).  This module only sequences those calls; graph()
records the whole sequence of one decode into a CUDA graph.
"""

from __future__ import annotations

import numpy as np

from . import Graph, decode_window_batch, window_assemble


def plan(num_layers: int, W: int, C: int):
    """(first layer, layers, is last) of each window over num_layers layers."""
    if not (1 <= C <= W):
        raise ValueError("need 1 <= C <= W")
    out, a = [], 0
    while a + W < num_layers:
        out.append((a, W, False))
        a += C
    out.append((a, num_layers - a, True))
    return out


class SlidingWindow:
    """Decoder for many streams of one stream graph: `stream` is a Graph of the
    whole history whose detectors are numbered layer by layer, `layer_size`
    detectors per layer."""

    def __init__(self, stream: Graph, layer_size: int, W: int, C: int):
        n = stream.num_detectors
        if layer_size < 1 or n % layer_size:
            raise ValueError("the stream's detectors must form whole layers of layer_size")
        self.stream = stream
        self.nz = int(layer_size)
        self.W, self.C = W, C
        self.windows = []
        for a, nl, last in plan(n // self.nz, W, C):
            g = Graph.window(stream, a * self.nz, nl * self.nz)
            bits = np.zeros(g.words * 32, np.uint8)
            bits[:(g.num_detectors if last else C * self.nz)] = 1
            g.set_commit_region(np.packbits(bits, bitorder="little").view(np.uint32))
            self.windows.append((a, nl, last, g))

    def decode(self, syndromes, num_streams: int, stream=None):
        """syndromes: int32 CUDA tensor [num_streams * stream words] (uint32 rows).
        Returns (observable int64 [S] holding the uint64 bits, status int32 [S])."""
        import torch
        dev = syndromes.device
        S = int(num_streams)
        sw = self.stream.words
        obs = torch.zeros(S, dtype=torch.int64, device=dev)
        status = torch.zeros(S, dtype=torch.int32, device=dev)
        carry_prev, prev = None, None
        for a, nl, last, g in self.windows:
            rows = torch.empty(S * g.words, dtype=torch.int32, device=dev)
            if carry_prev is None:
                window_assemble(syndromes, sw, a * self.nz, nl * self.nz, rows, g.words, S, stream=stream)
            else:
                pa, pnl, pg = prev
                overlap = (pa + pnl - a) * self.nz   # the previous window's layers this one shares
                window_assemble(syndromes, sw, a * self.nz, nl * self.nz, rows, g.words, S,
                                carry_rows=carry_prev, carry_words=pg.words,
                                carry_bit_begin=(a - pa) * self.nz, carry_bits=overlap, stream=stream)
            carry = torch.empty_like(rows)
            decode_window_batch([g], rows, obs, carry, status, num_shots=S, stream=stream)
            carry_prev, prev = carry, (a, nl, g)
        return obs, status

    def graph(self, syndromes, num_streams: int):
        """Record decode(syndromes, num_streams) into a CUDA graph (torch).
        Returns (graph, obs, status): graph.replay() decodes whatever the
        `syndromes` tensor holds at that time into the same obs / status
        tensors.  One uncaptured decode of the same shape runs first (it sizes
        the library's workspace); replays must not overlap other decodes on
        the device."""
        import torch
        self.decode(syndromes, num_streams)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            obs, status = self.decode(syndromes, num_streams)
        return g, obs, status
