"""Binding of the CPU/GPU pipeline of the numeric stage (include/sc_pipeline.h):
argument marshalling and buffer setup only.  Host factorisation threads, the
copy stream and the assembly all run in the native library.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence

import numpy as np
import scipy.sparse as sp

from . import _native, abi, sc
from .sc import SCError, _stream_ptr


class Pipeline:
    """Numeric stage of a batch in `nchunks` chunks: host Cholesky of chunk
    c+1 overlapped with the H2D copy and GPU assembly of chunk c.

    subdomains: the problem's subdomains (K, fixed, B^T, lambda map);
    factored: their FactoredSubdomain (host.factorize_problem), which fix the
    ordering and the L patterns the per-chunk plans are made for.
    """

    def __init__(self, subdomains: Sequence, factored: Sequence, n_dual: int, nchunks: int = 4,
                 device="cuda", nthreads: int = 0):
        import torch
        self.lib = _native.pipe_lib()
        nsub = len(subdomains)
        assert len(factored) == nsub and nsub > 0
        nchunks = max(1, min(int(nchunks), nsub))
        bounds = [round(c * nsub / nchunks) for c in range(nchunks + 1)]
        self._keep: List[object] = []
        self.subs = (abi.PipeSubdomain * nsub)()
        for i, (sd, fs) in enumerate(zip(subdomains, factored)):
            K = sp.csc_matrix(sd.K)
            K.sort_indices()
            arrs = [np.ascontiguousarray(K.indptr, np.int64), np.ascontiguousarray(K.indices, np.int32),
                    np.ascontiguousarray(K.data, np.float64), np.ascontiguousarray(np.asarray(sd.fixed), np.int32),
                    np.ascontiguousarray(fs.L.perm, np.int32)]
            self._keep += arrs
            s = self.subs[i]
            s.n = K.shape[0]
            s.K_colptr, s.K_rowind, s.K_val = arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data
            s.nfixed = len(arrs[3])
            s.fixed = arrs[3].ctypes.data if len(arrs[3]) else None
            s.perm = arrs[4].ctypes.data
        self.plans = [sc.Plan(factored[bounds[c]:bounds[c + 1]], n_dual).upload(device) for c in range(nchunks)]
        self.bounds = bounds
        lmax = max(p.sizes.L_values for p in self.plans)
        self.L_bufs = [torch.empty(max(1, lmax), dtype=torch.float64, device=device) for _ in range(min(2, nchunks))]
        ws_bytes = max(p.sizes.ws_bytes for p in self.plans)
        self.ws = torch.empty(max(256, ws_bytes), dtype=torch.uint8, device=device)
        self.F = [p.new_F(device) for p in self.plans]
        self.chunks = (abi.PipeChunk * nchunks)()
        for c, p in enumerate(self.plans):
            ch = self.chunks[c]
            ch.lo, ch.hi = bounds[c], bounds[c + 1]
            ch.plan = p.h.value
            ch.L_dev = self.L_bufs[c % len(self.L_bufs)].data_ptr()
            ch.F_dev = self.F[c].data_ptr()
            ch.ws_dev = self.ws.data_ptr()
            ch.ws_bytes = self.ws.numel()
        h = ctypes.c_void_p()
        st = self.lib.scp_create(ctypes.byref(h), nsub, self.subs, nchunks, self.chunks, int(nthreads))
        self.h = h
        if st != abi.SC_OK:
            msg = self.lib.scp_last_error(h).decode() if h.value else "scp_create failed"
            if h.value:
                self.lib.scp_destroy(h)
                self.h = ctypes.c_void_p()
            raise SCError(st, msg)

    def run(self, stream=None) -> dict:
        t = abi.PipeTimes()
        st = self.lib.scp_run(self.h, _stream_ptr(stream), ctypes.byref(t))
        if st != abi.SC_OK:
            raise SCError(st, self.lib.scp_last_error(self.h).decode())
        return {k: getattr(t, k) for k, _ in abi.PipeTimes._fields_}

    def export(self, i: int):
        """F_i (dense m x m, device) of subdomain i of the batch."""
        c = next(c for c in range(len(self.plans)) if self.bounds[c] <= i < self.bounds[c + 1])
        return self.plans[c].export(self.F[c], i - self.bounds[c])

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                self.lib.scp_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass
