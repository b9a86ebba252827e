"""Binding of the GPU implicit dual-operator application (include/sc_implicit.h):
argument marshalling only.  q = sum_i B_i L_i^{-T} L_i^{-1} B_i^T lambda_i runs
in the library's CUDA kernel; the plan is built on the host by the library.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence

import numpy as np

from . import _native, abi
from .sc import SCError, _stream_ptr


class ImplicitPlan:
    """sci_plan + its device buffers, for a list of factored subdomains
    (the objects :class:`paper_2509_21037_gb300.sc.Plan` takes).
    cluster_min_work: -1 automatic, 0 every subdomain on an 8-CTA cluster,
    a large value none; pairs: 0 automatic, 1 every subdomain whose tree
    splits on a CTA pair, -1 none (include/sc_implicit.h, sci_options)."""

    def __init__(self, subdomains: Sequence, n_dual: int, cluster_min_work: int = -1, pairs: int = 0):
        self.lib = _native.sc_lib()
        self.nsub = len(subdomains)
        self.n_dual = int(n_dual)
        keep: List[np.ndarray] = []
        descs = (abi.SubdomainDesc * max(1, self.nsub))()
        for i, fs in enumerate(subdomains):
            arrs = [np.ascontiguousarray(fs.L.colptr, np.int64), np.ascontiguousarray(fs.L.rowind, np.int32),
                    np.ascontiguousarray(fs.bt_colptr, np.int32), np.ascontiguousarray(fs.bt_rowind, np.int32),
                    np.ascontiguousarray(fs.bt_sign, np.int8), np.ascontiguousarray(fs.lambda_map, np.int32)]
            keep += arrs
            d = descs[i]
            d.n, d.m = fs.n, fs.m
            d.L_colptr, d.L_rowind, d.Bt_colptr, d.Bt_rowind, d.Bt_sign, d.lambda_map = \
                [a.ctypes.data if a.size else None for a in arrs]
        h = ctypes.c_void_p()
        opt = abi.ImplicitOptions()
        opt.cluster_min_work = int(cluster_min_work)
        opt.pairs = int(pairs)
        st = self.lib.sci_plan(ctypes.byref(h), self.nsub, descs, self.n_dual, ctypes.byref(opt))
        self.h = h
        if st != abi.SC_OK:
            msg = self.lib.sci_last_error(h).decode() if h.value else "sci_plan failed"
            if h.value:
                self.lib.sci_destroy(h)
                self.h = ctypes.c_void_p()
            raise SCError(st, msg)
        self.sizes = abi.ImplicitSizes()
        self._check(self.lib.sci_get_sizes(self.h, ctypes.byref(self.sizes)))
        self.plan_dev = None
        self.ws = None

    def _check(self, st: int):
        if st != abi.SC_OK:
            raise SCError(st, self.lib.sci_last_error(self.h).decode())

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                self.lib.sci_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass

    def export_plan(self) -> np.ndarray:
        buf = np.zeros(self.sizes.plan_bytes, np.uint8)
        self._check(self.lib.sci_export_plan(self.h, buf.ctypes.data, buf.size))
        return buf

    def upload(self, device="cuda", stream=None):
        import torch
        self.plan_dev = torch.empty(max(256, self.sizes.plan_bytes), dtype=torch.uint8, device=device)
        self._check(self.lib.sci_upload_plan(self.h, self.plan_dev.data_ptr(), self.plan_dev.numel(),
                                             _stream_ptr(stream)))
        self.ws = torch.empty(max(256, self.sizes.ws_bytes), dtype=torch.uint8, device=device)
        return self

    def apply(self, L_values, lam, q, stream=None):
        self._check(self.lib.sci_apply(self.h, L_values.data_ptr(), lam.data_ptr(), q.data_ptr(),
                                       self.ws.data_ptr(), self.ws.numel(), _stream_ptr(stream)))

    def device_status(self, stream=None) -> int:
        return self.lib.sci_device_status(self.h, self.ws.data_ptr(), _stream_ptr(stream))
