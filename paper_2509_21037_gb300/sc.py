"""Python binding over the C ABI (include/sc.h): argument marshalling only.

PyTorch provides device memory (caller-owned buffers) and streams; every step
of the assembly and of the application runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np

from . import _native, abi


class SCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{abi.STATUS.get(status, status)}: {msg}")
        self.status = status


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Plan:
    """sc_plan + the device buffers it needs (plan tables, workspace).

    ``subdomains`` is a list of :class:`paper_2509_21037_gb300.host.FactoredSubdomain`
    (L pattern, B^T in L's ordering, lambda map).
    """

    def __init__(self, subdomains: Sequence, n_dual: int, precision: int = abi.SC_FP64, n_slices: int = 0,
                 sub_slices: Optional[Sequence[int]] = None, ws_limit: int = 0, persistent: bool = False,
                 tile: int = abi.SC_TILE_32, sub_tile: Optional[Sequence[int]] = None, poll_limit: int = 0):
        self.lib = _native.sc_lib()
        self.nsub = len(subdomains)
        self.n_dual = int(n_dual)
        keep: List[np.ndarray] = []       # arrays must outlive sc_plan
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
            bv = getattr(fs, "bt_val", None)
            if bv is not None:
                bv = np.ascontiguousarray(bv, np.float64)
                keep.append(bv)
                d.Bt_val = bv.ctypes.data if bv.size else None
        h = ctypes.c_void_p()
        opt = abi.Options()
        opt.precision = precision
        opt.n_slices = n_slices
        opt.ws_limit = int(ws_limit)
        opt.persistent = int(bool(persistent))
        opt.tile = int(tile)
        opt.poll_limit = int(poll_limit)
        if sub_slices is not None:
            self._sub_slices = np.ascontiguousarray(np.asarray(sub_slices), dtype=np.int8)
            assert len(self._sub_slices) == self.nsub
            opt.sub_slices = self._sub_slices.ctypes.data
        if sub_tile is not None:
            self._sub_tile = np.ascontiguousarray(np.asarray(sub_tile), dtype=np.int8)
            assert len(self._sub_tile) == self.nsub
            opt.sub_tile = self._sub_tile.ctypes.data
        st = self.lib.sc_plan(ctypes.byref(h), self.nsub, descs, self.n_dual, ctypes.byref(opt))
        self.h = h
        if st != abi.SC_OK:
            msg = self.lib.sc_last_error(h).decode() if h.value else "sc_plan failed"
            if h.value:
                self.lib.sc_destroy(h)
                self.h = ctypes.c_void_p()
            raise SCError(st, msg)
        self.sizes = abi.Sizes()
        self._check(self.lib.sc_get_sizes(self.h, ctypes.byref(self.sizes)))
        self.stats = abi.Stats()
        self._check(self.lib.sc_get_stats(self.h, ctypes.byref(self.stats)))
        self.F_offsets = np.zeros(self.nsub + 1, np.int64)
        self.L_offsets = np.zeros(self.nsub + 1, np.int64)
        self._check(self.lib.sc_get_offsets(self.h, self.F_offsets.ctypes.data, self.L_offsets.ctypes.data))
        self.m = [fs.m for fs in subdomains]
        self.n = [fs.n for fs in subdomains]
        self.plan_dev = None
        self.ws = None

    # -- helpers
    def _check(self, st: int):
        if st != abi.SC_OK:
            raise SCError(st, self.lib.sc_last_error(self.h).decode())

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                self.lib.sc_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass

    # -- device side
    def upload(self, device="cuda", stream=None):
        import torch
        self.plan_dev = torch.empty(max(1, self.sizes.plan_bytes), dtype=torch.uint8, device=device)
        self._check(self.lib.sc_upload_plan(self.h, self.plan_dev.data_ptr(), self.plan_dev.numel(),
                                            _stream_ptr(stream)))
        self.ws = torch.empty(max(256, self.sizes.ws_bytes), dtype=torch.uint8, device=device)
        return self

    def new_F(self, device="cuda"):
        import torch
        return torch.empty(max(1, self.sizes.F_doubles), dtype=torch.float64, device=device)

    def assemble(self, L_values, F, stream=None, ws=None):
        ws = self.ws if ws is None else ws
        self._check(self.lib.sc_assemble_batch(self.h, L_values.data_ptr(), F.data_ptr(), ws.data_ptr(),
                                               ws.numel(), _stream_ptr(stream)))

    def device_status(self, stream=None, ws=None) -> int:
        ws = self.ws if ws is None else ws
        return self.lib.sc_device_status(self.h, ws.data_ptr(), _stream_ptr(stream))

    def apply(self, F, lam, q, stream=None):
        self._check(self.lib.sc_apply(self.h, F.data_ptr(), lam.data_ptr(), q.data_ptr(), _stream_ptr(stream)))

    def apply_fixed(self, F, lam, q, stream=None):
        """q = F * lambda on the integer pipes (include/sc.h, sc_apply_fixed)."""
        self._check(self.lib.sc_apply_fixed(self.h, F.data_ptr(), lam.data_ptr(), q.data_ptr(),
                                            _stream_ptr(stream)))

    def apply_mixed(self, F, lam, q, fp64_quarters: int = 2, stream=None):
        """q = F * lambda with the tiles split between the FP64 pipe and the
        integer pipes (include/sc.h, sc_apply_mixed)."""
        self._check(self.lib.sc_apply_mixed(self.h, F.data_ptr(), lam.data_ptr(), q.data_ptr(), int(fp64_quarters),
                                            _stream_ptr(stream)))

    def digits_size(self) -> int:
        """Bytes of the digit form of F (include/sc.h, sc_apply_digits_size)."""
        import ctypes
        n = ctypes.c_int64(0)
        self._check(self.lib.sc_apply_digits_size(self.h, ctypes.byref(n)))
        return int(n.value)

    def prepare_digits(self, F, Fd=None, stream=None):
        """The digit form of a tile-packed operator F for apply_digits
        (sc_apply_digits_prepare); allocated here when Fd is None."""
        import torch
        if Fd is None:
            Fd = torch.empty(max(16, self.digits_size()), dtype=torch.uint8, device=F.device)
        self._check(self.lib.sc_apply_digits_prepare(self.h, F.data_ptr(), Fd.data_ptr(), _stream_ptr(stream)))
        return Fd

    def apply_digits(self, Fd, lam, q, stream=None):
        """q = F * lambda on the tensor cores from the digit form
        (include/sc.h, sc_apply_digits)."""
        self._check(self.lib.sc_apply_digits(self.h, Fd.data_ptr(), lam.data_ptr(), q.data_ptr(),
                                             _stream_ptr(stream)))

    def digits_status(self, Fd, stream=None) -> int:
        """Status of the apply_digits calls on Fd since the last check
        (sc_apply_digits_status: synchronises the stream, resets the word):
        abi.SC_OK or abi.SC_ERR_TIMEOUT."""
        return self.lib.sc_apply_digits_status(self.h, Fd.data_ptr(), _stream_ptr(stream))

    def export(self, F, i: int, dst=None, stream=None):
        import torch
        m = self.m[i]
        if dst is None:
            dst = torch.empty((m, m), dtype=torch.float64, device=F.device)
        # column-major m x m with ld = m  ==  row-major transposed view
        self._check(self.lib.sc_export_F(self.h, F.data_ptr(), i, dst.data_ptr(), max(1, m), _stream_ptr(stream)))
        return dst.t()

    def pack(self, mats: Sequence, device="cuda"):
        """The inverse of ``export``: dense symmetric m_i x m_i matrices, in
        each subdomain's local multiplier order, tile-packed into a buffer of
        this plan's F layout (lower 32x32 tiles, diagonal tiles full, padding
        zero), so that ``apply`` runs any operator of F's shape, e.g. a
        preconditioner sum_i B_i M_i B_i^T."""
        import torch
        assert len(mats) == self.nsub
        buf = torch.zeros(max(1, self.sizes.F_doubles), dtype=torch.float64, device=device)
        for i, M in enumerate(mats):
            m = self.m[i]
            nt = (m + 31) // 32
            if nt == 0:
                continue
            A = torch.zeros((nt * 32, nt * 32), dtype=torch.float64, device=device)
            A[:m, :m] = torch.as_tensor(np.asarray(M, dtype=np.float64), device=device)
            # tiles[I, J, c, r] = A[32 I + r, 32 J + c]; tile (I, J) is number I (I + 1) / 2 + J
            T = A.reshape(nt, 32, nt, 32).permute(0, 2, 3, 1)
            I, J = torch.tril_indices(nt, nt, device=device)
            tiles = T[I, J].reshape(-1)
            off = int(self.F_offsets[i])
            assert int(self.F_offsets[i + 1]) - off == tiles.numel()
            buf[off:off + tiles.numel()] = tiles
        return buf

    def add_symmetric(self, F, i: int, rows, cols, vals):
        """F_i[r, c] += v and F_i[c, r] += v (once for r == c) for entries
        with r >= c, in place in the tile-packed layout (the lower tile holds
        an off-diagonal-tile pair once; a diagonal tile stores both entries)."""
        self.add_symmetric_batch(F, [(i, rows, cols, vals)])

    def add_symmetric_batch(self, F, entries):
        """``add_symmetric`` for several subdomains at once: entries is a
        sequence of (i, rows, cols, vals); one scatter-add on F's device."""
        import torch
        off, val = [], []
        for i, rows, cols, vals in entries:
            r = np.asarray(rows, np.int64)
            c = np.asarray(cols, np.int64)
            v = np.asarray(vals, np.float64)
            assert np.all(r >= c) and len(r) == len(c) == len(v)
            assert np.all(r < self.m[i]) and np.all(c >= 0)
            I, J = r // 32, c // 32
            base = int(self.F_offsets[i]) + (I * (I + 1) // 2 + J) * 1024
            off.append(base + r % 32 + 32 * (c % 32))
            val.append(v)
            mirror = (I == J) & (r != c)             # a diagonal tile holds the mirror entry too
            off.append(base[mirror] + c[mirror] % 32 + 32 * (r[mirror] % 32))
            val.append(v[mirror])
        if not off or sum(len(o) for o in off) == 0:
            return
        idx = torch.from_numpy(np.concatenate(off)).to(F.device)
        F.index_add_(0, idx, torch.from_numpy(np.concatenate(val)).to(F.device))

    def enable_stage_timing(self, on: bool = True):
        self._check(self.lib.sc_enable_stage_timing(self.h, int(on)))

    def stage_times(self):
        """Elapsed ms of the last timed assembly: (prep, trsm, syrk)."""
        ms = (ctypes.c_float * 3)()
        self._check(self.lib.sc_stage_times(self.h, ms, 3))
        return tuple(float(x) for x in ms)

    def stats_dict(self) -> dict:
        return {k: getattr(self.stats, k) for k, _ in abi.Stats._fields_}


def concat_L_values(subdomains) -> np.ndarray:
    return np.concatenate([fs.L.values for fs in subdomains]) if subdomains else np.zeros(0)
