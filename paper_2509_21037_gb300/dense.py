"""Dense comparator: the paper's original GPU assembly (Sec. 3.1) through cuBLAS.

Per subdomain: dense L (n x n), dense B^T (n x m); DTRSM Y = L^{-1} B^T over the
full right-hand side, then DSYRK F = Y^T Y.  No sparsity is used.  The dense
operands are built once with torch (setup, not part of the timed region).
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence

import numpy as np

from . import _native


class DenseRunner:
    def __init__(self, fs: Sequence, device, emulation: int = 0, nstreams: int = 4):
        import torch
        self.lib = _native.dense_lib()
        self.h = ctypes.c_void_p()
        rc = self.lib.scd_create(ctypes.byref(self.h), int(emulation))
        if rc != 0:
            raise RuntimeError(f"scd_create failed ({rc})")
        self.dev = device
        self.L, self.Bt0, self.Y, self.F = [], [], [], []
        for f in fs:
            n, m = f.n, f.m
            cols = np.repeat(np.arange(n), np.diff(f.L.colptr))
            Lt = torch.zeros((n, n), dtype=torch.float64, device=device)       # Lt[c, r] = L[r, c]
            Lt[torch.from_numpy(cols).to(device), torch.from_numpy(f.L.rowind.astype(np.int64)).to(device)] = \
                torch.from_numpy(f.L.values).to(device)
            bcols = np.repeat(np.arange(m), np.diff(f.bt_colptr))
            Bt = torch.zeros((m, n), dtype=torch.float64, device=device)       # Bt[j, r] = B^T[r, j]
            Bt[torch.from_numpy(bcols).to(device), torch.from_numpy(f.bt_rowind.astype(np.int64)).to(device)] = \
                torch.from_numpy(f.bt_sign.astype(np.float64)).to(device)
            self.L.append(Lt)
            self.Bt0.append(Bt)
            self.Y.append(torch.empty_like(Bt))
            self.F.append(torch.zeros((m, m), dtype=torch.float64, device=device))
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max(1, nstreams))]

    def run(self) -> None:
        """TRSM + SYRK for every subdomain, round-robin over the streams; the
        caller's current stream waits for all of them."""
        import torch
        cur = torch.cuda.current_stream(self.dev)
        for s in self.streams:
            s.wait_stream(cur)
        for i in range(len(self.L)):
            s = self.streams[i % len(self.streams)]
            with torch.cuda.stream(s):
                self.Y[i].copy_(self.Bt0[i])
                n, m = self.L[i].shape[0], self.Bt0[i].shape[0]
                rc = self.lib.scd_trsm_syrk(self.h, n, m, self.L[i].data_ptr(), self.Y[i].data_ptr(),
                                            self.F[i].data_ptr(), s.cuda_stream)
                if rc != 0:
                    raise RuntimeError(f"scd_trsm_syrk failed ({rc})")
        for s in self.streams:
            cur.wait_stream(s)

    def full_F(self, i: int) -> np.ndarray:
        Fcm = self.F[i].t().cpu().numpy()     # column-major buffer viewed as [row, col]
        low = np.tril(Fcm)
        return low + np.tril(Fcm, -1).T

    def __del__(self):
        try:
            if self.h.value:
                self.lib.scd_destroy(self.h)
                self.h = ctypes.c_void_p()
        except Exception:
            pass


def assemble_dense(fs: Sequence, device, emulation: int = 0) -> List[np.ndarray]:
    import torch
    r = DenseRunner(fs, device, emulation, nstreams=1)
    r.run()
    torch.cuda.synchronize(device)
    return [r.full_F(i) for i in range(len(fs))]
