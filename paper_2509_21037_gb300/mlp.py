"""Binding of the variant-predicting MLP (include/sc_mlp.h): argument
marshalling only; every forward, backward and optimiser step runs in the
library's CUDA kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native


class Shape(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("n_out", ctypes.c_int32)]


def _lib():
    lib = _native.sc_lib()
    if not getattr(lib, "_mlp_typed", False):
        P = ctypes.POINTER(Shape)
        vp = ctypes.c_void_p
        lib.sc_mlp_param_count.argtypes = [P]
        lib.sc_mlp_param_count.restype = ctypes.c_int64
        lib.sc_mlp_workspace_floats.argtypes = [P, ctypes.c_int32]
        lib.sc_mlp_workspace_floats.restype = ctypes.c_int64
        lib.sc_mlp_forward.argtypes = [P, vp, vp, ctypes.c_int32, vp, vp, vp]
        lib.sc_mlp_forward.restype = ctypes.c_int
        lib.sc_mlp_loss_grad.argtypes = [P, vp, vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp]
        lib.sc_mlp_loss_grad.restype = ctypes.c_int
        lib.sc_mlp_adam.argtypes = [ctypes.c_int64, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_int32, vp]
        lib.sc_mlp_adam.restype = ctypes.c_int
        lib._mlp_typed = True
    return lib


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc})")


class MLP:
    """3-layer ReLU MLP on the GPU; params/grads/Adam moments are torch tensors."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, device="cuda", seed: int = 0):
        import torch
        self.lib = _lib()
        self.shape = Shape(n_in, n_hidden, n_out)
        self.dims = (n_in, n_hidden, n_out)
        n = self.lib.sc_mlp_param_count(ctypes.byref(self.shape))
        rng = np.random.default_rng(seed)
        p = np.zeros(n, np.float32)
        o = 0
        for fan_in, fan_out in [(n_in, n_hidden), (n_hidden, n_hidden), (n_hidden, n_out)]:
            k = fan_in * fan_out
            p[o:o + k] = rng.standard_normal(k) * np.sqrt(2.0 / fan_in)    # He initialisation
            o += k + fan_out
        self.device = device
        self.params = torch.from_numpy(p).to(device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.mu = np.zeros(n_in, np.float32)
        self.sd = np.ones(n_in, np.float32)

    def _ws(self, batch):
        import torch
        return torch.empty(max(1, self.lib.sc_mlp_workspace_floats(ctypes.byref(self.shape), batch)),
                           dtype=torch.float32, device=self.device)

    def forward(self, X):
        """X: torch float32 [B, n_in] on the device -> [B, n_out]."""
        import torch
        B = X.shape[0]
        Y = torch.empty((B, self.dims[2]), dtype=torch.float32, device=self.device)
        _check(self.lib.sc_mlp_forward(ctypes.byref(self.shape), self.params.data_ptr(), X.data_ptr(), B,
                                       Y.data_ptr(), self._ws(B).data_ptr(), None), "sc_mlp_forward")
        return Y

    def loss_grad(self, X, T, mask):
        import torch
        B = X.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        _check(self.lib.sc_mlp_loss_grad(ctypes.byref(self.shape), self.params.data_ptr(), X.data_ptr(),
                                         T.data_ptr(), mask.data_ptr(), B, self.grads.data_ptr(), loss.data_ptr(),
                                         self._ws(B).data_ptr(), None), "sc_mlp_loss_grad")
        return loss

    def adam(self, lr=3e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        _check(self.lib.sc_mlp_adam(self.params.numel(), self.params.data_ptr(), self.grads.data_ptr(),
                                    self.m.data_ptr(), self.v.data_ptr(), lr, b1, b2, eps, self.step, None),
               "sc_mlp_adam")

    # ---- training on normalised features
    def fit(self, X: np.ndarray, T: np.ndarray, mask: np.ndarray, epochs: int = 2000, lr: float = 3e-3):
        import torch
        self.mu = X.mean(0).astype(np.float32)
        self.sd = (X.std(0) + 1e-6).astype(np.float32)
        Xd = torch.from_numpy(((X - self.mu) / self.sd).astype(np.float32)).to(self.device)
        Td = torch.from_numpy(T.astype(np.float32)).to(self.device)
        Md = torch.from_numpy(mask.astype(np.float32)).to(self.device)
        hist = []
        for e in range(epochs):
            loss = self.loss_grad(Xd, Td, Md)
            self.adam(lr=lr)
            if e % 100 == 0 or e == epochs - 1:
                hist.append(float(loss.item()))
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        import torch
        Xd = torch.from_numpy(((X - self.mu) / self.sd).astype(np.float32)).to(self.device)
        return self.forward(Xd).cpu().numpy()
