"""Learned WENO-weight surrogate: parameter storage, training loop and
training-set assembly over the C ABI of ``include/wenoc.h`` (the
``wc_mlp_*`` entry points).

Every arithmetic step -- feature extraction, plain-weight targets, forward,
backward and Adam -- runs in the library's CUDA kernels (tensor cores for
the network).  This module allocates device tensors, draws the batch indices
and loops.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import wenoc
from .wenoc import WcError, _dptr, _stream, lib

IN, NW = 32, 9


def nparam():
    return lib().wc_mlp_nparam()


def param_bytes():
    return lib().wc_mlp_param_bytes()


def _check(st, what):
    if st != 0:
        raise WcError(st, what)


class Surrogate:
    """FP32 masters + Adam moments + the BF16/FP32 parameter block used by
    the kernels, on one CUDA device."""

    def __init__(self, seed=0, device="cuda", master=None):
        n = nparam()
        if master is None:
            host = np.zeros(n, dtype=np.float32)
            _check(lib().wc_mlp_init_master(host.ctypes.data_as(ctypes.c_void_p), int(seed)),
                   "init")
            master = torch.from_numpy(host)
        self.master = torch.as_tensor(master, dtype=torch.float32).to(device).contiguous()
        self.params = torch.zeros(param_bytes(), dtype=torch.uint8, device=device)
        self.grads = torch.zeros(n, dtype=torch.float32, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.step = 0
        self.pack()

    def pack(self, stream=None):
        _check(lib().wc_mlp_pack(_dptr(self.master), _dptr(self.params), _stream(stream)),
               "pack")

    def forward(self, X, Y=None, stream=None):
        n = X.shape[0]
        Y = torch.empty((n, NW), dtype=torch.float32, device=X.device) if Y is None else Y
        _check(lib().wc_mlp_forward(_dptr(X), n, _dptr(self.params), _dptr(Y),
                                    _dptr(self.status), _stream(stream)), "forward")
        return Y

    def gradients(self, X, T, idx, stream=None):
        """Loss and gradients of one batch (grads are accumulated; cleared first)."""
        self.grads.zero_()
        self.loss.zero_()
        _check(lib().wc_mlp_gradients(_dptr(X), _dptr(T), _dptr(idx), idx.numel(),
                                      _dptr(self.params), _dptr(self.grads), _dptr(self.loss),
                                      _dptr(self.status), _stream(stream)), "gradients")
        return self.loss, self.grads

    def train_step(self, X, T, idx, lr, stream=None):
        self.step += 1
        _check(lib().wc_mlp_train_step(_dptr(X), _dptr(T), _dptr(idx), idx.numel(),
                                       _dptr(self.params), _dptr(self.master),
                                       _dptr(self.grads), _dptr(self.m), _dptr(self.v),
                                       float(lr), self.step, _dptr(self.loss),
                                       _dptr(self.status), _stream(stream)), "train_step")

    def check_status(self):
        s = int(self.status.item())
        if s:
            raise WcError(7, f"surrogate kernel status {s}")

    def train(self, ts, steps, batch=8192, lr=2e-3, lr_final=2e-4, seed=0, interesting=0.5,
              log_every=0):
        """Adam over ``steps`` batches of ``ts`` (a TrainingSet): a fraction
        ``interesting`` of every batch comes from the rows whose plain weights
        are not the ideal ones, the rest uniformly from all rows.  Cosine
        learning-rate decay from lr to lr_final.  Returns the per-step losses
        (FP32 mean squared weight error of each batch, before its update)."""
        rng = np.random.default_rng(seed)
        ni = int(batch * interesting) if ts.n_interesting > 0 else 0
        losses = torch.zeros(steps, dtype=torch.float32, device=self.master.device)
        idx_all = np.empty((steps, batch), dtype=np.int32)
        if ni:
            idx_all[:, :ni] = ts.interesting_rows[rng.integers(0, ts.n_interesting,
                                                               (steps, ni))]
        idx_all[:, ni:] = rng.integers(0, ts.nrows, (steps, batch - ni))
        idx_dev = torch.from_numpy(idx_all).to(self.master.device)
        for k in range(steps):
            lr_k = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * k / max(steps, 1)))
            self.loss.zero_()
            self.train_step(ts.X, ts.T, idx_dev[k], lr_k)
            losses[k] = self.loss[0]
            if log_every and (k % log_every == 0 or k == steps - 1):
                print(f"  step {k:6d}  lr {lr_k:.2e}  loss {losses[k].item():.3e}")
        torch.cuda.synchronize()
        self.check_status()
        return losses.cpu().numpy()


class TrainingSet:
    """Feature rows and plain-weight targets of every face side of given
    states, in device memory (X BF16 [rows][32], T FP32 [rows][9])."""

    def __init__(self, capacity, device="cuda"):
        self.cap = int(capacity)
        self.X = torch.zeros((self.cap, IN), dtype=torch.bfloat16, device=device)
        self.T = torch.zeros((self.cap, NW), dtype=torch.float32, device=device)
        self.lst = torch.zeros(self.cap, dtype=torch.int64, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.nrows = 0

    def add(self, grid: "wenoc.Grid", U, directions=None):
        """Appends the rows of every direction of state U (FP64 [NV][...])."""
        dirs = range(grid.desc.dim) if directions is None else directions
        for d in dirs:
            rows = 2 * grid.ncell
            if self.nrows + rows > self.cap:
                raise ValueError("training set full")
            grid.mlp_features(U, d, self.X, self.T, self.nrows, self.lst, self.count)
            self.nrows += rows

    def finish(self):
        torch.cuda.synchronize()
        n = min(int(self.count.item()), self.cap)
        self.interesting_rows = self.lst[:n].cpu().numpy().astype(np.int64)
        self.n_interesting = n
        return self
