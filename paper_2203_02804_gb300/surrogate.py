"""Learned surrogate of the tensor-train pricer for the d=5 call on the minimum.

An ensemble of small multilayer perceptrons maps the option's parameters to the
log-price the TT pricer computes, trained on prices that pricer generates.  A
quote whose ensemble members disagree by more than `tol` (in log-price, i.e.
relative price) goes back to the TT pricer, which thereby also judges the
surrogate.  The paper has no learned component (it names a better starting
point for TT-cross at high dimension as open, Section VI).

Network: 15 -> 256 -> 256 -> 256 -> 256 -> 1, SiLU on the hidden layers,
FP32 master weights trained by the library's kernels (include/ttmlp.h:
tiled GEMMs, fused activation, Adam); bfloat16 copies of the weights for
inference, whose 256-wide layers run on the tensor cores (tcgen05.mma
kind::f16, bfloat16 activations, FP32 accumulation in tensor memory).

Features (15): S0_j / K (5), sigma_j = sqrt(Cov_jj) (5), the mean off-diagonal
correlation, K / 100, T, r, and the mean damping -alpha.  Targets are
log(price / K); both are standardised with the training set's mean and
standard deviation.  PyTorch only holds device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import ttprice

SIZES = (15, 256, 256, 256, 256, 1)
LINEAR, SILU = 0, 1
_F, _I, _P, _LL = ctypes.c_float, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong


def _bind(lib):
    if getattr(lib, "_mlp_bound", False):
        return lib
    lib.tt_mlp_forward.argtypes = [_P, _I, _I, _P, _P, _I, _I, _P, _P, _P]
    lib.tt_mlp_forward_bf16.argtypes = [_P, _I, _I, _P, _P, _I, _I, _P, _P, _P]
    lib.tt_mlp_backward.argtypes = [_P, _P, _P, _I, _I, _P, _I, _I, _P, _P, _P, _P]
    lib.tt_mlp_mse.argtypes = [_P, _P, _I, _P, _P, _P]
    lib.tt_mlp_adam.argtypes = [_P, _P, _P, _P, _LL, _F, _F, _F, _F, _I, _P]
    lib.tt_mlp_to_bf16.argtypes = [_P, _P, _LL, _P]
    lib.tt_mlp_ensemble.argtypes = [_P, _I, _I, _P, _P, _P]
    lib.tt_mlp_gather.argtypes = [_P, _P, _I, _I, _P, _P]
    lib.tt_mlp_forward_tc.argtypes = [_P, _I, _I, _P, _P, _I, _I, _P, _P, _P]
    for f in ("forward", "forward_bf16", "forward_tc", "backward", "mse", "adam", "to_bf16", "ensemble", "gather"):
        getattr(lib, "tt_mlp_" + f).restype = ctypes.c_int
    lib._mlp_bound = True
    return lib


def _ptr(t) -> int:
    return t.data_ptr() if t is not None else 0


def _ok(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc})")


def features(problems: Sequence) -> np.ndarray:
    """Raw (unstandardised) features of d=5 calls on the minimum, float64 [n, 15]."""
    out = np.empty((len(problems), 15))
    for i, p in enumerate(problems):
        sig = np.sqrt(np.diag(p.cov))
        corr = p.cov / np.outer(sig, sig)
        d = len(sig)
        rho = (corr.sum() - d) / (d * (d - 1))
        out[i, :5] = np.asarray(p.spot) / p.strike
        out[i, 5:10] = sig
        out[i, 10:] = [rho, p.strike / 100.0, p.maturity, p.rate, -float(np.mean(p.damping))]
    return out


class Net:
    """One network: FP32 master weights and Adam moments on the device."""

    def __init__(self, seed: int, sizes=SIZES, device: int = 0):
        import torch

        self.torch, self.device, self.sizes = torch, device, tuple(sizes)
        self.lib = _bind(ttprice.load_library())
        self.stream = torch.cuda.current_stream(device)
        rng = np.random.default_rng(seed)
        dev = f"cuda:{device}"
        # He initialisation, biases zero
        self.w = [torch.tensor(rng.standard_normal((o, i)) * np.sqrt(2.0 / i), dtype=torch.float32, device=dev)
                  for i, o in zip(sizes[:-1], sizes[1:])]
        self.b = [torch.zeros(o, dtype=torch.float32, device=dev) for o in sizes[1:]]
        self.params = [t for pair in zip(self.w, self.b) for t in pair]
        self.grads = [torch.zeros_like(t) for t in self.params]
        self.m = [torch.zeros_like(t) for t in self.params]
        self.v = [torch.zeros_like(t) for t in self.params]
        self.w16 = None
        self.step_no = 0
        self._bufs = {}

    def _buffers(self, batch: int):
        if batch not in self._bufs:
            t, dev = self.torch, f"cuda:{self.device}"
            z = [t.empty((batch, o), dtype=t.float32, device=dev) for o in self.sizes[1:]]
            a = [t.empty((batch, o), dtype=t.float32, device=dev) for o in self.sizes[1:]]
            g = [t.empty((batch, o), dtype=t.float32, device=dev) for o in self.sizes[1:]]
            self._bufs[batch] = (z, a, g)
        return self._bufs[batch]

    def forward(self, x, bf16: bool = False):
        """x: device float32 [batch, 15] (contiguous); returns the output buffer [batch, 1]."""
        batch = x.shape[0]
        z, a, _ = self._buffers(batch)
        s = self.stream.cuda_stream
        inp = x
        last = len(self.w) - 1
        for l in range(len(self.w)):
            act = LINEAR if l == last else SILU
            i, o = self.sizes[l], self.sizes[l + 1]
            if bf16:
                rc = self.lib.tt_mlp_forward_bf16(_ptr(inp), batch, i, _ptr(self.w16[l]), _ptr(self.b[l]), o, act,
                                                  _ptr(z[l]), _ptr(a[l]), s)
            else:
                rc = self.lib.tt_mlp_forward(_ptr(inp), batch, i, _ptr(self.w[l]), _ptr(self.b[l]), o, act,
                                             _ptr(z[l]), _ptr(a[l]), s)
            _ok(rc, "tt_mlp_forward")
            inp = a[l]
        return a[last]

    def backward(self, x, dy):
        """Gradients of the loss into self.grads, given dL/d(output) in dy [batch, 1] (overwritten)."""
        batch = x.shape[0]
        z, a, g = self._buffers(batch)
        s = self.stream.cuda_stream
        da = dy
        for l in range(len(self.w) - 1, -1, -1):
            act = LINEAR if l == len(self.w) - 1 else SILU
            i, o = self.sizes[l], self.sizes[l + 1]
            inp = x if l == 0 else a[l - 1]
            dx = g[l - 1] if l > 0 else None
            rc = self.lib.tt_mlp_backward(_ptr(inp), _ptr(z[l]), _ptr(da), batch, i, _ptr(self.w[l]), o, act,
                                          _ptr(dx), _ptr(self.grads[2 * l]), _ptr(self.grads[2 * l + 1]), s)
            _ok(rc, "tt_mlp_backward")
            da = dx

    def adam(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_no += 1
        s = self.stream.cuda_stream
        for p, gr, m, v in zip(self.params, self.grads, self.m, self.v):
            _ok(self.lib.tt_mlp_adam(_ptr(p), _ptr(gr), _ptr(m), _ptr(v), p.numel(), lr, beta1, beta2, eps,
                                     self.step_no, s), "tt_mlp_adam")

    def to_bf16(self):
        t = self.torch
        self.w16 = [t.empty(w.shape, dtype=t.int16, device=w.device) for w in self.w]
        for w, w16 in zip(self.w, self.w16):
            _ok(self.lib.tt_mlp_to_bf16(_ptr(w), _ptr(w16), w.numel(), self.stream.cuda_stream), "tt_mlp_to_bf16")
        # tensor-core copies: inputs padded with zero columns to a multiple of 16
        self.w16tc = []
        for w in self.w:
            o, i = w.shape
            ip = -(-i // 16) * 16
            wp = t.zeros((o, ip), dtype=t.float32, device=w.device)
            wp[:, :i] = w
            w16 = t.empty((o, ip), dtype=t.int16, device=w.device)
            _ok(self.lib.tt_mlp_to_bf16(_ptr(wp), _ptr(w16), wp.numel(), self.stream.cuda_stream), "tt_mlp_to_bf16")
            self.w16tc.append(w16)

    def tc_layers(self) -> int:
        """Leading layers that run on the tensor cores (outputs a multiple of 16, <= 256)."""
        n = 0
        for o in self.sizes[1:]:
            if o % 16 or o > 256 or self.sizes[n] > 256:
                break
            n += 1
        return n

    def forward_tc(self, x16):
        """x16: device bfloat16 (int16 storage) [batch, in padded to 16]; the leading
        layers on the tensor cores (bfloat16 activations, FP32 accumulation), the rest
        on the bfloat16-weight path; returns the output buffer [batch, 1]."""
        t = self.torch
        batch = x16.shape[0]
        z, a, _ = self._buffers(batch)
        s = self.stream.cuda_stream
        ntc = self.tc_layers()
        key = ("tc", batch)
        if key not in self._bufs:
            self._bufs[key] = [t.empty((batch, o), dtype=t.int16, device=x16.device) for o in self.sizes[1:]]
        h16 = self._bufs[key]
        inp = x16
        last = len(self.w) - 1
        for l in range(ntc):
            act = LINEAR if l == last else SILU
            i, o = self.w16tc[l].shape[1], self.sizes[l + 1]
            fp32_out = l == ntc - 1  # the next layer reads FP32
            _ok(self.lib.tt_mlp_forward_tc(_ptr(inp), batch, i, _ptr(self.w16tc[l]), _ptr(self.b[l]), o, act,
                                           _ptr(a[l]) if fp32_out else 0, 0 if fp32_out else _ptr(h16[l]), s),
                "tt_mlp_forward_tc")
            inp = h16[l]
        out = a[ntc - 1] if ntc else None
        for l in range(ntc, len(self.w)):
            act = LINEAR if l == last else SILU
            i, o = self.sizes[l], self.sizes[l + 1]
            _ok(self.lib.tt_mlp_forward_bf16(_ptr(out), batch, i, _ptr(self.w16[l]), _ptr(self.b[l]), o, act,
                                             _ptr(z[l]), _ptr(a[l]), s), "tt_mlp_forward_bf16")
            out = a[l]
        return out


def train(net: Net, x, y, epochs: int, batch: int, lr: float, seed: int,
          lr_final: Optional[float] = None) -> List[float]:
    """Minibatch Adam on device data x [n, 15], y [n, 1] (standardised); the learning
    rate decays geometrically to lr_final.  Returns the mean loss of each epoch."""
    torch = net.torch
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    xb = torch.empty((batch, x.shape[1]), dtype=torch.float32, device=x.device)
    yb = torch.empty((batch, 1), dtype=torch.float32, device=x.device)
    dy = torch.empty((batch, 1), dtype=torch.float32, device=x.device)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    losses = []
    steps = epochs * (n // batch)
    decay = (lr_final / lr) ** (1.0 / max(1, steps)) if lr_final else 1.0
    s = net.stream.cuda_stream
    cur = lr
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(x.device)
        tot = torch.zeros(1, dtype=torch.float32, device=x.device)
        for k in range(n // batch):
            idx = perm[k * batch:(k + 1) * batch]
            _ok(net.lib.tt_mlp_gather(_ptr(x), _ptr(idx), batch, x.shape[1], _ptr(xb), s), "gather x")
            _ok(net.lib.tt_mlp_gather(_ptr(y), _ptr(idx), batch, 1, _ptr(yb), s), "gather y")
            out = net.forward(xb)
            _ok(net.lib.tt_mlp_mse(_ptr(out), _ptr(yb), batch, _ptr(dy), _ptr(loss), s), "mse")
            tot += loss
            net.backward(xb, dy)
            net.adam(cur)
            cur *= decay
        losses.append(float(tot.item()) / max(1, n // batch))
    return losses


class Surrogate:
    """Ensemble of `members` networks with TT fallback."""

    def __init__(self, members: int = 4, seed: int = 0, device: int = 0, sizes=SIZES):
        self.nets = [Net(seed + 7919 * k, sizes, device) for k in range(members)]
        self.device = device
        self.fx = self.fy = None

    def fit(self, problems: Sequence, prices: np.ndarray, epochs: int = 20, batch: int = 1024,
            lr: float = 2e-3, lr_final: float = 2e-5) -> List[List[float]]:
        import torch

        f = features(problems)
        y = np.log(np.asarray(prices) / np.array([p.strike for p in problems]))[:, None]
        self.fx = (f.mean(0), f.std(0) + 1e-12)
        self.fy = (float(y.mean()), float(y.std()) + 1e-12)
        dev = f"cuda:{self.device}"
        x = torch.tensor((f - self.fx[0]) / self.fx[1], dtype=torch.float32, device=dev).contiguous()
        t = torch.tensor((y - self.fy[0]) / self.fy[1], dtype=torch.float32, device=dev).contiguous()
        hist = []
        for k, net in enumerate(self.nets):
            hist.append(train(net, x, t, epochs, batch, lr, seed=1000 + k, lr_final=lr_final))
            net.to_bf16()
        return hist

    def standardise(self, problems: Sequence):
        """Device float32 [n, 15] standardised features."""
        import torch

        f = features(problems)
        return torch.tensor((f - self.fx[0]) / self.fx[1], dtype=torch.float32,
                            device=f"cuda:{self.device}").contiguous()

    def standardise_tc(self, problems: Sequence):
        """Device bfloat16 (int16 storage) [n, 16] standardised features, zero-padded."""
        import torch

        f = (features(problems) - self.fx[0]) / self.fx[1]
        fp = np.zeros((f.shape[0], 16), dtype=np.float32)
        fp[:, :f.shape[1]] = f
        src = torch.tensor(fp, device=f"cuda:{self.device}")
        dst = torch.empty(src.shape, dtype=torch.int16, device=src.device)
        net0 = self.nets[0]
        _ok(net0.lib.tt_mlp_to_bf16(_ptr(src), _ptr(dst), src.numel(), net0.stream.cuda_stream), "to_bf16")
        return dst

    def predict_device(self, x):
        """Ensemble members on device features: bfloat16 [n, 16] (tensor-core layers, from
        standardise_tc) or float32 [n, 15] (bfloat16 weights, FP32 activations); returns
        device (mean, spread) of the standardised log-price."""
        import torch

        n = x.shape[0]
        tc = x.dtype == torch.int16
        preds = torch.empty((len(self.nets), n), dtype=torch.float32, device=x.device)
        for k, net in enumerate(self.nets):
            preds[k].copy_((net.forward_tc(x) if tc else net.forward(x, bf16=True))[:, 0])
        mean = torch.empty(n, dtype=torch.float32, device=x.device)
        spread = torch.empty(n, dtype=torch.float32, device=x.device)
        net0 = self.nets[0]
        _ok(net0.lib.tt_mlp_ensemble(_ptr(preds), len(self.nets), n, _ptr(mean), _ptr(spread),
                                     net0.stream.cuda_stream), "ensemble")
        return mean, spread

    def predict_log(self, problems: Sequence) -> Tuple[np.ndarray, np.ndarray]:
        """(mean, spread) over the members of log(price / K), via the tensor-core layers."""
        mean, spread = self.predict_device(self.standardise_tc(problems))
        mu, sd = self.fy
        return mean.cpu().numpy().astype(np.float64) * sd + mu, spread.cpu().numpy().astype(np.float64) * sd

    def quote(self, problems: Sequence, pricer=None, tol: float = 1e-4, memory=None):
        """Prices from the ensemble mean; quotes whose members spread by more than
        `tol` in log-price are priced by `pricer` (a ttprice.Pricer) instead, warm
        started from `memory` (a PivotMemory) when given.
        Returns (prices, mask of the quotes the TT pricer gave, spread)."""
        mean, spread = self.predict_log(problems)
        k = np.array([p.strike for p in problems])
        prices = k * np.exp(mean)
        back = spread > tol
        if pricer is not None and back.any():
            idx = np.flatnonzero(back)
            todo = [problems[i] for i in idx]
            if memory is not None:
                todo = memory.warm(todo)
            _, tt, _ = pricer.evaluate(todo)
            prices[idx] = tt
        return prices, back, spread


class PivotMemory:
    """Warm starts for the TT fallback from the surrogate's training data.

    TT-cross starts from random column sets (Section IV.B); the pivots it
    converges to move little with the option's parameters.  The TT solves that
    produced the surrogate's training prices also leave their final right index
    sets (tt_price_pivots); a quote sent back to TT is warm started from the
    pivots of the nearest training problem in the surrogate's standardised
    feature space (the inputs its networks see).  The pivots are a set of grid
    multi-indices per bond, not a quantity a regression output fits, so the
    learned part here is the feature space and the memory, not a network head."""

    def __init__(self, problems: Sequence, records: Sequence[np.ndarray], fx):
        f = features(problems)
        self.fx = fx
        self.z = (f - fx[0]) / fx[1]
        self.records = list(records)
        self.shape = [(p.d, p.n_grid, p.payoff) for p in problems]

    def nearest(self, problems: Sequence) -> np.ndarray:
        q = (features(problems) - self.fx[0]) / self.fx[1]
        d2 = (q * q).sum(1)[:, None] - 2.0 * q @ self.z.T + (self.z * self.z).sum(1)[None, :]
        return np.argmin(d2, axis=1)

    def warm(self, problems: Sequence) -> List:
        """The problems with warm_sets from their nearest neighbour of the same shape
        (d, N, payoff); a problem of another shape is left cold."""
        out = []
        for p, j in zip(problems, self.nearest(problems)):
            same = self.shape[j] == (p.d, p.n_grid, p.payoff)
            out.append(p.with_(warm_sets=self.records[j]) if same else p)
        return out
