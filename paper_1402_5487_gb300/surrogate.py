"""Learned surrogate of K lattice steps (binding of the plbm_sur_* calls).

Workflow (every numerical step runs in libplbm's kernels; this module marshals
arguments and keeps the bookkeeping):

1. ``generate`` runs Kelvin-Helmholtz trajectories on the batched solver
   (D2Q25 {0,+-1,+-3}^2, theta0 = 1, omega = 1.3, periodic L x L; per seed a
   layer width delta in {L/80, L/64, L/40} and amplitude u0 in [0.06, 0.1];
   snapshots every K steps after a burn-in) and packs the moments of every
   snapshot into an FP32 NHWC stack on the device.
2. ``fit_norm`` takes per-field means and standard deviations of the inputs
   and of the K-step changes from the stack (host statistics of a sample).
3. ``Surrogate.train`` runs Adam steps on minibatches assembled on the device.
4. ``Surrogate.advance`` moves lattices forward by K steps with
   reconstruction and LBM fallback (plbm_sur_advance).
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import inputs as I
from . import plbm
from .batch import Batch

V5 = I.SET_013
THETA0 = 1.0
OMEGA = 1.3
DELTAS = (80.0, 64.0, 40.0)


def trajectory_instance(seed: int, L: int = 256):
    """Seeded KH variant: delta = L / {80, 64, 40}, u0 in [0.06, 0.1]."""
    rng = np.random.default_rng(50_000 + seed)
    div = DELTAS[int(rng.integers(0, len(DELTAS)))]
    u0 = float(rng.uniform(0.06, 0.1))
    return I.Instance(index=seed, L=L, v=V5, omega=OMEGA, theta0=THETA0, kind="kh", seed=seed), L / div, u0


def trajectory_fields(seed: int, L: int = 256):
    inst, delta, u0 = trajectory_instance(seed, L)
    return I.kh_fields(L, theta0=THETA0, seed=seed, u0=u0, delta=delta)


def generate(seeds, L=256, K=32, snaps=9, burn=64, chunk=250, torch=None):
    """FP32 NHWC snapshot stack [len(seeds) * snaps][L*L][4] (torch CUDA tensor)."""
    import torch as _torch
    torch = torch or _torch
    seeds = list(seeds)
    npix = L * L
    stack = torch.empty((len(seeds) * snaps, npix, 4), dtype=torch.float32, device="cuda")
    planes = torch.empty((4, npix), dtype=torch.float64, device="cuda")
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0:c0 + chunk]
        insts = [trajectory_instance(s, L)[0] for s in part]
        b = Batch(insts, prec="f32")
        for s, sol in zip(part, b.solvers):
            sol.init(*trajectory_fields(s, L))
        b.step(burn, "persistent_graph")
        for k in range(snaps):
            if k:
                b.step(K, "persistent_graph")
            for j, sol in enumerate(b.solvers):
                st = plbm.lib().plbm_moments(sol.h, *[planes[i].data_ptr() for i in range(4)], 1)
                if st != plbm.PLBM_OK:
                    raise plbm.PlbmError(st, plbm.last_error(sol.h))
                dst = stack[(c0 + j) * snaps + k]
                st = plbm.lib().plbm_sur_pack_fields(*[planes[i].data_ptr() for i in range(4)], npix,
                                                     dst.data_ptr(), b.stream.cuda_stream)
                if st != plbm.PLBM_OK:
                    raise plbm.PlbmError(st, "pack")
        b.stream.synchronize()
        st, bad = b.check()
        b.close()
        if st != plbm.PLBM_OK:
            raise RuntimeError("trajectory %d diverged" % bad)
    torch.cuda.synchronize()
    return stack


def pairs_of(ntraj, snaps):
    """(s0, s1) snapshot indices of consecutive snapshots of every trajectory."""
    return np.array([(t * snaps + k, t * snaps + k + 1) for t in range(ntraj) for k in range(snaps - 1)],
                    dtype=np.int32)


def fit_norm(stack, pairs, sample=512, seed=0):
    rng = np.random.default_rng(seed)
    sel = rng.choice(len(pairs), size=min(sample, len(pairs)), replace=False)
    a = stack[pairs[sel, 0]].cpu().numpy().astype(np.float64)
    b = stack[pairs[sel, 1]].cpu().numpy().astype(np.float64)
    d = b - a
    mean_in = a.reshape(-1, 4).mean(0)
    std_in = a.reshape(-1, 4).std(0)
    mean_d = d.reshape(-1, 4).mean(0)
    std_d = d.reshape(-1, 4).std(0)
    std_in = np.where(std_in > 0, std_in, 1.0)
    std_d = np.where(std_d > 0, std_d, 1.0)
    return mean_in, std_in, mean_d, std_d


class Surrogate:
    def __init__(self, max_batch, H=256, W=256, seed=0, stream=None):
        import torch
        self.torch = torch
        self.B, self.H, self.W = max_batch, H, W
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p()
        st = plbm.lib().plbm_sur_create(max_batch, H, W, seed, self.stream.cuda_stream, ctypes.byref(h))
        if st != plbm.PLBM_OK:
            raise plbm.PlbmError(st, plbm.last_error(None))
        self.h = h
        self.n = plbm.lib().plbm_sur_num_params()
        self.x = torch.empty((max_batch, H, W, 4), dtype=torch.bfloat16, device="cuda")
        self.y = torch.empty((max_batch, H, W, 4), dtype=torch.float32, device="cuda")
        self.out = torch.empty((max_batch, H, W, 4), dtype=torch.float32, device="cuda")
        self.norm = None

    def _ok(self, st):
        if st != plbm.PLBM_OK:
            raise plbm.PlbmError(st, plbm.lib().plbm_sur_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            plbm.lib().plbm_sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor_path(self, tcgen05: bool):
        """tcgen05.mma (True, default) or mma.sync (False) for the 64 -> 64 convolutions,
        their backward-data passes and their weight gradients."""
        self._ok(plbm.lib().plbm_sur_set_option(self.h, 1, 1 if tcgen05 else 0))

    def set_conserve(self, on: bool):
        """Project predicted fields onto the old global mass, momentum and energy
        before the drift gate of advance (PLBM_SUR_OPT_CONSERVE)."""
        self._ok(plbm.lib().plbm_sur_set_option(self.h, 2, 1 if on else 0))

    def set_wait_ns(self, ns: int):
        """Budget of each bounded wait of the tcgen05 kernels (PLBM_SUR_OPT_WAIT_NS)."""
        self._ok(plbm.lib().plbm_sur_set_option(self.h, 3, int(ns)))

    def set_mean_penalty(self, lam: float):
        """Weight of the lattice-mean error term of the training loss."""
        self._ok(plbm.lib().plbm_sur_set_mean_penalty(self.h, float(lam)))

    def check(self):
        return int(plbm.lib().plbm_sur_check(self.h))

    def set_norm(self, mean_in, std_in, mean_d, std_d):
        self.norm = tuple(np.asarray(a, dtype=np.float64) for a in (mean_in, std_in, mean_d, std_d))
        arrs = [(ctypes.c_float * 4)(*[float(v) for v in a]) for a in self.norm]
        self._ok(plbm.lib().plbm_sur_set_norm(self.h, *arrs))

    def params(self):
        p = np.empty(self.n, dtype=np.float32)
        g = np.empty(self.n, dtype=np.float32)
        self._ok(plbm.lib().plbm_sur_get_params(self.h, p.ctypes.data, g.ctypes.data))
        return p, g

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n
        self._ok(plbm.lib().plbm_sur_set_params(self.h, p.ctypes.data))

    def forward(self, x, B):
        self._ok(plbm.lib().plbm_sur_forward(self.h, int(B), x.data_ptr(), self.out.data_ptr()))
        self.stream.synchronize()
        return self.out[:B]

    def backward(self, x, dout, B):
        self._ok(plbm.lib().plbm_sur_backward(self.h, int(B), x.data_ptr(), dout.data_ptr()))
        return self.params()[1]

    def tensor(self, kind, layer, B):
        """Copy of a stored activation (kind 0) or pre-activation gradient (kind 1)."""
        torch = self.torch
        if kind == 0 and layer == 6:
            out = torch.empty((B, self.H, self.W, 4), dtype=torch.float32, device="cuda")
        else:
            out = torch.empty((B, self.H, self.W, 64), dtype=torch.bfloat16, device="cuda")
        self._ok(plbm.lib().plbm_sur_copy(self.h, int(kind), int(layer), int(B), out.data_ptr()))
        return out

    def train(self, stack, pairs, steps, batch=16, lr=1e-3, lr_end=None, seed=0, log_every=0, noise=0.0):
        """Adam steps on random minibatches of `pairs`; returns the list of (step, loss).
        noise: standard deviation of the normal perturbation added to the normalised
        inputs of every minibatch (plbm_sur_assemble_noise; 0 = none)."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        npix = self.H * self.W
        # every minibatch's pair indices on the device before the first step: the
        # steps run on the surrogate's stream while the host goes ahead, so an
        # index buffer rewritten per step would be read by a later step's copy
        sels = np.empty((steps, batch, 2), dtype=np.int32)
        order = rng.permutation(len(pairs))
        pos = 0
        for it in range(steps):
            if pos + batch > len(order):
                order = rng.permutation(len(pairs))
                pos = 0
            sels[it] = pairs[order[pos:pos + batch]]
            pos += batch
        pairs_all = torch.from_numpy(sels).to("cuda")
        torch.cuda.current_stream().synchronize()
        losses = []
        lr_end = lr if lr_end is None else lr_end
        for it in range(steps):
            self._ok(plbm.lib().plbm_sur_assemble_noise(self.h, stack.data_ptr(), npix, pairs_all[it].data_ptr(),
                                                        batch, self.x.data_ptr(), self.y.data_ptr(), float(noise),
                                                        (int(seed) << 32) + it))
            frac = it / max(1, steps - 1)
            lr_t = lr * (lr_end / lr) ** frac
            want = log_every and (it % log_every == 0 or it == steps - 1)
            loss = ctypes.c_float()
            self._ok(plbm.lib().plbm_sur_train_step(self.h, batch, self.x.data_ptr(), self.y.data_ptr(),
                                                    float(lr_t), ctypes.byref(loss) if want else None))
            if want:
                losses.append((it, loss.value))
        self.stream.synchronize()
        return losses

    def evaluate(self, stack, pairs, batch=None):
        """(network MSE, persistence MSE) in normalised units over the given pairs.

        Persistence predicts no change, i.e. the normalised target -mean_d / std_d."""
        torch = self.torch
        batch = batch or self.B
        npix = self.H * self.W
        pairs_dev = torch.empty((batch, 2), dtype=torch.int32, device="cuda")
        persist = torch.tensor((-self.norm[2] / self.norm[3]).astype(np.float32), device="cuda")
        se = sp = 0.0
        count = 0
        for i in range(0, len(pairs), batch):
            sel = pairs[i:i + batch]
            B = len(sel)
            pairs_dev[:B].copy_(torch.from_numpy(np.ascontiguousarray(sel)))
            torch.cuda.synchronize()
            self._ok(plbm.lib().plbm_sur_assemble(self.h, stack.data_ptr(), npix, pairs_dev.data_ptr(), B,
                                                  self.x.data_ptr(), self.y.data_ptr()))
            out = self.forward(self.x, B)
            y = self.y[:B]
            se += float(((out - y) ** 2).sum())
            sp += float(((persist - y) ** 2).sum())
            count += y.numel()
        return se / count, sp / count

    def advance(self, solvers, K=32, tol=1e-4):
        """Advance the given Solver handles by K steps; returns the fallback flags."""
        n = len(solvers)
        hs = (ctypes.c_void_p * n)(*[s.h.value if hasattr(s.h, "value") else s.h for s in solvers])
        flags = (ctypes.c_int * n)()
        self._ok(plbm.lib().plbm_sur_advance(self.h, hs, n, int(K), float(tol), flags))
        self.n_last = n
        return list(flags)

    def last_drift(self):
        """Drift of every lattice of the last advance (the quantity compared with tol)."""
        out = np.empty(self.n_last, dtype=np.float64)
        self._ok(plbm.lib().plbm_sur_last_drift(self.h, out.ctypes.data, self.n_last))
        return out
