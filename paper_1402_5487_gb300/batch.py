"""Batched sweeps of many lattices (ctypes binding of the plbm_batch_* calls).

``draw_instances`` turns the seeded candidate draws of ``inputs.batch_candidates``
into an admissible sweep with the library's own host gates: the positivity
range of Sec. 3.1 (``plbm_positivity``: every r_i >= 0 for |u| <= u_max at
theta0) and linear stability (``plbm_linear_stability``: max |lambda| <= 1 + 1e-9
at u = 0 and u = (u_max, 0) on a 48 x 48 wave-vector grid plus both k axes at
384 points; unstable bands of these lattices can be narrower than the spacing
of a 16 x 16 grid and sit on the axes).  u_max is 0.1 for
Kelvin-Helmholtz layers and 1e-3 for shear waves.

``Batch`` owns one plbm_batch: instances are ordinary handles for init and
output, steps go through one of the four launch schemes, and ``autotune``
caches the chosen persistent-kernel shape in a JSON file.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import inputs as I
from . import plbm

PERSISTENT = 0
PERSISTENT_GRAPH = 1
PER_INSTANCE = 2
PER_INSTANCE_GRAPH = 3
MODES = {"persistent": PERSISTENT, "persistent_graph": PERSISTENT_GRAPH,
         "per_instance": PER_INSTANCE, "per_instance_graph": PER_INSTANCE_GRAPH}
ORDERS = {"contiguous": 0, "interleaved": 1}   # PLBM_BATCH_ORDER_*


def admissible(v, omega, theta0, u_max, nk=48):
    """(accepted, min r, max |lambda|) by the library's host gates."""
    min_r = plbm.positivity(2, v, theta0, u_max)
    if min_r < 0.0:
        return False, min_r, None
    lim = 1.0 + 1e-9
    lam = plbm.linear_stability(2, v, omega, theta0, u_max, nk, stop_above=lim)
    if lam <= lim:
        lam = max(lam, plbm.linear_stability(2, v, omega, theta0, 0.0, nk, stop_above=lim))
    return lam <= lim, min_r, lam


def draw_instances(n=256, seed=1000, size_lo=64, size_hi=1024, **kw):
    """Admissible instances of the batched sweep and the acceptance statistics."""
    out, tried = [], 0
    for k, L, kind, cands in I.batch_candidates(n, seed, size_lo, size_hi, **kw):
        u_max = 0.1 if kind == "kh" else 1e-3
        for v, om, th in cands:
            tried += 1
            ok, _, _ = admissible(v, om, th, u_max)
            if ok:
                out.append(I.Instance(index=k, L=L, v=v, omega=om, theta0=th, kind=kind, seed=seed + k))
                break
        else:
            raise RuntimeError("instance %d: no admissible candidate" % k)
    return out, {"instances": n, "candidates_tried": tried, "acceptance": n / tried}


class Batch:
    """n lattices advanced together (see include/plbm.h, plbm_batch_*)."""

    def __init__(self, instances, prec="f32", device=0, stream=None):
        """prec: storage precision of every instance whose own ``prec`` is None."""
        import torch
        self.torch = torch
        self.instances = list(instances)
        self.prec = prec
        self.precs = [inst.prec or prec for inst in self.instances]
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        n = len(self.instances)
        descs = (plbm.PlbmDesc * n)()
        self._keep = []
        for i, inst in enumerate(self.instances):
            d, keep = plbm.make_desc(2, inst.v, inst.omega, inst.L, inst.L, theta0=inst.theta0, prec=self.precs[i],
                                     isothermal=inst.isothermal, device=device,
                                     u_max=0.1 if inst.kind == "kh" else 1e-3)
            descs[i] = d
            self._keep.append(keep)
        b = ctypes.c_void_p()
        st = plbm.lib().plbm_batch_create(descs, n, self.stream.cuda_stream, ctypes.byref(b))
        if st != plbm.PLBM_OK:
            raise plbm.PlbmError(st, plbm.lib().plbm_batch_last_error(None).decode())
        self.b = b
        self.solvers = []
        for i, inst in enumerate(self.instances):
            h = plbm._H()
            self._ok(plbm.lib().plbm_batch_instance(self.b, i, ctypes.byref(h)))
            self.solvers.append(plbm.Solver._wrap(h, 2, inst.v, inst.L, inst.L, self.precs[i], self.stream, torch))

    def _ok(self, st):
        if st != plbm.PLBM_OK:
            raise plbm.PlbmError(st, plbm.lib().plbm_batch_last_error(self.b).decode())

    @property
    def nodes(self) -> int:
        return sum(inst.L * inst.L for inst in self.instances)

    def init(self):
        """Initial fields of every instance (host FP64, inputs.instance_fields)."""
        for inst, s in zip(self.instances, self.solvers):
            rho, ux, uy, th = I.instance_fields(inst)
            s.init(rho, ux, uy, None if inst.isothermal else th)

    def groups(self):
        """(row-paired instances, plain-layout instances, persistent launches per step)."""
        vals = [ctypes.c_int() for _ in range(3)]
        self._ok(plbm.lib().plbm_batch_groups(self.b, *[ctypes.byref(v) for v in vals]))
        return tuple(v.value for v in vals)

    def step(self, n=1, mode="persistent_graph"):
        self._ok(plbm.lib().plbm_batch_step(self.b, int(n), MODES[mode] if isinstance(mode, str) else int(mode)))

    def check(self):
        bad = ctypes.c_int()
        st = plbm.lib().plbm_batch_check(self.b, ctypes.byref(bad))
        return st, bad.value

    def set_config(self, block_x, ctas_per_sm):
        self._ok(plbm.lib().plbm_batch_set_config(self.b, int(block_x), int(ctas_per_sm)))

    def set_order(self, order):
        """"contiguous" or "interleaved" tile order of the persistent kernel."""
        self._ok(plbm.lib().plbm_batch_set_order(self.b, ORDERS[order] if isinstance(order, str) else int(order)))

    @property
    def order(self):
        return {v: k for k, v in ORDERS.items()}[plbm.lib().plbm_batch_get_order(self.b)]

    def info(self):
        vals = [ctypes.c_int() for _ in range(5)]
        self._ok(plbm.lib().plbm_batch_info(self.b, *[ctypes.byref(v) for v in vals]))
        keys = ("instances", "total_tiles", "block_x", "ctas", "max_ctas_per_sm")
        return dict(zip(keys, (v.value for v in vals)))

    def cache_key(self):
        n = self.nodes
        paired, plain, _ = self.groups()
        return "%s/d2q25/%d-instances/%d-paired/%d-Mnodes" % ("+".join(sorted(set(self.precs))), len(self.instances),
                                                             paired, int(round(n / 1e6)))

    def autotune(self, steps_per_trial=6, cache_path=None):
        """Pick the persistent-kernel shape (cached in JSON by precision, count and size)."""
        key = self.cache_key()
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as fh:
                cache = json.load(fh)
        if key in cache:
            c = cache[key]
            self.set_config(c["block_x"], c["ctas_per_sm"])
            self.set_order(c.get("order", "contiguous"))
            return dict(c, cached=True)
        bx, cps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._ok(plbm.lib().plbm_batch_tune(self.b, int(steps_per_trial), ctypes.byref(bx), ctypes.byref(cps),
                                            ctypes.byref(ms)))
        c = {"block_x": bx.value, "ctas_per_sm": cps.value, "order": self.order, "ms_per_step": ms.value}
        if cache_path:
            cache[key] = c
            d = os.path.dirname(os.path.abspath(cache_path))
            os.makedirs(d, exist_ok=True)
            with open(cache_path, "w") as fh:
                json.dump(cache, fh, indent=1)
        return dict(c, cached=False)

    def close(self):
        if getattr(self, "b", None):
            for s in self.solvers:
                s.close()
            plbm.lib().plbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
