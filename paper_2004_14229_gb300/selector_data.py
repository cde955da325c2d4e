"""Training data of the parameter selector, measured by the method itself.

For every measurement problem (workloads.selector_problems) the product is
computed at Chebyshev orders 2..7, once with the default high-frequency level
l_hf (Eq. 11's rule) and once with l_hf - 1, and compared with exact rows of
Eq. (1) summed directly on the GPU (dfdm_direct_rows): the relative l2 error
on sampled rows.  Orders up to 5 use the tensor-core form (their errors, above
1e-5, are far above its ~1e-6 rounding), orders 6 and 7 the FP64 form (or, for
problems measured with the tensor-core form only, orders 2..6 in that form).
For a tolerance tol, the label of every level l of the problem is
  * order: the smallest measured order whose error (default l_hf) is <= tol / 3
    (a safety factor, so that the network's picks meet tol; one above the
    highest measured order when none is), scaled to (order - 2) / 8;
  * direction flag: 1 when l <= l_hf_needed, where l_hf_needed = l_hf - 1 if
    that coarser choice still meets tol / 3 at the chosen order, else l_hf;
and its features are dfdm_selector_features(kappa, root side, l, N, tol).
"""
import numpy as np

from . import FP64, TC_FP16X3, Plan, Selector, direct_rows
from .workloads import sample_rows

ORDERS = (2, 3, 4, 5, 6, 7)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class _Reference:
    """Direct-sum rows of one problem (computed once)."""

    def __init__(self, p, nrows, seed):
        import torch
        self.p = p
        self.rows = sample_rows(p["targets"].shape[0], nrows, seed)
        self.x64 = torch.from_numpy(np.ascontiguousarray(p["x"], dtype=np.complex128)).cuda()
        self.x32 = self.x64.to(torch.complex64)
        self.ref = direct_rows(torch.from_numpy(p["targets"]).cuda(), torch.from_numpy(p["sources"]).cuda(),
                               p["kappa"], self.x64, torch.from_numpy(self.rows).cuda()).cpu().numpy()

    def error(self, order, l_hf, tc_max=5):
        p = self.p
        prec = TC_FP16X3 if order <= tc_max else FP64
        with Plan(p["targets"], p["sources"], p["kappa"], order=order, max_depth=p["max_depth"], l_hf=l_hf,
                  precision=prec) as pl:
            y = pl.apply(self.x32 if prec == TC_FP16X3 else self.x64).cpu().numpy()[self.rows]
        return _rel(y.astype(np.complex128), self.ref)


def default_l_hf(p):
    """l_hf of the rule (Eq. 11) for problem p, as the library sets it."""
    with Plan(p["targets"], p["sources"], p["kappa"], order=2, max_depth=p["max_depth"], precision=FP64) as probe:
        return probe.stats()["l_hf"]


def evaluate(p, order, l_hf, nrows=64, seed=13):
    """Relative error on sampled direct-sum rows of the product with the given
    order and l_hf (orders above 7 are measured at 7)."""
    return _Reference(p, nrows, seed).error(min(max(order, 2), ORDERS[-1]), l_hf)


def far_field_blocks(p):
    """N_C of problem p's plan (0: every pair is nearfield, the product is
    exact at any order)."""
    with Plan(p["targets"], p["sources"], p["kappa"], order=2, max_depth=p["max_depth"], precision=FP64) as probe:
        return probe.stats()["n_coupling"]


def measure(problems, orders=ORDERS, nrows=64, seed=13, tc_max=5, require_far=False):
    """One record per problem: kappa, N, depth, root side, default l_hf, the
    measured orders and the error of every (order, l_hf shift) in {0, -1}.
    Orders up to tc_max use the tensor-core form, higher ones FP64.
    require_far: skip problems without admissible blocks (their error says
    nothing about the interpolation order)."""
    recs = []
    for p in problems:
        if require_far and far_field_blocks(p) == 0:
            continue
        ref = _Reference(p, nrows, seed)
        lhf0 = default_l_hf(p)
        err = {}
        for shift in (0, -1):
            lhf = lhf0 + shift
            if lhf < -1 or (shift < 0 and lhf0 < 0):
                continue
            for o in orders:
                err[(o, shift)] = ref.error(o, lhf, tc_max)
        recs.append(dict(kappa=p["kappa"], n=p["targets"].shape[0], depth=p["max_depth"], root_side=1.0,
                         l_hf=lhf0, err=err, orders=tuple(orders)))
    return recs


SAFETY = 3.0   # labels ask for an error of tol / SAFETY: the network's picks then meet tol


def labels(rec, tol, orders=ORDERS, safety=SAFETY):
    """(order needed, l_hf needed) of one record at tolerance tol (the
    record's own measured orders when it lists them; one above the highest
    when none suffices)."""
    orders = rec.get("orders", orders)
    goal = tol / safety
    ok = [o for o in orders if rec["err"][(o, 0)] <= goal]
    o_need = min(ok) if ok else orders[-1] + 1
    lhf_need = rec["l_hf"]
    o_chk = min(o_need, orders[-1])
    if (o_chk, -1) in rec["err"] and rec["err"][(o_chk, -1)] <= goal:
        lhf_need = rec["l_hf"] - 1
    return o_need, lhf_need


def make_samples(recs, tols, orders=ORDERS):
    """(X (m x 4), T (m x 2)) float32 training samples."""
    X, T = [], []
    for r in recs:
        for tol in tols:
            o_need, lhf_need = labels(r, tol, orders)
            for lv in range(min(2, r["depth"]), r["depth"] + 1):
                X.append(Selector.features(r["kappa"], r["root_side"], lv, r["n"], tol))
                T.append(((o_need - 2) / 8.0, 1.0 if lv <= lhf_need else 0.0))
    return np.asarray(X, dtype=np.float32), np.asarray(T, dtype=np.float32)
