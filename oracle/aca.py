"""Partially pivoted adaptive cross approximation (ACA) of a coupling matrix.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing here is shared
with, imported by, or imports the CUDA path.

Sect. 2.7 (closing remark) of Of & Watschinger compresses every stored
coupling matrix A_{c,t x s} (n x n, n = (m+1)^3) into U V^* with U, V of k
columns, built by a partially pivoted ACA (Bebendorf / Rjasanow).  The paper
states no stopping tolerance; reading A1: the usual relative criterion
|u_k| |v_k| <= tol ||S_k||_F, with S_k the current approximation and its
Frobenius norm updated term by term, and tol a parameter of the product.

The method reads one row and one column of A per step (here from the full
matrix; evaluating those entries of f_c directly would give the same numbers).
Step k:
  1. the residual of row i_k:  r = A[i_k, :] - sum_l u_l[i_k] v_l
  2. pivot column j_k: the largest |r|; v_k = r / r[j_k]
  3. u_k = A[:, j_k] - sum_l v_l[j_k] u_l  (the residual of column j_k)
  4. ||S_k||^2 = ||S_{k-1}||^2 + |u_k|^2 |v_k|^2
                 + 2 Re sum_{l<k} (u_l^H u_k)(v_l^H v_k)
  5. stop when |u_k| |v_k| <= tol ||S_k||; otherwise the next row is the
     largest |u_k| among rows not used yet.
A row whose residual vanishes is marked used and the next unused row taken
(a zero matrix gives rank 0).  Then A ~ sum_k u_k v_k^T = U V^* with
U = [u_k], V = conj([v_k]).
"""
import numpy as np


def aca_partial(a, tol, max_rank=None):
    """(U, V) with a ~ U @ V.conj().T, U (m x k), V (n x k), by the steps in
    the module docstring; max_rank bounds k (default min(m, n))."""
    a = np.asarray(a, dtype=np.complex128)
    m, n = a.shape
    kmax = min(m, n) if max_rank is None else min(int(max_rank), m, n)
    us, vs = [], []
    used = np.zeros(m, dtype=bool)
    fro2 = 0.0
    i = 0
    while len(us) < kmax:
        row = a[i, :].copy()
        for u, v in zip(us, vs):
            row -= u[i] * v
        used[i] = True
        j = int(np.argmax(np.abs(row)))
        if row[j] == 0:
            if used.all():
                break
            i = int(np.flatnonzero(~used)[0])
            continue
        v = row / row[j]
        u = a[:, j].copy()
        for ul, vl in zip(us, vs):
            u -= vl[j] * ul
        nu2 = float(np.vdot(u, u).real)
        nv2 = float(np.vdot(v, v).real)
        cross = sum(np.vdot(ul, u) * np.vdot(vl, v) for ul, vl in zip(us, vs))
        fro2 += nu2 * nv2 + 2.0 * float(np.real(cross))
        us.append(u)
        vs.append(v)
        if np.sqrt(nu2 * nv2) <= tol * np.sqrt(max(fro2, 0.0)):
            break
        if used.all():
            break
        cand = np.where(used, -1.0, np.abs(u))
        i = int(np.argmax(cand))
    if not us:
        return np.zeros((m, 0), dtype=np.complex128), np.zeros((n, 0), dtype=np.complex128)
    return np.stack(us, axis=1), np.conj(np.stack(vs, axis=1))
