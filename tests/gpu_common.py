"""Helpers shared by the GPU tests (not a test module)."""
import numpy as np


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def morton_key(ijk, level):
    key = 0
    for bit in range(level):
        for a in range(3):
            key |= ((int(ijk[a]) >> bit) & 1) << (3 * bit + a)
    return key


def gpu_apply(plan, x, nrhs=None):
    import torch
    dt = torch.complex128 if plan.precision == 0 else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dt, device="cuda")
    y = plan.apply(xt)
    torch.cuda.synchronize()
    return y.cpu().numpy()
