"""Helpers shared by the GPU parity tests (device transfer, plan export decoding)."""
import numpy as np
import torch

import paper_2103_13042_gb300 as P


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def plan_mask(plan: "P.Plan"):
    """(survivor mask [bd, bd, bd] as surv[i, k, j], split-flag mask) from the exported queues."""
    tp, kk = plan.export()
    bd = plan.bd
    surv = np.zeros((bd, bd, bd), dtype=bool)
    flag = np.zeros((bd, bd, bd), dtype=bool)
    for t in range(bd * bd):
        i, j = divmod(t, bd)
        ks = kk[tp[t]:tp[t + 1]]
        kv = (ks & 0x3FF).astype(np.int64)
        assert np.all(np.diff(kv) > 0), "survivors of a tile must be listed in increasing k"
        surv[i, kv, j] = True
        flag[i, kv, j] = (ks & 0x8000) != 0
    return surv, flag


def band_ok(gpu_surv, ora_surv, p, tau, band=1e-12):
    """Every disagreement lies within `band` relative of tau."""
    diff = gpu_surv != ora_surv
    if not diff.any():
        return True
    return bool(np.all(np.abs(p[diff] - tau) <= band * tau))
