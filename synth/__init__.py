"""Seeded synthetic inputs for SpAMM (shared by the CPU oracle and the CUDA path).

This module only draws numbers: it holds none of the method's arithmetic (no
norms, no products, no thresholds).  Every generator returns a C-contiguous
float32 N x N array, drawn in row-major order from numpy's PCG64 generator so
that both sides of a parity test see identical bits.

Matrix families (paper section 2.1 defines decay matrices; the concrete
recipes are the synthetic workloads of the SpAMM hot path):

* ``exp_decay_su``     a_ij = exp(-alpha |i-j|) * s_ij * u_ij, s = +-1, u ~ U[0.5, 1]
* ``alg_decay_signed`` a_ij = (|i-j| + 1)^(-q) * s_ij, s = +-1
* ``exp_decay_normal`` a_ij = exp(-alpha |i-j|) * z_ij, z ~ N(0, 1)
* ``near_sparse``      ReLU(z_ij), then each remaining entry zeroed with prob. 0.7
* ``table1_matrix``    a_ij = 0.1 / (|i-j|^0.1 + 1)   (Section 4.1, Table 1 workload)
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20210324


def config_seed(config_index: int, instance: int = 0, operand: str = "A") -> int:
    """Seed convention: base + 1000*config + instance, operand B offset by 500."""
    return SEED_BASE + 1000 * config_index + instance + (500 if operand == "B" else 0)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _dist_rows(r0: int, r1: int, n: int) -> np.ndarray:
    i = np.arange(r0, r1, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    return np.abs(i - j)


_ROW_CHUNK = 1024


def exp_decay_su(n: int, alpha: float, seed: int) -> np.ndarray:
    """exp(-alpha|i-j|) * s * u, s uniform on {-1,+1}, u ~ U[0.5,1]; s drawn first, then u."""
    g = _rng(seed)
    s = g.integers(0, 2, size=(n, n), dtype=np.int8)
    u = g.uniform(0.5, 1.0, size=(n, n))
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, _ROW_CHUNK):
        r1 = min(n, r0 + _ROW_CHUNK)
        mag = np.exp(-alpha * _dist_rows(r0, r1, n))
        sign = 2.0 * s[r0:r1].astype(np.float64) - 1.0
        out[r0:r1] = (mag * sign * u[r0:r1]).astype(np.float32)
    return out


def alg_decay_signed(n: int, q: float, seed: int) -> np.ndarray:
    """(|i-j|+1)^(-q) * s, s uniform on {-1,+1}."""
    g = _rng(seed)
    s = g.integers(0, 2, size=(n, n), dtype=np.int8)
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, _ROW_CHUNK):
        r1 = min(n, r0 + _ROW_CHUNK)
        mag = (_dist_rows(r0, r1, n) + 1.0) ** (-q)
        sign = 2.0 * s[r0:r1].astype(np.float64) - 1.0
        out[r0:r1] = (mag * sign).astype(np.float32)
    return out


def exp_decay_normal(n: int, alpha: float, seed: int) -> np.ndarray:
    """exp(-alpha|i-j|) * z, z ~ N(0,1) (float64 draws, row chunks in order)."""
    g = _rng(seed)
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, _ROW_CHUNK):
        r1 = min(n, r0 + _ROW_CHUNK)
        z = g.standard_normal(size=(r1 - r0, n))
        out[r0:r1] = (np.exp(-alpha * _dist_rows(r0, r1, n)) * z).astype(np.float32)
    return out


def near_sparse(n: int, seed: int, drop: float = 0.7) -> np.ndarray:
    """ReLU(N(0,1)), then every surviving entry zeroed independently with probability ``drop``."""
    g = _rng(seed)
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, _ROW_CHUNK):
        r1 = min(n, r0 + _ROW_CHUNK)
        z = g.standard_normal(size=(r1 - r0, n)).astype(np.float32)
        keep = g.uniform(size=(r1 - r0, n)) >= drop
        out[r0:r1] = np.where((z > 0) & keep, z, np.float32(0.0))
    return out


def rect_decay_normal(m: int, k: int, alpha: float, seed: int) -> np.ndarray:
    """m x k: exp(-alpha |i k/m - j|) * z, z ~ N(0,1): decay away from the stretched diagonal
    (rectangular operands of the general form; z drawn in one row-major block)."""
    g = _rng(seed)
    z = g.standard_normal(size=(m, k))
    i = np.arange(m, dtype=np.float64)[:, None] * (k / m)
    j = np.arange(k, dtype=np.float64)[None, :]
    return (np.exp(-alpha * np.abs(i - j)) * z).astype(np.float32)


def rect_near_sparse(m: int, k: int, seed: int, drop: float = 0.7) -> np.ndarray:
    """m x k ReLU(N(0,1)) with each remaining entry zeroed with probability ``drop`` (normals
    drawn first, then the uniforms, each in one row-major block)."""
    g = _rng(seed)
    z = g.standard_normal(size=(m, k))
    keep = g.uniform(size=(m, k)) >= drop
    return np.where((z > 0) & keep, z, 0.0).astype(np.float32)


def table1_matrix(n: int) -> np.ndarray:
    """Deterministic algebraic-decay matrix 0.1/(|i-j|^0.1 + 1) used for Table 1."""
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, _ROW_CHUNK):
        r1 = min(n, r0 + _ROW_CHUNK)
        out[r0:r1] = (0.1 / (_dist_rows(r0, r1, n) ** 0.1 + 1.0)).astype(np.float32)
    return out


def block_constant(exps: np.ndarray, signs: np.ndarray, leaf: int) -> np.ndarray:
    """Matrix whose (I,K) leaf block is the constant signs[I,K] * 2^exps[I,K] (tiny hand cases)."""
    bd = exps.shape[0]
    vals = (signs.astype(np.float64) * np.exp2(exps.astype(np.float64))).astype(np.float32)
    return np.kron(vals, np.ones((leaf, leaf), dtype=np.float32)).astype(np.float32)


# ---------------------------------------------------------------------------
# Mixed workloads (batched instances, learned-tau training matrices)
# ---------------------------------------------------------------------------

def batch_specs(count: int, seed: int, n_lo: int = 256, n_hi: int = 4096):
    """Instance specs: N log-uniform on [n_lo, n_hi]; decay family 50/50 exponential / algebraic.

    Exponential: alpha ~ U[0.2, 1.5], entries exp(-alpha|i-j|) * N(0,1).
    Algebraic:   q ~ U[2, 4],        entries (|i-j|+1)^(-q) * (+-1).
    Returns a list of dicts with keys n, kind, rate, seed_a, seed_b.
    """
    g = _rng(seed)
    specs = []
    for t in range(count):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = "exp" if g.uniform() < 0.5 else "alg"
        rate = float(g.uniform(0.2, 1.5)) if kind == "exp" else float(g.uniform(2.0, 4.0))
        specs.append({"n": n, "kind": kind, "rate": rate,
                      "seed_a": seed + 10 * t + 1, "seed_b": seed + 10 * t + 2})
    return specs


def spec_matrices(spec) -> tuple[np.ndarray, np.ndarray]:
    """Draw the (A, B) pair of one instance spec from :func:`batch_specs`."""
    n, rate = spec["n"], spec["rate"]
    if spec["kind"] == "exp":
        return (exp_decay_normal(n, rate, spec["seed_a"]),
                exp_decay_normal(n, rate, spec["seed_b"]))
    return (alg_decay_signed(n, rate, spec["seed_a"]),
            alg_decay_signed(n, rate, spec["seed_b"]))


def training_specs(count: int, seed: int, sizes=(1024, 2048, 4096, 8192)):
    """Specs for learned-tau data: N from ``sizes``, families and rates as in :func:`batch_specs`."""
    g = _rng(seed)
    specs = []
    for t in range(count):
        n = int(sizes[int(g.integers(0, len(sizes)))])
        kind = "exp" if g.uniform() < 0.5 else "alg"
        rate = float(g.uniform(0.2, 1.5)) if kind == "exp" else float(g.uniform(2.0, 4.0))
        specs.append({"n": n, "kind": kind, "rate": rate,
                      "seed_a": seed + 10 * t + 1, "seed_b": seed + 10 * t + 2})
    return specs


# Named workloads -----------------------------------------------------------

def workload_c1(tau_free: bool = True):
    """N=1024, A = B = exp(-0.5|i-j|) s u, leaf 32."""
    a = exp_decay_su(1024, 0.5, config_seed(0))
    return a, a.copy()


def workload_c2(n: int = 8192):
    """N=8192 independent algebraic decay (q=3) with random signs, leaf 64."""
    return (alg_decay_signed(n, 3.0, config_seed(1, operand="A")),
            alg_decay_signed(n, 3.0, config_seed(1, operand="B")))


def mlp_init(seed: int, sizes=(65, 64, 64, 1)) -> np.ndarray:
    """Flat initial parameters: W_l, b_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), FP32, in layer order."""
    g = _rng(seed)
    parts = []
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        bound = 1.0 / math.sqrt(fi)
        parts.append(g.uniform(-bound, bound, size=fo * fi))
        parts.append(g.uniform(-bound, bound, size=fo))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# Device-side draws of the same families (training data for the learned-tau
# network, where thousands of large matrices are needed and host generation
# would dominate).  Seeded with torch's device generator: deterministic for a
# given seed and device, but NOT the same bits as the numpy generators above,
# so nothing here feeds a parity test against the oracle.
# ---------------------------------------------------------------------------

def spec_matrices_device(spec, device):
    """(A, B) float32 device tensors of a spec from :func:`training_specs` / :func:`batch_specs`."""
    import torch
    n, rate = int(spec["n"]), float(spec["rate"])
    idx = torch.arange(n, device=device, dtype=torch.float32)
    dist = (idx[:, None] - idx[None, :]).abs()
    if spec["kind"] == "exp":
        mag = torch.exp(-rate * dist)
    else:
        mag = (dist + 1.0).pow(-rate)
    out = []
    for seed in (spec["seed_a"], spec["seed_b"]):
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        if spec["kind"] == "exp":
            z = torch.randn(n, n, generator=g, device=device, dtype=torch.float32)
        else:
            z = torch.randint(0, 2, (n, n), generator=g, device=device).to(torch.float32) * 2.0 - 1.0
        out.append((mag * z).contiguous())
    return out[0], out[1]


def near_sparse_device(n: int, seed: int, device, drop: float = 0.7):
    """ReLU(N(0,1)) with each remaining entry zeroed with probability ``drop``, drawn on the
    device (torch's seeded generator; the large near-sparse workload, never an oracle input)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty(n, n, device=device, dtype=torch.float32)
    rows = max(1, (1 << 26) // n)          # bounded temporaries
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        z = torch.randn(r1 - r0, n, generator=g, device=device, dtype=torch.float32)
        keep = torch.rand(r1 - r0, n, generator=g, device=device) >= drop
        out[r0:r1] = torch.where((z > 0) & keep, z, torch.zeros((), device=device))
    return out
