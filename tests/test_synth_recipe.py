"""The seeded input generators follow the recipes they state (shapes, value distributions,
seeds), so that every workload is the one its description names."""
import math

import numpy as np
import pytest

import synth


def _dist(n):
    i = np.arange(n)
    return np.abs(i[:, None] - i[None, :]).astype(np.float64)


def test_seed_convention():
    assert synth.config_seed(0) == 20210324
    assert synth.config_seed(2, 7) == 20210324 + 2000 + 7
    assert synth.config_seed(1, operand="B") == 20210324 + 1000 + 500


def test_generators_are_deterministic_float32_contiguous():
    for f in (lambda s: synth.exp_decay_su(50, 0.5, s), lambda s: synth.alg_decay_signed(50, 2.0, s),
              lambda s: synth.exp_decay_normal(50, 0.3, s), lambda s: synth.near_sparse(50, s)):
        a, b, c = f(3), f(3), f(4)
        assert a.dtype == np.float32 and a.flags.c_contiguous and a.shape == (50, 50)
        assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_exp_decay_su_magnitudes_and_signs():
    n, alpha = 200, 0.5
    a = synth.exp_decay_su(n, alpha, 11).astype(np.float64)
    ratio = np.abs(a) / np.exp(-alpha * _dist(n))
    ok = np.exp(-alpha * _dist(n)) > 1e-30          # FP32 keeps the ratio where not underflowed
    assert ratio[ok].min() >= 0.5 * (1 - 1e-6) and ratio[ok].max() <= 1.0 * (1 + 1e-6)
    assert abs(np.mean(ratio[ok]) - 0.75) < 0.01      # u ~ U[0.5, 1]
    assert abs(np.mean(np.sign(a[ok])) ) < 0.02         # signs +-1 equally likely


def test_alg_decay_signed_is_exact_power_law():
    n, q = 150, 2.5
    a = synth.alg_decay_signed(n, q, 12)
    assert np.array_equal(np.abs(a), ((_dist(n) + 1.0) ** (-q)).astype(np.float32))
    assert abs(np.mean(np.sign(a))) < 0.02


def test_exp_decay_normal_standardised_entries():
    n, alpha = 300, 0.05
    a = synth.exp_decay_normal(n, alpha, 13).astype(np.float64)
    z = a / np.exp(-alpha * _dist(n))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_near_sparse_density_and_values():
    """ReLU(N(0,1)) keeps half the entries, the 70% drop keeps 30% of those: 15% non-zero,
    each a half-normal value (mean sqrt(2/pi))."""
    a = synth.near_sparse(400, 14)
    nz = a[a != 0]
    assert abs(nz.size / a.size - 0.15) < 0.005
    assert (nz > 0).all() and abs(nz.mean() - math.sqrt(2 / math.pi)) < 0.01


def test_table1_matrix_formula():
    n = 70
    a = synth.table1_matrix(n)
    assert np.array_equal(a, (0.1 / (_dist(n) ** 0.1 + 1.0)).astype(np.float32))
    assert a[0, 0] == np.float32(0.1) and a[0, 1] == np.float32(0.05)   # 0^0.1 = 0, 1^0.1 = 1


def test_batch_specs_follow_the_mix():
    specs = synth.batch_specs(2000, 15)
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 256 and ns.max() <= 4096
    logs = np.log(ns)
    assert abs(logs.mean() - (math.log(256) + math.log(4096)) / 2) < 0.05   # log-uniform
    kinds = [s["kind"] for s in specs]
    assert abs(kinds.count("exp") / len(kinds) - 0.5) < 0.04
    for s in specs:
        lo, hi = (0.2, 1.5) if s["kind"] == "exp" else (2.0, 4.0)
        assert lo <= s["rate"] <= hi
    seeds = [s["seed_a"] for s in specs] + [s["seed_b"] for s in specs]
    assert len(set(seeds)) == len(seeds)


@pytest.mark.parametrize("kind", ["exp", "alg"])
def test_spec_matrices_use_the_stated_family(kind):
    spec = {"n": 64, "kind": kind, "rate": 0.7 if kind == "exp" else 3.0, "seed_a": 1, "seed_b": 2}
    a, b = synth.spec_matrices(spec)
    if kind == "exp":
        assert np.array_equal(a, synth.exp_decay_normal(64, 0.7, 1))
        assert np.array_equal(b, synth.exp_decay_normal(64, 0.7, 2))
    else:
        assert np.array_equal(a, synth.alg_decay_signed(64, 3.0, 1))
        assert np.array_equal(b, synth.alg_decay_signed(64, 3.0, 2))


def test_mlp_init_ranges():
    theta = synth.mlp_init(16)
    assert theta.dtype == np.float32 and theta.size == 65 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    w1 = theta[:65 * 64]
    assert np.abs(w1).max() <= 1 / math.sqrt(65) and np.abs(w1).max() > 0.9 / math.sqrt(65)
    w3 = theta[-65:-1]
    assert np.abs(w3).max() <= 1 / math.sqrt(64)


def test_named_workloads():
    a, b = synth.workload_c2(256)
    assert np.array_equal(a, synth.alg_decay_signed(256, 3.0, synth.config_seed(1)))
    assert np.array_equal(b, synth.alg_decay_signed(256, 3.0, synth.config_seed(1, operand="B")))


def test_rect_generators_follow_their_recipes():
    a = synth.rect_decay_normal(30, 70, 0.2, 9)
    z = np.random.Generator(np.random.PCG64(9)).standard_normal((30, 70))
    i = np.arange(30)[:, None] * (70 / 30)
    j = np.arange(70)[None, :]
    assert a.shape == (30, 70) and a.dtype == np.float32
    assert np.array_equal(a, (np.exp(-0.2 * np.abs(i - j)) * z).astype(np.float32))
    b = synth.rect_near_sparse(400, 300, 10)
    assert b.shape == (400, 300) and (b >= 0).all()
    assert abs((b > 0).mean() - 0.15) < 0.01
