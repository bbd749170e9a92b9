"""What the trained learned-tau network gains over the method without it.

On fresh seeded decay pairs (a seed used neither for training nor for the
held-out evaluation) the committed network's tau must meet the target error
in most cases, and the time to an admissible tau (prediction, one error check,
bisection only on a miss: spamm_tau_select with the network) must need fewer
error evaluations than plain bisection on the error (spamm_tau_select without
it), which stays the fallback and the arbiter.
"""
import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from paper_2103_13042_gb300 import tau_train as TT

pytestmark = pytest.mark.gpu


def test_trained_network_beats_bisection():
    W = P.load_tau_weights()
    dev = torch.device("cuda", 0)
    specs = synth.training_specs(12, synth.config_seed(4) + 31337, sizes=(1024, 2048))
    meters = {}
    hits, net_evals, bis_evals, ratios = 0, [], [], []
    total = 0
    for sp in specs:
        A, B = synth.spec_matrices_device(sp, dev)
        m = meters.get(sp["n"]) or meters.setdefault(sp["n"], TT.ErrorMeter(sp["n"], dev))
        m.setup(A, B)
        for eps in (1e-4, 1e-6):
            total += 1
            tau_p = m.plan.tau_predict(m.nA, m.nB, eps, W)
            e_p = m.error(tau_p)
            tau_b, n_b, e_b = m.select(eps)          # plain bisection: spamm_tau_select
            assert e_b <= eps                       # the arbiter's own answer is admissible
            assert m.error(tau_b) == e_b
            tau_n, n_n, e_n = m.select(eps, W)       # network, one check, bisection on a miss
            assert e_n <= eps
            bis_evals.append(n_b)
            net_evals.append(n_n)
            if e_p <= eps:
                hits += 1
                assert n_n == 1 and tau_n == tau_p
                ratios.append(tau_p / tau_b)
            else:
                assert n_n == 1 + n_b and tau_n == tau_b
    assert hits / total >= 0.75, hits / total
    assert np.mean(net_evals) < 0.5 * np.mean(bis_evals), (np.mean(net_evals), np.mean(bis_evals))
    # a hit is not an over-cautious tau: within three decades of the largest admissible one
    assert np.median(ratios) > 1e-3
