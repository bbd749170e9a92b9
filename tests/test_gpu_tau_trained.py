"""What the trained learned-tau network gains over the method without it.

On fresh seeded decay pairs (a seed used neither for training nor for the
held-out evaluation) the committed network's tau must meet the target error
in most cases, and the time to an admissible tau (prediction, one error check,
bisection only on a miss) must need fewer error evaluations than plain
bisection on the error, which stays the fallback and the arbiter.
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
            tau_b, n_b = TT.bisect_on_error(m, eps, tau0=m.ab * eps)
            e_b = m.error(tau_b)
            assert e_b <= eps                       # the arbiter's own answer is admissible
            bis_evals.append(n_b)
            if e_p <= eps:
                hits += 1
                net_evals.append(1)
                ratios.append(tau_p / tau_b)
            else:
                net_evals.append(1 + n_b)
    assert hits / total >= 0.75, hits / total
    assert np.mean(net_evals) < 0.5 * np.mean(bis_evals), (np.mean(net_evals), np.mean(bis_evals))
    # a hit is not an over-cautious tau: within three decades of the largest admissible one
    assert np.median(ratios) > 1e-3
