"""The library's default search parameters are the values the paper prints.

vrprpd_alns_params_default and vrprpd_brkga_params_default are host-only C
functions (no CUDA call), read here through the C ABI on the CPU and compared
with the paper's ALNS hyperparameter table (Section 4.2, Table "ALNS
hyperparameters") and BRKGA hyperparameter table with the text around it
(Section 4.4.3-4.4.4).
"""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2602_23685_gb300.build import build
    return ctypes.CDLL(build())


def test_alns_defaults_are_the_papers_table(lib):
    from paper_2602_23685_gb300._search_sig import AlnsParams
    p = AlnsParams()
    lib.vrprpd_alns_params_default(ctypes.byref(p))
    assert p.T0 == 0.30                        # initial temperature coefficient
    assert p.alpha == 0.9998                   # cooling rate
    assert p.reheat == 0.50                    # reheat factor
    assert p.stagnation == 2000                # stagnation threshold, iterations
    assert p.tau == 100                        # weight update interval
    assert p.r == 0.1                          # reaction factor
    assert (p.sigma1, p.sigma2, p.sigma3) == (33, 9, 13)   # scores (also Section 4.2.1's text)
    assert p.w_min == 0.1                      # minimum operator weight
    assert p.ls_pickup_every == 200            # pickup repositioning interval
    assert p.ls_relocate_every == 500          # cross-agent relocation interval
    assert p.sync_every == 1000                # intra-GPU global best check interval
    # removal size: 0 selects the formula max(4, floor(0.05 n)) and max(4, floor(q_max / 2))
    assert (p.q_min, p.q_max) == (0, 0)
    assert p.wait_limit_ns > 0                 # not a search parameter: the bounded device waits


def test_brkga_defaults_are_the_papers_table(lib):
    from paper_2602_23685_gb300._search_sig import BrkgaParams
    p = BrkgaParams()
    lib.vrprpd_brkga_params_default(ctypes.byref(p))
    assert p.pop == 30000                      # population size N_p
    assert p.generations == 20000              # the fixed budget T of generations
    assert p.elite_frac == pytest.approx(0.15) and p.mutant_frac == pytest.approx(0.15)
    assert p.rho == pytest.approx(0.7)         # elite bias in crossover
    assert p.eps == pytest.approx(0.03)        # warm-start perturbation U(-0.03, 0.03)
    assert p.warm_variants == 20               # 20 warm-start seeds
    assert p.warm_slots < 0                    # negative: 15% of P_0, worked out by the run
