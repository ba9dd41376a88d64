"""Pins for the oracle's Beverton-Holt resource (S2 "Resource Consumption"):
R' = r' R / (1 + R/K) - C 2^-16 with the growth rate r' = r + r_sd z drawn
every generation (z: the Irwin-Hall(12) normal)."""
import dataclasses
import math

import numpy as np
from scipy import stats as sps

import oracle
import spegg_synth as S


def resource_only(r, r_sd, K=1e5, n=200, seed=5):
    """A population that eats nothing (attack 0) and always survives, so the
    resource follows the Beverton-Holt map alone."""
    w = S.consumer_resource(n=n, n_loci=32, K=K, mu=0.0, seed=seed)
    w = dataclasses.replace(w, surv_table=S.constant_table(S.CERTAIN), attack=np.zeros(4096, np.uint32),
                            eco_model=1, eco_r=r, eco_r_sd=r_sd)
    return w, oracle.OraclePopulation.from_workload(w)


def test_first_step_and_fixed_point():
    K, r = 1e5, 2.0
    w, p = resource_only(r, 0.0, K)
    R = p.step(80)["R"]
    R0 = w.eco_R0
    assert R[0] == (r * R0) / (1.0 + R0 / K)
    assert abs(R[-1] - K * (r - 1.0)) < 1e-9 * K  # stable fixed point K (r - 1)
    assert np.all(np.diff(R) >= 0)  # monotone approach from below (exactly at K (r - 1) in the end)


def test_growth_rate_draws_follow_the_irwin_hall_normal():
    K, r, sd = 1e5, 2.0, 0.3
    w, p = resource_only(r, sd, K)
    R = np.concatenate([[w.eco_R0], p.step(3000)["R"]])
    rg = R[1:] * (1.0 + R[:-1] / K) / R[:-1]  # the growth rate each generation used
    z = (rg - r) / sd
    n = len(z)
    assert np.all(np.abs(z) <= 6.0 + 1e-9)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5 / math.sqrt(n)
    assert sps.kstest(z, "norm").pvalue > 1e-3


def test_consumption_is_subtracted():
    """With consumption the update is the same map minus C 2^-16."""
    w = S.with_beverton_holt(S.consumer_resource(n=3000, n_loci=32, K=1e6, mu=0.0), r=2.0, r_sd=0.0)
    p = oracle.OraclePopulation.from_workload(w)
    st = p.step(6)
    R = np.concatenate([[w.eco_R0], st["R"]])
    for t in range(6):
        expect = (2.0 * R[t]) / (1.0 + R[t] / w.eco_K) - float(st["consumption"][t]) * (1.0 / 65536.0)
        assert st["R"][t] == max(expect, 0.0)
