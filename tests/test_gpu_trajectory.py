"""1 ns trajectories of the 64 x 32 x 1 film (4 nm cells, RK4 at h = 0.1 ps,
10,000 steps) on the GPU against the CPU oracle: within 1e-4 in m after
1 ns, with full demag at every sub-step (FP64 and FP32 fields) and with the
order-3 extrapolation companion run (FP64 and FP32 fields)."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2107_06729_gb300 import workloads as W
from gpu_util import gpu_run

pytestmark = pytest.mark.gpu

T_END = 1e-9


@functools.lru_cache(maxsize=None)
def _oracle(p):
    cfg = W.film_config1(seed=0)
    integ = dict(cfg["integrator"], extrap_order=p)
    sim = O.Simulation(cfg["mesh"], cfg["material"], cfg["field"], integ, cfg["m0"])
    sim.run(T_END)
    m = sim.m()
    st = sim.stats()
    sim.close()
    return m, st


@pytest.mark.parametrize("prec,p", [("fp64", -1), ("fp64", 3), ("fp32", -1), ("fp32", 3)])
def test_film_1ns_trajectory_within_1e4(prec, p):
    cfg = W.film_config1(seed=0)
    integ = dict(cfg["integrator"], extrap_order=p)
    got, gs = gpu_run(cfg["mesh"], cfg["material"], cfg["field"], integ, cfg["m0"], T_END, prec)
    ref, rs = _oracle(p)
    assert gs["accepted"] == rs["accepted"] == 10000
    assert np.abs(got - ref).max() < 1e-4
    if prec == "fp64":
        assert O.epsilon(got, ref) < 1e-8
