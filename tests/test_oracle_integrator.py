"""Pins for the oracle's LLG right-hand side (Eq. 1), field terms, Butcher
tableaux (Eq. 3-4), controller (Eq. 5), demag extrapolation (Eq. 6) and
error metric (Eq. 7).  Each check is fixed by mathematics or by the paper,
not by re-running the oracle's own formula: rooted-tree order conditions,
the analytic macrospin solution, energy dissipation, measured convergence
orders min(n, p+1) (Sec. II after Eq. 6), and the paper's printed
controller constants (tests/golden/controller_constants.json)."""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2107_06729_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- tableaux --
def rooted_trees(order):
    """All rooted trees with `order` nodes; a tree is a sorted tuple of its
    child subtrees."""
    if order == 1:
        return [()]
    out = set()

    def parts(n, maxpart):
        if n == 0:
            yield []
            return
        for k in range(min(n, maxpart), 0, -1):
            for rest in parts(n - k, k):
                yield [k] + rest

    for p in parts(order - 1, order - 1):
        choices = [rooted_trees(k) for k in p]
        for combo in itertools.product(*choices):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def tree_order(t):
    return 1 + sum(tree_order(c) for c in t)


def gamma_tree(t):
    g = tree_order(t)
    for c in t:
        g *= gamma_tree(c)
    return g


def elementary_weight(t, w, A):
    def g(tt):
        v = np.ones(len(w))
        for c in tt:
            v = v * (A @ g(c))
        return v
    return float(w @ g(t))


def test_tree_counts():
    # number of rooted trees of order 1..6 is 1, 1, 2, 4, 9, 20
    assert [len(rooted_trees(k)) for k in range(1, 7)] == [1, 1, 2, 4, 9, 20]


EMBEDDED = {  # method: (order of c, order of chat)
    "RK4": (4, 4), "HEUN12": (2, 1), "RK23": (3, 2), "RKF45": (4, 5),
    "RKCK45": (4, 5), "RKDP54": (5, 4), "RKF56": (5, 6),
}


@pytest.mark.parametrize("method", list(EMBEDDED))
def test_order_conditions(method):
    T = O.tableau(method)
    A = T["b"]
    a = T["a"]
    assert np.allclose(A.sum(axis=1), a, atol=1e-15)  # row sums equal the nodes
    assert np.allclose(np.tril(A, -1), A)  # explicit
    n, nh = EMBEDDED[method]
    assert T["order"] == n
    for w, order in [(T["c"], n), (T["chat"], nh)]:
        for k in range(1, order + 1):
            for t in rooted_trees(k):
                assert elementary_weight(t, w, A) == pytest.approx(1.0 / gamma_tree(t), abs=1e-13)
        # and not one order higher (the stated order is exact)
        if method != "RK4" or w is T["c"]:
            misses = [abs(elementary_weight(t, w, A) - 1.0 / gamma_tree(t)) > 1e-10
                      for t in rooted_trees(order + 1)]
            assert any(misses)


def test_stage_counts_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_claims.json")))["substeps"]
    assert O.tableau("RK4")["s"] == g["RK4"]
    T = O.tableau("RK23")  # 4 stages, FSAL: 3 new evaluations per step
    assert T["fsal"] and T["s"] - 1 == g["RK23"]
    # FSAL: the last stage's input is the solution (last row = solution weights, c_s = 0)
    assert np.allclose(T["b"][-1, :-1], T["c"][:-1]) and T["c"][-1] == 0
    assert O.tableau("RKF56")["s"] == g["RKF56"]
    D = O.tableau("RKDP54")
    assert D["fsal"] and np.allclose(D["b"][-1, :-1], D["c"][:-1]) and D["c"][-1] == 0


# -------------------------------------------------------------- Eq. 6 ------
@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_lagrange_weights_reproduce_polynomials(p):
    rng = np.random.default_rng(p)
    # nodes: current and previous step-start times (<= 0), target ahead
    h = rng.uniform(0.5, 2.0, size=p)
    nodes = -np.concatenate([[0.0], np.cumsum(h)])
    for tau in [0.0, 0.3, 1.0, 1.7]:
        w = O.lagrange_weights(nodes, tau)
        assert w.sum() == pytest.approx(1.0, abs=1e-12)
        for deg in range(p + 1):
            assert (w * nodes ** deg).sum() == pytest.approx(tau ** deg, rel=1e-10, abs=1e-10)
    if p == 0:
        assert O.lagrange_weights(nodes, 0.7)[0] == 1.0  # hold last value
    # at a node the weights are the unit vector
    w = O.lagrange_weights(nodes, nodes[-1])
    assert np.allclose(w, np.eye(p + 1)[-1], atol=1e-12)


def test_extrapolation_degree_p_is_not_exact_for_degree_p_plus_1():
    nodes = -np.arange(4.0)
    w = O.lagrange_weights(nodes, 1.0)
    # degree-4 monomial: Lagrange error = prod (tau - t_j) = 1*2*3*4 = 24
    assert (w * nodes ** 4).sum() == pytest.approx(1.0 - 24.0, abs=1e-12)


# -------------------------------------------------------------- Eq. 5 ------
def test_controller_constants_and_properties():
    g = json.load(open(os.path.join(GOLDEN, "controller_constants.json")))
    emax = g["e_max"]
    for n in [2, 3, 4, 5]:
        # fixed point: an error of exactly safety*e_max keeps h
        assert O.controller_factor(g["safety"] * emax, emax, n, g["cmin"], g["cmax"]) == pytest.approx(1.0)
        # an error 2^(n+1) times larger halves the step
        e = g["safety"] * emax * 1.5 ** -(n + 1)
        c1 = O.controller_factor(e, emax, n, g["cmin"], g["cmax"])
        c2 = O.controller_factor(e * 2 ** (n + 1), emax, n, g["cmin"], g["cmax"])
        assert c1 == pytest.approx(1.5) and c2 == pytest.approx(c1 / 2)
        assert O.controller_factor(0.0, emax, n, g["cmin"], g["cmax"]) == g["cmax"]
        assert O.controller_factor(1e30, emax, n, g["cmin"], g["cmax"]) == g["cmin"]
        es = np.logspace(-12, 2, 50)
        cs = [O.controller_factor(e, emax, n, g["cmin"], g["cmax"]) for e in es]
        assert all(x >= y for x, y in zip(cs, cs[1:]))


# -------------------------------------------------------- field terms ------
def test_rhs_is_orthogonal_to_m_and_zero_for_parallel_field():
    rng = np.random.default_rng(0)
    m = rng.normal(size=(3, 2, 3, 4))
    m /= np.linalg.norm(m, axis=0)
    H = rng.normal(size=m.shape) * 1e5
    F = O.llg_rhs(2.211e5, 0.1, m, H)
    assert np.abs((m * F).sum(axis=0)).max() < 1e-9 * np.abs(F).max()
    F0 = O.llg_rhs(2.211e5, 0.1, m, 3.0 * m)
    assert np.abs(F0).max() < 1e-15 * 2.211e5 * 3.0 * 10
    # |F| = gamma/(1+a^2) |m x H| sqrt(1 + a^2) for unit m
    a = 0.3
    F = O.llg_rhs(2.0, a, m, H)
    cross = np.cross(m, H, axis=0)
    assert np.allclose(np.linalg.norm(F, axis=0),
                       2.0 / np.sqrt(1 + a * a) * np.linalg.norm(cross, axis=0), rtol=1e-12)


def test_exchange_closed_forms():
    n = (6, 5, 3)
    d = (2e-9, 3e-9, 1e-9)
    mesh = {"n": n, "d": d}
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": 0.0, "gamma": 1.0}
    cex = 2 * 1.3e-11 / (W.MU0 * 8e5)
    u = np.ones((3,) + n[::-1]) / np.sqrt(3)
    assert np.abs(O.exchange_anisotropy(mesh, mat, u)).max() < 1e-6
    # quadratic profile along y: interior Laplacian = 2*q/dy^2
    y = np.arange(n[1], dtype=float)
    m = np.zeros((3,) + n[::-1])
    m[0] = (0.01 * y ** 2)[None, :, None]
    H = O.exchange_anisotropy(mesh, mat, m)
    assert np.allclose(H[0][:, 1:-1, :], cex * 0.02 / d[1] ** 2, rtol=1e-12)
    # free boundary: the missing neighbour is the cell itself
    assert np.allclose(H[0][:, 0, :], cex * (m[0][:, 1, :] - m[0][:, 0, :]) / d[1] ** 2, rtol=1e-12)
    # self-adjointness: sum a.L(b) = sum b.L(a)
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=(2, 3) + n[::-1])
    la, lb = O.exchange_anisotropy(mesh, mat, a), O.exchange_anisotropy(mesh, mat, b)
    assert (a * lb).sum() == pytest.approx((b * la).sum(), rel=1e-12)


def test_anisotropy_closed_form():
    mesh = {"n": (1, 1, 1), "d": (1e-9, 1e-9, 1e-9)}
    ku = np.array([0.6, 0.8, 0.0])
    mat = {"Ms": 5e5, "A": 0.0, "K": 4e4, "ku": tuple(ku), "alpha": 0.0, "gamma": 1.0}
    m = np.array([0.0, 0.6, 0.8]).reshape(3, 1, 1, 1)
    H = O.exchange_anisotropy(mesh, mat, m).ravel()
    assert np.allclose(H, 2 * 4e4 / (W.MU0 * 5e5) * 0.48 * ku, rtol=1e-14)


def test_applied_field_pulse_window():
    f = {"H0": (1.0, 2.0, 3.0), "pulse": (0.0, 10.0, 0.0), "t_on": 1e-12, "t_off": 2e-12}
    mesh = {"n": (1, 1, 1), "d": (1, 1, 1)}
    mat = {"Ms": 1.0, "alpha": 0.0, "gamma": 1.0}
    assert np.allclose(O.applied_field(mesh, mat, f, 0.5e-12), [1, 2, 3])
    assert np.allclose(O.applied_field(mesh, mat, f, 1e-12), [1, 12, 3])
    assert np.allclose(O.applied_field(mesh, mat, f, 2e-12), [1, 2, 3])


# ---------------------------------------------------- whole integrator ----
def macrospin_exact(m0, gamma, alpha, Hz, t):
    gp = gamma / (1 + alpha * alpha)
    th0 = np.arccos(m0[2])
    ph0 = np.arctan2(m0[1], m0[0])
    mz = np.tanh(gp * alpha * Hz * t + np.arctanh(np.cos(th0)))
    ph = ph0 + gp * Hz * t
    st = np.sqrt(1 - mz * mz)
    return np.array([st * np.cos(ph), st * np.sin(ph), mz])


@pytest.mark.parametrize("method,p", [("RK4", -1), ("RK4", 3), ("RKDP54", -1), ("RKDP54", 4),
                                      ("RK23", 2), ("RKF45", 4), ("RKF56", 5), ("HEUN12", -1)])
def test_macrospin_matches_analytic_solution(method, p):
    """A single cubic cell feels a self field parallel to m, so it precesses
    in the applied field exactly as the analytic Landau-Lifshitz solution."""
    m0 = np.array([0.8, 0.0, -0.6])
    Hz = 1e5
    gamma, alpha = 2.211e5, 0.1
    mesh = {"n": (1, 1, 1), "d": (3e-9, 3e-9, 3e-9)}
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": alpha, "gamma": gamma}
    fld = {"H0": (0.0, 0.0, Hz)}
    h = 2e-14 if method != "HEUN12" else 1e-15
    sim = O.Simulation(mesh, mat, fld, {"method": method, "extrap_order": p, "adaptive": False, "h": h},
                       m0.reshape(3, 1, 1, 1))
    t_end = 50e-12
    sim.run(t_end)
    got = sim.m().ravel()
    ref = macrospin_exact(m0, gamma, alpha, Hz, t_end)
    tol = 1e-9 if method != "HEUN12" else 1e-6
    assert np.abs(got - ref).max() < tol
    st = sim.stats()
    assert st["t"] == t_end


def _energy(mesh, mat, fld, N6, m):
    """E/(mu0 V Ms) = -sum m.(H_app + H_d/2 + (H_ex + H_an)/2)."""
    Ha = np.array(fld["H0"]).reshape(3, 1, 1, 1)
    Hd = O.demag_fft(N6, mat["Ms"], m)
    He = O.exchange_anisotropy(mesh, mat, m)
    return -(m * (Ha + 0.5 * Hd + 0.5 * He)).sum()


def test_energy_decreases_with_damping_and_is_conserved_without():
    n, d = (8, 6, 2), (4e-9, 4e-9, 4e-9)
    mesh = {"n": n, "d": d}
    fld = {"H0": tuple(W.mT((10.0, -5.0, 0.0)))}
    N6 = O.newell_octant(*n, *d)
    m0 = W.m_smooth(n, seed=3)
    for alpha in [0.5, 0.0]:
        mat = {"Ms": 8e5, "A": 1.3e-11, "K": 2e4, "ku": (0.0, 1.0, 0.0), "alpha": alpha,
               "gamma": W.GAMMA}
        sim = O.Simulation(mesh, mat, fld, {"method": "RK4", "extrap_order": -1, "adaptive": False,
                                            "h": 2e-14}, m0, N6=N6)
        E = [_energy(mesh, mat, fld, N6, m0)]
        for k in range(1, 21):
            sim.run(k * 1e-12)
            E.append(_energy(mesh, mat, fld, N6, sim.m()))
        E = np.array(E)
        if alpha > 0:
            assert np.all(np.diff(E) < 0)
            assert E[-1] < E[0] - 1e-3 * abs(E[0])
        else:
            assert np.abs(E - E[0]).max() < 1e-7 * abs(E[0])


CONV_N, CONV_D = (8, 8, 2), (4e-9, 4e-9, 4e-9)


@pytest.fixture(scope="module")
def conv_problem():
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": 0.02, "gamma": W.GAMMA}
    fld = {"H0": tuple(W.mT((-24.6, 4.3, 0.0)))}
    N6 = O.newell_octant(*CONV_N, *CONV_D)
    return mat, fld, N6, W.m_smooth(CONV_N, seed=1)


def _slopes(conv_problem, method, p, h0=0.4e-12, T=10e-12):
    mat, fld, N6, m0 = conv_problem

    def run(pp, h):
        s = O.Simulation({"n": CONV_N, "d": CONV_D}, mat, fld,
                         {"method": method, "extrap_order": pp, "adaptive": False, "h": h}, m0, N6=N6)
        s.run(T)
        return s.m()

    ref = run(-1, h0 / 64)
    errs = [np.abs(run(p, h0 / 2 ** k) - ref).max() for k in range(1, 4)]
    return [np.log2(errs[i] / errs[i + 1]) for i in range(2)]


@pytest.mark.parametrize("method,p,expect", [
    ("RK4", -1, 4), ("RK4", 3, 4), ("RK4", 2, 3), ("RK4", 1, 2), ("RK4", 0, 1),
    ("RKDP54", -1, 5), ("RKDP54", 4, 5), ("RKDP54", 3, 4),
    ("RK23", -1, 3), ("RK23", 2, 3),
    ("RKF45", -1, 4), ("RKF45", 4, 4),
])
def test_convergence_order_is_min_of_method_and_extrapolation(conv_problem, method, p, expect):
    """Sec. II after Eq. 6: an order-p extrapolation has error O(h^(p+1)),
    so the global order is min(n, p+1)."""
    sl = _slopes(conv_problem, method, p)
    assert sl[-1] == pytest.approx(expect, abs=0.3)


def test_single_cell_extrapolated_equals_full():
    # on a 1x1x1 mesh the non-self field G vanishes, so Eq. 6 is exact
    m0 = np.array([0.36, 0.48, 0.8]).reshape(3, 1, 1, 1)
    mesh = {"n": (1, 1, 1), "d": (2e-9, 3e-9, 1e-9)}
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": 0.05, "gamma": W.GAMMA}
    fld = {"H0": (2e4, -1e4, 5e3)}
    # (a non-FSAL method: FSAL reuse in full mode is a different, valid path)
    for method, ps in [("RKF45", [-1, 4, 0]), ("RKDP54", [4, 1])]:
        out = []
        for p in ps:
            s = O.Simulation(mesh, mat, fld, {"method": method, "extrap_order": p, "adaptive": True,
                                              "h": 1e-13, "tol": 1e-6}, m0)
            s.run(20e-12)
            out.append(s.m().ravel())
        for o in out[1:]:
            assert np.abs(out[0] - o).max() < 1e-13


# ------------------------------------------ cells without material (R11) --
@pytest.mark.parametrize("method,p", [("RKDP54", 4), ("RK4", -1), ("RKF56", 5)])
def test_one_particle_in_vacuum_equals_the_single_cell_mesh(method, p):
    """A magnetic cell surrounded by cells with m = 0 (no material) moves
    exactly like the same cell alone on a 1 x 1 x 1 mesh: the empty cells
    add nothing to its demag sum (only the self term remains), their m = 0
    in its exchange stencil only adds a field parallel to m (no torque), and
    they stay exactly 0 themselves."""
    mesh1 = {"n": (1, 1, 1), "d": (4e-9, 4e-9, 4e-9)}
    mesh4 = {"n": (4, 4, 1), "d": (4e-9, 4e-9, 4e-9)}
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 5e4, "ku": (1.0, 0.0, 0.0), "alpha": 0.05, "gamma": W.GAMMA}
    fld = {"H0": (2e4, -1e4, 5e3)}
    mc = np.array([0.36, 0.48, 0.8])
    m1 = mc.reshape(3, 1, 1, 1)
    m4 = np.zeros((3, 1, 4, 4))
    m4[:, 0, 2, 1] = mc
    integ = {"method": method, "extrap_order": p, "adaptive": method != "RK4", "h": 1e-13, "tol": 1e-6}
    a = O.Simulation(mesh1, mat, fld, integ, m1)
    b = O.Simulation(mesh4, mat, fld, integ, m4)
    a.run(10e-12)
    b.run(10e-12)
    ma, mb = a.m(), b.m()
    assert a.stats()["accepted"] == b.stats()["accepted"]
    assert np.abs(mb[:, 0, 2, 1] - ma[:, 0, 0, 0]).max() < 1e-12
    mb[:, 0, 2, 1] = 0.0
    assert np.all(mb == 0.0)
    # the particle did move
    assert np.abs(ma[:, 0, 0, 0] - mc).max() > 1e-2


def test_checkerboard_particles_keep_the_vacuum_empty_and_unit_length():
    """The checkerboard stand-in (2 x 2-cell particles on alternate squares,
    no exchange): after 5 ps the empty squares are still exactly 0 and the
    particle cells unit vectors; with the array's dipolar coupling the
    particles' states differ from the uncoupled single-particle motion."""
    n = (8, 8, 1)
    mesh = {"n": n, "d": (5e-9, 5e-9, 5e-9)}
    mat = {"Ms": 8e5, "A": 0.0, "K": 0.0, "alpha": 0.02, "gamma": W.GAMMA}
    fld = {"H0": (20e3, 1e3, 0.0)}
    mask = W.checkerboard_mask(n, 2)
    m0 = W.m_uniform_noise(n, direction=(0.0, 1.0, 0.0), noise=0.05, seed=3) * mask
    s = O.Simulation(mesh, mat, fld, {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13,
                                      "tol": 1e-6}, m0)
    s.run(5e-12)
    m = s.m()
    assert np.all(m[:, mask[0] == 0] == 0.0)
    r = np.linalg.norm(m, axis=0)[mask[0] == 1]
    assert np.abs(r - 1.0).max() < 1e-12
    assert np.abs(m - m0).max() > 1e-3


def test_adaptive_controller_rejects_and_tracks_tolerance():
    n, d = (8, 8, 1), (4e-9, 4e-9, 4e-9)
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": 0.02, "gamma": W.GAMMA}
    fld = {"H0": tuple(W.mT((-24.6, 4.3, 0.0)))}
    N6 = O.newell_octant(*n, *d)
    m0 = W.m_uniform_noise(n, seed=0, noise=0.3)
    ref = O.Simulation({"n": n, "d": d}, mat, fld, {"method": "RKDP54", "extrap_order": -1,
                                                    "adaptive": False, "h": 5e-15}, m0, N6=N6)
    ref.run(20e-12)
    errs = []
    for tol in [1e-4, 1e-6]:
        s = O.Simulation({"n": n, "d": d}, mat, fld, {"method": "RKDP54", "extrap_order": 4,
                                                      "adaptive": True, "h": 1e-12, "tol": tol}, m0, N6=N6)
        s.run(20e-12)
        st = s.stats()
        assert st["rejected"] >= 1  # a 1 ps first step is far too large
        assert st["t"] == 20e-12
        attempts = st["accepted"] + st["rejected"]
        # stage 1 once per step start, stages 2..7 once per attempt
        assert st["exact_evals"] + st["extrap_evals"] == attempts * 6 + st["accepted"]
        assert st["exact_evals"] < st["extrap_evals"]
        errs.append(np.abs(s.m() - ref.m()).max())
    assert errs[1] < errs[0] / 10


def test_forced_accept_at_hmin():
    n, d = (4, 4, 1), (4e-9, 4e-9, 4e-9)
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "alpha": 0.02, "gamma": W.GAMMA}
    m0 = W.m_random(n, seed=5)
    s = O.Simulation({"n": n, "d": d}, mat, {"H0": (0, 0, 0)},
                     {"method": "RK23", "extrap_order": -1, "adaptive": True, "h": 1e-13, "tol": 1e-30,
                      "hmin": 1e-13}, m0)
    s.run(1e-12)
    st = s.stats()
    assert st["forced"] == st["accepted"] == 10 and st["rejected"] == 0


def test_epsilon_metric():
    a = W.m_random((3, 2, 1), seed=1)
    assert O.epsilon(a, a) == 0.0
    b = a.copy()
    b[:, 0, 0, 0] = -a[:, 0, 0, 0]
    assert O.epsilon(a, b) == pytest.approx(2.0 / 6)


def test_epsilon_over_time_samples():
    """Eq. 7 with time samples of <m> as its points: zero for equal
    histories; a constant offset d gives |d|; one differing sample out of S
    gives |difference| / S; the sample counts must agree."""
    rng = np.random.default_rng(3)
    mbar = rng.uniform(-1, 1, size=(3, 40))
    assert O.epsilon_time(mbar, mbar) == 0.0
    d = np.array([3e-3, -4e-3, 0.0])
    assert O.epsilon_time(mbar + d.reshape(3, 1), mbar) == pytest.approx(5e-3, rel=1e-12)
    other = mbar.copy()
    other[:, 7] += np.array([0.0, 0.0, 0.2])
    assert O.epsilon_time(other, mbar) == pytest.approx(0.2 / 40, rel=1e-12)
    with pytest.raises(ValueError):
        O.epsilon_time(mbar, mbar[:, :39])


# ------------------------------------------------------ ABM2 (reading R10) --
ABM_N, ABM_D = (6, 4, 2), (4e-9, 4e-9, 4e-9)
ABM_MAT = {"Ms": 8e5, "A": 1.3e-11, "K": 3e4, "ku": (0.0, 1.0, 0.0), "alpha": 0.05, "gamma": W.GAMMA}
ABM_FLD = {"H0": tuple(W.mT((-20.0, 6.0, 3.0)))}


def _field_rhs(N6, t, m):
    """F(t, m) of Eq. 1 assembled from the separately pinned field terms."""
    mesh = {"n": ABM_N, "d": ABM_D}
    H = (O.demag_fft(N6, ABM_MAT["Ms"], m) + O.exchange_anisotropy(mesh, ABM_MAT, m)
         + O.applied_field(mesh, ABM_MAT, ABM_FLD, t).reshape(3, 1, 1, 1))
    return O.llg_rhs(ABM_MAT["gamma"], ABM_MAT["alpha"], m, H)


def _abm_run(method, h, t_end, N6, m0):
    s = O.Simulation({"n": ABM_N, "d": ABM_D}, ABM_MAT, ABM_FLD,
                     {"method": method, "extrap_order": -1, "adaptive": False, "h": h}, m0, N6=N6)
    s.run(t_end)
    out = s.m(), s.stats()
    s.close()
    return out


def test_abm2_first_step_is_heun():
    """With no previous derivative the AB2 predictor is an Euler step, and
    Euler predictor + trapezoidal corrector is Heun's method."""
    N6 = O.newell_octant(*ABM_N, *ABM_D)
    m0 = W.m_smooth(ABM_N, seed=5)
    h = 5e-14
    a, sa = _abm_run("ABM2", h, h, N6, m0)
    b, sb = _abm_run("HEUN12", h, h, N6, m0)
    assert np.abs(a - b).max() < 1e-15
    assert sa["last_err"] == pytest.approx(sb["last_err"], rel=1e-12)


def test_abm2_steps_are_adams_bashforth_predictor_and_trapezoid_corrector():
    """Steps 2 and 3 (the third clipped to half a step, w = 1/2) rebuilt from
    the field terms: P = m + h [(1 + w/2) F_n - (w/2) F_(n-1)], then
    m + h/2 [F_n + F(t + h, P)], renormalised."""
    N6 = O.newell_octant(*ABM_N, *ABM_D)
    m0 = W.m_smooth(ABM_N, seed=6)
    h = 5e-14
    m1, _ = _abm_run("ABM2", h, h, N6, m0)
    F0 = _field_rhs(N6, 0.0, m0)

    def step(m, t, hh, F_n, F_prev, w):
        P = m + hh * ((1 + w / 2) * F_n - (w / 2) * F_prev)
        M = m + hh / 2 * (F_n + _field_rhs(N6, t + hh, P))
        return M / np.linalg.norm(M, axis=0, keepdims=True), np.linalg.norm(M - P, axis=0).max()  # R4

    F1 = _field_rhs(N6, h, m1)
    m2, _ = step(m1, h, h, F1, F0, 1.0)
    got2, _ = _abm_run("ABM2", h, 2 * h, N6, m0)
    assert np.abs(got2 - m2).max() < 1e-14
    F2 = _field_rhs(N6, 2 * h, m2)
    m3, e3 = step(m2, 2 * h, h / 2, F2, F1, 0.5)
    got3, st3 = _abm_run("ABM2", h, 2.5 * h, N6, m0)
    assert np.abs(got3 - m3).max() < 1e-14
    assert st3["accepted"] == 3 and st3["last_err"] == pytest.approx(e3, rel=1e-9)


@pytest.mark.parametrize("p,expect", [(-1, 2), (1, 2), (0, 1)])
def test_abm2_convergence_order(conv_problem, p, expect):
    """ABM2 is second order; with extrapolation of order p the global order
    is min(2, p + 1) (Sec. II after Eq. 6)."""
    sl = _slopes(conv_problem, "ABM2", p)
    assert sl[-1] == pytest.approx(expect, abs=0.3)


def test_abm2_two_evaluations_per_step_and_adaptive_run():
    """Two right-hand-side evaluations per attempt (Sec. III: 2 sub-steps),
    one exact demag and one Eq. 6 extrapolation once primed; the adaptive
    controller keeps the error at or below e_max."""
    N6 = O.newell_octant(*ABM_N, *ABM_D)
    m0 = W.m_smooth(ABM_N, seed=7)
    s = O.Simulation({"n": ABM_N, "d": ABM_D}, ABM_MAT, ABM_FLD,
                     {"method": "ABM2", "extrap_order": 1, "adaptive": True, "h": 1e-13, "tol": 1e-5},
                     m0, N6=N6)
    s.run(20e-12)
    st = s.stats()
    s.close()
    att = st["accepted"] + st["rejected"]
    assert st["exact_evals"] + st["extrap_evals"] == 2 * att - st["rejected"]
    # every attempt after priming (the first accepted step and the
    # rejections before it run in full mode) extrapolates its second field
    assert att - 1 - st["rejected"] <= st["extrap_evals"] <= att - 1
    assert st["last_err"] <= 1e-5
    assert st["t"] == pytest.approx(20e-12, rel=1e-15)
