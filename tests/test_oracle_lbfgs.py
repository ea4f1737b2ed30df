"""Pins of the optimiser: Algorithm 1 against the paper's H_k formula, and P7."""
import numpy as np
import scipy.optimize as so

from oracle import lbfgs as L


def test_two_loop_equals_product_formula_and_secant():
    rng = np.random.default_rng(0)
    n = 7
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + np.eye(n)
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(n)
        pairs.append((s, A @ s))
    h0 = float(pairs[-1][0] @ pairs[-1][1] / (pairs[-1][1] @ pairs[-1][1]))
    g = rng.standard_normal(n)
    Hm = L.hessian_product_form(pairs, h0, n)
    assert np.abs(L.two_loop(g, pairs, h0) - Hm @ g).max() <= 1e-13 * np.abs(Hm @ g).max()
    # secant equation of the newest pair: H_k phi_{k-1} = varkappa_{k-1}
    assert np.abs(L.two_loop(pairs[-1][1], pairs, h0) - pairs[-1][0]).max() <= 1e-13


def _quad(seed=0, n=50):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T / n + 0.3 * np.eye(n)
    b = rng.standard_normal(n)
    lo = np.full(n, -0.3)
    hi = np.full(n, 0.4)
    lo[::7] = -np.inf
    f = lambda x: 0.5 * x @ A @ x - b @ x
    fg = lambda x: (f(x), A @ x - b)
    return A, b, lo, hi, f, fg


def test_p7_matches_scipy_lbfgsb_and_kkt():
    A, b, lo, hi, f, fg = _quad()
    ref = so.minimize(fg, np.zeros(50), jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                      options=dict(ftol=1e-16, gtol=1e-14, maxiter=5000)).x
    for mem in (20, 0):
        res = L.projected_lbfgs(f, fg, np.zeros(50), lo, hi, np.full(50, 2.0), mem=mem,
                                max_iter=2000, rtol=0.0)
        x = res.x
        assert np.abs(x - ref).max() < 1e-6
        g = A @ x - b
        free = (x > lo) & (x < hi)
        assert np.abs(g[free]).max() < 1e-6
        assert np.all(g[x <= lo] >= -1e-9) and np.all(g[x >= hi] <= 1e-9)


def test_line_search_failure_stops_and_reports():
    A, b, lo, hi, f, fg = _quad(1, 10)
    calls = []

    def bad(x):  # every trial point is worse: the search must fail and reset
        calls.append(1)
        return f(x) + 1e6

    res = L.projected_lbfgs(bad, fg, np.zeros(10), lo[:10], hi[:10], np.ones(10), max_iter=5)
    assert res.stopped == "line_search"
    assert res.history[-1]["alpha"] == 0.0
    assert len(calls) == 2 * 21      # the first direction and the reset, 21 trials each


def test_projection():
    z = np.array([-2.0, 0.5, 3.0])
    assert np.all(L.project(z, np.array([-1.0, 0, 0]), np.array([1.0, 1, 2])) == [-1.0, 0.5, 2.0])


def test_p7_reaches_the_exact_kkt_point():
    """The box-constrained quadratic's minimiser in closed form: with the active set of the
    solution, the free components solve A_ff x_f = b_f - A_fa x_a.  The projected gradient
    (l = 0) reaches it to rounding; with l = 20 the Armijo test on J stops the iteration where
    J's decrease falls below its rounding (x then within about 1e-8 of the minimiser, as is
    scipy's L-BFGS-B)."""
    A, b, lo, hi, f, fg = _quad()
    ref = so.minimize(fg, np.zeros(50), jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                      options=dict(ftol=1e-16, gtol=1e-14, maxiter=5000)).x
    act_lo, act_hi = ref <= lo + 1e-12, ref >= hi - 1e-12
    free = ~(act_lo | act_hi)
    x_star = np.where(act_lo, lo, np.where(act_hi, hi, 0.0))
    x_star[free] = np.linalg.solve(A[np.ix_(free, free)], b[free] - A[np.ix_(free, ~free)] @ x_star[~free])
    g = A @ x_star - b                    # KKT signs of the closed-form point
    assert np.abs(g[free]).max() < 1e-12
    assert np.all(g[act_lo] >= 0) and np.all(g[act_hi] <= 0)
    assert np.abs(ref - x_star).max() < 1e-7
    for mem, tol in ((0, 1e-11), (20, 1e-7)):
        res = L.projected_lbfgs(f, fg, np.zeros(50), lo, hi, np.full(50, 2.0), mem=mem, max_iter=2000, rtol=0.0)
        assert np.abs(res.x - x_star).max() < tol, (mem, np.abs(res.x - x_star).max())
