"""GPU parity of the matrix-free equilibration (cone_problem_equilibrate)
against the FP64 oracle (oracle/equil.py), through the C ABI, on both solver
programs.

* the scalings D, E, sigma, rho agree with the oracle's (same iterations,
  probes and seed; the random signs come from each side's own SplitMix64);
* the first 20 iterates of the equilibrated iteration agree with the
  oracle's within 1e-5 (relative l2, scaled coordinates);
* equilibrated solves return points of the original problem: FP64-rechecked
  residuals <= 1e-4, objectives within 1e-4 of an independent optimum, and
  the certificates of infeasible / unbounded problems;
* on the small deconvolution the equilibrated iteration stops at 1e-4 in far
  fewer iterations than the plain one.
"""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import cones, equil, linop, scs
from paper_1609_03488_b300 import synth
from tests.helpers import fp32_conv_trajectory, fp64_residuals, objective_rel_err, rel

pytestmark = pytest.mark.gpu
ENGINES = ["graph", "team", "grid"]
EQ = dict(iters=10, probes=8, seed=0x5EED)


@pytest.fixture(scope="module")
def B():
    from paper_1609_03488_b300 import build
    build.build()
    from paper_1609_03488_b300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


FAMILIES = {
    "deconv": lambda: synth.deconv(n_x=300, L=30, seed=synth.BASE_SEED + 1),
    # 304 padded taps: the graph engine evaluates the convolution by FFTs
    # with the scalings folded in; a narrow kernel and the generator's own
    # sigma = L/10
    "deconv_fft": lambda: synth.deconv(n_x=3000, L=300, sigma=3.0, seed=synth.BASE_SEED + 1),
    "deconv_fft_wide": lambda: synth.deconv(n_x=3000, L=300, seed=synth.BASE_SEED + 1),
    # the same wide kernel (sigma = L/10) evaluated by the direct sum
    "deconv_direct_wide": lambda: _direct(synth.deconv(n_x=3000, L=300, seed=synth.BASE_SEED + 1)),
    "lasso_fp8": lambda: synth.lasso(m_d=301, p=151, seed=synth.BASE_SEED + 3, storage="fp8"),
    "lp_bf16": lambda: synth.lp(m_d=301, n_x=151, density=0.05, seed=synth.BASE_SEED + 4, storage="bf16"),
    "mixed": lambda: synth.mixed_cone_problem(np.random.default_rng(402), n=8, soc_sizes=(3, 1, 5), z=2, l=4),
}


def _direct(prob):
    return dict(prob, A=synth.with_conv_method(prob["A"], "direct"))


def _eq_problem(B, ctx, prob):
    P = B.cone_problem_create(ctx, prob)
    B.equilibrate(P, **EQ)
    return P


@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_scalings_match_oracle(B, ctx, family):
    prob = FAMILIES[family]()
    P = _eq_problem(B, ctx, prob)
    D, E, sigma, rho = B.scaling(P)
    ref = equil.equilibrate(scs.Operator(prob["A"]), prob["cone"], prob["b"], prob["c"], **EQ)
    assert rel(D, ref["D"]) <= 1e-4 and rel(E, ref["E"]) <= 1e-4, (rel(D, ref["D"]), rel(E, ref["E"]))
    assert sigma == pytest.approx(ref["sigma"], rel=1e-4) and rho == pytest.approx(ref["rho"], rel=1e-4)
    for lo, hi in equil.soc_blocks(prob["cone"]):
        assert np.all(D[lo:hi] == D[lo])


_CONV_BAR = {}


def _conv_bar(family, prob):
    """Per-iterate bar of a wide-kernel family: the larger of 1e-5 and twice
    how far float32 rounding of the convolution alone (scipy's
    single-precision FFT, or a float32 direct sum, in the FP64 oracle) moves
    that iterate (tests/test_conv_rounding.py)."""
    if family not in _CONV_BAR:
        method = "direct" if "direct" in family else "fft"
        exact, pert = fp32_conv_trajectory(prob, 20, method, equilibrate=EQ)
        _CONV_BAR[family] = [max(1e-5, 2 * rel(pert["traj_u"][k], exact["traj_u"][k]),
                                 2 * rel(pert["traj_v"][k], exact["traj_v"][k])) for k in range(20)]
    return _CONV_BAR[family]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_equilibrated_trajectory_matches_oracle(B, ctx, family, engine):
    prob = FAMILIES[family]()
    ref = scs.problem_solve(prob, max_iters=20, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3,
                            trajectory=20, equilibrate=EQ)
    bar = _conv_bar(family, prob) if family.startswith(("deconv_fft", "deconv_direct")) else [1e-5] * 20
    P = _eq_problem(B, ctx, prob)
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for k in (1, 5, 20):
        st = B.settings(max_iters=k, check_interval=10 ** 6, cg_fixed_iters=3, engine=engine)
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        eu = rel(uv[:N], ref["traj_u"][k - 1])
        ev = rel(uv[N:], ref["traj_v"][k - 1])
        assert eu <= bar[k - 1] and ev <= bar[k - 1], (family, engine, k, eu, ev, bar[k - 1])


@pytest.mark.parametrize("engine", ENGINES)
def test_equilibrated_solutions(B, ctx, engine):
    # small deconvolution against NNLS; LP against HiGHS; lasso and mixed
    # cones against the oracle's FP64 optimum (unequilibrated)
    dec = synth.deconv(n_x=1000, L=100, seed=synth.BASE_SEED + 1)
    K = linop.densify(dec["A"]["parts"][2]["parts"][0]["parts"][0])
    _, nnls = so.nnls(K, dec["meta"]["b_obs"], maxiter=50000)
    lp = synth.lp(m_d=300, n_x=150, density=0.05, seed=synth.BASE_SEED + 4)
    Dl = linop.densify(lp["A"]["parts"][0])
    hi = so.linprog(lp["c"], A_ub=Dl, b_ub=lp["b"][:300], bounds=(0, None), method="highs").fun
    las = synth.lasso(m_d=400, p=200, seed=synth.BASE_SEED + 3, storage="bf16")
    mix = synth.mixed_cone_problem(np.random.default_rng(403), n=8, soc_sizes=(3, 1, 5), z=2, l=4)
    cases = [(dec, nnls, 2e-5), (lp, hi, 1e-5),
             (las, scs.problem_solve(las, eps=1e-9, max_iters=200000)["pobj"], 1e-5),
             (mix, scs.problem_solve(mix, eps=1e-10, max_iters=400000)["pobj"], 1e-5)]
    for prob, p_star, eps in cases:
        P = _eq_problem(B, ctx, prob)
        info, x, y, s = B.solve(P, B.settings(eps=eps, max_iters=300000, engine=engine))
        assert info["status_name"] == "solved", info
        assert max(fp64_residuals(prob, x, y, s)) <= 1e-4, fp64_residuals(prob, x, y, s)
        assert objective_rel_err(prob["c"] @ x, p_star) <= 1e-4, (prob["c"] @ x, p_star)
        assert info["pobj"] == pytest.approx(prob["c"] @ x, rel=1e-5, abs=1e-7)
        assert cones.dist_to_cone(s, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(s))
        assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(y))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("kind", ["infeasible", "unbounded"])
def test_equilibrated_certificates(B, ctx, engine, kind):
    rng = np.random.default_rng(201 if kind == "infeasible" else 301)
    D, b_d, c = synth.random_tiny_lp(rng, 3, 3, kind)
    prob = synth.dense_lp(D, b_d, c)
    P = _eq_problem(B, ctx, prob)
    info, x, y, s = B.solve(P, B.settings(eps=1e-5, eps_infeas=1e-5, engine=engine))
    assert info["status_name"] == kind, info
    A = linop.densify(prob["A"])
    if kind == "infeasible":
        assert abs(prob["b"] @ y + 1.0) < 1e-5
        assert np.linalg.norm(A.T @ y) <= 1e-4
        assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-6
    else:
        assert abs(prob["c"] @ x + 1.0) < 1e-5
        assert np.linalg.norm(A @ x + s) <= 1e-4
        assert cones.dist_to_cone(s, prob["cone"]) <= 1e-5


@pytest.mark.parametrize("engine", ENGINES)
def test_equilibration_cuts_the_small_deconvolution_iterations(B, ctx, engine):
    prob = synth.deconv(n_x=1000, L=100, seed=synth.BASE_SEED + 1)
    plain = B.solve(B.cone_problem_create(ctx, prob), B.settings(eps=1e-4, engine=engine))[0]
    eqd = B.solve(_eq_problem(B, ctx, prob), B.settings(eps=1e-4, engine=engine))[0]
    ref = scs.problem_solve(prob, eps=1e-4, max_iters=100000, linsys="cg", equilibrate=EQ)
    assert plain["status_name"] == eqd["status_name"] == "solved"
    assert eqd["iters"] * 4 < plain["iters"], (eqd["iters"], plain["iters"])
    assert abs(eqd["iters"] - ref["iters"]) <= 2 * 10, (eqd["iters"], ref["iters"])


@pytest.mark.parametrize("method", ["direct", "fft"])
def test_equilibrated_fft_deconvolution_solution(B, ctx, method):
    """The scaled FFT convolution inside a whole solve: n = 2000, L = 400,
    against scipy's NNLS; both evaluation methods reach it."""
    prob = synth.deconv(n_x=2000, L=400, seed=synth.BASE_SEED + 9)
    prob["A"] = synth.with_conv_method(prob["A"], method)
    K = linop.densify(prob["A"]["parts"][2]["parts"][0]["parts"][0])
    _, nnls = so.nnls(K, prob["meta"]["b_obs"], maxiter=50000)
    P = _eq_problem(B, ctx, prob)
    info, x, y, s = B.solve(P, B.settings(eps=2e-5, max_iters=300000, engine="graph"))
    assert info["status_name"] == "solved", info
    assert max(fp64_residuals(prob, x, y, s)) <= 1e-4, fp64_residuals(prob, x, y, s)
    assert objective_rel_err(prob["c"] @ x, nnls) <= 1e-4, (prob["c"] @ x, nnls)


def test_equilibrate_arguments_and_state(B, ctx):
    P = B.cone_problem_create(ctx, synth.lp(m_d=50, n_x=25, density=0.1, seed=3))
    for bad in (dict(iters=-1), dict(iters=101), dict(probes=0), dict(probes=2000)):
        with pytest.raises(B.CfError) as e:
            B.equilibrate(P, **{**EQ, **bad})
        assert e.value.code == B.CF_E_INVALID
    D, E, sg, rh = B.scaling(P)
    assert np.all(D == 1) and np.all(E == 1) and sg == rh == 1.0
    B.equilibrate(P, **EQ)
    with pytest.raises(B.CfError) as e:
        B.equilibrate(P, **EQ)
    assert e.value.code == B.CF_E_STATE


def test_equilibrated_batch_equals_solo(B, ctx):
    probs = [synth.lp(m_d=m, n_x=m // 2, density=0.03, seed=50 + m, storage="bf16") for m in (120, 250, 400, 700)]
    probs.append(synth.deconv(n_x=400, L=40, seed=7))
    Ps = [_eq_problem(B, ctx, p) for p in probs]
    st = B.settings(engine="team")
    solo = [B.solve(P, st) for P in Ps]
    infos, xs, ys, ss = B.solve_batch(Ps, st)
    for (i0, x0, y0, s0), i1, x1, y1, s1, prob in zip(solo, infos, xs, ys, ss, probs):
        assert i0["iters"] == i1["iters"] and i1["status_name"] == "solved"
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(y0, y1)
        np.testing.assert_array_equal(s0, s1)
        assert max(fp64_residuals(prob, x1, y1, s1)) <= 1e-4


@pytest.mark.parametrize("engine", ["auto", "graph"])
def test_equilibrated_serving_equals_solo(B, ctx, engine):
    rng = np.random.default_rng(78)
    probs = [synth.deconv(n_x=300, L=30, seed=1), synth.lasso(m_d=300, p=150, seed=2, storage="bf16"),
             synth.lp(m_d=200, n_x=100, density=0.05, seed=3), synth.mixed_cone_problem(rng),
             synth.lp(m_d=500, n_x=250, density=0.02, seed=5, storage="bf16")]
    Ps = [_eq_problem(B, ctx, p) for p in probs]
    st = B.settings(engine=engine)
    solo = [B.solve(P, st) for P in Ps]
    srv = B.Server(ctx, 100 << 20, 4)
    order = [0, 1, 2, 3, 4, 3, 1]
    tickets = [(i, srv.submit(Ps[i], st)) for i in order]
    for i, t in tickets:
        info, x, y, s = srv.wait(t, Ps[i])
        assert info["iters"] == solo[i][0]["iters"]
        np.testing.assert_array_equal(x, solo[i][1])
        np.testing.assert_array_equal(y, solo[i][2])
        np.testing.assert_array_equal(s, solo[i][3])
    srv.close()
