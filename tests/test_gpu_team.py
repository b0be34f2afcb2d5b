"""GPU checks of the team engine's schedules (one persistent kernel per solve
or batch; a problem runs on one CTA or on a thread-block cluster), against
the FP64 oracle through the C ABI.

* every schedule shape -- one-CTA teams of 256 / 1024 threads, cluster teams
  of 2, 4 and 8 CTAs, CSR rows on 1 or 32 lanes -- keeps the first 20
  iterates within 1e-5 of the oracle's on convolution, dense (FP8, with row
  scales; adjoint with row-group partials) and CSR (BF16, ragged sizes)
  operators;
* a batch that mixes cluster teams and one-CTA teams returns, bit for bit,
  what each problem returns alone under the same schedule;
* the autotuner times its candidates, installs a valid schedule, and the
  problems then solve to the 1e-4 residuals (re-checked in FP64);
* CF_ENGINE_AUTO sends unsupported problems (operator products, more than 4
  second-order cones, long convolutions, wide dense leaves) to the graph
  engine, and CF_ENGINE_TEAM refuses them.
"""
import numpy as np
import pytest

from oracle import cones, scs
from paper_1609_03488_b300 import synth
from tests.helpers import fp64_residuals, objective_rel_err, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1609_03488_b300 import build
    build.build()
    from paper_1609_03488_b300 import binding
    return binding


def _ctx(B, **sched):
    c = B.Context(0)
    if sched:
        B.set_schedule(c, **sched)
    return c


SCHEDULES = {
    "cta256": dict(cluster=1, threads=256),
    "cta1024_lanes32": dict(cluster=1, threads=1024, csr_nnz_per_lane=1),
    "cluster2": dict(cluster=2, threads=512, team_bytes=0.0),
    "cluster4_lanes1": dict(cluster=4, threads=256, team_bytes=0.0, csr_nnz_per_lane=64),
    "cluster8": dict(cluster=8, threads=1024, team_bytes=0.0),
    "cta512x2": dict(cluster=1, threads=512, ctas_per_sm=2),
    "cta256x4_cluster2": dict(cluster=2, threads=256, ctas_per_sm=4, team_bytes=0.0),
}

FAMILIES = {
    "deconv": lambda: synth.deconv(n_x=1000, L=100, seed=synth.BASE_SEED + 1),
    "lasso_fp8": lambda: synth.lasso(m_d=601, p=301, seed=synth.BASE_SEED + 3, storage="fp8"),
    "lp_bf16": lambda: synth.lp(m_d=301, n_x=151, density=0.05, seed=synth.BASE_SEED + 4, storage="bf16"),
}


@pytest.mark.parametrize("sched", sorted(SCHEDULES))
@pytest.mark.parametrize("family", sorted(FAMILIES))
def test_schedule_trajectories_match_oracle(B, sched, family):
    ctx = _ctx(B, **SCHEDULES[sched])
    prob = FAMILIES[family]()
    ref = scs.problem_solve(prob, max_iters=20, check_interval=10 ** 6, linsys="cg", cg_fixed_steps=3,
                            trajectory=20)
    P = B.cone_problem_create(ctx, prob)
    N = prob["A"]["n"] + prob["A"]["m"] + 1
    for k in (1, 5, 20):
        st = B.settings(max_iters=k, check_interval=10 ** 6, cg_fixed_iters=3, engine="team")
        uv = np.empty(2 * N)
        info = B.cf_info()
        B.check(B.lib.solve(P.h, B.C.byref(st), None, None, None, None, B._ptr(uv), B.C.byref(info)), "solve")
        assert info.iters == k and info.cg_iters_total == 3 * k and info.kernel_launches == 1
        eu = rel(uv[:N], ref["traj_u"][k - 1])
        ev = rel(uv[N:], ref["traj_v"][k - 1])
        assert eu <= 1e-5 and ev <= 1e-5, (sched, k, eu, ev)


@pytest.mark.parametrize("sched", ["cluster2", "cluster8"])
def test_cluster_team_solutions(B, sched):
    """Mixed cones (zero, nonnegative, three second-order cones) and a lasso
    solved by cluster teams: FP64 residuals and objective vs the oracle."""
    ctx = _ctx(B, **SCHEDULES[sched])
    rng = np.random.default_rng(401)
    for prob in (synth.mixed_cone_problem(rng, n=8, soc_sizes=(3, 1, 5), z=2, l=4),
                 synth.lasso(m_d=400, p=200, seed=synth.BASE_SEED + 3, storage="bf16")):
        ref = scs.problem_solve(prob, eps=1e-10, max_iters=400000)
        assert ref["status"] == scs.SOLVED
        P = B.cone_problem_create(ctx, prob)
        info, x, y, s = B.solve(P, B.settings(eps=1e-5, engine="team"))
        assert info["status_name"] == "solved", info
        assert max(fp64_residuals(prob, x, y, s)) <= 1e-4
        assert objective_rel_err(prob["c"] @ x, ref["pobj"]) <= 1e-4
        assert cones.dist_to_cone(s, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(s))
        assert cones.dist_to_dual_cone(y, prob["cone"]) <= 1e-5 * (1 + np.linalg.norm(y))


def _lp_batch(count, seed):
    sizes = synth.lp_batch_sizes(count=count, m_lo=60, m_hi=900, seed=seed)
    return [synth.lp(m_d=m, n_x=n, density=max(d, 0.02), seed=sd, storage="bf16" if i % 2 else "fp32")
            for i, (m, n, d, sd) in enumerate(sizes)]


def test_mixed_batch_equals_solo(B):
    """A cluster schedule whose size threshold splits the batch: the larger
    half on 4-CTA cluster teams, the rest on one-CTA teams, one launch."""
    probs = _lp_batch(24, 901) + [synth.deconv(n_x=700, L=40, seed=9),
                                  synth.lasso(m_d=300, p=150, seed=10, storage="fp8")]
    ctx = _ctx(B, cluster=4, threads=512)
    Ps = [B.cone_problem_create(ctx, p) for p in probs]
    sizes = [B.team_info(P)[1] for P in Ps]
    B.set_schedule(ctx, team_bytes=float(np.median(sizes)))
    st = B.settings(engine="team")
    solo = [B.solve(P, st) for P in Ps]
    infos, xs, ys, ss = B.solve_batch(Ps, st)
    assert sum(i["kernel_launches"] for i in infos) == 1
    for (i0, x0, y0, s0), i1, x1, y1, s1 in zip(solo, infos, xs, ys, ss):
        assert i0["iters"] == i1["iters"] and i0["status"] == i1["status"] == B.CF_SOLVED
        np.testing.assert_array_equal(x0, x1)
        np.testing.assert_array_equal(y0, y1)
        np.testing.assert_array_equal(s0, s1)
    for k in range(0, len(probs), 5):
        assert max(fp64_residuals(probs[k], xs[k], ys[k], ss[k])) <= 1e-4


def test_autotuner_installs_a_schedule_that_solves(B):
    ctx = _ctx(B)
    probs = _lp_batch(16, 902)
    Ps = [B.cone_problem_create(ctx, p) for p in probs]
    info = B.solve_batch_tune(Ps, iters=10)
    assert info["problems"] == 16 and info["candidates"] == 2 + 24 + 9
    assert info["best_ms"] > 0 and info["best_ms"] <= info["default_ms"]
    got = B.get_schedule(ctx)
    assert got == info["best"]
    assert got["cluster"] in (1, 2, 4, 8) and got["threads"] in (256, 512, 1024)
    infos, xs, ys, ss = B.solve_batch(Ps)
    for p, i, x, y, s in zip(probs, infos, xs, ys, ss):
        assert i["status_name"] == "solved", i
        assert max(fp64_residuals(p, x, y, s)) <= 1e-4


def test_auto_routing_and_unsupported_problems(B):
    ctx = _ctx(B)
    rng = np.random.default_rng(5)
    # a small supported problem: one launch per solve under CF_ENGINE_AUTO
    P = B.cone_problem_create(ctx, synth.lp(m_d=200, n_x=100, density=0.05, seed=3))
    info, *_ = B.solve(P)
    assert info["kernel_launches"] == 1
    B.set_schedule(ctx, auto_max_bytes=0.0)       # now everything is too large for AUTO
    info, *_ = B.solve(P)
    assert info["kernel_launches"] > 1
    B.set_schedule(ctx, auto_max_bytes=1e6)
    # unsupported: an operator product, 5 second-order cones, a long
    # convolution, a wide dense leaf
    D = rng.standard_normal((30, 20)).astype(np.float32)
    prod = {"A": synth.vstack([synth.product([synth.dense(D[:, :10]), synth.eye(10)]), synth.scale(-1.0, synth.eye(10))]),
            "b": np.concatenate([np.ones(30), np.zeros(10)]), "c": -np.ones(10),
            "cone": {"z": 0, "l": 40, "q": []}}
    many_soc = synth.mixed_cone_problem(rng, n=6, soc_sizes=(2, 2, 2, 2, 2), z=1, l=2)
    long_conv = synth.deconv(n_x=100, L=2100, seed=4)
    wide = synth.lasso(m_d=2, p=16400, seed=5)
    for prob, why in ((prod, "product"), (many_soc, "second-order"), (long_conv, "taps"), (wide, "columns")):
        P = B.cone_problem_create(ctx, prob)
        ok, _, reason = B.team_info(P)
        assert not ok and why in reason, reason
        info, *_ = B.solve(P, B.settings(max_iters=20))
        assert info["kernel_launches"] > 1, why        # AUTO took the graph engine
        with pytest.raises(B.CfError) as e:
            B.solve(P, B.settings(max_iters=20, engine="team"))
        assert e.value.code == B.CF_E_INVALID and why in str(e.value), str(e.value)


def test_schedule_validation(B):
    ctx = _ctx(B)
    assert B.get_schedule(ctx)["team_bytes"] == 256e3 and B.get_schedule(ctx)["auto_max_bytes"] == 1e6
    for bad in (dict(cluster=3), dict(threads=128), dict(csr_nnz_per_lane=0), dict(team_bytes=-1.0),
                dict(ctas_per_sm=3), dict(threads=1024, ctas_per_sm=2)):
        with pytest.raises(B.CfError) as e:
            B.set_schedule(ctx, **bad)
        assert e.value.code == B.CF_E_INVALID
    s = B.get_schedule(ctx)
    assert (s["cluster"], s["threads"], s["csr_nnz_per_lane"]) == (4, 512, 16)


def test_engine_switch_redoes_setup(B):
    """g = M^{-1} h computed by one program is not reused by the other (their
    float32 rounding differs): switching engines reruns the setup, and the
    same engine twice does not."""
    ctx = _ctx(B)
    P = B.cone_problem_create(ctx, synth.deconv(n_x=300, L=30, seed=12))
    runs = [B.solve(P, B.settings(max_iters=30, engine=e))[0] for e in ("team", "team", "graph", "team")]
    assert [r["setup_cg_iters"] > 0 for r in runs] == [True, False, True, True]
