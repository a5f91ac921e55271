"""Batched solves: many independent meshes (2D and 3D, different sizes) in one
persistent cooperative kernel, checked per mesh against the FP64 oracle, and
each mesh's result bitwise equal alone and in the mix (its arithmetic and
reduction order depend only on that mesh)."""
import numpy as np
import pytest

import oracle
from paper_2301_08357_gb300 import synthetic as S
from tests.gpu_util import upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    ctx = P.ps_ctx_create(0)
    yield P, torch, ctx
    P.ps_ctx_destroy(ctx)


def _cases():
    cs = [S.make_batch_case(i, lo=2e3, hi=3e4) for i in range(6)]
    cs.append(S.shuffle_case(S.make_c2(9), seed=2))
    c3 = S.make_c3(10)
    cs.append(c3)
    return cs


def _rhs(case, A):
    if "xstar" in case.extra:
        return A.apply(case.extra["xstar"]), case.x0
    return case.b, case.x0


def _batch(P, torch, meshes, bs, x0s, **kw):
    bd = [torch.as_tensor(b, dtype=torch.float64, device="cuda") for b in bs]
    xd = [torch.as_tensor(x, dtype=torch.float64, device="cuda").clone() for x in x0s]
    st, infos = P.ps_batch_solve(meshes, bd, xd, P.make_opts(**kw))
    return st, infos, [x.cpu().numpy() for x in xd]


def test_batch_matches_oracle_and_alone(env):
    P, torch, ctx = env
    cases = _cases()
    As = [oracle.PressureMatrix.from_case(c) for c in cases]
    rhs = [_rhs(c, A) for c, A in zip(cases, As)]
    meshes = [upload(P, ctx, c) for c in cases]
    try:
        st, infos, xs = _batch(P, torch, meshes, [r[0] for r in rhs], [r[1] for r in rhs], tol=1e-10)
        assert st == P.PS_OK
        for c, A, (b, x0), inf, x in zip(cases, As, rhs, infos, xs):
            assert inf.converged == 1 and inf.rel_res <= 1e-10, c.name
            assert A.residual(b, x) <= 1.05e-10, c.name
            assert np.all(x[c.dirichlet.astype(bool)] == 0.0)
        # alone (batch of one, and the default single-solve engine) == in the mix, bitwise
        for k in (0, 3, len(cases) - 1):
            st1, inf1, x1 = _batch(P, torch, [meshes[k]], [rhs[k][0]], [rhs[k][1]], tol=1e-10)
            assert np.array_equal(x1[0], xs[k]), cases[k].name
            assert inf1[0].iters_inner == infos[k].iters_inner
            bd = torch.as_tensor(rhs[k][0], device="cuda")
            xd = torch.as_tensor(rhs[k][1], device="cuda").clone()
            st2, inf2 = P.ps_pressure_solve(meshes[k], bd, xd, P.make_opts(tol=1e-10, engine=P.PS_ENGINE_PERSISTENT))
            assert np.array_equal(xd.cpu().numpy(), xs[k])
        # another batch order gives the same per-mesh results
        order = [5, 2, 7, 0, 6, 1, 4, 3]
        st3, inf3, x3 = _batch(P, torch, [meshes[i] for i in order], [rhs[i][0] for i in order],
                               [rhs[i][1] for i in order], tol=1e-10)
        for j, i in enumerate(order):
            assert np.array_equal(x3[j], xs[i])
        # error gate at the tightened tolerance
        st4, inf4, x4 = _batch(P, torch, meshes, [r[0] for r in rhs], [r[1] for r in rhs], tol=1e-13,
                               max_outer=12)
        for c, A, (b, x0), x in zip(cases, As, rhs, x4):
            xs_, _, _, _ = A.cg(b, x0_full=x0, precond=1, tol=1e-13)
            assert np.linalg.norm(x - xs_) <= 1e-9 * np.linalg.norm(xs_), c.name
    finally:
        for m in meshes:
            P.ps_mesh_free(m)


def test_batch_degenerate_members(env):
    P, torch, ctx = env
    cases = [S.make_c1(12), S.make_c2(5), S.make_c1(20)]
    As = [oracle.PressureMatrix.from_case(c) for c in cases]
    meshes = [upload(P, ctx, c) for c in cases]
    try:
        exact, _, _, _ = As[1].cg(cases[1].b, precond=1, tol=1e-14)
        bs = [np.zeros(cases[0].n_nodes), cases[1].b, cases[2].b]
        x0s = [np.zeros(cases[0].n_nodes), exact, np.zeros(cases[2].n_nodes)]
        st, infos, xs = _batch(P, torch, meshes, bs, x0s)
        assert st == P.PS_OK
        assert np.all(xs[0] == 0.0) and infos[0].iters_inner == 0
        assert infos[1].iters_inner == 0
        assert As[2].residual(cases[2].b, xs[2]) <= 1.05e-10
        # an iteration cap is reported per mesh
        st, infos, xs = _batch(P, torch, meshes, bs, x0s, max_iters=2, max_outer=1)
        assert st == P.PS_ENOTCONV
        assert infos[2].converged == 0 and infos[0].converged == 1
    finally:
        for m in meshes:
            P.ps_mesh_free(m)


def test_batch_rejects_bad_calls(env):
    P, torch, ctx = env
    c = S.make_c1(6)
    m = upload(P, ctx, c)
    try:
        b = torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        with pytest.raises(P.PressureError):
            P.ps_batch_solve([m, m], [b, b], [x, x])       # same mesh twice
        m2 = P.ps_mesh_upload(ctx, 2, c.coords, c.conn, c.dirichlet)
        with pytest.raises(P.PressureError) as e:
            P.ps_batch_solve([m, m2], [b, b], [x, x.clone()])   # coefficients not set
        assert e.value.status == P.PS_ESTATE
        P.ps_mesh_free(m2)
    finally:
        P.ps_mesh_free(m)
