"""Periodic boundaries by vertex merging (Section 3.6) through the C ABI
(ps_mesh_upload_periodic), against the merged-system oracle of
oracle/periodic.py: apply element by element (FP64 and FP32 bars of the apply
tests), solves in every engine (oracle residual gate, error gate against a
direct solve), merged vertices carrying their unknown's value, and a batch
mixing periodic and ordinary meshes giving each mesh its alone result.
"""
import numpy as np
import pytest

from oracle.periodic import PeriodicMatrix
from paper_2301_08357_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    assert torch.cuda.is_available()
    ctx = P.ps_ctx_create(0)
    yield P, torch, ctx
    P.ps_ctx_destroy(ctx)


def _upload(P, case, ctx, chunk=0):
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk,
                         periodic=case.extra["master"])
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    return m


def _oracle(case):
    return PeriodicMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.extra["master"], case.alpha,
                          case.beta, case.dt2)


CASES = [("2d_24", lambda: S.make_periodic_case(2, 24), 0),
         ("3d_8", lambda: S.make_periodic_case(3, 8), 0),
         ("3d_9_small_chunks", lambda: S.make_periodic_case(3, 9), 60)]


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)], ids=["f64", "f32"])
def test_periodic_apply_matches_oracle(env, name, make, chunk, prec, tol):
    P, torch, ctx = env
    case = make()
    A = _oracle(case)
    m = _upload(P, case, ctx, chunk)
    try:
        x = np.random.default_rng(3).standard_normal(case.n_nodes)
        dt = torch.float64 if prec == 2 else torch.float32
        xd = torch.as_tensor(x, dtype=dt, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        P.ps_pressure_apply(m, xd, yd, prec)
        y = yd.cpu().double().numpy()
        ref = A.apply(x)
        # bar relative to the size of the terms summed into each row
        scale = A.to_user(abs(A.A) @ np.abs(A.to_dofs(x)[A.free]))
        free = scale > 0
        assert np.all(np.isfinite(y))
        assert np.max(np.abs(y - ref)[free] / scale[free]) <= tol
        assert np.all(y[~free] == 0.0)
        # every merged vertex carries its unknown's row
        master = case.extra["master"]
        assert np.array_equal(y, y[master])
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode,engine", [(0, 0), (1, 0), (1, 1), (1, 3), (1, 2)],
                         ids=["fp64", "mixed_auto", "mixed_graph", "mixed_fused", "mixed_persistent"])
def test_periodic_solve_matches_oracle(env, name, make, chunk, mode, engine):
    P, torch, ctx = env
    case = make()
    A = _oracle(case)
    m = _upload(P, case, ctx, chunk)
    try:
        bd = torch.as_tensor(case.b, device="cuda")
        xd = torch.zeros(case.n_nodes, dtype=torch.float64, device="cuda")
        st, info = P.ps_pressure_solve(m, bd, xd, P.make_opts(mode=mode, engine=engine, tol=1e-10))
        x = xd.cpu().numpy()
        assert st == P.PS_OK
        assert A.residual(case.b, x) <= 1.05e-10
        assert np.array_equal(x, x[case.extra["master"]])
        xs = A.solve(case.b)
        xd.zero_()
        st, info = P.ps_pressure_solve(m, bd, xd, P.make_opts(mode=mode, engine=engine, tol=1e-13, max_outer=12))
        x = xd.cpu().numpy()
        assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    finally:
        P.ps_mesh_free(m)


def test_periodic_mesh_in_a_batch_equals_alone(env):
    P, torch, ctx = env
    per = S.make_periodic_case(3, 8)
    plain = S.make_batch_case(5, lo=2e3, hi=4e3)
    m1 = _upload(P, per, ctx)
    m2 = P.ps_mesh_upload(ctx, plain.dim, plain.coords, plain.conn, plain.dirichlet)
    P.ps_coeff_set(m2, plain.alpha, plain.beta, plain.dt2)
    try:
        b1, b2 = torch.as_tensor(per.b, device="cuda"), torch.as_tensor(plain.b, device="cuda")
        x1 = torch.zeros(per.n_nodes, dtype=torch.float64, device="cuda")
        x2 = torch.zeros(plain.n_nodes, dtype=torch.float64, device="cuda")
        st, infos = P.ps_batch_solve([m1, m2], [b1, b2], [x1, x2])
        assert st == P.PS_OK
        y1 = torch.zeros_like(x1)
        st, _ = P.ps_batch_solve([m1], [b1], [y1])
        assert torch.equal(x1, y1)
        assert _oracle(per).residual(per.b, x1.cpu().numpy()) <= 1.05e-10
    finally:
        P.ps_mesh_free(m1)
        P.ps_mesh_free(m2)
