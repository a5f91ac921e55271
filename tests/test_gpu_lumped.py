"""The mass-lumped operator (ps_mesh_set_mass) and the general-EOS projection
step solved by Newton's method (ps_projection_step_eos), through the C ABI,
against oracle/lumped.py.

Gates: the lumped apply element by element (FP64 and FP32 bars of the apply
tests); lumped solves in every engine (oracle residual gate 1e-10, error
against a direct solve 1e-9); switching the form back restores the consistent
operator bit for bit, also inside captured graphs; a lumped mesh batched with
a consistent one gets its alone result; the Newton projection step against the
oracle's (dP, P, W_u, H, rho K, number of Newton steps, residual history); at
the 64^3 size of the bench workload the GPU's dP meets the oracle's exact
nonlinear residual bar.
"""
import numpy as np
import pytest

import oracle
from oracle import lumped as L
from oracle import projection as PJ
from paper_2301_08357_gb300 import synthetic as S
from tests.gpu_util import upload

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


def _lumped(case):
    return L.LumpedMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)


CASES = [("c1_24", lambda: S.make_c1(24), 0),
         ("c2_8", lambda: S.make_c2(8), 0),
         ("c2_9_small_chunks", lambda: S.make_c2(9), 60),
         ("c2_8_shuffled", lambda: S.shuffle_case(S.make_c2(8), seed=3), 0)]


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)], ids=["f64", "f32"])
def test_lumped_apply_matches_oracle(env, name, make, chunk, prec, tol):
    P, torch, ctx = env
    case = make()
    A = _lumped(case)
    m = upload(P, ctx, case, chunk)
    try:
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        x = np.random.default_rng(3).standard_normal(case.n_nodes)
        dt = torch.float64 if prec == 2 else torch.float32
        xd = torch.as_tensor(x, dtype=dt, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        P.ps_pressure_apply(m, xd, yd, prec)
        y = yd.cpu().double().numpy()
        ref = A.apply(x)
        scale = A.extend(abs(A.A) @ np.abs(A.restrict(x)))
        free = ~case.dirichlet.astype(bool)
        assert np.all(np.isfinite(y))
        assert np.max(np.abs(y - ref)[free] / scale[free]) <= tol
        assert np.all(y[~free] == 0.0)
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("name,make,chunk", CASES[:3], ids=[c[0] for c in CASES[:3]])
@pytest.mark.parametrize("mode,engine", [(0, 0), (1, 1), (1, 3), (1, 2)],
                         ids=["fp64", "mixed_graph", "mixed_fused", "mixed_persistent"])
def test_lumped_solve_matches_oracle(env, name, make, chunk, mode, engine):
    P, torch, ctx = env
    case = make()
    A = _lumped(case)
    m = upload(P, ctx, case, chunk)
    try:
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        bd = torch.as_tensor(case.b, device="cuda")
        xd = torch.zeros(case.n_nodes, dtype=torch.float64, device="cuda")
        st, info = P.ps_pressure_solve(m, bd, xd, P.make_opts(mode=mode, engine=engine, tol=1e-10))
        assert st == P.PS_OK
        assert A.residual(case.b, xd.cpu().numpy()) <= 1.05e-10
        xs = A.solve(case.b)
        xd.zero_()
        st, info = P.ps_pressure_solve(m, bd, xd, P.make_opts(mode=mode, engine=engine, tol=1e-13, max_outer=12))
        assert np.linalg.norm(xd.cpu().numpy() - xs) <= 1e-9 * np.linalg.norm(xs)
    finally:
        P.ps_mesh_free(m)


def test_switching_the_mass_form(env):
    """Consistent -> lumped -> consistent: the apply comes back bit for bit,
    and a graph captured under one form is not replayed under the other."""
    P, torch, ctx = env
    case = S.make_c2(8)
    m = upload(P, ctx, case)
    try:
        x = torch.as_tensor(np.random.default_rng(4).standard_normal(case.n_nodes), device="cuda")
        y0, y1, y2 = (torch.empty_like(x) for _ in range(3))
        P.ps_pressure_apply(m, x, y0, 2)
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        P.ps_pressure_apply(m, x, y1, 2)
        P.ps_mesh_set_mass(m, P.PS_MASS_CONSISTENT)
        P.ps_pressure_apply(m, x, y2, 2)
        assert torch.equal(y0, y2) and not torch.equal(y0, y1)
        bd = torch.as_tensor(case.b, device="cuda")
        opts = P.make_opts(mode=1, engine=1, tol=1e-10)
        for form, A in ((P.PS_MASS_CONSISTENT, oracle.PressureMatrix.from_case(case)),
                        (P.PS_MASS_LUMPED, _lumped(case)),
                        (P.PS_MASS_CONSISTENT, oracle.PressureMatrix.from_case(case))):
            P.ps_mesh_set_mass(m, form)
            xd = torch.zeros_like(bd)
            st, _ = P.ps_pressure_solve(m, bd, xd, opts)
            assert st == P.PS_OK
            assert A.residual(case.b, xd.cpu().numpy()) <= 1.05e-10
        with pytest.raises(P.PressureError) as ei:
            P.ps_mesh_set_mass(m, 2)
        assert ei.value.status == P.PS_EINVAL
    finally:
        P.ps_mesh_free(m)


def test_lumped_mesh_in_a_batch_equals_alone(env):
    P, torch, ctx = env
    c1, c2 = S.make_c2(8), S.make_batch_case(5, lo=2e3, hi=4e3)
    m1, m2 = upload(P, ctx, c1), upload(P, ctx, c2)
    try:
        P.ps_mesh_set_mass(m1, P.PS_MASS_LUMPED)
        b1, b2 = torch.as_tensor(c1.b, device="cuda"), torch.as_tensor(c2.b, device="cuda")
        x1 = torch.zeros(c1.n_nodes, dtype=torch.float64, device="cuda")
        x2 = torch.zeros(c2.n_nodes, dtype=torch.float64, device="cuda")
        st, _ = P.ps_batch_solve([m1, m2], [b1, b2], [x1, x2])
        assert st == P.PS_OK
        y1 = torch.zeros_like(x1)
        P.ps_batch_solve([m1], [b1], [y1])
        assert torch.equal(x1, y1)
        assert _lumped(c1).residual(c1.b, x1.cpu().numpy()) <= 1.05e-10
        assert oracle.PressureMatrix.from_case(c2).residual(c2.b, x2.cpu().numpy()) <= 1.05e-10
    finally:
        P.ps_mesh_free(m1)
        P.ps_mesh_free(m2)


# ------------------------------------------------------------ general EOS
def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _eos_gpu(P, torch, m, case, n_picard, max_newton, ntol, dp0=None, **solve_kw):
    e = case.extra
    N, E, d = case.n_nodes, case.n_elems, case.dim
    dp = _dev(torch, np.zeros(N) if dp0 is None else dp0)
    outs = [torch.empty(N, dtype=torch.float64, device="cuda"),
            torch.empty(E * d, dtype=torch.float64, device="cuda"),
            torch.empty(E, dtype=torch.float64, device="cuda"),
            torch.empty(E, dtype=torch.float64, device="cuda")]
    st, info, res = P.ps_projection_step_eos(m, _dev(torch, e["rho"]), _dev(torch, e["wu"]), _dev(torch, e["we"]),
                                             _dev(torch, e["pn"]), dp, *outs, eos_a=e["eos_a"], eos_b=e["eos_b"],
                                             dt=e["dt"], n_picard=n_picard, max_newton=max_newton,
                                             newton_tol=ntol, solve_opts=P.make_opts(**solve_kw))
    p, wu, H, rhok = (o.cpu().numpy() for o in outs)
    return st, info, res, dp.cpu().numpy(), p, wu.reshape(E, d), H, rhok


def _eos_oracle(case, n_picard, max_newton, tol):
    e = case.extra
    return L.projection_step_eos(case.dim, case.coords, case.conn, case.dirichlet, e["rho"], e["wu"], e["we"],
                                 e["pn"], e["eos_a"], e["eos_b"], e["dt"], n_picard, max_newton, tol=tol)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _eos_upload(P, ctx, case):
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet)
    P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
    return m


EOS_CASES = [("3d_8", lambda: S.make_eos_case(3, 8)),
             ("2d_24_stiff", lambda: S.make_eos_case(2, 24, eos_b=2.0)),
             ("3d_8_ideal", lambda: S.make_eos_case(3, 8, eos_b=0.0))]


@pytest.mark.parametrize("name,make", EOS_CASES, ids=[c[0] for c in EOS_CASES])
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_eos_step_matches_oracle(env, name, make, mode):
    P, torch, ctx = env
    case = make()
    m = _eos_upload(P, ctx, case)
    try:
        st, info, res, dp, p, wu, H, rhok = _eos_gpu(P, torch, m, case, 2, 8, 1e-10, mode=mode, tol=1e-13,
                                                      max_outer=20)
        ref = _eos_oracle(case, 2, 8, 1e-10)
        assert st == P.PS_OK
        assert _rel(dp, ref["dp"]) <= 1e-9, _rel(dp, ref["dp"])
        assert _rel(p, ref["p"]) <= 1e-10
        assert _rel(wu, ref["wu"]) <= 1e-9
        assert _rel(H, ref["H"]) <= 1e-10
        assert _rel(rhok, ref["rhok"]) <= 1e-9
        assert np.all(dp[case.dirichlet.astype(bool)] == 0.0)
        for k in range(2):
            h_gpu = res[k][res[k] >= 0]
            h_ref = np.array(ref["hist"][k])
            # same number of checks; residuals above the solve's floor agree
            assert h_gpu.size == h_ref.size, (h_gpu, h_ref)
            big = h_ref > 1e-7
            assert np.allclose(h_gpu[big], h_ref[big], rtol=1e-4)
        if case.extra["eos_b"] == 0.0:
            assert ref["steps"] == [1, 1]
    finally:
        P.ps_mesh_free(m)


def test_eos_step_fixed_count_and_warm_start(env):
    P, torch, ctx = env
    case = S.make_eos_case(3, 8)
    m = _eos_upload(P, ctx, case)
    try:
        a = _eos_gpu(P, torch, m, case, 1, 3, 0.0)
        b = _eos_gpu(P, torch, m, case, 1, 3, 0.0)
        assert a[0] == P.PS_OK
        for u, v in zip(a[3:], b[3:]):
            assert np.array_equal(u, v)
        assert np.all(a[2][0] >= 0)                 # every check recorded (history requested)
        # starting from its own converged dP, Newton stops at the first check
        c = _eos_gpu(P, torch, m, case, 1, 3, 1e-8, dp0=a[3])
        assert c[0] == P.PS_OK and c[1].iters_inner == 0 and c[2][0][0] <= 1e-8
        # an unreachable tolerance reports PS_ENOTCONV with the outputs written
        d = _eos_gpu(P, torch, m, case, 1, 1, 1e-30)
        assert d[0] == P.PS_ENOTCONV and np.all(np.isfinite(d[3]))
    finally:
        P.ps_mesh_free(m)


def test_eos_step_full_size_residual_gate(env):
    """64^3 Kuhn cube (the bench workload), one Picard iteration: the oracle's
    exact nonlinear residual of the GPU's dP (its own H and c) meets the
    Newton bar, and the element outputs are the oracle's post-projection."""
    P, torch, ctx = env
    case = S.make_eos_case(3, 64)
    e = case.extra
    m = _eos_upload(P, ctx, case)
    try:
        st, info, res, dp, p, wu, H, rhok = _eos_gpu(P, torch, m, case, 1, 8, 1e-9)
        assert st == P.PS_OK
        a, b, dt = e["eos_a"], e["eos_b"], e["dt"]
        H1 = L.enthalpy(case.conn, e["pn"], e["rho"], a, b)
        c = PJ.rhs(3, case.coords, case.conn, case.dirichlet, np.zeros(case.n_nodes), H1,
                   PJ.kinetic(e["wu"], e["rho"], 3), e["wu"], e["we"], e["pn"], dt)
        K = oracle.PressureMatrix(3, case.coords, case.conn, case.dirichlet, case.alpha, H1, 1.0, part=2)
        q, _ = L.mass_sum(3, case.coords, case.conn, e["rho"], e["pn"] + dp, a, b)
        free = ~case.dirichlet.astype(bool)
        F = (q + dt * dt * K.apply(dp) - c)[free]
        assert np.linalg.norm(F) <= 2e-9 * np.linalg.norm(c[free])
        _, wu_o, _, rhok_o = PJ.post(3, case.coords, case.conn, e["pn"], dp, e["wu"], e["rho"], 1.4, dt)
        assert np.max(np.abs(wu - wu_o)) <= 1e-12 * np.abs(wu_o).max()
        assert np.max(np.abs(rhok - rhok_o)) <= 1e-12 * np.abs(rhok_o).max()
        H_o = L.enthalpy(case.conn, p, e["rho"], a, b)
        assert np.max(np.abs(H - H_o) / H_o) <= 1e-14
    finally:
        P.ps_mesh_free(m)


def test_eos_step_rejects_bad_state_and_input(env):
    P, torch, ctx = env
    case = S.make_eos_case(2, 8, eos_b=1.0)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet)
    try:
        with pytest.raises(P.PressureError) as ei:          # consistent mass
            _eos_gpu(P, torch, m, case, 1, 2, 1e-8)
        assert ei.value.status == P.PS_ESTATE
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        with pytest.raises(P.PressureError) as ei:          # max_newton out of range
            _eos_gpu(P, torch, m, case, 1, 0, 1e-8)
        assert ei.value.status == P.PS_EINVAL
        # a pressure so negative that Q'_i = a m_i + 2 b s_i P_i < 0 (H stays
        # positive through its quadratic term)
        bad = S.Case(case.name, case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2,
                     case.b, case.x0, extra=dict(case.extra, pn=np.full(case.n_nodes, -20.0)))
        with pytest.raises(P.PressureError) as ei:
            _eos_gpu(P, torch, m, bad, 1, 2, 1e-8)
        assert ei.value.status == P.PS_EINVAL
        st, *_ = _eos_gpu(P, torch, m, case, 1, 4, 1e-8)
        assert st == P.PS_OK
        # the ideal-gas step needs coefficients from ps_coeff_set again
        with pytest.raises(P.PressureError) as ei:
            P.ps_projection_step(m, *(torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(9)),
                                 gamma=1.4, dt=0.1, n_picard=1)
        assert ei.value.status == P.PS_ESTATE
    finally:
        P.ps_mesh_free(m)


def test_eos_step_rejects_periodic_meshes(env):
    P, torch, ctx = env
    case = S.make_periodic_case(2, 8)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, periodic=case.extra["master"])
    try:
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        N, E = case.n_nodes, case.n_elems
        z = lambda n: torch.ones(n, dtype=torch.float64, device="cuda")
        with pytest.raises(P.PressureError) as ei:
            P.ps_projection_step_eos(m, z(E), z(2 * E), z(E), z(N), z(N), z(N), z(2 * E), z(E), z(E), dt=0.1)
        assert ei.value.status == P.PS_EINVAL
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 6)])
def test_lumped_apply_on_periodic_mesh(env, dim, n):
    """Lumped mass on a mesh with merged periodic vertices: the merged operator
    P^T (diag(alpha m) + dt^2 K) P of the unmerged mesh (every vertex its own
    weight m_v, alpha from the master), built here from the oracle's pieces."""
    import scipy.sparse as sp
    from oracle.periodic import PeriodicMatrix
    P, torch, ctx = env
    case = S.make_periodic_case(dim, n)
    master = case.extra["master"]
    N = case.n_nodes
    Pm = PeriodicMatrix(dim, case.coords, case.conn, case.dirichlet, master, case.alpha, case.beta, case.dt2)
    K = oracle.PressureMatrix(dim, case.coords, case.conn, np.zeros(N, np.uint8), case.alpha, case.beta, 1.0,
                              part=2)
    assert np.array_equal(K.node_of_free, np.arange(N))
    mv = L.lumped_weights(dim, case.coords, case.conn)
    A_full = sp.diags(np.asarray(case.alpha)[master] * mv) + case.dt2 * K.scipy()
    Ad = (Pm.P.T @ A_full @ Pm.P).tocsr()[Pm.free][:, Pm.free]
    m = P.ps_mesh_upload(ctx, dim, case.coords, case.conn, case.dirichlet, periodic=master)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        x = np.random.default_rng(8).standard_normal(N)
        for prec, tol in ((2, 1e-12), (1, 2e-5)):
            dt = torch.float64 if prec == 2 else torch.float32
            xd = torch.as_tensor(x, dtype=dt, device="cuda")
            yd = torch.full_like(xd, float("nan"))
            P.ps_pressure_apply(m, xd, yd, prec)
            y = yd.cpu().double().numpy()
            xu = xd.cpu().double().numpy()
            xf = Pm.to_dofs(xu)[Pm.free]
            ref = Pm.to_user(Ad @ xf)
            scale = Pm.to_user(abs(Ad) @ np.abs(xf))
            free = scale > 0
            assert np.max(np.abs(y - ref)[free] / scale[free]) <= tol, prec
            assert np.array_equal(y, y[master])
    finally:
        P.ps_mesh_free(m)
