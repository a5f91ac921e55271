"""The projection stage (ps_projection_step: first guesses, Picard loop of
operator update / right-hand side / solve / post-projection, Sections
3.3-3.5) against the FP64 oracle of oracle/projection.py, through the C ABI.

Gates: dP, P, W_u, H and rho K element by element (node by node) against the
oracle's Picard loop at a tight solve tolerance; at the 64^3 size of the bench
workload, the GPU's dP meets the 1e-10 residual gate of the oracle's system
for the same enthalpy and right-hand side, and every element output matches
the oracle's post-projection formulas applied to the GPU's dP.
"""
import numpy as np
import pytest

import oracle
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


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _gpu_step(P, torch, m, case, n_picard, dp0=None, **solve_kw):
    e = case.extra
    N, E, d = case.n_nodes, case.n_elems, case.dim
    dp = _dev(torch, np.zeros(N) if dp0 is None else dp0)
    outs = [torch.empty(N, dtype=torch.float64, device="cuda"),
            torch.empty(E * d, dtype=torch.float64, device="cuda"),
            torch.empty(E, dtype=torch.float64, device="cuda"),
            torch.empty(E, dtype=torch.float64, device="cuda")]
    st, info = P.ps_projection_step(m, _dev(torch, e["rho"]), _dev(torch, e["wu"]), _dev(torch, e["we"]),
                                    _dev(torch, e["pn"]), dp, *outs, gamma=e["gamma"], dt=e["dt"],
                                    n_picard=n_picard, solve_opts=P.make_opts(**solve_kw))
    p, wu, H, rhok = (o.cpu().numpy() for o in outs)
    return st, info, dp.cpu().numpy(), p, wu.reshape(E, d), H, rhok


def _oracle_step(case, n_picard, dp0=None):
    e = case.extra
    return PJ.projection_step(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, e["rho"], e["wu"],
                              e["we"], e["pn"], e["gamma"], e["dt"], n_picard, dp0=dp0, tol=1e-13)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [("3d_8", lambda: S.make_projection_case(3, 8)),
         ("2d_24", lambda: S.make_projection_case(2, 24)),
         ("3d_8_shuffled", lambda: _shuffled(S.make_projection_case(3, 8), 5))]


def _shuffled(case, seed):
    """The same flow under a random node numbering and element order."""
    sh = S.shuffle_case(case, seed=seed)
    p, q = sh.extra["node_new_of_old"], sh.extra["elem_old_of_new"]
    e = case.extra
    pn = np.empty(case.n_nodes)
    pn[p] = e["pn"]
    sh.extra = {"rho": e["rho"][q], "wu": e["wu"][q], "we": e["we"][q], "pn": pn,
                "gamma": e["gamma"], "dt": e["dt"]}
    return sh


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_projection_step_matches_oracle(env, name, make, mode):
    P, torch, ctx = env
    case = make()
    m = upload(P, ctx, case)
    try:
        st, info, dp, p, wu, H, rhok = _gpu_step(P, torch, m, case, 2, mode=mode, tol=1e-13, max_outer=20)
        ref = _oracle_step(case, 2)
        assert st == P.PS_OK
        assert _rel(dp, ref["dp"]) <= 1e-9, _rel(dp, ref["dp"])
        # P and H move by dP only (|dP| ~ 0.1 |P|): bounded by the dP gate
        assert _rel(p, ref["p"]) <= 1e-10
        assert _rel(wu, ref["wu"]) <= 1e-9
        assert _rel(H, ref["H"]) <= 1e-10
        assert _rel(rhok, ref["rhok"]) <= 1e-9
        assert np.all(dp[case.dirichlet.astype(bool)] == 0.0)
        # the second solve's right-hand side (||b|| over free nodes) is the
        # oracle's (it depends on the first dP through H and rho K)
        b2 = ref["solves"][1]["b"][~case.dirichlet.astype(bool)]
        assert abs(info.bnorm - np.linalg.norm(b2)) <= 1e-8 * np.linalg.norm(b2)
        assert info.iters_outer >= 2            # summed over both Picard iterations
    finally:
        P.ps_mesh_free(m)


def test_projection_step_is_deterministic_and_warm_starts(env):
    P, torch, ctx = env
    case = S.make_projection_case(3, 10)
    m = upload(P, ctx, case)
    try:
        a = _gpu_step(P, torch, m, case, 2)
        b = _gpu_step(P, torch, m, case, 2)
        for u, v in zip(a[2:], b[2:]):
            assert np.array_equal(u, v)
        # the first solve warm-starts from dp: from its own converged
        # correction, a one-iteration step does no CG iteration at all
        a1 = _gpu_step(P, torch, m, case, 1)
        c1 = _gpu_step(P, torch, m, case, 1, dp0=a1[2])
        assert a1[1].iters_inner > 0 and c1[1].iters_inner == 0
        assert np.array_equal(c1[2], a1[2])
    finally:
        P.ps_mesh_free(m)


def test_projection_step_full_size_residual_gate(env):
    """64^3 Kuhn cube (the bench workload), one Picard iteration: the GPU's dP
    meets the 1e-10 residual gate of the oracle's system (A with beta = H^1,
    b from the oracle's right-hand side), and every element output equals the
    oracle's post-projection of the GPU's dP."""
    P, torch, ctx = env
    case = S.make_projection_case(3, 64)
    e = case.extra
    m = upload(P, ctx, case)
    try:
        st, info, dp, p, wu, H, rhok = _gpu_step(P, torch, m, case, 1)
        assert st == P.PS_OK
        H1 = PJ.enthalpy(case.conn, e["pn"], e["rho"], e["gamma"])
        b = PJ.rhs(3, case.coords, case.conn, case.dirichlet, case.alpha, H1, PJ.kinetic(e["wu"], e["rho"], 3),
                   e["wu"], e["we"], e["pn"], e["dt"])
        A = oracle.PressureMatrix(3, case.coords, case.conn, case.dirichlet, case.alpha, H1, e["dt"] ** 2)
        assert A.residual(b, dp) <= 1.05e-10
        p_o, wu_o, H_o, rhok_o = PJ.post(3, case.coords, case.conn, e["pn"], dp, e["wu"], e["rho"], e["gamma"],
                                         e["dt"])
        assert np.allclose(p, p_o, rtol=1e-15, atol=0)
        assert np.max(np.abs(wu - wu_o)) <= 1e-12 * np.abs(wu_o).max()
        assert np.max(np.abs(H - H_o) / H_o) <= 1e-14
        assert np.max(np.abs(rhok - rhok_o)) <= 1e-12 * np.abs(rhok_o).max()
    finally:
        P.ps_mesh_free(m)


def test_projection_step_rejects_bad_input(env):
    P, torch, ctx = env
    case = S.make_projection_case(2, 8)
    m = upload(P, ctx, case)
    try:
        bad = case.extra.copy()
        bad["rho"] = case.extra["rho"].copy()
        bad["rho"][3] = -1.0                       # negative density: H < 0
        case_bad = S.Case(case.name, case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta,
                          case.dt2, case.b, case.x0, extra=bad)
        with pytest.raises(P.PressureError) as ei:
            _gpu_step(P, torch, m, case_bad, 1)
        assert ei.value.status == P.PS_EINVAL
        with pytest.raises(P.PressureError) as ei:
            _gpu_step(P, torch, m, case, 0)
        assert ei.value.status == P.PS_EINVAL
        # the mesh still solves after the rejected calls
        st, *_ = _gpu_step(P, torch, m, case, 1)
        assert st == P.PS_OK
    finally:
        P.ps_mesh_free(m)
