"""Serving loop: pressure-solve requests from several simulated cases, each a
sequence of time steps whose beta drifts and whose solve warm-starts from the
case's previous pressure (Section 3.4: the solution at t^n is the first guess).

Checks: every served result meets the 1e-10 residual gate against the FP64
oracle's matrix for that step's beta; every result is bitwise the same as the
same sequence of solves run alone (batch of one); a budget that admits one
request at a time still completes everything in order; error paths.
"""
import numpy as np
import pytest

import oracle
from paper_2301_08357_gb300 import synthetic as S
from tests.gpu_util import upload

pytestmark = pytest.mark.gpu

N_STEPS = 3


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    ctx = P.ps_ctx_create(0)
    yield P, torch, ctx
    P.ps_ctx_destroy(ctx)


def _steps(case):
    """(beta, b) for each time step of the case, drawn from its own stream."""
    out = []
    beta, b = case.beta.copy(), case.b.copy()
    out.append((None, beta.copy(), b.copy()))
    for _ in range(N_STEPS - 1):
        beta, b = S.served_step_drift(case, beta, b)
        out.append((beta.copy(), beta.copy(), b.copy()))
    return out


def _serve(P, ctx, cases, meshes, steps, **srv_kw):
    srv = P.ps_server_create(ctx, **srv_kw)
    try:
        ids = [P.ps_server_add_case(srv, m) for m in meshes]
        tickets = []
        for k in range(N_STEPS):
            for ci, cid in enumerate(ids):
                beta_sub, _, b = steps[ci][k]
                tickets.append((ci, k, P.ps_solve_submit(srv, cid, b, beta_sub)))
        results = {}
        for ci, k, t in tickets:
            x = np.empty(cases[ci].n_nodes)
            st, info = P.ps_solve_wait(srv, t, 120.0, x)
            results[(ci, k)] = (st, info.as_dict(), x)
            P.ps_server_release(srv, t)
        stats = P.ps_server_get_stats(srv).as_dict()
    finally:
        P.ps_server_destroy(srv)
    return results, stats


def _alone(P, torch, case, mesh, steps):
    """The same sequence of solves, one mesh per batch."""
    P.ps_coeff_set(mesh, case.alpha, case.beta, case.dt2)
    x = torch.zeros(case.n_nodes, dtype=torch.float64, device="cuda")
    outs = []
    for beta_sub, beta, b in steps:
        if beta_sub is not None:
            P.ps_coeff_set_beta(mesh, beta_sub)
        bd = torch.as_tensor(b, device="cuda")
        st, infos = P.ps_batch_solve([mesh], [bd], [x])
        outs.append(x.cpu().numpy().copy())
    P.ps_coeff_set(mesh, case.alpha, case.beta, case.dt2)
    return outs


def test_served_results_match_oracle_and_alone(env):
    P, torch, ctx = env
    cases = [S.make_served_case(c, lo=1e3, hi=2e4, median=4e3) for c in range(5)]
    steps = [_steps(c) for c in cases]
    meshes = [upload(P, ctx, c) for c in cases]
    try:
        results, stats = _serve(P, ctx, cases, meshes, steps, max_slots=8, epoch_iters=16)
        assert stats["completed"] == len(cases) * N_STEPS and stats["failed"] == 0
        assert stats["peak_in_flight"] >= 2          # requests really overlapped
        for ci, c in enumerate(cases):
            for k in range(N_STEPS):
                st, info, x = results[(ci, k)]
                assert st == P.PS_OK and info["converged"] == 1
                A = oracle.PressureMatrix.from_case(c, beta=steps[ci][k][1])
                assert A.residual(steps[ci][k][2], x) <= 1.05e-10, (ci, k)
                assert info["seconds"] >= info["queue_seconds"] >= 0.0
        for ci, c in enumerate(cases):
            alone = _alone(P, torch, c, meshes[ci], steps[ci])
            for k in range(N_STEPS):
                assert np.array_equal(alone[k], results[(ci, k)][2]), (ci, k)
        # warm start: later steps need fewer iterations than a cold first step
        it0 = np.mean([results[(ci, 0)][1]["iters_inner"] for ci in range(len(cases))])
        it2 = np.mean([results[(ci, N_STEPS - 1)][1]["iters_inner"] for ci in range(len(cases))])
        assert it2 < it0
    finally:
        for m in meshes:
            P.ps_mesh_free(m)


def _alone_single(P, torch, case, mesh, steps):
    """The same sequence of solves through ps_pressure_solve (default options)."""
    P.ps_coeff_set(mesh, case.alpha, case.beta, case.dt2)
    x = torch.zeros(case.n_nodes, dtype=torch.float64, device="cuda")
    outs = []
    for beta_sub, beta, b in steps:
        if beta_sub is not None:
            P.ps_coeff_set_beta(mesh, beta_sub)
        bd = torch.as_tensor(b, device="cuda")
        st, info = P.ps_pressure_solve(mesh, bd, x, P.make_opts())
        assert st == P.PS_OK
        outs.append(x.cpu().numpy().copy())
    P.ps_coeff_set(mesh, case.alpha, case.beta, case.dt2)
    return outs


def test_single_lane_for_large_meshes(env):
    """single_nodes routes the cases with the larger meshes to the
    single-solve engine (each request alone, between epochs): their results
    equal the same sequence of ps_pressure_solve calls bitwise, the others equal
    the batch of one, and every result meets the oracle's gate."""
    P, torch, ctx = env
    cases = [S.make_served_case(c, lo=1e3, hi=2e4, median=4e3) for c in range(30, 36)]
    steps = [_steps(c) for c in cases]
    meshes = [upload(P, ctx, c) for c in cases]
    sizes = [c.n_nodes for c in cases]
    thr = int(np.median(sizes)) + 1
    single = [n >= thr for n in sizes]
    assert 0 < sum(single) < len(cases)
    try:
        results, stats = _serve(P, ctx, cases, meshes, steps, max_slots=8, epoch_iters=16, single_nodes=thr)
        assert stats["completed"] == len(cases) * N_STEPS and stats["failed"] == 0
        assert stats["single_solves"] == sum(single) * N_STEPS
        for ci, c in enumerate(cases):
            for k in range(N_STEPS):
                st, info, x = results[(ci, k)]
                assert st == P.PS_OK and info["converged"] == 1
                A = oracle.PressureMatrix.from_case(c, beta=steps[ci][k][1])
                assert A.residual(steps[ci][k][2], x) <= 1.05e-10, (ci, k)
        for ci, c in enumerate(cases):
            alone = (_alone_single if single[ci] else _alone)(P, torch, c, meshes[ci], steps[ci])
            for k in range(N_STEPS):
                assert np.array_equal(alone[k], results[(ci, k)][2]), (ci, k, single[ci])
    finally:
        for m in meshes:
            P.ps_mesh_free(m)


def test_budget_forces_queueing(env):
    P, torch, ctx = env
    cases = [S.make_served_case(c, lo=3e3, hi=4e3, median=3.5e3) for c in range(10, 13)]
    steps = [_steps(c) for c in cases]
    meshes = [upload(P, ctx, c) for c in cases]
    try:
        # a budget that fits the largest single request only (any two exceed it)
        sizes = sorted(P.ps_mesh_get_stats(m).solve_bytes for m in meshes)
        budget = sizes[-1] + 1
        assert sizes[0] + sizes[1] > budget
        results, stats = _serve(P, ctx, cases, meshes, steps, max_slots=8, epoch_iters=16,
                                hbm_budget_bytes=budget)
        assert stats["completed"] == len(cases) * N_STEPS
        assert stats["peak_in_flight"] == 1
        for ci, c in enumerate(cases):
            A = oracle.PressureMatrix.from_case(c, beta=steps[ci][N_STEPS - 1][1])
            assert A.residual(steps[ci][N_STEPS - 1][2], results[(ci, N_STEPS - 1)][2]) <= 1.05e-10
    finally:
        for m in meshes:
            P.ps_mesh_free(m)


def test_server_error_paths(env):
    P, torch, ctx = env
    c = S.make_served_case(20, lo=1e3, hi=3e3, median=2e3)
    m = upload(P, ctx, c)
    srv = P.ps_server_create(ctx, hbm_budget_bytes=1024)   # nothing fits
    try:
        cid = P.ps_server_add_case(srv, m)
        with pytest.raises(P.PressureError) as e:
            P.ps_server_add_case(srv, m)                     # one case per mesh
        assert e.value.status == P.PS_EINVAL
        with pytest.raises(P.PressureError) as e:
            P.ps_solve_submit(srv, cid + 5, c.b)
        assert e.value.status == P.PS_ENOTFOUND
        with pytest.raises(P.PressureError) as e:
            P.ps_solve_submit(srv, cid, c.b, -c.beta)
        assert e.value.status == P.PS_EINVAL
        t = P.ps_solve_submit(srv, cid, c.b)
        with pytest.raises(P.PressureError) as e:
            P.ps_solve_wait(srv, t, 30.0)
        assert e.value.status == P.PS_ENOMEM
        with pytest.raises(P.PressureError) as e:
            P.ps_solve_poll(srv, 987654)
        assert e.value.status == P.PS_ENOTFOUND
    finally:
        P.ps_server_destroy(srv)
        P.ps_mesh_free(m)
