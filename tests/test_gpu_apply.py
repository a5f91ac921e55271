"""Parity of the CUDA matrix-free operator apply (through the C ABI) with the
FP64 oracle's assembled sparse matrix, element by element.

Tolerances (per row i, scale s_i = sum_j |A_ij x_j|):
  FP64 apply:  |y_gpu - y_oracle| <= 1e-12 s_i   (summation-order rounding);
  FP32 apply:  |y_gpu - y_oracle| <= 2e-5  s_i   (FP32 geometry relative to a
               chunk origin and FP32 sums; inputs are the same float32 values).
Dirichlet rows are exactly 0 in both.  The apply is deterministic: two calls
give bitwise equal results.
"""
import numpy as np
import pytest

import oracle
from paper_2301_08357_gb300 import synthetic as S
from tests.gpu_util import row_scale_fast, sampled_rows, upload

pytestmark = pytest.mark.gpu

TOL = {2: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def P():
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure
    return pressure


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def ctx(P, torch_mod):
    c = P.ps_ctx_create(0)
    yield c
    P.ps_ctx_destroy(c)


CASES = [
    ("c1_64", lambda: S.make_c1(64), 0),
    ("c1_64_shuffled_chunk37", lambda: S.shuffle_case(S.make_c1(64)), 37),
    ("c1_tiny_n2", lambda: S.make_c1(2), 0),
    ("c2_n1_six_tets", lambda: S.make_c2(1), 0),
    ("c2_n6_chunk50", lambda: S.make_c2(6), 50),
    ("c2_n16", lambda: S.make_c2(16), 0),
    ("c2_n16_shuffled", lambda: S.shuffle_case(S.make_c2(16), seed=3), 0),
    ("c3_n12", lambda: S.make_c3(12), 0),
    ("batch_mesh_1", lambda: S.make_batch_case(1, lo=2e3, hi=5e3), 0),
]


def _gpu_apply(P, torch, m, x, prec):
    dt = torch.float32 if prec == 1 else torch.float64
    xd = torch.as_tensor(x, dtype=dt, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    P.ps_pressure_apply(m, xd, yd, prec)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [2, 1], ids=["f64", "f32"])
def test_apply_matches_oracle(P, torch_mod, ctx, name, make, chunk, prec):
    case = make()
    m = upload(P, ctx, case, chunk)
    try:
        A = oracle.PressureMatrix.from_case(case)
        rng = np.random.default_rng(11)
        for trial in range(2):
            x = rng.standard_normal(case.n_nodes)
            if trial == 1:       # smooth input: stiffness part nearly cancels
                x = np.sin(3 * case.coords[:, 0]) + case.coords[:, 1] ** 2
            if prec == 1:
                x = x.astype(np.float32).astype(np.float64)
            y = _gpu_apply(P, torch_mod, m, x, prec)
            yo = A.apply(x)
            sc = row_scale_fast(A, x)
            dirm = case.dirichlet.astype(bool)
            assert np.all(y[dirm] == 0.0)
            err = np.abs(y - yo)
            worst = np.max(err[~dirm] / np.maximum(sc[~dirm], 1e-300))
            assert worst <= TOL[prec], (name, prec, worst)
            y2 = _gpu_apply(P, torch_mod, m, x, prec)
            assert np.array_equal(y, y2)
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("prec", [2, 1], ids=["f64", "f32"])
def test_apply_sparse_and_zero_inputs(P, torch_mod, ctx, prec):
    """Chunks whose input is zero skip their element phase: an input that is
    nonzero on a few nodes only (most chunks zero, a few partly) still matches
    the oracle on every row, and a zero input gives exactly zero."""
    case = S.make_c2(12)
    m = upload(P, ctx, case, 96)
    try:
        rng = np.random.default_rng(21)
        x = np.zeros(case.n_nodes)
        idx = rng.choice(case.n_nodes, size=7, replace=False)
        x[idx] = rng.standard_normal(7)
        if prec == 1:
            x = x.astype(np.float32).astype(np.float64)
        y = _gpu_apply(P, torch_mod, m, x, prec)
        # rows of the nodes that share an element with a nonzero input; their
        # scale is element-level (sum over elements of |A^e_ij x_j|): assembled
        # off-diagonal entries can cancel between the elements around an edge
        near = np.zeros(case.n_nodes, bool)
        hit = np.isin(case.conn, idx).any(axis=1)
        near[case.conn[hit].ravel()] = True
        nodes = np.where(near)[0]
        yo, sc = sampled_rows(case, x, nodes)
        live = sc > 0
        assert np.max(np.abs(y[nodes] - yo)[live] / sc[live]) <= TOL[prec]
        assert np.all(y[nodes][~live] == 0.0)
        assert np.all(y[~near] == 0.0)
        z = _gpu_apply(P, torch_mod, m, np.zeros(case.n_nodes), prec)
        assert np.all(z == 0.0)
    finally:
        P.ps_mesh_free(m)


def test_apply_full_size_c2(P, torch_mod, ctx):
    """64^3 Kuhn cube (1,572,864 tets), both precisions, every row."""
    case = S.make_c2()
    m = upload(P, ctx, case)
    try:
        A = oracle.PressureMatrix.from_case(case)
        x = np.random.default_rng(5).standard_normal(case.n_nodes)
        for prec in (2, 1):
            xi = x.astype(np.float32).astype(np.float64) if prec == 1 else x
            y = _gpu_apply(P, torch_mod, m, xi, prec)
            yo = A.apply(xi)
            sc = row_scale_fast(A, xi)
            free = ~case.dirichlet.astype(bool)
            worst = np.max(np.abs(y - yo)[free] / sc[free])
            assert worst <= TOL[prec], (prec, worst)
    finally:
        P.ps_mesh_free(m)


def test_apply_full_size_c3_sampled(P, torch_mod, ctx):
    """160^3 Kuhn cube (24,576,000 tets): sampled rows computed one by one from
    the oracle's element matrices, plus Dirichlet rows exactly zero."""
    case = S.make_c3()
    m = upload(P, ctx, case)
    try:
        x = np.random.default_rng(6).standard_normal(case.n_nodes)
        rng = np.random.default_rng(7)
        nodes = np.unique(np.concatenate([rng.integers(0, case.n_nodes, 400),
                                          np.arange(0, 200), np.arange(case.n_nodes - 200, case.n_nodes)]))
        for prec in (2, 1):
            xi = x.astype(np.float32).astype(np.float64) if prec == 1 else x
            y = _gpu_apply(P, torch_mod, m, xi, prec)
            yo, sc = sampled_rows(case, xi, nodes)
            free = ~case.dirichlet[nodes].astype(bool)
            worst = np.max(np.abs(y[nodes] - yo)[free] / sc[free])
            assert worst <= TOL[prec], (prec, worst)
            assert np.all(y[case.dirichlet.astype(bool)] == 0.0)
    finally:
        P.ps_mesh_free(m)


def test_apply_rejects_bad_calls(P, torch_mod, ctx):
    case = S.make_c1(4)
    m = P.ps_mesh_upload(ctx, 2, case.coords, case.conn, case.dirichlet)
    try:
        x = torch_mod.zeros(case.n_nodes, dtype=torch_mod.float64, device="cuda")
        y = torch_mod.zeros_like(x)
        with pytest.raises(P.PressureError) as e:
            P.ps_pressure_apply(m, x, y, 2)     # before coeff_set
        assert e.value.status == P.PS_ESTATE
        with pytest.raises(P.PressureError) as e:
            P.ps_coeff_set(m, case.alpha, -case.beta, case.dt2)
        assert e.value.status == P.PS_EINVAL
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        with pytest.raises(P.PressureError):
            P.ps_pressure_apply(m, x, y, 3)     # unknown precision
        with pytest.raises(P.PressureError):
            P.ps_pressure_apply(m, x, x, 2)     # aliasing
    finally:
        P.ps_mesh_free(m)
