"""CPU-only checks of the C ABI library: it loads, exports every function that
include/pressure.h declares, and its host preprocessing (chunking, renumbering,
incidence lists) satisfies the invariants the kernels rely on.  No device
call is made here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pressure.h")


@pytest.fixture(scope="module")
def P():
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure
    return pressure


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_are_exported(P):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.check_output(["nm", "-D", "--defined-only", P.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (ps_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the binding wraps exactly these names
    for n in names:
        assert n in P.SIGNATURES, n


def test_binding_constants_match_the_header(P):
    """Every PS_* constant the header defines has the same value in the
    binding (the binding restates them; a drift would pass wrong flags)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = dict(re.findall(r"#define\s+(PS_[A-Z0-9_]+)\s+(-?\d+)", src))
    assert len(defs) >= 25
    for name, value in defs.items():
        assert hasattr(P, name), name
        assert getattr(P, name) == int(value), (name, getattr(P, name), value)


def test_struct_layouts_match_the_header(P, tmp_path):
    """Size and field offsets of every struct the binding mirrors equal those a
    C compiler gives the header's declarations (gcc, this host's ABI)."""
    structs = [P.ps_mesh_opts, P.ps_solve_opts, P.ps_projection_opts, P.ps_solve_info, P.ps_mesh_stats,
               P.ps_server_opts, P.ps_server_stats, P.ps_eos_opts]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pressure.h"', 'int main(void) {']
    expect = []
    for st in structs:
        name = st.__name__
        lines.append('  printf("%%s %%zu\\n", "%s", sizeof(%s));' % (name, name))
        expect.append("%s %d" % (name, C.sizeof(st)))
        for field, _ in st._fields_:
            lines.append('  printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (name, field, name, field))
            expect.append("%s.%s %d" % (name, field, getattr(st, field).offset))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = subprocess.check_output([str(exe)]).decode().split("\n")
    assert [g for g in got if g] == expect


def test_version_and_status_strings(P):
    assert "sm_103a" in P.ps_version()
    assert P.ps_status_str(P.PS_OK) == "ok"
    assert "budget" in P.ps_status_str(P.PS_ENOMEM)


@pytest.mark.parametrize("dim,n,chunk", [(2, 8, 0), (2, 17, 37), (3, 4, 0), (3, 7, 50), (3, 6, 1000)])
def test_prepare_invariants(P, dim, n, chunk):
    from paper_2301_08357_gb300 import synthetic as S
    case = (S.make_c1 if dim == 2 else S.make_c2)(n=n, seed=n)
    s = P.ps_debug_prepare(dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk)
    assert s.n_nodes == case.n_nodes and s.n_elems == case.n_elems
    assert s.n_free == case.n_free
    assert s.n_chunks >= 1
    if chunk:
        assert s.max_chunk_elems <= chunk
    assert s.chunk_node_refs >= case.n_nodes
    # shuffled numbering gives the same sizes and still passes the invariants
    sh = S.shuffle_case(case, seed=7)
    s2 = P.ps_debug_prepare(dim, sh.coords, sh.conn, sh.dirichlet, chunk_elems=chunk)
    assert s2.n_free == s.n_free


def test_prepare_split_lead(P):
    """The first split_lead chunks of the Morton chunk order are split in
    halves when there are at least four times as many chunks (the layout's
    invariants hold either way); fewer chunks are left alone; -1 = none."""
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_c2(n=16)                                   # 24,576 tets
    base = P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=96)
    assert base.n_chunks == 256
    for k in (1, 7, 64):
        s = P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=96, split_lead=k)
        assert s.n_chunks == base.n_chunks + k
        assert s.max_chunk_elems == 96 and s.n_free == base.n_free
        assert s.n_shared >= base.n_shared
    # 65 * 4 > 256 chunks: no split; -1: none; below -1: rejected
    assert P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=96,
                              split_lead=65).n_chunks == 256
    assert P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=96,
                              split_lead=-1).n_chunks == 256
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=96, split_lead=-2)


def test_prepare_chunk_node_cap(P):
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_c2(n=8)
    s = P.ps_debug_prepare(3, case.coords, case.conn, case.dirichlet, chunk_elems=512, chunk_nodes_max=64)
    assert s.max_chunk_nodes <= 64


def test_prepare_rejects_bad_input(P):
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_c1(n=4)
    bad = case.conn.copy()
    bad[3, 1] = case.n_nodes          # out of range
    with pytest.raises(P.PressureError) as e:
        P.ps_debug_prepare(2, case.coords, bad, case.dirichlet)
    assert e.value.status == P.PS_EINVAL
    flat = case.conn.copy()
    flat[0] = [0, 1, 2]               # collinear vertices on the bottom edge
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, case.coords, flat, case.dirichlet)
    rep = case.conn.copy()
    rep[0, 2] = rep[0, 0]             # repeated vertex
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, case.coords, rep, case.dirichlet)
    nanc = case.coords.copy()
    nanc[5, 0] = np.nan
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, nanc, case.conn, case.dirichlet)
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(4, case.coords, case.conn, case.dirichlet)


@pytest.mark.parametrize("dim,n,chunk", [(2, 8, 0), (2, 9, 40), (3, 4, 0), (3, 5, 60)])
def test_prepare_periodic_invariants(P, dim, n, chunk):
    from oracle.periodic import PeriodicMatrix
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_periodic_case(dim, n)
    master = case.extra["master"]
    s = P.ps_debug_prepare(dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk, periodic=master)
    A = PeriodicMatrix(dim, case.coords, case.conn, case.dirichlet, master, case.alpha, case.beta, case.dt2)
    assert s.n_nodes == case.n_nodes
    assert s.n_free == int(A.free.sum())
    # identity map = no merging
    s0 = P.ps_debug_prepare(dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk,
                            periodic=np.arange(case.n_nodes, dtype=np.int32))
    assert s0.n_free == case.n_free


def test_prepare_rejects_bad_periodic_maps(P):
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_periodic_case(2, 4)
    master = case.extra["master"]
    chained = master.copy()
    j = int(np.flatnonzero(master != np.arange(case.n_nodes))[0])    # a merged vertex
    i = int(np.flatnonzero(master == np.arange(case.n_nodes))[-1])   # some master
    chained[i] = j                                                  # master mapped onto a merged vertex
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, case.coords, case.conn, case.dirichlet, periodic=chained)
    mixed = case.dirichlet.copy()
    x0_merged = np.flatnonzero((master != np.arange(case.n_nodes)) & (case.dirichlet == 1))[0]
    mixed[x0_merged] = 0                                            # slave free, master Dirichlet
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, case.coords, case.conn, mixed, periodic=master)
    # one cell across the period: an element would hold two vertices of one unknown
    coords, conn = S.square_mesh(1)
    thin = S.periodic_master(coords, (1,))
    with pytest.raises(P.PressureError):
        P.ps_debug_prepare(2, coords, conn, None, periodic=thin)
