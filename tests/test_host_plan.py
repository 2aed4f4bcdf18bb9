"""The launch list of one coarse step (fblts_plan_step, host only) against the
structure of the scheme, on CPU.

Counted independently from Sec. 2.2 and Eq. fbrk32: an FB-RK(3,2) step is
three stages of four passes (cell, vertex, TRiSK / edge prep, edge), or of two
(cell, edge) under the operator splitting of Sec. 3.2; an FB-LTS step of the
pair (l, l+1) is the coarse advancement, one save, and per subcycle one
prediction plus the fine step (recursing for more levels), then one
correction; a coarse step adds the forcing launch and the step end; the
splitting adds a four-pass slow block per coarse step (and per fine step in
its Sec. 4.2 variant); classical RK4 is four stages of four passes.  The
cell-updates are the metric's definition, sum_l N_l prod_{m<l} M_m."""
import numpy as np
import pytest

import paper_2405_10505_gb300 as fb
from synth import basin, scenario


def expected_ops(L, M, split):
    stage = 2 if split else 4

    def step(l):
        if l == L - 1:
            return 3 * stage
        return 3 * stage + 1 + M[l] * (1 + (4 if split == 2 else 0) + step(l + 1)) + 1

    return 1 + (4 if split else 0) + step(0) + 1


def expected_cell_updates(level, M):
    mult = np.cumprod([1] + list(M))
    return int(sum(int(np.sum(level == l)) * int(mult[l]) for l in range(len(M) + 1)))


CASES = {
    "bump_m2": lambda: scenario.gaussian_bump_case(two_level=True),
    "bump_m5": lambda: scenario.gaussian_bump_case(two_level=True, M=5),
    "nested_3level": lambda: scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)),
    "basin_1_64": lambda: basin.basin_case(Ly=150e3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_launch_count_and_cell_updates(name):
    s = CASES[name]()
    L = len(s.M) + 1
    bytes_ = {}
    for split in (0, 1, 2):
        for prec in (fb.FP64, fb.FP32_TENDENCY):
            n, b, cu = fb.plan_step(s.mesh, s.fVertex, s.level, s.M, fb.make_params(s.dt, precision=prec, split=split))
            assert n == expected_ops(L, s.M, split), (split, prec)
            assert cu == expected_cell_updates(s.level, s.M)
            bytes_[split, prec] = b
    for split in (0, 1, 2):
        assert 0 < bytes_[split, fb.FP32_TENDENCY] < bytes_[split, fb.FP64]
    for prec in (fb.FP64, fb.FP32_TENDENCY):
        # the splitting drops the vertex and TRiSK passes of every stage; its
        # variant adds a slow block per fine step
        assert bytes_[1, prec] < bytes_[2, prec] < bytes_[0, prec]


def test_rk4_plan_and_its_checks():
    s = scenario.gaussian_bump_case(two_level=True)
    one = np.zeros(s.mesh.nCells, np.int32)
    n, b, cu = fb.plan_step(s.mesh, s.fVertex, one, [], fb.make_params(s.dt, scheme=fb.SCHEME_RK4))
    assert n == 1 + 4 * 4 + 1 and cu == s.mesh.nCells and b > 0
    for level, M, kw in ((s.level, s.M, {}), (one, [], dict(split=1)), (one, [], dict(scheme=9))):
        with pytest.raises(fb.FbltsError) as e:
            fb.plan_step(s.mesh, s.fVertex, level, M, fb.make_params(s.dt, **{"scheme": fb.SCHEME_RK4, **kw}))
        assert e.value.status == fb.E_ARG


def test_degenerate_meshes():
    """One level of a tiny periodic mesh (one FB-RK(3,2) step: 14 launches); an
    empty mesh and a level array that skips a level are rejected."""
    s = scenario.gaussian_bump_case(nx=4, ny=4, two_level=False)
    n, b, cu = fb.plan_step(s.mesh, s.fVertex, s.level, [], fb.make_params(s.dt))
    assert n == 1 + 12 + 1 and cu == 16 and b > 0
    d = fb.MeshDesc()
    import ctypes as C
    n_ = C.c_int64()
    assert fb.lib().fblts_plan_step(C.byref(d), C.byref(fb.make_params(1.0)), C.byref(n_), None, None) == fb.E_ARG
    two = scenario.gaussian_bump_case(two_level=True)
    skip = two.level * 2          # levels 0 and 2, none on level 1
    with pytest.raises(fb.FbltsError):
        fb.plan_step(two.mesh, two.fVertex, skip, [2, 2], fb.make_params(two.dt))


def _first_advancement(s, params, after):
    """Per stage 1..3, the cell and edge modes of the first coarse advancement
    that starts after op index ``after``."""
    n, _, _ = fb.plan_step(s.mesh, s.fVertex, s.level, s.M, params)
    cells, edges, i = {}, {}, after + 1
    while i < n and (len(cells) < 3 or len(edges) < 3):
        kind, stage, mode = fb.plan_op(s.mesh, s.fVertex, s.level, s.M, params, i)
        if kind == "cell" and stage not in cells:
            cells[stage] = mode
        if kind == "edge" and stage not in edges and stage in cells:
            edges[stage] = mode
        i += 1
    return cells, edges, i


@pytest.mark.parametrize("name", ["bump_m2", "nested_3level", "basin_1_64"])
def test_coarse_advancement_uses_the_shrinking_sets(name):
    """The stages of a pair's coarse advancement update exactly the paper's
    shrinking sets (Sec. 2.2, computed by the oracle): cells F^5, F^3, F^1 and
    edges F_E^4, F_E^2 plus the coarse region, and in stage 3 the IF-1 and
    interior edges only (velocity stage 3 is skipped on IF-2 edges)."""
    s = CASES[name]()
    import oracle
    cc, cd, ec, ed, st = oracle.regions(oracle.Mesh.from_scenario(s), s.level)
    params = fb.make_params(s.dt)
    after = 0
    for pair in range(len(s.M)):
        cells, edges, last = _first_advancement(s, params, after)
        coarse_c = np.isin(cc[pair], (oracle.RC_IF1, oracle.RC_IF2, oracle.RC_INT))
        coarse_e = np.isin(ec[pair], (oracle.RC_IF1, oracle.RC_IF2, oracle.RC_INT))
        fine_c, fine_e = cc[pair] == oracle.RC_FINE, ec[pair] == oracle.RC_FINE
        want_c = {1: fine_c & (cd[pair] <= 10), 2: fine_c & (cd[pair] <= 6), 3: fine_c & (cd[pair] <= 2)}
        want_e = {1: (fine_e & (ed[pair] <= 8)) | coarse_e, 2: (fine_e & (ed[pair] <= 4)) | coarse_e,
                  3: np.isin(ec[pair], (oracle.RC_IF1, oracle.RC_INT))}
        for k in (1, 2, 3):
            upd_c = np.isin(cells[k], (fb.SEG_STAGE, fb.SEG_IN_PLACE))
            upd_e = np.isin(edges[k], (fb.SEG_STAGE, fb.SEG_IN_PLACE))
            np.testing.assert_array_equal(upd_c, want_c[k] | coarse_c, err_msg=f"pair {pair} cell stage {k}")
            np.testing.assert_array_equal(upd_e, want_e[k], err_msg=f"pair {pair} edge stage {k}")
        # interior cells and edges are updated in place by stage 3
        np.testing.assert_array_equal(cells[3] == fb.SEG_IN_PLACE, cc[pair] == oracle.RC_INT)
        # the next pair's coarse advancement starts after this pair's first prediction
        while fb.plan_op(s.mesh, s.fVertex, s.level, s.M, params, last)[0] != "predict":
            last += 1
        after = last


@pytest.mark.parametrize("name", ["bump_m2", "nested_3level"])
def test_correction_sums_cover_if1_and_if2(name):
    """Every launch that accumulates the interface correction (Eq. if_correction)
    covers exactly IF-1 u IF-2 of one level pair, cells and edges alike; each
    pair step sets the sums once (k = 0) and adds for k = 1..M-1."""
    s = CASES[name]()
    import oracle
    cc, cd, ec, ed, st = oracle.regions(oracle.Mesh.from_scenario(s), s.level)
    params = fb.make_params(s.dt)
    n, _, _ = fb.plan_step(s.mesh, s.fVertex, s.level, s.M, params)
    sets = {(p, kind): [] for p in range(len(s.M)) for kind in ("cell", "edge")}
    for i in range(n):
        kind, stage, mode = fb.plan_op(s.mesh, s.fVertex, s.level, s.M, params, i)
        if kind not in ("cell", "edge"):
            continue
        acc = np.isin(mode, (fb.SEG_SUM_SET, fb.SEG_SUM_ADD))
        if not acc.any():
            continue
        cls = cc if kind == "cell" else ec
        pairs = [p for p in range(len(s.M)) if np.array_equal(acc, np.isin(cls[p], (oracle.RC_IF1, oracle.RC_IF2)))]
        assert len(pairs) == 1, (i, kind)
        assert stage == 3
        modes = set(np.unique(mode[acc]).tolist())
        assert len(modes) == 1
        sets[pairs[0], kind].append(modes.pop())
    steps = np.cumprod([1] + list(s.M))
    for p in range(len(s.M)):
        for kind in ("cell", "edge"):
            got = sets[p, kind]
            assert len(got) == steps[p] * s.M[p]
            assert got.count(fb.SEG_SUM_SET) == steps[p]
            assert all(got[j] == (fb.SEG_SUM_SET if j % s.M[p] == 0 else fb.SEG_SUM_ADD) for j in range(len(got)))


def test_op_bytes_add_up_to_the_step():
    """The per-op algorithmic bytes sum to fblts_plan_step's total; the moved
    count is never below the algorithmic one, and only the FP32 path's TRiSK
    and edge passes (the per-slot shares) and the padded-row cell pass move
    more than the arithmetic needs."""
    s = CASES["nested_3level"]()
    for prec in (fb.FP64, fb.FP32_TENDENCY):
        p = fb.make_params(s.dt, precision=prec)
        n, total, _ = fb.plan_step(s.mesh, s.fVertex, s.level, s.M, p)
        alg = moved = 0.0
        for i in range(n):
            a, mv = fb.plan_op_bytes(s.mesh, s.fVertex, s.level, s.M, p, i)
            kind = fb.plan_op(s.mesh, s.fVertex, s.level, s.M, p, i)[0]
            assert mv >= a >= 0.0
            if mv > a:
                assert (prec == fb.FP32_TENDENCY and kind in ("trisk", "edge", "cell")) or \
                    (prec == fb.FP64 and kind == "cell"), (prec, kind)
            alg += a
            moved += mv
        assert abs(alg - total) <= 1e-9 * total
        assert moved >= alg
