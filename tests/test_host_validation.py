"""Mesh validation of fblts_mesh_create, exercised through the host-only
fblts_mesh_regions (the same validation and classification, no device): each
corruption of a valid mesh is rejected with its status and a message, and a
valid mesh whose weightsOnEdge are not the kite-fraction TRiSK weights is
accepted and planned with the explicit-list edge pass instead of the
cell-side TRiSK pass."""
import copy

import numpy as np
import pytest

import paper_2405_10505_gb300 as fb
from synth import scenario


@pytest.fixture(scope="module")
def bump():
    return scenario.gaussian_bump_case(two_level=True)


def _mesh_with(s, **arrays):
    m = copy.copy(s.mesh)
    for k, v in arrays.items():
        setattr(m, k, v)
    return m


def _status(s, mesh=None, level=None, M=None):
    try:
        fb.mesh_regions(mesh or s.mesh, s.fVertex, s.level if level is None else level,
                        s.M if M is None else M, 0)
    except fb.FbltsError as e:
        return e.status, fb.last_error()
    return fb.OK, ""


def test_valid_mesh_is_accepted(bump):
    assert _status(bump)[0] == fb.OK


def test_corruptions_are_rejected(bump):
    m = bump.mesh
    coe = m.cellsOnEdge.copy()
    coe[5, 1] = m.nCells + 3
    area = m.areaCell.copy()
    area[7] = -1.0
    dc = m.dcEdge.copy()
    dc[11] = 0.0
    eoc = m.edgesOnCell.copy()
    eoc[3, 0] = eoc[40, 0] if eoc[40, 0] not in eoc[3] else eoc[41, 0]
    cases = [
        (_mesh_with(bump, cellsOnEdge=coe), fb.E_MESH, "cellsOnEdge"),
        (_mesh_with(bump, areaCell=area), fb.E_MESH, "area"),
        (_mesh_with(bump, dcEdge=dc), fb.E_MESH, "dcEdge"),
        (_mesh_with(bump, edgesOnCell=eoc), fb.E_MESH, "edgesOnCell"),
    ]
    for mesh, want, word in cases:
        st, msg = _status(bump, mesh=mesh)
        assert st == want and word in msg, (word, st, msg)


def test_level_errors_are_rejected(bump):
    bad = bump.level.copy()
    bad[0] = -1
    st, msg = _status(bump, level=bad)                          # level out of range
    assert st == fb.E_REGIONS and "out of range" in msg
    skip = bump.level * 2
    skip[np.flatnonzero(bump.level == 0)[0]] = 1                # level 1 present, but the disk
    st, msg = _status(bump, level=skip, M=[2, 2])               # borders level 0 directly
    assert st == fb.E_REGIONS and "joins levels" in msg
    assert _status(bump, M=[0])[0] == fb.E_ARG                  # M < 1


def test_non_kite_weights_plan_the_explicit_list_pass(bump):
    p = fb.make_params(bump.dt, precision=fb.FP32_TENDENCY)
    kinds = [fb.plan_op(bump.mesh, bump.fVertex, bump.level, bump.M, p, i)[0] for i in range(5)]
    assert kinds == ["forcing", "cell", "vertex", "trisk", "edge"]
    w = bump.mesh.weightsOnEdge * (1.0 + 1e-3 * np.random.default_rng(3).standard_normal(bump.mesh.weightsOnEdge.shape))
    other = _mesh_with(bump, weightsOnEdge=w)
    kinds = [fb.plan_op(other, bump.fVertex, bump.level, bump.M, p, i)[0] for i in range(5)]
    assert kinds == ["forcing", "cell", "vertex", "edge_prep", "edge"]
