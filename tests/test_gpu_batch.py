"""Batched ensemble (fblts_batch_*) against each member advanced alone.

A batch shares launches between members but runs the same per-element
arithmetic.  In graph-branch mode the members' own kernels run, so every
member comes out bitwise equal to the same state advanced alone with
fblts_lts_advance.  The merged kernels are compiled separately, where the
compiler may contract a different set of float multiply-adds, so there (and
through the online tuning rounds, which try merged shapes) each member must
agree with its alone run within the FP32 path's tolerance: h 1e-6 relative,
u 1e-5 of max |u|.
"""
import numpy as np
import pytest

import paper_2405_10505_gb300 as fb
from synth import scenario
from tests.gpu_util import make_state, rel_errors

pytestmark = pytest.mark.gpu


def _members():
    # uneven meshes: hex and irregular Voronoi cells (8- and 12-slot rows),
    # 2 and 3 levels, M = 2 / 4, forcing off / wind + drag / vortex
    return [
        scenario.gaussian_bump_case(two_level=True),
        scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3),
        scenario.jittered_voronoi_case(),
        scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)),
        scenario.shelf_case(nx=40, ny=32, dc=2e3, M=4, width=10e3, vortex=True),
    ]


def _alone(cases, n):
    out = []
    for s in cases:
        st = make_state(s, precision=fb.FP32_TENDENCY)
        fb.lts_advance(st, n)
        out.append(fb.state_read(st))
    return out


@pytest.mark.parametrize("opts", [dict(autotune=True),
                                  dict(autotune=False, threads_per_block=128, ctas_per_sm=2, tile_order=1),
                                  dict(autotune=False, threads_per_block=256, ctas_per_sm=0, tile_order=0),
                                  dict(autotune=False, mode=1),
                                  dict(autotune=False, mode=2, threads_per_block=128, ctas_per_sm=8),
                                  dict(autotune=False, mode=3)])
def test_batch_equals_members_alone(opts):
    cases = _members()
    n = 15                                   # more rounds than the 13 tuning candidates
    ref = _alone(cases, n)
    states = [make_state(s, precision=fb.FP32_TENDENCY) for s in cases]
    b = fb.batch_create(states, **opts)
    fb.batch_advance(b, 4)
    fb.batch_advance(b, n - 4)
    fb.batch_synchronize(b)
    info = fb.batch_info(b)
    assert info.members == len(cases) and info.rounds == n
    if info.mode == 0:
        assert info.launches_per_round < info.member_launches_per_round
    if opts["autotune"]:
        assert info.tuned == 1
    for st, (h0, u0) in zip(states, ref):
        h, u = fb.state_read(st)
        if not opts["autotune"] and opts.get("mode") == 1:
            assert np.array_equal(h, h0) and np.array_equal(u, u0)
        else:
            dh, du = rel_errors(h, u, h0, u0)
            assert dh <= 1e-6 and du <= 1e-5, (dh, du)
    fb.batch_destroy(b)


def test_batch_then_alone_continues_the_same_run():
    cases = _members()[:3]
    ref = _alone(cases, 6)
    states = [make_state(s, precision=fb.FP32_TENDENCY) for s in cases]
    b = fb.batch_create(states, autotune=False, mode=1)
    fb.batch_advance(b, 3)
    fb.batch_destroy(b)
    for st in states:
        fb.lts_advance(st, 3)                 # the device step counter went on in the batch
    for st, (h0, u0) in zip(states, ref):
        h, u = fb.state_read(st)
        assert np.array_equal(h, h0) and np.array_equal(u, u0)


def test_batch_rejects_bad_members():
    s = scenario.gaussian_bump_case(two_level=True)
    st32 = make_state(s, precision=fb.FP32_TENDENCY)
    st64 = make_state(s, precision=fb.FP64)
    with pytest.raises(fb.FbltsError):
        fb.batch_create([st32, st64])
    with pytest.raises(fb.FbltsError):
        fb.batch_create([st32, st32])
    with pytest.raises(fb.FbltsError):
        fb.batch_create([st32], autotune=False, threads_per_block=100)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_mixes_schemes(mode):
    """Members with the operator splitting (both variants) and RK4 beside a
    plain FB-LTS member: every launch kind and segment mode goes through the
    merged kernels, and each member equals its alone run."""
    bump = scenario.gaussian_bump_case(two_level=True)
    shelf = scenario.shelf_case(nx=40, ny=32, dc=2e3, M=4, width=10e3, vortex=True)
    one = np.zeros(bump.mesh.nCells, np.int32)
    kinds = [dict(s=bump), dict(s=bump, split=1), dict(s=shelf, split=2),
             dict(s=bump, level=one, M=[], scheme=fb.SCHEME_RK4, dt=bump.dt / 2)]

    def state(k):
        return make_state(k["s"], level=k.get("level"), M=k.get("M"), precision=fb.FP32_TENDENCY,
                          split=k.get("split", 0), scheme=k.get("scheme", fb.SCHEME_FBLTS), dt=k.get("dt"))

    n = 8
    ref = []
    for k in kinds:
        st = state(k)
        fb.lts_advance(st, n)
        ref.append(fb.state_read(st))
    states = [state(k) for k in kinds]
    b = fb.batch_create(states, autotune=False, mode=mode)
    fb.batch_advance(b, n)
    fb.batch_synchronize(b)
    for st, (h0, u0) in zip(states, ref):
        h, u = fb.state_read(st)
        if mode == 1:
            assert np.array_equal(h, h0) and np.array_equal(u, u0)
        else:
            dh, du = rel_errors(h, u, h0, u0)
            assert dh <= 1e-6 and du <= 1e-5, (dh, du)
    fb.batch_destroy(b)


def test_batch_members_match_oracle():
    """Every member of a tuned batch, after 100 rounds (the 13 tuning rounds
    among them), against the FP64 oracle's FB-LTS run of the same scenario
    (Sec. 2.2) at the FP32 path's bar: h 1e-6 relative, u 1e-5 of max |u|."""
    import oracle
    cases = _members()
    n = 100
    states = [make_state(s, precision=fb.FP32_TENDENCY) for s in cases]
    b = fb.batch_create(states, autotune=True)
    fb.batch_advance(b, n)
    fb.batch_synchronize(b)
    assert fb.batch_info(b).tuned == 1
    for s, st in zip(cases, states):
        h, u = fb.state_read(st)
        ho, uo = oracle.fblts(oracle.Mesh.from_scenario(s), oracle.scenario_params(s), s.level, s.M, s.h0,
                              s.u0, s.dt, n)
        dh, du = rel_errors(h, u, ho, uo)
        assert dh <= 1e-6 and du <= 1e-5, (s.name, dh, du)
    fb.batch_destroy(b)
