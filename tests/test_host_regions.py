"""The library's host-side region classification (fblts_mesh_regions: the
band keys that order cells and edges so each set of Sec. 2.2 is one index
range) against the oracle's own region builder, on CPU.

The two are separate implementations: the library classifies by breadth-first
distances inside build_host_mesh, the oracle by its own layer search.  For
every level pair, every cell and edge must get the same class (fine, IF-1,
IF-2, interior, outside) and every fine cell and edge the same F^b band
b = ceil(D/2) (D the layer distance to the coarse region, capped at 6), which
is what decides the shrinking sets F^5 / F^3 / F^1 and F_E^4 / F_E^2."""
import numpy as np
import pytest

import oracle
import paper_2405_10505_gb300 as fb
from synth import basin, scenario

CASES = {
    "bump_2level": lambda: scenario.gaussian_bump_case(two_level=True),
    "nested_3level": lambda: scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3)),
    "shelf_walls": lambda: scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3),
    "jittered_voronoi": lambda: scenario.jittered_voronoi_case(),
    "basin_1_64": lambda: basin.basin_case(Ly=150e3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_library_regions_equal_oracle_regions(name):
    s = CASES[name]()
    m = oracle.Mesh.from_scenario(s)
    cc, cd, ec, ed, st = oracle.regions(m, s.level)
    assert st == oracle.OM_OK
    assert len(s.M) >= 1
    for pair in range(len(s.M)):
        lc, lb, lec, leb = fb.mesh_regions(s.mesh, s.fVertex, s.level, s.M, pair)
        np.testing.assert_array_equal(lc, cc[pair])
        np.testing.assert_array_equal(lec, ec[pair])
        fine, efine = cc[pair] == oracle.RC_FINE, ec[pair] == oracle.RC_FINE
        np.testing.assert_array_equal(lb[fine], np.minimum(6, (cd[pair][fine] + 1) // 2))
        np.testing.assert_array_equal(leb[efine], np.minimum(6, (ed[pair][efine] + 1) // 2))
        # every class of the pair is present (the test sees each set)
        assert {0, 1, 2, 3} <= set(np.unique(lc).tolist())


def test_regions_reject_a_bad_pair():
    s = scenario.gaussian_bump_case(two_level=True)
    with pytest.raises(fb.FbltsError) as e:
        fb.mesh_regions(s.mesh, s.fVertex, s.level, s.M, 1)
    assert e.value.status == fb.E_ARG


def test_library_promotes_levels_like_the_generator():
    """FBLTS_MESH_PROMOTE_LEVELS: nested disks placed without the separation
    the band order needs are refused as given and accepted with the flag; the
    levels the library then uses (read back from the region classes: a cell's
    level is the number of pairs in whose fine region it lies) are those of
    the generator's promotion rule (level l-1 cells closer than 17 layers to
    level >= l+1 move to level l, until stable)."""
    s = scenario.nested_disk_case(nx=64, ny=64, radii=(190e3, 50e3))
    Lx, Ly = s.mesh.period
    dx = scenario._min_image(s.mesh.xCell - Lx / 2, Lx)
    dy = scenario._min_image(s.mesh.yCell - Ly / 2, Ly)
    r2 = dx ** 2 + dy ** 2
    raw = np.zeros(s.mesh.nCells, np.int32)
    raw[r2 <= 190e3 ** 2] = 1
    raw[r2 <= 50e3 ** 2] = 2
    with pytest.raises(fb.FbltsError) as e:
        fb.mesh_regions(s.mesh, s.fVertex, raw, s.M, 0)
    assert e.value.status == fb.E_REGIONS
    want = scenario.enforce_level_separation(s.mesh, raw, min_sep=17)
    assert not np.array_equal(want, raw)
    got = np.zeros(s.mesh.nCells, np.int32)
    for pair in range(2):
        cc, _, _, _ = fb.mesh_regions(s.mesh, s.fVertex, raw, s.M, pair, promote=True)
        got += (cc == fb.REGION_FINE).astype(np.int32)
    np.testing.assert_array_equal(got, want)
