"""The allocation-free diagnostics entry point against the allocating one.

Some callers cannot allocate device memory while they run (they own all
device memory through their own pool, or cudaMalloc/cudaFree would
synchronise the device inside their loop).  fblts_diagnostics_static serves
them with scratch in a static device array; it must give the same totals as
fblts_diagnostics, call after call, with the tolerance the other diagnostics
tests use.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_diagnostics_match_fblts_diagnostics_twice():
    import torch

    import paper_2405_10505_gb300 as fb
    from synth import scenario
    from tests.gpu_util import make_state

    s = scenario.shelf_case(nx=64, ny=48, dc=2e3, M=4, width=10e3)
    st = make_state(s)
    for call in range(2):
        fb.lts_advance(st, 5)
        mass, absvort = fb.diagnostics(st)
        h, u = fb.state_read(st)
        d_h = torch.from_numpy(h).to("cuda")
        d_u = torch.from_numpy(u).to("cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        fb.diagnostics_static(st.mesh, d_h.data_ptr(), d_u.data_ptr(), out.data_ptr(), None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        assert got[0] == pytest.approx(mass, rel=1e-13), (call, got[0], mass)
        assert got[1] == pytest.approx(absvort, rel=1e-12), (call, got[1], absvort)
