"""belief_correct_noalloc: the Bayes correction for callers that cannot
allocate device memory (a loop that must not call cudaMalloc once running,
or a host that owns every device allocation).  Its scratch is a fixed array
inside the library, shared by every call, so these tests check it against
the workspace-taking belief_correct and the oracle's Bayes update on
consecutive calls, and check that an oversized grid is refused.  The file is named to run last."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import _native as N
    from paper_1810_00204_gb300 import api
    return N, api


def _call_noalloc(N, model, bbar, z, out, pz):
    return N.lib().belief_correct_noalloc(C.byref(model.struct), C.c_void_p(bbar.data_ptr()), int(z),
                                          C.c_void_p(out.data_ptr()), C.c_void_p(pz.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("make", [lambda: WL.mid(3, H=96, W=70), lambda: WL.large(1)])
def test_noalloc_matches_workspace_version_on_consecutive_calls(mods, make):
    N, api = mods
    w = make()
    m = api.Model(w)
    rng = np.random.default_rng(17)
    out = torch.empty((m.H, m.P), dtype=torch.float32, device="cuda")
    pz = torch.empty(1, dtype=torch.float32, device="cuda")
    # two calls in a row share the library's scratch; the second must not see
    # anything the first left behind
    for call, z in enumerate((2, w.B)):
        b = rng.random(w.H * w.W) * (1 - w.occ.ravel())
        b = (b / b.sum()).astype(np.float32)
        bbar_o = O.predict(w, b.astype(np.float64), call).astype(np.float32)  # the oracle's prediction
        bbar = m.to_grid(bbar_o.reshape(w.H, w.W))
        ref, ref_pz = api.belief_correct(m, bbar, z)
        out.fill_(-1.0)
        pz.fill_(-1.0)
        assert _call_noalloc(N, m, bbar, z, out, pz) == N.QV_OK
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        o = out.cpu().numpy()
        assert np.abs(o - r).max() <= REL * np.abs(r).max(), f"call {call}"
        assert abs(pz.item() - ref_pz.item()) <= REL * abs(ref_pz.item()), f"call {call}"
        assert o[:, w.W:].max(initial=0.0) == 0.0  # padding columns stay empty
        # and directly against the oracle's Bayes update of the same bbar
        ob, opz = O.correct(w, bbar_o.astype(np.float64), z)
        assert np.abs(o[:, :w.W].ravel() - ob).max() <= REL * np.abs(ob).max(), f"call {call} vs oracle"
        assert abs(pz.item() - opz) <= REL * abs(opz), f"call {call} P(z) vs oracle"


def test_noalloc_refuses_grids_beyond_its_scratch(mods):
    N, api = mods
    w = WL.tiny(0)
    m = api.Model(w)
    big = N.qv_model_t(m.struct.H, m.struct.W, m.struct.pitch, m.struct.d_cell, m.struct.num_beacons,
                       m.struct.goal, m.struct.slip, m.struct.accuracy, m.struct.discount, None,
                       m.struct.d_beacons, m.struct.sense_range)
    big.W = 2048
    big.pitch = 2048
    big.H = N.QV_NOALLOC_MAX_CELLS // 2048 + 1
    x = torch.empty(1, dtype=torch.float32, device="cuda")
    st = N.lib().belief_correct_noalloc(C.byref(big), C.c_void_p(x.data_ptr()), 0, C.c_void_p(x.data_ptr()),
                                        C.c_void_p(x.data_ptr()), None)
    assert st == N.QV_ERR_INVALID
    assert b"static scratch" in N.lib().qv_last_error()
