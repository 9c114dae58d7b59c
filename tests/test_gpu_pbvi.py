"""GPU parity of the PBVI lower bound (Sec. IV-B, Eq. 8): the pessimistic
start, belief set expansion, one backup, V_PBVI and the whole schedule
through the C ABI against the oracle on the same inputs.

The oracle takes Eq. 8's argmaxes as written (exact ties to the lowest
index).  Where one of a point's decisions is a near-tie in the oracle's own
scores (best and second-best candidates within 1e-4 * scale), FP32 and FP64
may order the candidates differently, so the test replays the oracle's
decisions for that point into the GPU backup (qv_pbvi_backup_fixed); every
other decision is the GPU's own and must equal the oracle's.  Where only
sampled points of a backup are recomputed by the oracle (or for V_PBVI's
vector), a near-tie is reported instead: the GPU's pick must score within
the margin of the oracle's best.  Values |d| <= 1e-5 * max(|ref|, 1) (FP32
against FP64) for one backup, 1e-4 after a schedule of many backups.
Sampled observations match except at draws the oracle flags as lying within
1e-6 of a CDF step."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL
from test_gpu_parity import _close

pytestmark = pytest.mark.gpu

REL = 1e-5
GAP = 1e-4


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _dead(w):
    d = w.occ.ravel().astype(bool).copy()
    d[w.goal] = True
    return d


def _beliefs(w, m, seed, support=None):
    """m random FP32 beliefs on the free cells (dense, or on `support` cells)."""
    rng = np.random.default_rng(seed)
    free = np.flatnonzero(w.occ.ravel() == 0)
    out = np.zeros((m, w.H * w.W), np.float32)
    for j in range(m):
        idx = free if support is None else rng.choice(free, size=min(support, len(free)), replace=False)
        out[j, idx] = rng.random(len(idx)).astype(np.float32)
        out[j] /= out[j].sum()
    return out


def _vectors(w, m, seed):
    rng = np.random.default_rng([5, seed])
    G = rng.normal(-10.0, 15.0, (m, w.H * w.W)).astype(np.float32)
    G[:, _dead(w)] = 0.0
    return G


def _grid(m, a):
    a = np.asarray(a, np.float32)
    return m.to_grid(a.reshape(-1, m.H, m.W))


def _flat(m, t):
    return m.from_grid(t).reshape(t.shape[0], -1).astype(np.float64)


def _check_argmax(got, scores, scale, what):
    """got: chosen index; scores: the oracle's candidates (FP64)."""
    s = np.sort(scores)
    top = s[-1]
    if len(s) > 1 and top - s[-2] > GAP * scale:
        assert got == int(np.argmax(scores)), f"{what}: {got} vs {int(np.argmax(scores))}"
    else:
        assert scores[got] >= top - GAP * scale, f"{what}: pick {got} scores {scores[got]} < max {top}"


def _near(scores, scale):
    s = np.sort(np.asarray(scores))
    return len(s) > 1 and s[-1] - s[-2] <= GAP * scale


def _oracle_fixes(o, scale):
    """The oracle's a* and winners for every point with a near-tie among
    its decisions (any action's Q, any observation's vectors); -1 elsewhere,
    where the GPU decides on its own."""
    nB, _, nz, _ = o["score"].shape
    fa = np.full(nB, -1, np.int32)
    fb = np.full((nB, nz), -1, np.int32)
    for j in range(nB):
        near = _near(o["q"][j], scale) or any(_near(o["score"][j, a, z], scale) for a in range(5)
                                               for z in range(nz))
        if near:
            fa[j] = o["astar"][j]
            fb[j] = o["best"][j]
    return fa, fb


def test_init_matches_oracle(api):
    for w in (WL.tiny(0), WL.diff(0, H=40, W=36), WL.mid(1, H=67, W=45)):
        m = api.Model(w)
        got = m.from_grid(api.pbvi_init(m)).reshape(-1)
        _close(got, O.pbvi_init(w), rel=1e-6, floor=1.0, what="alpha0")


@pytest.mark.parametrize("make", [lambda: WL.tiny(0), lambda: WL.tiny(3, H=13, W=17),
                                  lambda: WL.mid(1, H=67, W=45), lambda: WL.large(0, H=96, W=80)])
def test_expand_matches_oracle(api, make):
    w = make()
    m = api.Model(w)
    B = _beliefs(w, 24, 1)
    B[0] = w.b0.ravel()
    for rnd in (0, 5):
        g = api.pbvi_expand(m, _grid(m, B), rnd, seed=7)
        o = O.pbvi_expand(w, B.astype(np.float64), rnd, seed=7)
        assert np.array_equal(g["action"].cpu().numpy(), o["action"])
        gz = g["obs"].cpu().numpy()
        bad = (gz != o["obs"]) & (o["boundary"] == 0)
        assert not bad.any(), f"{int(bad.sum())} observations differ away from a CDF step"
        gp = _flat(m, g["points"])
        for j in np.flatnonzero(gz == o["obs"]):
            _close(gp[j], o["points"][j], what=f"point {j}")


def _backup_case(api, w, nB, nG, seed, support=None):
    m = api.Model(w)
    B = _beliefs(w, nB, seed, support)
    G = _vectors(w, nG, seed)
    pb = api.Pbvi(m, max(nB, nG))
    pb.set_points(_grid(m, B))
    o = O.pbvi_backup(w, B.astype(np.float64), G.astype(np.float64), want_score=True)
    scale = max(1.0, float(np.abs(o["q"]).max()))
    fa, fb = _oracle_fixes(o, scale)
    r = pb.backup(_grid(m, G), fix_astar=fa, fix_best=fb)
    torch.cuda.synchronize()
    gv = r["value"].cpu().numpy()
    ga = r["astar"].cpu().numpy()
    gb = r["best"].cpu().numpy()
    gq = r["q"].cpu().numpy()
    _close(gq, o["q"], floor=scale, what="Q_b(a)")
    _close(gv, o["value"], floor=scale, what="value")
    # every decision, the GPU's own or replayed at a near-tie, is the oracle's
    assert np.array_equal(ga, o["astar"]), "a*"
    assert np.array_equal(gb, o["best"]), "winning vectors"
    GG = _flat(m, r["G"])
    for j in range(nB):
        _close(GG[j], o["G"][j], floor=scale, what=f"alpha of point {j}")
        # the new vector gives the backed-up value at its own point
        assert abs(GG[j] @ B[j].astype(np.float64) - gv[j]) <= REL * scale * 10
        assert np.all(GG[j][_dead(w)] == 0.0)
    return m, pb, int((fa >= 0).sum())


@pytest.mark.parametrize("make,nB,nG", [(lambda: WL.tiny(0), 5, 4), (lambda: WL.tiny(2, H=13, W=17), 7, 3),
                                       (lambda: WL.diff(1, H=24, W=20), 6, 6)])
def test_backup_matches_oracle(api, make, nB, nG):
    _backup_case(api, make(), nB, nG, 3)


def test_backup_many_tiles_and_pieces(api):
    # 330 rows (3 tiles of 128) by 65 vectors (one tile), 17 labels, sparse
    # beliefs so the oracle's literal sums stay short
    w = WL.mid(2, H=67, W=45)
    _backup_case(api, w, 66, 65, 4, support=40)


def test_backup_ragged_vector_tiles(api):
    # 60 points (300 rows: 3 row tiles, the last ragged) by 300 vectors (two
    # column tiles of 256, the second ragged), sparse beliefs
    w = WL.mid(3, H=67, W=45)
    _backup_case(api, w, 60, 300, 5, support=40)


def test_backup_at_1024_points_sampled(api):
    # the benchmarked size: 1024 points on the mid map, one backup against
    # 1024 vectors (the test's own dense beliefs and vectors); the oracle's
    # Eq. 8 backup at sampled points against the same vectors gives the same
    # value and a*
    w = WL.mid(0)
    m = api.Model(w)
    B = _beliefs(w, 1024, 11)
    G = _vectors(w, 1024, 11)
    pb = api.Pbvi(m, 1024)
    pb.set_points(_grid(m, B))
    r = pb.backup(_grid(m, G))
    torch.cuda.synchronize()
    gv = r["value"].cpu().numpy()
    ga = r["astar"].cpu().numpy()
    pts = [0, 1023]  # one oracle call: its points run in parallel
    o = O.pbvi_backup(w, B[pts].astype(np.float64), G.astype(np.float64))
    for t, j in enumerate(pts):
        scale = max(1.0, float(np.abs(o["q"][t]).max()))
        assert abs(gv[j] - o["value"][t]) <= REL * scale * 10, j
        _check_argmax(int(ga[j]), o["q"][t], scale, f"a* of point {j}")


def test_value_matches_oracle(api):
    w = WL.mid(1, H=40, W=52)
    m = api.Model(w)
    G = _vectors(w, 70, 2)
    b = _beliefs(w, 90, 2, support=60)
    pb = api.Pbvi(m, 96)
    pb.set_points(_grid(m, b[:1]))
    v, arg = pb.value(_grid(m, G), _grid(m, b))
    s = b.astype(np.float64) @ G.astype(np.float64).T
    scale = max(1.0, float(np.abs(s).max()))
    _close(v.cpu().numpy(), s.max(axis=1), floor=scale, what="V_PBVI")
    for j, a in enumerate(arg.cpu().numpy()):
        _check_argmax(int(a), s[j], scale, f"V_PBVI vector of belief {j}")


@pytest.mark.parametrize("seed", [0, 1])
def test_solve_matches_oracle_schedule(api, seed):
    # the schedule of pbvi_solve, run on both sides backup by backup: the
    # oracle on its own FP64 chain, the GPU on its own FP32 chain with the
    # oracle's decisions replayed at the points where they are near-ties
    rounds, iters = 3, 12
    w = WL.tiny(seed, H=10, W=11)
    m = api.Model(w)
    B = w.b0.ravel().astype(np.float64)[None].copy()
    G = O.pbvi_init(w)[None]
    nmax = 1 << rounds
    Bg = torch.zeros((nmax, m.H, m.P), dtype=torch.float32, device="cuda")
    Bg[0] = m.b0()
    Gg = torch.zeros_like(Bg)
    Gg[0] = api.pbvi_init(m)
    G2 = torch.empty_like(Gg)
    pb = api.Pbvi(m, nmax)
    nB = nG = 1
    replayed = 0
    for r in range(rounds + 1):
        pb.set_points(Bg[:nB])
        for _ in range(iters):
            o = O.pbvi_backup(w, B, G, want_score=True)
            scale = max(1.0, float(np.abs(o["q"]).max()))
            fa, fb = _oracle_fixes(o, scale)
            replayed += int((fa >= 0).sum())
            res = pb.backup(Gg[:nG], out=G2[:nB], fix_astar=fa, fix_best=fb)
            assert np.array_equal(res["astar"].cpu().numpy(), o["astar"])
            assert np.array_equal(res["best"].cpu().numpy(), o["best"])
            Gg, G2 = G2, Gg
            nG = nB
            G = o["G"]
        if r < rounds:
            e = O.pbvi_expand(w, B, r, seed=seed)
            assert int(e["boundary"].sum()) == 0
            api.pbvi_expand(m, Bg[:nB], r, seed, out=Bg[nB:2 * nB])
            B = np.concatenate([B, e["points"]])
            nB *= 2
    gB = _flat(m, Bg[:nB])
    assert gB.shape == B.shape
    _close(gB, B, rel=1e-4, what="belief set")
    ov = O.pbvi_value(G, B)
    scale = max(1.0, float(np.abs(ov).max()))
    gv, _ = pb.value(Gg[:nG], Bg[:nB])
    _close(gv.cpu().numpy(), ov, rel=1e-4, floor=scale, what="V_PBVI at the points")
    _close(_flat(m, Gg[:nG]), G, rel=1e-4, floor=scale, what="alpha-vectors")


def test_full_size_lower_bound(api):
    # the mid map: 64 points after six expansion rounds; V_PBVI below V_FIB
    # at every point (both solved on the GPU: a property at any size)
    w = WL.mid(0)
    m = api.Model(w)
    g = api.pbvi_solve(m, rounds=6, iters=8, seed=3)
    fib = api.fib_value_iterate(m, dtype="f32")["Q"]
    B = _flat(m, g["B"])
    F = m.from_grid(fib).reshape(5, -1).astype(np.float64)
    vf = (B @ F.T).max(axis=1)
    vp = g["value"].cpu().numpy()
    assert np.all(vp <= vf + 1e-4 * np.maximum(1.0, np.abs(vf)))


def test_large_map_backup_sampled(api):
    # the 512x512 map: a backup of the test's own points against its own
    # vectors, the oracle's Eq. 8 backup at sampled points
    w = WL.large(1)
    m = api.Model(w)
    B = _beliefs(w, 8, 4, support=4000)
    G = _vectors(w, 6, 4)
    pb = api.Pbvi(m, 8)
    pb.set_points(_grid(m, B))
    r = pb.backup(_grid(m, G))
    gv = r["value"].cpu().numpy()
    ga = r["astar"].cpu().numpy()
    o = O.pbvi_backup(w, B[3:5].astype(np.float64), G.astype(np.float64))
    for t, j in enumerate((3, 4)):
        scale = max(1.0, float(np.abs(o["q"][t]).max()))
        assert abs(gv[j] - o["value"][t]) <= REL * scale * 10, j
        _check_argmax(int(ga[j]), o["q"][t], scale, f"a* of point {j}")


def test_errors(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(0)
    m = api.Model(w)
    pb = api.Pbvi(m, 4)
    G = torch.zeros((8, m.H, m.P), dtype=torch.float32, device="cuda")
    with pytest.raises(N.QVError) as ei:
        pb.backup(G[:1])                      # no point set yet
    assert ei.value.status == N.QV_ERR_INVALID
    with pytest.raises(N.QVError):
        pb.set_points(G[:5])                  # more points than the handle holds
    pb.set_points(_grid(m, _beliefs(w, 2, 0)))
    with pytest.raises(N.QVError):
        pb.backup(G[:5])                      # more vectors than the handle holds
    with pytest.raises(N.QVError):
        pb.backup(G[:2], out=G[1:3])          # output overlaps the input
    r = pb.backup(G[:2])
    assert torch.isfinite(r["value"]).all()


def test_value_reuses_its_vectors_until_a_backup(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(1)
    m = api.Model(w)
    G = _grid(m, _vectors(w, 6, 1))
    b = _grid(m, _beliefs(w, 9, 1))
    pb = api.Pbvi(m, 16)
    pb.set_points(b[:3])
    v1, a1 = pb.value(G, b)
    v2, a2 = pb.value(None, b, nG=6)
    assert torch.equal(v1, v2) and torch.equal(a1, a2)
    with pytest.raises(N.QVError):
        pb.value(None, b, nG=5)          # a different count was not kept
    pb.backup(G)                          # reorders other vectors
    with pytest.raises(N.QVError) as ei:
        pb.value(None, b, nG=6)
    assert ei.value.status == N.QV_ERR_INVALID
