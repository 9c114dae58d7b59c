"""Thin Python binding over the C ABI of include/qvts.h.

Argument marshalling only: tensors in, device pointers and the current CUDA
stream out to libqvts.so.  Every step of the computation runs in the CUDA
library; nothing here computes any part of the method.  PyTorch provides the
device memory and the stream.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _native as N
from ._native import check, lib

__all__ = ["Model", "Plan", "qv_model_build", "mdp_value_iterate", "mdp_value_iterate_checkpointed",
           "mdp_value_backward", "belief_predict", "belief_correct", "leaf_value", "qv_tree_plan",
           "qv_tree_plan_batched", "qv_tree_backward", "autotune", "tune_clear", "pitch_of"]


def pitch_of(W: int) -> int:
    """QV_PITCH(W): row pitch in cells, a multiple of 8."""
    return (W + 7) // 8 * 8


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def qv_model_build(H, W, pitch, occ, beacons, B, sense_range, goal, cell, stream=None):
    """Cell words of one grid (occ uint8 [H][pitch], beacons int32 [B], cell int16 [H][pitch])."""
    check(lib().qv_model_build(H, W, pitch, _ptr(occ), _ptr(beacons), B, sense_range, goal, _ptr(cell),
                               _stream(stream)), "qv_model_build")
    return cell


class Model:
    """Device form of one generated problem: the padded grids, the cell words
    written by qv_model_build, and the qv_model_t that points at them."""

    def __init__(self, w, device="cuda", slip=None, accuracy=None, cost="workload", stream=None):
        self.w = w
        self.H, self.W = w.H, w.W
        self.P = pitch_of(w.W)
        self.B = w.B
        self.device = torch.device(device)
        occ = np.ones((self.H, self.P), np.uint8)
        occ[:, :self.W] = w.occ
        self.occ = torch.from_numpy(occ).to(self.device)
        self.beacons = torch.from_numpy(np.asarray([self.pcell(b) for b in w.beacons], np.int32)).to(self.device)
        self.goal = self.pcell(w.goal)
        self.cell = torch.empty((self.H, self.P), dtype=torch.int16, device=self.device)
        qv_model_build(self.H, self.W, self.P, self.occ, self.beacons, self.B, w.sense_range, self.goal,
                       self.cell, stream)
        c = w.cost if isinstance(cost, str) else cost
        self.cost = None if c is None else self.to_grid(c if torch.is_tensor(c) else np.asarray(c, np.float32))
        self.slip = float(w.slip if slip is None else slip)
        self.accuracy = float(w.accuracy if accuracy is None else accuracy)
        self.discount = float(w.discount)
        self.sense_range = int(w.sense_range)
        self.struct = N.qv_model_t(self.H, self.W, self.P, self.cell.data_ptr(), self.B, self.goal,
                                   self.slip, self.accuracy, self.discount,
                                   None if self.cost is None else self.cost.data_ptr(),
                                   self.beacons.data_ptr(), self.sense_range)

    def pcell(self, x: int) -> int:
        """Unpadded cell index r*W + c -> pitched index r*pitch + c."""
        r, c = divmod(int(x), self.W)
        return r * self.P + c

    def to_grid(self, a) -> torch.Tensor:
        """[..., H, W] array -> float32 [..., H, pitch] device tensor (padding 0)."""
        a = torch.as_tensor(np.asarray(a, np.float32) if not torch.is_tensor(a) else a)
        a = a.reshape(*a.shape[:-1], self.H, self.W) if a.shape[-1] == self.H * self.W else a
        out = torch.zeros(*a.shape[:-2], self.H, self.P, dtype=torch.float32, device=self.device)
        out[..., :self.W] = a.to(self.device, torch.float32)
        return out

    def from_grid(self, t: torch.Tensor) -> np.ndarray:
        """[..., H, pitch] -> numpy [..., H*W] (unpadded, row-major)."""
        t = t.reshape(*t.shape[:-1], self.H, self.P) if t.shape[-1] == self.H * self.P else t
        a = t[..., :self.W].detach().cpu().numpy()
        return a.reshape(*a.shape[:-2], self.H * self.W)

    def b0(self) -> torch.Tensor:
        return self.to_grid(self.w.b0)


def mdp_value_iterate(model: Model, dtype="f32", tol=None, max_sweeps=100000, truncated=None, stream=None):
    """Returns dict(V [H][pitch], Q [5][H][pitch] float32, sweeps, residual, status)."""
    w = model.w
    tol = w.vi_tol if tol is None else tol
    truncated = w.vi_truncated if truncated is None else truncated
    dt = N.QV_F64 if dtype in ("f64", torch.float64) else N.QV_F32
    V = torch.zeros((model.H, model.P), dtype=torch.float64 if dt == N.QV_F64 else torch.float32,
                    device=model.device)
    Q = torch.empty((5, model.H, model.P), dtype=torch.float32, device=model.device)
    nbytes = lib().mdp_value_iterate_workspace_bytes(C.byref(model.struct), dt)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.device)
    sweeps = C.c_int32(0)
    res = C.c_double(0)
    st = lib().mdp_value_iterate(C.byref(model.struct), dt, float(tol), int(max_sweeps), int(truncated), _ptr(V),
                                 _ptr(Q), _ptr(ws), nbytes, C.byref(sweeps), C.byref(res), _stream(stream))
    if st not in (N.QV_OK, N.QV_ERR_NOT_CONVERGED):
        check(st, "mdp_value_iterate")
    return dict(V=V, Q=Q, sweeps=sweeps.value, residual=res.value, status=st)


def fib_value_iterate(model: Model, dtype="f32", tol=None, max_sweeps=100000, truncated=None, want_alpha=True,
                      stream=None):
    """The Fast Informed Bound alpha-vectors (Eq. 7).  Returns dict(alpha
    [5][H][pitch] in `dtype` or None, Q [5][H][pitch] float32 -- the leaf
    alpha-vectors of a plan whose leaves take V_FIB -- sweeps, residual, status)."""
    w = model.w
    tol = w.vi_tol if tol is None else tol
    truncated = w.vi_truncated if truncated is None else truncated
    dt = N.QV_F64 if dtype in ("f64", torch.float64) else N.QV_F32
    alpha = None
    if want_alpha:
        alpha = torch.empty((5, model.H, model.P), dtype=torch.float64 if dt == N.QV_F64 else torch.float32,
                            device=model.device)
    Q = torch.empty((5, model.H, model.P), dtype=torch.float32, device=model.device)
    nbytes = lib().fib_value_iterate_workspace_bytes(C.byref(model.struct), dt)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.device)
    sweeps = C.c_int32(0)
    res = C.c_double(0)
    st = lib().fib_value_iterate(C.byref(model.struct), dt, float(tol), int(max_sweeps), int(truncated),
                                 _ptr(alpha), _ptr(Q), _ptr(ws), nbytes, C.byref(sweeps), C.byref(res),
                                 _stream(stream))
    if st not in (N.QV_OK, N.QV_ERR_NOT_CONVERGED):
        check(st, "fib_value_iterate")
    return dict(alpha=alpha, Q=Q, sweeps=sweeps.value, residual=res.value, status=st)


def pbvi_init(model: Model, stream=None) -> torch.Tensor:
    """The pessimistic PBVI start alpha_0 (R_min / (1 - gamma)), [H][pitch]."""
    a0 = torch.empty((model.H, model.P), dtype=torch.float32, device=model.device)
    check(lib().qv_pbvi_init(C.byref(model.struct), _ptr(a0), _stream(stream)), "qv_pbvi_init")
    return a0


def pbvi_expand(model: Model, B: torch.Tensor, rnd: int, seed: int, out=None, stream=None):
    """One round of belief set expansion: a new point from each of the nB
    points of B [nB][H][pitch].  Returns dict(points, action, obs, boundary)."""
    nB = B.shape[0]
    out = torch.empty_like(B) if out is None else out
    a = torch.empty(nB, dtype=torch.int32, device=B.device)
    z = torch.empty(nB, dtype=torch.int32, device=B.device)
    bd = torch.empty(nB, dtype=torch.int32, device=B.device)
    check(lib().qv_pbvi_expand(C.byref(model.struct), _ptr(B.contiguous()), nB, int(rnd), int(seed), _ptr(out),
                               _ptr(a), _ptr(z), _ptr(bd), _stream(stream)), "qv_pbvi_expand")
    return dict(points=out, action=a, obs=z, boundary=bd)


class Pbvi:
    """Point-based value iteration on one model (Eq. 8): a belief set of up
    to `max_points` points and the C ABI handle with its workspace."""

    def __init__(self, model: Model, max_points: int):
        self.model = model
        self.max_points = int(max_points)
        h = C.c_void_p()
        check(lib().qv_pbvi_create(C.byref(model.struct), self.max_points, C.byref(h)), "qv_pbvi_create")
        self.handle = h
        self.ws_bytes = lib().qv_pbvi_workspace_bytes(h)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=model.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = C.c_void_p(self.ws.data_ptr() + off)
        self.nB = 0

    def layout(self):
        seg = (C.c_int32 * (self.model.B + 2))()
        Kp = lib().qv_pbvi_layout(self.handle, seg)
        return Kp, list(seg)

    def set_points(self, B: torch.Tensor, stream=None):
        self.B = B.contiguous()
        self.nB = self.B.shape[0]
        check(lib().qv_pbvi_set_points(self.handle, _ptr(self.B), self.nB, self.ws_ptr, self.ws_bytes,
                                       _stream(stream)), "qv_pbvi_set_points")

    def backup(self, G: torch.Tensor, out=None, stream=None, fix_astar=None, fix_best=None):
        """One Eq. 8 backup at every point of the set given G [nG][H][pitch].
        Returns dict(G [nB][H][pitch], value, astar, best [nB][B+1], q [nB][5]).
        fix_astar [nB] / fix_best [nB][B+1] (int32 arrays, -1 = not fixed):
        decisions taken as given (qv_pbvi_backup_fixed)."""
        nB, m = self.nB, self.model
        out = torch.empty((nB, m.H, m.P), dtype=torch.float32, device=m.device) if out is None else out
        value = torch.empty(nB, dtype=torch.float32, device=m.device)
        astar = torch.empty(nB, dtype=torch.int32, device=m.device)
        best = torch.empty((nB, m.B + 1), dtype=torch.int32, device=m.device)
        q = torch.empty((nB, 5), dtype=torch.float32, device=m.device)
        fa = fb = None
        if fix_astar is not None:
            fa = torch.as_tensor(np.ascontiguousarray(np.asarray(fix_astar, np.int32).reshape(nB))).to(m.device)
        if fix_best is not None:
            fb = torch.as_tensor(np.ascontiguousarray(np.asarray(fix_best, np.int32).reshape(nB, m.B + 1))).to(m.device)
        self._fixed = (fa, fb)  # alive until the next backup (the launch reads them asynchronously)
        check(lib().qv_pbvi_backup_fixed(self.handle, _ptr(G.contiguous()), G.shape[0], _ptr(out), _ptr(value),
                                         _ptr(astar), _ptr(best), _ptr(q), _ptr(fa), _ptr(fb), _stream(stream)),
              "qv_pbvi_backup_fixed")
        return dict(G=out, value=value, astar=astar, best=best, q=q)

    def value(self, G: Optional[torch.Tensor], b: torch.Tensor, nG: Optional[int] = None, stream=None):
        """V_PBVI(b) and the maximising vector's index for beliefs b [nb][H][pitch].
        G = None (with nG) reuses the vectors of the previous call."""
        nb = b.shape[0]
        v = torch.empty(nb, dtype=torch.float32, device=b.device)
        arg = torch.empty(nb, dtype=torch.int32, device=b.device)
        n = G.shape[0] if G is not None else int(nG)
        check(lib().qv_pbvi_value(self.handle, None if G is None else _ptr(G.contiguous()), n, _ptr(b.contiguous()),
                                  nb, _ptr(v), _ptr(arg), _stream(stream)), "qv_pbvi_value")
        return v, arg

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().qv_pbvi_destroy(h)
            self.handle = None


def pbvi_solve(model: Model, rounds: int, iters: int, seed: int = 0, b0: Optional[torch.Tensor] = None,
               stream=None):
    """The PBVI schedule the oracle's pbvi_solve follows: from B = {b0} and
    Gamma = {alpha_0}, `rounds` times (`iters` Eq. 8 backups, then one
    expansion round), then `iters` more backups.  Returns dict(B, G, value,
    pbvi) with value = V_PBVI at every point."""
    nmax = 1 << rounds
    m = model
    B = torch.zeros((nmax, m.H, m.P), dtype=torch.float32, device=m.device)
    B[0] = m.b0() if b0 is None else b0
    pb = Pbvi(m, nmax)
    G = torch.zeros((nmax, m.H, m.P), dtype=torch.float32, device=m.device)
    G[0] = pbvi_init(m, stream)
    G2 = torch.empty_like(G)
    nB, nG = 1, 1
    for r in range(rounds + 1):
        pb.set_points(B[:nB], stream)
        for _ in range(iters):
            pb.backup(G[:nG], out=G2[:nB], stream=stream)
            G, G2 = G2, G
            nG = nB
        if r < rounds:
            pbvi_expand(m, B[:nB], r, seed, out=B[nB:2 * nB], stream=stream)
            nB *= 2
    v, _ = pb.value(G[:nG], B[:nB], stream)
    return dict(B=B[:nB], G=G[:nG], value=v, pbvi=pb)


class BestFirst:
    """Alg. 1's best-first planning loop on one model: U from the upper-bound
    alpha-vectors Qu (FP32 [5][H][pitch], e.g. FIB), L from PBVI (a Pbvi
    handle with its vectors G), K forward samples per (V-node, action)."""

    def __init__(self, model: Model, Qu: torch.Tensor, pbvi: "Pbvi", G: torch.Tensor, K=8, seed=0, episode=0,
                 max_depth=6, max_nodes=4096):
        self.model, self.Qu, self.pbvi, self.G = model, Qu, pbvi, G.contiguous()
        h = C.c_void_p()
        check(lib().qv_bf_create(C.byref(model.struct), _ptr(Qu), pbvi.handle, _ptr(self.G), self.G.shape[0],
                                 int(K), int(seed), int(episode), int(max_depth), int(max_nodes), C.byref(h)),
              "qv_bf_create")
        self.handle = h
        self.ws_bytes = lib().qv_bf_workspace_bytes(h)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=model.device)
        self.ws_ptr = C.c_void_p(self.ws.data_ptr() + (-self.ws.data_ptr()) % 256)

    def reset(self, b0: Optional[torch.Tensor] = None, stream=None):
        b = self.model.b0() if b0 is None else b0.contiguous()
        self._b0 = b
        check(lib().qv_bf_reset(self.handle, _ptr(b), self.ws_ptr, self.ws_bytes, _stream(stream)), "qv_bf_reset")

    def run(self, iters: int, stream=None):
        check(lib().qv_bf_run(self.handle, int(iters), _stream(stream)), "qv_bf_run")

    def set_replay(self, expand=None):
        """Fix the node expanded at iteration t to expand[t] where that is >= 0
        (qv_bf_set_replay); None clears it."""
        if expand is None:
            self._replay = None
            check(lib().qv_bf_set_replay(self.handle, None, 0), "qv_bf_set_replay")
            return
        self._replay = torch.as_tensor(np.ascontiguousarray(np.asarray(expand, np.int32))).to(self.model.device)
        check(lib().qv_bf_set_replay(self.handle, _ptr(self._replay), int(self._replay.numel())),
              "qv_bf_set_replay")

    def read(self, stream=None) -> dict:
        r = N.qv_bf_result_t()
        check(lib().qv_bf_read(self.handle, C.byref(r), _stream(stream)), "qv_bf_read")
        return dict(iterations=r.iterations, nodes=r.nodes, stopped=r.stopped, root_action=r.root_action,
                    U=r.U, L=r.L, H=r.H, E=r.E, q=list(r.q), boundary_samples=r.boundary_samples)

    def tree(self) -> dict:
        """Host copies of the tree's arrays (the first `nodes` entries)."""
        n = self.read()["nodes"]
        v = N.qv_bf_view_t()
        check(lib().qv_bf_view(self.handle, C.byref(v)), "qv_bf_view")
        base = self.ws.data_ptr()

        def arr(ptr, count, dt):
            off = ptr - base
            esz = torch.tensor([], dtype=dt).element_size()
            return self.ws[off:off + count * esz].view(dt)

        m = self.model
        out = {}
        for k, dt in (("parent", torch.int32), ("action", torch.int32), ("obs", torch.int32), ("depth", torch.int32),
                      ("weight", torch.float32), ("U", torch.float32), ("L", torch.float32), ("H", torch.float32),
                      ("E", torch.int32)):
            out[k] = arr(getattr(v, "d_" + k), n, dt).cpu().numpy()
        for k, dt in (("R", torch.float32), ("UQ", torch.float32), ("LQ", torch.float32), ("HQ", torch.float32),
                      ("EQ", torch.int32), ("first", torch.int32), ("count", torch.int32)):
            out[k] = arr(getattr(v, "d_" + k), n * 5, dt).view(n, 5).cpu().numpy()
        out["expanded"] = arr(v.d_expanded, v.max_nodes, torch.int32).cpu().numpy()
        out["belief"] = arr(v.d_belief, n * m.H * m.P, torch.float32).view(n, m.H, m.P)
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().qv_bf_destroy(h)
            self.handle = None


def run_episodes(model: Model, Q: torch.Tensor, b0s: Sequence[torch.Tensor], starts: Sequence[int], depth=3, K=8,
                 seed=0, max_steps=100, check_every=8, history=False, stream=None) -> dict:
    """Closed-loop episodes (Alg. 1's outer loop) of E = len(b0s) robots on
    one map: each step one batched plan (episode e plans from belief e with
    Philox episode word step * E + e), the true system's step (qv_env_step)
    and the belief update (qv_belief_update_batched), with no host wait
    inside a step; every `check_every` steps the host reads whether all
    episodes ended.  starts: unpadded cells.  Returns dict(steps, success,
    ret, states [E], steps_run) on the host; with history, also the states
    [steps_run + 1][E] and measurements [steps_run][E] (-1 once ended),
    copied on the device each step."""
    E = len(b0s)
    dev = model.device
    B = torch.stack([b.contiguous() for b in b0s]).contiguous()
    state = torch.tensor([model.pcell(int(s)) for s in starts], dtype=torch.int32, device=dev)
    obs = torch.full((E,), -1, dtype=torch.int32, device=dev)
    steps = torch.zeros(E, dtype=torch.int32, device=dev)
    ret = torch.zeros(E, dtype=torch.float32, device=dev)
    done = (state == model.goal).to(torch.int32)
    nws = lib().qv_belief_update_batched_workspace_bytes(C.byref(model.struct), E)
    ws = torch.empty(nws + 256, dtype=torch.uint8, device=dev)
    wsp = C.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
    stride = C.c_int32(0)
    hist_s = torch.full((max_steps + 1, E), -1, dtype=torch.int32, device=dev) if history else None
    hist_z = torch.full((max_steps, E), -1, dtype=torch.int32, device=dev) if history else None
    if history:
        hist_s[0].copy_(state)
    # one batched plan for every step: it reads the beliefs B in place, and
    # the step's Philox episode word t * E comes from a device word written
    # on the stream before each run
    plan = Plan([model] * E, [Q] * E, [B[e] for e in range(E)], depth=depth, K=K, seed=seed, episode=0,
                stream=stream)
    word = torch.zeros(1, dtype=torch.int32, device=dev)
    plan.set_episode_word(word)
    act = lib().qv_plan_actions_device(plan.handle, C.byref(stride))
    cs = torch.cuda.current_stream(dev) if stream is None else stream
    t = 0
    for t in range(max_steps):
        with torch.cuda.stream(cs):
            word.fill_(t * E)
        plan.run(stream)
        check(lib().qv_env_step(C.byref(model.struct), E, act, stride.value, _ptr(state), int(seed), t, _ptr(obs),
                                _ptr(steps), _ptr(ret), _ptr(done), _stream(stream)), "qv_env_step")
        check(lib().qv_belief_update_batched(C.byref(model.struct), E, _ptr(B), act, stride.value, _ptr(obs), wsp,
                                             nws, _stream(stream)), "qv_belief_update_batched")
        if history:
            hist_s[t + 1].copy_(state)
            hist_z[t].copy_(obs)
        if (t + 1) % check_every == 0 and bool(done.all()):
            t += 1
            break
    else:
        t = max_steps
    def unpad(a):
        return np.where(a >= 0, (a // model.P) * model.W + a % model.P, -1)

    out = dict(steps=steps.cpu().numpy(), success=done.cpu().numpy(), ret=ret.cpu().numpy(),
               states=unpad(state.cpu().numpy().astype(np.int64)), steps_run=t, beliefs=B)
    if history:
        out["state_history"] = unpad(hist_s[:t + 1].cpu().numpy().astype(np.int64))
        out["obs_history"] = hist_z[:t].cpu().numpy()
    return out


def forward_sample(model: Model, B: torch.Tensor, actions, paths, K: int, level=0, seed=0, episode=0, stream=None):
    """Alg. 4's ancestral sampler: K measurements for each (belief B[j],
    action actions[j]) with Philox path paths[j].  Returns int32 [n][K]."""
    n = B.shape[0]
    a = torch.as_tensor(actions, dtype=torch.int32, device=B.device).contiguous()
    pth = torch.as_tensor(paths, dtype=torch.int64, device=B.device).contiguous()
    z = torch.empty((n, K), dtype=torch.int32, device=B.device)
    nws = lib().qv_forward_sample_workspace_bytes(C.byref(model.struct), n)
    ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=B.device)
    check(lib().qv_forward_sample(C.byref(model.struct), n, _ptr(B.contiguous()), _ptr(a), _ptr(pth), int(level),
                                  int(seed), int(episode), int(K), _ptr(z), _ptr(ws), nws, _stream(stream)),
          "qv_forward_sample")
    return z


def mdp_value_iterate_checkpointed(model: Model, sweeps: int, every: int = 16, stream=None):
    """Exactly `sweeps` FP64 sweeps from V_0 = 0, keeping V_k at every k that
    is a multiple of `every` for mdp_value_backward.  Returns dict(V (FP64),
    Q (FP32 [5][H][pitch]), ckpt (FP64 [ceil(sweeps/every)][H][pitch]),
    sweeps, every)."""
    J = (int(sweeps) + int(every) - 1) // int(every)
    V = torch.empty((model.H, model.P), dtype=torch.float64, device=model.device)
    Q = torch.empty((5, model.H, model.P), dtype=torch.float32, device=model.device)
    ck = torch.empty((J, model.H, model.P), dtype=torch.float64, device=model.device)
    nbytes = lib().mdp_value_iterate_workspace_bytes(C.byref(model.struct), N.QV_F64)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.device)
    check(lib().mdp_value_iterate_checkpointed(C.byref(model.struct), int(sweeps), int(every), _ptr(V), _ptr(Q),
                                               _ptr(ck), _ptr(ws), nbytes, _stream(stream)),
          "mdp_value_iterate_checkpointed")
    return dict(V=V, Q=Q, ckpt=ck, sweeps=int(sweeps), every=int(every))


def mdp_value_backward(model: Model, vi: dict, Qbar: torch.Tensor, dslip: torch.Tensor,
                       dcost: Optional[torch.Tensor] = None, stream=None):
    """Accumulates dL/dslip (FP64 device scalar) and dL/dc (FP64 [H][pitch])
    through the checkpointed sweeps `vi`, given Qbar = dL/dQ (FP64 [5][H][pitch])."""
    nbytes = lib().mdp_value_backward_workspace_bytes(C.byref(model.struct), vi["every"])
    ws = torch.empty(nbytes, dtype=torch.uint8, device=model.device)
    check(lib().mdp_value_backward(C.byref(model.struct), vi["sweeps"], vi["every"], _ptr(vi["ckpt"]),
                                   _ptr(Qbar.contiguous()), _ptr(dslip), _ptr(dcost), _ptr(ws), nbytes,
                                   _stream(stream)), "mdp_value_backward")
    return dslip, dcost


def belief_predict(model: Model, b: torch.Tensor, action: int, out=None, stream=None):
    out = torch.empty_like(b) if out is None else out
    check(lib().belief_predict(C.byref(model.struct), _ptr(b), int(action), _ptr(out), _stream(stream)),
          "belief_predict")
    return out


def belief_correct(model: Model, bbar: torch.Tensor, z: int, out=None, stream=None):
    out = torch.empty_like(bbar) if out is None else out
    pz = torch.empty(1, dtype=torch.float32, device=bbar.device)
    nbytes = lib().belief_correct_workspace_bytes(C.byref(model.struct))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=bbar.device)
    check(lib().belief_correct(C.byref(model.struct), _ptr(bbar), int(z), _ptr(out), _ptr(pz), _ptr(ws), nbytes,
                               _stream(stream)), "belief_correct")
    return out, pz


def _check_tensor(t, shape, device, fn, what):
    """Raise ValueError unless t is a contiguous float32 tensor on `device`
    (a CUDA device) of the given shape, or of at least one element when
    shape is None."""
    want_dev = torch.device(device)
    ok = (torch.is_tensor(t) and t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()
          and t.device.index == (want_dev.index if want_dev.index is not None else torch.cuda.current_device())
          and t.numel() >= 1
          and (shape is None or tuple(t.shape) == tuple(shape)))
    if not ok:
        desc = (f"{tuple(t.shape)} {t.dtype} on {t.device}, contiguous={t.is_contiguous()}"
                if torch.is_tensor(t) else type(t).__name__)
        want = f"shape {tuple(shape)}" if shape is not None else "at least one element"
        raise ValueError(f"{fn}: {what} must be a contiguous float32 tensor on {device} with {want}, got {desc}")


def belief_correct_noalloc(model: Model, bbar: torch.Tensor, z: int, out: torch.Tensor, pz: torch.Tensor,
                           stream=None):
    """belief_correct without a workspace: the library keeps the reduction's
    scratch in a fixed device array, so the call itself allocates nothing.
    The caller provides `out` (like bbar) and `pz` (one float32 on the device).
    Every tensor is checked (float32, contiguous, on the model's device,
    bbar and out of shape (H, pitch)) before the library is called: the C ABI
    takes bare pointers and would write through a host or undersized one."""
    dev = model.device
    for t, what in ((bbar, "bbar"), (out, "out")):
        _check_tensor(t, (model.H, model.P), dev, "belief_correct_noalloc", what)
    _check_tensor(pz, None, dev, "belief_correct_noalloc", "pz")
    check(lib().belief_correct_noalloc(C.byref(model.struct), _ptr(bbar), int(z), _ptr(out), _ptr(pz),
                                       _stream(stream)), "belief_correct_noalloc")
    return out, pz


def leaf_value(model: Model, Q: torch.Tensor, b: torch.Tensor, stream=None):
    n = b.shape[0] if b.dim() == 3 else 1
    out = torch.empty(n, dtype=torch.float32, device=b.device)
    check(lib().leaf_value(C.byref(model.struct), _ptr(Q), _ptr(b.contiguous()), n, _ptr(out), _stream(stream)),
          "leaf_value")
    return out


def _params(depth, K, seed, episode, weight_mode, leaf_mode, replay, band_cells=0, items_per_cta=0, grid_ctas=0,
            deadline_ms=0.0, deepest_form=0):
    return N.qv_plan_params_t(int(depth), int(K), int(seed), int(episode), int(weight_mode), int(leaf_mode),
                              None if replay is None else replay.data_ptr(), int(band_cells), int(items_per_cta),
                              int(grid_ctas), float(deadline_ms), int(deepest_form))


def _result_dict(r: N.qv_plan_result_t, depth: int):
    return dict(action=int(r.action), value=float(r.value), q=np.array(list(r.q), np.float32),
                nodes_per_level=[int(r.nodes_per_level[l]) for l in range(depth + 1)],
                boundary_samples=int(r.boundary_samples), depth_reached=int(r.depth_reached))


class Plan:
    """One batch of E episodes laid out in a caller workspace (a torch tensor).

    run() launches the search (asynchronous, no host synchronisation);
    read() synchronises and returns the root results; capture_graph() turns
    later run() calls into one CUDA-graph launch; level() exposes the device
    arrays of one tree level as tensors viewing the workspace."""

    def __init__(self, models: Sequence[Model], Qs: Sequence[torch.Tensor], b0s: Sequence[torch.Tensor],
                 depth=2, K=4, seed=0, episode=0, weight_mode=N.QV_WEIGHT_FREQ, leaf_mode=N.QV_LEAF_FUSED,
                 replay: Optional[torch.Tensor] = None, stream=None, band_cells=0, items_per_cta=0, grid_ctas=0,
                 deadline_ms=0.0, deepest_form=0):
        self.models = list(models)
        self.E = len(self.models)
        self.depth, self.K = int(depth), int(K)
        self.Qs = [q.contiguous() for q in Qs]
        self.b0s = [b.contiguous() for b in b0s]
        self.replay = replay
        self.params = _params(depth, K, seed, episode, weight_mode, leaf_mode, replay, band_cells, items_per_cta,
                              grid_ctas, deadline_ms, deepest_form)
        self.mstructs = (N.qv_model_t * self.E)(*[m.struct for m in self.models])
        self.qptrs = (C.c_void_p * self.E)(*[q.data_ptr() for q in self.Qs])
        self.bptrs = (C.c_void_p * self.E)(*[b.data_ptr() for b in self.b0s])
        nbytes = lib().qv_plan_workspace_bytes(self.E, self.mstructs, C.byref(self.params))
        if nbytes == 0:
            raise N.QVError(N.QV_ERR_INVALID, "qv_plan_workspace_bytes")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.models[0].device)
        self.handle = C.c_void_p()
        check(lib().qv_plan_create(self.E, self.mstructs, self.qptrs, self.bptrs, C.byref(self.params),
                                   _ptr(self.ws), nbytes, C.byref(self.handle), _stream(stream)), "qv_plan_create")

    @property
    def workspace_bytes(self):
        return self.ws.numel()

    @property
    def grid(self) -> int:
        """CTAs of the plan's launch."""
        return int(lib().qv_plan_grid(self.handle))

    @property
    def tuning(self) -> dict:
        """The launch-shape knobs this plan was created with."""
        t = N.qv_tune_t()
        check(lib().qv_plan_tuning(self.handle, C.byref(t)), "qv_plan_tuning")
        return dict(band_cells=int(t.band_cells), items_per_cta=int(t.items_per_cta))

    def backward_workspace(self, nbytes: int) -> torch.Tensor:
        """Device scratch for qv_tree_backward, kept with the plan."""
        ws = getattr(self, "_bws", None)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.models[0].device)
            self._bws = ws
        return ws

    def run(self, stream=None):
        check(lib().qv_plan_run(self.handle, _stream(stream)), "qv_plan_run")

    def set_episode_word(self, word: Optional[torch.Tensor]):
        """Draw with the device uint32 word[0] + e (read at every run) as the
        Philox episode word of episode e (qv_plan_set_episode_word); None
        returns to the episode given at creation.  Drops a captured graph."""
        self._episode_word = word
        check(lib().qv_plan_set_episode_word(self.handle, _ptr(word)), "qv_plan_set_episode_word")

    def capture_graph(self, stream=None):
        s = torch.cuda.Stream() if stream is None else stream
        s.wait_stream(torch.cuda.current_stream())
        check(lib().qv_plan_capture_graph(self.handle, C.c_void_p(s.cuda_stream)), "qv_plan_capture_graph")
        torch.cuda.current_stream().wait_stream(s)

    def read(self, stream=None) -> List[dict]:
        res = (N.qv_plan_result_t * self.E)()
        check(lib().qv_plan_read(self.handle, res, _stream(stream)), "qv_plan_read")
        return [_result_dict(res[e], self.depth) for e in range(self.E)]

    def readback_buffer(self) -> torch.Tensor:
        """Pinned host bytes for read_async."""
        return torch.empty(lib().qv_plan_readback_bytes(self.handle), dtype=torch.uint8).pin_memory()

    def read_async(self, buf: torch.Tensor, stream=None):
        """Enqueue the copy of this plan's results into `buf` (no synchronisation)."""
        check(lib().qv_plan_read_async(self.handle, C.c_void_p(buf.data_ptr()), _stream(stream)),
              "qv_plan_read_async")

    def decode(self, buf: torch.Tensor) -> List[dict]:
        """Results from a buffer filled by read_async, once the stream has passed the copy."""
        res = (N.qv_plan_result_t * self.E)()
        check(lib().qv_plan_decode(self.handle, C.c_void_p(buf.data_ptr()), res), "qv_plan_decode")
        return [_result_dict(res[e], self.depth) for e in range(self.E)]

    def profile(self, stream=None) -> List[dict]:
        """One eager run with a CUDA event after every launch (synchronises)."""
        out = (N.qv_launch_time_t * 64)()
        n = C.c_int32(0)
        check(lib().qv_plan_profile(self.handle, out, 64, C.byref(n), _stream(stream)), "qv_plan_profile")
        return [dict(name=out[i].name.decode(), level=int(out[i].level), ms=float(out[i].ms))
                for i in range(n.value)]

    def _view(self, ptr, count, dtype, shape=None):
        if not ptr:
            return None
        esz = torch.tensor([], dtype=dtype).element_size()
        off = ptr - self.ws.data_ptr()
        if 0 <= off < self.ws.numel():
            t = self.ws[off:off + count * esz].view(dtype)
        else:  # level 0 belief is the caller's b0
            return None
        return t if shape is None else t.view(*shape)

    def level(self, e: int, l: int) -> dict:
        v = N.qv_level_view_t()
        check(lib().qv_plan_level(self.handle, e, l, C.byref(v)), "qv_plan_level")
        cap = v.cap
        n = int(self._view(v.d_count, 1, torch.int32).item())
        m = self.models[e]
        out = dict(count=n, cap=cap)
        for key, ptr, dt in (("parent", v.d_parent, torch.int32), ("action", v.d_action, torch.int32),
                             ("obs", v.d_obs, torch.int32), ("weight", v.d_weight, torch.float32),
                             ("pz", v.d_pz, torch.float32), ("value", v.d_value, torch.float32)):
            out[key] = self._view(ptr, cap, dt)[:n]
        for key, ptr, dt in (("R", v.d_R, torch.float32), ("UQ", v.d_UQ, torch.float32),
                             ("nchild", v.d_nchild, torch.int32)):
            t = self._view(ptr, cap * 5, dt, (cap, 5)) if ptr else None
            out[key] = None if t is None else t[:n]
        t = self._view(v.d_samples, cap * 5 * self.K, torch.int32, (cap, 5, self.K)) if v.d_samples else None
        out["samples"] = None if t is None else t[:n]
        t = self._view(v.d_leaf_arg, cap, torch.int32) if v.d_leaf_arg else None
        out["leaf_arg"] = None if t is None else t[:n]
        if l == 0:
            out["belief"] = self.b0s[e].view(1, m.H, m.P)
        else:
            t = self._view(v.d_belief, cap * m.H * m.P, torch.float32, (cap, m.H, m.P)) if v.d_belief else None
            out["belief"] = None if t is None else t[:n]
        return out

    def bounds(self, leaf_L: torch.Tensor, e: int = 0, stream=None) -> List[dict]:
        """AEMS fields of episode e (Alg. 5-7, Eq. 9) from the lower bound of
        every leaf (leaf_L [leaves], float32): per level dict(LV, HV, EV and,
        below the leaves, LQ, HQ, EQ [n][5]); EV/EQ index the leaf level."""
        nbytes = lib().qv_plan_bounds_workspace_bytes(self.handle, e)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.models[e].device)
        ptr = C.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
        check(lib().qv_plan_bounds(self.handle, e, _ptr(leaf_L.contiguous()), ptr, nbytes, _stream(stream)),
              "qv_plan_bounds")
        out = []
        for l in range(self.depth + 1):
            v = N.qv_bounds_view_t()
            check(lib().qv_plan_bounds_view(self.handle, e, l, ptr, C.byref(v)), "qv_plan_bounds_view")
            lv = N.qv_level_view_t()
            check(lib().qv_plan_level(self.handle, e, l, C.byref(lv)), "qv_plan_level")
            cap = lv.cap
            n = int(self._view(lv.d_count, 1, torch.int32).item())
            d = dict(count=n)

            def view(p_, count, dt):
                off = p_ - ws.data_ptr()
                return ws[off:off + 4 * count].view(dt)

            for key, p_, dt in (("LV", v.d_LV, torch.float32), ("HV", v.d_HV, torch.float32),
                                ("EV", v.d_EV, torch.int32)):
                d[key] = view(p_, cap, dt)[:n]
            for key, p_, dt in (("LQ", v.d_LQ, torch.float32), ("HQ", v.d_HQ, torch.float32),
                                ("EQ", v.d_EQ, torch.int32)):
                d[key] = view(p_, cap * 5, dt).view(cap, 5)[:n] if p_ else None
            out.append(d)
        out[0]["_ws"] = ws  # keeps the workspace the views point into alive
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib().qv_plan_destroy(h)
            self.handle = C.c_void_p()


def autotune(models: Sequence[Model], Qs: Sequence[torch.Tensor], b0s: Sequence[torch.Tensor], depth=2, K=4,
             seed=0, episode=0, weight_mode=N.QV_WEIGHT_FREQ, leaf_mode=N.QV_LEAF_FUSED, reps=5, grid_ctas=0,
             stream=None):
    """qv_plan_autotune: time every (band_cells, items_per_cta) candidate on
    these inputs; the best is cached in the library for plans of the same
    shape class created with the knobs left at 0.  Returns (best, all)."""
    E = len(models)
    ms = (N.qv_model_t * E)(*[m.struct for m in models])
    qp = (C.c_void_p * E)(*[q.data_ptr() for q in Qs])
    bp = (C.c_void_p * E)(*[b.data_ptr() for b in b0s])
    params = _params(depth, K, seed, episode, weight_mode, leaf_mode, None, grid_ctas=grid_ctas)
    nbytes = lib().qv_plan_autotune_workspace_bytes(E, ms, C.byref(params))
    if nbytes == 0:
        raise N.QVError(N.QV_ERR_INVALID, "qv_plan_autotune_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=models[0].device)
    best = N.qv_tune_t()
    allv = (N.qv_tune_t * 64)()
    n = C.c_int32(0)
    check(lib().qv_plan_autotune(E, ms, qp, bp, C.byref(params), _ptr(ws), nbytes, int(reps), C.byref(best), allv,
                                 64, C.byref(n), _stream(stream)), "qv_plan_autotune")
    conv = lambda t: dict(band_cells=int(t.band_cells), items_per_cta=int(t.items_per_cta), ms=float(t.ms))  # noqa: E731
    return conv(best), [conv(allv[i]) for i in range(n.value)]


def tune_clear():
    lib().qv_tune_clear()


def qv_tree_backward(plan: Plan, e: int = 0, dL: float = 1.0, Qbar=None, dslip=None, dacc=None, dcost=None,
                     db0=None, want_db0=True, stream=None):
    """Adjoint of episode e's root value (FREQ weights; samples and every
    argmax held fixed).  Accumulates into FP64 device tensors, created zeroed
    when not given: Qbar [5][H][pitch], dslip [1], dacc [1], dcost [H][pitch],
    db0 [H][pitch].  Asynchronous: nothing is read back."""
    m = plan.models[e]
    dev = m.device
    f64 = dict(dtype=torch.float64, device=dev)
    Qbar = torch.zeros((5, m.H, m.P), **f64) if Qbar is None else Qbar
    dslip = torch.zeros(1, **f64) if dslip is None else dslip
    dacc = torch.zeros(1, **f64) if dacc is None else dacc
    dcost = torch.zeros((m.H, m.P), **f64) if dcost is None else dcost
    if db0 is None and want_db0:
        db0 = torch.zeros((m.H, m.P), **f64)
    nbytes = lib().qv_tree_backward_workspace_bytes(plan.handle, int(e))
    if nbytes == 0:
        raise N.QVError(N.QV_ERR_INVALID, "qv_tree_backward_workspace_bytes")
    ws = plan.backward_workspace(nbytes)
    check(lib().qv_tree_backward(plan.handle, int(e), float(dL), _ptr(Qbar), _ptr(dslip), _ptr(dacc), _ptr(dcost),
                                 _ptr(db0), _ptr(ws), nbytes, _stream(stream)), "qv_tree_backward")
    return dict(Qbar=Qbar, dslip=dslip, dacc=dacc, dcost=dcost, db0=db0)


def qv_tree_plan(model: Model, Q: torch.Tensor, b0: torch.Tensor, depth=2, K=4, seed=0, episode=0,
                 weight_mode=N.QV_WEIGHT_FREQ, leaf_mode=N.QV_LEAF_FUSED, replay=None, keep=False, stream=None,
                 deadline_ms=0.0, deepest_form=0):
    """One plan from b0 to the chosen action (Alg. 1 inner loop, one step);
    deadline_ms > 0 stops at the first level that is final after the budget;
    deepest_form picks the deepest fused level's form (N.QV_DEEPEST_*)."""
    p = Plan([model], [Q], [b0], depth, K, seed, episode, weight_mode, leaf_mode, replay, stream,
             deadline_ms=deadline_ms, deepest_form=deepest_form)
    p.run(stream)
    r = p.read(stream)[0]
    return (r, p) if keep else r


def qv_tree_plan_batched(models, Qs, b0s, depth=3, K=8, seed=0, episode=0, weight_mode=N.QV_WEIGHT_FREQ,
                         leaf_mode=N.QV_LEAF_FUSED, stream=None):
    p = Plan(models, Qs, b0s, depth, K, seed, episode, weight_mode, leaf_mode, None, stream)
    p.run(stream)
    return p.read(stream)


class Model9:
    """The paper's experimental model (Sec. V) on one grid: nine actions,
    four occupancy sensors, r in {-2, -1, 0}; its value iteration and plans
    (tree shape fixed at creation: depth <= 3, K <= 16).  Grids are unpadded
    [H][W] tensors on the model's device."""

    def __init__(self, w, depth=None, K=None, device="cuda", stream=None):
        self.w = w
        self.H, self.W = w.H, w.W
        self.device = torch.device(device)
        self.depth = w.depth if depth is None else depth
        self.K = w.K if K is None else K
        self.occ = torch.from_numpy(np.ascontiguousarray(w.occ.astype(np.uint8))).to(self.device)
        self.struct = N.qv9_model_t(int(w.H), int(w.W), _ptr(self.occ), int(w.goal), float(w.slip),
                                    float(w.p_sensor), float(w.discount))
        h = C.c_void_p()
        check(lib().qv9_create(C.byref(self.struct), int(self.depth), int(self.K), C.byref(h)), "qv9_create")
        self.handle = h
        nbytes = lib().qv9_workspace_bytes(h)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = C.c_void_p(self.ws.data_ptr() + (-self.ws.data_ptr()) % 256)
        check(lib().qv9_set_workspace(h, self.ws_ptr, nbytes, _stream(stream)), "qv9_set_workspace")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib().qv9_destroy(h)
            self.handle = None

    def b0(self):
        return torch.from_numpy(np.ascontiguousarray(self.w.b0.astype(np.float32))).to(self.device)

    def value_iterate(self, dtype="f32", tol=None, max_sweeps=100000, truncated=0, stream=None):
        """dict(V [H][W] in dtype, Q [9][H][W] FP32, sweeps, residual)."""
        tdt = torch.float64 if dtype == "f64" else torch.float32
        V = torch.empty((self.H, self.W), dtype=tdt, device=self.device)
        Q = torch.empty((9, self.H, self.W), dtype=torch.float32, device=self.device)
        sw = C.c_int32(0)
        res = C.c_double(0.0)
        tol = self.w.vi_tol if tol is None else tol
        check(lib().qv9_value_iterate(self.handle, N.QV_F64 if dtype == "f64" else N.QV_F32, float(tol),
                                      int(max_sweeps), int(truncated), _ptr(V), _ptr(Q), C.byref(sw), C.byref(res),
                                      _stream(stream)), "qv9_value_iterate")
        return dict(V=V, Q=Q, sweeps=sw.value, residual=res.value)

    def _check_grid(self, t, shape, what):
        if tuple(t.shape) != shape or t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError(f"Model9: {what} must be a float32 CUDA tensor of shape {shape}, "
                             f"got {tuple(t.shape)} {t.dtype} on {t.device}")

    def plan(self, Q, b0=None, seed=None, episode=None, stream=None):
        """One plan: dict(action, value, q [9], nodes_per_level, boundary)."""
        self._check_grid(Q, (9, self.H, self.W), "Q")
        b0 = self.b0() if b0 is None else b0.contiguous()
        self._check_grid(b0, (self.H, self.W), "b0")
        r = N.qv9_plan_result_t()
        check(lib().qv9_plan(self.handle, _ptr(Q.contiguous()), _ptr(b0), int(self.w.seed if seed is None else seed),
                             int(self.w.episode if episode is None else episode), C.byref(r), _stream(stream)),
              "qv9_plan")
        return dict(action=r.action, value=r.value, q=np.array(r.q[:]),
                    nodes_per_level=[int(r.nodes_per_level[l]) for l in range(self.depth + 1)],
                    boundary=int(r.boundary_samples))

    def _view(self, ptr, count, dtype, shape):
        if not ptr or count == 0:
            return None
        esz = torch.tensor([], dtype=dtype).element_size()
        off = ptr - self.ws.data_ptr()
        return self.ws[off:off + count * esz].view(dtype).view(*shape)

    def level(self, l):
        """Level l of the last plan as device tensors (views of the workspace,
        valid until the next plan): count, parent, action, obs, weight, pz,
        value; belief [n][H][W], R and UQ [n][9] for the internal levels."""
        v = N.qv9_level_view_t()
        check(lib().qv9_level(self.handle, int(l), C.byref(v)), "qv9_level")
        n = v.count
        out = dict(count=n)
        for key, dt in (("parent", torch.int32), ("action", torch.int32), ("obs", torch.int32),
                        ("weight", torch.float32), ("pz", torch.float32), ("value", torch.float32)):
            out[key] = self._view(getattr(v, key), n, dt, (n,))
        out["belief"] = self._view(v.belief, n * self.H * self.W, torch.float32, (n, self.H, self.W))
        out["R"] = self._view(v.R, n * 9, torch.float32, (n, 9))
        out["UQ"] = self._view(v.UQ, n * 9, torch.float32, (n, 9))
        return out
