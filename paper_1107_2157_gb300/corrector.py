"""Learned coarse-grid corrector: training and serving drivers.

The drivers only sequence library calls; every arithmetic step runs in
libswe.so: the fine and coarse Lax-Wendroff solvers (swe_batch_*), the
block-average restriction (swe_downsample), the training targets, the
network's forward/backward/AdamW (swe_net_*), and the corrected coarse step
-- by default all coarse steps of a run in one fused persistent launch
(swe_batch_learned_step), otherwise one Lax-Wendroff launch plus the
network's launches per step.

Protocol (fine grid n_fine^2, coarse grid n_fine/factor, dt_coarse =
factor * dt_fine):
  * training pair at coarse step k of a trajectory: input c_k = R(u_f(4k)),
    target residual R(u_f(4k+4)) - LW_c(c_k), where R is the factor x factor
    block average and LW_c the coarse Lax-Wendroff step;
  * corrected step: c_{k+1} = LW_c(c_k) + NN(c_k), the h part of NN made
    zero-mean per image so the step keeps the Lax-Wendroff mass; the
    network reads c_k through its FP32 Lax-Wendroff increment
    LW_c(c_k) - c_k (normalised), which BF16 resolves far better than the
    state itself (h ~ 1 carries its curvature in the 4th digit);
  * error of a coarse run after K steps: RMS of h against R(u_f(4K)).
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Dict, List, Optional

import numpy as np

import swe_inputs as si

from .swe import Batch, Net, flatten_params, swe_downsample, swe_resample


@dataclasses.dataclass
class Setup:
    n_fine: int = 1024
    factor: int = 4
    dt_fine: float = 0.04
    coarse_steps: int = 64
    g: float = 9.8
    dam_fraction: float = 0.1

    @property
    def n_coarse(self) -> int:
        return self.n_fine // self.factor


def init_params(seed: int = 0, hidden: int = 32, out_scale: float = 0.01) -> np.ndarray:
    """He-style initial weights (W[ky][kx][c_in][c_out]), flat float32."""
    rng = np.random.default_rng(seed)

    def w(ci, co, scale):
        return rng.standard_normal((3, 3, ci, co)) * scale / math.sqrt(9 * ci)

    p = dict(W1=w(3, hidden, math.sqrt(2.0)), b1=np.zeros(hidden), W2=w(hidden, hidden, math.sqrt(2.0)),
             b2=np.zeros(hidden), W3=w(hidden, 3, out_scale), b3=np.zeros(3))
    return flatten_params(p)


class _Pair:
    """B fine instances and B coarse instances of the same trajectories."""

    def __init__(self, setup: Setup, B: int, stream):
        import torch
        self.s = setup
        self.B = B
        self.stream = stream
        nf, nc = setup.n_fine, setup.n_coarse
        self.fine = Batch([(nf, nf)] * B, 1.0, 1.0, setup.dt_fine, setup.g)
        self.coarse = Batch([(nc, nc)] * B, float(setup.factor), float(setup.factor),
                            setup.factor * setup.dt_fine, setup.g)
        self.next = torch.zeros((B, 3, nc, nc), dtype=torch.float32, device="cuda")
        self.target = torch.zeros_like(self.next)

    def close(self):
        self.fine.close()
        self.coarse.close()

    @staticmethod
    def geom(batch: Batch):
        p0, plane, pitch = batch.state_ptr(0)
        img = (batch.state_ptr(1)[0] - p0) // 4 if batch.n > 1 else 3 * plane
        return p0, img, plane, pitch

    def load(self, states: List[si.State]):
        sp = self.stream
        for i, st in enumerate(states):
            self.fine.set_state(i, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)), stream=sp)
        self.restrict_to_coarse()

    def restrict_to_coarse(self):
        f0, fimg, fpl, fpi = self.geom(self.fine)
        c0, cimg, cpl, cpi = self.geom(self.coarse)
        nc = self.s.n_coarse
        swe_downsample(self.s.factor, f0, fimg, fpl, fpi, c0, cimg, cpl, cpi, nc, nc, self.B, stream=self.stream)

    def restrict_to_next(self):
        f0, fimg, fpl, fpi = self.geom(self.fine)
        nc = self.s.n_coarse
        swe_downsample(self.s.factor, f0, fimg, fpl, fpi, self.next.data_ptr(), 3 * nc * nc, nc * nc, nc, nc, nc,
                       self.B, stream=self.stream)


def compute_norm(setup: Setup, seeds, B: int, stream) -> List[float]:
    """Scales from one pass over a chunk of trajectories: the median over
    images of the RMS Lax-Wendroff increment (h; momenta) and of the RMS
    target residual (h; momenta).  Medians keep the few dam-break images,
    whose shock residuals are two orders larger, from setting the scale."""
    import torch
    pair = _Pair(setup, B, stream)
    try:
        pair.load(si.corrector_states(seeds[:B], setup.n_fine, setup.dam_fraction))
        inc_h, inc_u, res_h, res_u = [], [], [], []
        for k in range(setup.coarse_steps):
            take = k % 4 == 0
            if take:
                torch.cuda.synchronize()
                c = np.stack([np.stack(pair.coarse.get_state(i)) for i in range(pair.B)])
            pair.coarse.step(1, stream=stream)
            pair.fine.step(setup.factor, stream=stream)
            if take:
                pair.restrict_to_next()
                torch.cuda.synchronize()
                lw = np.stack([np.stack(pair.coarse.get_state(i)) for i in range(pair.B)])
                nxt = pair.next.cpu().numpy()
                d, r = lw - c, nxt - lw
                inc_h += list(np.sqrt((d[:, 0] ** 2).mean(axis=(1, 2))))
                inc_u += list(np.sqrt((d[:, 1:] ** 2).mean(axis=(1, 2, 3))))
                res_h += list(np.sqrt((r[:, 0] ** 2).mean(axis=(1, 2))))
                res_u += list(np.sqrt((r[:, 1:] ** 2).mean(axis=(1, 2, 3))))
            pair.restrict_to_coarse()
        med = [max(float(np.median(v)), 1e-9) for v in (inc_h, inc_u, res_h, res_u)]
        return [0.0, med[0], med[1], med[2], med[3]]
    finally:
        pair.close()


def train(setup: Setup, seeds, B: int = 32, lr: float = 1e-3, epochs: int = 1, params: Optional[np.ndarray] = None,
          norm: Optional[List[float]] = None, clip: float = 1.0, log_every: int = 0, wd: float = 0.0,
          gen_batch: int = 64, passes: int = 1, seed: int = 0, target_clip: float = 0.0,
          loss_power: float = 1.5, loss_floor: float = 1.0) -> Dict:
    """Trains the corrector on trajectories generated on the fly.

    Trajectories are generated gen_batch at a time; all their (input, target)
    pairs over the coarse steps go to a device buffer -- the coarse state c_k,
    its Lax-Wendroff result LW_c(c_k) and the normalised target residual,
    clipped to +-target_clip (0 = no clip) -- which is shuffled and consumed
    in minibatches of B (``passes`` times).  The loss is the mean squared
    error, each image weighted by max(ms, loss_floor)^(-loss_power/2), ms
    the mean square of its target (loss_power = 0: plain MSE).  The network input is the increment
    LW_c(c_k) - c_k.  The learning rate follows a cosine from lr to lr/20.
    Returns dict(params, norm, losses, seconds, steps)."""
    import torch
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    seeds = list(seeds)
    gen_batch = min(gen_batch, len(seeds))
    if norm is None:
        norm = compute_norm(setup, seeds, min(gen_batch, 32), sp)
    nc = setup.n_coarse
    K = setup.coarse_steps
    P = gen_batch * K
    Xc = torch.zeros((P, 3, nc, nc), dtype=torch.float32, device="cuda")
    Xl = torch.zeros_like(Xc)
    T = torch.zeros_like(Xc)
    net = Net(B, nc, nc)
    net.set_params(init_params(0) if params is None else params)
    net.set_norm(*norm)
    net.set_loss_weighting(loss_power, loss_floor)
    pair = _Pair(setup, gen_batch, sp)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    chunks = [seeds[c:c + gen_batch] for c in range(0, len(seeds) - gen_batch + 1, gen_batch)]
    total = max(1, epochs * len(chunks) * passes * (P // B))
    img = 3 * nc * nc
    losses = []
    t0 = time.perf_counter()
    steps = 0
    try:
        for ep in range(epochs):
            for chunk in chunks:
                pair.load(si.corrector_states(chunk, setup.n_fine, setup.dam_fraction))
                for k in range(K):
                    sl = slice(k * gen_batch, (k + 1) * gen_batch)
                    pair.coarse.copy_states(Xc[sl].data_ptr(), stream=sp)
                    pair.coarse.step(1, stream=sp)
                    pair.coarse.copy_states(Xl[sl].data_ptr(), stream=sp)
                    pair.fine.step(setup.factor, stream=sp)
                    pair.restrict_to_next()
                    l0, limg, lpl, lpi = _Pair.geom(pair.coarse)
                    net.make_target(gen_batch, pair.next.data_ptr(), l0, limg, lpl, lpi, T[sl].data_ptr(),
                                    clip=target_clip, stream=sp)
                    pair.restrict_to_coarse()
                for _ in range(passes):
                    perm = torch.randperm(P, generator=gen).cuda()
                    Cs, Ls, Ts = Xc.index_select(0, perm), Xl.index_select(0, perm), T.index_select(0, perm)
                    for j in range(P // B):
                        frac = steps / total
                        lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * frac)))
                        net.prep_input(B, Ls[j * B].data_ptr(), img, nc * nc, nc, base_ptr=Cs[j * B].data_ptr(),
                                       stream=sp)
                        loss, _ = net.train_step(B, Ts[j * B].data_ptr(), lr=lr_t, wd=wd, clip=clip, stream=sp)
                        losses.append(loss)
                        steps += 1
                        if log_every and steps % log_every == 0:
                            print("step %d loss %.4e lr %.2e" % (steps, np.mean(losses[-log_every:]), lr_t),
                                  flush=True)
                    del Cs, Ls, Ts
        out = net.get_params()
    finally:
        pair.close()
        net.close()
    return dict(params=out, norm=norm, losses=losses, seconds=time.perf_counter() - t0, steps=steps)


def coarse_run(setup: Setup, states: List[si.State], params: Optional[np.ndarray], norm, project_mass=True,
               steps: Optional[int] = None, net: Optional[Net] = None, stream=None, timing=None, fused=True):
    """Coarse runs (plain LW if params is None, else LW + corrector) from the
    restricted initial states; returns the coarse Batch (caller closes)."""
    import torch
    sp = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    K = setup.coarse_steps if steps is None else steps
    B = len(states)
    pair = _Pair(setup, B, sp)
    pair.load(states)
    pair.fine.close()
    coarse = pair.coarse
    own = None
    if params is not None and net is None:
        # the fused step reads only the weights: no activation buffers needed
        own = net = Net(1, 8, 8) if fused else Net(B, setup.n_coarse, setup.n_coarse)
        net.set_params(params)
        net.set_norm(*norm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if params is None:
        coarse.step(K, stream=sp)
    elif fused:
        coarse.learned_step(net, K, project_mass=project_mass, stream=sp)
    else:
        for _ in range(K):
            c0 = _Pair.geom(coarse)[0]  # c_k stays in the other buffer after the step
            coarse.step(1, stream=sp)
            l0, limg, lpl, lpi = _Pair.geom(coarse)
            net.prep_input(B, l0, limg, lpl, lpi, base_ptr=c0, stream=sp)
            net.correct(B, l0, limg, lpl, lpi, project_mass=project_mass, stream=sp)
    torch.cuda.synchronize()
    if timing is not None:
        timing.append(time.perf_counter() - t0)
    if own is not None:
        own.close()
    return coarse


def fine_truth(setup: Setup, states: List[si.State], stream=None, timing=None, factor_out: Optional[int] = None,
               tune: bool = False):
    """Fine runs to the final time, restricted to the coarse grid: [B][3][nc][nc]."""
    import torch
    sp = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    B = len(states)
    pair = _Pair(setup, B, sp)
    try:
        for i, st in enumerate(states):
            pair.fine.set_state(i, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)), stream=sp)
        if tune:
            pair.fine.tune(stream=sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pair.fine.step(setup.coarse_steps * setup.factor, stream=sp)
        torch.cuda.synchronize()
        if timing is not None:
            timing.append(time.perf_counter() - t0)
        pair.restrict_to_next()
        torch.cuda.synchronize()
        return pair.next.cpu().numpy()
    finally:
        pair.close()


def load_fine(setup: Setup, states: List[si.State], stream=None) -> Batch:
    """The fine initial states in a fine batch (caller closes)."""
    import torch
    sp = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    b = Batch([(setup.n_fine, setup.n_fine)] * len(states), 1.0, 1.0, setup.dt_fine, setup.g)
    for i, st in enumerate(states):
        b.set_state(i, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)), stream=sp)
    return b


def plain_at(setup: Setup, fine0: Batch, N: int, stream=None, timing=None, tune: bool = False) -> np.ndarray:
    """The plain method at N x N cells (spacing n_fine / N, time step
    dt_fine n_fine / N) from the area average of the fine batch's current
    state, run to the coarse run's final time; returns its final state area
    averaged onto the coarse grid, [B][3][nc][nc]."""
    import torch
    sp = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    nf, nc, B = setup.n_fine, setup.n_coarse, fine0.n
    f = nf / N
    steps = setup.coarse_steps * setup.factor * N // nf
    assert steps * nf == setup.coarse_steps * setup.factor * N, "N must divide the fine time steps evenly"
    b = Batch([(N, N)] * B, f, f, setup.dt_fine * f, setup.g)
    try:
        f0, fimg, fpl, fpi = _Pair.geom(fine0)
        p0, img, pl, pi = _Pair.geom(b)
        swe_resample(f0, fimg, fpl, fpi, nf, nf, p0, img, pl, pi, N, N, B, stream=sp)
        if tune:
            b.tune(stream=sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(steps, stream=sp)
        torch.cuda.synchronize()
        if timing is not None:
            timing.append(time.perf_counter() - t0)
        out = torch.zeros((B, 3, nc, nc), dtype=torch.float32, device="cuda")
        p0, img, pl, pi = _Pair.geom(b)
        swe_resample(p0, img, pl, pi, N, N, out.data_ptr(), 3 * nc * nc, nc * nc, nc, nc, nc, B, stream=sp)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        b.close()


def rms_h_error_arrays(h: np.ndarray, truth: np.ndarray) -> np.ndarray:
    """Per-instance RMS of h ([B][3][nc][nc] arrays) against the truth."""
    return np.sqrt(((h[:, 0].astype(np.float64) - truth[:, 0]) ** 2).mean(axis=(1, 2)))


def rms_h_error(coarse: Batch, truth: np.ndarray) -> np.ndarray:
    """Per-instance RMS error of h against the restricted fine solution."""
    out = []
    for i in range(coarse.n):
        h = coarse.get_state(i)[0]
        out.append(float(np.sqrt(np.mean((h.astype(np.float64) - truth[i, 0]) ** 2))))
    return np.array(out)


def serve(setup: Setup, states: List[si.State], params: np.ndarray, norm, mass_tol: float = 1e-5,
          fallback: bool = True, project_mass: bool = True, stream=None, fused: bool = True) -> Dict:
    """Learned-coarse serving of a batch of instances with checks.

    Runs the corrected coarse step for every instance (all steps in one
    fused launch unless fused=False), then flags an
    instance whose relative mass drift exceeds ``mass_tol`` or whose depth
    became non-positive (or not finite) during the run; flagged instances are
    recomputed with the plain fine solver from their fine initial state and
    their output replaced by its restriction.  Returns dict(coarse: Batch
    (caller closes), flagged: bool array, seconds: wall time of the whole job
    including the fallback, learned_seconds, fallback_seconds)."""
    import torch
    from .swe import SWE_FLAG_NONPOSITIVE
    sp = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    B = len(states)
    K = setup.coarse_steps
    nc = setup.n_coarse
    pair = _Pair(setup, B, sp)
    pair.load(states)
    pair.fine.close()
    coarse = pair.coarse
    net = Net(1, 8, 8) if fused else Net(B, nc, nc)
    net.set_params(params)
    net.set_norm(*norm)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m0 = coarse.mass(stream=sp)
        if fused:
            coarse.learned_step(net, K, project_mass=project_mass, stream=sp)
        else:
            for _ in range(K):
                c0 = _Pair.geom(coarse)[0]
                coarse.step(1, stream=sp)
                l0, limg, lpl, lpi = _Pair.geom(coarse)
                net.prep_input(B, l0, limg, lpl, lpi, base_ptr=c0, stream=sp)
                net.correct(B, l0, limg, lpl, lpi, project_mass=project_mass, stream=sp)
        rc, flags = coarse.status(stream=sp)
        m1 = coarse.mass(stream=sp)
        t1 = time.perf_counter()
        drift = np.abs(m1 - m0) / np.abs(m0)
        bad = ((flags & SWE_FLAG_NONPOSITIVE) != 0) | ~np.isfinite(drift) | (drift > mass_tol)
        t_fb = 0.0
        if fallback and bad.any():
            idx = np.nonzero(bad)[0]
            fb = _Pair(setup, len(idx), sp)
            try:
                for j, i in enumerate(idx):
                    st = states[i]
                    fb.fine.set_state(j, *(a.astype(np.float32) for a in (st.h, st.hu, st.hv)), stream=sp)
                fb.fine.step(K * setup.factor, stream=sp)
                fb.restrict_to_next()
                for j, i in enumerate(idx):
                    f = fb.next[j]
                    coarse.set_state(int(i), f[0], f[1], f[2], stream=sp)
                torch.cuda.synchronize()
            finally:
                fb.close()
            t_fb = time.perf_counter() - t1
        return dict(coarse=coarse, flagged=bad, drift=drift, seconds=time.perf_counter() - t0,
                    learned_seconds=t1 - t0, fallback_seconds=t_fb, status=int(rc))
    finally:
        net.close()
