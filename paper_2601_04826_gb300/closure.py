"""Learned closure pipeline: level-4 training data, GPU training, runs to a final time.

Every numerical step runs in the library's kernels through the C ABI:
  * the level-N reference runs are a batched ensemble (zoomy_ensemble_step), one slip coefficient
    per member drawn from the lognormal law of the ensemble workload;
  * zoomy_closure_samples turns snapshots of those states into (features, targets) on the device;
  * zoomy_mlp_train_step trains the 6 -> 64 -> 64 -> 6 network (Adam) on device mini-batches;
  * zoomy_closure_set hands the trained FP32 weights to the closed level-1 solver.
torch only holds device memory and does the bookkeeping between calls (scale factors from max-abs
values, a seeded permutation of the samples); the paper's model itself trains no network, the
closure is the data-driven form of its exchangeable "material closure" (Sec. 1, Sec. 3.4).
"""
from __future__ import annotations

import numpy as np

from . import inputs, zoomy

NPARAMS = 4998
G = 9.81


def init_params(seed=0):
    """Glorot-normal weights, zero biases, in the library's parameter order (float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in ((6, 64), (64, 64), (64, 6)):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (a + b)), size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def generate_samples(nmembers=32, side=64, level=4, T=2.0, snapshots=8, seed=0, nu=0.01, cfl=0.45, h_dry=1e-6):
    """Run nmembers seeded bump members (side x side, walls, flat bed, slip ~ logNormal(-2, 0.5))
    with the level-`level` solver to about time T and extract every cell of `snapshots` evenly
    spaced snapshots per member.  Returns (F, Y, lam): device float32 [n, 6] raw features
    (h, u_m, v_m, alpha_1, beta_1, lambda), raw targets (alpha_2..4, beta_2..4) and the members'
    slip coefficients."""
    import torch

    _, lam, seeds = inputs.ensemble_members(nmembers, seed=seed)
    sides = np.full(nmembers, side, dtype=np.int64)
    Q0, offs = inputs.ensemble_state(sides, seeds, level)
    ctx = zoomy.zoomy_ensemble_create(sides, lam, level, nu=nu, g=G, cfl=cfl, h_dry=h_dry)
    try:
        Q = torch.tensor(Q0, dtype=torch.float32, device="cuda")
        ld = Q.stride(0)
        # steps per snapshot from the initial CFL step of the fastest member (dt varies little)
        smax = np.sqrt(G * (1.0 + 0.5)) * 1.2
        dt0 = cfl * (0.5 / side) / smax
        per = max(1, int(round(T / dt0 / snapshots)))
        ones = torch.ones(6, dtype=torch.float32, device="cuda")
        per_member = side * side
        cells = torch.arange(int(offs[-1]), dtype=torch.int64, device="cuda")
        F = torch.empty((snapshots * int(offs[-1]), 6), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(F)
        n = 0
        for _ in range(snapshots):
            zoomy.zoomy_ensemble_step(ctx, Q, ld, per, 0)
            for m in range(nmembers):
                c = cells[int(offs[m]):int(offs[m]) + per_member]
                zoomy.zoomy_closure_samples(Q, ld, level, c, per_member, float(lam[m]), h_dry, ones, ones,
                                            F[n:n + per_member], Y[n:n + per_member])
                n += per_member
        torch.cuda.synchronize()
    finally:
        zoomy.zoomy_mesh_destroy(ctx)
    return F, Y, np.asarray(lam)


def scales(F, Y):
    """in_scale = 1 / max|feature|, out_scale = max|target| per column (zoomy_sample_scales)."""
    ins, outs = zoomy.zoomy_sample_scales(F, Y, F.shape[0])
    return np.asarray(ins, dtype=np.float64), np.asarray(outs, dtype=np.float64)


def fit(F, Y, in_scale, out_scale, steps=3000, batch=16384, lr=3e-3, lr_final=1e-3, seed=0, params=None):
    """Train on mini-batches of a seeded permutation of the samples (deterministic).  Returns
    (params float32 [4998], list of (step, loss) every 500 steps).  F and Y are left unchanged."""
    import torch

    ins = torch.tensor(in_scale, dtype=torch.float32, device=F.device)
    outs = torch.tensor(out_scale, dtype=torch.float32, device=F.device)
    g = torch.Generator(device=F.device)
    g.manual_seed(seed)
    perm = torch.randperm(F.shape[0], generator=g, device=F.device)
    X = F[perm].contiguous()  # a shuffled copy, scaled in place by the library
    T = Y[perm].contiguous()
    zoomy.zoomy_sample_scale(X, T, X.shape[0], ins, outs)
    n = X.shape[0]
    batch = min(batch, n)
    nb = n // batch
    mlp = zoomy.zoomy_mlp_create(init_params(seed) if params is None else params)
    hist = []
    try:
        for it in range(steps):
            b = it % nb
            rate = lr if it < (2 * steps) // 3 else lr_final
            want = (it + 1) % 500 == 0
            loss = zoomy.zoomy_mlp_train_step(mlp, X[b * batch:], T[b * batch:], batch, rate, want_loss=want)
            if want:
                hist.append((it + 1, loss))
        p = zoomy.zoomy_mlp_get_params(mlp)
    finally:
        zoomy.zoomy_mlp_destroy(mlp)
    return p, hist


def advance_to(ctx, Q, T, chunk=256):
    """Advance a context's state with CFL steps and land exactly on time T (zoomy_advance).  Returns
    the number of steps taken."""
    _, steps = ctx.advance(Q, T, chunk)
    return steps


class Run:
    """One structured 2D FP32 run of a bump member: level `level`, or level 1 closed by a trained
    network (closure=(params, in_scale, out_scale)) evaluated on the schedule given (0: every stage
    input, 1: once per step)."""

    def __init__(self, side, level, lam, member_seed, nu=0.01, cfl=0.45, h_dry=1e-6, closure=None, schedule=0):
        lv = 1 if closure is not None else level
        self.ctx = zoomy.Context(zoomy.mesh_2d(side, side, bc=(1, 1, 1, 1)), lv,
                                 zoomy.friction(zoomy.FRICTION_SLIP_NEWTONIAN, C=lam, nu=nu), g=G, cfl=cfl,
                                 h_dry=h_dry, dtype=zoomy.FP32)
        self.ctx.cfl = cfl
        if closure is not None:
            p, i, o = closure
            zoomy.zoomy_closure_set(self.ctx.ctx, p, i, o, lam)
            zoomy.zoomy_closure_schedule(self.ctx.ctx, schedule)
        self.Q = self.initial(side, lv, member_seed)

    @staticmethod
    def initial(side, level, member_seed):
        """The member's initial state (the ensemble workload's Gaussian bump at rest, flat bed)."""
        import torch

        Q0, _ = inputs.gaussian_bump_2d(side, side, level, seed=int(member_seed), bathymetry=False)
        return torch.tensor(Q0, dtype=torch.float32, device="cuda")

    def autotune(self):
        """Tune the structured decomposition of a plain level-N run (the closed stage sizes its own)."""
        return self.ctx.autotune(self.Q)

    def run_to(self, T):
        return advance_to(self.ctx, self.Q, T)

    def mean_state(self):
        """(h, h u_m, h v_m) on the host, float64 [3, side^2]."""
        return self.Q[:3].double().cpu().numpy()

    def close(self):
        self.ctx.close()
