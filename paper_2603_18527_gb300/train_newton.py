"""Training and evaluation of an FNO preconditioner for the inner systems of
Newton's method on -Lap u - u^2 = f (App. Full Derivations, Nonlinear PDE
via Newton-Born Linearization; App. Experimental Setup, Newton linear
systems: N = 64, s = 1600, FNO with 25 channels, 2 NLFL layers and 20
modes, batch 50, weight decay 1e-6, inner rTol 1e-4) through the library's
C-ABI: ``newton_linearise`` for the trajectory states, ``newton_train_step``
(Eq. nl_bs_loss and the two Euclidean objectives) and ``newton_solve``.

The NPBS networks use the FNO's identity skip (M = I + N, zero projection at
start: the Born series); ``--no-skip`` trains the paper's plain FNO.

Training states: Newton trajectories with Born inner solves from the
perturbed initial guesses of ``synth.newton_instance``; every step m gives a
state (u_m, c_m, r_m).  The unrolled loss starts from an inner iterate delta
drawn per state from a bank: delta = 0 (the paper's G r), the network's own
inner iterates after 2 and 6 iterations (on-policy, refreshed every
``refresh`` steps), and a white-noise field (all frequencies, scaled so that
||J delta|| ~ ||r||).  Starting from smooth G r alone leaves the network
untrained on the high frequencies that float32 rounding of the inner
residual injects at inference, and the inner iteration then diverges.

    python -m paper_2603_18527_gb300.train_newton --compare --steps 2000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

import synth
from . import build, capi

N_DEFAULT = 64
LEVELS = (0, 2, 6)  # inner iterations of the on-policy snapshots; one more level holds white noise


def trajectories(ctx, insts, steps: int, alpha: float = 0.0):
    """States (u, f, u32, shift, r) of each instance's Newton trajectory (Born
    inner solves, inner rTol 1e-4) at Newton steps 0..steps-1: per-state
    records holding device tensors."""
    n = insts[0].n
    b = capi.Batch([(n, n)] * len(insts), h=[1.0 / (n + 1)] * len(insts))
    f = b.pack([i.f for i in insts], dtype=torch.float64)
    u = b.pack([i.u0 for i in insts], dtype=torch.float64)
    out = []
    for m in range(steps):
        sh, u32, r = capi.newton_linearise(ctx, b, u, f, alpha)
        for j, o in enumerate(b.offsets):
            out.append({"u": u[o:o + n * n].clone(), "f": f[o:o + n * n].clone(), "u32": u32[o:o + n * n].clone(),
                        "shift": sh[j], "r": r[o:o + n * n].clone()})
        capi.newton_solve(ctx, None, b, f, u, alpha=alpha, tol=0.0, max_steps=1, inner_rtol=1e-4)
    return out


class StateGroup:
    """A fixed batch of states packed in one layout, with its snapshot bank
    [levels + 1, extent] of inner iterates delta."""

    def __init__(self, states, seed: int):
        n = int(round(math.sqrt(states[0]["u32"].numel())))
        self.n = n
        self.b = capi.Batch([(n, n)] * len(states), h=[1.0 / (n + 1)] * len(states))
        E = self.b.extent
        self.u = torch.zeros(E, dtype=torch.float64, device="cuda")
        self.f = torch.zeros(E, dtype=torch.float64, device="cuda")
        self.u32 = torch.zeros(E, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(E, dtype=torch.complex64, device="cuda")
        for s, o in zip(states, self.b.offsets):
            self.u[o:o + n * n] = s["u"]
            self.f[o:o + n * n] = s["f"]
            self.u32[o:o + n * n] = s["u32"]
            self.r[o:o + n * n] = s["r"]
        self.shift = [s["shift"] for s in states]
        self.bank = torch.zeros((len(LEVELS) + 1, E), dtype=torch.complex64, device="cuda")
        # white noise with ||J delta|| ~ ||r||: ||J|| ~ 8/h^2 on the highest modes
        g = torch.Generator(device="cuda").manual_seed(seed)
        noise = torch.randn(E, dtype=torch.float32, device="cuda", generator=g)
        h2 = 1.0 / (n + 1) ** 2
        for o in self.b.offsets:
            seg = noise[o:o + n * n]
            rn = float(self.r[o:o + n * n].abs().norm())
            self.bank[-1, o:o + n * n] = (seg * (rn * h2 / 8.0 / max(float(seg.norm()), 1e-30))).to(torch.complex64)

    def refresh(self, ctx, net):
        """The network's inner iterates after LEVELS[l] iterations from delta = 0."""
        for l, k in enumerate(LEVELS):
            if k == 0:
                continue
            u = self.u.clone()
            capi.newton_solve(ctx, net, self.b, self.f, u, tol=0.0, max_steps=1, inner_rtol=0.0, inner_max_iter=k,
                              check_every=k)
            d = (u - self.u).to(torch.complex64)
            for o in self.b.offsets:
                seg = d[o:o + self.n * self.n]
                # a diverged iterate (non-finite, or far beyond the O(10) Newton corrections) restarts from zero
                if not bool(torch.isfinite(torch.view_as_real(seg)).all()) or float(seg.abs().max()) > 1e6:
                    seg.zero_()
            self.bank[l] = d

    def draw(self, rng) -> torch.Tensor:
        d = torch.empty(self.b.extent, dtype=torch.complex64, device="cuda")
        lv = rng.integers(0, self.bank.shape[0], size=len(self.shift))
        for j, o in enumerate(self.b.offsets):
            d[o:o + self.n * self.n] = self.bank[lv[j], o:o + self.n * self.n]
        return d


def make_net(n=N_DEFAULT, width=25, modes=20, layers=2, seed=0, skip=True):
    """The Newton FNO; skip: M = I + N (zero projection at start, the Born series)."""
    return capi.Net.fno(n, width, modes, layers, seed=seed, skip=skip)


def train(ctx, net, groups, steps, lr=1e-3, lr_min=1e-5, wd=1e-6, unroll=4, seed=0, loss="bs_reta", log=print,
          log_every=100, refresh=250):
    """Cosine-decayed steps of `loss`; the on-policy levels of the banks are
    refreshed every `refresh` steps (the Direct format's own iterates are not
    banked: its snapshots stay at zero and noise)."""
    rng = np.random.default_rng(seed)
    t0 = time.time()
    hist, skipped = [], 0
    for g in groups:
        g.bank[:len(LEVELS)].zero_()
    for s in range(steps):
        if s % refresh == 0 and s > 0 and loss != "dir":
            for g in groups:
                g.refresh(ctx, net)
        g = groups[int(rng.integers(len(groups)))]
        lr_s = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * s / max(1, steps)))
        try:
            v = capi.newton_train_step(ctx, net, g.b, g.shift, g.u32, g.r, g.draw(rng), unroll=unroll, lr=lr_s,
                                       weight_decay=wd, loss=loss)
        except capi.NpbsError as e:
            # a non-finite loss leaves the weights untouched (the step returns before its update)
            if e.status != capi.ERR_NONFINITE:
                raise
            skipped += 1
            continue
        hist.append(v)
        if (s + 1) % log_every == 0 or s == 0:
            log(json.dumps({"loss_kind": loss, "step": s + 1, "loss": float(np.mean(hist[-log_every:])),
                            "lr": lr_s, "skipped": skipped, "s": round(time.time() - t0, 1)}))
    return hist


def solve_stats(ctx, net, insts, direct=False, tol=1e-10, inner_rtol=1e-4, max_steps=12, inner_max=500):
    """Newton on the instances (one batch): converged count, Newton steps,
    inner iterations per Newton step, wall time."""
    n = insts[0].n
    b = capi.Batch([(n, n)] * len(insts), h=[1.0 / (n + 1)] * len(insts))
    f = b.pack([i.f for i in insts], dtype=torch.float64)
    u = b.pack([i.u0 for i in insts], dtype=torch.float64)
    torch.cuda.synchronize()
    t = time.time()
    st, rep = capi.newton_solve(ctx, net, b, f, u, tol=tol, max_steps=max_steps, inner_rtol=inner_rtol,
                                inner_max_iter=inner_max, check_every=1, direct=direct)
    ms = (time.time() - t) * 1e3
    ok = [j for j, x in enumerate(rep["status"]) if x == capi.OK]
    per_step = [rep["inner_iters"][j] / max(1, rep["steps"][j]) for j in ok]
    res = [x for x in rep["residual"] if np.isfinite(x)]
    return {"converged": f"{len(ok)}/{len(insts)}",
            "newton_steps_mean": float(np.mean([rep["steps"][j] for j in ok])) if ok else None,
            "inner_iters_per_step_mean": float(np.mean(per_step)) if per_step else None,
            "residual_median_finite": float(np.median(res)) if res else None, "solve_ms": round(ms, 1)}


def compare(ctx, groups, test, steps, log=print, **net_kw):
    """Direct + L_dir, NPBS + L_bs^l2 and NPBS + L_bs^R_N from the same
    initialisation and states, each solving in its own format."""
    res = {}
    for loss in ("dir", "bs_l2", "bs_reta"):
        # the Direct format feeds M the raw residual r - J delta: there M = I + N would start as an
        # unscaled Richardson step, which diverges, so the Direct network is the plain FNO
        kw = dict(net_kw, skip=net_kw.get("skip", True) and loss != "dir")
        net = make_net(**kw)
        t = time.time()
        hist = train(ctx, net, groups, steps, loss=loss, log=log)
        res[loss] = {"train_s": round(time.time() - t, 1),
                     "final_loss": float(np.mean(hist[-100:])) if hist else None,
                     **solve_stats(ctx, net, test, direct=loss == "dir")}
        log(json.dumps({"compare": loss, **res[loss]}))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=N_DEFAULT)
    ap.add_argument("--pool", type=int, default=500, help="training instances (4 Newton states each)")
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--batch", type=int, default=50)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--width", type=int, default=25)
    ap.add_argument("--modes", type=int, default=20)
    ap.add_argument("--layers", type=int, default=2)
    ap.add_argument("--compare", action="store_true")
    ap.add_argument("--no-skip", action="store_true", help="the paper's FNO without the identity skip")
    args = ap.parse_args()
    build.build()
    ctx = capi.Context(0)
    pool = [synth.newton_instance(args.grid, 20000 + j) for j in range(args.pool)]
    states = trajectories(ctx, pool, 4)
    rng = np.random.default_rng(0)
    order = rng.permutation(len(states))
    groups = [StateGroup([states[k] for k in order[i:i + args.batch]], seed=i)
              for i in range(0, len(order) - args.batch + 1, args.batch)]
    test = [synth.newton_instance(args.grid, 80000 + j) for j in range(args.test)]
    kw = dict(n=args.grid, width=args.width, modes=args.modes, layers=args.layers, skip=not args.no_skip)
    born = solve_stats(ctx, None, test)
    print(json.dumps({"born": born}), flush=True)
    if args.compare:
        res = compare(ctx, groups, test, args.steps, log=lambda s: print(s, flush=True), **kw)
        print(json.dumps({"grid": args.grid, "states": len(states), "steps": args.steps, "compare": res,
                          "born": born}), flush=True)
        return
    net = make_net(**kw)
    train(ctx, net, groups, args.steps, log=lambda s: print(s, flush=True))
    print(json.dumps({"npbs": solve_stats(ctx, net, test), "born": born}), flush=True)


if __name__ == "__main__":
    main()
