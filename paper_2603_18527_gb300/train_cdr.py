"""Training and evaluation of an FNO preconditioner for the CDR problems
(App. Full Derivations, CDR; App. Experimental Setup, CDR benchmark) through
the library's C-ABI: ``cdr_train_step`` (the metric-matched loss of Eq.
cdr_bs_loss in its unrolled form) and ``cdr_solve`` (NPBS with the CDR
operators, float64 stopping test).

The network reads the four coefficient channels (kappa, vx, vy, sigma).
Training states: at full convection speed the Born series diverges, so the
snapshots u from which the unrolled loss starts come from the network's own
NPBS iteration (on-policy): every ``refresh`` steps each pool instance gets
snapshots after 0, 2, 6, 14 and 30 iterations of the current network, and a
batch draws one level per instance.

    python -m paper_2603_18527_gb300.train_cdr --steps 2000 --out /tmp/cdr_fno.bin
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

LEVELS = (0, 2, 6, 14, 30)
BOUND = 1e4  # largest |u| kept as a training state (solutions are O(1): unit source, sigma ~ 1)


class Group:
    """A fixed batch of CDR instances on the device: layout, coefficient
    fields, source, background constants and a snapshot bank [levels, extent]."""

    def __init__(self, ctx, insts):
        self.insts = insts
        self.b = capi.Batch([(i.n, i.n) for i in insts], h=[i.h for i in insts])
        self.fields = capi.CdrFields(self.b, [i.kappa for i in insts], [i.vx for i in insts],
                                     [i.vy for i in insts], [i.sigma for i in insts])
        self.f = self.b.pack([i.f for i in insts])
        self.consts = capi.npbs_cdr_background(ctx, self.b, self.fields)
        self.bank = torch.zeros((len(LEVELS), self.b.extent), dtype=torch.complex64, device="cuda")

    def refresh(self, ctx, net, direct=False):
        """Snapshots of the current network's iteration (NPBS, or the Direct
        format) from u = 0."""
        u = torch.zeros(self.b.extent, dtype=torch.complex128, device="cuda")
        done = 0
        for l, k in enumerate(LEVELS):
            if k > done:
                capi.cdr_solve(ctx, net, self.b, self.consts, self.fields, self.f, self.fields.a, u, rtol=0.0,
                               max_iter=k - done, check_every=k - done, direct=direct)
                done = k
            snap = u.to(torch.complex64)
            # a diverged state (non-finite, or far beyond the O(1) solution) restarts from zero
            for o, (ny, nx) in zip(self.b.offsets, self.b.shapes):
                seg = snap[o:o + ny * nx]
                if not bool(torch.isfinite(torch.view_as_real(seg)).all()) or float(seg.abs().max()) > BOUND:
                    seg.zero_()
            self.bank[l] = snap

    def draw(self, rng) -> torch.Tensor:
        """One snapshot per instance at a random level."""
        u = torch.empty(self.b.extent, dtype=torch.complex64, device="cuda")
        lv = rng.integers(0, len(LEVELS), size=len(self.insts))
        for j, (o, (ny, nx)) in enumerate(zip(self.b.offsets, self.b.shapes)):
            u[o:o + ny * nx] = self.bank[lv[j], o:o + ny * nx]
        return u


def instances(n: int, count: int, seed0: int, speed=(0.5, 1.0)):
    rng = np.random.default_rng(seed0)
    return [synth.cdr_instance(n, seed=seed0 + j, speed=float(rng.uniform(*speed))) for j in range(count)]


def make_net(n=128, width=25, modes=32, layers=3, seed=0):
    return capi.Net.fno(n, width, modes, layers, seed=seed, coef_channels=4)


def train(ctx, net, groups, steps, lr=1e-3, lr_min=1e-4, wd=1e-6, unroll=4, refresh=250, seed=0, log=print,
          log_every=50, loss="bs_reta"):
    """Cosine-decayed AdamW steps of `loss`; the snapshot banks follow the
    iteration format the loss trains for (Direct for "dir", NPBS otherwise)."""
    rng = np.random.default_rng(seed)
    t0 = time.time()
    hist = []
    skipped = 0
    for g in groups:
        g.bank.zero_()
    for s in range(steps):
        if s % refresh == 0 and s > 0:
            for g in groups:
                g.refresh(ctx, net, direct=loss == "dir")
        g = groups[int(rng.integers(len(groups)))]
        lr_s = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * s / max(1, steps)))
        try:
            loss_v = capi.cdr_train_step(ctx, net, g.b, g.consts, g.fields, g.f, g.fields.a, g.draw(rng),
                                         unroll=unroll, lr=lr_s, weight_decay=wd, loss=loss)
        except capi.NpbsError as e:
            # a non-finite loss leaves the weights untouched (the step returns before its update)
            if e.status != capi.ERR_NONFINITE:
                raise
            skipped += 1
            continue
        hist.append(loss_v)
        if (s + 1) % log_every == 0 or s == 0:
            log(json.dumps({"loss_kind": loss, "step": s + 1, "loss": float(np.mean(hist[-log_every:])),
                            "lr": lr_s, "skipped": skipped, "s": round(time.time() - t0, 1)}))
    return hist


def solve_stats(ctx, net, groups, tol=1e-6, max_iter=1000, check_every=4, direct=False):
    """Iterations to ||f - A u|| / ||f|| <= tol (float64) over the groups:
    NPBS with `net`, the Direct format (direct), or the Born series (net None)."""
    its, rts, ok, ms = [], [], 0, 0.0
    for g in groups:
        u = torch.zeros(g.b.extent, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t = time.time()
        st, rep = capi.cdr_solve(ctx, net, g.b, g.consts, g.fields, g.f, g.fields.a if net else None, u, rtol=tol,
                                 max_iter=max_iter, check_every=check_every, direct=direct)
        ms += (time.time() - t) * 1e3
        its += list(rep["iters"])
        rts += [float(x) for x in rep["rtol"]]
        ok += sum(1 for x in rep["status"] if x == capi.OK)
    conv = [i for i, r in zip(its, rts) if r <= tol]
    return {"converged": f"{ok}/{len(its)}", "iters_mean": float(np.mean(its)), "iters_max": int(np.max(its)),
            "iters_mean_converged": float(np.mean(conv)) if conv else None, "solve_ms_total": round(ms, 1)}


def evaluate(ctx, net, groups, tol=1e-6, max_iter=1000, check_every=4):
    """NPBS with the network, and the Born series for reference."""
    return {"npbs": solve_stats(ctx, net, groups, tol, max_iter, check_every),
            "born": solve_stats(ctx, None, groups, tol, min(max_iter, 300), check_every)}


def compare(ctx, groups, tgroups, steps, tol=1e-6, max_iter=1000, log=print, **net_kw):
    """The CDR format/loss comparison: Direct + L_dir, NPBS + L_bs^l2 and
    NPBS + L_bs^Reta from the same initialisation, pool and step count, each
    solved in its own format."""
    res = {}
    for loss in ("dir", "bs_l2", "bs_reta"):
        net = make_net(**net_kw)
        t = time.time()
        hist = train(ctx, net, groups, steps, loss=loss, log=log)
        tr = time.time() - t
        res[loss] = {"train_s": round(tr, 1), "final_loss": float(np.mean(hist[-50:])) if hist else None,
                     **solve_stats(ctx, net, tgroups, tol, max_iter, direct=loss == "dir")}
        log(json.dumps({"compare": loss, **res[loss]}))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--pool", type=int, default=512)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--refresh", type=int, default=250)
    ap.add_argument("--width", type=int, default=25)
    ap.add_argument("--modes", type=int, default=32)
    ap.add_argument("--layers", type=int, default=3)
    ap.add_argument("--eval-count", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--out", default=None, help="checkpoint path (npbs_net_save format)")
    ap.add_argument("--compare", action="store_true",
                    help="train Direct + L_dir, NPBS + L_bs^l2 and NPBS + L_bs^Reta and compare their solves")
    args = ap.parse_args()
    build.build()
    ctx = capi.Context(0)
    pool = instances(args.grid, args.pool, 40000)
    groups = [Group(ctx, pool[i:i + args.batch]) for i in range(0, len(pool), args.batch)]
    test = instances(args.grid, args.eval_count, 90000)
    tgroups = [Group(ctx, test[i:i + args.batch]) for i in range(0, len(test), args.batch)]
    if args.compare:
        res = compare(ctx, groups, tgroups, args.steps, tol=args.tol, log=lambda s: print(s, flush=True),
                      n=args.grid, width=args.width, modes=args.modes, layers=args.layers)
        born = solve_stats(ctx, None, tgroups, args.tol, 300)
        print(json.dumps({"grid": args.grid, "steps": args.steps, "tol": args.tol, "pool": args.pool,
                          "test": args.eval_count, "compare": res, "born": born}), flush=True)
        return
    net = make_net(args.grid, args.width, args.modes, args.layers)
    print(json.dumps({"untrained": evaluate(ctx, net, tgroups[:1], tol=args.tol, max_iter=200)}), flush=True)
    t = time.time()
    train(ctx, net, groups, args.steps, lr=args.lr, refresh=args.refresh, log=lambda s: print(s, flush=True))
    train_s = time.time() - t
    if args.out:
        net.save(args.out)
    res = evaluate(ctx, net, tgroups, tol=args.tol)
    print(json.dumps({"grid": args.grid, "steps": args.steps, "train_s": round(train_s, 1), "tol": args.tol,
                      "eval": res}), flush=True)


if __name__ == "__main__":
    main()
