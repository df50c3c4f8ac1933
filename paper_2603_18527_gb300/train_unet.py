"""Train the residual-to-correction network (U-Net or FNO) with the library's own kernels.

Training tuples (medium, source, residual) come from the method itself
(the metric-matched objective, Eq. L_bs_Reta_integral): a pool of instances
of the contrast media law is iterated with plain CBS (``cbs_apply`` CBS_STEP)
and its iterates are banked at log-spaced iteration counts; every training
batch draws instances and snapshot counts from that bank, and
``npbs_train_step`` unrolls the NPBS iteration from those snapshots.
Evaluation compares ``npbs_solve`` with ``cbs_solve`` (iterations and time to
the rTol target) on held-out seeds.  Every step runs on the GPU in the
library; this module only marshals arguments.

    python -m paper_2603_18527_gb300.train_unet --grid 64 --steps 2000 --out net.bin
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2603_18527_gb300 import build, capi  # noqa: E402


def coefficient_channel(inst, scale_by_omega: bool) -> np.ndarray:
    """Third network input: n(x), or the local wavenumber omega n(x) so that one
    network serves several frequencies."""
    return inst.n * (inst.omega if scale_by_omega else 1.0)


class Pool:
    """A packed batch of instances with the library-side potential."""

    def __init__(self, ctx, insts, scale_by_omega=True):
        self.insts = insts
        self.b = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
        self.k2 = self.b.pack([i.k2 for i in insts])
        self.f = self.b.pack([i.f for i in insts])
        self.n = self.b.pack([coefficient_channel(i, scale_by_omega) for i in insts], dtype=torch.float32)
        self.V = torch.zeros_like(self.k2)
        capi.npbs_potential_from_k2(ctx, self.b, self.k2, self.V)


def snapshot_bank(ctx, pool: Pool, max_snap: int = 2048) -> tuple[list[int], torch.Tensor]:
    """CBS iterates of every pool instance at log-spaced iteration counts
    0, 1, 3, 7, ..., up to max_snap (one pass of in-place complex64 CBS_STEP
    applies over the whole pool); returns (counts, bank[count_index, extent])."""
    counts = [0]
    while counts[-1] * 2 + 1 <= max_snap:
        counts.append(counts[-1] * 2 + 1)
    u = torch.zeros(pool.b.extent, dtype=torch.complex64, device="cuda")
    bank = torch.zeros((len(counts), pool.b.extent), dtype=torch.complex64, device="cuda")
    done = 0
    for ci, m in enumerate(counts):
        while done < m:
            capi.cbs_apply(ctx, pool.b, pool.V, pool.f, u, u, capi.CBS_STEP)
            done += 1
        bank[ci].copy_(u)
    return counts, bank


def media(grid: int, count: int, seed0: int, waves=(20.0, 40.0)):
    """Contrast media law at any grid size (seed block seed0)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        N = grid
        W = max(2, N // 16)
        g = synth.grf(rng, N, N, max(2.0, 16.0 * N / 256))
        na, nb = rng.uniform(0.7, 1.6, size=2)
        n = na + (nb - na) * 0.5 * (1.0 + np.tanh(g / 0.25))
        wl = rng.uniform(*waves) * N / 256.0
        omega = 2.0 * math.pi * wl / (N - 2 * W)
        cy, cx = int(rng.integers(W, N - W)), int(rng.integers(W, N - W))
        yy, xx = np.mgrid[0:N, 0:N]
        f = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * 1.5 ** 2)).astype(np.complex128)
        out.append(synth.make_instance(n, omega, W, f, seed=seed0 + i, source_kind="gaussian"))
    return out


def train(ctx, net, grid=64, steps=1000, batch=32, unroll=4, lr=1e-3, wd=1e-6, pool_size=256, seed=3000,
          max_snap=2048, log_every=50, log=print, lr_min=None, loss="bs_reta"):
    """Metric-matched training on a pool of contrast media; each step draws
    `batch` instances and, for each, a CBS snapshot at a log-uniform iteration
    count, and runs one npbs_train_step (4 unrolled NPBS steps, AdamW).  With
    lr_min the learning rate follows a cosine from lr down to lr_min."""
    rng = np.random.default_rng(seed)
    insts = media(grid, pool_size, seed)
    pool = Pool(ctx, insts)
    counts, bank = snapshot_bank(ctx, pool, max_snap)
    np_ = grid * grid
    if pool.b.extent != pool_size * np_:
        raise ValueError("grid * grid must be a multiple of 32 (packed pool layout)")
    pV, pf = pool.V.view(pool_size, np_), pool.f.view(pool_size, np_)
    pn, pb = pool.n.view(pool_size, np_), bank.view(len(counts), pool_size, np_)
    history = []
    t0 = time.time()
    sb = capi.Batch([(grid, grid)] * batch, h=[1.0] * batch)
    for step in range(steps):
        idx = rng.choice(pool_size, size=batch, replace=False)
        ci = rng.integers(0, len(counts), size=batch)
        it = torch.from_numpy(idx).cuda()
        V = pV.index_select(0, it).reshape(-1)
        f = pf.index_select(0, it).reshape(-1)
        n = pn.index_select(0, it).reshape(-1)
        u0 = pb[torch.from_numpy(ci).cuda(), it].reshape(-1)
        sb.k0sq = [pool.b.k0sq[i] for i in idx]
        sb.eps = [pool.b.eps[i] for i in idx]
        lr_t = lr if lr_min is None else lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / max(1, steps)))
        val = capi.npbs_train_step(ctx, net, sb, V, f, n, u0, unroll=unroll, lr=lr_t, weight_decay=wd, loss=loss)
        history.append(val)
        if log and (step % log_every == 0 or step == steps - 1):
            log(json.dumps({"step": step, "loss": val, "mean_last": float(np.mean(history[-log_every:])),
                            "elapsed_s": round(time.time() - t0, 1)}))
    return history


def evaluate(ctx, net, grid=64, count=16, seed=9000, tol=1e-5, max_iter=20000, solvers=("cbs", "npbs")):
    """Iterations and time to `tol` on held-out media for CBS, NPBS (Eq.
    npbs_integral) and/or the Direct format (Eq. direct_iter, "direct")."""
    insts = media(grid, count, seed)
    pool = Pool(ctx, insts)
    res = {}
    for name in solvers:
        u = torch.zeros(pool.b.extent, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t = time.time()
        if name == "cbs":
            st, rep = capi.cbs_solve(ctx, pool.b, pool.k2, pool.f, u, rtol=tol, max_iter=max_iter, check_every=16)
        elif name == "direct":
            st, rep = capi.npbs_solve_direct(ctx, net, pool.b, pool.k2, pool.f, pool.n, u, rtol=tol,
                                             max_iter=max_iter, check_every=4)
        else:
            st, rep = capi.npbs_solve(ctx, net, pool.b, pool.k2, pool.f, pool.n, u, rtol=tol, max_iter=max_iter,
                                      check_every=4)
        torch.cuda.synchronize()
        res[name] = {"iters": rep["iters"], "rtol": rep["rtol"], "status": rep["status"],
                     "fallback": rep.get("fallback"), "seconds": time.time() - t}
    return res


def compare(ctx, nets, grid=256, count=64, seed=2000, tol=1e-5, max_iter=2500):
    """NPBS with each network of `nets` (name -> npbs_net) against plain CBS on
    `count` held-out media of the contrast law: converged count, mean and
    median iterations of the converged instances, CBS hand-overs by the
    divergence guard, and ms per solve (batch time / count)."""
    insts = media(grid, count, seed)
    pool = Pool(ctx, insts)
    out = {}
    for name, net in [("cbs", None)] + list(nets.items()):
        u = torch.zeros(pool.b.extent, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t = time.time()
        if net is None:
            st, rep = capi.cbs_solve(ctx, pool.b, pool.k2, pool.f, u, rtol=tol, max_iter=max_iter, check_every=16)
        else:
            st, rep = capi.npbs_solve(ctx, net, pool.b, pool.k2, pool.f, pool.n, u, rtol=tol, max_iter=max_iter,
                                      check_every=4)
        torch.cuda.synchronize()
        dt = time.time() - t
        it = np.array(rep["iters"])
        ok = np.array(rep["status"]) == capi.OK
        out[name] = {"converged": int(ok.sum()), "iters_mean_converged": float(it[ok].mean()) if ok.any() else None,
                     "iters_median_converged": float(np.median(it[ok])) if ok.any() else None,
                     "fallback": int(sum(rep.get("fallback") or [0])), "ms_per_solve": dt * 1e3 / count}
    return out


def ablation(ctx, grid=256, steps=2000, count=32, tol=1e-5, max_iter=2500, log=print):
    """The format / objective ablation of Sec. 4 (Table 2's U-Net row): three
    networks from the same initialisation on the same media pool and snapshot
    bank, trained with Eq. L_dir (Direct format), Eq. L_bs_l2 and Eq.
    L_bs_Reta_integral (NPBS format), each evaluated in its own format on
    `count` held-out media against CBS."""
    out = {}
    for kind in ("dir", "bs_l2", "bs_reta"):
        net = capi.Net(0, seed=0)
        t = time.time()
        hist = train(ctx, net, grid=grid, steps=steps, batch=32, pool_size=256, seed=5000, lr=1e-3, lr_min=2e-5,
                     log_every=max(1, steps // 4), log=log, loss=kind)
        solver = "direct" if kind == "dir" else "npbs"
        r = evaluate(ctx, net, grid=grid, count=count, seed=2000, tol=tol, max_iter=max_iter, solvers=("cbs", solver))
        res = {"train_s": round(time.time() - t, 1), "final_loss": float(np.mean(hist[-200:]))}
        for name, v in r.items():
            it = np.array(v["iters"])
            ok = np.array(v["status"]) == capi.OK
            res[name] = {"converged": int(ok.sum()), "iters_mean_converged": float(it[ok].mean()) if ok.any() else None,
                         "iters_median": float(np.median(it)), "seconds": round(v["seconds"], 3),
                         "fallback": int(sum(v.get("fallback") or [0]))}
        out[kind] = res
        if log:
            log(json.dumps({kind: res}))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=None, help="cosine decay of the learning rate down to this")
    ap.add_argument("--init", default="", help="start from these weights (.npz with 'params' or a saved network)")
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--loss", default="bs_reta", choices=["bs_reta", "bs_l2", "dir"],
                    help="training objective (Sec. 4): metric-matched, Euclidean bs, or Direct")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="")
    ap.add_argument("--eval", type=int, default=16)
    ap.add_argument("--max-snap", type=int, default=2048)
    ap.add_argument("--backbone", default="unet", choices=["unet", "fno"],
                    help="the residual-to-correction map: the 4-level U-Net or the FNO (App. Architectural "
                         "Instantiations; width / modes / layers below, the network is tied to --grid)")
    ap.add_argument("--fno-width", type=int, default=25)
    ap.add_argument("--fno-modes", type=int, default=45)
    ap.add_argument("--fno-layers", type=int, default=3)
    ap.add_argument("--fno-skip", action="store_true",
                    help="the FNO as M = I + N (zero projection at start: the Born series, npbs_net_fno_set_skip)")
    ap.add_argument("--compare-unet", default="",
                    help="after training, compare NPBS with this network and with the U-Net of this .npz on the "
                         "64 held-out media of the bench (seeds 2000+) against CBS")
    ap.add_argument("--ablation", action="store_true",
                    help="train and evaluate the three objectives (Direct+L_dir, NPBS+L_bs_l2, NPBS+L_bs_Reta)")
    args = ap.parse_args()
    build.build()
    ctx = capi.Context(0)
    if args.ablation:
        print(json.dumps(ablation(ctx, grid=args.grid, steps=args.steps)))
        return
    def fresh():
        if args.backbone == "fno":
            return capi.Net.fno(args.grid, args.fno_width, min(args.fno_modes, args.grid // 2 + 1), args.fno_layers,
                                seed=args.seed, skip=args.fno_skip)
        return capi.Net(0, seed=args.seed)

    if args.init.endswith(".npz"):
        net = fresh()
        net.set_params(np.load(args.init)["params"].astype(np.float32))
    elif args.init:
        net = capi.Net.load(args.init)
    else:
        net = fresh()
    train(ctx, net, grid=args.grid, steps=args.steps, batch=args.batch, lr=args.lr, max_snap=args.max_snap,
          pool_size=args.pool, lr_min=args.lr_min, loss=args.loss)
    if args.out.endswith(".npz"):
        np.savez_compressed(args.out, params=net.get_params().astype(np.float16))
    elif args.out:
        net.save(args.out)
    if args.compare_unet:
        unet = capi.Net(0, seed=0)
        unet.set_params(np.load(args.compare_unet)["params"].astype(np.float32))
        print(json.dumps({"compare": compare(ctx, {args.backbone: net, "unet": unet}, grid=args.grid)}))
    elif args.eval:
        solvers = ("cbs", "direct") if args.loss == "dir" else ("cbs", "npbs")
        print(json.dumps(evaluate(ctx, net, grid=args.grid, count=args.eval, solvers=solvers)))


if __name__ == "__main__":
    main()
