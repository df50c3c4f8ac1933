"""Mutation check of the oracle's pins (CPU only, not collected by pytest).

Plants one plausible mistake at a time (a dropped term, a wrong sign or
conjugate, swapped operands or indices, a different reading of a convention)
in a temporary copy of ``oracle/`` and runs the oracle pins
(``tests/test_oracle_{pins,unet,fno,cdr,newton}.py``) against it.
Every mutant must make at least one pin fail.

    python tests/oracle_mutation_check.py [index ...]

Exit status 1 if any mutant survives.  Takes a few minutes (4 mutants at a
time).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# (oracle file, label, text, replacement)
M = [
 ("helmholtz.py", "xi h dropped", "ky = 2.0 * math.pi * mode_index(ny) / (ny * h)", "ky = 2.0 * math.pi * mode_index(ny) / ny"),
 ("helmholtz.py", "xi nx/ny swapped", "kx = 2.0 * math.pi * mode_index(nx) / (nx * h)", "kx = 2.0 * math.pi * mode_index(nx) / (ny * h)"),
 ("helmholtz.py", "k0sq mean", "k0sq = 0.5 * (float(re.min()) + float(re.max()))", "k0sq = float(re.mean())"),
 ("helmholtz.py", "eps real part only", "eps = float((k2 - k0sq).abs().max())", "eps = float((k2.real - k0sq).abs().max())"),
 ("helmholtz.py", "symbol sign of i eta", "return xi_squared(ny, nx, h).to(C128) - complex(k0sq, eps)", "return xi_squared(ny, nx, h).to(C128) - complex(k0sq, -eps)"),
 ("helmholtz.py", "V without i eta", "return k2 - complex(k0sq, eps)", "return k2 - k0sq"),
 ("helmholtz.py", "gamma sign", "return 1j * V / eps", "return -1j * V / eps"),
 ("helmholtz.py", "gamma conj", "return 1j * V / eps", "return 1j * V.conj() / eps"),
 ("helmholtz.py", "G* without conj", "return torch.fft.ifft2(torch.fft.fft2(q) / lam.conj())", "return torch.fft.ifft2(torch.fft.fft2(q) / lam)"),
 ("helmholtz.py", "laplacian h dropped", "return torch.fft.ifft2(xi_squared(ny, nx, h).to(C128) * torch.fft.fft2(u))", "return torch.fft.ifft2(xi_squared(ny, nx).to(C128) * torch.fft.fft2(u))"),
 ("helmholtz.py", "A with conj k2", "return laplacian_neg(u, h) - k2 * u", "return laplacian_neg(u, h) - k2.conj() * u"),
 ("helmholtz.py", "born residual -f", "return green(p.V * u + p.f, p.lam) - u", "return green(p.V * u - p.f, p.lam) - u"),
 ("helmholtz.py", "cbs step sign", "return u + p.gamma * born_residual(p, u)", "return u - p.gamma * born_residual(p, u)"),
 ("helmholtz.py", "B order VG", "return x - green(p.V * x, p.lam)", "return x - p.V * green(x, p.lam)"),
 ("helmholtz.py", "B* order", "return y - p.V.conj() * green_adjoint(y, p.lam)", "return y - green_adjoint(p.V.conj() * y, p.lam)"),
 ("helmholtz.py", "B* no conj V", "return y - p.V.conj() * green_adjoint(y, p.lam)", "return y - p.V * green_adjoint(y, p.lam)"),
 ("helmholtz.py", "prec sweep without B", "return z + p.gamma * (v - op_B(p, z))", "return z + p.gamma * (v - z)"),
 ("helmholtz.py", "npbs sign", "u = u + M(born_residual(p, u))", "u = u - M(born_residual(p, u))"),
 ("helmholtz.py", "direct uses born residual", "u = u + M(true_residual(p, u))", "u = u + M(born_residual(p, u))"),
 ("helmholtz.py", "left residual sign", "return green(p.f - apply_A(u, p.k2, p.h), p.lam)", "return green(p.f + apply_A(u, p.k2, p.h), p.lam)"),
 ("helmholtz.py", "rtol squared norm", "/ torch.linalg.vector_norm(p.f))", "/ torch.linalg.vector_norm(p.f) ** 2)"),
 ("helmholtz.py", "odd-N mode order", "torch.where(n <= N // 2, n, n - N)", "torch.where(n < N // 2, n, n - N)"),
 ("unet.py", "gelu tanh", 'return Fnn.gelu(Fnn.conv2d(x, P[name + ".w"], P[name + ".b"], padding=1))', 'return Fnn.gelu(Fnn.conv2d(x, P[name + ".w"], P[name + ".b"], padding=1), approximate="tanh")'),
 ("unet.py", "max pool", "return Fnn.avg_pool2d(x, 2)", "return Fnn.max_pool2d(x, 2)"),
 ("unet.py", "concat order", "h = torch.cat([skips[lvl], u], dim=1)", "h = torch.cat([u, skips[lvl]], dim=1)"),
 ("unet.py", "rms sum", "return torch.sqrt((r.real ** 2 + r.imag ** 2).mean(dim=(-2, -1)))", "return torch.sqrt((r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1)))"),
 ("unet.py", "input re/im swapped", "x = torch.stack([r.real / sc, r.imag / sc, n], dim=1)", "x = torch.stack([r.imag / sc, r.real / sc, n], dim=1)"),
 ("unet.py", "output re/im swapped", "return sc * torch.complex(y[:, 0], y[:, 1])", "return sc * torch.complex(y[:, 1], y[:, 0])"),
 ("unet.py", "loss over norm not squared", "acc = acc + (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1)) / r0n", "acc = acc + (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1)).sqrt() / r0n.sqrt()"),
 ("unet.py", "adam no bias correction", "mhat = m / (1.0 - beta1 ** step)", "mhat = m"),
 ("unet.py", "adam coupled decay", "theta = theta * (1.0 - lr * weight_decay)", "grad = grad + weight_decay * theta"),
 ("unet.py", "bilinear up", "return x.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)", 'return Fnn.interpolate(x, scale_factor=2, mode="bilinear", align_corners=False)'),
 ("unet.py", "bs_l2 with G out", 'proj_out = (lambda v: batched_green(lam, v)) if kind == "bs_reta" else (lambda v: v)', 'proj_out = (lambda v: batched_green(lam, v)) if kind != "dir" else (lambda v: v)'),
 ("unet.py", "batched B order", "return x - torch.fft.ifft2(torch.fft.fft2(V * x) / lam)", "return x - V * torch.fft.ifft2(torch.fft.fft2(x) / lam)"),
 ("unet.py", "unrolled loss r update sign", "r = r - batched_op_B(V, lam, c)", "r = r + batched_op_B(V, lam, c)"),
 ("unet.py", "dir P_in G", 'proj_in = (lambda v: v) if kind == "dir" else (lambda v: batched_green(lam, v))', 'proj_in = (lambda v: batched_green(lam, v))'),
 ("helmholtz.py", "true residual sign", "return p.f - apply_A(u, p.k2, p.h)", "return apply_A(u, p.k2, p.h) - p.f"),
 ("unet.py", "adam eps inside sqrt", "theta = theta - lr * mhat / (torch.sqrt(vhat) + eps)", "theta = theta - lr * mhat / torch.sqrt(vhat + eps)"),
 ("unet.py", "pool after the level's convs", "        if lvl > 0:\n            h = _pool(h)\n        h = _conv_gelu(h, P, f\"enc{lvl}a\")", "        h = _conv_gelu(h, P, f\"enc{lvl}a\")\n        if lvl > 0:\n            h = _pool(h)"),
 ("fgmres.py", "rotation without conj", "Hm[i, j] = cs[i].conj() * a + sn[i].conj() * c", "Hm[i, j] = cs[i] * a + sn[i].conj() * c"),
 ("fgmres.py", "sign of g", "g[j + 1] = -sn[j] * gj", "g[j + 1] = sn[j] * gj"),
 ("fgmres.py", "dot operands swapped", "hij = _dot(Vb[i], w)", "hij = _dot(w, Vb[i])"),
 ("fgmres.py", "earlier rotations skipped", "for i in range(j):\n                a, c", "for i in range(0):\n                a, c"),
 ("fno.py", "retained rows <=", "return [k for k in range(n) if min(k, n - k) < m]", "return [k for k in range(n) if min(k, n - k) <= m]"),
 ("fno.py", "conv1x1 transposed", 'y = torch.einsum("oi,bihw->bohw", w, x)', 'y = torch.einsum("io,bihw->bohw", w, x)'),
 ("fno.py", "spectral weights conj", 'Yr = torch.einsum("bikl,iokl->bokl", Xr, W)', 'Yr = torch.einsum("bikl,iokl->bokl", Xr, W.conj())'),
 ("fno.py", "residual branch re/im swapped", "x = conv1x1(torch.stack([r.real, r.imag], dim=1), P[\"lift_r.w\"])", "x = conv1x1(torch.stack([r.imag, r.real], dim=1), P[\"lift_r.w\"])"),
 ("fno.py", "layer norm over channels too", "mu = a.mean(dim=(-2, -1), keepdim=True)", "mu = a.mean(dim=(-3, -2, -1), keepdim=True)"),
 ("fno.py", "skip subtracts the input", "return out + r if cfg.skip else out", "return out - r if cfg.skip else out"),
 ("cdr.py", "A convection sign", "+ p.vx * ux + p.vy * uy + p.sigma * u", "- p.vx * ux - p.vy * uy + p.sigma * u"),
 ("cdr.py", "L0 symbol convection sign", "lam = (k0 * (kx ** 2 + ky ** 2)).to(C128) + 1j * (v0x * kx + v0y * ky) + s0", "lam = (k0 * (kx ** 2 + ky ** 2)).to(C128) - 1j * (v0x * kx + v0y * ky) + s0"),
 ("cdr.py", "A* without the v g flux", "return -(ddx(p, p.kappa * gx + p.vx * g) + ddy(p, p.kappa * gy + p.vy * g)) + p.sigma * g", "return -(ddx(p, p.kappa * gx) + ddy(p, p.kappa * gy)) + p.sigma * g"),
 ("cdr.py", "G* without conj", "return torch.fft.ifft2(torch.fft.fft2(q) / p.lam.conj())", "return torch.fft.ifft2(torch.fft.fft2(q) / p.lam)"),
 ("cdr.py", "V drops dkappa", "return (ddx(p, dk * ux) + ddy(p, dk * uy)) - (p.vx - p.v0x) * ux", "return - (p.vx - p.v0x) * ux"),
 ("newton.py", "stencil centre 2", "return (4.0 * c - p[2:, 1:-1]", "return (2.0 * c - p[2:, 1:-1]"),
 ("newton.py", "jacobian factor 2 dropped", "return lap_D(x, h) - 2.0 * u * x", "return lap_D(x, h) - u * x"),
 ("newton.py", "sine matrix over N", "return torch.sin(math.pi * torch.outer(j, j) / (N + 1))", "return torch.sin(math.pi * torch.outer(j, j) / N)"),
 ("newton.py", "dst one axis", "return S @ q @ S", "return S @ q"),
 ("newton.py", "eigenvalue full angle", "* math.pi * h / 2.0) ** 2", "* math.pi * h) ** 2"),
 ("newton.py", "shift sign of the mean", "shift = alpha - 2.0 * float(u.real.mean())", "shift = alpha + 2.0 * float(u.real.mean())"),
 ("newton.py", "inverse normalisation 1D", "* (2.0 / (N + 1)) ** 2", "* (2.0 / (N + 1))"),
 ("newton.py", "V sign of u", "return (s.shift + 2.0 * s.u) * x", "return (s.shift - 2.0 * s.u) * x"),
 ("newton.py", "B* order", "return y - apply_V(s, green(s, y))", "return y - green(s, apply_V(s, y))"),
 ("newton.py", "born residual sign", "return green(s, r - jacobian(s.u, d, s.h))", "return green(s, r + jacobian(s.u, d, s.h))"),
 ("newton.py", "nonlinear residual u^2 sign", "return lap_D(u, h) - u * u - f", "return lap_D(u, h) + u * u - f"),
]
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_unet.py", "tests/test_oracle_fno.py", "tests/test_oracle_cdr.py",
        "tests/test_oracle_newton.py"]
def run(i):
    fn, label, a, b = M[i]
    d = tempfile.mkdtemp(prefix=f"mut{i}_")
    for sub in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=shutil.ignore_patterns("__pycache__", "test_gpu_*", "test_zz_*"))
    p = os.path.join(d, "oracle", fn)
    s = open(p).read()
    if s.count(a) < 1:
        return i, label, "PATTERN-MISSING", ""
    open(p, "w").write(s.replace(a, b, 1))
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=d, capture_output=True, text=True, env=env, timeout=900)
    shutil.rmtree(d, ignore_errors=True)
    last = [l for l in r.stdout.splitlines() if "FAILED" in l or "passed" in l or "failed" in l]
    return i, label, ("CAUGHT" if r.returncode != 0 else "SURVIVED"), (last[0] if last else r.stdout[-200:])


def main() -> int:
    idx = [int(a) for a in sys.argv[1:]] or list(range(len(M)))
    survived = 0
    with cf.ThreadPoolExecutor(4) as ex:
        for i, label, st, info in ex.map(run, idx):
            print(f"{i:2d} {st:9s} {label:30s} {info[:110]}", flush=True)
            survived += st != "CAUGHT"
    print(f"{len(idx) - survived}/{len(idx)} mutants caught")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
