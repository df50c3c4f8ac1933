"""Mutation check of the oracle's pins (CPU only, not collected by pytest).

Plants one plausible mistake at a time (a dropped term, a wrong sign or
conjugate, swapped operands or indices, a different reading of a convention)
in a temporary copy of ``oracle/`` and runs the oracle pins
(``tests/test_oracle_pins.py``, ``tests/test_oracle_unet.py``) against it.
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
]
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
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_unet.py", "-x", "-q", "-p", "no:cacheprovider"],
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
