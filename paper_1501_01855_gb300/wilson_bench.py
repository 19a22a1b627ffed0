"""Time the Wilson kernel K alone through the C ABI (ovl_bench_wilson), one sign-function
application (--sign ETA), or mixed-precision solves (--solve TOL).

    python -m paper_1501_01855_gb300.wilson_bench --dims 24 24 24 48 --prec f32 --nrhs 1

Unit links, a random input spinor, the kernel launched `--iters` times back to back on
the context stream and timed with CUDA events. Prints milliseconds per launch, the
algorithmic bytes of one launch (each input spinor read once, each output written once,
the links read once) and the rate they imply. `--variant` forces a kernel shape (0 one
thread per site, 1 direction split, 2 4D tiles, 3 lane pairs for double-float); the
default lets the create-time autotuner choose.
"""
import argparse

import numpy as np

from . import binding as B

PRECS = {"f64": B.OVL_PREC_F64, "f32": B.OVL_PREC_F32, "f16": B.OVL_PREC_F16, "df64": B.OVL_PREC_F64E}


def unit_links(dims):
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 48], metavar=("LX", "LY", "LZ", "LT"))
    ap.add_argument("--prec", choices=sorted(PRECS), default="f32")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--variant", type=int, default=-1, choices=[-1, 0, 1, 2, 3])
    ap.add_argument("--sign", type=float, default=0.0, metavar="ETA",
                    help="instead: one sign-function application to accuracy ETA on nrhs random "
                         "vectors, 20 poles")
    ap.add_argument("--solve", type=float, default=0.0, metavar="TOL",
                    help="instead: mixed-precision GMRESR(relSUMR) solves of nrhs Gaussian sources to "
                         "relative residual TOL (mu = 0.05, 20 poles, eps 0.3 links, seed 1002)")
    args = ap.parse_args(argv)
    if args.sign > 0:
        return sign_main(args)
    if args.solve > 0:
        return solve_main(args)
    p = B.ovl_params_default()
    p.a_override, p.b_override = 0.2, 2.6     # skip the Lanczos bound estimate
    p.wilson_variant = args.variant
    ctx = B.Overlap(tuple(args.dims), unit_links(args.dims), 1.4, 0.05, 8, 1e-3, params=p)
    prec = PRECS[args.prec]
    ms, nbytes = ctx.bench_wilson(prec, args.nrhs, args.iters)
    v = int(np.prod(args.dims))
    variant = ctx.wilson_tuning(prec)[0]
    print("Wilson K %s, %s, nrhs %d, variant %d: %.4f ms per launch, %.1f MB algorithmic, %.0f GB/s, "
          "%.2f G site-applications/s" % (args.prec, "x".join(map(str, args.dims)), args.nrhs, variant, ms,
                                          nbytes / 1e6, nbytes / ms / 1e6, v * args.nrhs / ms / 1e6))
    ctx.close()


def sign_main(args):
    import time
    p = B.ovl_params_default()
    p.a_override, p.b_override = 0.2, 2.6
    p.wilson_variant = args.variant
    ctx = B.Overlap(tuple(args.dims), unit_links(args.dims), 1.4, 0.05, 20, 1e-10, params=p)
    rng = np.random.default_rng(7)
    shp = (args.nrhs,) + tuple(reversed(args.dims)) + (4, 3)
    v = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    out = np.empty_like(v)
    t0 = time.perf_counter()
    for _ in range(args.iters):
        ctx.sign_apply(v, out, eta=args.sign, prec=PRECS[args.prec])
    dt = (time.perf_counter() - t0) / args.iters
    print("sign %s, %s, nrhs %d, eta %g: %.1f ms per application (host buffers)"
          % (args.prec, "x".join(map(str, args.dims)), args.nrhs, args.sign, dt * 1e3))
    ctx.close()


def solve_main(args):
    import time
    import synth
    dims = tuple(args.dims)
    U = synth.gauge_links(dims, 0.3, 1002)
    b = synth.gaussian_source(dims, 3002, nvec=args.nrhs)
    ctx = B.Overlap(dims, U, 1.4, 0.05, 20, 1e-10)
    x = np.zeros_like(b)
    ctx.solve(b, x, args.solve)            # warm-up: workspaces, graphs, step caps
    for _ in range(args.iters):
        x[...] = 0
        t0 = time.perf_counter()
        infos = ctx.solve(b, x, args.solve)
        dt = time.perf_counter() - t0
        print("solve %s, nrhs %d, tol %g: %.1f ms, true residual %.2e, inner iterations %d"
              % ("x".join(map(str, dims)), args.nrhs, args.solve, dt * 1e3,
                 max(i["true_residual"] for i in infos), infos[0]["inner_iters"]), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
