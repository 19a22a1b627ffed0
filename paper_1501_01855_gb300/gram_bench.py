"""Time the Gram block G = A^dag B alone through the C ABI (ovl_bench_gram).

    python -m paper_1501_01855_gb300.gram_bench --dims 16 16 16 32 --na 128 --nb 128 --prec f64

Random fields of na and nb spinors held by the library; the block launched `--iters`
times back to back on the context stream and timed with CUDA events, with the tensor-core
path (method 0, FP64-level accuracy) and the CUDA-core path (method 1, FP32 products).
Prints milliseconds per block and the rates that bound each path: complex
multiply-adds per second (na nb 12 V per block), the tensor-core BF16 rate the split
arithmetic implies (26 digit-pair products of 128 x 64 x 16 per 16 complex elements and
tile of 64 x 64 vectors), and the operand bytes read per second.
"""
import argparse

import numpy as np

from . import binding as B

PRECS = {"f64": B.OVL_PREC_F64, "f32": B.OVL_PREC_F32}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32], metavar=("LX", "LY", "LZ", "LT"))
    ap.add_argument("--na", type=int, default=128)
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--prec", choices=sorted(PRECS), default="f64")
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--method", type=int, default=-1, choices=[-1, 0, 1], help="-1: both")
    args = ap.parse_args(argv)
    dims = tuple(args.dims)
    lx, ly, lz, lt = dims
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    p = B.ovl_params_default()
    p.a_override, p.b_override = 0.2, 2.6
    ctx = B.Overlap(dims, u, 1.4, 0.05, 8, 1e-3, params=p)
    v = int(np.prod(dims))
    na, nb = args.na, args.nb
    cmacs = float(na) * nb * 12 * v
    tiles = -(-na // 64) * -(-nb // 64)
    # per stage of 16 complex elements: 2 K-steps x 26 MMAs of 128 x 64 x 16, 2 flops each
    tc_flops = tiles * (12.0 * v / 16) * 2 * 26 * (128 * 64 * 16) * 2
    sb = 192 if args.prec == "f64" else 96
    for method in ([0, 1] if args.method < 0 else [args.method]):
        ms = ctx.bench_gram(PRECS[args.prec], na, nb, method, args.iters)
        line = ("Gram %s, %s, %d x %d, method %d (%s): %.3f ms per block, %.2f T complex MAC/s, %.0f GB/s of operands"
                % (args.prec, "x".join(map(str, dims)), na, nb, method,
                   "tensor cores, FP64-level" if method == 0 else "CUDA cores, FP32 products", ms,
                   cmacs / (ms * 1e-3) / 1e12, (na + nb) * v * sb / (ms * 1e-3) / 1e9))
        if method == 0:
            line += ", %.0f TFLOP/s BF16 on the tensor pipe" % (tc_flops / (ms * 1e-3) / 1e12)
        print(line, flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
