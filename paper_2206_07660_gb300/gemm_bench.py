"""Timing of the split-TF32 tensor-core GEMM on given shapes (pseudo-random operands).

    python -m paper_2206_07660_gb300.gemm_bench --shape 40000 800 5408 1 1 [--bn 224] [--iters 5] [--f16]

A shape is M N K batch fp64out: C[z] (M x N, real) += A[z] (M x K) B (N x K)^T with
three TF32 products (hi*hi + hi*lo + lo*hi), fp64 accumulating output when fp64out = 1
and a plain fp32 store otherwise (--f16: fp16 pieces, kind::f16, instead of TF32
pieces).  --bn forces the N tile (32..128 ping-pong epilogue,
160..256 split epilogue); without it the per-shape autotuner picks the tile.  Prints one
line per shape: mean device milliseconds per launch (CUDA events) and tensor-pipe
TFLOP/s (2 M N K batch x 3 products).  Example shapes: the last step of the P~0 chain
at nao 52, naux 400, ntau 100 is 40000 800 5408 1 1 (M = ntau naux, N = 2 naux,
K = 2 nao^2); the first step of the Sigma~ chain there is 400 5408 800 100 0.
"""
import argparse
import ctypes

from .gw import load


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--shape", nargs=5, type=int, action="append", required=True, metavar=("M", "N", "K", "B", "F64"))
    p.add_argument("--bn", type=int, default=0, help="force this N tile (0: autotuner)")
    p.add_argument("--iters", type=int, default=5)
    p.add_argument("--f16", action="store_true", help="fp16 pieces (kind::f16) instead of TF32 pieces")
    args = p.parse_args(argv)
    lib = load()
    lib.gwdbg_umma_bench.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_double)]
    lib.gwdbg_umma_bench.restype = ctypes.c_int
    lib.gwdbg_umma_bench_f16.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_double)]
    lib.gwdbg_umma_bench_f16.restype = ctypes.c_int
    bench = lib.gwdbg_umma_bench_f16 if args.f16 else lib.gwdbg_umma_bench
    blk = 64 if args.f16 else 32
    lib.gwdbg_umma_force_bn.argtypes = [ctypes.c_int]
    lib.gwdbg_umma_force_bn.restype = ctypes.c_int
    old = lib.gwdbg_umma_force_bn(args.bn)
    rc = 0
    try:
        for (m, n, k, b, f) in args.shape:
            ms = ctypes.c_double()
            kpad = (k + blk - 1) // blk * blk
            st = bench(m, n, kpad, b, f, args.iters, ctypes.byref(ms))
            tf = 6.0 * m * n * kpad * b / (ms.value * 1e-3) / 1e12 if st == 0 and ms.value > 0 else 0.0
            print("M=%d N=%d K=%d batch=%d fp64out=%d bn=%s %s status=%d ms=%.3f tensor_TFLOP/s=%.1f"
                  % (m, n, kpad, b, f, args.bn or "auto", "f16" if args.f16 else "tf32", st, ms.value, tf),
                  flush=True)
            rc = rc or st
    finally:
        lib.gwdbg_umma_force_bn(old)
    return 0 if rc == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
