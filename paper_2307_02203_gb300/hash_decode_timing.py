"""Decoding throughput of the paper's NDF architecture (hash grid, Fourier
features, SnakeAlt encoder and decoder) on one GPU, with seeded parameters.

    python -m paper_2307_02203_gb300.hash_decode_timing [--grid X Y Z] [--mode tc|cached|fp32]
                                                        [--refs R] [--repeat K]

Prints milliseconds per decoded volume (CUDA events around K calls of
ndf_hash_infer, or one ndf_hash_infer_batch of R references when R > 1).
Decoding does not depend on training, so the parameters are the model's seeded
initialisation with a non-zero output layer.
"""
from __future__ import annotations

import argparse

import numpy as np


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--grid", type=int, nargs=3, default=[250, 352, 20], metavar=("X", "Y", "Z"))
    ap.add_argument("--mode", choices=["tc", "cached", "fp32"], default="tc")
    ap.add_argument("--refs", type=int, default=1, help="references per call")
    ap.add_argument("--repeat", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    from paper_2307_02203_gb300 import ndf

    X, Y, Z = args.grid
    N = X * Y * Z
    stream = torch.cuda.Stream()
    ctx = ndf.ndf_create(0, stream.cuda_stream)
    arch = ndf.ndf_hash_arch_default()
    m = ndf.ndf_hash_model_create(ctx, arch, ndf.NDF_MEASURE_PEARSON, False, 1, X, Y, Z)
    p = np.empty(ndf.ndf_hash_model_param_count(m), np.float32)
    ndf.ndf_hash_model_get_params(m, p)
    p[-129:-1] = np.random.default_rng(1).uniform(-0.3, 0.3, 128)  # output layer (0 at init)
    ndf.ndf_hash_model_set_params(m, p)
    mode = {"tc": (ndf.NDF_HASH_DECODE_TC, False), "cached": (ndf.NDF_HASH_DECODE_TC, True),
            "fp32": (ndf.NDF_HASH_DECODE_FP32, False)}[args.mode]
    ndf.ndf_hash_set_decode(m, *mode)
    R = max(1, args.refs)
    out = torch.empty((R, N), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(2)

    def call():
        refs = [int(r) for r in rng.integers(0, N, size=R)]
        if R == 1:
            ndf.ndf_hash_infer(m, refs[0], out[0])
        else:
            ndf.ndf_hash_infer_batch(m, refs, out)

    for _ in range(args.warmup):
        call()
    ndf.ndf_synchronize(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.repeat):
        call()
    e1.record(stream)
    ndf.ndf_synchronize(ctx)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (args.repeat * R)
    print(f"hash NDF decode ({args.mode}, {R} reference(s) per call, {X}x{Y}x{Z} = {N} vertices): "
          f"{ms:.4f} ms per volume")
    ndf.ndf_hash_model_free(m)
    ndf.ndf_destroy(ctx)


if __name__ == "__main__":
    main()
