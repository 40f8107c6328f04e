"""Check and time one split of the far field's multi-column FFT on the current GPU.

    python -m paper_1501_01652_gb300.fft_check --log2-len 20 --ncols 8 --radices 5,5,5,5 --tensor 1111

Seeded FP64 columns go through the built-in FP64 split and through the given one (passes of radix
2^r, the --tensor bits, first pass first, marking passes on the tensor cores); prints the largest
difference relative to the largest output and the time of the given split. A diagnostic for the
launch splits the autotuner chooses between (hankel_debug_fft_compare).
"""
import argparse

import paper_1501_01652_gb300 as hk


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2-len", type=int, default=20)
    ap.add_argument("--ncols", type=int, default=8)
    ap.add_argument("--radices", default="5,5,5,5")
    ap.add_argument("--tensor", default="1111", help="one digit per pass: 1 = tensor cores, 0 = FP64 pipe")
    ap.add_argument("--inverse", action="store_true")
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)
    radices = [int(r) for r in a.radices.split(",")]
    mask = sum(1 << i for i, ch in enumerate(a.tensor) if ch == "1")
    for _ in range(a.repeat):
        err, ms = hk.debug_fft_compare(a.log2_len, a.ncols, radices, mask, inverse=a.inverse)
        print("log2_len=%d ncols=%d radices=%s tensor=%s inverse=%d: max|diff|/max|out| = %.3e, %.3f ms"
              % (a.log2_len, a.ncols, radices, a.tensor, int(a.inverse), err, ms))


if __name__ == "__main__":
    main()
