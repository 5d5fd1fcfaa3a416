#!/usr/bin/env python
"""Writes precision_fp64_counts.txt: FP64 reference-decoder error counts for the precision study.

The study (Sec. IV-E, Eqs. 8-9) compares the GPU decoder's FP32, binary16 and 8-bit
fixed-point paths with the FP64 reference decoder on the same seeded frames and the same
perturbation stream.  Decoding 10^6 frames per point in FP64 takes about an hour of host
time, so the FP64 side is computed once here, by the reference decoder in ``oracle/`` only,
and stored as counts: frames, frame errors (any information bit wrong) and information-bit
errors per (study, Eb/N0).  The GPU test regenerates the same frames from the same seeds.

Frames of point j of a study: ``workload.frames(code, CHUNK, ebn0, seed=FRAME_SEED + j,
frame_offset=c * CHUNK)`` for chunks c = 0, 1, ...; perturbation key ``DECODER_SEED + j``,
frame id = index within the point (the chunk's frame offset plus the index in the chunk).

  python tests/golden/make_precision_golden.py [--threads N] [--only STUDY]

Points already present in the output file are kept (the script can be resumed).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1402_2773_gb300 import workload as wl  # noqa: E402

OUT = os.path.join(HERE, "precision_fp64_counts.txt")
CHUNK = 100_000
FRAME_SEED = 7000
DECODER_SEED = 11

# study -> (code factory name, Eb/N0 points, frames per point, decoder parameters)
STUDIES = {
    "c1_plain": ("code_c1", (3.5, 3.75, 4.0, 4.25, 4.5), 1_000_000,
                 dict(w=0.75, theta=-0.9, eta=0.96, lam=1.0, y_max=2.5, t_max=100, smooth_window=64,
                      variant=0)),
    "c2_sm": ("code_c2", (3.5, 3.625, 3.75, 3.875, 4.0), 100_000,
              dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300, smooth_window=64,
                   variant=3)),
}


def point_frames(code, eb, j, frames):
    """The point's frames in chunks: (frame offset, samples, transmitted words)."""
    for c in range(0, frames, CHUNK):
        F = min(CHUNK, frames - c)
        y, cw, sig = wl.frames(code, F, eb, seed=FRAME_SEED + j, frame_offset=c)
        yield c, y, cw, sig


def read_existing(path=OUT):
    done = {}
    if os.path.exists(path):
        for ln in open(path):
            if ln.startswith("#") or not ln.strip():
                continue
            p = ln.split()
            done[(p[0], float(p[1]))] = ln
    return done


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    O = oracle.load()
    done = read_existing()
    header = ("# FP64 reference decoder (oracle/), counts per point; regenerate with "
              "tests/golden/make_precision_golden.py\n"
              f"# frames: workload.frames(code, {CHUNK}, ebn0, seed={FRAME_SEED} + j, frame_offset=chunk start); "
              f"perturbation key {DECODER_SEED} + j; j = index of the point in its study\n"
              "# study ebn0_db frames frame_errors info_bit_errors info_bits_per_frame\n")
    lines = dict(done)
    for name, (factory, points, frames, prm) in STUDIES.items():
        if args.only and name != args.only:
            continue
        code = getattr(wl, factory)()
        info = code.encoder().info_pos
        p = oracle.make_params(**prm)
        for j, eb in enumerate(points):
            if (name, eb) in done:
                continue
            t0 = time.time()
            fe = be = 0
            for off, y, cw, sig in point_frames(code, eb, j, frames):
                bits, _, _ = O.decode_f64(code, y, sig, p, seed=DECODER_SEED + j, frame_offset=off,
                                          threads=args.threads)
                wrong = wl.unpack_bits(bits, code.n)[:, info] != wl.unpack_bits(cw, code.n)[:, info]
                fe += int(wrong.any(axis=1).sum())
                be += int(wrong.sum())
            lines[(name, eb)] = f"{name} {eb} {frames} {fe} {be} {len(info)}\n"
            with open(OUT + ".tmp", "w") as f:
                f.write(header)
                for key in sorted(lines, key=lambda k: (k[0], k[1])):
                    f.write(lines[key])
            os.replace(OUT + ".tmp", OUT)
            print(f"{name} {eb} dB: FER {fe / frames:.5f}, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
