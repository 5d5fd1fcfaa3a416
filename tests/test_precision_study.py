"""Reduced-precision decoding against the FP64 reference decoder (Sec. IV-E; FER/BER, 95 % intervals,
Eb/N0 shift).

Two studies, on the frames and perturbation streams that ``tests/golden/make_precision_golden.py``
decoded with the FP64 reference decoder (counts stored in ``precision_fp64_counts.txt``):
(1) the (3,6) N=1008 code, plain M-NGDBF (w = 0.75, theta = -0.9, eta = 0.96, T = 100,
Y_max = 2.5), 10^6 frames at each of 3.5 .. 4.5 dB in 0.25 dB steps; (2) the (6,32) N=2048
code with the SM-NGDBF parameters of the throughput workload (adaptive thresholds, smoothing,
T = 300), 10^5 frames at each of 3.5 .. 4.0 dB in 0.125 dB steps.

The GPU decodes the same frames in FP32, binary16 and 8-bit fixed point (NGDBF_FIXACC, Q = 8: the
held sample is the 8-bit Eq. 8 level code, the inversion function an exact int32 sum in steps of
Y_max 2^-16).  For each of the three, at every point, the FER must lie inside the FP64 decoder's
95 % Wilson interval, and the Eb/N0 shift -- the horizontal distance between the log-FER curves,
interpolated linearly in Eb/N0, at the FP64 FER of the middle point -- must be at most 0.1 dB.
Reported but not asserted: the paper's own fixed-point form (NGDBF_FIX, Eq. 9, where theta, w and
the perturbation are quantized to level centres too) and the uniform perturbation of Sec. V-B.
Set NGDBF_REPORT_DIR to write the numbers to precision_study.json there.
"""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

from paper_1402_2773_gb300 import ngdbf, workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_module():
    spec = importlib.util.spec_from_file_location("make_precision_golden",
                                                  os.path.join(GOLDEN_DIR, "make_precision_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


G = _golden_module()
FP64 = G.read_existing()

# variant name -> (precision, q_bits, extra variant bits, asserted)
VARIANTS = {"fp32": (ngdbf.NGDBF_FP32, 0, 0, True), "fp16": (ngdbf.NGDBF_FP16, 0, 0, True),
            "fix8": (ngdbf.NGDBF_FIXACC, 8, 0, True), "fix8_eq9": (ngdbf.NGDBF_FIX, 8, 0, False),
            "fp32_uniform": (ngdbf.NGDBF_FP32, 0, ngdbf.NGDBF_UNIFORM, False)}


def wilson(k, n, z=1.96):
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return max(0.0, c - h), min(1.0, c + h)


def ebn0_at(ebn0, fer_curve, target):
    """Eb/N0 where the piecewise-linear log10(FER) curve reaches target."""
    lf = [math.log10(max(f, 1e-12)) for f in fer_curve]
    lt = math.log10(target)
    for i in range(len(ebn0) - 1):
        a, b = lf[i], lf[i + 1]
        if (a - lt) * (b - lt) <= 0 and a != b:
            return ebn0[i] + (ebn0[i + 1] - ebn0[i]) * (a - lt) / (a - b)
    return float("nan")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2773_gb300 import _build
    _build.build_cuda()
    ngdbf.load()
    torch.cuda.set_device(0)


def _write_report(study, report):
    out = os.environ.get("NGDBF_REPORT_DIR")
    if not out:
        return
    os.makedirs(out, exist_ok=True)
    path = os.path.join(out, "precision_study.json")
    studies = {}
    if os.path.exists(path):
        with open(path) as f:
            studies = json.load(f)
    studies[study] = report
    with open(path, "w") as f:
        json.dump(studies, f, indent=1)


@pytest.mark.parametrize("study", list(G.STUDIES))
def test_precision_variants_match_fp64_reference(study):
    factory, points, frames, prm = G.STUDIES[study]
    missing = [eb for eb in points if (study, eb) not in FP64]
    assert not missing, f"FP64 counts missing for {study} at {missing}: run make_precision_golden.py"
    code = getattr(wl, factory)()
    info = torch.from_numpy(code.encoder().info_pos.astype(np.int64)).cuda()
    dc = ngdbf.DeviceCode.from_code(code)
    report = {"code": code.name, "params": prm, "frames_per_point": frames, "points": {}}
    fer = {v: [] for v in ["fp64", *VARIANTS]}
    nb = (code.n + 7) // 8
    shifts = torch.arange(8, device="cuda", dtype=torch.uint8)
    try:
        for j, eb in enumerate(points):
            p64 = FP64[(study, eb)].split()
            n64, fe64, be64, kinfo = int(p64[2]), int(p64[3]), int(p64[4]), int(p64[5])
            assert n64 == frames
            counts = {v: [0, 0] for v in VARIANTS}
            for off, y, cw, sig in G.point_frames(code, eb, j, frames):
                yt = torch.from_numpy(y).cuda()
                tx = ((torch.from_numpy(cw).cuda()[:, :, None] >> shifts) & 1).reshape(cw.shape[0], -1)[:, :code.n]
                tx = tx[:, info]
                for name, (prec, qb, extra, _) in VARIANTS.items():
                    gp = ngdbf.make_params(**dict(prm, variant=prm["variant"] | extra), precision=prec, q_bits=qb)
                    b, _, _ = dc.decode(yt, sig, gp, seed=G.DECODER_SEED + j, frame_offset=off)
                    rx = ((b[:, :, None] >> shifts) & 1).reshape(b.shape[0], nb * 8)[:, :code.n][:, info]
                    wrong = rx != tx
                    counts[name][0] += int(wrong.any(dim=1).sum())
                    counts[name][1] += int(wrong.sum())
            torch.cuda.synchronize()
            lo, hi = wilson(fe64, frames)
            pt = {"fp64": {"fer": fe64 / frames, "fer_ci95": [lo, hi], "ber_info": be64 / (frames * kinfo)}}
            fer["fp64"].append(fe64 / frames)
            for name, (fe, be) in counts.items():
                pt[name] = {"fer": fe / frames, "fer_ci95": list(wilson(fe, frames)),
                            "ber_info": be / (frames * kinfo), "inside_fp64_ci95": bool(lo <= fe / frames <= hi)}
                fer[name].append(fe / frames)
            report["points"][str(eb)] = pt
        target = fer["fp64"][len(points) // 2]
        e64 = ebn0_at(points, fer["fp64"], target)
        report["shift_reference_fer"] = target
        report["shift_db"] = {name: ebn0_at(points, fer[name], target) - e64 for name in VARIANTS}
    finally:
        dc.close()
        _write_report(study, report)
    for name, (_, _, _, asserted) in VARIANTS.items():
        if not asserted:
            continue
        outside = {eb: report["points"][str(eb)][name]["fer"] for eb in points
                   if not report["points"][str(eb)][name]["inside_fp64_ci95"]}
        assert not outside, f"{study} {name}: FER outside the FP64 95 % interval at {outside}"
        assert abs(report["shift_db"][name]) <= 0.1, f"{study} {name}: shift {report['shift_db'][name]:.3f} dB"
