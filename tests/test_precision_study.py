"""Reduced-precision decoding against the FP64 reference decoder (FER/BER, 95 % intervals, Eb/N0 shift).

Two studies.  (1) The (3,6) N=1008 code with the plain M-NGDBF parameters
(w = 0.75, theta = -0.9, eta = 0.96, T = 100, Y_max = 2.5) at Eb/N0 = 3.5, 4.0,
4.5 dB, 2*10^4 frames per point.  (2) The (6,32) N=2048 code with the SM-NGDBF
parameters of the throughput workload (adaptive thresholds, smoothing, T = 300)
at 3.5, 3.75, 4.0 dB, 5*10^3 frames per point (the FP64 reference decoder runs
on the host cores).  In each, the FP64 reference decoder and the GPU's FP32,
FP16 and 8-bit fixed-point paths decode the same seeded frames with the same
perturbation stream.  For each variant: the Eb/N0 shift -- the horizontal
distance between the log-FER curves, interpolated linearly in Eb/N0, at the
FP64 FER of the middle point -- must be at most 0.1 dB; FP32 and FP16 must also
lie inside the FP64 decoder's 95 % interval at every point.  The 8-bit fixed
point moves theta and w to their level values (Eq. 8), to which the
non-adaptive decoder is sensitive (Sec. IV-C); the study records whether its
FER is inside the FP64 interval and also compares it with the FP64 decoder run
on those quantized parameters.  Set NGDBF_REPORT_DIR to also write the numbers
to precision_study.json there.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1402_2773_gb300 import ngdbf, workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STUDIES = {
    "c1_plain": dict(code=wl.code_c1, name="peg(3,6) N=1008 M=504", ebn0=(3.5, 4.0, 4.5),
                     frames=int(os.environ.get("NGDBF_STUDY_FP64_FRAMES", "20000")),
                     params=dict(w=0.75, theta=-0.9, eta=0.96, lam=1.0, y_max=2.5, t_max=100,
                                 smooth_window=64, variant=0)),
    "c2_sm": dict(code=wl.code_c2, name="peg(6,32) N=2048 M=384", ebn0=(3.5, 3.75, 4.0),
                  frames=int(os.environ.get("NGDBF_STUDY_FP64_FRAMES_C2", "5000")),
                  params=dict(w=0.1875, theta=-0.7, eta=0.65, lam=0.993, y_max=2.0, t_max=300,
                              smooth_window=64, variant=3)),
}
VARIANTS = {"fp32": (ngdbf.NGDBF_FP32, 0), "fp16": (ngdbf.NGDBF_FP16, 0), "fix8": (ngdbf.NGDBF_FIX, 8)}


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


def quantized(v, q_bits, y_max):
    """The FP32-decided fixed-point level value of v (Eq. 8), in the units of v."""
    R = np.float32(2.0 ** q_bits / (2.0 * np.float32(y_max)))
    kmax = 2 ** (q_bits - 1) - 1
    a = np.float32(abs(np.float32(v))) * R
    k = int(np.floor(a)) if a < kmax else kmax
    b = k if v >= 0 else -k - 1
    return (2 * b + 1) * float(y_max) / 2 ** q_bits


@pytest.mark.parametrize("study", list(STUDIES))
def test_precision_variants_match_fp64_reference(study):
    st = STUDIES[study]
    EBN0, FRAMES_FP64, PARAMS = st["ebn0"], st["frames"], st["params"]
    code = st["code"]()
    O = oracle.load()
    dc = ngdbf.DeviceCode.from_code(code)
    info = code.encoder().info_pos
    report = {"code": st["name"], "params": PARAMS, "frames_per_point": FRAMES_FP64, "points": {}}
    refs = ["fp64", "fp64_fix8_params"]
    fer = {v: [] for v in [*refs, *VARIANTS]}
    # the FP64 decoder once more with theta and w replaced by their 8-bit fixed-point values:
    # separates the cost of quantizing the parameters from that of quantizing samples and noise
    qparams = dict(PARAMS, theta=quantized(PARAMS["theta"], 8, PARAMS["y_max"]),
                   w=quantized(PARAMS["w"], 8, PARAMS["y_max"]))
    report["fix8_parameter_values"] = {"theta": qparams["theta"], "w": qparams["w"]}
    inside = {}
    try:
        for j, eb in enumerate(EBN0):
            y, cw, sig = wl.frames(code, FRAMES_FP64, eb, seed=700 + j)
            tx = wl.unpack_bits(cw, code.n)[:, info]
            ok, ber = {}, {}
            for name, prm in (("fp64", PARAMS), ("fp64_fix8_params", qparams)):
                b64, _, _ = O.decode_f64(code, y, sig, oracle.make_params(**prm), seed=11 + j,
                                         threads=os.cpu_count() or 1)
                ok[name] = (b64 == cw).all(axis=1)
                ber[name] = float((wl.unpack_bits(b64, code.n)[:, info] != tx).mean())
            yt = torch.from_numpy(y).cuda()
            for name, (prec, qb) in VARIANTS.items():
                gp = ngdbf.make_params(**PARAMS, precision=prec, q_bits=qb)
                b, it, ps = dc.decode(yt, sig, gp, seed=11 + j)
                torch.cuda.synchronize()
                b = b.cpu().numpy()
                ok[name] = (b == cw).all(axis=1)
                ber[name] = float((wl.unpack_bits(b, code.n)[:, info] != tx).mean())
            n = FRAMES_FP64
            pt = {}
            for name in refs:
                k = int((~ok[name]).sum())
                pt[name] = {"fer": k / n, "fer_ci95": list(wilson(k, n)), "ber_info": ber[name]}
                fer[name].append(k / n)
            lo, hi = pt["fp64"]["fer_ci95"]
            for name in VARIANTS:
                k = int((~ok[name]).sum())
                # paired difference against FP64 on the same frames (McNemar normal approximation)
                n10 = int((ok["fp64"] & ~ok[name]).sum())
                n01 = int((~ok["fp64"] & ok[name]).sum())
                d = (n10 - n01) / n
                half = 1.96 * math.sqrt(n10 + n01) / n
                pt[name] = {"fer": k / n, "fer_ci95": list(wilson(k, n)), "ber_info": ber[name],
                            "fer_minus_fp64": d, "fer_minus_fp64_ci95": [d - half, d + half],
                            "inside_fp64_ci95": bool(lo <= k / n <= hi)}
                inside.setdefault(name, []).append(pt[name]["inside_fp64_ci95"])
                fer[name].append(k / n)
            rlo, rhi = pt["fp64_fix8_params"]["fer_ci95"]
            pt["fix8"]["inside_fp64_fix8_params_ci95"] = bool(rlo <= pt["fix8"]["fer"] <= rhi)
            report["points"][str(eb)] = pt
        target = fer["fp64"][1]
        e64 = ebn0_at(EBN0, fer["fp64"], target)
        report["shift_reference_fer"] = target
        report["shift_db"] = {name: ebn0_at(EBN0, fer[name], target) - e64 for name in VARIANTS}
        report["shift_db_fix8_vs_fp64_fix8_params"] = (ebn0_at(EBN0, fer["fix8"], target) -
                                                       ebn0_at(EBN0, fer["fp64_fix8_params"], target))
    finally:
        dc.close()
        out = os.environ.get("NGDBF_REPORT_DIR")
        if out:
            os.makedirs(out, exist_ok=True)
            path = os.path.join(out, "precision_study.json")
            studies = {}
            if os.path.exists(path):
                with open(path) as f:
                    studies = json.load(f)
                if "points" in studies:
                    studies = {}
            studies[study] = report
            with open(path, "w") as f:
                json.dump(studies, f, indent=1)
    # FP32 is the FP64 method in single precision; FP16 keeps every decision within the
    # FP64 interval; every variant costs at most 0.1 dB
    for name in ("fp32", "fp16"):
        assert all(inside[name]), f"{name} FER outside the FP64 interval: {report['points']}"
    for name in VARIANTS:
        assert abs(report["shift_db"][name]) <= 0.1, f"{name}: Eb/N0 shift {report['shift_db'][name]:.3f} dB"
