"""CPU checks of the FMA-pipe exp2 used beside the MUFU ex2 in the forward
kernels: the committed coefficient header is what its generator writes, the
polynomials meet their stated error bounds, and a float32 emulation of the
device function (range reduction s = n + f, Horner, exponent-field add) has
the relative error of its polynomial over the whole argument range."""
import os
import re
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2412_20884_gb300", "csrc")
HEADER = os.path.join(CSRC, "exp2_poly.cuh")


def _coefficients():
    text = open(HEADER).read()
    out = {}
    for deg in (3, 5):
        m = re.search(rf"float exp2_poly{deg}\(float f\) {{ return (.*); }}", text)
        nums = [float(x.rstrip("f")) for x in re.findall(r"-?\d+\.\d+(?:e-?\d+)?f", m.group(1))]
        # Horner text lists the leading coefficient first, then c_{deg-1} .. c_0
        out[deg] = np.array(nums[::-1], dtype=np.float32)
        assert len(nums) == deg + 1
    errs = {int(d): float(e) for d, e in re.findall(r"kExp2Poly(\d)Err = ([0-9.e+-]+);", text)}
    return out, errs


def test_header_matches_generator(tmp_path):
    before = open(HEADER).read()
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp2_poly.py")], check=True, capture_output=True)
    assert open(HEADER).read() == before


def test_polynomial_error_bounds():
    coef, errs = _coefficients()
    f = np.linspace(-0.5, 0.5, 200001)
    for deg, c in coef.items():
        p = np.polynomial.polynomial.polyval(f, c.astype(np.float64))
        err = np.max(np.abs(p / np.exp2(f) - 1.0))
        assert err <= errs[deg] * 1.0001, (deg, err, errs[deg])
    assert errs[3] < 1e-4 and errs[5] < 2e-7


def _exp2_fma_f32(s, c):
    """The device function's steps in float32 (fmaf emulated in float64 and rounded once)."""
    s = np.asarray(s, np.float32)
    t = np.maximum(s, np.float32(-125.0))
    r = (t + np.float32(12582912.0)).astype(np.float32)
    f = (t - (r - np.float32(12582912.0)).astype(np.float32)).astype(np.float32)
    p = np.full_like(f, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p.astype(np.float64) * f.astype(np.float64) + np.float64(c[k])).astype(np.float32)
    bits = (p.view(np.uint32) + (r.view(np.uint32) << np.uint32(23))).astype(np.uint32)
    return bits.view(np.float32)


def test_exp2_fma_emulation_over_the_argument_range():
    coef, errs = _coefficients()
    rng = np.random.default_rng(0)
    s = np.concatenate([-rng.uniform(0, 125, 200000), -rng.uniform(0, 1, 100000), [0.0, -0.5, -1.0, -124.9]])
    s = s.astype(np.float32)
    ref = np.exp2(s.astype(np.float64))
    for deg, c in coef.items():
        got = _exp2_fma_f32(s, c).astype(np.float64)
        rel = np.abs(got / ref - 1.0)
        # polynomial error plus a few float32 roundings in the Horner steps
        assert rel.max() <= errs[deg] + 4e-7, (deg, rel.max())
    # below the clamp the result stays tiny and positive
    tiny = _exp2_fma_f32(np.array([-200.0, -1e9], np.float32), coef[5]).astype(np.float64)
    assert np.all(tiny > 0) and np.all(tiny <= 2.0 ** -124)
