"""Mutation check of the oracle's pins (CPU only). Each case plants one plausible mistake
in a copy of the C oracle -- a wrong tap, sign, index or operand, a dropped term or
stage, a wrong border, threshold or tie rule, a wrong frame -- builds the copy in a
temporary directory, and runs the pins of test_oracle_pins.py against it: at least one
pin must fail for every mutant. The unchanged copy, run the same way, passes every pin.
The oracle itself is never modified."""
import concurrent.futures as cf
import inspect
import itertools
import os
import subprocess

import pytest

from oracle import chain as oc
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oc.__file__), "kf_oracle.c")

# name: (text in kf_oracle.c, exactly once; its replacement)
MUTANTS = {
    "convert divides by 256": ("/ 255.0;", "/ 256.0;"),
    "asymmetric Gaussian tap": ("4.0 / 16, 6.0 / 16, 4.0 / 16", "4.0 / 16, 6.0 / 16, 5.0 / 16"),
    "Gaussian-H reflects instead of clamping": (
        "clampi(x + k, 0, W - 1)",
        "clampi(x + k < 0 ? -(x + k) : (x + k > W - 1 ? 2 * (W - 1) - (x + k) : x + k), 0, W - 1)"),
    "Gaussian-V pass dropped": ("clampi(y + k, 0, H - 1)", "clampi(y, 0, H - 1)"),
    "Sobel x sign flipped": ("ix[(int64_t)y * W + x] = gx;", "ix[(int64_t)y * W + x] = -gx;"),
    "Sobel outputs transposed": (
        "ix[(int64_t)y * W + x] = gx;\n            iy[(int64_t)y * W + x] = gy;",
        "ix[(int64_t)y * W + x] = gy;\n            iy[(int64_t)y * W + x] = gx;"),
    "Prewitt weights instead of Sobel": ("s[3] = {1.0, 2.0, 1.0};", "s[3] = {1.0, 1.0, 1.0};"),
    "Sobel y one-sided difference": ("g[(int64_t)clampi(y - 1, 0, H - 1) * W + xx]",
                                     "g[(int64_t)clampi(y, 0, H - 1) * W + xx]"),
    "cross product uses Ix twice": ("pxy[i] = ix[i] * iy[i];", "pxy[i] = ix[i] * ix[i];"),
    "box 3 wide instead of 5": ("for (int dx = -2; dx <= 2; ++dx)", "for (int dx = -1; dx <= 1; ++dx)"),
    "box pads with zeros": (
        "s += in[(int64_t)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];",
        "if (y + dy >= 0 && y + dy < H && x + dx >= 0 && x + dx < W) s += in[(int64_t)(y + dy) * W + (x + dx)];"),
    "determinant loses its cross term": ("double det = sxx[i] * syy[i] - sxy[i] * sxy[i];",
                                         "double det = sxx[i] * syy[i];"),
    "trace term added": ("r[i] = det - k * tr * tr;", "r[i] = det + k * tr * tr;"),
    "trace not squared": ("r[i] = det - k * tr * tr;", "r[i] = det - k * tr;"),
    "Harris reads the sums in the wrong order": (
        "kfo_harris(n, m[KFO_SXX], m[KFO_SXY], m[KFO_SYY], k, m[KFO_R]);",
        "kfo_harris(n, m[KFO_SXX], m[KFO_SYY], m[KFO_SXY], k, m[KFO_R]);"),
    "box of the wrong product": ("kfo_box5(H, W, m[KFO_PXY], m[KFO_SXY]);",
                                 "kfo_box5(H, W, m[KFO_PXX], m[KFO_SXY]);"),
    "threshold not strict": ("int keep = c > thr;", "int keep = c >= thr;"),
    "strict local maximum (plateaus dropped)": (
        "if (r[(int64_t)yy * W + xx] > c) keep = 0;",
        "if ((dy || dx) && r[(int64_t)yy * W + xx] >= c) keep = 0;"),
    "NMS ignores the right-hand column": ("for (int dx = -1; dx <= 1 && keep; ++dx)",
                                          "for (int dx = -1; dx <= 0 && keep; ++dx)"),
    "ties go to the higher raster index": ("(r[q] == v && q < p)", "(r[q] == v && q > p)"),
    "points in ascending response": ("if (r[q] > v ||", "if (r[q] < v ||"),
    "LK gradients at half gain": ("double gx = ix[q] / 8.0, gy = iy[q] / 8.0,",
                                  "double gx = ix[q] / 4.0, gy = iy[q] / 4.0,"),
    "LK temporal difference reversed": ("gt = g_cur[q] - g_prev[q];", "gt = g_prev[q] - g_cur[q];"),
    "LK solve with the wrong diagonal": ("u[i] = -(a11 * b0 - a01 * b1) / det;",
                                         "u[i] = -(a00 * b0 - a01 * b1) / det;"),
    "LK never reports a singular window": ("if (fabs(det) <= 1e-12 * tr * tr) {",
                                           "if (det == 0.0 && tr == 0.0) {"),
    "LK window asymmetric": ("for (int dx = -win; dx <= win; ++dx)", "for (int dx = -win; dx < win; ++dx)"),
    "LK frames swapped": ("kfo_lk(H, W, gp, maps[KFO_G],", "kfo_lk(H, W, maps[KFO_G], gp,"),
    "LK against the unsmoothed previous frame": ("kfo_lk(H, W, gp,", "kfo_lk(H, W, fp,"),
    "volume tracks each frame against itself": (
        "in + (int64_t)(t - 1) * H * pitch, in + (int64_t)t * H * pitch",
        "in + (int64_t)t * H * pitch, in + (int64_t)t * H * pitch"),
}


def _pin_calls():
    """Every pin with each of its parameter sets, in source order (cheap pins first)."""
    fns = [f for n, f in inspect.getmembers(pins, inspect.isfunction) if n.startswith("test_")]
    fns.sort(key=lambda f: f.__code__.co_firstlineno)
    calls = []
    for f in fns:
        marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            calls.append((f.__name__, f, {}))
            continue
        grids = []
        for m in marks:
            names = [s.strip() for s in m.args[0].split(",")]
            grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]])
        for combo in itertools.product(*grids):
            kw = {k: v for d in combo for k, v in d.items()}
            calls.append((f.__name__, f, kw))
    return calls


def _build(path_c, path_so):
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-o", path_so, path_c, "-lm"],
                   check=True, capture_output=True)
    return path_so


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {"unchanged": src}
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, f"{name}: the planted text must occur exactly once"
        jobs[name] = src.replace(old, new)
    paths = {}
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {}
        for i, (name, text) in enumerate(jobs.items()):
            c, so = str(d / f"m{i}.c"), str(d / f"libm{i}.so")
            with open(c, "w") as fh:
                fh.write(text)
            futs[name] = ex.submit(_build, c, so)
        paths = {name: f.result() for name, f in futs.items()}
    return paths


def _failing_pin(monkeypatch, so):
    """Run the pins against the oracle built at `so`; the first failing pin, or None."""
    monkeypatch.setattr(oc, "build", lambda force=False: so)
    monkeypatch.setattr(oc, "_lib", None)
    try:
        for name, f, kw in _pin_calls():
            try:
                f(**kw)
            except Exception as e:  # an assertion, or numpy rejecting the mutant's output
                return f"{name}{kw or ''}: {type(e).__name__}"
        return None
    finally:
        oc._lib = None


def test_unchanged_copy_passes_every_pin(builds, monkeypatch):
    assert _failing_pin(monkeypatch, builds["unchanged"]) is None


@pytest.mark.parametrize("name", list(MUTANTS))
def test_every_planted_mistake_fails_a_pin(builds, monkeypatch, name):
    assert _failing_pin(monkeypatch, builds[name]) is not None, f"no pin catches: {name}"
