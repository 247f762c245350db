"""Mutation check of the oracle's pins (CPU only). Each case plants one plausible mistake
in a copy of an oracle -- a wrong tap, sign, index or operand, a dropped term or stage,
a wrong border, threshold or tie rule, a wrong frame, a one-sided halo -- and runs that
oracle's pins against the copy: at least one pin must fail for every mutant. The C
oracle's copies are built in a temporary directory; a Python oracle's copy is executed
as a fresh module and swapped in for the pin module's reference to it. The unchanged
copies, run the same way, pass every pin. The oracles themselves are never modified.
Changes that cannot alter any result are not listed (e.g. in the plan reference, every
external input of a group is stored by an earlier group by construction)."""
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
    "Ix without vertical smoothing": (
        "gx += s[d + 1] * (g[(int64_t)yy * W + clampi(x + 1, 0, W - 1)] -\n"
        "                                  g[(int64_t)yy * W + clampi(x - 1, 0, W - 1)]);",
        "gx += s[d + 1] * (g[(int64_t)y * W + clampi(x + 1, 0, W - 1)] -\n"
        "                                  g[(int64_t)y * W + clampi(x - 1, 0, W - 1)]);"),
    "Gaussian-V clamps to the width": ("clampi(y + k, 0, H - 1)", "clampi(y + k, 0, H - 1 < W - 1 ? H - 1 : W - 1)"),
    "trace is a difference": ("double tr = sxx[i] + syy[i];", "double tr = sxx[i] - syy[i];"),
    "convert ignores pitch": ("in[(int64_t)y * pitch + x] / 255.0", "in[(int64_t)y * W + x] / 255.0"),
    "count counts every pixel": ("count += keep;", "count += 1;"),
    "box 3 rows instead of 5": ("for (int dy = -2; dy <= 2; ++dy)\n                for (int dx = -2; dx <= 2; ++dx)",
                                "for (int dy = -1; dy <= 1; ++dy)\n                for (int dx = -2; dx <= 2; ++dx)"),
    "NMS ignores the row above": ("for (int dy = -1; dy <= 1 && keep; ++dy)", "for (int dy = 0; dy <= 1 && keep; ++dy)"),
    "volume masks at the width's stride": ("masks + (int64_t)t * H * pitch, pitch);", "masks + (int64_t)t * H * W, pitch);"),
    "selection keeps one too few": ("int pos = n < K ? n : K;", "int pos = n < K - 1 ? n : K - 1;"),
    "LK point coordinates swapped": ("int py = idx[i] / W, px = idx[i] % W;", "int py = idx[i] % W, px = idx[i] / W;"),
    "LK cross term from Iy twice": ("a01 += gx * gy;", "a01 += gy * gy;"),
    "LK v with the wrong sign": ("v[i] = -(a00 * b1 - a01 * b0) / det;", "v[i] = (a00 * b1 - a01 * b0) / det;"),
    "Iy sign flipped": ("iy[(int64_t)y * W + x] = gy;", "iy[(int64_t)y * W + x] = -gy;"),
    "Harris run with k = 0": ("kfo_harris(n, m[KFO_SXX], m[KFO_SXY], m[KFO_SYY], k, m[KFO_R]);",
                              "kfo_harris(n, m[KFO_SXX], m[KFO_SXY], m[KFO_SYY], 0.0, m[KFO_R]);"),
    "threshold not applied": ("int64_t count = kfo_nms(H, W, m[KFO_R], thr, mask, mask_pitch);",
                              "int64_t count = kfo_nms(H, W, m[KFO_R], -1e300, mask, mask_pitch);"),
    "selection shifts one too few": ("for (int i = last; i > pos; --i) idx[i] = idx[i - 1];",
                                     "for (int i = last; i > pos + 1; --i) idx[i] = idx[i - 1];"),
    "LK b from Ix only": ("b1 += gy * gt;", "b1 += gx * gt;"),
    "LK determinant sign": ("double det = a00 * a11 - a01 * a01;", "double det = a00 * a11 + a01 * a01;"),
    "LK window rows clamped to the width": ("clampi(py + dy, 0, H - 1) * W", "clampi(py + dy, 0, W - 1) * W"),
    "previous frame smoothed along x only": ("kfo_gauss_v(H, W, g1p, gp);", "memcpy(gp, g1p, sizeof(double) * n);"),
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


def _pin_calls(module=pins):
    """Every pin of `module` with each of its parameter sets, in source order (cheap pins
    first)."""
    fns = [f for n, f in inspect.getmembers(module, inspect.isfunction)
           if n.startswith("test_") and f.__module__ == module.__name__]
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


# ------------------------------------------------------------------ the Python oracles
# module: (pin modules and the name each binds the module to, {name: (text, replacement)})
PY_MUTANTS = {
    "pchain": (["test_pchain_oracle:op"], {
        "gray takes blue for green": ("150.0 * c[..., 1]", "150.0 * c[..., 2]"),
        "gray scale off": ("(256.0 * 255.0)", "(255.0 * 255.0)"),
        "IIR weights swapped": ("return y_prev + alpha * (g - y_prev)", "return g + alpha * (y_prev - g)"),
        "IIR first frame scaled": ("return g.copy()", "return alpha * g"),
        "Gaussian weights do not sum to one": ("w = {-1: 0.25, 0: 0.5, 1: 0.25}", "w = {-1: 0.25, 0: 0.25, 1: 0.25}"),
        "gradient one-sided": ("gx += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))",
                               "gx += s[d] * (_shift(G, d, 1) - _shift(G, d, 0))"),
        "gradient y along x": ("gy += s[d] * (_shift(G, 1, d) - _shift(G, -1, d))",
                               "gy += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))"),
        "L2 magnitude instead of L1": ("np.abs(gx) + np.abs(gy)", "np.hypot(gx, gy)"),
        "threshold not strict": ("mask = M > tau\n", "mask = M >= tau\n"),
        "regions transposed": ("r = (GRID * y // H) * GRID + (GRID * x // W)",
                               "r = (GRID * x // W) * GRID + (GRID * y // H)"),
        "region sums swapped": ("regions[r, 1] += x\n        regions[r, 2] += y",
                                "regions[r, 1] += y\n        regions[r, 2] += x"),
        "Kalman half-step transition": ("F = np.block([[I2, I2], [np.zeros((2, 2)), I2]])",
                                        "F = np.block([[I2, 0.5 * I2], [np.zeros((2, 2)), I2]])"),
        "Kalman process noise off": ("I2 / 3.0, I2 / 2.0", "I2 / 2.0, I2 / 2.0"),
        "Kalman prediction adds no noise": ("P = F @ P @ F.T + Q", "P = F @ P @ F.T"),
        "Kalman innovation reversed": ("s = s + K @ (z - Hm @ s)", "s = s + K @ (Hm @ s - z)"),
        "Kalman covariance not updated": ("P = (np.eye(4) - K @ Hm) @ P", "P = P"),
        "Kalman gain without the inverse": ("K = P @ Hm.T @ np.linalg.inv(S)", "K = P @ Hm.T"),
        "Kalman innovation covariance without R": ("S = Hm @ P @ Hm.T + R", "S = Hm @ P @ Hm.T"),
        "Kalman start transposed": ("s = np.array([z[0], z[1], 0.0, 0.0])", "s = np.array([z[1], z[0], 0.0, 0.0])"),
        "Kalman initial covariance swapped": ("P = np.diag([r, r, p0, p0])", "P = np.diag([p0, p0, r, r])"),
        "regions by width for rows": ("r = (GRID * y // H) * GRID + (GRID * x // W)",
                                      "r = (GRID * y // W) * GRID + (GRID * x // W)"),
        "magnitude of the sum": ("np.abs(gx) + np.abs(gy)", "np.abs(gx + gy)"),
        "Gaussian not separable": ("out += w[dy] * w[dx] * _shift(y, dy, dx)", "out += w[dy] * w[dy] * _shift(y, dy, dx)"),
        "count of the complement": ("return mask.astype(np.uint8), int(mask.sum()), regions",
                                    "return mask.astype(np.uint8), int((~mask).sum()), regions"),
        "IIR restarted every frame": ("        y = iir(y, Y)\n", "        y = iir(None, Y)\n"),
        "centroid transposed": ("z = np.array([sx / cnt, sy / cnt])", "z = np.array([sy / cnt, sx / cnt])"),
    }),
    "stbox": (["test_stbox_oracle:ost"], {
        "gray takes blue for green": ("150 * c[..., 1]", "150 * c[..., 2]"),
        "temporal window one frame late": ("comb(n, k) * g[max(t - n + k, 0)]", "comb(n, k) * g[max(t - n + k - 1, 0)]"),
        "temporal weights linear": ("comb(n, k) * g[max(t - n + k, 0)]", "(k + 1) * g[max(t - n + k, 0)]"),
        "Gaussian box weights": ("w = {-1: 1, 0: 2, 1: 1}", "w = {-1: 1, 0: 1, 1: 1}"),
        "Prewitt weights": ("s = {-1: 1, 0: 2, 1: 1}", "s = {-1: 1, 0: 1, 1: 1}"),
        "gradient y along x": ("gy += s[d] * (_shift(G, 1, d) - _shift(G, -1, d))",
                               "gy += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))"),
        "magnitude of the sum": ("return np.abs(gx) + np.abs(gy)", "return np.abs(gx + gy)"),
        "real-valued chain scaled twice": ("/ 2.0 ** n", "/ 2.0 ** (n + 1)"),
        "clipped reads spatial one-sided": ("cx = sum(spans(W, x, DX, DX))", "cx = sum(spans(W, x, 0, DX))"),
        "gray ignores red": ("77 * c[..., 0] + 150", "0 * c[..., 0] + 150"),
        "spatial reach 1": ("DX = 2  #", "DX = 1  #"),
        "model writes each box twice": ("+ x * x * t * bytes_out)", "+ 2 * x * x * t * bytes_out)"),
        "model boxes ignore t": ("B = W * H * T / (x * x * t)", "B = W * H * T / (x * x)"),
        "count of the previous frame": ("counts[t] = int(masks[t].sum())", "counts[t] = int(masks[max(t - 1, 0)].sum())"),
        "Sobel x one-sided": ("gx += s[d] * (_shift(G, d, 1) - _shift(G, d, -1))",
                              "gx += s[d] * (_shift(G, d, 1) - _shift(G, d, 0))"),
        "utilisation spatial halo one-sided": ("return x * x * t / ((x + 2 * DX) ** 2 * (t + n))",
                                               "return x * x * t / ((x + DX) ** 2 * (t + n))"),
        "clipped reads skip the first box": ("for s in range(0, N, b)]", "for s in range(b, N, b)]"),
        "real-valued chain skips the Gaussian": ("M = pchain.gradient(pchain.gauss3(z))[2]", "M = pchain.gradient(z)[2]"),
        "threshold scale doubled": ("return 261120 << n", "return 261120 << (n + 1)"),
        "threshold not strict": ("masks[t] = M > thr", "masks[t] = M >= thr"),
        "model halo one-sided": ("(x + 2 * DX) ** 2 * (t + n) * bytes_in", "(x + DX) ** 2 * (t + n) * bytes_in"),
        "model temporal halo two-sided": ("(t + n) * bytes_in", "(t + 2 * n) * bytes_in"),
        "clipped reads on the future side": ("ct = sum(spans(T, t, n, 0))", "ct = sum(spans(T, t, 0, n))"),
        "clipped reads not clipped at the end": ("min(s + b + r_hi, N) - max(s - r_lo, 0)",
                                                 "s + b + r_hi - max(s - r_lo, 0)"),
        "utilisation temporal halo two-sided": ("return x * x * t / ((x + 2 * DX) ** 2 * (t + n))",
                                                "return x * x * t / ((x + 2 * DX) ** 2 * (t + 2 * n))"),
    }),
    "partition": (["test_partition_oracle:op", "test_stbox_oracle:opart"], {
        "cut bit read off by one": ("if cuts >> i & 1:", "if cuts >> (i + 1) & 1:"),
        "one cut point too few": ("repeat=n - 1", "repeat=n - 2"),
        "halo is the maximum radius": ("return (sum(s.rx for s in stages[a:b + 1]), sum(s.ry",
                                       "return (max(s.rx for s in stages[a:b + 1]), sum(s.ry"),
        "spatial halo one-sided": ("(x + 2 * Rx) * (y + 2 * Ry) * (t + Rt) * stages[a].in_bytes",
                                   "(x + Rx) * (y + Ry) * (t + Rt) * stages[a].in_bytes"),
        "temporal halo two-sided": ("(t + Rt) * stages[a].in_bytes", "(t + 2 * Rt) * stages[a].in_bytes"),
        "group reads the last stage's input": ("stages[a].in_bytes", "stages[b].in_bytes"),
        "group writes the first stage's output": ("x * y * t * stages[b].out_bytes", "x * y * t * stages[a].out_bytes"),
        "on-chip rows one-sided": ("(2 * s.ry + 1) * s.in_bytes", "(s.ry + 1) * s.in_bytes"),
        "feasible if any group fits": ("return all(group_onchip(stages, a, b, box) <= onchip_limit",
                                       "return any(group_onchip(stages, a, b, box) <= onchip_limit"),
        "utilisation temporal halo two-sided": ("* (t + rt))", "* (t + 2 * rt))"),
        "on-chip temporal halo two-sided": ("return (x + 2 * Rx) * (t + Rt) * sum", "return (x + 2 * Rx) * (t + 2 * Rt) * sum"),
        "candidate groups repeat one and miss singletons": (
            "[(a, b) for a in range(n) for b in range(a, n)]",
            "[(a, b) for a in range(n) for b in range(a + 1, n)] + [(n - 1, n - 1)] * n"),
        "boxes ignore t": ("boxes = N * M * T / (x * y * t)", "boxes = N * M * T / (x * y)"),
        "Eq. 6 without its factor 2": ("x = (2.0 * beta * dx / dt) ** (1.0 / 3.0)",
                                       "x = (beta * dx / dt) ** (1.0 / 3.0)"),
        "brute force keeps the worst": ("if best is None or c < best[1]:", "if best is None or c > best[1]:"),
        "Sobel writes one map": ('Stage("sobel", 1, 1, 0, 1 * e, 2 * e)', 'Stage("sobel", 1, 1, 0, 1 * e, 1 * e)'),
    }),
    "dag": (["test_dag_oracle:od"], {
        "binomial weights unnormalised": ("/ 4.0 ** r", "/ 2.0 ** r"),
        "binomial row shifted": ("comb(2 * r, r + k)", "comb(2 * r, k + 1)"),
        "affine bias scaled": ("return a * a_in + b", "return a * (a_in + b)"),
        "product squares its first input": ("np.clip(a_in * b_in, -16.0, 16.0)", "np.clip(a_in * a_in, -16.0, 16.0)"),
        "stencil not separable": ("out += w[iy] * w[ix] * _shift(a_in, dy, dx)",
                                  "out += w[iy] * w[iy] * _shift(a_in, dy, dx)"),
        "max over the diagonal only": ("out = np.maximum(out, _shift(a_in, dy, dx))",
                                       "out = np.maximum(out, _shift(a_in, dy, dy))"),
        "frames wrap instead of clamping": ("xs = np.clip(np.arange(W) + dx, 0, W - 1)", "xs = (np.arange(W) + dx) % W"),
        "max starts at zero": ("out = np.full_like(a_in, -np.inf)", "out = np.zeros_like(a_in)"),
        "abs is the identity": ("return np.abs(a_in)", "return a_in"),
        "product saturates below only": ("np.clip(a_in * b_in, -16.0, 16.0)", "np.clip(a_in * b_in, -16.0, None)"),
        "node 0 divides by 256": ("frame_u8.astype(np.float64) / 255.0", "frame_u8.astype(np.float64) / 256.0"),
        "second input read from the first": ("nodes[i2] if i2 >= 0 else None", "nodes[i1] if i2 >= 0 else None"),
        "bound: node 0 rounded once": ("err = [2.0 * U32 * np.abs(nodes[0]) * grow]", "err = [U32 * np.abs(nodes[0]) * grow]"),
        "bound: affine ignores its input error": ("bound = abs(a) * e + U32 * (2.0 * abs(a) * x + abs(b) + y)",
                                                  "bound = U32 * (2.0 * abs(a) * x + abs(b) + y)"),
        "bound: product drops a cross term": ("exact = x * e2 + x2 * e + e * e2", "exact = x * e2 + e * e2"),
        "bound: stencil rounding of one pass": ("bound = _stencil_abs(e, r) + 2 * (2 * r + 1) * U32",
                                                "bound = _stencil_abs(e, r) + (2 * r + 1) * U32"),
        "bound: max3 keeps the centre only": ("bound = np.maximum(bound, _shift(e, dy, dx))",
                                              "bound = np.maximum(bound, _shift(e, 0, 0))"),
        "bound: abs drops the error": ("bound = e.copy()", "bound = 0.0 * e"),
    }),
    "mlp": (["test_mlp_oracle:mlp"], {
        "ReLU gate dropped in layer 2": ("dz2 = np.outer(dy, w3) * (z2 > 0)", "dz2 = np.outer(dy, w3)"),
        "back-propagation through W2 transposed": ("dz1 = (dz2 @ W2) * (z1 > 0)", "dz1 = (dz2 @ W2.T) * (z1 > 0)"),
        "loss derivative without its 2": ("dy = 2.0 * (y - t) / n", "dy = (y - t) / n"),
        "output bias gradient averaged": ("g_b3 = dy.sum()", "g_b3 = dy.mean()"),
        "W2 gradient from pre-activations": ("g_W2 = dz2.T @ h1", "g_W2 = dz2.T @ z1"),
        "first bias gradient averaged": ("g_b1 = dz1.sum(0)", "g_b1 = dz1.mean(0)"),
        "W2 unpacked transposed": ("W2 = p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH); o += WIDTH * WIDTH",
                                   "W2 = p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH).T; o += WIDTH * WIDTH"),
        "loss summed, not averaged": ("return float(np.mean((forward(p, x) - t) ** 2))",
                                      "return float(np.sum((forward(p, x) - t) ** 2))"),
        "forward subtracts the first bias": ("h1 = np.maximum(x @ W1.T + b1, 0.0)", "h1 = np.maximum(x @ W1.T - b1, 0.0)"),
    }),
    "dag_plan": (["test_dag_plan_oracle:odp"], {
        "3x3 max has no radius": ("return r if kind == 4 else (1 if kind == 5 else 0)", "return r if kind == 4 else 0"),
        "product's second input dropped": ("return [i1, i2] if kind == 3 and i2 != i1 else [i1]", "return [i1]"),
        "stored when read by the range's last stage": ("if c > b:", "if c >= b:"),
        "halo ignores the consumer's radius": ("h = max(h, halo[c] + radius(rows[c - 1]))", "h = max(h, halo[c])"),
        "input halo one-sided": ("(TX + 2 * h) * (TY + 2 * h) * (1 if e == 0 else 4)",
                                 "(TX + h) * (TY + h) * (1 if e == 0 else 4)"),
        "frame read as a float map": ("(1 if e == 0 else 4)", "4"),
        "stored maps as bytes": ("t += TX * TY * 4 * len(outs)", "t += TX * TY * len(outs)"),
        "slot size ignores input halos": ("hmax = max([0] + [halo[j] for j in list(ext) + sorted(live)])",
                                          "hmax = max([0] + [halo[j] for j in sorted(live)])"),
        "inputs read without their consumer's radius": ("ext[i] = max(ext.get(i, -1), halo[j] + radius(rows[j - 1]))",
                                                        "ext[i] = max(ext.get(i, -1), halo[j])"),
        "inlined inputs of inlined nodes dropped": ("                stack.append(i)\n", "                pass\n"),
        "slots never freed": ("if last.get(i) == j and i in slots:", "if False:"),
        "slots without halo": ("return taken * (TX + 2 * hmax) * (TY + 2 * hmax) * 4", "return taken * TX * TY * 4"),
        "brute force keeps the worst": ("if best is None or c < best[0] - 1e-9:", "if best is None or c > best[0] + 1e-9:"),
        "range cut bit off by one": ("if b == n or (cuts >> (b - 1)) & 1:", "if b == n or (cuts >> b) & 1:"),
    }),
}


def _module_from(modname: str, text: str):
    """Execute oracle source `text` as a fresh module (relative imports resolve in the
    oracle package); registered only while it runs, so nothing else sees it."""
    import sys
    import types
    name = f"oracle._planted_{modname}"
    m = types.ModuleType(name)
    m.__package__ = "oracle"
    sys.modules[name] = m
    try:
        exec(compile(text, f"<planted oracle/{modname}.py>", "exec"), m.__dict__)
    finally:
        del sys.modules[name]
    return m


def _py_failing_pin(monkeypatch, modname, module):
    import importlib
    import warnings
    binds, _ = PY_MUTANTS[modname]
    pin_mods = []
    for b in binds:
        mod_name, alias = b.split(":")
        pm = importlib.import_module(f"tests.{mod_name}")
        monkeypatch.setattr(pm, alias, module)
        pin_mods.append(pm)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")  # a planted mistake may overflow on its way to failing
        for pm in pin_mods:
            for name, f, kw in _pin_calls(pm):
                try:
                    f(**kw)
                except Exception as e:
                    return f"{pm.__name__}.{name}{kw or ''}: {type(e).__name__}"
    return None


def _py_source(modname):
    import importlib
    return open(importlib.import_module(f"oracle.{modname}").__file__).read()


@pytest.mark.parametrize("modname", list(PY_MUTANTS))
def test_unchanged_python_oracle_passes_every_pin(monkeypatch, modname):
    assert _py_failing_pin(monkeypatch, modname, _module_from(modname, _py_source(modname))) is None


@pytest.mark.parametrize("modname,name", [(m, n) for m, (_, ms) in PY_MUTANTS.items() for n in ms])
def test_every_planted_mistake_in_a_python_oracle_fails_a_pin(monkeypatch, modname, name):
    src = _py_source(modname)
    old, new = PY_MUTANTS[modname][1][name]
    assert src.count(old) == 1, f"{modname} / {name}: the planted text must occur exactly once"
    got = _py_failing_pin(monkeypatch, modname, _module_from(modname, src.replace(old, new)))
    assert got is not None, f"no pin catches: {modname} / {name}"
