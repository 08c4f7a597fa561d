"""Planted mistakes in the oracle: a copy of oracle/rs_oracle.c with one
plausible slip (a dropped term, a wrong sign, a swapped index, a transposed
operand) must fail at least one of the oracle's pin tests, and the unchanged
copy must pass them.  Copies, builds and pin runs live in a temporary
directory; the oracle itself is never modified."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "test_oracle_pins.py"
CONV = "test_oracle_conv_pins.py"
CODEC = "test_oracle_codec_pins.py"

# (name, pin file that must catch it, text of the oracle, planted text
#  [, oracle file: rs_oracle.c unless given])
MUTANTS = [
    # ray lattice, Eq. 1, binning, Eq. 4
    ("ray at the cell corner", PINS,
     "double x1 = g->c1 - g->h1 + ((double)i + 0.5) * d1;",
     "double x1 = g->c1 - g->h1 + (double)i * d1;"),
    ("ray spacing of the other axis", PINS,
     "double x2 = g->c2 - g->h2 + ((double)j + 0.5) * d2;",
     "double x2 = g->c2 - g->h2 + ((double)j + 0.5) * d1;"),
    ("shear sign on x1", PINS,
     "double y1 = (1.0 - mc->gamma) * x1 - mc->kappa_s * x1 - a1;",
     "double y1 = (1.0 + mc->gamma) * x1 - mc->kappa_s * x1 - a1;"),
    ("smooth matter dropped on x2", PINS,
     "double y2 = (1.0 + mc->gamma) * x2 - mc->kappa_s * x2 - a2;",
     "double y2 = (1.0 + mc->gamma) * x2 - a2;"),
    ("deflection added instead of subtracted", PINS,
     "double y2 = (1.0 + mc->gamma) * x2 - mc->kappa_s * x2 - a2;",
     "double y2 = (1.0 + mc->gamma) * x2 - mc->kappa_s * x2 + a2;"),
    ("deflection sign of one lens sum", PINS,
     "s1 += lm[k] * d1 / r2;", "s1 -= lm[k] * d1 / r2;"),
    ("mass dropped from the x2 term", PINS,
     "s2 += lm[k] * d2 / r2;", "s2 += d2 / r2;"),
    ("r^2 with a transposed operand", PINS,
     "double r2 = d1 * d1 + d2 * d2;", "double r2 = d1 * d1 + d2 * d1;"),
    ("singular ray skipped instead of counted", PINS,
     "        if (r2 == 0.0)\n            return 1;",
     "        if (r2 == 0.0)\n            continue;"),
    ("pixel row from the x1 coordinate", PINS,
     "*qo = (int64_t)floor(v);", "*qo = (int64_t)floor(u);"),
    ("map corner at the centre", PINS,
     "double u = (y1 - (mp->c1 - mp->width / 2.0)) / w;",
     "double u = (y1 - mp->c1) / w;"),
    ("closed top edge of the map", PINS,
     "u < (double)mp->npix && v < (double)mp->npix",
     "u <= (double)mp->npix && v < (double)mp->npix"),
    ("N_avg with one spacing twice", PINS,
     "return (w / d1) * (w / d2);", "return (w / d1) * (w / d1);"),
    ("N_avg inverted", PINS,
     "return (w / d1) * (w / d2);", "return (d1 / w) * (d2 / w);"),
    # lens field (Eq. 3, disk, Salpeter masses, generator)
    ("Eq. 3 without pi in the denominator", PINS,
     "double n = kappa_star * area / (pi * mean_mass);",
     "double n = kappa_star * area / mean_mass;"),
    ("disk radius not square-rooted", PINS,
     "double r = radius * sqrt(u_r);", "double r = radius * u_r;"),
    ("Salpeter exponent sign", PINS,
     "double e = 1.0 - slope;", "double e = slope - 1.0;"),
    ("masses not mean-normalised", PINS,
     "            m[k] = m[k] / mean;", "            m[k] = m[k];"),
    ("SplitMix64 last shift", PINS,
     "return z ^ (z >> 31);", "return z ^ (z >> 30);"),
    # MPD and probability sums
    ("counts above the last bin dropped", PINS,
     "        if (c > n_bins - 1)\n            c = n_bins - 1;",
     "        if (c > n_bins - 1)\n            continue;"),
    ("probability sum counts its threshold", PINS,
     "if ((double)c < thr)", "if ((double)c <= thr)"),
    # finite source (Eq. 6) and pixelFlux
    ("convolution kernel not flipped", CONV,
     "s += k[(a + h) * d + (b + h)] * m[wrap(q - a, n) * n + wrap(p - b, n)];",
     "s += k[(a + h) * d + (b + h)] * m[wrap(q + a, n) * n + wrap(p - b, n)];"),
    ("convolution wraps to the wrong axis", CONV,
     "s += k[(a + h) * d + (b + h)] * m[wrap(q - a, n) * n + wrap(p - b, n)];",
     "s += k[(a + h) * d + (b + h)] * m[wrap(q - b, n) * n + wrap(p - a, n)];"),
    ("pixelFlux x and y from one draw", CONV,
     "uint64_t hy = orc_splitmix64(seed, 2u * (uint64_t)t + 1u) >> 32;",
     "uint64_t hy = orc_splitmix64(seed, 2u * (uint64_t)t) >> 32;"),
    ("value histogram with open edges", CONV,
     "while (b < n_edges && edges[b] <= v[t])", "while (b < n_edges && edges[b] < v[t])"),
    ("Gaussian sigma of the wrong axis", CONV,
     "(y2 * y2) / (2.0 * p->sigma2 * p->sigma2)", "(y2 * y2) / (2.0 * p->sigma1 * p->sigma1)"),
    ("Gaussian without its factor 2", CONV,
     "exp(-(y1 * y1) / (2.0 * p->sigma1 * p->sigma1)", "exp(-(y1 * y1) / (p->sigma1 * p->sigma1)"),
    ("power law with the wrong sign", CONV,
     "return pow(r / p->r_scale, -p->index);", "return pow(r / p->r_scale, p->index);"),
    ("thin disc exponent", CONV,
     "double xi = pow(r / p->r_scale, 0.75)", "double xi = pow(r / p->r_scale, 0.5)"),
    ("central hole ignored", CONV,
     "if (!(q >= in2 && q < out2))", "if (!(q < out2))"),
    ("profile samples at cell corners", CONV,
     "sum += brightness(p, 2 * (b * S + s) + 1 - S, 2 * (a * S + t) + 1 - S,",
     "sum += brightness(p, 2 * (b * S + s) - S, 2 * (a * S + t) - S,"),
    ("kernel not normalised", CONV,
     "        k[t] = k[t] / total;", "        k[t] = k[t];"),
    ("point source by radius instead of diameter", CONV,
     "if (2.0 * p->r_out <= w)", "if (p->r_out <= w)"),
    # indexed maps (App. B)
    ("index bits one short", CODEC,
     "while (b < 32 && ((int64_t)1 << b) < distinct)",
     "while (b < 32 && ((int64_t)1 << b) < distinct - 1)"),
    ("packing MSB first", CODEC,
     "words[bit / 32] |= (uint32_t)1 << (bit % 32);",
     "words[bit / 32] |= (uint32_t)1 << (31 - bit % 32);"),
    ("table keeps duplicates", CODEC,
     "if (d == 0 || table[t] != table[d - 1])", "if (1)"),
    # previews and the colorbar (Sec. 3.2.1, Sec. 4.6)
    ("preview samples the pixel corner", CODEC,
     "int64_t q = (2 * r + 1) * n / (2 * s);", "int64_t q = r * n / s;"),
    ("gray level excludes its threshold", CODEC,
     "while (g < 255 && thr[g] <= v)", "while (g < 255 && thr[g] < v)"),
    ("colorbar interpolation truncated", CODEC,
     "+ cb * (i - pa) + (pb - pa) / 2) / (pb - pa));", "+ cb * (i - pa)) / (pb - pa));"),
    ("colorbar stops swapped", CODEC,
     "lut[3 * i + c] = (uint8_t)((ca * (pb - i) + cb * (i - pa)",
     "lut[3 * i + c] = (uint8_t)((cb * (pb - i) + ca * (i - pa)"),
    ("recoloured pixels transparent", CODEC,
     "rgba[4 * t + 3] = 255;", "rgba[4 * t + 3] = 0;"),
    # the Python side of the oracle (argument structs, closed forms, Eq. 6 by FFT)
    ("ray-grid half widths swapped", PINS,
     "g = Grid(job.c1, job.c2, job.half1, job.half2, job.n1, job.n2)",
     "g = Grid(job.c1, job.c2, job.half2, job.half1, job.n1, job.n2)", "__init__.py"),
    ("map centre coordinates swapped", PINS,
     "mp = Map(job.mc1, job.mc2, job.width, job.npix)",
     "mp = Map(job.mc2, job.mc1, job.width, job.npix)", "__init__.py"),
    ("macro magnification with the shear added", PINS,
     "return 1.0 / ((1.0 - kappa) ** 2 - gamma ** 2)",
     "return 1.0 / ((1.0 - kappa) ** 2 + gamma ** 2)", "__init__.py"),
    ("MPD normalised by the ray count", PINS,
     "return count_histogram(counts, n_bins) / float(np.asarray(counts).size)",
     "return count_histogram(counts, n_bins) / float(np.asarray(counts).sum())", "__init__.py"),
    ("FFT kernel image transposed", CONV,
     "img[a % n, b % n] += k[a + h, b + h]", "img[a % n, b % n] += k[b + h, a + h]",
     "__init__.py"),
    ("Eq. 3 arguments swapped", PINS,
     "lens_count(job.kappa_star, job.lens_radius)", "lens_count(job.lens_radius, job.kappa_star)",
     "__init__.py"),
]


def _slug(name: str) -> str:
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")


def _run(base: str, name: str, pins: str, old: str | None, new: str | None,
         target: str = "rs_oracle.c"):
    d = os.path.join(base, _slug(name))
    ign = shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "workloads"), os.path.join(d, "workloads"), ignore=ign)
    os.makedirs(os.path.join(d, "tests"))
    for f in ("__init__.py", "conftest.py", pins):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    if old is not None:
        path = os.path.join(d, "oracle", target)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) >= 1, f"{name}: text not found in the oracle"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new, 1))
        # a planted mistake must still compile: a build error is not a catch
        if target.endswith(".c"):
            cc = subprocess.run([os.environ.get("CC", "gcc"), "-fsyntax-only", "-fopenmp",
                                 "-std=c11", path], capture_output=True, text=True)
            assert cc.returncode == 0, f"{name}: the mutant does not compile\n{cc.stderr}"
        else:
            compile(src.replace(old, new, 1), path, "exec")
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", f"tests/{pins}", "-x", "-q"], cwd=d,
                       env=env, capture_output=True, text=True, timeout=900)
    return name, r


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    jobs = [("control " + p, p, None, None) for p in (PINS, CONV, CODEC)] + MUTANTS
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda m: _run(str(tmp_path), *m), jobs))
    controls = [(n, r) for n, r in results if n.startswith("control ")]
    for n, r in controls:
        assert r.returncode == 0, f"{n}: the unchanged oracle fails its pins\n{r.stdout[-2000:]}"
    # caught: a pin fails (or the mutant crashes its test process)
    survivors = [n for n, r in results if not n.startswith("control ") and r.returncode == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
