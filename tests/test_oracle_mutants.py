"""The oracle's pins catch plausible mistakes: each case below plants one mistake (a dropped term,
a wrong sign, index or operand) in a copy of oracle.c, compiles it in a temporary directory, and
runs the pin file that covers that part against it (ORACLE_LIBRARY); the run must fail.  The
oracle itself is never modified."""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

PINS = "test_oracle_pins"
LORB = "test_lorb_oracle"
MATCH = "test_match_oracle"

# (pin file, what, original text, replacement); the first occurrence is replaced
MUTANTS = [
    (PINS, "reflect-101 fold off by one", "if (i >= n) i = p - i;", "if (i >= n) i = p - i - 1;"),
    (PINS, "EXPAND weights transposed", "double wt = (2.0 * W5[dx + 2]) * (2.0 * W5[dy + 2]);",
     "double wt = (2.0 * W5[dx + 2]) * (2.0 * W5[dx + 2]);"),
    (PINS, "REDUCE folds with the wrong size", "int xx = reflect101(2 * k + m, nxf);", "int xx = reflect101(2 * k + m, nyf);"),
    (PINS, "Laplacian sign", "for (int c = 0; c < 3; ++c) lap[c] -= e[c];", "for (int c = 0; c < 3; ++c) lap[c] += e[c];"),
    (PINS, "blend not renormalised", "nn[c] = s > 1e-12 ? nn[c] / s : 0.0;", "nn[c] = s > 1e-12 ? nn[c] : 0.0;"),
    (PINS, "bilinear fractions swapped", "double fx = uc - i0, fy = vc - j0;", "double fx = vc - j0, fy = uc - i0;"),
    (PINS, "weights not normalised", "g[3] = s > 0.0 ? wr / s : 0.0;", "g[3] = s > 0.0 ? wr : 0.0;"),
    (PINS, "feather border distance", "if (c->W - 0.5 - u < m) m = c->W - 0.5 - u;", "if (c->W - 1.0 - u < m) m = c->W - 1.0 - u;"),
    (PINS, "gradient term a31 uses y", "gi[6] += -q * x * iw;", "gi[6] += -q * y * iw;"),
    (PINS, "gain gradient uses the gained value", "gg += 2.0 * r * s[i].B[c];", "gg += 2.0 * r * s[i].I[c];"),
    (PINS, "gradient term a12 uses v", "gi[1] += gu * y * iw;", "gi[1] += gv * y * iw;"),
    (PINS, "cylinder sin/cos swapped", "X = sin(t);\n        Y = (y - c->ccy) / c->cf;\n        Z = cos(t);",
     "X = cos(t);\n        Y = (y - c->ccy) / c->cf;\n        Z = sin(t);"),
    (PINS, "cylinder angle sign", "const double t = (x - c->ccx) / c->cf;", "const double t = (c->ccx - x) / c->cf;"),
    (PINS, "cylinder height not scaled", "Y = (y - c->ccy) / c->cf;", "Y = (y - c->ccy);"),
    (PINS, "seam owner off by one", "if (seam) g[3] = (s == (double)(i + 1)) ? 1.0 : 0.0;",
     "if (seam) g[3] = (s == (double)i) ? 1.0 : 0.0;"),
    (PINS, "seam owner without coverage", "if (wv[i] > 0.0 && wv[i] >= (1.0 - 1e-9) * wmax) owner = i;",
     "if (wv[i] >= (1.0 - 1e-9) * wmax) owner = i;"),
    (PINS, "seam ties to the last camera", "for (int i = 0; i < n && owner < 0; ++i)\n                    if (wv[i] > 0.0",
     "for (int i = n - 1; i >= 0 && owner < 0; --i)\n                    if (wv[i] > 0.0"),
    (PINS, "inverse cofactor sign", "inv[5] = -(a * f - c * d) / det;", "inv[5] = (a * f - c * d) / det;"),
    (PINS, "gain dropped from the sample", "rgb[ch] = c->gain * ((1.0 - fy) * top + fy * bot) / 255.0;",
     "rgb[ch] = ((1.0 - fy) * top + fy * bot) / 255.0;"),
    (PINS, "validity starts at the first pixel centre", "int valid = (u >= -0.5) && (u < c->W - 0.5)",
     "int valid = (u >= 0.0) && (u < c->W - 0.5)"),
    (PINS, "collapse skips the coarsest band", "for (int l = L - 2; l >= 0; --l) {\n#pragma omp parallel for",
     "for (int l = L - 3; l >= 0; --l) {\n#pragma omp parallel for"),
    (PINS, "output not masked by coverage", "int covered = *limg_at(&wsum, x, y) > 0.0;", "int covered = 1;"),
    (PINS, "output not clamped above", "(r[c] > 1.0 ? 1.0 : r[c])", "r[c]"),
    (PINS, "residual includes cameras that do not cover the pixel", "if (j != i && val[j]) r += s[i].I[c] - s[j].I[c];",
     "if (j != i) r += s[i].I[c] - s[j].I[c];"),
    (PINS, "gradient sampler fractions swapped", "double fx = uc - i0, fy = vc - j0;\n    int i1 = i0 + 1 < W ?",
     "double fx = vc - j0, fy = uc - i0;\n    int i1 = i0 + 1 < W ?"),
    (PINS, "gradient term a13 scaled by x", "gi[2] += gu * iw;", "gi[2] += gu * x * iw;"),
    (PINS, "v-derivative weighted by the v fraction",
     "s->dIv[c] = cv ? 0.0 : g * ((1.0 - fx) * (p10 - p00) + fx * (p11 - p01)) / 255.0;",
     "s->dIv[c] = cv ? 0.0 : g * ((1.0 - fy) * (p10 - p00) + fy * (p11 - p01)) / 255.0;"),
    (PINS, "clamped coordinates keep a derivative", "int cu = s->u < 0.0 || s->u > W - 1, cv = s->v < 0.0 || s->v > H - 1;",
     "int cu = 0, cv = 0;"),
    (LORB, "gray weights R/B swapped", "(77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8",
     "(29 * q[0] + 150 * q[1] + 77 * q[2] + 128) >> 8"),
    (LORB, "FAST-8 instead of FAST-9", "if (run_b >= 9 || run_d >= 9) return 1;", "if (run_b >= 8 || run_d >= 8) return 1;"),
    (LORB, "FAST non-strict brighter", "run_b = c > p + t ? run_b + 1 : 0;", "run_b = c >= p + t ? run_b + 1 : 0;"),
    (LORB, "forward difference Ix", "const int ix = (int)gray[q + 1] - (int)gray[q - 1];",
     "const int ix = (int)gray[q + 1] - (int)gray[q];"),
    (LORB, "Harris alpha doubled", "const int64_t r = 25 * (A * B - C * C) - (A + B) * (A + B);",
     "const int64_t r = 25 * (A * B - C * C) - 2 * (A + B) * (A + B);"),
    (LORB, "tensor weight transposed", "const int64_t w = binom5[dx + 2] * binom5[dy + 2];",
     "const int64_t w = binom5[dx + 2] * binom5[dx + 2];"),
    (LORB, "ties to the higher index", "return a->r > b->r || (a->r == b->r && a->idx < b->idx);",
     "return a->r > b->r || (a->r == b->r && a->idx > b->idx);"),
    (LORB, "BRIEF bits MSB-first", "if (s[0] > s[1]) d[b >> 3] |= (uint8_t)(1u << (b & 7));",
     "if (s[0] > s[1]) d[b >> 3] |= (uint8_t)(0x80u >> (b & 7));"),
    (LORB, "BRIEF non-strict", "if (s[0] > s[1]) d[b >> 3]", "if (s[0] >= s[1]) d[b >> 3]"),
    (LORB, "BRIEF smoothing transposed",
     "acc += binom5[dx + 2] * binom5[dy + 2] * gray[(int64_t)(py + dy) * W + px + dx];",
     "acc += binom5[dx + 2] * binom5[dx + 2] * gray[(int64_t)(py + dy) * W + px + dx];"),
    (MATCH, "Hamming by AND", "d += __builtin_popcount((unsigned)(a[k] ^ b[k]));",
     "d += __builtin_popcount((unsigned)(a[k] & b[k]));"),
    (MATCH, "LSH key bits MSB-first in a byte", "key |= (uint32_t)((d[bits[j] >> 3] >> (bits[j] & 7)) & 1u) << j;",
     "key |= (uint32_t)((d[bits[j] >> 3] >> (7 - (bits[j] & 7))) & 1u) << j;"),
    (MATCH, "ratio test inverted", "(long long)ratio_den * d1 < (long long)ratio_num * d2",
     "(long long)ratio_num * d1 < (long long)ratio_den * d2"),
    (MATCH, "probe ORs instead of flipping", "const uint32_t q = p < 0 ? q0 : (q0 ^ (1u << p));",
     "const uint32_t q = p < 0 ? q0 : (q0 | (1u << p));"),
    (MATCH, "max_dist strict", "d1 <= max_dist", "d1 < max_dist"),
    (MATCH, "quality order descending", "for (int j = i; j > 0 && mt[3 * (j - 1) + 2] > mt[3 * j + 2]; --j)",
     "for (int j = i; j > 0 && mt[3 * (j - 1) + 2] < mt[3 * j + 2]; --j)"),
    (MATCH, "DLT sign of the u terms", "m0[6] = -(u * x); m0[7] = -(u * y);", "m0[6] = (u * x); m0[7] = (u * y);"),
    (MATCH, "inlier threshold on image A's scale", "const double tn = inlier_px * sb;", "const double tn = inlier_px * sa;"),
    (MATCH, "schedule increment factor", "const long long num = 800000LL * n * (n - 1) * (n - 2);",
     "const long long num = 800000LL * n * (n - 1) * (n - 3);"),
    (MATCH, "de-normalisation sign", "const double Ta[9] = {sa, 0.0, -(sa * ca[0]),", "const double Ta[9] = {sa, 0.0, (sa * ca[0]),"),
    (MATCH, "normal equations cross term", "M[p][q] = M[p][q] + row0[p] * row0[q] + row1[p] * row1[q];",
     "M[p][q] = M[p][q] + row0[p] * row0[q] + row1[p] * row0[q];"),
    (MATCH, "sampling with replacement", "if (s[i] <= j) ++j;", "if (s[i] < j) ++j;"),
    (MATCH, "newest match not sampled", "idx[0] = n - 1;", "idx[0] = 0;"),
    (MATCH, "pivot threshold", "if (!(fabs(M[p][c]) >= 1e-12)) return 0;", "if (!(fabs(M[p][c]) >= 1e12)) return 0;"),
    (MATCH, "points behind the camera accepted", "const double w = h[6] * x + h[7] * y + 1.0;\n    if (!(w > 0.0)) return 0;",
     "const double w = h[6] * x + h[7] * y + 1.0;\n    if (!(w != 0.0)) return 0;"),
]


def _run_mutant(workdir, threads, pins, what, orig, repl):
    """Compile one mutant into its own directory and run its pin file against it: (exit code, tail
    of the output)."""
    src = open(SRC).read()
    d = tempfile.mkdtemp(dir=workdir)
    bad = os.path.join(d, "oracle_mutant.c")
    with open(bad, "w") as f:
        f.write(src.replace(orig, repl, 1))
    lib = os.path.join(d, "liboracle_mutant.so")
    oracle.compile_library(bad, lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins + ".py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT,
                       env=dict(os.environ, ORACLE_LIBRARY=lib, OMP_NUM_THREADS=str(threads)),
                       capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-1500:]


@pytest.fixture(scope="module")
def mutant_results(request, tmp_path_factory):
    """Runs of the selected mutants, several at a time (each pin run is mostly single-threaded);
    under pytest-xdist each worker runs only the mutant it is asked for."""
    workdir = str(tmp_path_factory.mktemp("mutants"))
    cores = os.cpu_count() or 2
    cache = {}
    if not os.environ.get("PYTEST_XDIST_WORKER"):
        wanted = {item.callspec.params["what"] for item in request.session.items
                  if item.module is request.module and hasattr(item, "callspec")}
        todo = [m for m in MUTANTS if m[1] in wanted and m[2] in open(SRC).read()]
        workers = max(1, min(len(todo), cores // 2))
        with ThreadPoolExecutor(workers) as ex:
            futs = {m[1]: ex.submit(_run_mutant, workdir, max(1, cores // workers), *m) for m in todo}
            cache.update({k: f.result() for k, f in futs.items()})

    def get(m):
        if m[1] not in cache:
            cache[m[1]] = _run_mutant(workdir, cores, *m)
        return cache[m[1]]
    return get


@pytest.mark.parametrize("pins,what,orig,repl", MUTANTS, ids=[m[1] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(mutant_results, pins, what, orig, repl):
    assert orig in open(SRC).read(), f"mutation site not found: {orig}"
    rc, out = mutant_results((pins, what, orig, repl))
    assert rc != 0, f"{what}: the pins in {pins}.py still pass\n{out}"
