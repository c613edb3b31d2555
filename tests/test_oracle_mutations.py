"""The pins in test_oracle.py must fail for plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong sign or index, a transposed operand, a lost
scale) in a temporary copy of oracle/oracle.c, compiles it, and runs the pin suite against that
copy in a subprocess: the suite has to fail.  Nothing here touches a GPU or the real oracle.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "sample scale dropped": ("double scale = sqrt((double)m / (double)s);", "double scale = 1.0;"),
    "philox output word swapped": ("uint64_t y1 = lo1;", "uint64_t y1 = lo0;"),
    "index from low half": ("idx[blk * 4 + q] = (int64_t)hi;", "idx[blk * 4 + q] = (int64_t)(lo % (uint64_t)m);"),
    "householder tau sign": ("tau = (beta - alpha) / beta;", "tau = (alpha - beta) / beta;"),
    "R_s sign normalisation dropped": ("double sgn = (d < 0.0) ? -1.0 : 1.0;", "double sgn = 1.0;"),
    "trsm transposed operand": ("for (int64_t k = 0; k < j; ++k) t -= x[k] * T[k * n + j];",
                                "for (int64_t k = 0; k < j; ++k) t -= x[k] * T[j * n + k];"),
    "gram diagonal dropped": ("for (int64_t q = p; q < n; ++q) P[p * n + q] += xp * x[q];",
                              "for (int64_t q = p + 1; q < n; ++q) P[p * n + q] += xp * x[q];"),
    "cholesky term dropped": ("for (int64_t k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];",
                              "for (int64_t k = 1; k < j; ++k) d -= R[k * n + j] * R[k * n + j];"),
    "triu product term dropped": ("for (int64_t k = i; k <= j; ++k) t += R2[i * n + k] * Rs[k * n + j];",
                                  "for (int64_t k = i; k < j; ++k) t += R2[i * n + k] * Rs[k * n + j];"),
    "second solve uses R_s": ("oracle_trsm_rows(A1, m, n, n, R1, Q, ldq, variant);",
                              "oracle_trsm_rows(A1, m, n, n, Rs, Q, ldq, variant);"),
    "hadamard parity sign flipped": ("(__builtin_popcountll(k & (uint64_t)i) & 1) ? -d[i] : d[i];",
                                     "(__builtin_popcountll(k & (uint64_t)i) & 1) ? d[i] : -d[i];"),
    "rademacher from the low bit": ("(w[q] >> 63) ? -1.0 : 1.0;", "(w[q] & 1) ? -1.0 : 1.0;"),
    "smoothing normalisation dropped": ("const double inv = 1.0 / sqrt((double)mp);", "const double inv = 1.0;"),
    "smoothing order one too large": ("while (p < m) p <<= 1;", "while (p <= m) p <<= 1;"),
    "smoothed sample scale uses m": ("const double scale = sqrt((double)mp / (double)s);",
                                     "const double scale = sqrt((double)m / (double)s);"),
    "dct first-row weight": ("const double w = k == 0 ? sqrt(1.0 / (double)mp) : sqrt(2.0 / (double)mp);",
                             "const double w = sqrt(2.0 / (double)mp);"),
    "scholqr3 shift dropped": ("for (int64_t i = 0; i < n; ++i) G[i * n + i] += sigma;",
                               "for (int64_t i = 0; i < n; ++i) G[i * n + i] += 0.0 * sigma;"),
    "dct half-sample shift dropped": ("const uint64_t r = ((2 * (uint64_t)i + 1) * k) % (4 * (uint64_t)mp);",
                                      "const uint64_t r = ((2 * (uint64_t)i) * k) % (4 * (uint64_t)mp);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique for {name!r}"
    with tempfile.TemporaryDirectory() as tmp:
        mutant_c = os.path.join(tmp, "mutant.c")
        mutant_so = os.path.join(tmp, "libmutant.so")
        open(mutant_c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                        "-o", mutant_so, mutant_c, "-lm"], check=True)
        env = dict(os.environ, RPQ_ORACLE_LIB=mutant_so)
        r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"),
                            os.path.join(ROOT, "tests", "test_oracle_smoothing.py"),
                            "-x", "-q", "-p", "no:cacheprovider", "-k", "not thread_count"],
                           env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"planted mistake {name!r} passed every pin:\n{r.stdout[-2000:]}"
