"""The float32 voxel-mean helper of the map build (a voxel's mean and
covariance are the binary64 mean of its points' values rounded to float32,
Sec. III-A) against exact rational arithmetic.

The helper is compiled for the host from the same header the kernel includes;
every operation in it is an explicitly rounded float32 operation, so the host
build behaves like the device code.  For each (hi, lo, n) with hi = RN32(hi + lo)
it either reports "not certified" (the kernel then evaluates the binary64
definition) or returns RN32(RN64(RN64(hi + lo) / n)) exactly.  Cases include
quotients placed within a few float64 ulps of float32 midpoints, binade edges,
exact quotients, negative sums and the guarded magnitude range."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "mean_rn32_harness.cpp")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("mean") / "mean_rn32")
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17", SRC, "-o", exe], check=True)

    def run(cases):
        inp = "".join(f"{h:08x} {l:08x} {n}\n" for h, l, n in cases)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [(int(a), int(b, 16)) for a, b in (ln.split() for ln in out.splitlines())]
    return run


def f32(bits):
    return float(np.uint32(bits).view(np.float32))


def bits32(x):
    return int(np.float32(x).view(np.uint32))


def truth(hb, lb, n):
    """RN32(RN64(RN64(hi + lo) / n)), the binary64 definition."""
    s = float(Fraction(f32(hb)) + Fraction(f32(lb)))   # RN64 of the exact sum
    q = float(Fraction(s) / n)                          # RN64 of the quotient
    return bits32(q)                                    # RN32 (ties to even)


def df_pair(S):
    """hi = RN32(S), lo = RN32(S - hi): a double-float pair with |lo| <= ulp(hi)/2."""
    hi = np.float32(float(S))
    lo = np.float32(float(S - Fraction(float(hi))))
    return bits32(hi), bits32(lo)


def gen_cases(rng, count):
    cases = []
    for _ in range(count):
        kind = rng.integers(0, 5)
        n = int(rng.choice([1, 2, 3, 5, 7, 10, 64, 1000, 65537, 1 << 24,
                            int(rng.integers(1, 50))]))
        if kind == 0:       # random sum of n float32 values near a common scale
            scale = 2.0 ** rng.integers(-40, 40)
            vals = (rng.normal(size=min(n, 50)) * scale).astype(np.float32)
            S = sum(Fraction(float(v)) for v in vals)
            cases.append((*df_pair(S), n))
        elif kind == 1:     # quotient near a float32 midpoint: S = (mid + tiny) n
            q = np.float32(rng.uniform(0.5, 2.0) * 2.0 ** rng.integers(-30, 30))
            qb = bits32(q)
            mid = (Fraction(float(q)) + Fraction(f32(qb + 1))) / 2
            tiny = Fraction(int(rng.integers(-8, 9)), 1) * mid * Fraction(1, 1 << 53)
            cases.append((*df_pair((mid + tiny) * n), n))
        elif kind == 2:     # exact quotient or binade edge
            q = np.float32(2.0 ** rng.integers(-30, 30))
            if rng.random() < 0.5:
                q = np.float32(f32(bits32(q) + int(rng.integers(-2, 3))))
            cases.append((*df_pair(Fraction(float(q)) * n), n))
        elif kind == 3:     # arbitrary hi with a random lo in [-ulp/2, ulp/2]
            hi = np.float32(rng.normal() * 2.0 ** rng.integers(-50, 50))
            ulp = Fraction(float(np.spacing(np.float32(abs(hi)))))
            lo_f = Fraction(int(rng.integers(-(1 << 20), 1 << 20)), 1 << 21) * ulp
            S = Fraction(float(hi)) + lo_f
            cases.append((*df_pair(S), n))
        else:               # lower binade neighbour of a power of two
            q = np.float32(2.0 ** rng.integers(-20, 20))
            below = f32(bits32(q) - 1)
            mid = (Fraction(float(q)) + Fraction(below)) / 2
            off = Fraction(int(rng.integers(-3, 4)), 1 << 60) * mid
            cases.append((*df_pair((mid + off) * n), n))
    return cases


def test_mean_rn32_matches_binary64_definition(harness):
    rng = np.random.default_rng(20220201)
    cases = gen_cases(rng, 6000)
    cases += [(bits32(0.0), bits32(0.0), 3), (bits32(-1.5), 0, 1), (bits32(3.0), 0, 3),
              (bits32(1e-30), 0, 7), (bits32(-2.0 ** 99), 0, 5)]
    got = harness(cases)
    certified = 0
    for (hb, lb, n), (ok, qb) in zip(cases, got):
        if ok:
            certified += 1
            assert qb == truth(hb, lb, n), (hex(hb), hex(lb), n, hex(qb), hex(truth(hb, lb, n)))
    # exact midpoints are decided too: only quotients within 2^-50 of a midpoint
    # without being on it are left to binary64
    assert certified >= 0.95 * len(cases)


def test_mean_rn32_certifies_typical_values(harness):
    """Ordinary coordinates and covariances are certified without fallback."""
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(3000):
        n = int(rng.integers(1, 40))
        vals = rng.uniform(-60, 60, size=n).astype(np.float32)
        cases.append((*df_pair(sum(Fraction(float(v)) for v in vals)), n))
    got = harness(cases)
    assert all(ok for ok, _ in got)
    for (hb, lb, n), (ok, qb) in zip(cases, got):
        assert qb == truth(hb, lb, n)


def test_mean_rn32_refuses_outside_guarded_range(harness):
    cases = [(bits32(2.0 ** -70), 0, 3), (bits32(2.0 ** 110), 0, 3), (bits32(1.0), 0, (1 << 24) + 1),
             (bits32(float("inf")), 0, 2), (bits32(float("nan")), 0, 2), (bits32(1.0), 0, 0)]
    assert all(ok == 0 for ok, _ in harness(cases))
