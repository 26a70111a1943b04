"""The arithmetic of the split FP64 scatter, checked on the CPU with NumPy:
the plan's choices (digit width b with K 2^(2b) <= 2^24, 50 bits per
operand, pair groups within 2^24, a Horner tail below 2^-26 of the leading
term), the balanced integer digits, exact FP32 sums of the slice products,
and the FP64 result against the FP64 product.  The same rules are what the
library's host planner and kernels implement for the tensor cores (Ozaki,
Ogita, Oishi and Rump 2012, error-free splitting); here an FP32 matrix
product stands in for the tensor-core MMAs with FP32 accumulation.  The
last test compiles the library's planner (csrc/split_plan.hpp) and checks
that it produces exactly the plan checked here."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def plan(K):
    """(bits, nsl, passes): passes = [(d, [(i, j, beta), ...]), ...]."""
    lim = 2.0 ** 24
    b = 7
    while b > 0 and K * 2.0 ** (2 * b) > lim:
        b -= 1
    nsl = -(-50 // b)
    dt = min(nsl, -(-26 // b))

    def D(i):
        return 2.0 ** (b if i == 0 else b - 1)

    passes = []
    for d in range(dt):
        cur, acc = [], 0.0
        for i in range(d + 1):
            bound = K * D(i) * D(d - i)
            if cur and acc + bound > lim:
                passes.append((d, cur))
                cur, acc = [], 0.0
            cur.append((i, d - i, 0.0 if not cur else 1.0))
            acc += bound
        passes.append((d, cur))
    tail = []
    for d in range(nsl - 1, dt - 1, -1):
        for i in range(d + 1):
            tail.append((i, d - i, 0.0 if not tail else (2.0 ** -b if i == 0 else 1.0)))
    if tail:
        passes.append((dt, tail))
    return b, nsl, passes


def split_rows(Z, bits, nsl):
    """Row scales mu (powers of two above max |row|) and integer digits
    [nsl][rows][K] with Z ~= mu sum_i d_i 2^(-bits (i+1))."""
    m = np.abs(Z).max(axis=1)
    e = np.where(m > 0, np.frexp(m)[1], 0)
    mu = np.ldexp(1.0, e)
    T = np.rint(np.ldexp(Z, (bits * nsl - e)[:, None])).astype(np.int64)
    half, mask = 1 << (bits - 1), (1 << bits) - 1
    digits = np.zeros((nsl,) + Z.shape, dtype=np.int64)
    for i in range(nsl - 1, 0, -1):
        r = ((T + half) & mask) - half
        digits[i] = r
        T = (T - r) >> bits
    digits[0] = T
    return mu, digits


def split_product(A, Bt):
    """A @ Bt.T to FP64 accuracy from FP32 products of integer digit slices."""
    K = A.shape[1]
    b, nsl, passes = plan(K)
    mu, da = split_rows(A, b, nsl)
    nu, db = split_rows(Bt, b, nsl)
    y = np.zeros((A.shape[0], Bt.shape[0]))
    for d, gemms in passes:
        P = np.zeros_like(y, dtype=np.float32)
        for i, j, beta in gemms:
            prod = da[i].astype(np.float32) @ db[j].astype(np.float32).T
            P = prod + np.float32(beta) * P
        y += np.ldexp(1.0, -b * (d + 2)) * mu[:, None] * nu[None, :] * P.astype(np.float64)
    return y


@pytest.mark.parametrize("K", [96, 384, 1536, 6144])
def test_plan_bounds(K):
    b, nsl, passes = plan(K)
    assert K * 2.0 ** (2 * b) <= 2.0 ** 24 and (b == 7 or K * 2.0 ** (2 * b + 2) > 2.0 ** 24)
    assert b * nsl >= 50
    pairs = sorted((i, j) for _, g in passes for i, j, _ in g)
    assert pairs == sorted((i, d - i) for d in range(nsl) for i in range(d + 1))
    D = lambda i: 2.0 ** (b if i == 0 else b - 1)
    dt = min(nsl, -(-26 // b))
    for d, g in passes:
        if d < dt and all(i + j == d for i, j, _ in g):
            assert sum(K * D(i) * D(j) for i, j, _ in g) <= 2.0 ** 24
    assert b * dt >= 26


def test_digits_are_balanced_and_exact():
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((40, 96)) * np.logspace(-30, 30, 40)[:, None]
    b, nsl, _ = plan(96)
    mu, d = split_rows(Z, b, nsl)
    assert np.abs(d[0]).max() <= 2 ** b and np.abs(d[1:]).max() <= 2 ** (b - 1)
    back = sum(np.ldexp(d[i].astype(np.float64), -b * (i + 1)) for i in range(nsl)) * mu[:, None]
    assert np.abs(back - Z).max(axis=1).max() <= 0.0 + np.max(mu * 2.0 ** (-b * nsl))


@pytest.mark.parametrize("K", [384, 1536, 6144])
def test_slice_products_are_exact_in_fp32(K):
    b, nsl, passes = plan(K)
    # worst-case digits: every entry at its bound, one sign
    da = np.full((nsl, 8, K), 2 ** (b - 1), dtype=np.int64)
    da[0] = 2 ** b
    for d, gemms in passes[:-1]:  # the exact passes (the last one is the Horner tail)
        P = np.zeros((8, 8), dtype=np.float32)
        exact = np.zeros((8, 8), dtype=np.int64)
        for i, j, beta in gemms:
            P = da[i].astype(np.float32) @ da[j].astype(np.float32).T + np.float32(beta) * P
            exact = da[i] @ da[j].T + int(beta) * exact
        assert np.array_equal(P.astype(np.int64), exact)


@pytest.mark.parametrize("K", [96, 1536])
def test_split_product_matches_fp64(K):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((64, K)) * np.logspace(-8, 8, 64)[:, None]
    Bt = rng.standard_normal((48, K))
    y = split_product(A, Bt)
    ref = A @ Bt.T
    err = np.abs(y - ref) / (np.abs(A).max(axis=1)[:, None] * np.abs(Bt).max(axis=1)[None, :] * K)
    assert err.max() < 1e-14
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-13


@pytest.fixture(scope="module")
def library_plan(tmp_path_factory):
    """split_plan of the library (csrc/split_plan.hpp), compiled on the host."""
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("plan") / "libplan.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2010_04559_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "split_plan_shim.cpp"), "-o", out],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.shim_split_plan.restype = ctypes.c_int

    def get(K):
        cap = 512
        I = (ctypes.c_int * cap)
        bits, nsl = ctypes.c_int(), ctypes.c_int()
        d, start, gi, gj = I(), I(), I(), I()
        beta = (ctypes.c_float * cap)()
        n = lib.shim_split_plan(K, ctypes.byref(bits), ctypes.byref(nsl), d, start, gi, gj,
                                beta, cap)
        assert n >= 0
        passes = [(d[p], [(gi[g], gj[g], float(beta[g])) for g in range(start[p], start[p + 1])])
                  for p in range(n)]
        return bits.value, nsl.value, passes
    return get


@pytest.mark.parametrize("K", [64, 96, 384, 1000, 1536, 4096, 6144, 8192, 16384, 65536, 2 ** 21])
def test_the_library_runs_the_plan_checked_here(library_plan, K):
    """The library's plan is, pass for pass and product for product, the plan
    whose bounds and exactness the tests above check (or none where the digit
    width would drop below 2 bits)."""
    b, nsl, passes = library_plan(K)
    if b == 0:
        assert K * 2.0 ** 4 > 2.0 ** 24 and passes == []
        return
    assert (b, nsl, passes) == plan(K)
