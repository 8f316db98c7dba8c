"""Direct tests of the device arithmetic helpers (rmhd_eval_math) against IEEE
arithmetic: the refined approximate FP64 reciprocal, reciprocal square root
and one-Newton-step quotient that replace IEEE divisions and square roots in
the kernels, and the integer-pipe FP64 <-> FP32 conversions of the mixed form
and the stage solves. References are computed in numpy's long double (80-bit
extended on x86, IEEE quad on Arm), so they are far more accurate than the
bounds checked.

Bounds: the series refinements leave an O(e^3) ~ 2^-57 truncation, with the
approximation's e <= 2^-19, plus the last FMA's rounding, so s_rcp and
s_rsqrt are within 2^-52 relative (about one ulp) on their domains; s_div1
keeps an O(e^2) ~ 2^-38 term (checked against 2^-36); f32_of rounds to
nearest with ties away from zero and f64_of is exact."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RCP, RSQRT, DIV1, F32, F64 = 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def ev():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1808_09721_gb300 import _lib
    from paper_1808_09721_gb300 import build as B
    B.build()
    lib = _lib.load()

    def run(which, x, a=None):
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
        ad = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda() if a is not None else None
        out = torch.full_like(xd, float("nan"))
        st = torch.cuda.current_stream()
        rc = lib.rmhd_eval_math(which, xd.numel(), C.c_void_p(xd.data_ptr()),
                                C.c_void_p(ad.data_ptr() if ad is not None else 0), C.c_void_p(out.data_ptr()),
                                C.c_void_p(st.cuda_stream))
        assert rc == 0
        st.synchronize()
        return out.cpu().numpy()
    return run


def _wide(rng, n, lo=-300.0, hi=300.0, signed=True):
    """n values 10^U(lo, hi) with random mantissas (and signs)."""
    x = 10.0 ** rng.uniform(lo, hi, n) * rng.uniform(1.0, 2.0, n)
    if signed:
        x *= rng.choice([-1.0, 1.0], n)
    return x


def _rel(got, ref):
    g, r = got.astype(np.longdouble), ref
    return np.abs(g - r) / np.abs(r)


def test_rcp_and_rsqrt_to_one_ulp(ev):
    rng = np.random.default_rng(1)
    x = np.concatenate([_wide(rng, 1_000_000),
                        # next to the smallest normal (inputs) and to 2^1021 (results near it)
                        2.0 ** rng.uniform(-1022, -1000, 20000), 2.0 ** rng.uniform(1000, 1021, 20000),
                        [1.0, -1.0, 2.0 ** -1022, 2.0 ** 1021, 3.0, 0.1]])
    ref = np.longdouble(1) / x.astype(np.longdouble)
    err = _rel(ev(RCP, x), ref)
    assert np.max(err) <= 2.0 ** -52, float(np.max(err))
    assert np.mean(err) <= 2.0 ** -53
    xp = np.abs(np.concatenate([_wide(rng, 1_000_000, signed=False), 2.0 ** rng.uniform(-1022, -1000, 20000),
                                2.0 ** rng.uniform(1000, 1023.9, 20000), [1.0, 4.0, 2.0 ** -1022, 0.3]]))
    ref = np.longdouble(1) / np.sqrt(xp.astype(np.longdouble))
    err = _rel(ev(RSQRT, xp), ref)
    assert np.max(err) <= 2.0 ** -52, float(np.max(err))
    assert np.mean(err) <= 2.0 ** -53


def test_div1_within_its_newton_bound(ev):
    rng = np.random.default_rng(2)
    x = _wide(rng, 1_000_000, -150.0, 150.0)
    a = _wide(rng, 1_000_000, -150.0, 150.0)
    ref = a.astype(np.longdouble) / x.astype(np.longdouble)
    err = _rel(ev(DIV1, x, a), ref)
    assert np.max(err) <= 2.0 ** -36, float(np.max(err))
    # the WENO3 weights' use: A / (A + 2 B) with A, B > 0 lies in (0, 1]
    A, Bv = _wide(rng, 200_000, -20, 20, False), _wide(rng, 200_000, -20, 20, False)
    w = ev(DIV1, A + 2.0 * Bv, A)
    ref = A.astype(np.longdouble) / (A + 2.0 * Bv).astype(np.longdouble)
    assert np.max(_rel(w, ref)) <= 2.0 ** -36


def test_integer_pipe_conversions(ev):
    rng = np.random.default_rng(3)
    # FP32 range, subnormals and overflow; random doubles are never exact ties
    x = np.concatenate([_wide(rng, 500_000, -37.0, 38.0), _wide(rng, 100_000, -45.5, -37.9),
                        _wide(rng, 1000, 38.6, 300.0), [0.0, -0.0, 1.0, -2.5]])
    got = ev(F32, x)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)
    # exact ties (a float plus half an ulp) round away from zero
    f = rng.uniform(1.0, 1.99, 1000).astype(np.float32).astype(np.float64) * rng.choice([-1.0, 1.0], 1000)
    half = 2.0 ** -24  # half an FP32 ulp in [1, 2)
    tie = f + np.sign(f) * half
    got = ev(F32, tie)
    away = (np.abs(f) + 2 * half) * np.sign(f)
    bits_ok = (np.abs(f) + 2 * half).astype(np.float32).astype(np.float64) == np.abs(f) + 2 * half
    assert np.all(bits_ok) and np.array_equal(got, away)
    # NaN and infinities give a signed infinity
    got = ev(F32, np.array([np.inf, -np.inf, np.nan]))
    assert got[0] == np.inf and got[1] == -np.inf and np.isinf(got[2])
    # FP32 -> FP64 is exact: normals, subnormals, zeros, infinities, NaN
    f32 = np.concatenate([rng.standard_normal(100_000).astype(np.float32) * np.float32(1e20),
                          (rng.integers(1, 2 ** 23, 10_000).astype(np.uint32)).view(np.float32),
                          np.array([0.0, -0.0, np.inf, -np.inf], dtype=np.float32)])
    got = ev(F64, f32.astype(np.float64))
    assert np.array_equal(got, f32.astype(np.float64))
    assert np.isnan(ev(F64, np.array([np.nan]))[0])
