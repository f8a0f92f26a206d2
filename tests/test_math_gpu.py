"""The kernels' single-precision function approximations (the library's
pdr_math.cuh and the response kernel's helpers) against FP64, each over its
whole stated input range, through the diagnostic entry point pdr_math_eval.

The Box-Muller pieces see exactly the 2^23 uniforms u = (2k + 1) / 2^24, so
they are checked at every one of them; the deviate itself at every value of
one word with the other word fixed at several values, both ways.  The other
functions are checked on dense grids of their argument ranges.  Each bound is
the one the source states for that function.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import binding, build
    build.build()
    return binding


def _ev(B, name, x, x2=None):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    x2t = None if x2 is None else torch.from_numpy(np.ascontiguousarray(x2)).cuda()
    if x.dtype == np.uint32:
        xt = xt.view(torch.float32)
        x2t = None if x2t is None else x2t.view(torch.float32)
    y = B.math_eval(name, xt, x2t)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


K = np.arange(1 << 23, dtype=np.uint32)
U = (2.0 * K.astype(np.float64) + 1.0) / 2.0**24   # every uniform the generator makes


def test_uniforms(B):
    w = (K << np.uint32(9)) | np.uint32(0x155)
    y = _ev(B, "u01", w)
    assert np.array_equal(y, U)


def test_ln_unit_at_every_uniform(B):
    y = _ev(B, "ln_unit", U.astype(np.float32))
    ref = np.log(U)
    rel = np.abs(y - ref) / np.abs(ref)
    print("ln_unit max rel", rel.max())
    assert rel.max() <= 6e-7


def test_cos_two_pi_at_every_uniform(B):
    y = _ev(B, "cos_two_pi", U.astype(np.float32))
    err = np.abs(y - np.cos(2 * np.pi * U))
    print("cos_two_pi max abs", err.max())
    assert err.max() <= 2.4e-7


@pytest.mark.parametrize("fixed", [0, 1, 0x2AAAAA, 0x400000, 0x7FFFFF])
def test_normal_at_every_word(B, fixed):
    """The deviate for every value of one word, the other at `fixed` (in its
    top 23 bits), both ways round."""
    wf = np.full(K.shape, np.uint32(fixed) << np.uint32(9), np.uint32)
    wk = K << np.uint32(9)
    uf = (2.0 * fixed + 1.0) / 2.0**24
    for wa, wb, ua, ub in ((wk, wf, U, uf), (wf, wk, uf, U)):
        y = _ev(B, "normal", wa, wb)
        ref = np.sqrt(-2.0 * np.log(ua)) * np.cos(2 * np.pi * ub)
        err = np.abs(y - ref)
        print("normal", fixed, "max abs", err.max())
        assert err.max() <= 1e-6


def _grid(lo, hi, n):
    return np.unique(np.linspace(lo, hi, n).astype(np.float32))


def test_asin_on_half_interval(B):
    x = _grid(0.0, 0.5, 1 << 24)
    y = _ev(B, "asin_half", x)
    ref = np.arcsin(x.astype(np.float64))
    rel = np.abs(y - ref) / np.maximum(ref, 1e-30)
    print("asin_half max rel", rel.max())
    assert rel.max() <= 2.4e-7


def test_sin_on_half_turn(B):
    x = _grid(0.0, np.float32(np.pi), 1 << 24)
    y = _ev(B, "sin_half_turn", x)
    err = np.abs(y - np.sin(x.astype(np.float64)))
    print("sin_half_turn max abs", err.max())
    assert err.max() <= 1.8e-7


def test_log1p_for_non_negative_arguments(B):
    x = np.concatenate([_grid(0.0, 0.25, 1 << 23), _grid(0.25, 4.0, 1 << 22),
                        np.geomspace(4.0, 1e8, 1 << 20).astype(np.float32), np.float32([0.0, 1e-30, 1e-12])])
    y = _ev(B, "log1p_pos", x)
    ref = np.log1p(x.astype(np.float64))
    rel = np.abs(y - ref) / np.maximum(ref, 1e-300)
    rel[ref == 0] = np.abs(y[ref == 0])
    print("log1p_pos max rel", rel.max())
    assert rel.max() <= 6e-7


def test_cosh_and_sinh(B):
    x = np.concatenate([_grid(-12.0, 12.0, 1 << 23), -_grid(0.0, 0.5, 1 << 20), _grid(0.0, 0.5, 1 << 20)])
    x64 = x.astype(np.float64)
    c = _ev(B, "cosh", x)
    s = _ev(B, "sinh", x)
    rc = np.abs(c / np.cosh(x64) - 1)
    rs = np.abs(s - np.sinh(x64)) / np.maximum(np.abs(np.sinh(x64)), 1e-30)
    rs[x64 == 0] = np.abs(s[x64 == 0])
    print("cosh max rel", rc.max(), "sinh max rel", rs.max())
    assert rc.max() <= 4e-7 and rs.max() <= 4e-7


def test_asinh(B):
    x = np.concatenate([_grid(-50.0, 50.0, 1 << 23), np.geomspace(50.0, 1e7, 1 << 20).astype(np.float32),
                        -np.geomspace(50.0, 1e7, 1 << 20).astype(np.float32)])
    y = _ev(B, "asinh", x)
    ref = np.arcsinh(x.astype(np.float64))
    err = np.abs(y - ref) / np.maximum(np.abs(ref), 1.0)
    print("asinh max err / max(|asinh|, 1)", err.max())
    assert err.max() <= 2.5e-7


def test_reciprocal_and_square_root(B):
    x = np.concatenate([np.geomspace(1e-20, 1e20, 1 << 22).astype(np.float32), _grid(0.5, 2.0, 1 << 22)])
    x64 = x.astype(np.float64)
    r = _ev(B, "rcp", x)
    q = _ev(B, "sqrt", x)
    rr = np.abs(r * x64 - 1)
    rq = np.abs(q / np.sqrt(x64) - 1)
    print("rcp max rel", rr.max(), "sqrt max rel", rq.max())
    assert rr.max() <= 2.0**-23 and rq.max() <= 2.0**-22


def _ff(B, name, x):
    hi = _ev(B, name + "_hi", x).astype(np.longdouble)
    lo = _ev(B, name + "_lo", x).astype(np.longdouble)
    return hi + lo


def test_float_float_exponential(B):
    x = np.concatenate([_grid(0.0, 88.0, 1 << 23), _grid(0.0, 1.0, 1 << 21)])
    ref = np.exp(x.astype(np.longdouble))
    rel = (np.abs(_ff(B, "exp_ff", x) - ref) / ref).astype(np.float64)
    print("exp_ff max rel", rel.max(), "= 2^", np.log2(rel.max()))
    assert rel.max() <= 2.0**-42


def test_float_float_sinh(B):
    x = np.concatenate([_grid(0.0, 88.0, 1 << 23), _grid(0.0, 1.0, 1 << 21), _grid(0.0, 1.0 / 32, 1 << 20),
                        np.geomspace(1e-30, 1e-2, 1 << 16).astype(np.float32)])
    ref = np.sinh(x.astype(np.longdouble))
    err = np.abs(_ff(B, "sinh_ff", x) - ref)
    rel = np.where(ref > 0, err / np.where(ref > 0, ref, 1), err).astype(np.float64)
    print("sinh_ff max rel", rel.max(), "= 2^", np.log2(rel.max()),
          "from 1/4 up", rel[x >= 0.25].max(), "= 2^", np.log2(rel[x >= 0.25].max()))
    assert rel.max() <= 2.0**-36 and rel[x >= 0.25].max() <= 2.0**-41


def test_unknown_function_is_rejected(B):
    x = torch.zeros(4, device="cuda")
    assert B.lib().pdr_math_eval(99, x.data_ptr(), None, x.data_ptr(), 4, None) == -1
