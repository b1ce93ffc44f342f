"""The library's own exponentials against CUDA's and against the function's
value in extended precision (GPU).

Eq. density's exp(c_f (p - p_ref)) and the expm1(c_f (p - p^n)) form of
Eq. vk's accumulation term run, for small arguments, through Taylor series
of the library's own (exp_fp64 and expm1_fp64 below |x| < 2^-5, expm1_f32
below |x| < 2^-7); larger arguments, NaN and infinities go to CUDA's exp /
expm1 / expm1f.  tpfa_math_eval evaluates them element-wise.

Bounds, from the series' Horner form: exp_fp64 is the rounding of
1 + x r with r's error scaled by |x| <= 2^-5, so within 0.57 ulp of exp(x);
expm1_fp64 and expm1_f32 are two roundings (the last fused multiply-add and
the product with x), a relative error of at most 2u (u the unit roundoff),
i.e. just over 2 ulp at worst.  The truncated terms are below 2^-35 of the
value.  The rounding errors are unbiased: a wrong or missing series term
shows as a systematic error at the top of the range (dropping x^3/24 from
expm1_f32 biases its top octave by about -0.13 ulp), so the mean signed
error of the top octave is held to 0.05 ulp.  CUDA's exp, expm1 and expm1f
are within 1 ulp of the function's value, so the library's results are
within the sum of the two bounds of CUDA's.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

LD = np.longdouble
EXTENDED = np.finfo(LD).nmant >= 63  # x86 extended or IEEE quad


def _math(fn, x):
    from paper_2304_11274_gb300.api import math_eval

    y = math_eval(fn, torch.as_tensor(x, device="cuda:0"))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _series_args(lim, dense=1 << 18):
    mags = np.geomspace(1e-300 if lim > 0.01 else 1e-44, lim, 4001)[:-1]
    x = np.concatenate([np.linspace(-lim, lim, dense + 1)[1:-1], mags, -mags,
                        [0.0, -0.0, 5e-324, -5e-324, 1e-310, -2.2e-308,
                         np.nextafter(lim, 0.0), -np.nextafter(lim, 0.0)]])
    return x


def _outer_args(lim):
    x = np.concatenate([np.linspace(-700.0, 700.0, 20001), np.geomspace(lim, 700.0, 2001),
                        -np.geomspace(lim, 700.0, 2001),
                        [lim, -lim, np.nextafter(lim, 1.0), 0.05, -0.05, 1.0, -1.0, 10.0, 709.7, -745.0,
                         -746.0, -1000.0]])
    return x[np.abs(x) >= lim]


def _ulp_error(y, truth, dtype):
    """(y - truth) in units of the spacing of `dtype` at truth (finite)."""
    with np.errstate(over="ignore", invalid="ignore"):
        t = truth.astype(dtype)
        sp = np.spacing(np.abs(t)).astype(LD)
    return (y.astype(LD) - truth) / sp


def _check_special(y, ref):
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    assert np.array_equal(np.isposinf(y), np.isposinf(ref))
    assert np.array_equal(np.isneginf(y), np.isneginf(ref))


def _ulps_apart(a, b, dtype):
    """Distance in units in the last place of `dtype` between finite a and b
    of the same sign (or zero)."""
    ai = np.abs(a.astype(dtype)).view(np.int64 if dtype == np.float64 else np.int32).astype(np.int64)
    bi = np.abs(b.astype(dtype)).view(np.int64 if dtype == np.float64 else np.int32).astype(np.int64)
    same_sign = (np.signbit(a) == np.signbit(b)) | (a == 0) | (b == 0)
    assert same_sign.all()
    return np.abs(ai - bi)


CASES = {
    # fn: (series bound in ulp against the value, torch reference, dtype, series limit, numpy truth)
    "exp_fp64": (0.57, torch.exp, np.float64, 2.0 ** -5, np.exp),
    "expm1_fp64": (2.01, torch.expm1, np.float64, 2.0 ** -5, np.expm1),
    "expm1_f32": (2.01, torch.expm1, np.float32, 2.0 ** -7, np.expm1),
}


def _cuda_ref(fn, x):
    _, tf, dtype, _, _ = CASES[fn]
    xt = torch.as_tensor(x, device="cuda:0")
    if dtype == np.float32:
        xt = xt.float()
    r = tf(xt).double()
    torch.cuda.synchronize()
    return r.cpu().numpy()


def _truth(fn, x):
    _, _, dtype, _, npf = CASES[fn]
    xa = x.astype(np.float32).astype(np.float64) if dtype == np.float32 else x
    with np.errstate(over="ignore"):
        return npf(xa.astype(LD))


@pytest.mark.parametrize("fn", sorted(CASES))
def test_series_range_against_the_function_and_cuda(fn):
    bound, _, dtype, lim, _ = CASES[fn]
    x = _series_args(lim)
    if dtype == np.float32:
        x = x[np.abs(x.astype(np.float32)) < lim]
    y = _math(fn, x)
    ref = _cuda_ref(fn, x)
    assert np.isfinite(y).all()
    if dtype == np.float32:
        assert np.array_equal(y.astype(np.float32).astype(np.float64), y)  # an FP32 result, widened
    apart = _ulps_apart(y, ref, dtype)
    assert apart.max() <= int(np.floor(bound + 1.0)) + 1, (fn, apart.max())
    if not EXTENDED:
        pytest.skip("numpy's long double is not wider than double here: only the CUDA comparison ran")
    err = _ulp_error(y, _truth(fn, x), dtype)
    assert np.abs(err).max() <= bound, (fn, float(np.abs(err).max()))
    top = np.abs(x.astype(np.float32) if dtype == np.float32 else x) >= lim / 2
    assert top.sum() > 10000
    assert abs(float(err[top].mean())) < 0.05, (fn, float(err[top].mean()))


@pytest.mark.parametrize("fn", sorted(CASES))
def test_outside_the_series_range_it_is_cudas_function(fn):
    """From the series limit to overflow and underflow, and at NaN and the
    infinities, the result is CUDA's function's (a series evaluated beyond
    its range would be far off there)."""
    _, _, dtype, lim, _ = CASES[fn]
    x = _outer_args(lim)
    if dtype == np.float32:
        x = x[np.abs(x.astype(np.float32)) >= lim]
    x = np.concatenate([x, [np.nan, np.inf, -np.inf]])
    y = _math(fn, x)
    ref = _cuda_ref(fn, x)
    _check_special(y, ref)
    fin = np.isfinite(ref)
    assert _ulps_apart(y[fin], ref[fin], dtype).max() <= 2
    assert np.isnan(y[-3]) and y[-2] == np.inf and y[-1] == (0.0 if fn == "exp_fp64" else -1.0)


def test_ragged_lengths_and_empty():
    """Every element of a length that is no multiple of the block is written;
    n = 0 launches nothing."""
    from paper_2304_11274_gb300.api import math_eval

    for n in [1, 255, 257, 100003]:
        x = torch.linspace(-0.03, 0.03, n, dtype=torch.float64, device="cuda:0")
        y = math_eval("expm1_fp64", x)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert torch.equal(torch.sign(y), torch.sign(x))
    assert math_eval("exp_fp64", torch.empty(0, dtype=torch.float64, device="cuda:0")).numel() == 0
