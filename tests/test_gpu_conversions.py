"""The FP64 <-> double-float conversions of the device path, bit for bit.

The solver carries its iterate, right-hand side and residual in double-float (hi + lo, two floats) and
converts from and to the caller's complex128 on the IEEE bit patterns with integer and FP32 instructions
(GB300's FP64 pipe is far slower).  Their definition is the FP64 one: hi = fl32(v), lo = fl32(v - hi) and
back hi + lo rounded to a double.  The second-order scheme's right-hand side is F = f (no correction
terms), so helm_build_rhs of an order-2 context runs exactly f -> double-float -> complex128, and F must
equal numpy's FP64 evaluation of the definition at every point, for values across the whole float range:
ordinary magnitudes, powers of two, values whose low part ties, zeros, tiny values outside the fast path
(below 2^-74) and large ones near the float limit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_07711_gb300 import Solver


def _reference(f):
    """hi + lo of the double-float split, both rounded as in IEEE FP64/FP32 arithmetic."""
    def part(v):
        hi = v.astype(np.float32)
        lo = (v - hi.astype(np.float64)).astype(np.float32)
        return hi.astype(np.float64) + lo.astype(np.float64)
    return part(f.real) + 1j * part(f.imag)


def _values(n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-35, 37, n)
    v = rng.standard_normal(n) * mag
    k = n // 8
    v[:k] = np.sign(v[:k]) * 2.0 ** rng.integers(-120, 120, k)                 # powers of two
    hi = v[k:2 * k].astype(np.float32).astype(np.float64)
    v[k:2 * k] = hi + np.spacing(hi.astype(np.float32)).astype(np.float64) / 2  # low part ties
    v[2 * k:2 * k + 16] = 0.0
    v[2 * k + 16:2 * k + 32] = rng.uniform(1e-35, 1e-25, 16)                    # below the fast path
    v[2 * k + 32:2 * k + 48] = rng.uniform(1e37, 3e38, 16)                      # near the float limit
    return rng.permutation(v)


def test_double_float_round_trip_is_the_fp64_definition():
    n = 24
    npts = n ** 3
    f = _values(npts, 1) + 1j * _values(npts, 2)
    S = Solver((n, n, n), np.full(npts, 100.0 + 0j), 10.0, order=2)
    F = S.build_rhs(torch.from_numpy(f.reshape(n, n, n)).cuda()).cpu().numpy().ravel()
    S.close()
    ref = _reference(f)
    assert np.array_equal(F, ref), int(np.sum(F != ref))
