"""The float path's own approximations against CUDA's functions and exact
values, on dense grids, through the library's test hook (bysdf_test_math,
computed with the kernels' build flags):

* atan2: the degree-8 polynomial in the octant's ratio (coefficients fitted
  by least squares on [0, 1]) against atan2f and float64 atan2, over every
  octant, the axes, zeros and points far from the origin (magnitudes below
  2^126, where the approximate division of the octant's ratio holds);
* the sine and cosine of the fiber normal's deviation (Taylor polynomials to
  degree 13 / 14 on [-pi/2, pi/2], sincosf beyond) against sinf / cosf and
  float64."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12724_gb300 import _native as N
    return N.load()


def call(lib, fn, x, y=None):
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda() if y is not None else None
    out = torch.empty_like(xt)
    rc = lib.bysdf_test_math(fn, xt.data_ptr(), yt.data_ptr() if yt is not None else None,
                             xt.numel(), out.data_ptr(), None)
    assert rc == 0, lib.bysdf_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_atan2_polynomial(lib):
    rng = np.random.default_rng(5)
    ang = np.linspace(-np.pi, np.pi, 400001)
    r = np.exp(rng.uniform(np.log(1e-20), np.log(1e20), ang.size))
    x = (r * np.cos(ang)).astype(np.float32)
    y = (r * np.sin(ang)).astype(np.float32)
    # axes, diagonals, zeros, tiny and huge components
    sp = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [-1, 1], [1, -1],
                   [-1, -1], [1e-30, 1.0], [1.0, 1e-30], [1e30, 1.0], [-1e30, -2e29]],
                  np.float32)
    x = np.concatenate([x, sp[:, 0]])
    y = np.concatenate([y, sp[:, 1]])
    mine = call(lib, 0, x, y)
    ref = call(lib, 1, x, y)
    exact = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    assert np.isfinite(mine).all()
    assert mine[-13] == 0.0                          # atan2(0, 0)
    # within a few 1e-7 rad of the exact value, like atan2f
    assert np.abs(mine - exact).max() <= 4e-7, np.abs(mine - exact).max()
    assert np.abs(ref - exact).max() <= 4e-7
    assert np.abs(mine - ref).max() <= 6e-7


def test_fiber_deviation_sincos(lib):
    x = np.concatenate([np.linspace(-np.pi / 2, np.pi / 2, 400001),
                        [0.0, 1e-30, -1e-30, 1.5707964, -1.5707964]]).astype(np.float32)
    s, c = call(lib, 2, x), call(lib, 3, x)
    rs, rc = call(lib, 4, x), call(lib, 5, x)
    xd = x.astype(np.float64)
    assert np.abs(s - np.sin(xd)).max() <= 2e-7
    assert np.abs(c - np.cos(xd)).max() <= 2e-7
    assert np.abs(s - rs).max() <= 2.5e-7 and np.abs(c - rc).max() <= 2.5e-7
    # tiny arguments keep their relative accuracy in the sine
    assert s[-4] == np.float32(1e-30) and s[-5] == 0.0
    # beyond pi/2 the library's sincosf takes over
    xb = np.array([2.0, -3.0, 100.0, 1e4], np.float32)
    assert np.array_equal(call(lib, 2, xb), call(lib, 4, xb))
    assert np.array_equal(call(lib, 3, xb), call(lib, 5, xb))
