"""Accuracy of the float-float elementary functions that the mixed prologue computes on the FP32 pipe
(gwl_ff_eval through the C ABI) against numpy's FP64 functions (correctly rounded to within 1 ulp).

The argument itself is held as a float pair (about 48 bits: |dx| <= 2^-48 |x|), so each bar is 3e-14
for the function plus the argument's representation error carried through it (2^-47 |x| for exp, sin
and cos; 2^-47 for ln).  The prologue needs ~1e-12 (the phase coefficients)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    from paper_1909_11873_gb300 import build, gwl
    build.build()
    return gwl


def run(g, x, fn):
    out = g.ff_eval(torch.from_numpy(np.ascontiguousarray(x)).cuda(), fn)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_ff_exp(g):
    x = np.concatenate([np.linspace(-20.0, 20.0, 20001), np.random.default_rng(0).uniform(-12, 3, 20000),
                        [0.0, -0.0, 1e-12, -1e-12]])
    ref = np.exp(x)
    assert np.all(np.abs(run(g, x, g.GWL_FF_EXP) - ref) / ref < 3e-14 + 2.0 ** -47 * np.abs(x))


def test_ff_log(g):
    x = np.concatenate([np.geomspace(1e-8, 1e8, 20001), np.random.default_rng(1).uniform(0.01, 2.0, 20000),
                        1.0 + np.linspace(-1e-6, 1e-6, 101)])
    ref = np.log(x)
    assert np.all(np.abs(run(g, x, g.GWL_FF_LOG) - ref) / np.maximum(np.abs(ref), 1.0) < 3e-14 + 2.0 ** -47)


@pytest.mark.parametrize("fn", ["sin", "cos"])
def test_ff_sin_cos(g, fn):
    """Absolute error over [-4 pi, 4 pi] (the prologue's angles lie in [-2 pi, 3 pi]), including quadrant
    boundaries (multiples of pi/4) and zeros."""
    k = np.arange(-16, 17)
    x = np.concatenate([np.linspace(-4 * np.pi, 4 * np.pi, 40001), k * np.pi / 4,
                        k * np.pi / 4 + 1e-9, k * np.pi / 4 - 1e-9,
                        np.random.default_rng(2).uniform(-7.0, 7.0, 20000)])
    code = g.GWL_FF_SIN if fn == "sin" else g.GWL_FF_COS
    ref = np.sin(x) if fn == "sin" else np.cos(x)
    assert np.all(np.abs(run(g, x, code) - ref) < 3e-14 + 2.0 ** -47 * np.abs(x))


@pytest.mark.parametrize("fn", ["sinpi", "cospi"])
def test_f32_sincospi(g, fn):
    """The FP32 sin(pi x), cos(pi x) of the mixed gradient's bin loop (a table of the 64th-cycle points and
    short series on the remainder, |u| <= pi/64, then the rotation) over |x| <= 1.5, with the quarter-turn
    boundaries and their neighbours: absolute error against FP64 at the FP32 argument below 2^-22 (the
    hardware sine's is ~4e-7), and exact values at the quarter turns' zeros and ones."""
    k = np.arange(-6, 7) / 4.0
    x = np.concatenate([np.linspace(-1.5, 1.5, 60001), k, np.nextafter(k.astype(np.float32), np.float32(2)),
                        np.nextafter(k.astype(np.float32), np.float32(-2)),
                        np.random.default_rng(3).uniform(-1.2, 1.2, 40000)]).astype(np.float32).astype(np.float64)
    code = g.GWL_F32_SINPI if fn == "sinpi" else g.GWL_F32_COSPI
    ref = np.sin(np.pi * x) if fn == "sinpi" else np.cos(np.pi * x)
    got = run(g, x, code)
    assert np.max(np.abs(got - ref)) < 2.0 ** -22
    # at the multiples of 1/2 the reduced argument is zero: the results are exactly 0 or +-1
    h = np.arange(-3, 4) / 2.0
    got_h = run(g, h, code)
    ref_h = np.round(np.sin(np.pi * h) if fn == "sinpi" else np.cos(np.pi * h))
    assert np.array_equal(np.abs(got_h), np.abs(ref_h)) and np.all(got_h * ref_h >= 0)
