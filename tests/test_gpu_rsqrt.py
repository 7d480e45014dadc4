"""Accuracy of the evaluation kernel's own reciprocal square roots (no CUDA
math-library routine is used for them) against a higher-precision reference:
numpy's long double 1/sqrt (at least 64 significant bits on both hosts),
over the seed's range x in [2^-126, 2^127] (EX: [2^-100, 2^100], where the
low float of the input pair is still normal).

FP64 form (x scaled into [1, 4), SFU seed refined in float-float and
assembled as a double on the integer pipe, one FP64 Newton step; and the
earlier five-DFMA form): at most 2 ulp of the correctly rounded result.  Float-float form of
the EX path: relative error at most 1e-13 (float-float carries about 48
bits; the input itself is rounded to a float-float pair).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00367_gb300 import build as nbbuild
    nbbuild.build()
    from paper_1812_00367_gb300 import nb as nbmod
    nbmod.load()
    return nbmod


def _inputs():
    rng = np.random.default_rng(11)
    parts = [
        np.exp2(rng.uniform(-125.9, 126.9, 200000)),           # the whole valid range
        10.0 ** rng.uniform(-10, 4, 200000),                   # r^2 + eps^2 of the workloads
        np.exp2(np.arange(-126, 127, dtype=np.float64)),       # powers of two
        1.0 + rng.uniform(-1e-3, 1e-3, 10000),                 # near 1
        np.nextafter(np.exp2(np.arange(-120, 120, 7.0)), np.inf),
    ]
    return np.concatenate(parts)


def _run(nb, which, x):
    xt = torch.as_tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    nb.nb_probe_rsqrt(which, xt, yt)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


@pytest.mark.parametrize("which", [0, 2])
def test_fp64_rsqrt_within_two_ulp(nb, which):
    x = _inputs()
    if which == 0:   # the three-DFMA form covers every positive normal double
        rng = np.random.default_rng(12)
        x = np.concatenate([x, np.exp2(rng.uniform(-1021.9, 1022.9, 100000)),
                            np.exp2(np.arange(-1022, 1023, dtype=np.float64)),
                            4.0 * (1.0 - rng.uniform(0.0, 1e-6, 10000))])
    y = _run(nb, which, x)
    ref = 1.0 / np.sqrt(x.astype(np.longdouble))
    ulp = np.spacing(ref.astype(np.float64))
    err = np.abs(y.astype(np.longdouble) - ref) / ulp
    assert np.all(np.isfinite(y))
    assert float(err.max()) <= 2.0, float(err.max())
    print(f"\nFP64 rsqrt form {which}: max {float(err.max()):.3f} ulp, mean {float(err.mean()):.3f} ulp")


def test_ex_rsqrt_relative_error(nb):
    # the low float of the input pair must stay normal: |x| within 2^+-100
    x = _inputs()
    x = x[(x >= 2.0 ** -100) & (x <= 2.0 ** 100)]
    y = _run(nb, 1, x)
    ref = 1.0 / np.sqrt(x.astype(np.longdouble))
    rel = np.abs(y.astype(np.longdouble) - ref) / ref
    assert float(rel.max()) <= 1e-13, float(rel.max())
    print(f"\nEX rsqrt: max relative error {float(rel.max()):.3e}")
