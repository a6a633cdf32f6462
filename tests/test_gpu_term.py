"""The mixed form's FP32 real-space term erfc(alpha r)/r (paper Eq. (3),
second term) on the GPU: the paired form the kernels use (two terms per lane
with FFMA2/FADD2/FMUL2) gives the scalar function's bits, and both stay
within a few FP32 roundings of FP64 with no systematic sign over the range
of alpha r the real-space sum covers (erfc(alpha r) down to the mixed
cutoff's 1e-10, x = alpha r up to 4.58).

Bound per term: 3.5e-7 (1 + x) relative.  A few roundings of 2^-24 each
give the constant; the rounding of x itself (through 1/r from r^2) enters
erfc(x) multiplied by |d ln erfc(x) / dx| ~ 2x, so the error grows with x
(measured: rms 5e-8 near x = 0 to 3.6e-7 at x = 4.3, largest 1.4e-6, about
linear in x).  Bias:
the mean signed error over a million terms, per range of x and overall,
below 1e-8 and 5e-9 (a relative bias of 1e-8 per term would be ~4e-7 of
the error floor of the fcc electron-gas energies, whose real-space sums add
millions of terms of one sign)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

special = pytest.importorskip("scipy.special")


@pytest.fixture(scope="module")
def ew():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    ewald.load()
    return ewald


def samples(alpha, n, seed):
    """r^2 (float32) with x = alpha r distributed like pair images in a
    volume (density ~ x^2 up to 4.58), plus log-uniform small x; odd n."""
    rng = np.random.default_rng(seed)
    x = np.concatenate([4.58 * rng.random(n // 2) ** (1 / 3), np.exp(rng.uniform(np.log(1e-3), np.log(4.58), n - n // 2))])
    return ((x / alpha) ** 2).astype(np.float32)


@pytest.mark.parametrize("alpha", [0.15685, 0.0586, 0.4595, 1.0])
def test_paired_term_equals_scalar_and_fp64(ew, alpha):
    r2 = samples(alpha, (1 << 20) + 1, seed=int(alpha * 1e4))
    sc, pa = ew.pair_terms(r2, alpha)
    assert np.array_equal(sc.view(np.uint32), pa.view(np.uint32))
    r = np.sqrt(r2.astype(np.float64))
    ref = special.erfc(alpha * r) / r
    rel = (sc.astype(np.float64) - ref) / ref
    vol = slice(0, r2.size // 2)                      # the volume-weighted half
    x = alpha * r
    print("alpha %g: max |rel| %.3e, mean rel (volume) %.3e, (all) %.3e"
          % (alpha, np.max(np.abs(rel)), np.mean(rel[vol]), np.mean(rel)))
    for lo, hi in ((0, 0.5), (0.5, 1), (1, 2), (2, 3), (3, 4), (4, 4.6)):
        m = (x >= lo) & (x < hi)
        print("  x in [%g, %g): n %d max |rel| %.3e mean %.3e rms %.3e" % (lo, hi, m.sum(), np.max(np.abs(rel[m])),
              np.mean(rel[m]), np.sqrt(np.mean(rel[m] ** 2))))
        assert abs(np.mean(rel[m])) <= 1e-8
    assert np.all(np.abs(rel) <= 3.5e-7 * (1 + x))
    assert abs(np.mean(rel)) <= 5e-9 and abs(np.mean(rel[vol])) <= 5e-9


def test_pair_terms_arguments(ew):
    with pytest.raises(ew.EwaldError):
        ew.pair_terms(np.array([1.0, 0.0], dtype=np.float32), 0.5)      # r^2 = 0
    with pytest.raises(ew.EwaldError):
        ew.pair_terms(np.array([1.0], dtype=np.float32), -1.0)
    sc, pa = ew.pair_terms(np.zeros(0, dtype=np.float32), 0.5)
    assert sc.size == 0 and pa.size == 0


@pytest.mark.parametrize("alpha", [0.15685, 0.4595])
def test_double_float_head_term_against_fp64(ew, alpha):
    """The tiered form's head-term arithmetic (double-float 1/r and erfc,
    FP32 pipe only) on the head range x = alpha r < 3.77 against the FP64
    definition.  Bound per term 2e-14 (1 + 2 x^2): the pairs carry 48 bits,
    so x = alpha r (alpha itself a float pair) is good to ~1e-14, and
    erfc(x) turns a relative error e of x into ~2 x^2 e (measured: 1.2e-14
    near x = 0 to 4.0e-13 at x = 3.6).  The magnitude-weighted mean error,
    which is what a sum of head terms sees, stays below 5e-15."""
    rng = np.random.default_rng(7)
    x = np.concatenate([3.77 * rng.random(200000) ** (1 / 3), np.exp(rng.uniform(np.log(1e-3), np.log(3.77), 50001))])
    r2 = (x / alpha) ** 2
    got = ew.pair_terms_df(r2, alpha)
    r = np.sqrt(r2)
    ref = special.erfc(alpha * r) / r
    rel = (got - ref) / ref
    vol = slice(0, 200000)                             # the volume-weighted part
    wbias = np.sum(got[vol] - ref[vol]) / np.sum(ref[vol])
    print("alpha %g: max |rel| %.3e, weighted mean %.3e" % (alpha, np.max(np.abs(rel)), wbias))
    assert np.all(np.abs(rel) <= 2e-14 * (1 + 2 * x ** 2))
    assert abs(wbias) <= 5e-15


def test_pair_terms_df_arguments(ew):
    with pytest.raises(ew.EwaldError):
        ew.pair_terms_df(np.array([1.0, -2.0]), 0.5)
    assert ew.pair_terms_df(np.zeros(0), 0.5).size == 0
