"""mlmc_icdf_mse: the mean square error of the approximate Normal (Sec. 3.4,
eq. mse_dyadic) computed by the library from its own FP64 table, against the
oracle's 40-digit closed forms (Method 1: 1 - E[Z~^2]; Method 3: the
decomposition with the exact least-squares lines; Method 2: the decomposition
with the coupled uniform in interval pi(j))."""
import pytest

from oracle import tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc
    return mlmc


def _tol(d):
    # the GPU table entries are within 2^d 1e-15 relative of the closed form
    # (adjacent quantiles lose about d bits); the MSE is 1 - E[Z~^2] with
    # E[Z~^2] < 1, so its absolute error is at most twice that
    return 2.0 ** (d + 1) * 1e-15 + 1e-15


@pytest.mark.parametrize("d", range(2, 15))
def test_method1_and_method3_mse(m, d):
    _, mse1 = tables.moments_m1(d)
    assert abs(m.icdf_mse(d, 1) - float(mse1)) <= _tol(d)
    assert abs(m.icdf_mse(d, 3) - float(tables.mse_m3(d))) <= _tol(d)
    assert m.icdf_mse(d, 3) >= m.icdf_mse(d, 1)


@pytest.mark.parametrize("d,n", [(4, 2), (8, 2), (10, 2), (12, 3)])
def test_method2_mse(m, d, n):
    o = tables.m2_optimise(d, n)
    ref = tables.m2_mse(o["values"], o["pi"], d)
    assert abs(m.icdf_mse(d, 2, n) - ref) <= _tol(d) + 1e-12


def test_mse_argument_checks(m):
    for args in ((1, 1, 0), (1, 15, 0), (4, 10, 0), (1, 10, 2), (2, 10, 3)):
        with pytest.raises(m.MLMCError) as e:
            m.icdf_mse(args[1], args[0], args[2])
        assert e.value.status == m.EINVAL
