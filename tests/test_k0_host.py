"""ls_k0_weight (host computation, no device) against the oracle: the ball-integral weight
every context uses, and the one-point trapezoid correction of Sec. 2.1, for 2D, 3D and the
3D Laplace kernel.  The two sides share no code: the library sums the lattice and integrates
radially with its own Gauss-Legendre panels and the C++ special functions, the oracle with
numpy / scipy."""

import math

import pytest

import oracle as O


@pytest.fixture(scope="module")
def LS():
    from paper_1408_4495_gb300 import build, ls
    build.build()
    return ls


@pytest.mark.parametrize("d,omega,h", [(2, 2 * math.pi * 2, 1 / 33), (2, 2 * math.pi * 32, 1 / 257),
                                       (3, 2 * math.pi * 1, 1 / 17), (3, 0.0, 1 / 65)])
def test_k0_weight_matches_the_oracle(LS, d, omega, h):
    ball = LS.k0_weight(d, omega, h, LS.LS_K0_BALL)
    ref = O.k0_weight(d, omega, h)
    assert abs(ball - ref) < 1e-13 * abs(ref)
    corr = LS.k0_weight(d, omega, h, LS.LS_K0_CORRECTED)
    refc = O.k0_corrected(d, omega, h)
    assert abs(corr - refc) < 1e-12 * abs(refc)


def test_k0_weight_rejects_bad_arguments(LS):
    for args in ((4, 1.0, 0.1, 0), (2, 0.0, 0.1, 0), (3, 1.0, -0.1, 0), (3, 1.0, 0.1, 7), (2, -1.0, 0.1, 1)):
        with pytest.raises(LS.LsError) as e:
            LS.k0_weight(*args)
        assert e.value.status == LS.LS_EINVAL
