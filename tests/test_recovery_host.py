"""pd_theta_to_apd (host code of the library) against the oracle's
physical-parameter recovery (Sec. 2.3, eqs. pd-lr-to-phys and
apd-lr-to-phys; the common shift of Sec. 5.5.3).  No GPU is involved: the
conversion is host arithmetic."""
import numpy as np
import pytest

import oracle as O
from paper_2605_20816_gb300 import pd, synth


@pytest.mark.parametrize("dim", [2, 3])
def test_power_diagram_matches_oracle(dim):
    y, w = synth.power_params(41 + dim, 12, dim=dim)
    th = O.theta_from_apd(dim, 1, y, w) + synth.random_theta(3, 1, dim + 1, 0.3)  # any gauge
    yo, wo, _, lo = O.theta_to_apd(dim, 1, th)
    yl, wl, Al, ll = pd.pd_theta_to_apd(dim, 1, th)
    assert Al is None and ll == lo == 0.0
    np.testing.assert_allclose(yl.numpy(), yo, rtol=0, atol=1e-13)
    np.testing.assert_allclose(wl.numpy(), wo, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,shift", [(2, 0.0), (2, 3.0), (3, 0.0), (3, 3.0)])
def test_anisotropic_matches_oracle(dim, shift):
    y, w, A = synth.apd_params(51 + dim, 10, dim=dim)
    th = O.theta_from_apd(dim, 2, y, w, A)
    # a common shift of the quadratic coefficients (Lemma 4.2) that leaves
    # metrics indefinite: the recovery must shift them back
    K = O.K(dim, 2)
    c = np.zeros(K)
    al = O.alpha(dim, 2)
    for k, a in enumerate(al):
        if sum(a) == 2 and max(a) == 2:
            c[k] = -shift * (2.0 / 3.0)     # -shift x_a^2 in Legendre: P_2 = (3 t^2 - 1) / 2
    th = th + c
    for margin in (1e-3, 0.25):
        yo, wo, Ao, lo = O.theta_to_apd(dim, 2, th, margin)
        yl, wl, Al, ll = pd.pd_theta_to_apd(dim, 2, th, margin)
        assert abs(ll - lo) <= 1e-12 * max(1.0, abs(lo))
        np.testing.assert_allclose(Al.numpy(), Ao, rtol=0, atol=1e-11)
        np.testing.assert_allclose(yl.numpy(), yo, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(wl.numpy(), wo, rtol=1e-10, atol=1e-10)
        assert np.linalg.eigvalsh(Al.numpy()).min() >= margin * (1 - 1e-9)


def test_errors():
    th = np.zeros((4, 6))
    with pytest.raises(pd.PdError) as e:
        pd.pd_theta_to_apd(2, 2, th, margin=0.0)
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PdError) as e:
        pd.pd_theta_to_apd(2, 3, np.zeros((4, 10)))
    assert e.value.code == pd.PD_ENOTSUP
    bad = th.copy()
    bad[1, 2] = np.nan
    with pytest.raises(pd.PdError) as e:
        pd.pd_theta_to_apd(2, 2, bad)
    assert e.value.code == pd.PD_ENAN
