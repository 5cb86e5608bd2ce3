"""The LPP-versus-GPP comparison of Sec. 4.2 on the polar-cap survey geometry (8 realisations
of a BBKS tidal field, 256^3, the cap theta < 60 deg, r in [1000, 1800] Mpc/h).

The paper finds that the LPP estimator on the locally projected field (case (a)) agrees with
the distant-observer set-up (case (c)), while the GPP estimator applied to the locally
projected field (case (b)) is biased at every scale.  Pinned here on the mean of the
realisations, with margins well outside their scatter (a few per cent per shell):
* |a / c - 1| < 3% for P_gd^(2) and P_+^(2) at k > 0.04 h/Mpc, < 15% above 0.01 h/Mpc (the
  windows of (a) and (c) differ, the paper's caveat, most at the largest scales);
* (b) falls below (c) by more than 15% (P_gd^(2)) and 50% (P_+^(2)) in every shell;
* P_+^(0) is the same in (a) and (b): the same projected field, and its kernel L_0 = 1 has no
  line of sight; the density monopole is the same in all three cases.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_lpp_agrees_with_distant_observer_and_gpp_on_local_projection_is_biased():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import lpp as L
    from paper_2202_11839_gb300 import los_cases as LC
    L.load_library()
    st = LC.LosStudy()
    mean, per = LC.run(st, seeds=range(1, 9))
    k = 0.5 * (st.k_edges[1:] + st.k_edges[:-1])
    a, b, c = (mean[x] for x in "abc")
    for slot, b_max in ((L.LPP_MOM_CROSS2, 0.85), (L.LPP_MOM_PLUS2, 0.5)):
        ra = a[slot].real / c[slot].real
        rb = b[slot].real / c[slot].real
        assert np.all(np.abs(ra[k > 0.04] - 1.0) < 0.03), (slot, ra)
        assert np.all(np.abs(ra[k > 0.01] - 1.0) < 0.15), (slot, ra)
        assert np.all(rb < b_max) and np.all(rb > 0.0), (slot, rb)
    np.testing.assert_allclose(a[L.LPP_MOM_PLUS0].real, b[L.LPP_MOM_PLUS0].real, rtol=1e-5)
    for x in "bc":
        np.testing.assert_allclose(mean[x][L.LPP_MOM_DD0].real, a[L.LPP_MOM_DD0].real, rtol=1e-5)
