"""Coarse lattice parameters (host logic of the C ABI, no GPU needed)."""

import pytest


def test_coarse_params_match_the_paper():
    """Section 4.3.2: tau_fine = 0.50012 with dx, dt scaled by r = 10 gives tau_coarse = 0.500012."""
    import paper_1312_0195_gb300 as lbm
    import synth
    u = synth.LatticeUnits(0.0025, 2.5e-5)
    fine = lbm.Params(nx=400, ny=400, tau=0.50012, nu=u.nu(2e-6), eps=0.8, gx=u.force(2.0))
    c = lbm.lbm_coarse_params(fine, 10)
    assert (c.nx, c.ny) == (40, 40)
    assert abs(c.tau - 0.500012) < 1e-15
    uc = synth.LatticeUnits(0.025, 2.5e-4)
    assert abs(c.nu - uc.nu(2e-6)) < 1e-18          # 8e-7: same physical nu on the coarse lattice
    assert abs(c.gx - uc.force(2.0)) < 1e-18        # G_c = r G_f
    assert c.eps == 0.8


def test_coarse_params_reject_bad_block():
    import paper_1312_0195_gb300 as lbm
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coarse_params(lbm.Params(nx=400, ny=400, tau=0.5), 7)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coarse_params(lbm.Params(nx=400, ny=400, tau=0.5), 0)
