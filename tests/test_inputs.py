"""The seeded synthetic workloads hold the shapes, ranges and structure the
library is measured and checked on (they stand in for the FAL-C Mg II h&k and
H I Ly-alpha runs of Sects. 6.1-6.2, with the atoms of Table 1), and the same
seed always gives the same arrays."""
import numpy as np

from paper_2505_20968_gb300 import inputs as I


def _vmax(atm):
    return float(np.sqrt((np.asarray(atm["v_kms"]) ** 2).sum(1)).max())


def test_mgii_workload_recipe():
    c = I.mgii()
    atm, quad = c["atm"], c["quad"]
    z = np.asarray(atm["z_km"])
    assert z.size == 70 and z[0] == -100.0 and abs(z[-1] - 2219.43) < 1e-9 and np.all(np.diff(z) > 0)
    lam = np.asarray(quad["grid"])
    assert lam.size == 200 and np.all(np.diff(lam) > 0) and quad["grid_kind"] == I.GRID_LAMBDA
    # both lines inside the grid, 70 nodes within 1 A of each
    for E in I.MGII_TABLE["E_u_cm"]:
        assert np.sum(np.abs(lam - 1e8 / E) <= 1.0 + 1e-9) >= 70
    assert 2 * quad["n_mu_half"] * quad["n_chi"] == 64
    assert np.all((atm["B_G"] >= 0) & (atm["B_G"] <= 100.0))
    assert abs(_vmax(atm) - 5.0) < 1e-12
    eps = np.asarray(atm["eps"])
    assert abs(eps[0] - 1e-3) < 1e-15 and abs(eps[-1] - 1e-6) < 1e-18
    assert 0.9e-4 < np.min(atm["a"]) and np.max(atm["a"]) < 1.1e-2
    assert 4000 < np.min(atm["T_K"]) and np.max(atm["T_K"]) < 1.2e4
    assert c["atom"]["E_u_cm"] == I.MGII_TABLE["E_u_cm"] and c["precision"] == "fp32"


def test_hi_lya_workload_recipe():
    c = I.hi_lya()
    atm, quad = c["atm"], c["quad"]
    assert len(atm["z_km"]) == 90 and len(quad["grid"]) == 150
    assert 2 * quad["n_mu_half"] * quad["n_chi"] == 96
    assert np.all((atm["B_G"] >= 0) & (atm["B_G"] <= 50.0))
    assert abs(_vmax(atm) - 5.0) < 1e-12
    assert 1.5e4 < np.max(atm["T_K"]) < 2.5e4
    assert I.hi_lya(mode=I.MODE_AA)["quad"]["mode"] == I.MODE_AA


def test_twolevel_slab_recipe():
    c = I.twolevel_slab()
    atm, quad = c["atm"], c["quad"]
    x = np.asarray(quad["grid"])
    t = -1.0 + np.arange(21) / 10.0
    assert np.allclose(x, 8.0 * np.sinh(3.0 * t) / np.sinh(3.0), rtol=0, atol=1e-12)
    assert len(atm["z_km"]) == 40 and quad["grid_kind"] == I.GRID_X
    assert np.ptp(atm["T_K"]) == 0.0 and np.max(np.abs(atm["B_G"])) == 0.0 and np.max(np.abs(atm["v_kms"])) == 0.0
    assert np.all(np.asarray(atm["a"]) == 1e-3) and np.all(np.asarray(atm["eps"]) == 1e-4)
    assert np.all(np.asarray(atm["r_el"]) == 0.1) and c["precision"] == "fp64"


def test_batch_is_ragged_within_its_ranges():
    cfgs = I.mgii_batch(n_inst=8)
    nz = [len(c["atm"]["z_km"]) for c in cfgs]
    nn = [len(c["quad"]["grid"]) for c in cfgs]
    assert all(50 <= v <= 130 for v in nz) and all(120 <= v <= 220 for v in nn)
    assert len(set(nz)) > 1 and len(set(nn)) > 1
    assert [c["seed"] for c in cfgs] == list(range(400, 408))


def test_seeded_and_deterministic():
    a, b, d = I.mgii(seed=7), I.mgii(seed=7), I.mgii(seed=8)
    for k in a["atm"]:
        assert np.array_equal(np.asarray(a["atm"][k]), np.asarray(b["atm"][k])), k
    assert not np.array_equal(a["atm"]["B_G"], d["atm"]["B_G"])
    assert np.array_equal(I.seeded_vector((3, 4), 5), I.seeded_vector((3, 4), 5))
