"""The pass rule the GPU parity tests use (tests/parity.py) rejects what it
must: planted errors just above the tolerance, non-finite values and
membership bits that disagree with the reference away from a level; it
excludes only points under the floor 1e-8 ||C||_F and forgives only
membership flips inside a level's pass band."""
import numpy as np

from tests.parity import atol_for, check_sigma

FRO = 10.0
N = 50


def _ref(k=200, seed=0):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-6, -5.2, k)  # above the 1e-7 floor, below 1e-6 ||C||_F = 1e-5


def _kw(rtol=1e-8):
    return dict(n=N, fro=FRO, schur_err=0.0, oracle_off=np.zeros(1), rtol=rtol)


def test_exact_values_pass_and_atol_is_the_stated_sum():
    ref = _ref()
    rep = check_sigma(ref.copy(), ref, **_kw())
    assert rep["n_bad"] == 0 and rep["n_included"] == ref.size
    assert atol_for(N, FRO, 1e-13, np.array([1e-16, 3e-16])) == 4.0 * (1e-13 + 3e-16 * FRO + N * 2.220446049250313e-16 * FRO)


def test_planted_relative_errors_are_caught_at_the_tolerance():
    ref = _ref()
    atol = atol_for(N, FRO, 0.0, np.zeros(1))
    band = 1e-8 * ref + atol
    inside = ref + 0.9 * band
    outside = ref - 1.1 * band
    assert check_sigma(inside, ref, **_kw())["n_bad"] == 0
    rep = check_sigma(outside, ref, **_kw())
    assert rep["n_bad"] == ref.size
    assert 1.0 < rep["worst_ratio"] < 1.2
    one = ref.copy()
    one[17] *= 1 + 1e-6  # one wrong point among 200
    assert check_sigma(one, ref, **_kw())["n_bad"] == 1


def test_non_finite_values_fail():
    ref = _ref(20)
    for bad in (np.nan, np.inf, -np.inf):
        sig = ref.copy()
        sig[3] = bad
        assert check_sigma(sig, ref, **_kw())["n_bad"] == 1


def test_only_points_under_the_floor_are_excluded():
    ref = np.array([1e-9, 5e-8, 1.01e-7, 0.3])  # floor = 1e-8 * 10 = 1e-7
    sig = ref * 2.0
    rep = check_sigma(sig, ref, **_kw())
    assert rep["n_included"] == 2 and rep["n_bad"] == 2


def test_membership_mismatch_and_in_band_flips():
    eps = (1e-1, 1e-3)
    ref = np.array([0.5, 5e-2, 5e-4, 1e-3 * (1 + 1e-12)])
    truth = np.zeros(ref.size, np.uint32)
    for i, e in enumerate(eps):
        truth |= (ref < e).astype(np.uint32) << np.uint32(i)
    rep = check_sigma(ref, ref, eps_levels=eps, member=truth, **_kw())
    assert rep["member_mismatch"] == 0 and rep["member_inband_flips"] == 0
    far = truth.copy()
    far[0] ^= np.uint32(1)  # sigma 0.5 is far from level 1e-1: a real mismatch
    rep = check_sigma(ref, ref, eps_levels=eps, member=far, **_kw())
    assert rep["member_mismatch"] == 1 and rep["member_inband_flips"] == 0
    near = truth.copy()
    near[3] ^= np.uint32(2)  # sigma within 1e-12 of level 1e-3: inside the band, forgiven and counted
    rep = check_sigma(ref, ref, eps_levels=eps, member=near, **_kw())
    assert rep["member_mismatch"] == 0 and rep["member_inband_flips"] == 1


def test_relative_target_holds_alone_above_1e_6_fro():
    # sigma_ref >= 1e-6 ||C||_F = 1e-5: atol no longer widens the band
    ref = np.array([2e-5, 1e-3, 0.5])
    atol = atol_for(N, FRO, 0.0, np.zeros(1))
    assert atol > 1e-8 * ref[0]  # the combined band alone would accept the planted error below
    sig = ref * (1 + 2e-8)
    rep = check_sigma(sig, ref, **_kw())
    assert rep["n_rel_only"] == 3 and rep["n_bad_rel"] == 3 and rep["n_bad"] == 3
    ok = ref * (1 + 0.9e-8)
    rep = check_sigma(ok, ref, **_kw())
    assert rep["n_bad"] == 0 and rep["max_rel_err_rel_only"] < 1e-8
    # just below the 1e-6 ||C||_F line the combined band applies
    rep = check_sigma(np.array([9.9e-6 * (1 + 2e-8)]), np.array([9.9e-6]), **_kw())
    assert rep["n_rel_only"] == 0 and rep["n_bad"] == 0
    # FP64 target
    rep = check_sigma(ref * (1 + 2e-10), ref, **_kw(rtol=1e-10))
    assert rep["n_bad_rel"] == 3
