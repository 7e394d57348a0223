"""Pass rule shared by the parity tests.

sigma passes iff |sigma - sigma_ref| <= rtol * sigma_ref + atol with
atol = 4 * (e_schur + e_oracle + n * eps64 * ||C||_F); points with
sigma_ref < 1e-8 ||C||_F are excluded from sigma parity but still compared
for epsilon-membership, where a point whose sigma_ref lies inside the pass
band of a level may legitimately differ (counted, expected ~0).

Where sigma_ref >= 1e-6 ||C||_F the relative target must hold on its own:
|sigma - sigma_ref| <= rtol * sigma_ref, without atol (a point failing it
counts in ``n_bad`` as well as ``n_bad_rel``)."""
import numpy as np

EPS64 = 2.220446049250313e-16


def atol_for(n, fro, schur_err, oracle_off):
    return 4.0 * (schur_err + float(np.max(oracle_off)) * fro + n * EPS64 * fro)


def check_sigma(sig, ref, *, n, fro, schur_err, oracle_off, rtol, eps_levels=(), member=None):
    sig = np.asarray(sig, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    atol = atol_for(n, fro, schur_err, oracle_off)
    incl = ref >= 1e-8 * fro
    rel_only = ref >= 1e-6 * fro
    err = np.abs(sig - ref)
    band = rtol * ref + atol
    bad_rel = rel_only & ~(err <= rtol * ref)
    bad = (incl & ~(err <= band)) | bad_rel
    report = {
        "n_points": int(sig.size), "n_included": int(incl.sum()), "n_bad": int(bad.sum()), "atol": atol,
        "max_rel_err_included": float(np.max(err[incl] / ref[incl])) if incl.any() else 0.0,
        "worst_ratio": float(np.max(err[incl] / band[incl])) if incl.any() else 0.0,
        "n_rel_only": int(rel_only.sum()), "n_bad_rel": int(bad_rel.sum()),
        "max_rel_err_rel_only": float(np.max(err[rel_only] / ref[rel_only])) if rel_only.any() else 0.0,
    }
    if member is not None and len(eps_levels):
        mem = np.asarray(member).astype(np.uint32)
        flips = 0
        unexplained = 0
        for i, e in enumerate(eps_levels):
            m_gpu = (mem >> np.uint32(i)) & 1
            m_ref = (ref < e).astype(np.uint32)
            diff = m_gpu != m_ref
            inband = np.abs(ref - e) <= band
            flips += int((diff & inband).sum())
            unexplained += int((diff & ~inband).sum())
        report["member_inband_flips"] = flips
        report["member_mismatch"] = unexplained
    return report
