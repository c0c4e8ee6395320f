"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (FP32 path, stated by the method's target): nu within 1e-5 relative,
with the noise unit of nu (1) as the floor for values near zero:
    |nu_gpu - nu_64| <= 1e-5 * max(|nu_64|, 1)
alpha within 1e-5 relative with its noise unit sigma_alpha = 1/sqrt(Phi) as floor.
Top-k lists must be identical except where the oracle's own values tie within
that tolerance; a slot where the velocity index differs must name a trajectory
whose oracle nu equals the GPU's within tolerance and deserves the rank within
twice the tolerance.
"""
import numpy as np

NU_RTOL = 1e-5


def nu_tol(nu_ref, rtol=NU_RTOL):
    return rtol * np.maximum(np.abs(nu_ref), 1.0)


def check_topk(gpu, ref, nu_of, rtol=NU_RTOL, max_mismatch_frac=0.01, check_alpha=True):
    """gpu: records [..., k] (binding RESULT_DTYPE); ref: oracle records [..., k];
    nu_of(flat_pixel_index, vidx) -> oracle nu of that trajectory.  Returns mismatch count."""
    g = gpu.reshape(-1, gpu.shape[-1])
    r = ref.reshape(-1, ref.shape[-1])
    assert g.shape == r.shape
    gv, rv = g["vidx"], r["vidx"]
    # the same number of valid results per pixel
    assert np.array_equal(gv >= 0, rv >= 0), "valid-slot pattern differs"
    valid = rv >= 0
    # sorted nu agrees slot by slot
    dn = np.abs(g["nu"][valid] - r["nu"][valid])
    tol = nu_tol(r["nu"][valid], rtol)
    bad = dn > tol
    assert not bad.any(), "nu differs beyond tolerance in %d slots (max excess %.3g)" % (
        bad.sum(), (dn - tol).max())
    same = gv == rv
    mism = np.argwhere(valid & ~same)
    for (p, i) in mism:
        nu_true = nu_of(p, int(gv[p, i]))
        assert abs(nu_true - g["nu"][p, i]) <= nu_tol(nu_true, rtol), (p, i, nu_true, g["nu"][p, i])
        assert abs(nu_true - r["nu"][p, i]) <= 2 * nu_tol(r["nu"][p, i], rtol), (p, i, nu_true, r["nu"][p, i])
    assert len(mism) <= max(2, max_mismatch_frac * valid.sum()), "%d slots name different velocities" % len(mism)
    m = valid & same
    if check_alpha and m.any():
        sig = 1.0 / np.sqrt(r["phi"][m])
        da = np.abs(g["alpha"][m] - r["alpha"][m])
        ta = rtol * np.maximum(np.abs(r["alpha"][m]), sig)
        assert np.all(da <= ta), "alpha differs beyond tolerance in %d slots" % (da > ta).sum()
        assert np.array_equal(g["nobs"][m], r["nobs"][m]), "nobs differs"
        dphi = np.abs(g["phi"][m] - r["phi"][m])
        assert np.all(dphi <= rtol * r["phi"][m]), "Phi differs beyond tolerance"
    return len(mism)


def oracle_nu_table(psi, phi, times, dx, dy):
    """nu of every (pixel, velocity) from oracle planes: [H*W][V] (-inf where Phi == 0)."""
    import oracle
    V = dx.shape[0]
    N, H, W = psi.shape
    out = np.full((H * W, V), -np.inf)
    for v in range(V):
        P, F, _ = oracle.sums_one_velocity(psi, phi, times, dx[v], dy[v])
        ok = (F > 0).ravel()
        out[ok, v] = (P.ravel()[ok] / np.sqrt(F.ravel()[ok]))
    return out
