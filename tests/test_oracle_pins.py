"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test names the paper passage whose definition it pins and the independent
source of the expected value: a library routine (scipy), a closed form, exact
rational arithmetic, a distributional law, a different formulation (numpy
slicing) or brute-force enumeration.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import signal, stats

import oracle
import synth


def _weights(sci, var, mask=None, bright=np.inf):
    bad = ~np.isfinite(sci) | ~np.isfinite(var) | (var <= 0) | (sci > bright)
    if mask is not None:
        bad |= mask != 0
    w = np.where(bad, 0.0, 1.0 / np.where(bad, 1.0, var.astype(np.float64)))
    nw = np.where(bad, 0.0, np.where(bad, 0.0, sci.astype(np.float64)) * w)
    return w, nw


def _asym_psf(K, rng):
    p = rng.uniform(0.1, 1.0, (K, K)).astype(np.float32)
    return (p / p.sum()).astype(np.float32)


# ---------------------------------------------------------------- psi / phi images (Sec. 2.1.5)

def test_psi_phi_equals_scipy_correlate2d():
    """psi = corr(n/s^2, T), phi = corr(1/s^2, T^2) with zero fill: scipy.signal.correlate2d."""
    rng = np.random.default_rng(10)
    N, H, W, K = 3, 23, 17, 7
    sci = rng.normal(0, 3, (N, H, W)).astype(np.float32)
    var = rng.uniform(0.5, 4.0, (N, H, W)).astype(np.float32)
    sci[0, 3, 4] = np.nan
    var[1, 10, 2] = -1.0
    var[2, 0, 0] = np.inf
    mask = (rng.random((N, H, W)) < 0.05).astype(np.uint8)
    psf = np.stack([_asym_psf(K, rng) for _ in range(N)])  # asymmetric: correlation != convolution
    psi, phi = oracle.psi_phi(sci, var, mask, psf)
    for e in range(N):
        w, nw = _weights(sci[e], var[e], mask[e])
        k = psf[e].astype(np.float64)
        exp_psi = signal.correlate2d(nw, k, mode="same", boundary="fill", fillvalue=0.0)
        exp_phi = signal.correlate2d(w, k * k, mode="same", boundary="fill", fillvalue=0.0)
        np.testing.assert_allclose(psi[e], exp_psi, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(phi[e], exp_phi, rtol=1e-12, atol=1e-14)


def test_psi_of_delta_image_is_reflected_psf():
    """Closed form: a unit delta at c gives psi(c - d) = T(d)/s^2 (cross-correlation orientation)."""
    rng = np.random.default_rng(11)
    H, W, K = 15, 19, 5
    r = K // 2
    sci = np.zeros((1, H, W), np.float32)
    cy, cx = 7, 9
    sci[0, cy, cx] = 1.0
    var = np.full((1, H, W), 2.0, np.float32)
    psf = _asym_psf(K, rng)[None]
    psi, _ = oracle.psi_phi(sci, var, None, psf)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            assert psi[0, cy - dy, cx - dx] == pytest.approx(psf[0, dy + r, dx + r] / 2.0, rel=1e-14)
    assert np.count_nonzero(psi) == K * K


def test_constant_image_interior_closed_form():
    """Constant n = c and s^2 = V, no mask: interior psi = c/V * sum T, phi = sum T^2 / V; edges smaller."""
    H, W, K = 20, 24, 7
    r = K // 2
    psf = synth.gaussian_psf(K, 1.3)[None]
    sci = np.full((1, H, W), 3.0, np.float32)
    var = np.full((1, H, W), 5.0, np.float32)
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    t = psf[0].astype(np.float64)
    assert np.allclose(psi[0, r:H - r, r:W - r], 3.0 / 5.0 * t.sum(), rtol=1e-13)
    assert np.allclose(phi[0, r:H - r, r:W - r], (t * t).sum() / 5.0, rtol=1e-13)
    assert phi[0, 0, 0] < phi[0, H // 2, W // 2]  # zero padding, no renormalisation


def test_masked_pixels_add_nothing():
    """Sec. 2.1.5: masked pixels get zero weight, so their values cannot change psi or phi."""
    rng = np.random.default_rng(12)
    st = synth.small_stack(12, 2, 16, 18, K=5, mask_frac=0.1)
    psi1, phi1 = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    sci2, var2 = st.sci.copy(), st.var.copy()
    m = st.mask != 0
    sci2[m] = rng.normal(0, 1e6, m.sum())
    var2[m] = rng.uniform(-5, 5, m.sum())
    psi2, phi2 = oracle.psi_phi(sci2, var2, st.mask, st.psf)
    assert np.array_equal(psi1, psi2) and np.array_equal(phi1, phi2)


def test_bright_pixel_limit_masks():
    """Sec. 5.2 bright-pixel mask: pixels above the limit behave as masked."""
    st = synth.small_stack(13, 1, 12, 12, K=5)
    sci = st.sci.copy()
    sci[0, 5, 6] = 500.0
    mask = np.zeros(sci.shape, np.uint8)
    mask[0, 5, 6] = 1
    a = oracle.psi_phi(sci, st.var, None, st.psf, bright_max=120.0)
    b = oracle.psi_phi(sci, st.var, mask, st.psf)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_point_definition_matches_planes():
    st = synth.small_stack(14, 3, 14, 11, K=5, nan_frac=0.05, mask_frac=0.05)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    for (e, y, x) in [(0, 0, 0), (1, 7, 5), (2, 13, 10), (2, 3, 9)]:
        a, b = oracle.psi_phi_at(st.sci[e], st.var[e], st.mask[e], st.psf[e], x, y)
        assert a == pytest.approx(psi[e, y, x], rel=1e-13, abs=1e-15)
        assert b == pytest.approx(phi[e, y, x], rel=1e-13, abs=1e-15)


# ---------------------------------------------------------------- trajectory pixels

def _exact_offset(v, dt):
    """floor(v_q t_q / 2^36 + 1/2) with exact rationals (v_q, t_q: nearest integers, ties away)."""
    def rnd(x):  # llround: nearest, halves away from zero, on the exact value of the double
        f = Fraction(x)
        a = abs(f)
        n = math.floor(a + Fraction(1, 2))
        return n if f >= 0 else -n
    vq = rnd(Fraction(v) * 65536)
    tq = rnd(Fraction(dt) * 1048576)
    return math.floor(Fraction(vq * tq, 2 ** 36) + Fraction(1, 2)), vq, tq


def test_offsets_match_exact_rationals():
    rng = np.random.default_rng(20)
    times = np.concatenate([[3.25], 3.25 + np.sort(rng.uniform(0, 3.0, 9))])
    vx = rng.uniform(-600, 600, 40)
    vy = rng.uniform(-600, 600, 40)
    dx, dy = oracle.offsets(times, vx, vy)
    for v in range(40):
        for e in range(times.size):
            dt = times[e] - times.min()
            assert dx[v, e] == _exact_offset(vx[v], dt)[0]
            assert dy[v, e] == _exact_offset(vy[v], dt)[0]


def test_offsets_round_half_up_and_reference_epoch():
    """v t exactly at k + 1/2 rounds up (also for negatives); the earliest epoch has offset 0."""
    cases = [(1.5, 1.0, 2), (2.5, 1.0, 3), (-2.5, 1.0, -2), (-1.5, 1.0, -1), (0.75, 2.0, 2),
             (-0.25, 2.0, 0), (3.0, 0.5, 2), (-3.0, 0.5, -1), (0.0, 5.0, 0), (10.0, 0.0, 0)]
    for v, t, expect in cases:
        times = np.array([7.0, 7.0 + t]) if t > 0 else np.array([7.0])
        dx, _ = oracle.offsets(times, np.array([v]), np.array([0.0]))
        assert dx[0, 0] == 0
        if t > 0:
            assert dx[0, 1] == expect, (v, t)
    # unordered epochs: offsets relative to the minimum time
    dx, dy = oracle.offsets(np.array([2.0, 1.0, 1.5]), np.array([4.0]), np.array([-4.0]))
    assert list(dx[0]) == [4, 0, 2] and list(dy[0]) == [-4, 0, -2]


# ---------------------------------------------------------------- coadd, scores, search (Sec. 2.1.5, 2.2)

def _stamp_psf(img, cy, cx, psf, scale):
    K = psf.shape[0]
    r = K // 2
    img[cy - r:cy + r + 1, cx - r:cx + r + 1] += (scale * psf).astype(np.float32)


def test_noiseless_injection_closed_form():
    """A noiseless source f*T_t on the trajectory pixels gives Psi_t = f S_t, Phi_t = S_t with
    S_t = sum T_t^2 / V_t, hence alpha = f and nu = f sqrt(sum_t S_t); it is also the top result."""
    rng = np.random.default_rng(30)
    N, H, W, K = 4, 40, 44, 7
    times = np.array([0.0, 0.4, 1.1, 1.7])
    vx, vy = synth.velocity_grid(8, 5, -math.pi, math.pi, 2.0, 6.0, angle_endpoint=False)
    dx, dy = oracle.offsets(times, vx, vy)
    vt = 13
    x0, y0 = 20, 22
    f = 8.0  # power of two: the float32 stamp f*T is exact
    V_t = rng.uniform(1.0, 3.0, N).astype(np.float32)
    psf = np.stack([_asym_psf(K, rng) for _ in range(N)])
    sci = np.zeros((N, H, W), np.float32)
    var = np.empty((N, H, W), np.float32)
    for e in range(N):
        var[e] = V_t[e]
        _stamp_psf(sci[e], y0 + dy[vt, e], x0 + dx[vt, e], psf[e], f)
    S = np.array([(psf[e].astype(np.float64) ** 2).sum() / np.float64(V_t[e]) for e in range(N)])
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    rec = oracle.search_pixels(psi, phi, times, dx, dy, 3, [x0], [y0])[0]
    P, F, n = oracle.sums_one_velocity(psi, phi, times, dx[vt], dy[vt])
    assert P[y0, x0] == pytest.approx(f * S.sum(), rel=1e-12)
    assert F[y0, x0] == pytest.approx(S.sum(), rel=1e-12)
    assert n[y0, x0] == N
    top = rec[0]
    assert np.array_equal(dx[top["vidx"]], dx[vt]) and np.array_equal(dy[top["vidx"]], dy[vt])
    assert top["nu"] == pytest.approx(f * math.sqrt(S.sum()), rel=1e-12)
    assert top["alpha"] == pytest.approx(f, rel=1e-12)
    assert top["nobs"] == N and rec[1]["nu"] < top["nu"]


def test_noise_only_nu_is_standard_normal():
    """With n ~ N(0, s^2) per pixel, Var(psi_t) = phi_t, so nu of a fixed trajectory is N(0, 1)."""
    rng = np.random.default_rng(31)
    N, H, W, K = 5, 160, 170, 7
    times = np.array([0.0, 0.3, 0.9, 1.2, 2.0])
    var = rng.uniform(1.0, 6.0, (N, H, W)).astype(np.float32)
    sci = (rng.standard_normal((N, H, W)) * np.sqrt(var)).astype(np.float32)
    psf = np.stack([synth.gaussian_psf(K, s) for s in rng.uniform(0.9, 1.4, N)])
    vx, vy = np.array([4.0]), np.array([-3.0])
    dx, dy = oracle.offsets(times, vx, vy)
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    P, F, n = oracle.sums_one_velocity(psi, phi, times, dx[0], dy[0])
    r = K // 2
    ys = np.arange(r + 8, H - r - 8, K + 1)   # disjoint PSF supports -> independent samples
    xs = np.arange(r + 1, W - r - 10, K + 1)
    nu = (P / np.sqrt(F))[np.ix_(ys, xs)].ravel()
    m = nu.size
    assert m > 300
    assert abs(nu.mean()) < 4.0 / math.sqrt(m)
    assert abs(nu.var() - 1.0) < 4.0 * math.sqrt(2.0 / m)
    assert stats.kstest(nu, "norm").pvalue > 1e-3


def _shift_stack(planes, times, dxv, dyv):
    """Textbook shift-and-stack with numpy slicing: sum_t planes_t(y + dy_t, x + dx_t), zero outside."""
    N, H, W = planes.shape
    out = np.zeros((H, W))
    cnt = np.zeros((H, W), np.int32)
    for e in np.argsort(times, kind="stable"):
        sx, sy = int(dxv[e]), int(dyv[e])
        ys, ye = max(0, -sy), min(H, H - sy)
        xs, xe = max(0, -sx), min(W, W - sx)
        if ys >= ye or xs >= xe:
            continue
        out[ys:ye, xs:xe] += planes[e, ys + sy:ye + sy, xs + sx:xe + sx]
        cnt[ys:ye, xs:xe] += 1
    return out, cnt


def test_coadd_equals_shift_and_stack():
    """Sec. 2.1.5: summing psi along the trajectory equals shifting the planes and stacking them."""
    st = synth.small_stack(32, 5, 30, 26, K=5, nan_frac=0.02, s_hi=9.0)
    psi, phi = oracle.psi_phi(st.sci, st.var, None, st.psf)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    for v in [0, 7, 21, 40, 63]:
        P, F, n = oracle.sums_one_velocity(psi, phi, st.times, dx[v], dy[v])
        P2, c2 = _shift_stack(psi, st.times, dx[v], dy[v])
        F2, _ = _shift_stack(phi, st.times, dx[v], dy[v])
        np.testing.assert_allclose(P, P2, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(F, F2, rtol=1e-13, atol=1e-15)
        assert np.array_equal(n, c2)


def _brute_topk(psi, phi, times, dx, dy, k, nu_min=-np.inf):
    V = dx.shape[0]
    N, H, W = psi.shape
    nu = np.full((V, H, W), -np.inf)
    for v in range(V):
        P, _ = _shift_stack(psi, times, dx[v], dy[v])
        F, _ = _shift_stack(phi, times, dx[v], dy[v])
        ok = F > 0
        nu[v][ok] = P[ok] / np.sqrt(F[ok])
    out = np.full((H, W, k), -1, np.int64)
    for y in range(H):
        for x in range(W):
            col = nu[:, y, x]
            valid = np.nonzero((col > -np.inf) & (col >= nu_min))[0]
            order = valid[np.lexsort((valid, -col[valid]))]
            out[y, x, :min(k, order.size)] = order[:k]
    return out, nu


def test_topk_equals_brute_force_sort_with_exact_ties():
    """Sec. 2.2 exhaustive search: the kept list is the full sort by (nu desc, vidx asc); duplicated
    velocities give bit-identical sums (exact ties broken by index)."""
    st = synth.small_stack(33, 3, 9, 11, K=3, mask_frac=0.05, n_angles=4, n_speeds=3, s_hi=3.0)
    vx = np.concatenate([st.vx, st.vx[:4], [0.01, 0.02]])
    vy = np.concatenate([st.vy, st.vy[:4], [0.0, 0.0]])
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    dx, dy = oracle.offsets(st.times, vx, vy)
    k = 5
    rec = oracle.search_region(psi, phi, st.times, dx, dy, k)
    expect, nu = _brute_topk(psi, phi, st.times, dx, dy, k)
    assert np.array_equal(rec["vidx"], expect)
    got = rec["nu"][expect >= 0]
    ref = np.take_along_axis(nu.transpose(1, 2, 0), np.maximum(expect, 0), axis=2)[expect >= 0]
    np.testing.assert_allclose(got, ref, rtol=1e-13)
    # thresholded list keeps only nu >= nu_min, in the same order
    rec2 = oracle.search_region(psi, phi, st.times, dx, dy, k, nu_min=0.5)
    expect2, _ = _brute_topk(psi, phi, st.times, dx, dy, k, nu_min=0.5)
    assert np.array_equal(rec2["vidx"], expect2)


def test_scaling_laws_exact():
    """n -> 2n doubles nu and alpha; s^2 -> 4 s^2 halves nu and keeps alpha (exact in binary FP)."""
    st = synth.small_stack(34, 4, 12, 13, K=5, var_lo=1.0, var_hi=3.0)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    base = oracle.search_region(*oracle.psi_phi(st.sci, st.var, None, st.psf), st.times, dx, dy, 3)
    two = oracle.search_region(*oracle.psi_phi(2 * st.sci, st.var, None, st.psf), st.times, dx, dy, 3)
    four = oracle.search_region(*oracle.psi_phi(st.sci, 4 * st.var, None, st.psf), st.times, dx, dy, 3)
    assert np.array_equal(two["vidx"], base["vidx"]) and np.array_equal(two["nu"], 2 * base["nu"])
    assert np.array_equal(two["alpha"], 2 * base["alpha"])
    assert np.array_equal(four["vidx"], base["vidx"]) and np.array_equal(four["nu"], base["nu"] / 2)
    assert np.array_equal(four["alpha"], base["alpha"])


def test_epoch_permutation_invariance():
    """Permuting (image, time) pairs together leaves every result unchanged."""
    st = synth.small_stack(35, 5, 12, 10, K=5, nan_frac=0.03)
    perm = np.array([3, 0, 4, 2, 1])
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    a = oracle.search_region(*oracle.psi_phi(st.sci, st.var, None, st.psf), st.times, dx, dy, 4)
    dxp, dyp = oracle.offsets(st.times[perm], st.vx, st.vy)
    b = oracle.search_region(*oracle.psi_phi(st.sci[perm], st.var[perm], None, st.psf[perm]),
                             st.times[perm], dxp, dyp, 4)
    assert np.array_equal(a, b)


def test_trajectory_from_images_matches_planes():
    st = synth.small_stack(36, 4, 20, 18, K=5, nan_frac=0.03, mask_frac=0.03)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    for v, x0, y0 in [(0, 3, 4), (17, 10, 10), (50, 17, 0), (63, 0, 19)]:
        P, F, n = oracle.sums_one_velocity(psi, phi, st.times, dx[v], dy[v])
        a, b, c = oracle.trajectory_from_images(st.sci, st.var, st.mask, st.psf, st.times, dx[v], dy[v],
                                                x0, y0)
        assert a == pytest.approx(P[y0, x0], rel=1e-12, abs=1e-14)
        assert b == pytest.approx(F[y0, x0], rel=1e-12, abs=1e-14)
        assert c == n[y0, x0]


def test_off_image_trajectory_is_invalid():
    """Epochs off the image add nothing; a trajectory with no valid epoch (Phi = 0) is never kept."""
    st = synth.small_stack(37, 3, 8, 8, K=3)
    times = np.array([0.0, 1.0, 2.0])
    vx = np.array([100.0, 1.0])
    vy = np.array([0.0, 0.0])
    dx, dy = oracle.offsets(times, vx, vy)
    var = st.var.copy()
    var[0] = -1.0   # epoch 0 fully masked -> phi_0 = 0 everywhere
    psi, phi = oracle.psi_phi(st.sci, var, None, st.psf)
    rec = oracle.search_region(psi, phi, times, dx, dy, 2)
    # velocity 0 leaves the image after t = 0 and epoch 0 has phi = 0: never valid.  Velocity 1
    # visits x0, x0 + 1, x0 + 2: nobs counts in-image epochs (masked or not), and at x0 = 7 only
    # the masked epoch 0 is inside, so Phi = 0 and nothing is kept.
    assert np.all(rec["vidx"][:, :7, 0] == 1)
    assert np.all(rec["nobs"][:, :6, 0] == 3) and np.all(rec["nobs"][:, 6, 0] == 2)
    assert np.all(rec["vidx"][:, 7, :] == -1) and np.all(rec["nu"][:, 7, :] == -np.inf)
    assert np.all(rec["vidx"][..., 1] == -1) and np.all(rec["nu"][..., 1] == -np.inf)


def test_search_from_images_matches_planes():
    """The point-evaluated search (used for sampled full-size checks) equals the plane search."""
    st = synth.small_stack(38, 4, 21, 19, K=5, nan_frac=0.03, mask_frac=0.03)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    px = np.array([0, 5, 18, 9, 3])
    py = np.array([0, 11, 20, 2, 17])
    a = oracle.search_pixels(psi, phi, st.times, dx, dy, 6, px, py)
    b = oracle.search_pixels_from_images(st.sci, st.var, st.mask, st.psf, st.times, dx, dy, 6, px, py)
    assert np.array_equal(a["vidx"], b["vidx"]) and np.array_equal(a["nobs"], b["nobs"])
    np.testing.assert_allclose(a["nu"][a["vidx"] >= 0], b["nu"][b["vidx"] >= 0], rtol=1e-12)


def _read_golden(name):
    """Parse a hand-worked fixture of tests/golden (format described in the file)."""
    from fractions import Fraction
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    d = dict(images=[], mask=[], velocities=[], trajectories=[], topk=[])
    cur = None
    for raw in open(path):
        line = raw.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "times":
            d["times"] = [float(t) for t in tok[1:]]
        elif tok[0] == "variance":
            d["variance"] = [float(t) for t in tok[1:]]
        elif tok[0] == "psf":
            d["psf"] = float(tok[1])
        elif tok[0] == "image":
            cur = []
            d["images"].append(cur)
        elif tok[0] == "mask":
            d["mask"].append(tuple(int(t) for t in tok[1:]))
        elif tok[0] == "velocity":
            d["velocities"].append((float(tok[2]), float(tok[3])))
        elif tok[0] == "trajectory":
            d["trajectories"].append((int(tok[1]), int(tok[2]), int(tok[3]), Fraction(tok[4]), Fraction(tok[5]),
                                      int(tok[6])))
        elif tok[0] == "topk":
            d["topk"].append((int(tok[1]), int(tok[2]), [int(t) for t in tok[3:]]))
        else:
            cur.append([float(t) for t in tok])
    return d


def test_hand_worked_coadd_example():
    """Sec. 2.1.5 / 2.2 on a hand-worked 3-epoch stack (tests/golden/coadd_hand_example.txt):
    exact Psi, Phi and nobs of ten trajectories (masked pixel, trajectories leaving the
    image, half-pixel offsets in both directions) and the top-k order of one start pixel."""
    d = _read_golden("coadd_hand_example.txt")
    sci = np.array(d["images"], np.float32)
    N, H, W = sci.shape
    var = np.stack([np.full((H, W), v, np.float32) for v in d["variance"]])
    mask = np.zeros((N, H, W), np.uint8)
    for e, x, y in d["mask"]:
        mask[e, y, x] = 1
    psf = np.full((N, 1, 1), d["psf"], np.float32)
    vx = np.array([v[0] for v in d["velocities"]])
    vy = np.array([v[1] for v in d["velocities"]])
    times = np.array(d["times"])
    psi, phi = oracle.psi_phi(sci, var, mask, psf)
    dx, dy = oracle.offsets(times, vx, vy)
    for x0, y0, v, P, F, nobs in d["trajectories"]:
        Pg, Fg, Ng = oracle.sums_one_velocity(psi, phi, times, dx[v], dy[v])
        assert Pg[y0, x0] == float(P) and Fg[y0, x0] == float(F) and Ng[y0, x0] == nobs, (x0, y0, v)
    for x0, y0, order in d["topk"]:
        rec = oracle.search_pixels(psi, phi, times, dx, dy, len(order), np.array([x0]), np.array([y0]))[0]
        assert list(rec["vidx"]) == order
        for r in rec:
            P, F = [(t[3], t[4]) for t in d["trajectories"] if (t[0], t[1], t[2]) == (x0, y0, r["vidx"])][0]
            assert r["nu"] == pytest.approx(float(P) / math.sqrt(float(F)), rel=1e-15)
            assert r["alpha"] == pytest.approx(float(P / F), rel=1e-15)


# ------------------------------------------------------------ Sec. 3.3 light-curve filter

def _flat_stack(N, H, W, flux_map):
    """1 x 1 PSF, unit variance: psi_t = n_t, phi_t = 1 at every pixel (Sec. 2.1.5 with T = 1)."""
    sci = np.asarray(flux_map, np.float32)
    var = np.ones((N, H, W), np.float32)
    psf = np.ones((N, 1, 1), np.float32)
    return sci, var, psf


def test_filter_rejects_exactly_the_interloper_epoch():
    """Constant flux 2 on a stationary trajectory in 8 epochs, one epoch with flux 32 (a bright
    interloper, Sec. 3.3).  With unit variances that epoch is 28 sigma from the other seven's
    flux and each other epoch 4 sigma from the rest: only the interloper goes, and the kept
    epochs give Psi = 14, Phi = 7, nu = 14 / sqrt(7), alpha = 2."""
    N, H, W = 8, 5, 5
    img = np.zeros((N, H, W), np.float32)
    img[:, 2, 2] = 2.0
    img[3, 2, 2] = 32.0
    sci, var, psf = _flat_stack(N, H, W, img)
    times = np.arange(N, dtype=np.float64) * 0.1
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    dx = np.zeros(N, np.int32)
    dy = np.zeros(N, np.int32)
    P, F, nk, nr, rej = oracle.filter_lightcurve(psi, phi, times, dx, dy, 2, 2, 5.0)
    assert (P, F, nk, nr) == (14.0, 7.0, 7, 1)
    assert list(np.nonzero(rej)[0]) == [3]
    # a lower threshold also takes the 4-sigma epochs: nothing then survives but the outlier's test
    P, F, nk, nr, rej = oracle.filter_lightcurve(psi, phi, times, dx, dy, 2, 2, 3.5)
    assert nr == N and nk == 0 and (P, F) == (0.0, 0.0)


def test_filter_keeps_a_clean_noiseless_source():
    """A noiseless point source on its exact trajectory: every epoch's flux equals the others',
    so nothing is rejected and the sums equal the unfiltered coadd."""
    rng = np.random.default_rng(31)
    N, H, W, K = 6, 40, 60, 7
    times = np.array([0.0, 0.3, 0.7, 1.2, 1.6, 2.0])
    psf1 = synth.gaussian_psf(K, 1.2)
    psf = np.stack([psf1] * N)
    var = np.stack([np.full((H, W), v, np.float32) for v in rng.uniform(2.0, 5.0, N)])
    sci = np.zeros((N, H, W), np.float32)
    v = (7.0, -4.0)
    for e, t in enumerate(times):
        sci[e, 25 + int(round(v[1] * t)) - K // 2: 25 + int(round(v[1] * t)) + K // 2 + 1,
            12 + int(round(v[0] * t)) - K // 2: 12 + int(round(v[0] * t)) + K // 2 + 1] = 8.0 * psf1
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    dx, dy = oracle.offsets(times, np.array([v[0]]), np.array([v[1]]))
    P, F, nk, nr, rej = oracle.filter_lightcurve(psi, phi, times, dx[0], dy[0], 12, 25, 5.0)
    P0, F0, n0 = oracle.sums_one_velocity(psi, phi, times, dx[0], dy[0])
    assert nr == 0 and nk == N and not rej.any()
    assert P == P0[25, 12] and F == F0[25, 12]
    assert P / F == pytest.approx(8.0, rel=1e-9)


def test_filter_rarely_rejects_pure_noise():
    """N(0, 1) noise, unit variance, no source: alpha_e - alpha_rest then has variance exactly
    1 / phi_e + 1 / (Phi - phi_e), so the statistic is N(0, 1).  A 5-sigma rejection has
    probability ~6e-7 per epoch (essentially none over ~48000 epochs); beyond 2 sigma lie
    4.55 % of them."""
    rng = np.random.default_rng(32)
    N, H, W = 8, 60, 100
    sci, var, psf = _flat_stack(N, H, W, rng.standard_normal((N, H, W)))
    times = np.arange(N) * 0.25
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    dx = np.zeros(N, np.int32)
    dy = np.zeros(N, np.int32)
    rej5 = rej2 = 0
    for y in range(H):
        for x in range(W):
            rej5 += oracle.filter_lightcurve(psi, phi, times, dx, dy, x, y, 5.0)[3]
            rej2 += oracle.filter_lightcurve(psi, phi, times, dx, dy, x, y, 2.0)[3]
    n = N * H * W
    assert rej5 <= 2
    # under the null, (alpha_e - alpha_rest) / sigma is exactly N(0, 1): 4.55 % beyond 2 sigma
    assert abs(rej2 / n - 0.0455) < 5 * math.sqrt(0.0455 * 0.9545 / n)


def test_filter_masked_epoch_and_permutation_invariance():
    """An epoch masked at the trajectory pixel (phi = 0 there with a 1 x 1 PSF) carries no
    information and is never rejected; permuting (epoch, time) pairs changes nothing."""
    N, H, W = 7, 4, 4
    img = np.zeros((N, H, W), np.float32)
    img[:, 1, 1] = 3.0
    img[5, 1, 1] = 300.0
    sci, var, psf = _flat_stack(N, H, W, img)
    mask = np.zeros((N, H, W), np.uint8)
    mask[5, 1, 1] = 1
    times = np.array([0.0, 0.5, 0.2, 0.9, 0.4, 0.7, 1.0])
    psi, phi = oracle.psi_phi(sci, var, mask, psf)
    z = np.zeros(N, np.int32)
    P, F, nk, nr, rej = oracle.filter_lightcurve(psi, phi, times, z, z, 1, 1, 5.0)
    assert nr == 0 and nk == N and (P, F) == (18.0, 6.0)
    perm = np.array([3, 0, 6, 1, 5, 2, 4])
    r2 = oracle.filter_lightcurve(psi[perm], phi[perm], times[perm], z, z, 1, 1, 5.0)
    assert r2[:4] == (P, F, nk, nr)


# ------------------------------------------------------------ Sec. 3.3 postage stamps and moments

def test_moments_of_hand_stamps():
    """A single pixel of value 5 at (2, -1): m00 = 5, centroid (2, -1), no spread.  Two unit
    pixels at (-1, 0) and (1, 0): centroid 0, mu20 = 1, mu02 = mu11 = 0.  An empty stamp: zeros."""
    r = 3
    s = np.zeros((7, 7), np.float32)
    s[-1 + r, 2 + r] = 5.0
    assert oracle.moments(s) == (5.0, 2.0, -1.0, 0.0, 0.0, 0.0)
    s = np.zeros((7, 7), np.float32)
    s[r, r - 1] = s[r, r + 1] = 1.0
    assert oracle.moments(s) == (2.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    assert oracle.moments(np.zeros((5, 5), np.float32)) == (0.0,) * 6


def test_moments_over_an_aperture_by_hand():
    """Unit pixels at (-1, 0) and (1, 0) and 100 at (3, 3).  Aperture 2 leaves the 100 out (it is
    4.24 px from the centre): the moments of the pair.  Aperture 5 takes it: m00 = 102, centroid
    (50/17, 50/17) and, worked out by hand with the deviations -67/17, -33/17, 1/17 in x and
    -50/17, -50/17, 1/17 in y, mu20 = 5678/29478, mu02 = mu11 = 5100/29478."""
    r = 4
    s = np.zeros((9, 9), np.float32)
    s[r, r - 1] = s[r, r + 1] = 1.0
    s[r + 3, r + 3] = 100.0
    assert oracle.moments(s, 2.0) == (2.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    m = oracle.moments(s, 5.0)
    assert m[0] == 102.0
    assert m[1] == pytest.approx(50.0 / 17.0, rel=1e-14) and m[2] == pytest.approx(50.0 / 17.0, rel=1e-14)
    assert m[3] == pytest.approx(5678.0 / 29478.0, rel=1e-12)
    assert m[4] == pytest.approx(5100.0 / 29478.0, rel=1e-12)
    assert m[5] == pytest.approx(5100.0 / 29478.0, rel=1e-12)
    # an aperture at least the stamp's corner distance takes every pixel: aperture 0's moments
    assert oracle.moments(s, 6.0) == oracle.moments(s, 0.0)


def test_moments_of_a_gaussian_in_an_aperture_follow_the_truncated_closed_form():
    """A centred isotropic Gaussian of width sigma inside a disk of radius R: r^2 / (2 sigma^2)
    is exponential, so <x^2> = sigma^2 (1 - u e^-u / (1 - e^-u)) with u = R^2 / (2 sigma^2).
    The sampled Gaussian on the pixel grid (sigma = 4 px) follows it to 3.5 % (the disk of pixel
    centres is jagged at its edge, more so for small R); centroid and mu11 are zero by symmetry."""
    sigma, r = 4.0, 12
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    g = np.exp(-(xx ** 2 + yy ** 2) / (2 * sigma ** 2)).astype(np.float32)
    for R in (5.0, 8.0, 11.0):
        u = R * R / (2 * sigma ** 2)
        want = sigma ** 2 * (1.0 - u * math.exp(-u) / (1.0 - math.exp(-u)))
        m00, mx, my, mu20, mu02, mu11 = oracle.moments(g, R)
        assert abs(mx) < 1e-12 and abs(my) < 1e-12 and abs(mu11) < 1e-12
        assert mu20 == pytest.approx(want, rel=0.035) and mu02 == pytest.approx(mu20, rel=1e-12)


def _c1_like_stamp(rng, source, snr=2.5, r=10):
    """A mean stamp of 12 DECam-shaped epochs (variance 80-120, PSF FWHM 3.5-4.5 px) along a
    trajectory, with a source of per-epoch PSF-fit SNR `snr` moving exactly along it, or none.
    Returns the stamp and the epochs' PSF sigmas."""
    times = synth.decam_times()
    N, H, W, K = times.size, 96, 96, 17
    var_t = rng.uniform(80.0, 120.0, N)
    sig = rng.uniform(3.5, 4.5, N) / synth.FWHM_PER_SIGMA
    sci = (rng.standard_normal((N, H, W)) * np.sqrt(var_t)[:, None, None]).astype(np.float32)
    x0, y0 = rng.uniform(30.0, 34.0), rng.uniform(40.0, 44.0)
    speed, ang = rng.uniform(4.5, 27.5), rng.uniform(-math.pi / 4, math.pi / 4)
    vx, vy = speed * math.cos(ang), speed * math.sin(ang)
    if source:
        flux = snr * math.sqrt(4.0 * math.pi * float(np.mean(sig ** 2)) * float(np.mean(var_t)))
        for e in range(N):
            synth.render_source(sci[e], x0 + vx * times[e], y0 + vy * times[e], flux, sig[e], K // 2)
    dx, dy = oracle.offsets(times, np.array([vx]), np.array([vy]))
    st = oracle.stamp(sci, None, dx[0], dy[0], int(math.floor(x0 + 0.5)), int(math.floor(y0 + 0.5)), r)
    return st, sig


def psf_moment_cuts(sig, aperture):
    """Cuts of a centred PSF seen through the aperture: the truncated second moment of each
    epoch's Gaussian (closed form above) averaged, plus 1/12 px^2 of pixel rounding; the variances
    within [0.4, 1.8] of it, |mu11| within half of it, the centroid within 1 px."""
    u = aperture ** 2 / (2 * sig ** 2)
    v0 = float(np.mean(sig ** 2 * (1 - u * np.exp(-u) / (1 - np.exp(-u))))) + 1.0 / 12.0
    return {"max_offset": 1.0, "min_var": 0.4 * v0, "max_var": 1.8 * v0, "max_mu11": 0.5 * v0}


def _passes(m, c):
    m00, mx, my, mu20, mu02, mu11 = m
    return (m00 > 0 and abs(mx) <= c["max_offset"] and abs(my) <= c["max_offset"] and
            c["min_var"] <= mu20 <= c["max_var"] and c["min_var"] <= mu02 <= c["max_var"] and
            abs(mu11) <= c["max_mu11"])


def test_aperture_moment_filter_keeps_faint_sources_and_drops_noise():
    """Sec. 3.3 reading: moments over a 3 px aperture with cuts from the PSF widths.  Seeded
    DECam-like mean stamps: at least 90 % of sources of per-epoch SNR 2.5 on their trajectory
    pass, and at most 6 % of pure-noise stamps.  Over the whole 21 x 21 stamp (aperture 0) the
    same sources pass at most 20 % of the time: the sky noise of the outer pixels dominates."""
    rng = np.random.default_rng(31)
    src = [_c1_like_stamp(rng, True) for _ in range(150)]
    noise = [_c1_like_stamp(rng, False) for _ in range(150)]
    ok_src = np.mean([_passes(oracle.moments(st, 3.0), psf_moment_cuts(sig, 3.0)) for st, sig in src])
    ok_noise = np.mean([_passes(oracle.moments(st, 3.0), psf_moment_cuts(sig, 3.0)) for st, sig in noise])
    ok_whole = np.mean([_passes(oracle.moments(st, 0.0), psf_moment_cuts(sig, 20.0)) for st, sig in src])
    assert ok_src >= 0.9, ok_src
    assert ok_noise <= 0.06, ok_noise
    assert ok_whole <= 0.2, ok_whole


def _moving_gaussian_stack(N, H, W, sigma, x0, y0, dx, dy, amp=100.0):
    """A noiseless Gaussian of width sigma centred on the integer trajectory pixels."""
    yy, xx = np.mgrid[0:H, 0:W]
    sci = np.zeros((N, H, W), np.float32)
    for e in range(N):
        cx, cy = x0 + dx[e], y0 + dy[e]
        sci[e] = (amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sigma ** 2))).astype(np.float32)
    return sci


def test_stamp_of_a_noiseless_source_is_its_profile():
    """Every epoch's stamp is the same sampled Gaussian, so the mean and the median coadds are
    that Gaussian; its centroid is the stamp centre, mu11 = 0 and mu20 = mu02 = sigma^2 to the
    accuracy of a sampled, truncated Gaussian (r = 6 sigma)."""
    N, H, W, sigma, r = 5, 60, 80, 1.5, 9
    dx = np.array([0, 4, 9, 13, 18], np.int32)
    dy = np.array([0, -2, -5, -7, -9], np.int32)
    sci = _moving_gaussian_stack(N, H, W, sigma, 25, 40, dx, dy)
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    profile = (100.0 * np.exp(-(xx ** 2 + yy ** 2) / (2 * sigma ** 2))).astype(np.float32)
    for med in (False, True):
        st = oracle.stamp(sci, None, dx, dy, 25, 40, r, median=med)
        assert np.allclose(st, profile, rtol=1e-6, atol=1e-6)
    m00, mx, my, mu20, mu02, mu11 = oracle.moments(oracle.stamp(sci, None, dx, dy, 25, 40, r))
    assert abs(mx) < 1e-9 and abs(my) < 1e-9 and abs(mu11) < 1e-9
    assert mu20 == pytest.approx(sigma ** 2, rel=1e-4) and mu02 == pytest.approx(sigma ** 2, rel=1e-4)


def test_median_stamp_ignores_a_single_epoch_interloper():
    """A bright source off the trajectory in one of 5 epochs: the median coadd is unchanged, the
    mean carries a fifth of it (Sec. 3.3: the moment filter rejects off-centre light)."""
    N, H, W, sigma, r = 5, 60, 80, 1.2, 6
    dx = np.array([0, 3, 6, 9, 12], np.int32)
    dy = np.zeros(N, np.int32)
    sci = _moving_gaussian_stack(N, H, W, sigma, 20, 30, dx, dy)
    clean_mean = oracle.stamp(sci, None, dx, dy, 20, 30, r)
    sci[2, 30 + 3, 20 + dx[2] + 4] += 500.0           # interloper 4 px right, 3 px down in epoch 2
    med = oracle.stamp(sci, None, dx, dy, 20, 30, r, median=True)
    mean = oracle.stamp(sci, None, dx, dy, 20, 30, r)
    assert np.array_equal(med, clean_mean)            # all epochs agreed before: same values
    assert mean[3 + r, 4 + r] == pytest.approx(clean_mean[3 + r, 4 + r] + 100.0, rel=1e-5)
    # by linearity: the clean stamp is centred, so the mean's centroid moves to 4 * 100 / (m00 + 100)
    m00 = float(np.sum(clean_mean, dtype=np.float64))
    assert oracle.moments(mean)[1] == pytest.approx(400.0 / (m00 + 100.0), rel=1e-5)
    assert oracle.moments(mean)[2] == pytest.approx(300.0 / (m00 + 100.0), rel=1e-5)
    assert abs(oracle.moments(med)[1]) < 1e-9


def test_stamp_skips_masked_nan_and_outside_pixels():
    """Masked or NaN pixels, and stamp pixels off the image, are left out of the coadd; a
    stamp pixel no epoch covers is 0; the median of an even count is the mean of the two
    middle values."""
    N, H, W = 4, 10, 10
    sci = np.zeros((N, H, W), np.float32)
    sci[:, 5, 5] = [1.0, 2.0, 10.0, 40.0]
    mask = np.zeros((N, H, W), np.uint8)
    mask[3, 5, 5] = 1                                  # drops the 40
    sci[2, 4, 5] = np.nan                              # a NaN above the centre in epoch 2
    z = np.zeros(N, np.int32)
    st = oracle.stamp(sci, mask, z, z, 5, 5, 1)
    assert st[1, 1] == pytest.approx(13.0 / 3.0)       # mean of 1, 2, 10
    med = oracle.stamp(sci, mask, z, z, 5, 5, 1, median=True)
    assert med[1, 1] == 2.0
    sci[1, 5, 5] = 4.0
    med = oracle.stamp(sci, mask, np.zeros(N, np.int32), z, 5, 5, 1, median=True)
    assert med[1, 1] == 4.0                            # middle of 1, 4, 10
    mask[2, 5, 5] = 1
    med = oracle.stamp(sci, mask, z, z, 5, 5, 1, median=True)
    assert med[1, 1] == 2.5                            # two values left: (1 + 4) / 2
    corner = oracle.stamp(sci, None, z, z, 0, 0, 2)
    assert np.all(corner[:2, :] == 0.0) and np.all(corner[:, :2] == 0.0)


# ------------------------------------------------------------ Sec. 3.3 DBSCAN de-duplication

def _hand_clusters():
    """Two clusters in velocity space (start pixel 0, w_vel = 1, eps = 1, min_samples = 4), each with
    one core point (a0 = (0, 0), b0 = (1.9, 0)) and three border points; p = (0.95, 0) lies at
    exactly the same distance 0.95 from both cores (float(1.9) = 2 float(0.95)) with only 3
    neighbours; q is noise; an empty slot (vidx -1) lies next to p."""
    v = [(0.0, 0.0), (-0.9, 0.0), (-0.5, 0.8), (-0.3, -0.9),          # A: a0..a3, indices 0-3
         (1.9, 0.0), (2.8, 0.0), (2.4, 0.8), (2.2, -0.9),             # B: b0..b3, indices 4-7
         (0.95, 0.0),                                                 # p, index 8
         (10.0, 10.0),                                                # q, index 9
         (0.95, 0.05)]                                                # empty slot, index 10
    vx = np.array([a for a, _ in v], np.float32)
    vy = np.array([b for _, b in v], np.float32)
    n = len(v)
    nu = np.arange(n, dtype=np.float64)
    nu[8] = 100.0                                      # p is A's best member
    vidx = np.zeros(n, np.int32)
    vidx[10] = -1
    return np.zeros(n, np.int32), np.zeros(n, np.int32), vx, vy, nu, vidx


def test_cluster_hand_example():
    x0, y0, vx, vy, nu, vidx = _hand_clusters()
    label, keep, core = oracle.cluster(x0, y0, vx, vy, nu, vidx, 1.0, 1.0, 1.0, 4)
    assert list(np.nonzero(core)[0]) == [0, 4]          # a0 has a1, a2, a3, p; b0 likewise
    # p ties between a0 and b0: the lower core index wins
    assert list(label) == [0, 0, 0, 0, 4, 4, 4, 4, 0, 9, -1]
    assert list(np.nonzero(keep)[0]) == [7, 8, 9]        # B's best is b3 (nu 7), A's is p, q alone
    # moved towards b0, p joins B
    vx2 = vx.copy()
    vx2[8] = np.float32(0.96)
    label2, _, _ = oracle.cluster(x0, y0, vx2, vy, nu, vidx, 1.0, 1.0, 1.0, 4)
    assert label2[8] == 4
    # the empty slot would have made p a core point (and merged A and B) had it counted
    vidx2 = vidx.copy()
    vidx2[10] = 3
    label3, _, core3 = oracle.cluster(x0, y0, vx, vy, nu, vidx2, 1.0, 1.0, 1.0, 4)
    assert core3[8] and label3[4] == 0 and label3[8] == 0


def _clumps(rng, n_clumps, per, spread_px, spread_v, n_noise, W=500, V=300.0):
    """Candidates around clump centres (start pixel, velocity) plus scattered ones."""
    x0, y0, vx, vy = [], [], [], []
    for _ in range(n_clumps):
        cx, cy = rng.integers(0, W, 2)
        cu, cv = rng.uniform(-V, V, 2)
        m = int(rng.integers(1, per + 1))
        x0 += list(np.clip(cx + rng.integers(-spread_px, spread_px + 1, m), 0, W - 1))
        y0 += list(np.clip(cy + rng.integers(-spread_px, spread_px + 1, m), 0, W - 1))
        vx += list(cu + rng.normal(0, spread_v, m))
        vy += list(cv + rng.normal(0, spread_v, m))
    x0 += list(rng.integers(0, W, n_noise))
    y0 += list(rng.integers(0, W, n_noise))
    vx += list(rng.uniform(-V, V, n_noise))
    vy += list(rng.uniform(-V, V, n_noise))
    n = len(x0)
    return (np.array(x0, np.int32), np.array(y0, np.int32), np.array(vx, np.float32), np.array(vy, np.float32),
            rng.normal(5.0, 2.0, n), np.where(rng.random(n) < 0.02, -1, 1).astype(np.int32))


def _scaled(x0, y0, vx, vy, w_pos, w_vel):
    return np.stack([x0.astype(np.float64) * w_pos, y0.astype(np.float64) * w_pos,
                     vx.astype(np.float64) * w_vel, vy.astype(np.float64) * w_vel], axis=1)


@pytest.mark.parametrize("min_samples", [2, 3, 5])
def test_cluster_against_sklearn_dbscan(min_samples):
    """Core points, the partition of core points and the noise set equal scikit-learn's DBSCAN on
    the weighted features; border points sit in a cluster that has a core point within eps."""
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(40 + min_samples)
    x0, y0, vx, vy, nu, vidx = _clumps(rng, 120, 12, 3, 4.0, 300)
    w_pos, w_vel, eps = 1.0, 0.5, 4.0
    label, keep, core = oracle.cluster(x0, y0, vx, vy, nu, vidx, w_pos, w_vel, eps, min_samples)
    ok = vidx >= 0
    feats = _scaled(x0, y0, vx, vy, w_pos, w_vel)[ok]
    db = sk.DBSCAN(eps=eps, min_samples=min_samples).fit(feats)
    idx = np.nonzero(ok)[0]
    sk_core = np.zeros(x0.size, bool)
    sk_core[idx[db.core_sample_indices_]] = True
    assert np.array_equal(core, sk_core)
    assert np.all(label[~ok] == -1) and not keep[~ok].any()
    sk_label = np.full(x0.size, -2)
    sk_label[idx] = db.labels_
    # the same partition of the core points
    pairs = {}
    for i in np.nonzero(core)[0]:
        assert pairs.setdefault(label[i], sk_label[i]) == sk_label[i]
    assert len(set(pairs.values())) == len(pairs)
    # noise: sklearn's -1 exactly where a point is its own group without being core
    own = ok & ~core & (label == np.arange(x0.size))
    assert np.array_equal(own, sk_label == -1)
    # border points: in a cluster with a core point within eps
    d2 = lambda i, j: float(np.sum((feats[np.searchsorted(idx, i)] - feats[np.searchsorted(idx, j)]) ** 2))
    for i in np.nonzero(ok & ~core & ~own)[0]:
        members = np.nonzero(core & (label == label[i]))[0]
        assert min(d2(i, j) for j in members) <= eps * eps * (1 + 1e-12)
    assert 10 < len(pairs) and own.sum() > 10
    if min_samples > 2:                              # with 2, every point with a neighbour is core
        assert (ok & ~core & ~own).sum() > 10


def test_cluster_min_samples_one_is_connected_components():
    """With min_samples = 1 every candidate is core and the groups are the connected components of
    the eps-neighbour graph (scipy), each labelled by its lowest index."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(41)
    x0, y0, vx, vy, nu, _ = _clumps(rng, 80, 10, 2, 1.0, 150)
    vidx = np.zeros(x0.size, np.int32)
    w_pos, w_vel, eps = 0.5, 1.0, 3.0
    label, keep, core = oracle.cluster(x0, y0, vx, vy, nu, vidx, w_pos, w_vel, eps, 1)
    assert core.all()
    f = _scaled(x0, y0, vx, vy, w_pos, w_vel)
    ncomp, comp = connected_components(csr_matrix(cdist(f, f) <= eps), directed=False)
    for c in range(ncomp):
        members = np.nonzero(comp == c)[0]
        assert np.all(label[members] == members.min())
        best = members[np.lexsort((members, -nu[members]))[0]]
        assert list(np.nonzero(keep[members])[0]) == [list(members).index(best)]
    assert ncomp < x0.size // 2


def test_cluster_permutation_relabels_consistently():
    rng = np.random.default_rng(42)
    x0, y0, vx, vy, nu, vidx = _clumps(rng, 60, 10, 3, 4.0, 100)
    args = (1.0, 0.5, 4.0, 3)
    label, keep, core = oracle.cluster(x0, y0, vx, vy, nu, vidx, *args)
    p = rng.permutation(x0.size)
    l2, k2, c2 = oracle.cluster(x0[p], y0[p], vx[p], vy[p], nu[p], vidx[p], *args)
    assert np.array_equal(c2, core[p]) and np.array_equal(k2, keep[p])
    # same groups: candidates share a label after permuting iff they did before (core points;
    # border points may choose another cluster only on an exact distance tie, absent here)
    for a, b in [(label, l2[np.argsort(p)])]:
        m = {}
        for u, w in zip(a, b):
            assert m.setdefault(u, w) == w


def test_elongated_psfs_are_normalised_and_not_separable():
    """The bench's non-separable PSFs: unit sum, the Gaussian's major-axis width kept, and a
    second singular value far above rounding (so the single-pass path is exercised)."""
    import synth
    base = np.stack([synth.gaussian_psf(17, s) for s in (1.5, 1.7, 1.9)])
    el = synth.elongate_psfs(base, seed=3)
    for e in range(3):
        p = el[e].astype(np.float64)
        assert abs(p.sum() - 1.0) < 1e-6
        sv = np.linalg.svd(p, compute_uv=False)
        assert sv[1] / sv[0] > 1e-4
        # the largest second moment along any axis is the base width (sampled, truncated at 8 px)
        d = np.arange(-8, 9, dtype=np.float64)
        yy, xx = np.meshgrid(d, d, indexing="ij")
        cov = np.array([[np.sum(p * xx * xx), np.sum(p * xx * yy)], [np.sum(p * xx * yy), np.sum(p * yy * yy)]])
        sig = math.sqrt(float(np.sum(base[e].astype(np.float64).sum(axis=0) * d ** 2)))
        assert np.linalg.eigvalsh(cov).max() == pytest.approx(sig ** 2, rel=2e-3)


# ------------------------------------------------------------ Sec. 5.3 likelihood bound over a span

def _traj_sums(psi, phi, dxv, dyv, x, y):
    N, H, W = psi.shape
    P = F = 0.0
    for t in range(N):
        xx, yy = x + dxv[t], y + dyv[t]
        if 0 <= xx < W and 0 <= yy < H:
            P += psi[t, yy, xx]
            F += phi[t, yy, xx]
    return P, F


@pytest.mark.parametrize("span", [1, 7, 64])
def test_span_bound_exceeds_every_nu_in_the_span(span):
    """Brute force on a masked noise stack with a source: for random rows, span starts (also
    partly off the image) and velocities, the bound is at least nu^2 of every trajectory of the
    span with Psi > 0."""
    st = synth.small_stack(71, 6, 40, 90, K=5, var_lo=1.0, var_hi=3.0, nan_frac=0.02, mask_frac=0.02,
                           n_angles=6, n_speeds=5, s_lo=2.0, s_hi=15.0, n_sources=2, flux=30.0)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    N, H, W = psi.shape
    r = oracle.snr2_span_max(psi, phi, span)
    rng = np.random.default_rng(span)
    checked = 0
    for _ in range(150):
        v = int(rng.integers(0, dx.shape[0]))
        y0 = int(rng.integers(0, H))
        x0 = int(rng.integers(-span + 1, W))
        b = oracle.span_bound(r, W, span, dx[v], dy[v], x0, y0)
        for x in range(max(x0, 0), min(x0 + span, W)):
            P, F = _traj_sums(psi, phi, dx[v], dy[v], x, y0)
            if P > 0 and F > 0:
                assert P * P / F <= b * (1 + 1e-12), (v, x, y0, P * P / F, b)
                checked += 1
    assert checked > 40


def test_span_bound_is_tight_for_a_noiseless_source():
    """Equality in Cauchy-Schwarz: psi_t / phi_t the same for every epoch (a noiseless source on
    its own trajectory, unit variance, one PSF) gives bound = nu^2 with a one-pixel span."""
    N, H, W = 5, 40, 60
    times = np.array([0.0, 0.5, 1.0, 1.5, 2.0])
    vx, vy = np.array([6.0]), np.array([-4.0])
    dx, dy = oracle.offsets(times, vx, vy)
    psf = np.stack([synth.gaussian_psf(5, 1.0)] * N)
    sci = np.zeros((N, H, W), np.float32)
    for t in range(N):
        sci[t, 25 + dy[0, t], 12 + dx[0, t]] = 16.0          # a delta at the trajectory pixel
    var = np.ones((N, H, W), np.float32)
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    r = oracle.snr2_span_max(psi, phi, 1)
    P, F = _traj_sums(psi, phi, dx[0], dy[0], 12, 25)
    assert oracle.span_bound(r, W, 1, dx[0], dy[0], 12, 25) == pytest.approx(P * P / F, rel=1e-12)
    # a single epoch and a one-pixel span: the bound is that pixel's psi^2 / phi
    r1 = oracle.snr2_span_max(psi[:1], phi[:1], 1)
    assert oracle.span_bound(r1, W, 1, dx[0, :1], dy[0, :1], 12, 25) == pytest.approx(
        psi[0, 25, 12] ** 2 / phi[0, 25, 12], rel=1e-15)


def test_span_bound_of_pure_noise_prunes_at_ten_sigma():
    """Unit-variance noise, no source: every 64-pixel span's bound stays below 10^2 (the single-
    epoch SNRs are N(0, 1), so each epoch's span maximum is a few units)."""
    rng = np.random.default_rng(72)
    N, H, W = 12, 24, 256
    sci = rng.standard_normal((N, H, W)).astype(np.float32)
    var = np.ones((N, H, W), np.float32)
    psf = np.stack([synth.gaussian_psf(7, 1.3)] * N)
    psi, phi = oracle.psi_phi(sci, var, None, psf)
    r = oracle.snr2_span_max(psi, phi, 64)
    times = np.linspace(0.0, 2.0, N)
    dx, dy = oracle.offsets(times, np.array([20.0, -35.0]), np.array([3.0, 8.0]))
    worst = max(oracle.span_bound(r, W, 64, dx[v], dy[v], x0, y0)
                for v in range(2) for y0 in range(H) for x0 in range(-63, W, 32))
    assert worst < 100.0
