"""Pins for the FP64 oracle: facts the paper and the mathematics fix, checked
without re-typing the oracle's own formulas.

Each test names the passage it rests on (section / equation of arXiv
1807.11534, or the cited method it reduces to).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1807_11534_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- operators

@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (6, 1), (5, 9), (17, 4)])
def test_div_is_minus_adjoint_of_grad(orc, shape):
    """Chambolle (2004) operators (cited in Section 2.1): <grad w, p> = -<w, div p>."""
    rng = np.random.default_rng(1)
    w = rng.normal(size=shape)
    p1, p2 = rng.normal(size=shape), rng.normal(size=shape)
    g1, g2 = orc.grad(w)
    d = orc.div(p1, p2)
    lhs = float(np.sum(g1 * p1) + np.sum(g2 * p2))
    rhs = -float(np.sum(w * d))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_grad_div_textbook_values(orc):
    """Forward differences with Neumann boundary: a ramp in i has gradient
    (1, 0) except on the last row; a constant unit field p1 has divergence
    +1 on the first row, 0 inside, -1 on the last row."""
    H, W = 5, 4
    ramp = np.repeat(np.arange(H, dtype=float)[:, None], W, axis=1)
    g1, g2 = orc.grad(ramp)
    exp1 = np.ones((H, W)); exp1[-1] = 0
    np.testing.assert_array_equal(g1, exp1)
    np.testing.assert_array_equal(g2, np.zeros((H, W)))
    d = orc.div(np.ones((H, W)), np.zeros((H, W)))
    exp = np.zeros((H, W)); exp[0] = 1; exp[-1] = -1
    np.testing.assert_array_equal(d, exp)
    d = orc.div(np.zeros((H, W)), np.ones((H, W)))
    exp = np.zeros((H, W)); exp[:, 0] = 1; exp[:, -1] = -1
    np.testing.assert_array_equal(d, exp)


# ----------------------------------------------------------------- fitting

def test_cv_term_is_affine_in_z(orc):
    """Eq. CV expands to f = 2 z (c2 - c1) + c1^2 - c2^2; for c1 = .3, c2 = .7
    this is 0.8 z - 0.4."""
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 2, (13, 11)).astype(np.float32)
    f64, f32 = orc.fitting(z, 0.3, 0.7)
    np.testing.assert_allclose(f64, 0.8 * z.astype(np.float64) - 0.4, atol=1e-14)
    assert f32.dtype == np.float32
    np.testing.assert_array_equal(f32, f64.astype(np.float32))
    # the sign decides the phase: f < 0 iff z is closer to c1
    assert np.all((f64 < 0) == (np.abs(z - 0.3) < np.abs(z - 0.7)))


def test_ds_term_distance_properties(orc):
    """Eq. DS: f = CV + gamma P, P the normalised distance to the markers:
    P = 0 on a marker, max P = 1, and on one row with a marker at column 0
    P(j) = j / (W-1)."""
    H, W = 1, 9
    z = np.full((H, W), 0.5, np.float32)  # CV = 0 at z = (c1+c2)/2
    f64, _ = orc.fitting(z, 0.3, 0.7, markers=np.array([[0, 0]]), gamma=2.0)
    np.testing.assert_allclose(f64[0], 2.0 * np.arange(W) / (W - 1), atol=1e-15)
    rng = np.random.default_rng(3)
    H, W = 20, 31
    m = np.stack([rng.integers(0, H, 5), rng.integers(0, W, 5)], 1)
    z = np.full((H, W), 0.5, np.float32)
    f64, _ = orc.fitting(z, 0.3, 0.7, markers=m, gamma=1.0)
    assert np.all(np.abs(f64[m[:, 0], m[:, 1]]) < 1e-15)
    assert abs(f64.max() - 1.0) < 1e-15
    # brute force on the distance itself
    yy, xx = np.mgrid[0:H, 0:W]
    dist = np.min(np.hypot(yy[..., None] - m[:, 0], xx[..., None] - m[:, 1]), axis=-1)
    np.testing.assert_allclose(f64, dist / dist.max(), atol=1e-14)


def test_class_means_match_numpy(orc):
    rng = np.random.default_rng(4)
    z = rng.normal(size=(40, 50)).astype(np.float32)
    lab = (rng.random((40, 50)) < 0.3).astype(np.uint8)
    c1, c2 = orc.class_means(z, lab)
    assert abs(c1 - z[lab == 1].astype(np.float64).mean()) < 1e-13
    assert abs(c2 - z[lab == 0].astype(np.float64).mean()) < 1e-13


# ------------------------------------------------------------------ domain

@pytest.mark.parametrize("q", [0.0, 0.013, 0.25, 0.5, 0.97, 1.0])
def test_quantile_delta_is_minimal_by_brute_force(orc, q):
    """Section 3: q-hat grows from 0 until the RD fraction reaches q.  Brute
    force: |RD(q-hat)| >= ceil(qn), and the next smaller threshold misses it."""
    rng = np.random.default_rng(5)
    f = rng.normal(0, 0.2, 500).astype(np.float32)
    f[::7] = f[3]  # ties
    delta = orc.quantile_delta(f, q)
    k = math.ceil(q * f.size)
    cnt = int(np.sum(np.abs(f) < np.float32(delta)))
    assert cnt >= k
    if k > 0:
        below = np.nextafter(np.float32(delta), np.float32(0))
        assert int(np.sum(np.abs(f) < below)) < k
    else:
        assert delta == 0.0 and cnt == 0


def test_domain_special_cases(orc):
    """Section 3: q = 0 gives RD empty (zero-thresholding of f); q = 1 gives
    Fg = Bg = empty (the conventional problem)."""
    rng = np.random.default_rng(6)
    f = rng.normal(0, 1, (9, 14)).astype(np.float32)
    f[0, 0] = 0.0
    reg0 = orc.domain(f, 0.0)
    assert not np.any(reg0 == 2)
    np.testing.assert_array_equal(reg0 == 1, f < 0)   # u0 = H(-f): f = 0 is background
    reg1 = orc.domain(f, np.inf)
    assert np.all(reg1 == 2)
    d = orc.quantile_delta(f, 1.0)
    assert np.all(orc.domain(f, d) == 2)


def test_pixel_and_tile_lists_brute_force(orc):
    rng = np.random.default_rng(7)
    f = rng.normal(0, 1, (37, 70)).astype(np.float32)
    reg = orc.domain(f, 0.2)
    pl = orc.pixel_list(reg)
    np.testing.assert_array_equal(pl, np.flatnonzero(reg.ravel() == 2))
    th, tw = 8, 32
    tl = orc.tile_list(reg, th, tw)
    ntx = -(-70 // tw)
    exp = [ty * ntx + tx for ty in range(-(-37 // th)) for tx in range(ntx)
           if np.any(reg[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw] == 2)]
    np.testing.assert_array_equal(tl, np.array(exp, np.int32))
    # tile-major numbering: same set as the row-major list, grouped by tile
    pt = orc.pixel_list_tiled(reg, th, tw)
    np.testing.assert_array_equal(np.sort(pt), pl)
    key = (pt // 70 // th) * ntx + (pt % 70) // tw
    assert np.all(np.diff(key) >= 0)
    for t in np.unique(key):
        seg_ = pt[key == t]
        assert np.all(np.diff(seg_) > 0)


# ------------------------------------------------------------------ solver

def _numpy_bresson_full(f, lam, theta, tau, iters):
    """The original, unrestricted dual iteration (Section 2.1) written
    independently with numpy slicing: no region logic at all."""
    f = f.astype(np.float64)
    u = (f < 0).astype(np.float64)
    p1 = np.zeros_like(u); p2 = np.zeros_like(u)
    v = np.clip(u - theta * lam * f, 0, 1)

    def dv(a, b):
        d = np.zeros_like(a)
        d[:-1, :] += a[:-1, :]; d[1:, :] -= a[:-1, :]
        d[:, :-1] += b[:, :-1]; d[:, 1:] -= b[:, :-1]
        return d

    for _ in range(iters):
        w = dv(p1, p2) - v / theta
        g1 = np.zeros_like(w); g1[:-1] = w[1:] - w[:-1]
        g2 = np.zeros_like(w); g2[:, :-1] = w[:, 1:] - w[:, :-1]
        den = 1 + tau * np.sqrt(g1 * g1 + g2 * g2)
        p1 = (p1 + tau * g1) / den; p2 = (p2 + tau * g2) / den
        u = v - theta * dv(p1, p2)
        v = np.clip(u - theta * lam * f, 0, 1)
    return u, v, p1, p2


def test_unrestricted_domain_is_the_original_method(orc):
    """Section 3: for q = 1 the restricted method is the conventional one."""
    P = synth.small_example(seed=0, H=40, W=52)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    st = orc.solve(f, orc.domain(f, np.inf), 1.0, 0.2, 0.125, iters=60)
    u, v, p1, p2 = _numpy_bresson_full(f, 1.0, 0.2, 0.125, 60)
    for a, b in ((st.u, u), (st.v, v), (st.p1, p1), (st.p2, p2)):
        np.testing.assert_allclose(a, b, atol=1e-12, rtol=0)


def test_empty_domain_is_zero_thresholding(orc):
    """Section 3: q = 0 gives the zero-thresholding of the fitting term:
    u = v = H(-f), rho = 0, and no increment."""
    P = synth.small_example(seed=1, H=33, W=45)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    st = orc.solve(f, orc.domain(f, 0.0), 1.0, iters=5)
    h = (f < 0).astype(np.float64)
    np.testing.assert_array_equal(st.u, h)
    np.testing.assert_array_equal(st.v, h)
    assert not st.p1.any() and not st.p2.any()
    assert np.all(st.hist == 0)


@pytest.mark.parametrize("delta", [0.05, 0.15, np.inf])
def test_dual_field_and_v_stay_feasible(orc, delta):
    """The fixed-point step keeps |rho| <= 1 (its denominator dominates the
    numerator once |rho^n| <= 1) and the v-step keeps v in [0, 1]."""
    P = synth.small_example(seed=2, H=48, W=40)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, delta)
    st = None
    for _ in range(4):
        st = orc.solve(f, reg, 1.0, iters=25, state=st)
        nrm = np.sqrt(st.p1 ** 2 + st.p2 ** 2)
        assert nrm.max() <= 1 + 1e-12
        assert st.v.min() >= 0 and st.v.max() <= 1
        assert np.all(st.p1[reg != 2] == 0) and np.all(st.p2[reg != 2] == 0)
        assert np.all(st.u[reg == 1] == 1) and np.all(st.u[reg == 0] == 0)


def test_large_lambda_gives_heaviside(orc):
    """Section 1: for large lambda the solution is f < 0 foreground, f > 0
    background.  With |rho| <= 1, |div rho| <= 4, so once
    theta lambda |f| >= 1 + 4 theta the v-step returns H(-f) exactly."""
    rng = np.random.default_rng(8)
    f = rng.uniform(0.05, 1.0, (30, 30)) * rng.choice([-1, 1], (30, 30))
    f = f.astype(np.float32)
    theta = 0.2
    lam = (1 + 4 * theta) / (theta * 0.05) * 1.01
    st = orc.solve(f, orc.domain(f, np.inf), lam, theta, 0.125, iters=40)
    np.testing.assert_array_equal(st.v, (f < 0).astype(np.float64))


@pytest.mark.slow
@pytest.mark.parametrize("r", [8, 12])
def test_disk_closed_form(orc, r):
    """f = -1 inside a disk of radius r, +1 outside (Chan-Esedoglu-Nikolova,
    the model Section 2 relaxes): the disk costs 2 pi r - lambda pi r^2 and
    any sub-disk is worse than one of the two ends, so the minimiser is empty
    for lambda < 2/r and the disk for lambda > 2/r."""
    n = 2 * r + 16
    f, inside = synth.disk_fitting(n, n, r)
    reg = orc.domain(f, np.inf)
    lam_c = 2.0 / r
    st = orc.solve(f, reg, 0.5 * lam_c, iters=3000, tol=1e-7)
    assert st.u.max() < 0.5 and st.v.max() < 0.5
    st = orc.solve(f, reg, 5.0 * lam_c, iters=3000, tol=1e-7)
    np.testing.assert_array_equal(st.u > 0.5, inside)


def test_rof_subproblem_matches_bounded_least_squares(orc):
    """The rho fixed point solves min_u TV(u) + ||u - v||^2/(2 theta)
    (Chambolle 2004; the u-equation of Section 2.1).  For v constant along
    columns this is 1-D TV denoising with weight theta, whose dual is a
    box-constrained least-squares problem solved here by scipy's BVLS."""
    lsq_linear = pytest.importorskip("scipy.optimize").lsq_linear
    rng = np.random.default_rng(9)
    H, W, theta = 20, 3, 0.2
    s = np.clip(np.repeat([0.2, 0.9, 0.4, 0.6], 5) + rng.normal(0, 0.1, H), 0, 1)
    v = np.repeat(s[:, None], W, axis=1)
    f = np.zeros((H, W), np.float32)
    reg = np.full((H, W), 2, np.uint8)
    z0 = np.zeros((H, W))
    st = orc.solve(f, reg, 0.0, theta, 0.125, iters=1, n_inner=60000,
                   state=orc.State(v.copy(), v.copy(), z0, z0, 0, np.zeros((0, 2))))
    D = np.diff(np.eye(H), axis=0)                     # (H-1) x H forward difference
    res = lsq_linear(D.T, s, bounds=(-theta, theta), method="bvls", tol=1e-14)
    x = s - D.T @ res.x
    for j in range(W):
        np.testing.assert_allclose(st.u[:, j], x, atol=2e-6)


def _smoothed_min(f, lam, theta, eps, relaxed_only=False):
    """Independent minimiser (scipy L-BFGS-B) of the Eq. DF energy (or of
    Eq. CR when relaxed_only) with TV smoothed as sqrt(a^2 + b^2 + e^2),
    e lowered by continuation from 1e-2 down to `eps`."""
    minimize = pytest.importorskip("scipy.optimize").minimize
    H, W = f.shape
    N = H * W
    f = f.astype(np.float64).ravel()

    def tv_and_grad(u, e):
        u = u.reshape(H, W)
        a = np.zeros_like(u); a[:-1] = u[1:] - u[:-1]
        b = np.zeros_like(u); b[:, :-1] = u[:, 1:] - u[:, :-1]
        r = np.sqrt(a * a + b * b + e * e)
        ga, gb = a / r, b / r
        g = np.zeros_like(u)
        g[1:] += ga[:-1]; g[:-1] -= ga[:-1]
        g[:, 1:] += gb[:, :-1]; g[:, :-1] -= gb[:, :-1]
        return r.sum(), g.ravel()

    if relaxed_only:
        def obj(x, e):
            t, g = tv_and_grad(x, e)
            return t + lam * np.dot(f, x), g + lam * f
        x = np.full(N, 0.5)
        bounds = [(0, 1)] * N
    else:
        def obj(x, e):
            u, v = x[:N], x[N:]
            t, g = tv_and_grad(u, e)
            dq = (u - v) / theta
            val = t + 0.5 * np.dot(u - v, u - v) / theta + lam * np.dot(f, v)
            return val, np.concatenate([g + dq, -dq + lam * f])
        x = np.full(2 * N, 0.5)
        bounds = [(None, None)] * N + [(0, 1)] * N
    e = 1e-2
    while True:
        res = minimize(obj, x, args=(e,), jac=True, method="L-BFGS-B", bounds=bounds,
                       options=dict(maxiter=200000, maxfun=400000, ftol=1e-16, gtol=1e-13,
                                    maxcor=50))
        x = res.x
        if e <= eps:
            break
        e = max(eps, e / 10)
    if relaxed_only:
        return res.fun, x.reshape(H, W)
    return res.fun, x[:N].reshape(H, W), x[N:].reshape(H, W)


@pytest.mark.parametrize("seed,lam", [(0, 2.0), (1, 4.0)])
def test_iteration_reaches_the_df_minimum(orc, seed, lam):
    """Section 2.1: alternating the u- and v-minimisations minimises Eq. DF.
    The converged oracle energy must equal an independent L-BFGS-B minimum of
    the (slightly smoothed) Eq. DF energy on a tiny image with an edge."""
    rng = np.random.default_rng(10 + seed)
    blk = np.zeros((5, 6), bool)
    blk[1:4, 1 + seed:4 + seed] = True
    f = (np.where(blk, -0.5, 0.5) + rng.normal(0, 0.3, (5, 6))).astype(np.float32)
    theta, eps = 0.2, 1e-7
    st = orc.solve(f, orc.domain(f, np.inf), lam, theta, 0.125, iters=40000, tol=1e-13)
    e = orc.energy(st.u, st.v, st.p1, st.p2, f, lam, theta)
    assert e["tv"] > 0.5                      # the solution has an edge
    emin, _, _ = _smoothed_min(f, lam, theta, eps)
    # smoothing only raises the energy (by at most N eps), and the iteration
    # cannot beat the true minimum: E_DF(oracle) >= emin - N eps
    assert e["edf"] >= emin - 30 * eps - 1e-9
    assert abs(e["edf"] - emin) <= 1e-5 * max(1.0, abs(emin))


def _restricted_min(f, region, lam, theta, eps):
    """Independent minimiser (scipy L-BFGS-B, TV smoothed by continuation as
    in _smoothed_min) of the energy whose alternating minimisation is the
    restricted iteration of Section 3:

        E_R(u, v) = sum_{x in RD} |grad u(x)| + (1/2 theta) sum_{all x} (u - v)^2
                    + lambda sum_{x in RD} f v,

    with v = H(-f) held on Fg and Bg, v in [0, 1] on RD, and u free at every
    pixel.  rho = 0 off RD keeps only RD's |grad u| terms (the dual of
    sum_RD |grad u| is <u, div rho> over rho supported on RD), and the rho
    equation evaluated at RD points reads theta div rho - v at fixed
    neighbours too, so the u of this energy off RD is v - theta div rho, an
    auxiliary value the method never reports (it reports the fixed 0 / 1
    there).  Returns (min, u, v)."""
    minimize = pytest.importorskip("scipy.optimize").minimize
    H, W = f.shape
    N = H * W
    rdm = region == 2
    rd = rdm.ravel()
    nr = int(rd.sum())
    vfix = (region == 1).astype(np.float64).ravel()
    fr = f.astype(np.float64).ravel()[rd]

    def obj(x, e):
        u = x[:N].reshape(H, W)
        v = vfix.copy()
        v[rd] = x[N:]
        a = np.zeros_like(u); a[:-1] = u[1:] - u[:-1]
        b = np.zeros_like(u); b[:, :-1] = u[:, 1:] - u[:, :-1]
        r = np.sqrt(a * a + b * b + e * e)
        ga = np.where(rdm, a / r, 0.0)
        gb = np.where(rdm, b / r, 0.0)
        g = np.zeros_like(u)
        g[1:] += ga[:-1]; g[:-1] -= ga[:-1]
        g[:, 1:] += gb[:, :-1]; g[:, :-1] -= gb[:, :-1]
        d = x[:N] - v
        val = r[rdm].sum() + 0.5 * np.dot(d, d) / theta + lam * np.dot(fr, x[N:])
        return val, np.concatenate([g.ravel() + d / theta, -d[rd] / theta + lam * fr])

    x = np.concatenate([vfix, np.full(nr, 0.5)])
    bounds = [(None, None)] * N + [(0, 1)] * nr
    e = 1e-2
    while True:
        res = minimize(obj, x, args=(e,), jac=True, method="L-BFGS-B", bounds=bounds,
                       options=dict(maxiter=200000, maxfun=400000, ftol=1e-16, gtol=1e-13,
                                    maxcor=50))
        x = res.x
        if e <= eps:
            break
        e = max(eps, e / 10)
    v = vfix.copy()
    v[rd] = x[N:]
    return res.fun, x[:N].reshape(H, W), v.reshape(H, W)


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("delta", [0.1, 0.3])
def test_restricted_iteration_reaches_the_restricted_minimum(orc, seed, delta):
    """Section 3 for 0 < q-hat < inf: at convergence the restricted iterate
    (u, v on RD) is the minimiser of E_R (see _restricted_min), found
    independently by L-BFGS-B.  RD pixels here border fixed Fg and Bg
    pixels on every side, so how a fixed neighbour enters the rho step (its
    v, its div rho) and which |grad u| terms count are all exercised."""
    rng = np.random.default_rng(20 + seed)
    H, W = 8, 9
    blk = np.zeros((H, W), bool)
    blk[2:6, 2 + seed:6 + seed] = True
    f = (np.where(blk, -0.4, 0.4) + rng.normal(0, 0.25, (H, W))).astype(np.float32)
    reg = orc.domain(f, delta)
    rd = reg == 2
    assert 4 <= rd.sum() <= H * W // 2 and (reg == 1).any() and (reg == 0).any()
    theta, lam, eps = 0.2, 2.0, 1e-7
    st = orc.solve(f, reg, lam, theta, 0.125, iters=100000, tol=1e-13)
    assert st.iters_done < 100000
    emin, um, vm = _restricted_min(f, reg, lam, theta, eps)
    np.testing.assert_allclose(st.u[rd], um[rd], rtol=0, atol=2e-5)
    np.testing.assert_allclose(st.v[rd], vm[rd], rtol=0, atol=2e-5)
    # E_R at the oracle's state (u off RD: the auxiliary v - theta div rho,
    # with div written here by its definition as minus the adjoint of the
    # forward difference): not below the smoothed minimum by more than the
    # smoothing's N_RD eps, and not above it
    d = np.zeros((H, W))
    d[:-1, :] += st.p1[:-1, :]; d[1:, :] -= st.p1[:-1, :]
    d[:, :-1] += st.p2[:, :-1]; d[:, 1:] -= st.p2[:, :-1]
    u = np.where(rd, st.u, st.v - theta * d)
    a = np.zeros_like(u); a[:-1] = u[1:] - u[:-1]
    b = np.zeros_like(u); b[:, :-1] = u[:, 1:] - u[:, :-1]
    er = (np.sqrt(a * a + b * b)[rd].sum() + 0.5 * np.sum((u - st.v) ** 2) / theta
          + lam * np.sum(f.astype(np.float64)[rd] * st.v[rd]))
    assert emin - rd.sum() * eps - 1e-9 <= er <= emin + 1e-7


def test_tv_textbook_value(orc):
    """Isotropic discrete TV (forward differences): one raised pixel inside a
    3x3 image has TV = 2 + sqrt(2) (its own corner term is sqrt(1 + 1), the
    pixels above and to the left each see a unit jump)."""
    u = np.zeros((3, 3)); u[1, 1] = 1.0
    z = np.zeros((3, 3))
    e = orc.energy(u, u, z, z, np.zeros((3, 3), np.float32), 1.0)
    assert abs(e["tv"] - (2 + math.sqrt(2))) < 1e-15


def test_duality_gap_and_brute_force_bounds(orc):
    """Weak duality (derived from TV(u) = max_{|p|<=1} <u, div p>): for any
    feasible pair D(p) <= min over u in [0,1] <= E_CR(v); the binary brute
    force minimum over all 2^9 labelings of a 3x3 image is itself above the
    relaxed minimum.  At convergence the gap shrinks with theta (Eq. DF
    approaches Eq. CR as theta -> 0)."""
    rng = np.random.default_rng(11)
    f = rng.normal(0, 0.7, (3, 3)).astype(np.float32)
    lam = 1.0
    best = np.inf
    for code in range(512):
        u = np.array([(code >> k) & 1 for k in range(9)], float).reshape(3, 3)
        e = orc.energy(u, u, np.zeros((3, 3)), np.zeros((3, 3)), f, lam)["ecr_u"]
        best = min(best, e)
    relaxed, _ = _smoothed_min(f, lam, 0.2, 1e-8, relaxed_only=True)
    assert relaxed <= best + 1e-6
    gaps = []
    for theta in (0.2, 0.05, 0.0125):
        st = orc.solve(f, orc.domain(f, np.inf), lam, theta, 0.125, iters=60000, tol=1e-13)
        e = orc.energy(st.u, st.v, st.p1, st.p2, f, lam, theta)
        assert e["dual"] <= relaxed + 1e-6 <= e["ecr_v"] + 2e-6
        assert e["gap"] >= -1e-12
        gaps.append(e["gap"])
    assert gaps[2] < gaps[0]
    assert gaps[2] < 0.05 * max(1.0, abs(best))
    # random feasible pairs obey weak duality too
    for k in range(20):
        p1, p2, v = synth.random_state(3, 3, seed=100 + k)
        e = orc.energy(v, v, p1, p2, f, lam)
        assert e["dual"] <= e["ecr_v"] + 1e-12


def test_df_energy_decreases_with_exact_inner_solves(orc):
    """With the rho fixed point run (nearly) to convergence each outer step,
    the alternation is exact block minimisation of Eq. DF, so E_DF(u^l, v^l)
    cannot increase."""
    P = synth.small_example(seed=3, H=24, W=24)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, np.inf)
    st = orc.solve(f, reg, 1.0, iters=1, n_inner=300)
    last = orc.energy(st.u, st.v, st.p1, st.p2, f, 1.0)["edf"]
    for _ in range(12):
        st = orc.solve(f, reg, 1.0, iters=1, n_inner=300, state=st)
        e = orc.energy(st.u, st.v, st.p1, st.p2, f, 1.0)["edf"]
        assert e <= last + 1e-9
        last = e


def test_stopping_rule_and_history(orc):
    """Section 4: the increments are the Euclidean norms of the change of u and
    v over one iteration (checked against consecutive warm-started states),
    and the solve stops at the first l with max(||du||, ||dv||) <= tol."""
    P = synth.small_example(seed=4, H=32, W=32)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, 0.2)
    full = orc.solve(f, reg, 1.0, iters=400)
    assert np.all(full.hist[:20] > 0)
    a = orc.solve(f, reg, 1.0, iters=7)
    b = orc.solve(f, reg, 1.0, iters=1, state=a)
    assert abs(full.hist[7, 0] - np.linalg.norm(b.u - a.u)) < 1e-14
    assert abs(full.hist[7, 1] - np.linalg.norm(b.v - a.v)) < 1e-14
    tol = 1e-2
    crit = np.max(full.hist, axis=1)
    l = int(np.argmax(crit <= tol)) + 1
    st = orc.solve(f, reg, 1.0, iters=400, tol=tol)
    assert st.iters_done == l
    np.testing.assert_allclose(st.hist, full.hist[:l], rtol=0, atol=0)


def test_initialisation_is_heaviside_of_minus_f(orc):
    """Section 1: u0 = H(-f) on the whole image, whatever the restriction;
    with H(0) = 0 a pixel with f = 0 starts in the background both when it is
    fixed (q-hat = 0) and when it lies in RD (any q-hat > 0)."""
    rng = np.random.default_rng(12)
    f = rng.normal(0, 0.2, (11, 13)).astype(np.float32)
    f[2, 3] = 0.0; f[5, 5] = -0.0; f[7, 1] = 1e-30
    h = (f < 0).astype(np.float64)
    for delta in (0.0, np.float32(1e-38), 0.1, np.inf):
        st = orc.solve(f, orc.domain(f, delta), 1.0, iters=0)
        np.testing.assert_array_equal(st.u, h)
        assert not st.p1.any() and not st.p2.any()


# ------------------------------------------------------------------ metrics

def test_errors_hand_computed(orc):
    """Section 4: E1 = |GT & O| / |GT | O| with 0.5 thresholds, E2 = sum of
    squared differences."""
    gt = np.array([0.9, 0.8, 0.1, 0.6, 0.2])
    us = np.array([0.7, 0.2, 0.3, 0.9, 0.6])
    # GT = {0, 1, 3}, O = {0, 3, 4}: intersection 2, union 4
    e1, e2 = orc.errors(us, gt)
    assert e1 == 0.5
    assert abs(e2 - np.sum((us - gt) ** 2)) < 1e-15
    assert orc.errors(np.zeros(4), np.zeros(4)) == (1.0, 0.0)


@pytest.mark.slow
def test_restriction_trend_like_table1(orc):
    """Table 1 (Section 4): q = 1 reproduces the full-domain result (E1 = 1 up
    to the loose 1e-2 stop) and has the smallest E2 of all q in every example
    of the paper's table.  The same must hold on a synthetic 128x128
    piecewise-constant image (here lambda = 1, where small shapes vanish in
    the full solution, so restriction costs accuracy until q -> 1)."""
    with open(os.path.join(GOLDEN, "table1_paper.json")) as fh:
        table = json.load(fh)
    for ex in table["examples"]:
        e1 = dict(zip(table["q"], ex["E1"]))
        e2 = dict(zip(table["q"], ex["E2"]))
        assert e1[1.0] == 1.0 and min(e2.values()) == e2[1.0]
    P = synth.small_example(seed=5, H=128, W=128)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    gt = orc.solve(f, orc.domain(f, np.inf), 1.0, iters=6000, tol=1e-9)
    res = {}
    for q in (0.0, 0.2, 0.4, 0.7, 0.9, 1.0):
        reg = orc.domain(f, orc.quantile_delta(f, q))
        st = orc.solve(f, reg, 1.0, iters=6000, tol=1e-2)
        res[q] = orc.errors(st.u, gt.u)
    assert res[1.0][0] >= 0.99
    assert all(res[1.0][1] < res[q][1] for q in res if q < 1.0)


# ------------------------------------------------------------- reverse mode

def _loss(orc, f, reg, lam, gu, gv, iters, theta=0.2, tau=0.125):
    st = orc.solve(f, reg, lam, theta, tau, iters)
    return float(np.sum(gu * st.u) + np.sum(gv * st.v))


@pytest.mark.parametrize("delta,seed", [(np.inf, 0), (0.25, 1), (0.12, 2)])
def test_reverse_mode_matches_central_differences(orc, delta, seed):
    """Reverse-mode gradient of L = <gu, u^K> + <gv, v^K> through the unrolled
    iteration against central finite differences in FP64 along random
    directions (f changes keep every pixel on its side of the threshold and
    of 0, so the partition and u0 stay fixed)."""
    rng = np.random.default_rng(20 + seed)
    H, W, K, lam = 9, 11, 12, 1.4
    f = (rng.uniform(0.05, 0.35, (H, W)) * rng.choice([-1, 1], (H, W))).astype(np.float32)
    reg = orc.domain(f, delta)
    gu = rng.normal(size=(H, W))
    gv = rng.normal(size=(H, W))
    gf, glam = orc.solve_grad(f, reg, lam, gu, gv, iters=K)
    assert np.all(gf[reg != 2] == 0)
    # f is float32 inside the oracle: the step actually taken is measured.  A
    # step that happens to carry some iterate across a kink of the clip shows
    # up as disagreement that does not shrink with h, so two step sizes are
    # tried and the closer one counts.
    for t in range(3):
        dirn = np.where(reg == 2, rng.normal(size=(H, W)), 0.0)
        best = np.inf
        for e in (16, 19):
            hstep = 2.0 ** -e
            fp = (f.astype(np.float64) + hstep * dirn).astype(np.float32)
            fm = (f.astype(np.float64) - hstep * dirn).astype(np.float32)
            fd = (_loss(orc, fp, reg, lam, gu, gv, K) - _loss(orc, fm, reg, lam, gu, gv, K)) / (2 * hstep)
            an = float(np.sum(gf * (fp.astype(np.float64) - fm) / (2 * hstep)))
            best = min(best, abs(fd - an) / max(1e-3, abs(an)))
        assert best <= 1e-5, best
    el = 1e-6
    fd = (_loss(orc, f, reg, lam + el, gu, gv, K) - _loss(orc, f, reg, lam - el, gu, gv, K)) / (2 * el)
    assert abs(fd - glam) <= 1e-5 * max(1.0, abs(glam)), (fd, glam)


# ------------------------------------------------------------ Chan-Vese loop

def test_update_means_is_the_class_mean_and_keeps_empty_classes(orc):
    rng = np.random.default_rng(41)
    z = rng.uniform(0, 1, (37, 53)).astype(np.float32)
    u = rng.uniform(-0.2, 1.2, (37, 53))
    c1, c2 = orc.update_means(z, u, 0.5, -7.0, -8.0)
    m = u > 0.5
    assert c1 == pytest.approx(float(np.sum(z[m].astype(np.float64))) / m.sum(), rel=1e-14)
    assert c2 == pytest.approx(float(np.sum(z[~m].astype(np.float64))) / (~m).sum(), rel=1e-14)
    # one class empty: it keeps the value it had
    c1, c2 = orc.update_means(z, np.zeros_like(u), 0.5, 0.25, 0.75)
    assert c1 == 0.25 and c2 == pytest.approx(float(np.mean(z.astype(np.float64))), rel=1e-14)


def test_update_means_minimises_the_fitting_energy_for_the_mask(orc):
    """For a fixed thresholded u the updated c1, c2 minimise
    sum (z-c1)^2 [u > 0.5] + (z-c2)^2 [u <= 0.5]: any other pair is worse."""
    rng = np.random.default_rng(42)
    z = rng.normal(0.5, 0.2, (40, 40)).astype(np.float32)
    u = rng.uniform(0, 1, (40, 40))
    c1, c2 = orc.update_means(z, u, 0.5, 0.3, 0.7)
    m = u > 0.5
    zz = z.astype(np.float64)

    def energy(a, b):
        return float(np.sum((zz[m] - a) ** 2) + np.sum((zz[~m] - b) ** 2))

    e0 = energy(c1, c2)
    for da, db in ((1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3), (0.05, -0.05)):
        assert energy(c1 + da, c2 + db) > e0


def test_chan_vese_one_outer_step_is_the_plain_solve(orc):
    P = synth.small_example(seed=5, H=48, W=64)
    st, used, _ = orc.chan_vese(P.z, 0.3, 0.7, 1.0, outer=1, iters=30, delta=0.2)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    ref = orc.solve(f, orc.domain(f, 0.2), 1.0, iters=30)
    assert used == (0.3, 0.7)
    np.testing.assert_array_equal(st.u, ref.u)
    np.testing.assert_array_equal(st.p1, ref.p1)


def test_chan_vese_finds_the_levels_of_a_noiseless_two_level_image(orc):
    """A disk at 0.3 on 0.7, starting from c = (0.35, 0.65): with lambda large
    enough the first solve segments the disk exactly, after which the class
    means are the two float32 levels and stay there."""
    H = W = 64
    yy, xx = np.mgrid[0:H, 0:W]
    disk = (yy - 31.5) ** 2 + (xx - 30.0) ** 2 < 18.0 ** 2
    z = np.where(disk, 0.3, 0.7).astype(np.float32)
    st, used, hist = orc.chan_vese(z, 0.35, 0.65, 40.0, outer=4, iters=60, delta=np.inf)
    assert np.array_equal(st.u > 0.5, disk)
    assert hist[1] == (float(np.float32(0.3)), float(np.float32(0.7)))
    assert used == hist[1] == hist[3]


# ------------------------------------------------- robust restriction (Conclusion)

@pytest.mark.parametrize("r", [0, 1, 2, 5])
def test_dilation_is_the_square_binary_dilation(orc, r):
    """RD grown by Chebyshev distance r = binary dilation of the RD mask by a
    (2r+1) x (2r+1) square (scipy.ndimage, zero outside the image); the other
    pixels keep their Fg / Bg code."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(40 + r)
    reg = rng.choice(np.array([0, 1, 2], np.uint8), size=(37, 53), p=[0.5, 0.45, 0.05])
    out = orc.dilate(reg, r)
    want = ndimage.binary_dilation(reg == 2, structure=np.ones((2 * r + 1, 2 * r + 1), bool))
    np.testing.assert_array_equal(out == 2, want)
    np.testing.assert_array_equal(out[~want], reg[~want])


def test_dilation_of_one_pixel_is_a_clipped_square(orc):
    reg = np.zeros((9, 12), np.uint8)
    reg[1, 10] = 2
    out = orc.dilate(reg, 3)
    want = np.zeros((9, 12), bool)
    want[0:5, 7:12] = True
    np.testing.assert_array_equal(out == 2, want)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_box_mean_is_the_clipped_window_mean(orc, r):
    """Inside the image the local mean equals scipy's uniform filter (a
    running-sum implementation, so within float32 rounding); at a corner it
    is the mean of the (r+1) x (r+1) window that remains; a constant field is
    kept exactly."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(7 + r)
    f = rng.normal(0, 0.4, (30, 41)).astype(np.float32)
    m = orc.box_mean(f, r)
    ref = ndimage.uniform_filter(f.astype(np.float64), 2 * r + 1, mode="constant")
    inner = (slice(r, -r), slice(r, -r))
    np.testing.assert_allclose(m[inner], ref[inner], rtol=0, atol=2e-7)
    assert m[0, 0] == np.float32(np.mean(f[: r + 1, : r + 1].astype(np.float64)))
    assert m[-1, -1] == np.float32(np.mean(f[-r - 1:, -r - 1:].astype(np.float64)))
    c = np.full((11, 13), 0.3125, np.float32)
    assert np.all(orc.box_mean(c, r) == np.float32(0.3125))
    np.testing.assert_array_equal(orc.box_mean(f, 0), f)


def test_robust_partition_reduces_to_the_plain_one(orc):
    """With fbar = f there is no sign disagreement: the Section 3 partition."""
    f = np.random.default_rng(3).normal(0, 0.3, (25, 33)).astype(np.float32)
    f[2, 2] = 0.0
    np.testing.assert_array_equal(orc.domain_robust(f, f, 0.1), orc.domain(f, 0.1))
    m = orc.box_mean(f, 1)
    reg = orc.domain_robust(f, m, 0.0)   # empty threshold: only the sign disagreements
    np.testing.assert_array_equal(reg == 2, (f < 0) != (m < 0))
    np.testing.assert_array_equal(reg[reg != 2], np.where(f < 0, 1, 0)[reg != 2])


def test_robust_restriction_trend_with_strong_noise(orc):
    """The Conclusion expects noisy f to need a more robust restriction.  With
    N(0, 0.25) noise (a fifth of the pixels have the wrong sign of f):
    restricting on the local mean of f (plus the sign disagreements) at
    |RD|/N ~ 0.25 agrees with the full-domain result much better than the
    plain |f| threshold at the same size, and better than the plain one at
    twice the size; growing the plain RD by one pixel also helps."""
    P = synth.noisy_example(seed=0)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    full = orc.solve(f, orc.domain(f, math.inf), 2.0, iters=600).u > 0.5

    def e1(**kw):
        reg = orc.robust_region(f, **kw)
        m = orc.solve(f, reg, 2.0, iters=600).u > 0.5
        return float(np.mean(m == full)), float(np.mean(reg == 2))

    e_plain, a_plain = e1(q=0.25)
    e_half, _ = e1(q=0.5)
    e_rob, a_rob = e1(q=0.05, smooth=1)
    e_q1, _ = e1(q=0.1)
    e_dil, _ = e1(q=0.1, radius=1)
    assert abs(a_rob - a_plain) < 0.03
    assert e_rob > e_plain + 0.08
    assert e_rob > e_half
    assert e_dil > e_q1


# ------------------------------------- restricted primal-dual solver (Conclusion)

def _tv_lp_1d(f, lam, region):
    """The 1-D restricted problem as a linear program (scipy's HiGHS): the
    unknowns are u at the RD pixels; for every RD pixel j < W-1 a term
    |u_{j+1} - u_j| (u fixed to H(-f) outside RD); plus lam * f_j u_j over RD."""
    opt = pytest.importorskip("scipy.optimize")
    W = f.shape[0]
    rd = np.flatnonzero(region == 2)
    col = {j: k for k, j in enumerate(rd)}
    fixed = np.where(region == 1, 1.0, 0.0)
    edges = [j for j in rd if j < W - 1]
    nu, ne = len(rd), len(edges)
    c = np.concatenate([lam * f[rd].astype(np.float64), np.ones(ne)])
    A, b = [], []
    for e, j in enumerate(edges):
        for sgn in (1.0, -1.0):   # t_e >= sgn (u_{j+1} - u_j)
            r = np.zeros(nu + ne)
            rhs = 0.0
            r[nu + e] = -1.0
            r[col[j]] -= sgn
            if (j + 1) in col:
                r[col[j + 1]] += sgn
            else:
                rhs -= sgn * fixed[j + 1]
            A.append(r)
            b.append(rhs)
    res = opt.linprog(c, A_ub=np.array(A) if A else None, b_ub=np.array(b) if b else None,
                      bounds=[(0, 1)] * nu + [(0, None)] * ne, method="highs")
    assert res.status == 0
    return res.fun


def _restricted_objective_1d(u, f, lam, region):
    rd = region == 2
    W = f.shape[0]
    tv = sum(abs(u[j + 1] - u[j]) for j in range(W - 1) if rd[j])
    return tv + lam * float(np.sum(f[rd].astype(np.float64) * u[rd]))


@pytest.mark.parametrize("delta", [math.inf, 0.4, 0.15])
def test_pd_reaches_the_linear_programming_minimum_in_1d(orc, delta):
    """With one row, the restricted Eq. CR is a linear program; the
    primal-dual iterate reaches its optimum (scipy HiGHS, an independent
    solver) on the full domain and on restricted ones."""
    rng = np.random.default_rng(11)
    f = rng.normal(0, 0.5, (1, 70)).astype(np.float32)
    lam = 1.3
    reg = orc.domain(f, delta)
    st = orc.solve_pd(f, reg, lam, iters=20000)
    got = _restricted_objective_1d(st.u[0], f[0], lam, reg[0])
    want = _tv_lp_1d(f[0], lam, reg[0])
    assert got == pytest.approx(want, abs=1e-6)
    assert np.all(st.u[reg != 2] == np.where(reg[reg != 2] == 1, 1.0, 0.0))


def test_pd_duality_gap_closes_on_a_noisy_image(orc):
    """Weak duality (gap >= 0 for every |p| <= 1) and the gap shrinking to ~0
    (strong duality of Eq. CR); the primal-dual p is the negative of the dual
    variable in the energy's convention (TV(u) = max <u, div p>)."""
    P = synth.noisy_example(seed=0, H=40, W=48)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, math.inf)
    gaps = []
    for it in (100, 2000, 8000):
        st = orc.solve_pd(f, reg, 2.0, iters=it)
        assert np.max(np.hypot(st.p1, st.p2)) <= 1 + 1e-12
        e = orc.energy(st.u, st.u, -st.p1, -st.p2, f, 2.0)
        gaps.append(e["ecr_u"] - e["dual"])
        assert gaps[-1] >= -1e-9
    assert gaps[1] < 0.05 * gaps[0]
    assert gaps[2] < 2e-5 * abs(e["ecr_u"])


def test_pd_is_at_least_as_low_as_the_dual_iteration_on_eq_cr(orc):
    """Both methods work on the same restricted Eq. CR; the DF iteration
    minimises its theta-relaxation, so its v is feasible but not optimal for
    Eq. CR, while the primal-dual iterate converges to the minimum."""
    P = synth.noisy_example(seed=2, H=40, W=48)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, math.inf)
    pd = orc.solve_pd(f, reg, 2.0, iters=6000)
    df = orc.solve(f, reg, 2.0, iters=3000)
    e_pd = orc.energy(pd.u, pd.u, pd.p1, pd.p2, f, 2.0)["ecr_u"]
    e_df = orc.energy(df.u, df.v, df.p1, df.p2, f, 2.0)["ecr_v"]
    assert e_pd <= e_df + 1e-4


def test_pd_special_cases(orc):
    """Empty RD keeps u = H(-f) and p = 0; large lambda gives u = H(-f) on RD
    too (the fitting term dominates every TV change)."""
    f = np.random.default_rng(5).normal(0, 0.3, (20, 24)).astype(np.float32)
    f[f == 0] = 0.1
    st = orc.solve_pd(f, orc.domain(f, 0.0), 1.0, iters=50)
    np.testing.assert_array_equal(st.u, (f < 0).astype(float))
    assert not st.p1.any() and not st.p2.any()
    g = np.where(np.abs(f) < 0.05, np.sign(f) * 0.05, f).astype(np.float32)
    st = orc.solve_pd(g, orc.domain(g, 0.2), 1e4, iters=50)
    np.testing.assert_array_equal(st.u, (g < 0).astype(float))


def test_pd_two_pixel_worked_example(orc):
    """Two pixels in one row, f = (-0.5, 0.5), lambda = 0.1, sigma = tau =
    s = 1/sqrt(8), worked by hand through Chambolle and Pock's Algorithm 1
    (extrapolation ubar = 2u' - u):
      u0 = (1, 0) = ubar0, p = 0.  Only p2 at the first pixel is free (the
      last column's p2 never enters div).
      it 1: p2 = -s (|.| < 1); div p = (-s, s);
            u = (1 - s (s - 0.05), s (s - 0.05)) = (0.892678, 0.107322);
            ubar = 2u - u0 = (0.785355, 0.214645)
      it 2: p2 = -s + s (0.214645 - 0.785355) = -0.555330;
            u1 = 0.892678 + s (-0.555330 + 0.05) = 0.714016
    (without the extrapolation step it would be 0.687156)."""
    f = np.array([[-0.5, 0.5]], np.float32)
    reg = orc.domain(f, math.inf)
    st = orc.solve_pd(f, reg, 0.1, iters=1)
    assert st.u[0] == pytest.approx([0.892678, 0.107322], abs=1e-6)
    assert st.p2[0, 0] == pytest.approx(-0.353553, abs=1e-6)
    st = orc.solve_pd(f, reg, 0.1, iters=2)
    assert st.p2[0, 0] == pytest.approx(-0.555330, abs=1e-6)
    assert st.u[0, 0] == pytest.approx(0.714016, abs=1e-6)


# ------------------------------------------------------------- 3-D volumes

@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 7), (4, 1, 6), (3, 5, 1), (4, 6, 9)])
def test_div3_is_minus_adjoint_of_grad3(orc, shape):
    rng = np.random.default_rng(sum(shape))
    w = rng.normal(size=shape)
    p = [rng.normal(size=shape) for _ in range(3)]
    g = orc.grad3(w)
    lhs = float(sum(np.sum(a * b) for a, b in zip(g, p)))
    rhs = -float(np.sum(w * orc.div3(*p)))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_grad3_textbook_values(orc):
    """A ramp along the slices has gradient (0, 0, 1) except on the last
    slice; a unit field p3 has divergence +1 on the first slice, 0 inside,
    -1 on the last."""
    D, H, W = 5, 3, 4
    ramp = np.broadcast_to(np.arange(D, dtype=float)[:, None, None], (D, H, W)).copy()
    g1, g2, g3 = orc.grad3(ramp)
    assert not g1.any() and not g2.any()
    assert np.all(g3[:-1] == 1.0) and np.all(g3[-1] == 0.0)
    d = orc.div3(np.zeros((D, H, W)), np.zeros((D, H, W)), np.ones((D, H, W)))
    assert np.all(d[0] == 1.0) and np.all(d[1:-1] == 0.0) and np.all(d[-1] == -1.0)


def test_volume_of_one_slice_is_the_image_solve(orc):
    P = synth.small_example(seed=4, H=30, W=41)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    reg = orc.domain(f, 0.2)
    a = orc.solve3(f[None], reg[None], 1.0, iters=80)
    b = orc.solve(f, reg, 1.0, iters=80)
    for k in ("u", "v", "p1", "p2"):
        np.testing.assert_array_equal(getattr(a, k)[0], getattr(b, k))
    assert not a.p3.any()


def test_volume_constant_along_slices_solves_every_slice_as_the_image(orc):
    """f repeated over the slices: the slice differences vanish, so every
    slice follows the image iteration (p3 stays 0)."""
    P = synth.small_example(seed=6, H=24, W=37)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    f3 = np.repeat(f[None], 5, axis=0)
    a = orc.solve3(f3, orc.domain(f3, 0.25), 1.0, iters=60)
    b = orc.solve(f, orc.domain(f, 0.25), 1.0, iters=60)
    assert not a.p3.any()
    for z in range(5):
        np.testing.assert_allclose(a.u[z], b.u, atol=1e-13)
        np.testing.assert_allclose(a.p1[z], b.p1, atol=1e-13)


@pytest.mark.parametrize("perm", [(1, 0, 2), (2, 1, 0), (0, 2, 1)])
def test_volume_solve_commutes_with_axis_permutations(orc, perm):
    """The iteration treats the three axes alike (isotropic TV, the same
    boundary rule on each), so permuting the axes of f permutes u, v and the
    components of p."""
    rng = np.random.default_rng(8)
    f = rng.normal(0, 0.3, (6, 9, 11)).astype(np.float32)
    reg = orc.domain(f, 0.25)
    a = orc.solve3(f, reg, 1.5, iters=40)
    fp = np.ascontiguousarray(f.transpose(perm))
    b = orc.solve3(fp, np.ascontiguousarray(reg.transpose(perm)), 1.5, iters=40)
    np.testing.assert_allclose(b.u, a.u.transpose(perm), atol=1e-12)
    np.testing.assert_allclose(b.v, a.v.transpose(perm), atol=1e-12)
    # component k of p belongs to axis (1, 2, 0)[k] of the array (rows, columns, slices)
    comp_axis = {0: 2, 1: 0, 2: 1}   # array axis -> component index
    pa = (a.p1, a.p2, a.p3)
    pb = (b.p1, b.p2, b.p3)
    for new_axis, old_axis in enumerate(perm):
        np.testing.assert_allclose(pb[comp_axis[new_axis]], pa[comp_axis[old_axis]].transpose(perm),
                                   atol=1e-12)


def test_openmp_build_gives_the_same_bits(orc):
    """The OpenMP build of the oracle (all cores, used for the full-size
    parity tests and the timed CPU baseline) computes every element with the
    same operations as the serial build and sums the increments in the same
    order: identical iterates and history."""
    if not orc.has_omp():
        pytest.skip("no OpenMP in this compiler")
    P = synth.small_example(seed=5, H=61, W=77)
    _, f = orc.fitting(P.z, 0.3, 0.7)
    for delta in (0.15, np.inf):
        reg = orc.domain(f, delta)
        a = orc.solve(f, reg, 1.0, iters=120, n_inner=2)
        b = orc.solve(f, reg, 1.0, iters=120, n_inner=2, parallel=True)
        for x, y in ((a.u, b.u), (a.v, b.v), (a.p1, b.p1), (a.p2, b.p2), (a.hist, b.hist)):
            np.testing.assert_array_equal(x, y)
        c = orc.solve(f, reg, 1.0, iters=500, tol=1e-2, parallel=True)
        d = orc.solve(f, reg, 1.0, iters=500, tol=1e-2)
        assert c.iters_done == d.iters_done
