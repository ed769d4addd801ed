"""Pins for the FP64 CPU oracle: each function is tied to something other than
itself -- published test vectors, library routines (numpy, scipy), closed
forms, identities from the paper, invariants and brute force.  A dropped term,
a wrong sign or index, a missing conjugate or a transposed operand anywhere in
the oracle fails at least one test here."""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage, stats

import oracle as O
from paper_1605_02164_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _img(H, W, d, seed, cells=5, noise=8.0):
    return synth.voronoi_image(H, W, d, cells, noise, seed=seed).astype(np.float64)


def _full_C(d, seed, lo=25.0 ** 2, hi=60.0 ** 2):
    return synth.spd_eig_range(d, lo, hi, seed)


# ---------------------------------------------------------------- sampling ---

def test_splitmix64_known_answer():
    g = json.load(open(os.path.join(GOLD, "splitmix64_vectors.json")))
    got = [O.splitmix64(g["seed"], i) for i in range(len(g["outputs"]))]
    assert got == [int(v) for v in g["outputs"]]


@pytest.mark.parametrize("N", [1, 10, 20, 63, 64, 65, 100])
def test_sample_Y_is_binomial(N):
    """Prop. 2: X ~ B(N, 1/2) per component, independent; Y = N - 2X."""
    d, K = 3, 6000
    Y = O.sample_Y(d, N, K, seed=12345 + N)
    assert Y.min() >= -N and Y.max() <= N
    assert np.all((N - Y) % 2 == 0)
    X = (N - Y) // 2
    # mean and variance of the binomial
    se = math.sqrt(N / 4 / X.size)
    assert abs(X.mean() - N / 2) < 5 * se
    assert abs(X.var() / (N / 4) - 1) < 0.1
    # goodness of fit on the bins with enough mass
    k = np.arange(N + 1)
    pmf = stats.binom.pmf(k, N, 0.5)
    cnt = np.bincount(X.ravel(), minlength=N + 1)
    keep = pmf * X.size >= 20
    obs = np.append(cnt[keep], cnt[~keep].sum())
    exp = np.append(pmf[keep], pmf[~keep].sum()) * X.size
    if exp[-1] < 1e-9:
        obs, exp = obs[:-1], exp[:-1]
    exp *= obs.sum() / exp.sum()
    if len(obs) > 1:
        assert stats.chisquare(obs, exp).pvalue > 1e-4
    # components uncorrelated
    if N > 1:
        cc = np.corrcoef(X.T)
        assert np.abs(cc - np.eye(d)).max() < 0.08


def test_sample_Y_depends_on_seed_and_is_reproducible():
    a = O.sample_Y(3, 10, 50, 7)
    assert np.array_equal(a, O.sample_Y(3, 10, 50, 7))
    assert not np.array_equal(a, O.sample_Y(3, 10, 50, 8))
    # prefix property: the draw order is t-major, so fewer terms is a prefix
    assert np.array_equal(O.sample_Y(3, 10, 20, 7), a[:20])


# --------------------------------------------------------------- whitening ---

@pytest.mark.parametrize("d", [1, 2, 3, 6, 8])
def test_cholesky_matches_numpy(d):
    C = _full_C(d, 100 + d)
    assert np.allclose(O.cholesky(C), np.linalg.cholesky(C), rtol=1e-12, atol=1e-9)


def test_not_spd_rejected():
    C = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky(C)
    with pytest.raises(np.linalg.LinAlgError):
        O.whiten(C, 0)


@pytest.mark.parametrize("d", [1, 2, 3, 6])
@pytest.mark.parametrize("mode", [0, 1])
def test_whitening(d, mode):
    """Eq. COB: x^T C^{-1} x = |W x|^2 for all x, i.e. W^T W = C^{-1}."""
    C = _full_C(d, 200 + d)
    Wm = O.whiten(C, mode)
    assert np.allclose(Wm @ C @ Wm.T, np.eye(d), atol=1e-12)
    assert np.allclose(Wm.T @ Wm, np.linalg.inv(C), rtol=1e-10, atol=1e-16)
    if mode == 0:
        assert np.allclose(Wm, np.linalg.inv(np.linalg.cholesky(C)), rtol=1e-10, atol=1e-16)
        assert np.allclose(np.triu(Wm, 1), 0)
    else:
        lam, V = np.linalg.eigh(C)  # ascending
        alpha = np.linalg.norm(Wm, axis=1)
        assert np.allclose(alpha, 1 / np.sqrt(lam), rtol=1e-10)
        rows = Wm / alpha[:, None]
        assert np.allclose(np.abs(np.sum(rows * V.T, axis=1)), 1.0, atol=1e-9)


def test_eigen_whitening_isotropic_is_identity_scaled():
    """Section 4: C = sigma_r^2 I gives Q = I and alpha_k = 1/sigma_r."""
    Wm = O.whiten(np.diag([40.0 ** 2] * 3), 1)
    assert np.allclose(Wm, np.eye(3) / 40.0, atol=0)


@pytest.mark.parametrize("mode", [0, 1])
def test_freqs_quadratic_invariant(mode):
    """omega_t = W^T Y_t / sqrt(N) implies omega_t^T C omega_t = |Y_t|^2 / N."""
    d, N, K = 3, 10, 64
    C = _full_C(d, 301)
    Y = O.sample_Y(d, N, K, 9)
    om = O.freqs(O.whiten(C, mode), Y, N)
    q = np.einsum("ti,ij,tj->t", om, C, om)
    assert np.allclose(q, np.sum(Y.astype(float) ** 2, axis=1) / N, rtol=1e-12, atol=1e-14)


def test_freqs_isotropic_closed_form():
    """Section 4 setting: C = sigma_r^2 I gives omega_t = Y_t / (sigma_r sqrt(N))."""
    N, K, sr = 10, 16, 40.0
    Y = O.sample_Y(3, N, K, 3)
    om = O.freqs(O.whiten(np.diag([sr * sr] * 3), 0), Y, N)
    assert np.allclose(om, Y / (sr * math.sqrt(N)), rtol=1e-15, atol=0)


def test_radius_rule():
    """Section 1: window [-3 sigma_s, 3 sigma_s]^2 on the integer grid."""
    assert [O.radius(s) for s in (3, 5, 8, 1, 2.3, 10, 0.2)] == [9, 15, 24, 3, 6, 30, 0]


# ---------------------------------------------------- part A: direct filter ---

def test_direct_two_pixel_closed_form_full_C():
    """Eqs. BF/normal on a 1x2 image: each output mixes the two pixels with
    weights omega(0)=1 and omega(1) phi(delta), phi taken from scipy's
    multivariate normal density (ratio to its peak)."""
    d = 3
    C = _full_C(d, 401)
    f = np.array([[[10.0, 70.0]], [[200.0, 150.0]], [[30.0, 90.0]]])  # (3, 1, 2)
    s = 1.3
    out = O.direct(f, s, C, r=1)
    mvn = stats.multivariate_normal(mean=np.zeros(d), cov=C)
    delta = f[:, 0, 1] - f[:, 0, 0]
    phi = mvn.pdf(delta) / mvn.pdf(np.zeros(d))
    w1 = math.exp(-1.0 / (2 * s * s))
    a, b = f[:, 0, 0], f[:, 0, 1]
    assert np.allclose(out[:, 0, 0], (a + w1 * phi * b) / (1 + w1 * phi), rtol=1e-12)
    assert np.allclose(out[:, 0, 1], (b + w1 * phi * a) / (1 + w1 * phi), rtol=1e-12)


def test_direct_diagonal_offset_weight():
    """A 2x2 image with one bright pixel: the diagonal neighbour has spatial
    weight exp(-2/(2 s^2)), the edge neighbours exp(-1/(2 s^2))."""
    s, sr = 0.9, 50.0
    f = np.zeros((1, 2, 2))
    f[0, 0, 0] = 100.0
    out = O.direct(f, s, np.array([[sr * sr]]), r=1)
    w1, w2 = math.exp(-1 / (2 * s * s)), math.exp(-2 / (2 * s * s))
    phi = math.exp(-0.5 * 100.0 ** 2 / sr ** 2)
    assert math.isclose(out[0, 1, 1], (w2 * phi * 100.0) / (1 + 2 * w1 + w2 * phi), rel_tol=1e-12)
    assert math.isclose(out[0, 0, 0], 100.0 / (1 + (2 * w1 + w2) * phi), rel_tol=1e-12)


def _normalised_blur(f, s, r):
    u = np.arange(-r, r + 1)
    w = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2 * s * s))
    num = np.stack([ndimage.correlate(c, w, mode="constant", cval=0.0) for c in f])
    den = ndimage.correlate(np.ones(f.shape[1:]), w, mode="constant", cval=0.0)
    return num / den


@pytest.mark.parametrize("d", [1, 3])
def test_direct_infinite_range_is_gaussian_blur(d):
    """sigma_r -> infinity: phi == 1, so B[f] is the truncated, normalised
    Gaussian blur (scipy.ndimage with zero padding, divided by the blurred 1)."""
    f = _img(13, 17, d, 5)
    s = 1.7
    r = O.radius(s)
    out = O.direct(f, s, np.eye(d) * 1e16, r=r)
    assert np.allclose(out, _normalised_blur(f, s, r), rtol=1e-10, atol=1e-9)


def test_direct_fixed_point_hull_identity():
    d = 3
    C = _full_C(d, 402)
    const = np.ones((d, 9, 11)) * np.array([10.0, 120.0, 250.0])[:, None, None]
    assert np.allclose(O.direct(const, 2.0, C), const, rtol=0, atol=1e-12)
    f = _img(12, 10, d, 6)
    s = 1.2
    r = O.radius(s)
    out = O.direct(f, s, C, r=r)
    fmax = np.stack([ndimage.maximum_filter(c, size=2 * r + 1, mode="nearest") for c in f])
    fmin = np.stack([ndimage.minimum_filter(c, size=2 * r + 1, mode="nearest") for c in f])
    assert np.all(out <= fmax + 1e-9) and np.all(out >= fmin - 1e-9)
    # r = 0: the window is the pixel alone
    assert np.array_equal(O.direct(f, 0.2, C), f)


def test_direct_equivariance():
    """Transposing the image transposes the output (catches x/y swaps on a
    non-square image); permuting channels with C permuted alike permutes the
    output channels (catches a transposed C or a channel index mix-up)."""
    d = 3
    C = _full_C(d, 403)
    f = _img(9, 14, d, 7)
    s = 1.5
    out = O.direct(f, s, C)
    outT = O.direct(np.ascontiguousarray(f.transpose(0, 2, 1)), s, C)
    assert np.allclose(outT, out.transpose(0, 2, 1), rtol=1e-12, atol=1e-10)
    p = [2, 0, 1]
    outP = O.direct(f[p], s, C[np.ix_(p, p)])
    assert np.allclose(outP, out[p], rtol=1e-12, atol=1e-10)


# ---------------------------------------------- part B: the MC estimator ---

@pytest.mark.parametrize("d,H,W,s,N,K", [(1, 11, 13, 1.4, 10, 9), (2, 10, 7, 1.0, 7, 5),
                                         (3, 12, 15, 1.6, 10, 12), (6, 8, 9, 1.0, 10, 4)])
def test_shiftable_equals_pairwise(d, H, W, s, N, K):
    """Eqs. bigExp-denom: exchanging the sums turns the pairwise form into the
    shiftable one; the two are the same number up to rounding."""
    f = _img(H, W, d, 11 + d)
    Wm = O.whiten(_full_C(d, 500 + d), 0)
    Y = O.sample_Y(d, N, K, 13)
    b1 = O.mcsf(f, s, Wm, N, Y)
    pix = np.array([[y, x] for y in range(H) for x in range(W)])
    b2 = O.mcsf_pairwise(f, s, Wm, N, Y, pix)
    scale = np.abs(b2["Zre"]).max()
    assert np.allclose(b1["Zre"].ravel(), b2["Zre"], rtol=0, atol=1e-12 * scale)
    assert np.allclose(b1["Pre"].reshape(d, -1).T, b2["Pre"], rtol=0, atol=1e-12 * scale * 255)


@pytest.mark.parametrize("d,N,mode", [(1, 1, 0), (1, 6, 0), (2, 3, 0), (2, 4, 1), (3, 4, 0), (3, 3, 1)])
def test_prop2_exhaustive_equals_raised_cosine(d, N, mode):
    """Prop. 2 (Eq. expansion): the expectation over X ~ B(N,1/2)^d of the
    product of complex exponentials is the product of cos^N, so Algorithm 1
    over all Y with binomial weights equals the direct filter with the
    raised-cosine kernel of Eq. approx."""
    f = _img(8, 7, d, 21 + d)
    Wm = O.whiten(_full_C(d, 600 + d, lo=15.0 ** 2, hi=40.0 ** 2), mode)
    s = 1.0
    ex = O.mcsf_exhaustive(f, s, Wm, N)
    rc, Zrc = O.rc_direct(f, s, Wm, N, return_Z=True)
    assert np.allclose(ex["Zre"], Zrc, rtol=1e-10, atol=1e-12)
    assert np.allclose(ex["S"], rc, rtol=1e-9, atol=1e-8)
    assert np.abs(ex["Zim"]).max() < 1e-12 and np.abs(ex["Pim"]).max() < 1e-9


def test_mcsf_infinite_range_is_gaussian_blur():
    """sigma_r -> infinity makes every frequency ~0, H_t == 1, and Algorithm 1
    reduces to the truncated normalised Gaussian blur."""
    d = 3
    f = _img(14, 11, d, 31)
    s = 1.5
    Wm = O.whiten(np.eye(d) * 1e24, 0)
    Y = O.sample_Y(d, 10, 8, 5)
    out = O.mcsf(f, s, Wm, 10, Y)["S"]
    assert np.allclose(out, _normalised_blur(f, s, O.radius(s)), rtol=1e-9, atol=1e-8)


def test_mcsf_constant_image_fixed_point():
    d = 3
    f = np.ones((d, 10, 9)) * np.array([3.0, 77.0, 241.5])[:, None, None]
    Wm = O.whiten(_full_C(d, 700), 0)
    Y = O.sample_Y(d, 10, 16, 6)
    b = O.mcsf(f, 1.3, Wm, 10, Y)
    assert np.allclose(b["S"], f, rtol=0, atol=1e-10)
    assert np.all(b["Zre"] > 0)


def test_mcsf_default_weights_are_uniform():
    d = 2
    f = _img(7, 6, d, 41)
    Wm = O.whiten(_full_C(d, 701), 0)
    Y = O.sample_Y(d, 10, 6, 2)
    a = O.mcsf(f, 1.0, Wm, 10, Y)
    b = O.mcsf(f, 1.0, Wm, 10, Y, weights=np.full(6, 1 / 6))
    assert np.allclose(a["Pre"], b["Pre"], rtol=1e-14) and np.allclose(a["Zre"], b["Zre"], rtol=1e-14)


def test_mcsf_unbiased():
    """Eq. finalApprox is an unbiased Monte Carlo estimate of Eq. MCinterp:
    over many seeds the mean of (Re P, Re Z) approaches the exhaustive sums
    and the mean of the imaginary parts approaches 0 (within 4.5 standard errors)."""
    d, N, K, M = 2, 4, 4, 300
    f = _img(6, 5, d, 51, cells=3)
    Wm = O.whiten(np.diag([20.0 ** 2, 30.0 ** 2]), 0)
    s = 1.0
    ex = O.mcsf_exhaustive(f, s, Wm, N)
    Ps, Zs, Zi = [], [], []
    for m in range(M):
        b = O.mcsf(f, s, Wm, N, O.sample_Y(d, N, K, 10_000 + m))
        Ps.append(b["Pre"])
        Zs.append(b["Zre"])
        Zi.append(b["Zim"])
    for arr, target in ((np.array(Ps), ex["Pre"]), (np.array(Zs), ex["Zre"]), (np.array(Zi), 0 * ex["Zre"])):
        mean = arr.mean(0)
        se = arr.std(0, ddof=1) / math.sqrt(M) + 1e-12
        assert np.all(np.abs(mean - target) <= 4.5 * se)


# ------------------------------------------------- part C: raised cosine ---

def test_raised_cosine_converges_to_gaussian():
    """Prop. 1: cos^N(alpha t / sqrt N) -> exp(-alpha^2 t^2 / 2), so the
    raised-cosine filter approaches the direct filter as N grows."""
    d = 3
    f = _img(10, 10, d, 61)
    C = _full_C(d, 800, lo=30.0 ** 2, hi=50.0 ** 2)
    Wm = O.whiten(C, 0)
    s = 1.0
    A = O.direct(f, s, C)
    errs = [np.abs(O.rc_direct(f, s, Wm, N) - A).max() for N in (10, 40, 160, 640)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 0.1 * errs[0] and errs[3] < 0.05


def test_raised_cosine_hull_even_order():
    d = 3
    f = _img(11, 9, d, 62)
    Wm = O.whiten(_full_C(d, 801), 0)
    s = 1.0
    r = O.radius(s)
    out = O.rc_direct(f, s, Wm, 10)
    fmax = np.stack([ndimage.maximum_filter(c, size=2 * r + 1, mode="nearest") for c in f])
    fmin = np.stack([ndimage.minimum_filter(c, size=2 * r + 1, mode="nearest") for c in f])
    assert np.all(out <= fmax + 1e-9) and np.all(out >= fmin - 1e-9)


def test_fig1_kernel_1d():
    """Fig. 1 setting (alpha = 1/30, N = 20, T = 200, t in [-255, 255]): the
    exhaustive average of cos(omega t) over Y equals cos^N(alpha t / sqrt N)
    (Prop. 2 in closed form), the raised cosine stays within 0.02 of the
    Gaussian, and one T = 200 Monte Carlo draw stays within 5/sqrt(T)."""
    g = json.load(open(os.path.join(GOLD, "paper_experiments.json")))["fig1_kernel"]
    alpha, N, T = g["alpha"], g["N"], g["T"]
    t = np.linspace(g["range"][0], g["range"][1], 1021)
    Wm = O.whiten(np.array([[1.0 / alpha ** 2]]), 0)
    Yall, wts = O.exhaustive_Y(1, N)
    om = O.freqs(Wm, Yall, N)[:, 0]
    exact = (wts[:, None] * np.cos(om[:, None] * t[None, :])).sum(0)
    rc = np.cos(alpha * t / math.sqrt(N)) ** N
    gauss = np.exp(-0.5 * (alpha * t) ** 2)
    assert np.abs(exact - rc).max() < 1e-13
    assert np.abs(rc - gauss).max() < 0.02
    omT = O.freqs(Wm, O.sample_Y(1, N, T, 2016), N)[:, 0]
    mc = np.cos(omT[:, None] * t[None, :]).mean(0)
    assert np.abs(mc - rc).max() < 5 / math.sqrt(T)


# ------------------------------------------------------------ Eq. MSE ---

def test_mse_definitions():
    B = np.zeros((3, 2, 2))
    S = np.ones((3, 2, 2)) * 2.0
    assert O.mse(B, S) == 4.0
    assert math.isclose(O.mse_db(B, S), 10 * math.log10(4.0))
    assert math.isclose(O.psnr(B, S), 10 * math.log10(255.0 ** 2 / 4.0))


def test_fig5_error_decreases_with_T_and_is_subpixel():
    """Section 4 / Fig. 5 (qualitative; the Dome image is not available): at
    sigma_s = 1, sigma_r = 30, N = 10 the MSE between the direct filter and
    MCSF falls as T grows and is below 1 (sub-pixel) for T > 300.  Parity
    unpinned as a number: only the trend and the threshold are checked."""
    g = json.load(open(os.path.join(GOLD, "paper_experiments.json")))["fig5_error"]
    d = 3
    f = synth.voronoi_image(48, 48, d, 8, 10.0, seed=77).astype(np.float64)
    C = np.diag([g["sigma_r"] ** 2.0] * d)
    s, N = g["sigma_s"], g["N"][0]
    A = O.direct(f, s, C)
    Wm = O.whiten(C, 0)
    res = {}
    for T in (25, 100, 400):
        res[T] = np.mean([O.mse(A, O.mcsf(f, s, Wm, N, O.sample_Y(d, N, T, 9000 + 31 * T + m))["S"])
                          for m in range(4)])
    assert res[25] > res[100] > res[400]
    assert res[400] < 1.0


def test_fig5_variance_falls_as_one_over_T_and_saturates_in_N():
    """Section 4 / Fig. 5: the MC error of Algorithm 1 behaves as variance / T
    (Prop. 2 makes the estimator an average of T iid terms, so its variance is
    1/T of one term's), and for a fixed large T the MSE hardly changes from
    N = 10 to N = 20 (the paper's saturation in N).  Checked on a 64 x 64
    synthetic stand-in at sigma_s = 1, sigma_r = 30, 4 seeds per point."""
    d = 3
    f = synth.voronoi_image(64, 64, d, 8, 10.0, seed=1001).astype(np.float64)
    C = np.diag([30.0 ** 2] * d)
    A = O.direct(f, 1.0, C)
    Wm = O.whiten(C, 0)
    m = {}
    for N in (10, 20):
        for T in (40, 640):
            m[N, T] = np.mean([O.mse(A, O.mcsf(f, 1.0, Wm, N, O.sample_Y(d, N, T, 60_000 + 17 * T + N + k))["S"])
                               for k in range(4)])
    slope = math.log(m[10, 640] / m[10, 40]) / math.log(16.0)
    assert -1.3 < slope < -0.7, slope
    assert abs(10 * math.log10(m[20, 640] / m[10, 640])) < 1.5


# ---------------------------------------------------------------- CIE-Lab ---

def _lab_of(rgb):
    return O.rgb_to_lab(np.asarray(rgb, np.float64).T.reshape(3, 1, -1))[:, 0, :].T


def test_lab_tabulated_colours():
    """Section 4 (Fig. 4) filters in CIE-Lab.  The transform is pinned to the
    tabulated L*a*b* of the sRGB primaries, secondaries and mid grey
    (tests/golden/srgb_lab_reference.json, sources cited there)."""
    g = json.load(open(os.path.join(GOLD, "srgb_lab_reference.json")))
    names = list(g["colours"])
    got = _lab_of([g["colours"][k]["rgb"] for k in names])
    for k, v in zip(names, got):
        assert np.abs(v - np.array(g["colours"][k]["lab"])).max() < g["tolerance"], (k, v)


def test_lab_white_black_grey_axis():
    """White is (100, 0, 0) and black (0, 0, 0) by construction of the white
    point; every grey has a* = b* = 0 and L* increases with the grey level."""
    w, k = _lab_of([[255, 255, 255], [0, 0, 0]])
    assert np.abs(w - [100, 0, 0]).max() < 1e-12 and np.abs(k).max() < 1e-12
    grey = _lab_of([[v, v, v] for v in np.linspace(0, 255, 52)])
    assert np.abs(grey[:, 1:]).max() < 1e-12
    assert np.all(np.diff(grey[:, 0]) > 0)


def test_lab_round_trip_and_continuity():
    """lab_to_rgb inverts rgb_to_lab (also outside [0, 255], no clipping), and
    both piecewise definitions meet at their break points: the sRGB one at
    0.04045 up to the ~1e-6 step its published rounded constants leave, the
    CIE one at Y/Yn = (6/29)^3, i.e. L* = 116 (6/29) - 16 = 8."""
    rng = np.random.default_rng(5)
    f = rng.uniform(-20, 275, (3, 17, 23))
    assert np.abs(O.lab_to_rgb(O.rgb_to_lab(f)) - f).max() < 1e-9
    v = 0.04045 * 255
    a, b = _lab_of([[v - 1e-9] * 3, [v + 1e-9] * 3])
    assert abs(a[0] - b[0]) < 1e-5
    lo, hi = 0.0, 255.0  # grey level where L* crosses 8, by bisection
    for _ in range(80):
        mid = (lo + hi) / 2
        if _lab_of([[mid] * 3])[0, 0] < 116 * (6 / 29) - 16:
            lo = mid
        else:
            hi = mid
    a, b = _lab_of([[lo - 1e-7] * 3, [lo + 1e-7] * 3])
    assert abs(a[0] - b[0]) < 1e-5


# ------------------------------------------------------- recursive (Deriche) ---

DERICHE_FIT = (1.680, 3.735, 1.783, 0.6318, -0.6803, -0.2598, 1.723, 1.997)  # Deriche 1993, Gaussian fit


def _deriche_closed_form(n, s):
    a0, a1, b0, w0, c0, c1, b1, w1 = DERICHE_FIT
    t = np.abs(n) / s
    return (a0 * np.cos(w0 * t) + a1 * np.sin(w0 * t)) * np.exp(-b0 * t) + \
        (c0 * np.cos(w1 * t) + c1 * np.sin(w1 * t)) * np.exp(-b1 * t)


@pytest.mark.parametrize("s", [1.5, 3.0, 8.0, 25.0])
def test_deriche_recursion_equals_its_closed_form(s):
    """Section 3 names Deriche's recursive Gaussian for the O(1) convolution.
    The 4th-order causal + anticausal recursions (coefficients from the
    z-transform of the two damped sinusoids) reproduce the closed-form kernel
    h(|x|) h(|y|) of the fit exactly, and that kernel is within ~1e-3 of the
    Gaussian it approximates (peak 1)."""
    n = 301
    x = np.zeros((n, n))
    x[150, 150] = 1.0
    h = O.deriche_blur(x, s)
    m = np.arange(n) - 150
    cf = _deriche_closed_form(m, s)
    assert np.abs(h - np.outer(cf, cf)).max() < 1e-10
    g = np.exp(-m ** 2 / (2 * s * s))
    assert np.abs(h - np.outer(g, g)).max() < 1.5e-3


def test_deriche_zero_state_is_zero_padding():
    """Zero state at both ends of every line = zeros outside the image (R5)."""
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 255, (23, 31))
    pad = np.zeros((23 + 80, 31 + 80))
    pad[40:63, 40:71] = img
    a = O.deriche_blur(img, 4.0)
    b = O.deriche_blur(pad, 4.0)[40:63, 40:71]
    assert np.abs(a - b).max() < 1e-9 * np.abs(a).max()


def test_mcsf_deriche_shiftable_equals_pairwise():
    """Algorithm 1 with the recursive blur equals the pairwise sum with the
    closed-form recursive kernel over the whole image (Eqs. bigExp-denom)."""
    d, H, W, N, K, s = 3, 9, 11, 10, 4, 2.0
    f = synth.voronoi_image(H, W, d, 4, 10.0, seed=5).astype(np.float64)
    C = np.diag([40.0 ** 2] * d)
    Wm = O.whiten(C, 0)
    Y = O.sample_Y(d, N, K, 77)
    S = O.mcsf_deriche(f, s, Wm, N, Y)["S"]
    pix = np.array([(y, x) for y in range(H) for x in range(W)], np.int32)
    pw = O.mcsf_deriche_pairwise(f, s, Wm, N, Y, pix)
    assert np.allclose(pw.T.reshape(d, H, W), S, rtol=1e-9, atol=1e-9)


def test_mcsf_deriche_infinite_range_and_constant_image():
    """sigma_r -> inf: the recursive MCSF is the normalised recursive blur
    (w * f) / (w * 1); a constant image is a fixed point."""
    d, H, W, s = 3, 20, 17, 3.0
    f = synth.voronoi_image(H, W, d, 5, 10.0, seed=8).astype(np.float64)
    Wm = O.whiten(np.eye(d) * 1e16, 0)
    Y = O.sample_Y(d, 10, 6, 3)
    S = O.mcsf_deriche(f, s, Wm, 10, Y)["S"]
    one = O.deriche_blur(np.ones((H, W)), s)
    for c in range(d):
        assert np.allclose(S[c], O.deriche_blur(f[c], s) / one, rtol=1e-9)
    g = np.full((d, H, W), 77.0)
    S = O.mcsf_deriche(g, s, O.whiten(np.eye(d) * 900.0, 0), 10, O.sample_Y(d, 10, 5, 4))["S"]
    assert np.abs(S - 77.0).max() < 1e-9
