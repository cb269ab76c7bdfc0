"""The FP32 decision margins of the FP32-mixed self-gravity walk, checked on the
CPU with numpy's IEEE float32 arithmetic (the same round-to-nearest additions,
subtractions and minima the kernel performs).  The walk takes a node's
opening decision in FP32 only when it is certain: inside a margin it falls back
to the FP64 test.  These tests place particles within a few units in the last
place of box faces and of the opening radius and check that a "certain" FP32
answer always equals the FP64 one."""
import numpy as np

TWO_M24 = 2.0 ** -24


def _split(v):
    hi = np.float32(v)
    lo = np.float32(v - np.float64(hi))
    return hi, lo


def _face_decision(p, lo_box, hi_box, origin, L):
    """(certain_outside, certain_inside) as the FP32 walk computes them."""
    mb = np.float32(4.0 * L * TWO_M24)
    ph = np.float32(p - origin)                  # head of the particle coordinate
    blo = np.float32(lo_box - origin)
    bhi = np.float32(hi_box - origin)
    d = np.minimum(ph - blo, bhi - ph)           # float32 arithmetic, per axis
    dmin = np.min(d, axis=-1)
    return dmin < -mb, dmin >= mb


def test_box_margin_never_contradicts_fp64():
    rng = np.random.default_rng(7)
    origin = np.array([-1.0, -1.0, -1.0])
    L = 2.002
    trials = 200_000
    lo_box = origin + rng.uniform(0, 1.5, (trials, 3))
    hi_box = lo_box + rng.uniform(0.01, 0.5, (trials, 3))
    # particles on or a few ulps (of the box's coordinates) away from a face
    p = rng.uniform(lo_box - 0.05, hi_box + 0.05)
    ax = rng.integers(0, 3, trials)
    face = np.where(rng.random(trials) < 0.5, lo_box[np.arange(trials), ax],
                    hi_box[np.arange(trials), ax])
    ulps = rng.integers(-8, 9, trials) * np.spacing(np.float32(2.0)).astype(np.float64)
    p[np.arange(trials), ax] = face + ulps
    out_c, in_c = _face_decision(p, lo_box, hi_box, origin, L)
    inside64 = np.all((p >= lo_box) & (p <= hi_box), axis=1)
    assert not np.any(out_c & inside64)
    assert not np.any(in_c & ~inside64)
    # the margin is not so wide that nothing is decided in FP32
    assert (out_c | in_c).mean() > 0.5


def _open_decision(p, c, size, theta, origin, L, rsq_ulps):
    """(certain_accept, certain_reject) of s < theta |p - c| as the walk takes it."""
    aL = np.float32(8.0 * L * TWO_M24)
    ph, pl = _split(p - origin)
    ch, cl = _split(c - origin)
    r = (ph - ch) + (pl - cl)                    # float32
    # the kernel fuses these products into FMAs; separate roundings here differ
    # from it by about an ulp, far inside the 2e-6 margin
    R2 = np.float32(r[..., 0] * r[..., 0]) + np.float32(r[..., 1] * r[..., 1])
    R2 = np.float32(R2 + np.float32(r[..., 2] * r[..., 2]))
    inv = np.float32(1.0 / np.sqrt(R2.astype(np.float64)))
    inv = np.float32(inv * (1.0 + rsq_ulps * 2.0 ** -23))   # rsqrtf is approximate
    Rf = np.float32(R2 * inv)
    th = np.float32(theta)
    s = np.float32(size)
    acc_c = s * np.float32(1.0 + 1e-6) < th * (Rf * np.float32(1.0 - 2e-6) - aL)
    rej_c = s * np.float32(1.0 - 1e-6) > th * (Rf * np.float32(1.0 + 2e-6) + aL)
    return acc_c, rej_c


def test_opening_margin_never_contradicts_fp64():
    rng = np.random.default_rng(11)
    origin = np.array([-1.0, -1.0, -1.0])
    L = 2.002
    theta = 0.5
    trials = 200_000
    c = rng.uniform(-0.9, 0.9, (trials, 3))
    direction = rng.normal(size=(trials, 3))
    direction /= np.linalg.norm(direction, axis=1, keepdims=True)
    R = rng.uniform(0.02, 1.0, trials)
    p = c + direction * R[:, None]
    r = p - c
    R64 = np.sqrt((r[:, 0] * r[:, 0] + r[:, 1] * r[:, 1]) + r[:, 2] * r[:, 2])
    # node sizes at the opening radius, a few ulps either side
    size = theta * R64 * (1.0 + rng.integers(-6, 7, trials) * 2.0 ** -52)
    for ulps in (-3, 0, 3):
        acc_c, rej_c = _open_decision(p, c, size, theta, origin, L, ulps)
        accept64 = size < theta * R64
        assert not np.any(acc_c & ~accept64)
        assert not np.any(rej_c & accept64)
    # away from the radius the FP32 test decides
    size_far = theta * R64 * rng.choice([0.9, 1.1], trials)
    acc_c, rej_c = _open_decision(p, c, size_far, theta, origin, L, 0)
    assert (acc_c | rej_c).all()


def _fma32(a, b, c):
    """float32 fused multiply-add: the product of two float32 values is exact in
    float64, so one rounding of the float64 sum to float32 (double rounding is
    rare enough not to matter against the margin)."""
    return np.float32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def test_neighbour_prefilter_margin_never_contradicts_fp64():
    """The search's FP32 prefilter: separations from cell-relative FP32 offsets
    (each within err32 = 2^-20 cs of the truth), r^2 - lo and r^2 - hi from
    fused multiply-adds, and a band of half-width margin around (2 h)^2 left to
    the exact FP64 test.  Outside the band the FP32 answer must be FP64's."""
    rng = np.random.default_rng(5)
    trials = 200_000
    lo_grid = np.zeros(3)
    h = rng.uniform(0.004, 0.006, trials)
    cs = np.full(3, 0.0125)                       # cell side >= 2 h_max
    cs32 = cs.astype(np.float32)
    err32 = np.float32(cs[0] * 2.0 ** -20)
    esum = np.float32(3 * err32)
    esq = np.float32(3 * err32 * err32)
    xa = rng.uniform(0.2, 0.8, (trials, 3))
    direction = rng.normal(size=(trials, 3))
    direction /= np.linalg.norm(direction, axis=1, keepdims=True)
    # neighbours at (2h)(1 + k ulps), on both sides of the support radius
    k = rng.integers(-40, 41, trials)
    xb = xa + direction * (2 * h * (1 + k * 2.0 ** -52))[:, None]
    ia = np.floor((xa - lo_grid) / cs).astype(np.int64)
    ib = np.floor((xb - lo_grid) / cs).astype(np.int64)
    shift = ib - ia                               # -1, 0 or +1 per axis here
    assert np.abs(shift).max() <= 1
    off_a = np.float32(xa - (lo_grid + ia * cs))
    off_b = np.float32(xb - (lo_grid + ib * cs))
    cand = np.float32(off_b + np.float32(shift.astype(np.float32) * cs32))
    d = np.float32(cand - off_a)
    two_h = np.float32(2.0) * np.float32(h)
    lim = np.float32(two_h * two_h)
    margin = np.float32(2.0) * (np.float32(2.0) * two_h * esum + esq
                                + np.float32(4.76837158203125e-07) * lim)
    lo_lim, hi_lim = np.float32(lim - margin), np.float32(lim + margin)
    t = _fma32(d[:, 0], d[:, 0], -lo_lim)
    t = _fma32(d[:, 1], d[:, 1], t)
    t = _fma32(d[:, 2], d[:, 2], t)
    u = np.float32(t + np.float32(lo_lim - hi_lim))
    certain_in = t < 0
    certain_out = u >= 0
    dx = xb - xa
    r2 = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
    in64 = r2 < (2 * h) * (2 * h)
    assert not np.any(certain_in & ~in64)
    assert not np.any(certain_out & in64)
    # the band is narrow: 0.1% away from the radius nothing reaches the FP64 test
    xb_far = xa + direction * (2 * h * rng.choice([0.999, 1.001], trials))[:, None]
    ib2 = np.floor((xb_far - lo_grid) / cs).astype(np.int64)
    off_b2 = np.float32(xb_far - (lo_grid + ib2 * cs))
    d2 = np.float32(np.float32(off_b2 + np.float32((ib2 - ia).astype(np.float32) * cs32)) - off_a)
    t2 = _fma32(d2[:, 2], d2[:, 2], _fma32(d2[:, 1], d2[:, 1], _fma32(d2[:, 0], d2[:, 0], -lo_lim)))
    u2 = np.float32(t2 + np.float32(lo_lim - hi_lim))
    assert ((t2 < 0) | (u2 >= 0)).all()
