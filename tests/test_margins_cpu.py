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
