"""Seeded input generators shared by the GPU tests (coordinates only: none
of the method's arithmetic)."""
import numpy as np

from paper_2212_08284_gb300 import synth


def face_coords(rng, box, n, count, lo, hi):
    """FP32 coordinates next to the leaf faces k L / n - L / 2, k = lo .. hi:
    the first half on a face or up to three FP32 steps either side of it, the
    second half 1 to 4 times n 2^-20 leaf edges away from it (just outside the
    band that the binning's FP32 screen hands to the FP64 chain)."""
    k = rng.integers(lo, hi + 1, size=count)
    h = box / n
    far = np.arange(count) >= count // 2
    delta = rng.uniform(1.0, 4.0, size=count) * n * 2.0 ** -20 * h * rng.choice([-1.0, 1.0], size=count)
    v = (k * h - box / 2 + np.where(far, delta, 0.0)).astype(np.float32)
    steps = np.where(far, 0, rng.integers(-3, 4, size=count))
    for s in range(3):
        up, dn = steps > s, steps < -s
        v[up] = np.nextafter(v[up], np.float32(np.inf))
        v[dn] = np.nextafter(v[dn], np.float32(-np.inf))
    return v


def face_box(nonperiodic=False, seed=2212, count=4000):
    """The 24,000-atom water box at n = 14 with one coordinate of `count`
    atoms next to a leaf face (periodic: faces up to one box length outside
    the box, which wrap; non-periodic: clipped into [-L/2, L/2))."""
    b = synth.config_box(2)
    n = 14
    rng = np.random.default_rng(seed)
    idx = rng.choice(b.n, size=count, replace=False)
    axis = rng.integers(0, 3, size=count)
    fc = face_coords(rng, b.box, n, count, 0 if nonperiodic else -n, n if nonperiodic else 2 * n)
    if nonperiodic:
        hi = np.float32(b.box / 2)
        if float(hi) >= b.box / 2:
            hi = np.nextafter(hi, np.float32(-np.inf))
        lo = np.float32(-b.box / 2)
        if float(lo) < -b.box / 2:
            lo = np.nextafter(lo, np.float32(np.inf))
        fc = np.clip(fc, lo, hi)
    x = b.x.copy()
    x[idx, axis] = fc
    b.x = x.astype(np.float32)
    return b, n


def clustered_one_leaf(n_atoms=4096, box=20.0, n=5, leaf=(2, 3, 1), seed=11):
    """n_atoms uniform in one leaf (every other leaf empty), charges +-0.5."""
    rng = np.random.default_rng(seed)
    h = box / n
    lo = -box / 2 + np.array(leaf) * h
    x = (lo + rng.uniform(0.02, 0.98, size=(n_atoms, 3)) * h).astype(np.float32)
    q = rng.choice([-0.5, 0.5], size=n_atoms).astype(np.float32)
    return synth.Box(x=x, q=q, mu=np.zeros((n_atoms, 3), np.float32), theta=np.zeros((n_atoms, 6), np.float32),
                     box=box), n


def clustered_half_in_eight(seed=12):
    """The 24,000-atom water box with half its atoms (a random subset) moved
    uniformly into the 2 x 2 x 2 leaves around a corner of the box at n = 14
    (leaves 13 and 0 of each axis: the block straddles the periodic
    boundary)."""
    b = synth.config_box(2)
    n = 14
    h = b.box / n
    rng = np.random.default_rng(seed)
    idx = rng.choice(b.n, size=b.n // 2, replace=False)
    x = b.x.astype(np.float64).copy()
    x[idx] = -b.box / 2 + rng.uniform(-0.98, 0.98, size=(idx.size, 3)) * h
    x[x < -b.box / 2] += b.box
    b.x = x.astype(np.float32)
    return b, n


def heavy_leaf_box(seed=5):
    """1,000 atoms of a 3,000-atom water box (31.1 A, n = 7) moved onto a
    jittered 10 x 10 x 10 lattice (0.44 A) inside leaf (3, 1, 5), charges only."""
    b = synth.small_box(1000, 31, box=31.1)
    n = 7
    h = b.box / n
    rng = np.random.default_rng(seed)
    idx = rng.choice(b.n, size=1000, replace=False)
    g = (np.arange(10) + 0.5) / 10.0
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    lat = lat + rng.uniform(-0.15, 0.15, size=lat.shape) / 10.0
    x = b.x.astype(np.float64).copy()
    x[idx] = -b.box / 2 + (np.array([3, 1, 5]) + lat) * h
    b.x = x.astype(np.float32)
    b.mu[:] = 0
    b.theta[:] = 0
    return b, n


def uniform_box(n_atoms, box=60.0, seed=0):
    """n_atoms uniform in [-box/2, box/2)^3, normal charges."""
    rng = np.random.default_rng(seed)
    x = ((rng.random((n_atoms, 3)) - 0.5) * box).astype(np.float32)
    q = rng.normal(size=n_atoms).astype(np.float32)
    return synth.Box(x=x, q=q, mu=np.zeros((n_atoms, 3), np.float32), theta=np.zeros((n_atoms, 6), np.float32),
                     box=box, name="uniform")
