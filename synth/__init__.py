"""Seeded synthetic inputs for the EBSD template-matching indexer.

This module only *generates inputs*: a Kikuchi-like spherical master pattern
sampled on a Lambert equal-area square grid, orientation sets (uniform random,
an S^2 x S^1 grid restricted to the cubic fundamental zone, a smooth
orientation field for a map), pattern-centre jitter and a Poisson/background
noise model.  It holds none of the indexer's arithmetic (no projection onto
the detector, no filtering, no correlation, no refinement): both the FP64 CPU
oracle and the CUDA path take what is generated here as their inputs, so the
two never share code through this module.

The paper's master pattern comes from a Bloch-wave simulation (DynamicS,
"SO(3) Library Generation" section) and its maps are experimental; neither is
available, so the band-sum master below and the generators stand in for them
with the paper's sizes (128 x 128 patterns, PC ranges of the Demonstrations
section, ~4,000-template cubic libraries).
"""
from __future__ import annotations

import functools
import math

import numpy as np

# ---------------------------------------------------------------------------
# geometry defaults (Bruker-style pattern centre, 70 degree sample tilt)
# ---------------------------------------------------------------------------
DEFAULT_PC = (0.5, 0.5, 0.6)
SAMPLE_TILT_DEG = 70.0
DETECTOR_TILT_DEG = 0.0

# electron wavelength at 20 kV in picometres
WAVELENGTH_PM = 8.59


def _family_normals(hkl):
    """All distinct plane normals {hkl} of a cubic crystal, one of each +/- pair."""
    h, k, l = hkl
    seen = set()
    out = []
    import itertools
    for perm in set(itertools.permutations((h, k, l))):
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    v = (sx * perm[0], sy * perm[1], sz * perm[2])
                    key = max(v, tuple(-c for c in v))
                    if key in seen:
                        continue
                    seen.add(key)
                    out.append(v)
    a = np.array(sorted(out), dtype=np.float64)
    return a / np.linalg.norm(a, axis=1, keepdims=True)


# (hkl, |F|^2 proxy) per crystal; lattice parameter in pm
CRYSTALS = {
    # diamond cubic (Si-like): {111}, {220}, {004}, {311}
    "diamond": dict(a_pm=543.1, families=[((1, 1, 1), 32.0), ((2, 2, 0), 64.0),
                                          ((0, 0, 4), 64.0), ((3, 1, 1), 32.0)]),
    # BCC (alpha-Fe-like): h+k+l even
    "bcc": dict(a_pm=286.65, families=[((1, 1, 0), 4.0), ((2, 0, 0), 4.0), ((2, 1, 1), 4.0),
                                       ((2, 2, 0), 4.0), ((3, 1, 0), 4.0)]),
}


def band_table(crystal: str, lowest_halfwidth_deg: float = 1.5, debye_waller_a2: float = 0.5):
    """Per-band (normal, weight, sigma_rad) of the synthetic master pattern.

    Band half-width sigma is proportional to the Bragg angle (so to 1/d), scaled
    so that the lowest-order band has ``lowest_halfwidth_deg``; the weight is
    |F|^2 times a Debye-Waller factor exp(-B |g|^2 / 4) (|g| in 1/Angstrom).
    """
    spec = CRYSTALS[crystal]
    a = spec["a_pm"]
    rows = []
    thetas = []
    for hkl, f2 in spec["families"]:
        g = math.sqrt(sum(c * c for c in hkl)) / a          # 1/pm
        theta_b = math.asin(WAVELENGTH_PM * g / 2.0)
        thetas.append(theta_b)
        g_a = g * 100.0                                     # 1/Angstrom
        w = f2 * math.exp(-debye_waller_a2 * g_a * g_a / 4.0)
        rows.append((hkl, w, theta_b))
    scale = math.radians(lowest_halfwidth_deg) / min(thetas)
    wmax = max(r[1] for r in rows)
    normals, weights, sigmas = [], [], []
    for hkl, w, theta_b in rows:
        n = _family_normals(hkl)
        normals.append(n)
        weights.append(np.full(len(n), w / wmax))
        sigmas.append(np.full(len(n), scale * theta_b))
    return np.concatenate(normals), np.concatenate(weights), np.concatenate(sigmas)


def lambert_square_to_sphere(X, Y):
    """Inverse of the Rosca (2010) equal-area square map, northern hemisphere.

    (X, Y) in [-sqrt(pi/2), sqrt(pi/2)]^2 -> unit vector with z >= 0.
    Used here only to know which direction each master-grid cell samples.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    out = np.zeros(X.shape + (3,))
    absX, absY = np.abs(X), np.abs(Y)
    m1 = (absY <= absX) & (absX > 0)
    m2 = (absY > absX)
    # region |Y| <= |X|
    Xa, Ya = X[m1], Y[m1]
    f = (2.0 * Xa / np.pi) * np.sqrt(np.maximum(np.pi - Xa * Xa, 0.0))
    ang = np.pi * Ya / (4.0 * Xa)
    out[m1, 0] = f * np.cos(ang)
    out[m1, 1] = f * np.sin(ang)
    out[m1, 2] = 1.0 - 2.0 * Xa * Xa / np.pi
    # region |X| < |Y|
    Xb, Yb = X[m2], Y[m2]
    f = (2.0 * Yb / np.pi) * np.sqrt(np.maximum(np.pi - Yb * Yb, 0.0))
    ang = np.pi * Xb / (4.0 * Yb)
    out[m2, 0] = f * np.sin(ang)
    out[m2, 1] = f * np.cos(ang)
    out[m2, 2] = 1.0 - 2.0 * Yb * Yb / np.pi
    # origin
    m0 = ~(m1 | m2)
    out[m0, 2] = 1.0
    return out


def master_grid_directions(M: int):
    """Directions sampled by a 2 x M x M master grid: [hemisphere, row, col, xyz].

    Cell (a, b) of hemisphere h has its centre at X = L(2(b+0.5)/M - 1),
    Y = L(2(a+0.5)/M - 1), L = sqrt(pi/2); hemisphere 1 is the mirror z -> -z.
    """
    L = math.sqrt(math.pi / 2.0)
    c = L * (2.0 * (np.arange(M) + 0.5) / M - 1.0)
    Y, X = np.meshgrid(c, c, indexing="ij")
    north = lambert_square_to_sphere(X, Y)
    south = north.copy()
    south[..., 2] *= -1.0
    return np.stack([north, south])


@functools.lru_cache(maxsize=8)
def master_pattern(crystal: str = "bcc", M: int = 1024, background: float = 0.25) -> np.ndarray:
    """Kikuchi-like master pattern [2, M, M] float32 on the Lambert square grid.

    I(n) = background + sum_bands w_b sech^2(asin(n . g_b) / sigma_b): one
    sech^2 band centred on the great circle of each plane normal g_b.  The sum
    is invariant under the 24 proper cubic rotations because every family is
    closed under them.  Returned read-only (cached).
    """
    normals, weights, sigmas = band_table(crystal)
    dirs = master_grid_directions(M).reshape(-1, 3).astype(np.float32)
    out = np.full(dirs.shape[0], background, dtype=np.float32)
    chunk = 1 << 18
    for s in range(0, dirs.shape[0], chunk):
        d = dirs[s:s + chunk]
        dots = np.clip(d @ normals.T.astype(np.float32), -1.0, 1.0)
        ang = np.arcsin(dots) / sigmas.astype(np.float32)
        sech2 = 1.0 / np.cosh(np.clip(ang, -40, 40)) ** 2
        out[s:s + chunk] += sech2 @ weights.astype(np.float32)
    out = out.reshape(2, M, M)
    out.setflags(write=False)
    return out


# ---------------------------------------------------------------------------
# small quaternion helpers for *generating* orientation sets (w, x, y, z)
# ---------------------------------------------------------------------------
def _qmul(a, b):
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def _canon(q):
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    return np.where(q[..., :1] < 0, -q, q)


def _axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    ang = np.asarray(ang, dtype=np.float64)[..., None]
    return np.concatenate([np.cos(ang / 2), np.sin(ang / 2) * axis], axis=-1)


def _rotvec_to_quat(v):
    v = np.asarray(v, dtype=np.float64)
    ang = np.linalg.norm(v, axis=-1, keepdims=True)
    safe = np.where(ang > 0, ang, 1.0)
    axis = np.where(ang > 0, v / safe, np.array([1.0, 0.0, 0.0]))
    return np.concatenate([np.cos(ang / 2), np.sin(ang / 2) * axis], axis=-1)


def random_quaternions(n: int, seed: int) -> np.ndarray:
    """n uniformly random unit quaternions (Shoemake 1992), w >= 0, float64 [n, 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u1, u2, u3 = rng.random((3, n))
    q = np.stack([np.sqrt(u1) * np.cos(2 * np.pi * u3),
                  np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3)], axis=-1)
    return _canon(q)


def in_cubic_fundamental_zone(q: np.ndarray) -> np.ndarray:
    """True where q lies in the cubic (432) Rodrigues fundamental zone."""
    q = _canon(np.asarray(q, dtype=np.float64))
    w = np.maximum(q[..., 0], 1e-300)
    r = np.abs(q[..., 1:]) / w[..., None]
    return (r.max(axis=-1) <= math.sqrt(2.0) - 1.0 + 1e-12) & (r.sum(axis=-1) <= 1.0 + 1e-12)


def so3_grid_cubic_fz(step_deg: float) -> np.ndarray:
    """Equispaced S^2 x S^1 grid of SO(3), kept where it falls in the cubic FZ.

    Follows the construction the paper describes for its MTEX library: the
    polar angle of S^2 is split equidistantly, each ring's azimuth is sampled in
    proportion to its circumference, and the rotation about each S^2 point (the
    S^1 factor) is split linearly.  Orientation = Bunge (phi1, Phi, phi2) with
    (phi1, Phi) from the S^2 point and phi2 from S^1.
    """
    d = math.radians(step_deg)
    n_polar = max(1, int(round(math.pi / d)))
    n_s1 = max(1, int(round(2 * math.pi / d)))
    qs = []
    for i in range(n_polar + 1):
        Phi = math.pi * i / n_polar
        n_az = max(1, int(round(2 * math.pi * math.sin(Phi) / d)))
        for j in range(n_az):
            phi1 = 2 * math.pi * (j + 0.5 * (i % 2)) / n_az
            for k in range(n_s1):
                phi2 = 2 * math.pi * k / n_s1
                qs.append((phi1, Phi, phi2))
    e = np.array(qs)
    q = euler_bunge_to_quat(e)
    return np.ascontiguousarray(q[in_cubic_fundamental_zone(q)])


def euler_bunge_to_quat(e: np.ndarray) -> np.ndarray:
    """Bunge (phi1, Phi, phi2) -> quaternion of Rz(phi1) Rx(Phi) Rz(phi2), w >= 0."""
    e = np.asarray(e, dtype=np.float64)
    z = np.array([0.0, 0.0, 1.0])
    x = np.array([1.0, 0.0, 0.0])
    q1 = _axis_angle(np.broadcast_to(z, e.shape), e[:, 0])
    q2 = _axis_angle(np.broadcast_to(x, e.shape), e[:, 1])
    q3 = _axis_angle(np.broadcast_to(z, e.shape), e[:, 2])
    return _canon(_qmul(_qmul(q1, q2), q3))


def perturb(q: np.ndarray, max_deg: float, seed: int) -> np.ndarray:
    """q composed with a random rotation whose rotation-vector components are U(-max, max) deg."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = np.radians(rng.uniform(-max_deg, max_deg, size=(len(q), 3)))
    return _canon(_qmul(np.asarray(q, dtype=np.float64), _rotvec_to_quat(v)))


def smooth_orientation_map(ny: int, nx: int, seed: int, amp_deg: float = 10.0,
                           jitter_deg: float = 2.0, n_modes: int = 8) -> np.ndarray:
    """Ground-truth orientations [ny*nx, 4] of a synthetic map.

    A random base orientation composed with a smooth rotation-vector field (a
    sum of ``n_modes`` random plane waves, at most ``amp_deg`` per component)
    and a per-point uniform jitter of +/- ``jitter_deg`` per component.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    base = random_quaternions(1, seed + 1000)[0]
    yy, xx = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    field = np.zeros((ny, nx, 3))
    for _ in range(n_modes):
        f = rng.uniform(-2.0, 2.0, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.uniform(-1.0, 1.0, size=3)
        field += np.sin(2 * np.pi * (f[0] * yy + f[1] * xx) + ph)[..., None] * a
    field *= amp_deg / max(np.abs(field).max(), 1e-12)
    field = np.radians(field.reshape(-1, 3))
    field += np.radians(rng.uniform(-jitter_deg, jitter_deg, size=field.shape))
    q = _qmul(np.broadcast_to(base, (field.shape[0], 4)), _rotvec_to_quat(field))
    return np.ascontiguousarray(_canon(q))


def jittered_pcs(n: int, seed: int, pc=DEFAULT_PC, jitter: float = 0.005) -> np.ndarray:
    """Per-pattern pattern centres [n, 3]: pc + U(-jitter, jitter) per component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asarray(pc, dtype=np.float64)[None, :] + rng.uniform(-jitter, jitter, size=(n, 3))


def add_noise(clean: np.ndarray, pcs: np.ndarray, peak, seed: int,
              bg_sigma_frac: float = 0.35, bg_frac: float = 0.6) -> np.ndarray:
    """Noisy detector images from noise-free ones.

    lambda = peak * (bg_frac * B + (1 - bg_frac) * I_hat), where B is a
    Gaussian background hump (sigma = bg_sigma_frac * width) centred on the
    pattern centre and I_hat is the clean image rescaled to [0, 1]; each pixel
    is a Poisson draw of lambda.  ``peak`` is a scalar or one value per image.
    Returns float32 [n, H, W].
    """
    clean = np.asarray(clean, dtype=np.float64)
    n, H, W = clean.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    peak = np.broadcast_to(np.asarray(peak, dtype=np.float64), (n,))
    rows = np.arange(H) + 0.5
    cols = np.arange(W) + 0.5
    out = np.empty((n, H, W), dtype=np.float32)
    s2 = (bg_sigma_frac * W) ** 2
    for i in range(n):
        cx, cy = pcs[i, 0] * W, pcs[i, 1] * H
        B = np.exp(-((rows[:, None] - cy) ** 2 + (cols[None, :] - cx) ** 2) / (2 * s2))
        c = clean[i]
        lo, hi = c.min(), c.max()
        Ih = (c - lo) / (hi - lo) if hi > lo else np.zeros_like(c)
        lam = peak[i] * (bg_frac * B + (1 - bg_frac) * Ih)
        out[i] = rng.poisson(lam).astype(np.float32)
    return out


def random_images(n: int, H: int, W: int, seed: int) -> np.ndarray:
    """Plain seeded Gaussian images [n, H, W] float32 (for transform-level tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, H, W)).astype(np.float32)


# ---------------------------------------------------------------------------
# workload recipes (inputs only; projection is done by the caller)
# ---------------------------------------------------------------------------
def config_parity_64(seed: int = 0) -> dict:
    """Plain search parity workload: diamond-cubic master (2 x 1024^2), 300
    uniformly random library orientations, 16 random test orientations,
    64 x 64 detector, PC (0.5, 0.5, 0.6), Poisson peak 200 + background."""
    return dict(name="xcf64_T300_P16", crystal="diamond", M=1024, n=64, pc=DEFAULT_PC,
                master=master_pattern("diamond", 1024),
                lib_q=random_quaternions(300, seed), truth_q=random_quaternions(16, seed + 1),
                pcs=np.broadcast_to(np.asarray(DEFAULT_PC), (16, 3)).copy(), peak=200.0,
                noise_seed=seed + 2, max_iter=2)


def config_map_128(seed: int = 0, ny: int = 100, nx: int = 100, step_deg: float = 5.35) -> dict:
    """Search + refinement workload: BCC master (2 x 1024^2), 128 x 128
    detector, ~4,000 library orientations (S^2 x S^1 grid in the cubic
    fundamental zone, step 5.35 deg), a ny x nx map of orientations (smooth
    random field +-10 deg plus +-2 deg jitter), PC (0.5, 0.5, 0.6) jittered by
    +-0.005 per pattern, Poisson peak 100 counts + background, refinement to
    convergence (at most 10 iterations)."""
    P = ny * nx
    return dict(name=f"xcf128_T{len(so3_grid_cubic_fz(step_deg))}_P{P}", crystal="bcc", M=1024, n=128,
                pc=DEFAULT_PC, master=master_pattern("bcc", 1024), lib_q=so3_grid_cubic_fz(step_deg),
                truth_q=smooth_orientation_map(ny, nx, seed + 1), pcs=jittered_pcs(P, seed + 2),
                peak=100.0, noise_seed=seed + 3, max_iter=10)


def config_ndp_128(seed: int = 0, ny: int = 100, nx: int = 100, step_deg: float = 2.5) -> dict:
    """NDP dictionary-indexing workload: the 128 x 128 map of config_map_128
    (same orientations, PCs and noise) against the library spacing the paper
    gives the NDP (2.5 deg: 39,784 orientations in the cubic fundamental
    zone), top-4 BF16 candidates rescored in FP32, then the same refinement."""
    wl = config_map_128(seed=seed, ny=ny, nx=nx)
    wl["lib_q"] = so3_grid_cubic_fz(step_deg)
    wl["name"] = f"ndp128_T{len(wl['lib_q'])}_P{ny * nx}"
    wl["k"] = 4
    return wl


def config_precision_256(seed: int = 0, P: int = 50000, step_deg: float = 3.14) -> dict:
    """Precision-form workload: BCC master (2 x 1024^2), 256 x 256 detector,
    ~20,000 library orientations (S^2 x S^1 FZ grid, 3.14 deg), P patterns at
    uniformly random orientations, PC (0.5, 0.5, 0.6) jittered by +-0.005,
    Poisson peak drawn per pattern from U[50, 500]; screen top-32, FP32
    rescore, two refinement iterations."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    lib_q = so3_grid_cubic_fz(step_deg)
    return dict(name=f"xcf256_T{len(lib_q)}_P{P}", crystal="bcc", M=1024, n=256, pc=DEFAULT_PC,
                master=master_pattern("bcc", 1024), lib_q=lib_q, truth_q=random_quaternions(P, seed + 1),
                pcs=jittered_pcs(P, seed + 2), peak=rng.uniform(50.0, 500.0, size=P), noise_seed=seed + 3,
                max_iter=2, k=32)


# detector (width, height), FZ grid step (deg), patterns per map for the batched form:
# detectors {96, 128, 160, 200, 256}^2 (cropped to 64, 128, 128, 128, 256),
# libraries ~1,000-20,000 orientations, 2,000-40,000 patterns per map
BATCHED_MAPS = (
    ((96, 96), 8.5, 40000),
    ((128, 128), 5.35, 4000),
    ((160, 160), 6.75, 3000),
    ((200, 200), 8.5, 4000),
    ((256, 256), 8.5, 2000),
    ((96, 96), 3.14, 2000),
    ((128, 128), 8.5, 8000),
    ((160, 160), 5.35, 2000),
)


def config_batched(seed: int = 0, maps=BATCHED_MAPS, scale: float = 1.0) -> dict:
    """Batched-form workload: several maps with different detectors and
    libraries indexed together.  Per map: BCC master (shared, 2 x 1024^2), an
    S^2 x S^1 FZ library at the map's step, patterns at uniformly random
    orientations, PC (0.5, 0.5, 0.6) jittered by +-0.005, Poisson peak drawn
    from U[50, 500].  ``scale`` multiplies every map's pattern count."""
    out = []
    for i, ((W, H), step, P) in enumerate(maps):
        P = max(2, int(P * scale))
        rng = np.random.Generator(np.random.PCG64(seed * 1000 + 17 * i + 5))
        out.append(dict(W=W, H=H, step=step, lib_q=so3_grid_cubic_fz(step),
                        truth_q=random_quaternions(P, seed * 1000 + 17 * i + 1),
                        pcs=jittered_pcs(P, seed * 1000 + 17 * i + 2), peak=rng.uniform(50.0, 500.0, size=P)))
    sizes = "_".join(f"{m['W']}T{len(m['lib_q'])}P{len(m['truth_q'])}" for m in out)
    return dict(name=f"maps{len(out)}_{sizes}", master=master_pattern("bcc", 1024), pc=DEFAULT_PC, maps=out,
                noise_seed=seed + 3)


# channel widths of the proposal network's five stride-2 convolutions and its hidden layer
CNN_CHANNELS = (1, 32, 64, 64, 128, 128)
CNN_HIDDEN = 256


def cnn_init_params(k: int = 8, seed: int = 0) -> np.ndarray:
    """Initial parameters of the proposal network as one float32 array in the
    order conv1 W, b, ..., conv5 W, b, fc1 W, b, fc2 W, b: weights uniform in
    +-sqrt(6 / fan_in) (He et al. 2015), biases 0.01 for the ReLU layers and 0
    for the output layer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    ch = CNN_CHANNELS
    for l in range(5):
        fan = ch[l] * 9
        parts.append(rng.uniform(-1, 1, ch[l + 1] * ch[l] * 9) * np.sqrt(6.0 / fan))
        parts.append(np.full(ch[l + 1], 0.01))
    parts.append(rng.uniform(-1, 1, CNN_HIDDEN * ch[5]) * np.sqrt(6.0 / ch[5]))
    parts.append(np.full(CNN_HIDDEN, 0.01))
    parts.append(rng.uniform(-1, 1, 6 * k * CNN_HIDDEN) * np.sqrt(6.0 / CNN_HIDDEN))
    parts.append(np.zeros(6 * k))
    return np.concatenate(parts).astype(np.float32)


def config_learned_128(seed: int = 0, n_train: int = 200000, n_test: int = 100000, step_deg: float = 5.35,
                       n_cal: int = 4000) -> dict:
    """Learned-form workload: the 128 x 128 map generator (BCC master 2 x 1024^2,
    PC (0.5, 0.5, 0.6) jittered by +-0.005) with orientations uniform over
    SO(3), Poisson peak drawn per pattern from U[50, 500]; n_train training
    and n_test test patterns; the ~4,000-orientation FZ library for the
    fallback search; refinement to convergence (at most 10 iterations); n_cal
    separate calibration patterns for the fallback threshold."""
    rng = np.random.Generator(np.random.PCG64(seed + 11))
    lib_q = so3_grid_cubic_fz(step_deg)
    return dict(name=f"learned128_T{len(lib_q)}_train{n_train}_test{n_test}", n=128, pc=DEFAULT_PC,
                master=master_pattern("bcc", 1024), lib_q=lib_q,
                train_q=random_quaternions(n_train, seed + 12), train_pcs=jittered_pcs(n_train, seed + 13),
                train_peak=rng.uniform(50.0, 500.0, size=n_train),
                test_q=random_quaternions(n_test, seed + 14), test_pcs=jittered_pcs(n_test, seed + 15),
                test_peak=rng.uniform(50.0, 500.0, size=n_test),
                cal_q=random_quaternions(n_cal, seed + 17), cal_pcs=jittered_pcs(n_cal, seed + 18),
                cal_peak=rng.uniform(50.0, 500.0, size=n_cal), noise_seed=seed + 16, max_iter=10, k=8)
