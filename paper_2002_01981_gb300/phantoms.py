"""Seeded synthetic phantoms: the inputs both the CUDA path and the oracle read.

This module generates raw FP32 volumes only.  It holds none of the method's
arithmetic (no normalisation, no neighbourhood, no clustering) and imports
neither the CUDA binding nor the oracle.

The paper's own data are not available here: the "cube within a cube"
synthetic set (section 6.2, 181x217x181, re-created at 32^2 ... 854^2) and the
Brainweb volume (section 6.3, 181x217 axial slices, 1-20% noise).  These
piecewise-constant phantoms stand in for them at the paper's sizes and noise
range: nested ellipses / ellipsoids of 3-6 grey levels, an optional smooth
multiplicative bias field, and Gaussian or Rician noise.

Arrays are (nz, ny, nx) float32, x fastest.  ``pitch_x`` pads the fastest
axis (with zeros) to a multiple of 4 elements (16 bytes) as the library's
tensor maps require; ``unpad`` drops the padding again.
"""
import numpy as np


def pitch_for(nx, align=4):
    return (nx + align - 1) // align * align


def pad_pitch(vol, align=4):
    """Copy (nz, ny, nx) into a zero-padded (nz, ny, pitch_x) float32 array."""
    nz, ny, nx = vol.shape
    out = np.zeros((nz, ny, pitch_for(nx, align)), dtype=np.float32)
    out[:, :, :nx] = vol
    return out


def _grid(shape):
    nz, ny, nx = shape
    z = (np.arange(nz, dtype=np.float64) + 0.5)[:, None, None]
    y = (np.arange(ny, dtype=np.float64) + 0.5)[None, :, None]
    x = (np.arange(nx, dtype=np.float64) + 0.5)[None, None, :]
    return z, y, x


def nested_ellipsoids(shape, levels, radii, centre=None):
    """Piecewise-constant label field: level k inside ellipsoid k (outer first).

    radii: list of (rz, ry, rx) semi-axes in voxels, outermost first;
    levels: intensity of the background followed by one per ellipsoid.
    """
    nz, ny, nx = shape
    z, y, x = _grid(shape)
    cz, cy, cx = centre if centre is not None else (nz / 2.0, ny / 2.0, nx / 2.0)
    img = np.full(shape, float(levels[0]))
    for k, (rz, ry, rx) in enumerate(radii):
        rz = max(rz, 1e-9)
        inside = ((x - cx) / rx) ** 2 + ((y - cy) / ry) ** 2 + ((z - cz) / rz) ** 2 <= 1.0
        if nz == 1:
            inside = ((x - cx) / rx) ** 2 + ((y - cy) / ry) ** 2 <= 1.0
            inside = np.broadcast_to(inside, shape)
        img = np.where(inside, float(levels[k + 1]), img)
    return img


def bias_field(shape, amplitude=0.1):
    """b = 1 + a (2 (0.5 x/nx + 0.3 y/ny + 0.2 z/nz) - 1), within [1-a, 1+a]."""
    nz, ny, nx = shape
    z, y, x = _grid(shape)
    return 1.0 + amplitude * (2.0 * (0.5 * x / nx + 0.3 * y / ny + 0.2 * z / nz) - 1.0)


def rician(img, sigma, rng):
    n1 = rng.normal(0.0, sigma, img.shape)
    n2 = rng.normal(0.0, sigma, img.shape)
    return np.sqrt((img + n1) ** 2 + n2 ** 2)


def gaussian(img, sigma, rng):
    return img + rng.normal(0.0, sigma, img.shape)


def ellipse_slice(n=64, seed=1, sigma=0.05):
    """64x64 four-class slice: concentric ellipses centred (32, 32) with
    semi-axes (28, 22), (20, 15), (11, 8) at 0.3 / 0.6 / 0.9 on a 0.0
    background, plus i.i.d. N(0, sigma^2) noise."""
    s = n / 64.0
    shape = (1, n, n)
    img = nested_ellipsoids(shape, [0.0, 0.3, 0.6, 0.9],
                            [(0, 22 * s, 28 * s), (0, 15 * s, 20 * s), (0, 8 * s, 11 * s)],
                            centre=(0.5, n / 2.0, n / 2.0))
    rng = np.random.default_rng(seed)
    return gaussian(img, sigma, rng).astype(np.float32)


BRAIN_LEVELS = [0.0, 0.25, 0.55, 0.85]          # background / CSF / GM / WM
BRAIN_RADII = [(0.42, 0.44, 0.40), (0.36, 0.38, 0.34), (0.22, 0.25, 0.21)]


def brain_phantom(shape=(181, 217, 181), seed=2, sigma=0.07, bias=0.1,
                  levels=None, radii=None):
    """Nested-ellipsoid brain stand-in (default 181x217x181 as (nz, ny, nx)):
    background/CSF/GM/WM at 0/0.25/0.55/0.85, a +-10% linear bias field and
    Rician noise of standard deviation ``sigma``."""
    nz, ny, nx = shape
    levels = BRAIN_LEVELS if levels is None else levels
    radii = BRAIN_RADII if radii is None else radii
    ax = [(fz * nz, fy * ny, fx * nx) for fz, fy, fx in radii]
    img = nested_ellipsoids(shape, levels, ax)
    if bias:
        img = img * bias_field(shape, bias)
    rng = np.random.default_rng(seed)
    return rician(img, sigma, rng).astype(np.float32)


def brain_slice(n, seed=2, sigma=0.07):
    """n x n 2D slice of the brain stand-in (the paper's 32 ... 854 sweep)."""
    ax = [(1e-9, fy * n, fx * n) for _, fy, fx in BRAIN_RADII]
    img = nested_ellipsoids((1, n, n), BRAIN_LEVELS, ax, centre=(0.5, n / 2.0, n / 2.0))
    img = img * bias_field((1, n, n), 0.1)
    rng = np.random.default_rng(seed)
    return rician(img, sigma, rng).astype(np.float32)


SWEEP_SIZES = (32, 55, 95, 165, 285, 493, 854)


def multi_tissue(shape=(256, 256, 256), seed=5, sigma=0.1,
                 levels=(0.0, 0.2, 0.35, 0.5, 0.7, 0.9)):
    """Background plus five nested tissues, Rician noise (c = 6 workload)."""
    nz, ny, nx = shape
    fr = [0.45, 0.38, 0.30, 0.22, 0.12]
    radii = [(f * nz, f * 1.05 * ny, f * 0.95 * nx) for f in fr]
    img = nested_ellipsoids(shape, list(levels), radii)
    rng = np.random.default_rng(seed)
    return rician(img, sigma, rng).astype(np.float32)


def gaussian_phantom(shape=(128, 128, 128), seed=4, sigma=0.09):
    """Brain-like nested ellipsoids (0/0.25/0.55/0.85, no bias) plus i.i.d.
    Gaussian noise (the c = 4 differentiation workload)."""
    nz, ny, nx = shape
    ax = [(fz * nz, fy * ny, fx * nx) for fz, fy, fx in BRAIN_RADII]
    img = nested_ellipsoids(shape, BRAIN_LEVELS, ax)
    rng = np.random.default_rng(seed)
    return gaussian(img, sigma, rng).astype(np.float32)


def piecewise_cube(n=4, levels=(0.0, 1.0), seed=None, sigma=0.0, nz=None):
    """Tiny noise-free (or lightly noisy) piecewise-constant volume whose
    classes split along x: used by brute-force and fixed-point tests."""
    nz = n if nz is None else nz
    k = len(levels)
    img = np.empty((nz, n, n))
    for ix in range(n):
        img[:, :, ix] = levels[min(ix * k // n, k - 1)]
    if sigma:
        img = gaussian(img, sigma, np.random.default_rng(seed))
    return img.astype(np.float32)


def uneven_volumes(count=48, seed=3, lo=64, hi=224, sigmas=(0.03, 0.07, 0.12)):
    """Batch of phantoms of uneven size: each dim ~ U{lo..hi}, c ~ U{4,5,6},
    Rician sigma cycled.  Returns a list of (volume, c)."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        nz, ny, nx = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        c = int(rng.integers(4, 7))
        levels = list(np.linspace(0.0, 0.9, c))
        fr = np.linspace(0.45, 0.15, c - 1)
        radii = [(f, f * 1.05, f * 0.95) for f in fr]
        vol = brain_phantom((nz, ny, nx), seed=seed + k, sigma=sigmas[k % len(sigmas)],
                            bias=0.1, levels=levels, radii=radii)
        out.append((vol, c))
    return out


def random_memberships(shape, c, seed=0, padded_pitch=None):
    """Random positive memberships summing to 1 over the c clusters (inputs for
    single-iteration tests), float32 of shape (c,) + shape; with
    ``padded_pitch`` the x axis is zero-padded to that length."""
    rng = np.random.default_rng(seed)
    u = rng.random((c,) + tuple(shape)) + 0.05
    u = (u / u.sum(axis=0, keepdims=True)).astype(np.float32)
    if padded_pitch is not None:
        out = np.zeros((c,) + tuple(shape[:-1]) + (padded_pitch,), dtype=np.float32)
        out[..., :shape[-1]] = u
        return out
    return u
