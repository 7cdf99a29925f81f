"""Synthetic SAR-shaped scenes (the paper names no dataset).

Recipe (one numpy PCG64 stream per workload, children of
SeedSequence(20230131)):
* grid x_j = (j + 1/2)/N on [0, 1];
* Gaussian bump a * exp(-(x - c)^2 / (2 w^2)), w the standard deviation;
* point scatterer: its complex amplitude added at the nearest sample
  round(x N - 1/2), clipped to the grid;
* complex amplitude: |a| ~ U[0.5, 1], phase ~ U[0, 2 pi);
* SNR_dB = 10 log10(mean |f_clean|^2 / sigma^2); complex noise has real and
  imaginary parts ~ N(0, sigma^2 / 2), real noise ~ N(0, sigma^2).
"""
import numpy as np

SEED = 20230131


def config_rng(idx, sub=None):
    """Generator for workload ``idx`` (0-based); ``sub`` spawns a child."""
    ss = np.random.SeedSequence(SEED).spawn(8)[idx]
    if sub is not None:
        ss = ss.spawn(sub + 1)[sub]
    return np.random.Generator(np.random.PCG64(ss))


def _grid(n):
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _phase(rng, k):
    return np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=k))


def real_noise(rng, n, sigma):
    return rng.normal(0.0, sigma, size=n)


def add_noise_snr(rng, clean, snr_db):
    """Complex white noise at the given SNR (returns noisy, sigma)."""
    p = float(np.mean(np.abs(clean) ** 2))
    sigma = np.sqrt(p / (10.0 ** (snr_db / 10.0)))
    noise = (rng.normal(0.0, sigma / np.sqrt(2.0), size=clean.shape)
             + 1j * rng.normal(0.0, sigma / np.sqrt(2.0), size=clean.shape))
    return clean + noise, sigma


def line_1d_bumps(rng, n, nbumps=5, sigma=0.05):
    """Real line: Gaussian bumps (a ~ U[0.5,1], c ~ U[0.1,0.9], w ~ U[0.01,0.05])
    plus N(0, sigma^2) noise.  Returns (noisy, clean) float64."""
    x = _grid(n)
    a = rng.uniform(0.5, 1.0, nbumps)
    c = rng.uniform(0.1, 0.9, nbumps)
    w = rng.uniform(0.01, 0.05, nbumps)
    clean = np.zeros(n)
    for k in range(nbumps):
        clean += a[k] * np.exp(-(x - c[k]) ** 2 / (2 * w[k] ** 2))
    noisy = clean + real_noise(rng, n, sigma)
    return noisy, clean


def line_1d_scatterers(rng, n, nscat=50, nbumps=3, bump_w=0.05, snr_db=20.0):
    """Complex line: point scatterers over a smooth background of complex
    Gaussian bumps, plus complex white noise.  Returns (noisy, clean) c128."""
    x = _grid(n)
    clean = np.zeros(n, dtype=np.complex128)
    if nbumps:
        amp = rng.uniform(0.5, 1.0, nbumps) * _phase(rng, nbumps)
        c = rng.uniform(0.1, 0.9, nbumps)
        for k in range(nbumps):
            clean += amp[k] * np.exp(-(x - c[k]) ** 2 / (2 * bump_w ** 2))
    pos = rng.uniform(0.0, 1.0, nscat)
    amp = rng.uniform(0.5, 1.0, nscat) * _phase(rng, nscat)
    idx = np.clip(np.round(pos * n - 0.5).astype(np.int64), 0, n - 1)
    np.add.at(clean, idx, amp)
    noisy, _ = add_noise_snr(rng, clean, snr_db)
    return noisy, clean


def image_2d_scene(rng, ny, nx, nscat=200, nrect=5, snr_db=10.0,
                   rect_min=16, rect_max=256):
    """Complex image F[y, x]: point scatterers + rectangles of uniform
    amplitude U[0.3, 0.8] with one random phase each, plus complex noise.
    Rectangle sides ~ U{rect_min..rect_max} pixels (clipped to the image).
    Returns (noisy, clean) complex128 arrays of shape (ny, nx)."""
    clean = np.zeros((ny, nx), dtype=np.complex128)
    for _ in range(nrect):
        h = int(rng.integers(min(rect_min, ny), min(rect_max, ny) + 1))
        w = int(rng.integers(min(rect_min, nx), min(rect_max, nx) + 1))
        y0 = int(rng.integers(0, max(ny - h, 0) + 1))
        x0 = int(rng.integers(0, max(nx - w, 0) + 1))
        a = rng.uniform(0.3, 0.8) * _phase(rng, 1)[0]
        clean[y0:y0 + h, x0:x0 + w] += a
    py = rng.uniform(0.0, 1.0, nscat)
    px = rng.uniform(0.0, 1.0, nscat)
    amp = rng.uniform(0.5, 1.0, nscat) * _phase(rng, nscat)
    iy = np.clip(np.round(py * ny - 0.5).astype(np.int64), 0, ny - 1)
    ix = np.clip(np.round(px * nx - 0.5).astype(np.int64), 0, nx - 1)
    np.add.at(clean, (iy, ix), amp)
    noisy, _ = add_noise_snr(rng, clean, snr_db)
    return noisy, clean


def batch_lines(rng, nlines=256, dmin=14, dmax=18, snr_db=15.0,
                bmin=128.0, bmax=1024.0, rmax_choices=(8, 16, 32, 64)):
    """Range lines of uneven length: log2 length ~ U{dmin..dmax}, 10-40
    scatterers each, B ~ U[bmin, bmax], R_max drawn from rmax_choices.
    Returns a list of dicts (x, clean, d, B, rmax)."""
    out = []
    for _ in range(nlines):
        d = int(rng.integers(dmin, dmax + 1))
        nscat = int(rng.integers(10, 41))
        B = float(rng.uniform(bmin, bmax))
        rmax = int(rng.choice(rmax_choices))
        x, clean = line_1d_scatterers(rng, 2 ** d, nscat=nscat, nbumps=0,
                                      snr_db=snr_db)
        out.append(dict(x=x, clean=clean, d=d, B=B, rmax=rmax))
    return out


def deconv_scene_2d(rng, ny, nx, nscat=100):
    """Sparse complex scene (point scatterers) for the deconvolution
    workload; the caller convolves it and adds noise.  complex128."""
    scene = np.zeros((ny, nx), dtype=np.complex128)
    py = rng.uniform(0.0, 1.0, nscat)
    px = rng.uniform(0.0, 1.0, nscat)
    amp = rng.uniform(0.5, 1.0, nscat) * _phase(rng, nscat)
    iy = np.clip(np.round(py * ny - 0.5).astype(np.int64), 0, ny - 1)
    ix = np.clip(np.round(px * nx - 0.5).astype(np.int64), 0, nx - 1)
    np.add.at(scene, (iy, ix), amp)
    return scene


# ---------------------------------------------------------------- Sec. 7 examples
# The paper's analytic test signals (Examples 1-3), sampled at the cell
# centres x_j = a + dx/2 + j dx, j < N = 2^(K-1) - 1, dx = (b - a)/N, and
# zero-padded at the end to 2^K per axis.  The printed noise levels are read
# as standard deviations.  Each returns (noisy, clean, N, B) with B = 2^K /
# (Delta_x / dx), the sinc bandwidth in this library's units (the grid
# spacing of the padded axis is 1 / 2^K).

def _paper_grid(a, b, K):
    N = 2 ** (K - 1) - 1
    dx = (b - a) / N
    return a + dx / 2 + dx * np.arange(N, dtype=np.float64), dx, N


def paper_example_1d(example, K, rng):
    """Example 1: f = exp(-(3x/10)^2) (0.4 sin 8 pi x - 0.7 cos 6 pi x) on
    [-10, 10], noise 0.02, Delta_x = 4 dx.  Example 2: f = exp(-(3x)^2)
    (0.9 sin(2 pi x / (5 dx)) + 1.4 cos(pi x / (3 dx))) on [-1, 1], noise 0.01,
    Delta_x = 2 dx."""
    if example == 1:
        x, dx, N = _paper_grid(-10.0, 10.0, K)
        f = np.exp(-(3 * x / 10) ** 2) * (0.4 * np.sin(8 * np.pi * x) - 0.7 * np.cos(6 * np.pi * x))
        sd, lobe = 0.02, 4.0
    elif example == 2:
        x, dx, N = _paper_grid(-1.0, 1.0, K)
        f = np.exp(-(3 * x) ** 2) * (0.9 * np.sin(2 * np.pi * x / (5 * dx))
                                     + 1.4 * np.cos(np.pi * x / (3 * dx)))
        sd, lobe = 0.01, 2.0
    else:
        raise ValueError("1D examples are 1 and 2")
    n = 2 ** K
    clean = np.zeros(n)
    clean[:N] = f
    noisy = clean.copy()
    noisy[:N] += real_noise(rng, N, sd)
    return noisy, clean, N, n / lobe


def paper_example_2d(K, rng):
    """Example 3: f = exp(-((2x)^2 + (2y)^2)) (sin 2 pi x - cos 7 pi y
    + cos 4 pi x y - sin 3 pi x y) on [-1, 1]^2, noise 0.1, Delta_x = 2 dx;
    returned as F[y, x] (rows y, columns x: x is the fast index, so the plain
    QTT chain -- column bits first -- takes the x bits first)."""
    x, dx, N = _paper_grid(-1.0, 1.0, K)
    X, Y = np.meshgrid(x, x, indexing="ij")
    f = np.exp(-((2 * X) ** 2 + (2 * Y) ** 2)) * (np.sin(2 * np.pi * X) - np.cos(7 * np.pi * Y)
                                                 + np.cos(4 * np.pi * X * Y)
                                                 - np.sin(3 * np.pi * X * Y))
    n = 2 ** K
    clean = np.zeros((n, n))
    clean[:N, :N] = f
    noisy = clean.copy()
    noisy[:N, :N] += rng.normal(0.0, 0.1, size=(N, N))
    return noisy.T.copy(), clean.T.copy(), N, n / 2.0


# ---------------------------------------------------------------- TT-RSVD draws
def rsvd_omega_blocks(d, rmax, p, rng, dtype=np.float64):
    """Seeded N(0, 1) test matrices of the max rank TT-RSVD (Sec. 5 (2),
    App. A Alg. 4) for a vector of length 2^d: one n_k x (rmax + p) block per
    level k = 1..d-1 (n_k = 2^(d-k)), column-major, one after the other (the
    layout qtt_decompose_rsvd reads).  Returns (flat, omega) with
    omega(k, n, l) the FP64 block of level k."""
    l = rmax + p
    sizes = [2 ** (d - k) * l for k in range(1, d)]
    flat = rng.standard_normal(int(sum(sizes))).astype(dtype)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    def omega(k, n, ll):
        assert ll == l and n == 2 ** (d - k)
        return flat[offs[k - 1]:offs[k]].reshape((n, l), order="F").astype(np.float64)

    return flat, omega
