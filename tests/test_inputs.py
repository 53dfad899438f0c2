"""The seeded input generators hold the recipe they state: determinism in the
seed, layout [nz][ny][nx], the lognormal field's spectral slope, unit
variance and zeroed margin, the Plummer sphere's profile and noise bound, and
the batch sizes' range.  CPU only."""
import numpy as np

from paper_2606_13793_gb300 import inputs


def test_generators_are_deterministic_in_the_seed():
    for gen in (inputs.lognormal, inputs.plummer, inputs.gaussian_blobs):
        a, b, c = gen(24, seed=5), gen(24, seed=5), gen(24, seed=6)
        assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert inputs.batch_sizes(16, seed=3) == inputs.batch_sizes(16, seed=3)


def test_layout_is_z_y_x():
    shape = (40, 24, 16)  # (nx, ny, nz)
    for gen in (inputs.lognormal, inputs.plummer, inputs.gaussian_blobs):
        assert gen(shape, seed=1).shape == (16, 24, 40)
    rho = inputs.point_mass(shape, (3, 5, 7))
    assert rho.shape == (16, 24, 40) and rho[7, 5, 3] == 1.0 and rho.sum() == 1.0


def test_lognormal_spectrum_variance_and_margin():
    n = 64
    rho = inputs.lognormal(n, seed=11, pad_frac=0.0, dtype=np.float64)
    assert rho.min() > 0
    delta = np.log(rho) + 0.5  # rho = exp(delta - 1/2)
    assert abs(delta.mean()) < 1e-5 and abs(delta.std() - 1.0) < 1e-5
    # shell-averaged power of delta against |k|: slope -2.5 over the resolved range
    pk = np.abs(np.fft.fftn(delta)) ** 2
    f = np.fft.fftfreq(n)
    kk = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    edges = np.geomspace(2.0 / n, 0.4, 12)
    k_mid, p_mid = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (kk >= lo) & (kk < hi)
        k_mid.append(kk[m].mean())
        p_mid.append(pk[m].mean())
    slope = np.polyfit(np.log(k_mid), np.log(p_mid), 1)[0]
    assert abs(slope + 2.5) < 0.15, slope
    # the margin: floor(0.1 n) cells on every face are empty, the rest is not
    rho = inputs.lognormal((40, 30, 20), seed=11)
    nz, ny, nx = rho.shape
    for axis, m in ((2, nx), (1, ny), (0, nz)):
        pad = int(np.floor(0.1 * m))
        edge = np.take(rho, list(range(pad)) + list(range(m - pad, m)), axis=axis)
        assert not edge.any()
    assert rho[2:18, 3:27, 4:36].min() > 0


def test_plummer_profile_and_noise():
    n = 48
    rho = inputs.plummer(n, seed=4, noise=0.01, dtype=np.float64)
    rng = np.random.default_rng(4)
    a = rng.uniform(4.0, 20.0)  # the generator's first draw
    rho0 = 3.0 / (4.0 * np.pi * a ** 3)
    z, y, x = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    r2 = (x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2
    smooth = rho0 * (1.0 + r2 / (a * a)) ** -2.5
    noise = rho - smooth
    assert noise.min() >= 0 and noise.max() < 0.01 * rho0
    assert abs(noise.mean() / (0.005 * rho0) - 1.0) < 0.05  # U[0, 0.01 rho0): mean 0.005 rho0


def test_batch_sizes_come_from_the_choices():
    sizes = inputs.batch_sizes(64, seed=2606)
    assert len(sizes) == 64 and set(sizes) <= {64, 96, 128, 192} and len(set(sizes)) > 1
