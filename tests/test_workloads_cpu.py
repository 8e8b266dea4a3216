"""The seeded input recipes match the statistics the clumpy-medium configuration
states: a Gaussian random field with power spectrum P(k) ~ k^(-11/3), a
lognormal density with sigma_ln = 1 and unit mean in expectation, turbulent
velocities with sigma = 10 km/s per component, and fields held constant over
the bricks of the stated lattice."""
import numpy as np

from paper_1709_10187_gb300 import workloads as W


def _shell_spectrum(g):
    n = g.shape[0]
    p = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(n) ** 2] * 3, indexing="ij")))
    kb = np.round(k * n).astype(int)
    num = np.bincount(kb.ravel(), weights=p.ravel())
    cnt = np.bincount(kb.ravel())
    shells = np.arange(len(num))
    sel = (shells >= 2) & (shells <= n // 3) & (cnt > 0)
    return shells[sel] / n, num[sel] / cnt[sel]


def test_random_field_has_the_stated_spectral_slope():
    rng = np.random.default_rng(3)
    for slope in (-11.0 / 3.0, -2.0):
        g = W.gaussian_random_field(64, slope, rng)
        assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
        k, pk = _shell_spectrum(g)
        fit = np.polyfit(np.log(k), np.log(pk), 1)[0]
        assert abs(fit - slope) < 0.1, (slope, fit)


def test_clumpy_medium_statistics_and_brick_lattice():
    med = W.clumpy_medium(n=64, J=8, x_max=8.0, brick=1, packets=1, seed=0x5EED0005)
    ln = np.log(med.n_rel)
    assert abs(ln.std() - 1.0) < 1e-9                      # sigma_ln = 1
    assert abs(ln.mean() + 0.5) < 1e-9                     # mean of ln rho = -sigma_ln^2 / 2
    assert 0.6 < med.n_rel.mean() < 1.6                    # <rho> = 1 in expectation (a steep spectrum: few modes)
    assert np.allclose(med.v_kms.std(axis=0), 10.0, rtol=1e-9)
    assert np.allclose(med.v_kms.mean(axis=0), 0.0, atol=1e-9)
    # bricks of 8 cells with a boundary at cell index 3: values constant over
    # every brick, partial bricks at the faces
    mb = W.clumpy_medium(n=16, J=8, x_max=8.0, brick=8, offset=3, packets=1, seed=11)
    nbx, c, sh = W.brick_lattice(16, 8, 3)
    assert nbx == 3 and sh == 5 and c[2] == 0 and c[3] == 1 and c[10] == 1 and c[11] == 2
    rho = mb.n_rel.reshape(16, 16, 16)  # (z, y, x), axis 0 fastest in the flat array
    for bz in range(nbx):
        for by in range(nbx):
            for bx in range(nbx):
                blk = rho[np.ix_(c == bz, c == by, c == bx)]
                assert np.all(blk == blk.flat[0])
    assert mb.full.sum() == 1  # only the middle brick lies wholly inside the cube


def test_batched_instances_follow_their_stated_laws():
    # 512 instances: slab or sphere with p = 1/2; tau0 log-uniform in [1e4, 1e8],
    # T log-uniform in [1e2, 1e5] K, 32..256 cells (a sphere: the nearest cube
    # root per axis), 128..512 bins, packets log-uniform in [1e4, 1e6]; bins at
    # least a Doppler width wide and the grid covering 4 (a tau0)^(1/3)
    from scipy.stats import kstest
    ws = W.batched_instances()
    assert len(ws) == 512
    sph = np.array([w.sphere for w in ws])
    assert abs(sph.mean() - 0.5) < 4.0 * np.sqrt(0.25 / 512)
    lt = np.log10([w.tau0 for w in ws])
    lT = np.log10([w.T for w in ws])
    lp = np.log10([w.packets for w in ws])
    assert lt.min() >= 4.0 and lt.max() <= 8.0 and kstest((lt - 4.0) / 4.0, "uniform").pvalue > 1e-3
    assert lT.min() >= 2.0 and lT.max() <= 5.0 and kstest((lT - 2.0) / 3.0, "uniform").pvalue > 1e-3
    assert lp.min() >= 4.0 - 1e-9 and lp.max() <= 6.0 + 1e-9 and kstest((lp - 4.0) / 2.0, "uniform").pvalue > 1e-3
    for w in ws:
        assert 128 <= w.J <= 512
        if w.sphere:
            assert w.ndim == 3 and w.n[0] == w.n[1] == w.n[2] and 3 <= w.n[0] <= 6  # cube roots of 32..256
        else:
            assert w.ndim == 1 and 32 <= w.n[0] <= 256
        a = 4.702e-4 / np.sqrt(w.T / 1.0e4)
        dx = (w.x_max - w.x_min) / w.J
        assert dx >= 1.0 - 1e-12 and w.x_max >= 4.0 * (a * w.tau0) ** (1.0 / 3.0) - 1e-9
    # the 1 % scale the default benchmark walks keeps each instance's law, scaled
    small = W.batched_instances(packet_scale=0.01)
    assert all(s.packets == max(1, round(0.01 * w.packets)) or abs(s.packets - 0.01 * w.packets) <= 1.0
               for s, w in zip(small, ws))


def test_named_configurations_carry_their_stated_sizes():
    from oracle import coracle as C
    # the slab (C1, C2) and sphere (C3) configurations
    for w, cells, bins, xm, tau0, npk in ((W.C1, (64, 1, 1), 128, 30.0, 1.0e5, 100_000),
                                         (W.C2, (256, 1, 1), 512, 60.0, 1.0e7, 10_000_000),
                                         (W.C3, (64, 64, 64), 128, 80.0, 1.0e7, 10_000_000)):
        assert (w.n, w.J, w.x_max, -w.x_min, w.tau0, w.packets, w.T) == (cells, bins, xm, xm, tau0, npk, 1.0e4)
    assert W.C3.sphere and W.C3_V20.vmax_kms == 20.0 and W.C3_V200.vmax_kms == 200.0
    # the paper's a tau0 = 1e9, T = 10 K slab: |x| <= 2.5 (a tau0)^(1/3); Fig. 2 with
    # dz ~ 0.01 R, dx ~ 0.05 (a tau0)^(1/3) (P1); the time-dependent test and the
    # n_z = 101, n_x = 51 choice with dz ~ 0.02 R, dx ~ 0.1 (a tau0)^(1/3) (P2)
    for w, dz, dx in ((W.P1, 0.01, 0.05), (W.P2, 0.02, 0.1)):
        atau = C.damping(w.T) * w.tau0
        assert w.T == 10.0 and abs(atau / 1.0e9 - 1.0) < 1e-5
        s = atau ** (1.0 / 3.0)
        assert abs(w.x_max / (2.5 * s) - 1.0) < 1e-3 and w.x_min == -w.x_max
        assert abs((2.0 * w.R / w.n[0]) / (dz * w.R) - 1.0) < 0.02
        assert abs(((w.x_max - w.x_min) / w.J) / (dx * s) - 1.0) < 0.02
    assert (W.P2.n[0], W.P2.J) == (101, 51)
