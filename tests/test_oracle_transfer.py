"""Pins of the oracle's walk and of whole transfer runs against closed forms,
conservation laws, symmetries and the analytic solutions the paper compares
with (Sects. 3.4, 4.5, App. B).  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth

THREADS = 8


def _chi2_sym(counts):
    """p-value that a histogram symmetric about its centre is symmetric."""
    from scipy.stats import chi2
    c = np.asarray(counts, float)
    a, b = c[: c.size // 2], c[::-1][: c.size // 2]
    m = (a + b) > 0
    stat = ((a[m] - b[m]) ** 2 / (a[m] + b[m])).sum()
    return chi2.sf(stat, m.sum())


# ---------------------------------------------------------------- walk
def _brute_leaf(tree, p, k):
    """Leaf containing p + eps k, by scanning every leaf."""
    h = tree.leaf_size()
    lo = tree.leaf_ijk * h[:, None]
    hi = lo + h[:, None]
    ok = np.ones(tree.nleaf, bool)
    for ax in range(3):
        if k[ax] < 0:
            ok &= (lo[:, ax] < p[ax]) & (p[ax] <= hi[:, ax])
        else:
            ok &= (lo[:, ax] <= p[ax]) & (p[ax] < hi[:, ax])
    idx = np.nonzero(ok)[0]
    assert idx.size <= 1
    return int(idx[0]) if idx.size else -1


def test_locate_matches_brute_force():
    """Root descent (Sect. 4.3) finds the same leaf as a scan of all leaves,
    including points exactly on faces, edges and corners."""
    wl = synth.sphere(n_packets=1, base=2, max_level=5)
    o = oracle.Oracle(wl)
    tree = wl.medium.tree
    rng = np.random.default_rng(5)
    pts = list(rng.random((300, 3)))
    # points on cell boundaries at several levels
    for lv in (2, 3, 4, 5):
        q = rng.integers(1, 1 << lv, (60, 3)) / float(1 << lv)
        pts += list(q)
    for i, p in enumerate(pts):
        k = rng.normal(size=3)
        if i % 7 == 0:
            k[i % 3] = 0.0
        leaf, lv, ijk = o.locate(p, k)
        assert leaf == _brute_leaf(tree, p, k)
        if leaf >= 0:
            assert lv == tree.leaf_level[leaf] and tuple(ijk) == tuple(tree.leaf_ijk[leaf])


def test_ray_tau_closed_form_sphere():
    """From the centre of a uniform static sphere at line centre: path = R
    and tau = tau0 (Tasitsiomi's H(a,0) = 1); cells crossed on a uniform grid =
    1 + sum |delta i|."""
    tau0 = 1e3
    wl = synth.sphere(tau0=tau0, T=1e4, n_packets=1, base=4, max_level=4)
    o = oracle.Oracle(wl)
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    rng = np.random.default_rng(2)
    R = wl.domain.size
    # the leaf fields are stored in float32: expected tau uses the stored density
    n64 = synth.density_for_tau0(wl.lines[0], 1e4, tau0, R * wl.medium.box_cm)
    tau0 = tau0 * float(wl.medium.n_HI[0]) / n64
    for _ in range(200):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        p = np.array([0.5, 0.5, 0.5])
        tau, cells, lens, n = o.ray_tau(p, k, nu0, cap=1000)
        assert abs(lens.sum() / R - 1) < 1e-14
        assert abs(tau / tau0 - 1) < 1e-12
        end = p + R * k
        i0 = np.where(k < 0, np.ceil(p * 16) - 1, np.floor(p * 16)).astype(int)
        i1 = np.floor(end * 16).astype(int)
        assert n == 1 + np.abs(i1 - i0).sum()


def test_walk_on_graded_tree_matches_brute_force():
    """The neighbour-search walk (Sect. 4.3: same father, then the neighbour
    across the face, then the root) on a graded octree: the midpoint of every
    segment lies in the leaf the walk reports (by a scan of all leaves), and
    the summed path equals the analytic distance to the sphere border."""
    wl = synth.sphere(n_packets=1, base=2, max_level=6)
    o = oracle.Oracle(wl)
    tree = wl.medium.tree
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    c = np.array(wl.domain.centre)
    R = wl.domain.size
    rng = np.random.default_rng(17)
    nseg = 0
    for i in range(90):
        r = R * rng.random() ** (1 / 3) * 0.99
        v = rng.normal(size=3)
        p = c + v / np.linalg.norm(v) * r
        if i < 20:
            p = np.round(p * 64) / 64          # start on faces, edges and corners
        k = rng.normal(size=3)
        if i % 10 == 0:
            k[i % 3] = 0.0                      # rays inside a face plane
        k /= np.linalg.norm(k)
        tau, cells, lens, n = o.ray_tau(p, k, nu0, cap=100000)
        assert n == len(cells) > 0
        b = float(np.dot(p - c, k))
        t_border = -b + math.sqrt(b * b - (float(np.dot(p - c, p - c)) - R * R))
        assert abs(lens.sum() - t_border) <= 1e-12 * max(t_border, 1.0)
        s = np.concatenate([[0.0], np.cumsum(lens)])
        for j in range(n):
            if lens[j] < 1e-9:
                continue                        # a zero-length step through an edge or corner
            mid = p + 0.5 * (s[j] + s[j + 1]) * k
            assert _brute_leaf(tree, mid, k) == cells[j], (i, j)
            nseg += 1
    assert nseg > 500


def test_ray_tau_periodic_slab():
    """Slab (periodic x,y, Sect. 4): a grazing ray from the mid-plane wraps
    many times; its path to the border is (1/2)/|k_z| and tau = tau0/|k_z|."""
    tau0 = 1e2
    wl = synth.slab(tau0=tau0, T=1e4, n_packets=1)
    o = oracle.Oracle(wl)
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    tau0 = tau0 * float(wl.medium.n_HI[0]) / synth.density_for_tau0(wl.lines[0], 1e4, tau0, 0.5 * wl.medium.box_cm)
    for kz in [0.9, -0.3, 0.05, -0.01]:
        k = np.array([math.sqrt(1 - kz * kz) * 0.6, math.sqrt(1 - kz * kz) * 0.8, kz])
        tau, cells, lens, n = o.ray_tau([0.31, 0.77, 0.5], k, nu0, cap=100000)
        assert abs(lens.sum() * abs(kz) / 0.5 - 1) < 1e-12
        assert abs(tau * abs(kz) / tau0 - 1) < 1e-11


# ---------------------------------------------------------------- transfer
def test_conservation_no_dust():
    """Every packet escapes a dust-free medium (Sect. 4.4: status flags);
    the escape spectrum holds every packet."""
    wl = synth.slab(tau0=1e3, T=1e4, n_packets=500)
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    assert np.all(out["status"] == oracle.ESCAPED)
    assert tal["spec"].sum() == 500
    assert np.all(out["nscatt"] > 0)


def test_escape_spectrum_is_the_histogram_of_escapes():
    """Sect. 4.4 tallies: the escape spectrum is the histogram of the escaped
    packets' external frequencies on the detector axis, bin for bin."""
    wl = synth.slab(tau0=1e3, T=1e4, n_packets=800)
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    det = wl.detector
    esc = out["status"] == oracle.ESCAPED
    h, _ = np.histogram(out["nu"][esc], bins=np.linspace(det.nu_lo, det.nu_hi, det.nbin + 1))
    assert np.array_equal(tal["spec"], h)


def test_slab_symmetry():
    """Static slab without recoil: escape through +z and -z equally likely,
    spectrum symmetric in x (Sect. 3.4.2)."""
    from scipy.stats import binomtest
    wl = synth.slab(tau0=1e4, T=1e4, n_packets=3000)
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    up = int((out["pos"][:, 2] > 0.5).sum())
    assert binomtest(up, 3000, 0.5).pvalue > 1e-3
    assert _chi2_sym(tal["spec"]) > 1e-3


@pytest.mark.parametrize("tau0", [10.0, 1e3])
def test_mean_free_path(tau0):
    """Mean distance to the first scattering = (n_HI sigma_0)^-1 (App. B)."""
    n = 20000
    wl = synth.sphere(tau0=tau0, T=100.0, n_packets=n, base=3, max_level=3)
    wl.physics.max_scatt = 1
    out, _ = oracle.Oracle(wl).run(threads=THREADS)
    first = out["path"][out["status"] == oracle.CAPPED]
    lam = wl.domain.size / tau0   # box units; Tasitsiomi H(a,0) = 1
    assert first.size > 0.999 * n
    assert abs(first.mean() / lam - 1) < 4 / math.sqrt(first.size)


@pytest.mark.parametrize("tau_d", [1.0, 2.5])
def test_pure_absorber(tau_d):
    """No H I, albedo 0: a central source escapes with probability
    exp(-tau_dust) (Sect. 3.1.2 / 3.2.2)."""
    from scipy.stats import binomtest
    n = 20000
    wl = synth.sphere(tau0=0.0, T=1e4, tau_dust=tau_d, n_packets=n, base=3, max_level=4)
    wl.dust.albedo = 0.0
    out, _ = oracle.Oracle(wl).run(threads=THREADS)
    esc = int((out["status"] == oracle.ESCAPED).sum())
    assert esc + int((out["status"] == oracle.ABSORBED).sum()) == n
    assert binomtest(esc, n, math.exp(-tau_d)).pvalue > 1e-3


@pytest.mark.parametrize("tau_d", [5.0, 20.0])
def test_interaction_choice_dust_vs_line(tau_d):
    """Sect. 3.2: the first interaction is with dust with probability
    tau_d / (tau_d + tau_HI) at the packet's frequency.  Slab with
    half-thickness tau0 = 10 in H I at line centre (Tasitsiomi's H(a,0) = 1)
    and tau_d in dust of albedo 0, packets emitted at x = 0, one interaction
    each: dust interactions are the absorptions."""
    from scipy.stats import binomtest
    n = 20000
    wl = synth.slab(tau0=10.0, T=1e4, n_packets=n, tau_dust=tau_d, albedo=0.0)
    wl.physics.max_scatt = 1
    out, _ = oracle.Oracle(wl).run(threads=THREADS)
    absorbed = int((out["status"] == oracle.ABSORBED).sum())
    capped = int((out["status"] == oracle.CAPPED).sum())
    assert absorbed + capped >= n - 2          # escaping before any interaction: e^-(10 + tau_d)
    assert binomtest(absorbed, absorbed + capped, tau_d / (tau_d + 10.0)).pvalue > 1e-3


@pytest.mark.parametrize("tau0", [10.0, 1e3])
@pytest.mark.parametrize("mesh", ["one_cell", "grid"])
def test_error_budget_direction_preserving(tau0, mesh):
    """Sect. 4.5: with scatterings that keep the direction, every packet
    travels exactly R; one cell: error ~1e-15 (tau=10) .. 1e-13 (1e6);
    64^3 mesh: ~3 eps per cell crossed."""
    n = 400
    if mesh == "one_cell":
        wl = synth.sphere(tau0=tau0, T=1e4, n_packets=n, base=1, max_level=1)
        wl.domain = synth.Domain(0, (0.25, 0.25, 0.25), 0.2)
        wl.packets.pos[:] = 0.25
    else:
        wl = synth.sphere(tau0=tau0, T=1e4, n_packets=n, base=6, max_level=6)
    wl.physics.keep_direction = 1
    out, _ = oracle.Oracle(wl).run(threads=THREADS)
    R = wl.domain.size
    rel = out["path"] / R - 1
    assert np.all(out["status"] == oracle.ESCAPED)
    assert np.abs(rel).max() < 1e-12
    assert np.all(out["nscatt"] > 0) or tau0 < 100


def _mean_abs_x(shape):
    from scipy.integrate import quad
    num = quad(lambda y: y * shape(y), 0, 20, limit=200)[0]
    den = quad(shape, 0, 20, limit=200)[0]
    return num / den


def _escape_x(wl, out):
    ln = wl.lines[0]
    nu0, dnu = synth.nu_of(ln.lambda_A), synth.doppler_width(ln, wl.medium.T[0])
    return (out["nu"] - nu0) / dnu


@pytest.mark.slow
def test_neufeld_slab_and_harrington():
    """Extremely thick static slab (a tau0 = 1.5e3, T = 10 K, no recoil,
    isotropic; Sect. 3.4.2): the spectrum follows Neufeld (1990),
    J(x) ~ x^2 / cosh(sqrt(pi^3/54) |x|^3 / (a tau0)), whose peaks sit at
    |x| ~ 1.066 (a tau0)^(1/3); <N_scatt> is near Harrington's 1.612 tau0."""
    wl = synth.slab(tau0=1e5, T=10.0, n_packets=600)
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    x = _escape_x(wl, out)
    ln = wl.lines[0]
    dnu = synth.doppler_width(ln, 10.0)
    a = ln.A_ul / (4 * math.pi * dnu)
    at3 = (a * 1e5) ** (1 / 3)
    c = math.sqrt(math.pi ** 3 / 54)
    mx = _mean_abs_x(lambda y: 2 * y * y * math.exp(-c * y ** 3) / (1 + math.exp(-2 * c * y ** 3))) * at3
    assert abs(np.abs(x).mean() / mx - 1) < 0.06
    ratio = out["nscatt"].mean() / 1e5
    assert 1.4 < ratio < 2.2


@pytest.mark.slow
def test_dijkstra_sphere():
    """Thick static sphere (a tau0 = 1.5e3): J(x) ~ x^2 / (1 + cosh(
    sqrt(2 pi^3/27) |x|^3/(a tau0))) (Dijkstra et al. 2006, Sect. 3.4.2)."""
    wl = synth.sphere(tau0=1e5, T=10.0, n_packets=600, isotropic=1)
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    x = _escape_x(wl, out)
    ln = wl.lines[0]
    dnu = synth.doppler_width(ln, 10.0)
    a = ln.A_ul / (4 * math.pi * dnu)
    at3 = (a * 1e5) ** (1 / 3)
    c = math.sqrt(2 * math.pi ** 3 / 27)
    mx = _mean_abs_x(lambda y: 2 * y * y * math.exp(-c * y ** 3) / (1 + math.exp(-c * y ** 3)) ** 2) * at3
    assert abs(np.abs(x).mean() / mx - 1) < 0.06
    assert _chi2_sym(np.histogram(x, np.linspace(-40, 40, 41))[0]) > 1e-3


def test_peeling_flux_equals_escape():
    """Peeling (Sect. 5.1): for a static sphere with isotropic scattering,
    4 pi times the peeled flux per packet equals the escape fraction in every
    direction, and the peeled spectra match the escape spectrum."""
    n = 1500
    wl = synth.sphere(tau0=1e3, T=1e4, n_packets=n, base=3, max_level=4, isotropic=1, xrange=20)
    wl.detector.dirs = synth.PEEL_DIRS_3.copy()
    wl.detector.npix = 8
    wl.detector.fov = 1.0
    wl.physics.tau_stop = math.inf
    out, tal = oracle.Oracle(wl).run(threads=THREADS)
    flux = 4 * math.pi * tal["pspec"].sum(1) / n
    assert np.all(np.abs(flux - 1) < 0.06)
    img = 4 * math.pi * tal["pimg"].sum((1, 2)) / n
    assert np.allclose(img, flux, rtol=1e-9)
    esc = tal["spec"] / n
    for d in range(3):
        ps = 4 * math.pi * tal["pspec"][d] / n
        xs = np.arange(esc.size)
        assert abs((ps * xs).sum() / ps.sum() - (esc * xs).sum() / esc.sum()) < 2.0


def test_peeled_images_of_a_transparent_sphere():
    """Peeling at emission (Sect. 5.1) through an empty medium: each packet
    adds 1/(4 pi) (isotropic emission, e^-0 = 1) to the pixel where its
    birth point projects on the image plane of each direction (axes e_u, e_v
    orthonormal to the direction) and to the channel of its frequency."""
    n = 600
    wl = synth.sphere(tau0=0.0, T=1e4, n_packets=n, base=3, max_level=4)
    wl.detector.dirs = synth.PEEL_DIRS_3.copy()
    wl.detector.npix, wl.detector.fov = 16, 1.0
    rng = np.random.default_rng(23)
    c = np.array(wl.domain.centre)
    r = wl.domain.size * rng.random(n) ** (1 / 3) * 0.999
    v = rng.normal(size=(n, 3))
    pos = c + v / np.linalg.norm(v, axis=1)[:, None] * r[:, None]
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    nu = synth.nu_of(wl.lines[0].lambda_A) + rng.uniform(-20, 20, n) * synth.doppler_width(wl.lines[0], 1e4)
    pk = synth.Packets(pos, d, nu, np.arange(n, dtype=np.uint64) + 5)
    wl.physics.tau_stop = math.inf
    out, tal = oracle.Oracle(wl).run(packets=pk, threads=THREADS)
    assert np.all(out["status"] == oracle.ESCAPED) and np.all(out["nscatt"] == 0)
    det = wl.detector
    npix = det.npix
    img = np.zeros((3, npix, npix))
    spec = np.zeros((3, det.nbin))
    for di, ko in enumerate(det.dirs):
        ko = ko / np.linalg.norm(ko)
        eu, ev = oracle.onb(ko)
        assert abs(np.dot(eu, ko)) < 1e-15 and abs(np.dot(ev, ko)) < 1e-15
        rel = pos - np.array(det.centre)
        iu = np.floor((rel @ eu / det.fov + 0.5) * npix).astype(int)
        iv = np.floor((rel @ ev / det.fov + 0.5) * npix).astype(int)
        ok = (iu >= 0) & (iu < npix) & (iv >= 0) & (iv < npix)
        np.add.at(img[di], (iv[ok], iu[ok]), 1.0 / (4 * math.pi))
        ch = np.floor((nu - det.nu_lo) / (det.nu_hi - det.nu_lo) * det.nbin).astype(int)
        okc = (ch >= 0) & (ch < det.nbin)
        np.add.at(spec[di], ch[okc], 1.0 / (4 * math.pi))
    assert np.allclose(tal["pimg"].reshape(3, npix, npix), img, rtol=1e-12, atol=1e-15)
    assert np.allclose(tal["pspec"].reshape(3, -1), spec, rtol=1e-12, atol=1e-15)


def test_expanding_sphere_redshift():
    """Outflow (Sect. 3.4.2, expanding sphere): photons escape mostly on the
    red side of the line; in an infalling sphere (v -> -v) on the blue side,
    by the same amount (the two media are mirror images in frequency)."""
    res = {}
    for sign in (1.0, -1.0):
        wl = synth.expanding_sphere(N_HI=1e18, v_max_kms=200.0 * sign, tau_dust=0.0, n_packets=400, npix=4, nchan=8)
        wl.physics.recoil = 0
        out, _ = oracle.Oracle(wl).run(threads=8)
        h = wl.lines[0]
        x = (out["nu"] - synth.nu_of(h.lambda_A)) / synth.doppler_width(h, 1e4)
        res[sign] = x
    m_out, m_in = res[1.0].mean(), res[-1.0].mean()
    se = math.sqrt(res[1.0].var() / 400 + res[-1.0].var() / 400)
    assert m_out < -5 * res[1.0].std() / 20 and m_in > 5 * res[-1.0].std() / 20
    assert abs(m_out + m_in) < 4 * se


def test_dusty_slab_resonant_trapping():
    """Lya through an absorbing slab (Sect. 3.4.2, the escape fraction of a
    dusty slab): resonant scattering lengthens the paths, so a line photon is
    absorbed far more often than a continuum photon crossing the same dust;
    without dust every packet escapes."""
    n = 800
    f = {}
    for name, tau0, td in (("lya", 1e4, 0.1), ("continuum", 0.0, 0.1), ("no dust", 1e4, 0.0)):
        wl = synth.slab(tau0=tau0, T=100.0, tau_dust=td, albedo=0.0, n_packets=n)
        out, _ = oracle.Oracle(wl).run(threads=8)
        f[name] = (out["status"] == oracle.ESCAPED).mean()
    assert f["no dust"] == 1.0
    # continuum from the mid-plane, isotropic: escape probability E2(tau_d)
    from scipy.special import expn
    se = math.sqrt(0.25 / n)
    assert abs(f["continuum"] - expn(2, 0.1)) < 4 * se, f
    assert f["lya"] < f["continuum"] - 6 * se, f
