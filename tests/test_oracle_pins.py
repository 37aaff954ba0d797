"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics:
hand-worked profiles, closed forms of layered media, the multiple-reflection
series, invariants of Eq. 1, exactness of trilinear sampling on linear
fields, rotation algebra, a library Philox, statistics of the speckle model,
blur identities and finite differences of the gradient."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- profiles

def test_hand_worked_profiles():
    cases = json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"]
    for c in cases:
        for method in (0, 1):
            d0, det = oracle.profile(c["Z"], c["a"], c["mode"], method)
            np.testing.assert_allclose(d0, c["d0"], rtol=0, atol=1e-14, err_msg=c["name"])
            np.testing.assert_allclose(det, c["det"], rtol=0, atol=1e-14, err_msg=c["name"])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("m", [0, 3, 9])
def test_two_layer_single_echo(mode, m):
    # Z1 in cells 0..m, Z2 beyond: one echo R a^{2(m+1)} at row m, none elsewhere
    S, a, z1, z2 = 14, 0.987, 1.5, 2.7
    Z = np.array([z1] * (m + 1) + [z2] * (S - m))
    I_ = oracle.echoes(Z, a, mode)
    r = (z2 - z1) / (z1 + z2)
    expect = np.zeros(S)
    expect[m] = (abs(r) if mode == 0 else r) * a ** (2 * (m + 1))
    np.testing.assert_allclose(I_, expect, rtol=0, atol=1e-15)


def test_homogeneous_medium_renders_zero():
    vol = I.Volume(np.full((12, 10, 9), 1.6, np.float32), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    fan = I.Fan(7, 40, math.radians(50), 9.0, 5.0, 0.5)
    pose = np.array([4.0, 4.5, 0.0, 0.1, -0.05, 0.3])
    for mode in (0, 1):
        img, ill = oracle.render(vol, pose, fan, I.Params(mode=mode))
        assert np.all(img == 0.0) and not ill.any()


@pytest.mark.parametrize("mode", [0, 1])
def test_three_layer_airy_sum(mode):
    # Layers Z1 (cells 0..m), Z2 (L cells), Z3: the full-depth profile is the
    # Airy sum  a^{2m} [a^2 R1 + a^2 T1 T1' rho2 / (1 - R1' rho2)],
    # rho2 = a^{2L} R2, and the echoes sit at rows m and m+L.
    m, L, S, a = 4, 5, 16, 0.99
    z1, z2, z3 = 1.4, 2.9, 1.7
    Z = np.array([z1] * (m + 1) + [z2] * L + [z3] * (S - m - L))
    d0, _ = oracle.profile(Z, a, mode)

    def co(x, y):
        r = (y - x) / (x + y)
        return (abs(r), abs(r)) if mode == 0 else (r, -r), 2 * y / (x + y), 2 * x / (x + y)

    (R1, R1p), T1, T1p = co(z1, z2)
    (R2, _), _, _ = co(z2, z3)
    rho2 = a ** (2 * L) * R2
    full = a ** (2 * m) * (a * a * R1 + a * a * T1 * T1p * rho2 / (1 - R1p * rho2))
    assert abs(d0[-1] - full) < 1e-15
    I_ = np.diff(d0)
    nz = np.nonzero(np.abs(I_) > 1e-15)[0]
    assert list(nz) == [m, m + L]
    assert abs(I_[m] - a ** (2 * (m + 1)) * R1) < 1e-15


def _series_by_bounce(Z, a, mode, k, orders):
    """d_0^(k) as the multiple-reflection series: generation g holds the
    waves that turned downward g times at an interface (R' events); each
    generation is propagated exactly through transmissions and upward
    reflections.  Returns the partial sums after each generation."""
    S = len(Z) - 1
    R = np.zeros(S); Rp = np.zeros(S); T = np.zeros(S); Tp = np.zeros(S)
    for i in range(S):
        z1, z2 = Z[i], Z[i + 1]
        r = (z2 - z1) / (z1 + z2)
        R[i], Rp[i] = (abs(r), abs(r)) if mode == 0 else (r, -r)
        T[i], Tp[i] = 2 * z2 / (z1 + z2), 2 * z1 / (z1 + z2)
    fwd = np.zeros(k + 1)   # forward amplitude entering cell i at its near face
    fwd[0] = 1.0
    sums, total = [], 0.0
    for _ in range(orders):
        # forward sweep: forward waves travel down; at each interface they
        # transmit (stay in this generation) or reflect upward
        up_src = np.zeros(k + 1)  # upward wave created at the near face of cell i
        f = fwd.copy()
        for i in range(k):
            up_src[i] += a * a * R[i] * f[i]
            f[i + 1] += a * T[i] * f[i]
        # f[k] leaves the truncated ray (d_k = 0)
        # upward sweep: backward waves travel up, transmitting (upward) or
        # reflecting downward into the next generation
        nxt = np.zeros(k + 1)
        b = 0.0
        for i in range(k, -1, -1):
            b = b + up_src[i] if i < k else up_src[i]
            if i == 0:
                total += b
                break
            nxt[i] += Rp[i - 1] * b
            b = a * Tp[i - 1] * b
        fwd = nxt
        sums.append(total)
    return np.array(sums)


@pytest.mark.parametrize("mode", [0, 1])
def test_multiple_reflection_series_converges_to_solve(mode):
    rng = np.random.default_rng(11)
    for trial in range(6):
        S = int(rng.integers(2, 7))
        Z = rng.uniform(1.0, 3.0, size=S + 1)
        a = float(rng.uniform(0.9, 1.0))
        d0, _ = oracle.profile(Z, a, mode)
        for k in range(1, S + 1):
            sums = _series_by_bounce(Z, a, mode, k, 60)
            assert abs(sums[-1] - d0[k]) < 1e-12
            if k >= 2:
                # the first generation is the single-scattering sum
                single = 0.0
                amp = 1.0
                for i in range(k):
                    z1, z2 = Z[i], Z[i + 1]
                    r = (z2 - z1) / (z1 + z2)
                    Ri = abs(r) if mode == 0 else r
                    single += amp * a * a * Ri
                    amp *= a * a * (2 * z2 / (z1 + z2)) * (2 * z1 / (z1 + z2))
                assert abs(sums[0] - single) < 1e-14


def test_banded_equals_dense():
    rng = np.random.default_rng(5)
    for mode in (0, 1):
        Z = rng.uniform(1.3, 1.8, size=41)
        Z[17:19] = 7.8
        a = 0.993
        d0b, detb = oracle.profile(Z, a, mode, 0)
        d0d, detd = oracle.profile(Z, a, mode, 1)
        np.testing.assert_allclose(d0b, d0d, rtol=0, atol=1e-13)
        np.testing.assert_allclose(detb, detd, rtol=1e-12, atol=1e-13)


def test_determinant_is_product_of_interface_denominators():
    # det(A_k) = prod_i (1 - R'_i rho_{i+1}^{(k)}): the denominators met when
    # the recurrences are eliminated from the deepest interface upward.
    rng = np.random.default_rng(3)
    for mode in (0, 1):
        Z = rng.uniform(1.2, 3.5, size=12)
        a = 0.97
        _, det = oracle.profile(Z, a, mode)
        for k in range(1, len(Z)):
            rho, prod = 0.0, 1.0
            for i in range(k - 1, -1, -1):
                R, Rp, T, Tp = oracle.coeffs(Z[i], Z[i + 1], mode)
                prod *= 1.0 - Rp * rho
                rho = a * a * (R + T * Tp * rho / (1.0 - Rp * rho))
            assert abs(det[k] - prod) < 1e-13


def test_literal_profile_monotone_and_signed_bounded():
    # literal mode: every path amplitude is non-negative, so deeper systems
    # only add echo energy up to the first pole
    rng = np.random.default_rng(8)
    Z = 1.54 + rng.normal(0.0, 0.01, size=300)
    d0, det = oracle.profile(Z, 0.995, 0)
    assert (det > 1e-6).all()
    assert (np.diff(d0) >= 0).all()
    Z = rng.uniform(1.38, 1.70, size=300)
    d0, det = oracle.profile(Z, 0.995, 0)
    first = int(np.argmax(det < 1e-6)) if (det < 1e-6).any() else len(det)
    assert first > 2 and (np.diff(d0[:first]) >= 0).all()
    for _ in range(20):
        Z = rng.uniform(1.0, 8.0, size=60)
        d0, det = oracle.profile(Z, 1.0, 1)
        assert np.abs(d0).max() <= 1.0 + 1e-12


def test_coefficient_invariants():
    rng = np.random.default_rng(2)
    for _ in range(200):
        z1, z2 = rng.uniform(0.5, 9.0, size=2)
        R, Rp, T, Tp = oracle.coeffs(z1, z2, 0)
        assert 0 <= R <= 1 and R == Rp
        r, rp, T2, Tp2 = oracle.coeffs(z1, z2, 1)
        assert abs(1 + r - T2) < 1e-15 and abs(1 - r - Tp2) < 1e-15 and rp == -r
        assert abs(T2 * Tp2 - (1 - r * r)) < 1e-15
        assert abs(R - abs(r)) < 1e-16


# -------------------------------------------------------------- geometry

def _vol(data, sp=(1.0, 1.0, 1.0), org=(0.0, 0.0, 0.0)):
    return I.Volume(np.ascontiguousarray(data, dtype=np.float32), sp, org)


def test_trilinear_reproduces_linear_fields_and_clamps():
    nz, ny, nx = 6, 7, 9
    sp, org = (0.5, 1.5, 2.0), (3.0, -1.0, 2.5)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    px, py, pz = org[0] + sp[0] * xx, org[1] + sp[1] * yy, org[2] + sp[2] * zz
    c = (0.25, -0.5, 0.125, 2.0)
    data = c[0] * px + c[1] * py + c[2] * pz + c[3]
    vol = _vol(data, sp, org)
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = np.array([org[0] + rng.uniform(0, sp[0] * (nx - 1)), org[1] + rng.uniform(0, sp[1] * (ny - 1)),
                      org[2] + rng.uniform(0, sp[2] * (nz - 1))])
        v, g = oracle.trilinear(vol, p)
        assert abs(v - (c[0] * p[0] + c[1] * p[1] + c[2] * p[2] + c[3])) < 1e-5
        np.testing.assert_allclose(g, c[:3], atol=1e-5)
    # voxel centres give the stored value
    v, _ = oracle.trilinear(vol, [org[0] + 2 * sp[0], org[1] + 3 * sp[1], org[2] + 4 * sp[2]])
    assert v == float(np.float32(data[4, 3, 2]))
    # outside: border value, no gradient across the clamped axis
    v, g = oracle.trilinear(vol, [org[0] - 5.0, org[1] + 1.5 * sp[1], org[2] + 1.0 * sp[2]])
    v2, _ = oracle.trilinear(vol, [org[0], org[1] + 1.5 * sp[1], org[2] + 1.0 * sp[2]])
    assert v == v2 and g[0] == 0.0 and g[1] != 0.0


def test_rotation_algebra():
    rng = np.random.default_rng(4)
    for _ in range(10):
        r = rng.uniform(-3, 3, size=3)
        R, dR = oracle.rotation(r)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        h = 1e-6
        for q in range(3):
            e = np.zeros(3); e[q] = h
            fd = (oracle.rotation(r + e)[0] - oracle.rotation(r - e)[0]) / (2 * h)
            np.testing.assert_allclose(dR[q], fd, atol=1e-8)
    # R = Rz(pi/2): x -> y, y -> -x
    R, _ = oracle.rotation([0, 0, math.pi / 2])
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    # ZYX order: Rz(a) Ry(b) applied to x
    a, b = 0.3, 0.4
    R, _ = oracle.rotation([0, b, a])
    np.testing.assert_allclose(R @ [1, 0, 0], [math.cos(a) * math.cos(b), math.sin(a) * math.cos(b), -math.sin(b)],
                               atol=1e-15)


def test_fan_geometry():
    fan = I.Fan(5, 8, math.radians(60), 40.0, 5.0, 0.5)
    pose = np.array([1.0, 2.0, 3.0, 0.0, 0.0, 0.0])
    ds = fan.depth / fan.n_samples
    for j, th in enumerate(np.linspace(-math.pi / 6, math.pi / 6, 5)):
        pos = oracle.ray_positions(pose, fan, j)
        np.testing.assert_allclose(pos[0], [1 + 0.5 * ds * math.sin(th), 2.0, 3 + 0.5 * ds * math.cos(th)], atol=1e-14)
        np.testing.assert_allclose(np.diff(pos, axis=0), np.tile([ds * math.sin(th), 0, ds * math.cos(th)], (8, 1)),
                                   atol=1e-13)
    one = I.Fan(1, 4, 1.0, 4.0)
    pos = oracle.ray_positions(pose, one, 0)
    np.testing.assert_allclose(pos[:, :2], np.tile([1.0, 2.0], (5, 1)), atol=1e-15)


def test_attenuation_round_trip_in_decibels():
    fan = I.Fan(4, 256, 1.0, 60.0, 5.0, 0.5)
    a = oracle.attenuation(fan)
    # round trip over the full depth: -2 alpha f depth[cm] dB
    assert abs(20 * math.log10(a ** (2 * 256)) - (-2 * 0.5 * 5.0 * 6.0)) < 1e-9


# ---------------------------------------------------------------- Philox

def test_philox_matches_triton_library_routine():
    """Philox4x32-10 against triton's philox, run by triton's CPU interpreter
    in a subprocess (the interpreter is switched on by an environment
    variable read at import)."""
    import subprocess
    import sys
    pytest.importorskip("triton")
    code = r'''
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
sys.path.insert(0, %r)
import numpy as np, torch, triton, triton.language as tl
import oracle

@triton.jit
def k(out_ptr, seed, c0_ptr, c1, c2, c3, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c0_ptr + offs)
    z = c0 * 0
    a, b, c, d = tl.philox(seed, c0, z + c1, z + c2, z + c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)

N = 64
bad = 0
for seed, c1, c2, c3 in [(0, 0, 0, 0), (0x1234567890ABCDEF, 7, 3, 1), (42, 1000, 511, 1)]:
    c0 = torch.arange(N, dtype=torch.int32) * 104729 + 17
    out = torch.zeros(N * 4, dtype=torch.int32)
    k[(1,)](out, seed, c0, c1, c2, c3, N=N)
    got = out.view(N, 4).numpy().view(np.uint32)
    ref = np.array([oracle.philox([int(c0[i]), c1, c2, c3], [seed & 0xffffffff, seed >> 32]) for i in range(N)])
    bad += int((got != ref).sum())
print("MISMATCH", bad)
''' % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if "MISMATCH" not in r.stdout:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    assert "MISMATCH 0" in r.stdout


def test_philox_bytes_uniform():
    counts = np.zeros(256)
    for i in range(3000):
        w = oracle.philox([i, 1, 2, 3], [99, 0])
        for x in w:
            for s in (0, 8, 16, 24):
                counts[(int(x) >> s) & 255] += 1
    n = counts.sum()
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)


# --------------------------------------------------------------- speckle

def test_speckle_off_is_one_and_statistics():
    S = 64
    p = I.Params(speckle=0)
    assert np.all(oracle.speckle(p, 0, 3, S) == 1.0)
    p = I.Params(Ar=0.1, pr=1.0, Ag=0.05, pg=0.5, Lr=2, gshift=0)
    M = np.array([oracle.speckle(p, 5, j, S) for j in range(400)])
    z = (np.arange(S) + 1) / S
    var = 0.1 ** 2 * z ** 2 + 0.05 ** 2 * z
    assert abs(M.mean() - 1.0) < 0.01
    ratio = M.var(axis=0)[S // 2:] / var[S // 2:]
    assert 0.8 < ratio.mean() < 1.2


def test_radial_term_is_a_moving_average():
    # with the grain term off, n_r(k) and n_r(k+d) share 2L+1-d of their
    # 2L+1 white terms: correlation (2L+1-d)/(2L+1), zero beyond 2L
    S, L = 64, 3
    p = I.Params(Ar=1.0, pr=0.0, Ag=0.0, Lr=L)
    X = np.array([oracle.speckle(p, 1, j, S) for j in range(600)]) - 1.0
    for d in (1, 3, 6, 8):
        c = np.mean(X[:, :-d] * X[:, d:]) / np.mean(X * X)
        assert abs(c - max(0, 2 * L + 1 - d) / (2 * L + 1)) < 0.06


def test_grain_cells_grow_with_depth():
    S, gs = 200, 1
    p = I.Params(Ar=0.0, Ag=1.0, pg=0.0, gshift=gs)
    m = oracle.speckle(p, 2, 7, S)
    for b in range(4):
        k0, k1 = -(-b * S // 4), -(-(b + 1) * S // 4)
        L = 2 ** (gs + b)
        for s in range(k0, k1, L):
            seg = m[s:min(s + L, k1)]
            assert np.all(seg == seg[0])
        # consecutive cells almost surely differ
        starts = list(range(k0, k1, L))
        assert sum(m[s] != m[s - 1] for s in starts[1:]) >= len(starts) - 3


# ------------------------------------------------------------------ blur

def test_blur_identities():
    rng = np.random.default_rng(1)
    y = rng.normal(size=(23, 17))
    ident = I.Params(sigma0=1e-9, sigma1=0.0)
    assert np.array_equal(oracle.blur(ident, y), y)
    p = I.Params(sigma0=0.5, sigma1=1.5)
    const = np.full((23, 17), 2.5)
    np.testing.assert_allclose(oracle.blur(p, const), const, rtol=1e-15)
    x = rng.normal(size=(23, 17)); w = rng.normal(size=(23, 17))
    assert abs(np.sum(oracle.blur(p, x) * w) - np.sum(x * oracle.blur_T(p, w))) < 1e-12
    # an interior impulse spreads as the normalised Gaussian of its row
    d = np.zeros((40, 8)); d[20, 5] = 1.0
    out = oracle.blur(p, d)
    sig = 0.5 + 1.5 * 6 / 8
    W = int(math.ceil(3 * 2.0))
    w_ = np.exp(-np.arange(-W, W + 1) ** 2 / (2 * sig * sig))
    np.testing.assert_allclose(out[20 - W:21 + W, 5], w_ / w_.sum(), rtol=1e-14)
    assert np.all(out[:, :5] == 0) and np.all(out[:, 6:] == 0)


# ------------------------------------------------------------- gradients

def test_profile_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    for mode in (0, 1):
        Z = rng.uniform(1.3, 2.5, size=15)
        a = 0.98
        gd0 = rng.normal(size=15)
        gd0[0] = 0.0
        g = oracle.profile_grad(Z, a, mode, gd0)
        h = 1e-6
        for i in range(15):
            e = np.zeros(15); e[i] = h
            fd = (np.dot(gd0, oracle.profile(Z + e, a, mode)[0]) - np.dot(gd0, oracle.profile(Z - e, a, mode)[0])) / (2 * h)
            assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd))


def test_render_gradient_matches_finite_differences():
    rng = np.random.default_rng(12)
    data = 1.5 + 0.15 * rng.random((10, 9, 11))
    data[5:7, :, :] += 0.8
    vol = I.Volume(data.astype(np.float32), (1.0, 1.2, 0.9), (0.5, -0.3, 0.2))
    fan = I.Fan(6, 24, math.radians(40), 7.0, 6.0, 0.6)
    pose = np.array([5.3, 4.9, 0.4, 0.05, -0.07, 0.2])
    for params in (I.Params(seed=3), I.Params(seed=3, mode=1, sigma0=0.4, sigma1=1.0)):
        img, ill = oracle.render(vol, pose, fan, params)
        assert not ill.any()
        G = rng.normal(size=img.shape)
        gvol, gpose = oracle.render_grad(vol, pose, fan, params, G)

        def loss(v=vol, p=pose):
            return float(np.sum(G * oracle.render(v, p, fan, params)[0]))

        h = 1e-6
        for q in range(6):
            e = np.zeros(6); e[q] = h
            fd = (loss(p=pose + e) - loss(p=pose - e)) / (2 * h)
            assert abs(fd - gpose[q]) < 1e-6 * max(1.0, abs(fd)), (q, fd, gpose[q])
        # the volume is float32: perturb in float64 copies through the float32
        # path with a step that float32 represents exactly
        hv = 2.0 ** -12
        for idx in [(5, 4, 5), (6, 2, 3), (3, 7, 8), (5, 5, 5)]:
            dp = data.astype(np.float32).copy(); dm = dp.copy()
            dp[idx] += np.float32(hv); dm[idx] -= np.float32(hv)
            fd = (loss(v=I.Volume(dp, vol.spacing, vol.origin)) - loss(v=I.Volume(dm, vol.spacing, vol.origin))) / (2 * hv)
            assert abs(fd - gvol[idx]) < 2e-5 * max(1.0, abs(fd)), (idx, fd, gvol[idx])


def _layered_ray(layers, S, ds=1.0):
    """One straight-down ray whose sample k sits exactly on voxel centre k of
    a volume layered along z: returns (vol, pose, fan) with Z_k = layers[k]."""
    z = np.asarray(layers, np.float32)
    vol = I.Volume(np.broadcast_to(z[:, None, None], (z.size, 3, 3)).copy(), (ds, ds, ds), (0.0, 0.0, 0.0))
    pose = np.array([1.0, 1.0, -0.5 * ds, 0.0, 0.0, 0.0])     # sample k at z = k ds
    fan = I.Fan(1, S, 0.0, S * ds, 5.0, 0.5)
    return vol, pose, fan


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_gain_reading_two_layer_equals_in_system(mode):
    # one interface: a single echo R a^{2(m+1)} at row m in both attenuation readings
    S, m = 20, 7
    z1, z2 = float(np.float32(1.5)), float(np.float32(2.6))      # the volume stores float32
    vol, pose, fan = _layered_ray([z1] * (m + 1) + [z2] * (S - m), S)
    a = oracle.attenuation(fan)
    r = (z2 - z1) / (z1 + z2)
    expect = np.zeros(S)
    expect[m] = (abs(r) if mode == 0 else r) * a ** (2 * (m + 1))
    for atten in (0, 1):
        img, _ = oracle.render(vol, pose, fan, I.Params(mode=mode, speckle=0, blur=0, atten=atten))
        np.testing.assert_allclose(img[0], expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_gain_reading_three_layer_airy(mode):
    # two interfaces at rows m and m+L: with the depth gain the second echo is
    # a^{2(m+L+1)} T1 T1' R2 / (1 - R1' R2) (lossless multiple reflections),
    # inside the system it is a^{2(m+L+1)} T1 T1' R2 / (1 - R1' a^{2L} R2)
    S, m, L = 24, 5, 6
    z1, z2, z3 = (float(np.float32(v)) for v in (1.4, 2.9, 1.7))
    vol, pose, fan = _layered_ray([z1] * (m + 1) + [z2] * L + [z3] * (S - m - L), S)
    a = oracle.attenuation(fan)

    def co(x, y):
        r = (y - x) / (x + y)
        return (abs(r), abs(r)) if mode == 0 else (r, -r), 2 * y / (x + y), 2 * x / (x + y)

    (R1, R1p), T1, T1p = co(z1, z2)
    (R2, _), _, _ = co(z2, z3)
    g = a ** (2 * (m + L + 1))
    gain_img, _ = oracle.render(vol, pose, fan, I.Params(mode=mode, speckle=0, blur=0, atten=1))
    sys_img, _ = oracle.render(vol, pose, fan, I.Params(mode=mode, speckle=0, blur=0, atten=0))
    assert abs(gain_img[0, m + L] - g * T1 * T1p * R2 / (1 - R1p * R2)) < 1e-14
    assert abs(sys_img[0, m + L] - g * T1 * T1p * R2 / (1 - R1p * a ** (2 * L) * R2)) < 1e-14
    assert abs(gain_img[0, m + L] - sys_img[0, m + L]) > 1e-6
