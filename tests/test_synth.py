"""Pins for the seeded input generator (Philox4x32-10 + Box-Muller)."""
import numpy as np
import pytest
from scipy import stats

import synth


def philox_generic(ctr, key, width, m0, m1, w0, w1, rounds=10):
    """Philox-4xW round function and key schedule (Salmon et al., SC'11)."""
    mask = (1 << width) - 1
    c = [int(x) for x in ctr]
    k = [int(x) for x in key]
    for _ in range(rounds):
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> width, p0 & mask
        hi1, lo1 = p1 >> width, p1 & mask
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
        k = [(k[0] + w0) & mask, (k[1] + w1) & mask]
    return c


def test_philox_round_structure_matches_numpy_4x64():
    # numpy's Philox is the 4x64-10 member of the same family; its round
    # function and key schedule are those of the 4x32 variant with 64-bit
    # words.  numpy increments the counter before producing a block.
    for key, ctr0 in [([12345, 678], 5), ([0, 0], 0), ([2**64 - 1, 3], 2**40)]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64))
        raw = [int(x) for x in bg.random_raw(4)]
        mine = philox_generic([ctr0 + 1, 0, 0, 0], key, 64, 0xD2E7470EE14C6C93,
                              0xCA5A826395121157, 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
        assert raw == mine


def test_philox4x32_c_matches_generic():
    rng = np.random.default_rng(1)
    for _ in range(200):
        c = [int(x) for x in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        k = [int(x) for x in rng.integers(0, 2**32, size=2, dtype=np.uint64)]
        assert synth.philox4x32_10(c, k) == philox_generic(
            c, k, 32, 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85)


def test_ln32_accuracy_on_whole_uniform_grid():
    # Every input the generator can produce: k * 2^-24, k = 1 .. 2^24.
    k = np.arange(1, 2**24 + 1, dtype=np.float64)
    x = (k * 2.0**-24).astype(np.float32)
    got = synth.ln32_array(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    err = np.abs(got - ref)
    # absolute error within a few binary32 ulps of |ln x| (ln x = 0 at x = 1 exactly)
    assert got[-1] == 0.0
    assert np.all(err <= 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-12)


def test_cossin_accuracy_on_whole_angle_grid():
    xb = (np.arange(2**24, dtype=np.uint64) << 8).astype(np.uint32)
    c, s = synth.cossin_turns_array(xb)
    ang = 2.0 * np.pi * (xb >> 8).astype(np.float64) * 2.0**-24
    assert np.max(np.abs(c - np.cos(ang))) < 3e-7
    assert np.max(np.abs(s - np.sin(ang))) < 3e-7
    # exact special angles
    assert synth.cossin_turns(0) == (1.0, 0.0)
    c4, s4 = synth.cossin_turns(0x40000000)  # quarter turn
    assert abs(c4) < 1e-7 and s4 == 1.0


def fma32(a, b, c):
    """Correctly rounded binary32 fused multiply-add, emulated in binary64: a*b is
    exact in binary64, the sum is rounded to odd (TwoSum error, then the last bit
    forced), and the odd-rounded binary64 value rounds correctly to binary32
    (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums: proved
    algorithms using rounding to odd", IEEE Trans. Computers 2008)."""
    p = np.float64(a) * np.float64(b)
    c = np.float64(c)
    s = p + c
    bb = s - p
    err = (p - (s - bb)) + (c - bb)
    if err != 0.0 and (np.array([s]).view(np.uint64)[0] & 1) == 0:
        s = np.nextafter(s, np.inf if err > 0 else -np.inf)
    return np.float32(s)


def test_fma32_emulation_on_hard_cases():
    # a*b + c whose exact value sits just beside a binary32 rounding boundary
    one = np.float32(1.0)
    eps = np.float32(2.0**-23)
    assert fma32(one + eps, one + eps, -one) == np.float32(2.0**-22 + 2.0**-46)
    assert fma32(one + eps, one - eps, -one) == np.float32(-(2.0**-46))
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a, b, c = (np.float32(v) for v in rng.standard_normal(3))
        exact = np.longdouble(a) * np.longdouble(b) + np.longdouble(c)
        got = fma32(a, b, c)
        lo, hi = np.nextafter(got, np.float32(-np.inf)), np.nextafter(got, np.float32(np.inf))
        assert abs(np.longdouble(got) - exact) <= min(abs(np.longdouble(lo) - exact),
                                                     abs(np.longdouble(hi) - exact))


def _emulated_normals_block(seed, stream, b):
    """Second implementation of the generator recipe in numpy binary32 scalars,
    operation by operation, to catch transcription errors in synth.c."""
    f32 = np.float32
    x = philox_generic([b & 0xFFFFFFFF, b >> 32, stream, 0], [seed & 0xFFFFFFFF, seed >> 32],
                       32, 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85)
    out = []
    for p in range(2):
        xa, xb = x[2 * p], x[2 * p + 1]
        ua = f32((xa >> 8) + 1) * f32(2.0**-24)
        # ln
        bits = np.array([ua], dtype=np.float32).view(np.uint32)[0]
        e = int((bits >> 23) & 0xFF) - 127
        mf = np.array([(bits & 0x7FFFFF) | 0x3F800000], dtype=np.uint32).view(np.float32)[0]
        if mf > f32(float.fromhex("0x1.6a09e6p+0")):
            mf = mf * f32(0.5)
            e += 1
        s = (mf - f32(1)) / (mf + f32(1))
        z = s * s
        q = f32(float.fromhex("0x1.745d18p-4"))
        for cst in ["0x1.c71c72p-4", "0x1.24924ap-3", "0x1.99999ap-3", "0x1.555556p-2"]:
            q = fma32(q, z, f32(float.fromhex(cst)))
        t = (s * z) * q
        lnm = (s + t) * f32(2)
        ef = f32(e)
        ln = ef * f32(float.fromhex("0x1.62e4p-1")) + fma32(ef, f32(float.fromhex("0x1.7f7d1cp-20")), lnm)
        rad = np.sqrt(f32(-2) * ln, dtype=np.float32)
        # cos/sin
        o = xb >> 29
        r = f32((xb >> 8) & 0x1FFFFF) * f32(2.0**-21)
        if o & 1:
            tt, quad, neg = f32(1) - r, ((o + 1) >> 1) & 3, True
        else:
            tt, quad, neg = r, (o >> 1) & 3, False
        psi = tt * f32(float.fromhex("0x1.921fb6p-1"))
        zz = psi * psi
        ps = f32(float.fromhex("0x1.71de3ap-19"))
        for cst in ["-0x1.a01a02p-13", "0x1.111112p-7", "-0x1.555556p-3"]:
            ps = fma32(ps, zz, f32(float.fromhex(cst)))
        sp = fma32(psi * zz, ps, psi)
        pc = f32(float.fromhex("-0x1.27e4fcp-22"))
        for cst in ["0x1.a01a02p-16", "-0x1.6c16c2p-10", "0x1.555556p-5", "-0x1.0p-1"]:
            pc = fma32(pc, zz, f32(float.fromhex(cst)))
        cp = fma32(pc, zz, f32(1))
        if neg:
            sp = -sp
        c, s_ = [(cp, sp), (-sp, cp), (-cp, -sp), (sp, -cp)][quad]
        out += [rad * c, rad * s_]
    return np.array(out, dtype=np.float32)


def test_normals_bit_exact_against_numpy_emulation():
    rng = np.random.default_rng(5)
    for seed in [0, 1, 2**40 + 17]:
        for b in [0, 1, 12345, int(rng.integers(0, 2**40))]:
            got = synth.normals(seed, 0, 4 * b, 4)
            ref = _emulated_normals_block(seed, 0, b)
            assert got.view(np.uint32).tolist() == ref.view(np.uint32).tolist()
        got = synth.normals(seed, 1, 4 * 77, 4)
        assert got.view(np.uint32).tolist() == _emulated_normals_block(seed, 1, 77).view(
            np.uint32).tolist()


def test_normals_are_standard_gaussian():
    z = synth.normals(3, 0, 0, 1 << 21).astype(np.float64)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 5e-3
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # Box-Muller with 24-bit uniforms caps |z| at sqrt(2 ln 2^24) ~ 5.77
    assert np.max(np.abs(z)) <= np.sqrt(2 * 24 * np.log(2)) + 1e-5


def test_gaussian_matrix_layout_and_scale():
    m, N = 37, 64
    A = synth.gaussian_matrix(11, m, N)
    z = synth.normals(11, 0, 0, m * N).reshape(m, N)
    scale = synth.gauss_scale(m)
    assert scale == np.float32(1.0 / np.sqrt(m))
    assert np.array_equal(A, (z * scale).astype(np.float32))
    part = synth.gaussian_matrix(11, m, N, row0=5, nrows=7)
    assert np.array_equal(part, A[5:12])


def test_measurements_noise_level():
    P = synth.make_problem(32, 0.3, 0, 6, 1e3, noise_c=1e-2)
    y = P.A.astype(np.float64) @ P.ubar.astype(np.float64).ravel()
    assert P.sigma == pytest.approx(1e-2 * np.linalg.norm(y) / np.sqrt(P.m), rel=1e-12)
    noise = P.f.astype(np.float64) - y
    assert np.std(noise) == pytest.approx(P.sigma, rel=0.2)


def test_phantom_is_deterministic_piecewise_constant():
    a = synth.phantom(64, 6, 3)
    b = synth.phantom(64, 6, 3)
    c = synth.phantom(64, 6, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert len(np.unique(a)) <= 7
    g = synth.phantom(128, 12, 1, rect_grid=True)
    assert g.shape == (128, 128) and len(np.unique(g)) <= 12 + 64 + 1


def test_sampled_m_matches_workloads():
    assert synth.sampled_m(32, 0.3) == 307
    assert synth.sampled_m(128, 0.3) == 4915
    assert synth.sampled_m(256, 0.2) == 13107
    assert synth.sampled_m(96, 0.1) == 921


def test_measure_seeded_equals_materialised():
    for n, ratio, seed in [(16, 0.3, 3), (48, 0.1, 9)]:
        P = synth.make_problem(n, ratio, seed, 4, 1e3)
        Q = synth.make_problem(n, ratio, seed, 4, 1e3, materialise=False)
        assert Q.A is None
        assert np.array_equal(P.f, Q.f) and P.sigma == Q.sigma


def test_uneven_shapes_cover_the_grid():
    shapes = [synth.uneven_shape(s) for s in range(1, 65)]
    assert all(n in synth.UNEVEN_SIDES and r in synth.UNEVEN_RATIOS for n, r in shapes)
    assert {n for n, _ in shapes} == set(synth.UNEVEN_SIDES)
    assert {r for _, r in shapes} == set(synth.UNEVEN_RATIOS)
    assert shapes == [synth.uneven_shape(s) for s in range(1, 65)]   # seeded
