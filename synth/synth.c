/*
 * Seeded synthetic inputs for the TV/L2 reconstruction problem
 *     min_u  sum_i ||D_i u||_2 + (mu/2) ||A u - f||_2^2
 * (Xiao & Yang, "A Fast Algorithm for Total Variation Image Reconstruction
 * from Random Projections", Sec. 1, eqs. (obser) and (tv)).
 *
 * This file generates INPUTS only: the Gaussian encoding matrix A, the
 * measurement noise, and the measurements f = A*ubar + noise.  It contains
 * none of the solver's arithmetic.  Both the CPU oracle's tests and the GPU
 * path's tests/benchmark draw their inputs from here.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), a counter-based generator, so that
 * any entry A[i][j] is a pure function of (seed, i*N + j) and can be
 * regenerated anywhere.  Gaussians come from the Box-Muller transform
 * (Box & Muller, Ann. Math. Stat. 1958) with a natural logarithm and a
 * sine/cosine written here from their Taylor series; every floating-point
 * operation is a single IEEE binary32 operation in a fixed order -- the
 * polynomial steps are fused multiply-adds (C99 fmaf, one rounding), every
 * other step a plain operation (this translation unit must be compiled with
 * -ffp-contract=off so that nothing else is fused) -- so the values are
 * bit-reproducible on any IEEE machine.
 *
 * The generator recipe, stated once (the GPU path implements the same recipe
 * independently for in-kernel regeneration):
 *   element e of stream s  ->  block b = e >> 2, lane = e & 3
 *   (x0,x1,x2,x3) = Philox4x32-10(counter = (lo32(b), hi32(b), s, 0),
 *                                 key     = (lo32(seed), hi32(seed)))
 *   lanes 0,1 use the pair (x0,x1); lanes 2,3 use the pair (x2,x3)
 *   pair (xa,xb):  ua = ((xa >> 8) + 1) * 2^-24         in (0, 1]
 *                  rad = sqrt(-2 * ln(ua))
 *                  angle = 2*pi*(xb >> 8)*2^-24        (via cossin_turns)
 *                  even lane -> rad*cos(angle), odd lane -> rad*sin(angle)
 *   A[i][j] = binary32( z(e = i*N + j, s = 0) * scale ),
 *   scale   = binary32( 1 / sqrt((double) m) )
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

#define SYNTH_EXPORT __attribute__((visibility("default")))

/* Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

SYNTH_EXPORT void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                                      uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float f_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ln(x) for x in (0, 1], x a normal binary32.  x = 2^e * mfrac with
 * mfrac in [sqrt(1/2), sqrt(2)); ln(mfrac) = 2*atanh(s), s = (mfrac-1)/(mfrac+1),
 * atanh(s) = s + s^3/3 + s^5/5 + ... truncated after s^11/11 (|s| <= 0.1716,
 * truncation error below 2^-30 relative). ln 2 = LN2_HI + LN2_LO with LN2_HI
 * carrying 16 significant bits so that e*LN2_HI is exact. */
SYNTH_EXPORT float synth_ln(float x)
{
    const float SQRT2 = 0x1.6a09e6p+0f;
    const float LN2_HI = 0x1.62e4p-1f;
    const float LN2_LO = 0x1.7f7d1cp-20f;
    const float Q3 = 0x1.555556p-2f, Q5 = 0x1.99999ap-3f, Q7 = 0x1.24924ap-3f,
                Q9 = 0x1.c71c72p-4f, Q11 = 0x1.745d18p-4f;
    uint32_t b = bits_from_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float mf = f_from_bits((b & 0x7fffffu) | 0x3f800000u);
    if (mf > SQRT2) { mf = mf * 0.5f; e += 1; }
    float num = mf - 1.0f;
    float den = mf + 1.0f;
    float s = num / den;
    float z = s * s;
    float q = Q11;
    q = fmaf(q, z, Q9);
    q = fmaf(q, z, Q7);
    q = fmaf(q, z, Q5);
    q = fmaf(q, z, Q3);
    float t = s * z;
    t = t * q;
    float lnm = s + t;
    lnm = lnm * 2.0f;
    float ef = (float)e;
    float hi = ef * LN2_HI;
    float lo = fmaf(ef, LN2_LO, lnm);
    return hi + lo;
}

/* cos and sin of 2*pi*(xb >> 8)*2^-24.  The top 3 bits pick the octant o and
 * the next 21 bits the position r in it (exact).  angle = (o + r)*pi/4
 * = Q*pi/2 + sgn*psi with psi in [0, pi/4]; sin/cos of psi by Taylor series to
 * psi^9 / psi^10 (remainder below 2^-29). */
SYNTH_EXPORT void synth_cossin_turns(uint32_t xb, float* c_out, float* s_out)
{
    const float PI_4 = 0x1.921fb6p-1f;
    const float S3 = -0x1.555556p-3f, S5 = 0x1.111112p-7f, S7 = -0x1.a01a02p-13f,
                S9 = 0x1.71de3ap-19f;
    const float C2 = -0x1.0p-1f, C4 = 0x1.555556p-5f, C6 = -0x1.6c16c2p-10f,
                C8 = 0x1.a01a02p-16f, C10 = -0x1.27e4fcp-22f;
    uint32_t o = xb >> 29;
    uint32_t rbits = (xb >> 8) & 0x1fffffu;
    float r = (float)rbits * 0x1.0p-21f;
    float t;
    uint32_t quad;
    int neg;
    if (o & 1u) { t = 1.0f - r; quad = ((o + 1u) >> 1) & 3u; neg = 1; }
    else        { t = r;        quad = (o >> 1) & 3u;        neg = 0; }
    float psi = t * PI_4;
    float z = psi * psi;
    float ps = S9;
    ps = fmaf(ps, z, S7);
    ps = fmaf(ps, z, S5);
    ps = fmaf(ps, z, S3);
    float sp = psi * z;
    sp = fmaf(sp, ps, psi);
    float pc = C10;
    pc = fmaf(pc, z, C8);
    pc = fmaf(pc, z, C6);
    pc = fmaf(pc, z, C4);
    pc = fmaf(pc, z, C2);
    float cp = fmaf(pc, z, 1.0f);
    if (neg) sp = -sp;
    float c, s;
    switch (quad) {
        case 0: c = cp;  s = sp;  break;
        case 1: c = -sp; s = cp;  break;
        case 2: c = -cp; s = -sp; break;
        default: c = sp; s = -cp; break;
    }
    *c_out = c;
    *s_out = s;
}

/* Standard normal deviates for elements e0 .. e0+count-1 of stream s. */
static void normals_block(uint64_t seed, uint32_t stream, uint64_t b, float z[4])
{
    uint32_t ctr[4] = { (uint32_t)b, (uint32_t)(b >> 32), stream, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    synth_philox4x32_10(ctr, key, x);
    for (int p = 0; p < 2; ++p) {
        uint32_t xa = x[2 * p], xb = x[2 * p + 1];
        float ua = (float)((xa >> 8) + 1u) * 0x1.0p-24f;
        float l = synth_ln(ua);
        float v = -2.0f * l;
        float rad = sqrtf(v);
        float c, s;
        synth_cossin_turns(xb, &c, &s);
        z[2 * p] = rad * c;
        z[2 * p + 1] = rad * s;
    }
}

SYNTH_EXPORT void synth_normals(uint64_t seed, uint32_t stream, uint64_t e0, int64_t count,
                                float* out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        uint64_t e = e0 + (uint64_t)k;
        float z[4];
        normals_block(seed, stream, e >> 2, z);
        out[k] = z[e & 3u];
    }
}

/* scale = binary32(1/sqrt(m)), computed in binary64 then rounded once. */
SYNTH_EXPORT float synth_gauss_scale(int m)
{
    return (float)(1.0 / sqrt((double)m));
}

/* Rows [row0, row0+nrows) of the m x N Gaussian encoding matrix, row-major,
 * A[i][j] = binary32(z(i*N + j, stream 0) * scale). */
SYNTH_EXPORT void synth_gaussian_rows(uint64_t seed, int m, int64_t N, int64_t row0,
                                      int64_t nrows, float* out)
{
    const float scale = synth_gauss_scale(m);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nrows; ++i) {
        const uint64_t base = (uint64_t)(row0 + i) * (uint64_t)N;
        float* orow = out + i * N;
        int64_t j = 0;
        while (j < N) {
            uint64_t e = base + (uint64_t)j;
            float z[4];
            normals_block(seed, 0u, e >> 2, z);
            for (uint32_t l = (uint32_t)(e & 3u); l < 4u && j < N; ++l, ++j)
                orow[j] = z[l] * scale;
        }
    }
}

/* Measurements f = A*ubar + sigma*eps (eq. obser with additive Gaussian noise):
 * y = A*ubar accumulated in binary64 per row, sigma = c * ||y|| / sqrt(m)
 * (c times the RMS of A*ubar), eps_i = z(i, stream 1 of noise_seed),
 * f_i = binary32(y_i + sigma*eps_i).  Returns sigma. */
SYNTH_EXPORT double synth_measure(const float* A, int m, int64_t N, const float* ubar,
                                  double c, uint64_t noise_seed, float* f_out)
{
    double* y = (double*)malloc(sizeof(double) * (size_t)m);
    float* eps = (float*)malloc(sizeof(float) * (size_t)m);
    if (!y || !eps) { free(y); free(eps); return -1.0; }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        const float* a = A + (int64_t)i * N;
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += (double)a[j] * (double)ubar[j];
        y[i] = acc;
    }
    double ss = 0.0;
    for (int i = 0; i < m; ++i) ss += y[i] * y[i];
    double sigma = c * sqrt(ss) / sqrt((double)m);
    synth_normals(noise_seed, 1u, 0u, m, eps);
    for (int i = 0; i < m; ++i) f_out[i] = (float)(y[i] + sigma * (double)eps[i]);
    free(y);
    free(eps);
    return sigma;
}

/* The same measurements without a stored A: row i of A is generated, as in
 * synth_gaussian_rows, while it is multiplied with ubar (same binary64
 * accumulation order), so f equals synth_measure's for the same seed. */
SYNTH_EXPORT double synth_measure_seeded(uint64_t seed, int m, int64_t N, const float* ubar,
                                         double c, uint64_t noise_seed, float* f_out)
{
    double* y = (double*)malloc(sizeof(double) * (size_t)m);
    float* eps = (float*)malloc(sizeof(float) * (size_t)m);
    if (!y || !eps) { free(y); free(eps); return -1.0; }
    const float scale = synth_gauss_scale(m);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < m; ++i) {
        const uint64_t base = (uint64_t)i * (uint64_t)N;
        double acc = 0.0;
        int64_t j = 0;
        while (j < N) {
            uint64_t e = base + (uint64_t)j;
            float z[4];
            normals_block(seed, 0u, e >> 2, z);
            for (uint32_t l = (uint32_t)(e & 3u); l < 4u && j < N; ++l, ++j)
                acc += (double)(z[l] * scale) * (double)ubar[j];
        }
        y[i] = acc;
    }
    double ss = 0.0;
    for (int i = 0; i < m; ++i) ss += y[i] * y[i];
    double sigma = c * sqrt(ss) / sqrt((double)m);
    synth_normals(noise_seed, 1u, 0u, m, eps);
    for (int i = 0; i < m; ++i) f_out[i] = (float)(y[i] + sigma * (double)eps[i]);
    free(y);
    free(eps);
    return sigma;
}

/* Array forms of the two elementary functions, for tests. */
SYNTH_EXPORT void synth_ln_array(int64_t count, const float* x, float* out)
{
    for (int64_t i = 0; i < count; ++i) out[i] = synth_ln(x[i]);
}

SYNTH_EXPORT void synth_cossin_array(int64_t count, const uint32_t* xb, float* c, float* s)
{
    for (int64_t i = 0; i < count; ++i) synth_cossin_turns(xb[i], &c[i], &s[i]);
}
