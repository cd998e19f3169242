// Counter-based Gaussian generator shared by the kernels that produce the
// encoding matrix: k_gen.cu writes A to memory, k_regen.cu regenerates it tile
// by tile inside the product kernel.  The recipe is stated at the top of
// k_gen.cu; every floating-point step is a single binary32 operation with
// round-to-nearest (explicit __f*_rn intrinsics: the polynomial steps are fused
// multiply-adds, nothing else is contracted), which makes the values identical
// to the host-side input generator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tvcs {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c[0];
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ float gen_ln(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float mf = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    const bool big = mf > 0x1.6a09e6p+0f;   // selects, not branches
    mf = big ? __fmul_rn(mf, 0.5f) : mf;
    e += big ? 1 : 0;
    const float s = __fdiv_rn(__fsub_rn(mf, 1.0f), __fadd_rn(mf, 1.0f));
    const float z = __fmul_rn(s, s);
    float q = 0x1.745d18p-4f;
    q = __fmaf_rn(q, z, 0x1.c71c72p-4f);
    q = __fmaf_rn(q, z, 0x1.24924ap-3f);
    q = __fmaf_rn(q, z, 0x1.99999ap-3f);
    q = __fmaf_rn(q, z, 0x1.555556p-2f);
    const float t = __fmul_rn(__fmul_rn(s, z), q);
    const float lnm = __fmul_rn(__fadd_rn(s, t), 2.0f);
    const float ef = (float)e;
    const float hi = __fmul_rn(ef, 0x1.62e4p-1f);
    const float lo = __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnm);
    return __fadd_rn(hi, lo);
}

__device__ __forceinline__ void gen_cossin(uint32_t xb, float& c, float& s)
{
    const uint32_t o = xb >> 29;
    const float r = __fmul_rn((float)((xb >> 8) & 0x1fffffu), 0x1.0p-21f);
    const bool odd = (o & 1u) != 0u;
    const float t = odd ? __fsub_rn(1.0f, r) : r;
    const uint32_t quad = ((o + (odd ? 1u : 0u)) >> 1) & 3u;
    const float psi = __fmul_rn(t, 0x1.921fb6p-1f);
    const float z = __fmul_rn(psi, psi);
    float ps = 0x1.71de3ap-19f;
    ps = __fmaf_rn(ps, z, -0x1.a01a02p-13f);
    ps = __fmaf_rn(ps, z, 0x1.111112p-7f);
    ps = __fmaf_rn(ps, z, -0x1.555556p-3f);
    float sp = __fmaf_rn(__fmul_rn(psi, z), ps, psi);
    float pc = -0x1.27e4fcp-22f;
    pc = __fmaf_rn(pc, z, 0x1.a01a02p-16f);
    pc = __fmaf_rn(pc, z, -0x1.6c16c2p-10f);
    pc = __fmaf_rn(pc, z, 0x1.555556p-5f);
    pc = __fmaf_rn(pc, z, -0x1.0p-1f);
    const float cp = __fmaf_rn(pc, z, 1.0f);
    if (odd) sp = -sp;
    // rotate by quad quarter turns: (c, s) = (cp, sp), (-sp, cp), (-cp, -sp), (sp, -cp)
    const bool swap = (quad & 1u) != 0u;
    const float cc = swap ? sp : cp;
    const float ss = swap ? cp : sp;
    c = (quad == 1u || quad == 2u) ? -cc : cc;
    s = (quad >= 2u) ? -ss : ss;
}

// Four consecutive standard normals of block b of stream `stream`.
__device__ __forceinline__ float4 gen_normals4(uint64_t seed, uint32_t stream, uint64_t b)
{
    uint32_t c[4] = {(uint32_t)b, (uint32_t)(b >> 32), stream, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    float z[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float ua = __fmul_rn((float)((c[2 * p] >> 8) + 1u), 0x1.0p-24f);
        const float rad = __fsqrt_rn(__fmul_rn(-2.0f, gen_ln(ua)));
        float cs, sn;
        gen_cossin(c[2 * p + 1], cs, sn);
        z[2 * p] = __fmul_rn(rad, cs);
        z[2 * p + 1] = __fmul_rn(rad, sn);
    }
    return make_float4(z[0], z[1], z[2], z[3]);
}

}  // namespace tvcs
