// Rows a1-a5 of one IADM/FTVCS iteration for many 128 x 128 images at once, one
// block per image, with every 128-point transform held in the registers of one
// warp (Xiao & Yang, Sec. 2.1-2.2: the w-step of eq. (iadmw) with reading C1 and
// the shrink of eq. (shrink), the right-hand side of eq. (eqnorm11) times beta
// in increment form, the FFT solve with the eigenvalues of D^T D, the stop
// norms of eq. (stop)).  The same arithmetic as usolve_steps.cuh, laid out so
// that no phase needs a block barrier: a warp owns whole rows (phases A and C)
// or whole columns (phase B) of the image.
//
// 128-point DFT in one warp.  Lane l holds x[l + 32 j], j = 0..3.  With
// c = l + 32 j and k = k1 + 4 k2 (k1 = 0..3, k2 = 0..31),
//     X[k1 + 4 k2] = sum_l W32^(l k2) * [ W128^(l k1) * sum_j x[l + 32 j] W4^(j k1) ],
// so a radix-4 DFT in registers, a twiddle, and for each k1 a 32-point DFT
// across the lanes (five radix-2 butterfly stages through shuffles, decimation
// in frequency: lane l ends with k2 = bitrev5(l)).  The inverse runs the mirror
// image (decimation in time from that order, twiddle, inverse radix-4), so a
// forward transform followed by its inverse needs no reordering.  Rows of the
// image are read with lane l holding the contiguous columns c = 4 l + j (one
// 16-byte access per lane and plane, a column shift in one shuffle); their
// forward transform takes the other factor order, k = k1 + 32 k2 (k1 = 0..31):
//     X[k1 + 32 k2] = sum_j W4^(j k2) * [ W128^(j k1) * sum_l x[4 l + j] W32^(l k1) ],
// the same 32-point lane stages first (lane l ends with k1 = bitrev5(l)), then a
// twiddle and the radix-4 DFT in registers.
//
// Phases (8 warps):
//   A  per pair of rows (r0, r0+1), each warp down a stripe of 16 rows: the
//      multiplier update and shrink of the two rows from u, w, lambda in global
//      memory (L2), the right-hand side of the pair packed into one complex row,
//      its forward transform, and the split into the two rows' half spectra,
//      stored column-major in shared memory (the spectrum of the image never
//      leaves the SM);
//   B  per column q = 0..64: forward transform, divide by beta Lambda_pq + mu/tau,
//      inverse transform, in registers;
//   C  per pair of rows: the packed inverse row transform (through the same
//      forward code on the conjugate), u += d, bf16 planes, the norms (each
//      lane's 8 squares of a pair in binary32, then double-single across pairs);
// then the block's sums and eq. (stop).  Shared memory: the half spectrum
// (65 columns of 129 complex values) and one 128-value exchange row per warp:
// 75 KB; two images per SM (256 images in one wave), with the registers of
// that occupancy holding the next pair's loads while a pair is transformed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "usolve_steps.cuh"

namespace tvcs {

namespace {

constexpr int RG_NN = 128;
constexpr int RG_N = RG_NN * RG_NN;
constexpr int RG_Q = RG_NN / 2 + 1;      // columns of the half spectrum
constexpr int RG_QS = RG_NN + 1;         // column stride (complex)
constexpr int RG_WARPS = 8;
constexpr int RG_T = RG_WARPS * 32;
constexpr int RG_XS = RG_NN + RG_NN / 16;   // exchange row of a warp, one pad per 16 values
constexpr int RG_TWK = 11;   // per-lane twiddles (3 in-lane, 5 lane stages, 3 for the contiguous rows)
constexpr size_t RG_SMEM = ((size_t)RG_Q * RG_QS * 8 + 15) / 16 * 16 + (size_t)RG_WARPS * RG_XS * 8 + 64 * 8 +
                           (size_t)RG_TWK * 32 * 8;

__device__ __forceinline__ int bitrev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

// padded position of value c in a warp's exchange row (conflict-free for the
// natural and the bit-reversed orders used here)
__device__ __forceinline__ int xpos(int c) { return c + (c >> 4); }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Per-lane twiddles, in a shared table twl[k][lane] (the same for every warp):
// k = 0..2 the in-lane W128^(l (k+1)); k = 3 + s, for lane stage s (half h = 16 >> s),
// W_{2h}^(l mod h) on the lanes that take the difference (l & h) and exactly 1 on
// the others, so that every lane runs the same butterfly (a product by 1 is exact);
// k = 8..10 the W128^(bitrev5(l) (k-7)) of the contiguous-row transform.
// Forward values (exp(-2 pi i t / n)); the inverse uses their conjugates.
__device__ __forceinline__ float2 lane_twiddle(const float2* __restrict__ tw128, int k, int l)
{
    int t;
    if (k < 3) {
        t = (l * (k + 1)) & (RG_NN - 1);
    } else if (k >= 8) {
        t = (bitrev5(l) * (k - 7)) & (RG_NN - 1);
    } else {
        const int h = 16 >> (k - 3);
        if ((l & h) == 0) return make_float2(1.f, 0.f);
        t = (4 * (l & (h - 1)) * (16 / h)) & (RG_NN - 1);   // exponent of W32, in W128 steps
    }
    const float2 c = tw128[t];   // (cos, sin)(2 pi t / 128)
    return make_float2(c.x, -c.y);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)   // a * conj(b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Forward radix-4 DFT of the four values of a lane, W4 = -i.
__device__ __forceinline__ void radix4_fwd(float2 v[4])
{
    const float2 s02 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    const float2 d02 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    const float2 s13 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    const float2 d13 = make_float2(v[1].y - v[3].y, v[3].x - v[1].x);   // -i (v1 - v3)
    v[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
    v[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
    v[1] = make_float2(d02.x + d13.x, d02.y + d13.y);
    v[3] = make_float2(d02.x - d13.x, d02.y - d13.y);
}

// For each of the four values of a lane, the forward 32-point DFT across the
// lanes (lane l holds element l in, coefficient bitrev5(l) out).
__device__ __forceinline__ void lanes_fwd(float2 v[4], const float2* __restrict__ twl, int l)
{
#pragma unroll
    for (int s = 0; s < 5; ++s) {   // decimation in frequency across the lanes
        // upper lanes (l & h) == 0 keep v + p, the others (p - v) W: one signed
        // sum and a product by the lane's twiddle (1 on the upper lanes, and on
        // every lane in the last stage, where it is left out)
        const int h = 16 >> s;
        const float sg = (l & h) ? -1.f : 1.f;
        const float2 ws = twl[(3 + (s < 4 ? s : 0)) * 32 + l];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float2 p = shfl_xor2(v[k1], h);
            v[k1] = make_float2(fmaf(sg, v[k1].x, p.x), fmaf(sg, v[k1].y, p.y));
            if (s < 4) v[k1] = cmulf(v[k1], ws);
        }
    }
}

// Forward: v[j] = x[l + 32 j] in, v[k1] = X[k1 + 4 bitrev5(l)] out.
__device__ __forceinline__ void fft128_fwd(float2 v[4], const float2* __restrict__ twl, int l)
{
    radix4_fwd(v);
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[k1] = cmulf(v[k1], twl[(k1 - 1) * 32 + l]);
    lanes_fwd(v, twl, l);
}

// Forward on contiguous columns: v[j] = x[4 l + j] in, v[k2] = X[bitrev5(l) + 32 k2] out.
__device__ __forceinline__ void fft128_fwd_c(float2 v[4], const float2* __restrict__ twl, int l)
{
    lanes_fwd(v, twl, l);
#pragma unroll
    for (int j = 1; j < 4; ++j) v[j] = cmulf(v[j], twl[(7 + j) * 32 + l]);
    radix4_fwd(v);
}

// Inverse (unnormalised): v[k1] = X[k1 + 4 bitrev5(l)] in, v[j] = x[l + 32 j] out.
__device__ __forceinline__ void fft128_inv(float2 v[4], const float2* __restrict__ twl, int l)
{
#pragma unroll
    for (int s = 4; s >= 0; --s) {   // decimation in time across the lanes
        // lanes (l & h) != 0 send v conj(W) and keep p - own, the others send v and
        // keep own + p (twiddle 1 on the upper lanes and in the first stage)
        const int h = 16 >> s;
        const float sg = (l & h) ? -1.f : 1.f;
        const float2 ws = twl[(3 + (s < 4 ? s : 0)) * 32 + l];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float2 own = s < 4 ? cmulc(v[k1], ws) : v[k1];
            const float2 p = shfl_xor2(own, h);
            v[k1] = make_float2(fmaf(sg, own.x, p.x), fmaf(sg, own.y, p.y));
        }
    }
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[k1] = cmulc(v[k1], twl[(k1 - 1) * 32 + l]);
    {   // inverse radix 4, W4^-1 = +i
        const float2 s02 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 d02 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 s13 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 d13 = make_float2(v[3].y - v[1].y, v[1].x - v[3].x);   // +i (v1 - v3)
        v[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
        v[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
        v[1] = make_float2(d02.x + d13.x, d02.y + d13.y);
        v[3] = make_float2(d02.x - d13.x, d02.y - d13.y);
    }
}

// Rows with lane l holding columns 4 l + j: the value at column c - 1 (periodic;
// column 4 l - 1 is lane l - 1's last value, lane 0 takes lane 31's).
__device__ __forceinline__ void shift_left_cols(const float v[4], float out[4], int l)
{
    out[0] = __shfl_sync(0xffffffffu, v[3], (l + 31) & 31);
    out[1] = v[0];
    out[2] = v[1];
    out[3] = v[2];
}

// The value at column c + 1 (column 4 l + 4 is lane l + 1's first value, lane 31
// takes lane 0's).
__device__ __forceinline__ void shift_right_cols(const float v[4], float out[4], int l)
{
    out[0] = v[1];
    out[1] = v[2];
    out[2] = v[3];
    out[3] = __shfl_sync(0xffffffffu, v[0], (l + 1) & 31);
}

__device__ __forceinline__ void ld4(const float* __restrict__ p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}

__device__ __forceinline__ void st4(float* __restrict__ p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Multiplier update of eq. (udlamb) (when an iteration is pending), shrink of
// eq. (shrink) and y = beta (w - Du) - lambda for one row held as columns
// 4 l + j: uc is the row, ud the row below it (periodic), l1/l2 the
// multipliers (updated in place), wo1/wo2 the previous w (read when pending).
__device__ __forceinline__ void shrink_row(const float (&uc)[4], const float (&ud)[4], float (&l1)[4],
                                           float (&l2)[4], const float (&wo1)[4], const float (&wo2)[4],
                                           int pending, float beta, float inv_beta, int l,
                                           float (&y1)[4], float (&y2)[4], float (&w1)[4], float (&w2)[4])
{
    float up[4];
    shift_right_cols(uc, up, l);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float d1 = up[j] - uc[j];
        const float d2 = ud[j] - uc[j];
        if (pending) {
            l1[j] -= beta * (wo1[j] - d1);
            l2[j] -= beta * (wo2[j] - d2);
        }
        const float z1 = d1 + l1[j] * inv_beta, z2 = d2 + l2[j] * inv_beta;
        const float nz = sqrtf(z1 * z1 + z2 * z2);
        float a1 = 0.0f, a2 = 0.0f;
        if (nz > inv_beta) {
            const float sc = (nz - inv_beta) / nz;
            a1 = sc * z1;
            a2 = sc * z2;
        }
        w1[j] = a1;
        w2[j] = a2;
        y1[j] = beta * (a1 - d1) - l1[j];
        y2[j] = beta * (a2 - d2) - l2[j];
    }
}

// What the pair of rows (r0, r0 + 1) reads besides the carried row r0 of u:
// u rows r0 + 1, r0 + 2 (periodic), the multipliers, w (when pending) and g
// of rows r0, r0 + 1.
struct PairIn {
    float u[2][4];
    float l1[2][4], l2[2][4], w1[2][4], w2[2][4];
};

// The first two stream-K partials of g for the pair's rows (the second 0 past the
// last segment), loaded with the pair's other inputs.
struct PairG {
    float g[2][4];
    float g1[2][4];
    int s0[2], ns[2];   // each row's (tile's) first segment and segment count
};

// Where g comes from: the partial tiles of G = A^T R, whose 128-row tile t holds
// row t of a 128 x 128 image: g at pixel (t, c) is the sum of
// ws[(slot_s cols + col) 128 + c] over the tile's segments s.
struct GSrc {
    const float* ws;
    const int* tsb;
    const int* ss;
    int cols, col;
};

__device__ __forceinline__ void load_pair(PairIn& in, const float* __restrict__ u,
                                          const float* __restrict__ lsrc, const float* __restrict__ wsrc,
                                          int r0, int l, int pending)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int gi = (r0 + h) * RG_NN + 4 * l;
        ld4(u + ((r0 + 1 + h) & (RG_NN - 1)) * RG_NN + 4 * l, in.u[h]);
        ld4(lsrc + gi, in.l1[h]);
        ld4(lsrc + RG_N + gi, in.l2[h]);
        if (pending) {
            ld4(wsrc + gi, in.w1[h]);
            ld4(wsrc + RG_N + gi, in.w2[h]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) in.w1[h][j] = in.w2[h][j] = 0.0f;
        }
    }
}

__device__ __forceinline__ void load_g(PairG& in, const GSrc& gs, int r0, int l)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int s0 = gs.tsb[r0 + h], ns = gs.tsb[r0 + h + 1] - s0;
        in.s0[h] = s0;
        in.ns[h] = ns;
        const float* p0 = gs.ws + ((size_t)gs.ss[s0] * gs.cols + gs.col) * RG_NN;
        const float* p1 = ns > 1 ? gs.ws + ((size_t)gs.ss[s0 + 1] * gs.cols + gs.col) * RG_NN : nullptr;
        ld4(p0 + 4 * l, in.g[h]);
        if (p1) {
            ld4(p1 + 4 * l, in.g1[h]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) in.g1[h][j] = 0.0f;
        }
    }
}

// g of row r0 + h at columns 4 l + j, bitwise the fix-up's sum: it adds from +0
// the first GEMM_FX_SEG partials (zeros past the last segment), then the rest, in
// K order.  A sum that starts at +0 is never -0 after its first addition, and x + 0
// is x for every other x, so the padding zeros change nothing: the sum from +0 over
// the tile's segments in order is the same value.
__device__ __forceinline__ void g_row(const PairG& in, const GSrc& gs, int h, int l, float (&g)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float d = 0.f;
        d += in.g[h][j];
        d += in.g1[h][j];   // 0 for a one-segment tile: the same value
        g[j] = d;
    }
    for (int q = 2; q < in.ns[h]; ++q) {   // tiles of more than two segments
        const float* p = gs.ws + ((size_t)gs.ss[in.s0[h] + q] * gs.cols + gs.col) * RG_NN;
        float t[4];
        ld4(p + 4 * l, t);
#pragma unroll
        for (int j = 0; j < 4; ++j) g[j] += t[j];
    }
}

}  // namespace

// Image b = blockIdx.x, with the conventions of k_usolve_img (per-image mu and
// tau, control block, bf16 planes at row img_slot[b]).
__global__ void __launch_bounds__(RG_T, 2) k_usolve_reg128(
    float* __restrict__ u, float* __restrict__ wbuf, float* __restrict__ lbuf,
    const float* __restrict__ g, const float2* __restrict__ tw_g, const float* __restrict__ s2_g,
    float beta, float mu_over_tau, float mu, Ctrl* __restrict__ ctrl, int mode,
    const float* __restrict__ mu_img, const float* __restrict__ tau_img, float tau,
    unsigned short* __restrict__ u_hi, unsigned short* __restrict__ u_lo,
    const int* __restrict__ img_slot, const float* __restrict__ gws, const int* __restrict__ gtsb,
    const int* __restrict__ gss, int gws_cols, const int* __restrict__ img_slot_prev)
{
    constexpr int NN = RG_NN, N = RG_N;
    pdl_release();   // the next GEMM may start its first copies of A (it waits before reading u)
    GSrc gs{gws, gtsb, gss, gws_cols, 0};
    {
        const int b = blockIdx.x;
        u += (size_t)b * N;
        wbuf += (size_t)b * 4 * N;
        lbuf += (size_t)b * 4 * N;
        gs.col = img_slot_prev ? img_slot_prev[b] : b;
        ctrl += b;
        if (u_hi) {
            const int row = img_slot ? img_slot[b] : b;
            if (row >= 0) {
                u_hi += (size_t)row * N;
                u_lo += (size_t)row * N;
            } else {
                u_hi = u_lo = nullptr;
            }
        }
        if (mu_img) {
            mu = mu_img[b];
            mu_over_tau = mu / (tau_img ? tau_img[b] : tau);
        }
    }
    extern __shared__ __align__(16) unsigned char smem[];
    float2* spec = reinterpret_cast<float2*>(smem);                     // spec[q QS + p]
    float2* xrow_all = reinterpret_cast<float2*>(smem + ((size_t)RG_Q * RG_QS * 8 + 15) / 16 * 16);
    float2* red = xrow_all + RG_WARPS * RG_XS;                          // [64]
    float2* twl = red + 64;                                             // [RG_TWK][32]
    const int tid = threadIdx.x, l = tid & 31, warp = tid >> 5;
    float2* xrow = xrow_all + warp * RG_XS;

    if (mode == MODE_ITER) {
        const int done = ctrl->done;   // stable during this kernel
        if (tid == 0) ctrl->skip = done;
        if (done) return;              // uniform across the block
    }
    const int pending = ctrl->pending;
    const int par = ctrl->wpar;
    const float* wsrc = wbuf + (size_t)par * 2 * N;
    const float* lsrc = lbuf + (size_t)par * 2 * N;
    float* wdst = wbuf + (size_t)(par ^ 1) * 2 * N;
    float* ldst = lbuf + (size_t)(par ^ 1) * 2 * N;
    for (int e = tid; e < RG_TWK * 32; e += RG_T) twl[e] = lane_twiddle(tw_g, e >> 5, e & 31);
    __syncthreads();
    const float inv_beta = 1.0f / beta;

    // ---------------- phase A: pairs of rows ----------------
    // Warp w owns the stripe of rows 16 w .. 16 w + 15 (eight pairs), so that
    // each pair shares its upper u row and the y2 row above it with the pair
    // before: one shrink per row, plus one for the row above the stripe.  The
    // loads of the next pair are issued before the transform of the current
    // one, which hides their latency.
    constexpr int PPW = NN / 2 / RG_WARPS;
    const int R0 = warp * 2 * PPW;
    float ucur[4], y2prev[4];   // u row r0 and y2 of row r0 - 1
    {
        const int rp = (R0 - 1 + NN) & (NN - 1);
        const int gi = rp * NN + 4 * l;
        float ur[4], lr1[4], lr2[4], wr1[4] = {0.f, 0.f, 0.f, 0.f}, wr2[4] = {0.f, 0.f, 0.f, 0.f};
        ld4(u + gi, ur);
        ld4(u + R0 * NN + 4 * l, ucur);
        ld4(lsrc + gi, lr1);
        ld4(lsrc + N + gi, lr2);
        if (pending) {
            ld4(wsrc + gi, wr1);
            ld4(wsrc + N + gi, wr2);
        }
        float y1d[4], w1d[4], w2d[4];
        shrink_row(ur, ucur, lr1, lr2, wr1, wr2, pending, beta, inv_beta, l, y1d, y2prev, w1d, w2d);
    }
    PairIn cur;
    PairG gp;   // g of the pair (or its partials), loaded with the pair's other inputs
    load_pair(cur, u, lsrc, wsrc, R0, l, pending);
    load_g(gp, gs, R0, l);
#pragma unroll 1
    for (int k = 0; k < PPW; ++k) {
        const int r0 = R0 + 2 * k;
        float y1[2][4], y2[2][4], w1[4], w2[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // rows r0 + h: multiplier update, shrink, y
            if (h == 0)
                shrink_row(ucur, cur.u[0], cur.l1[0], cur.l2[0], cur.w1[0], cur.w2[0], pending, beta,
                           inv_beta, l, y1[0], y2[0], w1, w2);
            else
                shrink_row(cur.u[0], cur.u[1], cur.l1[1], cur.l2[1], cur.w1[1], cur.w2[1], pending, beta,
                           inv_beta, l, y1[1], y2[1], w1, w2);
            const int gi = (r0 + h) * NN + 4 * l;
            st4(wdst + gi, w1);
            st4(wdst + N + gi, w2);
            st4(ldst + gi, cur.l1[h]);
            st4(ldst + N + gi, cur.l2[h]);
        }
        // right-hand side of rows r0, r0+1 packed: z = rhs[r0] + i rhs[r0+1]
        float2 v[4];
        float ym[2][4];
        shift_left_cols(y1[0], ym[0], l);
        shift_left_cols(y1[1], ym[1], l);
        float g0[4], g1[4];
        g_row(gp, gs, 0, l, g0);
        g_row(gp, gs, 1, l, g1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float rr0 = ym[0][j] - y1[0][j] + y2prev[j] - y2[0][j] - mu * g0[j];
            const float rr1 = ym[1][j] - y1[1][j] + y2[0][j] - y2[1][j] - mu * g1[j];
            v[j] = make_float2(rr0, rr1);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ucur[j] = cur.u[1][j];
            y2prev[j] = y2[1][j];
        }
        if (k + 1 < PPW) {
            load_pair(cur, u, lsrc, wsrc, r0 + 2, l, pending);
            load_g(gp, gs, r0 + 2, l);
        }
        fft128_fwd_c(v, twl, l);
        // exchange row: Z[k] at its padded position, then the split of the pair
        const int br = bitrev5(l);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) xrow[xpos(br + 32 * k2)] = v[k2];
        __syncwarp();
        for (int q = l; q < RG_Q; q += 32) {
            const float2 a = xrow[xpos(q)];
            const float2 bb = xrow[xpos((NN - q) & (NN - 1))];
            spec[q * RG_QS + r0] = make_float2(0.5f * (a.x + bb.x), 0.5f * (a.y - bb.y));
            spec[q * RG_QS + r0 + 1] = make_float2(0.5f * (a.y + bb.y), -0.5f * (a.x - bb.x));
        }
        __syncwarp();   // the exchange row is free for the next pair
    }
    __syncthreads();

    // ---------------- phase B: columns ----------------
    float s2p[4];   // s2 of the rows p = k1 + 4 bitrev5(l) this lane holds after a forward transform
    {
        const int br = bitrev5(l);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) s2p[k1] = s2_g[k1 + 4 * br];
    }
    for (int q = warp; q < RG_Q; q += RG_WARPS) {
        float2* col = spec + q * RG_QS;
        float2 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = col[l + 32 * j];
        fft128_fwd(v, twl, l);
        const float s2q = s2_g[q];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float rd = 1.0f / (beta * (s2p[k1] + s2q) + mu_over_tau);
            v[k1].x *= rd;
            v[k1].y *= rd;
        }
        fft128_inv(v, twl, l);
#pragma unroll
        for (int j = 0; j < 4; ++j) col[l + 32 * j] = v[j];
    }
    __syncthreads();

    // ---------------- phase C: pairs of rows ----------------
    const float sc = 1.0f / (float)N;
    float2 du2 = make_float2(0.f, 0.f), u2 = make_float2(0.f, 0.f);
    for (int pr = warp; pr < NN / 2; pr += RG_WARPS) {
        const int r0 = 2 * pr;
        float du2p = 0.f, u2p = 0.f;   // this lane's 8 squares of the pair, in binary32
        float uo[2][4];   // u of the pair at columns 4 l + j, loaded before the transform that hides the latency
#pragma unroll
        for (int h = 0; h < 2; ++h) ld4(u + (r0 + h) * NN + 4 * l, uo[h]);
        // packed inverse input Z[q] = X[q] + i Y[q] (q >= 65 by conjugate symmetry);
        // transformed with the forward code on conj(Z): x = conj(F(conj Z))
        float2 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = l + 32 * j;
            const bool lo = q < RG_Q;
            const int qq = lo ? q : NN - q;
            float2 X = spec[qq * RG_QS + r0];
            float2 Y = spec[qq * RG_QS + r0 + 1];
            if (qq == 0 || 2 * qq == NN) {   // exactly real bins
                X.y = 0.f;
                Y.y = 0.f;
            }
            if (!lo) {
                X.y = -X.y;
                Y.y = -Y.y;
            }
            v[j] = make_float2(X.x - Y.y, -(X.y + Y.x));   // conj(X + i Y)
        }
        fft128_fwd(v, twl, l);
        const int br = bitrev5(l);
        // conj of the result, through the exchange row into natural column order
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) xrow[xpos(k1 + 4 * br)] = make_float2(v[k1].x, -v[k1].y);
        __syncwarp();
        float2 z[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) z[j] = xrow[xpos(4 * l + j)];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gi = (r0 + h) * NN + 4 * l;
            float nw[4];
            unsigned short hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float d = (h == 0 ? z[j].x : z[j].y) * sc;
                const float o = uo[h][j];
                du2p = fmaf(d, d, du2p);
                u2p = fmaf(o, o, u2p);
                nw[j] = o + d;
                // bf16 hi = RN(u), lo = RN(u - hi)
                const __nv_bfloat16 hb = __float2bfloat16_rn(nw[j]);
                hi[j] = __bfloat16_as_ushort(hb);
                lo[j] = __bfloat16_as_ushort(__float2bfloat16_rn(nw[j] - __bfloat162float(hb)));
            }
            st4(u + gi, nw);
            if (u_hi) {   // four bf16 values in one 8-byte store per plane
                *reinterpret_cast<uint2*>(u_hi + gi) =
                    make_uint2(hi[0] | ((unsigned)hi[1] << 16), hi[2] | ((unsigned)hi[3] << 16));
                *reinterpret_cast<uint2*>(u_lo + gi) =
                    make_uint2(lo[0] | ((unsigned)lo[1] << 16), lo[2] | ((unsigned)lo[3] << 16));
            }
        }
        // the pair's sums (relative error at most 8 x 2^-24) into the double-single
        // totals of eq. (stop)
        du2 = ds_add(du2, make_float2(du2p, 0.f));
        u2 = ds_add(u2, make_float2(u2p, 0.f));
        __syncwarp();
    }
    block_sum_ds2(du2, u2, red);
    if (tid == 0) step_stop(ctrl, par, mode, ds_value(du2), ds_value(u2));
}

bool usolve_reg_configure()
{
    if (cudaFuncSetAttribute(k_usolve_reg128, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RG_SMEM) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

void launch_usolve_reg128(const TvArgs& a, cudaStream_t s)
{
    k_usolve_reg128<<<a.nimg > 0 ? a.nimg : 1, RG_T, RG_SMEM, s>>>(
        a.u, a.w, a.lam, a.g, a.tw, a.s2, a.beta, a.mu_over_tau, a.mu, a.ctrl, a.mode, a.mu_img,
        a.tau_img, a.tau, a.u_hi, a.u_lo, a.img_slot, a.gws, a.gtsb, a.gss, a.gws_cols, a.img_slot_prev);
}

}  // namespace tvcs
