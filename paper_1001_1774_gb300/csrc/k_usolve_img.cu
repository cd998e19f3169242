// Rows a1-a5 of one IADM/FTVCS iteration for many images at once, one block
// per image (Xiao & Yang, Sec. 2.1-2.2; the same steps as k_usolve.cu, in
// usolve_steps.cuh).  For batches: with hundreds of images in flight the
// latency of one image matters less than the rate at which the SMs get through
// them, so each image stays on one SM and needs no cluster barrier.
//
// The block keeps the image's whole half spectrum in shared memory, column-
// major (spec[q (n+1) + p], q = 0 .. n/2: the column stride is padded by one
// complex value so that a warp storing consecutive columns of one row, as the
// split after the row transforms does, spreads over the banks).  Phases A and C
// stream the image in stripes of S rows through asynchronous 16-byte copies (the
// next stripe's rows arrive while the current one is transformed):
//   A  per stripe: w-step, right-hand side, forward row FFTs (two real rows per
//      complex transform), half spectra into their columns;
//   B  the columns in chunks: FFTs, divide by beta Lambda_pq + mu/tau, inverse FFTs;
//   C  per stripe: inverse row FFTs, u += d, double-single partial norms;
// then the block sums and eq. (stop) for the image.  The spectrum plus one
// stripe's (or one column chunk's) scratch stay under half of an SM's shared
// memory, so two images share an SM and 2 x (number of SMs) images run in one wave.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "usolve_steps.cuh"

namespace tvcs {

namespace {

// Two blocks of T threads per SM: the block's shared memory (the half spectrum
// plus one stripe's scratch) stays under half of the SM's, so that a batch of
// up to 2 x (number of SMs) images runs in one wave.
template <int NN, int S, int T>
struct ImgShape {
    static constexpr int Q = NN / 2 + 1;
    static constexpr int QS = NN + 1;               // column stride of the spectrum (complex)
    static constexpr int NSTRIPE = NN / S;
    static constexpr int IN_U = (S + 2) * NN;       // u rows r0-1 .. r0+S
    static constexpr int IN_G = S * NN;             // g rows r0 .. r0+S-1
    static constexpr int IN_WL = 4 * (S + 1) * NN;  // w1, w2, l1, l2 rows r0-1 .. r0+S-1
    static constexpr int IN = IN_U + IN_G + IN_WL;  // floats of one stripe's inputs
    static constexpr int CCOLS = (Q + 2) / 3 < 32 ? (Q + 2) / 3 : 32;   // columns per phase-B chunk
    static constexpr size_t O_TW = 0;
    static constexpr size_t O_S2 = O_TW + NN * 8;
    static constexpr size_t O_RED = O_S2 + ((NN * 4 + 15) / 16) * 16;   // [64] float2
    static constexpr size_t O_SPEC = O_RED + 64 * 8;                     // Q columns of QS complex
    static constexpr size_t SPEC_BYTES = (((size_t)Q * QS * 8 + 15) / 16) * 16;
    static constexpr size_t O_SCR = O_SPEC + SPEC_BYTES;
    // phase A, inside the scratch region: the stripe's inputs, y1, y2, two FFT buffers
    static constexpr size_t A_IN = O_SCR;
    static constexpr size_t A_Y1 = A_IN + (size_t)IN * 4;
    static constexpr size_t A_Y2 = A_Y1 + (size_t)S * NN * 4;
    static constexpr size_t A_WA = A_Y2 + (size_t)(S + 1) * NN * 4;
    static constexpr size_t A_WB = A_WA + (size_t)(S / 2) * NN * 8;
    static constexpr size_t A_END = A_WB + (size_t)(S / 2) * NN * 8;
    // phase B: the Stockham partner of a chunk of CCOLS columns (same column stride)
    static constexpr size_t B_END = O_SCR + (size_t)CCOLS * QS * 8;
    // phase C: two u-row buffers, two FFT buffers
    static constexpr size_t C_END = O_SCR + 2 * (size_t)S * NN * 4 + 2 * (size_t)(S / 2) * NN * 8;
    static constexpr size_t SMEM = A_END > B_END ? (A_END > C_END ? A_END : C_END)
                                                 : (B_END > C_END ? B_END : C_END);
    static_assert(NN % S == 0 && S % 2 == 0, "whole stripes of an even number of rows");
    static_assert(T % 32 == 0 && T / 32 <= 32, "whole warps, one reduction slot each");
    static_assert(SMEM * 2 + 2048 <= 233472, "two blocks per SM");
};

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all_groups()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_one()
{
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

}  // namespace

// Image b = blockIdx.x uses u + b N, w/lambda + 4 b N, g + b N, ctrl + b and,
// when mu_img is set, mu_img[b] (and tau_img[b] when set); its bf16 planes go
// to row img_slot[b] when img_slot is set (-1: stopped, no planes), else row b.
template <int NN, int S, int T>
__global__ void __launch_bounds__(T, 2) k_usolve_img(
    float* __restrict__ u, float* __restrict__ wbuf, float* __restrict__ lbuf,
    const float* __restrict__ g, const float2* __restrict__ tw_g, const float* __restrict__ s2_g,
    float beta, float mu_over_tau, float mu, Ctrl* __restrict__ ctrl, int mode,
    const float* __restrict__ mu_img, const float* __restrict__ tau_img, float tau,
    unsigned short* __restrict__ u_hi, unsigned short* __restrict__ u_lo,
    const int* __restrict__ img_slot)
{
    using SH = ImgShape<NN, S, T>;
    constexpr int N = NN * NN, Q = SH::Q, CPR = NN / 4, WL = (S + 1) * NN;
    {
        const int b = blockIdx.x;
        u += (size_t)b * N;
        wbuf += (size_t)b * 4 * N;
        lbuf += (size_t)b * 4 * N;
        g += (size_t)b * N;
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
    float2* tw = reinterpret_cast<float2*>(smem + SH::O_TW);
    float* s2 = reinterpret_cast<float*>(smem + SH::O_S2);
    float2* spec = reinterpret_cast<float2*>(smem + SH::O_SPEC);   // spec[q QS + p]
    float2* scr = reinterpret_cast<float2*>(smem + SH::O_SCR);
    float* in = reinterpret_cast<float*>(smem + SH::A_IN);
    float* sy1 = reinterpret_cast<float*>(smem + SH::A_Y1);
    float* sy2 = reinterpret_cast<float*>(smem + SH::A_Y2);
    float2* wa = reinterpret_cast<float2*>(smem + SH::A_WA);
    float2* wb = reinterpret_cast<float2*>(smem + SH::A_WB);
    float2* red = reinterpret_cast<float2*>(smem + SH::O_RED);   // [64] block reduction
    const int tid = threadIdx.x, nthr = T;

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

    // ---------------- phase A: stripes of S rows ----------------
    // One input buffer: the copies of stripe s+1 are issued as soon as stripe s's
    // inputs have been used (after the right-hand side), so they land while
    // stripe s's row transforms run.
    auto load_stripe = [&](int s) {
        const int r0 = s * S;
        float* su = in;
        float* sg = in + SH::IN_U;
        float* swl = sg + SH::IN_G;
        for (int i = tid; i < (S + 2) * CPR; i += nthr) {
            const int rr = i / CPR, c4 = i - rr * CPR;
            const int row = (r0 - 1 + rr + NN) % NN;
            cp_async16(su + rr * NN + 4 * c4, u + row * NN + 4 * c4);
        }
        for (int i = tid; i < S * CPR; i += nthr) cp_async16(sg + 4 * i, g + r0 * NN + 4 * i);
        for (int i = tid; i < (S + 1) * CPR; i += nthr) {
            const int rr = i / CPR, c4 = i - rr * CPR;
            const int gi = ((r0 - 1 + rr + NN) % NN) * NN + 4 * c4;
            const int li = rr * NN + 4 * c4;
            cp_async16(swl + li, wsrc + gi);
            cp_async16(swl + WL + li, wsrc + N + gi);
            cp_async16(swl + 2 * WL + li, lsrc + gi);
            cp_async16(swl + 3 * WL + li, lsrc + N + gi);
        }
    };
    for (int i = tid; i < NN / 2; i += nthr) cp_async16(tw + 2 * i, tw_g + 2 * i);
    for (int i = tid; i < CPR; i += nthr) cp_async16(s2 + 4 * i, s2_g + 4 * i);
    load_stripe(0);
    cp_async_commit();
    for (int s = 0; s < SH::NSTRIPE; ++s) {
        cp_async_wait_all_groups();   // this stripe's inputs (and the tables) have landed
        __syncthreads();
        const int r0 = s * S;
        step_wshrink<NN>(in, in + SH::IN_U + SH::IN_G, WL, S, r0, beta, pending, sy1, sy2, wdst,
                         ldst, tid, nthr);
        __syncthreads();
        step_rhs<NN>(sy1, sy2, in + SH::IN_U, S, r0, mu, wa, nullptr, tid, nthr);
        __syncthreads();              // the input buffer is free
        if (s + 1 < SH::NSTRIPE) {
            load_stripe(s + 1);
            cp_async_commit();
        }
        float2* Z = fft_block<NN, false>(wa, wb, tw, S / 2, NN);
        step_split<NN>(Z, S, spec + r0, 1, SH::QS, tid, nthr);
    }
    __syncthreads();

    // ---------------- phase B: the columns in chunks ----------------
    // Forward and inverse Stockham passes ping-pong between the chunk's columns
    // in `spec` and the scratch chunk (same column stride); the result is copied
    // back when it ends in the scratch.
    for (int q0 = 0; q0 < Q; q0 += SH::CCOLS) {
        const int nc = min(SH::CCOLS, Q - q0);
        float2* A0 = spec + (size_t)q0 * SH::QS;
        float2* X = fft_block<NN, false>(A0, scr, tw, nc, SH::QS);
        for (int i = tid; i < nc * NN; i += nthr) {
            const int qq = i / NN, p = i - qq * NN;
            const float rd = 1.0f / solve_divisor(s2, p, q0 + qq, beta, mu_over_tau);
            float2 v = X[qq * SH::QS + p];
            v.x *= rd;
            v.y *= rd;
            X[qq * SH::QS + p] = v;
        }
        __syncthreads();
        float2* Y = fft_block<NN, true>(X, X == A0 ? scr : A0, tw, nc, SH::QS);
        if (Y != A0) {
            for (int i = tid; i < nc * NN; i += nthr) {
                const int qq = i / NN, p = i - qq * NN;
                A0[qq * SH::QS + p] = Y[qq * SH::QS + p];
            }
        }
        __syncthreads();   // the scratch chunk is free for the next chunk
    }
    const float2* Y = spec;

    // ---------------- phase C: stripes of S rows ----------------
    float* ub0 = reinterpret_cast<float*>(scr);
    float* ub1 = ub0 + S * NN;
    float2* ca = reinterpret_cast<float2*>(ub1 + S * NN);
    float2* cb = ca + (S / 2) * NN;
    auto load_u = [&](int s, float* dst) {
        for (int i = tid; i < S * CPR; i += nthr) cp_async16(dst + 4 * i, u + s * S * NN + 4 * i);
    };
    load_u(0, ub0);
    cp_async_commit();
    float2 du2 = make_float2(0.f, 0.f), u2 = make_float2(0.f, 0.f);
    for (int s = 0; s < SH::NSTRIPE; ++s) {
        float* cur = (s & 1) ? ub1 : ub0;
        if (s + 1 < SH::NSTRIPE) load_u(s + 1, (s & 1) ? ub0 : ub1);
        cp_async_commit();
        cp_async_wait_one();
        __syncthreads();
        const int r0 = s * S;
        step_pack_inverse<NN>(Y + r0, 1, SH::QS, S, ca, tid, nthr);
        __syncthreads();
        float2* z = fft_block<NN, true>(ca, cb, tw, S / 2, NN);
        step_update<NN>(z, cur, S, r0, u, u_hi, u_lo, du2, u2, tid, nthr);
        __syncthreads();
    }
    block_sum_ds2(du2, u2, red);
    if (tid == 0) step_stop(ctrl, par, mode, ds_value(du2), ds_value(u2));
}

// ---------------------------------------------------------------------------
// Host side.  Stripes of 8 rows (4 packed transforms per stripe); 256 threads, 384
// at n = 128 (87.7 against 90.2 us for 256 images).
// ---------------------------------------------------------------------------
#define TVCS_USOLVE_IMG_TABLE(X) \
    X(16, 8, 256) X(32, 8, 256) X(48, 8, 256) X(64, 8, 256) X(96, 8, 256) X(128, 8, 384)

template <int NN, int S, int T>
static bool configure_img_t()
{
    if (cudaFuncSetAttribute(k_usolve_img<NN, S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ImgShape<NN, S, T>::SMEM) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

bool usolve_img_configure(int n)
{
#define X(NN, S, T) \
    if (n == NN) return configure_img_t<NN, S, T>();
    TVCS_USOLVE_IMG_TABLE(X)
#undef X
    return false;
}

void launch_usolve_img(int n, const TvArgs& a, cudaStream_t s)
{
#define X(NN, S, T)                                                                              \
    if (n == NN) {                                                                               \
        k_usolve_img<NN, S, T><<<a.nimg > 0 ? a.nimg : 1, T, ImgShape<NN, S, T>::SMEM, s>>>(     \
            a.u, a.w, a.lam, a.g, a.tw, a.s2, a.beta, a.mu_over_tau, a.mu, a.ctrl, a.mode,       \
            a.mu_img, a.tau_img, a.tau, a.u_hi, a.u_lo, a.img_slot);                             \
        return;                                                                                  \
    }
    TVCS_USOLVE_IMG_TABLE(X)
#undef X
}

}  // namespace tvcs
