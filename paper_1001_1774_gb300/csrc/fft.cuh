// Shared-memory mixed-radix (8, 4, 3, 2) Stockham FFT of compile-time length NN,
// used for the u-step of eq. (eqnorm11): the 2D DFT diagonalises D^T D under
// periodic boundary (Sec. 2.1), so the u-solve is a forward 2D FFT, a divide
// by beta*Lambda_pq + mu/tau and an inverse 2D FFT.
//
// Stage s with radix R and Ns = product of the earlier radices computes, for
// j in [0, NN/R), k = j mod Ns:
//   v_r = x[j + r*NN/R] * W^(r*k*NN/(Ns*R)),  V = DFT_R(v),
//   y[(j/Ns)*Ns*R + k + r*Ns] = V_r,
// W = exp(-2 pi i/NN) (forward) or its conjugate (inverse, unnormalised).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tvcs {

// Radix of stage s for length n = 2^e 3^t: the fewest stages (e = 3a + 2b + c
// with as many 8s as possible, a lone remainder 2 turned into 4 x 4 when an 8
// can give way), in increasing radix order: 2s, 3s, 4s, 8s.  Small radices go
// first, where a stage's outputs are scattered with stride R, so that the
// eight-way scatter of a radix-8 stage happens only where its outputs are
// contiguous (Ns large).
__host__ __device__ constexpr int fft_radix(int n, int s)
{
    int m = n, e = 0, t = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++e;
    }
    while (m % 3 == 0) {
        m /= 3;
        ++t;
    }
    if (m != 1) return 0;   // only 2^e 3^t
    int n8 = e / 3, n4 = 0, n2 = 0;
    if (e % 3 == 1) {
        if (n8 > 0) {
            --n8;
            n4 = 2;
        } else {
            n2 = 1;
        }
    } else if (e % 3 == 2) {
        n4 = 1;
    }
    if (s < n2) return 2;
    s -= n2;
    if (s < t) return 3;
    s -= t;
    if (s < n4) return 4;
    s -= n4;
    if (s < n8) return 8;
    return 0;
}

__host__ __device__ constexpr int fft_nstages(int n)
{
    int s = 0;
    while (fft_radix(n, s) != 0) ++s;
    return s;
}

__host__ __device__ constexpr int fft_ns(int n, int s)
{
    int p = 1;
    for (int i = 0; i < s; ++i) p *= fft_radix(n, i);
    return p;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Multiply by -i (forward) or +i (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* v)
{
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if constexpr (R == 8) {
        // two 4-point transforms of the even and odd entries, joined with
        // W8^k = exp(-+i pi k/4): 1, (1 -+ i)/sqrt 2, -+i, (-1 -+ i)/sqrt 2
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<4, INV>(e);
        dft_small<4, INV>(o);
        const float h = 0.707106781186547524f;   // 1/sqrt 2
        const float2 t1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                              : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        const float2 t2 = mul_mi<INV>(o[2]);
        const float2 t3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                              : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], t1);
        v[5] = csub(e[1], t1);
        v[2] = cadd(e[2], t2);
        v[6] = csub(e[2], t2);
        v[3] = cadd(e[3], t3);
        v[7] = csub(e[3], t3);
    } else {  // R == 3: w = exp(-+2 pi i/3) = -1/2 -+ i sqrt(3)/2
        const float h = 0.866025403784438647f;  // sqrt(3)/2
        float2 a = v[0], b = v[1], c = v[2];
        float2 s = cadd(b, c), d = csub(b, c);
        float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
        // -+ i*h*d
        float2 e = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);
        v[0] = cadd(a, s);
        v[1] = cadd(t, e);
        v[2] = csub(t, e);
    }
}

// One Stockham stage over `nfft` transforms stored with distance `dist`.
template <int NN, int S, bool INV>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                          const float2* __restrict__ tw, int nfft, int dist,
                                          int tid, int nthr)
{
    constexpr int R = fft_radix(NN, S);
    constexpr int NS = fft_ns(NN, S);
    constexpr int L = NN / R;          // butterflies per transform
    constexpr int TSTEP = NN / (NS * R);
    const int total = nfft * L;
    for (int idx = tid; idx < total; idx += nthr) {
        const int f = idx / L;
        const int j = idx - f * L;
        const int k = j % NS;
        const float2* s = src + f * dist;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = s[j + r * L];
            if (r > 0 && NS > 1) {
                const int t = (r * k * TSTEP) % NN;
                float2 w = tw[t];
                if (!INV) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        dft_small<R, INV>(v);
        float2* d = dst + f * dist;
        const int base = (j / NS) * NS * R + k;
        if constexpr (NS == 1 && R % 2 == 0) {
            // the R outputs are contiguous: 16-byte stores (a warp then writes whole
            // 128-byte lines instead of R-way conflicting 8-byte stores) where the
            // address is 16-byte aligned
            if ((reinterpret_cast<uintptr_t>(d + base) & 15u) == 0) {
                float4* d4 = reinterpret_cast<float4*>(d + base);
#pragma unroll
                for (int r = 0; r < R; r += 2) d4[r / 2] = make_float4(v[r].x, v[r].y, v[r + 1].x, v[r + 1].y);
                continue;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * NS] = v[r];
    }
}

// Recursion end: S == number of stages.
template <int NN, bool INV, int S, bool END = (S == fft_nstages(NN))>
struct FftRun;

template <int NN, bool INV, int S>
struct FftRun<NN, INV, S, true> {
    static __device__ __forceinline__ float2* run(float2* a, float2*, const float2*, int, int, int,
                                                  int)
    {
        return a;
    }
};

template <int NN, bool INV, int S>
struct FftRun<NN, INV, S, false> {
    static __device__ __forceinline__ float2* run(float2* a, float2* b, const float2* tw, int nfft,
                                                  int dist, int tid, int nthr)
    {
        fft_stage<NN, S, INV>(a, b, tw, nfft, dist, tid, nthr);
        __syncthreads();
        return FftRun<NN, INV, S + 1>::run(b, a, tw, nfft, dist, tid, nthr);
    }
};

// Transforms `nfft` sequences of length NN held in shared memory at a (element
// i of transform f at a[f*dist + i]); b is scratch of the same size.  Every
// thread of the block must call it; the input must be visible (synchronised)
// before the call.  Returns the buffer holding the result (a or b).
template <int NN, bool INV>
__device__ __forceinline__ float2* fft_block(float2* a, float2* b, const float2* tw, int nfft,
                                             int dist)
{
    return FftRun<NN, INV, 0>::run(a, b, tw, nfft, dist, threadIdx.x, blockDim.x);
}

}  // namespace tvcs
