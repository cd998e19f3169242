// Counter-based Gaussian encoding matrix, generated on the device.
//
// Recipe (every floating-point step a single IEEE binary32 operation with
// round-to-nearest -- fused multiply-adds where the recipe says so, nothing
// else contracted: the explicit __f*_rn intrinsics fix each step):
//   element e of stream s -> block b = e >> 2, lane = e & 3
//   (x0..x3) = Philox4x32-10(counter (lo32 b, hi32 b, s, 0), key (lo32 seed, hi32 seed))
//              (Salmon, Moraes, Dror, Shaw, SC'11: multipliers 0xD2511F53,
//              0xCD9E8D57, key increments 0x9E3779B9, 0xBB67AE85)
//   lanes 0,1 take (x0,x1), lanes 2,3 take (x2,x3); for a pair (xa, xb):
//     ua  = ((xa >> 8) + 1) * 2^-24,  rad = sqrt(-2 ln ua)       (Box-Muller, 1958)
//     ln  : ua = 2^e m, m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
//           ln m = 2 (s + s^3/3 + ... + s^11/11) (Horner in s^2 with fused
//           multiply-adds), ln 2 split in a 16-bit head and a tail
//     angle 2 pi (xb >> 8) 2^-24: octant o = xb >> 29, r = ((xb >> 8) & 0x1fffff) 2^-21,
//           angle = Q pi/2 +- psi with psi = t pi/4, t = r or 1 - r; sin psi and
//           cos psi by Taylor series to degree 9 and 10 (Horner, fused
//           multiply-adds)
//     even lane: rad * cos, odd lane: rad * sin
//   A[i][j] = z(i*N + j) * scale, scale = binary32(1/sqrt(m)) (passed in).
// The same values are produced by the host-side input generator; tests check
// the two bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gen.cuh"
#include "kernels.h"

namespace tvcs {

// A (m x N, row-major) with N a multiple of 4: each thread writes one float4.
__global__ void k_gen_gauss(float4* __restrict__ A, long long total4, uint64_t seed, float scale)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total4;
         q += (long long)gridDim.x * blockDim.x) {
        const float4 z = gen_normals4(seed, 0u, (uint64_t)q);
        A[q] = make_float4(__fmul_rn(z.x, scale), __fmul_rn(z.y, scale), __fmul_rn(z.z, scale),
                           __fmul_rn(z.w, scale));
    }
}

void launch_gen_gauss(float* A, int m, int64_t N, uint64_t seed, float scale, cudaStream_t s)
{
    const long long total4 = (long long)m * N / 4;
    int grid = (int)((total4 + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    k_gen_gauss<<<grid, 256, 0, s>>>(reinterpret_cast<float4*>(A), total4, seed, scale);
}

}  // namespace tvcs
