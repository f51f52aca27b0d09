// Epilogue of the tensor-core Gram tiles (Q formation in the BF16 store and
// the fused recompute inside the sweep): BF16 Q entries from the FP32 Gram
// accumulators read out of tensor memory, one row chunk of 32 columns at a
// time.  Both kernels call the same code, so the recomputed tiles equal the
// stored ones bit for bit.
#pragma once

#include "common.cuh"

namespace gabp {

// Bit c set where column 32 cc + c of tile row r is a pair the tile owns:
// both nodes exist (i = I T + r < n, j = J T + 32 cc + c < n) and, on a
// diagonal tile, j > i.
__device__ __forceinline__ uint32_t chunk_valid(int n, int I, int J, int r, int cc)
{
    if (I * T + r >= n) return 0u;
    const int hi = min(32, n - (J * T + 32 * cc));
    const int lo = I == J ? max(0, r - 32 * cc + 1) : 0;
    if (hi <= 0 || lo >= hi) return 0u;
    const uint32_t upto = hi == 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);   // lo < hi <= 32, so lo < 32
}

// out = BF16 q_ij for the 32 columns of one row chunk (0 where `valid` has no
// bit): q_ij = y_i y_j (exp(-gamma d2) + lambda^2), d2 = max(0, ||x_i||^2 +
// ||x_j||^2 - 2 g_ij) with g the Gram values of the chunk.  Lane c of the warp
// holds y_j and ||x_j||^2 of column c (yl, sl); they reach the other lanes by
// shuffles.  exp is the hardware-based __expf: its relative error (a few 1e-6
// for these arguments) is far below the BF16 rounding of the entries.
__device__ __forceinline__ void q_chunk_bf16(const float (&g)[32], float yi, float si, float yl, float sl,
                                             float gamma, float lam2, uint32_t valid, uint4 (&out)[4])
{
    uint32_t w[16];
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
        float q2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float yj = __shfl_sync(0xffffffffu, yl, c + u);
            const float sj = __shfl_sync(0xffffffffu, sl, c + u);
            const float d2 = fmaxf(0.f, si + sj - 2.f * g[c + u]);
            const float q = yi * yj * (__expf(-gamma * d2) + lam2);
            q2[u] = ((valid >> (c + u)) & 1u) ? q : 0.f;
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(q2[0], q2[1]);
        w[c / 2] = *reinterpret_cast<const uint32_t*>(&h);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

}  // namespace gabp
