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

// log2(e): K = exp(-gamma d2) = 2^(-gamma log2(e) d2).
constexpr float kLog2e = 1.4426950408889634f;

// The column constants of one 32-column chunk, staged in shared memory by
// the warp that uses them: b[c] = -gamma log2(e) ||x_j||^2 and sy[c] = the
// sign bit of y_j, for column j = J T + 32 cc + c.
struct ColChunk {
    alignas(16) float b[32];
    alignas(16) uint32_t sy[32];
};

// Lane c writes column c's constants from its y_j (yl) and ||x_j||^2 (sl)
// (0 beyond n: such columns are masked out).  The first __syncwarp keeps the
// previous chunk's constants until every lane has read them.
__device__ __forceinline__ void stage_cols(ColChunk& cs, float yl, float sl, float gamma, int lane)
{
    __syncwarp();
    cs.b[lane] = -gamma * kLog2e * sl;
    cs.sy[lane] = __float_as_uint(yl) & 0x80000000u;
    __syncwarp();
}

// 2^t by the hardware approximation (relative error of a few units in the
// last place of FP32, far below the BF16 rounding of the Q entries).
__device__ __forceinline__ float ex2_approx(float t)
{
    float r;
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
}

// out = BF16 q_ij for the 16 columns h0 .. h0 + 15 (h0 = 0 or 16) of one row
// chunk (0 where `valid` has no bit): q_ij = y_i y_j (exp(-gamma d2) +
// lambda^2), d2 = max(0, ||x_i||^2 + ||x_j||^2 - 2 g_ij) with g the Gram
// values of those columns, evaluated as 2^min(0, a_i + b_j + c2 g_ij) with
// a_i = -gamma log2(e) ||x_i||^2, b_j from the staged column constants and
// c2 = 2 gamma log2(e); the label product y_i y_j = +-1 is applied as a sign
// flip (sign bits syi ^ sy_j).
__device__ __forceinline__ void q_half_bf16(const float (&g)[16], int h0, float ai, uint32_t syi, const ColChunk& cs,
                                            float c2, float lam2, uint32_t valid, uint4 (&out)[2])
{
    uint32_t w[8];
#pragma unroll
    for (int c = 0; c < 16; c += 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(&cs.b[h0 + c]);
        const uint4 s4 = *reinterpret_cast<const uint4*>(&cs.sy[h0 + c]);
        const float bj[4] = {b4.x, b4.y, b4.z, b4.w};
        const uint32_t sj[4] = {s4.x, s4.y, s4.z, s4.w};
        float q4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float t = fminf(fmaf(c2, g[c + u], bj[u]) + ai, 0.f);
            const float q = ex2_approx(t) + lam2;
            const float qs = __uint_as_float(__float_as_uint(q) ^ syi ^ sj[u]);
            q4[u] = ((valid >> (h0 + c + u)) & 1u) ? qs : 0.f;
        }
        __nv_bfloat162 p0 = __floats2bfloat162_rn(q4[0], q4[1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(q4[2], q4[3]);
        w[c / 2] = *reinterpret_cast<const uint32_t*>(&p0);
        w[c / 2 + 1] = *reinterpret_cast<const uint32_t*>(&p1);
    }
    out[0] = make_uint4(w[0], w[1], w[2], w[3]);
    out[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

}  // namespace gabp
