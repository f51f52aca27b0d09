// Epilogue of the tensor-core Gram tiles (Q formation in the BF16 store and
// the fused recompute inside the sweep): BF16 Q entries from the FP32 Gram
// accumulators read out of tensor memory, 16 columns of a row at a time, with
// the column constants of the tile staged once in shared memory.  Both
// kernels call the same code, so the recomputed tiles equal the stored ones
// bit for bit.
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

// The column constants of a tile's 128 columns, staged in shared memory by
// the epilogue warp that uses them: b[c] = -gamma log2(e) ||x_j||^2 and the
// sign bits of the labels y_j, two columns to a word (column 2 w in bit 15
// of s2[w], column 2 w + 1 in bit 31: the sign bits of a BF16 pair), for
// column j = J T + c.
struct ColTile {
    alignas(16) float b[T];
    alignas(16) uint32_t s2[T / 2];
};

// Lane l writes the constants of columns 32 cc + l for the chunks cc in
// [cc0, cc1) from the labels y and the norms sqb of the column block J
// (zeros beyond n: such columns are masked out).  The first __syncwarp keeps
// the previous tile's constants until every lane has read them.
__device__ __forceinline__ void stage_tile_cols(ColTile& ct, const float* __restrict__ y,
                                                const float* __restrict__ sqb, int n, int J, float gamma,
                                                int lane, int cc0, int cc1)
{
    float yl[4], sl[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int j = J * T + 32 * cc + lane;
        const bool in = cc >= cc0 && cc < cc1 && j < n;
        yl[cc] = in ? y[j] : 0.f;
        sl[cc] = in ? sqb[j] : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc < cc0 || cc >= cc1) continue;
        ct.b[32 * cc + lane] = -gamma * kLog2e * sl[cc];
        const uint32_t sg = __float_as_uint(yl[cc]) & 0x80000000u;
        const uint32_t other = __shfl_xor_sync(0xffffffffu, sg, 1);
        if (!(lane & 1)) ct.s2[16 * cc + lane / 2] = (sg >> 16) | other;
    }
    __syncwarp();
}

// 2^t by the hardware approximation (relative error of a few units in the
// last place of FP32, far below the BF16 rounding of the Q entries), with
// results below the smallest normal FP32 value flushed to 0: such kernel
// values (gamma d2 > 87) only matter without the bias term (lambda = 0),
// where they stand for entries below 1.2e-38 of a matrix whose diagonal is
// at least 1.
__device__ __forceinline__ float ex2_approx(float t)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
}

// out = BF16 q_ij for the 16 columns c0 .. c0 + 15 of one tile row (c0 a
// multiple of 16), as eight BF16 pairs: q_ij = y_i y_j (exp(-gamma d2) +
// lambda^2), d2 = max(0, ||x_i||^2 + ||x_j||^2 - 2 g_ij) with g the Gram values
// of those columns, evaluated as 2^min(0, a_i + b_j + c2 g_ij) with
// a_i = -gamma log2(e) ||x_i||^2, b_j from the staged column constants and
// c2 = 2 gamma log2(e), two columns per instruction where the arithmetic
// allows.  The label product y_i y_j = +-1 is applied to the rounded pair as
// a flip of its sign bits (rounding to nearest is symmetric, so this equals
// rounding the signed value); si2 holds the sign bit of y_i in bits 15 and
// 31.  Columns whose bit in `valid` (bit u for column c0 + u) is clear
// come out +0.
__device__ __forceinline__ void q_half_bf16(const float (&g)[16], int c0, float ai, uint32_t si2, const ColTile& ct,
                                            float c2, float lam2, uint32_t valid, uint4 (&out)[2])
{
    const float2 c22 = make_float2(c2, c2), ai2 = make_float2(ai, ai), lam22 = make_float2(lam2, lam2);
    uint32_t w[8];
#pragma unroll
    for (int c = 0; c < 16; c += 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(&ct.b[c0 + c]);
        const uint2 s = *reinterpret_cast<const uint2*>(&ct.s2[(c0 + c) / 2]);
        const float2 t01 = __fadd2_rn(__ffma2_rn(c22, make_float2(g[c], g[c + 1]), make_float2(b4.x, b4.y)), ai2);
        const float2 t23 = __fadd2_rn(__ffma2_rn(c22, make_float2(g[c + 2], g[c + 3]), make_float2(b4.z, b4.w)), ai2);
        const float2 q01 = __fadd2_rn(make_float2(ex2_approx(fminf(t01.x, 0.f)), ex2_approx(fminf(t01.y, 0.f))), lam22);
        const float2 q23 = __fadd2_rn(make_float2(ex2_approx(fminf(t23.x, 0.f)), ex2_approx(fminf(t23.y, 0.f))), lam22);
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(q01.x, q01.y);
        const __nv_bfloat162 p1 = __floats2bfloat162_rn(q23.x, q23.y);
        w[c / 2] = *reinterpret_cast<const uint32_t*>(&p0) ^ s.x ^ si2;
        w[c / 2 + 1] = *reinterpret_cast<const uint32_t*>(&p1) ^ s.y ^ si2;
    }
    if (valid != 0xffffu) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t lo = 0u - ((valid >> (2 * k)) & 1u), hi = 0u - ((valid >> (2 * k + 1)) & 1u);
            w[k] &= (lo & 0x0000ffffu) | (hi & 0xffff0000u);
        }
    }
    out[0] = make_uint4(w[0], w[1], w[2], w[3]);
    out[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

}  // namespace gabp
