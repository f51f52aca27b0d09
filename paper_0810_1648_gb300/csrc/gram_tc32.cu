// FP32-accurate Gram tiles on the 5th-generation tensor cores (tcgen05),
// fused with the RBF kernel, labels and bias: the FP32 Q tiles of the plain
// form, the FP32 copy the BF16 store keeps for its refinement residuals, and
// the |Q| row sums that set the weighted diagonal (Section 5 computes the
// kernel matrix once; Section 3.1 weights the diagonal by those sums;
// Section 1.1 defines D_ij = y_i y_j K(x_i, x_j)).
//
// Three BF16 planes.  Every FP32 feature is split as x = x1 + x2 + x3 with
// x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (both differences
// are exact in FP32), so x1 + x2 + x3 carries x to about 2^-27 of its size.
// The dot product keeps the six plane products with a + b <= 4,
//   x.y ~ x1.y3 + x2.y2 + x3.y1 + x1.y2 + x2.y1 + x1.y1,
// issued smallest first; the dropped ones are below 2^-26 of |x||y|.  The
// tensor cores multiply BF16 exactly; their FP32 accumulation drops low bits
// (toward zero), so each 64-feature chunk gets a fresh accumulator and the
// chunks are added on the CUDA cores (round to nearest).  The squared norms in
// d^2 = ||x_i||^2 + ||x_j||^2 - 2 x_i.x_j come from the same products (the
// diagonal of the diagonal tiles, a first pass): for near pairs, where K is
// large, the norms and the Gram value then carry the same truncation, which
// cancels in d^2 instead of shrinking every K by ~2 gamma ||x||^2 x 1e-8.
//
// k_form_q_tc32 is persistent with warp roles: warp 0 streams the six 16 KB
// operand blocks of each (tile, chunk) into a two-stage shared-memory ring;
// warp 1 allocates 512 TMEM columns (four 128 x 128 FP32 accumulators, one per
// K-step) and one thread issues the 24 MMAs of a chunk (6 products x K = 64
// in steps of 16); warps 2-9 (two per TMEM lane quarter, one per column half)
// add each chunk's accumulators into registers, then form the Q entries
// (norm expansion, clamp, expf, bias, labels), store them, and reduce |Q| over
// rows (four interleaved partial sums), over columns
// (a warp transpose-sum, then the four lane quarters in shared memory) and to
// the tile maximum.  Instances chained behind the listed one (the points of a
// parameter grid over the same features) take their Q tiles from the same
// Gram sums.
#include "common.cuh"
#include "ptx.cuh"

#include <float.h>

namespace gabp {

namespace {

constexpr int NPLANE = 3;
constexpr int T3_EPI_WARPS = 8;
constexpr int T3_THREADS = (2 + T3_EPI_WARPS) * 32;
constexpr int T3_STAGES = 2;
constexpr size_t T3_STAGE_BYTES = (size_t)2 * NPLANE * BLK_BYTES;   // A planes, then B planes: 96 KB
// Accumulators per 64-feature chunk: one per K-step of 16 features, each
// receiving the step's five small products first and its x1.y1 product last,
// so that no x1.y1 partial sum passes through a truncating tensor-core
// addition; the chunk value is their sum on the CUDA cores (round to
// nearest).  Measured against the FP64 oracle (n = 2048, with the norms from
// the same products): mean relative error of K -2e-8 with four accumulators
// against +1.2e-6 with one (clustered data, gamma ||x||^2 ~ 24), +1.2e-7
// against +2.6e-7 (m = 128); formation 1.01 against 0.83 ms at n = 20000,
// m = 128.  With four, TMEM holds one chunk at a time.
constexpr int T3_NACC = 4;
static_assert(T3_NACC == 1 || T3_NACC == 2 || T3_NACC == 4, "1, 2 or 4 accumulators per chunk");
constexpr int T3_NBUF = T3_NACC == 4 ? 1 : 2;
constexpr uint32_t T3_TMEM_COLS = (uint32_t)(T3_NACC * T3_NBUF * T <= 256 ? 256 : 512);
constexpr uint32_t T3_IDESC = idesc_bf16_f32(T, T);
constexpr int T3_PRODUCTS = 6;

// Plane pairs (a, b) of the kept products, smallest first.
__device__ __forceinline__ int prod_a(int q) { return q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 3 ? 0 : q == 4 ? 1 : 0; }
__device__ __forceinline__ int prod_b(int q) { return q == 0 ? 2 : q == 1 ? 1 : q == 2 ? 0 : q == 3 ? 1 : q == 4 ? 0 : 0; }

// The three BF16 planes of x.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& b1, __nv_bfloat16& b2, __nv_bfloat16& b3)
{
    b1 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b1);
    b2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b2);
    b3 = __float2bfloat16_rn(r2);
}

// Offset (in 16-byte units) of row rr's 8-feature group kg inside a packed
// 128 x 64 block: 8-row x 16-byte core matrices, K-adjacent ones 128 bytes
// apart, 8-row groups 1024 bytes apart (the canonical K-major layout).
__device__ __forceinline__ size_t core_off16(int rr, int kg)
{
    return (size_t)((rr / 8) * (KCH / 8) + kg) * 8 + (rr % 8);
}

// Row r (of Nt*T, zero beyond n) and 8-feature group gk of chunk kc -> the
// three planes' blocks ((I nkc + kc) 3 + plane).
__device__ __forceinline__ void pack3_group(const float* __restrict__ Xf, int n, int m, int nkc, int r, int gk,
                                            uint4* __restrict__ Xp3)
{
    const int kc = gk / (KCH / 8), kg = gk % (KCH / 8);
    const int I = r / T, rr = r % T;
    __align__(16) __nv_bfloat16 v[NPLANE][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int k = kc * KCH + kg * 8 + u;
        split3((r < n && k < m) ? Xf[(size_t)r * m + k] : 0.f, v[0][u], v[1][u], v[2][u]);
    }
#pragma unroll
    for (int pl = 0; pl < NPLANE; ++pl) {
        const size_t blk = ((size_t)I * nkc + kc) * NPLANE + pl;
        Xp3[blk * (BLK_BYTES / 16) + core_off16(rr, kg)] = *reinterpret_cast<const uint4*>(v[pl]);
    }
}

__global__ void k_pack3(const float* __restrict__ Xf, int n, int m, int nkc, int Nt, uint4* __restrict__ Xp3)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long groups = (long long)nkc * (KCH / 8);
    if (e >= (long long)Nt * T * groups) return;
    pack3_group(Xf, n, m, nkc, (int)(e / groups), (int)(e % groups), Xp3);
}

// Listed node blocks (32 rows, 8 threads a row); the last block of an
// instance also writes the zero rows that pad its last tile.
__global__ void k_pack3_list(const Inst* __restrict__ tab, const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    const int rl = threadIdx.x >> 3, gsub = threadIdx.x & 7;
    const int r = nb.y * 32 + rl, n = p.n;
    const bool last = nb.y == (n - 1) / 32;
    uint4* Xp3 = static_cast<uint4*>(const_cast<void*>(p.Xp3));
    const int groups = p.nkc * (KCH / 8);
    for (int rw = r; rw < p.Nt * T; rw += 32) {
        for (int gk = gsub; gk < groups; gk += 8) pack3_group(p.X, n, p.m, p.nkc, rw, gk, Xp3);
        if (!last) break;
    }
}

struct T3Smem {
    unsigned long long xfull[T3_STAGES], xempty[T3_STAGES];
    unsigned long long accfull[T3_NBUF], accempty[T3_NBUF];
    unsigned long long drain;
    uint32_t tmem_base;
    int abort;
    float colsum[4][T];                 // per lane quarter: column sums over its 32 rows
    float rowsum[2][T];                 // per column half: row sums
    float tmx[T3_EPI_WARPS];
    alignas(16) uint32_t cy[T3_EPI_WARPS][64];   // a warp's 64 columns: sign bits of the labels
    alignas(16) float cs[T3_EPI_WARPS][64];   // and FP32 norms
};

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(T3_EPI_WARPS * 32) : "memory"); }

// After it, lane l of the warp holds the sum over the 32 lanes of v[l]
// (a fixed butterfly: 31 shuffles for 32 values).
__device__ __forceinline__ float transpose_sum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool hi = (lane & w) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = hi ? v[k] : v[k + w];
            const float keep = hi ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// FP32 Q entries of 32 columns of one tile row from the Gram values g,
// the staged column sign bits sy and norms sn: q = y_i y_j (exp(-gamma d2) +
// lambda^2), d2 = max(0, ||x_i||^2 + ||x_j||^2 - 2 g); the label product is a
// flip of the sign bit (y = +-1).  Not FULL: entries outside the pair set
// (i >= n, column j0 + cb + c >= n, or c + cb <= rdiag on a diagonal tile)
// are 0.  Adds |q| to the row sums rs4[c % 4].
template <bool FULL>
__device__ __forceinline__ void q_chunk32(const float* g, const uint32_t* sy, const float* sn, float si, uint32_t syi,
                                          float ngam, float lam2, int i, int n, int cb, int j0, int rdiag,
                                          float (&q)[32], float (&rs4)[4])
{
#pragma unroll
    for (int c4 = 0; c4 < 32; c4 += 4) {
        const uint4 y4 = *reinterpret_cast<const uint4*>(sy + c4);
        const float4 s4 = *reinterpret_cast<const float4*>(sn + c4);
        const uint32_t yj[4] = {y4.x, y4.y, y4.z, y4.w};
        const float sj[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float d2 = fmaxf(0.f, si + sj[t] - 2.f * g[c4 + t]);
            const float e = expf(ngam * d2) + lam2;
            float qv = __uint_as_float(__float_as_uint(e) ^ syi ^ yj[t]);
            if (!FULL) {
                const int c = cb + c4 + t;
                const bool valid = i < n && j0 + c < n && c > rdiag;
                qv = valid ? qv : 0.f;
            }
            q[c4 + t] = qv;
            rs4[t] += fabsf(qv);
        }
    }
}

__global__ void __launch_bounds__(T3_THREADS, 1)
    k_form_q_tc32(const Inst* __restrict__ tab, const int4* __restrict__ work, long long ntiles, int norms_only)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* ops = align_smem(smem_raw, 1024);
    T3Smem& sm = *reinterpret_cast<T3Smem*>(ops + T3_STAGES * T3_STAGE_BYTES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < T3_STAGES; ++s) { mbar_init(&sm.xfull[s], 1); mbar_init(&sm.xempty[s], 1); }
        for (int b = 0; b < T3_NBUF; ++b) { mbar_init(&sm.accfull[b], 1); mbar_init(&sm.accempty[b], T3_EPI_WARPS); }
        mbar_init(&sm.drain, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, T3_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sm.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ operand producer
        if (lane == 0) {
            const uint64_t pol = l2_evict_first_policy();
            int stage = 0;
            uint32_t ph = 0;
            bool run = true;
            for (long long L = blockIdx.x; L < ntiles && run; L += gridDim.x) {
                const int4 w = work[L];
                const Inst& p = tab[w.x];
                const unsigned char* Xp3 = static_cast<const unsigned char*>(p.Xp3);
                const int I = w.y, J = w.z, nkc = p.nkc;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*(volatile int*)&sm.abort || !mbar_wait(&sm.xempty[stage], ph ^ 1u)) {
                        sm.abort = 1;
                        record_error(p.ctrl, ST_ETIMEOUT, L);
                        run = false;
                        break;
                    }
                    unsigned char* S = ops + (size_t)stage * T3_STAGE_BYTES;
                    mbar_arrive_expect_tx(&sm.xfull[stage], (uint32_t)T3_STAGE_BYTES);
#pragma unroll
                    for (int pl = 0; pl < NPLANE; ++pl) {
                        bulk_load(S + (size_t)pl * BLK_BYTES, Xp3 + (((size_t)I * nkc + kc) * NPLANE + pl) * BLK_BYTES,
                                  BLK_BYTES, &sm.xfull[stage], pol);
                        bulk_load(S + (size_t)(NPLANE + pl) * BLK_BYTES,
                                  Xp3 + (((size_t)J * nkc + kc) * NPLANE + pl) * BLK_BYTES, BLK_BYTES, &sm.xfull[stage],
                                  pol);
                    }
                    if (++stage == T3_STAGES) { stage = 0; ph ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool run = true;
            for (long long L = blockIdx.x; L < ntiles && run; L += gridDim.x) {
                const Inst& p = tab[work[L].x];
                Ctrl* ctrl = p.ctrl;
                const int nkc = p.nkc;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*(volatile int*)&sm.abort || !mbar_wait(&sm.accempty[acc], aph ^ 1u) ||
                        !mbar_wait(&sm.xfull[stage], ph)) {
                        sm.abort = 1;
                        record_error(ctrl, ST_ETIMEOUT, L);
                        run = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* S = ops + (size_t)stage * T3_STAGE_BYTES;
                    constexpr int SPA = (KCH / 16) / T3_NACC;   // K-steps per accumulator
#pragma unroll
                    for (int a = 0; a < T3_NACC; ++a) {
                        const uint32_t d = tbase + (uint32_t)(acc * T3_NACC + a) * T;
#pragma unroll
                        for (int q = 0; q < T3_PRODUCTS; ++q) {
#pragma unroll
                            for (int s = a * SPA; s < (a + 1) * SPA; ++s) {
                                const uint64_t ad = smem_desc(S + (size_t)prod_a(q) * BLK_BYTES + s * 256, 128, 1024);
                                const uint64_t bd =
                                    smem_desc(S + (size_t)(NPLANE + prod_b(q)) * BLK_BYTES + s * 256, 128, 1024);
                                tc_mma_bf16(d, ad, bd, T3_IDESC, (q != 0 || s != a * SPA) ? 1u : 0u);
                            }
                        }
                    }
                    tc_commit(&sm.xempty[stage]);
                    tc_commit(&sm.accfull[acc]);
                    if (++stage == T3_STAGES) { stage = 0; ph ^= 1u; }
                    if (++acc == T3_NBUF) { acc = 0; aph ^= 1u; }
                }
            }
            // every MMA issued above must finish before the columns are freed
            tc_commit(&sm.drain);
            if (!mbar_wait(&sm.drain, 0u)) sm.abort = 1;
        }
    } else {
        // --------------------------------------------------------- epilogue
        // warp w reads TMEM lanes 32 (w % 4) ..: rows 32 g + lane, columns
        // [64 half, 64 half + 64)
        const int ew = warp - 2, g = warp & 3, half = ew >> 2;
        const int r = 32 * g + lane, c0 = 64 * half;
        const int etid = tid - 64;
        int acc = 0;
        uint32_t aph = 0;
        for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
            const int4 w = work[L];
            const int nkc = tab[w.x].nkc;
            float ga[64];
#pragma unroll
            for (int c = 0; c < 64; ++c) ga[c] = 0.f;
            bool ok = true;
            for (int kc = 0; kc < nkc; ++kc) {
                const bool stop = __shfl_sync(0xffffffffu, *(volatile int*)&sm.abort, 0) != 0;
                if (stop || !mbar_wait_warp(&sm.accfull[acc], aph)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // the chunk's accumulators added to the running sums in order,
                // 16 columns at a time
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int a = 0; a < T3_NACC; ++a) {
                        float v[16];
                        tmem_ld16(tbase + (uint32_t)(acc * T3_NACC + a) * T + ((uint32_t)(32 * g) << 16) +
                                      (uint32_t)(c0 + 16 * j),
                                  v);
                        if (kc == 0 && a == 0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c) ga[16 * j + c] = v[c];
                        } else {
                            // two columns per instruction, each rounded as a scalar add
#pragma unroll
                            for (int c = 0; c < 16; c += 2) {
                                const float2 t2 = __fadd2_rn(make_float2(ga[16 * j + c], ga[16 * j + c + 1]),
                                                             make_float2(v[c], v[c + 1]));
                                ga[16 * j + c] = t2.x;
                                ga[16 * j + c + 1] = t2.y;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.accempty[acc]);
                if (++acc == T3_NBUF) { acc = 0; aph ^= 1u; }
            }
            if (!ok && lane == 0) {
                sm.abort = 1;
                record_error(tab[w.x].ctrl, ST_ETIMEOUT, L);
            }
            epi_bar();   // every epilogue warp takes the stop decision together
            if (*(volatile int*)&sm.abort) break;
            const int I = w.y, J = w.z;
            const int i = I * T + r;
            if (norms_only) {
                // diagonal tile: x_i . x_i is the Gram value at (r, r), held by the
                // warp of r's lane quarter whose column half contains r
                if (half == (g >> 1)) {
                    float d = 0.f;
#pragma unroll
                    for (int c = 0; c < 64; ++c) d = (c0 + c == r) ? ga[c] : d;
                    for (int k = w.x; k >= 0; k = tab[k].form_next - 1)
                        if (i < tab[k].n) tab[k].sq3[i] = d;
                }
                continue;
            }
            for (int k = w.x; k >= 0;) {
                const Inst& p = tab[k];
                const int n = p.n;
                // this warp's 64 column labels and norms
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = J * T + c0 + 32 * u + lane;
                    sm.cy[ew][32 * u + lane] = j < n ? (__float_as_uint(p.y[j]) & 0x80000000u) : 0u;
                    sm.cs[ew][32 * u + lane] = j < n ? p.sq3[j] : 0.f;
                }
                __syncwarp();
                const float si = i < n ? p.sq3[i] : 0.f, ngam = -p.gamma, lam2 = p.lam2;
                const uint32_t syi = i < n ? (__float_as_uint(p.y[i]) & 0x80000000u) : 0u;
                // interior tile: every pair valid
                const bool full = I != J && (I + 1) * T <= n && (J + 1) * T <= n;
                float* qt = p.qref ? p.qref + (size_t)w.w * TT + (size_t)r * T + c0 : nullptr;
                float rs4[4] = {0.f, 0.f, 0.f, 0.f}, tmx = 0.f;   // row sum in four interleaved parts
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float q[32];
                    if (full)
                        q_chunk32<true>(ga + 32 * u, sm.cy[ew] + 32 * u, sm.cs[ew] + 32 * u, si, syi, ngam, lam2,
                                        0, 0, 0, 0, 0, q, rs4);
                    else
                        q_chunk32<false>(ga + 32 * u, sm.cy[ew] + 32 * u, sm.cs[ew] + 32 * u, si, syi, ngam, lam2,
                                         i, n, c0 + 32 * u, J * T, I == J ? r : -1, q, rs4);
                    if (p.tilemax) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) tmx = fmaxf(tmx, fabsf(q[c]));
                    }
                    if (qt) {
#pragma unroll
                        for (int c4 = 0; c4 < 32; c4 += 4)
                            *reinterpret_cast<float4*>(qt + 32 * u + c4) = make_float4(q[c4], q[c4 + 1], q[c4 + 2], q[c4 + 3]);
                    }
#pragma unroll
                    for (int c = 0; c < 32; ++c) q[c] = fabsf(q[c]);
                    sm.colsum[g][c0 + 32 * u + lane] = transpose_sum32(q, lane);
                }
                sm.rowsum[half][r] = (rs4[0] + rs4[1]) + (rs4[2] + rs4[3]);
                tmx = warp_max_f(tmx);
                if (lane == 0) sm.tmx[ew] = tmx;
                epi_bar();
                // per-node slot partials (fixed order): row sums of the tile's rows,
                // column sums of its columns; both roles on a diagonal tile
                // (slot sl.x of the row block, sl.y of the column block).  Where
                // rfix is set they are added to the nodes' fixed-point sums instead.
                int x = -1, off = 0, role = 0;
                float v = 0.f;
                if (I == J) {
                    if (etid < T) {
                        x = I * T + etid;
                        off = etid;
                        v = (sm.rowsum[0][etid] + sm.rowsum[1][etid]) +
                            (((sm.colsum[0][etid] + sm.colsum[1][etid]) + sm.colsum[2][etid]) + sm.colsum[3][etid]);
                    }
                } else if (etid < T) {
                    x = I * T + etid;
                    off = etid;
                    v = sm.rowsum[0][etid] + sm.rowsum[1][etid];
                } else if (etid < 2 * T) {
                    off = etid - T;
                    x = J * T + off;
                    role = 1;
                    v = ((sm.colsum[0][off] + sm.colsum[1][off]) + sm.colsum[2][off]) + sm.colsum[3][off];
                }
                if (x >= 0 && x < n) {
                    if (p.rfix) {
                        atomicAdd(p.rfix + x, (unsigned long long)rsum_fix(v, pow2i(rsum_shift(n, lam2))));
                    } else {
                        const int2 sl = tile_slots(p, w);
                        p.part[(size_t)(role ? sl.y : sl.x) * T + off] = v;
                    }
                }
                if (etid == 0 && p.tilemax) {
                    float m2 = 0.f;
                    for (int e = 0; e < T3_EPI_WARPS; ++e) m2 = fmaxf(m2, sm.tmx[e]);
                    p.tilemax[w.w] = m2;
                }
                epi_bar();   // shared sums read before the next instance or tile writes them
                k = p.form_next - 1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, T3_TMEM_COLS);
    }
}

constexpr size_t t3_smem_bytes() { return 1024 + T3_STAGES * T3_STAGE_BYTES + sizeof(T3Smem); }

}  // namespace

size_t pack3_bytes(int Nt, int m) { return (size_t)NPLANE * Nt * bf16_chunks(m) * BLK_BYTES; }

cudaError_t launch_pack3(const float* Xf, int n, int m, int Nt, void* Xp3, cudaStream_t s)
{
    const int nkc = bf16_chunks(m);
    const long long total = (long long)Nt * T * nkc * (KCH / 8);
    k_pack3<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Xf, n, m, nkc, Nt, static_cast<uint4*>(Xp3));
    return cudaGetLastError();
}

cudaError_t launch_pack3_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) k_pack3_list<<<nblocks, 256, 0, s>>>(tab, nbl);
    return cudaGetLastError();
}

cudaError_t launch_form_q_tc32(const Inst* tab, const int4* work, long long ntiles, int norms_only, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_form_q_tc32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)t3_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int sms = num_sms();
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_form_q_tc32<<<grid, T3_THREADS, t3_smem_bytes(), s>>>(tab, work, ntiles, norms_only);
    return cudaGetLastError();
}

}  // namespace gabp
