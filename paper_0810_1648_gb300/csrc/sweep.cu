// The synchronous broadcast-GaBP round (Algorithm 2, Section 4) on the
// device: a pair sweep over the stored upper triangle followed by a per-node
// finalize that forms the next aggregates, the residual and the stop test.
//
// Round t, information form (H = P mu):
//   sweep    for every pair {i < j} with q = Q_ij, from the aggregates of t
//            (Ptilde, htilde = Ptilde mutilde) and the pair's messages:
//              d_i = Ptilde_i - P_ji,  d_j = Ptilde_j - P_ij   (cavities)
//              P_ij <- -q^2 / d_i,     H_ij <- -q (htilde_i - H_ji) / d_i
//              P_ji <- -q^2 / d_j,     H_ji <- -q (htilde_j - H_ij) / d_j
//            node j collects (P_ij, H_ij), node i collects (P_ji, H_ji);
//            both collect q mutilde of the other end for r(t).
//   finalize Ptilde_i(t+1) = Q_ii + sum_k P_ki, htilde_i(t+1) = b_i + sum_k H_ki,
//            mutilde = htilde / Ptilde (Step 2), r_i(t) = b_i - Q_ii mutilde_i(t)
//            - sum_j Q_ij mutilde_j(t) with FP64 cross-tile sums, and the
//            Step-3 test ||r(t)||_inf < tol in the last CTA to finish.
//
// The sweep is bound by HBM bandwidth: per pair it reads 16 B of messages and
// 4 B of Q (2 B in BF16) and writes 16 B; once the P messages sit at their
// fixed point it writes only the 8 B of H (messages stored in BF16 halve the
// message bytes).  Messages and Q arrive in shared memory through bulk copies
// issued by a producer warp well ahead of use; consumer warp w takes rows w
// and w + 8 of each 16-row chunk, each lane four of their columns laid out so
// that every warp access to a row is one contiguous 512-byte span (lane_col).
// Row sums go through one warp reduction per two rows (four with BF16
// messages), column sums stay in registers and meet in shared memory, and each
// node's per-tile sums go to its own slot (common.cuh), so the reduction order
// is fixed and the result reproducible.
#include "common.cuh"
#include "ptx.cuh"
#include "qtile_epi.cuh"

#include <algorithm>
#include <float.h>
#include <type_traits>

namespace gabp {

namespace {

// Named barrier of the CW consumer warps.
template <int CW>
__device__ __forceinline__ void consumer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(CW * 32) : "memory"); }


// ---- pair sweep -----------------------------------------------------------
// Persistent CTAs walk the tile list with stride gridDim.x.  A producer warp
// publishes each tile's parameters and bulk-copies its row and column
// aggregates into a double-buffered tile slot, then streams the tile as
// chunks of rc<MSG>() rows of messages (and, when Q is stored, of Q) into a
// stages<MSG>()-deep shared-memory ring, running ahead across tile boundaries;
// the consumers follow the tiles it publishes.  Eight consumer warps take two
// rows of each chunk, update their pairs from shared memory and store the new
// messages straight to global memory with 128-bit streaming stores.  Only the
// pairs the tile owns are copied: whole chunks for interior tiles, the c > r
// part of each row on diagonal tiles, the first `cols` columns on the last
// tile column (one row per producer lane).
//
// Two kernels share the producer and consumer code:
//   k_sweep<QT>   Q stored (FP32 or BF16) and streamed with the messages;
//   k_sweep_rc    Q recomputed in every sweep: a second producer streams the
//                 BF16 feature blocks of the tile, one thread issues tcgen05
//                 MMAs into a double-buffered TMEM accumulator, four warps
//                 turn the Gram rows into BF16 Q values in a double-buffered
//                 shared-memory Q tile, which the consumers read in place of
//                 a stored tile (bitwise the same values as the BF16 store).
// Rows per ring stage (16), two per consumer warp (eight consumer warps in
// both kernels, so that the recomputed and the stored form sum in the same
// order).
constexpr int RC_ROWS = 16;
template <class MSG>
__host__ __device__ constexpr int rc() { return RC_ROWS; }
constexpr int STAGES = 4;                     // barrier slots of the stage ring (upper bound)
// Ring stages used by a message type (both keep ~80 KB of rows in flight).
template <class MSG>
__host__ __device__ constexpr int stages() { return MSG::NSTAGE; }
constexpr int SWEEP_THREADS = NTHREADS + 32;  // + one producer warp
// 1/d for the cavity precisions: the hardware approximate reciprocal
// refined by one Newton-Raphson step r <- r (2 - d r) (error within about one
// unit in the last place for normal positive d; checked against IEEE division
// by gabp_selftest_reciprocal).
__device__ __forceinline__ float rcp_nr(float d)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return fmaf(r, fmaf(-d, r, 1.0f), r);
}

// Message storage: FP32 pairs (plain and precision forms) or BF16 pairs
// (precision forms with refinement).  Arithmetic is FP32 either way; sums use
// the stored (rounded) values so that the aggregates match the messages the
// next round reads.
struct MsgF32 {
    using T2 = float2;
    static constexpr bool MIXED = false;   // no BF16 halves to read directly
    static __device__ __forceinline__ T2 pack(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ float2 unpack(T2 v) { return v; }
    static __device__ __forceinline__ bool same(T2 a, T2 b) { return (a.x == b.x) & (a.y == b.y); }
    // 1/q of the frozen-P update: the refined reciprocal; 0 for |q| below the
    // smallest normal float, where P = -q^2 / d is 0 (the reciprocal of a
    // flushed subnormal would be inf, and 0 * inf a NaN)
    static __device__ __forceinline__ float qinv(float q) { return fabsf(q) >= FLT_MIN ? rcp_nr(q) : 0.f; }
    // the same where |q| >= FLT_MIN is known (no guard)
    static __device__ __forceinline__ float qinv_normal(float q) { return rcp_nr(q); }
    // a lane's pairs of a row: columns 2 lane + {0, 1} and 64 + 2 lane + {0, 1}
    // (each access of the warp is one contiguous 512-byte span)
    static constexpr int G = 2;
    static constexpr int NSTAGE = 2;   // ring stages of 16 rows (40 KB with FP32 Q)
    static constexpr int SPC = 1;      // stages per row-sum reduction
    // diagonal and edge tiles: only the owned pairs of each row are copied
    // (one copy per row; the form is bandwidth bound, so bytes count)
    static constexpr bool WHOLE_ROWS = false;
    static __device__ __forceinline__ void load4(const T2* row, int lane, T2 (&v)[4])
    {
        const float4 a = *reinterpret_cast<const float4*>(row + 2 * lane);
        const float4 b = *reinterpret_cast<const float4*>(row + 64 + 2 * lane);
        v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
        v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
    }
    static __device__ __forceinline__ void store4(T2* row, int lane, const T2 (&v)[4])
    {
        __stcs(reinterpret_cast<float4*>(row + 2 * lane), make_float4(v[0].x, v[0].y, v[1].x, v[1].y));
        __stcs(reinterpret_cast<float4*>(row + 64 + 2 * lane), make_float4(v[2].x, v[2].y, v[3].x, v[3].y));
    }
};
struct MsgBF16 {
    using T2 = unsigned;   // two BF16 values, the first in the low half
    // Mixed-precision arithmetic reads a BF16 half of a stored word as an FP32
    // operand (exact widening) in the same instruction, with no unpacking:
    // lo_minus / hi_minus = half - c, add_lo / add_hi: s += half.
    static constexpr bool MIXED = true;
    static __device__ __forceinline__ float lo_minus(T2 w, float c)
    {
        float d;
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tsub.rn.f32.bf16 %0, l, %2;\n\t}" : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    static __device__ __forceinline__ float hi_minus(T2 w, float c)
    {
        float d;
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tsub.rn.f32.bf16 %0, h, %2;\n\t}" : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    static __device__ __forceinline__ void add_lo(float& s, T2 w)
    {
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.bf16 %0, l, %0;\n\t}" : "+f"(s) : "r"(w));
    }
    static __device__ __forceinline__ void add_hi(float& s, T2 w)
    {
        asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.bf16 %0, h, %0;\n\t}" : "+f"(s) : "r"(w));
    }
    static __device__ __forceinline__ T2 pack(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    static __device__ __forceinline__ float2 unpack(T2 v)
    {
        return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
    }
    static __device__ __forceinline__ bool same(T2 a, T2 b) { return a == b; }
    // 1/q of the frozen-P update: the hardware reciprocal alone (its error,
    // about 2^-23, vanishes in the BF16 rounding of the stored H), clamped to
    // +-3e38 so that |q| below the smallest normal float (flushed: inf) gives a
    // finite factor of P = 0
    static __device__ __forceinline__ float qinv(float q)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
        return fmaxf(fminf(r, 3.0e38f), -3.0e38f);
    }
    // the same where |q| >= FLT_MIN is known (no clamp)
    static __device__ __forceinline__ float qinv_normal(float q)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
        return r;
    }
    // a lane's pairs of a row: columns 4 lane + {0 .. 3} (16 bytes; each
    // access of the warp is one contiguous 512-byte span)
    static constexpr int G = 4;
    static constexpr int NSTAGE = 4;   // ring stages of 16 rows (20 KB with BF16 Q)
    // two stages per row-sum reduction (four rows per consumer warp): half the
    // shuffles of this instruction-bound form per pair
    static constexpr int SPC = 2;
    // diagonal and edge tiles also move 16 whole rows per copy (the unowned
    // entries are masked by the consumers): sixteen times fewer bulk copies
    // for a few percent more bytes, faster for this instruction-heavy form
    static constexpr bool WHOLE_ROWS = true;
    static __device__ __forceinline__ void load4(const T2* row, int lane, T2 (&v)[4])
    {
        const uint4 u = *reinterpret_cast<const uint4*>(row + 4 * lane);
        v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
    }
    static __device__ __forceinline__ void store4(T2* row, int lane, const T2 (&v)[4])
    {
        __stcs(reinterpret_cast<uint4*>(row + 4 * lane), make_uint4(v[0], v[1], v[2], v[3]));
    }
};

template <class MSG>
__host__ __device__ constexpr size_t pchunk() { return (size_t)rc<MSG>() * T * sizeof(typename MSG::T2); }

// Resident sweep CTAs per SM: two for both message types (three for the
// BF16-message kernel spilled registers and ran slower than two).
template <class MSG>
__host__ __device__ constexpr int sweep_ctas() { return 2; }
template <class MSG>
__host__ __device__ constexpr size_t state_chunk() { return 2 * pchunk<MSG>(); }

// What the producer publishes to the consumers for each tile it streams
// (double-buffered by tile parity, completed through tfull[slot]).
struct TileInfo {
    void* Pst;          // the tile's P message block
    void* Hst;          // the tile's H message block
    float* part;        // the instance's slot partial sums
    long long plen;     // floats of each partial array
    Ctrl* ctrl;
    long long L;        // work-list index (error records)
    int n, Nt, I, J;
    int sR, sC;         // the tile's slots: row block's, column block's
    int t, zero_h, frozen, end;
    int qnormal;        // every off-diagonal |q| >= FLT_MIN (lambda^2 >= 2 FLT_MIN)
};

// Shared state of the producer and the CW consumer warps.
template <int CW>
struct SweepTail {
    static constexpr int kCW = CW;
    unsigned long long full[STAGES], empty[STAGES];
    unsigned long long tfull[2], tempty[2];
    int cabort;                        // consumer-side stop, decided at a tile barrier
    TileInfo info[2];
    alignas(16) float agg[2][6][T];    // per slot: row block {Ptilde, htilde, mu}, column block {same}
    float cp[CW][T], ch[CW][T], cr[CW][T];
    float rp[T], rh[T], rr[T];
};

// Barriers and flags of the stage ring and the tile slots (one thread).
template <int CW>
__device__ __forceinline__ void init_tail(SweepTail<CW>& sm)
{
    for (int s = 0; s < STAGES; ++s) {
        mbar_init(&sm.full[s], 1);
        mbar_init(&sm.empty[s], CW);
    }
    for (int s = 0; s < 2; ++s) {
        mbar_init(&sm.tfull[s], 1);
        mbar_init(&sm.tempty[s], CW);
    }
    sm.cabort = 0;
}

// Ring stage = P messages of rc<MSG>() rows, their H messages, then (stored Q) their Q values.
template <typename QT>
struct QBytes { static constexpr size_t v = sizeof(QT); };
template <>
struct QBytes<void> { static constexpr size_t v = 0; };

template <typename QT, class MSG>
__host__ __device__ constexpr size_t stage_bytes() { return state_chunk<MSG>() + (size_t)rc<MSG>() * T * QBytes<QT>::v; }

template <typename QT, class MSG>
__host__ __device__ constexpr size_t sweep_smem_bytes()
{
    return 128 + stages<MSG>() * stage_bytes<QT, MSG>() + sizeof(SweepTail<NWARPS>);
}

// Producer (one warp).  For every tile it streams: publishes the tile's
// parameters and bulk-copies its row and column aggregates into the tile slot,
// then streams the message (and stored Q) rows through the stage ring.
// Interior tiles move rc<MSG>() whole rows per copy; diagonal and edge tiles copy each
// row's needed span, one row per lane.  QT = void: messages only.
template <typename QT, class MSG, size_t SB, class Tail>
__device__ __forceinline__ void sweep_producer(const Inst* __restrict__ tab, const int4* __restrict__ work,
                                               long long ntiles, Tail& sm, unsigned char* ring,
                                               volatile int* abort_flag, int lane, int stage_no)
{
    constexpr size_t QB = QBytes<QT>::v;
    constexpr size_t MB = sizeof(typename MSG::T2);
    constexpr size_t SC = state_chunk<MSG>(), PC = pchunk<MSG>();
    const uint64_t pol = l2_evict_first_policy();
    const uint64_t pol_keep = l2_evict_last_policy();
    int stage = 0, slot = 0;
    uint32_t phase = 0, tph = 0;
    auto stopped = [&]() { return __shfl_sync(0xffffffffu, abort_flag ? *abort_flag : 0, 0) != 0; };
    for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
        const int4 w = work[L];
        const Inst& p = tab[w.x];
        Ctrl* ctrl = p.ctrl;
        if (*(volatile const int*)&ctrl->done) continue;      // instance finished: tile skipped
        const int t = *(volatile const int*)&ctrl->t;
        const bool zero = t == 0;
        const int n = p.n, I = w.y, J = w.z;
        const int rows = min(T, n - I * T), cols = min(T, n - J * T);
        const bool diag = (I == J);
        const typename MSG::T2* sp = static_cast<const typename MSG::T2*>(p.Pst) + (size_t)w.w * TT;
        const typename MSG::T2* sh = static_cast<const typename MSG::T2*>(p.Hst) + (size_t)w.w * TT;
        const unsigned char* qt = QB ? static_cast<const unsigned char*>(p.qstore) + (size_t)w.w * TT * QB : nullptr;
        // tile slot: parameters + aggregates
        if (stopped() || !mbar_wait_warp(&sm.tempty[slot], tph ^ 1u)) {
            if (lane == 0) {
                record_error(ctrl, ST_ETIMEOUT, L);
                if (abort_flag) *abort_flag = 1;
            }
            return;
        }
        if (lane == 0) {
            TileInfo& ti = sm.info[slot];
            ti.Pst = const_cast<typename MSG::T2*>(sp);
            ti.Hst = const_cast<typename MSG::T2*>(sh);
            ti.part = p.part;
            ti.plen = (long long)part_len(p);
            ti.ctrl = ctrl;
            ti.L = L;
            ti.n = n; ti.Nt = p.Nt; ti.I = I; ti.J = J;
            const int2 sl = tile_slots(p, w);
            ti.sR = sl.x; ti.sC = sl.y;
            ti.t = t;
            ti.zero_h = *(volatile const int*)&ctrl->zero_h;
            ti.frozen = *(volatile const int*)&ctrl->p_frozen;
            // q = +-(K + lambda^2) with K >= 0: |q| >= lambda^2, also after the
            // rounding of a BF16 store
            ti.qnormal = p.lam2 >= 2.f * FLT_MIN;
            ti.end = 0;
            mbar_arrive_expect_tx(&sm.tfull[slot], 6 * T * sizeof(float));
        }
        __syncwarp();
        if (lane < 6) {
            // Ptilde and htilde from the previous stage's aggregates in a
            // staged round; mutilde (residual partials) from the round's start
            const int a = lane % 3;
            const float* base = (stage_no > 0 && a < 2) ? p.aggmid + (size_t)a * p.npad
                                                        : p.agg + (size_t)(t & 1) * 3 * p.npad + (size_t)a * p.npad;
            const float* agg = base + (size_t)(lane < 3 ? I : J) * T;
            bulk_load(&sm.agg[slot][lane][0], agg, T * sizeof(float), &sm.tfull[slot], pol_keep);
        }
        if (++slot == 2) { slot = 0; tph ^= 1u; }
        // message / Q rows
        constexpr int RC = rc<MSG>();
        const int nch = (rows + RC - 1) / RC;
        for (int c = 0; c < nch; ++c) {
            if (stopped() || !mbar_wait_warp(&sm.empty[stage], phase ^ 1u)) {
                if (lane == 0) {
                    record_error(ctrl, ST_ETIMEOUT, L);
                    if (abort_flag) *abort_flag = 1;
                }
                return;
            }
            unsigned char* S = ring + (size_t)stage * SB;
            unsigned long long* bar = &sm.full[stage];
            const int r0 = c * RC, nr = min(RC, rows - r0);
            if (MSG::WHOLE_ROWS || (!diag && cols == T)) {
                const uint32_t bq = (uint32_t)(nr * T * QB);
                const uint32_t bs = zero ? 0u : (uint32_t)(nr * T * MB);
                if (lane == 0) mbar_arrive_expect_tx(bar, bq + 2 * bs);
                __syncwarp();
                if (QB && lane == 0) bulk_load(S + SC, qt + (size_t)r0 * T * QB, bq, bar, pol);
                if (!zero && lane == 1) bulk_load(S, sp + (size_t)r0 * T, bs, bar, pol);
                if (!zero && lane == 2) bulk_load(S + PC, sh + (size_t)r0 * T, bs, bar, pol);
            } else {
                // row r0 + lane: columns [c0, c1) with c0, c1 multiples of 8
                // (16-byte granules of every array) covering the pairs it owns
                const int c1 = min(T, (cols + 7) & ~7);
                const int r = r0 + lane, c0 = diag ? ((r + 1) & ~7) : 0;
                const bool has = lane < nr && c0 < c1 && (!diag || r + 1 < cols);
                const uint32_t mine = has ? (uint32_t)((c1 - c0) * (QB + (zero ? 0 : 2 * MB))) : 0u;
                const uint32_t bytes = __reduce_add_sync(0xffffffffu, mine);
                if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
                __syncwarp();
                if (has) {
                    if (QB)
                        bulk_load(S + SC + ((size_t)lane * T + c0) * QB, qt + ((size_t)r * T + c0) * QB,
                                  (uint32_t)((c1 - c0) * QB), bar, pol);
                    if (!zero) {
                        const size_t o = ((size_t)lane * T + c0) * MB;
                        const uint32_t b2 = (uint32_t)((c1 - c0) * MB);
                        bulk_load(S + o, sp + (size_t)r * T + c0, b2, bar, pol);
                        bulk_load(S + PC + o, sh + (size_t)r * T + c0, b2, bar, pol);
                    }
                }
            }
            if (++stage == stages<MSG>()) { stage = 0; phase ^= 1u; }
        }
    }
    // end of this CTA's tiles
    if (!stopped() && mbar_wait_warp(&sm.tempty[slot], tph ^ 1u) && lane == 0) {
        sm.info[slot].end = 1;
        mbar_arrive(&sm.tfull[slot]);
    }
}

// Column slot k = 0..3 of a lane in a 128-column row: G consecutive columns
// in each of 4 / G groups of 32 G columns (G = 2 for FP32 messages, 4 for
// BF16 messages), so that every warp access to a row is contiguous.
template <int G>
__device__ __forceinline__ constexpr int lane_col(int lane, int k)
{
    return (k / G) * 32 * G + G * lane + k % G;
}

// The four slot values of a lane from / to a row of FP32 or BF16 scalars.
template <int G>
__device__ __forceinline__ void ld4(const float* row, int lane, float (&o)[4])
{
    if constexpr (G == 4) {
        const float4 a = *reinterpret_cast<const float4*>(row + 4 * lane);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else {
        const float2 a = *reinterpret_cast<const float2*>(row + 2 * lane);
        const float2 b = *reinterpret_cast<const float2*>(row + 64 + 2 * lane);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}
template <int G>
__device__ __forceinline__ void ld4(const __nv_bfloat16* row, int lane, float (&o)[4])
{
    if constexpr (G == 4) {
        const uint2 u = *reinterpret_cast<const uint2*>(row + 4 * lane);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    } else {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + 2 * lane));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + 64 + 2 * lane));
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}
template <int G>
__device__ __forceinline__ void st4(float* row, int lane, const float (&o)[4])
{
    if constexpr (G == 4) {
        *reinterpret_cast<float4*>(row + 4 * lane) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        *reinterpret_cast<float2*>(row + 2 * lane) = make_float2(o[0], o[1]);
        *reinterpret_cast<float2*>(row + 64 + 2 * lane) = make_float2(o[2], o[3]);
    }
}

// Sums the eight values {x0 .. x7} over the warp in a fixed order:
// afterwards every lane of the group (lane / 4) % 8 = k holds the total of
// value k (nine shuffles: the three sums of two rows, or the H and residual
// sums of four rows once P is frozen).
__device__ __forceinline__ float reduce_scatter8x(const float (&x)[8], int lane)
{
    const bool hi = (lane & 16) != 0;
    float y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        y[k] = (hi ? x[k + 4] : x[k]) + __shfl_xor_sync(0xffffffffu, hi ? x[k] : x[k + 4], 16);
    const bool b8 = (lane & 8) != 0;
    float z[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
        z[k] = (b8 ? y[k + 2] : y[k]) + __shfl_xor_sync(0xffffffffu, b8 ? y[k] : y[k + 2], 8);
    const bool b4 = (lane & 4) != 0;
    float v = (b4 ? z[1] : z[0]) + __shfl_xor_sync(0xffffffffu, b4 ? z[0] : z[1], 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}
// The three sums {P, H, R} of two rows: values {a0, a1, a2, 0, b0, b1, b2, 0}.
__device__ __forceinline__ float reduce_scatter8(float a0, float a1, float a2, float b0, float b1, float b2,
                                                 int lane)
{
    const float x[8] = {a0, a1, a2, 0.f, b0, b1, b2, 0.f};
    return reduce_scatter8x(x, lane);
}

// Sums the four values {a0, a1, a2, a3} over the warp in a fixed order:
// afterwards every lane of the group (lane / 8) % 4 = k holds the total of
// value k (six shuffles: the three sums of one row, or the H and residual
// sums of two rows once P is frozen).
__device__ __forceinline__ float reduce_scatter4(float a0, float a1, float a2, float a3, int lane)
{
    const float x[4] = {a0, a1, a2, a3};
    const bool hi = (lane & 16) != 0;
    float y[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
        y[k] = (hi ? x[k + 2] : x[k]) + __shfl_xor_sync(0xffffffffu, hi ? x[k] : x[k + 2], 16);
    const bool b8 = (lane & 8) != 0;
    float v = (b8 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, b8 ? y[0] : y[1], 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// Per-tile column values a consumer lane needs for its row updates.
struct ColVals {
    float P[4], H[4], M[4];      // aggregates of the lane's four columns
    float aP[4], aH[4], aR[4];   // column partial sums
};

// Two-wide FP32 arithmetic (one instruction for two lanes of values; each
// half rounds exactly as the scalar operation would).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// c - b, bitwise equal to the scalar subtraction (the product -1 * b is exact)
__device__ __forceinline__ float2 sub2(float2 c, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, c); }

// Updates the lane's four pairs (r, lane_col(lane, k)) of chunk row r held in
// shared memory.  FULL: interior tile, every column valid (no
// predicates); FROZEN: the P messages are at their fixed point (no P stores,
// no P sums).  Adds the lane's share of the row sums to rs[0..2] (P, H,
// residual).  Whole 4-pair groups are stored: on diagonal and edge tiles the
// slots outside the pair set are never read, so writing them is harmless.
// The arithmetic runs on the column pairs {0, 1} and {2, 3} two at a time; a
// lane's row sums add columns {0, 2} and {1, 3} first, then the two halves.
template <bool FULL, bool FROZEN, bool QN, class MSG, class QSrc>
__device__ __forceinline__ void update_row(const QSrc& qsrc, const unsigned char* S, int lr, int lane, int r,
                                           int cols, bool diag, int it, bool zero, bool zero_h, float rP,
                                           float rH, float rM, ColVals& cv, typename MSG::T2* __restrict__ gp,
                                           typename MSG::T2* __restrict__ gh, float (&rs)[3], bool& bad,
                                           bool& changed)
{
    using T2 = typename MSG::T2;
    const T2* Sp = reinterpret_cast<const T2*>(S) + (size_t)lr * T;
    const T2* Sh = reinterpret_cast<const T2*>(S + pchunk<MSG>()) + (size_t)lr * T;
    float q[4];
    qsrc.template q4<MSG::G>(S, lr, r, lane, it, q);
    bool v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = lane_col<MSG::G>(lane, k);
        v[k] = FULL || (c < cols && (!diag || c > r));
    }
    T2 pw[4], hw[4], nw[4];   // stored words
    float2 pv[4], hv[4];
    if (zero) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { pw[k] = MSG::pack(0.f, 0.f); pv[k] = make_float2(0.f, 0.f); }
    } else {
        MSG::load4(Sp, lane, pw);                               // {P_ij, P_ji}
#pragma unroll
        for (int k = 0; k < 4; ++k) pv[k] = MSG::unpack(pw[k]);
    }
    const float2 rH2 = make_float2(rH, rH);
    if (FROZEN) {
        if (zero_h) {
#pragma unroll
            for (int k = 0; k < 4; ++k) { hw[k] = MSG::pack(0.f, 0.f); hv[k] = make_float2(0.f, 0.f); }
        } else {
            MSG::load4(Sh, lane, hw);                           // {H_ij, H_ji}
            if constexpr (!MSG::MIXED) {
#pragma unroll
                for (int k = 0; k < 4; ++k) hv[k] = MSG::unpack(hw[k]);
            }
        }
        // With P at its fixed point, P_ij = -q^2 / d_i, so the H update
        // -q (htilde_i - H_ji) / d_i equals P_ij (htilde_i - H_ji) / q: one
        // reciprocal per pair, no cavity subtraction (the cavities were
        // checked when these P values were formed).  For |q| below the
        // smallest normal float (q = 0, or an RBF value exp(-gamma d^2) that
        // underflowed to a subnormal) q^2 is 0, so P = 0 and H comes out 0
        // (MSG::qinv keeps the factor finite).
#pragma unroll
        for (int k = 0; k < 4; k += 2) {
            float2 hx, hy;   // new H_ij, H_ji
            if constexpr (MSG::MIXED) {
                // P (H_ji - htilde_i) (-1 / q): the same value, read from the BF16 halves
                const float2 nqi = QN ? make_float2(MSG::qinv_normal(-q[k]), MSG::qinv_normal(-q[k + 1]))
                                      : make_float2(MSG::qinv(-q[k]), MSG::qinv(-q[k + 1]));
                const float2 er = make_float2(MSG::hi_minus(hw[k], rH), MSG::hi_minus(hw[k + 1], rH));
                const float2 ec = make_float2(MSG::lo_minus(hw[k], cv.H[k]), MSG::lo_minus(hw[k + 1], cv.H[k + 1]));
                hx = mul2(mul2(make_float2(pv[k].x, pv[k + 1].x), er), nqi);
                hy = mul2(mul2(make_float2(pv[k].y, pv[k + 1].y), ec), nqi);
            } else {
                const float2 qi = QN ? make_float2(MSG::qinv_normal(q[k]), MSG::qinv_normal(q[k + 1]))
                                     : make_float2(MSG::qinv(q[k]), MSG::qinv(q[k + 1]));
                const float2 dr = sub2(rH2, make_float2(hv[k].y, hv[k + 1].y));              // htilde_i - H_ji
                const float2 dc = sub2(make_float2(cv.H[k], cv.H[k + 1]), make_float2(hv[k].x, hv[k + 1].x));
                hx = mul2(mul2(make_float2(pv[k].x, pv[k + 1].x), dr), qi);
                hy = mul2(mul2(make_float2(pv[k].y, pv[k + 1].y), dc), qi);
            }
            nw[k] = MSG::pack(hx.x, hy.x);
            nw[k + 1] = MSG::pack(hx.y, hy.y);
        }
    } else {
        float2 inv[4];
        {
            T2 npw[4];
            float2 sp = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float di = rP - pv[k].y;        // cavity Ptilde_i - P_ji
                const float dj = cv.P[k] - pv[k].x;   // cavity Ptilde_j - P_ij
                bad |= v[k] & !((di > 0.f) & (dj > 0.f));
                inv[k] = make_float2(rcp_nr(di), rcp_nr(dj));
                const float q2 = q[k] * q[k];
                npw[k] = MSG::pack(-q2 * inv[k].x, -q2 * inv[k].y);
                changed |= v[k] & !MSG::same(npw[k], pw[k]);
            }
            MSG::store4(gp + r * T, lane, npw);
#pragma unroll
            for (int k = 0; k < 4; k += 2) {
                float2 a = MSG::unpack(npw[k]), b = MSG::unpack(npw[k + 1]);
                if (!FULL) {
                    if (!v[k]) a = make_float2(0.f, 0.f);
                    if (!v[k + 1]) b = make_float2(0.f, 0.f);
                }
                sp = add2(sp, make_float2(a.y, b.y));
                const float2 ap = add2(make_float2(cv.aP[k], cv.aP[k + 1]), make_float2(a.x, b.x));
                cv.aP[k] = ap.x; cv.aP[k + 1] = ap.y;
            }
            rs[0] += sp.x + sp.y;
        }
        if (zero || zero_h) {
#pragma unroll
            for (int k = 0; k < 4; ++k) hv[k] = make_float2(0.f, 0.f);
        } else {
            MSG::load4(Sh, lane, hw);                           // {H_ij, H_ji}
#pragma unroll
            for (int k = 0; k < 4; ++k) hv[k] = MSG::unpack(hw[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            nw[k] = MSG::pack(-q[k] * (rH - hv[k].y) * inv[k].x, -q[k] * (cv.H[k] - hv[k].x) * inv[k].y);
    }
    MSG::store4(gh + r * T, lane, nw);
    // sums over the valid pairs: H into the row / column sums, q mu of the
    // other end into the residual sums
    // (slots outside the pair set add zeros; their column aggregates may lie
    // beyond n and are not read)
    float qv[4], mv[4];
    T2 nwv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qv[k] = q[k];
        mv[k] = cv.M[k];
        nwv[k] = nw[k];
        if (!FULL && !v[k]) { nwv[k] = MSG::pack(0.f, 0.f); qv[k] = 0.f; mv[k] = 0.f; }
    }
    const float2 rM2 = make_float2(rM, rM);
    float2 sh = make_float2(0.f, 0.f), sr = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
        const float2 q01 = make_float2(qv[k], qv[k + 1]);
        if constexpr (MSG::MIXED) {
            MSG::add_hi(sh.x, nwv[k]);
            MSG::add_hi(sh.y, nwv[k + 1]);
            MSG::add_lo(cv.aH[k], nwv[k]);
            MSG::add_lo(cv.aH[k + 1], nwv[k + 1]);
        } else {
            const float2 n0 = MSG::unpack(nwv[k]), n1 = MSG::unpack(nwv[k + 1]);
            sh = add2(sh, make_float2(n0.y, n1.y));
            const float2 ah = add2(make_float2(cv.aH[k], cv.aH[k + 1]), make_float2(n0.x, n1.x));
            cv.aH[k] = ah.x; cv.aH[k + 1] = ah.y;
        }
        sr = fma2(q01, make_float2(mv[k], mv[k + 1]), sr);
        const float2 ar = fma2(q01, rM2, make_float2(cv.aR[k], cv.aR[k + 1]));
        cv.aR[k] = ar.x; cv.aR[k + 1] = ar.y;
    }
    rs[1] += sh.x + sh.y;
    rs[2] += sr.x + sr.y;
}

// Per-tile constants of one consumer warp.
// (The rest of the tile's parameters stay in the tile slot, sm.info[slot],
// and are read again where needed, so that they take no registers in the
// pair loop.)
struct TileCtx {
    int cw, lane, rows, cols;
    bool diag;
    int it;
    bool zero, zero_h;
    int slot;   // the tile slot: aggregates sm.agg[slot] (rows 0..2, columns 3..5), parameters sm.info[slot]
};

// One tile's chunk rows for one consumer warp: waits for each ring stage,
// updates its row, releases the stage; leaves the warp's row sums in
// sm.rp/rh/rr and its column partials in sm.cp (not when FROZEN), sm.ch and
// sm.cr.  Specialised per tile kind so that a frozen-P tile keeps neither the
// column P values nor their sums in registers.
template <int CW, bool FULL, bool FROZEN, bool QN, int SB, class MSG, class QSrc>
__device__ __forceinline__ void consume_tile(const QSrc& qsrc, SweepTail<CW>& sm, const unsigned char* ring,
                                             const TileCtx& tc, typename MSG::T2* __restrict__ gp,
                                             typename MSG::T2* __restrict__ gh, int& stage, uint32_t& phase,
                                             bool& abort, bool& bad, bool& changed)
{
    const int cw = tc.cw, lane = tc.lane, rows = tc.rows;
    constexpr int G = MSG::G;
    const float (*ag)[T] = sm.agg[tc.slot];
    ColVals cv;
    ld4<G>(ag[4], lane, cv.H);
    ld4<G>(ag[5], lane, cv.M);
    if (!FROZEN) ld4<G>(ag[3], lane, cv.P);
#pragma unroll
    for (int k = 0; k < 4; ++k) cv.aP[k] = cv.aH[k] = cv.aR[k] = 0.f;
    // A group of SPC consecutive ring stages (RPS rows of each per warp) is
    // reduced together: RPW = SPC * RPS rows of the warp, cw + CW u.
    constexpr int RC = rc<MSG>(), SPC = MSG::SPC, RPS = RC / CW, RPW = SPC * RPS;
    static_assert(RPS * CW == RC && (RPW == 1 || RPW == 2 || RPW == 4), "1, 2 or 4 rows per consumer warp and group");
    const int nst = (rows + RC - 1) / RC;   // ring stages of this tile
#pragma unroll 1
    for (int ch = 0; ch < nst; ch += SPC) {
        float rs[RPW][3];
#pragma unroll
        for (int g = 0; g < SPC; ++g) {
#pragma unroll
            for (int u = 0; u < RPS; ++u) rs[g * RPS + u][0] = rs[g * RPS + u][1] = rs[g * RPS + u][2] = 0.f;
            if (SPC > 1 && ch + g >= nst) continue;   // a tile with an odd number of stages
            if (!abort && !mbar_wait_warp(&sm.full[stage], phase)) {
                abort = true;
                if (lane == 0) record_error(sm.info[tc.slot].ctrl, ST_ETIMEOUT, sm.info[tc.slot].L);
            }
            if (!abort) {
                const unsigned char* S = ring + (size_t)stage * SB;
#pragma unroll
                for (int u = 0; u < RPS; ++u) {
                    const int lr = cw + CW * u, r = (ch + g) * RC + lr;
                    if (FULL || r < rows)
                        update_row<FULL, FROZEN, QN, MSG>(qsrc, S, lr, lane, r, tc.cols, tc.diag, tc.it, tc.zero,
                                                      tc.zero_h, ag[0][r], ag[1][r], ag[2][r], cv, gp, gh,
                                                      rs[g * RPS + u], bad, changed);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
            if (++stage == stages<MSG>()) { stage = 0; phase ^= 1u; }
        }
        // row sums {P, H, R} of the warp's rows over the warp; group row u is
        // tile row ch RC + cw + CW u
        const int r0 = ch * RC + cw;
        if constexpr (RPW == 4 && FROZEN) {
            // the P sums of a frozen round are not needed
            const float x[8] = {rs[0][1], rs[0][2], rs[1][1], rs[1][2], rs[2][1], rs[2][2], rs[3][1], rs[3][2]};
            const float v = reduce_scatter8x(x, lane);
            const int qi = (lane >> 2) & 7, r = r0 + CW * (qi >> 1);
            if ((lane & 3) == 0 && r < rows) ((qi & 1) ? sm.rr : sm.rh)[r] = v;
        } else if constexpr (RPW == 4) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float v = reduce_scatter8(rs[2 * h][0], rs[2 * h][1], rs[2 * h][2], rs[2 * h + 1][0],
                                                rs[2 * h + 1][1], rs[2 * h + 1][2], lane);
                const int qi = (lane >> 2) & 7, qv = qi & 3, r = r0 + CW * (2 * h + (qi >> 2));
                if ((lane & 3) == 0 && qv < 3 && r < rows) (qv == 0 ? sm.rp : (qv == 1 ? sm.rh : sm.rr))[r] = v;
            }
        } else if constexpr (RPW == 2 && FROZEN) {
            const float v = reduce_scatter4(rs[0][1], rs[0][2], rs[1][1], rs[1][2], lane);
            const int qi = (lane >> 3) & 3, r = r0 + CW * (qi >> 1);
            if ((lane & 7) == 0 && r < rows) ((qi & 1) ? sm.rr : sm.rh)[r] = v;
        } else if constexpr (RPW == 2) {
            const float v = reduce_scatter8(rs[0][0], rs[0][1], rs[0][2], rs[1][0], rs[1][1], rs[1][2], lane);
            const int qi = (lane >> 2) & 7, qv = qi & 3, r = r0 + CW * (qi >> 2);
            if ((lane & 3) == 0 && qv < 3 && r < rows) (qv == 0 ? sm.rp : (qv == 1 ? sm.rh : sm.rr))[r] = v;
        } else {
            const float v = reduce_scatter4(rs[0][0], rs[0][1], rs[0][2], 0.f, lane);
            const int qv = (lane >> 3) & 3;
            if ((lane & 7) == 0 && qv < 3 && r0 < rows) (qv == 0 ? sm.rp : (qv == 1 ? sm.rh : sm.rr))[r0] = v;
        }
    }
    if (!FROZEN) st4<G>(sm.cp[cw], lane, cv.aP);
    st4<G>(sm.ch[cw], lane, cv.aH);
    st4<G>(sm.cr[cw], lane, cv.aR);
}

// Consumers (256 threads, ctid = 0..255, consumer warp cw = ctid / 32).
// QSrc supplies q for a pair and the per-tile hand-shake of a recomputed Q tile.
template <int CW, size_t SB, class MSG, class QSrc>
__device__ __forceinline__ void sweep_consumers(const Inst* __restrict__ tab, const int4* __restrict__ work,
                                                long long ntiles, SweepTail<CW>& sm, const unsigned char* ring,
                                                int ctid, QSrc& qsrc)
{
    const int cw = ctid >> 5, lane = ctid & 31;
    int stage = 0;
    uint32_t phase = 0;
    bool abort = false;
    int it = 0, slot = 0;
    uint32_t tph = 0;
    for (;;) {
        // next tile from the producer (bounded wait; the stop is taken by all
        // consumer warps together at the tile barrier)
        if (!mbar_wait_warp(&sm.tfull[slot], tph) && lane == 0) {
            sm.cabort = 1;
            if (blockIdx.x < ntiles) record_error(tab[work[blockIdx.x].x].ctrl, ST_ETIMEOUT, -1);
        }
        consumer_bar<CW>();   // also: the previous tile's sums are read out
        if (*(volatile int*)&sm.cabort) break;
        if (sm.info[slot].end) break;
        bool changed = false, bad = false;
        TileCtx tc;
        typename MSG::T2 *gp, *gh;
        bool full, frozen, qnormal;
        {
            const TileInfo& ti = sm.info[slot];
            const int n = ti.n, I = ti.I, J = ti.J;
            tc.cw = cw;
            tc.lane = lane;
            tc.rows = min(T, n - I * T);
            tc.cols = min(T, n - J * T);
            tc.diag = (I == J);
            tc.it = it;
            tc.zero = (ti.t == 0);   // Step 1: all messages 0, nothing to read
            tc.zero_h = ti.zero_h != 0;
            tc.slot = slot;
            full = !tc.diag && tc.cols == T;
            frozen = ti.frozen != 0;
            qnormal = ti.qnormal != 0;
            gp = static_cast<typename MSG::T2*>(ti.Pst);
            gh = static_cast<typename MSG::T2*>(ti.Hst);
        }
        if (!abort && !qsrc.tile_begin(it, lane)) {
            abort = true;
            if (lane == 0) record_error(sm.info[slot].ctrl, ST_ETIMEOUT, sm.info[slot].L);
        }
        if (full) {
            if (frozen && qnormal)
                consume_tile<CW, true, true, true, SB, MSG>(qsrc, sm, ring, tc, gp, gh, stage, phase, abort, bad, changed);
            else if (frozen)
                consume_tile<CW, true, true, false, SB, MSG>(qsrc, sm, ring, tc, gp, gh, stage, phase, abort, bad, changed);
            else consume_tile<CW, true, false, false, SB, MSG>(qsrc, sm, ring, tc, gp, gh, stage, phase, abort, bad, changed);
        } else {
            if (frozen) consume_tile<CW, false, true, false, SB, MSG>(qsrc, sm, ring, tc, gp, gh, stage, phase, abort, bad, changed);
            else consume_tile<CW, false, false, false, SB, MSG>(qsrc, sm, ring, tc, gp, gh, stage, phase, abort, bad, changed);
        }
        // the tile's remaining parameters, read before the slot is released
        const TileInfo ti = sm.info[slot];
        Ctrl* ctrl = ti.ctrl;
        const int I = ti.I;
        const int rows = tc.rows, cols = tc.cols;
        const bool diag = tc.diag;
        frozen = ti.frozen != 0;
        float* partP = ti.part;
        float* partH = partP + ti.plen;
        float* partR = partH + ti.plen;
        const size_t oR = (size_t)ti.sR * T, oC = (size_t)ti.sC * T;
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.tempty[slot]);   // tile slot free for the producer
        if (++slot == 2) { slot = 0; tph ^= 1u; }
        __syncwarp();
        qsrc.tile_end(it, lane);
        consumer_bar<CW>();
        // With frozen P the P sums are unchanged from the previous round and
        // the finalize keeps Ptilde; the P slots are not written.
        if (diag) {
            if (ctid < rows) {
                float P = sm.rp[ctid], H = sm.rh[ctid], R = sm.rr[ctid];
#pragma unroll
                for (int w = 0; w < CW; ++w) { P += sm.cp[w][ctid]; H += sm.ch[w][ctid]; R += sm.cr[w][ctid]; }
                const size_t o = oR + ctid;
                if (!frozen) partP[o] = P;
                partH[o] = H; partR[o] = R;
            }
        } else if (ctid < T) {
            if (ctid < rows) {
                const size_t o = oR + ctid;
                if (!frozen) partP[o] = sm.rp[ctid];
                partH[o] = sm.rh[ctid]; partR[o] = sm.rr[ctid];
            }
        } else {
            const int c = ctid - T;
            if (c < cols) {
                float P = 0.f, H = 0.f, R = 0.f;
#pragma unroll
                for (int w = 0; w < CW; ++w) { P += sm.cp[w][c]; H += sm.ch[w][c]; R += sm.cr[w][c]; }
                const size_t o = oC + c;
                if (!frozen) partP[o] = P;
                partH[o] = H; partR[o] = R;
            }
        }
        if (bad) record_error(ctrl, ST_ENUMERIC, (long long)I * T);
        // P fixed-point detection: one flag per instance and round
        if (__any_sync(0xffffffffu, changed) && lane == 0 && !*(volatile int*)&ctrl->p_changed)
            atomicExch(&ctrl->p_changed, 1);
        ++it;
    }
}

// Q streamed with the messages: it sits after the messages in each ring stage.
template <typename QT, class MSG>
struct StoredQ {
    __device__ __forceinline__ bool tile_begin(int, int) { return true; }
    __device__ __forceinline__ void tile_end(int, int) {}
    // q of the lane's four pairs of chunk row cw
    template <int G>
    __device__ __forceinline__ void q4(const unsigned char* S, int cw, int, int lane, int, float (&q)[4]) const
    {
        ld4<G>(reinterpret_cast<const QT*>(S + state_chunk<MSG>()) + (size_t)cw * T, lane, q);
    }
};

template <typename QT, class MSG>
__global__ void __launch_bounds__(SWEEP_THREADS, sweep_ctas<MSG>())
    k_sweep(const Inst* __restrict__ tab, const int4* __restrict__ work, const Sched* __restrict__ sched, int stage_no)
{
    const long long ntiles = sched->ntiles;
    work += sched->off;
    constexpr size_t SB = stage_bytes<QT, MSG>();

    extern __shared__ unsigned char smem_raw[];
    unsigned char* ring = align_smem(smem_raw, 128);
    SweepTail<NWARPS>& sm = *reinterpret_cast<SweepTail<NWARPS>*>(ring + stages<MSG>() * SB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        init_tail(sm);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == NWARPS) {
        sweep_producer<QT, MSG, SB>(tab, work, ntiles, sm, ring, nullptr, lane, stage_no);
        return;
    }
    StoredQ<QT, MSG> qsrc;
    sweep_consumers<NWARPS, SB, MSG>(tab, work, ntiles, sm, ring, tid, qsrc);
}

// ---- fused recompute ------------------------------------------------------
constexpr int RC_XSTAGES = 2;
// Consumer warps (two rows of each 16-row stage each).  Sixteen consumers
// (one row each, 88 registers a thread) measured slower with an earlier
// consumer (0.71 / 0.51 of the copy peak against 0.77 / 0.53 with eight).
// Eight also keep the summation order of the stored-Q sweep, so recomputed
// and stored forms agree bitwise.
constexpr int RC_CW = 8;
constexpr int RC_THREADS = (7 + RC_CW) * 32;   // 3 role warps + 4 epilogue + 8 consumers
constexpr uint32_t RC_TMEM_COLS = 256;
constexpr size_t RC_QTILE = (size_t)TT * sizeof(__nv_bfloat16);   // 32 KB

struct RcExtra {
    unsigned long long xfull[RC_XSTAGES], xempty[RC_XSTAGES];
    unsigned long long accfull[2], accempty[2];
    unsigned long long qfull[2], qempty[2];
    unsigned long long drain;
    uint32_t tmem_base;
    int abort;
    ColTile cols[4];    // column constants of the current tile, one set per epilogue warp
};

template <class MSG>
__host__ __device__ constexpr size_t rc_smem_bytes()
{
    return 1024 + stages<MSG>() * state_chunk<MSG>() + RC_XSTAGES * 2 * BLK_BYTES + 2 * RC_QTILE + sizeof(SweepTail<RC_CW>) +
           sizeof(RcExtra);
}

// Q from the shared-memory tile written by the epilogue warps.
struct RecomputedQ {
    const __nv_bfloat16* qtile;   // [2][T][T]
    RcExtra* ex;
    __device__ __forceinline__ bool tile_begin(int it, int)
    {
        return mbar_wait_warp(&ex->qfull[it & 1], (uint32_t)((it >> 1) & 1));
    }
    __device__ __forceinline__ void tile_end(int it, int lane)
    {
        if (lane == 0) mbar_arrive(&ex->qempty[it & 1]);
    }
    // The tile's rows are stored with their 16-byte chunks permuted: chunk c
    // of row r sits at chunk c ^ (r % 8), so that the epilogue's stores (one
    // row per lane, the same chunk) spread over all banks; a consumer warp
    // still reads one row's 256 contiguous bytes.
    template <int G>
    __device__ __forceinline__ void q4(const unsigned char*, int, int r, int lane, int it, float (&q)[4]) const
    {
        const unsigned char* row = reinterpret_cast<const unsigned char*>(qtile + (size_t)(it & 1) * TT + (size_t)r * T);
        const int sw = r & 7;
        if constexpr (G == 4) {
            const uint2 u = *reinterpret_cast<const uint2*>(row + (((lane >> 1) ^ sw) << 4) + ((lane & 1) << 3));
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
            q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
        } else {
            const int o = ((lane >> 2) ^ sw) << 4 | ((lane & 3) << 2);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + o));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + 128 + o));
            q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
        }
    }
};

template <class MSG>
__global__ void __launch_bounds__(RC_THREADS, 1)
    k_sweep_rc(const Inst* __restrict__ tab, const int4* __restrict__ work, const Sched* __restrict__ sched,
               int stage_no)
{
    const long long ntiles = sched->ntiles;
    work += sched->off;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* ring = align_smem(smem_raw, 1024);
    unsigned char* xops = ring + stages<MSG>() * state_chunk<MSG>();                // [2][A, B]
    __nv_bfloat16* qtile = reinterpret_cast<__nv_bfloat16*>(xops + RC_XSTAGES * 2 * BLK_BYTES);
    SweepTail<RC_CW>& sm = *reinterpret_cast<SweepTail<RC_CW>*>(reinterpret_cast<unsigned char*>(qtile) + 2 * RC_QTILE);
    RcExtra& ex = *reinterpret_cast<RcExtra*>(reinterpret_cast<unsigned char*>(&sm) + sizeof(SweepTail<RC_CW>));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        init_tail(sm);
        for (int s = 0; s < RC_XSTAGES; ++s) { mbar_init(&ex.xfull[s], 1); mbar_init(&ex.xempty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ex.accfull[b], 1);
            mbar_init(&ex.accempty[b], 4);
            mbar_init(&ex.qfull[b], 4);
            mbar_init(&ex.qempty[b], RC_CW);
        }
        mbar_init(&ex.drain, 1);
        ex.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) tmem_alloc(&ex.tmem_base, RC_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = ex.tmem_base;
    volatile int* abort_flag = &ex.abort;

    if (warp == 0) {
        sweep_producer<void, MSG, state_chunk<MSG>()>(tab, work, ntiles, sm, ring, abort_flag, lane, stage_no);
    } else if (warp == 1) {
        // feature blocks of each tile
        if (lane == 0) {
            const uint64_t pol = l2_evict_first_policy();
            int xs = 0;
            uint32_t ph = 0;
            bool run = true;
            for (long long L = blockIdx.x; L < ntiles && run; L += gridDim.x) {
                const int4 w = work[L];
                const Inst& p = tab[w.x];
                Ctrl* ctrl = p.ctrl;
                if (*(volatile const int*)&ctrl->done) continue;
                const unsigned char* Xp = static_cast<const unsigned char*>(p.Xp);
                const int I = w.y, J = w.z, nkc = p.nkc;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*abort_flag || !mbar_wait(&ex.xempty[xs], ph ^ 1u)) {
                        *abort_flag = 1;
                        record_error(ctrl, ST_ETIMEOUT, L);
                        run = false;
                        break;
                    }
                    unsigned char* A = xops + (size_t)xs * 2 * BLK_BYTES;
                    mbar_arrive_expect_tx(&ex.xfull[xs], 2 * BLK_BYTES);
                    bulk_load(A, Xp + ((size_t)I * nkc + kc) * BLK_BYTES, BLK_BYTES, &ex.xfull[xs], pol);
                    bulk_load(A + BLK_BYTES, Xp + ((size_t)J * nkc + kc) * BLK_BYTES, BLK_BYTES, &ex.xfull[xs], pol);
                    if (++xs == RC_XSTAGES) { xs = 0; ph ^= 1u; }
                }
            }
        }
    } else if (warp == 2) {
        // MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(T, T);
            int xs = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
                const Inst& p = tab[work[L].x];
                Ctrl* ctrl = p.ctrl;
                if (*(volatile const int*)&ctrl->done) continue;
                const int nkc = p.nkc;
                if (*abort_flag || !mbar_wait(&ex.accempty[acc], aph ^ 1u)) {
                    *abort_flag = 1;
                    record_error(ctrl, ST_ETIMEOUT, L);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tbase + (uint32_t)acc * T;
                bool ok = true;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*abort_flag || !mbar_wait(&ex.xfull[xs], ph)) {
                        *abort_flag = 1;
                        record_error(ctrl, ST_ETIMEOUT, L);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* A = xops + (size_t)xs * 2 * BLK_BYTES;
#pragma unroll
                    for (int s = 0; s < KCH / 16; ++s) {
                        const uint64_t ad = smem_desc(A + s * 256, 128, 1024);
                        const uint64_t bd = smem_desc(A + BLK_BYTES + s * 256, 128, 1024);
                        tc_mma_bf16(d, ad, bd, IDESC, (kc | s) != 0);
                    }
                    tc_commit(&ex.xempty[xs]);
                    if (++xs == RC_XSTAGES) { xs = 0; ph ^= 1u; }
                }
                if (!ok) break;
                tc_commit(&ex.accfull[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1u; }
            }
            tc_commit(&ex.drain);
            if (!mbar_wait(&ex.drain, 0u)) *abort_flag = 1;
        }
    } else if (warp < 7) {
        // epilogue: TMEM rows -> BF16 Q tile in shared memory
        const int g = warp & 3, r = 32 * g + lane;
        int it = 0;
        for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
            const int4 w = work[L];
            const Inst& p = tab[w.x];
            Ctrl* ctrl = p.ctrl;
            if (*(volatile const int*)&ctrl->done) continue;
            const int n = p.n;
            const int acc = it & 1;
            const uint32_t par = (uint32_t)((it >> 1) & 1);
            const bool stop = __shfl_sync(0xffffffffu, *abort_flag, 0) != 0;
            if (stop || !mbar_wait_warp(&ex.accfull[acc], par) || !mbar_wait_warp(&ex.qempty[acc], par ^ 1u)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    record_error(ctrl, ST_ETIMEOUT, L);
                }
                break;
            }
            tc_fence_after();
            const int I = w.y, J = w.z, i = I * T + r;
            const float* y = p.y;
            const float* sqb = p.sqb;
            const float gamma = p.gamma, lam2 = p.lam2;
            const float yi = i < n ? y[i] : 0.f, si = i < n ? sqb[i] : 0.f;
            stage_tile_cols(ex.cols[g], y, sqb, n, J, gamma, lane, 0, T / 32);
            const float ai = -gamma * kLog2e * si, c2 = 2.f * gamma * kLog2e;
            const uint32_t s1 = __float_as_uint(yi) & 0x80000000u, si2 = s1 | (s1 >> 16);
            uint4* qrow = reinterpret_cast<uint4*>(qtile + (size_t)acc * TT + (size_t)r * T);   // 16 chunks
            const int sw = r & 7;   // chunk c stored at c ^ sw (see RecomputedQ)
#pragma unroll 1
            for (int cc = 0; cc < T / 32; ++cc) {
                const uint32_t valid = chunk_valid(n, I, J, r, cc);
                float v[32];
                tmem_ld32(tbase + (uint32_t)acc * T + ((uint32_t)(32 * g) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float vh[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) vh[u] = v[16 * h + u];
                    uint4 out[2];
                    q_half_bf16(vh, 32 * cc + 16 * h, ai, si2, ex.cols[g], c2, lam2, (valid >> (16 * h)) & 0xffffu, out);
                    qrow[(4 * cc + 2 * h) ^ sw] = out[0];
                    qrow[(4 * cc + 2 * h + 1) ^ sw] = out[1];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&ex.accempty[acc]);
                mbar_arrive(&ex.qfull[acc]);
            }
            ++it;
        }
    } else {
        RecomputedQ qsrc{qtile, &ex};
        sweep_consumers<RC_CW, state_chunk<MSG>(), MSG>(tab, work, ntiles, sm, ring, tid - 7 * 32, qsrc);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tbase, RC_TMEM_COLS);
    }
}

// Compensated FP32 accumulation (Knuth's TwoSum): s + c carries the running
// sum with an error term, so sums of a few hundred FP32 partials keep close to
// 48 bits without using the (slow) FP64 pipe.
__device__ __forceinline__ void acc2(float& s, float& c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// Node x's next aggregates {Ptilde, htilde, mutilde} from its slot sums (P,
// H) and its residual r_x(t) = b_x - Q_xx mutilde_x(t) - R in FP64; returns
// |r_x| (inf for a non-finite one) and flags a non-positive or non-finite
// aggregate.
__device__ __forceinline__ double finalize_node(const Inst& p, Ctrl* ctrl, int x, int t, bool frozen, double P,
                                                double H, double R)
{
    const float* cur = p.agg + (size_t)(t & 1) * 3 * p.npad;
    float* nxt = p.agg + (size_t)((t + 1) & 1) * 3 * p.npad;
    const double qd = p.qdiag[x], bx = p.b[x];
    const float Pn = frozen ? cur[x] : (float)(qd + P);
    const float hn = (float)(bx + H);
    const float mn = hn / Pn;
    nxt[x] = Pn;
    nxt[p.npad + x] = hn;
    nxt[2 * p.npad + x] = mn;
    const double r = bx - qd * (double)cur[2 * p.npad + x] - R;
    double absr = fabs(r);
    if (!(absr <= DBL_MAX)) absr = INFINITY;
    if (!(Pn > 0.f) || !isfinite(Pn) || !isfinite(mn)) record_error(ctrl, ST_ENUMERIC, x);
    return absr;
}

// Run by the last node block of an instance to finish a round: ||r(t)||_inf,
// the stop test (Step 3: k* = t when it is below tol, the limit otherwise),
// the exact P-freeze flag, and the round counter.
__device__ __forceinline__ void finalize_decide(const Inst& p, Ctrl* ctrl, int t)
{
    __threadfence();
    const double rmax = __longlong_as_double((long long)atomicAdd(&ctrl->rmax_bits, 0ull));
    const int status = atomicAdd(&ctrl->status, 0);
    if (p.rhist && t < p.rhist_cap) p.rhist[t] = rmax;
    if (status != 0) {
        ctrl->done = 1;
        ctrl->kstar = t;
        ctrl->rinf = rmax;
    } else if (rmax < ctrl->tol) {
        ctrl->done = 1;
        ctrl->kstar = t;
        ctrl->converged = 1;
        ctrl->rinf = rmax;
    } else if (t + 1 >= ctrl->limit) {
        ctrl->done = 1;
        ctrl->kstar = t + 1;
    }
    // No P message changed in this round: P is at its floating-point fixed
    // point (its recursion does not involve b or H), so later rounds would
    // rewrite the same values; they stop writing them.
    if (!ctrl->p_frozen && t > 0 && atomicAdd(&ctrl->p_changed, 0) == 0) {
        ctrl->p_frozen = 1;
        ctrl->t_frozen = t + 1;
    }
    ctrl->p_changed = 0;
    ctrl->t = t + 1;
    ctrl->zero_h = 0;
    ctrl->rmax_bits = 0ull;
    ctrl->blocks_done = 0u;
    __threadfence();
}

// Compensated sums of node x's slots k = k0, k0 + step, ... (of the
// slot_count of its block) of NA partial arrays (P, H[, R]), eight loads of
// each in flight; P reads as 0 when frozen (Ptilde is kept then).
template <int NA>
__device__ __forceinline__ void slot_sums(const Inst& p, int x, int k0, int step, bool frozen, float (&s)[NA],
                                          float (&c)[NA])
{
    const int X = x / T, ns = slot_count(p, X);
    const size_t len = part_len(p);
    const float* part = p.part + (size_t)slot_begin(p, X) * T + (x - X * T);
#pragma unroll
    for (int a = 0; a < NA; ++a) s[a] = c[a] = 0.f;
    int k = k0;
    for (; k + 7 * step < ns; k += 8 * step) {
        float v[NA][8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const size_t o = a * len + (size_t)(k + u * step) * T;
                v[a][u] = (a == 0 && frozen) ? 0.f : part[o];
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int a = 0; a < NA; ++a) acc2(s[a], c[a], v[a][u]);
    }
    for (; k < ns; k += step)
#pragma unroll
        for (int a = 0; a < NA; ++a) acc2(s[a], c[a], (a == 0 && frozen) ? 0.f : part[a * len + (size_t)k * T]);
}

// Node-block units of a round's finalize.  Blocks [0, nsmall) of the list
// belong to instances with at most kWarpFinNt tile rows and are finalized one
// warp per block, eight blocks per unit; the others take a whole CTA each
// (eight warps over the slots, then one reduction).  An instance's blocks all
// take the same mode, so its arithmetic does not depend on the other
// instances of the list.
__device__ __forceinline__ int fin_units(const Sched* sc, int& usmall)
{
    usmall = (sc->nsmall + 7) / 8;
    return usmall + (sc->nblocks - sc->nsmall);
}

// Per node x: compensated sums of its slots, next aggregates, residual
// r_x(t) in FP64, max |r| -> ctrl; the last node block of an instance to
// finish decides.  Five CTAs per SM (48 registers a thread), so that one
// CTA per 32-node block of n = 20000 (625) runs in a single wave.
__global__ void __launch_bounds__(256, 5)
    k_finalize(const Inst* __restrict__ tab, const int2* __restrict__ nbl, const Sched* __restrict__ sched)
{
    int usmall;
    const int units = fin_units(sched, usmall), nsmall = sched->nsmall;
    __shared__ float red[6][8][32];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        if (u < usmall) {
            // ---- one warp per node block
            const int bi = 8 * u + g;
            if (bi >= nsmall) continue;
            const int2 nb = nbl[bi];
            const Inst& p = tab[nb.x];
            Ctrl* ctrl = p.ctrl;
            if (*(volatile int*)&ctrl->done) continue;
            const int t = *(volatile int*)&ctrl->t;
            const bool frozen = *(volatile int*)&ctrl->p_frozen != 0;
            const int x = nb.y * 32 + lane, n = p.n;
            double absr = 0.0;
            if (x < n) {
                float sv[3], cv[3];
                slot_sums<3>(p, x, 0, 1, frozen, sv, cv);
                absr = finalize_node(p, ctrl, x, t, frozen, (double)sv[0] + (double)cv[0],
                                     (double)sv[1] + (double)cv[1], (double)sv[2] + (double)cv[2]);
            }
            absr = warp_max_d(absr);
            if (lane == 0) atomicMax(&ctrl->rmax_bits, (unsigned long long)__double_as_longlong(absr));
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
                if (prev == (unsigned)((n + 31) / 32 - 1)) finalize_decide(p, ctrl, t);
            }
            continue;
        }
        // ---- one CTA per node block: warp g sums slots g, g + 8, ...
        const int2 nb = nbl[nsmall + (u - usmall)];
        const Inst& p = tab[nb.x];
        Ctrl* ctrl = p.ctrl;
        if (*(volatile int*)&ctrl->done) continue;
        const int t = *(volatile int*)&ctrl->t;
        const bool frozen = *(volatile int*)&ctrl->p_frozen != 0;
        const int x = nb.y * 32 + lane, n = p.n;
        float sv[3] = {0.f, 0.f, 0.f}, cv[3] = {0.f, 0.f, 0.f};
        if (x < n) slot_sums<3>(p, x, g, 8, frozen, sv, cv);
        __syncthreads();   // red[] of the previous node block is consumed
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            red[2 * a][g][lane] = sv[a];
            red[2 * a + 1][g][lane] = cv[a];
        }
        __syncthreads();
        if (g == 0) {
            double absr = 0.0;
            if (x < n) {
                float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    acc2(a[0], a[1], red[0][w][lane]); a[1] += red[1][w][lane];
                    acc2(a[2], a[3], red[2][w][lane]); a[3] += red[3][w][lane];
                    acc2(a[4], a[5], red[4][w][lane]); a[5] += red[5][w][lane];
                }
                absr = finalize_node(p, ctrl, x, t, frozen, (double)a[0] + (double)a[1], (double)a[2] + (double)a[3],
                                     (double)a[4] + (double)a[5]);
            }
            absr = warp_max_d(absr);
            if (lane == 0)
                atomicMax(&ctrl->rmax_bits, (unsigned long long)__double_as_longlong(absr));
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
            s_last = (prev == (unsigned)((n + 31) / 32 - 1));
        }
        __syncthreads();
        if (s_last && tid == 0) finalize_decide(p, ctrl, t);
    }
}

// Node x's P and residual (when `with_p`) and H slot partials := 0, the sums
// of all-zero messages: the staged schedule's stage finalize reads the slots
// of tiles not yet swept in a round, and under the tile-sparse option the
// slots of dropped tiles are never written by a sweep.
__device__ __forceinline__ void zero_slots(const Inst& p, int x, bool with_p)
{
    const int X = x / T, ns = slot_count(p, X);
    const size_t len = part_len(p);
    float* partP = p.part + (size_t)slot_begin(p, X) * T + (x - X * T);
    float* partH = partP + len;
    float* partR = partH + len;
    for (int k = 0; k < ns; ++k) {
        if (with_p) {
            partP[(size_t)k * T] = 0.f;
            partR[(size_t)k * T] = 0.f;
        }
        partH[(size_t)k * T] = 0.f;
    }
}

// The whole matrix's sum_{j != i} |Q_ij| of node x: the formation's slot sums
// (array 0) added in fixed point (rsum_fix), or the first pass's sums of the
// tile-sparse option (the same value).
__device__ __forceinline__ double offdiag_abs_sum(const Inst& p, int x)
{
    if (p.rsum) return p.rsum[x];
    const int X = x / T, ns = slot_count(p, X), sh = rsum_shift(p.n, p.lam2);
    const double scale = pow2i(sh);
    const float* s0 = p.part + (size_t)slot_begin(p, X) * T + (x - X * T);
    long long a = 0;
    for (int k = 0; k < ns; ++k) a += rsum_fix(s0[(size_t)k * T], scale);
    return rsum_unfix(a, sh);
}

// Between the stages of a staged round: Ptilde and htilde of every node from
// all of its slot partials (slots of tiles not yet swept in this round still
// hold the sums of their current messages) into aggmid, for the next stage;
// with frozen P, Ptilde is kept.  No residual and no stop test: those come
// with the round's last stage (k_finalize).  Same node-block units as
// k_finalize.
__device__ __forceinline__ void stage_node(const Inst& p, int x, int t, bool frozen, double P, double H)
{
    const float* cur = p.agg + (size_t)(t & 1) * 3 * p.npad;
    p.aggmid[x] = frozen ? cur[x] : (float)((double)p.qdiag[x] + P);
    p.aggmid[p.npad + x] = (float)((double)p.b[x] + H);
}

__global__ void __launch_bounds__(256)
    k_finalize_stage(const Inst* __restrict__ tab, const int2* __restrict__ nbl, const Sched* __restrict__ sched)
{
    int usmall;
    const int units = fin_units(sched, usmall), nsmall = sched->nsmall;
    __shared__ float red[4][8][32];
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        if (u < usmall) {
            const int bi = 8 * u + g;
            if (bi >= nsmall) continue;
            const int2 nb = nbl[bi];
            const Inst& p = tab[nb.x];
            if (*(volatile int*)&p.ctrl->done) continue;
            const int t = *(volatile int*)&p.ctrl->t;
            const bool frozen = *(volatile int*)&p.ctrl->p_frozen != 0;
            const int x = nb.y * 32 + lane;
            if (x < p.n) {
                float sv[2], cv[2];
                slot_sums<2>(p, x, 0, 1, frozen, sv, cv);
                stage_node(p, x, t, frozen, (double)sv[0] + (double)cv[0], (double)sv[1] + (double)cv[1]);
            }
            continue;
        }
        const int2 nb = nbl[nsmall + (u - usmall)];
        const Inst& p = tab[nb.x];
        Ctrl* ctrl = p.ctrl;
        if (*(volatile int*)&ctrl->done) continue;   // the same node block for the whole CTA
        const int t = *(volatile int*)&ctrl->t;
        const bool frozen = *(volatile int*)&ctrl->p_frozen != 0;
        const int x = nb.y * 32 + lane, n = p.n;
        float sv[2] = {0.f, 0.f}, cv[2] = {0.f, 0.f};
        if (x < n) slot_sums<2>(p, x, g, 8, frozen, sv, cv);
        __syncthreads();   // red[] of the previous node block is consumed
        red[0][g][lane] = sv[0]; red[1][g][lane] = cv[0];
        red[2][g][lane] = sv[1]; red[3][g][lane] = cv[1];
        __syncthreads();
        if (g == 0 && x < n) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                acc2(a[0], a[1], red[0][w][lane]); a[1] += red[1][w][lane];
                acc2(a[2], a[3], red[2][w][lane]); a[3] += red[3][w][lane];
            }
            stage_node(p, x, t, frozen, (double)a[0] + (double)a[1], (double)a[2] + (double)a[3]);
        }
    }
}

__global__ void k_reset(Inst p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl* c = p.ctrl;
        c->t = 0;
        c->zero_h = 0;
        c->p_frozen = 0;
        c->p_changed = 0;
        c->done = 1;
        c->kstar = 0;
        c->converged = 0;
        c->rmax_bits = 0ull;
        c->blocks_done = 0u;
    }
    if (x >= p.n) return;
    zero_slots(p, x, true);
    const float qd = p.qdiag[x], bx = p.b0[x];
    const_cast<float*>(p.b)[x] = bx;
    p.agg[x] = qd;
    p.agg[p.npad + x] = bx;
    p.agg[2 * p.npad + x] = bx / qd;
}

// Correction system Q d = r with the current P messages: b := r, the H
// messages restart from 0, so htilde = b and mutilde = b / Ptilde.  Over a
// list of node blocks; block 0 of an instance flags the H restart.
__global__ void k_refine_rhs_list(const Inst* __restrict__ tab, const StopOp* __restrict__ ops,
                                  const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    Ctrl* c = p.ctrl;
    const int t = *(volatile int*)&c->t;
    const int x = nb.y * 32 + threadIdx.x;
    if (nb.y == 0 && threadIdx.x == 0) c->zero_h = 1;
    if (threadIdx.x >= 32 || x >= p.n) return;
    zero_slots(p, x, false);   // the H messages restart from 0
    float* cur = p.agg + (size_t)(t & 1) * 3 * p.npad;
    const float bx = ops[nb.x].r_out[x];
    const_cast<float*>(p.b)[x] = bx;
    cur[p.npad + x] = bx;
    cur[2 * p.npad + x] = bx / cur[x];
}

// acc = mutilde(buf) (first pass) or acc += mutilde(buf), over node blocks.
__global__ void k_axpy_list(const Inst* __restrict__ tab, const StopOp* __restrict__ ops,
                            const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    const StopOp& op = ops[nb.x];
    const int x = nb.y * 32 + threadIdx.x;
    if (threadIdx.x >= 32 || x >= p.n || !op.acc) return;
    const float m = p.agg[(size_t)(op.axpy_buf & 1) * 3 * p.npad + 2 * (size_t)p.npad + x];
    op.acc[x] = op.axpy_first ? m : op.acc[x] + m;
}

// Failure-detection self test: one thread waits, with the same bounded wait
// the sweep uses, on an mbarrier that nothing ever arrives on, and reports
// ST_ETIMEOUT when the limit runs out (the kernel then returns normally).
__global__ void k_selftest_wait(unsigned long long limit_ns, int* status)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *status = mbar_wait(&bar, 0u, limit_ns) ? (int)ST_OK : (int)ST_ETIMEOUT;
    }
}

// Reciprocal self test: out[i] = rcp_nr(d[i]).
__global__ void k_selftest_rcp(const float* __restrict__ d, float* __restrict__ out, int cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) out[i] = rcp_nr(d[i]);
}

// Row x's diagonal margin Q_xx - R_x into the instance's running
// max_i 1 / (Q_ii - R_i) (the control block is zeroed before formation):
// with all margins positive Q is strictly diagonally dominant and Varah's
// bound ||mu - Q^-1 b||_inf <= ||b - Q mu||_inf / min_i (Q_ii - R_i) holds for
// any mu; a row without a positive margin records +inf (no bound).
__device__ __forceinline__ void note_margin(Ctrl* c, float qd, double R)
{
    const double mg = (double)qd - R;
    const double inv = mg > 0.0 ? 1.0 / mg : INFINITY;
    atomicMax(&c->inv_margin_bits, (unsigned long long)__double_as_longlong(inv));
}

// Diagonal rule (Section 3.1) from the |Q| row-sum partials of the Q
// formation, then Algorithm 2 Step 1: messages 0, so Ptilde = Q_ii,
// htilde = b_i, mutilde = b_i / Q_ii.  CTA 0 resets the control block.
__global__ void k_init(Inst p, int diag_rule, float delta)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl* c = p.ctrl;
        c->t = 0;
        c->done = 1;
        c->limit = 0;
        c->kstar = 0;
        c->converged = 0;
        c->rmax_bits = 0ull;
        c->blocks_done = 0u;
        c->tol = 0.0;
        c->rinf = -1.0;
    }
    if (x >= p.n) return;
    const double R = offdiag_abs_sum(p, x);
    zero_slots(p, x, true);   // all messages start at 0
    const double lam2 = p.lam2;
    const double base = 1.0 + lam2 + 1.0 / (double)p.C;
    double qd = base;
    if (diag_rule == 0) {
        const double dom = (1.0 + (double)delta) * R;
        qd = dom > base ? dom : base;
    }
    const float qf = (float)qd, bx = p.b[x];
    p.qdiag[x] = qf;
    p.agg[x] = qf;
    p.agg[p.npad + x] = bx;
    p.agg[2 * p.npad + x] = bx / qf;
    note_margin(p.ctrl, qf, R);
}

__global__ void k_row_abs_sums(Inst p, double* __restrict__ rsum)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < p.n) {
        const long long a = reinterpret_cast<const long long*>(rsum)[x];
        rsum[x] = rsum_unfix(a, rsum_shift(p.n, p.lam2));
    }
}

// k_init over listed node blocks (block 0 of an instance resets its control block).
__global__ void k_init_list(const Inst* __restrict__ tab, const int2* __restrict__ nbl, int diag_rule, float delta)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    if (nb.y == 0 && threadIdx.x == 0) {
        Ctrl* c = p.ctrl;
        c->t = 0;
        c->done = 1;
        c->limit = 0;
        c->kstar = 0;
        c->converged = 0;
        c->rmax_bits = 0ull;
        c->blocks_done = 0u;
        c->tol = 0.0;
        c->rinf = -1.0;
    }
    const int x = nb.y * 32 + threadIdx.x;
    if (threadIdx.x >= 32 || x >= p.n) return;
    const double R = offdiag_abs_sum(p, x);
    zero_slots(p, x, true);   // all messages start at 0
    const double lam2 = p.lam2;
    const double base = 1.0 + lam2 + 1.0 / (double)p.C;
    double qd = base;
    if (diag_rule == 0) {
        const double dom = (1.0 + (double)delta) * R;
        qd = dom > base ? dom : base;
    }
    const float qf = (float)qd, bx = p.b[x];
    p.qdiag[x] = qf;
    p.agg[x] = qf;
    p.agg[p.npad + x] = bx;
    p.agg[2 * p.npad + x] = bx / qf;
    note_margin(p.ctrl, qf, R);
}

__global__ void k_begin_list(Inst* tab, const int2* __restrict__ list, const double* __restrict__ tols, int count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    Ctrl* c = tab[list[k].x].ctrl;
    const int iters = list[k].y;
    c->limit = c->t + iters;
    c->tol = tols[k];
    c->converged = 0;
    c->kstar = c->t;
    c->rinf = -1.0;
    c->rmax_bits = 0ull;
    c->blocks_done = 0u;
    c->done = (c->status != 0 || iters <= 0) ? 1 : 0;
}

__global__ void k_begin(Inst* tab, int ninst, int iters, double tol)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ninst) return;
    Ctrl* c = tab[k].ctrl;
    c->limit = c->t + iters;
    c->tol = tol;
    c->converged = 0;
    c->kstar = c->t;
    c->rinf = -1.0;
    c->rmax_bits = 0ull;
    c->blocks_done = 0u;
    c->done = (c->status != 0 || iters <= 0) ? 1 : 0;
}

__global__ void k_get_pairs(Inst p, const long long* __restrict__ ij, long long cnt, float4* __restrict__ out)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    const long long i = ij[2 * e], j = ij[2 * e + 1];
    const long long I = i / T, J = j / T, Nt = p.Nt;
    long long L = I * Nt - I * (I - 1) / 2 + (J - I);
    if (p.slab) L = p.slab[L];   // -1: a dropped tile, whose messages are 0
    const int r = (int)(i - I * T), c = (int)(j - J * T);
    if (p.ctrl->t == 0 || L < 0) {
        out[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const size_t o = (size_t)L * TT + r * T + c;
        float2 a, b;
        if (p.msg_bf16) {
            a = __bfloat1622float2(static_cast<const __nv_bfloat162*>(p.Pst)[o]);
            b = __bfloat1622float2(static_cast<const __nv_bfloat162*>(p.Hst)[o]);
        } else {
            a = static_cast<const float2*>(p.Pst)[o];
            b = static_cast<const float2*>(p.Hst)[o];
        }
        out[e] = make_float4(a.x, a.y, b.x, b.y);
    }
}

}  // namespace

void launch_init(const Inst& p, int diag_rule, float delta, cudaStream_t s)
{
    k_init<<<(p.n + 255) / 256, 256, 0, s>>>(p, diag_rule, delta);
}

void launch_row_abs_sums(const Inst& p, double* rsum, cudaStream_t s)
{
    k_row_abs_sums<<<(p.n + 255) / 256, 256, 0, s>>>(p, rsum);
}

void launch_reset(const Inst& p, cudaStream_t s) { k_reset<<<(p.n + 255) / 256, 256, 0, s>>>(p); }

void launch_refine_rhs_list(const Inst* tab, const StopOp* ops, const int2* nbl, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) k_refine_rhs_list<<<nblocks, 32, 0, s>>>(tab, ops, nbl);
}

void launch_axpy_list(const Inst* tab, const StopOp* ops, const int2* nbl, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) k_axpy_list<<<nblocks, 32, 0, s>>>(tab, ops, nbl);
}

void launch_init_list(const Inst* tab, const int2* nbl, int nblocks, int diag_rule, float delta, cudaStream_t s)
{
    if (nblocks > 0) k_init_list<<<nblocks, 32, 0, s>>>(tab, nbl, diag_rule, delta);
}

void launch_begin_list(Inst* tab, const int2* list, const double* tols, int count, cudaStream_t s)
{
    if (count > 0) k_begin_list<<<(count + 127) / 128, 128, 0, s>>>(tab, list, tols, count);
}

void launch_begin(Inst* tab, int ninst, int iters, double tol, cudaStream_t s)
{
    k_begin<<<(ninst + 127) / 128, 128, 0, s>>>(tab, ninst, iters, tol);
}

int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

RoundGrid round_grid(long long max_tiles, int max_nblocks, int q_mode, int ctas_per_sm, int msg_bf16)
{
    const int sms = num_sms();
    RoundGrid g;
    const int dflt = msg_bf16 ? sweep_ctas<MsgBF16>() : sweep_ctas<MsgF32>();
    const long long per_sm = q_mode == 2 ? 1 : (ctas_per_sm > 0 ? std::min(ctas_per_sm, dflt) : dflt);
    const long long gs = (long long)sms * per_sm;
    g.sweep = (int)(max_tiles < gs ? (max_tiles > 0 ? max_tiles : 1) : gs);
    const int gf = sms * 8;
    g.finalize = max_nblocks < gf ? (max_nblocks > 0 ? max_nblocks : 1) : gf;
    return g;
}

cudaError_t prepare_sweep_rc()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep_rc<MsgF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rc_smem_bytes<MsgF32>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep_rc<MsgBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rc_smem_bytes<MsgBF16>());
}

cudaError_t prepare_sweep()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep<float, MsgF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep_smem_bytes<float, MsgF32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep<__nv_bfloat16, MsgF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sweep_smem_bytes<__nv_bfloat16, MsgF32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep<__nv_bfloat16, MsgBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sweep_smem_bytes<__nv_bfloat16, MsgBF16>());
    return e;
}

void launch_round(const Inst* tab, const int4* work, const int2* nbl, const Sched* sched, int nstages,
                  const RoundGrid& g, int q_mode, int msg_bf16, cudaStream_t s, cudaEvent_t* ev)
{
    for (int st = 0; st < nstages; ++st) {
        const Sched* sc = sched + st;
        if (ev && st == 0) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
        if (q_mode == 2 && msg_bf16)
            k_sweep_rc<MsgBF16><<<g.sweep, RC_THREADS, rc_smem_bytes<MsgBF16>(), s>>>(tab, work, sc, st);
        else if (q_mode == 2)
            k_sweep_rc<MsgF32><<<g.sweep, RC_THREADS, rc_smem_bytes<MsgF32>(), s>>>(tab, work, sc, st);
        else if (q_mode == 1 && msg_bf16)
            k_sweep<__nv_bfloat16, MsgBF16>
                <<<g.sweep, SWEEP_THREADS, sweep_smem_bytes<__nv_bfloat16, MsgBF16>(), s>>>(tab, work, sc, st);
        else if (q_mode == 1)
            k_sweep<__nv_bfloat16, MsgF32>
                <<<g.sweep, SWEEP_THREADS, sweep_smem_bytes<__nv_bfloat16, MsgF32>(), s>>>(tab, work, sc, st);
        else
            k_sweep<float, MsgF32>
                <<<g.sweep, SWEEP_THREADS, sweep_smem_bytes<float, MsgF32>(), s>>>(tab, work, sc, st);
        if (ev && st == nstages - 1) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
        if (st < nstages - 1)
            k_finalize_stage<<<g.finalize, 256, 0, s>>>(tab, nbl, sched);
        else
            k_finalize<<<g.finalize, 256, 0, s>>>(tab, nbl, sched);
    }
}

void launch_get_pairs(const Inst& p, const long long* ij, long long cnt, float4* out, cudaStream_t s)
{
    if (cnt > 0) k_get_pairs<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(p, ij, cnt, out);
}

}  // namespace gabp

namespace gabp {
cudaError_t launch_selftest_rcp(const float* d, float* out, int cnt, cudaStream_t s)
{
    if (cnt > 0) k_selftest_rcp<<<(cnt + 255) / 256, 256, 0, s>>>(d, out, cnt);
    return cudaGetLastError();
}

cudaError_t launch_selftest_wait(unsigned long long limit_ns, int* status_dev, cudaStream_t s)
{
    k_selftest_wait<<<1, 32, 0, s>>>(limit_ns, status_dev);
    return cudaGetLastError();
}
}  // namespace gabp
