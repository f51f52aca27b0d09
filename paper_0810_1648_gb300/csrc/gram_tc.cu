// BF16 Gram tiles on the 5th-generation tensor cores (tcgen05), fused with the
// RBF kernel, labels and bias, for the precision form of the solver: Q tiles
// from BF16 features with FP32 accumulation (Section 5 computes the kernel
// matrix once; Section 3 adds the bias term; Section 1.1 defines
// D_ij = y_i y_j K(x_i, x_j)).
//
// Operand layout.  The features are rounded to BF16 once and packed per
// 128-row tile and 64-feature chunk into a 16 KB block in the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices stored as
// contiguous 128-byte blocks, K-adjacent core matrices 128 bytes apart,
// 8-row groups 1024 bytes apart.  One bulk copy then moves a ready operand.
// Row norms are taken from the same rounded values, so d^2_ii is 0.
//
// k_form_q_tc is a persistent kernel with warp roles: warp 0 streams the A/B
// operand blocks of each tile into a 4-stage shared-memory ring; warp 1
// allocates 256 TMEM columns (two 128 x 128 FP32 accumulators) and one of its
// threads issues the MMAs (M = N = 128, K = 16 per instruction); warps 2-5
// read the accumulator rows back from TMEM (warp w reads lanes
// 32*(w%4)..+31), apply d^2 = max(0, s_i + s_j - 2G), exp, labels and bias,
// and write the tile's Q values in BF16.  The accumulator is double buffered
// so the epilogue of one tile overlaps the MMAs of the next.
#include "common.cuh"
#include "ptx.cuh"
#include "qtile_epi.cuh"

#include <float.h>

namespace gabp {

namespace {

constexpr int XSTAGES = 4;
constexpr int TC_THREADS = 10 * 32;   // producer, MMA issuer, 8 epilogue warps
constexpr int TC_EPI_WARPS = 8;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t IDESC = idesc_bf16_f32(T, T);

// Packs FP32 rows into the BF16 core-matrix blocks (zero padding for rows >= n
// and features >= m); one thread per (row, 8-feature group).
__global__ void k_pack_bf16(const float* __restrict__ Xf, int n, int m, int nkc, int Nt,
                            uint4* __restrict__ Xp)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long groups = (long long)nkc * (KCH / 8);
    if (e >= (long long)Nt * T * groups) return;
    const int r = (int)(e / groups), gk = (int)(e % groups);
    const int kc = gk / (KCH / 8), kg = gk % (KCH / 8);
    const int I = r / T, rr = r % T;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int k = kc * KCH + kg * 8 + u;
        v[u] = __float2bfloat16_rn((r < n && k < m) ? Xf[(size_t)r * m + k] : 0.f);
    }
    const size_t blk = (size_t)I * nkc + kc;
    const size_t off16 = blk * (BLK_BYTES / 16) + (size_t)((rr / 8) * (KCH / 8) + kg) * 8 + (rr % 8);
    Xp[off16] = *reinterpret_cast<const uint4*>(v);
}

// Listed node blocks (32 rows): packing (8 threads per row over the 8-feature
// groups) and the BF16 row norms.  The last block of an instance also writes
// the zero rows that pad its last 128-row tile, so the packed operand needs no
// clearing beforehand.
__global__ void k_pack_list(const Inst* __restrict__ tab, const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    const int rl = threadIdx.x >> 3, gsub = threadIdx.x & 7;
    const int r = nb.y * 32 + rl, n = p.n, m = p.m, nkc = p.nkc;
    const int Nt = p.Nt;
    const bool last = nb.y == (n - 1) / 32;
    const float* Xf = p.X;
    uint4* Xp = static_cast<uint4*>(const_cast<void*>(p.Xp));
    const int groups = nkc * (KCH / 8);
    for (int rw = r; rw < Nt * T; rw += 32) {
        const int I = rw / T, rr = rw % T;
        for (int gk = gsub; gk < groups; gk += 8) {
            const int kc = gk / (KCH / 8), kg = gk % (KCH / 8);
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = kc * KCH + kg * 8 + u;
                v[u] = __float2bfloat16_rn((rw < n && k < m) ? Xf[(size_t)rw * m + k] : 0.f);
            }
            const size_t blk = (size_t)I * nkc + kc;
            Xp[blk * (BLK_BYTES / 16) + (size_t)((rr / 8) * (KCH / 8) + kg) * 8 + (rr % 8)] =
                *reinterpret_cast<const uint4*>(v);
        }
        if (!last) break;
    }
    if (gsub == 0 && r < n) {
        float sacc = 0.f;
        for (int k = 0; k < m; ++k) {
            const float v = __bfloat162float(__float2bfloat16_rn(Xf[(size_t)r * m + k]));
            sacc = fmaf(v, v, sacc);
        }
        const_cast<float*>(p.sqb)[r] = sacc;
    }
}

// ||bf16(x_i)||^2 in FP32 from the rounded values.
__global__ void k_norms_bf16(const float* __restrict__ Xf, int n, int m, float* __restrict__ sqb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int k = 0; k < m; ++k) {
        const float v = __bfloat162float(__float2bfloat16_rn(Xf[(size_t)i * m + k]));
        s = fmaf(v, v, s);
    }
    sqb[i] = s;
}

struct TcSmem {
    unsigned long long xfull[XSTAGES], xempty[XSTAGES];
    unsigned long long accfull[2], accempty[2];
    unsigned long long drain;
    uint32_t tmem_base;
    int abort;
    ColTile cols[TC_EPI_WARPS];    // column constants of the current tile, one set per epilogue warp
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_form_q_tc(const Inst* __restrict__ tab, const int4* __restrict__ work, long long ntiles)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = align_smem(smem_raw, 1024);
    unsigned char* ops = base;                                   // XSTAGES x (A block, B block)
    TcSmem& sm = *reinterpret_cast<TcSmem*>(base + XSTAGES * 2 * BLK_BYTES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < XSTAGES; ++s) { mbar_init(&sm.xfull[s], 1); mbar_init(&sm.xempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&sm.accfull[b], 1); mbar_init(&sm.accempty[b], TC_EPI_WARPS); }
        mbar_init(&sm.drain, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, TMEM_COLS);
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
                const unsigned char* Xp = static_cast<const unsigned char*>(p.Xp);
                const int I = w.y, J = w.z, nkc = p.nkc;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*(volatile int*)&sm.abort || !mbar_wait(&sm.xempty[stage], ph ^ 1u)) {
                        sm.abort = 1;
                        record_error(p.ctrl, ST_ETIMEOUT, L);
                        run = false;
                        break;
                    }
                    unsigned char* A = ops + (size_t)stage * 2 * BLK_BYTES;
                    mbar_arrive_expect_tx(&sm.xfull[stage], 2 * BLK_BYTES);
                    bulk_load(A, Xp + ((size_t)I * nkc + kc) * BLK_BYTES, BLK_BYTES, &sm.xfull[stage], pol);
                    bulk_load(A + BLK_BYTES, Xp + ((size_t)J * nkc + kc) * BLK_BYTES, BLK_BYTES, &sm.xfull[stage],
                              pol);
                    if (++stage == XSTAGES) { stage = 0; ph ^= 1u; }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
                const Inst& p = tab[work[L].x];
                Ctrl* ctrl = p.ctrl;
                const int nkc = p.nkc;
                if (*(volatile int*)&sm.abort || !mbar_wait(&sm.accempty[acc], aph ^ 1u)) {
                    sm.abort = 1;
                    record_error(ctrl, ST_ETIMEOUT, L);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tbase + (uint32_t)acc * T;
                bool ok = true;
                for (int kc = 0; kc < nkc; ++kc) {
                    if (*(volatile int*)&sm.abort || !mbar_wait(&sm.xfull[stage], ph)) {
                        sm.abort = 1;
                        record_error(ctrl, ST_ETIMEOUT, L);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* A = ops + (size_t)stage * 2 * BLK_BYTES;
#pragma unroll
                    for (int s = 0; s < KCH / 16; ++s) {
                        const uint64_t ad = smem_desc(A + s * 256, 128, 1024);
                        const uint64_t bd = smem_desc(A + BLK_BYTES + s * 256, 128, 1024);
                        tc_mma_bf16(d, ad, bd, IDESC, (kc | s) != 0);
                    }
                    tc_commit(&sm.xempty[stage]);
                    if (++stage == XSTAGES) { stage = 0; ph ^= 1u; }
                }
                if (!ok) break;
                tc_commit(&sm.accfull[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1u; }
            }
            // every MMA issued above must finish before the columns are freed
            tc_commit(&sm.drain);
            if (!mbar_wait(&sm.drain, 0u)) sm.abort = 1;
        }
    } else {
        // --------------------------------------------------------- epilogue
        // warp w may read TMEM lanes 32 (w % 4) ..: two warps per lane
        // quarter, one per half of the 128 columns
        const int g = warp & 3, half = (warp - 2) >> 2;
        const int r = 32 * g + lane;
        int acc = 0;
        uint32_t aph = 0;
        for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
            const int4 w = work[L];
            const bool stop = __shfl_sync(0xffffffffu, *(volatile int*)&sm.abort, 0) != 0;
            if (stop || !mbar_wait_warp(&sm.accfull[acc], aph)) {
                if (lane == 0) {
                    sm.abort = 1;
                    record_error(tab[w.x].ctrl, ST_ETIMEOUT, L);
                }
                break;
            }
            tc_fence_after();
            const int I = w.y, J = w.z;
            const int i = I * T + r;
            // the listed instance and every one chained behind it (same
            // features) take their BF16 Q tile from this accumulator
            ColTile& cs = sm.cols[warp - 2];
            for (int k = w.x; k >= 0;) {
                const Inst& p = tab[k];
                const int n = p.n;
                const float* y = p.y;
                const float* sqb = p.sqb;
                const float gamma = p.gamma, lam2 = p.lam2;
                const float yi = i < n ? y[i] : 0.f, si = i < n ? sqb[i] : 0.f;
                stage_tile_cols(cs, y, sqb, n, J, gamma, lane, 2 * half, 2 * half + 2);
                const float ai = -gamma * kLog2e * si, c2 = 2.f * gamma * kLog2e;
                const uint32_t s1 = __float_as_uint(yi) & 0x80000000u, si2 = s1 | (s1 >> 16);
                __nv_bfloat16* qrow = static_cast<__nv_bfloat16*>(p.qstore) + (size_t)w.w * TT + (size_t)r * T;
#pragma unroll 1
                for (int cc = 2 * half; cc < 2 * half + 2; ++cc) {
                    const uint32_t valid = chunk_valid(n, I, J, r, cc);
                    uint4* dst = reinterpret_cast<uint4*>(qrow + 32 * cc);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float v[16];
                        tmem_ld16(tbase + (uint32_t)acc * T + ((uint32_t)(32 * g) << 16) + (uint32_t)(32 * cc + 16 * h),
                                  v);
                        uint4 out[2];
                        q_half_bf16(v, 32 * cc + 16 * h, ai, si2, cs, c2, lam2, (valid >> (16 * h)) & 0xffffu, out);
                        dst[2 * h] = out[0];
                        dst[2 * h + 1] = out[1];
                    }
                }
                k = p.form_next - 1;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.accempty[acc]);
            if (++acc == 2) { acc = 0; aph ^= 1u; }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, TMEM_COLS);
    }
}

constexpr size_t tc_smem_bytes() { return 1024 + XSTAGES * 2 * BLK_BYTES + sizeof(TcSmem); }

}  // namespace

cudaError_t launch_pack_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) k_pack_list<<<nblocks, 256, 0, s>>>(tab, nbl);
    return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const float* Xf, int n, int m, int nkc, int Nt, void* Xp, float* sqb, cudaStream_t s)
{
    const long long total = (long long)Nt * T * nkc * (KCH / 8);
    k_pack_bf16<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Xf, n, m, nkc, Nt, static_cast<uint4*>(Xp));
    k_norms_bf16<<<(n + 255) / 256, 256, 0, s>>>(Xf, n, m, sqb);
    return cudaGetLastError();
}

cudaError_t launch_form_q_tc(const Inst* tab, const int4* work, long long ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_form_q_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_form_q_tc<<<grid, TC_THREADS, tc_smem_bytes(), s>>>(tab, work, ntiles);
    return cudaGetLastError();
}

int bf16_chunks(int m) { return (m + KCH - 1) / KCH; }
size_t bf16_pack_bytes(int Nt, int m) { return (size_t)Nt * bf16_chunks(m) * BLK_BYTES; }

}  // namespace gabp
