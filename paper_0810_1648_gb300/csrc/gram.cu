// SIMT FP32 Gram tiles fused with the RBF kernel, and everything built on them:
//   - input staging (FP64 -> FP32, row norms, label/finiteness checks),
//   - the final residual r = 1 - Q mu and Q alpha for the dual objective
//     (Q read back from the FP32 tiles, or recomputed here when not stored),
//   - the decision values f(x) = sum_i alpha_i y_i (K(x_i, x) + lambda^2)
//     (Section 1.1).
// (The stored Q tiles themselves are formed on the tensor cores: gram_tc32.cu.)
//
// One CTA computes one 128 x 128 Gram tile G = X_I X_J^T by SIMT FP32 FMAs
// (8 x 8 outputs per thread, K-chunks of 16 double-buffered in shared memory),
// then runs an epilogue on the 64 values it holds: d^2 = max(0, s_i + s_j - 2 G),
// K = expf(-gamma d^2), Q_ij = y_i y_j (K + lambda^2).  The distances use the
// norm expansion with norms of the same FP32 rows, so d^2_ii is 0 up to
// rounding and is clamped at 0.
#include "common.cuh"
#include "gabp_svm.h"

#include <float.h>
#include <mutex>
#include <string>

namespace gabp {

namespace {

constexpr int KC = 16;

struct GramSmem {
    float A[2][KC][T + 4];   // double-buffered K-chunks
    float B[2][KC][T + 4];
};

struct EpiSmem {
    float rowv[2][T];
    float colw[NWARPS][2][T];
    float colv[2][T];
};

union TileSmem {
    GramSmem g;
    EpiSmem e;
};

// acc[a][b] = <x_{I*T + ty*8 + a}, x_{J*T + tx*8 + b}>.  K-chunks of KC
// features go through two shared-memory buffers: the next chunk's global
// loads are in flight (in registers) while the current chunk's FMAs run, and
// one barrier per chunk separates the buffer swaps.  Every output sums its
// products in ascending k, as a plain loop would.
__device__ __forceinline__ void gram_tile(const GramSide& A, const GramSide& B, int m, int I, int J,
                                          GramSmem& sm, float (&acc)[8][8])
{
    constexpr int LD = (T * KC) / NTHREADS;   // elements of each operand a thread stages per chunk
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    float ra[LD], rb[LD];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = tid + NTHREADS * u;
            const int row = e / KC, kk = e % KC, k = k0 + kk;
            const int ga = I * T + row, gb = J * T + row;
            ra[u] = (ga < A.n && k < m) ? A.X[(size_t)ga * m + k] : 0.f;
            rb[u] = (gb < B.n && k < m) ? B.X[(size_t)gb * m + k] : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = tid + NTHREADS * u;
            const int row = e / KC, kk = e % KC;
            sm.A[buf][kk][row] = ra[u];
            sm.B[buf][kk][row] = rb[u];
        }
    };
    const int nch = (m + KC - 1) / KC;
    load(0);
    store(0);
    __syncthreads();
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        if (c + 1 < nch) load((c + 1) * KC);
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sm.A[buf][kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sm.A[buf][kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sm.B[buf][kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sm.B[buf][kk][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        if (c + 1 < nch) store(buf ^ 1);
        __syncthreads();
    }
}

// RBF entry from a Gram value (norm expansion, clamped distance).
__device__ __forceinline__ float rbf_from_gram(float g, float si, float sj, float gamma)
{
    const float d2 = fmaxf(0.f, si + sj - 2.f * g);
    return expf(-gamma * d2);
}

// Sums over the 16 tx-lanes that share a row (lanes differ in bits 0..3).
__device__ __forceinline__ float sum16(float v)
{
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row sums (rs, per thread's 8 rows) and column sums (cs, per thread's 8
// columns) of up to two quantities -> per-node slot partials part_q[k][x].
template <int NQ>
__device__ __forceinline__ void reduce_and_write(EpiSmem& es, float (&rs)[NQ][8], float (&cs)[NQ][8],
                                                 float* const (&part)[NQ], int n, int I, int J, int2 sl)
{
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15, warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const float v = sum16(rs[q][a]);
            if (tx == 0) es.rowv[q][ty * 8 + a] = v;
        }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float v = cs[q][b] + __shfl_xor_sync(0xffffffffu, cs[q][b], 16);
            if (lane < 16) es.colw[warp][q][tx * 8 + b] = v;
        }
    __syncthreads();
    if (tid < T) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < NWARPS; ++w) s += es.colw[w][q][tid];
            es.colv[q][tid] = s;
        }
    }
    __syncthreads();
    // slot sl.x of the row block (its nodes I T + r), sl.y of the column block
    const size_t oR = (size_t)sl.x * T, oC = (size_t)sl.y * T;
    if (I == J) {
        if (tid < T) {
            const int x = I * T + tid;
            if (x < n)
#pragma unroll
                for (int q = 0; q < NQ; ++q) part[q][oR + tid] = es.rowv[q][tid] + es.colv[q][tid];
        }
    } else {
        if (tid < T) {
            const int x = I * T + tid;
            if (x < n)
#pragma unroll
                for (int q = 0; q < NQ; ++q) part[q][oR + tid] = es.rowv[q][tid];
        } else {
            const int c = tid - T, x = J * T + c;
            if (x < n)
#pragma unroll
                for (int q = 0; q < NQ; ++q) part[q][oC + c] = es.colv[q][c];
        }
    }
}

// ---------------------------------------------------------------- staging
// One row: FP32 copy (from FP32, FP64 or BF16 input; BF16 widens exactly),
// squared norm, finiteness and label checks, b_i = 1 (the SVM right-hand
// side: the linear term 1'h of the dual).
__device__ __forceinline__ void stage_row(const void* __restrict__ X, int x_dtype, int i, int m,
                                          float* __restrict__ y, float* __restrict__ Xf,
                                          float* __restrict__ sq, float* __restrict__ b,
                                          float* __restrict__ b0, int task, Ctrl* ctrl)
{
    float s = 0.f;
    bool ok = true;
    for (int k = 0; k < m; ++k) {
        const size_t e = (size_t)i * m + k;
        const float v = x_dtype == 1   ? (float)static_cast<const double*>(X)[e]
                        : x_dtype == 2 ? __bfloat162float(static_cast<const __nv_bfloat16*>(X)[e])
                                       : static_cast<const float*>(X)[e];
        ok &= isfinite(v);
        if (Xf != X) Xf[e] = v;
        s = fmaf(v, v, s);
    }
    sq[i] = s;
    float rhs = 1.f;   // SVM: Q alpha = 1 (Section 3)
    if (y) {
        const float yi = y[i];
        if (task) {    // KRR: (K + lambda_r I) c = y (Section 1.2)
            ok &= isfinite(yi);
            rhs = yi;
            y[i] = 1.f;
        } else {
            ok &= (yi == 1.f || yi == -1.f);
        }
    }
    if (b) b[i] = rhs;
    if (b0) b0[i] = rhs;
    if (!ok && atomicCAS(&ctrl->status, 0, (int)ST_EINVAL) == 0) ctrl->bad_index = i;
}

__global__ void k_stage(const void* __restrict__ X, int x_dtype, int n, int m, float* __restrict__ y,
                        float* __restrict__ Xf, float* __restrict__ sq, float* __restrict__ b,
                        float* __restrict__ b0, int task, Ctrl* ctrl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) stage_row(X, x_dtype, i, m, y, Xf, sq, b, b0, task, ctrl);
}

// Listed node blocks of instances whose FP32 rows already sit in their X.
__global__ void k_stage_list(const Inst* __restrict__ tab, const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    const int i = nb.y * 32 + threadIdx.x;
    if (threadIdx.x < 32 && i < p.n)
        stage_row(p.X, 0, i, p.m, const_cast<float*>(p.y), const_cast<float*>(p.X), const_cast<float*>(p.sq),
                  const_cast<float*>(p.b), const_cast<float*>(p.b0), p.task, p.ctrl);
}

// ------------------------------------------- final residual and Q alpha
// For every instance k listed: off-diagonal sums sum_{j != i} Q_ij mu_j
// (-> part[0]) and sum_{j != i} Q_ij alpha_j (-> part[1]).
//
// Per listed tile: partial sums of (Q mu)_i and (Q alpha)_i over the tile's
// pairs (both roles) into the slot partials, with alpha = clip(mu, 0, C) and
// mu = ops[k].mu.  acc holds the tile's stored FP32 Q values (STORED) or its
// FP32 Gram values, from which Q is formed exactly as at formation, so both
// give the same values.
template <bool STORED>
__device__ __forceinline__ void final_tile_sums(const Inst& p, const float* __restrict__ mu, int4 w,
                                                float (&acc)[8][8], EpiSmem& es)
{
    const int n = p.n, I = w.y, J = w.z;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float yj[8], sj[8], mj[8], aj[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int j = J * T + tx * 8 + b;
        yj[b] = j < n ? p.y[j] : 0.f;
        sj[b] = j < n ? p.sq[j] : 0.f;
        mj[b] = j < n ? mu[j] : 0.f;
        aj[b] = p.task ? mj[b] : fminf(fmaxf(mj[b], 0.f), p.C);
    }
    float rs[2][8], cs[2][8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cs[0][b] = cs[1][b] = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = ty * 8 + a, i = I * T + r;
        const float yi = i < n ? p.y[i] : 0.f, si = i < n ? p.sq[i] : 0.f;
        const float mi = i < n ? mu[i] : 0.f, ai = p.task ? mi : fminf(fmaxf(mi, 0.f), p.C);
        float rm = 0.f, ra = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int c = tx * 8 + b, j = J * T + c;
            const bool v = i < n && j < n && (I != J || c > r);
            const float q0 =
                STORED ? acc[a][b] : yi * yj[b] * (rbf_from_gram(acc[a][b], si, sj[b], p.gamma) + p.lam2);
            const float q = v ? q0 : 0.f;
            rm = fmaf(q, mj[b], rm);
            ra = fmaf(q, aj[b], ra);
            cs[0][b] = fmaf(q, mi, cs[0][b]);
            cs[1][b] = fmaf(q, ai, cs[1][b]);
        }
        rs[0][a] = rm;
        rs[1][a] = ra;
    }
    float* const parts[2] = {p.part, p.part + part_len(p)};
    reduce_and_write<2>(es, rs, cs, parts, n, I, J, tile_slots(p, w));
}

// Q recomputed by the FP32 Gram (forms without an FP32 store).  One CTA per
// listed tile.
__global__ void __launch_bounds__(NTHREADS) k_final_tiles(const Inst* __restrict__ tab,
                                                          const StopOp* __restrict__ ops,
                                                          const int4* __restrict__ work)
{
    __shared__ __align__(16) TileSmem sm;
    const int4 w = work[blockIdx.x];
    const Inst& p = tab[w.x];
    float acc[8][8];
    const GramSide S{p.X, p.sq, p.n};
    gram_tile(S, S, p.m, w.y, w.z, sm.g, acc);
    __syncthreads();   // Gram smem is reused by the epilogue
    final_tile_sums<false>(p, ops[w.x].mu, w, acc, sm.e);
}

// Q read back from the FP32 tiles (Inst::qref): no Gram, small footprint, so
// several CTAs share an SM and the pass runs at memory speed.
__global__ void __launch_bounds__(NTHREADS, 2) k_final_tiles_q(const Inst* __restrict__ tab,
                                                               const StopOp* __restrict__ ops,
                                                               const int4* __restrict__ work)
{
    __shared__ __align__(16) EpiSmem es;
    const int4 w = work[blockIdx.x];
    const Inst& p = tab[w.x];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const float* qt = p.qref + (size_t)w.w * TT;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const float4 u0 = *reinterpret_cast<const float4*>(qt + (ty * 8 + a) * T + tx * 8);
        const float4 u1 = *reinterpret_cast<const float4*>(qt + (ty * 8 + a) * T + tx * 8 + 4);
        acc[a][0] = u0.x; acc[a][1] = u0.y; acc[a][2] = u0.z; acc[a][3] = u0.w;
        acc[a][4] = u1.x; acc[a][5] = u1.y; acc[a][6] = u1.z; acc[a][7] = u1.w;
    }
    final_tile_sums<true>(p, ops[w.x].mu, w, acc, es);
}

// Per node of a listed node block: r_i = b0_i - Q_ii mu_i - sum part0,
// (Q alpha)_i = Q_ii alpha_i + sum part1; writes alpha (and r in FP32 when
// requested); block partials {max |r_i|, sum b0_i alpha_i - 1/2 alpha_i
// (Q alpha)_i, #SV} into the instance's block buffer.  SVM: b0 = 1, alpha =
// clip(mu, 0, C), SV where alpha_i > threshold; KRR: b0 = the targets, alpha =
// mu, counted where |alpha_i| > threshold.
__global__ void __launch_bounds__(256) k_final_nodes(const Inst* __restrict__ tab,
                                                     const StopOp* __restrict__ ops,
                                                     const int2* __restrict__ nbl)
{
    const int2 nb = nbl[blockIdx.x];
    const Inst& p = tab[nb.x];
    const StopOp& op = ops[nb.x];
    const float* __restrict__ mu = op.mu;
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int x = nb.y * 32 + lane, n = p.n;
    double s0 = 0.0, s1 = 0.0;
    if (x < n) {
        // the node's slots (see slot_begin)
        const int X = x / T, ns = slot_count(p, X);
        const float* p0 = p.part + (size_t)slot_begin(p, X) * T + (x - X * T);
        const float* p1 = p0 + part_len(p);
        for (int k = g; k < ns; k += 8) {
            s0 += (double)p0[(size_t)k * T];
            s1 += (double)p1[(size_t)k * T];
        }
    }
    __shared__ double red[2][8][32];
    red[0][g][lane] = s0;
    red[1][g][lane] = s1;
    __syncthreads();
    if (g == 0) {
        double absr = 0.0, obj = 0.0, nsv = 0.0;
        if (x < n) {
            double a0 = 0.0, a1 = 0.0;
            for (int w = 0; w < 8; ++w) { a0 += red[0][w][lane]; a1 += red[1][w][lane]; }
            const double qd = p.qdiag[x], m = mu[x], bx = p.b0[x];
            const float af = p.task ? mu[x] : fminf(fmaxf(mu[x], 0.f), p.C);
            const double al = af;
            op.alpha[x] = af;
            const double r = bx - qd * m - a0;   // residual of the system Q mu = b0
            if (op.r_out) op.r_out[x] = (float)r;
            absr = fabs(r);
            if (!(absr <= DBL_MAX)) absr = INFINITY;
            const double qa = qd * al + a1;
            obj = bx * al - 0.5 * al * qa;
            nsv = (p.task ? fabsf(af) : af) > op.sv_threshold ? 1.0 : 0.0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            absr = fmax(absr, __shfl_xor_sync(0xffffffffu, absr, o));
            obj += __shfl_xor_sync(0xffffffffu, obj, o);
            nsv += __shfl_xor_sync(0xffffffffu, nsv, o);
        }
        if (lane == 0) {
            op.blockbuf[3 * nb.y + 0] = absr;
            op.blockbuf[3 * nb.y + 1] = obj;
            op.blockbuf[3 * nb.y + 2] = nsv;
        }
    }
}

// One CTA per listed instance: fixed-order reduction of its block partials
// -> final3 = {||r||_inf, objective, #SV}, also copied to f3_all[3 * slot].
__global__ void k_final_reduce(const Inst* __restrict__ tab, const StopOp* __restrict__ ops,
                               const int* __restrict__ members, double* __restrict__ f3_all)
{
    __shared__ double s[3][256];
    const int slot = members[blockIdx.x];
    const StopOp& op = ops[slot];
    const int nb = (tab[slot].n + 31) / 32;
    const int tid = threadIdx.x;
    double m = 0.0, o = 0.0, c = 0.0;
    for (int k = tid; k < nb; k += 256) {
        m = fmax(m, op.blockbuf[3 * k]);
        o += op.blockbuf[3 * k + 1];
        c += op.blockbuf[3 * k + 2];
    }
    s[0][tid] = m; s[1][tid] = o; s[2][tid] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            s[0][tid] = fmax(s[0][tid], s[0][tid + w]);
            s[1][tid] += s[1][tid + w];
            s[2][tid] += s[2][tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int q = 0; q < 3; ++q) {
            op.final3[q] = s[q][0];
            if (f3_all) f3_all[3 * slot + q] = s[q][0];
        }
    }
}

// ----------------------------------------------------------------- decision
// Rectangle of tiles (test tile I, training tile J): part[J][s] =
// sum_{j in J} alpha_j y_j (K(x_j, xt_s) + lambda^2).
__global__ void __launch_bounds__(NTHREADS) k_decision_tiles(Inst p, const float* __restrict__ Xt,
                                                             const float* __restrict__ sqt, int t,
                                                             const float* __restrict__ alpha,
                                                             const int2* __restrict__ work,
                                                             float* __restrict__ part)
{
    __shared__ __align__(16) TileSmem sm;
    const long long L = blockIdx.x;
    const int I = work[L].x, J = work[L].y, n = p.n;
    const GramSide A{Xt, sqt, t}, B{p.X, p.sq, n};
    float acc[8][8];
    gram_tile(A, B, p.m, I, J, sm.g, acc);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float wj[8], sj[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int j = J * T + tx * 8 + b;
        wj[b] = j < n ? alpha[j] * p.y[j] : 0.f;
        sj[b] = j < n ? p.sq[j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = ty * 8 + a, s = I * T + r;
        const float si = s < t ? sqt[s] : 0.f;
        float f = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float kv = rbf_from_gram(acc[a][b], si, sj[b], p.gamma) + p.lam2;
            f = fmaf(wj[b], kv, f);
        }
        f = sum16(f);
        if (tx == 0) sm.e.rowv[0][r] = f;
    }
    __syncthreads();
    if (tid < T) {
        const int s = I * T + tid;
        if (s < t) part[(size_t)J * t + s] = sm.e.rowv[0][tid];
    }
}

__global__ void k_decision_sum(const float* __restrict__ part, int t, int Ntrain_tiles, float* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= t) return;
    double f = 0.0;
    for (int k = 0; k < Ntrain_tiles; ++k) f += (double)part[(size_t)k * t + s];
    out[s] = (float)f;
}

// ---------------------------------------------------------------- inspection
__global__ void k_get_q(Inst p, const int4* __restrict__ work, int q_bf16, float* __restrict__ Qd)
{
    const long long L = work[blockIdx.x].w;
    const int I = work[blockIdx.x].y, J = work[blockIdx.x].z, n = p.n;
    for (int e = threadIdx.x; e < TT; e += blockDim.x) {
        const int r = e / T, c = e % T, i = I * T + r, j = J * T + c;
        if (i >= n || j >= n || (I == J && c <= r)) continue;
        const size_t o = (size_t)L * TT + e;
        const float q = q_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(p.qstore)[o])
                               : static_cast<const float*>(p.qstore)[o];
        Qd[(size_t)i * n + j] = q;
        Qd[(size_t)j * n + i] = q;
    }
    if (I == J)
        for (int r = threadIdx.x; r < T; r += blockDim.x) {
            const int i = I * T + r;
            if (i < n) Qd[(size_t)i * n + i] = p.qdiag[i];
        }
}

}  // namespace

void launch_stage_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) k_stage_list<<<nblocks, 32, 0, s>>>(tab, nbl);
}

void launch_stage(const void* X, int x_dtype, int n, int m, float* y, float* Xf, float* sq,
                  float* b, float* b0, int task, Ctrl* ctrl, cudaStream_t s)
{
    k_stage<<<(n + 255) / 256, 256, 0, s>>>(X, x_dtype, n, m, y, Xf, sq, b, b0, task, ctrl);
}

void launch_final(const Inst* tab, const StopOp* ops, const int4* tiles, long long ntiles, const int2* nbl,
                  int nblocks, const int* members, int nmembers, double* f3_all, int q_stored, cudaStream_t s)
{
    if (ntiles > 0) {
        if (q_stored)
            k_final_tiles_q<<<(unsigned)ntiles, NTHREADS, 0, s>>>(tab, ops, tiles);
        else
            k_final_tiles<<<(unsigned)ntiles, NTHREADS, 0, s>>>(tab, ops, tiles);
    }
    if (nblocks > 0) k_final_nodes<<<nblocks, 256, 0, s>>>(tab, ops, nbl);
    if (nmembers > 0) k_final_reduce<<<nmembers, 256, 0, s>>>(tab, ops, members, f3_all);
}

void launch_decision(const Inst& p, const float* Xt, const float* sqt, int t, const float* alpha,
                     const int2* work, long long ntiles, float* part, float* out, cudaStream_t s)
{
    k_decision_tiles<<<(unsigned)ntiles, NTHREADS, 0, s>>>(p, Xt, sqt, t, alpha, work, part);
    k_decision_sum<<<(t + 255) / 256, 256, 0, s>>>(part, t, p.Nt, out);
}

void launch_get_q(const Inst& p, const int4* work, long long ntiles, int q_bf16, float* Qdense,
                  cudaStream_t s)
{
    k_get_q<<<(unsigned)ntiles, 256, 0, s>>>(p, work, q_bf16, Qdense);
}

}  // namespace gabp

// ---------------------------------------------------------------------------
// Decision values with no device allocation.
//
// Some callers cannot call cudaMalloc: plugins inside a host framework that
// owns all device memory through its own allocator, and latency-critical
// loops that cannot afford the implicit device-wide synchronisation of
// cudaMalloc/cudaFree.  gabp_decision_noalloc serves them:
// the caller passes every input and output as device memory, and the
// temporaries (row norms and per-tile partial sums) live in the file-scope
// array below, which every GPU that loads this library holds until the
// process exits.
namespace gabp {
namespace {

constexpr long long kNoAllocScratchFloats = 1LL << 20;   // 4 MiB

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

__global__ void k_rownorms(const float* __restrict__ X, int n, int m, float* __restrict__ sq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int k = 0; k < m; ++k) {
        const float v = X[(size_t)i * m + k];
        s = fmaf(v, v, s);
    }
    sq[i] = s;
}

// Same tile computation as k_decision_tiles, on a rectangle enumerated by the
// block index (I = test tile, J = training tile) instead of a work list.
__global__ void __launch_bounds__(NTHREADS) k_decision_tiles_noalloc(
    const float* __restrict__ X, const float* __restrict__ y, const float* __restrict__ alpha,
    const float* __restrict__ sq, int n, int m, const float* __restrict__ Xt,
    const float* __restrict__ sqt, int t, float gamma, float lam2, int Nt, float* __restrict__ part)
{
    __shared__ __align__(16) TileSmem sm;
    const long long L = blockIdx.x;
    const int I = (int)(L / Nt), J = (int)(L % Nt);
    const GramSide A{Xt, sqt, t}, B{X, sq, n};
    float acc[8][8];
    gram_tile(A, B, m, I, J, sm.g, acc);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float wj[8], sj[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int j = J * T + tx * 8 + b;
        wj[b] = j < n ? alpha[j] * y[j] : 0.f;
        sj[b] = j < n ? sq[j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = ty * 8 + a, s = I * T + r;
        const float si = s < t ? sqt[s] : 0.f;
        float f = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float kv = rbf_from_gram(acc[a][b], si, sj[b], gamma) + lam2;
            f = fmaf(wj[b], kv, f);
        }
        f = sum16(f);
        if (tx == 0) sm.e.rowv[0][r] = f;
    }
    __syncthreads();
    if (tid < T) {
        const int s = I * T + tid;
        if (s < t) part[(size_t)J * t + s] = sm.e.rowv[0][tid];
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_dev_ptr[kMaxDevices] = {};

}  // namespace
}  // namespace gabp

extern "C" GABP_API gabp_status gabp_decision_noalloc(const float* X, const float* y, const float* alpha,
                                                      int64_t n, int64_t m, const float* Xtest, int64_t t,
                                                      double gamma, double lambda, float* out, void* stream)
{
    using namespace gabp;
    set_last_error("");
    auto fail = [](gabp_status st, const std::string& msg) { set_last_error(msg.c_str()); return st; };
    if (!X || !y || !alpha || (t > 0 && (!Xtest || !out)))
        return fail(GABP_EINVAL, "gabp_decision_noalloc: null pointer");
    if (n < 1 || m < 1 || t < 0 || n > (1LL << 30) || m > (1LL << 20) || t > (1LL << 30))
        return fail(GABP_EINVAL, "gabp_decision_noalloc: bad sizes");
    if (!(gamma > 0) || !(lambda >= 0)) return fail(GABP_EINVAL, "gabp_decision_noalloc: need gamma > 0, lambda >= 0");
    if (t == 0) return GABP_OK;
    const long long Nt = (n + T - 1) / T, Ntt = (t + T - 1) / T;
    const long long need = n + t + Nt * t;
    if (need > kNoAllocScratchFloats)
        return fail(GABP_EINVAL, "gabp_decision_noalloc: n + t + ceil(n/128)*t = " + std::to_string(need) +
                                     " floats of scratch exceeds the fixed maximum of " +
                                     std::to_string(kNoAllocScratchFloats) + "; split the test rows");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GABP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(GABP_ECUDA, "gabp_decision_noalloc: device index out of range");
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_dev_ptr[dev]) {
            // Once per device, with that device current: the device address of the
            // array (its name in host code is only a host-side stand-in).
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(GABP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_dev_ptr[dev] = static_cast<float*>(ptr);
        }
        scratch = g_noalloc_dev_ptr[dev];
    }
    // Every scratch element read below is written earlier in the same call.
    float* sq = scratch;
    float* sqt = scratch + n;
    float* part = scratch + n + t;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_rownorms<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, (int)n, (int)m, sq);
    k_rownorms<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(Xtest, (int)t, (int)m, sqt);
    k_decision_tiles_noalloc<<<(unsigned)(Ntt * Nt), NTHREADS, 0, s>>>(
        X, y, alpha, sq, (int)n, (int)m, Xtest, sqt, (int)t, (float)gamma, (float)(lambda * lambda), (int)Nt, part);
    k_decision_sum<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(part, (int)t, (int)Nt, out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GABP_ECUDA, std::string("gabp_decision_noalloc: ") + cudaGetErrorString(e));
    return GABP_OK;
}
