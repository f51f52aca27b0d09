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
// 4 B of Q and writes 16 B.  Each CTA owns one 128 x 128 tile; warp w takes
// rows w, w+8, ...; lane l takes columns l, l+32, l+64, l+96, so every warp
// load or store of messages covers 512 contiguous bytes.  The next row's loads
// are issued before the current row's arithmetic and stores.  Row sums go
// through warp shuffles, column sums stay in registers and meet in shared
// memory, and each node's per-tile sums go to its own slot (common.cuh), so
// the reduction order is fixed and the result reproducible.
#include "common.cuh"

#include <float.h>

namespace gabp {

namespace {

template <typename QT>
struct RowData {
    float q[4];
    float4 s[4];
};

template <typename QT>
__device__ __forceinline__ void load_row(RowData<QT>& d, const QT* __restrict__ qt, const float4* st,
                                         int r, int lane, int cols, bool diag, bool zero)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = lane + 32 * k;
        const bool v = c < cols && (!diag || c > r);
        d.q[k] = v ? to_f(qt[r * T + c]) : 0.f;
        d.s[k] = (v && !zero) ? __ldcs(&st[r * T + c]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <typename QT>
__global__ void __launch_bounds__(NTHREADS, 2) k_sweep(Inst p, const int2* __restrict__ work)
{
    const Ctrl* ctrl = p.ctrl;
    if (*(volatile const int*)&ctrl->done) return;
    const int t = *(volatile const int*)&ctrl->t;
    const long long L = blockIdx.x;
    const int2 tile = work[L];
    const int I = tile.x, J = tile.y, n = p.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    __shared__ float sRow[3][T], sCol[3][T];
    __shared__ float sCp[NWARPS][T], sCh[NWARPS][T], sCr[NWARPS][T];
    __shared__ float sRp[T], sRh[T], sRr[T];

    const float* agg = p.agg + (size_t)(t & 1) * 3 * p.npad;
    {
        const int rc = tid < T ? tid : tid - T;
        const int x = (tid < T ? I : J) * T + rc;
        const bool v = x < n;
        float* dst0 = tid < T ? sRow[0] : sCol[0];
        float* dst1 = tid < T ? sRow[1] : sCol[1];
        float* dst2 = tid < T ? sRow[2] : sCol[2];
        dst0[rc] = v ? agg[x] : 1.f;
        dst1[rc] = v ? agg[p.npad + x] : 0.f;
        dst2[rc] = v ? agg[2 * p.npad + x] : 0.f;
    }
    __syncthreads();

    const int rows = min(T, n - I * T), cols = min(T, n - J * T);
    const bool diag = (I == J);
    const bool zero = (t == 0);   // Step 1: all messages 0, nothing to read
    float cP[4], cH[4], cM[4], aP[4], aH[4], aR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = lane + 32 * k;
        cP[k] = sCol[0][c];
        cH[k] = sCol[1][c];
        cM[k] = sCol[2][c];
        aP[k] = aH[k] = aR[k] = 0.f;
    }
    float4* st = p.state + (size_t)L * TT;
    const QT* qt = static_cast<const QT*>(p.qstore) + (size_t)L * TT;
    bool bad = false;

    RowData<QT> cur, nxt;
    int r = warp;
    if (r < rows) load_row(cur, qt, st, r, lane, cols, diag, zero);
    for (; r < rows; r += NWARPS) {
        const int rn = r + NWARPS;
        if (rn < rows) load_row(nxt, qt, st, rn, lane, cols, diag, zero);
        const float rP = sRow[0][r], rH = sRow[1][r], rM = sRow[2][r];
        float sp = 0.f, sh = 0.f, sr = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            const bool v = c < cols && (!diag || c > r);
            if (v) {
                const float q = cur.q[k];
                const float4 s = cur.s[k];       // {P_ij, P_ji, H_ij, H_ji}
                const float di = rP - s.y;       // Ptilde_i - P_ji
                const float dj = cP[k] - s.x;    // Ptilde_j - P_ij
                bad |= !(di > 0.f && di <= FLT_MAX && dj > 0.f && dj <= FLT_MAX);
                const float ii = __frcp_rn(di), ij = __frcp_rn(dj);
                const float q2 = q * q;
                const float nPij = -q2 * ii;
                const float nPji = -q2 * ij;
                const float nHij = -q * (rH - s.w) * ii;
                const float nHji = -q * (cH[k] - s.z) * ij;
                __stcs(&st[r * T + c], make_float4(nPij, nPji, nHij, nHji));
                sp += nPji;
                sh += nHji;
                sr = fmaf(q, cM[k], sr);
                aP[k] += nPij;
                aH[k] += nHij;
                aR[k] = fmaf(q, rM, aR[k]);
            }
        }
        sp = warp_sum(sp);
        sh = warp_sum(sh);
        sr = warp_sum(sr);
        if (lane == 0) { sRp[r] = sp; sRh[r] = sh; sRr[r] = sr; }
        if (rn < rows) cur = nxt;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = lane + 32 * k;
        sCp[warp][c] = aP[k];
        sCh[warp][c] = aH[k];
        sCr[warp][c] = aR[k];
    }
    if (bad) {
        Ctrl* cw = p.ctrl;
        if (atomicCAS(&cw->status, 0, (int)ST_ENUMERIC) == 0) cw->bad_index = (long long)I * T;
    }
    __syncthreads();

    float* partP = p.part;
    float* partH = partP + (size_t)p.Nt * n;
    float* partR = partH + (size_t)p.Nt * n;
    if (diag) {
        if (tid < rows) {
            float P = sRp[tid], H = sRh[tid], R = sRr[tid];
#pragma unroll
            for (int w = 0; w < NWARPS; ++w) { P += sCp[w][tid]; H += sCh[w][tid]; R += sCr[w][tid]; }
            const size_t o = (size_t)I * n + I * T + tid;
            partP[o] = P; partH[o] = H; partR[o] = R;
        }
    } else if (tid < T) {
        if (tid < rows) {
            const size_t o = (size_t)J * n + I * T + tid;
            partP[o] = sRp[tid]; partH[o] = sRh[tid]; partR[o] = sRr[tid];
        }
    } else {
        const int c = tid - T;
        if (c < cols) {
            float P = 0.f, H = 0.f, R = 0.f;
#pragma unroll
            for (int w = 0; w < NWARPS; ++w) { P += sCp[w][c]; H += sCh[w][c]; R += sCr[w][c]; }
            const size_t o = (size_t)I * n + J * T + c;
            partP[o] = P; partH[o] = H; partR[o] = R;
        }
    }
}

// Per node x: FP64 sums of its Nt slots (32 nodes x 8 slot groups per CTA),
// next aggregates, residual r_x(t), CTA max |r| -> ctrl, last CTA decides.
__global__ void __launch_bounds__(256) k_finalize(Inst p)
{
    Ctrl* ctrl = p.ctrl;
    if (*(volatile int*)&ctrl->done) return;
    const int t = *(volatile int*)&ctrl->t;
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int x = blockIdx.x * 32 + lane, n = p.n, Nt = p.Nt;
    const float* partP = p.part;
    const float* partH = partP + (size_t)Nt * n;
    const float* partR = partH + (size_t)Nt * n;
    double sP = 0.0, sH = 0.0, sR = 0.0;
    if (x < n)
        for (int k = g; k < Nt; k += 8) {
            const size_t o = (size_t)k * n + x;
            sP += (double)partP[o];
            sH += (double)partH[o];
            sR += (double)partR[o];
        }
    __shared__ double red[3][8][32];
    __shared__ int s_last;
    red[0][g][lane] = sP;
    red[1][g][lane] = sH;
    red[2][g][lane] = sR;
    __syncthreads();
    if (g == 0) {
        double absr = 0.0;
        if (x < n) {
            double P = 0.0, H = 0.0, R = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) { P += red[0][w][lane]; H += red[1][w][lane]; R += red[2][w][lane]; }
            const float* cur = p.agg + (size_t)(t & 1) * 3 * p.npad;
            float* nxt = p.agg + (size_t)((t + 1) & 1) * 3 * p.npad;
            const double qd = p.qdiag[x], bx = p.b[x];
            const float Pn = (float)(qd + P);
            const float hn = (float)(bx + H);
            const float mn = hn / Pn;
            nxt[x] = Pn;
            nxt[p.npad + x] = hn;
            nxt[2 * p.npad + x] = mn;
            const double r = bx - qd * (double)cur[2 * p.npad + x] - R;
            absr = fabs(r);
            if (!(absr <= DBL_MAX)) absr = INFINITY;
            if (!(Pn > 0.f) || !isfinite(mn)) {
                if (atomicCAS(&ctrl->status, 0, (int)ST_ENUMERIC) == 0) ctrl->bad_index = x;
            }
        }
        absr = warp_max_d(absr);
        if (lane == 0)
            atomicMax(&ctrl->rmax_bits, (unsigned long long)__double_as_longlong(absr));
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(&ctrl->blocks_done, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && tid == 0) {
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
        ctrl->t = t + 1;
        ctrl->rmax_bits = 0ull;
        ctrl->blocks_done = 0u;
        __threadfence();
    }
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
    double R = 0.0;
    for (int k = 0; k < p.Nt; ++k) R += (double)p.part[(size_t)k * p.n + x];
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
}

__global__ void k_begin(Ctrl* c, int iters, double tol)
{
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
    const long long L = I * Nt - I * (I - 1) / 2 + (J - I);
    const int r = (int)(i - I * T), c = (int)(j - J * T);
    out[e] = (p.ctrl->t == 0) ? make_float4(0.f, 0.f, 0.f, 0.f) : p.state[L * TT + r * T + c];
}

}  // namespace

void launch_init(const Inst& p, int diag_rule, float delta, cudaStream_t s)
{
    k_init<<<(p.n + 255) / 256, 256, 0, s>>>(p, diag_rule, delta);
}

void launch_begin(const Inst& p, int iters, double tol, cudaStream_t s)
{
    k_begin<<<1, 1, 0, s>>>(p.ctrl, iters, tol);
}

void launch_round(const Inst& p, const int2* work, long long ntiles, int q_mode, cudaStream_t s,
                  cudaEvent_t* ev)
{
    if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
    if (q_mode == 1)
        k_sweep<__nv_bfloat16><<<(unsigned)ntiles, NTHREADS, 0, s>>>(p, work);
    else
        k_sweep<float><<<(unsigned)ntiles, NTHREADS, 0, s>>>(p, work);
    if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
    k_finalize<<<(p.n + 31) / 32, 256, 0, s>>>(p);
}

void launch_get_pairs(const Inst& p, const long long* ij, long long cnt, float4* out, cudaStream_t s)
{
    if (cnt > 0) k_get_pairs<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(p, ij, cnt, out);
}

}  // namespace gabp
