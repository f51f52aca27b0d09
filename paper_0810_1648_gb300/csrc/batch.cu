// Batched and served forms: many GaBP SVM instances of uneven size swept
// together, one persistent launch per synchronous round for all of them.
//
// An Engine owns a device table of instances (Inst), their control blocks in
// one contiguous array (one copy reads every instance's progress), and the
// combined tile list and node-block list of the live instances.  A round is
// the same pair-sweep + finalize pair the single-instance solver uses; the
// kernels look each tile's instance up in the table and skip instances that
// have stopped, so a captured chunk of rounds stays valid while instances
// finish, leave and join.  Each instance keeps its own round counter,
// iteration limit, tolerance and stop decision (Algorithm 2, Step 3, per
// instance).
//
// gabp_batch_solve runs a fixed set to completion; gabp_server_* admits
// instances as they arrive, by device-memory budget, forms their Q on a side
// stream while the others keep sweeping, and retires them as they converge
// (continuous batching).  The end-of-solve work of the instances that stopped
// in a chunk (final residual, refinement restart, result copy) runs on a
// third stream during the next chunk; the round lists are rebuilt on the
// device from a membership mask.  The schedule knobs (persistent sweep CTAs
// per SM, rounds per convergence check) are chosen by measuring candidates on
// the actual set; results are cached per shape signature.  The engine of a
// thread's last gabp_batch_solve is kept for its next compatible call.
#include "common.cuh"
#include "gabp_svm.h"

#include <algorithm>
#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace gabp {

namespace {

size_t aup(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device memory of one instance (one allocation), carved like the handle's.
struct MemberPlan {
    size_t X, vec, agg, part, state, q, qref, rhist, final3, blockbuf, xp, xp3, total;
};

// alias_x: FP32 features in device memory are read in place (no copy).
// The total is a multiple of 1024 bytes, so instances can be packed into one
// allocation back to back.
MemberPlan member_plan(int64_t n, int64_t m, int q_mode, int msg_bf16, bool alias_x)
{
    const int Nt = (int)((n + T - 1) / T);
    const long long nt = tri_tiles(Nt);
    const size_t npad = aup((size_t)n, 128);
    MemberPlan p{};
    p.X = alias_x ? 0 : aup((size_t)n * m * 4, 256);
    p.vec = aup(npad * 4, 256);
    p.agg = aup(8 * npad * 4, 256);   // 2 x {P, h, mu} + staged {P, h}
    p.part = aup((size_t)4 * Nt * Nt * T * 4, 256);   // slot partials: Nt slots of T nodes per block row
    p.state = 2 * aup((size_t)nt * TT * (msg_bf16 ? 4 : 8), 256);
    p.q = q_mode == 0 ? aup((size_t)nt * TT * 4, 256) : q_mode == 1 ? aup((size_t)nt * TT * 2, 256) : 0;
    p.qref = q_mode == 1 ? aup((size_t)nt * TT * 4, 256) : 0;   // FP32 copy for the refinement residuals
    p.rhist = 0;
    p.final3 = 256;
    p.blockbuf = aup((size_t)3 * ((n + 31) / 32) * 8, 256);
    p.xp = q_mode != 0 ? aup(bf16_pack_bytes(Nt, (int)m), 1024) : 0;
    p.xp3 = aup(pack3_bytes(Nt, (int)m), 1024);   // the FP32 Gram's three BF16 planes
    p.total = aup(p.X + 10 * p.vec + p.agg + p.part + p.state + p.q + p.qref + p.final3 + p.blockbuf + p.xp + p.xp3 +
                  3072, 1024);
    return p;
}

struct Member {
    bool used = false;
    bool formed = false;     // Q formation finished (event)
    bool active = false;     // in the round lists
    bool finished = false;   // results available
    Inst inst{};
    void* mem = nullptr;
    size_t bytes = 0;
    long long ntiles = 0;
    int nblk = 0;
    float* alpha = nullptr;
    float* mu_acc = nullptr;
    float* r32 = nullptr;
    double* final3 = nullptr;
    double* blockbuf = nullptr;
    cudaEvent_t ready = nullptr;   // formation done (shared by the instances formed together)
    int evg = -1;                  // its group, while the instance still holds it
    // request bookkeeping
    int iters = 0;
    double tol = 0;
    int refine_left = 0;
    int refine_done = 0;
    bool refining = false;
    bool staged = false;     // rows checked and normed already (FP64 / device input)
    const void* src_x = nullptr;  // the caller's features (instances over the same ones share Gram tiles)
    int t_first_stop = 0;
    gabp_result res{};
    float* out_alpha = nullptr;  // caller buffer
    float* out_mu = nullptr;     // caller buffer for the unclipped means, or null
    int out_dev = 0;
    int64_t ticket = -1;
};

struct TuneKey {
    int q_mode;
    int msg_bf16;
    int nstages;
    long long tiles_bucket;
    int members_bucket;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(q_mode, msg_bf16, nstages, tiles_bucket, members_bucket) <
               std::tie(o.q_mode, o.msg_bf16, o.nstages, o.tiles_bucket, o.members_bucket);
    }
};
struct TuneVal {
    int ctas_per_sm;
    int chunk;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

// Host wall time of the phases of the last gabp_batch_solve (milliseconds).
struct BatchPhases {
    double form_ms, tune_ms, rounds_ms, stop_ms, total_ms;
    int64_t chunks, launches;
    double add_ms;   // host part of form_ms: allocating and enqueuing every instance
};
thread_local BatchPhases g_last_phases{};

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}


// Copies `count` words of W bytes from a host buffer the GPU reads coherently
// (pageable memory on a system with cudaDevAttrPageableMemoryAccess) into
// device memory; grid-stride.
template <class W>
__global__ void k_fetch(const W* __restrict__ src, W* __restrict__ dst, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// The round lists of the live instances (live[k] != 0), built on the device
// so that a membership change costs one small copy and one launch instead of
// host loops over every tile: tiles grouped by stage and, within a stage, by
// instance in slot order, each instance's tiles (I, J) of the stage's band
// I-major (the order the sweeps' results do not depend on, kept anyway);
// node blocks of the instances finalized one warp per block first; and every
// stage's Sched.  Every CTA computes all offsets (the instances go through in
// chunks of blockDim with a block-wide scan); instance k's entries are written
// by one warp of CTA k % gridDim.x, so the writing is spread over the GPU.
constexpr int kListThreads = 1024;

// Exclusive scan over the block (blockDim.x a multiple of 32, at most 1024):
// warp-shuffle scans, then one scan of the warp totals.  sc[blockDim.x - 1]
// holds the block's total afterwards, until the next call.
__device__ __forceinline__ long long block_scan_excl(long long v, long long* sc)
{
    __shared__ long long wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)blockDim.x >> 5;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    __syncthreads();   // wsum and sc of the previous call are consumed
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        wsum[lane] = w;   // inclusive scan of the warp totals
    }
    __syncthreads();
    const long long incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    sc[tid] = incl;
    __syncthreads();
    return incl - v;
}

__global__ void __launch_bounds__(kListThreads)
    k_build_lists(const Inst* __restrict__ tab, const int* __restrict__ live, int cap, int S,
                  int4* __restrict__ work, int2* __restrict__ nbl, Sched* __restrict__ sched)
{
    __shared__ long long sc[kListThreads];
    __shared__ long long m_off[kListThreads];
    __shared__ int m_k[kListThreads], m_a[kListThreads], m_b[kListThreads], m_c[kListThreads];
    __shared__ long long s_tiles[kMaxStages];
    __shared__ long long s_blocks[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)blockDim.x >> 5;
    // ---- tiles, stage by stage
    long long base = 0;
    for (int s = 0; s < S; ++s) {
        long long carry = 0;
        for (int c0 = 0; c0 < cap; c0 += (int)blockDim.x) {
            const int k = c0 + tid;
            long long cnt = 0;
            int Nt = 0, Bs = 0, Be = 0;
            if (k < cap && live[k]) {
                Nt = tab[k].Nt;
                int B[kMaxStages + 1];
                stage_bounds(Nt, S, B);
                Bs = B[s];
                Be = B[s + 1];
                const long long w = Be - Bs;
                cnt = (long long)Bs * w + w * (w + 1) / 2;
            }
            const long long ex = block_scan_excl(cnt, sc);
            m_off[tid] = base + carry + ex;
            m_k[tid] = cnt > 0 ? k : -1;
            m_a[tid] = Nt;
            m_b[tid] = Bs;
            m_c[tid] = Be;
            const long long total = sc[blockDim.x - 1];
            __syncthreads();
            for (int i = warp; i < (int)blockDim.x; i += nw) {
                if (m_k[i] < 0 || m_k[i] % (int)gridDim.x != (int)blockIdx.x) continue;
                const int kk = m_k[i], nt = m_a[i], bs = m_b[i], be = m_c[i];
                long long o = m_off[i];
                for (int I = 0; I < be; ++I) {
                    const int J0 = I > bs ? I : bs;
                    const long long Lrow = (long long)I * nt - (long long)I * (I - 1) / 2 - I;
                    for (int J = J0 + lane; J < be; J += 32)
                        work[o + (J - J0)] = make_int4(kk, I, J, (int)(Lrow + J));
                    o += be - J0;
                }
            }
            carry += total;
            __syncthreads();
        }
        if (tid == 0) s_tiles[s] = carry;
        base += carry;
    }
    // ---- node blocks: instances with at most kWarpFinNt tile rows first
    long long bbase = 0;
    for (int g = 0; g < 2; ++g) {
        long long carry = 0;
        for (int c0 = 0; c0 < cap; c0 += (int)blockDim.x) {
            const int k = c0 + tid;
            long long cnt = 0;
            if (k < cap && live[k]) {
                const int Nt = tab[k].Nt;
                if ((Nt <= kWarpFinNt) == (g == 0)) cnt = (tab[k].n + 31) / 32;
            }
            const long long ex = block_scan_excl(cnt, sc);
            m_off[tid] = bbase + carry + ex;
            m_k[tid] = cnt > 0 ? k : -1;
            m_a[tid] = (int)cnt;
            const long long total = sc[blockDim.x - 1];
            __syncthreads();
            for (int i = warp; i < (int)blockDim.x; i += nw) {
                if (m_k[i] < 0 || m_k[i] % (int)gridDim.x != (int)blockIdx.x) continue;
                for (int b = lane; b < m_a[i]; b += 32) nbl[m_off[i] + b] = make_int2(m_k[i], b);
            }
            carry += total;
            __syncthreads();
        }
        if (tid == 0) s_blocks[g] = carry;
        bbase += carry;
    }
    __syncthreads();
    if (blockIdx.x == 0 && tid < S) {
        long long off = 0;
        for (int s2 = 0; s2 < tid; ++s2) off += s_tiles[s2];
        Sched q{};
        q.ntiles = s_tiles[tid];
        q.nblocks = (int)(s_blocks[0] + s_blocks[1]);
        q.ninst = cap;
        q.off = off;
        q.nsmall = (int)s_blocks[0];
        sched[tid] = q;
    }
}

}  // namespace

// ---------------------------------------------------------------- Engine
class Engine {
  public:
    std::string err;
    gabp_status fail(gabp_status st, const std::string& m)
    {
        err = m;
        set_last_error(m.c_str());
        return st;
    }
#define EK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(GABP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    int q_mode = 0, diag_rule = 0, x_dtype = 0, ptr_mode = 0, msg_bf16 = 0, task = 0, bias_mode = 0;
    bool host_direct = false;   // the GPU reads pageable host memory coherently
    int nstages = 1;   // message schedule: 1 synchronous, > 1 staged
    double delta = 0.1, sv_threshold = 0.0, bias_lambda = 0.0;
    double handover = 1e-4, inner = 1e-2;   // refinement schedule
    double t_rebuild = 0;                    // host ms spent rebuilding the round lists
    int64_t rebuilds = 0;
    int cap_members = 0;
    long long cap_tiles = 0;
    int cap_nblk = 0;
    cudaStream_t stream = nullptr, side = nullptr;
    bool own_stream = false;
    Inst* d_tab = nullptr;
    Ctrl* d_ctrl = nullptr;
    int4* d_work = nullptr;
    int2* d_nbl = nullptr;
    Sched* d_sched = nullptr;
    int* d_live = nullptr;        // instances in the round lists (list build input)
    int* h_live = nullptr;        // its pinned mirror
    Ctrl* h_ctrl = nullptr;       // pinned mirror
    Inst* h_tab = nullptr;        // pinned staging of the instance table (uploaded per formation group)
    double* h_f3 = nullptr;       // pinned {residual, objective, #SV} per slot
    StopOp* h_ops = nullptr;      // pinned end-of-solve operations per slot
    StopOp* d_ops = nullptr;
    double* d_f3 = nullptr;
    int4* d_stop_tiles = nullptr; // lists of the instances being finished
    int2* d_stop_nbl = nullptr;
    int* d_stop_members = nullptr;
    int2* d_begin_list = nullptr;
    double* d_begin_tol = nullptr;
    int2* d_restart_list = nullptr;   // the refinement restarts' begin list (stop handling)
    double* d_restart_tol = nullptr;
    cudaStream_t sstream = nullptr;   // end-of-solve handling beside the rounds
    std::vector<Member> mem;
    RoundGrid grid{};
    int ctas_per_sm = 0;
    int chunk = 16;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<int> pending;     // added, Q not formed yet
    char* arena = nullptr;        // one allocation for a known set of instances (gabp_batch_solve)
    size_t arena_size = 0, arena_off = 0;
    struct EvGroup {
        cudaEvent_t ev = nullptr;
        int refs = 0;             // instances not yet activated or released
    };
    std::vector<EvGroup> evg;
    long long live_tiles = 0;     // tiles in the current lists
    bool lists_dirty = true;
    size_t bytes_in_use = 0;
    int64_t launches = 0;

    ~Engine()
    {
        if (stream) cudaStreamSynchronize(stream);
        if (side) cudaStreamSynchronize(side);
        if (sstream) cudaStreamSynchronize(sstream);
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        for (auto& m : mem) release(m);
        if (arena) cudaFreeAsync(arena, stream);
        if (stream) cudaStreamSynchronize(stream);
        if (d_tab) cudaFree(d_tab);
        for (auto& g : evg) cudaEventDestroy(g.ev);
        if (h_tab) cudaFreeHost(h_tab);
        if (h_live) cudaFreeHost(h_live);
        if (h_ctrl) cudaFreeHost(h_ctrl);
        if (h_f3) cudaFreeHost(h_f3);
        if (h_ops) cudaFreeHost(h_ops);
        if (side) cudaStreamDestroy(side);
        if (sstream) cudaStreamDestroy(sstream);
        if (rejoin_ev) cudaEventDestroy(rejoin_ev);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    gabp_status init(int members, long long tiles, int nblk, const gabp_svm_opts& o)
    {
        q_mode = o.q_mode;
        msg_bf16 = o.msg_bf16;
        task = o.task;
        nstages = o.stages > 1 ? o.stages : 1;
        bias_mode = o.bias_mode;
        bias_lambda = o.bias_lambda;
        diag_rule = o.diag_rule;
        delta = o.diag_delta > 0 ? o.diag_delta : 0.1;
        x_dtype = o.x_dtype;
        ptr_mode = o.ptr_mode;
        sv_threshold = o.sv_threshold;
        handover = refine_handover(o.refine_handover, o.msg_bf16);
        inner = refine_inner(o.refine_inner, o.msg_bf16);
        cap_members = members;
        cap_tiles = std::max<long long>(tiles, 1);
        cap_nblk = std::max(nblk, 1);
        if (o.stream) {
            stream = (cudaStream_t)o.stream;
        } else {
            EK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        EK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        {
            int dev = 0, pma = 0;
            EK(cudaGetDevice(&dev));
            if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) pma = 0;
            host_direct = pma != 0;
        }
        EK(cudaStreamCreateWithFlags(&sstream, cudaStreamNonBlocking));
        EK(cudaEventCreateWithFlags(&rejoin_ev, cudaEventDisableTiming));
        {
            // keep freed instance memory in the stream-ordered pool for reuse
            int dev = 0;
            cudaMemPool_t pool;
            EK(cudaGetDevice(&dev));
            EK(cudaDeviceGetDefaultMemPool(&pool, dev));
            uint64_t keep = UINT64_MAX;
            EK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        EK(prepare_sweep());
        if (q_mode == 2) EK(prepare_sweep_rc());
        const size_t b_tab = aup((size_t)cap_members * sizeof(Inst), 256);
        const size_t b_ctrl = aup((size_t)cap_members * sizeof(Ctrl), 256);
        const size_t b_work = aup((size_t)cap_tiles * sizeof(int4), 256);
        const size_t b_nbl = aup((size_t)cap_nblk * sizeof(int2), 256);
        const size_t b_ops = aup((size_t)cap_members * sizeof(StopOp), 256);
        const size_t b_f3 = aup((size_t)cap_members * 3 * sizeof(double), 256);
        const size_t b_mem = aup((size_t)cap_members * sizeof(int), 256);
        const size_t b_bl = aup((size_t)cap_members * sizeof(int2), 256);
        const size_t b_bt = aup((size_t)cap_members * sizeof(double), 256);
        char* base = nullptr;
        const size_t b_sched = aup((size_t)kMaxStages * sizeof(Sched), 256);
        const size_t b_live = aup((size_t)cap_members * sizeof(int), 256);
        EK(cudaMalloc((void**)&base,
                      b_tab + b_ctrl + 2 * b_work + 2 * b_nbl + b_ops + b_f3 + b_mem + 2 * b_bl + 2 * b_bt + b_sched + b_live));
        size_t off = 0;
        auto carve = [&](size_t bytes) { char* r = base + off; off += bytes; return r; };
        d_tab = (Inst*)carve(b_tab);
        d_ctrl = (Ctrl*)carve(b_ctrl);
        d_work = (int4*)carve(b_work);
        d_nbl = (int2*)carve(b_nbl);
        d_stop_tiles = (int4*)carve(b_work);
        d_stop_nbl = (int2*)carve(b_nbl);
        d_ops = (StopOp*)carve(b_ops);
        d_f3 = (double*)carve(b_f3);
        d_stop_members = (int*)carve(b_mem);
        d_begin_list = (int2*)carve(b_bl);
        d_begin_tol = (double*)carve(b_bt);
        d_restart_list = (int2*)carve(b_bl);
        d_restart_tol = (double*)carve(b_bt);
        d_sched = (Sched*)carve(b_sched);   // one per stage
        d_live = (int*)carve(b_live);
        EK(cudaMemsetAsync(d_ctrl, 0, b_ctrl, stream));
        EK(cudaMemsetAsync(d_sched, 0, b_sched, stream));
        EK(cudaMallocHost((void**)&h_ctrl, (size_t)cap_members * sizeof(Ctrl)));
        EK(cudaMallocHost((void**)&h_tab, (size_t)cap_members * sizeof(Inst)));
        EK(cudaMallocHost((void**)&h_live, (size_t)cap_members * sizeof(int)));
        EK(cudaMallocHost((void**)&h_f3, (size_t)cap_members * 3 * sizeof(double)));
        EK(cudaMallocHost((void**)&h_ops, (size_t)cap_members * sizeof(StopOp)));
        std::memset(h_ops, 0, (size_t)cap_members * sizeof(StopOp));
        mem.resize((size_t)cap_members);
        set_grid(0);
        EK(cudaStreamSynchronize(stream));
        return GABP_OK;
    }

    void set_grid(int cps)
    {
        ctas_per_sm = cps;
        grid = round_grid(cap_tiles, cap_nblk, q_mode, cps, msg_bf16);
    }

    void release(Member& m)
    {
        if (m.mem) cudaFreeAsync(m.mem, stream);
        drop_ready(m);
        if (m.used) bytes_in_use -= m.bytes;
        m = Member{};
    }

    // The instance no longer needs its formation event (its wait is enqueued,
    // or it is released); the event of a group is reused once all let go.
    void drop_ready(Member& m)
    {
        if (m.evg >= 0) --evg[(size_t)m.evg].refs;
        m.evg = -1;
    }

    bool alias_x() const { return ptr_mode == 1 && x_dtype == 0; }

    // Host-to-device copy of an input array.  Where the GPU reads pageable
    // host memory coherently (cudaDevAttrPageableMemoryAccess, e.g. a Grace
    // CPU over NVLink-C2C), unregistered host buffers are pulled by a kernel
    // instead of the driver's staged copy, which blocks the calling thread;
    // pinned or registered buffers go by DMA.
    gabp_status fetch(void* dst, const void* src, size_t bytes, cudaStream_t s)
    {
        cudaPointerAttributes a{};
        const bool pageable = host_direct && cudaPointerGetAttributes(&a, src) == cudaSuccess &&
                              a.type == cudaMemoryTypeUnregistered;
        cudaGetLastError();   // clear a failed attribute query
        if (!pageable || bytes % 4 != 0 || ((uintptr_t)src | (uintptr_t)dst) % 4 != 0) {
            EK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
            return GABP_OK;
        }
        // a few CTAs: enough loads in flight for the link, few SM slots taken
        // from the sweeps that run beside admission
        constexpr size_t kFetchCtas = 32;
        if ((((uintptr_t)src | (uintptr_t)dst) % 16) == 0 && bytes % 16 == 0) {
            const size_t c = bytes / 16;
            const unsigned g = (unsigned)std::min<size_t>((c + 255) / 256, kFetchCtas);
            k_fetch<uint4><<<std::max(1u, g), 256, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), c);
        } else {
            const size_t c = bytes / 4;
            const unsigned g = (unsigned)std::min<size_t>((c + 255) / 256, kFetchCtas);
            k_fetch<unsigned><<<std::max(1u, g), 256, 0, s>>>(static_cast<const unsigned*>(src),
                                                               static_cast<unsigned*>(dst), c);
        }
        EK(cudaGetLastError());
        ++launches;
        return GABP_OK;
    }
    // labels in device memory are read in place unless the task rewrites them
    bool alias_y() const { return ptr_mode == 1 && task != GABP_TASK_KRR; }

    // Instance memory of a known set in one allocation (carved by add()).
    gabp_status reserve(size_t bytes)
    {
        if (fault_mask() > 0 && (fault_mask() & FAULT_ALLOC))
            return fail(GABP_ENOMEM, "injected device allocation failure (GABP_FAULT=alloc)");
        EK(cudaMallocAsync((void**)&arena, bytes, side));
        arena_size = bytes;
        arena_off = 0;
        return GABP_OK;
    }

    // Whether this engine, kept from an earlier gabp_batch_solve of the same
    // thread, can serve a call with these sizes and options as it is.
    bool compatible(int members, long long tiles, int nblk, const gabp_svm_opts& o) const
    {
        const bool same_stream = o.stream ? (!own_stream && stream == (cudaStream_t)o.stream) : own_stream;
        return same_stream && members <= cap_members && cap_members <= 2 * members + 64 && tiles <= cap_tiles &&
               nblk <= cap_nblk && q_mode == o.q_mode && msg_bf16 == o.msg_bf16 && task == o.task &&
               nstages == (o.stages > 1 ? o.stages : 1) && bias_mode == o.bias_mode &&
               bias_lambda == o.bias_lambda && diag_rule == o.diag_rule &&
               delta == (o.diag_delta > 0 ? o.diag_delta : 0.1) && x_dtype == o.x_dtype && ptr_mode == o.ptr_mode &&
               sv_threshold == o.sv_threshold && handover == refine_handover(o.refine_handover, o.msg_bf16) &&
               inner == refine_inner(o.refine_inner, o.msg_bf16);
    }

    // Ready for the next call: no instances, zeroed control blocks, the
    // default schedule; buffers, streams, events and captured graphs stay.
    gabp_status reuse()
    {
        for (auto& m : mem) m = Member{};
        pending.clear();
        sb.stopped.clear();
        rejoin.clear();
        rejoin_event = false;
        for (auto& g : evg) g.refs = 0;
        lists_dirty = true;
        live_tiles = 0;
        bytes_in_use = 0;
        launches = 0;
        t_rebuild = 0;
        rebuilds = 0;
        chunk = 16;
        set_grid(0);
        std::memset(h_ops, 0, (size_t)cap_members * sizeof(StopOp));
        EK(cudaMemsetAsync(d_ctrl, 0, (size_t)cap_members * sizeof(Ctrl), stream));
        EK(cudaMemsetAsync(d_sched, 0, (size_t)kMaxStages * sizeof(Sched), stream));
        return GABP_OK;
    }

    // End of a call: instance memory back to the pool, every copy to the
    // caller's buffers done.
    gabp_status end_call()
    {
        EK(cudaStreamSynchronize(side));
        EK(cudaStreamSynchronize(sstream));
        for (auto& m : mem) release(m);
        if (arena) {
            EK(cudaFreeAsync(arena, stream));
            arena = nullptr;
            arena_size = arena_off = 0;
        }
        EK(cudaStreamSynchronize(stream));
        return GABP_OK;
    }

    int free_slot() const
    {
        for (int k = 0; k < cap_members; ++k)
            if (!mem[(size_t)k].used) return k;
        return -1;
    }

    // Allocates and forms one instance in `slot` on the side stream.
    gabp_status add(int slot, const gabp_problem& pr, float* out_alpha, float* out_mu, int out_dev)
    {
        Member& M = mem[(size_t)slot];
        const int64_t n = pr.n, m = pr.m;
        if (n < 2 || m < 1 || !pr.X || !pr.y) return fail(GABP_EINVAL, "problem needs n >= 2, m >= 1, X and y");
        if (!(pr.gamma > 0) || !(pr.gamma <= FLT_MAX) || !(pr.C > 0) || !std::isfinite(pr.C))
            return fail(GABP_EINVAL, "problem needs gamma in (0, FLT_MAX] and finite C > 0");
        const MemberPlan pl = member_plan(n, m, q_mode, msg_bf16, alias_x());
        M = Member{};
        M.used = true;
        M.bytes = pl.total;
        bytes_in_use += pl.total;
        cudaStream_t s = side;
        char* b = nullptr;
        if (arena) {
            if (arena_off + pl.total > arena_size) return fail(GABP_ENOMEM, "instance memory exhausted");
            b = arena + arena_off;
            arena_off += pl.total;
        } else {
            if (fault_mask() > 0 && (fault_mask() & FAULT_ALLOC)) {
                M = Member{};
                bytes_in_use -= pl.total;
                return fail(GABP_ENOMEM, "injected device allocation failure (GABP_FAULT=alloc)");
            }
            EK(cudaMallocAsync(&M.mem, pl.total, s));
            b = static_cast<char*>(M.mem);
        }
        size_t off = 0;
        auto take = [&](size_t bytes) { void* r = b + off; off += bytes; return r; };
        Inst& p = M.inst;
        p.n = (int)n;
        p.Nt = (int)((n + T - 1) / T);
        p.m = (int)m;
        p.npad = (int)aup((size_t)n, 128);
        p.X = alias_x() ? static_cast<const float*>(pr.X) : (const float*)take(pl.X);
        p.sq = (const float*)take(pl.vec);
        p.y = alias_y() ? pr.y : (const float*)take(pl.vec);
        p.b = (const float*)take(pl.vec);
        p.b0 = (const float*)take(pl.vec);
        p.qdiag = (float*)take(pl.vec);
        M.alpha = (float*)take(pl.vec);
        p.sqb = (const float*)take(pl.vec);
        M.mu_acc = (float*)take(pl.vec);
        M.r32 = (float*)take(pl.vec);
        p.sq3 = (float*)take(pl.vec);
        p.agg = (float*)take(pl.agg);
        p.aggmid = p.agg + (size_t)6 * p.npad;
        p.part = (float*)take(pl.part);
        p.nslot = (long long)p.Nt * p.Nt;   // dense slot layout
        p.srow = nullptr;
        p.tslot = nullptr;
        p.rsum = nullptr;
        p.Pst = take(pl.state / 2);
        p.Hst = take(pl.state / 2);
        p.msg_bf16 = msg_bf16;
        p.qstore = pl.q ? take(pl.q) : nullptr;
        p.qref = pl.qref ? (float*)take(pl.qref) : (q_mode == 0 ? (float*)p.qstore : nullptr);
        M.final3 = (double*)take(pl.final3);
        M.blockbuf = (double*)take(pl.blockbuf);
        p.nkc = bf16_chunks((int)m);
        if (pl.xp) {
            off = aup(off, 1024);
            p.Xp = take(pl.xp);
        }
        off = aup(off, 1024);
        p.Xp3 = take(pl.xp3);
        p.ctrl = d_ctrl + slot;
        p.rhist = nullptr;
        p.rhist_cap = 0;
        // bias feature lambda (Section 3): 1/n for the SVM, off for KRR unless set
        const double lam = bias_mode == 1 ? bias_lambda : (task == GABP_TASK_KRR ? 0.0 : 1.0 / (double)n);
        p.gamma = (float)pr.gamma;
        p.lam2 = (float)(lam * lam);
        p.C = (float)(task == GABP_TASK_KRR ? 1.0 / pr.C : pr.C);   // KRR: C is the ridge
        p.task = task;
        M.ntiles = tri_tiles(p.Nt);
        M.nblk = (int)((n + 31) / 32);
        M.out_alpha = out_alpha;
        M.out_mu = out_mu;
        M.out_dev = out_dev;
        M.src_x = pr.X;
        M.res.status = GABP_OK;
        M.res.alpha = out_alpha;
        M.res.mu = out_mu;
        // (the table entry and the control block are uploaded by form_pending)
        h_tab[slot] = p;
        if (!alias_y()) {
            if (ptr_mode) EK(cudaMemcpyAsync((void*)p.y, pr.y, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
            else if (gabp_status st = fetch((void*)p.y, pr.y, (size_t)n * 4, s)) return st;
        }
        if (x_dtype == 0) {
            // FP32 rows: read in place from device memory, else copied into X;
            // the batched staging of form_pending() checks them
            if (!alias_x())
                if (gabp_status st = fetch((void*)p.X, pr.X, (size_t)n * m * 4, s)) return st;
        } else {
            // FP64 / BF16 input: widen to FP32 and check now
            EK(cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s));
            const void* src = pr.X;
            void* tmp = nullptr;
            if (!ptr_mode) {
                EK(cudaMallocAsync(&tmp, (size_t)n * m * x_elem_bytes(x_dtype), s));
                if (gabp_status st = fetch(tmp, pr.X, (size_t)n * m * x_elem_bytes(x_dtype), s)) return st;
                src = tmp;
            }
            launch_stage(src, x_dtype, (int)n, (int)m, const_cast<float*>(p.y), (float*)p.X, (float*)p.sq,
                         (float*)p.b, const_cast<float*>(p.b0), p.task, p.ctrl, s);
            ++launches;
            if (tmp) EK(cudaFreeAsync(tmp, s));
            M.staged = true;
        }
        pending.push_back(slot);
        return GABP_OK;
    }

    // Forms Q for every instance added since the last call, one launch per
    // kernel over all of them (staging checks, BF16 packing, FP32 Gram / row
    // sums, diagonal rule + Step 1, tensor-core BF16 Q), on the side stream.
    gabp_status form_pending()
    {
        if (pending.empty()) return GABP_OK;
        NvtxRange nv("gabp.batch.formation");
        cudaStream_t s = side;
        // Instances over the same features (a parameter grid) are chained
        // behind the first: the FP32 and the tensor-core Gram tiles are
        // computed once for all (form_next goes up with the table entries).
        std::map<std::tuple<const void*, int, int>, int> tail;
        std::vector<int> leaders;
        for (int k : pending) {
            const Member& M = mem[(size_t)k];
            auto key = std::make_tuple(M.src_x, M.inst.n, M.inst.m);
            auto it = tail.find(key);
            h_tab[k].form_next = 0;
            if (it == tail.end()) {
                tail.emplace(key, k);
                leaders.push_back(k);
            } else {
                h_tab[it->second].form_next = k + 1;
                it->second = k;
            }
        }
        // table entries (one copy per run of consecutive slots) and control
        // blocks of the FP32-input instances (one memset per run)
        std::vector<int> sl(pending);
        std::sort(sl.begin(), sl.end());
        for (size_t a = 0; a < sl.size();) {
            size_t e = a + 1;
            while (e < sl.size() && sl[e] == sl[e - 1] + 1) ++e;
            EK(cudaMemcpyAsync(d_tab + sl[a], h_tab + sl[a], (e - a) * sizeof(Inst), cudaMemcpyHostToDevice, s));
            a = e;
        }
        for (size_t a = 0; a < sl.size();) {
            if (mem[(size_t)sl[a]].staged) { ++a; continue; }
            size_t e = a + 1;
            while (e < sl.size() && sl[e] == sl[e - 1] + 1 && !mem[(size_t)sl[e]].staged) ++e;
            EK(cudaMemsetAsync(d_ctrl + sl[a], 0, (e - a) * sizeof(Ctrl), s));
            a = e;
        }
        std::vector<int4> tiles_lead, diag_lead;
        std::vector<int2> nb, nb_stage;
        for (int k : leaders) {
            const int Nt = mem[(size_t)k].inst.Nt;
            int L = 0;
            for (int I = 0; I < Nt; ++I)
                for (int J = I; J < Nt; ++J, ++L) {
                    tiles_lead.push_back(make_int4(k, I, J, L));
                    if (I == J) diag_lead.push_back(make_int4(k, I, J, L));
                }
        }
        for (int k : pending) {
            const Member& M = mem[(size_t)k];
            for (int b = 0; b < M.nblk; ++b) {
                nb.push_back(make_int2(k, b));
                if (!M.staged) nb_stage.push_back(make_int2(k, b));
            }
        }
        int4* d_tl = nullptr;
        int4* d_dl = nullptr;
        int2* d_n = nullptr;
        int2* d_ns = nullptr;
        EK(cudaMallocAsync((void**)&d_tl, tiles_lead.size() * sizeof(int4) + 16, s));
        EK(cudaMallocAsync((void**)&d_dl, diag_lead.size() * sizeof(int4) + 16, s));
        EK(cudaMemcpyAsync(d_dl, diag_lead.data(), diag_lead.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        EK(cudaMallocAsync((void**)&d_n, nb.size() * sizeof(int2) + 16, s));
        EK(cudaMallocAsync((void**)&d_ns, nb_stage.size() * sizeof(int2) + 16, s));
        EK(cudaMemcpyAsync(d_tl, tiles_lead.data(), tiles_lead.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        EK(cudaMemcpyAsync(d_n, nb.data(), nb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        if (!nb_stage.empty())
            EK(cudaMemcpyAsync(d_ns, nb_stage.data(), nb_stage.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        launch_stage_list(d_tab, d_ns, (int)nb_stage.size(), s);
        if (q_mode != 0) EK(launch_pack_list(d_tab, d_n, (int)nb.size(), s));
        EK(launch_pack3_list(d_tab, d_n, (int)nb.size(), s));
        launch_form_norms(d_tab, d_dl, (long long)diag_lead.size(), s);
        launch_form_q(d_tab, d_tl, (long long)tiles_lead.size(), s);
        launch_init_list(d_tab, d_n, (int)nb.size(), diag_rule, (float)delta, s);
        if (q_mode == 1) EK(launch_form_q_tc(d_tab, d_tl, (long long)tiles_lead.size(), s));
        launches += q_mode == 0 ? 5 : (q_mode == 1 ? 7 : 6);
        EK(cudaGetLastError());
        size_t g = 0;
        while (g < evg.size() && evg[g].refs > 0) ++g;
        if (g == evg.size()) {
            evg.emplace_back();
            EK(cudaEventCreateWithFlags(&evg[g].ev, cudaEventDisableTiming));
        }
        EK(cudaEventRecord(evg[g].ev, s));
        evg[g].refs = (int)pending.size();
        for (int k : pending) {
            mem[(size_t)k].ready = evg[g].ev;
            mem[(size_t)k].evg = (int)g;
        }
        EK(cudaFreeAsync(d_tl, s));
        EK(cudaFreeAsync(d_dl, s));
        EK(cudaFreeAsync(d_n, s));
        EK(cudaFreeAsync(d_ns, s));
        // (pageable host-to-device copies return once the data is staged, so
        // the host lists may go out of scope; the kernels run on asynchronously)
        pending.clear();
        return GABP_OK;
    }

    // Arms several formed instances with one launch (their own iters / tol).
    gabp_status activate_list(const std::vector<int>& slots)
    {
        if (slots.empty()) return GABP_OK;
        std::vector<int2> bl;
        std::vector<double> bt;
        for (int k : slots) {
            Member& M = mem[(size_t)k];
            EK(cudaStreamWaitEvent(stream, M.ready, 0));
            drop_ready(M);
            const double t0 = (q_mode != 0 && M.refine_left > 0) ? std::max(M.tol, handover) : M.tol;
            bl.push_back(make_int2(k, M.iters));
            bt.push_back(t0);
            M.formed = true;
            M.active = true;
        }
        EK(cudaMemcpyAsync(d_begin_list, bl.data(), bl.size() * sizeof(int2), cudaMemcpyHostToDevice, stream));
        EK(cudaMemcpyAsync(d_begin_tol, bt.data(), bt.size() * sizeof(double), cudaMemcpyHostToDevice, stream));
        launch_begin_list(d_tab, d_begin_list, d_begin_tol, (int)bl.size(), stream);
        ++launches;
        lists_dirty = true;
        return GABP_OK;
    }

    gabp_status rebuild()
    {
        if (!lists_dirty) return GABP_OK;
        const auto t0 = std::chrono::steady_clock::now();
        struct Acc {   // host time of the list rebuilds
            double& t;
            std::chrono::steady_clock::time_point t0;
            ~Acc() { t += ms_since(t0); }
        } acc{t_rebuild, t0};
        ++rebuilds;
        // membership on the host, the lists themselves on the device (in
        // stream order before the next chunk)
        long long tiles = 0, blocks = 0;
        for (int k = 0; k < cap_members; ++k) {
            const Member& M = mem[(size_t)k];
            const bool in = M.used && M.active;
            h_live[k] = in ? 1 : 0;
            if (in) {
                tiles += M.ntiles;
                blocks += M.nblk;
            }
        }
        if (tiles > cap_tiles || blocks > cap_nblk) return fail(GABP_ENOMEM, "batch lists exceed their capacity");
        EK(cudaMemcpyAsync(d_live, h_live, (size_t)cap_members * sizeof(int), cudaMemcpyHostToDevice, stream));
        k_build_lists<<<std::max(1, std::min(cap_members, num_sms())), kListThreads, 0, stream>>>(
            d_tab, d_live, cap_members, nstages, d_work, d_nbl, d_sched);
        EK(cudaGetLastError());
        ++launches;
        live_tiles = tiles;
        lists_dirty = false;
        return GABP_OK;
    }

    gabp_status graph_for(int rounds, cudaGraphExec_t* out)
    {
        const int key = rounds * 16 + ctas_per_sm;
        auto it = graphs.find(key);
        if (it != graphs.end()) { *out = it->second; return GABP_OK; }
        cudaGraph_t g = nullptr;
        EK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < rounds; ++k)
            launch_round(d_tab, d_work, d_nbl, d_sched, nstages, grid, q_mode, msg_bf16, stream);
        EK(cudaStreamEndCapture(stream, &g));
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        EK(e);
        graphs[key] = ex;
        *out = ex;
        return GABP_OK;
    }

    // One captured chunk of rounds over the live lists, then every control
    // block read back; launch_chunk returns at once, wait_chunk waits.
    gabp_status launch_chunk(int rounds)
    {
        NvtxRange nv("gabp.batch.launch_rounds");
        if (gabp_status st = take_rejoin()) return st;
        if (gabp_status st = rebuild()) return st;
        if (live_tiles > 0) {
            cudaGraphExec_t g = nullptr;
            if (gabp_status st = graph_for(rounds, &g)) return st;
            EK(cudaGraphLaunch(g, stream));
            launches += 2LL * rounds;
        }
        EK(cudaMemcpyAsync(h_ctrl, d_ctrl, (size_t)cap_members * sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
        return GABP_OK;
    }
    gabp_status wait_chunk()
    {
        NvtxRange nv("gabp.batch.wait_rounds");
        EK(cudaStreamSynchronize(stream));
        return GABP_OK;
    }

    // Records the results of a stopped instance from its final residual /
    // objective / #SV (in h_f3) and queues the copy of alpha to the caller.
    gabp_status finish(int slot, const Ctrl& c, cudaStream_t ss)
    {
        Member& M = mem[(size_t)slot];
        const double* f3 = h_f3 + 3 * (size_t)slot;
        const cudaMemcpyKind kind = M.out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (M.out_alpha) EK(cudaMemcpyAsync(M.out_alpha, M.alpha, (size_t)M.inst.n * 4, kind, ss));
        // the means the final pass used (the refined accumulator or the round k* aggregates)
        if (M.out_mu && h_ops[(size_t)slot].mu)
            EK(cudaMemcpyAsync(M.out_mu, h_ops[(size_t)slot].mu, (size_t)M.inst.n * 4, kind, ss));
        M.res.residual_inf = f3[0];
        M.res.dual_objective = f3[1];
        M.res.n_support = (int64_t)std::llround(f3[2]);
        M.res.iters_done = c.t;
        // a stop on the tolerance (Step 3), confirmed by the final FP64-summed residual
        // (an unrefined BF16 solve stops on its own matrix; residual_inf is the FP32-Gram one)
        M.res.converged = M.refining ? (f3[0] < M.tol ? 1 : 0)
                                     : (c.converged && (q_mode != 0 || f3[0] < M.tol)) ? 1 : 0;
        M.res.refine_passes = M.refine_done;
        {
            double inv = 0.0;
            std::memcpy(&inv, &c.inv_margin_bits, sizeof inv);
            M.res.margin = inv > 0 ? 1.0 / inv : 0.0;
            M.res.err_bound = M.res.margin > 0 ? f3[0] / M.res.margin : INFINITY;
        }
        if (c.status == ST_ENUMERIC) M.res.status = GABP_ENUMERIC;
        else if (c.status == ST_EINVAL) M.res.status = GABP_EINVAL;
        else if (c.status == ST_ETIMEOUT) M.res.status = GABP_ETIMEOUT;
        else if (c.status != 0) M.res.status = GABP_ECUDA;
        M.finished = true;
        M.active = false;
        lists_dirty = true;
        return GABP_OK;
    }

    // End-of-solve handling of the instances that stopped in a chunk, in two
    // halves so that it can run on its own stream while the other instances
    // sweep the next chunk:
    //   stop_begin (after the chunk's control blocks were read): the stopped
    //     instances leave the lists; their final passes (refinement axpy,
    //     final residual / objective / #SV) are queued on `ss`, one launch per
    //     kernel over all of them;
    //   stop_end: waits for those passes and decides per instance: the next
    //     defect-correction pass (right-hand side and restart queued on `ss`;
    //     the instance rejoins the lists at the next chunk launch) or finish
    //     (results recorded, alpha copied to the caller's buffer on `ss`).
    struct StopBatch {
        std::vector<int> stopped;
        std::vector<char> ref;
        std::vector<Ctrl> snap;   // control blocks as the chunk left them
        std::vector<int4> tiles;
        std::vector<int2> nb;
    } sb;
    std::vector<int> rejoin;      // restarted, join the lists at the next launch
    bool rejoin_event = false;    // rejoin_ev orders their restart before that launch
    cudaEvent_t rejoin_ev = nullptr;

    gabp_status stop_begin(cudaStream_t ss, int* running)
    {
        NvtxRange nv("gabp.batch.stop_begin");
        int run = 0;
        sb.stopped.clear();
        sb.ref.clear();
        sb.snap.clear();
        sb.tiles.clear();
        sb.nb.clear();
        for (int k = 0; k < cap_members; ++k) {
            Member& M = mem[(size_t)k];
            if (!M.used || !M.active) continue;
            if (!h_ctrl[k].done) { ++run; continue; }
            sb.stopped.push_back(k);
        }
        if (running) *running = run;
        if (sb.stopped.empty()) return GABP_OK;
        // 1. final residual (and, in the precision form, the refined means)
        for (size_t u = 0; u < sb.stopped.size(); ++u) {
            const int k = sb.stopped[u];
            Member& M = mem[(size_t)k];
            const Ctrl& c = h_ctrl[k];
            sb.snap.push_back(c);
            M.active = false;
            lists_dirty = true;
            StopOp& op = h_ops[(size_t)k];
            op = StopOp{};
            op.alpha = M.alpha;
            op.blockbuf = M.blockbuf;
            op.final3 = M.final3;
            op.sv_threshold = (float)sv_threshold;
            const bool ref = c.status == 0 && q_mode != 0 && (M.refining || M.refine_left > 0);
            sb.ref.push_back(ref ? 1 : 0);
            if (ref) {
                // Defect correction on the FP32-Gram residual: accumulate the
                // means (or the correction) and form r = 1 - Q32 mu_acc.
                op.acc = M.mu_acc;
                op.axpy_buf = c.kstar;
                op.axpy_first = M.refining ? 0 : 1;
                op.mu = M.mu_acc;
                op.r_out = M.r32;
                if (M.refining) ++M.refine_done;
                M.refining = true;
            } else {
                op.mu = M.refining ? M.mu_acc
                                   : M.inst.agg + (size_t)(c.kstar & 1) * 3 * M.inst.npad + 2 * (size_t)M.inst.npad;
            }
            const int Nt = M.inst.Nt;
            int L = 0;
            for (int I = 0; I < Nt; ++I)
                for (int J = I; J < Nt; ++J, ++L) sb.tiles.push_back(make_int4(k, I, J, L));
            for (int b = 0; b < M.nblk; ++b) sb.nb.push_back(make_int2(k, b));
        }
        EK(cudaMemcpyAsync(d_ops, h_ops, (size_t)cap_members * sizeof(StopOp), cudaMemcpyHostToDevice, ss));
        EK(cudaMemcpyAsync(d_stop_tiles, sb.tiles.data(), sb.tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, ss));
        EK(cudaMemcpyAsync(d_stop_nbl, sb.nb.data(), sb.nb.size() * sizeof(int2), cudaMemcpyHostToDevice, ss));
        EK(cudaMemcpyAsync(d_stop_members, sb.stopped.data(), sb.stopped.size() * sizeof(int), cudaMemcpyHostToDevice,
                           ss));
        launch_axpy_list(d_tab, d_ops, d_stop_nbl, (int)sb.nb.size(), ss);
        launch_final(d_tab, d_ops, d_stop_tiles, (long long)sb.tiles.size(), d_stop_nbl, (int)sb.nb.size(),
                     d_stop_members, (int)sb.stopped.size(), d_f3, q_mode != 2, ss);   // FP32 tiles kept unless recomputing
        launches += 4;
        EK(cudaGetLastError());
        EK(cudaMemcpyAsync(h_f3, d_f3, (size_t)cap_members * 3 * sizeof(double), cudaMemcpyDeviceToHost, ss));
        return GABP_OK;
    }

    gabp_status stop_end(cudaStream_t ss, std::vector<int>* finished)
    {
        if (sb.stopped.empty()) return GABP_OK;
        NvtxRange nv("gabp.batch.stop_end");
        EK(cudaStreamSynchronize(ss));
        // 2. next correction pass, or done
        std::vector<int2> rnb, blist;
        std::vector<double> btol;
        for (size_t u = 0; u < sb.stopped.size(); ++u) {
            const int k = sb.stopped[u];
            Member& M = mem[(size_t)k];
            const double rn = h_f3[3 * (size_t)k];
            if (sb.ref[u] && rn >= M.tol && M.refine_left > 0) {
                // solve Q_bf d = r with the P messages kept (H restarted)
                --M.refine_left;
                for (int b = 0; b < M.nblk; ++b) rnb.push_back(make_int2(k, b));
                blist.push_back(make_int2(k, M.iters));
                btol.push_back(std::max(M.tol * 0.5, inner * rn));
                rejoin.push_back(k);
                continue;
            }
            const Ctrl& c = sb.snap[u];
            if (!sb.ref[u] && q_mode == 0 && c.status == 0 && c.converged && rn >= M.tol && c.t < M.iters) {
                // the in-round stop test (compensated FP32 sums) passed, the
                // final FP64-summed residual did not: the same solve goes on
                // from its current messages (Algorithm 2, Step 3)
                blist.push_back(make_int2(k, M.iters - c.t));
                btol.push_back(M.tol);
                rejoin.push_back(k);
                continue;
            }
            if (gabp_status st = finish(k, sb.snap[u], ss)) return st;
            if (finished) finished->push_back(k);
        }
        if (!blist.empty()) {
            if (!rnb.empty())
                EK(cudaMemcpyAsync(d_stop_nbl, rnb.data(), rnb.size() * sizeof(int2), cudaMemcpyHostToDevice, ss));
            EK(cudaMemcpyAsync(d_restart_list, blist.data(), blist.size() * sizeof(int2), cudaMemcpyHostToDevice, ss));
            EK(cudaMemcpyAsync(d_restart_tol, btol.data(), btol.size() * sizeof(double), cudaMemcpyHostToDevice, ss));
            launch_refine_rhs_list(d_tab, d_ops, d_stop_nbl, (int)rnb.size(), ss);
            launch_begin_list(d_tab, d_restart_list, d_restart_tol, (int)blist.size(), ss);
            launches += 2;
            EK(cudaGetLastError());
            if (ss != stream) {
                EK(cudaEventRecord(rejoin_ev, ss));
                rejoin_event = true;
            }
        }
        sb.stopped.clear();
        // (pageable host-to-device copies return once their data is staged,
        // so the host lists above may go out of scope)
        return GABP_OK;
    }

    // Restarted instances join the lists (before a chunk launch).
    gabp_status take_rejoin()
    {
        if (rejoin.empty()) return GABP_OK;
        if (rejoin_event) EK(cudaStreamWaitEvent(stream, rejoin_ev, 0));
        rejoin_event = false;
        for (int k : rejoin) mem[(size_t)k].active = true;
        rejoin.clear();
        lists_dirty = true;
        return GABP_OK;
    }

    // Instances not finished yet.
    int unfinished() const
    {
        int u = 0;
        for (const auto& M : mem) u += (M.used && !M.finished) ? 1 : 0;
        return u;
    }

    // Restart every active instance from Step 1 (used after tuning runs).
    gabp_status reset_all()
    {
        for (int k = 0; k < cap_members; ++k) {
            Member& M = mem[(size_t)k];
            if (!M.used || !M.active) continue;
            launch_reset(M.inst, stream);
            ++launches;
        }
        EK(cudaStreamSynchronize(stream));
        return GABP_OK;
    }

    // Picks sweep CTAs per SM and the chunk length by timing candidate
    // schedules for a few rounds of the real set (then restarts it).
    gabp_status autotune(int iters)
    {
        NvtxRange nv("gabp.batch.autotune");
        long long tiles = 0;
        int members = 0;
        for (auto& M : mem)
            if (M.used && M.active) { tiles += M.ntiles; ++members; }
        TuneKey key{q_mode, msg_bf16, nstages, tiles >> 8, members >> 3};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                set_grid(it->second.ctas_per_sm);
                chunk = it->second.chunk;
                return GABP_OK;
            }
        }
        const int probe = std::max(1, std::min(4, iters));
        std::vector<int> cands = q_mode == 2 ? std::vector<int>{1}
                                 : (msg_bf16 ? std::vector<int>{1, 2, 3} : std::vector<int>{1, 2});
        float best = 1e30f;
        int best_c = cands[0];
        cudaEvent_t e0, e1;
        EK(cudaEventCreate(&e0));
        EK(cudaEventCreate(&e1));
        double round_ms = 1.0;
        for (int c : cands) {
            set_grid(c);
            for (int k = 0; k < cap_members; ++k)
                if (mem[(size_t)k].used && mem[(size_t)k].active) launch_begin(d_tab + k, 1, probe, 0.0, stream);
            if (gabp_status st = rebuild()) return st;
            cudaGraphExec_t g = nullptr;
            if (gabp_status st = graph_for(probe, &g)) return st;
            EK(cudaEventRecord(e0, stream));
            EK(cudaGraphLaunch(g, stream));
            EK(cudaEventRecord(e1, stream));
            EK(cudaEventSynchronize(e1));
            float ms = 0.f;
            EK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_c = c; round_ms = ms / probe; }
            if (gabp_status st = reset_all()) return st;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_grid(best_c);
        // rounds per convergence check: keep the host check (~0.05 ms) under
        // about 2% of the rounds it covers, within [4, 64]
        int ch = 4;
        while (ch < 64 && 0.05 / (ch * round_ms) > 0.02) ch *= 2;
        chunk = ch;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneVal{best_c, chunk};
        return GABP_OK;
    }
};

// The engine of this thread's last gabp_batch_solve, kept for the next call
// with compatible sizes and options (its lists, tables, streams and captured
// round graphs are reused; instance memory is not kept).  Freed by
// gabp_batch_release; deliberately not destroyed at thread exit, where the
// CUDA runtime may already be shut down.
thread_local Engine* g_batch_engine = nullptr;

}  // namespace gabp

using gabp::Engine;
using gabp::ms_since;

extern "C" {

gabp_status gabp_batch_solve(const gabp_problem* probs, int64_t count, const gabp_svm_opts* opts, int32_t iters,
                             double tol, gabp_result* results)
{
    using namespace gabp;
    set_last_error("");
    if (!probs || !results || count < 1 || count > (1 << 20)) {
        set_last_error("gabp_batch_solve: need problems, results and 1 <= count <= 2^20");
        return GABP_EINVAL;
    }
    if (iters < 0 || std::isnan(tol)) {
        set_last_error("gabp_batch_solve: bad iters or tol");
        return GABP_EINVAL;
    }
    if (fault_mask() < 0) {
        set_last_error("GABP_FAULT holds an unknown token (known: alloc, nan, timeout)");
        return GABP_EINVAL;
    }
    gabp_svm_opts o;
    gabp_svm_opts_default(&o);
    if (opts) o = *opts;
    if (o.diag_delta == 0) o.diag_delta = 0.1;
    if (o.q_mode < 0 || o.q_mode > 2 || o.refine < 0 || o.refine > 64 || o.msg_bf16 < 0 || o.msg_bf16 > 1 ||
        (o.msg_bf16 && o.q_mode == 0) || o.task < 0 || o.task > 1 || o.stages < 0 || o.stages > kMaxStages ||
        o.sparse_tau != 0.f || o.x_dtype < 0 || o.x_dtype > 2 || o.ptr_mode < 0 || o.ptr_mode > 1 ||
        (o.bias_mode == 1 && (!(o.bias_lambda >= 0) || !(o.bias_lambda * o.bias_lambda <= FLT_MAX)))) {
        set_last_error("gabp_batch_solve: bad q_mode, refine, msg_bf16, task, x_dtype, ptr_mode or bias");
        return GABP_EINVAL;
    }
    long long tiles = 0, nblk = 0;
    size_t bytes = 0;
    for (int64_t k = 0; k < count; ++k) {
        const gabp_problem& p = probs[k];
        if (p.n < 2 || p.m < 1 || p.n > (1 << 30) || !p.X || !p.y || !(p.gamma > 0) ||
            !(p.gamma <= FLT_MAX) || !(p.C > 0) || !std::isfinite(p.C)) {
            set_last_error(("gabp_batch_solve: problem " + std::to_string(k) + " is invalid").c_str());
            return GABP_EINVAL;
        }
        const long long Nt = (p.n + T - 1) / T;
        tiles += tri_tiles(Nt);
        nblk += (p.n + 31) / 32;
        bytes += member_plan(p.n, p.m, o.q_mode, o.msg_bf16, o.ptr_mode == 1 && o.x_dtype == 0).total;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_last_error("no CUDA device");
        return GABP_ECUDA;
    }
    size_t free_b = 0;
    device_available(&free_b, false);   // instance memory comes from the stream-ordered pool
    if (bytes + ((size_t)512 << 20) > free_b) {
        set_last_error(("gabp_batch_solve: needs " + std::to_string(bytes / 1e9) + " GB of device memory").c_str());
        return GABP_ENOMEM;
    }
    using clk = std::chrono::steady_clock;
    const auto t_all = clk::now();
    BatchPhases ph{};
    std::unique_ptr<Engine> Ep;
    if (g_batch_engine && g_batch_engine->compatible((int)count, tiles, (int)nblk, o)) {
        Ep.reset(g_batch_engine);
        g_batch_engine = nullptr;
        if (gabp_status st = Ep->reuse()) return st;
    } else {
        delete g_batch_engine;
        g_batch_engine = nullptr;
        Ep.reset(new Engine);
        if (gabp_status st = Ep->init((int)count, tiles, (int)nblk, o)) return st;
    }
    Engine& E = *Ep;
    auto t0 = clk::now();
    if (gabp_status st = E.reserve(bytes)) return st;
    for (int64_t k = 0; k < count; ++k) {
        if (gabp_status st = E.add((int)k, probs[k], results[k].alpha, results[k].mu, o.ptr_mode)) return st;
        E.mem[(size_t)k].iters = iters;
        E.mem[(size_t)k].tol = tol;
        E.mem[(size_t)k].refine_left = o.q_mode != 0 ? o.refine : 0;
        E.mem[(size_t)k].ticket = k;
        // formation of each group of instances starts while the next are added
        if ((k + 1) % 64 == 0)
            if (gabp_status st = E.form_pending()) return st;
    }
    ph.add_ms = ms_since(t0);
    if (gabp_status st = E.form_pending()) return st;
    if (cudaStreamSynchronize(E.side) != cudaSuccess) return E.fail(GABP_ECUDA, "formation failed");
    // labels / features validated by the staging kernels
    if (cudaMemcpy(E.h_ctrl, E.d_ctrl, (size_t)count * sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return E.fail(GABP_ECUDA, "control read failed");
    for (int64_t k = 0; k < count; ++k)
        if (E.h_ctrl[k].status != 0)
            return E.fail(GABP_EINVAL, "problem " + std::to_string(k) + ": non-finite feature or label not +-1");
    {
        std::vector<int> all((size_t)count);
        for (int64_t k = 0; k < count; ++k) all[(size_t)k] = (int)k;
        if (gabp_status st = E.activate_list(all)) return st;
    }
    cudaStreamSynchronize(E.stream);
    ph.form_ms = ms_since(t0);
    t0 = clk::now();
    if (o.chunk <= 0) {
        if (gabp_status st = E.autotune(iters)) return st;
        const double t0 = (o.q_mode != 0 && o.refine > 0) ? std::max(tol, E.handover) : tol;
        for (int64_t k = 0; k < count; ++k) gabp::launch_begin(E.d_tab + k, 1, iters, t0, E.stream);
    } else {
        E.chunk = o.chunk;
    }
    ph.tune_ms = ms_since(t0);
    // The end-of-solve work of the instances that stopped in one chunk runs
    // on its own stream while the others sweep the next chunk; restarted
    // instances (refinement) join again one chunk later.
    const int max_loops = (int)(((long long)iters * (1 + o.refine)) / std::max(1, E.chunk) + 8 * (2 + o.refine) + 8);
    int running = (int)count;
    for (int loop = 0; loop < max_loops && running > 0; ++loop) {
        t0 = clk::now();
        if (gabp_status st = E.launch_chunk(E.chunk)) return st;
        ph.rounds_ms += ms_since(t0);
        t0 = clk::now();
        if (gabp_status st = E.stop_end(E.sstream, nullptr)) return st;
        ph.stop_ms += ms_since(t0);
        t0 = clk::now();
        if (gabp_status st = E.wait_chunk()) return st;
        ph.rounds_ms += ms_since(t0);
        t0 = clk::now();
        if (gabp_status st = E.stop_begin(E.sstream, nullptr)) return st;
        ph.stop_ms += ms_since(t0);
        running = E.unfinished();
        ++ph.chunks;
    }
    ph.launches = E.launches;
    ph.total_ms = ms_since(t_all);
    g_last_phases = ph;
    if (running > 0) return E.fail(GABP_ECUDA, "batch did not reach its stop condition");
    gabp_status worst = GABP_OK;
    for (int64_t k = 0; k < count; ++k) {
        gabp_result r = E.mem[(size_t)k].res;
        r.alpha = results[k].alpha;
        r.mu = results[k].mu;
        results[k] = r;
        if (r.status != GABP_OK && worst == GABP_OK) worst = (gabp_status)r.status;
    }
    if (gabp_status st = E.end_call()) return st;
    g_batch_engine = Ep.release();
    if (worst != GABP_OK) set_last_error("one or more problems failed; see their result status");
    return worst;
}

gabp_status gabp_batch_release(void)
{
    gabp::set_last_error("");
    delete gabp::g_batch_engine;
    gabp::g_batch_engine = nullptr;
    return GABP_OK;
}

gabp_status gabp_batch_last_phases(double* out7)
{
    if (!out7) return GABP_EINVAL;
    const gabp::BatchPhases& p = gabp::g_last_phases;
    out7[0] = p.form_ms;
    out7[1] = p.tune_ms;
    out7[2] = p.rounds_ms;
    out7[3] = p.stop_ms;
    out7[4] = p.total_ms;
    out7[5] = (double)p.chunks;
    out7[6] = p.add_ms;
    return GABP_OK;
}

// ------------------------------------------------------------------ server
struct gabp_server_s {
    Engine E;
    gabp_server_cfg cfg{};
    size_t budget = 0;
    std::deque<std::pair<int64_t, gabp_problem>> queue;
    std::map<int64_t, std::pair<float*, float*>> outs;   // {alpha, mu} caller buffers
    std::map<int64_t, gabp_result> done;
    std::deque<int64_t> fresh;   // finished, not yet reported by gabp_server_completed
    std::vector<int> forming;   // slots whose Q formation runs on the side stream
    int64_t next_ticket = 0;
    // host wall time (ms) per phase of gabp_server_step, since creation
    double t_admit = 0, t_activate = 0, t_rounds = 0, t_stop = 0, t_total = 0;
    int64_t steps = 0;
};

gabp_status gabp_server_create(const gabp_server_cfg* cfg, gabp_server_t* out)
{
    using namespace gabp;
    set_last_error("");
    if (!cfg || !out) { set_last_error("gabp_server_create: null argument"); return GABP_EINVAL; }
    *out = nullptr;
    gabp_server_cfg c = *cfg;
    if (c.max_members <= 0) c.max_members = 64;
    if (c.max_members > 4096 || c.iters < 0 || std::isnan(c.tol) || c.opts.q_mode < 0 || c.opts.q_mode > 2 ||
        (c.opts.msg_bf16 && c.opts.q_mode == 0) || c.opts.task < 0 || c.opts.task > 1 || c.opts.stages < 0 ||
        c.opts.stages > kMaxStages || c.opts.sparse_tau != 0.f || c.opts.x_dtype < 0 || c.opts.x_dtype > 2 ||
        c.opts.ptr_mode < 0 || c.opts.ptr_mode > 1 || (c.opts.bias_mode == 1 &&
         (!(c.opts.bias_lambda >= 0) || !(c.opts.bias_lambda * c.opts.bias_lambda <= FLT_MAX)))) {
        set_last_error("gabp_server_create: bad configuration");
        return GABP_EINVAL;
    }
    if (c.opts.diag_delta == 0) c.opts.diag_delta = 0.1;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { set_last_error("no CUDA device"); return GABP_ECUDA; }
    size_t free_b = 0;
    device_available(&free_b, false);   // instance memory comes from the stream-ordered pool
    size_t budget = c.hbm_budget_bytes > 0 ? (size_t)c.hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    if (budget + ((size_t)1 << 30) > free_b) budget = free_b > ((size_t)2 << 30) ? free_b - ((size_t)2 << 30) : 0;
    // list capacities: every tile of state costs TT * 16 bytes, so the budget bounds them
    const long long cap_tiles = (long long)(budget / ((size_t)TT * (c.opts.msg_bf16 ? 8 : 16))) + 1;
    const int cap_nblk = (int)std::min<long long>(cap_tiles * 4 + 1024, 1LL << 28);
    gabp_server_t s = new gabp_server_s();
    if (gabp_status st = s->E.init(c.max_members, cap_tiles, cap_nblk, c.opts)) { delete s; return st; }
    s->E.chunk = c.opts.chunk > 0 ? c.opts.chunk : 8;
    s->cfg = c;
    s->budget = budget;
    *out = s;
    return GABP_OK;
}

gabp_status gabp_server_submit(gabp_server_t s, const gabp_problem* p, float* alpha_out, int64_t* ticket)
{
    return gabp_server_submit_ex(s, p, alpha_out, nullptr, ticket);
}

gabp_status gabp_server_submit_ex(gabp_server_t s, const gabp_problem* p, float* alpha_out, float* mu_out,
                                  int64_t* ticket)
{
    gabp::set_last_error("");
    if (!s || !p || !ticket) { gabp::set_last_error("gabp_server_submit: null argument"); return GABP_EINVAL; }
    if (p->n < 2 || p->m < 1 || !p->X || !p->y || !(p->gamma > 0) || !(p->gamma <= FLT_MAX) || !(p->C > 0) ||
        !std::isfinite(p->C)) {
        gabp::set_last_error("gabp_server_submit: invalid problem");
        return GABP_EINVAL;
    }
    const int64_t t = s->next_ticket++;
    s->queue.emplace_back(t, *p);
    s->outs[t] = std::make_pair(alpha_out, mu_out);
    *ticket = t;
    return GABP_OK;
}

gabp_status gabp_server_step(gabp_server_t s, int32_t* active, int32_t* queued, int32_t* completed)
{
    using namespace gabp;
    set_last_error("");
    if (!s) { set_last_error("gabp_server_step: null server"); return GABP_EINVAL; }
    Engine& E = s->E;
    using clk = std::chrono::steady_clock;
    const auto t_step = clk::now();
    auto t0 = t_step;
    // 1. one chunk of rounds over every live instance (with the ones the
    //    previous step restarted): launched now, waited for after the work
    //    below, which overlaps it
    if (gabp_status st = E.take_rejoin()) return st;
    bool any = false;
    for (auto& M : E.mem) any |= (M.used && M.active);
    if (any) {
        if (gabp_status st = E.launch_chunk(E.chunk)) return st;
        s->t_rounds += ms_since(t0);
    }
    // 1b. the instances that stopped in the previous chunk: results or the
    //     next refinement pass (their final passes ran on the stop stream)
    {
        t0 = clk::now();
        std::vector<int> fin;
        if (gabp_status st = E.stop_end(E.sstream, &fin)) return st;
        if (!fin.empty()) {
            // alpha copies done before the memory is released
            if (cudaStreamSynchronize(E.sstream) != cudaSuccess) return E.fail(GABP_ECUDA, "result copies failed");
            for (int slot : fin) {
                Member& M = E.mem[(size_t)slot];
                gabp_result r = M.res;
                r.alpha = M.out_alpha;
                r.mu = M.out_mu;
                s->done[M.ticket] = r;
                s->fresh.push_back(M.ticket);
                E.release(M);
            }
        }
        s->t_stop += ms_since(t0);
    }
    // 2. admission, first come first served, by device-memory budget and free
    //    slots; formation on the side stream
    t0 = clk::now();
    while (!s->queue.empty()) {
        const auto& front = s->queue.front();
        const size_t need = member_plan(front.second.n, front.second.m, s->cfg.opts.q_mode, s->cfg.opts.msg_bf16,
                                        E.alias_x()).total;
        if (need > s->budget) {
            gabp_result r{};
            r.status = GABP_ENOMEM;
            r.alpha = s->outs[front.first].first;
            r.mu = s->outs[front.first].second;
            s->done[front.first] = r;
            s->fresh.push_back(front.first);
            s->queue.pop_front();
            continue;
        }
        const int slot = E.free_slot();
        if (slot < 0 || E.bytes_in_use + need > s->budget) break;
        const int64_t t = front.first;
        if (gabp_status st = E.add(slot, front.second, s->outs[t].first, s->outs[t].second, s->cfg.opts.ptr_mode)) {
            if (st != GABP_ENOMEM) return st;
            // the instance's memory could not be had: the request completes with
            // GABP_ENOMEM and the server goes on with the others
            gabp_result r{};
            r.status = GABP_ENOMEM;
            r.alpha = s->outs[t].first;
            r.mu = s->outs[t].second;
            s->done[t] = r;
            s->fresh.push_back(t);
            s->queue.pop_front();
            continue;
        }
        Member& M = E.mem[(size_t)slot];
        M.ticket = t;
        M.iters = s->cfg.iters;
        M.tol = s->cfg.tol;
        M.refine_left = s->cfg.opts.q_mode != 0 ? s->cfg.opts.refine : 0;
        s->forming.push_back(slot);
        s->queue.pop_front();
    }
    if (gabp_status st = E.form_pending()) return st;
    s->t_admit += ms_since(t0);
    // 3. end of the chunk: the instances that stopped leave the lists, their
    //    final passes go to the stop stream (finished at the next step)
    if (any) {
        t0 = clk::now();
        if (gabp_status st = E.wait_chunk()) return st;
        s->t_rounds += ms_since(t0);
        t0 = clk::now();
        if (gabp_status st = E.stop_begin(E.sstream, nullptr)) return st;
        s->t_stop += ms_since(t0);
    }
    // 4. instances whose Q is ready join the sweeps from the next chunk
    t0 = clk::now();
    std::vector<int> ready;
    for (size_t k = 0; k < s->forming.size();) {
        const int slot = s->forming[k];
        cudaError_t q = cudaEventQuery(E.mem[(size_t)slot].ready);
        if (q == cudaSuccess) {
            ready.push_back(slot);
            s->forming.erase(s->forming.begin() + (long)k);
        } else if (q == cudaErrorNotReady) {
            ++k;
        } else {
            return E.fail(GABP_ECUDA, std::string("formation: ") + cudaGetErrorString(q));
        }
    }
    if (gabp_status st = E.activate_list(ready)) return st;
    s->t_activate += ms_since(t0);
    s->t_total += ms_since(t_step);
    ++s->steps;
    int act = 0;
    for (auto& M : E.mem) act += M.used ? 1 : 0;
    if (active) *active = act;
    if (queued) *queued = (int32_t)s->queue.size();
    if (completed) *completed = (int32_t)s->done.size();
    return GABP_OK;
}

gabp_status gabp_server_poll(gabp_server_t s, int64_t ticket, gabp_result* res, int32_t* done)
{
    gabp::set_last_error("");
    if (!s || !done) { gabp::set_last_error("gabp_server_poll: null argument"); return GABP_EINVAL; }
    auto it = s->done.find(ticket);
    *done = it != s->done.end() ? 1 : 0;
    if (*done && res) *res = it->second;
    return GABP_OK;
}

gabp_status gabp_server_completed(gabp_server_t s, int64_t* tickets, int32_t cap, int32_t* count)
{
    gabp::set_last_error("");
    if (!s || !count || (cap > 0 && !tickets) || cap < 0) {
        gabp::set_last_error("gabp_server_completed: bad argument");
        return GABP_EINVAL;
    }
    int32_t k = 0;
    while (k < cap && !s->fresh.empty()) {
        tickets[k++] = s->fresh.front();
        s->fresh.pop_front();
    }
    *count = k;
    return GABP_OK;
}

gabp_status gabp_server_phases(gabp_server_t s, double* out8)
{
    gabp::set_last_error("");
    if (!s || !out8) { gabp::set_last_error("gabp_server_phases: null argument"); return GABP_EINVAL; }
    out8[0] = s->t_admit;
    out8[1] = s->t_activate;
    out8[2] = s->E.t_rebuild;
    out8[3] = s->t_rounds - s->E.t_rebuild;
    out8[4] = s->t_stop;
    out8[5] = s->t_total;
    out8[6] = (double)s->steps;
    out8[7] = (double)s->E.rebuilds;
    return GABP_OK;
}

gabp_status gabp_server_destroy(gabp_server_t s)
{
    gabp::set_last_error("");
    delete s;
    return GABP_OK;
}

}  // extern "C"
