// C ABI of the GaBP SVM solver (declared in include/gabp_svm.h): handle
// lifetime, argument checks, the device memory plan, the solve loop with its
// captured CUDA graphs, and the host-side views of the results.  All
// arithmetic of the method runs in the kernels of gram.cu and sweep.cu.
#include "common.cuh"
#include "gabp_svm.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

using namespace gabp;

namespace {

thread_local std::string g_err;

gabp_status fail(gabp_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
gabp_status fail(gabp_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(GABP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
    } while (0)

constexpr int kRhistCap = 1 << 16;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

void gabp::set_last_error(const char* msg) { g_err = msg; }

cudaError_t gabp::device_available(size_t* avail, bool trim)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e != cudaSuccess) return e;
    if (trim) {
        e = cudaMemPoolTrimTo(pool, 0);
        if (e != cudaSuccess) return e;
    }
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return e;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        reserved = used = 0;
    }
    *avail = free_b + (reserved > used ? (size_t)(reserved - used) : 0);
    return cudaSuccess;
}

int gabp::fault_mask()
{
    const char* v = std::getenv("GABP_FAULT");
    if (!v || !*v) return 0;
    int bits = 0;
    std::string tok;
    for (const char* c = v;; ++c) {
        if (*c == ',' || *c == 0) {
            if (tok == "alloc") bits |= FAULT_ALLOC;
            else if (tok == "nan") bits |= FAULT_NAN;
            else if (tok == "timeout") bits |= FAULT_TIMEOUT;
            else if (!tok.empty()) return -1;
            tok.clear();
            if (*c == 0) break;
        } else {
            tok += *c;
        }
    }
    return bits;
}

struct gabp_svm_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gabp_svm_opts opts{};
    int64_t n = 0, m = 0;
    int Nt = 0, npad = 0;
    long long ntiles = 0;
    double gamma = 0, C = 0, lambda = 0, delta = 0;
    void* pool = nullptr;
    size_t pool_bytes = 0;
    // tile-sparse option: the message state and Q of the kept tiles live in a
    // second allocation sized after the tile-maxima pass (grown on refit)
    void* spool = nullptr;
    size_t spool_bytes = 0;
    float* tilemax = nullptr;       // per-tile maxima (formation's first pass)
    int* slab = nullptr;            // slab of every tile in the compacted storage, -1 = dropped
    int* srow = nullptr;            // compacted slot space: block row I owns [srow[I], srow[I + 1])
    int2* tslot = nullptr;          // slots {row role, column role} of each kept tile (by slab)
    double* rsum = nullptr;         // the whole matrix's sum_{j != i} |Q_ij| (first pass), per node
    long long nslot = 0;            // slots of the compacted slot space
    Inst inst{};
    Inst* d_tab = nullptr;          // device copy of inst (a one-instance batch)
    int4* work_all = nullptr;       // every tile {0, I, J, L}, row by row (formation)
    int4* work = nullptr;           // the swept tiles, grouped by stage (= work_all's tiles when dense)
    int4* work_diag = nullptr;      // the diagonal tiles {0, I, I, L} (the tensor-core norms pass)
    long long nlive = 0;            // tiles in `work`
    int2* nbl = nullptr;            // node blocks {0, b}
    Sched* sched = nullptr;   // one per stage
    int nstages = 1;
    StopOp* d_ops = nullptr;        // end-of-solve operation of the one instance
    int* d_members = nullptr;       // {0}
    RoundGrid grid{};
    float* alpha = nullptr;
    double* final3 = nullptr;
    double* blockbuf = nullptr;
    Ctrl* hctrl = nullptr;          // pinned mirror of the control block
    double* hfinal = nullptr;       // pinned {rinf, objective, nsv}
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> ev;   // 2 per bracketed round when captured with profiling on
    };
    std::map<std::pair<int, int>, Graph> graphs;   // by (rounds, profiling stride)
    int profiling = 0;   // 0 off, k >= 1: the pair sweep of every k-th round is bracketed by events
    gabp_svm_profile prof{};
    bool solved = false;
    bool formed = false;            // the last create/refit formed Q completely (else only refit/destroy are valid)
    int kstar = 0;
    float* mu_acc = nullptr;        // refined means (precision form)
    float* r32 = nullptr;           // FP32 residual of the accurate matrix (refinement)
    const float* mean_src = nullptr;  // device array holding the means of the last solve
    gabp_svm_stats stats{};
};

namespace {

gabp_status check_handle(gabp_svm_t h)
{
    if (!h) return fail(GABP_EINVAL, "null handle");
    return GABP_OK;
}

// Handle whose last create/refit completed (a failed refit leaves only
// refit and destroy valid).
gabp_status check_formed(gabp_svm_t h)
{
    if (gabp_status s = check_handle(h)) return s;
    if (!h->formed) return fail(GABP_ESTATE, "the last refit failed; refit again before using the handle");
    return GABP_OK;
}

// Device memory plan of one handle (bytes, 256-aligned sub-buffers).
struct Plan {
    size_t X, vec, agg, part, state, q, qref, work, tilemax, sparse, ctrl, rhist, final3, blockbuf, xp, xp3, tab, nbl,
        total;
};

// Bytes of the per-pair arrays (messages, stored Q, FP32 copy) for `tiles` tiles.
size_t pair_bytes(long long tiles, int q_mode, int msg_bf16)
{
    const size_t tt = (size_t)tiles * TT;
    return 2 * align_up(tt * (msg_bf16 ? 4 : 8), 256) +
           (q_mode == GABP_Q_F32 ? align_up(tt * 4, 256) : q_mode == GABP_Q_BF16 ? align_up(tt * 2, 256) : 0) +
           (q_mode == GABP_Q_BF16 ? align_up(tt * 4, 256) : 0);
}

// Bytes of the four slot-partial arrays for `nslot` slots of T nodes.
size_t part_bytes(long long nslot) { return align_up((size_t)4 * nslot * T * sizeof(float), 256); }

Plan make_plan(int64_t n, int64_t m, int Nt, long long ntiles, int npad, int q_mode, int msg_bf16, bool sparse)
{
    Plan p{};
    // the tile-sparse option keeps a second tile list (the swept tiles), the
    // tile maxima, the slab map, the compacted slot space (srow, tslot) and
    // the first pass's row sums; its per-pair arrays and slot partials are
    // allocated later, for the kept tiles only (pair_bytes, part_bytes)
    p.tilemax = sparse ? 2 * align_up((size_t)ntiles * sizeof(float), 256) : 0;
    p.sparse = sparse ? align_up((size_t)(Nt + 1) * sizeof(int), 256) + align_up((size_t)ntiles * sizeof(int2), 256) +
                            align_up((size_t)n * sizeof(double), 256)
                      : 0;
    p.xp = q_mode != GABP_Q_F32 ? align_up(bf16_pack_bytes(Nt, (int)m), 1024) : 0;
    p.xp3 = align_up(pack3_bytes(Nt, (int)m), 1024);   // the FP32 Gram's three BF16 planes
    p.X = align_up((size_t)n * m * sizeof(float), 256);
    p.vec = align_up((size_t)npad * sizeof(float), 256);
    p.agg = align_up((size_t)8 * npad * sizeof(float), 256);   // 2 x {P, h, mu} + staged {P, h}
    p.part = sparse ? 0 : part_bytes((long long)Nt * Nt);
    const long long dense_tiles = sparse ? 0 : ntiles;
    p.state = 2 * align_up((size_t)dense_tiles * TT * (msg_bf16 ? 4 : 8), 256);
    p.q = q_mode == GABP_Q_F32 ? align_up((size_t)dense_tiles * TT * sizeof(float), 256)
        : q_mode == GABP_Q_BF16 ? align_up((size_t)dense_tiles * TT * sizeof(__nv_bfloat16), 256)
        : 0;
    // the BF16 store keeps an FP32 copy for the refinement residuals
    p.qref = q_mode == GABP_Q_BF16 ? align_up((size_t)dense_tiles * TT * sizeof(float), 256) : 0;
    p.work = (sparse ? 2 : 1) * align_up((size_t)ntiles * sizeof(int4), 256) + align_up((size_t)Nt * sizeof(int4), 256);
    p.tab = align_up(align_up(sizeof(Inst), 16) + kMaxStages * align_up(sizeof(Sched), 16) + sizeof(StopOp) + 64, 256);
    p.nbl = align_up((size_t)((n + 31) / 32) * sizeof(int2), 256);
    p.ctrl = align_up(sizeof(Ctrl), 256);
    p.rhist = align_up((size_t)kRhistCap * sizeof(double), 256);
    p.final3 = 256;
    p.blockbuf = align_up((size_t)3 * ((n + 31) / 32) * sizeof(double), 256);
    p.total = p.X + 10 * p.vec + p.agg + p.part + p.state + p.q + p.qref + p.work + p.tilemax + p.sparse + p.ctrl + p.rhist +
              p.final3 + p.blockbuf + p.xp + p.xp3 + p.tab + p.nbl + 2048;
    return p;
}

void clear_graphs(gabp_svm_t h)
{
    for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto e : kv.second.ev) cudaEventDestroy(e);
    }
    h->graphs.clear();
}

// The swept tile list after formation.  Dense: every tile (the list built at
// create, grouped by stage).  Tile-sparse: the diagonal tiles and every tile
// whose largest |Q_ij| exceeds sparse_tau, grouped by stage, each given the
// next slab of the compacted per-pair storage (h->slab maps every tile to its
// slab, -1 for a dropped one).  The diagonal rule keeps the row sums of the
// whole matrix, so dropping a tile changes only its own entries (and the
// matrix stays diagonally dominant).
gabp_status build_sweep_list(gabp_svm_t h)
{
    h->stats.tiles_total = h->ntiles;
    if (!(h->opts.sparse_tau > 0)) {
        h->nlive = h->ntiles;
        h->stats.tiles_kept = h->ntiles;
        return GABP_OK;
    }
    cudaStream_t s = h->stream;
    std::vector<float> mx((size_t)h->ntiles);
    CK(cudaMemcpyAsync(mx.data(), h->tilemax, mx.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int Nt = h->Nt;
    auto L_of = [Nt](int I, int J) { return (long long)I * Nt - (long long)I * (I - 1) / 2 + (J - I); };
    const float tau = h->opts.sparse_tau;
    std::vector<int4> wl;
    std::vector<int> slab((size_t)h->ntiles, -1);
    int B[kMaxStages + 1];
    stage_bounds(Nt, h->nstages, B);
    const int nblk = (int)((h->n + 31) / 32);
    Sched sc[kMaxStages];
    for (int st = 0; st < h->nstages; ++st) {
        const long long off = (long long)wl.size();
        for (int I = 0; I < Nt; ++I)
            for (int J = std::max(I, B[st]); J < B[st + 1]; ++J) {
                const long long L = L_of(I, J);
                if (I == J || mx[(size_t)L] > tau) {
                    slab[(size_t)L] = (int)wl.size();
                    wl.push_back(make_int4(0, I, J, (int)wl.size()));
                }
            }
        sc[st] = Sched{(long long)wl.size() - off, nblk, 1, off, Nt <= kWarpFinNt ? nblk : 0, 0};
    }
    h->nlive = (long long)wl.size();
    h->stats.tiles_kept = h->nlive;
    // compacted slot space: block row I's slots are its kept tiles (row or
    // column block I) in the order of their other block index
    std::vector<int> cnt((size_t)Nt + 1, 0), srow((size_t)Nt + 1, 0);
    std::vector<std::vector<int>> other((size_t)Nt);
    for (const int4& w : wl) {
        other[(size_t)w.y].push_back(w.z);
        if (w.z != w.y) other[(size_t)w.z].push_back(w.y);
    }
    for (int I = 0; I < Nt; ++I) {
        std::sort(other[(size_t)I].begin(), other[(size_t)I].end());
        srow[(size_t)I + 1] = srow[(size_t)I] + (int)other[(size_t)I].size();
    }
    auto slot_of = [&](int I, int k) {
        const auto& o = other[(size_t)I];
        return srow[(size_t)I] + (int)(std::lower_bound(o.begin(), o.end(), k) - o.begin());
    };
    std::vector<int2> tslot(wl.size());
    for (size_t e = 0; e < wl.size(); ++e) tslot[e] = make_int2(slot_of(wl[e].y, wl[e].z), slot_of(wl[e].z, wl[e].y));
    h->nslot = srow[(size_t)Nt];
    CK(cudaMemcpyAsync(h->work, wl.data(), wl.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->slab, slab.data(), slab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->srow, srow.data(), srow.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->tslot, tslot.data(), tslot.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->sched, sc, (size_t)h->nstages * sizeof(Sched), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // the host lists go out of scope
    return GABP_OK;
}

// Tile-sparse option: the second allocation holds at least `need` bytes
// (kept when large enough, else replaced; its contents are not kept).
// GABP_ENOMEM when that does not fit in free device memory.
gabp_status ensure_spool(gabp_svm_t h, size_t need, const char* what)
{
    need += 1024;
    if (need <= h->spool_bytes) return GABP_OK;
    CK(cudaStreamSynchronize(h->stream));
    if (h->spool) CK(cudaFree(h->spool));
    h->spool = nullptr;
    h->spool_bytes = 0;
    size_t free_b = 0;
    CK(device_available(&free_b, true));   // cudaMalloc below: the pool's unused memory back first
    const size_t margin = (size_t)256 << 20;
    if (need + margin > free_b)
        return fail(GABP_ENOMEM, "%s need %.2f GB of device memory, %.2f GB free", what, need / 1e9, free_b / 1e9);
    cudaError_t e = cudaMalloc(&h->spool, need);
    if (e != cudaSuccess) return fail(GABP_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    h->spool_bytes = need;
    return GABP_OK;
}

// Tile-sparse option: per-pair arrays for the h->nlive kept tiles and the
// slot partials of the compacted slot space (nslot slots), in the second
// allocation.
gabp_status ensure_pair_storage(gabp_svm_t h, long long nslot)
{
    Inst& p = h->inst;
    const int qm = h->opts.q_mode, mb = h->opts.msg_bf16;
    char what[64];
    snprintf(what, sizeof(what), "the %lld kept tiles", h->nlive);
    if (gabp_status st = ensure_spool(h, pair_bytes(h->nlive, qm, mb) + part_bytes(nslot), what)) return st;
    const size_t tt = (size_t)h->nlive * TT;
    char* b = static_cast<char*>(h->spool);
    const size_t st = align_up(tt * (mb ? 4 : 8), 256);
    p.Pst = b;
    p.Hst = b + st;
    b += 2 * st;
    p.qstore = nullptr;
    p.qref = nullptr;
    if (qm == GABP_Q_F32) {
        p.qstore = b;
        p.qref = (float*)b;
        b += align_up(tt * 4, 256);
    } else if (qm == GABP_Q_BF16) {
        p.qstore = b;
        p.qref = (float*)(b + align_up(tt * 2, 256));
        b += align_up(tt * 2, 256) + align_up(tt * 4, 256);
    }
    p.part = (float*)b;
    p.nslot = nslot;
    p.srow = h->srow;
    p.tslot = h->tslot;
    p.rsum = h->rsum;
    return GABP_OK;
}

gabp_status stage_and_form(gabp_svm_t h, const void* X, const float* y)
{
    NvtxRange nv("gabp.formation");
    cudaStream_t s = h->stream;
    const int64_t n = h->n, m = h->m;
    const bool dev = h->opts.ptr_mode == 1;
    const int xd = h->opts.x_dtype;
    Inst& p = h->inst;
    p.gamma = (float)h->gamma;
    p.lam2 = (float)(h->lambda * h->lambda);
    // KRR: C is the ridge lambda_r; inside, 1/C enters the diagonal floor
    // 1 + lambda^2 + 1/C as the SVM's 2-norm soft margin does
    p.C = (float)(h->opts.task == GABP_TASK_KRR ? 1.0 / h->C : h->C);
    p.task = h->opts.task;
    clear_graphs(h);
    h->solved = false;
    h->formed = false;
    h->kstar = 0;
    h->mean_src = nullptr;

    if (h->opts.sparse_tau > 0) {
        // formation's first pass stores nothing and records the tile maxima
        p.tilemax = h->tilemax;
        p.slab = nullptr;
        p.qstore = nullptr;
        p.qref = nullptr;
    }
    CK(cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s));
    CK(cudaMemcpyAsync(h->d_tab, &p, sizeof(Inst), cudaMemcpyHostToDevice, s));
    // labels -> device copy (validated by the staging kernel, which also sets b = 1)
    CK(cudaMemcpyAsync((void*)p.y, y, (size_t)n * sizeof(float),
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (fault_mask() > 0 && (fault_mask() & FAULT_NAN)) {
        // the handle's own copy of the labels (targets) gets a NaN in row n / 2
        static const float kNaN = NAN;
        CK(cudaMemcpyAsync((void*)(p.y + n / 2), &kNaN, sizeof(float), cudaMemcpyHostToDevice, s));
    }
    void* tmp = nullptr;
    const void* src = X;
    if (!dev) {
        if (xd != 0) {   // FP64 / BF16 rows: widened to FP32 by the staging kernel
            CK(cudaMallocAsync(&tmp, (size_t)n * m * x_elem_bytes(xd), s));
            CK(cudaMemcpyAsync(tmp, X, (size_t)n * m * x_elem_bytes(xd), cudaMemcpyHostToDevice, s));
            src = tmp;
        } else {
            CK(cudaMemcpyAsync((void*)p.X, X, (size_t)n * m * sizeof(float), cudaMemcpyHostToDevice, s));
            src = p.X;
        }
    }
    launch_stage(src, xd, (int)n, (int)m, const_cast<float*>(p.y), (float*)p.X, (float*)p.sq, (float*)p.b,
                 const_cast<float*>(p.b0), p.task, p.ctrl, s);
    h->prof.kernel_launches += 1;
    CK(cudaGetLastError());
    if (tmp) CK(cudaFreeAsync(tmp, s));
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->hctrl->status != 0)
        return fail(GABP_EINVAL, h->opts.task == GABP_TASK_KRR ? "row %lld: non-finite feature or target"
                                                                : "row %lld: non-finite feature or label not +-1",
                    (long long)h->hctrl->bad_index);
    // the FP32 rows as three BF16 planes for the tensor-core FP32 Gram, and
    // the norms from the same products (diagonal tiles)
    CK(launch_pack3(p.X, (int)n, (int)m, h->Nt, (void*)p.Xp3, s));
    launch_form_norms(h->d_tab, h->work_diag, h->Nt, s);
    CK(cudaGetLastError());
    h->prof.kernel_launches += 2;
    if (h->opts.sparse_tau > 0) {
        // Tile-sparse option.  Pass 1 over every tile: tile maxima and |Q|
        // row sums (the whole matrix's, for the diagonal rule), Q not
        // stored; the row sums are added into per-node fixed-point sums
        // (in rsum's memory, converted to rsum in place).  Then the kept-tile
        // list, the compacted slot space and the kept tiles' storage (which
        // replaces the dense slots), and pass 2 over the kept tiles only:
        // their FP32 values (the store, or the FP32 copy beside the BF16
        // store; the row sums it writes into the compacted slots are not
        // used, the diagonal rule takes rsum), the diagonal rule and Step 1,
        // and the BF16 tiles.  Recompute needs no second pass.
        if (h->opts.q_mode != GABP_Q_F32)
            CK(launch_pack_bf16(p.X, (int)n, (int)m, p.nkc, h->Nt, (void*)p.Xp, (float*)p.sqb, s));
        p.part = nullptr;
        p.nslot = 0;
        p.srow = nullptr;
        p.tslot = nullptr;
        p.rsum = nullptr;
        p.rfix = reinterpret_cast<unsigned long long*>(h->rsum);
        CK(cudaMemsetAsync(h->rsum, 0, (size_t)n * sizeof(double), s));
        CK(cudaMemcpyAsync(h->d_tab, &p, sizeof(Inst), cudaMemcpyHostToDevice, s));
        launch_form_q(h->d_tab, h->work_all, h->ntiles, s);
        launch_row_abs_sums(p, h->rsum, s);
        CK(cudaGetLastError());
        h->prof.kernel_launches += h->opts.q_mode != GABP_Q_F32 ? 4 : 2;
        p.rfix = nullptr;
        if (gabp_status st = build_sweep_list(h)) return st;
        if (gabp_status st = ensure_pair_storage(h, h->nslot)) return st;
        p.tilemax = nullptr;
        p.slab = h->slab;
        CK(cudaMemcpyAsync(h->d_tab, &p, sizeof(Inst), cudaMemcpyHostToDevice, s));
        if (h->opts.q_mode != GABP_Q_RECOMPUTE) {
            launch_form_q(h->d_tab, h->work, h->nlive, s);
            h->prof.kernel_launches += 1;
        }
        launch_init(p, h->opts.diag_rule, (float)h->delta, s);
        h->prof.kernel_launches += 1;
        CK(cudaGetLastError());
        if (h->opts.q_mode == GABP_Q_BF16) {
            CK(launch_form_q_tc(h->d_tab, h->work, h->nlive, s));
            h->prof.kernel_launches += 1;
        }
    } else if (h->opts.q_mode == GABP_Q_F32) {
        launch_form_q(h->d_tab, h->work_all, h->ntiles, s);
        CK(cudaGetLastError());
        if (gabp_status st = build_sweep_list(h)) return st;
        launch_init(p, h->opts.diag_rule, (float)h->delta, s);
        h->prof.kernel_launches += 2;
        CK(cudaGetLastError());
    } else {
        // Precision form: the diagonal weighting uses the FP32 Gram's row sums
        // (the accurate matrix), whose tiles the BF16 store also keeps as the
        // FP32 copy for its refinement residuals; the off-diagonal entries
        // the sweeps read come from the BF16 tensor-core Gram.
        CK(launch_pack_bf16(p.X, (int)n, (int)m, p.nkc, h->Nt, (void*)p.Xp, (float*)p.sqb, s));
        launch_form_q(h->d_tab, h->work_all, h->ntiles, s);
        CK(cudaGetLastError());
        if (gabp_status st = build_sweep_list(h)) return st;
        launch_init(p, h->opts.diag_rule, (float)h->delta, s);
        CK(cudaGetLastError());
        h->prof.kernel_launches += 4;
        if (h->opts.q_mode == GABP_Q_BF16) {
            CK(launch_form_q_tc(h->d_tab, h->work_all, h->ntiles, s));
            h->prof.kernel_launches += 1;
        }
    }
    CK(cudaStreamSynchronize(s));
    h->formed = true;
    return GABP_OK;
}

void destroy_all(gabp_svm_t h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    clear_graphs(h);
    if (h->pool) cudaFree(h->pool);
    if (h->spool) cudaFree(h->spool);
    if (h->hctrl) cudaFreeHost(h->hctrl);
    if (h->hfinal) cudaFreeHost(h->hfinal);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Whether round k of a captured chunk has its pair sweep bracketed by events
// (every `stride`-th round: k = stride - 1, 2 stride - 1, ...), and its pair.
static bool bracketed(int stride, int k) { return stride > 0 && k % stride == stride - 1; }

// A captured chunk of `rounds` synchronous rounds; with profiling on, the
// pair sweep of every profiling-th round in it is bracketed by two
// event-record nodes.
gabp_status get_graph(gabp_svm_t h, int rounds, gabp_svm_s::Graph** out)
{
    const int stride = h->profiling;
    const auto key = std::make_pair(rounds, stride);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) { *out = &it->second; return GABP_OK; }
    gabp_svm_s::Graph G;
    if (stride > 0) {
        G.ev.resize((size_t)2 * (rounds / stride));
        for (auto& e : G.ev) CK(cudaEventCreate(&e));
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < rounds; ++k)
        launch_round(h->d_tab, h->work, h->nbl, h->sched, h->nstages, h->grid, h->opts.q_mode, h->opts.msg_bf16,
                     h->stream, bracketed(stride, k) ? &G.ev[(size_t)2 * (k / stride)] : nullptr);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(GABP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(GABP_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    auto res = h->graphs.emplace(key, std::move(G));
    *out = &res.first->second;
    return GABP_OK;
}

// Runs up to `iters` synchronous rounds from the current state with the
// residual test `tol`, as captured graphs of `chunk` rounds, reading the
// control block after each replay.  *out = the final control block.
gabp_status run_rounds(gabp_svm_t h, int iters, double tol, Ctrl* out)
{
    NvtxRange nv("gabp.rounds");
    cudaStream_t s = h->stream;
    Inst& p = h->inst;
    launch_begin(h->d_tab, 1, iters, tol, s);
    h->prof.kernel_launches += 1;
    CK(cudaGetLastError());
    if (iters > 0 && fault_mask() > 0 && (fault_mask() & FAULT_TIMEOUT)) {
        // as if a bounded device wait of the first round ran out: the round's
        // finalize stops the solve and the status reaches the host
        static const int kTimeout = ST_ETIMEOUT;
        CK(cudaMemcpyAsync(&p.ctrl->status, &kTimeout, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (iters > 0) {
        const int len = tol > 0 ? std::min<int>(h->opts.chunk, iters) : iters;
        gabp_svm_s::Graph* g = nullptr;
        if (gabp_status st = get_graph(h, len, &g)) return st;
        const int max_chunks = (iters + len - 1) / len + 1;
        int t_before = h->hctrl->t;
        for (int c = 0; c < max_chunks; ++c) {
            CK(cudaGraphLaunch(g->exec, s));
            h->prof.kernel_launches += 2 * len;
            CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const int ran = h->hctrl->t - t_before;
            if (!g->ev.empty()) {
                const int stride = h->profiling;
                for (int k = 0; k < ran && k < len; ++k) {
                    if (!bracketed(stride, k)) continue;
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, g->ev[(size_t)2 * (k / stride)], g->ev[(size_t)2 * (k / stride) + 1]));
                    h->prof.sweep_ms += ms;
                    h->prof.sweep_launches += 1;
                    if (t_before + k == 0) h->prof.sweep_launches_zero_state += 1;
                    if (h->hctrl->p_frozen && t_before + k >= h->hctrl->t_frozen) h->prof.sweep_launches_p_frozen += 1;
                }
            }
            t_before = h->hctrl->t;
            if (h->hctrl->done) break;
        }
    }
    const Ctrl c = *h->hctrl;
    *out = c;
    if (!c.done) return fail(GABP_ECUDA, "solve loop did not reach its stop condition");
    if (c.status == ST_ENUMERIC)
        return fail(GABP_ENUMERIC, "nonpositive or non-finite cavity precision near node %lld in round %d",
                    c.bad_index, c.kstar);
    if (c.status == ST_ETIMEOUT)
        return fail(GABP_ETIMEOUT, "a bounded device wait ran out in round %d (tile %lld)", c.kstar, c.bad_index);
    if (c.status != 0) return fail(GABP_ECUDA, "device status %d", c.status);
    return GABP_OK;
}

}  // namespace

extern "C" {

void gabp_svm_opts_default(gabp_svm_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->diag_rule = GABP_DIAG_DOMINANT;
    o->diag_delta = 0.1;
    o->q_mode = GABP_Q_F32;
    o->chunk = 16;
}

const char* gabp_last_error(void) { return g_err.c_str(); }

int32_t gabp_version(void) { return GABP_SVM_VERSION; }

gabp_status gabp_svm_create(const void* X, const float* y, int64_t n, int64_t m, double gamma,
                            double C, gabp_svm_t* out)
{
    gabp_svm_opts o;
    gabp_svm_opts_default(&o);
    return gabp_svm_create_ex(X, y, n, m, gamma, C, &o, out);
}

gabp_status gabp_svm_create_ex(const void* X, const float* y, int64_t n, int64_t m, double gamma,
                               double C, const gabp_svm_opts* opts, gabp_svm_t* out)
{
    g_err.clear();
    if (!out) return fail(GABP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!X || !y) return fail(GABP_EINVAL, "X or y is NULL");
    if (n < 2 || m < 1) return fail(GABP_EINVAL, "need n >= 2 and m >= 1 (got n=%lld m=%lld)",
                                    (long long)n, (long long)m);
    if (n > (int64_t)1 << 30 || m > (int64_t)1 << 20 || n * m > ((int64_t)1 << 40))
        return fail(GABP_EINVAL, "n or m too large");
    if (!(gamma > 0) || !(gamma <= FLT_MAX)) return fail(GABP_EINVAL, "gamma must be > 0 and within FP32 range");
    if (!(C > 0) || !std::isfinite(C)) return fail(GABP_EINVAL, "C must be finite and > 0");
    gabp_svm_opts o;
    gabp_svm_opts_default(&o);
    if (opts) {
        o = *opts;
        if (o.diag_delta == 0) o.diag_delta = 0.1;
        if (o.chunk <= 0) o.chunk = 16;
    }
    if (o.x_dtype < 0 || o.x_dtype > 2) return fail(GABP_EINVAL, "x_dtype must be 0 (f32), 1 (f64) or 2 (bf16)");
    if (o.ptr_mode != 0 && o.ptr_mode != 1) return fail(GABP_EINVAL, "ptr_mode must be 0 or 1");
    if (o.diag_rule != GABP_DIAG_DOMINANT && o.diag_rule != GABP_DIAG_SOFT2)
        return fail(GABP_EINVAL, "unknown diag_rule");
    if (!(o.diag_delta > 0) || !std::isfinite(o.diag_delta)) return fail(GABP_EINVAL, "diag_delta must be > 0");
    if (o.bias_mode == 1 && (!(o.bias_lambda >= 0) || !(o.bias_lambda * o.bias_lambda <= FLT_MAX)))
        return fail(GABP_EINVAL, "bias_lambda must be >= 0 with lambda^2 within FP32 range");
    if (o.q_mode != GABP_Q_F32 && o.q_mode != GABP_Q_BF16 && o.q_mode != GABP_Q_RECOMPUTE)
        return fail(GABP_EINVAL, "unknown q_mode %d", o.q_mode);
    if (o.refine < 0 || o.refine > 64) return fail(GABP_EINVAL, "refine must be in [0, 64]");
    if (o.msg_bf16 != 0 && (o.msg_bf16 != 1 || o.q_mode == GABP_Q_F32))
        return fail(GABP_EINVAL, "msg_bf16 = 1 needs a precision form (q_mode BF16 or recompute)");
    if (o.task != GABP_TASK_SVM && o.task != GABP_TASK_KRR) return fail(GABP_EINVAL, "unknown task %d", o.task);
    if (o.stages < 0 || o.stages > kMaxStages) return fail(GABP_EINVAL, "stages must be in [0, %d]", kMaxStages);
    if (!(o.sparse_tau >= 0) || !std::isfinite(o.sparse_tau)) return fail(GABP_EINVAL, "sparse_tau must be >= 0");
    const int faults = fault_mask();
    if (faults < 0) return fail(GABP_EINVAL, "GABP_FAULT holds an unknown token (known: alloc, nan, timeout)");

    int dev = 0, ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(GABP_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    CK(cudaGetDevice(&dev));

    gabp_svm_t h = new (std::nothrow) gabp_svm_s();
    if (!h) return fail(GABP_ENOMEM, "host allocation failed");
    h->device = dev;
    h->opts = o;
    h->n = n;
    h->m = m;
    h->Nt = (int)((n + T - 1) / T);
    h->npad = (int)align_up((size_t)n, T);   // whole tiles: the sweep copies aggregate blocks of T
    h->ntiles = tri_tiles(h->Nt);
    h->gamma = gamma;
    h->C = C;
    h->lambda = o.bias_mode == 1 ? o.bias_lambda : (o.task == GABP_TASK_KRR ? 0.0 : 1.0 / (double)n);
    h->delta = o.diag_delta;
    h->nstages = o.stages > 1 ? o.stages : 1;

    const Plan pl = make_plan(n, m, h->Nt, h->ntiles, h->npad, o.q_mode, o.msg_bf16, o.sparse_tau > 0);
    size_t free_b = 0;
    e = device_available(&free_b, true);   // cudaMalloc below: the pool's unused memory back first
    if (e != cudaSuccess) { destroy_all(h); return fail(GABP_ECUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e)); }
    const size_t margin = (size_t)256 << 20;
    if (pl.total + margin > free_b) {
        destroy_all(h);
        return fail(GABP_ENOMEM, "needs %.2f GB of device memory, %.2f GB free", pl.total / 1e9, free_b / 1e9);
    }
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { destroy_all(h); return fail(GABP_ECUDA, "stream: %s", cudaGetErrorString(e)); }
        h->own_stream = true;
    }
    e = prepare_sweep();
    if (e == cudaSuccess && o.q_mode == GABP_Q_RECOMPUTE) e = prepare_sweep_rc();
    if (e != cudaSuccess) { destroy_all(h); return fail(GABP_ECUDA, "sweep kernel setup: %s", cudaGetErrorString(e)); }
    if (faults & FAULT_ALLOC) {
        destroy_all(h);
        return fail(GABP_ENOMEM, "injected device allocation failure (GABP_FAULT=alloc)");
    }
    e = cudaMalloc(&h->pool, pl.total);
    if (e != cudaSuccess) { destroy_all(h); return fail(GABP_ENOMEM, "cudaMalloc(%zu): %s", pl.total, cudaGetErrorString(e)); }
    h->pool_bytes = pl.total;
    if (cudaMallocHost(&h->hctrl, sizeof(Ctrl)) != cudaSuccess ||
        cudaMallocHost(&h->hfinal, 4 * sizeof(double)) != cudaSuccess) {
        destroy_all(h);
        return fail(GABP_ENOMEM, "pinned host allocation failed");
    }
    char* base = static_cast<char*>(h->pool);
    size_t off = 0;
    auto take = [&](size_t bytes) { void* r = base + off; off += bytes; return r; };
    Inst& p = h->inst;
    p.n = (int)n;
    p.Nt = h->Nt;
    p.m = (int)m;
    p.npad = h->npad;
    p.X = (const float*)take(pl.X);
    p.sq = (const float*)take(pl.vec);
    p.y = (const float*)take(pl.vec);
    p.b = (const float*)take(pl.vec);
    p.b0 = (const float*)take(pl.vec);
    p.qdiag = (float*)take(pl.vec);
    h->alpha = (float*)take(pl.vec);
    p.sq3 = (float*)take(pl.vec);
    p.sqb = (const float*)take(pl.vec);
    h->mu_acc = (float*)take(pl.vec);
    h->r32 = (float*)take(pl.vec);
    p.agg = (float*)take(pl.agg);
    p.aggmid = p.agg + (size_t)6 * h->npad;
    p.part = pl.part ? (float*)take(pl.part) : nullptr;   // tile-sparse: with the kept tiles' arrays
    p.nslot = (long long)h->Nt * h->Nt;
    p.srow = nullptr;
    p.tslot = nullptr;
    p.rsum = nullptr;
    p.Pst = take(pl.state / 2);
    p.Hst = take(pl.state / 2);
    p.msg_bf16 = o.msg_bf16;
    p.qstore = pl.q ? take(pl.q) : nullptr;
    p.qref = pl.qref ? (float*)take(pl.qref) : (o.q_mode == GABP_Q_F32 ? (float*)p.qstore : nullptr);
    h->work_diag = (int4*)take(align_up((size_t)h->Nt * sizeof(int4), 256));
    const size_t wbytes = pl.work - align_up((size_t)h->Nt * sizeof(int4), 256);
    if (o.sparse_tau > 0) {
        h->work_all = (int4*)take(wbytes / 2);
        h->work = (int4*)take(wbytes / 2);
        h->tilemax = (float*)take(pl.tilemax / 2);
        h->slab = (int*)take(pl.tilemax / 2);
        h->srow = (int*)take(align_up((size_t)(h->Nt + 1) * sizeof(int), 256));
        h->tslot = (int2*)take(align_up((size_t)h->ntiles * sizeof(int2), 256));
        h->rsum = (double*)take(align_up((size_t)n * sizeof(double), 256));
    } else {
        h->work = h->work_all = (int4*)take(wbytes);   // formation walks the swept list
    }
    {
        char* tb = (char*)take(pl.tab);
        h->d_tab = (Inst*)tb;
        h->sched = (Sched*)(tb + align_up(sizeof(Inst), 16));   // one per stage
        h->d_ops = (StopOp*)(tb + align_up(sizeof(Inst), 16) + kMaxStages * align_up(sizeof(Sched), 16));
        h->d_members = (int*)((char*)h->d_ops + align_up(sizeof(StopOp), 16));
    }
    h->nbl = (int2*)take(pl.nbl);
    p.ctrl = (Ctrl*)take(pl.ctrl);
    p.rhist = (double*)take(pl.rhist);
    p.rhist_cap = kRhistCap;
    h->final3 = (double*)take(pl.final3);
    h->blockbuf = (double*)take(pl.blockbuf);
    p.nkc = bf16_chunks((int)m);
    if (pl.xp) {
        off = align_up(off, 1024);
        p.Xp = take(pl.xp);
    }
    off = align_up(off, 1024);
    p.Xp3 = take(pl.xp3);

    // Tile work list: the upper triangle, row by row within each stage (one
    // stage = all of it under the synchronous schedule); tile storage index
    // L(I,J) = I*Nt - I(I-1)/2 + (J-I).
    std::vector<int4> wl;
    wl.reserve((size_t)h->ntiles);
    int B[kMaxStages + 1];
    stage_bounds(h->Nt, h->nstages, B);
    const int nblk = (int)((n + 31) / 32);
    Sched sc[kMaxStages];
    for (int st = 0; st < h->nstages; ++st) {
        const long long off = (long long)wl.size();
        for (int I = 0; I < h->Nt; ++I)
            for (int J = std::max(I, B[st]); J < B[st + 1]; ++J)
                wl.push_back(make_int4(0, I, J, (int)((long long)I * h->Nt - (long long)I * (I - 1) / 2 + (J - I))));
        sc[st] = Sched{(long long)wl.size() - off, nblk, 1, off, h->Nt <= kWarpFinNt ? nblk : 0, 0};
    }
    std::vector<int2> nb((size_t)nblk);
    for (int b = 0; b < nblk; ++b) nb[(size_t)b] = make_int2(0, b);
    std::vector<int4> wd((size_t)h->Nt);
    for (int I = 0; I < h->Nt; ++I)
        wd[(size_t)I] = make_int4(0, I, I, (int)((long long)I * h->Nt - (long long)I * (I - 1) / 2));
    h->grid = round_grid(h->ntiles, nblk, o.q_mode, 0, o.msg_bf16);
    h->nlive = h->ntiles;
    e = cudaMemcpyAsync(h->work_all, wl.data(), wl.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->nbl, nb.data(), nb.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->work_diag, wd.data(), wd.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->sched, sc, (size_t)h->nstages * sizeof(Sched), cudaMemcpyHostToDevice, h->stream);
    const int zero_slot = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_members, &zero_slot, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { destroy_all(h); return fail(GABP_ECUDA, "work list copy: %s", cudaGetErrorString(e)); }

    gabp_status st = stage_and_form(h, X, y);
    if (st != GABP_OK) { std::string msg = g_err; destroy_all(h); g_err = msg; return st; }
    *out = h;
    return GABP_OK;
}

gabp_status gabp_svm_refit(gabp_svm_t h, const void* X, const float* y, double gamma, double C)
{
    g_err.clear();
    if (gabp_status s = check_handle(h)) return s;
    if (!X || !y) return fail(GABP_EINVAL, "X or y is NULL");
    if (!(gamma > 0) || !(gamma <= FLT_MAX)) return fail(GABP_EINVAL, "gamma must be > 0 and within FP32 range");
    if (!(C > 0) || !std::isfinite(C)) return fail(GABP_EINVAL, "C must be finite and > 0");
    h->gamma = gamma;
    h->C = C;
    return stage_and_form(h, X, y);
}

gabp_status gabp_svm_solve(gabp_svm_t h, int32_t iters, double tol, float* alpha, double* residual_inf,
                           int32_t* iters_done)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    if (iters < 0) return fail(GABP_EINVAL, "iters must be >= 0");
    if (std::isnan(tol)) return fail(GABP_EINVAL, "tol is NaN");
    cudaStream_t s = h->stream;
    Inst& p = h->inst;
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->hctrl->status != 0) return fail(GABP_ESTATE, "state is invalid after an earlier failure; refit first");
    const bool refine = h->opts.q_mode != GABP_Q_F32 && h->opts.refine > 0;
    const bool same_matrix = h->opts.q_mode == GABP_Q_F32;   // the sweeps and the final pass see one Q
    if (refine) {
        // The refined solve always starts from Step 1 (b = 1, messages 0).
        launch_reset(p, s);
        h->prof.kernel_launches += 1;
    }
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int t0 = h->hctrl->t;
    if ((long long)t0 + (long long)iters * (1 + h->opts.refine) >= (long long)INT_MAX)
        return fail(GABP_EINVAL, "too many rounds");
    Ctrl c{};
    // With refinement ahead, the BF16 solve only needs to reach about the BF16
    // error level of its matrix (and messages) before the first correction.
    const double handover = refine_handover(h->opts.refine_handover, h->opts.msg_bf16);
    if (gabp_status st = run_rounds(h, iters, refine ? std::max(tol, handover) : tol, &c)) return st;
    h->kstar = c.kstar;
    const float* mu = p.agg + (size_t)(c.kstar & 1) * 3 * p.npad + 2 * (size_t)p.npad;
    int refine_done = 0;
    StopOp op{};
    op.alpha = h->alpha;
    op.blockbuf = h->blockbuf;
    op.final3 = h->final3;
    op.sv_threshold = (float)h->opts.sv_threshold;
    const int nblk = (int)((h->n + 31) / 32);
    auto final_pass = [&](const StopOp& o) -> gabp_status {
        NvtxRange nv("gabp.final_pass");
        CK(cudaMemcpyAsync(h->d_ops, &o, sizeof(StopOp), cudaMemcpyHostToDevice, s));
        if (o.acc) launch_axpy_list(h->d_tab, h->d_ops, h->nbl, nblk, s);
        launch_final(h->d_tab, h->d_ops, h->work, h->nlive, h->nbl, nblk, h->d_members, 1, nullptr,
                     h->inst.qref != nullptr, s);
        h->prof.kernel_launches += o.acc ? 4 : 3;
        CK(cudaGetLastError());
        return GABP_OK;
    };
    if (refine) {
        // Defect correction: mu_acc solves the BF16 system; r = 1 - Q32 mu_acc
        // with the FP32-Gram matrix and FP64 sums; GaBP on the BF16 system with
        // right-hand side r (P messages kept, H restarted) gives the
        // correction d; mu_acc += d; repeat until ||r||_inf < tol.
        int buf = c.kstar, first = 1;
        for (int it = 0; it <= h->opts.refine; ++it) {
            StopOp o = op;
            o.mu = h->mu_acc;
            o.acc = h->mu_acc;
            o.axpy_buf = buf;
            o.axpy_first = first;
            o.r_out = h->r32;
            if (gabp_status st = final_pass(o)) return st;
            if (!first) ++refine_done;
            first = 0;
            CK(cudaMemcpyAsync(h->hfinal, h->final3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const double rn = h->hfinal[0];
            if (!(rn >= tol) || it == h->opts.refine) break;
            StopOp rr = op;
            rr.r_out = h->r32;
            CK(cudaMemcpyAsync(h->d_ops, &rr, sizeof(StopOp), cudaMemcpyHostToDevice, s));
            launch_refine_rhs_list(h->d_tab, h->d_ops, h->nbl, nblk, s);
            h->prof.kernel_launches += 1;
            const double inner = std::max(tol * 0.5, refine_inner(h->opts.refine_inner, h->opts.msg_bf16) * rn);
            Ctrl ci{};
            if (gabp_status st = run_rounds(h, iters, inner, &ci)) return st;
            buf = ci.kstar;
        }
        mu = h->mu_acc;
    } else {
        // The stop test of the rounds sums the residual in compensated FP32;
        // the reported residual comes from the final pass (FP32 tile
        // partials, FP64 sums).  When both are residuals of the same matrix
        // (Q stored in FP32), a stop counts once the reported residual is
        // below tol too; until then the rounds go on from where they stopped
        // (Algorithm 2, Step 3), within the iteration limit.  (An unrefined
        // BF16 solve stops on its own matrix; its reported residual is that
        // of the FP32-Gram matrix.)
        for (;;) {
            StopOp o = op;
            o.mu = mu;
            if (gabp_status st = final_pass(o)) return st;
            CK(cudaMemcpyAsync(h->hfinal, h->final3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const long long left = (long long)t0 + iters - (long long)c.t;
            if (!same_matrix || !c.converged || h->hfinal[0] < tol || left <= 0) break;
            if (gabp_status st = run_rounds(h, (int)left, tol, &c)) return st;
            h->kstar = c.kstar;
            mu = p.agg + (size_t)(c.kstar & 1) * 3 * p.npad + 2 * (size_t)p.npad;
        }
    }
    CK(cudaMemcpyAsync(h->hfinal, h->final3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (alpha)
        CK(cudaMemcpyAsync(alpha, h->alpha, (size_t)h->n * sizeof(float),
                           h->opts.ptr_mode == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->solved = true;
    h->mean_src = mu;
    gabp_svm_stats& S = h->stats;
    S.n = h->n;
    S.m = h->m;
    S.sweeps_total = h->hctrl->t;
    S.kstar = c.kstar;
    S.converged = refine ? (h->hfinal[0] < tol ? 1 : 0)
                         : (c.converged && (!same_matrix || h->hfinal[0] < tol)) ? 1 : 0;
    S.residual_inf = h->hfinal[0];
    {
        double inv = 0.0;
        std::memcpy(&inv, &h->hctrl->inv_margin_bits, sizeof inv);
        S.margin = inv > 0 ? 1.0 / inv : 0.0;   // 1/inf = 0: some row is not strictly dominant
        S.err_bound = S.margin > 0 ? S.residual_inf / S.margin : INFINITY;
    }
    S.dual_objective = h->hfinal[1];
    S.n_support = (int64_t)std::llround(h->hfinal[2]);
    S.refine_passes = refine_done;
    if (residual_inf) *residual_inf = h->hfinal[0];
    if (iters_done) *iters_done = refine ? (h->hctrl->t - t0) : (c.kstar - t0);
    return GABP_OK;
}

gabp_status gabp_svm_get_mean(gabp_svm_t h, float* mu)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    if (!mu) return fail(GABP_EINVAL, "mu is NULL");
    const Inst& p = h->inst;
    const float* src = h->mean_src ? h->mean_src : p.agg + 2 * (size_t)p.npad;
    CK(cudaMemcpyAsync(mu, src, (size_t)h->n * sizeof(float),
                       h->opts.ptr_mode == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GABP_OK;
}

gabp_status gabp_svm_get_aggregates(gabp_svm_t h, float* Pt, float* ht, float* mu)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    const Inst& p = h->inst;
    CK(cudaMemcpyAsync(h->hctrl, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const float* base = p.agg + (size_t)(h->hctrl->t & 1) * 3 * p.npad;
    const cudaMemcpyKind kind = h->opts.ptr_mode == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    float* dst[3] = {Pt, ht, mu};
    for (int a = 0; a < 3; ++a)
        if (dst[a]) CK(cudaMemcpyAsync(dst[a], base + (size_t)a * p.npad, (size_t)h->n * sizeof(float), kind, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GABP_OK;
}

gabp_status gabp_svm_decision(gabp_svm_t h, const void* Xtest, int64_t t, float* out)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    if (!h->solved) return fail(GABP_ESTATE, "no solve yet");
    if (t < 0 || (t > 0 && (!Xtest || !out))) return fail(GABP_EINVAL, "bad test set");
    if (t == 0) return GABP_OK;
    if (t > ((int64_t)1 << 30)) return fail(GABP_EINVAL, "t too large");
    NvtxRange nv("gabp.decision");
    cudaStream_t s = h->stream;
    const bool dev = h->opts.ptr_mode == 1;
    const int xd = h->opts.x_dtype;
    const int64_t m = h->m;
    const int Ntt = (int)((t + T - 1) / T);
    const long long ntl = (long long)Ntt * h->Nt;
    const size_t bx = align_up((size_t)t * m * sizeof(float), 256), bsq = align_up((size_t)t * 4, 256);
    const size_t bin = (!dev && xd != 0) ? align_up((size_t)t * m * x_elem_bytes(xd), 256) : 0;
    const size_t bpart = align_up((size_t)h->Nt * t * sizeof(float), 256);
    const size_t bw = align_up((size_t)ntl * sizeof(int2), 256), bout = align_up((size_t)t * 4, 256);
    char* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, bx + bsq + bin + bpart + bw + bout, s));
    float* Xt = (float*)tmp;
    float* sqt = (float*)(tmp + bx);
    void* in = tmp + bx + bsq;
    float* part = (float*)(tmp + bx + bsq + bin);
    int2* w = (int2*)(tmp + bx + bsq + bin + bpart);
    float* dout = (float*)(tmp + bx + bsq + bin + bpart + bw);
    std::vector<int2> wl((size_t)ntl);
    size_t k = 0;
    for (int I = 0; I < Ntt; ++I)
        for (int J = 0; J < h->Nt; ++J) wl[k++] = make_int2(I, J);
    gabp_status st = GABP_OK;
    auto run = [&]() -> gabp_status {
        CK(cudaMemcpyAsync(w, wl.data(), wl.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        const void* src = Xtest;
        if (!dev) {
            if (xd != 0) {
                CK(cudaMemcpyAsync(in, Xtest, (size_t)t * m * x_elem_bytes(xd), cudaMemcpyHostToDevice, s));
                src = in;
            } else {
                CK(cudaMemcpyAsync(Xt, Xtest, (size_t)t * m * sizeof(float), cudaMemcpyHostToDevice, s));
                src = Xt;
            }
        }
        CK(cudaMemcpyAsync(h->hctrl, h->inst.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int saved_status = h->hctrl->status;
        launch_stage(src, xd, (int)t, (int)m, nullptr, Xt, sqt, nullptr, nullptr, 0, h->inst.ctrl, s);
        h->prof.kernel_launches += 1;
        CK(cudaMemcpyAsync(h->hctrl, h->inst.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->hctrl->status != saved_status) {
            CK(cudaMemsetAsync(&h->inst.ctrl->status, 0, sizeof(int), s));
            CK(cudaStreamSynchronize(s));
            return fail(GABP_EINVAL, "test row %lld: non-finite feature", h->hctrl->bad_index);
        }
        launch_decision(h->inst, Xt, sqt, (int)t, h->alpha, w, ntl, part, dev ? out : dout, s);
        h->prof.kernel_launches += 2;
        CK(cudaGetLastError());
        if (!dev) CK(cudaMemcpyAsync(out, dout, (size_t)t * sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return GABP_OK;
    };
    st = run();
    cudaFreeAsync(tmp, s);
    cudaStreamSynchronize(s);
    return st;
}

gabp_status gabp_svm_support(gabp_svm_t h, int32_t* idx, int64_t cap, int64_t* count)
{
    g_err.clear();
    if (gabp_status s = check_handle(h)) return s;
    if (!h->solved) return fail(GABP_ESTATE, "no solve yet");
    if (!count || (cap > 0 && !idx)) return fail(GABP_EINVAL, "bad output");
    std::vector<float> a((size_t)h->n);
    CK(cudaMemcpyAsync(a.data(), h->alpha, a.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int64_t c = 0;
    const float th = (float)h->opts.sv_threshold;
    const bool krr = h->opts.task == GABP_TASK_KRR;
    for (int64_t i = 0; i < h->n; ++i)
        if ((krr ? std::fabs(a[(size_t)i]) : a[(size_t)i]) > th) {
            if (c < cap) idx[c] = (int32_t)i;
            ++c;
        }
    *count = c;
    return GABP_OK;
}

gabp_status gabp_svm_get_stats(gabp_svm_t h, gabp_svm_stats* st)
{
    g_err.clear();
    if (gabp_status s = check_handle(h)) return s;
    if (!st) return fail(GABP_EINVAL, "stats is NULL");
    h->stats.n = h->n;
    h->stats.m = h->m;
    h->stats.lambda = h->lambda;
    h->stats.gamma = h->gamma;
    h->stats.C = h->C;
    h->stats.diag_delta = h->delta;
    h->stats.device_bytes = (int64_t)(h->pool_bytes + h->spool_bytes);
    h->stats.q_mode = h->opts.q_mode;
    h->stats.diag_rule = h->opts.diag_rule;
    *st = h->stats;
    return GABP_OK;
}

gabp_status gabp_svm_get_q(gabp_svm_t h, float* Q)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    if (!Q) return fail(GABP_EINVAL, "Q is NULL");
    if (h->opts.q_mode == GABP_Q_RECOMPUTE) return fail(GABP_ESTATE, "Q is not stored in recompute mode");
    if (h->n > 46340) return fail(GABP_EINVAL, "n too large for a dense copy");
    const size_t bytes = (size_t)h->n * h->n * sizeof(float);
    float* d = nullptr;
    CK(cudaMallocAsync((void**)&d, bytes, h->stream));
    CK(cudaMemsetAsync(d, 0, bytes, h->stream));
    launch_get_q(h->inst, h->work, h->nlive, h->opts.q_mode == GABP_Q_BF16, d, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Q, d, bytes, h->opts.ptr_mode == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            h->stream);
    cudaFreeAsync(d, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(GABP_ECUDA, "get_q: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return GABP_OK;
}

gabp_status gabp_svm_get_pairs(gabp_svm_t h, const int64_t* i, const int64_t* j, int64_t cnt, float* out)
{
    g_err.clear();
    if (gabp_status s = check_formed(h)) return s;
    if (cnt < 0 || (cnt > 0 && (!i || !j || !out))) return fail(GABP_EINVAL, "bad pair list");
    if (cnt == 0) return GABP_OK;
    std::vector<long long> ij((size_t)cnt * 2);
    for (int64_t k = 0; k < cnt; ++k) {
        if (i[k] < 0 || j[k] >= h->n || i[k] >= j[k])
            return fail(GABP_EINVAL, "pair %lld: need 0 <= i < j < n", (long long)k);
        ij[2 * k] = i[k];
        ij[2 * k + 1] = j[k];
    }
    long long* dij = nullptr;
    float4* dout = nullptr;
    CK(cudaMallocAsync((void**)&dij, ij.size() * sizeof(long long), h->stream));
    CK(cudaMallocAsync((void**)&dout, (size_t)cnt * sizeof(float4), h->stream));
    CK(cudaMemcpyAsync(dij, ij.data(), ij.size() * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    launch_get_pairs(h->inst, dij, cnt, dout, h->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dout, (size_t)cnt * sizeof(float4), cudaMemcpyDeviceToHost, h->stream));
    cudaFreeAsync(dij, h->stream);
    cudaFreeAsync(dout, h->stream);
    CK(cudaStreamSynchronize(h->stream));
    return GABP_OK;
}

gabp_status gabp_svm_set_profiling(gabp_svm_t h, int32_t on)
{
    g_err.clear();
    if (gabp_status s = check_handle(h)) return s;
    if (on < 0) return fail(GABP_EINVAL, "profiling stride must be >= 0");
    h->profiling = on;
    return GABP_OK;
}

gabp_status gabp_svm_get_profile(gabp_svm_t h, gabp_svm_profile* out, int32_t reset)
{
    g_err.clear();
    if (gabp_status s = check_handle(h)) return s;
    if (!out) return fail(GABP_EINVAL, "out is NULL");
    *out = h->prof;
    if (reset) {
        const int64_t kl = h->prof.kernel_launches;
        h->prof = gabp_svm_profile{};
        h->prof.kernel_launches = kl;
    }
    return GABP_OK;
}

gabp_status gabp_selftest_bounded_wait(int64_t limit_ns)
{
    g_err.clear();
    if (limit_ns <= 0 || limit_ns > 10000000000LL) return fail(GABP_EINVAL, "limit_ns must be in (0, 1e10]");
    int* d = nullptr;
    int hst = -1;
    CK(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = launch_selftest_wait((unsigned long long)limit_ns, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&hst, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(GABP_ECUDA, "selftest: %s", cudaGetErrorString(e));
    if (hst == ST_ETIMEOUT) return fail(GABP_ETIMEOUT, "bounded device wait ran out after %lld ns", (long long)limit_ns);
    return hst == ST_OK ? GABP_OK : fail(GABP_ECUDA, "selftest returned %d", hst);
}

gabp_status gabp_selftest_reciprocal(const float* d, float* out, int64_t cnt)
{
    g_err.clear();
    if (cnt < 0 || cnt > (1LL << 30) || (cnt > 0 && (!d || !out))) return fail(GABP_EINVAL, "bad arguments");
    float *dd = nullptr, *dout = nullptr;
    CK(cudaMalloc(&dd, (size_t)cnt * 4 + 4));
    CK(cudaMalloc(&dout, (size_t)cnt * 4 + 4));
    cudaError_t e = cudaMemcpy(dd, d, (size_t)cnt * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_selftest_rcp(dd, dout, (int)cnt, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)cnt * 4, cudaMemcpyDeviceToHost);
    cudaFree(dd);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(GABP_ECUDA, "selftest_reciprocal: %s", cudaGetErrorString(e));
    return GABP_OK;
}

gabp_status gabp_svm_destroy(gabp_svm_t h)
{
    g_err.clear();
    destroy_all(h);
    return GABP_OK;
}

}  // extern "C"
