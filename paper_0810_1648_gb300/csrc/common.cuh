// Internal declarations shared by the CUDA sources of the GaBP SVM library.
//
// Geometry.  Q and the message state are kept for the upper triangle only,
// cut into T x T pair tiles (I, J) with I <= J, tile I holding nodes
// [I*T, I*T + T).  Tile L of the work list owns the contiguous slab
// [L*T*T, (L+1)*T*T) of every per-pair array, row-major inside the tile:
// pair (r, c) of the tile is node pair (I*T + r, J*T + c).  On diagonal
// tiles only c > r is used; on edge tiles only nodes < n.
//
// Per-pair message state (information form of Algorithm 2), two arrays in
// the tile layout: Pst = float2 {P_ij, P_ji} and Hst = float2 {H_ij, H_ji},
// i = I*T + r < j = J*T + c, where P_ij is the precision of the message
// i -> j and H_ij = P_ij mu_ij.  They are separate so that, once the P
// recursion (which does not depend on b) sits at its floating-point fixed
// point, a round reads P and streams only H.
//
// Per-node partial sums: every kernel that reduces over pairs writes, for
// node x and tile index k along the other axis, one value into
// part[a][k][x] (a = which sum).  For node x in tile row X = x / T the slot
// k > X comes from tile (X, k) (x as a row), k < X from tile (k, X) (x as a
// column) and k = X from the diagonal tile (both roles added).  Every slot is
// written exactly once per pass, so the reduction order is fixed.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace gabp {

constexpr int T = 128;                 // pair tile edge
constexpr int TT = T * T;
constexpr int NTHREADS = 256;          // threads per tile CTA
constexpr int NWARPS = NTHREADS / 32;
constexpr int KCH = 64;                   // features per BF16 operand block
constexpr int BLK_BYTES = T * KCH * 2;    // one 128 x 64 BF16 operand block (16 KB)

enum Status : int {
    ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENUMERIC = 4,
    ST_ETIMEOUT = 5, ST_ESTATE = 6
};

// Device-resident control block of one solver instance.  Kernels of a sweep
// read `t` and `done` from here, so a captured chunk of sweeps can be
// replayed from any starting round.
struct Ctrl {
    int t;                    // message updates applied since create/refit
    int done;                 // set once the solve must stop
    int limit;                // stop when t reaches this
    int kstar;                // round whose aggregates are the answer
    int converged;            // 1 if the residual test stopped the solve
    int status;               // first error (Status), 0 if none
    int zero_h;               // next sweep treats the H messages as 0 (restart of the b-dependent part)
    int p_frozen;             // P messages at their fixed point: sweeps no longer write them
    int p_changed;            // some P message changed in the current round
    int t_frozen;             // first round run with frozen P (valid when p_frozen)
    long long bad_index;      // offending node (or pair row) of the first error
    unsigned int blocks_done; // last-block-done counter of the finalize kernel
    unsigned long long rmax_bits;  // running max |r_i| of the round (bits of a nonnegative double)
    unsigned long long inv_margin_bits;  // max_i 1 / (Q_ii - R_i), R_i = sum_{j != i} |Q_ij| (bits of a
                                         // nonnegative double; +inf where a row is not strictly dominant),
                                         // set at formation: Varah's bound ||mu - Q^-1 b||_inf <=
                                         // ||b - Q mu||_inf * it
    double tol;
    double rinf;              // ||r(kstar)||_inf as seen by the convergence test
};

// One solver instance as the kernels see it.
struct Inst {
    int n;            // nodes (training points)
    int Nt;           // tiles per axis = ceil(n / T)
    int m;            // features
    int npad;         // stride of the per-node arrays inside agg
    const float* X;   // n x m FP32, row-major
    const float* sq;  // ||x_i||^2 of the FP32 rows
    const float* y;   // labels +-1
    const float* b;   // working right-hand side (b0, or a refinement residual)
    const float* b0;  // the problem's right-hand side: ones (SVM), the targets (KRR)
    float* qdiag;     // Q_ii
    void* Pst;        // ntiles * TT precision messages {P_ij, P_ji} (float2, or bf16x2 when msg_bf16)
    void* Hst;        // ntiles * TT information messages {H_ij, H_ji}
    void* qstore;     // ntiles * TT values of Q (float or bf16), or nullptr
    float* tilemax;   // per tile, the largest off-diagonal |Q_ij| (tile-sparse option), or nullptr
    const int* slab;  // tile-sparse option: slab of tile L = I Nt - I (I - 1) / 2 + (J - I) in the
                      // per-pair arrays (kept tiles are stored compacted), -1 for a dropped
                      // tile; nullptr = slab L (dense storage)
    float* qref;      // ntiles * TT FP32 values of Q for the residual passes (the FP32
                      // store itself, a separate copy beside the BF16 store, or nullptr
                      // when Q is recomputed)
    float* agg;       // [2][3][npad]: double-buffered {Ptilde, htilde, mutilde}
    float* aggmid;    // [2][npad]: {Ptilde, htilde} between the stages of a staged round
    float* part;      // [4][nslot][T] slot partial sums (slot_begin / slot_count / tile_slots)
    long long nslot;  // slots of each partial array: Nt * Nt, or the kept ones (tile-sparse option)
    const int* srow;  // tile-sparse option: block row I owns slots [srow[I], srow[I + 1]); nullptr = dense
    const int2* tslot;// tile-sparse option: slots {row role, column role} of swept tile w.w; nullptr = dense
    const double* rsum;  // tile-sparse option: the whole matrix's sum_{j != i} |Q_ij| per node (formation's
                         // first pass), for the diagonal rule; nullptr = summed from the slots
    unsigned long long* rfix;  // formation: where set, the |Q| row-sum partials are added to these
                               // per-node fixed-point sums (rsum_fix) instead of written to slots
    Ctrl* ctrl;
    double* rhist;    // ||r(t)||_inf per round (rhist_cap entries)
    int rhist_cap;
    float gamma;      // RBF width
    float lam2;       // lambda^2
    float C;          // box constant
    const void* Xp;   // BF16 features packed in tensor-core operand blocks (precision form)
    const float* sqb; // ||bf16(x_i)||^2
    int nkc;          // 64-feature chunks of Xp and Xp3
    const void* Xp3;  // the FP32 features as three BF16 planes in operand blocks (FP32 Gram on the tensor cores)
    float* sq3;       // x_i . x_i from the same tensor-core products as the Gram tiles (the norms the
                      // FP32 formation uses, so that the rounding of the norms and of the Gram values
                      // cancels in ||x_i||^2 + ||x_j||^2 - 2 x_i . x_j for near pairs)
    int msg_bf16;     // messages stored in BF16 (precision forms)
    int task;         // 0 SVM (labels in Q, alpha clipped to [0, C]), 1 KRR (y = 1 in Q, alpha unclipped)
    int form_next;    // formation: 1 + the next instance built from the same features (its Q
                      // tiles come from the same Gram tiles), 0 = none
};

// Slot partials.  Every node has one slot per tile it belongs to (a tile
// whose row block or column block is the node's block), ordered by the
// tile's other block index; slot s of an instance covers floats [s T, s T + T)
// of each partial array, one per node of the block.  Dense instances give
// block row I the slots I Nt .. I Nt + Nt - 1 (slot I Nt + k for the tile with
// block k); under the tile-sparse option block row I owns the compacted slots
// [srow[I], srow[I + 1]) of its kept tiles, in the same order, so that a
// node's sum over its slots adds the same values in the same order as the
// dense sum over all slots (those of dropped tiles hold 0).
__host__ __device__ inline long long slot_begin(const Inst& p, int I)
{
    return p.srow ? (long long)p.srow[I] : (long long)I * p.Nt;
}
__host__ __device__ inline int slot_count(const Inst& p, int I) { return p.srow ? p.srow[I + 1] - p.srow[I] : p.Nt; }
// Slots of the tile of work entry w = {instance, I, J, index}: {the row
// block's (its nodes I T + r), the column block's (nodes J T + c)}.
__host__ __device__ inline int2 tile_slots(const Inst& p, int4 w)
{
    if (p.tslot) return p.tslot[w.w];
    return make_int2(w.y * p.Nt + w.z, w.z * p.Nt + w.y);
}
// Floats of each partial array.
__host__ __device__ inline size_t part_len(const Inst& p) { return (size_t)p.nslot * T; }

// The |Q| row sums R_i = sum_{j != i} |Q_ij| of the diagonal rule are added up
// in fixed point: each FP32 slot partial v becomes the integer nearest to
// v 2^s, the integers are summed, and R_i = (that sum) 2^-s.  Integer addition
// does not depend on the order of its terms, so the dense slot sums and the
// tile-sparse first pass's atomic sums (no slots) give the same R bit for bit.
// s is the largest shift that keeps every possible sum below 2^62: each entry
// is at most 1 + lambda^2 (an RBF value plus the bias term; 1% room for the
// rounding of the entries), a row has fewer than n of them.  The resolution
// 2^-s is below 1e-15 R_max.
__host__ __device__ inline int rsum_shift(int n, float lam2)
{
    int e = 0;
    frexp(1.01 * (double)(n > 2 ? n : 2) * (1.0 + (double)lam2), &e);   // bound < 2^e
    return 62 - e;
}
// 2^s for |s| < 1000, built from the exponent field.
__device__ __forceinline__ double pow2i(int s) { return __longlong_as_double((long long)(1023 + s) << 52); }
__device__ __forceinline__ long long rsum_fix(float v, double scale) { return __double2ll_rn((double)v * scale); }
__device__ __forceinline__ double rsum_unfix(long long a, int shift) { return __ll2double_rn(a) * pow2i(-shift); }

// Work of one round over a set of instances (device resident, so that a
// captured round stays valid while the set changes).  Tile list entries are
// int4 {instance, I, J, tile index within the instance}; node-block list
// entries are int2 {instance, block of 32 nodes}.
// Under the staged (block Gauss-Seidel) schedule a round has one Sched per
// stage, each naming its segment [off, off + ntiles) of the tile list.
struct Sched {
    long long ntiles;
    int nblocks;
    int ninst;
    long long off;
    int nsmall;   // node blocks [0, nsmall) of the list: instances with Nt <= kWarpFinNt (one warp each at finalize)
    int pad_;
};
constexpr int kWarpFinNt = 32;
constexpr int kMaxStages = 16;

// Stage boundaries of the staged schedule for Nt tile rows: B[0] = 0,
// B[S] = Nt, B[s] = the smallest b with S b (b + 1) / 2 >= s Nt (Nt + 1) / 2
// (about equal tile counts per stage); tile (I, J) runs in the stage whose
// range [B[s], B[s+1]) holds J.
__host__ __device__ inline void stage_bounds(int Nt, int S, int* B)
{
    const long long tot = (long long)Nt * (Nt + 1) / 2;
    B[0] = 0;
    for (int s = 1; s < S; ++s) {
        long long b = B[s - 1];
        while (b < Nt && (long long)S * (b * (b + 1) / 2) < (long long)s * tot) ++b;
        B[s] = (int)b;
    }
    B[S] = Nt;
}

// What the end-of-solve kernels do for one instance (indexed by its slot):
// final residual / objective / alpha of the means `mu`, the FP32 residual to
// r_out when not null, and (refinement) acc = mu(axpy_buf) or acc += it first.
struct StopOp {
    const float* mu;
    float* r_out;
    float* alpha;
    double* blockbuf;
    double* final3;
    float* acc;
    int axpy_buf;
    int axpy_first;
    float sv_threshold;
    int pad;
};

// Launch shapes of one round (persistent sweep CTAs, finalize CTAs).
struct RoundGrid {
    int sweep = 1;
    int finalize = 1;
};

// Gram operands: rows [0, n) of an n x m FP32 matrix with row norms sq.
struct GramSide {
    const float* X;
    const float* sq;
    int n;
};

// ---- launchers (defined in the .cu files) --------------------------------
// Inputs: convert/validate X and y, row norms, right-hand sides.  SVM (task 0):
// y must be +-1, b = b0 = 1.  KRR (task 1): y holds finite targets, which move
// to b and b0, and y becomes 1 (no labels in Q).  y, b, b0 may be null (test
// points).  Returns nothing; errors go to ctrl->status.
void launch_stage(const void* X, int x_dtype, int n, int m, float* y, float* Xf, float* sq,
                  float* b, float* b0, int task, Ctrl* ctrl, cudaStream_t s);
// Bytes of one feature of the input layout x_dtype (0 FP32, 1 FP64, 2 BF16).
inline size_t x_elem_bytes(int x_dtype) { return x_dtype == 1 ? 8 : x_dtype == 2 ? 2 : 4; }
// Refinement schedule of the precision forms (0 selects the default): the
// first solve hands over to the defect correction at ||r||_inf < handover, each
// correction pass stops at inner * ||r||_inf of its right-hand side.
inline double refine_handover(float opt, int msg_bf16) { return opt > 0 ? opt : (msg_bf16 ? 1e-3 : 1e-4); }
inline double refine_inner(float opt, int msg_bf16) { return opt > 0 ? opt : (msg_bf16 ? 3e-2 : 1e-2); }

// Q formation (FP32-accurate Gram on the tensor cores from three BF16 planes,
// fused with exp, labels and bias) + |Q| row-sum partials; the FP32 tiles are
// stored into Inst::qref where it is set (the FP32 store, or the FP32 copy the
// BF16 store keeps for its refinement residuals), the tile maxima into
// Inst::tilemax where it is set.  Needs Inst::Xp3 packed first.
// norms_only = 1: over a list of diagonal tiles (I, I), writes Inst::sq3 of the
// listed instances (and those chained behind them) and nothing else; it must
// run before the formation of their other tiles.
cudaError_t launch_form_q_tc32(const Inst* tab, const int4* work, long long ntiles, int norms_only, cudaStream_t s);
inline void launch_form_q(const Inst* tab, const int4* work, long long ntiles, cudaStream_t s)
{
    (void)launch_form_q_tc32(tab, work, ntiles, 0, s);   // errors surface at the caller's cudaGetLastError
}
inline void launch_form_norms(const Inst* tab, const int4* diag_work, long long ntiles, cudaStream_t s)
{
    (void)launch_form_q_tc32(tab, diag_work, ntiles, 1, s);
}
// The three BF16 planes of FP32 rows (zero padding to whole tiles and chunks).
cudaError_t launch_pack3(const float* Xf, int n, int m, int Nt, void* Xp3, cudaStream_t s);
cudaError_t launch_pack3_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s);
size_t pack3_bytes(int Nt, int m);
// Precision form: BF16 operand packing + norms, and the tensor-core Q formation (BF16 store).
cudaError_t launch_pack_bf16(const float* Xf, int n, int m, int nkc, int Nt, void* Xp, float* sqb, cudaStream_t s);
cudaError_t launch_form_q_tc(const Inst* tab, const int4* work, long long ntiles, cudaStream_t s);
int bf16_chunks(int m);
size_t bf16_pack_bytes(int Nt, int m);
// Restart: Step-1 aggregates from the stored diagonal and b, t = 0.
void launch_reset(const Inst& p, cudaStream_t s);

// Diagonal rule, Step-1 aggregates and control reset.
void launch_init(const Inst& p, int diag_rule, float delta, cudaStream_t s);
// rsum[x] = R_x from the fixed-point sums that the formation's first pass
// added into rfix (the same memory, converted in place).
void launch_row_abs_sums(const Inst& p, double* rsum, cudaStream_t s);
// Solve control: arm the control blocks of tab[0..ninst) for `iters` more rounds with tolerance `tol`.
void launch_begin(Inst* tab, int ninst, int iters, double tol, cudaStream_t s);
int num_sms();
// Grid of a round for up to max_tiles tiles and max_nblocks node blocks
// (ctas_per_sm: sweep CTAs per SM for the stored-Q kernels, 0 = default).
RoundGrid round_grid(long long max_tiles, int max_nblocks, int q_mode, int ctas_per_sm, int msg_bf16);
// Raises the dynamic shared-memory limit of the pair-sweep kernels (once per device).
cudaError_t prepare_sweep();
// Fused-recompute form: also raises the shared-memory limit of its sweep kernel.
cudaError_t prepare_sweep_rc();
// One round over every live instance of tab: pair sweep then per-node
// finalize.  When ev is not null, ev[0] is recorded before the (first stage's)
// pair sweep and ev[1] after the (last stage's) pair sweep.
// nstages > 1: the staged schedule, sched[0 .. nstages-1] one per stage, a
// stage finalize (aggregates only) between the stages.
void launch_round(const Inst* tab, const int4* work, const int2* nbl, const Sched* sched, int nstages,
                  const RoundGrid& g, int q_mode, int msg_bf16, cudaStream_t s, cudaEvent_t* ev = nullptr);
// Final FP32-Gram residual r = 1 - Q mu (FP64 sums), dual objective and
// alpha = clip(mu, 0, C) of the listed instances (their tiles, node blocks
// and slots), per ops[slot]; results in ops[slot].final3 and f3_all[3 slot].
// q_stored: the instances keep FP32 Q tiles (Inst::qref), read instead of
// recomputing the Gram.
void launch_final(const Inst* tab, const StopOp* ops, const int4* tiles, long long ntiles, const int2* nbl,
                  int nblocks, const int* members, int nmembers, double* f3_all, int q_stored, cudaStream_t s);
// Refinement over listed node blocks: acc (+)= mutilde (ops[slot].axpy_*).
void launch_axpy_list(const Inst* tab, const StopOp* ops, const int2* nbl, int nblocks, cudaStream_t s);
// Refinement over listed node blocks: b := ops[slot].r_out, H restarts.
void launch_refine_rhs_list(const Inst* tab, const StopOp* ops, const int2* nbl, int nblocks, cudaStream_t s);
// Formation over listed node blocks of several instances (FP32 rows already in X):
// staging checks / norms / b = 1; BF16 packing + norms; diagonal rule + Step 1.
void launch_stage_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s);
cudaError_t launch_pack_list(const Inst* tab, const int2* nbl, int nblocks, cudaStream_t s);
void launch_init_list(const Inst* tab, const int2* nbl, int nblocks, int diag_rule, float delta, cudaStream_t s);
// Arms listed instances: list entries {slot, iters} with their tolerances.
void launch_begin_list(Inst* tab, const int2* list, const double* tols, int count, cudaStream_t s);
// Decision values for t test rows (Xt FP32, sqt norms) using alpha.
void launch_decision(const Inst& p, const float* Xt, const float* sqt, int t, const float* alpha,
                     const int2* work, long long ntiles, float* part, float* out, cudaStream_t s);
// Gather helpers for inspection.
void launch_get_q(const Inst& p, const int4* work, long long ntiles, int q_bf16, float* Qdense,
                  cudaStream_t s);
void launch_get_pairs(const Inst& p, const long long* ij, long long cnt, float4* out,
                      cudaStream_t s);

// Reciprocal used by the pair sweep, evaluated on d[0..cnt) (device arrays).
cudaError_t launch_selftest_rcp(const float* d, float* out, int cnt, cudaStream_t s);
// Bounded-wait self test: writes ST_ETIMEOUT to *status_dev once limit_ns ran out.
cudaError_t launch_selftest_wait(unsigned long long limit_ns, int* status_dev, cudaStream_t s);
// Sets the thread-local message returned by gabp_last_error().
void set_last_error(const char* msg);
// Device memory available to the library: cudaMemGetInfo's free bytes plus
// what the device's default stream-ordered pool holds reserved but unused
// (instance memory of the batched and served forms goes back to that pool and
// stays reserved for reuse).  trim = true first returns the pool's unused
// memory to the device (for plain cudaMalloc callers).
cudaError_t device_available(size_t* avail, bool trim);
// Host-side fault injection for tests of the failure paths: the environment
// variable GABP_FAULT holds comma-separated tokens, read at each public call:
//   alloc    the call's device allocation fails (create, batch, server admission)
//   nan      a non-finite label or target reaches the staging checks (create, refit)
//   timeout  the device reports a bounded wait that ran out during the next rounds
// Returns the FAULT_* bits, or -1 for an unknown token.
enum FaultBits { FAULT_ALLOC = 1, FAULT_NAN = 2, FAULT_TIMEOUT = 4 };
int fault_mask();

// NVTX range over a host-side phase (formation, rounds, final pass,
// refinement, decision, batch and server phases), shown by profilers that
// record NVTX; without one attached a push/pop pair costs a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- small device helpers --------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// Tile index along the triangle -> slot k for node x (see the header comment).
__host__ __device__ __forceinline__ long long tri_tiles(long long Nt) { return Nt * (Nt + 1) / 2; }

}  // namespace gabp
