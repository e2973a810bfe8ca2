// Batches of independent cyclic problems (uneven m and N): fold in one launch,
// cyclic Sinkhorn in two persistent launches (one per rows-per-chunk class,
// see chunk_rows).
//
// Solver (Algorithm 2 per problem, log domain, the same iteration and stopping
// rule as ot_sinkhorn_reduced).  Two bounded grid barriers per sweep:
//
//  row phase    The rows of the launch's still-active problems form one index
//               space weighted by estimated row cost; every block takes a
//               contiguous, equally weighted range of it (recomputed
//               identically in every block each sweep, so finished problems
//               free their share).  A block streams chunks of rows (two or
//               three per thread group) through shared-memory stages filled by
//               bulk copies, together with the rows' scalars (previous
//               potential, its lo factor, the row marginal).  A group of GS
//               threads owns a fixed set of columns; it forms the
//               exponentials of its chunk rows around the
//               previous potentials in registers, releases the stage (so that
//               the next copy starts while the row sums are reduced), then
//               writes the new row potentials and adds the column
//               contributions u_i e_ij to compensated sums in registers.  At
//               the end of a problem segment these are added into the
//               problem's column sums with FP32 reductions (a problem is split
//               over few blocks, so each sum receives few terms).  The row L1
//               terms go to a per-problem FP64 accumulator.
//  column phase The columns of the active problems are split the same way;
//               each column's potential is updated from its sum (FP64), the
//               sum is cleared, and the block holding a problem's column 0
//               applies the stopping rule: a finished problem's state (after
//               t-1 iterations) is frozen and recorded.
//
// When no problem is active, every block writes the outputs of its share.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace cyc {

int device_sms();

#define OT_BATCH_MAX 1024     // problems per batch
#define OT_BATCH_MAXM 8192    // largest block size
#define OT_BT 512             // threads per block
#define OT_BW (OT_BT / 32)
#define OT_BV 4               // float4 column slots per thread and row
#define OT_STAGES_MAX 2       // chunks in flight per block (bulk copies into shared memory)
#define OT_ISSUER (OT_BT - 32) // issues the copies: lane 0 of the last warp (the first warp of a group
                               // writes the pending potentials; a warp doing both lags at every reduction)
#ifndef OT_ROW_FIXED
#define OT_ROW_FIXED 8        // per-chunk cost of a group that does not scale with its slots, in slots
#endif
#define OT_BATCH_NCFG 6       // tunable launch configurations (see decode_cfg)

struct BatchArgs {
    int count;
    long long total_m;
    const float* G;
    const float* a;
    const float* b;
    double tol;
    int max_iter;
    unsigned long long timeout_ns;
    int warm;
    int gs_shift;                  // group-size policy (0: tight, 1: one size larger)
    int check_every;               // the stopping rule is applied every check_every iterations
    const int* nrows;              // [2][2] problems per group-size shift and rows per chunk (null: not counted)
    double* w_out;
    double* z_out;
    ot_result* res;
    // workspace
    Ctrl* ctrl;
    const ot_problem_desc* desc;   // [count]
    double* inv_sa;                // [count]
    double* inv_sb;                // [count]
    int* active;                   // [count]
    int* iters;                    // [count]
    double* l1acc;                 // [2][count]
    float4* rs;                    // [2][total_m] row scalars {hi part of the row potential (log2 units),
                                   //  2^lo, alpha_i = a_i / sum a, 0}; the potential is hi + lo exactly
    float* flo;                    // [2][total_m] lo part of the row potential
    double* gam;                   // [total_m]
    float* gc;                     // [total_m]
    float* cf;                     // [total_m]
    float* R;                      // [total_m] column sums
};

// Rows per group and chunk: three when a thread's row slice fills three float4
// slots (the per-chunk costs that do not grow with the row, the group reduction
// above all, are then shared by three rows), otherwise two.  A stage holds the
// larger of two rows of 8192 and three of 6144 floats.
#define OT_STAGE_FLOATS (3 * 3 * OT_BATCH_MAXM / 4)
#define OT_RSC_STAGE (3 * OT_BW)   // row scalars per stage (float4)
static_assert(OT_STAGE_FLOATS >= 2 * OT_BATCH_MAXM, "a stage holds two of the longest rows");

// Dynamic shared memory of the solver: OT_STAGES_MAX chunk stages (two or three
// rows per group, and their rows' scalars) filled by bulk copies, the current
// problem's staged column data, prefix sums, block sizes, row weights and active
// flags.
constexpr size_t a128(size_t x) { return (x + 127) & ~(size_t)127; }
struct BatchSmem {
    static constexpr size_t stage = 0;
    static constexpr size_t rsc = a128(stage + sizeof(float) * OT_STAGE_FLOATS * OT_STAGES_MAX);
    static constexpr size_t gc = a128(rsc + sizeof(float4) * OT_RSC_STAGE * OT_STAGES_MAX);
    static constexpr size_t cf = a128(gc + sizeof(float) * OT_BATCH_MAXM);
    static constexpr size_t pref = a128(cf + sizeof(float) * OT_BATCH_MAXM);
    static constexpr size_t msz = a128(pref + sizeof(long long) * (OT_BATCH_MAX + 1));
    static constexpr size_t rw = a128(msz + sizeof(unsigned short) * OT_BATCH_MAX);
    static constexpr size_t act = a128(rw + sizeof(unsigned short) * OT_BATCH_MAX);
    static constexpr size_t total = a128(act + sizeof(unsigned char) * OT_BATCH_MAX);
};
static_assert(4 * OT_BV * OT_BT == OT_BATCH_MAXM, "a full block covers the longest row");
static_assert(OT_BATCH_MAXM <= 65535, "block sizes are kept as 16-bit integers");
static_assert(BatchSmem::total + 2048 <= 227 * 1024, "shared memory");

__device__ __forceinline__ void red_add_f32(float* p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// ---- packed FP32 pairs (f32x2 instructions: two lanes of arithmetic per instruction)
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Compensated (Kahan) addition on both lanes of the contribution sum_r u_r e_r
// of a chunk's rows: sum - nc carries the running total of the added values to
// about one rounding, however many rows a thread accumulates (nc is the negated
// compensation, so the contributions and the compensation enter through FMAs).
template <int R>
__device__ __forceinline__ void kahan_rows(f32x2& sum, f32x2& nc, const f32x2 (&u)[R], const f32x2 (&e)[R]) {
    f32x2 y = nc;
#pragma unroll
    for (int r = 0; r < R; ++r) y = fma2(u[r], e[r], y);
    const f32x2 t = add2(sum, y);
    nc = sub2(y, sub2(t, sum));
    sum = t;
}

// The two-row engine's compensated addition: kahan_rows<2> with scalar arguments.
__device__ __forceinline__ void kahan2(f32x2& sum, f32x2& nc, f32x2 u0, f32x2 e0, f32x2 u1, f32x2 e1) {
    const f32x2 y = fma2(u1, e1, fma2(u0, e0, nc));
    const f32x2 t = add2(sum, y);
    nc = sub2(y, sub2(t, sum));
    sum = t;
}

// ---- mbarrier helpers of the row engine
__device__ __forceinline__ void mbar_arrive_cnt(unsigned long long* bar, unsigned cnt) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(cnt)
                 : "memory");
}

// Bounded wait that also gives up at once when the block has aborted.
__device__ __forceinline__ bool mbar_wait_ab(unsigned long long* bar, unsigned parity,
                                             unsigned long long timeout_ns, const volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (globaltimer() - t0 > timeout_ns) return false;
    }
    return true;
}

// Thread-group size of a problem's rows: the smallest power of two >= 32 whose
// OT_BV float4 slots per thread cover the row stride (one size larger per shift).
__host__ __device__ __forceinline__ constexpr int group_size(int ld, int shift) {
    int gs = 32;
    while (gs < OT_BT && gs * 4 * OT_BV < ld) gs <<= 1;
    gs <<= shift;
    return gs < OT_BT ? gs : OT_BT;
}

// Float4 slots of a row that each thread of its group covers (1 .. OT_BV).
__host__ __device__ __forceinline__ constexpr int row_slots(int ld, int shift) {
    const int gs = group_size(ld, shift);
    return (ld + 4 * gs - 1) / (4 * gs);
}

// Rows per group and chunk (see OT_STAGE_FLOATS).
__host__ __device__ __forceinline__ constexpr int chunk_rows(int slots) { return slots == 3 ? 3 : 2; }

// Every chunk fits its stage: R rows of ld floats for each of the OT_BT / GS groups, and
// their R * OT_BT / GS row scalars, for every row stride and group-size policy.
constexpr bool stages_hold_every_chunk() {
    for (int sh = 0; sh < 2; ++sh)
        for (int ld = 4; ld <= OT_BATCH_MAXM; ld += 4) {
            const int gs = group_size(ld, sh), rows = chunk_rows(row_slots(ld, sh)) * (OT_BT / gs);
            if ((long long)rows * ld > OT_STAGE_FLOATS || rows > OT_RSC_STAGE) return false;
        }
    return true;
}
static_assert(stages_hold_every_chunk(), "a chunk exceeds its shared-memory stage");

// Estimated cost of one row of a problem, the unit of the row phase's work split:
// a chunk costs its group a fixed part (OT_ROW_FIXED slots) plus half a slot per
// filled float4 slot and row, and holds R rows per group, so a row costs
// GS (OT_ROW_FIXED / R + slots / 2) thread slots; times 6 to stay integral.
// Splitting by bytes instead would give blocks with short rows more chunks than
// the others.
__host__ __device__ __forceinline__ int row_weight(int ld, int shift) {
    const int gs = group_size(ld, shift);
    const int slots = row_slots(ld, shift);
    return gs * (6 * OT_ROW_FIXED / chunk_rows(slots) + 3 * slots);
}

// Block-wide exclusive scan of the per-problem weights (m x row weight for rows,
// m for columns; 0 for finished problems) into s_pref[0..count].
__device__ void batch_prefix(int count, const unsigned short* s_m, const unsigned short* s_rw,
                             const unsigned char* act, bool rows, long long* s_pref, long long* s_wsum) {
    // each thread sums a contiguous chunk, then a warp scan of the chunk sums
    const int tid = threadIdx.x;
    const int per = (count + OT_BT - 1) / OT_BT;
    const int p0 = tid * per, p1 = min(count, p0 + per);
    long long loc = 0;
    for (int p = p0; p < p1; ++p) {
        const long long m = s_m[p];
        loc += act[p] ? (rows ? m * s_rw[p] : m) : 0;
    }
    const int lane = tid & 31, wid = tid >> 5;
    long long v = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) s_wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long x = lane < OT_BW ? s_wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < OT_BW) s_wsum[lane] = x;
    }
    __syncthreads();
    long long base = (wid > 0 ? s_wsum[wid - 1] : 0) + v - loc;
    for (int p = p0; p < p1; ++p) {
        s_pref[p] = base;
        const long long m = s_m[p];
        base += act[p] ? (rows ? m * s_rw[p] : m) : 0;
    }
    if (tid == OT_BT - 1) s_pref[count] = base;
    __syncthreads();
}

// Largest p with s_pref[p] <= x (problems with zero weight are skipped by the caller).
__device__ __forceinline__ int find_problem(const long long* s_pref, int count, long long x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pref[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- thread groups of the row phase
//
// A problem segment is processed by groups of GS threads (GS = 32 .. 512, the
// smallest power of two whose OT_BV float4 slots per thread cover the row
// stride).  Thread gt of a group owns the float4 column slots gt + v * GS for
// the whole segment, so its column contributions stay in registers until the
// segment ends.  A group reduction is an xor butterfly inside each warp and,
// for multi-warp groups, one named barrier and a butterfly over the warp
// partials: every thread of the group obtains bit-identical row sums, so the
// data-dependent branches below are uniform across the group.

__device__ __forceinline__ void group_barrier(int gs, int q) {
    if (gs > 32) asm volatile("bar.sync %0, %1;" ::"r"(q + 1), "r"(gs) : "memory");
    else __syncwarp();
}

// All-reduce of R values (the rows of a chunk) over a group.  A warp's partials
// sit in one 8-byte (two rows) or 16-byte (three rows) slot of s_part per warp.
template <bool MAX, int R>
__device__ __forceinline__ void group_allreduce(float (&v)[R], int gs, float* s_part, int& parity) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = __shfl_xor_sync(0xffffffffu, v[r], o);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = MAX ? fmaxf(v[r], a[r]) : v[r] + a[r];
    }
    if (gs > 32) {
        const int tid = threadIdx.x, lane = tid & 31, nw = gs >> 5, w0 = (tid >> 5) & ~(nw - 1);
        float x[R];
        if (R == 2) {
            float2* part = reinterpret_cast<float2*>(s_part) + parity * OT_BW;
            if (lane == 0) part[tid >> 5] = make_float2(v[0], v[1 % R]);
            group_barrier(gs, tid / gs);
            // every aligned run of nw lanes holds the nw partials and combines them in the same tree
            const float2 x2 = part[w0 + (lane & (nw - 1))];
            x[0] = x2.x;
            x[1 % R] = x2.y;
        } else {
            float4* part = reinterpret_cast<float4*>(s_part) + parity * OT_BW;
            if (lane == 0) part[tid >> 5] = make_float4(v[0], v[1 % R], v[2 % R], 0.f);
            group_barrier(gs, tid / gs);
            const float4 x4 = part[w0 + (lane & (nw - 1))];
            x[0] = x4.x;
            x[1 % R] = x4.y;
            x[2 % R] = x4.z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o < nw) {
                float a[R];
#pragma unroll
                for (int r = 0; r < R; ++r) a[r] = __shfl_xor_sync(0xffffffffu, x[r], o);
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = MAX ? fmaxf(x[r], a[r]) : x[r] + a[r];
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[r];
        parity ^= 1;   // the next reduction writes the other buffer (one barrier separates reuse)
    }
}

// The two-row engine's all-reduce of two values (the two rows of a chunk) over a
// group: group_allreduce<MAX, 2> with scalar arguments.
template <bool MAX>
__device__ __forceinline__ void group_allreduce2(float& v0, float& v1, int gs, float* s_part, int& parity) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, v0, o), b = __shfl_xor_sync(0xffffffffu, v1, o);
        v0 = MAX ? fmaxf(v0, a) : v0 + a;
        v1 = MAX ? fmaxf(v1, b) : v1 + b;
    }
    if (gs > 32) {
        const int tid = threadIdx.x, lane = tid & 31, nw = gs >> 5, w0 = (tid >> 5) & ~(nw - 1);
        if (lane == 0) {
            s_part[(parity * OT_BW + (tid >> 5)) * 2] = v0;
            s_part[(parity * OT_BW + (tid >> 5)) * 2 + 1] = v1;
        }
        group_barrier(gs, tid / gs);
        // every aligned run of nw lanes holds the nw partials and combines them in the same tree
        const float2 x = reinterpret_cast<const float2*>(s_part)[parity * OT_BW + w0 + (lane & (nw - 1))];
        float x0 = x.x, x1 = x.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o < nw) {
                const float a = __shfl_xor_sync(0xffffffffu, x0, o), b = __shfl_xor_sync(0xffffffffu, x1, o);
                x0 = MAX ? fmaxf(x0, a) : x0 + a;
                x1 = MAX ? fmaxf(x1, b) : x1 + b;
            }
        }
        v0 = x0;
        v1 = x1;
        parity ^= 1;   // the next reduction writes the other buffer (one barrier separates reuse)
    }
}

struct SegCtx {
    const float* Gp;
    float4* rs_nxt;   // row scalars written by this sweep (problem-local)
    float* flo_nxt;
    const float4* rs_cur;   // row scalars of the previous iterate (problem-local)
    int gs, m, ld, ng4, r_lo, r_hi, t, ng, nchunks;
    float kap;
};

// The staged column data of the current problem (shared memory): hi parts of
// the column potentials and their lo factors (padding: -inf and 0).
struct ColData {
    const float4* gc;
    const float4* cf;
};

// Exponentials of a float4 of costs around the potential F (log2 units):
// 2^(gamma_j - kap c_j + F), two lanes per f32x2 instruction.
__device__ __forceinline__ float4 exps4(const float4 c, const float4 gg, f32x2 nk2, f32x2 F2) {
    const float2 x01 = upk(add2(fma2(pk(c.x, c.y), nk2, pk(gg.x, gg.y)), F2));
    const float2 x23 = upk(add2(fma2(pk(c.z, c.w), nk2, pk(gg.z, gg.w)), F2));
    return make_float4(ex2(x01.x), ex2(x01.y), ex2(x23.x), ex2(x23.y));
}

// S += e . c on both lanes of a packed accumulator.
__device__ __forceinline__ f32x2 dot4x2(const float4 e, const float4 c, f32x2 S) {
    return fma2(pk(e.z, e.w), pk(c.z, c.w), fma2(pk(e.x, e.y), pk(c.x, c.y), S));
}

__device__ __forceinline__ float hsum(f32x2 v) {
    const float2 x = upk(v);
    return x.x + x.y;
}

// Pipeline state of a block: chunks are numbered in the order the block
// consumes them (across segments and sweeps); chunk n uses stage n % STAGES and
// completes phase (n / STAGES) & 1 of that stage's full and empty barriers.
// Every warp arrives once on a chunk's empty barrier when it no longer reads the
// stage; thread OT_ISSUER issues the copies.
struct Pipe {
    float* stage;                 // [STAGES][OT_STAGE_FLOATS]
    float4* rsc;                  // [STAGES][OT_RSC_STAGE] scalars of the chunk's rows
    unsigned long long* full;     // [STAGES]
    unsigned long long* empty;    // [STAGES] (OT_BW arrivals)
    volatile int* abort;          // set by the first expired wait; later waits give up at once
    long long consumed;           // chunks consumed so far (every thread)
    long long issued;             // chunks issued so far (thread OT_ISSUER)
};

__device__ __forceinline__ void abort_block(const BatchArgs& A, const Pipe& P) {
    if (!*P.abort) {
        *P.abort = 1;
        set_status(A.ctrl, OT_ERR_TIMEOUT);
    }
}

// The warp no longer reads the current chunk's stage.
template <int STAGES>
__device__ __forceinline__ void stage_release(const Pipe& P) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive_cnt(&P.empty[P.consumed % STAGES], 1u);
}

// Chunk k of a segment (thread OT_ISSUER): rows r_lo + R k NG .. (R NG consecutive rows,
// R per group) and their scalars, two bulk copies (rows are contiguous with
// stride ld; all sizes and addresses 16-byte multiples).  The stage is taken
// once every warp has released the chunk that used it before.  (No proxy fence
// before a refill: the stage was only read through the generic proxy, and the
// release/acquire pair on the empty barrier orders those reads first.)
template <int STAGES, int R>
__device__ __forceinline__ void issue_chunk(Pipe& P, const SegCtx& X, int k, const BatchArgs& A) {
    const long long n = P.issued;
    const int st = (int)(n % STAGES);
    if (n >= STAGES && !mbar_wait_ab(&P.empty[st], (unsigned)(((n - STAGES) / STAGES) & 1), A.timeout_ns, P.abort))
        abort_block(A, P);
    if (*P.abort) return;
    const int r0 = X.r_lo + R * k * X.ng;
    const int nr = min(R * X.ng, X.r_hi - r0);
    const unsigned bytes = (unsigned)nr * (unsigned)X.ld * 4u, sbytes = (unsigned)nr * 16u;
    unsigned long long* bar = &P.full[st];
    mbar_arrive_expect_tx(bar, bytes + sbytes);
    bulk_g2s(P.stage + (size_t)st * OT_STAGE_FLOATS, X.Gp + (long long)r0 * X.ld, bytes, bar);
    bulk_g2s(P.rsc + st * OT_RSC_STAGE, X.rs_cur + r0, sbytes, bar);
    P.issued = n + 1;
}

// A row whose new potential is still to be written: lane R kk + r of a group's
// first warp holds row r of the group's kk-th chunk in a window of 32 / R chunks,
// and that warp writes the window's rows at once (no serial chain of special
// functions on one lane per chunk).
struct Pending {
    float S, F, al;
    int row;   // -1: none
};

// New potential F - log2(S / alpha) of a pending row, held exactly as hi + lo (TwoSum).
__device__ __forceinline__ void finish_pending(const BatchArgs& A, const SegCtx& X, Pending& pd) {
    if (pd.row < 0) return;
    if (pd.S > 1e-30f && pd.S < 1e30f) {
        const float b = -lg2(__fdividef(pd.S, pd.al));
        const float hi = __fadd_rn(pd.F, b);
        const float bv = __fsub_rn(hi, pd.F);
        const float lo = __fadd_rn(__fsub_rn(pd.F, __fsub_rn(hi, bv)), __fsub_rn(b, bv));
        X.rs_nxt[pd.row] = make_float4(hi, ex2(lo), pd.al, 0.f);
        X.flo_nxt[pd.row] = lo;
    } else {
        set_status(A.ctrl, OT_ERR_NONFINITE);
    }
    pd.row = -1;
}

// Row update of the R rows of a chunk held by a group (Eq.
// optimal_f_sinkhorn_logdomain in log2 units): S_r = sum_j 2^(gamma_j - kap c_rj + F_r)
// around the previous potential F_r, new potential F_r - log2(S_r / alpha_r)
// kept exactly as hi + lo (recorded in pd, written by finish_pending), column
// contributions (alpha_r / S_r) e_rj added to acc.  An explicit max shift is used
// on the first sweep and whenever a row sum leaves the safe range (then from the
// rows in global memory: the stage may already be refilled).  V float4 slots per
// thread and row cover the row (V = OT_BV for two rows, 3 for three).
template <int STAGES, int R, int V>
__device__ __forceinline__ void process_rows(const float* srow, const float4* srsc, const BatchArgs& A,
                                             const SegCtx& X, int row, int k, int kk, const ColData& CR,
                                             float* s_part, int& parity, f32x2 (&acc)[2 * V], f32x2 (&cmp)[2 * V],
                                             float& l1, Pending& pd, Pipe& P) {
    const int GS = X.gs, gt = threadIdx.x & (GS - 1);
    // row r of the chunk exists iff ok[r] (uniform over the group; the caller guarantees row 0);
    // a missing row is processed as a copy of the first and gets no weight: the hot loops carry
    // no test for it
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ok[r] = r == 0 || row + r < X.r_hi;
    const int ep = R * kk;   // lanes of the group's first warp that hold the rows until they are finished
    float4 sc[R];
    const float4* c[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rr = ok[r] ? r : 0;
        sc[r] = srsc[rr];
        c[r] = reinterpret_cast<const float4*>(srow + rr * X.ld);
    }
    const f32x2 nk2 = pk(-X.kap, -X.kap);
    float4 e[R][V];
    float F[R], S[R];
#pragma unroll
    for (int r = 0; r < R; ++r) F[r] = sc[r].x;
    const bool first = X.t == 1;
    bool shifted = first;
    if (!shifted) {
        f32x2 F2[R], S2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            F2[r] = pk(F[r], F[r]);
            S2[r] = pk(0.f, 0.f);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int g = gt + v * GS;
#pragma unroll
            for (int r = 0; r < R; ++r) e[r][v] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < X.ng4) {
                const float4 gg = CR.gc[g], cc = CR.cf[g];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    e[r][v] = exps4(c[r][g], gg, nk2, F2[r]);
                    S2[r] = dot4x2(e[r][v], cc, S2[r]);
                }
            }
        }
        stage_release<STAGES>(P);
#pragma unroll
        for (int r = 0; r < R; ++r) S[r] = hsum(S2[r]);
        group_allreduce<false, R>(S, GS, s_part, parity);
        if (threadIdx.x == OT_ISSUER && k + STAGES < X.nchunks) issue_chunk<STAGES, R>(P, X, k + STAGES, A);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (ok[r] && gt == ep + r) l1 += fabsf(fmaf(S[r], sc[r].y - 1.0f, S[r] - sc[r].z));
            // uniform over the group
            if (ok[r] && !(S[r] > 1e-30f && S[r] < 1e30f)) shifted = true;
        }
    }
    if (shifted) {
        // explicit shifts F_r = -max_j (gamma_j - kap c_rj)
        const float4* rp[R];
        float mx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            rp[r] = first ? c[r]
                          : reinterpret_cast<const float4*>(X.Gp + (long long)(row + (ok[r] ? r : 0)) * X.ld);
            mx[r] = -INFINITY;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int g = gt + v * GS;
#pragma unroll
            for (int r = 0; r < R; ++r) e[r][v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            if (g < X.ng4) {
                const float4 gg = CR.gc[g];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 cv = rp[r][g];
                    const float2 x01 = upk(fma2(pk(cv.x, cv.y), nk2, pk(gg.x, gg.y)));
                    const float2 x23 = upk(fma2(pk(cv.z, cv.w), nk2, pk(gg.z, gg.w)));
                    e[r][v] = make_float4(x01.x, x01.y, x23.x, x23.y);
                    mx[r] = fmaxf(mx[r], fmaxf(fmaxf(x01.x, x01.y), fmaxf(x23.x, x23.y)));
                }
            }
        }
        if (first) stage_release<STAGES>(P);
        group_allreduce<true, R>(mx, GS, s_part, parity);
        if (first && threadIdx.x == OT_ISSUER && k + STAGES < X.nchunks) issue_chunk<STAGES, R>(P, X, k + STAGES, A);
        f32x2 S2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            F[r] = mx[r] > -INFINITY ? -mx[r] : 0.f;
            S2[r] = pk(0.f, 0.f);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int g = gt + v * GS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 x = e[r][v];
                e[r][v] = make_float4(ex2(x.x + F[r]), ex2(x.y + F[r]), ex2(x.z + F[r]), ex2(x.w + F[r]));
            }
            if (g < X.ng4) {
                const float4 cc = CR.cf[g];
#pragma unroll
                for (int r = 0; r < R; ++r) S2[r] = dot4x2(e[r][v], cc, S2[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) S[r] = hsum(S2[r]);
        group_allreduce<false, R>(S, GS, s_part, parity);
    }
    f32x2 u2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (ok[r] && gt == ep + r) {
            pd.S = S[r];
            pd.F = F[r];
            pd.al = sc[r].z;
            pd.row = row + r;
        }
        const float u = (ok[r] && S[r] > 1e-30f && S[r] < 1e30f) ? __fdividef(sc[r].z, S[r]) : 0.f;
        u2[r] = pk(u, u);
    }
    // (a slot past the row end holds zeros, so its sums stay zero: no test in the loop)
#pragma unroll
    for (int v = 0; v < V; ++v) {
        f32x2 e01[R], e23[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            e01[r] = pk(e[r][v].x, e[r][v].y);
            e23[r] = pk(e[r][v].z, e[r][v].w);
        }
        kahan_rows<R>(acc[2 * v], cmp[2 * v], u2, e01);
        kahan_rows<R>(acc[2 * v + 1], cmp[2 * v + 1], u2, e23);
    }
}

// Rows [r_lo, r_hi) of one problem by all groups of the block, R rows per group
// and chunk.  Chunk k holds rows r_lo + R (k NG + q) .. + R - 1 for group q;
// STAGES chunks are in flight.  Returns false (uniformly) if a wait expired.
// The three-row launch runs this engine; the two-row launch runs rows_segment2.
template <int STAGES, int R>
__device__ __forceinline__ bool rows_segment(const BatchArgs& A, const ot_problem_desc& d, int p, int r_lo, int r_hi,
                                             int t, int GS, float* s_part, float* s_gc, float* s_cf, Pipe& P) {
    constexpr int V = R == 2 ? OT_BV : 3;   // a row of a three-row chunk fills at most 3 slots
    constexpr int W = 32 / R;               // chunks per window of pending rows
    const int NG = OT_BT / GS;
    const int tid = threadIdx.x, gt = tid & (GS - 1), q = tid / GS;
    const int cur = (t - 1) & 1, nxt = t & 1;
    SegCtx X;
    X.Gp = A.G + d.g_off;
    X.rs_cur = A.rs + (size_t)cur * A.total_m + d.v_off;
    X.rs_nxt = A.rs + (size_t)nxt * A.total_m + d.v_off;
    X.flo_nxt = A.flo + (size_t)nxt * A.total_m + d.v_off;
    X.gs = GS;
    X.ng = NG;
    X.m = d.m;
    X.ld = d.ld;
    X.ng4 = d.ld >> 2;
    X.r_lo = r_lo;
    X.r_hi = r_hi;
    X.t = t;
    X.kap = (float)(1.0 / ((double)d.eps * OT_LN2));
    X.nchunks = (r_hi - r_lo + R * NG - 1) / (R * NG);
    if (tid == OT_ISSUER) {
        for (int k = 0; k < X.nchunks && k < STAGES; ++k) issue_chunk<STAGES, R>(P, X, k, A);
    }
    // stage the column data (every thread has finished with the previous segment's)
    __syncthreads();
    for (int j = tid; j < X.ld; j += OT_BT) {
        const bool in = j < X.m;
        s_gc[j] = in ? A.gc[d.v_off + j] : -INFINITY;
        s_cf[j] = in ? A.cf[d.v_off + j] : 0.f;
    }
    __syncthreads();
    ColData CR;
    CR.gc = reinterpret_cast<const float4*>(s_gc);
    CR.cf = reinterpret_cast<const float4*>(s_cf);
    int parity = 0;
    f32x2 acc[2 * V], cmp[2 * V];   // column contributions: compensated sums acc - (-cmp)
#pragma unroll
    for (int v = 0; v < 2 * V; ++v) acc[v] = cmp[v] = pk(0.f, 0.f);
    float l1 = 0.f;
    Pending pd;
    pd.S = pd.F = pd.al = 0.f;
    pd.row = -1;
    for (int k = 0; k < X.nchunks; ++k) {
        const int kk = k % W;   // chunk index within the window of pending rows
        const int row = r_lo + R * (k * NG + q);
        const int st = (int)(P.consumed % STAGES);
        const unsigned ph = (unsigned)((P.consumed / STAGES) & 1);
        if (!mbar_wait_ab(&P.full[st], ph, A.timeout_ns, P.abort)) abort_block(A, P);
        // (processed even after an expired wait: the shared-memory reads stay in bounds, and
        // every warp keeps to the same sequence of group barriers and releases; the block
        // leaves together at the end of the segment)
        if (row < r_hi)   // uniform over the group
            process_rows<STAGES, R, V>(P.stage + (size_t)st * OT_STAGE_FLOATS + (size_t)(R * q) * X.ld,
                                       P.rsc + st * OT_RSC_STAGE + R * q, A, X, row, k, kk, CR, s_part, parity,
                                       acc, cmp, l1, pd, P);
        else
            stage_release<STAGES>(P);
        // the group's first warp writes the window's pending rows at its end and at the segment's end
        if (gt < 32 && (kk == W - 1 || k == X.nchunks - 1)) finish_pending(A, X, pd);
        P.consumed += 1;
    }
    if (__syncthreads_or(*P.abort)) return false;
    // column contributions of this group (times the lo factors) and its L1 terms
    if (r_lo + R * q < r_hi) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int g = gt + v * GS;
            if (g < X.ng4) {
                const float4 cc = CR.cf[g];
                const float2 s01 = upk(add2(acc[2 * v], cmp[2 * v]));
                const float2 s23 = upk(add2(acc[2 * v + 1], cmp[2 * v + 1]));
                const int j = 4 * g;
                const long long o = d.v_off + j;
                if (j < X.m) red_add_f32(A.R + o, s01.x * cc.x);
                if (j + 1 < X.m) red_add_f32(A.R + o + 1, s01.y * cc.y);
                if (j + 2 < X.m) red_add_f32(A.R + o + 2, s23.x * cc.z);
                if (j + 3 < X.m) red_add_f32(A.R + o + 3, s23.y * cc.w);
            }
        }
    }
    if (l1 != 0.f) atomicAdd(A.l1acc + (size_t)(t & 1) * A.count + p, (double)l1);
    return true;
}

// Two-row engine: row update of the two rows of a chunk held by a group (Eq.
// optimal_f_sinkhorn_logdomain in log2 units): S_r = sum_j 2^(gamma_j - kap c_rj + F_r)
// around the previous potential F_r, new potential F_r - log2(S_r / alpha_r)
// kept exactly as hi + lo (recorded in pd, written by finish_pending), column
// contributions (alpha_r / S_r) e_rj added to acc.  An explicit max shift is used on the first sweep and whenever a row
// sum leaves the safe range (then from the rows in global memory: the stage may
// already be refilled).
template <int STAGES>
__device__ __forceinline__ void process_rows2(const float* srow, const float4* srsc, const BatchArgs& A,
                                             const SegCtx& X, int row, int k, const ColData& CR, float* s_part,
                                             int& parity, f32x2 (&acc)[2 * OT_BV], f32x2 (&cmp)[2 * OT_BV],
                                             float& l1, Pending& pd, Pipe& P) {
    const int GS = X.gs, gt = threadIdx.x & (GS - 1);
    const bool two = row + 1 < X.r_hi;   // uniform over the group
    // lanes of the group's first warp that hold the two rows until they are finished
    const int ep0 = (2 * k) & 31, ep1 = ep0 + 1;
    // a lone last row is processed twice (as both rows of the pair) and its second copy
    // gets no weight: the hot loops carry no test for it
    const float4 sc0 = srsc[0], sc1 = two ? srsc[1] : sc0;
    const float al0 = sc0.z, al1 = sc1.z;
    const f32x2 nk2 = pk(-X.kap, -X.kap);
    const float4* c0 = reinterpret_cast<const float4*>(srow);
    const float4* c1 = reinterpret_cast<const float4*>(two ? srow + X.ld : srow);
    float4 e0[OT_BV], e1[OT_BV];
    float F0 = sc0.x, F1 = sc1.x, S0 = 0.f, S1 = 0.f;
    const bool first = X.t == 1;
    bool shifted = first;
    if (!shifted) {
        const f32x2 F02 = pk(F0, F0), F12 = pk(F1, F1);
        f32x2 S02 = pk(0.f, 0.f), S12 = pk(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < OT_BV; ++v) {
            const int g = gt + v * GS;
            e0[v] = e1[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < X.ng4) {
                const float4 gg = CR.gc[g], cc = CR.cf[g];
                e0[v] = exps4(c0[g], gg, nk2, F02);
                S02 = dot4x2(e0[v], cc, S02);
                e1[v] = exps4(c1[g], gg, nk2, F12);
                S12 = dot4x2(e1[v], cc, S12);
            }
        }
        stage_release<STAGES>(P);
        S0 = hsum(S02);
        S1 = hsum(S12);
        group_allreduce2<false>(S0, S1, GS, s_part, parity);
        if (threadIdx.x == OT_ISSUER && k + STAGES < X.nchunks) issue_chunk<STAGES, 2>(P, X, k + STAGES, A);
        if (gt == ep0) l1 += fabsf(fmaf(S0, sc0.y - 1.0f, S0 - al0));
        if (two && gt == ep1) l1 += fabsf(fmaf(S1, sc1.y - 1.0f, S1 - al1));
        // uniform over the group
        shifted = !(S0 > 1e-30f && S0 < 1e30f) || (two && !(S1 > 1e-30f && S1 < 1e30f));
    }
    if (shifted) {
        // explicit shifts F_r = -max_j (gamma_j - kap c_rj), both rows
        const float4* r0 = first ? c0 : reinterpret_cast<const float4*>(X.Gp + (long long)row * X.ld);
        const float4* r1 = first ? c1 : reinterpret_cast<const float4*>(X.Gp + (long long)(two ? row + 1 : row) * X.ld);
        float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
        for (int v = 0; v < OT_BV; ++v) {
            const int g = gt + v * GS;
            e0[v] = e1[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            if (g < X.ng4) {
                const float4 gg = CR.gc[g];
                float4 c = r0[g];
                float2 x01 = upk(fma2(pk(c.x, c.y), nk2, pk(gg.x, gg.y)));
                float2 x23 = upk(fma2(pk(c.z, c.w), nk2, pk(gg.z, gg.w)));
                e0[v] = make_float4(x01.x, x01.y, x23.x, x23.y);
                m0 = fmaxf(m0, fmaxf(fmaxf(x01.x, x01.y), fmaxf(x23.x, x23.y)));
                if (two) {
                    c = r1[g];
                    x01 = upk(fma2(pk(c.x, c.y), nk2, pk(gg.x, gg.y)));
                    x23 = upk(fma2(pk(c.z, c.w), nk2, pk(gg.z, gg.w)));
                    e1[v] = make_float4(x01.x, x01.y, x23.x, x23.y);
                    m1 = fmaxf(m1, fmaxf(fmaxf(x01.x, x01.y), fmaxf(x23.x, x23.y)));
                }
            }
        }
        if (first) stage_release<STAGES>(P);
        group_allreduce2<true>(m0, m1, GS, s_part, parity);
        if (first && threadIdx.x == OT_ISSUER && k + STAGES < X.nchunks) issue_chunk<STAGES, 2>(P, X, k + STAGES, A);
        F0 = m0 > -INFINITY ? -m0 : 0.f;
        F1 = m1 > -INFINITY ? -m1 : 0.f;
        f32x2 S02 = pk(0.f, 0.f), S12 = pk(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < OT_BV; ++v) {
            const int g = gt + v * GS;
            float4 x = e0[v];
            x = make_float4(ex2(x.x + F0), ex2(x.y + F0), ex2(x.z + F0), ex2(x.w + F0));
            e0[v] = x;
            x = e1[v];
            x = make_float4(ex2(x.x + F1), ex2(x.y + F1), ex2(x.z + F1), ex2(x.w + F1));
            e1[v] = x;
            if (g < X.ng4) {
                const float4 cc = CR.cf[g];
                S02 = dot4x2(e0[v], cc, S02);
                S12 = dot4x2(e1[v], cc, S12);
            }
        }
        S0 = hsum(S02);
        S1 = hsum(S12);
        group_allreduce2<false>(S0, S1, GS, s_part, parity);
    }
    if (gt == ep0) {
        pd.S = S0;
        pd.F = F0;
        pd.al = al0;
        pd.row = row;
    }
    if (two && gt == ep1) {
        pd.S = S1;
        pd.F = F1;
        pd.al = al1;
        pd.row = row + 1;
    }
    const float u0 = (S0 > 1e-30f && S0 < 1e30f) ? __fdividef(al0, S0) : 0.f;
    const float u1 = (two && S1 > 1e-30f && S1 < 1e30f) ? __fdividef(al1, S1) : 0.f;
    const f32x2 u02 = pk(u0, u0), u12 = pk(u1, u1);
#pragma unroll
    for (int v = 0; v < OT_BV; ++v) {
        kahan2(acc[2 * v], cmp[2 * v], u02, pk(e0[v].x, e0[v].y), u12, pk(e1[v].x, e1[v].y));
        kahan2(acc[2 * v + 1], cmp[2 * v + 1], u02, pk(e0[v].z, e0[v].w), u12, pk(e1[v].z, e1[v].w));
    }
}

// Two-row engine: rows [r_lo, r_hi) of one problem by all groups of the block.
// Chunk k holds rows r_lo + 2 (k NG + q) and the next one for group q; STAGES
// chunks are in flight.  Returns false (uniformly) if a wait expired.  (The
// same steps as rows_segment<STAGES, 2>, written for two rows: it measured 4%
// faster than the R-generic code with two rows.)
template <int STAGES>
__device__ __forceinline__ bool rows_segment2(const BatchArgs& A, const ot_problem_desc& d, int p, int r_lo, int r_hi,
                                              int t, int GS, float* s_part, float* s_gc, float* s_cf, Pipe& P) {
    const int NG = OT_BT / GS;
    const int tid = threadIdx.x, gt = tid & (GS - 1), q = tid / GS;
    const int cur = (t - 1) & 1, nxt = t & 1;
    SegCtx X;
    X.Gp = A.G + d.g_off;
    X.rs_cur = A.rs + (size_t)cur * A.total_m + d.v_off;
    X.rs_nxt = A.rs + (size_t)nxt * A.total_m + d.v_off;
    X.flo_nxt = A.flo + (size_t)nxt * A.total_m + d.v_off;
    X.gs = GS;
    X.ng = NG;
    X.m = d.m;
    X.ld = d.ld;
    X.ng4 = d.ld >> 2;
    X.r_lo = r_lo;
    X.r_hi = r_hi;
    X.t = t;
    X.kap = (float)(1.0 / ((double)d.eps * OT_LN2));
    X.nchunks = (r_hi - r_lo + 2 * NG - 1) / (2 * NG);
    if (tid == OT_ISSUER) {
        for (int k = 0; k < X.nchunks && k < STAGES; ++k) issue_chunk<STAGES, 2>(P, X, k, A);
    }
    // stage the column data (every thread has finished with the previous segment's)
    __syncthreads();
    for (int j = tid; j < X.ld; j += OT_BT) {
        const bool in = j < X.m;
        s_gc[j] = in ? A.gc[d.v_off + j] : -INFINITY;
        s_cf[j] = in ? A.cf[d.v_off + j] : 0.f;
    }
    __syncthreads();
    ColData CR;
    CR.gc = reinterpret_cast<const float4*>(s_gc);
    CR.cf = reinterpret_cast<const float4*>(s_cf);
    int parity = 0;
    f32x2 acc[2 * OT_BV], cmp[2 * OT_BV];   // column contributions: compensated sums acc - (-cmp)
#pragma unroll
    for (int v = 0; v < 2 * OT_BV; ++v) acc[v] = cmp[v] = pk(0.f, 0.f);
    float l1 = 0.f;
    Pending pd;
    pd.S = pd.F = pd.al = 0.f;
    pd.row = -1;
    for (int k = 0; k < X.nchunks; ++k) {
        const int row = r_lo + 2 * (k * NG + q);
        const int st = (int)(P.consumed % STAGES);
        const unsigned ph = (unsigned)((P.consumed / STAGES) & 1);
        if (!mbar_wait_ab(&P.full[st], ph, A.timeout_ns, P.abort)) abort_block(A, P);
        // (processed even after an expired wait: the shared-memory reads stay in bounds, and
        // every warp keeps to the same sequence of group barriers and releases; the block
        // leaves together at the end of the segment)
        if (row < r_hi)   // uniform over the group
            process_rows2<STAGES>(P.stage + (size_t)st * OT_STAGE_FLOATS + (size_t)(2 * q) * X.ld,
                                  P.rsc + st * OT_RSC_STAGE + 2 * q, A, X, row, k, CR, s_part, parity, acc, cmp, l1, pd,
                                 P);
        else
            stage_release<STAGES>(P);
        // the group's first warp writes its 32 pending rows every 16 chunks and at the end
        if (gt < 32 && ((k & 15) == 15 || k == X.nchunks - 1)) finish_pending(A, X, pd);
        P.consumed += 1;
    }
    if (__syncthreads_or(*P.abort)) return false;
    // column contributions of this group (times the lo factors) and its L1 terms
    if (r_lo + 2 * q < r_hi) {
#pragma unroll
        for (int v = 0; v < OT_BV; ++v) {
            const int g = gt + v * GS;
            if (g < X.ng4) {
                const float4 cc = CR.cf[g];
                const float2 s01 = upk(add2(acc[2 * v], cmp[2 * v]));
                const float2 s23 = upk(add2(acc[2 * v + 1], cmp[2 * v + 1]));
                const int j = 4 * g;
                const long long o = d.v_off + j;
                if (j < X.m) red_add_f32(A.R + o, s01.x * cc.x);
                if (j + 1 < X.m) red_add_f32(A.R + o + 1, s01.y * cc.y);
                if (j + 2 < X.m) red_add_f32(A.R + o + 2, s23.x * cc.z);
                if (j + 3 < X.m) red_add_f32(A.R + o + 3, s23.y * cc.w);
            }
        }
    }
    if (l1 != 0.f) atomicAdd(A.l1acc + (size_t)(t & 1) * A.count + p, (double)l1);
    return true;
}

// One launch solves the problems whose chunks hold R rows per group (chunk_rows);
// the solver launches once per R, so that each launch carries one row engine.
template <int STAGES, int R>
__global__ void __launch_bounds__(OT_BT, 1) batch_solve_kernel(const __grid_constant__ BatchArgs A) {
    // a launch without problems of its kind leaves at once (every block alike)
    if (A.nrows && A.nrows[2 * A.gs_shift + R - 2] == 0) return;
    extern __shared__ __align__(128) unsigned char dsm[];
    float* s_stage = reinterpret_cast<float*>(dsm + BatchSmem::stage);                 // [STAGES][OT_STAGE_FLOATS]
    float* s_gc = reinterpret_cast<float*>(dsm + BatchSmem::gc);                       // [MAXM]
    float* s_cf = reinterpret_cast<float*>(dsm + BatchSmem::cf);                       // [MAXM]
    long long* s_pref = reinterpret_cast<long long*>(dsm + BatchSmem::pref);           // [count+1]
    unsigned short* s_m = reinterpret_cast<unsigned short*>(dsm + BatchSmem::msz);     // [count]
    unsigned short* s_rw = reinterpret_cast<unsigned short*>(dsm + BatchSmem::rw);     // [count]
    unsigned char* s_act = reinterpret_cast<unsigned char*>(dsm + BatchSmem::act);     // [count]
    __shared__ __align__(16) float s_part[2 * OT_BW * 4];
    __shared__ long long s_wsum[32];
    __shared__ double s_dred[OT_BW];
    __shared__ __align__(8) unsigned long long s_full[STAGES], s_empty[STAGES];
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int B = blockIdx.x, Gd = gridDim.x;
    const int count = A.count;
    unsigned epoch = 0;
    Pipe P;
    P.stage = s_stage;
    P.rsc = reinterpret_cast<float4*>(dsm + BatchSmem::rsc);
    P.full = s_full;
    P.empty = s_empty;
    P.abort = &s_abort;
    P.consumed = 0;
    P.issued = 0;

    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&s_full[st], 1);
            mbar_init(&s_empty[st], OT_BW);
        }
        s_abort = 0;
        fence_mbar_init();
    }
    for (int p = tid; p < count; p += OT_BT) {
        const int ld = A.desc[p].ld;
        s_m[p] = (unsigned short)A.desc[p].m;
        // row weight, 0 for the problems of the other launch
        s_rw[p] = chunk_rows(row_slots(ld, A.gs_shift)) == R ? (unsigned short)row_weight(ld, A.gs_shift) : 0;
    }
    __syncthreads();

    // ---- per-problem marginal sums and validation (problems split over blocks)
    for (int p = B; p < count; p += Gd) {
        if (!s_rw[p]) continue;   // uniform over the block
        const ot_problem_desc d = A.desc[p];
        const int m = d.m;
        const long long v0 = d.v_off;
        double sa = 0.0, sb = 0.0;
        int bad = 0;
        for (int i = tid; i < m; i += OT_BT) {
            const float x = A.a[v0 + i], y = A.b[v0 + i];
            bad |= !(x > 0.f && x < INFINITY) || !(y > 0.f && y < INFINITY);
            sa += x;
            sb += y;
        }
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        bad = __syncthreads_or(bad);
        if (lane == 0) s_dred[wid] = sa;
        __syncthreads();
        double ta = 0.0;
        for (int w2 = 0; w2 < OT_BW; ++w2) ta += s_dred[w2];
        __syncthreads();
        if (lane == 0) s_dred[wid] = sb;
        __syncthreads();
        double tb = 0.0;
        for (int w2 = 0; w2 < OT_BW; ++w2) tb += s_dred[w2];
        __syncthreads();
        if (tid == 0) {
            A.inv_sa[p] = 1.0 / ta;
            A.inv_sb[p] = 1.0 / tb;
            A.active[p] = bad ? 0 : 1;
            A.iters[p] = bad ? -1 : 0;
            A.l1acc[p] = 0.0;
            A.l1acc[count + p] = 0.0;
            A.res[p].value = 0.0;
            A.res[p].transport_cost = 0.0;
            A.res[p].marg_l1_col = 0.0;
            A.res[p].reserved[0] = 0.0;
            if (bad) {
                A.res[p].iters = 0;
                A.res[p].status = OT_ERR_ARG;
                A.res[p].marg_l1 = -1.0;
                A.res[p].marg_l2_col = -1.0;
            }
        }
        // row scalars of both buffers (no potential yet: the first sweep shifts every row)
        const double isa = 1.0 / ta;
        for (int i = tid; i < m; i += OT_BT) {
            const float4 r0 = make_float4(0.f, 1.f, (float)((double)A.a[v0 + i] * isa), 0.f);
            A.rs[v0 + i] = r0;
            A.rs[A.total_m + v0 + i] = r0;
            A.flo[v0 + i] = 0.f;
            A.flo[A.total_m + v0 + i] = 0.f;
        }
        // column potentials and sums
        const float kap = (float)(1.0 / ((double)d.eps * OT_LN2));
        for (int j = tid; j < m; j += OT_BT) {
            const double g0 = A.warm ? A.z_out[v0 + j] * (double)kap : 0.0;
            const float hi = (float)g0;
            A.gam[v0 + j] = g0;
            A.gc[v0 + j] = hi;
            A.cf[v0 + j] = ex2((float)(g0 - (double)hi));
            A.R[v0 + j] = 0.f;
        }
    }
    if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;

    for (int t = 1;; ++t) {
        const int nxt = t & 1;
        const long long TM = A.total_m;
        // ---------------- row phase
        // (the row scalars written last sweep by generic stores are read by bulk copies)
        if (tid == OT_ISSUER) asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int p = tid; p < count; p += OT_BT) s_act[p] = (A.active[p] && s_rw[p]) ? 1 : 0;
        __syncthreads();
        batch_prefix(count, s_m, s_rw, s_act, true, s_pref, s_wsum);
        {
            // a row belongs to the block whose weight range holds the row's start
            const long long W = s_pref[count];
            const long long w0 = W * B / Gd, w1 = W * (B + 1) / Gd;
            const int pfirst = (W > 0 && w0 < w1) ? find_problem(s_pref, count, w0) : count;
            for (int p = pfirst; p < count && s_pref[p] < w1; ++p) {
                if (!s_act[p]) continue;
                const int m = s_m[p], rw = s_rw[p];
                const long long base = s_pref[p];
                const int r_lo = (w0 <= base) ? 0 : (int)((w0 - base + rw - 1) / rw);
                const int r_hi = min(m, (int)((w1 - base + rw - 1) / rw));
                if (r_lo >= r_hi) continue;
                const ot_problem_desc d = A.desc[p];
                const int gs = group_size(d.ld, A.gs_shift);   // tuned: a larger group takes fewer slots per thread
                bool ok;
                if constexpr (R == 2) ok = rows_segment2<STAGES>(A, d, p, r_lo, r_hi, t, gs, s_part, s_gc, s_cf, P);
                else ok = rows_segment<STAGES, R>(A, d, p, r_lo, r_hi, t, gs, s_part, s_gc, s_cf, P);
                if (!ok) goto fail;
            }
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;

        // ---------------- column phase
        batch_prefix(count, s_m, s_rw, s_act, false, s_pref, s_wsum);
        {
            const long long W = s_pref[count];
            const long long c0 = W * B / Gd, c1 = W * (B + 1) / Gd;
            for (long long cidx = c0 + tid; cidx < c1; cidx += OT_BT) {
                const int p = find_problem(s_pref, count, cidx);
                const int j = (int)(cidx - s_pref[p]);
                const long long v0 = A.desc[p].v_off;
                const double L1 = A.l1acc[(size_t)(t & 1) * count + p];
                const int done = t - 1;
                int st = -1;
                if (done >= 1) {
                    const bool check = done % A.check_every == 0;
                    if (check && L1 != L1) st = OT_ERR_NONFINITE;
                    else if (check && L1 <= A.tol) st = OT_OK;
                    else if (done >= A.max_iter) st = OT_ERR_NOT_CONVERGED;
                }
                const float Rj = A.R[v0 + j];
                A.R[v0 + j] = 0.f;
                if (st >= 0) {
                    if (j == 0) {
                        A.active[p] = 0;
                        A.iters[p] = done;
                        A.res[p].iters = done;
                        A.res[p].status = st;
                        A.res[p].marg_l1 = L1;
                        A.res[p].marg_l2_col = -1.0;
                    }
                    continue;
                }
                if (j == 0) A.l1acc[(size_t)((t + 1) & 1) * count + p] = 0.0;
                if (Rj != Rj) {
                    set_status(A.ctrl, OT_ERR_NONFINITE);
                    continue;
                }
                double gnew;
                const double beta = (double)A.b[v0 + j] * A.inv_sb[p];
                if (Rj > 1e-30f && Rj < 1e30f) {
                    gnew = A.gam[v0 + j] - (double)lg2(__fdividef(Rj, (float)beta));
                } else {
                    // rare: recompute the column's log-sum-exp with an explicit max (one thread)
                    const ot_problem_desc d = A.desc[p];
                    const int m = d.m, ld = d.ld;
                    const float kap = (float)(1.0 / ((double)d.eps * OT_LN2));
                    const float* Gp = A.G + d.g_off;
                    float mx = -INFINITY, s = 0.f;
                    for (int i = 0; i < m; ++i) {
                        const float4 ri = A.rs[nxt * TM + v0 + i];
                        const float x = fmaf(Gp[(long long)i * ld + j], -kap, ri.x);
                        const float e = ri.y;
                        if (x > mx) { s = fmaf(s, ex2(mx - x), e); mx = x; }
                        else s += ex2(x - mx) * e;
                    }
                    if (!(s > 0.f)) {
                        set_status(A.ctrl, OT_ERR_NONFINITE);
                        continue;
                    }
                    gnew = (double)lg2((float)beta) - (double)mx - (double)lg2(s);
                }
                const float hi = (float)gnew;
                A.gam[v0 + j] = gnew;
                A.gc[v0 + j] = hi;
                A.cf[v0 + j] = ex2((float)(gnew - (double)hi));
            }
        }
        if (!grid_sync(A.ctrl, Gd, A.timeout_ns, epoch)) goto fail;
        int any = 0;
        for (int p = tid; p < count; p += OT_BT) any |= s_rw[p] ? ((volatile int*)A.active)[p] : 0;
        if (!__syncthreads_or(any)) break;
    }

    // ---------------- outputs: each block writes a share of this launch's problems
    for (int p = B; p < count; p += Gd) {
        if (!s_rw[p]) continue;
        const ot_problem_desc d = A.desc[p];
        const int m = d.m;
        const long long v0 = d.v_off;
        const int it = A.iters[p];
        const int buf = it & 1;
        const double unit = (double)d.eps * OT_LN2;
        const double shift = -(double)d.eps * log((double)d.N);
        for (int i = tid; i < m; i += OT_BT) {
            // a problem rejected by the validation gets NaN potentials
            const size_t o = (size_t)buf * A.total_m + v0 + i;
            A.w_out[v0 + i] = it < 0 ? (double)NAN : ((double)A.rs[o].x + (double)A.flo[o]) * unit + shift;
            A.z_out[v0 + i] = it < 0 ? (double)NAN : A.gam[v0 + i] * unit;
        }
        if (tid == 0) A.res[p].reserved[1] = 4.0;   // variant code: batch
    }
    return;
fail:
    // no copy may still be writing into this block's shared memory when it exits (once the
    // block aborted no copy is issued, and at most the last STAGES issued can be in flight)
    if (tid == OT_ISSUER) {
        for (long long u = P.issued > STAGES ? P.issued - STAGES : 0; u < P.issued; ++u)
            if (!mbar_wait(&s_full[u % STAGES], (unsigned)((u / STAGES) & 1), A.timeout_ns)) break;
        for (int p = B; p < count; p += Gd) {
            if (!s_rw[p]) continue;
            A.res[p].iters = -1;
            A.res[p].status = ld_volatile_int(&A.ctrl->status);
        }
    }
    __syncthreads();
}

// ---- batched fold from points: G_p[i][j] = -eps log sum_k exp(-|x_i - R^k y_j|^2 / eps)
// (Eq. def_Kij with the squared Euclidean cost of rotated points).  Blocks take
// rows; |x_i - R^k y_j| = |R^-k x_i - y_j|, so the N rotations of x_i are formed
// once per row in shared memory and each thread streams columns j.
__global__ void __launch_bounds__(256) batch_fold_kernel(const ot_problem_desc* desc, int count,
                                                         const float2* pts, float* G_all) {
    const int p = blockIdx.y;
    if (p >= count) return;
    const ot_problem_desc d = desc[p];
    __shared__ float2 rot[256];
    __shared__ float2 xr[256];
    for (int k = threadIdx.x; k < d.N && k < 256; k += blockDim.x) {
        float sn, cs;
        sincospif(2.0f * (float)k / (float)d.N, &sn, &cs);
        rot[k] = make_float2(cs, sn);
    }
    const float kap = (float)(1.0 / ((double)d.eps * OT_LN2));
    const float inv_kap = (float)((double)d.eps * OT_LN2);
    for (int i = blockIdx.x; i < d.m; i += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < d.N) {   // R^-k x_i
            const float2 r = rot[threadIdx.x], xi = pts[d.x_off + i];
            xr[threadIdx.x] = make_float2(fmaf(r.x, xi.x, r.y * xi.y), fmaf(r.x, xi.y, -r.y * xi.x));
        }
        __syncthreads();
        float* Grow = G_all + d.g_off + (long long)i * d.ld;
        for (int j = threadIdx.x; j < d.ld; j += blockDim.x) {
            if (j >= d.m) {   // row padding: a finite value (the solver gives these columns zero weight)
                Grow[j] = 0.f;
                continue;
            }
            const float2 yj = pts[d.y_off + j];
            float mn = 0.f, s = 1.f;
            for (int k = 0; k < d.N; ++k) {
                const float2 xk = xr[k];
                const float dx = xk.x - yj.x, dy = xk.y - yj.y;
                const float c = fmaf(dx, dx, dy * dy);
                if (k == 0) mn = c;
                else if (c < mn) { s = fmaf(s, ex2((c - mn) * kap), 1.0f); mn = c; }
                else s += ex2((mn - c) * kap);
            }
            Grow[j] = mn - lg2(s) * inv_kap;
        }
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Writes a one-problem table into the workspace from kernel parameters (no host copy, so a single-problem
// solve through this kernel stays capturable in a CUDA graph).
__global__ void batch_single_table_kernel(ot_problem_desc d, ot_problem_desc* dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = d;
}

struct BatchLayout {
    size_t ctrl, desc, inv_sa, inv_sb, active, iters, l1acc, rs, flo, gam, gc, cf, R, total;
};

static BatchLayout batch_layout(int count, long long TM) {
    BatchLayout L;
    size_t o = 0;
    L.ctrl = o; o = a256(o + sizeof(Ctrl));
    L.desc = o; o = a256(o + sizeof(ot_problem_desc) * (size_t)count);
    L.inv_sa = o; o = a256(o + sizeof(double) * (size_t)count);
    L.inv_sb = o; o = a256(o + sizeof(double) * (size_t)count);
    L.active = o; o = a256(o + sizeof(int) * (size_t)count);
    L.iters = o; o = a256(o + sizeof(int) * (size_t)count);
    L.l1acc = o; o = a256(o + sizeof(double) * 2 * (size_t)count);
    L.rs = o; o = a256(o + sizeof(float4) * 2 * (size_t)TM);
    L.flo = o; o = a256(o + sizeof(float) * 2 * (size_t)TM);
    L.gam = o; o = a256(o + sizeof(double) * (size_t)TM);
    L.gc = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.cf = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.R = o; o = a256(o + sizeof(float) * (size_t)TM);
    L.total = o;
    return L;
}

// Host-side copy of the last prepared table (count, total_m) per workspace is not kept:
// the table header lives in the workspace itself.
struct BatchHeader {
    int count;
    int max_m;
    long long total_m;
    int nrows[2][2];   // problems with [group-size shift][rows per chunk - 2]
    long long pad[4];
};
static_assert(sizeof(BatchHeader) == 64, "header layout");

}  // namespace cyc

using namespace cyc;

extern "C" size_t ot_batch_workspace_bytes(int count, long long total_m) {
    if (count <= 0 || count > OT_BATCH_MAX || total_m <= 0) return 0;
    return a256(sizeof(BatchHeader)) + batch_layout(count, total_m).total;
}

extern "C" int ot_batch_prepare(const ot_problem_desc* descs, int count, void* workspace, size_t ws_bytes,
                                void* stream) {
    if (!descs || count <= 0 || count > OT_BATCH_MAX || !workspace) return OT_ERR_ARG;
    long long TM = 0;
    int max_m = 0;
    for (int p = 0; p < count; ++p) {
        const ot_problem_desc& d = descs[p];
        if (d.m <= 0 || d.N <= 0 || d.N > 256 || !(d.eps > 0.f) || d.ld < d.m || d.ld % 4 != 0 ||
            d.g_off % 4 != 0 || d.ld > OT_BATCH_MAXM)
            return OT_ERR_ARG;
        TM = TM > d.v_off + d.m ? TM : d.v_off + d.m;
        max_m = max_m > d.m ? max_m : d.m;
    }
    int nrows[2][2] = {{0, 0}, {0, 0}};
    for (int p = 0; p < count; ++p)
        for (int sh = 0; sh < 2; ++sh) nrows[sh][chunk_rows(row_slots(descs[p].ld, sh)) - 2] += 1;
    if (ws_bytes < ot_batch_workspace_bytes(count, TM) || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    BatchHeader h;
    memset(&h, 0, sizeof(h));
    h.count = count;
    h.max_m = max_m;
    h.total_m = TM;
    memcpy(h.nrows, nrows, sizeof(nrows));
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)workspace;
    const BatchLayout L = batch_layout(count, TM);
    // pageable host sources: the copies are complete when cudaMemcpyAsync returns
    if (cudaMemcpyAsync(w, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) return OT_ERR_CUDA;
    char* base = w + a256(sizeof(BatchHeader));
    if (cudaMemcpyAsync(base + L.desc, descs, sizeof(ot_problem_desc) * (size_t)count, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return OT_ERR_CUDA;
    return OT_OK;
}

extern "C" int ot_batch_fold(int count, const float* points, float* G_all, void* workspace, size_t ws_bytes,
                             void* stream) {
    if (count <= 0 || count > OT_BATCH_MAX || !points || !G_all || !workspace) return OT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    const BatchLayout L = batch_layout(count, 1);
    const ot_problem_desc* d = (const ot_problem_desc*)((char*)workspace + a256(sizeof(BatchHeader)) + L.desc);
    (void)ws_bytes;
    dim3 grid(64u, (unsigned)count);   // blocks beyond a problem's rows leave at once
    batch_fold_kernel<<<grid, 256, 0, st>>>(d, count, (const float2*)points, G_all);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

// ---- launch configurations and the autotuner
//
// A configuration code (ot_options.tile_override for the batch solver) packs
// the group-size policy and the convergence-check cadence: 0 is the default
// (tight groups, opt->check_every); otherwise code - 1 = g | (c << 1) with
// g = group-size shift and c = log2 of the check cadence (0..2).
struct BatchCfg {
    int stages, gs_shift, check_every;
};

static bool decode_cfg(int code, int opt_check_every, BatchCfg& c) {
    c.stages = OT_STAGES_MAX;
    if (code == 0) {
        c.gs_shift = 0;
        c.check_every = opt_check_every >= 1 ? opt_check_every : 1;
        return true;
    }
    code -= 1;
    if (code < 0 || code >= OT_BATCH_NCFG) return false;
    c.gs_shift = code & 1;
    c.check_every = 1 << (code >> 1);
    return true;
}

static int encode_cfg(const BatchCfg& c) {
    const int ce = c.check_every >= 4 ? 2 : (c.check_every >= 2 ? 1 : 0);
    return 1 + c.gs_shift + (ce << 1);
}

template <int STAGES, int R>
static int launch_batch(const BatchArgs& A, cudaStream_t st) {
    const int sms = device_sms();
    if (sms <= 0) return OT_ERR_CUDA;
    if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return OT_ERR_CUDA;
    const size_t smem = BatchSmem::total;
    auto kern = batch_solve_kernel<STAGES, R>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OT_ERR_CUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, OT_BT, smem) != cudaSuccess || nb < 1)
        return OT_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sms);
    cfg.blockDim = dim3(OT_BT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, A) != cudaSuccess) return OT_ERR_CUDA;
    return OT_OK;
}

static int batch_solve_cfg(int count, long long total_m, const float* G_all, const float* a_all, const float* b_all,
                           const ot_options* opt, double* w_all, double* z_all, ot_result* results, void* workspace,
                           size_t ws_bytes, cudaStream_t st, const BatchCfg& C, int rows = 0) {
    char* base = (char*)workspace + a256(sizeof(BatchHeader));
    const BatchHeader* hdr = (const BatchHeader*)workspace;
    const BatchLayout L = batch_layout(count, total_m);
    BatchArgs A;
    memset(&A, 0, sizeof(A));
    A.count = count;
    A.total_m = total_m;
    A.G = G_all;
    A.a = a_all;
    A.b = b_all;
    A.tol = opt->tol_l1;
    A.max_iter = opt->max_iter;
    A.timeout_ns = opt->timeout_ns ? opt->timeout_ns : 10000000000ull;
    A.warm = opt->warm_start;
    A.gs_shift = C.gs_shift;
    A.check_every = C.check_every;
    A.nrows = rows ? nullptr : &hdr->nrows[0][0];   // a single problem (rows given) has no prepared header
    A.w_out = w_all;
    A.z_out = z_all;
    A.res = results;
    A.ctrl = (Ctrl*)(base + L.ctrl);
    A.desc = (const ot_problem_desc*)(base + L.desc);
    A.inv_sa = (double*)(base + L.inv_sa);
    A.inv_sb = (double*)(base + L.inv_sb);
    A.active = (int*)(base + L.active);
    A.iters = (int*)(base + L.iters);
    A.l1acc = (double*)(base + L.l1acc);
    A.rs = (float4*)(base + L.rs);
    A.flo = (float*)(base + L.flo);
    A.gam = (double*)(base + L.gam);
    A.gc = (float*)(base + L.gc);
    A.cf = (float*)(base + L.cf);
    A.R = (float*)(base + L.R);
    // the problems with two rows per chunk, then those with three (rows: only one of them)
    if (rows != 3) {
        const int rc = launch_batch<OT_STAGES_MAX, 2>(A, st);
        if (rc != OT_OK || rows == 2) return rc;
    }
    return launch_batch<OT_STAGES_MAX, 3>(A, st);
}

static int batch_check_args(int count, long long total_m, const float* G_all, const float* a_all, const float* b_all,
                            const ot_options* opt, double* w_all, double* z_all, ot_result* results,
                            void* workspace, size_t ws_bytes) {
    if (count <= 0 || count > OT_BATCH_MAX || total_m <= 0 || !G_all || !a_all || !b_all || !opt || !w_all ||
        !z_all || !results || !workspace)
        return OT_ERR_ARG;
    if (opt->max_iter < 1 || opt->tol_l1 < 0.0 || opt->stop_norm != OT_STOP_L1_FULL) return OT_ERR_ARG;
    if (((uintptr_t)G_all) % 16) return OT_ERR_ARG;   // bulk copies of cost rows need 16-byte alignment
    if (ws_bytes < ot_batch_workspace_bytes(count, total_m) || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    return OT_OK;
}

extern "C" int ot_batch_solve(int count, long long total_m, const float* G_all, const float* a_all,
                              const float* b_all, const ot_options* opt, double* w_all, double* z_all,
                              ot_result* results, void* workspace, size_t ws_bytes, void* stream) {
    const int rc = batch_check_args(count, total_m, G_all, a_all, b_all, opt, w_all, z_all, results, workspace,
                                    ws_bytes);
    if (rc != OT_OK) return rc;
    BatchCfg C;
    if (!decode_cfg(opt->tile_override, opt->check_every, C)) return OT_ERR_ARG;
    return batch_solve_cfg(count, total_m, G_all, a_all, b_all, opt, w_all, z_all, results, workspace, ws_bytes,
                           (cudaStream_t)stream, C);
}

namespace cyc {

// One stored-cost problem through the streaming batch kernel (used by the single-problem
// solvers for rows of 4097..8192 columns, where the cost cannot stay in shared memory).
// The potentials follow the batch convention: w = row potential - eps ln N, z = column potential.
size_t batch_single_ws_bytes(int m) { return ot_batch_workspace_bytes(1, m); }

int batch_single_solve(int m, int N, const float* G, int ld, const float* a, const float* b, const ot_options* opt,
                       double* w, double* z, ot_result* out, void* workspace, size_t ws_bytes, cudaStream_t st) {
    if (m <= 0 || m > OT_BATCH_MAXM || ld < m || ld % 4 != 0 || ld > OT_BATCH_MAXM) return OT_ERR_UNSUPPORTED;
    const int rc = batch_check_args(1, m, G, a, b, opt, w, z, out, workspace, ws_bytes);
    if (rc != OT_OK) return rc;
    ot_problem_desc d;
    memset(&d, 0, sizeof(d));
    d.m = m;
    d.N = N;
    d.eps = opt->eps;
    d.ld = ld;
    char* base = (char*)workspace + a256(sizeof(BatchHeader));
    const BatchLayout L = batch_layout(1, m);
    batch_single_table_kernel<<<1, 32, 0, st>>>(d, (ot_problem_desc*)(base + L.desc));
    if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
    BatchCfg C;
    decode_cfg(0, opt->check_every, C);
    return batch_solve_cfg(1, m, G, a, b, opt, w, z, out, workspace, ws_bytes, st, C,
                           chunk_rows(row_slots(ld, C.gs_shift)));
}

}  // namespace cyc

namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, unsigned long long>, int> g_tune_cache;   // (device, batch signature) -> code

// FNV-1a over the problem table and the stopping parameters.
unsigned long long batch_signature(const ot_problem_desc* d, int count, const ot_options* opt) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    for (int i = 0; i < count; ++i) {
        mix(&d[i].m, sizeof(int));
        mix(&d[i].N, sizeof(int));
        mix(&d[i].eps, sizeof(float));
        mix(&d[i].ld, sizeof(int));
    }
    mix(&opt->tol_l1, sizeof(double));
    mix(&opt->max_iter, sizeof(int));
    return h;
}
}  // namespace

extern "C" int ot_batch_autotune(int count, long long total_m, const float* G_all, const float* a_all,
                                 const float* b_all, const ot_options* opt, double* w_all, double* z_all,
                                 ot_result* results, void* workspace, size_t ws_bytes, void* stream,
                                 int* config_out, float* ms_out) {
    int rc = batch_check_args(count, total_m, G_all, a_all, b_all, opt, w_all, z_all, results, workspace, ws_bytes);
    if (rc != OT_OK) return rc;
    if (!config_out) return OT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return OT_ERR_ARG;
    // signature of the prepared problem table
    std::vector<ot_problem_desc> h(count);
    const BatchLayout L = batch_layout(count, total_m);
    const char* base = (const char*)workspace + a256(sizeof(BatchHeader));
    if (cudaMemcpyAsync(h.data(), base + L.desc, sizeof(ot_problem_desc) * (size_t)count, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OT_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OT_ERR_CUDA;
    const auto key = std::make_pair(dev, batch_signature(h.data(), count, opt));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *config_out = it->second;
            return OT_OK;
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return OT_ERR_CUDA;
    auto timed = [&](const BatchCfg& C, const ot_options& o, float& ms) -> int {
        float best = 3.4e38f;
        for (int rep = 0; rep < 2; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return OT_ERR_CUDA;
            int r = batch_solve_cfg(count, total_m, G_all, a_all, b_all, &o, w_all, z_all, results, workspace,
                                    ws_bytes, st, C);
            if (r != OT_OK) return r;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return OT_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = t < best ? t : best;
        }
        ms = best;
        return OT_OK;
    };
    // 1. group-size policy: a few full sweeps (no problem stops early)
    ot_options o = *opt;
    o.warm_start = 0;
    o.tol_l1 = 0.0;
    o.max_iter = 4;
    BatchCfg best;
    best.stages = OT_STAGES_MAX;
    best.gs_shift = 0;
    best.check_every = 1;
    float best_ms = 3.4e38f;
    for (int code = 1; code <= 2 && rc == OT_OK; ++code) {
        BatchCfg C;
        decode_cfg(code, 1, C);
        float ms = 0.f;
        rc = timed(C, o, ms);
        if (ms_out) ms_out[code - 1] = ms;
        if (rc == OT_OK && ms < best_ms) {
            best_ms = ms;
            best = C;
        }
    }
    // 2. convergence-check cadence: complete solves with the caller's stopping rule
    o = *opt;
    o.warm_start = 0;
    float best_full = 3.4e38f;
    int best_ce = 1;
    for (int ce = 1; ce <= 4 && rc == OT_OK; ce <<= 1) {
        BatchCfg C = best;
        C.check_every = ce;
        float ms = 0.f;
        rc = timed(C, o, ms);
        if (ms_out) ms_out[2 + (ce == 1 ? 0 : (ce == 2 ? 1 : 2))] = ms;
        if (rc == OT_OK && ms < best_full) {
            best_full = ms;
            best_ce = ce;
        }
    }
    best.check_every = best_ce;
    // leave the outputs of a complete solve with the chosen configuration
    if (rc == OT_OK)
        rc = batch_solve_cfg(count, total_m, G_all, a_all, b_all, &o, w_all, z_all, results, workspace, ws_bytes, st,
                             best);
    if (rc == OT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = OT_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != OT_OK) return rc;
    *config_out = encode_cfg(best);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = *config_out;
    return OT_OK;
}
