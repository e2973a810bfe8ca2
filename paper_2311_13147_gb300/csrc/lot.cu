// Reduced LOT of Theorem 1 on the GPU: the small linear program (Eq.
// small_problem_CLOT)
//
//     min <G, S>  s.t.  S 1 = alpha,  S^T 1 = beta,  S >= 0,
//
// with G the min-fold of the cost blocks (Eq. definition_G) and alpha, beta the
// base marginals (mass 1/N each).  Its optimal value is the C-LOT value, and
// Eq. optimal_solution_problem_CLOT unfolds S into the block-circulant plan.
// Sec. 5.2 solves this problem with the network simplex; so does this file, as
// a primal network simplex on the complete bipartite graph of m sources
// (nodes 0..m-1), m sinks (nodes m..2m-1) and an artificial root (node 2m):
//
//  costs    pivoting runs on integer costs: g_ij = rint(G_ij 2^k) with 2^k the
//           largest power of two keeping |g| < 2^30, so reduced costs and
//           potentials are exact 64-bit integers (no tolerance; FP64, slow on
//           this GPU, stays out of the parallel loops).  The plan is optimal
//           for these costs and within 2^-k per unit of mass, about
//           1e-9 max|G|, of the optimum for the FP32 costs;
//  start    every source sends its supply to the root and the root feeds every
//           sink, over artificial arcs of cost M = (max|g| + 1)(2m + 1), a
//           strongly feasible spanning tree (a zero-flow arc points away from
//           the root);
//  pricing  reduced costs g_ij - pi(i) + pi(m + j) of a block of rows, in
//           parallel over the block's threads; the most negative one enters
//           if it is negative, else the next block of rows is priced, and a
//           full pass without a candidate proves optimality;
//  pivot    one thread: the entering arc closes a cycle with the tree paths
//           from its ends up to their common ancestor; the flow on the cycle's
//           backward arcs bounds the step, and of the blocking arcs the last
//           one met when going round the cycle from that ancestor leaves (the
//           rule that keeps the tree strongly feasible, so degenerate pivots
//           cannot cycle); the cut-off subtree is re-hung from the entering
//           arc by reversing the parent pointers on the path between them;
//  duals    every node's potential is the signed sum of arc costs on its path
//           to the root (pi(x) = c + pi(parent) over an arc x -> parent,
//           pi(x) = pi(parent) - c over parent -> x): recomputed from the tree
//           after each pivot by pointer jumping over all nodes in parallel.
//           A node's jump pointer and partial sum share one 64-bit word, so
//           every read sees a consistent pair and the jumps need no barrier
//           between reads and writes (one per pass, about log2 depth passes).
//
// One thread block solves one problem and holds its tree in shared memory, 18
// bytes per node: the potential with the jump pointer (one 64-bit word), the
// FP64 flow on the node's parent arc, and the parent and the arc's direction
// in 16 bits (an original arc is fixed by its two ends, and points from the
// source to the sink; an arc to the root is artificial).  A launch solves
// `count` problems of one size at once.
// Every loop has a bound; a tree found inconsistent ends the solve with
// OT_ERR_NONFINITE instead of looping.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

#define LOT_BT 1024
#define LOT_BW (LOT_BT / 32)
#define LOT_MAXM 5120
#define LOT_PRICE_ARCS 16384                                 // arcs priced per step (whole rows)
#define LOT_PPT (LOT_PRICE_ARCS / LOT_BT)                    // arcs per thread and step
#define LOT_MAX_ROUNDS 20                                    // pointer-jumping rounds (2^20 > any depth)

struct LotArgs {
    int count, m, N;
    const float* a;        // [count][m] unnormalised
    const float* b;
    const float* G;        // [count][m][m]
    long long max_pivots;
    float* S;              // [count][m][m]
    double* u;             // [count][m]
    double* v;
    ot_result* res;        // [count]
    double* sums;          // [count][2m] row and column sums of the returned plan (workspace)
};

// Block minimum of (value, index) pairs; ties go to the smaller index.  Every
// thread returns the result.
__device__ __forceinline__ void lot_argmin(long long& v, int& idx, long long* s_v, int* s_i) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    if (lane == 0) {
        s_v[w] = v;
        s_i[w] = idx;
    }
    __syncthreads();
    if (w == 0) {
        v = s_v[lane];
        idx = s_i[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov < v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        if (lane == 0) {
            s_v[LOT_BW] = v;
            s_i[LOT_BW] = idx;
        }
    }
    __syncthreads();
    v = s_v[LOT_BW];
    idx = s_i[LOT_BW];
}

__device__ __forceinline__ double lot_sum(double x, double* s_v) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) s_v[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < LOT_BW; ++k) t += s_v[k];   // same order in every thread
    return t;
}

// A node's word: jump pointer in the top 14 bits, potential (|pi| < 2^46) as a
// 50-bit two's-complement field below it.
#define LOT_PB 50
#define LOT_MARK 0x3fff   // jump-pointer value marking a node during a pivot (above any node index)

__device__ __forceinline__ long long lot_pack(int anc, long long pi) {
    return (long long)(((unsigned long long)anc << LOT_PB) | ((unsigned long long)pi & ((1ull << LOT_PB) - 1)));
}
__device__ __forceinline__ int lot_anc(long long w) { return (int)((unsigned long long)w >> LOT_PB); }
__device__ __forceinline__ long long lot_pi(long long w) { return (long long)((unsigned long long)w << (64 - LOT_PB)) >> (64 - LOT_PB); }

// Original arc between node x and its parent y (one a source, the other a sink).
__device__ __forceinline__ int lot_arc(int x, int y, int m) {
    return x < m ? x * m + (y - m) : y * m + (x - m);
}

// One pivot (a single thread).  pu[x] = 2 parent + up (up = 1 when x's parent
// arc points from x to the parent; the root is its own parent), flow[x] the
// flow on that arc; the jump-pointer fields of the words serve as marks here
// (every one is the root when a pivot starts).  Returns 0 or an OT_ERR_*.
__device__ int lot_pivot(int e, int m, unsigned short* pu, long long* word, double* flow) {
    const int V = 2 * m + 1, R = 2 * m;
    const int u = e / m, v = m + (e - (e / m) * m);
    // common ancestor w: mark the path from u to the root, climb from v to a mark
    int x = u;
    for (int s = 0;; ++s) {
        if (s > V) return OT_ERR_NONFINITE;
        word[x] = lot_pack(LOT_MARK, lot_pi(word[x]));
        if (x == R) break;
        x = pu[x] >> 1;
    }
    int w = v;
    for (int s = 0; lot_anc(word[w]) != LOT_MARK; ++s) {
        if (s > V) return OT_ERR_NONFINITE;
        w = pu[w] >> 1;
    }
    // leaving arc: the cycle runs w -> ... -> u (down), u -> v, v -> ... -> w (up).
    // Backward arcs: on the u side those pointing up, on the v side those pointing
    // down.  Of the blocking arcs the last in that order leaves: on the u side the
    // deepest (strict <, climbing from u), on the v side the highest (<=, climbing
    // from v, and after every u-side arc).
    double delta = INFINITY;
    int leave = -1, leave_u = 0;
    int len = 0;
    for (x = u; x != w; x = pu[x] >> 1) {
        if (++len > V) return OT_ERR_NONFINITE;
        if ((pu[x] & 1) && flow[x] < delta) {
            delta = flow[x];
            leave = x;
            leave_u = 1;
        }
    }
    for (x = v; x != w; x = pu[x] >> 1) {
        if (++len > V) return OT_ERR_NONFINITE;
        if (!(pu[x] & 1) && flow[x] <= delta) {
            delta = flow[x];
            leave = x;
            leave_u = 0;
        }
    }
    if (leave < 0 || !(delta < INFINITY)) return OT_ERR_NONFINITE;   // cannot happen: every cycle has a backward arc
    for (x = u; x != w; x = pu[x] >> 1) flow[x] += (pu[x] & 1) ? -delta : delta;
    for (x = v; x != w; x = pu[x] >> 1) flow[x] += (pu[x] & 1) ? delta : -delta;
    // re-hang: q is the entering arc's end inside the cut-off subtree; the path
    // q -> ... -> leave is reversed, each node taking over its old child's arc
    // (the reversed path holds original arcs only: an artificial arc joins a node
    // to the root, which stays above the leaving arc)
    const int q = leave_u ? u : v;
    int np = leave_u ? v : u;
    int nup = leave_u ? 1 : 0;   // u -> v points up from u, down to v
    double nfl = delta;
    x = q;
    for (int s = 0;; ++s) {
        if (s > V) return OT_ERR_NONFINITE;
        const int op = pu[x] >> 1, oup = pu[x] & 1;
        const double ofl = flow[x];
        pu[x] = (unsigned short)(2 * np + nup);
        flow[x] = nfl;
        if (x == leave) break;
        np = x;
        nup = oup ^ 1;   // the same arc seen from the other end
        nfl = ofl;
        x = op;
    }
    return OT_OK;
}

__global__ void __launch_bounds__(LOT_BT, 1) lot_simplex_kernel(const __grid_constant__ LotArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int m = A.m, V = 2 * m + 1, R = 2 * m;
    long long* word = reinterpret_cast<long long*>(dsm);                  // [V] jump pointer + potential
    double* flow = reinterpret_cast<double*>(word + V);                   // [V] flow on the parent arc
    unsigned short* pu = reinterpret_cast<unsigned short*>(flow + V);     // [V] 2 parent + up
    __shared__ double s_v[LOT_BW + 1];
    __shared__ long long s_q[LOT_BW + 1];
    __shared__ int s_i[LOT_BW + 1];
    __shared__ int s_err;

    const int p = blockIdx.x, tid = threadIdx.x;
    const long long mm = (long long)m * m;
    const float* G = A.G + (size_t)p * mm;
    const float* a = A.a + (size_t)p * m;
    const float* b = A.b + (size_t)p * m;
    double* sums = A.sums + (size_t)p * 2 * m;
    float* S = A.S + (size_t)p * mm;
    ot_result* res = A.res + p;

    // ---- marginal sums, cost bound and validation
    double sa = 0.0, sb = 0.0;
    int bad = 0;
    for (int i = tid; i < m; i += LOT_BT) {
        const float x = a[i], y = b[i];
        bad |= !(x >= 0.f && x < INFINITY) || !(y >= 0.f && y < INFINITY);
        sa += x;
        sb += y;
    }
    float gmax = 0.f;
    for (long long e = tid; e < mm; e += LOT_BT) {
        const float c = fabsf(G[e]);
        bad |= !(c < INFINITY);
        gmax = fmaxf(gmax, c);
    }
    bad = __syncthreads_or(bad);
    sa = lot_sum(sa, s_v);
    sb = lot_sum(sb, s_v);
    gmax = warp_max(gmax);
    __syncthreads();
    if ((tid & 31) == 0) s_v[tid >> 5] = gmax;
    __syncthreads();
    for (int k = 0; k < LOT_BW; ++k) gmax = fmaxf(gmax, (float)s_v[k]);
    if (bad || !(sa > 0.0) || !(sb > 0.0)) {
        for (long long e = tid; e < mm; e += LOT_BT) S[e] = NAN;
        for (int i = tid; i < m; i += LOT_BT) {
            A.u[(size_t)p * m + i] = NAN;
            A.v[(size_t)p * m + i] = NAN;
        }
        if (tid == 0) {
            res->iters = 0;
            res->status = OT_ERR_ARG;
            res->marg_l1 = res->marg_l1_col = res->marg_l2_col = -1.0;
            res->value = res->transport_cost = NAN;
            res->reserved[0] = NAN;
            res->reserved[1] = 6.0;   // variant code: reduced LOT
        }
        return;
    }
    const double ia = 1.0 / (sa * (double)A.N), ib = 1.0 / (sb * (double)A.N);
    // integer costs rint(G 2^k) with |g| < 2^30; |potentials| <= 2 M + V 2^30 < 2^46
    const int k2 = gmax > 0.f ? min(100, max(-120, 29 - ilogbf(gmax))) : 0;
    const float sc = ldexpf(1.0f, k2);
    const long long M = ((long long)ldexpf(gmax, k2) + 1) * (long long)V;

    // ---- strongly feasible artificial start
    for (int x = tid; x < V; x += LOT_BT) {
        if (x == R) {
            pu[x] = (unsigned short)(2 * R);
            flow[x] = 0.0;
            word[x] = lot_pack(R, 0);
        } else if (x < m) {
            const double al = (double)a[x] * ia;
            const int up = al > 0.0 ? 1 : 0;   // a zero supply hangs below the root with zero flow
            pu[x] = (unsigned short)(2 * R + up);
            flow[x] = al;
            word[x] = lot_pack(R, up ? M : -M);
        } else {
            pu[x] = (unsigned short)(2 * R);   // root -> sink
            flow[x] = (double)b[x - m] * ib;
            word[x] = lot_pack(R, -M);
        }
    }
    if (tid == 0) s_err = 0;

    // ---- pivots
    const int rb = max(1, min(m, LOT_PRICE_ARCS / m));   // rows per pricing step (rb m <= LOT_PRICE_ARCS)
    const int qstep = LOT_BT / m, rstep = LOT_BT - (LOT_BT / m) * m;
    const int npt = (V + LOT_BT - 1) / LOT_BT;            // tree nodes per thread
    long long piv = 0;
    int status = OT_OK;
    int cursor = 0, scanned = 0;
    for (;;) {
        __syncthreads();   // potentials and the previous reduction's results are settled
        const int r1 = min(m, cursor + rb);
        long long best = 0x7fffffffffffffffll;
        int be = 0x7fffffff;
        {
            // arcs e = cursor m + tid + k LOT_BT of rows [cursor, r1): all loads issued up front
            const int e_end = r1 * m;
            int e = cursor * m + tid;
            int r = e / m, j = e - r * m;
#pragma unroll
            for (int k = 0; k < LOT_PPT; ++k) {
                if (e < e_end) {
                    const long long rc = (long long)__float2int_rn(G[e] * sc) - lot_pi(word[r]) + lot_pi(word[m + j]);
                    if (rc < best) {
                        best = rc;
                        be = e;
                    }
                }
                e += LOT_BT;
                j += rstep;
                r += qstep;
                if (j >= m) {
                    j -= m;
                    ++r;
                }
            }
        }
        lot_argmin(best, be, s_q, s_i);
        scanned += r1 - cursor;
        cursor = r1 == m ? 0 : r1;
        if (best >= 0) {
            if (scanned >= m) break;   // a full pass found no improving arc: optimal
            continue;
        }
        scanned = 0;
        if (piv >= A.max_pivots) {
            status = OT_ERR_NOT_CONVERGED;
            break;
        }
        if (tid == 0) s_err = lot_pivot(be, m, pu, word, flow);
        __syncthreads();
        if (s_err != OT_OK) {
            status = s_err;
            break;
        }
        ++piv;
        // potentials by pointer jumping: word[x] = (anc, pi(x) - pi(anc)) until anc is the root
        for (int k = 0; k < npt; ++k) {
            const int x = tid + k * LOT_BT;
            if (x < V) {
                if (x == R) {
                    word[x] = lot_pack(R, 0);
                } else {
                    const int y = pu[x] >> 1;
                    const long long c = y == R ? M : (long long)__float2int_rn(G[lot_arc(x, y, m)] * sc);
                    word[x] = lot_pack(y, (pu[x] & 1) ? c : -c);
                }
            }
        }
        __syncthreads();
        // passes: each owned node jumps to its pointer's pointer and adds its partial sum.
        // Only a node's owner writes its word, and every word (one 64-bit shared-memory
        // access) satisfies the invariant, so reads racing with writes are harmless; a
        // jump pointer only moves up, and a pass that finds every pointer at the root ends
        int rounds = 0;
        {
            volatile long long* vw = word;
            for (;;) {
                int any = 0;
                for (int k = 0; k < npt; ++k) {
                    const int x = tid + k * LOT_BT;
                    if (x >= V) break;
                    const long long w = vw[x];
                    const int y = lot_anc(w);
                    if (y != R) {
                        const long long w2 = vw[y];
                        vw[x] = lot_pack(lot_anc(w2), lot_pi(w) + lot_pi(w2));
                        any = 1;
                    }
                }
                if (!__syncthreads_or(any)) break;
                if (++rounds > LOT_MAX_ROUNDS) break;   // uniform; caught below
            }
        }
        if (rounds > LOT_MAX_ROUNDS) {
            status = OT_ERR_NONFINITE;
            break;
        }
    }
    __syncthreads();

    // ---- outputs: the plan from the basic flows, duals u_i = pi(i) - pi(0), v_j = pi(0) - pi(m + j)
    for (long long e = tid; e < mm; e += LOT_BT) S[e] = 0.f;
    for (int k = tid; k < 2 * m; k += LOT_BT) sums[k] = 0.0;
    __syncthreads();
    double val = 0.0, art = 0.0;
    for (int x = tid; x < V; x += LOT_BT) {
        if (x == R) continue;
        const int y = pu[x] >> 1;
        if (y != R) {
            const int arc = lot_arc(x, y, m);
            const float f = (float)flow[x];
            S[arc] = f;
            val += flow[x] * (double)G[arc];   // the LP value from the FP64 flows
            const int i = arc / m, j = arc - i * m;
            atomicAdd(&sums[i], (double)f);
            atomicAdd(&sums[m + j], (double)f);
        } else {
            art += flow[x];
        }
    }
    const long long p0 = lot_pi(word[0]);
    const double unit = ldexp(1.0, -k2);
    double dual = 0.0, l1r = 0.0, l1c = 0.0, l2c = 0.0;
    __syncthreads();
    for (int i = tid; i < m; i += LOT_BT) {
        const double al = (double)a[i] * ia, be2 = (double)b[i] * ib;
        const double ui = (double)(lot_pi(word[i]) - p0) * unit, vj = (double)(p0 - lot_pi(word[m + i])) * unit;
        A.u[(size_t)p * m + i] = ui;
        A.v[(size_t)p * m + i] = vj;
        dual += al * ui + be2 * vj;
        l1r += fabs(sums[i] - al);
        const double dc = sums[m + i] - be2;
        l1c += fabs(dc);
        l2c += dc * dc;
    }
    val = lot_sum(val, s_v);
    art = lot_sum(art, s_v);
    dual = lot_sum(dual, s_v);
    l1r = lot_sum(l1r, s_v);
    l1c = lot_sum(l1c, s_v);
    l2c = lot_sum(l2c, s_v);
    if (tid == 0) {
        // flow left on artificial arcs beyond rounding means M was too small (not expected)
        if (status == OT_OK && art > 1e-9 / (double)A.N) status = OT_ERR_NOT_CONVERGED;
        const double Nd = (double)A.N;
        res->iters = (int)(piv < 0x7fffffff ? piv : 0x7fffffff);
        res->status = status;
        res->marg_l1 = Nd * l1r;            // full scale: the N row blocks of the plan are alike
        res->marg_l1_col = Nd * l1c;
        res->marg_l2_col = sqrt(Nd * l2c);
        res->value = Nd * val;              // full scale: the C-LOT value is N <G, S> (mass 1/N, Theorem 1)
        res->transport_cost = Nd * val;
        res->reserved[0] = Nd * dual;       // N (<alpha, u> + <beta, v>): equals value at optimality
        res->reserved[1] = 6.0;             // variant code: reduced LOT
    }
}

size_t lot_smem_bytes(int m) { return (size_t)18 * (2 * (size_t)m + 1) + 16; }
static_assert(2 * (2 * LOT_MAXM + 1) < 0xffff, "parent and direction fit 16 bits");
static_assert(2 * LOT_MAXM < LOT_MARK, "node indices fit the 14-bit jump pointer, below the mark");

}  // namespace cyc

using namespace cyc;

static size_t lot_a256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" size_t ot_lot_workspace_bytes(int count, int m) {
    if (count <= 0 || m <= 0 || m > LOT_MAXM) return 0;
    return lot_a256(sizeof(double) * (size_t)count * 2 * (size_t)m);
}

extern "C" int ot_lot_reduced(int count, int m, int N, const float* a_base, const float* b_base, const float* G,
                              const ot_options* opt, float* S, double* u, double* v, ot_result* out, void* workspace,
                              size_t ws_bytes, void* stream) {
    if (count <= 0 || m <= 0 || N <= 0 || !a_base || !b_base || !G || !opt || !S || !u || !v || !out)
        return OT_ERR_ARG;
    if (opt->max_iter < 1) return OT_ERR_ARG;
    if (m > LOT_MAXM) return OT_ERR_UNSUPPORTED;
    const size_t need = ot_lot_workspace_bytes(count, m);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace) % 256) return OT_ERR_WORKSPACE;
    LotArgs A;
    memset(&A, 0, sizeof(A));
    A.count = count;
    A.m = m;
    A.N = N;
    A.a = a_base;
    A.b = b_base;
    A.G = G;
    A.max_pivots = opt->max_iter;
    A.S = S;
    A.u = u;
    A.v = v;
    A.res = out;
    A.sums = (double*)workspace;
    const size_t smem = lot_smem_bytes(m);
    if (cudaFuncSetAttribute(lot_simplex_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return OT_ERR_CUDA;
    lot_simplex_kernel<<<count, LOT_BT, smem, (cudaStream_t)stream>>>(A);
    return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}
