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
//  pricing  reduced costs g_ij - pi(i) + pi(m + j) of a block of rows (about
//           16384 arcs), in parallel over the block's threads, four arcs per
//           16-byte load when m is a multiple of 4; the most negative one enters
//           if it is negative, else the next block of rows is priced, and a
//           full pass without a candidate proves optimality;
//  tree     besides parent pointers, every node has its position in a preorder
//           of the tree and its subtree size, so that a subtree is the
//           contiguous range [pos, pos + size) and "y is an ancestor of x" is
//           a range test;
//  pivot    one warp: the entering arc closes a cycle with the tree paths
//           from its ends up to their common ancestor, found by climbing from
//           each end (two lanes at once) until the range holds the other end;
//           the paths are recorded, and the rest of the pivot runs over them
//           in parallel.  The flow on the cycle's backward arcs bounds the
//           step, and of the blocking arcs the last one met when going round
//           the cycle from that ancestor leaves (the rule that keeps the tree
//           strongly feasible, so degenerate pivots cannot cycle); the cut-off subtree T is re-hung from the entering
//           arc by reversing the parent pointers on the path between them,
//           and only the subtree sizes on the cycle change outside T;
//  duals    every node's potential is the signed sum of arc costs on its path
//           to the root (pi(x) = c + pi(parent) over an arc x -> parent,
//           pi(x) = pi(parent) - c over parent -> x).  A pivot changes the
//           potentials of T only, all by the entering arc's reduced cost (the
//           potentials are exact integers, so the shift is exact), and moves
//           T's range next to its new parent: the re-rooted subtree's preorder
//           is the old range of each node on the reversed path minus that of
//           the node below it, concatenated from the entering end up.  One
//           parallel pass over the nodes applies the shift, the new positions
//           (a binary search on the nested ranges of the reversed path) and
//           the path's new sizes.
//
// One thread block (CTA 0 of a cluster, when several price) solves one problem
// and holds its tree in shared memory, 22 bytes per node: the potential with
// the subtree size (one 64-bit word), the FP64 flow on the node's parent arc,
// the parent and the arc's direction in 16 bits (an original arc is fixed by
// its two ends, and points from the source to the sink; an arc to the root is
// artificial), the preorder position, and one slot of the pivot's path buffer.
// A launch solves `count` problems of one size at once.  Every loop has a bound;
// a tree found inconsistent (also by a check of every potential against its
// parent arc after the last pivot) ends the solve with OT_ERR_NONFINITE instead
// of looping.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace cyc {

#define LOT_BT 1024
#define LOT_BW (LOT_BT / 32)
#define LOT_MAXM 5120
#define LOT_PRICE_ARCS 16384                                 // arcs priced per step (whole rows)
#define LOT_PPT (LOT_PRICE_ARCS / LOT_BT)                    // arcs per thread and pass

// Passes of LOT_PRICE_ARCS arcs per pricing step: a wider block finds better entering
// arcs (fewer pivots: on the paper's synthetic costs 68072 -> 33011 at m = 5000 with
// four passes) but costs more per scan, which pays only when the pivots are dear.
__device__ __forceinline__ int lot_price_passes(int m) { return m >= 4000 ? 4 : m >= 1500 ? 2 : 1; }

#define LOT_NPT ((2 * LOT_MAXM + 1 + LOT_BT - 1) / LOT_BT)   // tree nodes per thread, at most
#define LOT_CPK 256                                          // reversed-path ranges kept packed for the move pass
#define LOT_CLUSTER_MIN_M 800   // clusters per instance from this m (Table 1: 37.5 vs 41.5 ms at m = 1000; slower at m <= 500)

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
    unsigned long long timeout_ns;   // bound on each wait between the CTAs of a cluster
    int debug_flags;                 // OT_DEBUG_WITHHOLD_ARRIVAL: CTA 1 withholds its first candidate
};

// ---- thread-block cluster helpers (one instance per cluster of CL CTAs)
__device__ __forceinline__ unsigned lot_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address of this variable in CTA `rank` of the cluster (the shared layout is the same in every CTA).
__device__ __forceinline__ unsigned lot_mapa(const void* p, unsigned rank) {
    unsigned a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
    return a;
}
__device__ __forceinline__ void lot_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void lot_remote_arrive(unsigned addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ long long lot_ld_remote64(unsigned addr) {
    long long v;
    asm volatile("ld.shared::cluster.b64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int lot_ld_remote32(unsigned addr) {
    int v;
    asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void lot_st_remote64(unsigned addr, long long v) {
    asm volatile("st.shared::cluster.b64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void lot_st_remote32(unsigned addr, int v) {
    asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Bounded wait for phase `parity` of a barrier that other CTAs of the cluster arrive on.
__device__ __forceinline__ bool lot_wait_cluster(unsigned long long* bar, unsigned parity, unsigned long long timeout_ns) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer() - t0 > timeout_ns) return false;
    }
}

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
        v = lane < LOT_BW ? s_v[lane] : 0x7fffffffffffffffll;
        idx = lane < LOT_BW ? s_i[lane] : 0x7fffffff;
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

// A node's word: pi 2^14 + size, the potential (|pi| < 2^46) above the subtree
// size (1 <= size <= 2m + 1 < 2^14).  Adding d 2^14 shifts the potential, adding
// d the size.
#define LOT_SB 14
__device__ __forceinline__ long long lot_pack(long long pi, int size) { return pi * (1ll << LOT_SB) + size; }
__device__ __forceinline__ long long lot_pi(long long w) { return w >> LOT_SB; }
__device__ __forceinline__ int lot_size(long long w) { return (int)(w & ((1ll << LOT_SB) - 1)); }

// Original arc between node x and its parent y (one a source, the other a sink).
__device__ __forceinline__ int lot_arc(int x, int y, int m) {
    return x < m ? x * m + (y - m) : y * m + (x - m);
}

// Reduced costs of the arcs [e0, e0 + NP LOT_PRICE_ARCS) below e_end, four consecutive
// arcs of one row per 16-byte load (m % 4 == 0, 16-byte aligned costs); the most
// negative one (the first on ties) is merged into (best, be).
template <int NP>
__device__ __forceinline__ void lot_price_vec4(const float* G, const long long* word, int m, int e0, int e_end,
                                               float sc, long long& best, int& be) {
    const float4* G4 = reinterpret_cast<const float4*>(G);
#pragma unroll
    for (int k = 0; k < NP * LOT_PPT / 4; ++k) {
        const int e = e0 + 4 * ((int)threadIdx.x + k * LOT_BT);
        if (e < e_end) {
            const float4 c4 = G4[e >> 2];
            const int r = e / m, j = e - r * m;
            const long long pr = lot_pi(word[r]);
            const longlong2 w01 = *reinterpret_cast<const longlong2*>(word + m + j);
            const longlong2 w23 = *reinterpret_cast<const longlong2*>(word + m + j + 2);
            const long long r0 = (long long)__float2int_rn(c4.x * sc) - pr + lot_pi(w01.x);
            const long long r1 = (long long)__float2int_rn(c4.y * sc) - pr + lot_pi(w01.y);
            const long long r2 = (long long)__float2int_rn(c4.z * sc) - pr + lot_pi(w23.x);
            const long long r3 = (long long)__float2int_rn(c4.w * sc) - pr + lot_pi(w23.y);
            if (r0 < best) { best = r0; be = e; }
            if (r1 < best) { best = r1; be = e + 1; }
            if (r2 < best) { best = r2; be = e + 2; }
            if (r3 < best) { best = r3; be = e + 3; }
        }
    }
}

// What the parallel pass of a pivot needs: T = the old range [a0, a0 + s), its
// new parent at old position P, the reversed path p_0..p_{k-1} (p_0 the entering
// end, p_{k-1} the node whose parent arc left; p_t = chain[t] when dir = 1,
// chain[V - 1 - t] when dir = -1) and the potential shift.
struct LotMove {
    int a0, s, P, k, dir;
    int lbase, lcap;   // free part of the path buffer, [lbase, lbase + lcap): T's node list
    long long sigma;
};

__device__ __forceinline__ int lot_path_at(const unsigned short* chain, int V, int dir, int t) {
    return dir > 0 ? chain[t] : chain[V - 1 - t];
}

// Warp minimum of (flow, rank) pairs: the smaller flow, then the smaller rank.
__device__ __forceinline__ void lot_warp_argmin(double& f, int& r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, f, o);
        const int orr = __shfl_xor_sync(0xffffffffu, r, o);
        if (of < f || (of == f && orr < r)) {
            f = of;
            r = orr;
        }
    }
}

// One pivot by the 32 lanes of one warp, on the entering arc e with reduced cost
// rc < 0.  pu[x] = 2 parent + up (up = 1 when x's parent arc points from x to the
// parent; the root is its own parent), flow[x] the flow on that arc, pos and the
// size field of word the preorder ranges.  Updates the flows, the parent
// pointers of the reversed path and the sizes on the cycle outside T; T's
// potentials, positions and sizes are left to the block's parallel pass.
// Returns 0 or an OT_ERR_* (the same value in every lane).
//
//  1. lane 0 climbs from u, lane 1 from v, each until the node's range holds the
//     other end (both stop at the common ancestor w), recording the nodes below
//     w: the u side from chain[0] up, the v side from chain[V - 1] down;
//  2. the cycle runs w -> ... -> u (down), u -> v, v -> ... -> w (up); its
//     backward arcs are those pointing up on the u side and down on the v side,
//     and of the blocking ones the last met in that order leaves: ranked, the v
//     side's from the highest down come first, then the u side's from the
//     deepest up, and the warp takes the smallest (flow, rank);
//  3. the step moves along both sides in parallel;
//  4. the path from the entering end q to the leaving node is reversed, each node
//     taking over its old child's arc (all of a lane group's reads before its
//     writes, groups from the leaving end down, so no old value is overwritten
//     before it is read); the reversed path holds original arcs only, since an
//     artificial arc joins a node to the root, which stays above the leaving arc;
//  5. the leaving node's old ancestors below w lose T's size, the new parent's
//     gain it.
__device__ int lot_pivot_warp(int e, long long rc, int m, unsigned short* pu, unsigned short* pos, long long* word,
                              double* flow, unsigned short* chain, unsigned* cpk, LotMove* mv) {
    const int V = 2 * m + 1, lane = threadIdx.x & 31;
    const int u = e / m, v = m + (e - (e / m) * m);
    // 1. the two climbs
    int len = 0;
    if (lane < 2) {
        int x = lane == 0 ? u : v;
        const int po = pos[lane == 0 ? v : u];
        for (;;) {
            const int px = pos[x], sx = lot_size(word[x]), nx = pu[x] >> 1;   // one round trip per step
            if (px <= po && po < px + sx) break;
            if (len >= V) {
                len = V + 1;   // inconsistent tree
                break;
            }
            chain[lane == 0 ? len : V - 1 - len] = (unsigned short)x;
            ++len;
            x = nx;
        }
    }
    const int ku = __shfl_sync(0xffffffffu, len, 0), kv = __shfl_sync(0xffffffffu, len, 1);
    if (ku + kv > V - 1) return OT_ERR_NONFINITE;
    __syncwarp();
    // 2. the leaving arc
    double f = INFINITY;
    int r = 0x7fffffff;
    for (int t = lane; t < ku + kv; t += 32) {
        const bool vside = t < kv;
        const int x = vside ? chain[V - 1 - t] : chain[t - kv];
        const int up = pu[x] & 1;
        if (vside ? !up : up) {
            const double fx = flow[x];
            const int rx = vside ? kv - 1 - t : t;   // v side: highest first; then u side: deepest first
            if (fx < f || (fx == f && rx < r)) {
                f = fx;
                r = rx;
            }
        }
    }
    lot_warp_argmin(f, r);
    if (r == 0x7fffffff || !(f < INFINITY)) return OT_ERR_NONFINITE;   // cannot happen: every cycle has a backward arc
    const double delta = f;
    const int leave_u = r >= kv;
    const int li = leave_u ? r - kv : kv - 1 - r;   // the leaving node's index along its side
    const int leave = leave_u ? chain[li] : chain[V - 1 - li];
    // 3. the step
    if (delta > 0.0) {
        for (int t = lane; t < ku + kv; t += 32) {
            const bool vside = t < kv;
            const int x = vside ? chain[V - 1 - t] : chain[t - kv];
            const bool upx = pu[x] & 1;
            flow[x] += (vside ? upx : !upx) ? delta : -delta;
        }
    }
    __syncwarp();
    // 4. re-hang along p_0 = q .. p_li = leave
    const int dir = leave_u ? 1 : -1;
    const int nparent = leave_u ? v : u;
    const int s = lot_size(word[leave]);
    for (int t0 = (li / 32) * 32; t0 >= 0; t0 -= 32) {
        const int t = t0 + lane;
        int npu = 0;
        double nfl = 0.0;
        if (t <= li) {
            if (t == 0) {
                npu = 2 * nparent + (leave_u ? 1 : 0);   // u -> v points up from u, down to v
                nfl = delta;
            } else {
                const int c = lot_path_at(chain, V, dir, t - 1);   // the old child on the path
                npu = 2 * c + ((pu[c] & 1) ^ 1);                   // the same arc seen from the other end
                nfl = flow[c];
            }
        }
        __syncwarp();
        if (t <= li) {
            const int x = lot_path_at(chain, V, dir, t);
            pu[x] = (unsigned short)npu;
            flow[x] = nfl;
            // the path's (unchanged) range, packed for the move pass's binary search
            if (t < LOT_CPK) cpk[t] = (unsigned)pos[x] | ((unsigned)lot_size(word[x]) << 16);
        }
        __syncwarp();
    }
    // 5. sizes on the cycle outside T
    for (int t = lane; t < ku + kv; t += 32) {
        const bool vside = t < kv;
        const int i = vside ? t : t - kv;    // index along its side
        const int x = vside ? chain[V - 1 - t] : chain[t - kv];
        if (vside == (bool)leave_u) {
            word[x] += s;                    // the new parent's side, up to w
        } else if (i > li) {
            word[x] -= s;                    // above the leaving node on its side
        }
    }
    if (lane == 0) {
        mv->a0 = pos[leave];
        mv->s = s;
        mv->P = pos[nparent];
        mv->k = li + 1;
        mv->dir = dir;
        mv->lbase = ku;
        mv->lcap = V - ku - kv;
        mv->sigma = leave_u ? rc : -rc;   // the entering arc's reduced cost becomes 0
    }
    return OT_OK;
}

// Node x after the move mv, packed in 32 bits: the new position (bits 0-13), x in
// T (bit 14: its potential shifts by mv.sigma), x on the reversed path (bit 15)
// with its new subtree size (bits 16-29).  Reads old positions and the sizes of
// the path's nodes, which the pass writes only after a barrier.
// The old range of the reversed path's node t: packed when t < LOT_CPK, else from the tree.
__device__ __forceinline__ void lot_path_range(int t, int V, const LotMove& mv, const unsigned short* pos,
                                               const long long* word, const unsigned short* chain,
                                               const unsigned* cpk, int& p, int& sz) {
    if (t < LOT_CPK) {
        const unsigned v = cpk[t];
        p = (int)(v & 0xffffu);
        sz = (int)(v >> 16);
    } else {
        const int c = lot_path_at(chain, V, mv.dir, t);
        p = pos[c];
        sz = lot_size(word[c]);
    }
}

__device__ __forceinline__ unsigned lot_move_node(int x, int V, const LotMove& mv, const unsigned short* pos,
                                                  const long long* word, const unsigned short* chain,
                                                  const unsigned* cpk) {
    const int xp = pos[x];
    if (xp >= mv.a0 && xp < mv.a0 + mv.s) {
        // the first path node whose range holds xp (the ranges grow along the path)
        int lo = 0, hi = mv.k - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            int cp, cs;
            lot_path_range(mid, V, mv, pos, word, chain, cpk, cp, cs);
            if (cp <= xp && xp < cp + cs)
                hi = mid;
            else
                lo = mid + 1;
        }
        int cp, cs, off, psz = 0;
        lot_path_range(lo, V, mv, pos, word, chain, cpk, cp, cs);
        if (lo == 0) {
            off = xp - cp;
        } else {
            int pp;
            lot_path_range(lo - 1, V, mv, pos, word, chain, cpk, pp, psz);
            off = psz + xp - cp - (xp >= pp + psz ? psz : 0);
        }
        const unsigned np = (unsigned)((mv.P < mv.a0 ? mv.P + 1 : mv.P + 1 - mv.s) + off);
        if (xp != cp) return np | 0x4000u;   // positions are unique: xp == cp exactly for the path node
        return np | 0xC000u | ((unsigned)(lo == 0 ? mv.s : mv.s - psz) << 16);   // a reversed path's new size
    }
    if (mv.P < mv.a0) return (unsigned)((xp > mv.P && xp < mv.a0) ? xp + mv.s : xp);
    return (unsigned)((xp >= mv.a0 + mv.s && xp <= mv.P) ? xp - mv.s : xp);
}

// CL > 1: one instance per cluster of CL CTAs.  CTA 0 (the owner) holds the tree and
// pivots; every CTA keeps a copy of the potentials and prices its own part of a
// pricing block CL times as wide (one pass each), and the owner takes the most
// negative reduced cost over the parts (the smallest arc on ties, so the choice is
// the single-CTA one over the wide block).  Per round the other CTAs hand their
// candidates to the owner and the owner hands back its decision through mbarriers
// with bounded waits; after a pivot they shift their copies over the re-hung
// subtree's node list (or copy all potentials when the move took the full pass).
template <int CL>
__global__ void __launch_bounds__(LOT_BT, 1) lot_simplex_kernel(const __grid_constant__ LotArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int m = A.m, V = 2 * m + 1, R = 2 * m;
    long long* word = reinterpret_cast<long long*>(dsm);                  // [V] potential + subtree size
    double* flow = reinterpret_cast<double*>(word + V);                   // [V] flow on the parent arc
    unsigned short* pu = reinterpret_cast<unsigned short*>(flow + V);     // [V] 2 parent + up
    unsigned short* pos = pu + V;                                         // [V] preorder position
    unsigned short* chain = pos + V;                                      // [V] a pivot's reversed path
    __shared__ double s_v[LOT_BW + 1];
    __shared__ long long s_q[LOT_BW + 1];
    __shared__ int s_i[LOT_BW + 1];
    __shared__ int s_err;
    __shared__ LotMove s_mv;
    __shared__ unsigned s_cpk[LOT_CPK];
    __shared__ int s_cnt;
    // cluster hand-offs (CL > 1)
    __shared__ __align__(8) unsigned long long mb_cand, mb_go;
    __shared__ long long s_cv[CL > 1 ? CL : 1];
    __shared__ int s_ce[CL > 1 ? CL : 1];
    __shared__ long long s_best;
    __shared__ int s_be, s_dec, s_flag;
    __shared__ float s_gmax;
    __shared__ int s_bad;

    const int rank = CL > 1 ? (int)lot_rank() : 0;
    const int p = blockIdx.x / CL, tid = threadIdx.x;
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
    {
        // the cost bound over this CTA's share of the instance's costs (all of them when CL = 1)
        const long long e0 = mm * rank / CL, e1 = mm * (rank + 1) / CL;
        for (long long e = e0 + tid; e < e1; e += LOT_BT) {
            const float c = fabsf(G[e]);
            bad |= !(c < INFINITY);
            gmax = fmaxf(gmax, c);
        }
    }
    bad = __syncthreads_or(bad);
    sa = lot_sum(sa, s_v);
    sb = lot_sum(sb, s_v);
    gmax = warp_max(gmax);
    __syncthreads();
    if ((tid & 31) == 0) s_v[tid >> 5] = gmax;
    __syncthreads();
    for (int k = 0; k < LOT_BW; ++k) gmax = fmaxf(gmax, (float)s_v[k]);
    if constexpr (CL > 1) {
        if (tid == 0) {
            s_gmax = gmax;
            s_bad = bad;
            mbar_init(&mb_cand, CL - 1);
            mbar_init(&mb_go, 1);
            fence_mbar_init();
        }
        lot_cluster_sync();   // every CTA's share and barriers are ready
        if (tid == 0) {
            float g = 0.f;
            int bd = 0;
            for (int r = 0; r < CL; ++r) {
                g = fmaxf(g, __int_as_float(lot_ld_remote32(lot_mapa(&s_gmax, (unsigned)r))));
                bd |= lot_ld_remote32(lot_mapa(&s_bad, (unsigned)r));
            }
            s_v[LOT_BW] = g;
            s_flag = bd;
        }
        __syncthreads();
        gmax = (float)s_v[LOT_BW];
        bad = s_flag;
    }
    if (bad || !(sa > 0.0) || !(sb > 0.0)) {
        for (long long e = tid; e < mm; e += LOT_BT) S[e] = NAN;
        for (int i = tid; i < m; i += LOT_BT) {
            A.u[(size_t)p * m + i] = NAN;
            A.v[(size_t)p * m + i] = NAN;
        }
        if (tid == 0 && rank == 0) {
            res->iters = 0;
            res->status = OT_ERR_ARG;
            res->marg_l1 = res->marg_l1_col = res->marg_l2_col = -1.0;
            res->value = res->transport_cost = NAN;
            res->reserved[0] = NAN;
            res->reserved[1] = 6.0;   // variant code: reduced LOT
        }
        if constexpr (CL > 1) lot_cluster_sync();   // no CTA leaves while a peer may read it
        return;
    }
    const double ia = 1.0 / (sa * (double)A.N), ib = 1.0 / (sb * (double)A.N);
    // integer costs rint(G 2^k) with |g| < 2^30; |potentials| <= 2 M + V 2^30 < 2^46
    const int k2 = gmax > 0.f ? min(100, max(-120, 29 - ilogbf(gmax))) : 0;
    const float sc = ldexpf(1.0f, k2);
    const long long M = ((long long)ldexpf(gmax, k2) + 1) * (long long)V;

    // ---- strongly feasible artificial start: the root (position 0) and every other
    // node as a leaf below it, at position x + 1
    for (int x = tid; x < V; x += LOT_BT) {
        if (x == R) {
            pu[x] = (unsigned short)(2 * R);
            flow[x] = 0.0;
            word[x] = lot_pack(0, V);
            pos[x] = 0;
        } else if (x < m) {
            const double al = (double)a[x] * ia;
            const int up = al > 0.0 ? 1 : 0;   // a zero supply hangs below the root with zero flow
            pu[x] = (unsigned short)(2 * R + up);
            flow[x] = al;
            word[x] = lot_pack(up ? M : -M, 1);
            pos[x] = (unsigned short)(x + 1);
        } else {
            pu[x] = (unsigned short)(2 * R);   // root -> sink
            flow[x] = (double)b[x - m] * ib;
            word[x] = lot_pack(-M, 1);
            pos[x] = (unsigned short)(x + 1);
        }
    }
    if (tid == 0) s_err = 0;

    // ---- pivots
    const int npass = CL > 1 ? 1 : lot_price_passes(m);
    const int rb = max(1, min(m, npass * LOT_PRICE_ARCS / m));   // rows per CTA and pricing step (rb m <= npass LOT_PRICE_ARCS)
    const int qstep = LOT_BT / m, rstep = LOT_BT - (LOT_BT / m) * m;
    const bool vec4 = (m & 3) == 0 && ((uintptr_t)A.G & 15) == 0;   // rows of whole, aligned float4s
    long long piv = 0;
    int status = OT_OK;
    int cursor = 0, scanned = 0;
    unsigned round = 0;
    for (;; ++round) {
        __syncthreads();   // potentials and the previous reduction's results are settled
        // this step's rows [cursor, rend), CTA `rank` taking the part [r0, r1)
        const int rend = min(m, cursor + CL * rb);
        const int per = (rend - cursor + CL - 1) / CL;
        const int r0 = min(rend, cursor + rank * per), r1 = min(rend, r0 + per);
        long long best = 0x7fffffffffffffffll;
        int be = 0x7fffffff;
        const int e_end = r1 * m;
        if (r0 >= r1) {
            // no rows for this CTA in a short last step
        } else if (vec4) {
            // all NP passes' loads in one unrolled sequence (independent, so all in flight)
            if (npass == 4)
                lot_price_vec4<4>(G, word, m, r0 * m, e_end, sc, best, be);
            else if (npass == 2)
                lot_price_vec4<2>(G, word, m, r0 * m, e_end, sc, best, be);
            else
                lot_price_vec4<1>(G, word, m, r0 * m, e_end, sc, best, be);
        } else {
            for (int ps = 0; ps < npass; ++ps) {
                // arcs e = cursor m + ps LOT_PRICE_ARCS + tid + k LOT_BT below e_end: a pass's loads issued up front
                int e = r0 * m + ps * LOT_PRICE_ARCS + tid;
                int r = e / m, j = e - r * m;
#pragma unroll
                for (int k = 0; k < LOT_PPT; ++k) {
                    if (e < e_end) {
                        const long long rc =
                            (long long)__float2int_rn(G[e] * sc) - lot_pi(word[r]) + lot_pi(word[m + j]);
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
        }
        lot_argmin(best, be, s_q, s_i);
        bool timed_out = false;
        if constexpr (CL > 1) {
            // the parts' candidates meet at the owner
            if (rank != 0) {
                // (fault injection for tests: CTA 1 never hands in its first candidate, so the
                // owner's bounded wait expires and the solve reports OT_ERR_TIMEOUT)
                const bool withhold = (A.debug_flags & OT_DEBUG_WITHHOLD_ARRIVAL) && rank == 1 && round == 0;
                if (tid == 0 && !withhold) {
                    lot_st_remote64(lot_mapa(&s_cv[rank], 0u), best);
                    lot_st_remote32(lot_mapa(&s_ce[rank], 0u), be);
                    lot_remote_arrive(lot_mapa(&mb_cand, 0u));
                }
            } else {
                if (tid == 0) {
                    int to = !lot_wait_cluster(&mb_cand, round & 1u, A.timeout_ns);
                    long long bv = best;
                    int bi = be;
                    for (int r = 1; r < CL; ++r) {
                        const long long v = s_cv[r];
                        const int i = s_ce[r];
                        if (v < bv || (v == bv && i < bi)) {
                            bv = v;
                            bi = i;
                        }
                    }
                    s_best = bv;
                    s_be = bi;
                    s_flag = to;
                }
                __syncthreads();
                best = s_best;
                be = s_be;
                timed_out = s_flag != 0;
            }
        }
        scanned += rend - cursor;
        cursor = rend == m ? 0 : rend;
        // the owner decides: 0 no improving arc in this step, 1 pivot, 2 stop
        int dec = 0;
        if (rank == 0) {
            if (timed_out) {
                status = OT_ERR_TIMEOUT;
                dec = 2;
            } else if (best >= 0) {
                dec = scanned >= m ? 2 : 0;   // a full pass found no improving arc: optimal
            } else if (piv >= A.max_pivots) {
                status = OT_ERR_NOT_CONVERGED;
                dec = 2;
            } else {
                dec = 1;
                scanned = 0;
            }
        }
        if (CL > 1 && rank != 0) {
            // the owner's decision, and after a pivot the new potentials.  Thread 0 alone reads
            // the decision and the move's fields from the owner (one round trip, and no
            // thousand-fold requests at the owner's shared memory); the list of T's nodes is read
            // in 4-byte words of two entries (the path buffer starts at byte 20 (2m + 1), a
            // multiple of 4 but not of 8, and has 16 spare bytes after it).
            if (tid == 0) {
                int d = 2;
                if (lot_wait_cluster(&mb_go, round & 1u, A.timeout_ns)) {
                    d = lot_ld_remote32(lot_mapa(&s_dec, 0u));
                    if (d == 1) {
                        const unsigned mva = lot_mapa(&s_mv, 0u);
                        const int k = lot_ld_remote32(mva + offsetof(LotMove, k));
                        const int sz = lot_ld_remote32(mva + offsetof(LotMove, s));
                        const int lbase = lot_ld_remote32(mva + offsetof(LotMove, lbase));
                        const int lcap = lot_ld_remote32(mva + offsetof(LotMove, lcap));
                        const long long sig = lot_ld_remote64(mva + offsetof(LotMove, sigma));
                        const int cnt = lot_ld_remote32(lot_mapa(&s_cnt, 0u));
                        s_mv.sigma = sig;
                        s_mv.lbase = lbase;
                        // list length, or -1: the move took the full pass, copy every potential
                        s_mv.k = (k <= LOT_CPK && sz <= lcap) ? min(cnt, lcap) : -1;
                    }
                }
                s_flag = d;
            }
            __syncthreads();
            dec = s_flag;
            if (dec == 1) {
                const long long sig = s_mv.sigma;
                const int nT = s_mv.k, lbase = s_mv.lbase;
                if (nT >= 0) {
                    // entries [lbase, lbase + nT) of the owner's path buffer, by 4-byte words
                    const int w0 = lbase >> 1, w1 = (lbase + nT + 1) >> 1;
                    const unsigned ca = lot_mapa(chain, 0u);
                    for (int wi = w0 + tid; wi < w1; wi += LOT_BT) {
                        const unsigned v = (unsigned)lot_ld_remote32(ca + 4u * (unsigned)wi);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int i = 2 * wi + h;
                            const int x = (int)((v >> (16 * h)) & 0xffffu);
                            if (i >= lbase && i < lbase + nT && x < V) word[x] += sig * (1ll << LOT_SB);
                        }
                    }
                } else {
                    const unsigned wa = lot_mapa(word, 0u);
                    for (int x = tid; x < V; x += LOT_BT) word[x] = lot_ld_remote64(wa + 8u * (unsigned)x);
                }
            }
            if (dec == 2) break;
            continue;
        }
        // the owner (or the only CTA)
        auto release = [&](int d) {
            if constexpr (CL > 1) {
                if (tid == 0) s_dec = d;
                __syncthreads();   // the decision, the move and T's list are written
                if (tid == 0) {
                    asm volatile("fence.acq_rel.cluster;" ::: "memory");
                    for (int r = 1; r < CL; ++r) lot_remote_arrive(lot_mapa(&mb_go, (unsigned)r));
                }
            }
        };
        if (dec != 1) {
            release(dec);
            if (dec == 2) break;
            continue;
        }
        {
            // the next pricing block's costs into L2 while the pivot runs
            const size_t b0 = (size_t)cursor * m * 4, b1 = (size_t)min(m, cursor + rb) * m * 4;
            for (size_t off = b0 + (size_t)tid * 128; off < b1; off += (size_t)LOT_BT * 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)G + off));
        }
        if (tid < 32) {
            const int st = lot_pivot_warp(be, best, m, pu, pos, word, flow, chain, s_cpk, &s_mv);
            if (tid == 0) {
                s_err = st;
                s_cnt = 0;
            }
        }
        __syncthreads();
        if (s_err != OT_OK) {
            status = s_err;
            release(2);
            break;
        }
        ++piv;
        // T's potentials, every moved position and the reversed path's sizes
        const LotMove mv = s_mv;
        if (mv.k <= LOT_CPK && mv.s <= mv.lcap) {
            // the path's ranges are all packed, so no node's update reads another's:
            // nodes between T and its new place move at once; T's nodes are listed in
            // the free part of the path buffer (one append per warp), then updated
            unsigned short* list = chain + mv.lbase;
            for (int k = 0; k < LOT_NPT; ++k) {
                const int x = tid + k * LOT_BT;
                const int xp = x < V ? pos[x] : -1;
                const bool inT = xp >= mv.a0 && xp < mv.a0 + mv.s;
                if (x < V && !inT) {
                    if (mv.P < mv.a0) {
                        if (xp > mv.P && xp < mv.a0) pos[x] = (unsigned short)(xp + mv.s);
                    } else if (xp >= mv.a0 + mv.s && xp <= mv.P) {
                        pos[x] = (unsigned short)(xp - mv.s);
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, inT);
                if (ball) {
                    int base = 0;
                    if ((tid & 31) == 0) base = atomicAdd(&s_cnt, __popc(ball));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const int slot = base + __popc(ball & ((1u << (tid & 31)) - 1u));
                    if (inT && slot < mv.lcap) list[slot] = (unsigned short)x;   // s slots fit; a corrupt tree cannot overflow
                }
            }
            __syncthreads();
            const int nT = min(s_cnt, mv.lcap);   // == mv.s in a consistent tree
            for (int i = tid; i < nT; i += LOT_BT) {
                const int x = list[i];
                const unsigned r = lot_move_node(x, V, mv, pos, word, chain, s_cpk);
                pos[x] = (unsigned short)(r & 0x3fffu);
                long long w = word[x] + mv.sigma * (1ll << LOT_SB);
                if (r & 0x8000u) w += (long long)(r >> 16) - lot_size(w);
                word[x] = w;
            }
        } else {
            // all reads, a barrier, then all writes
            unsigned nx[LOT_NPT];
#pragma unroll
            for (int k = 0; k < LOT_NPT; ++k) {
                const int x = tid + k * LOT_BT;
                if (x < V) nx[k] = lot_move_node(x, V, mv, pos, word, chain, s_cpk);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < LOT_NPT; ++k) {
                const int x = tid + k * LOT_BT;
                if (x < V) {
                    pos[x] = (unsigned short)(nx[k] & 0x3fffu);
                    if (nx[k] & 0x4000u) {
                        long long w = word[x] + mv.sigma * (1ll << LOT_SB);
                        if (nx[k] & 0x8000u) w += (long long)(nx[k] >> 16) - lot_size(w);
                        word[x] = w;
                    }
                }
            }
        }
        release(1);
    }
    __syncthreads();
    if (rank != 0) {
        if constexpr (CL > 1) lot_cluster_sync();
        return;
    }
    // every potential against its parent arc: a wrong incremental update shows here
    {
        int bad_tree = 0;
        for (int x = tid; x < V; x += LOT_BT) {
            if (x == R) {
                bad_tree |= lot_pi(word[x]) != 0;
                continue;
            }
            const int y = pu[x] >> 1;
            const long long c = y == R ? M : (long long)__float2int_rn(G[lot_arc(x, y, m)] * sc);
            bad_tree |= lot_pi(word[x]) != lot_pi(word[y]) + ((pu[x] & 1) ? c : -c);
        }
        if (__syncthreads_or(bad_tree) && status == OT_OK) status = OT_ERR_NONFINITE;
    }

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
    if constexpr (CL > 1) lot_cluster_sync();   // the peers no longer read this CTA
}

size_t lot_smem_bytes(int m) { return (size_t)22 * (2 * (size_t)m + 1) + 16; }
static_assert(2 * (2 * LOT_MAXM + 1) < 0xffff, "parent and direction fit 16 bits");
static_assert(2 * LOT_MAXM + 1 < (1 << LOT_SB), "subtree sizes fit their 14-bit field");

}  // namespace cyc

using namespace cyc;

static size_t lot_a256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int CL>
static cudaError_t lot_prepare(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(lot_simplex_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

static void lot_cfg(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int CL, int count, size_t smem,
                    cudaStream_t st) {
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(count * CL), 1, 1);
    cfg.blockDim = dim3(LOT_BT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

// How many clusters of c CTAs (one instance each) can be resident at once.
static bool lot_clusters_resident(int c, size_t smem, int* n) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    lot_cfg(cfg, attr, c, 1, smem, 0);
    cudaError_t e;
    switch (c) {
        case 8: e = lot_prepare<8>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(n, lot_simplex_kernel<8>, &cfg); break;
        case 4: e = lot_prepare<4>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(n, lot_simplex_kernel<4>, &cfg); break;
        case 2: e = lot_prepare<2>(smem); if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(n, lot_simplex_kernel<2>, &cfg); break;
        default: return false;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();   // an unsupported cluster shape only rules that size out
        *n = 0;
    }
    return true;
}

static int lot_launch(int CL, int count, size_t smem, const LotArgs& A, cudaStream_t st) {
    if (CL == 1) {
        if (lot_prepare<1>(smem) != cudaSuccess) return OT_ERR_CUDA;
        lot_simplex_kernel<1><<<count, LOT_BT, smem, st>>>(A);
        return cudaGetLastError() == cudaSuccess ? OT_OK : OT_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    lot_cfg(cfg, attr, CL, count, smem, st);
    cudaError_t e;
    switch (CL) {
        case 8: e = cudaLaunchKernelEx(&cfg, lot_simplex_kernel<8>, A); break;
        case 4: e = cudaLaunchKernelEx(&cfg, lot_simplex_kernel<4>, A); break;
        case 2: e = cudaLaunchKernelEx(&cfg, lot_simplex_kernel<2>, A); break;
        default: return OT_ERR_CUDA;
    }
    return e == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

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
    A.timeout_ns = opt->timeout_ns ? opt->timeout_ns : 10000000000ull;
    A.debug_flags = opt->debug_flags;
    const size_t smem = lot_smem_bytes(m);
    // CTAs per instance: from m = LOT_CLUSTER_MIN_M (below it a pivot is cheaper than the
    // hand-offs between CTAs), the largest of 8, 4, 2 for which every CTA prices a full
    // block (CL LOT_PRICE_ARCS <= m^2) and all `count` clusters are resident at once; else one
    const int cls[3] = {8, 4, 2};
    int CL = 1;
    if (!(opt->debug_flags & OT_DEBUG_NO_CLUSTER) && m >= LOT_CLUSTER_MIN_M) {
        for (int c : cls) {
            if ((long long)c * LOT_PRICE_ARCS > (long long)m * m) continue;
            int ncl = 0;
            if (!lot_clusters_resident(c, smem, &ncl)) return OT_ERR_CUDA;
            if (ncl >= count) {
                CL = c;
                break;
            }
        }
    }
    return lot_launch(CL, count, smem, A, (cudaStream_t)stream);
}
