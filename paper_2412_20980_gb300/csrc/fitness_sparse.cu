// Sparse fitness: work proportional to what a member's deletion disturbs,
// for graphs whose labels do not fit in shared memory (Section III-C, Eq. 13;
// PC(G) and MCN of Table "Whole").
//
// The upload's BFS forest numbers every component from its top hub, so a
// node's tree parent is its lowest-numbered neighbour and a node's children
// carry consecutive numbers.  Deleting a member's set D cuts each touched
// component's tree into pieces: the root's piece (root live) and one piece
// below every live child of a deleted node (a "top").  Per member:
//  1. deletion bitmap in shared memory; the distinct deleted nodes listed;
//     each touched component counts its deleted nodes;
//  2. every top re-picks its first live lower-numbered neighbour q (none: the
//     top is a terminal of its own) and hops to the first top or tree root
//     met walking up the tree from q.  Hops strictly decrease, so following
//     them ends at a terminal (a live tree root or a top that re-picked
//     nothing), and the pieces whose chains end at one terminal are joined;
//  3. terminals form classes (union-find): every top chained to a top that
//     re-picked nothing unites that terminal's class with the terminals of
//     its first live neighbours outside its piece (neighbour sampling: after
//     the top hub is deleted, thousands of its children re-pick nothing and
//     would otherwise each list a whole subtree); per touched component the
//     class of one reference terminal becomes R: the root if it is live,
//     else the terminal whose chained tops carry the most subtree nodes (any
//     choice is exact; this one keeps the lists short);
//  4. the pieces of the classes other than R are listed, grown down the tree
//     from their tops; every listed node's arcs unite classes (an arc to an
//     unlisted live node joins R, since every unlisted live node of the
//     component lies in R's class);
//  5. classes apart from R count their listed nodes; R's set is the
//     component's size less its deleted nodes less those classes, so
//     PC = PC(G) - sum over touched components of C(size, 2) + the new terms
//     (MCN: the largest of those and of the largest untouched component).
// Nothing inside a piece that stays joined is read, and nothing is done per
// node of the graph.  One CTA per member at a time, persistent over a work
// queue; its per-node state (hops, classes, counts, per-component sums) lives
// in the CTA's own slice of global scratch, which it clears after every
// member (entries start as -1 / 0 when the scratch is allocated).
#include <climits>

#include "gapa_internal.cuh"
#include "tree16.cuh"

namespace {

using gapa_dev::bm_test;
using gapa_dev::objective_add;
using gapa_dev::Team;
using gapa_dev::team_sum_ll;
using gapa_dev::tree16l_owner;
using gapa_dev::tree16l_scan;

constexpr int kSpBlock = 1024;
constexpr int kSpLinkScan = 4;              // adjacency entries a top samples for links
constexpr int kSpInFlight = 4;              // tops per thread resolved together in the re-pick pass
constexpr int kSpForestShift = 28;          // order entry: member | forest << 28
constexpr int kSpMemberMask = (1 << kSpForestShift) - 1;

template <typename Col>
struct SpGraph {
    int n;
    const int* perm;      // original id -> BFS number
    const int* tparent;   // tree parent (roots: itself)
    const int2* palt;     // (tree parent, second lower-numbered neighbour or -1)
    const int* lo_ptr;    // lower-numbered neighbours, ascending (CSR)
    const int* lo_col;
    const int* fptr;      // full adjacency in BFS numbers (CSR)
    const Col* fcol;
    const int2* kids;     // (first child, number of children)
    const int* croot;     // root of the node's component tree (-1: a single-node component)
    const int* csize;     // size of the component, at its root
    const int* sub;       // subtree size
    const int* bysize;    // component roots by decreasing size (MCN)
    int ncomp;
    int giant;            // root of the largest component
    long long pc0;        // sum over components of C(size, 2)
    int objective;        // 0: PC, 1: MCN
};

// The forests of one graph (forest 0 on G; 1, 2, 3 on G without the edges of the top hub, of the two
// top hubs, of the second hub; an absent forest has kids == nullptr).
template <typename Col>
struct SpGraphs {
    SpGraph<Col> f[kSpForests];
};

// One CTA's slice of the scratch (n entries each).  Reads go through L2 only
// (__ldcg; a slice moves between SMs from one launch to the next, and within
// a phase the union-find entries change under other threads' atomics); what a
// phase writes, later phases read after a barrier.
struct SpSlot {
    int* hop;                  // live tops: hop, then terminal; -1 elsewhere
    int* cls;                  // terminals: class link (terminal + 1; 0 = R); listed nodes: their class; -1 elsewhere
    unsigned* cnt;             // terminals: chained subtree weight, then class size; 0 elsewhere
    int* list;                 // listed nodes
    int* tl;                   // live tops
    int* th;                   // hop of the live top at the same position of tl (then its terminal)
    int* cl;                   // touched components (roots), single-node components excepted
    unsigned long long* cacc;  // component roots: deleted << 32 | nodes apart from R; 0 elsewhere
    unsigned long long* best;  // component roots whose root is deleted: weight << 32 | ~terminal
};

__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ldcg(const unsigned* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg(const unsigned long long* p) { return __ldcg(p); }

__host__ __device__ __forceinline__ size_t sp_bitmap_bytes(int n) { return ((((size_t)n + 31) >> 5) * 4 + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ size_t sp_smem_bytes(int n, int k) {
    return sp_bitmap_bytes(n) + (((size_t)2 * k + 1) * 4 + 15) / 16 * 16 + (size_t)3 * kSpBlock * 4;
}

// Class of value a (terminal + 1; 0 = R): the root's value r, with the links
// on the way that still lie below r pointed at it.  Links always point to
// smaller values and only ever move to ancestors, so a link above r (another
// thread compressed past r after r was hooked) ends the compression: every
// node written lies strictly between a and r on a's path, and r is its
// ancestor.
__device__ __forceinline__ int sp_find(int* cls, int a) {
    int r = a;
    while (r != 0) {
        const int p = ldcg(&cls[r - 1]);
        if (p == r) break;
        r = p;
    }
    while (a > r) {
        const int p = ldcg(&cls[a - 1]);
        if (p <= r) break;
        cls[a - 1] = r;
        a = p;
    }
    return r;
}

// Union of two classes: the larger value hooks under the smaller, so R (0) is never hooked.
__device__ __forceinline__ void sp_unite(int* cls, int a, int b) {
    a = sp_find(cls, a);
    b = sp_find(cls, b);
    while (a != b) {
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(&cls[a - 1], a, b);
        if (old == a) return;
        a = sp_find(cls, old);
        b = sp_find(cls, b);
    }
}

// Warp-aggregated append of v (where want) to a list; called by all lanes.  Returns v's
// position (-1 where not wanted).
__device__ __forceinline__ int sp_append(bool want, int v, int lane, int* count, int* list) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return -1;
    int first = 0;
    if (lane == 0) first = atomicAdd(count, __popc(m));
    first = __shfl_sync(0xffffffffu, first, 0);
    const int at = first + __popc(m & ((1u << lane) - 1));
    if (want) list[at] = v;
    return want ? at : -1;
}

// The terminal of live node w's piece: walk up to the first top (its terminal) or tree root.
template <typename Col>
__device__ __forceinline__ int sp_terminal_of(const SpGraph<Col>& g, const unsigned* dead, const int* hop, int w,
                                              int p) {
    while (true) {
        if (p == w) return w;
        if (bm_test(dead, p)) return ldcg(&hop[w]);
        w = p;
        p = __ldg(&g.tparent[w]);
    }
}

// Forest of every member and its cost estimate: a member that deletes the top hub (h0) and / or the
// second hub (h1) is evaluated on the forest of G without those hubs' edges, where deleting them cuts
// nothing (forest 2: both, 1: h0, 3: h1, 0: neither; an absent forest falls back to forest 0); the
// estimate is the sum over its genes of (children + 1) in that forest, read through a table by
// original node id.
struct SpCostArgs {
    const int* cost[kSpForests];  // null: forest absent
    int hub0, hub1;
};

__global__ void __launch_bounds__(128) sp_cost_kernel(const int* __restrict__ pop, int k, int n, SpCostArgs a,
                                                      unsigned* __restrict__ est, int* __restrict__ forest) {
    __shared__ unsigned long long part[4];
    __shared__ int s_f;
    const int m = blockIdx.x, t = threadIdx.x;
    const int* genes = pop + (size_t)m * k;
    int h0 = 0, h1 = 0;
    for (int j = t; j < k; j += 128) {
        const int d = __ldg(&genes[j]);
        h0 |= d == a.hub0;
        h1 |= d == a.hub1;
    }
    h0 = __syncthreads_or(h0);
    h1 = __syncthreads_or(h1);
    if (t == 0) {
        int f = 0;
        if (h0 && h1 && a.cost[2]) f = 2;
        else if (h0 && a.cost[1]) f = 1;
        else if (h1 && a.cost[3]) f = 3;
        s_f = f;
    }
    __syncthreads();
    const int* cost = a.cost[s_f];
    unsigned long long c = 0;
    for (int j = t; j < k; j += 128) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n) c += (unsigned)__ldg(&cost[d]);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((t & 31) == 0) part[t >> 5] = c;
    __syncthreads();
    if (t == 0) {
        const unsigned long long tot = part[0] + part[1] + part[2] + part[3];
        est[m] = tot > 0xFFFFFFFFull ? 0xFFFFFFFFu : (unsigned)tot;
        forest[m] = s_f;
    }
}

// Members by decreasing estimate (a counting sort on the estimate's bit length; one CTA), so that
// the persistent CTAs take the costliest members first and none starts late; entry = member |
// forest << 28.
__global__ void __launch_bounds__(1024) sp_order_kernel(const unsigned* __restrict__ est,
                                                        const int* __restrict__ forest, int s,
                                                        int* __restrict__ order) {
    __shared__ int cnt[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < s; m += blockDim.x) atomicAdd(&cnt[__clz(est[m])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < 33; ++c) {
            const int x = cnt[c];
            cnt[c] = acc;
            acc += x;
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < s; m += blockDim.x)
        order[atomicAdd(&cnt[__clz(est[m])], 1)] = m | (forest[m] << kSpForestShift);
}

template <typename Col>
__global__ void __launch_bounds__(kSpBlock, 1) cc_sparse_kernel(const __grid_constant__ SpGraphs<Col> gs, SpSlot base,
                                                               size_t stride, const int* __restrict__ pop, int s,
                                                               int k, long long* __restrict__ fit, int* head,
                                                               int* status, const int* __restrict__ order) {
    extern __shared__ __align__(16) unsigned char sp_smem[];
    __shared__ long long red[32];
    __shared__ int s_member, s_forest, s_nd, s_nt, s_nterm, s_ncl, s_gdel, s_nlist;
    const Team tm{(int)threadIdx.x, (int)blockDim.x, 0};
    const int tid = tm.tid, T = tm.T, lane = tid & 31, n = gs.f[0].n;
    const int words = (n + 31) >> 5;
    unsigned* dead = reinterpret_cast<unsigned*>(sp_smem);
    int* D = reinterpret_cast<int*>(sp_smem + sp_bitmap_bytes(n));
    int* Doff = D + k;  // nd + 1 entries
    int* s_off = reinterpret_cast<int*>(sp_smem + sp_smem_bytes(n, k) - (size_t)3 * kSpBlock * 4);
    int* s_first = s_off + T;
    int* s_val = s_first + T;
    int* ws = reinterpret_cast<int*>(red);
    const size_t o = (size_t)blockIdx.x * stride;
    int* const hop = base.hop + o;
    int* const cls = base.cls + o;
    unsigned* const cnt = base.cnt + o;
    int* const list = base.list + o;
    int* const tl = base.tl + o;
    int* const th = base.th + o;
    int* const cl = base.cl + o;
    unsigned long long* const cacc = base.cacc + o;
    unsigned long long* const best = base.best + o;
    constexpr int F = kSpInFlight;

    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(head, 1);
            const int e = q < s ? order[q] : q;
            s_member = q < s ? (e & kSpMemberMask) : q;
            s_forest = q < s ? (e >> kSpForestShift) : 0;
            s_nd = 0;
            s_nt = 0;
            s_nterm = 0;
            s_ncl = 0;
            s_gdel = 0;
            s_nlist = 0;
        }
        for (int w = tid; w < words; w += T) dead[w] = 0u;
        tm.sync();
        const int m = s_member;
        if (m >= s) break;
        const SpGraph<Col>& g = gs.f[s_forest];  // this member's forest
        const int* genes = pop + (size_t)m * k;

        // 1. perturbation P^(A, p) of Eq. 13 in BFS numbering; distinct deleted nodes listed
        for (int j0 = 0; j0 < k; j0 += F * T) {
            int b[F];
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int j = j0 + u * T + tid;
                b[u] = -1;
                if (j < k) {
                    const int d = __ldg(&genes[j]);
                    if ((unsigned)d < (unsigned)n) b[u] = d;
                    else atomicOr(status, GAPA_DEV_BAD_GENE);
                }
            }
#pragma unroll
            for (int u = 0; u < F; ++u)
                if (b[u] >= 0) b[u] = __ldg(&g.perm[b[u]]);
#pragma unroll
            for (int u = 0; u < F; ++u) {
                bool fresh = false;
                if (b[u] >= 0) {
                    const unsigned bit = 1u << (b[u] & 31);
                    fresh = !(atomicOr(&dead[b[u] >> 5], bit) & bit);
                }
                sp_append(fresh, b[u], lane, &s_nd, D);
            }
        }
        tm.sync();
        const int nd = s_nd;
        // children per deleted node -> offsets of the tops; deleted nodes per touched component
        int ntops;
        {
            const int per = (nd + T - 1) / T, lo = min(nd, tid * per), hi = min(nd, lo + per);
            int sum = 0;
#pragma unroll 4
            for (int i = lo; i < hi; ++i) sum += __ldg(&g.kids[D[i]].y);
            int at = tree16l_scan(tm, sum, ws, &ntops);
            for (int i = lo; i < hi; ++i) {
                Doff[i] = at;
                at += __ldg(&g.kids[D[i]].y);
            }
            if (tid == 0) Doff[nd] = ntops;
        }
        {
            int gdel = 0;  // deletions in the largest component, summed in shared memory
            for (int i0 = tid & ~31; i0 < nd; i0 += T) {
                const int i = i0 + lane;
                int c = i < nd ? __ldg(&g.croot[D[i]]) : -1;  // -1: a single-node component
                if (c >= 0 && c == g.giant) {
                    ++gdel;
                    c = -1;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, c);
                if (c >= 0 && lane == __ffs(peers) - 1) {
                    const unsigned long long old = atomicAdd(&cacc[c], (unsigned long long)__popc(peers) << 32);
                    if (old == 0ull) {
                        cl[atomicAdd(&s_ncl, 1)] = c;
                        if (!bm_test(dead, c)) cls[c] = c + 1;  // a live tree root is a terminal
                    }
                }
            }
            gdel = __reduce_add_sync(0xffffffffu, gdel);
            if (lane == 0 && gdel) atomicAdd(&s_gdel, gdel);
        }
        tm.sync();
        if (tid == 0 && s_gdel) {
            const int c = g.giant;
            cacc[c] = (unsigned long long)s_gdel << 32;
            cl[s_ncl++] = c;
            if (!bm_test(dead, c)) cls[c] = c + 1;
        }

        // 2. re-pick and hop of every top; the live tops are also listed compactly (tl) for the
        // passes below.  F tops per thread are resolved together (their loads overlap).
        for (int base_i = 0; base_i < ntops; base_i += F * T) {
            int t[F], q[F], y[F];
            int2 pa[F];
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int i = base_i + u * T + tid;
                t[u] = -1;
                if (i < ntops) {
                    const int ow = tree16l_owner(Doff, nd, i);
                    t[u] = __ldg(&g.kids[D[ow]].x) + i - Doff[ow];
                }
            }
#pragma unroll
            for (int u = 0; u < F; ++u) {
                if (t[u] >= 0 && bm_test(dead, t[u])) t[u] = -1;  // a deleted child is no top
                pa[u] = t[u] >= 0 ? __ldg(&g.palt[t[u]]) : make_int2(0, -1);
            }
#pragma unroll
            for (int u = 0; u < F; ++u) {
                q[u] = t[u];
                if (t[u] < 0 || pa[u].y < 0) continue;
                if (!bm_test(dead, pa[u].y)) {
                    q[u] = pa[u].y;
                } else {
                    const int end = __ldg(&g.lo_ptr[t[u] + 1]);
                    for (int e = __ldg(&g.lo_ptr[t[u]]) + 2; e < end; ++e) {
                        const int w = __ldg(&g.lo_col[e]);
                        if (!bm_test(dead, w)) {
                            q[u] = w;
                            break;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < F; ++u) y[u] = q[u] != t[u] ? __ldg(&g.tparent[q[u]]) : -1;
#pragma unroll
            for (int u = 0; u < F; ++u) {
                if (t[u] < 0) continue;
                int x = q[u];
                if (q[u] != t[u]) {
                    int p = y[u];  // walk up to the first top or tree root
                    while (p != x && !bm_test(dead, p)) {
                        x = p;
                        p = __ldg(&g.tparent[x]);
                    }
                }
                hop[t[u]] = x;
                y[u] = x;
            }
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int at = sp_append(t[u] >= 0, t[u], lane, &s_nt, tl);
                if (at >= 0) th[at] = y[u];
            }
        }
        tm.sync();
        const int nt = s_nt;
        // terminal of every top: its hop chain followed (F tops per thread together, chains of a few
        // hops) and compressed; tops that re-picked nothing start their class and are listed densely
        // (in `list`, free until the listing); subtree weight of the chained tops at terminals whose
        // component root is deleted
        for (int base_j = 0; base_j < nt; base_j += F * T) {
            int t[F], x[F];
            bool act[F];
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int j = base_j + u * T + tid;
                t[u] = j < nt ? ldcg(&tl[j]) : -1;
                x[u] = j < nt ? ldcg(&th[j]) : -1;
            }
            bool any = false;
#pragma unroll
            for (int u = 0; u < F; ++u) {
                act[u] = t[u] >= 0 && x[u] != t[u];
                any |= act[u];
            }
            while (any) {
                int h[F];
#pragma unroll
                for (int u = 0; u < F; ++u) h[u] = act[u] ? ldcg(&hop[x[u]]) : 0;
                any = false;
#pragma unroll
                for (int u = 0; u < F; ++u) {
                    if (!act[u]) continue;
                    if (h[u] == -1 || h[u] == x[u]) {  // a tree root or a top that re-picked nothing
                        act[u] = false;
                    } else {
                        x[u] = h[u];
                        any = true;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < F; ++u) {
                int key = -1;
                unsigned wgt = 0;
                const bool term = t[u] >= 0 && x[u] == t[u];
                if (term) {
                    cls[t[u]] = t[u] + 1;
                } else if (t[u] >= 0) {
                    hop[t[u]] = x[u];
                    th[base_j + u * T + tid] = x[u];
                }
                if (t[u] >= 0) {
                    // x is a top that re-picked nothing, or a live tree root (never weighed)
                    const int cx = __ldg(&g.croot[x[u]]);
                    if (cx >= 0 && bm_test(dead, cx)) {
                        key = x[u];
                        wgt = (unsigned)__ldg(&g.sub[t[u]]);
                    }
                }
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const unsigned tot = __reduce_add_sync(peers, wgt);
                if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], tot);
                sp_append(term, t[u], lane, &s_nterm, list);
            }
        }
        tm.sync();
        const int nterm = s_nterm;

        // sampled links: a terminal unites its class with the classes of its first live neighbours
        // outside its own piece (at most two)
        for (int j = tid; j < nterm; j += T) {
            const int t = ldcg(&list[j]);
            const int beg = __ldg(&g.fptr[t]);
            const int cntw = min(__ldg(&g.fptr[t + 1]) - beg, kSpLinkScan);
            int w[kSpLinkScan], pw[kSpLinkScan];
#pragma unroll
            for (int e = 0; e < kSpLinkScan; ++e) w[e] = e < cntw ? (int)__ldg(&g.fcol[beg + e]) : -1;
#pragma unroll
            for (int e = 0; e < kSpLinkScan; ++e) {
                if (w[e] >= 0 && bm_test(dead, w[e])) w[e] = -1;
                pw[e] = w[e] >= 0 ? __ldg(&g.tparent[w[e]]) : -1;
            }
            int links = 0;
#pragma unroll
            for (int e = 0; e < kSpLinkScan; ++e) {
                if (w[e] < 0 || pw[e] == t || links == 2) continue;
                const int b = sp_terminal_of(g, dead, hop, w[e], pw[e]);
                if (b == t) continue;  // a neighbour chained to this terminal links nothing
                sp_unite(cls, t + 1, b + 1);
                ++links;
            }
        }
        tm.sync();

        // 3. reference terminal of components whose root is deleted
        for (int j = tid; j < nterm; j += T) {
            const int t = ldcg(&list[j]);
            const int c = __ldg(&g.croot[t]);
            if (bm_test(dead, c))
                atomicMax(&best[c], ((unsigned long long)ldcg(&cnt[t]) << 32) | (unsigned long long)(~(unsigned)t));
        }
        tm.sync();
        // the reference's class becomes R (one thread per touched component; classes never span two)
        const int ncl = s_ncl;
        for (int i = tid; i < ncl; i += T) {
            const int c = ldcg(&cl[i]);
            int r;
            if (!bm_test(dead, c)) {
                r = c + 1;
            } else {
                const unsigned long long bk = ldcg(&best[c]);
                if (bk == 0ull) continue;  // no live node left in the component
                r = (int)(~(unsigned)(bk & 0xFFFFFFFFull)) + 1;
            }
            r = sp_find(cls, r);
            while (r != 0) {
                const int old = atomicCAS(&cls[r - 1], r, 0);
                if (old == r) break;
                r = sp_find(cls, old);
            }
        }
        tm.sync();
        // every terminal's and live root's link straight to its class root (0: R)
        for (int j = tid; j < nterm; j += T) sp_find(cls, ldcg(&list[j]) + 1);
        for (int i = tid; i < ncl; i += T) {
            const int c = ldcg(&cl[i]);
            if (!bm_test(dead, c)) sp_find(cls, c + 1);
        }
        tm.sync();

        // 4. listing: tops whose class is not R, then their pieces down the tree
        for (int base_j = 0; base_j < nt; base_j += F * T) {
            int t[F], x[F];
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int j = base_j + u * T + tid;
                t[u] = j < nt ? ldcg(&tl[j]) : -1;
                x[u] = j < nt ? ldcg(&th[j]) : -1;
            }
            int cx[F];
#pragma unroll
            for (int u = 0; u < F; ++u) cx[u] = t[u] >= 0 ? ldcg(&cls[x[u]]) : 0;
#pragma unroll
            for (int u = 0; u < F; ++u) {
                bool want = false;
                if (t[u] >= 0) {
                    if (x[u] == t[u]) cnt[t[u]] = 0u;  // the weight has served
                    if (cx[u] != 0) {
                        if (x[u] != t[u]) cls[t[u]] = x[u] + 1;  // a terminal keeps its class link
                        want = true;
                    }
                }
                sp_append(want, t[u], lane, &s_nlist, list);
            }
        }
        tm.sync();
        {
            int head_i = 0, tail = s_nlist;
            while (head_i < tail) {
                for (int u0 = head_i; u0 < tail; u0 += T) {
                    const int idx = u0 + tid;
                    int2 ch = make_int2(0, 0);
                    int cl = 0;
                    if (idx < tail) {
                        const int u = ldcg(&list[idx]);
                        ch = __ldg(&g.kids[u]);
                        cl = ldcg(&cls[u]);
                    }
                    int total;
                    const int off = tree16l_scan(tm, ch.y, ws, &total);
                    s_off[tid] = off;
                    s_first[tid] = ch.x;
                    s_val[tid] = cl;
                    tm.sync();
                    const int owners = min(T, tail - u0);
                    for (int i0 = tid & ~31; i0 < total; i0 += T) {
                        const int i = i0 + lane;
                        bool want = false;
                        int x = 0;
                        if (i < total) {
                            const int ow = tree16l_owner(s_off, owners, i);
                            x = s_first[ow] + i - s_off[ow];
                            if (!bm_test(dead, x)) {
                                cls[x] = s_val[ow];
                                want = true;
                            }
                        }
                        sp_append(want, x, lane, &s_nlist, list);
                    }
                    tm.sync();
                }
                head_i = tail;
                tail = s_nlist;
                tm.sync();  // every thread has read the length before the next round appends
            }
        }
        const int nl = s_nlist;

        // join along the listed nodes' arcs (a class already joined to R scans nothing)
        for (int v0 = 0; v0 < nl; v0 += T) {
            const int idx = v0 + tid;
            int v = 0, b = 0, d = 0;
            if (idx < nl) {
                v = ldcg(&list[idx]);
                if (sp_find(cls, ldcg(&cls[v])) != 0) {
                    b = __ldg(&g.fptr[v]);
                    d = __ldg(&g.fptr[v + 1]) - b;
                }
            }
            int total;
            const int off = tree16l_scan(tm, d, ws, &total);
            s_off[tid] = off;
            s_first[tid] = b;
            s_val[tid] = v;
            tm.sync();
            const int owners = min(T, nl - v0);
            for (int i = tid; i < total; i += T) {
                const int ow = tree16l_owner(s_off, owners, i);
                const int w = (int)__ldg(&g.fcol[s_first[ow] + i - s_off[ow]]);
                if (bm_test(dead, w)) continue;
                const int cv = ldcg(&cls[s_val[ow]]), cw = ldcg(&cls[w]);
                if (cw == -1) sp_unite(cls, cv, 0);
                else if (cw != cv) sp_unite(cls, cv, cw);
            }
            tm.sync();
        }

        // 5. sizes of the classes apart from R, and per component the nodes apart from R
        for (int i0 = tid & ~31; i0 < nl; i0 += T) {
            const int i = i0 + lane;
            int r = 0, c = -1;
            if (i < nl) {
                const int v = ldcg(&list[i]);
                r = sp_find(cls, ldcg(&cls[v]));
                if (r != 0) c = __ldg(&g.croot[v]);
            }
            const unsigned pr = __match_any_sync(0xffffffffu, r);
            if (r != 0 && lane == __ffs(pr) - 1) atomicAdd(&cnt[r - 1], (unsigned)__popc(pr));
            const unsigned pc = __match_any_sync(0xffffffffu, c);
            if (c >= 0 && lane == __ffs(pc) - 1) atomicAdd(&cacc[c], (unsigned long long)__popc(pc));
        }
        tm.sync();
        const bool mx = g.objective != 0;
        long long acc = 0;
        for (int i = tid; i < nl; i += T) {
            const int v = ldcg(&list[i]);
            if (ldcg(&cls[v]) == v + 1) acc = objective_add(acc, (long long)ldcg(&cnt[v]), g.objective);
        }
        for (int i = tid; i < ncl; i += T) {
            const int c = ldcg(&cl[i]);
            const unsigned long long a = ldcg(&cacc[c]);
            const long long cs = __ldg(&g.csize[c]);
            const long long rs = cs - (long long)(a >> 32) - (long long)(a & 0xFFFFFFFFull);
            if (mx) acc = rs > acc ? rs : acc;
            else acc += rs * (rs - 1) / 2 - cs * (cs - 1) / 2;
        }
        long long tot = team_sum_ll(tm, acc, red, mx);
        if (tid == 0) {
            if (mx) {
                // the largest untouched component
                for (int j = 0; j < g.ncomp; ++j) {
                    const int c = __ldg(&g.bysize[j]);
                    const bool touched = __ldg(&g.csize[c]) == 1 ? bm_test(dead, c) : ldcg(&cacc[c]) != 0ull;
                    if (!touched) {
                        const long long cs = __ldg(&g.csize[c]);
                        tot = cs > tot ? cs : tot;
                        break;
                    }
                }
                fit[m] = tot;
            } else {
                fit[m] = g.pc0 + tot;
            }
        }
        tm.sync();

        // clear what this member wrote
        for (int j0 = tid; j0 < nt; j0 += F * T) {
            int t[F];
#pragma unroll
            for (int u = 0; u < F; ++u) t[u] = j0 + u * T < nt ? ldcg(&tl[j0 + u * T]) : -1;
#pragma unroll
            for (int u = 0; u < F; ++u)
                if (t[u] >= 0) {
                    hop[t[u]] = -1;
                    cls[t[u]] = -1;
                }
        }
        for (int i0 = tid; i0 < nl; i0 += F * T) {
            int v[F];
#pragma unroll
            for (int u = 0; u < F; ++u) v[u] = i0 + u * T < nl ? ldcg(&list[i0 + u * T]) : -1;
#pragma unroll
            for (int u = 0; u < F; ++u)
                if (v[u] >= 0) {
                    cls[v[u]] = -1;
                    cnt[v[u]] = 0u;
                }
        }
        for (int i = tid; i < ncl; i += T) {
            const int c = ldcg(&cl[i]);
            cacc[c] = 0ull;
            best[c] = 0ull;
            cls[c] = -1;
        }
        tm.sync();
    }
}

template <typename Col>
SpGraph<Col> sp_graph(const gapa_ctx* c, const SparseForest& f, const Col* fcol) {
    SpGraph<Col> g;
    g.n = c->g.n;
    g.perm = f.perm;
    g.tparent = f.tparent;
    g.palt = f.palt;
    g.lo_ptr = f.lo_ptr;
    g.lo_col = f.lo_col;
    g.fptr = f.fptr;
    g.fcol = fcol;
    g.kids = f.kids;
    g.croot = f.croot;
    g.csize = f.csize;
    g.sub = f.sub;
    g.bysize = f.bysize;
    g.ncomp = f.ncomp;
    g.giant = f.giant;
    g.pc0 = f.pc0;
    g.objective = c->objective;
    return g;
}

template <typename Col>
SpGraphs<Col> sp_graphs(const gapa_ctx* c) {
    SpGraphs<Col> gs;
    for (int i = 0; i < kSpForests; ++i) {
        const SparseForest& f = c->g.spf[i];
        if constexpr (sizeof(Col) == 2) gs.f[i] = sp_graph<Col>(c, f, f.fcol16);
        else gs.f[i] = sp_graph<Col>(c, f, reinterpret_cast<const Col*>(f.fcol32));
    }
    return gs;
}

}  // namespace

bool gapa_sparse_fits(const gapa_ctx* c, int k) {
    return c->g.sp_nforests > 0 && c->sp_smem_max > 0 && sp_smem_bytes(c->g.n, k) <= c->sp_smem_max;
}

int gapa_sparse_init(gapa_ctx* c) {
    int rc = gapa_set_smem_limit((const void*)cc_sparse_kernel<int>, c->smem_optin, &c->sp_smem_max);
    size_t other = 0;
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_sparse_kernel<unsigned short>, c->smem_optin, &other);
    if (other < c->sp_smem_max) c->sp_smem_max = other;
    return rc;
}

// Scratch of the persistent CTAs: nine n-entry arrays per CTA (hops, classes,
// counts, listed nodes, live tops, their hops, touched components: int32;
// per-component sums and reference keys: int64), set to -1 / 0 once here and
// left that way by every member.
int gapa_sparse_prepare(gapa_ctx* c, int s) {
    const int n = c->g.n;
    const size_t stride = ((size_t)n + 63) & ~(size_t)63;
    // member order, estimates and forests (3 ints per member)
    if ((size_t)3 * std::max(s, 1) > c->sp_order_cap) {
        int rc = gapa_reserve((void**)&c->sp_order, &c->sp_order_cap, (size_t)3 * std::max(s, 1), sizeof(int));
        if (rc != GAPA_OK) return rc;
    }
    if (c->sp_scratch && c->sp_stride == stride) return GAPA_OK;  // (also inside a stream capture)
    const size_t smem = sp_smem_bytes(n, 0);
    int per_sm = 0;
    GAPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cc_sparse_kernel<int>, kSpBlock, smem));
    if (per_sm < 1) per_sm = 1;
    const int slots = c->num_sms * per_sm;
    const size_t bytes = (size_t)slots * stride * (7 * 4 + 2 * 8) + 64;
    cudaFree(c->sp_scratch);
    c->sp_scratch = nullptr;
    c->sp_scratch_cap = 0;
    if (cudaMalloc(&c->sp_scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "sparse fitness scratch of %zu bytes", bytes);
    }
    c->sp_scratch_cap = bytes;
    c->sp_stride = stride;
    c->sp_slots = slots;
    const size_t ints = (size_t)slots * stride;
    char* p = static_cast<char*>(c->sp_scratch);
    // hop, cls = -1; cnt, list, tl, th, cl = 0; cacc, best = 0; the queue head last
    GAPA_CUDA(cudaMemset(p, 0xFF, ints * 8));
    GAPA_CUDA(cudaMemset(p + ints * 8, 0, ints * 20 + ints * 16 + 64));
    GAPA_CUDA(cudaDeviceSynchronize());
    return GAPA_OK;
}

int gapa_launch_fitness_sparse(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                               int* kernels) {
    if (!gapa_sparse_fits(c, k)) return gapa_fail(GAPA_ERR_INVALID_ARG, "sparse fitness: shared memory too small");
    int rc = gapa_sparse_prepare(c, s);
    if (rc != GAPA_OK) return rc;
    const size_t ints = (size_t)c->sp_slots * c->sp_stride;
    char* p = static_cast<char*>(c->sp_scratch);
    SpSlot b;
    b.hop = reinterpret_cast<int*>(p);
    b.cls = reinterpret_cast<int*>(p + ints * 4);
    b.cnt = reinterpret_cast<unsigned*>(p + ints * 8);
    b.list = reinterpret_cast<int*>(p + ints * 12);
    b.tl = reinterpret_cast<int*>(p + ints * 16);
    b.th = reinterpret_cast<int*>(p + ints * 20);
    b.cl = reinterpret_cast<int*>(p + ints * 24);
    b.cacc = reinterpret_cast<unsigned long long*>(p + ints * 28);
    b.best = reinterpret_cast<unsigned long long*>(p + ints * 36);
    int* head = reinterpret_cast<int*>(p + ints * 44);
    GAPA_CUDA(cudaMemsetAsync(head, 0, sizeof(int), st));
    const size_t smem = sp_smem_bytes(c->g.n, k);
    const int grid = std::min(c->sp_slots, std::max(s, 1));
    // every member's forest and cost estimate, then the members costliest first
    unsigned* est = reinterpret_cast<unsigned*>(c->sp_order + s);
    int* forest = c->sp_order + 2 * (size_t)s;
    SpCostArgs ca;
    for (int i = 0; i < kSpForests; ++i) ca.cost[i] = c->g.spf[i].kids ? c->g.spf[i].cost : nullptr;
    ca.hub0 = c->g.sp_hub[0];
    ca.hub1 = c->g.sp_hub[1];
    sp_cost_kernel<<<s, 128, 0, st>>>(pop, k, c->g.n, ca, est, forest);
    sp_order_kernel<<<1, 1024, 0, st>>>(est, forest, s, c->sp_order);
    if (c->g.packed16)
        cc_sparse_kernel<unsigned short><<<grid, kSpBlock, smem, st>>>(sp_graphs<unsigned short>(c), b, c->sp_stride,
                                                                        pop, s, k, reinterpret_cast<long long*>(fit),
                                                                        head, c->status, c->sp_order);
    else
        cc_sparse_kernel<int><<<grid, kSpBlock, smem, st>>>(sp_graphs<int>(c), b, c->sp_stride, pop, s, k,
                                                             reinterpret_cast<long long*>(fit), head, c->status,
                                                             c->sp_order);
    GAPA_CUDA(cudaGetLastError());
    if (kernels) *kernels = 3;
    return GAPA_OK;
}
