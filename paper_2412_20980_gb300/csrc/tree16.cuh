// Shared-memory TREE fitness pipeline for graphs of at most 65536 nodes,
// written for a "team": a group of warps of one CTA that evaluates one
// population member with its own slice of shared memory and its own named
// barrier.  A whole CTA is one team (barrier 0); the batched persistent kernel
// splits a CTA into 2, 4 or 8 teams so that small graphs run several members
// per CTA.
//
// Fitness (Section III-C, Eq. 13; PC(G) of Table "Whole"): pairwise
// connectivity of G with the member's genes deleted.  Nodes are in BFS
// numbering (every tree parent precedes its child); see fitness.cu for the
// phases.
#pragma once

#include "gapa_internal.cuh"

namespace gapa_dev {

struct Team {
    int tid;  // thread index within the team
    int T;    // team size (a multiple of 32)
    int bar;  // named barrier id (0 = the whole CTA)
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory");
    }
};

// Path halving.  Invariant: a non-root's parent has a smaller id, so the
// walk terminates; roots change only by CAS in uf_unite.
__device__ __forceinline__ int uf_find(volatile int* lab, int x) {
    while (true) {
        const int p = lab[x];
        if (p == x) return x;
        const int gp = lab[p];
        if (gp == p) return p;
        lab[x] = gp;
        x = gp;
    }
}

// Root of x by a read-only walk.  Used once no hooking is left: every write
// then is an owner storing its node's final root, so no walk can leave a
// stale (non-root) ancestor behind, which path halving could.
__device__ __forceinline__ int uf_root(volatile int* lab, int x) {
    int p = lab[x];
    while (p != x) {
        x = p;
        p = lab[x];
    }
    return x;
}

// Union of the trees of live nodes a and b: hook the larger root under the
// smaller with a CAS on the root's slot; retry from the new parent on a race.
__device__ __forceinline__ void uf_unite(volatile int* lab, int a, int b) {
    a = uf_find(lab, a);
    b = uf_find(lab, b);
    while (a != b) {
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS((int*)&lab[a], a, b);
        if (old == a) return;
        a = uf_find(lab, old);
        b = uf_find(lab, b);
    }
}

__device__ __forceinline__ bool bm_test(const unsigned* bm, int v) { return (bm[v >> 5] >> (v & 31)) & 1u; }

// Sum (or, with mx, maximum) of non-negative values over the team; valid in
// team thread 0.  red: 32 slots of this team.
__device__ __forceinline__ long long team_sum_ll(const Team& tm, long long v, long long* red, bool mx = false) {
    for (int o = 16; o > 0; o >>= 1) {
        const long long x = __shfl_down_sync(0xffffffffu, v, o);
        v = mx ? (x > v ? x : v) : v + x;
    }
    const int warp = tm.tid >> 5, lane = tm.tid & 31;
    if (lane == 0) red[warp] = v;
    tm.sync();
    long long tot = 0;
    if (warp == 0) {
        tot = lane < (tm.T >> 5) ? red[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) {
            const long long x = __shfl_down_sync(0xffffffffu, tot, o);
            tot = mx ? (x > tot ? x : tot) : tot + x;
        }
    }
    return tot;
}

// A component of c nodes in the objective: C(c, 2) summed for PC, c maxed for MCN.
__device__ __forceinline__ long long objective_add(long long acc, long long c, int objective) {
    return objective ? (c > acc ? c : acc) : acc + c * (c - 1) / 2;
}

struct Tree16Graph {
    int n;
    const int* perm;     // original id -> BFS number
    const int2* palt;    // (tree parent, second lower-numbered neighbour or -1)
    const int* lo_ptr;   // lower-numbered neighbours (CSR)
    const int* lo_col;
    const unsigned* nontree;  // non-tree edges a<<16|b
    int num_nontree;
    const int* fptr;          // full adjacency in BFS numbering (CSR, 16-bit ids)
    const unsigned short* fcol;
    int join_mode;            // 0: per member, 1: non-tree edges, 2: scan outside the giant piece
    int mean_deg_x16;         // 16 * 2E / n, rounded up
    int objective;            // 0: PC, 1: MCN
    // cut-local variant only
    const int* tparent;       // tree parent per node (roots: itself), padded to a multiple of 4 entries
    const int4* kids;         // children in at most two runs: x .. x+y-1, then z+y .. z+y+w-1
    const int* roots;         // the BFS root of every component
    int num_roots;
    int list_bytes;           // bytes of the member's list region
};

// Shared-memory bytes of one member: labels + deleted-node bitmap (reused as
// a node list once the labels are set) + four team-wide scalars.
__host__ __device__ __forceinline__ size_t tree16_smem_bytes(int n) {
    return (size_t)n * 4 + (size_t)((n + 31) >> 5) * 4 + 16;
}

// The label pick of live node v: its tree parent if live, else its first
// live lower-numbered neighbour, else v; -1 for a deleted v.
__device__ __forceinline__ int tree16_pick(const unsigned* dead, const Tree16Graph& g, int v, int2 pa) {
    if (bm_test(dead, v)) return -1;
    if (pa.x == v || !bm_test(dead, pa.x)) return pa.x;
    if (pa.y < 0) return v;
    if (!bm_test(dead, pa.y)) return pa.y;
    const int beg = __ldg(&g.lo_ptr[v]) + 2, end = __ldg(&g.lo_ptr[v + 1]);
    for (int e = beg; e < end; ++e) {
        const int w = __ldg(&g.lo_col[e]);
        if (!bm_test(dead, w)) return w;
    }
    return v;
}

// Unite every live node of a warp's `cnt` nodes (node of lane j: nodes[j],
// -1 for none) with its live neighbours.  The arcs of the warp's nodes are
// laid end to end and dealt out one per lane; a lane finds its node by binary
// search over the warp's degree prefix sums.
__device__ __forceinline__ void tree16_scan_warp(volatile int* lab, const Tree16Graph& g, int v, int lane) {
    int b = 0, d = 0;
    if (v >= 0) {
        b = __ldg(&g.fptr[v]);
        d = __ldg(&g.fptr[v + 1]) - b;
    }
    int incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int s0 = 0; s0 < total; s0 += 32) {
        const int idx = s0 + lane;
        int lo = 0, hi = 31;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            if (__shfl_sync(0xffffffffu, incl, mid) > idx) hi = mid; else lo = mid + 1;
        }
        const int ov = __shfl_sync(0xffffffffu, v, lo), ob = __shfl_sync(0xffffffffu, b, lo),
                  oi = __shfl_sync(0xffffffffu, incl, lo), od = __shfl_sync(0xffffffffu, d, lo);
        if (idx < total) {
            const int w = __ldg(&g.fcol[ob + idx - (oi - od)]);
            const int lw = lab[w];
            if (lw != -1 && lw != lab[ov]) uf_unite(lab, ov, w);
        }
    }
}

// Root of live node v (labels may carry count bits above bit 16).
__device__ __forceinline__ int tree16_root16(volatile int* lab, int v) {
    int x = lab[v] & 0xFFFF;
    while (true) {
        const int q = lab[x] & 0xFFFF;
        if (q == x) return x;
        x = q;
    }
}

// One member: lab = n labels, dead = (n+31)/32 bitmap words followed by four
// scalars (all in this team's shared memory).  Deleted nodes end as -1.
//
// Phases: deletion bitmap; labels (tree parent, or on a deleted parent the
// first live lower-numbered neighbour, or the node itself); flatten every
// piece onto its top node.  The piece of the first live node R is the giant
// candidate: R has no live lower-numbered neighbour, so it is its piece's
// root and the smallest live id, and no union ever hooks it under another
// root.  The live nodes outside R's piece are listed (in the bitmap's words,
// which nothing reads any more) and counted; then the pieces are joined,
// either by letting only the listed nodes scan their adjacency (an edge
// inside R's piece joins nothing) or along every non-tree edge, whichever is
// cheaper (an arc scan costs about half a non-tree edge).  Sizes: only listed nodes can end outside R's
// component, so only they walk to their roots; R's component has the other
// live nodes plus the listed ones that reached R.  Without room for the list
// every live node walks and counts.
__device__ __forceinline__ void tree16_member(const Team& tm, volatile int* lab, unsigned* dead, const Tree16Graph& g,
                                              const int* __restrict__ genes, int k, long long* out, long long* red,
                                              int* status) {
    const int tid = tm.tid, T = tm.T, n = g.n, lane = tid & 31;
    const int words = (n + 31) >> 5;
    volatile int* scalar = reinterpret_cast<volatile int*>(dead + words);  // R, mode, list length, live
    for (int w = tid; w < words; w += T) dead[w] = 0u;
    tm.sync();
    // perturbation P^(A, p) of Eq. 13 in BFS numbering
    for (int j = tid; j < k; j += T) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n) {
            const int b = __ldg(&g.perm[d]);
            atomicOr(&dead[b >> 5], 1u << (b & 31));
        } else {
            atomicOr(status, GAPA_DEV_BAD_GENE);
        }
    }
    tm.sync();
    if (tid == 0) {
        int f = -1;
        for (int w = 0; w < words; ++w) {
            const unsigned live = ~dead[w];
            if (live) {
                f = (w << 5) + __ffs(live) - 1;
                break;
            }
        }
        scalar[0] = f < n ? f : -1;
        scalar[2] = 0;
    }
    // labels, four nodes per thread per step
    constexpr int kU = 4;
    for (int base = tid; base < n; base += kU * T) {
        int2 pa[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = base + u * T;
            pa[u] = v < n ? __ldg(&g.palt[v]) : make_int2(0, -1);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int v = base + u * T;
            if (v < n) lab[v] = tree16_pick(dead, g, v, pa[u]);
        }
    }
    tm.sync();
    const int R = scalar[0];
    // flatten (owner writes only) and list the live nodes outside R's piece
    int* list = reinterpret_cast<int*>(dead);
    long long live_out = 0;  // live << 32 | outside
    for (int base = 0; base < n; base += T) {
        const int v = base + tid;
        int r = -1;
        if (v < n) {
            const int p = lab[v];
            if (p != -1) {
                r = p == v ? v : uf_root(lab, p);
                if (p != v) lab[v] = r;
            }
        }
        const bool outside = r >= 0 && r != R;
        live_out += (r >= 0 ? (1ll << 32) : 0) + (outside ? 1 : 0);
        const unsigned m = __ballot_sync(0xffffffffu, outside);
        if (m) {
            int first = 0;
            if (lane == 0) first = atomicAdd((int*)&scalar[2], __popc(m));
            first = __shfl_sync(0xffffffffu, first, 0);
            const int slot = first + __popc(m & ((1u << lane) - 1));
            if (outside && slot < words) list[slot] = v;
        }
    }
    live_out = team_sum_ll(tm, live_out, red);
    if (tid == 0) {
        const long long outside = live_out & 0xFFFFFFFFll;
        // scanning costs about half as much per arc as uniting along a non-tree edge
        const bool scan = g.join_mode == 2 || (g.join_mode == 0 && outside * g.mean_deg_x16 <= 32ll * g.num_nontree);
        scalar[1] = (scan ? 1 : 0) | (outside <= words ? 2 : 0);
        scalar[3] = (int)(live_out >> 32);
    }
    tm.sync();
    const int mode = scalar[1], listed = scalar[2];
    const bool have_list = (mode & 2) != 0;
    const int nw = T >> 5;
    if ((mode & 1) && have_list) {
        // the listed nodes scan their adjacency, 32 per warp step
        for (int i0 = (tid >> 5) * 32; i0 < listed; i0 += nw * 32)
            tree16_scan_warp(lab, g, i0 + lane < listed ? list[i0 + lane] : -1, lane);
    } else if (mode & 1) {
        // the same over every node, skipping the groups of 32 with nobody outside R's piece
        for (int base = (tid >> 5) * 32; base < n; base += nw * 32) {
            const int v = base + lane;
            const int l = v < n ? lab[v] : -1;
            const bool outside = l != -1 && l != R;
            if (!__ballot_sync(0xffffffffu, outside)) continue;
            tree16_scan_warp(lab, g, outside ? v : -1, lane);
        }
    } else {
        // join the pieces along the non-tree edges, four per 16-byte load
        const uint4* e4 = reinterpret_cast<const uint4*>(g.nontree);
        const int quads = g.num_nontree >> 2;
        int q = tid;
        uint4 w = q < quads ? __ldg(&e4[q]) : make_uint4(0, 0, 0, 0);
        while (q < quads) {
            const int qn = q + T;
            const uint4 wn = qn < quads ? __ldg(&e4[qn]) : make_uint4(0, 0, 0, 0);
            const int a0 = (int)(w.x >> 16), b0 = (int)(w.x & 0xFFFFu), a1 = (int)(w.y >> 16), b1 = (int)(w.y & 0xFFFFu);
            const int a2 = (int)(w.z >> 16), b2 = (int)(w.z & 0xFFFFu), a3 = (int)(w.w >> 16), b3 = (int)(w.w & 0xFFFFu);
            const int la0 = lab[a0], lb0 = lab[b0], la1 = lab[a1], lb1 = lab[b1];
            const int la2 = lab[a2], lb2 = lab[b2], la3 = lab[a3], lb3 = lab[b3];
            if (la0 != lb0 && la0 != -1 && lb0 != -1) uf_unite(lab, la0, lb0);
            if (la1 != lb1 && la1 != -1 && lb1 != -1) uf_unite(lab, la1, lb1);
            if (la2 != lb2 && la2 != -1 && lb2 != -1) uf_unite(lab, la2, lb2);
            if (la3 != lb3 && la3 != -1 && lb3 != -1) uf_unite(lab, la3, lb3);
            q = qn;
            w = wn;
        }
        for (int e = quads * 4 + tid; e < g.num_nontree; e += T) {
            const unsigned x = __ldg(&g.nontree[e]);
            const int a = (int)(x >> 16), b = (int)(x & 0xFFFFu);
            const int la = lab[a], lb = lab[b];
            if (la != lb && la != -1 && lb != -1) uf_unite(lab, la, lb);
        }
    }
    tm.sync();
    // sizes: a root's slot becomes (members below it) << 16 | its id; a
    // root's own slot may already carry count bits, so it is classified by
    // the masked id; -1 (deleted) can equal no root slot because root ids are
    // below 65535.
    long long acc = 0;
    if (have_list) {
        long long joined = 0;  // listed nodes whose component is R's
        for (int i = tid; i < listed; i += T) {
            const int v = list[i];
            const int x = tree16_root16(lab, v);
            if (x == R) ++joined;
            else if (x != v) atomicAdd((unsigned*)&lab[x], 1u << 16);
        }
        joined = team_sum_ll(tm, joined, red);
        if (tid == 0) {
            const long long c = (long long)scalar[3] - listed + joined;  // R's component
            acc = objective_add(0, c, g.objective);
        }
        tm.sync();
        for (int i = tid; i < listed; i += T) {
            const int v = list[i];
            const unsigned l = (unsigned)lab[v];
            if ((int)(l & 0xFFFFu) == v) acc = objective_add(acc, (long long)(l >> 16) + 1, g.objective);
        }
    } else {
        // every live non-root walks to its root and adds itself: R's members by
        // one ballot, the other roots grouped with match_any
        for (int base = 0; base < n; base += T) {
            const int v = base + tid;
            int key = -1;
            if (v < n) {
                const int l = lab[v];
                if (l != -1 && (l & 0xFFFF) != v) key = tree16_root16(lab, v);
            }
            const unsigned giant = __ballot_sync(0xffffffffu, key >= 0 && key == R);
            if (giant && lane == 0) atomicAdd((unsigned*)&lab[R], (unsigned)__popc(giant) << 16);
            const bool other = key >= 0 && key != R;
            if (__any_sync(0xffffffffu, other)) {
                const unsigned peers = __match_any_sync(0xffffffffu, other ? key : -1);
                if (other && lane == __ffs(peers) - 1) atomicAdd((unsigned*)&lab[key], (unsigned)__popc(peers) << 16);
            }
        }
        tm.sync();
        for (int v = tid; v < n; v += T) {
            const unsigned l = (unsigned)lab[v];
            if (l != 0xFFFFFFFFu && (int)(l & 0xFFFFu) == v)
                acc = objective_add(acc, (long long)(l >> 16) + 1, g.objective);
        }
    }
    const long long tot = team_sum_ll(tm, acc, red, g.objective != 0);
    if (tid == 0) *out = tot;
}

// ---------------------------------------------------------------------------
// Cut-local variant.  Same fitness as tree16_member, with work proportional
// to what the deletion disturbs instead of to n:
//  * the tree-parent array is copied into the labels by one bulk copy
//    (cp.async.bulk, completion on an mbarrier), so every live node whose
//    parent is live already holds its final pick;
//  * only the children of deleted nodes are re-picked (first live lower-
//    numbered neighbour, else themselves); these "tops" start the pieces the
//    deletion cut off;
//  * each top walks to its root; a top whose root is not R (the first live
//    node, a root forever) seeds the list of nodes outside R's piece, and so
//    does every other live component root;
//  * the list grows level by level down the tree (a node's children have
//    consecutive numbers), each listed node taking its piece root as label;
//  * the pieces are joined either by the listed nodes' adjacency (an arc to
//    an unlisted live node unites with R directly, since every unlisted live
//    node lies in R's piece) or, for long lists, by giving every unlisted
//    live node R as label and uniting along the non-tree edges as
//    tree16_member does; then the sizes are counted on the list.
// Work items (children of a set of nodes, arcs of the listed nodes) are dealt
// out over the whole team through a team-wide prefix sum, so that one deleted
// hub with hundreds of children does not hold up a single warp.
// A member with repeated genes, or whose list outgrows its region or half the
// graph, or whose tree below the seeds is deeper than kLocalLevels, runs
// tree16_member (and so does, by the caller's choice, one whose cost
// estimate says the list will be long).

constexpr int kLocalLevels = 256;
constexpr long long kLocalSpinLimit = 1ll << 24;

// Layout of one member: labels (n rounded up to a multiple of 4, so the bulk
// copy moves whole 16-byte units), the list region, eight team scalars and
// the mbarrier.  The list region holds, from its start, the deletion bitmap
// (until the re-picks are done) and then the list (16-bit node ids); at its
// end four arrays of one int per team thread for the dealing rounds, and
// the bitmap of listed nodes.
__host__ __device__ __forceinline__ size_t tree16l_lab_ints(int n) { return ((size_t)n + 3) & ~(size_t)3; }
__host__ __device__ __forceinline__ size_t tree16l_bitmap_bytes(int n) {
    return ((((size_t)n + 31) >> 5) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t tree16l_scratch_bytes(int team) { return (size_t)4 * team * 4; }
__host__ __device__ __forceinline__ size_t tree16l_min_list_bytes(int n, int team) {
    return 2 * tree16l_bitmap_bytes(n) + tree16l_scratch_bytes(team);
}
__host__ __device__ __forceinline__ size_t tree16l_smem_bytes(int n, size_t list_bytes) {
    return tree16l_lab_ints(n) * 4 + list_bytes + 32 + 16;
}

__device__ __forceinline__ unsigned tree16l_smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool tree16l_wait(unsigned bar, unsigned parity) {
    for (long long i = 0; i < kLocalSpinLimit; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Exclusive prefix sum of v over the team in thread order; *total = the sum.
// ws: 32 ints of team scratch, free again after the caller's next barrier.
// Contains two team barriers.
__device__ __forceinline__ int tree16l_scan(const Team& tm, int v, int* ws, int* total) {
    const int lane = tm.tid & 31, warp = tm.tid >> 5, nw = tm.T >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) ws[warp] = incl;
    tm.sync();
    if (warp == 0) {
        int x = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) ws[lane] = x;
    }
    tm.sync();
    *total = ws[nw - 1];
    return (warp ? ws[warp - 1] : 0) + incl - v;
}

// The owner of item i among `owners` owners with exclusive offsets off[]:
// the last owner whose offset is at most i (owners without items share the
// next one's offset and come before it).
__device__ __forceinline__ int tree16l_owner(const int* off, int owners, int i) {
    int lo = 0, hi = owners - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Warp-aggregated append of val (where want) to the 16-bit list, marking it
// in the listed-node bitmap; entries past cap are dropped (the caller sees
// the count exceed cap).  Called by all lanes of a warp.
__device__ __forceinline__ void tree16l_append(bool want, int val, int lane, volatile int* count,
                                               unsigned short* list, int cap, unsigned* listed_bm) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    int first = 0;
    if (lane == 0) first = atomicAdd((int*)count, __popc(m));
    first = __shfl_sync(0xffffffffu, first, 0);
    const int slot = first + __popc(m & ((1u << lane) - 1));
    if (want && slot < cap) {
        list[slot] = (unsigned short)val;
        atomicOr(&listed_bm[val >> 5], 1u << (val & 31));
    }
}

// Join step for the arc (a, b) of a listed node once the list is complete:
// two listed ends unite their sets; a listed end and an unlisted live one
// unite with R.
__device__ __forceinline__ void tree16l_join_edge(volatile int* lab, const unsigned* listed_bm, int R, int a, int b) {
    const bool la = bm_test(listed_bm, a), lb = bm_test(listed_bm, b);
    if (!la && !lb) return;
    if (la && lb) {
        if (lab[a] != lab[b]) uf_unite(lab, a, b);
        return;
    }
    const int x = la ? a : b, y = la ? b : a;
    if (lab[y] != -1 && lab[x] != R) uf_unite(lab, x, R);
}

// Child of owner o for item i of a dealing round (owner records: first item,
// first run start | length << 16, second run start less the first's length).
__device__ __forceinline__ int tree16l_child(const int* s_off, const int* s_run, const int* s_run2, int o, int i) {
    const int r = i - s_off[o];
    const unsigned run = (unsigned)s_run[o];
    return r < (int)(run >> 16) ? (int)(run & 0xFFFFu) + r : s_run2[o] + r;
}

// Owner records of the team's chunk of genes j0 .. j0+T-1 (node, children
// runs; the first chunk's come from registers), their exclusive offsets and
// *total items.  Returns the thread's gene node (-1: none).  Ends with a team
// barrier.
__device__ __forceinline__ int tree16l_gene_chunk(const Team& tm, const Tree16Graph& g, const int* __restrict__ genes,
                                                  int k, int j0, int b0, int4 ch0, int* s_off, int* s_run,
                                                  int* s_run2, int* ws, int* total) {
    int b = b0;
    int4 ch = ch0;
    if (j0 > 0) {
        b = -1;
        ch = make_int4(0, 0, 0, 0);
        const int j = j0 + tm.tid;
        if (j < k) {
            const int d = __ldg(&genes[j]);
            if ((unsigned)d < (unsigned)g.n) {
                b = __ldg(&g.perm[d]);
                ch = __ldg(&g.kids[b]);
            }
        }
    }
    const int off = tree16l_scan(tm, ch.y + ch.w, ws, total);
    s_off[tm.tid] = off;
    s_run[tm.tid] = (int)((unsigned)ch.x | ((unsigned)ch.y << 16));
    s_run2[tm.tid] = ch.z;
    tm.sync();
    return b;
}

// lab: the member's labels; region: its list region (g.list_bytes); scal_base:
// its eight scalars followed by the mbarrier.  Returns through *out like
// tree16_member.
__device__ __forceinline__ void tree16_member_local(const Team& tm, volatile int* lab, unsigned* region,
                                                    int* scal_base, const Tree16Graph& g,
                                                    const int* __restrict__ genes, int k, long long* out,
                                                    long long* red, int* status) {
    const int tid = tm.tid, T = tm.T, n = g.n, lane = tid & 31;
    const int words = (n + 31) >> 5;
    volatile int* scalar = scal_base;  // 0 R, 1 list length, 2 repeated genes, 3 live, 4 labels landed
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(scal_base + 8);
    const unsigned bar_a = tree16l_smem_u32(bar);
    unsigned* dead = region;
    unsigned short* list = reinterpret_cast<unsigned short*>(region);
    const int bm_bytes = (int)tree16l_bitmap_bytes(n);
    char* tail_area = reinterpret_cast<char*>(region) + g.list_bytes - bm_bytes - (int)tree16l_scratch_bytes(T);
    // dealing rounds: per owner its first item, its children's first run (start | length << 16),
    // the start of the second run less the first run's length, and a value (piece root, node)
    int* s_off = reinterpret_cast<int*>(tail_area);
    int* s_run = s_off + T;
    int* s_run2 = s_run + T;
    int* s_own = s_run2 + T;
    unsigned* listed_bm = reinterpret_cast<unsigned*>(s_own + T);

    const int cap = (int)((tail_area - reinterpret_cast<char*>(region)) >> 1);
    int* ws = reinterpret_cast<int*>(red);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int w = tid; w < words; w += T) {
        dead[w] = 0u;
        listed_bm[w] = 0u;
    }
    tm.sync();
    if (tid == 0) {
        // labels <- tree parents, in chunks of at most 32 KB (the fence orders this team's earlier
        // generic-proxy use of the labels before the async-proxy writes)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const unsigned bytes = (unsigned)(tree16l_lab_ints(n) * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        const unsigned dst = tree16l_smem_u32((const void*)lab);
        for (unsigned o = 0; o < bytes; o += 32768u) {
            const unsigned len = bytes - o < 32768u ? bytes - o : 32768u;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dst + o),
                "l"(reinterpret_cast<const char*>(g.tparent) + o), "r"(len), "r"(bar_a)
                : "memory");
        }
    }
    // perturbation P^(A, p) of Eq. 13 in BFS numbering; count the distinct
    // deleted nodes and the repeated genes.  The first T genes keep their
    // node, first child and number of children in registers.
    long long fresh_dup = 0;  // distinct << 32 | repeated
    int b0 = -1;
    int4 ch0 = make_int4(0, 0, 0, 0);
    for (int j = tid; j < k; j += T) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n) {
            const int b = __ldg(&g.perm[d]);
            const unsigned bit = 1u << (b & 31);
            const unsigned old = atomicOr(&dead[b >> 5], bit);
            fresh_dup += (old & bit) ? 1 : (1ll << 32);
            if (j == tid) {
                b0 = b;
                ch0 = __ldg(&g.kids[b]);
            }
        } else {
            atomicOr(status, GAPA_DEV_BAD_GENE);
        }
    }
    fresh_dup = team_sum_ll(tm, fresh_dup, red);  // (includes a team barrier: the bitmap is complete)
    if ((tid >> 5) == 0) {
        // R = the first live node
        int f = -1;
        for (int w0 = 0; w0 < words && f < 0; w0 += 32) {
            const int w = w0 + lane;
            unsigned live = w < words ? ~dead[w] : 0u;
            if (w == words - 1 && (n & 31)) live &= (1u << (n & 31)) - 1u;
            const unsigned m = __ballot_sync(0xffffffffu, live != 0u);
            if (m) {
                const int src = __ffs(m) - 1;
                const unsigned lw = __shfl_sync(0xffffffffu, live, src);
                f = ((w0 + src) << 5) + __ffs(lw) - 1;
            }
        }
        if (lane == 0) {
            scalar[0] = f;
            scalar[1] = 0;
            scalar[2] = (fresh_dup & 0xFFFFFFFFll) != 0;
            scalar[3] = n - (int)(fresh_dup >> 32);
        }
    }
    // the labels must have landed before anyone reads or writes them
    bool ok = tree16l_wait(bar_a, 0u);
    if (!ok) {
        atomicOr(status, GAPA_DEV_TIMEOUT);
        tree16l_wait(bar_a, 0u);  // bounded: the copy may still be in flight
    }
    if (tid == 0) scalar[4] = ok;
    tm.sync();
    ok = scalar[4] != 0;  // thread 0's view, the same for the whole team
    // the copy has landed: the mbarrier's memory may be reused
    if (tid == 0 && ok) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar_a) : "memory");
    if (!ok) {
        if (tid == 0) *out = -1;
        return;
    }
    const int R = scalar[0];
    if (R < 0) {  // every node deleted
        if (tid == 0) *out = 0;
        return;
    }
    if (scalar[2]) {  // repeated genes: the per-gene passes below would list tops twice
        tree16_member(tm, lab, region, g, genes, k, out, red, status);
        return;
    }
    // re-pick the children of the deleted nodes
    int tops_total = 0;
    for (int j0 = 0; j0 < k; j0 += T) {
        const int b = tree16l_gene_chunk(tm, g, genes, k, j0, b0, ch0, s_off, s_run, s_run2, ws, &tops_total);
        if (b >= 0) lab[b] = -1;
        const int owners = min(T, k - j0);
        for (int i = tid; i < tops_total; i += T) {
            const int c = tree16l_child(s_off, s_run, s_run2, tree16l_owner(s_off, owners, i), i);
            if (!bm_test(dead, c)) lab[c] = tree16_pick(dead, g, c, __ldg(&g.palt[c]));
        }
        tm.sync();
    }
    // from here a deleted node is a label of -1; the bitmap's words become the list.
    // Seeds: tops whose root is not R (each top takes its root as label)
    for (int j0 = 0; j0 < k; j0 += T) {
        if (k > T)  // one chunk: the offsets are still in place
            tree16l_gene_chunk(tm, g, genes, k, j0, b0, ch0, s_off, s_run, s_run2, ws, &tops_total);
        const int owners = min(T, k - j0);
        for (int i0 = tid & ~31; i0 < tops_total; i0 += T) {
            const int i = i0 + lane;
            bool want = false;
            int c = 0;
            if (i < tops_total) {
                c = tree16l_child(s_off, s_run, s_run2, tree16l_owner(s_off, owners, i), i);
                const int l = lab[c];
                if (l != -1) {
                    const int r = l == c ? c : uf_root(lab, l);
                    if (r != l) lab[c] = r;
                    want = r != R;
                }
            }
            tree16l_append(want, c, lane, &scalar[1], list, cap, listed_bm);
        }
        tm.sync();
    }
    for (int i0 = tid & ~31; i0 < g.num_roots; i0 += T) {
        const int i = i0 + lane;
        const int rho = i < g.num_roots ? __ldg(&g.roots[i]) : -1;
        tree16l_append(rho >= 0 && rho != R && lab[rho] == rho, rho, lane, &scalar[1], list, cap, listed_bm);
    }
    tm.sync();
    // the list grows one tree level per round; the children of up to T listed
    // nodes per dealing step
    // (a list past half the graph is cheaper in the full pipeline)
    const int lim = min(cap, max(n / 2, 256));
    int head = 0, tail = scalar[1], level = 0;
    while (head < tail && tail <= lim && level < kLocalLevels) {
        for (int u0 = head; u0 < tail; u0 += T) {
            const int idx = u0 + tid;
            int4 ch = make_int4(0, 0, 0, 0);
            int r = 0;
            if (idx < tail) {
                const int u = list[idx];
                ch = __ldg(&g.kids[u]);
                r = lab[u];
            }
            int total;
            const int off = tree16l_scan(tm, ch.y + ch.w, ws, &total);
            s_off[tid] = off;
            s_run[tid] = (int)((unsigned)ch.x | ((unsigned)ch.y << 16));
            s_run2[tid] = ch.z;
            s_own[tid] = r;
            tm.sync();
            const int owners = min(T, tail - u0);
            for (int i0 = tid & ~31; i0 < total; i0 += T) {
                const int i = i0 + lane;
                bool want = false;
                int x = 0;
                if (i < total) {
                    const int o = tree16l_owner(s_off, owners, i);
                    x = tree16l_child(s_off, s_run, s_run2, o, i);
                    if (lab[x] != -1) {
                        lab[x] = s_own[o];
                        want = true;
                    }
                }
                tree16l_append(want, x, lane, &scalar[1], list, cap, listed_bm);
            }
            tm.sync();
        }
        head = tail;
        tail = scalar[1];
        ++level;
        tm.sync();  // every thread has read the new length before the next round appends
    }
    if (tail > lim || head < tail) {  // list overflow or a tree too deep: the full pipeline
        tree16_member(tm, lab, region, g, genes, k, out, red, status);
        return;
    }
    const int listed = tail;
    // join: the listed nodes' arcs, or (long lists) the non-tree edges, four
    // per 16-byte load, after a pass that labels R's piece
    if ((long long)listed * g.mean_deg_x16 <= 4ll * g.num_nontree) {
        for (int v0 = 0; v0 < listed; v0 += T) {
            const int idx = v0 + tid;
            int v = 0, b = 0, d = 0;
            if (idx < listed) {
                v = list[idx];
                b = __ldg(&g.fptr[v]);
                d = __ldg(&g.fptr[v + 1]) - b;
            }
            int total;
            const int off = tree16l_scan(tm, d, ws, &total);
            s_off[tid] = off;
            s_run2[tid] = b;
            s_own[tid] = v;
            tm.sync();
            const int owners = min(T, listed - v0);
            for (int i = tid; i < total; i += T) {
                const int o = tree16l_owner(s_off, owners, i);
                const int w = __ldg(&g.fcol[s_run2[o] + i - s_off[o]]);
                tree16l_join_edge(lab, listed_bm, R, s_own[o], w);
            }
            tm.sync();
        }
    } else {
        // every unlisted live node lies in R's piece: give it R as label, then
        // unite along the non-tree edges whose ends carry different labels
        for (int v = tid; v < n; v += T)
            if (!bm_test(listed_bm, v) && lab[v] != -1) lab[v] = R;
        tm.sync();
        const uint4* e4 = reinterpret_cast<const uint4*>(g.nontree);
        const int quads = g.num_nontree >> 2;
        int q = tid;
        uint4 w = q < quads ? __ldg(&e4[q]) : make_uint4(0, 0, 0, 0);
        while (q < quads) {
            const int qn = q + T;
            const uint4 wn = qn < quads ? __ldg(&e4[qn]) : make_uint4(0, 0, 0, 0);
            const int a0 = (int)(w.x >> 16), b0 = (int)(w.x & 0xFFFFu), a1 = (int)(w.y >> 16), b1 = (int)(w.y & 0xFFFFu);
            const int a2 = (int)(w.z >> 16), b2 = (int)(w.z & 0xFFFFu), a3 = (int)(w.w >> 16), b3 = (int)(w.w & 0xFFFFu);
            const int la0 = lab[a0], lb0 = lab[b0], la1 = lab[a1], lb1 = lab[b1];
            const int la2 = lab[a2], lb2 = lab[b2], la3 = lab[a3], lb3 = lab[b3];
            if (la0 != lb0 && la0 != -1 && lb0 != -1) uf_unite(lab, la0, lb0);
            if (la1 != lb1 && la1 != -1 && lb1 != -1) uf_unite(lab, la1, lb1);
            if (la2 != lb2 && la2 != -1 && lb2 != -1) uf_unite(lab, la2, lb2);
            if (la3 != lb3 && la3 != -1 && lb3 != -1) uf_unite(lab, la3, lb3);
            q = qn;
            w = wn;
        }
        for (int e = quads * 4 + tid; e < g.num_nontree; e += T) {
            const unsigned x = __ldg(&g.nontree[e]);
            const int a = (int)(x >> 16), b = (int)(x & 0xFFFFu);
            const int la = lab[a], lb = lab[b];
            if (la != lb && la != -1 && lb != -1) uf_unite(lab, la, lb);
        }
        tm.sync();
    }
    // sizes on the list (see tree16_member)
    long long joined = 0;
    for (int i = tid; i < listed; i += T) {
        const int v = list[i];
        const int x = tree16_root16(lab, v);
        if (x == R) ++joined;
        else if (x != v) atomicAdd((unsigned*)&lab[x], 1u << 16);
    }
    joined = team_sum_ll(tm, joined, red);
    long long acc = 0;
    if (tid == 0) acc = objective_add(0, (long long)scalar[3] - listed + joined, g.objective);
    tm.sync();
    for (int i = tid; i < listed; i += T) {
        const int v = list[i];
        const unsigned l = (unsigned)lab[v];
        if ((int)(l & 0xFFFFu) == v) acc = objective_add(acc, (long long)(l >> 16) + 1, g.objective);
    }
    const long long tot = team_sum_ll(tm, acc, red, g.objective != 0);
    if (tid == 0) *out = tot;
}
}  // namespace gapa_dev
