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

}  // namespace gapa_dev
