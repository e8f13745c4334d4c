// Forest-piece evaluation of one population member: the fitness of
// Section III-C (Eq. 13; PC(G) of Table "Whole") without a per-node label
// array, so that several members share one SM.
//
// At upload the graph gets a spanning forest whose parents precede their
// children (BFS numbering), the subtree size sz of every node, a preorder
// position pre (a subtree is the interval [pre, pre + sz) of positions) and
// the root of every node's tree.  Deleting the member's node set D cuts the
// forest into pieces, each rooted at a live child of a deleted node (a "top")
// or at a live root of a tree in a component that contains a deleted node (a
// component may span several trees of the forest); a component without
// deleted nodes stays whole.  Then:
//
//  1. piece sizes by subtraction: a piece rooted at p has sz[p] nodes less
//     the subtrees of the deleted nodes whose parent lies in the piece (the
//     piece of a live node is found by walking up the forest until the parent
//     is deleted or the node is a root);
//  2. every top re-picks a live lower-numbered neighbour (its tree parent is
//     deleted), and the two pieces are united (union-find over piece ids);
//  3. the class with the most nodes is taken as the giant; every live node
//     of every other piece is enumerated from its piece's preorder interval
//     and each of its arcs to a live node of another piece unites the two
//     pieces' classes.  An edge between two nodes of the giant class joins
//     nothing new, and every other edge has an end outside it, so the classes
//     are then the components of G[V \ D];
//  4. the objective: the sum of C(size, 2) (PC) or the largest size (MCN)
//     over the classes, plus the untouched components.
//
// A member is evaluated by a team of warps; the walks up the forest read a
// 16-bit copy of the forest's parents that the CTA keeps in shared memory
// for all its teams.  Shared memory per member: the deleted-node bitmap, a
// bitmap of the components already seen, the distinct deleted nodes, an
// open-addressing table from a piece's root node to its id, and per piece its
// root, union-find parent, size and class size (which holds the re-pick
// target until the classes are summed).  A member whose pieces or distinct
// deletions exceed the capacities, or whose nodes outside the giant class
// exceed the enumeration budget, returns false (the caller evaluates it
// another way).
#pragma once

#include "tree16.cuh"

namespace gapa_dev {

struct PieceGraph {
    int n;
    const int* perm;             // original id -> forest number
    const int* tparent;          // forest parent (roots: itself); parents precede children
    const int2* palt;            // (tree parent, second lower-numbered neighbour or -1)
    const int* lo_ptr;           // lower-numbered neighbours (CSR, ascending)
    const int* lo_col;
    const int* fptr;             // full adjacency in forest numbers (CSR, 16-bit ids)
    const unsigned short* fcol;
    const int4* kids;            // children in at most two runs (see Tree16Graph::kids)
    const int* sz;               // subtree size
    const int* pre;              // preorder position
    const unsigned short* at;    // node at each preorder position
    const int* crep;             // smallest root of each node's component (its representative)
    const int* nroot;            // next root of the same component, ascending (-1: none)
    const int* csize;            // component size, at the representative
    const int* roots;            // every root
    int num_roots;
    long long tree_pc;           // sum over the components of G of C(size, 2)
    int objective;               // 0: PC, 1: MCN
};

// Byte offsets of one member's (team's) shared memory (computed on the host).
struct PieceLayout {
    int T;       // threads per team
    int words;   // bitmap words
    int dcap;    // distinct deleted nodes (later: pieces outside the giant class)
    int hbits;   // log2 of the table slots
    int pcap;    // pieces
    int vcap;    // enumeration budget outside the giant class (preorder positions)
    unsigned off_dead, off_seen, off_listed, off_scr, off_dl, off_hash, off_pn, off_pu, off_ps, off_acc, off_pst, bytes;
};

__host__ __device__ __forceinline__ unsigned piece_align16(size_t x) { return (unsigned)((x + 15) & ~(size_t)15); }

// Bytes of the CTA's 16-bit copy of the forest parents.
__host__ __device__ __forceinline__ unsigned piece_parents_bytes(int n) { return piece_align16((size_t)n * 2); }

constexpr int kPieceSlots = 4;  // genes (and preorder positions) a thread keeps in registers per pass

// Layout of one team for a graph of n nodes, k genes, T threads and `budget` bytes; pcap = 0 when
// it does not fit.  The table has at least 4/3 slots per piece (load at most 0.75).
inline PieceLayout piece_layout(int n, int k, int T, size_t budget) {
    PieceLayout L{};
    L.T = T;
    L.words = (n + 31) >> 5;
    size_t o = 0;
    L.off_dead = 0;
    o = piece_align16((size_t)L.words * 4);
    L.off_seen = (unsigned)o;
    o = piece_align16(o + (size_t)L.words * 4);
    L.off_listed = (unsigned)o;
    o = piece_align16(o + (size_t)L.words * 4);
    L.off_scr = (unsigned)o;  // ws[32], three dealing arrays of T ints, red[32] (8 B), scalars[16]
    o = piece_align16(o + (size_t)(32 + 3 * T) * 4 + 32 * 8 + 16 * 4);
    L.dcap = k < 64 ? 64 : k;
    L.off_dl = (unsigned)o;
    o = piece_align16(o + (size_t)L.dcap * 4);
    L.vcap = n / 4 > 4096 ? n / 4 : 4096;
    if (o >= budget) return L;
    const size_t rest = budget - o;
    int best_p = 0, best_h = 0;
    for (int hb = 6; hb <= 16; ++hb) {
        const size_t hs = (size_t)1 << hb;
        if (hs * 4 + 80 > rest) break;
        // per piece: root (2 B), union-find parent, size, class size, subtree size (4 B each)
        size_t p = (rest - hs * 4 - 80) / 18;
        if (p > hs * 3 / 4) p = hs * 3 / 4;
        if (p > 65535) p = 65535;
        if ((int)p > best_p) {
            best_p = (int)p;
            best_h = hb;
        }
    }
    if (best_p < 64) return L;
    L.hbits = best_h;
    L.pcap = best_p & ~7;
    const size_t hs = (size_t)1 << L.hbits, pc = (size_t)L.pcap;
    L.off_hash = (unsigned)o;
    o = piece_align16(o + hs * 4);
    L.off_pn = (unsigned)o;
    o = piece_align16(o + pc * 2);
    L.off_pu = (unsigned)o;
    o = piece_align16(o + pc * 4);
    L.off_ps = (unsigned)o;
    o = piece_align16(o + pc * 4);
    L.off_acc = (unsigned)o;
    o = piece_align16(o + pc * 4);
    L.off_pst = (unsigned)o;
    o = piece_align16(o + pc * 4);
    L.bytes = (unsigned)o;
    if (o > budget) L.pcap = 0;
    return L;
}

constexpr unsigned kPieceEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned piece_hash(int key, int hbits) {
    return ((unsigned)key * 0x9E3779B1u) >> (32 - hbits);
}

// Piece id of the piece rooted at node `key` (-1: none).
__device__ __forceinline__ int piece_lookup(const unsigned* hash, int hbits, int key) {
    const unsigned mask = (1u << hbits) - 1u;
    unsigned h = piece_hash(key, hbits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const unsigned e = hash[h];
        if (e == kPieceEmpty) return -1;
        if ((int)(e >> 16) == key) return (int)(e & 0xFFFFu);
        h = (h + 1) & mask;
    }
    return -1;
}

// The root of the piece holding live node y: up the forest (the shared-memory copy of the
// parents) until the parent is deleted (y is then a top) or y is a root.  Parents have smaller
// numbers, so the walk ends.
__device__ __forceinline__ int piece_walk(const unsigned short* tp, const unsigned* dead, int y) {
    while (true) {
        const int p = tp[y];
        if (p == y || bm_test(dead, p)) return y;
        y = p;
    }
}

// The owner of item i among `owners` owners with exclusive offsets off[].
__device__ __forceinline__ int piece_owner(const int* off, int owners, int i) {
    int lo = 0, hi = owners - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One arc (x, y) of the live node x of piece pi, a piece outside the giant class: a live y that is
// not listed (in no piece outside the giant class) marks pi as touching the giant (flag[pi] = 2);
// a listed y of another piece unites the two pieces' classes.
__device__ __forceinline__ void piece_join_arc(const unsigned short* tp, const unsigned* dead, const unsigned* listed,
                                               const unsigned* hash, int hbits, int* pu, int* flag, volatile int* err,
                                               int x, int px, int pi, int y) {
    if (y == px || bm_test(dead, y)) return;
    if (!bm_test(listed, y)) {
        flag[pi] = 2;
        return;
    }
    const int py = tp[y];
    if (py == x) return;  // a child of x: the same piece
    const int z = (py == y || bm_test(dead, py)) ? y : piece_walk(tp, dead, py);
    const int j = piece_lookup(hash, hbits, z);
    if (j < 0) *err = 1;
    else if (j != pi) uf_unite(pu, pi, j);
}

// The arcs e0, e0+step, ... < e1 of x (eight reads in flight at a time).
__device__ __forceinline__ void piece_join_arcs(const PieceGraph& g, const unsigned short* tp, const unsigned* dead,
                                                const unsigned* listed, const unsigned* hash, int hbits, int* pu,
                                                int* flag, volatile int* err, int x, int pi, int e0, int e1,
                                                int step) {
    const int px = tp[x];
    for (int e = e0; e < e1; e += 8 * step) {
        int y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = e + u * step < e1 ? (int)__ldg(&g.fcol[e + u * step]) : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (y[u] >= 0) piece_join_arc(tp, dead, listed, hash, hbits, pu, flag, err, x, px, pi, y[u]);
    }
}

// acc[r] += v for the lanes with `active`, one atomic per distinct r in the warp (the pieces of
// one class, which is mostly the giant, would otherwise queue on one shared-memory word).  Called
// by all lanes of the warp.
__device__ __forceinline__ void piece_class_add(int* acc, int r, int v, bool active) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const unsigned same = __match_any_sync(act, r);
    const int tot = (int)__reduce_add_sync(same, (unsigned)v);
    if (__ffs(same) - 1 == (int)(threadIdx.x & 31)) atomicAdd(&acc[r], tot);
}

// Warp-aggregated slot in a list counted by *count (valid for the lanes with `want`).
__device__ __forceinline__ int piece_append_slot(bool want, volatile int* count) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return -1;
    const int lane = threadIdx.x & 31;
    int first = 0;
    if (lane == __ffs(m) - 1) first = atomicAdd((int*)count, __popc(m));
    first = __shfl_sync(0xffffffffu, first, __ffs(m) - 1);
    return want ? first + __popc(m & ((1u << lane) - 1u)) : -1;
}

// Evaluates one member with team tm (T = L.T threads, named barrier); *out = its objective.
// tp: the CTA's shared-memory copy of g's parents.  Returns false (nothing written) when the member
// exceeds the layout's capacities.  Every return is taken by the whole team.  The global reads are
// batched so that a member waits for few dependent round trips: genes, their forest numbers, the
// deleted nodes' subtree sizes and children, the tops' parent pairs and subtree sizes, and, outside
// the giant class, preorder positions, nodes, adjacency ranges and arcs.
__device__ __forceinline__ bool piece_member(const Team& tm, const PieceGraph& g, const PieceLayout& L,
                                             unsigned char* sm, const unsigned short* tp,
                                             const int* __restrict__ genes, int k, long long* out, int* status) {
    const int tid = tm.tid, T = tm.T;
    const int n = g.n;
    unsigned* dead = reinterpret_cast<unsigned*>(sm + L.off_dead);
    unsigned* seen = reinterpret_cast<unsigned*>(sm + L.off_seen);
    unsigned* listed = reinterpret_cast<unsigned*>(sm + L.off_listed);
    int* ws = reinterpret_cast<int*>(sm + L.off_scr);
    int* s_off = ws + 32;
    int* s_a = s_off + T;
    int* s_b = s_a + T;
    long long* red = reinterpret_cast<long long*>(s_b + T);
    volatile int* scal = reinterpret_cast<int*>(red + 32);  // 0 pieces, 1 distinct, 2 overflow, 3 giant, 4 outside
    unsigned* dl = reinterpret_cast<unsigned*>(sm + L.off_dl);  // node << 16 | (subtree size - 1)
    unsigned* hash = reinterpret_cast<unsigned*>(sm + L.off_hash);
    unsigned short* pn = reinterpret_cast<unsigned short*>(sm + L.off_pn);
    int* pu = reinterpret_cast<int*>(sm + L.off_pu);
    int* ps = reinterpret_cast<int*>(sm + L.off_ps);
    int* acc = reinterpret_cast<int*>(sm + L.off_acc);
    int* pst = reinterpret_cast<int*>(sm + L.off_pst);
    const int hs = 1 << L.hbits;

    for (int w = tid; w < L.words; w += T) {
        dead[w] = 0u;
        seen[w] = 0u;
        listed[w] = 0u;
    }
    for (int h = tid; h < hs; h += T) hash[h] = kPieceEmpty;
    if (tid == 0) {
        scal[0] = 0;
        scal[1] = 0;
        scal[2] = 0;
        scal[4] = 0;
    }
    tm.sync();

    // 1. the deletion set (Eq. 13) in forest numbers; its distinct nodes with their subtree sizes
    for (int j0 = 0; j0 < k; j0 += kPieceSlots * T) {
        int b[kPieceSlots], zb[kPieceSlots];
#pragma unroll
        for (int u = 0; u < kPieceSlots; ++u) {
            const int j = j0 + u * T + tid;
            b[u] = j < k ? __ldg(&genes[j]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kPieceSlots; ++u) {
            const int j = j0 + u * T + tid;
            if (j < k && (unsigned)b[u] >= (unsigned)n) atomicOr(status, GAPA_DEV_BAD_GENE);
            b[u] = (j < k && (unsigned)b[u] < (unsigned)n) ? __ldg(&g.perm[b[u]]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kPieceSlots; ++u) zb[u] = b[u] >= 0 ? __ldg(&g.sz[b[u]]) : 0;
#pragma unroll
        for (int u = 0; u < kPieceSlots; ++u) {
            bool fresh = false;
            if (b[u] >= 0) {
                const unsigned bit = 1u << (b[u] & 31);
                fresh = !(atomicOr(&dead[b[u] >> 5], bit) & bit);
            }
            const int slot = piece_append_slot(fresh, &scal[1]);
            if (fresh) {
                if (slot < L.dcap) dl[slot] = ((unsigned)b[u] << 16) | (unsigned)(zb[u] - 1);
                else scal[2] = 1;
            }
        }
    }
    tm.sync();
    if (scal[2]) return false;
    const int nd = scal[1];
    if (nd >= n) {  // every node deleted
        if (tid == 0) *out = 0;
        tm.sync();
        return true;
    }

    // 2. pieces: the live children of the deleted nodes (the class-size slot holds the re-pick, a
    // live lower-numbered neighbour), and the live roots of the trees of every component holding
    // deleted nodes; those components' C(size, 2) leave the untouched total.  The children runs
    // of the thread's first kPieceSlots deleted nodes are read at once.
    long long dirty = 0;
    int4 kch[kPieceSlots];
    int krep[kPieceSlots];
#pragma unroll
    for (int u = 0; u < kPieceSlots; ++u) {
        const int r = u * T + tid;
        const int b = r < nd ? (int)(dl[r] >> 16) : 0;
        kch[u] = r < nd ? __ldg(&g.kids[b]) : make_int4(0, 0, 0, 0);
        krep[u] = r < nd ? __ldg(&g.crep[b]) : -1;
    }
    for (int r0 = 0, u = 0; r0 < nd; r0 += T, ++u) {
        const int r = r0 + tid;
        int4 ch = make_int4(0, 0, 0, 0);
        int rep = -1;
        if (u < kPieceSlots) {
#pragma unroll
            for (int v = 0; v < kPieceSlots; ++v)
                if (v == u) {
                    ch = kch[v];
                    rep = krep[v];
                }
        } else if (r < nd) {
            const int b = (int)(dl[r] >> 16);
            ch = __ldg(&g.kids[b]);
            rep = __ldg(&g.crep[b]);
        }
        if (rep >= 0) {
            const unsigned bit = 1u << (rep & 31);
            // (most deleted nodes share one component: read the bit before taking it)
            if (!(seen[rep >> 5] & bit) && !(atomicOr(&seen[rep >> 5], bit) & bit)) {
                const long long csz = __ldg(&g.csize[rep]);
                dirty += csz * (csz - 1) / 2;
                for (int rt = rep; rt >= 0; rt = __ldg(&g.nroot[rt])) {
                    if (bm_test(dead, rt)) continue;
                    const int i = atomicAdd((int*)&scal[0], 1);
                    if (i < L.pcap) {
                        const int z = __ldg(&g.sz[rt]);
                        pn[i] = (unsigned short)rt;
                        acc[i] = rt;
                        pu[i] = i;
                        ps[i] = z;
                        pst[i] = z;
                    }
                }
            }
        }
        int total;
        const int off = tree16l_scan(tm, ch.y + ch.w, ws, &total);
        s_off[tid] = off;
        s_a[tid] = (int)((unsigned)ch.x | ((unsigned)ch.y << 16));
        s_b[tid] = ch.z;
        tm.sync();
        const int owners = min(T, nd - r0);
        for (int it0 = 0; it0 < total; it0 += T) {
            const int it = it0 + tid;
            int c = -1, w = 0, z = 0;
            if (it < total) {
                const int o = piece_owner(s_off, owners, it);
                const int q = it - s_off[o];
                const unsigned run = (unsigned)s_a[o];
                c = q < (int)(run >> 16) ? (int)(run & 0xFFFFu) + q : s_b[o] + q;
                if (bm_test(dead, c)) c = -1;
            }
            if (c >= 0) {
                const int2 pa = __ldg(&g.palt[c]);  // pa.x, the tree parent, is deleted
                z = __ldg(&g.sz[c]);
                w = c;
                if (pa.y >= 0 && !bm_test(dead, pa.y)) {
                    w = pa.y;
                } else if (pa.y >= 0) {
                    for (int e = __ldg(&g.lo_ptr[c]) + 2, e1 = __ldg(&g.lo_ptr[c + 1]); e < e1; ++e) {
                        const int x = __ldg(&g.lo_col[e]);
                        if (!bm_test(dead, x)) {
                            w = x;
                            break;
                        }
                    }
                }
            }
            const int i = piece_append_slot(c >= 0, &scal[0]);
            if (c >= 0 && i < L.pcap) {
                pn[i] = (unsigned short)c;
                acc[i] = w;
                pu[i] = i;
                ps[i] = z;
                pst[i] = z;
            }
        }
        tm.sync();
    }
    const int np = scal[0];
    if (np > L.pcap) return false;
    // the table: piece root -> id
    for (int i = tid; i < np; i += T) {
        const int key = pn[i];
        const unsigned e = ((unsigned)key << 16) | (unsigned)i;
        const unsigned mask = (unsigned)hs - 1u;
        unsigned h = piece_hash(key, L.hbits);
        for (int probe = 0; probe < hs && atomicCAS(&hash[h], kPieceEmpty, e) != kPieceEmpty; ++probe)
            h = (h + 1) & mask;  // at most 3/4 of the slots are taken: an empty one is always reached
    }
    tm.sync();

    // 3. sizes by subtraction (one atomic per piece and warp: most go to the giant piece), then
    // the re-pick unions
    for (int r0 = 0; r0 < nd; r0 += T) {
        const int r = r0 + tid;
        int i = -1, v = 0;
        if (r < nd) {
            const unsigned e = dl[r];
            const int b = (int)(e >> 16);
            const int p = tp[b];
            if (p != b && !bm_test(dead, p)) {
                i = piece_lookup(hash, L.hbits, piece_walk(tp, dead, p));
                if (i < 0) scal[2] = 1;
                else v = -(int)((e & 0xFFFFu) + 1u);
            }
        }
        piece_class_add(ps, i < 0 ? 0 : i, v, i >= 0);
    }
    for (int i = tid; i < np; i += T) {
        const int w = acc[i];
        if (w == pn[i]) continue;
        const int j = piece_lookup(hash, L.hbits, piece_walk(tp, dead, w));
        if (j < 0) scal[2] = 1;
        else uf_unite(pu, i, j);
    }
    tm.sync();
    for (int i = tid; i < np; i += T) acc[i] = 0;
    tm.sync();
    if (scal[2]) {
        atomicOr(status, GAPA_DEV_CAPACITY);  // a piece root missing from the table: not expected
        return false;
    }

    // 4. class sizes; the giant class; the pieces outside it (listed in the distinct-deletion
    // slots, free now) and their preorder volume
    for (int i0 = 0; i0 < np; i0 += T) {
        const int i = i0 + tid;
        const bool on = i < np;
        piece_class_add(acc, on ? uf_find(pu, i) : 0, on ? ps[i] : 0, on);
    }
    tm.sync();
    long long key = -1;
    for (int i = tid; i < np; i += T)
        if (pu[i] == i) {
            const long long x = ((long long)acc[i] << 20) | (long long)(0xFFFFF - i);
            key = x > key ? x : key;
        }
    key = team_sum_ll(tm, key + 1, red, true);
    if (tid == 0) scal[3] = key > 0 ? 0xFFFFF - (int)((key - 1) & 0xFFFFF) : -1;
    tm.sync();
    const int giant = scal[3];
    long long vol = 0;
    for (int i0 = 0; i0 < np; i0 += T) {
        const int i = i0 + tid;
        const bool outside = i < np && uf_find(pu, i) != giant;
        if (i < np) acc[i] = outside;
        if (outside) vol += pst[i];
        const int slot = piece_append_slot(outside, &scal[4]);
        if (outside && slot < L.dcap) dl[slot] = (unsigned)i;
    }
    vol = team_sum_ll(tm, vol, red);
    if (tid == 0) scal[2] = vol > L.vcap || scal[4] > L.dcap;
    tm.sync();
    if (scal[2]) return false;
    const int nout = scal[4];

    // 5. the live nodes of the pieces outside the giant class: a first pass marks them in
    // `listed`, a second takes their arcs.  An arc to a live node that is not listed reaches the
    // giant class (flag 2 in the class-size slot, united below); an arc to a listed node of
    // another piece unites the two pieces' classes.  The pieces' preorder positions are dealt out
    // over the team; a node of more than 32 arcs has them split over the lanes of its warp.  When
    // the outside pieces fit one dealing of at most kPieceSlots rounds, the first pass keeps its
    // nodes in registers for the second.
    const bool keep = nout <= T;
    int kx[kPieceSlots], kp[kPieceSlots];
#pragma unroll
    for (int u = 0; u < kPieceSlots; ++u) kx[u] = -1;
    int rounds = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int o0 = 0; o0 < nout; o0 += T) {
            const int oi = o0 + tid;
            int cnt = 0, pi = 0;
            if (oi < nout) {
                pi = (int)dl[oi];
                cnt = pst[pi];
            }
            const int pre_c = cnt ? __ldg(&g.pre[pn[pi]]) : 0;
            int total;
            const int off = tree16l_scan(tm, cnt, ws, &total);
            s_off[tid] = off;
            s_a[tid] = pre_c;
            s_b[tid] = pi;
            tm.sync();
            const int owners = min(T, nout - o0);
            const bool kept = pass == 1 && keep && (total + T - 1) / T <= kPieceSlots;
            if (pass == 0) rounds = (total + T - 1) / T;
            for (int p0 = 0, u = 0; p0 < total; p0 += T, ++u) {
                int x = -1, xp = 0;
                if (kept) {
#pragma unroll
                    for (int v = 0; v < kPieceSlots; ++v)
                        if (v == u) {
                            x = kx[v];
                            xp = kp[v];
                        }
                } else {
                    const int it = p0 + tid;
                    if (it < total) {
                        const int o = piece_owner(s_off, owners, it);
                        xp = s_b[o];
                        x = __ldg(&g.at[s_a[o] + it - s_off[o]]);
                        if (bm_test(dead, x)) {
                            x = -1;
                        } else {
                            // x belongs to piece xp unless a deleted node lies between it and the root
                            const int top = pn[xp];
                            for (int y = x; y != top;) {
                                const int p = tp[y];
                                if (p == y) {  // a root other than the piece's: not its subtree
                                    scal[2] = 1;
                                    x = -1;
                                    break;
                                }
                                if (bm_test(dead, p)) {
                                    x = -1;
                                    break;
                                }
                                y = p;
                            }
                        }
                    }
                }
                if (pass == 0) {
                    if (x >= 0) atomicOr(&listed[x >> 5], 1u << (x & 31));
                    if (keep) {
#pragma unroll
                        for (int v = 0; v < kPieceSlots; ++v)
                            if (v == u) {
                                kx[v] = x;
                                kp[v] = xp;
                            }
                    }
                    continue;
                }
                int e0 = 0, deg = 0;
                if (x >= 0) {
                    e0 = __ldg(&g.fptr[x]);
                    deg = __ldg(&g.fptr[x + 1]) - e0;
                }
                const bool heavy = deg > 32;
                if (deg && !heavy)
                    piece_join_arcs(g, tp, dead, listed, hash, L.hbits, pu, acc, &scal[2], x, xp, e0, e0 + deg, 1);
                unsigned pending = __ballot_sync(0xffffffffu, heavy);
                while (pending) {  // the warp's heavy nodes, one at a time, arcs split over the lanes
                    const int src = __ffs(pending) - 1;
                    pending &= pending - 1;
                    const int xs = __shfl_sync(0xffffffffu, x, src);
                    const int pis = __shfl_sync(0xffffffffu, xp, src);
                    const int es = __shfl_sync(0xffffffffu, e0, src);
                    const int ds = __shfl_sync(0xffffffffu, deg, src);
                    piece_join_arcs(g, tp, dead, listed, hash, L.hbits, pu, acc, &scal[2], xs, pis, es + tm.tid % 32,
                                    es + ds, 32);
                }
            }
            tm.sync();
        }
    }
    (void)rounds;
    if (scal[2]) {
        atomicOr(status, GAPA_DEV_CAPACITY);
        return false;
    }
    for (int i = tid; i < np; i += T)
        if (acc[i] == 2) uf_unite(pu, i, giant);
    tm.sync();
    for (int i = tid; i < np; i += T) acc[i] = 0;
    tm.sync();
    for (int i0 = 0; i0 < np; i0 += T) {
        const int i = i0 + tid;
        const bool on = i < np;
        piece_class_add(acc, on ? uf_find(pu, i) : 0, on ? ps[i] : 0, on);
    }
    tm.sync();

    // 6. the objective over the classes and the untouched components
    long long obj = 0;
    for (int i = tid; i < np; i += T)
        if (pu[i] == i) obj = objective_add(obj, acc[i], g.objective);
    if (g.objective) {
        for (int r = tid; r < g.num_roots; r += T) {
            const int rt = __ldg(&g.roots[r]);
            if (__ldg(&g.crep[rt]) == rt && !bm_test(seen, rt)) obj = objective_add(obj, __ldg(&g.csize[rt]), 1);
        }
    } else {
        obj -= dirty;
    }
    obj = team_sum_ll(tm, obj, red, g.objective != 0);
    if (tid == 0) *out = g.objective ? obj : obj + g.tree_pc;
    tm.sync();
    return true;
}

}  // namespace gapa_dev
