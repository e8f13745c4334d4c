// Batched critical-node-detection fitness: for every population member, the
// pairwise connectivity of G with the member's genes deleted
// (Section III-C, Eq. 13: node deletion removes all incident edges; PC(G) of
// Table "Whole": sum over components C of |C|(|C|-1)/2).
//
// One CTA evaluates one member.  Labels live in shared memory when the graph
// fits (4 bytes per node), else in a global scratch slice per member.  The
// deletion set is encoded in the labels themselves (kDead), so no separate
// bitmap is kept.  Components are found by union-find with CAS hooking of the
// larger root under the smaller and path halving; sizes are counted into the
// root slots with warp-aggregated atomics; the int64 sum is reduced with
// warp shuffles.
#include <climits>
#include <mutex>

#include "gapa_internal.cuh"
#include "tree16.cuh"
#include "piece.cuh"

namespace {

constexpr int kDead = INT_MIN;
using gapa_dev::bm_test;
using gapa_dev::uf_find;
using gapa_dev::uf_root;
using gapa_dev::uf_unite;

__device__ __forceinline__ void edge_op(volatile int* lab, int u, int v) {
    if (lab[u] == kDead || lab[v] == kDead) return;
    uf_unite(lab, u, v);
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* red, bool mx = false) {
    const gapa_dev::Team tm{(int)threadIdx.x, (int)blockDim.x, 0};
    return gapa_dev::team_sum_ll(tm, v, red, mx);  // valid in thread 0
}

// Labels: every node its own root, then the perturbation P^(A, p) of Eq. 13
// marks the deleted nodes.
__device__ __forceinline__ void init_labels(volatile int* lab, int n, const int* __restrict__ genes, int k,
                                            int* status) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int v = tid; v < n; v += T) lab[v] = v;
    __syncthreads();
    for (int j = tid; j < k; j += T) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n)
            lab[d] = kDead;
        else
            atomicOr(status, GAPA_DEV_BAD_GENE);
    }
    __syncthreads();
}

// Hooking, plain: every undirected edge once, two edges per 16-byte load.
__device__ __forceinline__ void hook_all_edges(volatile int* lab, int num_edges, const int2* __restrict__ edges) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int pairs = num_edges >> 1;
    const int4* e4 = reinterpret_cast<const int4*>(edges);
    int q = tid;
    int4 w = q < pairs ? __ldg(&e4[q]) : make_int4(0, 0, 0, 0);
    while (q < pairs) {
        const int qn = q + T;
        const int4 wn = qn < pairs ? __ldg(&e4[qn]) : make_int4(0, 0, 0, 0);  // prefetch
        edge_op(lab, w.x, w.y);
        edge_op(lab, w.z, w.w);
        q = qn;
        w = wn;
    }
    if ((num_edges & 1) && tid == 0) {
        const int2 last = __ldg(&edges[num_edges - 1]);
        edge_op(lab, last.x, last.y);
    }
    __syncthreads();
}

// Hooking, sampled: (1) every live node is joined to its first kSample live
// neighbours in CSR order; (2) the tree of the first live probe node (the
// highest-degree nodes) is taken as the giant tree G; (3) every live node not
// in G joins all its live neighbours.  Exact: an edge {v,w} is either joined
// in (3) from an endpoint outside G, or both endpoints were seen inside G.
constexpr int kSample = 2;

__device__ __forceinline__ void hook_sampled(volatile int* lab, int n, const int* __restrict__ row_ptr,
                                             const int* __restrict__ col, const int* __restrict__ probe,
                                             int* sh_root) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int v = tid; v < n; v += T) {
        if (lab[v] == kDead) continue;
        const int beg = __ldg(&row_ptr[v]), end = __ldg(&row_ptr[v + 1]);
        int linked = 0;
        for (int e = beg; e < end && linked < kSample; ++e) {
            const int w = __ldg(&col[e]);
            if (lab[w] == kDead) continue;
            uf_unite(lab, v, w);
            ++linked;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int r = -1;
        for (int q = 0; q < kProbe && r < 0; ++q) {
            const int p = __ldg(&probe[q]);
            if (p < n && lab[p] != kDead) r = uf_root(lab, p);
        }
        *sh_root = r;
    }
    __syncthreads();
    const int giant = *sh_root;
    for (int v = tid; v < n; v += T) {
        if (lab[v] == kDead) continue;
        if (giant >= 0) {
            const int r = uf_find(lab, v);
            if (r == giant || r == uf_find(lab, giant)) continue;
        }
        const int beg = __ldg(&row_ptr[v]), end = __ldg(&row_ptr[v + 1]);
        for (int e = beg; e < end; ++e) {
            const int w = __ldg(&col[e]);
            if (lab[w] != kDead) uf_unite(lab, v, w);
        }
    }
    __syncthreads();
}

// Hooking, tree (32-bit ids; the 16-bit shared-memory pipeline is in
// tree16.cuh): labels start as the parents of a BFS spanning forest of G in
// BFS numbering (parent < child), so the forest already joins every live node
// to its live ancestors.  A live node whose tree parent is deleted takes its
// first live lower-numbered neighbour as parent instead (the top of a new
// piece only if there is none).  Each piece is flattened onto its top node,
// and the pieces are joined along the non-tree edges; an edge whose endpoints
// already share a label costs two shared-memory reads.
template <int kDeadV>
__device__ __forceinline__ void join_edge(volatile int* lab, int a, int b) {
    const int la = lab[a], lb = lab[b];
    if (la == lb || la == kDeadV || lb == kDeadV) return;
    uf_unite(lab, la, lb);
}

template <bool kPacked16, int kDeadV>
__device__ __forceinline__ void hook_tree(volatile int* lab, int n, const int* __restrict__ tparent,
                                          const int2* __restrict__ palt,
                                          const int* __restrict__ lo_ptr, const int* __restrict__ lo_col,
                                          const int* __restrict__ perm, const void* __restrict__ nontree,
                                          int num_nontree, const int* __restrict__ genes, int k, int* status) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int v = tid; v < n; v += T) lab[v] = __ldg(&tparent[v]);
    __syncthreads();
    // perturbation P^(A, p) of Eq. 13 in BFS numbering
    for (int j = tid; j < k; j += T) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n)
            lab[__ldg(&perm[d])] = kDeadV;
        else
            atomicOr(status, GAPA_DEV_BAD_GENE);
    }
    __syncthreads();
    // cut: a live node whose parent is deleted re-attaches to its first live
    // lower-numbered neighbour, or tops its own piece.  Deadness is final here,
    // so reading it while other slots change is safe.
    for (int v = tid; v < n; v += T) {
        const int p = lab[v];
        if (p == kDeadV || p == v || lab[p] != kDeadV) continue;
        int q = v;
        const int beg = __ldg(&lo_ptr[v]) + 1, end = __ldg(&lo_ptr[v + 1]);  // entry 0 is the tree parent
        for (int e = beg; e < end; ++e) {
            const int w = __ldg(&lo_col[e]);
            if (lab[w] != kDeadV) {
                q = w;
                break;
            }
        }
        lab[v] = q;
    }
    __syncthreads();
    // flatten every piece onto its top node (owner writes only)
    for (int v = tid; v < n; v += T) {
        const int p = lab[v];
        if (p != kDeadV && p != v) lab[v] = uf_root(lab, p);
    }
    __syncthreads();
    // join the pieces along the non-tree edges
    if (kPacked16) {
        const uint4* e4 = reinterpret_cast<const uint4*>(nontree);
        const int quads = num_nontree >> 2;
        int q = tid;
        uint4 w = q < quads ? __ldg(&e4[q]) : make_uint4(0, 0, 0, 0);
        while (q < quads) {
            const int qn = q + T;
            const uint4 wn = qn < quads ? __ldg(&e4[qn]) : make_uint4(0, 0, 0, 0);
            // all eight labels first, then the (rarely failing) comparisons
            const int a0 = (int)(w.x >> 16), b0 = (int)(w.x & 0xFFFFu), a1 = (int)(w.y >> 16), b1 = (int)(w.y & 0xFFFFu);
            const int a2 = (int)(w.z >> 16), b2 = (int)(w.z & 0xFFFFu), a3 = (int)(w.w >> 16), b3 = (int)(w.w & 0xFFFFu);
            const int la0 = lab[a0], lb0 = lab[b0], la1 = lab[a1], lb1 = lab[b1];
            const int la2 = lab[a2], lb2 = lab[b2], la3 = lab[a3], lb3 = lab[b3];
            if (la0 != lb0) join_edge<kDeadV>(lab, a0, b0);
            if (la1 != lb1) join_edge<kDeadV>(lab, a1, b1);
            if (la2 != lb2) join_edge<kDeadV>(lab, a2, b2);
            if (la3 != lb3) join_edge<kDeadV>(lab, a3, b3);
            q = qn;
            w = wn;
        }
        const unsigned* e1 = reinterpret_cast<const unsigned*>(nontree);
        for (int e = quads * 4 + tid; e < num_nontree; e += T) {
            const unsigned x = __ldg(&e1[e]);
            join_edge<kDeadV>(lab, (int)(x >> 16), (int)(x & 0xFFFFu));
        }
    } else {
        const int4* e4 = reinterpret_cast<const int4*>(nontree);
        const int pairs = num_nontree >> 1;
        int q = tid;
        int4 w = q < pairs ? __ldg(&e4[q]) : make_int4(0, 0, 0, 0);
        while (q < pairs) {
            const int qn = q + T;
            const int4 wn = qn < pairs ? __ldg(&e4[qn]) : make_int4(0, 0, 0, 0);
            join_edge<kDeadV>(lab, w.x, w.y);
            join_edge<kDeadV>(lab, w.z, w.w);
            q = qn;
            w = wn;
        }
        if ((num_nontree & 1) && tid == 0) {
            const int2 x = __ldg(reinterpret_cast<const int2*>(nontree) + (num_nontree - 1));
            join_edge<kDeadV>(lab, x.x, x.y);
        }
    }
    __syncthreads();
}

// Component sizes and the int64 sum of C(size, 2) (PC(G) of Table "Whole").
__device__ __forceinline__ void count_pc(volatile int* lab, int n, long long* out, long long* red, int objective) {
    const int tid = threadIdx.x, T = blockDim.x;
    // flatten: every live node points at its root
    for (int v = tid; v < n; v += T) {
        const int l = lab[v];
        if (l != kDead && l != v) lab[v] = uf_root(lab, l);
    }
    __syncthreads();
    // roots become counters: -1 for the root itself
    for (int v = tid; v < n; v += T)
        if (lab[v] == v) lab[v] = -1;
    __syncthreads();
    // every other live node adds itself to its root's counter (warp-aggregated)
    const int lane = tid & 31;
    for (int base = 0; base < n; base += T) {
        const int v = base + tid;
        int key = -1;
        if (v < n) {
            const int l = lab[v];
            if (l >= 0) key = l;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd((int*)&lab[key], -__popc(peers));
    }
    __syncthreads();
    // sum of C(size, 2) over roots
    long long acc = 0;
    for (int v = tid; v < n; v += T) {
        const int l = lab[v];
        if (l < 0 && l != kDead) acc = gapa_dev::objective_add(acc, -(long long)l, objective);
    }
    const long long tot = block_sum_ll(acc, red, objective != 0);
    if (tid == 0) *out = tot;
}

int smem_block_for(int n) {
    // enough threads to cover the graph, at most 1024; multiples of 32
    if (n <= 2048) return 256;
    if (n <= 8192) return 512;
    return 1024;
}

struct GraphArgs {
    int n, num_edges;
    const int2* edges;
    const int* row_ptr;
    const int* col;
    const int* probe;
    const int* perm;
    const int* tparent;
    const int* lo_ptr;
    const int* lo_col;
    const int2* palt;
    const void* nontree;
    int num_nontree;
    const int* fptr;
    const unsigned short* fcol16;
    int join_mode;
    int mean_deg_x16;
    int objective;
    const int4* kids;
    const int* roots;
    int num_roots;
    int list_bytes;
    const unsigned* est;  // cut-local kernel: per-member cost estimates (may be null)
    DeviceForest alt;     // cut-local kernel: the second forest (alt.perm null: none)
};

enum Variant : int { V_EDGES = 0, V_SAMPLED = 1, V_TREE16 = 2, V_TREE32 = 3, V_TREE16L = 4 };

template <int kVar>
__device__ __forceinline__ void member_pc(volatile int* lab, const GraphArgs& g, const int* __restrict__ genes, int k, int m,
                                          long long* out, int* status, long long* red, int* sh_root,
                                          bool use_alt = false) {
    if (kVar == V_TREE16 || kVar == V_TREE16L) {
        // the whole CTA is one team; the deleted-node bitmap sits right after the labels
        const gapa_dev::Team tm{(int)threadIdx.x, (int)blockDim.x, 0};
        // the cut-local kernel leaves members expected to list over a quarter of the nodes (the
        // BFS tree shattered) to the full pipeline from the start
        const bool full = kVar == V_TREE16 || (g.est && __ldg(&g.est[m]) > (unsigned)(g.n / 4));
        unsigned* region = (unsigned*)(lab + gapa_dev::tree16l_lab_ints(g.n));
        int* scal = (int*)region + g.list_bytes / 4;
        if (kVar == V_TREE16L && use_alt && !full) {
            // the second forest: the same graph in its own numbering (its own constant record, so
            // that every field stays a kernel-parameter read)
            const DeviceForest& a = g.alt;
            const gapa_dev::Tree16Graph tb{g.n,           a.perm,          a.palt,          a.lo_ptr,
                                           a.lo_col,      a.nontree,       a.num_nontree,   a.fptr,
                                           a.fcol16,      g.join_mode,     g.mean_deg_x16,  g.objective,
                                           a.tparent,     a.kids,          a.roots,         a.num_roots,
                                           g.list_bytes};
            gapa_dev::tree16_member_local(tm, lab, region, scal, tb, genes, k, out, red, status);
            return;
        }
        const gapa_dev::Tree16Graph t16{g.n,           g.perm,          g.palt,          g.lo_ptr,
                                        g.lo_col,      (const unsigned*)g.nontree,      g.num_nontree,
                                        g.fptr,        g.fcol16,        g.join_mode,     g.mean_deg_x16,
                                        g.objective,   g.tparent,       g.kids,          g.roots,
                                        g.num_roots,   g.list_bytes};
        if (full)
            gapa_dev::tree16_member(tm, lab, (unsigned*)(lab + g.n), t16, genes, k, out, red, status);
        else
            gapa_dev::tree16_member_local(tm, lab, region, scal, t16, genes, k, out, red, status);
        return;
    }
    if (kVar == V_TREE32) {
        hook_tree<false, kDead>(lab, g.n, g.tparent, g.palt, g.lo_ptr, g.lo_col, g.perm,
                                g.nontree, g.num_nontree, genes, k, status);
    } else {
        init_labels(lab, g.n, genes, k, status);
        if (kVar == V_SAMPLED)
            hook_sampled(lab, g.n, g.row_ptr, g.col, g.probe, sh_root);
        else
            hook_all_edges(lab, g.num_edges, g.edges);
    }
    count_pc(lab, g.n, out, red, g.objective);
}

// Edge genes: every node stays; a member's genes are edge ids (CSR order of
// the edges {u, v}, u < v, the order of g.edges) whose edges are removed.
// Labels and the removed-edge mask in shared memory; union-find over the
// remaining edges, then the sizes and the objective.
__global__ void __launch_bounds__(1024) cc_edge_genes_kernel(GraphArgs g, const int* __restrict__ pop, int k,
                                                             long long* __restrict__ fit, int* status) {
    extern __shared__ int smem_lab[];
    __shared__ long long red[32];
    volatile int* lab = smem_lab;
    unsigned* gone = reinterpret_cast<unsigned*>(smem_lab + g.n);
    const int tid = threadIdx.x, T = blockDim.x;
    const int words = (g.num_edges + 31) >> 5;
    const int* genes = pop + (size_t)blockIdx.x * k;
    for (int v = tid; v < g.n; v += T) lab[v] = v;
    for (int w = tid; w < words; w += T) gone[w] = 0u;
    __syncthreads();
    for (int j = tid; j < k; j += T) {
        const int e = __ldg(&genes[j]);
        if ((unsigned)e < (unsigned)g.num_edges)
            atomicOr(&gone[e >> 5], 1u << (e & 31));
        else
            atomicOr(status, GAPA_DEV_BAD_GENE);
    }
    __syncthreads();
    for (int e = tid; e < g.num_edges; e += T) {
        if ((gone[e >> 5] >> (e & 31)) & 1u) continue;
        const int2 ed = __ldg(&g.edges[e]);
        if (lab[ed.x] != lab[ed.y]) uf_unite(lab, ed.x, ed.y);
    }
    __syncthreads();
    count_pc(lab, g.n, &fit[blockIdx.x], red, g.objective);
}

size_t edge_genes_smem(int n, int num_edges) { return (size_t)n * 4 + (size_t)((num_edges + 31) / 32) * 4; }

// One CTA per member, labels in shared memory; with `order`, CTA i takes
// member order[i] (CTAs start roughly in index order, so the members
// expected to be costliest start first and the launch has no long tail).
template <int kVar>
__global__ void __launch_bounds__(1024) cc_smem_kernel(GraphArgs g, const int* __restrict__ pop, int k,
                                                       long long* __restrict__ fit, int* status,
                                                       const int* __restrict__ order) {
    extern __shared__ int smem_lab[];
    __shared__ long long red[32];
    __shared__ int sh_root;
    const int e = order ? __ldg(&order[blockIdx.x]) : (int)blockIdx.x;
    const int i = e & 0x3FFFFFFF;  // bit 30: evaluate on the second forest
    member_pc<kVar>(smem_lab, g, pop + (size_t)i * k, k, i, &fit[i], status, red, &sh_root, (e >> 30) & 1);
}

// Cost estimate of every member for the cut-local kernel under each forest:
// the sum over its genes of the nodes that deleting the gene alone leaves in
// pieces to be listed (cost tables by original node id; one 128-thread CTA
// per member, four genes in flight per thread; saturates at 2^31 - 1).
// cut2 null: one forest.
__global__ void __launch_bounds__(128) local_cost_kernel(const int* __restrict__ pop, int k, int n,
                                                         const int* __restrict__ cut, const int* __restrict__ cut2,
                                                         unsigned* __restrict__ est, unsigned* __restrict__ est2) {
    __shared__ long long part[2][4];
    const int m = blockIdx.x, t = threadIdx.x;
    const int* genes = pop + (size_t)m * k;
    long long c = 0, c2 = 0;
    int j = t;
    for (; j + 384 < k; j += 512) {
        int d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = __ldg(&genes[j + 128 * u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = (unsigned)d[u] < (unsigned)n;
            c += ok ? __ldg(&cut[d[u]]) : 0;
            c2 += ok && cut2 ? __ldg(&cut2[d[u]]) : 0;
        }
    }
    for (; j < k; j += 128) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n) {
            c += __ldg(&cut[d]);
            if (cut2) c2 += __ldg(&cut2[d]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        c2 += __shfl_down_sync(0xffffffffu, c2, o);
    }
    if ((t & 31) == 0) {
        part[0][t >> 5] = c;
        part[1][t >> 5] = c2;
    }
    __syncthreads();
    if (t == 0) {
        const long long s1 = (part[0][0] + part[0][1]) + (part[0][2] + part[0][3]);
        const long long s2 = (part[1][0] + part[1][1]) + (part[1][2] + part[1][3]);
        est[m] = (unsigned)(s1 < 0x7FFFFFFFll ? s1 : 0x7FFFFFFFll);
        est2[m] = cut2 ? (unsigned)(s2 < 0x7FFFFFFFll ? s2 : 0x7FFFFFFFll) : 0xFFFFFFFFu;
    }
}

// Members by decreasing bit length of their lower estimate (a counting sort
// over the 33 values of its count of leading zeros, in one CTA; the order
// within a class is arbitrary).  order[i] = member | 1 << 30 when the second
// forest has the lower estimate; est_min[m] = the lower estimate.
__global__ void __launch_bounds__(1024) local_order_kernel(const unsigned* __restrict__ est,
                                                           const unsigned* __restrict__ est2, int s,
                                                           int* __restrict__ order, unsigned* __restrict__ est_min) {
    __shared__ int cnt[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < s; m += blockDim.x) {
        const unsigned a = est[m], b = est2[m], e = b < a ? b : a;
        est_min[m] = e;
        atomicAdd(&cnt[__clz(e)], 1);
    }
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
    for (int m = threadIdx.x; m < s; m += blockDim.x) {
        const unsigned e = est_min[m];
        order[atomicAdd(&cnt[__clz(e)], 1)] = m | (est2[m] < est[m] ? (1 << 30) : 0);
    }
}

// One CTA per member, labels in a global scratch slice per CTA.
template <int kVar>
__global__ void __launch_bounds__(1024) cc_global_kernel(GraphArgs g, const int* __restrict__ pop, int k,
                                                         long long* __restrict__ fit, int* status, int* labels,
                                                         int member_base) {
    __shared__ long long red[32];
    __shared__ int sh_root;
    const int i = member_base + blockIdx.x;
    member_pc<kVar>(labels + (size_t)blockIdx.x * g.n, g, pop + (size_t)i * k, k, i, &fit[i], status, red, &sh_root);
}

// Forest-piece kernel: a persistent CTA of kPieceTeams teams of kPieceThreads threads per SM.
// The CTA serves one forest: it copies that forest's parents (16-bit) into shared memory, then
// every team takes members of that forest from the forest's queue (costliest first) and
// evaluates them (piece.cuh).  Members that exceed the teams' capacities are appended to `defer`
// for cc_list_kernel.  ctl: [0] deferred count, [1] [2] members per forest, [3] [4] queue heads.
constexpr int kPieceThreads = 256;
constexpr int kPieceTeams = 4;

struct PieceArgs {
    gapa_dev::PieceGraph g1, g2;
    gapa_dev::PieceLayout L;
};

__global__ void __launch_bounds__(kPieceThreads* kPieceTeams, 1)
    cc_piece_kernel(PieceArgs a, const int* __restrict__ pop, int k, long long* __restrict__ fit, int* status,
                    const int* __restrict__ list, int* __restrict__ defer, int* ctl) {
    extern __shared__ __align__(16) unsigned char smem_piece[];
    __shared__ int team_next[kPieceTeams];
    const int c1 = __ldcg(&ctl[1]), c2 = __ldcg(&ctl[2]), total = c1 + c2;
    // the first g1 CTAs serve the first forest (at least one CTA per forest with members)
    int g1 = (int)(((long long)gridDim.x * c1 + total / 2) / (total > 0 ? total : 1));
    if (c1 > 0 && g1 < 1) g1 = 1;
    if (c2 > 0 && g1 > (int)gridDim.x - 1) g1 = (int)gridDim.x - 1;
    if (c2 == 0) g1 = gridDim.x;
    const int f = (int)blockIdx.x < g1 ? 0 : 1;
    const gapa_dev::PieceGraph& g = f ? a.g2 : a.g1;
    const int count = f ? c2 : c1;
    const int* flist = list + (f ? c1 : 0);
    unsigned short* tp = reinterpret_cast<unsigned short*>(smem_piece);
    for (int v = threadIdx.x; v < g.n; v += blockDim.x) tp[v] = (unsigned short)__ldg(&g.tparent[v]);
    __syncthreads();
    const int team = threadIdx.x / kPieceThreads;
    const gapa_dev::Team tm{(int)threadIdx.x - team * kPieceThreads, kPieceThreads, 1 + team};
    unsigned char* tsm = smem_piece + gapa_dev::piece_parents_bytes(g.n) + (size_t)team * a.L.bytes;
    while (true) {
        if (tm.tid == 0) team_next[team] = atomicAdd(&ctl[3 + f], 1);
        tm.sync();
        const int idx = team_next[team];
        tm.sync();
        if (idx >= count) break;
        const int e = __ldg(&flist[idx]);
        const int m = e & 0x3FFFFFFF;
        const bool done = gapa_dev::piece_member(tm, g, a.L, tsm, tp, pop + (size_t)m * k, k, &fit[m], status);
        if (!done && tm.tid == 0) defer[atomicAdd(&ctl[0], 1)] = e;
    }
}

// Members by forest (the one with the lower estimate; the first forest on ties), and within each
// forest by decreasing bit length of the estimate (a counting sort over 2 x 33 classes in one CTA;
// the order within a class is arbitrary); est_min[m] = the lower estimate.  Also resets the
// forest-piece kernel's counters (see cc_piece_kernel).
__global__ void __launch_bounds__(1024) piece_order_kernel(const unsigned* __restrict__ est,
                                                           const unsigned* __restrict__ est2, int s,
                                                           int* __restrict__ order, unsigned* __restrict__ est_min,
                                                           int* __restrict__ ctl) {
    __shared__ int cnt[66];
    if (threadIdx.x < 66) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int m = threadIdx.x; m < s; m += blockDim.x) {
        const unsigned a = est[m], b = est2[m];
        const bool second = b < a;
        const unsigned e = second ? b : a;
        est_min[m] = e;
        atomicAdd(&cnt[33 * second + __clz(e)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < 66; ++c) {
            const int x = cnt[c];
            cnt[c] = acc;
            acc += x;
            if (c == 32) ctl[1] = acc;
        }
        ctl[2] = acc - ctl[1];
        ctl[0] = 0;
        ctl[3] = 0;
        ctl[4] = 0;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < s; m += blockDim.x) {
        const unsigned a = est[m], b = est2[m];
        const bool second = b < a;
        order[atomicAdd(&cnt[33 * second + __clz(second ? b : a)], 1)] = m | (second ? (1 << 30) : 0);
    }
}

// The deferred members, with the cut-local TREE kernel (which runs the full pipeline for members
// estimated to list over a quarter of the nodes): CTAs stride over list[0 .. *count).
template <int kVar>
__global__ void __launch_bounds__(1024) cc_list_kernel(GraphArgs g, const int* __restrict__ pop, int k,
                                                       long long* __restrict__ fit, int* status,
                                                       const int* __restrict__ list, const int* count) {
    extern __shared__ int smem_lab[];
    __shared__ long long red[32];
    __shared__ int sh_root;
    const int cnt = *count;
    for (int x = blockIdx.x; x < cnt; x += gridDim.x) {
        const int e = list[x];
        const int i = e & 0x3FFFFFFF;
        member_pc<kVar>(smem_lab, g, pop + (size_t)i * k, k, i, &fit[i], status, red, &sh_root, (e >> 30) & 1);
        __syncthreads();  // the shared memory is reused by the next member
    }
}

template <int kVar>
int launch_variant(gapa_ctx* c, const GraphArgs& ga, const int32_t* pop, int s, int k, long long* f,
                   cudaStream_t st, int* kernels = nullptr, const unsigned* est_in = nullptr) {
    const int n = ga.n;
    const size_t lab_bytes = kVar == V_TREE16    ? gapa_dev::tree16_smem_bytes(n)
                             : kVar == V_TREE16L ? gapa_dev::tree16l_smem_bytes(n, (size_t)ga.list_bytes)
                                                 : (size_t)n * 4;
    if (lab_bytes <= c->fit_smem_max) {
        const int* order = nullptr;
        unsigned* est_min = nullptr;
        if (kVar == V_TREE16L && s > 1 && s <= kOrderCap) {
            // estimates under both forests (precomputed by the operator kernel, or here), then the order
            unsigned* e1 = gapa_estimate_buffer(c);
            unsigned* e2 = e1 + kOrderCap;
            est_min = e2 + kOrderCap;
            if (!est_in) {
                const bool alt = c->g.has_alt;
                local_cost_kernel<<<s, 128, 0, st>>>(pop, k, n, c->g.cut, alt ? c->g.alt.cut : nullptr, e1, e2);
                if (kernels) *kernels += 1;
            }
            const unsigned* a = est_in ? est_in : e1;
            local_order_kernel<<<1, 1024, 0, st>>>(a, a + kOrderCap, s, c->g.order, est_min);
            order = c->g.order;
            if (kernels) *kernels += 1;
        }
        GraphArgs gl = ga;
        gl.est = est_min;
        cc_smem_kernel<kVar><<<s, smem_block_for(n), lab_bytes, st>>>(gl, pop, k, f, c->status, order);
        GAPA_CUDA(cudaGetLastError());
        return GAPA_OK;
    }
    if constexpr (kVar == V_TREE16 || kVar == V_TREE16L) {
        // 16-bit ids are chosen at upload only when the labels fit in shared memory
        return gapa_fail(GAPA_ERR_STATE, "16-bit tree labels need shared memory");
    } else {
        int rc = gapa_fitness_prepare(c, s);
        if (rc != GAPA_OK) return rc;
        const int wave = (int)(c->labels_cap / (size_t)n);
        for (int base = 0; base < s; base += wave) {
            const int cnt = s - base < wave ? s - base : wave;
            cc_global_kernel<kVar><<<cnt, 1024, 0, st>>>(ga, pop, k, f, c->status, c->labels, base);
            GAPA_CUDA(cudaGetLastError());
        }
        return GAPA_OK;
    }
}


gapa_dev::PieceGraph piece_graph(const gapa_ctx* c, bool second) {
    const DeviceGraph& g = c->g;
    gapa_dev::PieceGraph p{};
    p.n = g.n;
    p.tree_pc = g.tree_pc;
    p.objective = c->objective;
    if (!second) {
        p.perm = g.perm;
        p.tparent = g.tparent;
        p.palt = g.palt;
        p.lo_ptr = g.lo_ptr;
        p.lo_col = g.lo_col;
        p.fptr = g.fptr;
        p.fcol = g.fcol16;
        p.kids = g.kids;
        p.sz = g.sz;
        p.pre = g.pre;
        p.at = g.at;
        p.crep = g.crep;
        p.nroot = g.nroot;
        p.csize = g.csize;
        p.roots = g.roots;
        p.num_roots = g.num_roots;
    } else {
        const DeviceForest& a = g.alt;
        p.perm = a.perm;
        p.tparent = a.tparent;
        p.palt = a.palt;
        p.lo_ptr = a.lo_ptr;
        p.lo_col = a.lo_col;
        p.fptr = a.fptr;
        p.fcol = a.fcol16;
        p.kids = a.kids;
        p.sz = a.sz;
        p.pre = a.pre;
        p.at = a.at;
        p.crep = a.crep;
        p.nroot = a.nroot;
        p.csize = a.csize;
        p.roots = a.roots;
        p.num_roots = a.num_roots;
    }
    return p;
}

// The fitness phase with the forest-piece kernel: estimates (unless the operator kernel wrote
// them), the order by forest and cost, the piece kernel, then the deferred members.  Falls back to
// the cut-local TREE kernel when the layout does not fit.
int launch_piece(gapa_ctx* c, const GraphArgs& ga, const int32_t* pop, int s, int k, long long* f, cudaStream_t st,
                 int* kernels, const unsigned* est_in) {
    const int n = ga.n;
    const size_t parents = gapa_dev::piece_parents_bytes(n);
    const size_t avail = c->piece_smem_max > parents ? c->piece_smem_max - parents : 0;
    const gapa_dev::PieceLayout L = gapa_dev::piece_layout(n, k, kPieceThreads, avail / kPieceTeams);
    const size_t lab_bytes = gapa_dev::tree16l_smem_bytes(n, (size_t)ga.list_bytes);
    if (L.pcap < 512 || s < 2 || s > kOrderCap || lab_bytes > c->fit_smem_max)
        return launch_variant<V_TREE16L>(c, ga, pop, s, k, f, st, kernels, est_in);
    unsigned* e1 = gapa_estimate_buffer(c);
    unsigned* e2 = e1 + kOrderCap;
    unsigned* est_min = e2 + kOrderCap;
    int* defer = c->g.order + 4 * kOrderCap;
    int* ctl = defer + kOrderCap;
    if (!est_in) {
        local_cost_kernel<<<s, 128, 0, st>>>(pop, k, n, c->g.cut, c->g.has_alt ? c->g.alt.cut : nullptr, e1, e2);
        if (kernels) *kernels += 1;
    }
    const unsigned* a = est_in ? est_in : e1;
    piece_order_kernel<<<1, 1024, 0, st>>>(a, a + kOrderCap, s, c->g.order, est_min, ctl);
    PieceArgs pa;
    pa.g1 = piece_graph(c, false);
    pa.g2 = c->g.has_alt ? piece_graph(c, true) : pa.g1;
    pa.L = L;
    const int grid = std::max(2, std::min(c->num_sms, (s + kPieceTeams - 1) / kPieceTeams));
    const size_t bytes = parents + (size_t)kPieceTeams * L.bytes;
    cc_piece_kernel<<<grid, kPieceThreads * kPieceTeams, bytes, st>>>(pa, pop, k, f, c->status, c->g.order, defer,
                                                                       ctl);
    GAPA_CUDA(cudaGetLastError());
    GraphArgs gl = ga;
    gl.est = est_min;
    cc_list_kernel<V_TREE16L><<<std::min(s, 2 * c->num_sms), smem_block_for(n), lab_bytes, st>>>(gl, pop, k, f,
                                                                                               c->status, defer, ctl);
    GAPA_CUDA(cudaGetLastError());
    if (kernels) *kernels += 3;
    return GAPA_OK;
}

}  // namespace

// The sparse kernel: on request, and by AUTO where the labels exceed shared memory.
static bool sparse_selected(const gapa_ctx* c) {
    return c->g.sp_nforests > 0 &&
           (c->fitness_variant == GAPA_FITNESS_SPARSE ||
            (c->fitness_variant == GAPA_FITNESS_AUTO && !c->g.packed16 && (size_t)c->g.n * 4 > c->fit_smem_max));
}

int gapa_fitness_prepare(gapa_ctx* c, int s) {
    const size_t lab_bytes = (size_t)c->g.n * 4;
    const bool tree = c->fitness_variant != GAPA_FITNESS_EDGES && c->fitness_variant != GAPA_FITNESS_SAMPLED;
    if (sparse_selected(c)) {
        int rc = gapa_sparse_prepare(c, s);
        if (rc != GAPA_OK) return rc;
    }
    if (tree) return (c->g.packed16 || lab_bytes <= c->fit_smem_max) ? GAPA_OK : gapa_ig_prepare(c, s);
    if (lab_bytes <= c->fit_smem_max) return GAPA_OK;
    // global labels: process members in waves of at most `wave` CTAs
    const size_t wave = (size_t)(s < 4 * c->num_sms ? s : 4 * c->num_sms);
    return gapa_reserve((void**)&c->labels, &c->labels_cap, wave * (size_t)c->g.n, sizeof(int));
}

int gapa_fitness_block_for(int n) { return smem_block_for(n); }

namespace {
// Read-bandwidth probe: 16-byte loads over the buffer, grid-strided, four in
// flight per thread; one word per CTA keeps the loads live.
__global__ void __launch_bounds__(256) read_probe_kernel(const uint4* __restrict__ buf, size_t n16, int passes,
                                                         unsigned* __restrict__ sink) {
    unsigned acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(&buf[i]), b = __ldcg(&buf[i + stride]), c = __ldcg(&buf[i + 2 * stride]),
                        d = __ldcg(&buf[i + 3 * stride]);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(&buf[i]);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(&sink[blockIdx.x], acc);
}
}  // namespace

int gapa_launch_read_probe(const void* buf, size_t bytes, int passes, int grid, unsigned* sink, cudaStream_t st) {
    read_probe_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const uint4*>(buf), bytes / 16, passes, sink);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

// AUTO picks the cut-local kernel above this many nodes: on smaller graphs the full pipeline is as
// fast or faster (whole 100-generation runs: 40.5k against 34.0k generations/s at n = 1000, even at
// n = 2000, 1.12-1.31 x for the cut-local kernel from n = 4000 to 12000)
static constexpr int kLocalAutoMinNodes = 2049;

static bool local_selected(const gapa_ctx* c) {
    return c->g.packed16 && c->g.local_list_bytes > 0 &&
           ((c->fitness_variant == GAPA_FITNESS_AUTO && c->g.n >= kLocalAutoMinNodes) ||
            c->fitness_variant == GAPA_FITNESS_TREE_LOCAL);
}

// The forest-piece kernel: by request only (it needs the cut-local kernel's forests and cost tables).
static bool piece_selected(const gapa_ctx* c) {
    return c->g.packed16 && c->g.local_list_bytes > 0 && c->g.sz && c->fitness_variant == GAPA_FITNESS_PIECE;
}

bool gapa_fitness_uses_estimates(const gapa_ctx* c, int s) {
    return (local_selected(c) || piece_selected(c)) && s > 1 && s <= kOrderCap && c->genes == GAPA_GENES_NODES &&
           (c->objective == GAPA_OBJECTIVE_PC || c->objective == GAPA_OBJECTIVE_MCN);
}

unsigned* gapa_estimate_buffer(gapa_ctx* c) { return reinterpret_cast<unsigned*>(c->g.order + kOrderCap); }

int gapa_launch_fitness(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                        const unsigned* est) {
    if (s <= 0) return GAPA_OK;
    ProfileScope prof(c, st, 0, s);
    const int n = c->g.n;
    long long* f = reinterpret_cast<long long*>(fit);
    GraphArgs ga;
    ga.n = n;
    ga.num_edges = c->g.num_edges;
    ga.edges = c->g.edges;
    ga.row_ptr = c->g.row_ptr;
    ga.col = c->g.col;
    ga.probe = c->g.probe;
    ga.perm = c->g.perm;
    ga.tparent = c->g.tparent;
    ga.lo_ptr = c->g.lo_ptr;
    ga.lo_col = c->g.lo_col;
    ga.palt = c->g.palt;
    ga.nontree = c->g.nontree;
    ga.num_nontree = c->g.num_nontree;
    ga.fptr = c->g.fptr;
    ga.fcol16 = c->g.fcol16;
    ga.join_mode = c->fitness_variant == GAPA_FITNESS_TREE_JOIN ? 1 : c->fitness_variant == GAPA_FITNESS_TREE_SCAN ? 2 : 0;
    ga.mean_deg_x16 = c->g.mean_deg_x16;
    ga.objective = c->objective;
    ga.kids = c->g.kids;
    ga.roots = c->g.roots;
    ga.num_roots = c->g.num_roots;
    ga.list_bytes = c->g.local_list_bytes;
    ga.est = nullptr;
    ga.alt = c->g.alt;
    if (c->objective == GAPA_OBJECTIVE_SIXDST_PC || c->objective == GAPA_OBJECTIVE_SIXDST_MCN) {
        if (c->genes != GAPA_GENES_NODES) return gapa_fail(GAPA_ERR_INVALID_ARG, "SixDST objectives take node genes");
        return gapa_launch_fitness_sixdst(c, pop, s, k, fit, st, &prof.kernels);
    }
    if (c->genes == GAPA_GENES_EDGES) {
        const size_t bytes = edge_genes_smem(n, c->g.num_edges);
        if (bytes > c->fit_smem_max)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "edge genes: labels and edge mask (%zu bytes) exceed shared memory",
                             bytes);
        cc_edge_genes_kernel<<<s, smem_block_for(n), bytes, st>>>(ga, pop, k, f, c->status);
        GAPA_CUDA(cudaGetLastError());
        return GAPA_OK;
    }
    if (sparse_selected(c) && gapa_sparse_fits(c, k)) return gapa_launch_fitness_sparse(c, pop, s, k, fit, st, &prof.kernels);
    switch (c->fitness_variant) {
        case GAPA_FITNESS_EDGES:
            return launch_variant<V_EDGES>(c, ga, pop, s, k, f, st);
        case GAPA_FITNESS_SAMPLED:
            return launch_variant<V_SAMPLED>(c, ga, pop, s, k, f, st);
        default:
            if (c->g.packed16) {
                if (piece_selected(c) && c->objective <= GAPA_OBJECTIVE_MCN)
                    return launch_piece(c, ga, pop, s, k, f, st, &prof.kernels, est);
                if (local_selected(c)) return launch_variant<V_TREE16L>(c, ga, pop, s, k, f, st, &prof.kernels, est);
                return launch_variant<V_TREE16>(c, ga, pop, s, k, f, st);
            }
            if ((size_t)n * 4 <= c->fit_smem_max) return launch_variant<V_TREE32>(c, ga, pop, s, k, f, st);
            // labels too large for shared memory: interleaved member groups in global memory
            return gapa_launch_fitness_ig(c, pop, s, k, fit, st, &prof.kernels);
    }
}

int gapa_fitness_kernels_init(gapa_ctx* c) {
    int rc = gapa_set_smem_limit((const void*)cc_smem_kernel<V_EDGES>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_smem_kernel<V_SAMPLED>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_smem_kernel<V_TREE16>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_smem_kernel<V_TREE16L>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_list_kernel<V_TREE16L>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_piece_kernel, c->smem_optin, &c->piece_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_smem_kernel<V_TREE32>, c->smem_optin, &c->fit_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)cc_edge_genes_kernel, c->smem_optin, &c->fit_smem_max);
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free fitness (gapa_fitness_noalloc).
//
// For callers that must not allocate device memory: latency-critical loops
// that cannot take cudaMalloc's implicit synchronisation, and processes whose
// device memory is owned by another allocator under a fixed budget.  The call
// blocks (it reads the status word back and synchronises the stream).  The
// caller passes the graph as a device edge list and the population and output
// as device arrays; the label scratch is the file-scope array below, which
// every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocLabels = (size_t)GAPA_NOALLOC_MAX_LABELS;  // 8 Mi int32 = 32 MiB
__device__ __align__(256) int g_noalloc_labels[kNoAllocLabels];
__device__ int g_noalloc_status;

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int* g_noalloc_labels_addr[kNoAllocMaxDevices];
int* g_noalloc_status_addr[kNoAllocMaxDevices];

// Union-find over a caller-supplied edge list (pairs of int32), every
// endpoint checked against [0, n) because the list was not validated.
__device__ __forceinline__ void hook_edge_list_checked(volatile int* lab, int n, int num_edges,
                                                       const int* __restrict__ edges, int* status) {
    for (int e = threadIdx.x; e < num_edges; e += blockDim.x) {
        const int u = __ldg(&edges[2 * (size_t)e]), v = __ldg(&edges[2 * (size_t)e + 1]);
        if ((unsigned)u >= (unsigned)n || (unsigned)v >= (unsigned)n) {
            atomicOr(status, GAPA_DEV_BAD_EDGE);
            continue;
        }
        if (u != v) edge_op(lab, u, v);
    }
    __syncthreads();
}

// One CTA per member; labels in the static scratch, slice blockIdx.x of the wave.
__global__ void __launch_bounds__(1024) cc_noalloc_kernel(int n, int num_edges, const int* __restrict__ edges,
                                                          const int* __restrict__ pop, int k,
                                                          long long* __restrict__ fit, int* status, int* labels,
                                                          int member_base) {
    __shared__ long long red[32];
    const int i = member_base + blockIdx.x;
    volatile int* lab = labels + (size_t)blockIdx.x * n;
    init_labels(lab, n, pop + (size_t)i * k, k, status);
    hook_edge_list_checked(lab, n, num_edges, edges, status);
    count_pc(lab, n, &fit[i], red, 0);  // pairwise connectivity
}

// Device addresses of the static arrays on the current device, looked up once.
int noalloc_setup(int dev, int** labels, int** status) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return gapa_fail(GAPA_ERR_INVALID_ARG, "device %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_labels_addr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_labels);
        if (e != cudaSuccess) return gapa_cuda_fail(e, "cudaGetSymbolAddress(label scratch)");
        e = cudaGetSymbolAddress(&b, g_noalloc_status);
        if (e != cudaSuccess) return gapa_cuda_fail(e, "cudaGetSymbolAddress(status word)");
        g_noalloc_labels_addr[dev] = (int*)a;
        g_noalloc_status_addr[dev] = (int*)b;
    }
    *labels = g_noalloc_labels_addr[dev];
    *status = g_noalloc_status_addr[dev];
    return GAPA_OK;
}

}  // namespace

extern "C" int gapa_fitness_noalloc(int device, void* cuda_stream, int32_t n, int32_t num_edges,
                                    const int32_t* edges_dev, const int32_t* pop_dev, int32_t s, int32_t k,
                                    int64_t* fit_dev) {
    if (n < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "n must be >= 1 (got %d)", n);
    if ((size_t)n > kNoAllocLabels)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "n = %d exceeds the static scratch of %zu labels", n, kNoAllocLabels);
    if (num_edges < 0 || s < 0 || k < 0) return gapa_fail(GAPA_ERR_INVALID_ARG, "negative size");
    if ((long long)s * k >= (1LL << 31)) return gapa_fail(GAPA_ERR_INVALID_ARG, "s*k must be below 2^31");
    if (s == 0) return GAPA_OK;
    if (!fit_dev || (k > 0 && !pop_dev) || (num_edges > 0 && !edges_dev))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return gapa_fail(GAPA_ERR_CUDA, "cudaGetDevice failed");
    if (prev != device) {
        const cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return gapa_cuda_fail(e, "cudaSetDevice");
    }
    auto restore = [&](int rc) {
        if (prev != device) cudaSetDevice(prev);
        return rc;
    };
    int* labels = nullptr;
    int* status = nullptr;
    int rc = noalloc_setup(device, &labels, &status);
    if (rc != GAPA_OK) return restore(rc);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return restore(gapa_cuda_fail(e, "clearing the status word"));
    const int wave = (int)(kNoAllocLabels / (size_t)n);
    for (int base = 0; base < s; base += wave) {
        const int cnt = s - base < wave ? s - base : wave;
        cc_noalloc_kernel<<<cnt, 1024, 0, st>>>(n, num_edges, edges_dev, pop_dev, k,
                                                 reinterpret_cast<long long*>(fit_dev), status, labels, base);
        e = cudaGetLastError();
        if (e != cudaSuccess) return restore(gapa_cuda_fail(e, "cc_noalloc_kernel launch"));
    }
    int h = 0;
    e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return restore(gapa_cuda_fail(e, "gapa_fitness_noalloc"));
    if (h & GAPA_DEV_BAD_EDGE) return restore(gapa_fail(GAPA_ERR_DEVICE, "an edge endpoint outside [0, n)"));
    if (h & GAPA_DEV_BAD_GENE) return restore(gapa_fail(GAPA_ERR_DEVICE, "a gene outside [0, n)"));
    return restore(GAPA_OK);
}

// ---------------------------------------------------------------------------
// Batched instances: a persistent kernel pulls packets (instance, members)
// from a work queue ordered by decreasing graph size; a CTA of 1024 threads
// splits into `teams` teams of 1024/teams threads, each evaluating one member
// of the packet with its own slice of shared memory and its own named barrier
// (1 + team), so small graphs run several members per CTA.
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(1024, 1) fitness_batched_kernel(const BatchDesc* __restrict__ d,
                                                                  const BatchPacket* __restrict__ pk, int npk,
                                                                  int* head, int buf, unsigned smem_bytes,
                                                                  int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long red[8][32];
    __shared__ int sh_p;
    while (true) {
        if (threadIdx.x == 0) sh_p = atomicAdd(head, 1);
        __syncthreads();
        const int p = sh_p;
        __syncthreads();
        if (p >= npk) break;
        const BatchPacket q = pk[p];
        const BatchDesc& bd = d[q.b];
        const int T = (int)blockDim.x / q.teams;
        const int team = (int)threadIdx.x / T;
        if (team < q.cnt) {
            const gapa_dev::Team tm{(int)threadIdx.x - team * T, T, 1 + team};
            const unsigned slice = (smem_bytes / (unsigned)q.teams) & ~15u;
            int* lab = reinterpret_cast<int*>(smem + (size_t)team * slice);
            const gapa_dev::Tree16Graph g{bd.n,        bd.perm,      bd.palt,        bd.lo_ptr,   bd.lo_col,
                                          bd.nontree,  bd.num_nontree, bd.fptr,      bd.fcol16,   0,
                                          bd.mean_deg_x16, bd.objective, bd.tparent, bd.kids,     bd.roots,
                                          bd.num_roots, bd.list_bytes};
            const int member = q.i0 + team;
            const int* genes = bd.pop[buf] + (size_t)member * bd.p.k;
            long long* out = reinterpret_cast<long long*>(bd.fit[buf]) + member;
            // the cut-local kernel with the operator kernels' estimates: the cheaper forest, or the
            // full pipeline for a member expected to shatter both
            bool local = bd.list_bytes > 0, alt = false;
            if (local && bd.p.est_out) {
                const unsigned e1 = bd.p.est_out[member], e2 = bd.p.est_out[bd.p.est_stride + member];
                const unsigned e = e2 < e1 ? e2 : e1;
                if (e > (unsigned)(bd.n / 4)) local = false;
                alt = e2 < e1 && bd.alt.perm != nullptr;
            }
            unsigned* region = reinterpret_cast<unsigned*>(lab + gapa_dev::tree16l_lab_ints(bd.n));
            int* scal = reinterpret_cast<int*>(region) + bd.list_bytes / 4;
            if (local && alt) {
                const DeviceForest& a = bd.alt;
                const gapa_dev::Tree16Graph tb{bd.n,         a.perm,          a.palt,          a.lo_ptr,
                                               a.lo_col,     a.nontree,       a.num_nontree,   a.fptr,
                                               a.fcol16,     0,               bd.mean_deg_x16, bd.objective,
                                               a.tparent,    a.kids,          a.roots,         a.num_roots,
                                               bd.list_bytes};
                gapa_dev::tree16_member_local(tm, lab, region, scal, tb, genes, bd.p.k, out, red[team], status);
            } else if (local) {
                gapa_dev::tree16_member_local(tm, lab, region, scal, g, genes, bd.p.k, out, red[team], status);
            } else {
                gapa_dev::tree16_member(tm, lab, reinterpret_cast<unsigned*>(lab + bd.n), g, genes, bd.p.k, out,
                                        red[team], status);
            }
        }
        __syncthreads();
    }
}

}  // namespace

int gapa_launch_fitness_batched(const BatchDesc* d, const BatchPacket* pk, int npk, int* head, int buf,
                                size_t smem, int grid, int* status, cudaStream_t st) {
    if (npk <= 0) return GAPA_OK;
    GAPA_CUDA(cudaMemsetAsync(head, 0, sizeof(int), st));
    fitness_batched_kernel<<<grid, 1024, smem, st>>>(d, pk, npk, head, buf, (unsigned)smem, status);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_fitness_batched_init(size_t optin, size_t* max_dyn) {
    return gapa_set_smem_limit((const void*)fitness_batched_kernel, optin, max_dyn);
}

int gapa_fitness_batched_occupancy(size_t smem, int* blocks_per_sm) {
    GAPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fitness_batched_kernel, 1024, smem));
    return GAPA_OK;
}
