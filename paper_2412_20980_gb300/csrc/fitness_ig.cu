// Batched fitness for graphs whose labels do not fit in shared memory
// (Section III-C, Eq. 13; PC(G) of Table "Whole").
//
// Members are evaluated in groups of kM = 8 whose labels are interleaved,
// L[v * 8 + m] for member m of the group, so one 32-byte sector holds a node's
// labels for the whole group: every non-tree edge costs two sector reads for
// eight members, and the edge list streams from HBM once per group.  Several
// groups run per batch, as many as keep their labels within an L2-sized
// budget.  The phases are those of the shared-memory TREE kernel (tree-parent
// labels in BFS numbering, deleted nodes, cut with fallback parents, flatten,
// join along non-tree edges); the last flatten turns the roots into counters,
// sizes are counted into them and the int64 sums of C(size, 2) are reduced per
// member.  Each phase is one
// grid-wide kernel; thread t of a group handles (node t/8, member t%8) in a
// grid-stride loop, so the eight lanes of a node share one sector.
//
// Deleting hubs near the top of the BFS tree shatters it into many pieces,
// and uniting them edge by edge in L2 is slow, so two steps come between the
// cut and the join: every live node also links to up to two live neighbours
// among the first entries of its adjacency (neighbour sampling), and the
// first live node of each member - the smallest live id, hence a root
// forever - names the giant candidate.  The nodes outside its piece then scan
// their adjacency, unless that is more work than the non-tree edge list, in
// which case the group joins along the non-tree edges as before.  These steps
// pay off on graphs with many non-tree edges per node (at least 4); sparser
// graphs go straight from the cut to the join.
#include <climits>

#include "gapa_internal.cuh"

namespace {

constexpr int kM = 8;
constexpr int kDead = INT_MIN;
constexpr int kIgBlock = 256;

__device__ __forceinline__ volatile int* slot(int* L, int x, int m) { return (volatile int*)(L + (size_t)x * kM + m); }

// Path halving on member m's view (parents have smaller BFS numbers).
__device__ __forceinline__ int ig_find(int* L, int m, int x) {
    while (true) {
        const int p = *slot(L, x, m);
        if (p == x) return x;
        const int gp = *slot(L, p, m);
        if (gp == p) return p;
        *slot(L, x, m) = gp;
        x = gp;
    }
}

// The top of x's chain: a node that points at itself or, once roots have
// become counters, holds a negative count.  No live chain passes a deleted
// node, so a negative label on a chain is always a counter.
__device__ __forceinline__ int ig_top(int* L, int m, int x) {
    int p = *slot(L, x, m);
    while (p != x && p >= 0) {
        x = p;
        p = *slot(L, x, m);
    }
    return x;
}

__device__ __forceinline__ void ig_unite(int* L, int m, int a, int b) {
    a = ig_find(L, m, a);
    b = ig_find(L, m, b);
    while (a != b) {
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(L + (size_t)a * kM + m, a, b);
        if (old == a) return;
        a = ig_find(L, m, old);
        b = ig_find(L, m, b);
    }
}

struct IgArgs {
    int n, k, s, member_base;  // members [member_base, member_base + 8 * groups) of the population
    const int* pop;
    const int* perm;
    const int* tparent;
    const int2* palt;
    const int* lo_ptr;
    const int* lo_col;
    const int2* nontree;
    int num_nontree;
    int* L;  // [groups][n][8]
    long long* fit;
    int* status;
    int objective;  // 0: PC, 1: MCN
    const int* fptr;  // full adjacency in BFS numbers (CSR)
    const int* fcol;
    int* giant;                  // [groups][8] first live node of each member (-1: none)
    unsigned long long* work;    // [groups][8] adjacency entries of the nodes outside the giant piece
    int sampled;                 // 1: the sampling / giant / scan steps run before the join
};

constexpr int kLinkScan = 4;  // adjacency entries a node looks at for its sampled links

// a group's last slots may hold no member of the population
__device__ __forceinline__ bool ig_real_member(const IgArgs& a, int m) {
    return a.member_base + (int)blockIdx.y * kM + m < a.s;
}

// whether the group's piece scan replaces the join (decided from the work counts)
__device__ __forceinline__ bool ig_group_scans(const IgArgs& a) {
    const unsigned long long* w = a.work + (size_t)blockIdx.y * kM;
    unsigned long long tot = 0;
#pragma unroll
    for (int m = 0; m < kM; ++m) tot += w[m];
    return tot <= 2ull * kM * (unsigned long long)a.num_nontree;
}

__device__ __forceinline__ int* group_labels(const IgArgs& a) { return a.L + (size_t)blockIdx.y * a.n * kM; }
__device__ __forceinline__ size_t gthreads() { return (size_t)gridDim.x * blockDim.x; }
__device__ __forceinline__ size_t gtid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }

// labels = tree parents for all eight members; fitness slots cleared
__global__ void __launch_bounds__(kIgBlock) ig_init_kernel(IgArgs a) {
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM;
    for (size_t t = gtid(); t < total; t += gthreads()) L[t] = __ldg(&a.tparent[t / kM]);
    if (blockIdx.x == 0 && threadIdx.x < kM) {
        const int member = a.member_base + blockIdx.y * kM + threadIdx.x;
        if (member < a.s) a.fit[member] = 0;
    }
}

// perturbation P^(A, p) of Eq. 13: deleted nodes of each member
__global__ void __launch_bounds__(kIgBlock) ig_dead_kernel(IgArgs a) {
    int* L = group_labels(a);
    const size_t total = (size_t)a.k * kM;
    for (size_t t = gtid(); t < total; t += gthreads()) {
        const int m = (int)(t / a.k), j = (int)(t % a.k);
        const int member = a.member_base + blockIdx.y * kM + m;
        if (member >= a.s) continue;
        const int d = __ldg(&a.pop[(size_t)member * a.k + j]);
        if ((unsigned)d < (unsigned)a.n)
            L[(size_t)__ldg(&a.perm[d]) * kM + m] = kDead;
        else
            atomicOr(a.status, GAPA_DEV_BAD_GENE);
    }
}

// cut: a live node whose tree parent is deleted takes its first live
// lower-numbered neighbour, or tops its own piece (deadness is final here)
__global__ void __launch_bounds__(kIgBlock) ig_cut_kernel(IgArgs a) {
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM;
    for (size_t t = gtid(); t < total; t += gthreads()) {
        const int v = (int)(t / kM), m = (int)(t % kM);
        const int p = *slot(L, v, m);
        if (p == kDead || p == v || *slot(L, p, m) != kDead) continue;
        int q = v;
        const int2 pa = __ldg(&a.palt[v]);
        if (pa.y >= 0) {
            if (*slot(L, pa.y, m) != kDead) {
                q = pa.y;
            } else {
                const int beg = __ldg(&a.lo_ptr[v]) + 2, end = __ldg(&a.lo_ptr[v + 1]);
                for (int e = beg; e < end; ++e) {
                    const int w = __ldg(&a.lo_col[e]);
                    if (*slot(L, w, m) != kDead) {
                        q = w;
                        break;
                    }
                }
            }
        }
        *slot(L, v, m) = q;
    }
}

// every live node points at the top of its piece / its root (owner writes only;
// a label already there is not rewritten).  kCounters: the last flatten also
// turns every root into a counter (-1), the start of the size count; a
// concurrent walk stops at a root either way.
constexpr int kFlatInFlight = 4;  // items per thread resolved together by ig_flatten_kernel
constexpr int kLinkInFlight = 4;  // items per thread loaded together by ig_link_kernel

template <bool kCounters>
__global__ void __launch_bounds__(kIgBlock) ig_flatten_kernel(IgArgs a) {
    // kFlatInFlight items per thread in flight: their labels, then their parents' labels, are
    // loaded together; only a chain longer than two steps walks on alone.  Parents have smaller
    // numbers and the items go in increasing node order, so most parents are flat already.
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM, G = gthreads();
    size_t t = gtid();
    for (; t + (kFlatInFlight - 1) * G < total; t += kFlatInFlight * G) {
        int p[kFlatInFlight], q[kFlatInFlight];
#pragma unroll
        for (int u = 0; u < kFlatInFlight; ++u) p[u] = *slot(L, (int)((t + u * G) / kM), (int)((t + u * G) % kM));
#pragma unroll
        for (int u = 0; u < kFlatInFlight; ++u) {
            const int v = (int)((t + u * G) / kM), m = (int)((t + u * G) % kM);
            int x = p[u];
            if (p[u] != kDead && p[u] != v) x = *slot(L, p[u], m);
            q[u] = x;
        }
#pragma unroll
        for (int u = 0; u < kFlatInFlight; ++u) {
            const int v = (int)((t + u * G) / kM), m = (int)((t + u * G) % kM);
            if (p[u] == kDead) continue;
            if (p[u] == v) {
                if (kCounters) *slot(L, v, m) = -1;
                continue;
            }
            const int r = (q[u] == p[u] || q[u] < 0) ? p[u] : ig_top(L, m, q[u]);
            if (r != p[u]) *slot(L, v, m) = r;
        }
    }
    for (; t < total; t += G) {
        const int v = (int)(t / kM), m = (int)(t % kM);
        const int p = *slot(L, v, m);
        if (p == kDead) continue;
        if (p == v) {
            if (kCounters) *slot(L, v, m) = -1;
            continue;
        }
        const int r = ig_top(L, m, p);
        if (r != p) *slot(L, v, m) = r;
    }
}

// first live node of every member of the group (one warp per member; the
// smallest live id), and the work counters cleared
__global__ void __launch_bounds__(kIgBlock) ig_giant_kernel(IgArgs a) {
    int* L = group_labels(a);
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (m >= kM) return;
    const int member = a.member_base + blockIdx.y * kM + m;
    int f = -1;
    if (member < a.s) {
        for (int base = 0; base < a.n; base += 32) {
            const int v = base + lane;
            const unsigned live = __ballot_sync(0xffffffffu, v < a.n && *slot(L, v, m) != kDead);
            if (live) {
                f = base + __ffs(live) - 1;
                break;
            }
        }
    }
    if (lane == 0) {
        a.giant[(size_t)blockIdx.y * kM + m] = f;
        a.work[(size_t)blockIdx.y * kM + m] = 0ull;
    }
}

// neighbour sampling: every live node unites with up to two live neighbours of
// another piece among its first kLinkScan adjacency entries
__global__ void __launch_bounds__(kIgBlock) ig_link_kernel(IgArgs a) {
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM, G = gthreads();
    size_t t = gtid();
    // kLinkInFlight items per thread in flight: their labels, adjacency bounds, first neighbours
    // and those neighbours' labels are loaded together before any union.  A neighbour's label read
    // early that equals the node's current label still proves both in one set (sets only merge),
    // so skipping it is exact.
    for (; t + (kLinkInFlight - 1) * G < total; t += kLinkInFlight * G) {
        int v[kLinkInFlight], m[kLinkInFlight], beg[kLinkInFlight], cnt[kLinkInFlight];
#pragma unroll
        for (int u = 0; u < kLinkInFlight; ++u) {
            v[u] = (int)((t + u * G) / kM);
            m[u] = (int)((t + u * G) % kM);
            cnt[u] = (ig_real_member(a, m[u]) && *slot(L, v[u], m[u]) != kDead) ? 1 : 0;
        }
#pragma unroll
        for (int u = 0; u < kLinkInFlight; ++u) {
            if (!cnt[u]) continue;
            beg[u] = __ldg(&a.fptr[v[u]]);
            cnt[u] = min(__ldg(&a.fptr[v[u] + 1]) - beg[u], kLinkScan);
        }
        int w[kLinkInFlight][kLinkScan], lw[kLinkInFlight][kLinkScan];
#pragma unroll
        for (int e = 0; e < kLinkScan; ++e)
#pragma unroll
            for (int u = 0; u < kLinkInFlight; ++u) w[u][e] = e < cnt[u] ? __ldg(&a.fcol[beg[u] + e]) : -1;
#pragma unroll
        for (int e = 0; e < kLinkScan; ++e)
#pragma unroll
            for (int u = 0; u < kLinkInFlight; ++u) {
                int x = kDead;
                if (w[u][e] >= 0) x = *slot(L, w[u][e], m[u]);
                lw[u][e] = x;
            }
#pragma unroll
        for (int u = 0; u < kLinkInFlight; ++u) {
            int linked = 0;
#pragma unroll
            for (int e = 0; e < kLinkScan; ++e) {
                if (e >= cnt[u] || linked >= 2 || lw[u][e] == kDead) continue;
                if (lw[u][e] != *slot(L, v[u], m[u])) ig_unite(L, m[u], v[u], w[u][e]);
                ++linked;
            }
        }
    }
    for (; t < total; t += G) {
        const int v = (int)(t / kM), m = (int)(t % kM);
        if (!ig_real_member(a, m) || *slot(L, v, m) == kDead) continue;
        const int beg = __ldg(&a.fptr[v]);
        const int end = min(__ldg(&a.fptr[v + 1]), beg + kLinkScan);
        int linked = 0;
        for (int e = beg; e < end && linked < 2; ++e) {
            const int w = __ldg(&a.fcol[e]);
            const int lw = *slot(L, w, m);
            if (lw == kDead) continue;
            if (lw != *slot(L, v, m)) ig_unite(L, m, v, w);
            ++linked;
        }
    }
}

// adjacency entries of the live nodes outside the giant candidate's piece, per member
__global__ void __launch_bounds__(kIgBlock) ig_outside_kernel(IgArgs a) {
    int* L = group_labels(a);
    __shared__ unsigned long long acc_m[kM];
    if (threadIdx.x < kM) acc_m[threadIdx.x] = 0ull;
    __syncthreads();
    const size_t total = (size_t)a.n * kM;
    const int m = (int)(gtid() % kM);
    const int R = a.giant[(size_t)blockIdx.y * kM + m];
    unsigned long long acc = 0;
    for (size_t t = ig_real_member(a, m) ? gtid() : total; t < total; t += gthreads()) {
        const int v = (int)(t / kM);
        const int l = *slot(L, v, m);
        if (l != kDead && l != R) acc += (unsigned long long)(__ldg(&a.fptr[v + 1]) - __ldg(&a.fptr[v]));
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 16);
    acc += __shfl_down_sync(0xffffffffu, acc, 8);
    if ((threadIdx.x & 31) < kM) atomicAdd(&acc_m[threadIdx.x & 31], acc);
    __syncthreads();
    if (threadIdx.x < kM && acc_m[threadIdx.x])
        atomicAdd(&a.work[(size_t)blockIdx.y * kM + threadIdx.x], acc_m[threadIdx.x]);
}

// the nodes outside the giant candidate's piece unite with their live
// neighbours (an edge inside that piece joins nothing)
__global__ void __launch_bounds__(kIgBlock) ig_scan_kernel(IgArgs a) {
    if (!ig_group_scans(a)) return;
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM;
    for (size_t t = gtid(); t < total; t += gthreads()) {
        const int v = (int)(t / kM), m = (int)(t % kM);
        const int l = *slot(L, v, m);
        if (l == kDead || l == a.giant[(size_t)blockIdx.y * kM + m] || !ig_real_member(a, m)) continue;
        const int end = __ldg(&a.fptr[v + 1]);
        for (int e = __ldg(&a.fptr[v]); e < end; ++e) {
            const int w = __ldg(&a.fcol[e]);
            const int lw = *slot(L, w, m);
            if (lw != kDead && lw != *slot(L, v, m)) ig_unite(L, m, v, w);
        }
    }
}

// join the pieces along the non-tree edges: lane m of an edge handles member m
__global__ void __launch_bounds__(kIgBlock) ig_join_kernel(IgArgs a) {
    if (a.sampled && ig_group_scans(a)) return;
    int* L = group_labels(a);
    const size_t total = (size_t)a.num_nontree * kM;
    for (size_t t = gtid(); t < total; t += gthreads()) {
        const int m = (int)(t % kM);
        const int2 e = __ldcs(&a.nontree[t / kM]);  // streamed once per group: evict first, keep labels in L2
        // quick check through L1: a stale label is still an ancestor (or the node itself) at some
        // earlier moment, so equal labels prove a common tree; unequal ones go to union-find
        const int la = L[(size_t)e.x * kM + m], lb = L[(size_t)e.y * kM + m];
        if (la == lb || la == kDead || lb == kDead) continue;
        ig_unite(L, m, la, lb);
    }
}

// every other live node adds itself to its root's counter; a thread keeps a
// run of equal roots in a register and flushes it when the root changes
__global__ void __launch_bounds__(kIgBlock) ig_count_kernel(IgArgs a) {
    int* L = group_labels(a);
    const size_t total = (size_t)a.n * kM;
    const size_t stride = gthreads();  // a multiple of 8: a thread keeps its member
    const int m = (int)(gtid() % kM);
    int run_root = -1, run = 0;
    for (size_t t = gtid(); t < total; t += stride) {
        const int v = (int)(t / kM);
        const int l = *slot(L, v, m);
        if (l < 0) continue;  // deleted node or a root (counter)
        if (l != run_root) {
            if (run) atomicAdd(L + (size_t)run_root * kM + m, -run);
            run_root = l;
            run = 0;
        }
        ++run;
    }
    // the last runs: most threads end on the same root (the giant piece's), so the
    // four lanes of a warp with this thread's member whose root equals their first
    // lane's add their runs together, and one atomic carries them
    const int lane = threadIdx.x & 31;
    const int r0 = __shfl_sync(0xffffffffu, run_root, lane & (kM - 1));
    int part = run_root == r0 ? run : 0;
    if (run && run_root != r0) atomicAdd(L + (size_t)run_root * kM + m, -run);
    part += __shfl_down_sync(0xffffffffu, part, 16);
    part += __shfl_down_sync(0xffffffffu, part, 8);
    if (lane < kM && part) atomicAdd(L + (size_t)r0 * kM + m, -part);
}

// Per member, the int64 sum of C(size, 2) over roots (PC) or the largest size
// (MCN): block reduce, then one atomic per member.
__global__ void __launch_bounds__(kIgBlock) ig_sum_kernel(IgArgs a) {
    int* L = group_labels(a);
    __shared__ unsigned long long acc_m[kM];
    if (threadIdx.x < kM) acc_m[threadIdx.x] = 0ull;
    __syncthreads();
    const size_t total = (size_t)a.n * kM;
    const int m = (int)(gtid() % kM);
    const bool mx = a.objective != 0;
    unsigned long long acc = 0;
    for (size_t t = gtid(); t < total; t += gthreads()) {
        const int l = *slot(L, (int)(t / kM), m);
        if (l < 0 && l != kDead) {
            const unsigned long long c = (unsigned long long)(-(long long)l);
            acc = mx ? (c > acc ? c : acc) : acc + c * (c - 1) / 2;
        }
    }
    // lanes with equal (lane % 8) share a member: reduce over lanes 8 apart
    for (int o = 16; o >= 8; o >>= 1) {
        const unsigned long long x = __shfl_down_sync(0xffffffffu, acc, o);
        acc = mx ? (x > acc ? x : acc) : acc + x;
    }
    if ((threadIdx.x & 31) < kM) {
        if (mx) atomicMax(&acc_m[threadIdx.x & 31], acc);
        else atomicAdd(&acc_m[threadIdx.x & 31], acc);
    }
    __syncthreads();
    if (threadIdx.x < kM) {
        const int member = a.member_base + blockIdx.y * kM + threadIdx.x;
        if (member < a.s) {
            if (mx) atomicMax((unsigned long long*)&a.fit[member], acc_m[threadIdx.x]);
            else atomicAdd((unsigned long long*)&a.fit[member], acc_m[threadIdx.x]);
        }
    }
}

constexpr size_t kIgLabelBudget = 64ull << 20;  // labels of a batch of groups kept within this many bytes (R-MAT 2^20: two groups; 48 MB (one group) took 11.3 ms per 256 members, 64 MB 8.2, 96 MB 9.8)

int ig_groups_per_batch(int n, int s) {
    const size_t per_group = (size_t)n * kM * sizeof(int);
    size_t g = kIgLabelBudget / per_group;
    if (g < 1) g = 1;
    const size_t need = ((size_t)s + kM - 1) / kM;
    if (g > need) g = need;
    if (g > 65535) g = 65535;
    return (int)g;
}

}  // namespace

int gapa_ig_prepare(gapa_ctx* c, int s) {
    const int groups = ig_groups_per_batch(c->g.n, s < 1 ? 1 : s);
    int rc = gapa_reserve((void**)&c->labels, &c->labels_cap, (size_t)groups * c->g.n * kM, sizeof(int));
    // work counters (8 bytes) and giant ids (4 bytes) per member of a batch
    if (rc == GAPA_OK) rc = gapa_reserve(&c->ig_aux, &c->ig_aux_cap, (size_t)groups * kM, 12);
    return rc;
}

int gapa_launch_fitness_ig(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                           int* kernels) {
    const int n = c->g.n;
    int rc = gapa_ig_prepare(c, s);
    if (rc != GAPA_OK) return rc;
    const int gpb = ig_groups_per_batch(n, s);
    IgArgs a;
    a.n = n;
    a.k = k;
    a.s = s;
    a.pop = pop;
    a.perm = c->g.perm;
    a.tparent = c->g.tparent;
    a.palt = c->g.palt;
    a.lo_ptr = c->g.lo_ptr;
    a.lo_col = c->g.lo_col;
    a.nontree = reinterpret_cast<const int2*>(c->g.nontree);
    a.num_nontree = c->g.num_nontree;
    a.L = c->labels;
    a.fit = reinterpret_cast<long long*>(fit);
    a.status = c->status;
    a.objective = c->objective;
    a.fptr = c->g.fptr;
    a.fcol = c->g.fcol32;
    a.work = reinterpret_cast<unsigned long long*>(c->ig_aux);
    a.giant = reinterpret_cast<int*>(a.work + (size_t)gpb * kM);
    a.sampled = (long long)a.num_nontree >= 4ll * n ? 1 : 0;
    // grid: enough CTAs to fill the GPU a few times over, a multiple of the SM count
    const size_t work = (size_t)n * kM;
    int bx = (int)((work + kIgBlock - 1) / kIgBlock);
    const int cap = c->num_sms * 8;
    const int per_batch_cap = gpb > 0 ? (cap + gpb - 1) / gpb : cap;
    if (bx > per_batch_cap) bx = per_batch_cap < 1 ? 1 : per_batch_cap;
    const size_t ework = (size_t)a.num_nontree * kM;
    int bxe = (int)((ework + kIgBlock - 1) / kIgBlock);
    if (bxe > per_batch_cap) bxe = per_batch_cap < 1 ? 1 : per_batch_cap;
    if (bxe < 1) bxe = 1;
    const int groups_total = (s + kM - 1) / kM;
    for (int g0 = 0; g0 < groups_total; g0 += gpb) {
        const int gcount = groups_total - g0 < gpb ? groups_total - g0 : gpb;
        a.member_base = g0 * kM;
        const dim3 grid(bx, gcount), egrid(bxe, gcount);
        ig_init_kernel<<<grid, kIgBlock, 0, st>>>(a);
        ig_dead_kernel<<<grid, kIgBlock, 0, st>>>(a);
        ig_cut_kernel<<<grid, kIgBlock, 0, st>>>(a);
        ig_flatten_kernel<false><<<grid, kIgBlock, 0, st>>>(a);
        if (a.sampled) {
            ig_giant_kernel<<<dim3(1, gcount), kIgBlock, 0, st>>>(a);
            ig_link_kernel<<<grid, kIgBlock, 0, st>>>(a);
            ig_flatten_kernel<false><<<grid, kIgBlock, 0, st>>>(a);
            ig_outside_kernel<<<grid, kIgBlock, 0, st>>>(a);
            ig_scan_kernel<<<grid, kIgBlock, 0, st>>>(a);
        }
        if (a.num_nontree > 0) ig_join_kernel<<<egrid, kIgBlock, 0, st>>>(a);
        ig_flatten_kernel<true><<<grid, kIgBlock, 0, st>>>(a);
        ig_count_kernel<<<grid, kIgBlock, 0, st>>>(a);
        ig_sum_kernel<<<grid, kIgBlock, 0, st>>>(a);
        GAPA_CUDA(cudaGetLastError());
        if (kernels) *kernels = (g0 == 0 ? 0 : *kernels) + (a.num_nontree > 0 ? 8 : 7) + (a.sampled ? 5 : 0);
    }
    return GAPA_OK;
}
