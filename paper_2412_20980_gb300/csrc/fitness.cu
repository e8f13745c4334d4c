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

#include "gapa_internal.cuh"

namespace {

constexpr int kDead = INT_MIN;

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

__device__ __forceinline__ void edge_op(volatile int* lab, int u, int v) {
    if (lab[u] == kDead || lab[v] == kDead) return;
    uf_unite(lab, u, v);
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    long long tot = 0;
    if (warp == 0) {
        tot = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    return tot;  // valid in thread 0
}

// The whole per-member pipeline on a label array `lab` of n ints that only
// this CTA touches.
__device__ __forceinline__ void member_pc(volatile int* lab, int n, int num_edges, const int2* __restrict__ edges,
                                          const int* __restrict__ genes, int k, long long* out, int* status,
                                          long long* red) {
    const int tid = threadIdx.x, T = blockDim.x;
    // labels: every node its own root
    for (int v = tid; v < n; v += T) lab[v] = v;
    __syncthreads();
    // perturbation P^(A, p): mark the deleted nodes
    for (int j = tid; j < k; j += T) {
        const int d = __ldg(&genes[j]);
        if ((unsigned)d < (unsigned)n)
            lab[d] = kDead;
        else
            atomicOr(status, GAPA_DEV_BAD_GENE);
    }
    __syncthreads();
    // hooking over every undirected edge once, two edges per 16-byte load
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
    // flatten: every live node points at its root
    for (int v = tid; v < n; v += T) {
        const int l = lab[v];
        if (l != kDead && l != v) lab[v] = uf_find(lab, v);
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
        if (l < 0 && l != kDead) {
            const long long c = -(long long)l;
            acc += c * (c - 1) / 2;
        }
    }
    const long long tot = block_sum_ll(acc, red);
    if (tid == 0) *out = tot;
}

__global__ void __launch_bounds__(1024) cc_smem_kernel(int n, int num_edges, const int2* __restrict__ edges,
                                                       const int* __restrict__ pop, int k,
                                                       long long* __restrict__ fit, int* status) {
    extern __shared__ int smem_lab[];
    __shared__ long long red[32];
    const int i = blockIdx.x;
    member_pc(smem_lab, n, num_edges, edges, pop + (size_t)i * k, k, &fit[i], status, red);
}

__global__ void __launch_bounds__(1024) cc_global_kernel(int n, int num_edges, const int2* __restrict__ edges,
                                                         const int* __restrict__ pop, int k,
                                                         long long* __restrict__ fit, int* status,
                                                         int* labels, int member_base) {
    __shared__ long long red[32];
    const int i = member_base + blockIdx.x;
    member_pc(labels + (size_t)blockIdx.x * n, n, num_edges, edges, pop + (size_t)i * k, k, &fit[i], status, red);
}


int smem_block_for(int n) {
    // enough threads to cover the graph, at most 1024; multiples of 32
    if (n <= 2048) return 256;
    if (n <= 8192) return 512;
    return 1024;
}

}  // namespace

int gapa_fitness_prepare(gapa_ctx* c, int s) {
    const size_t lab_bytes = (size_t)c->g.n * 4;
    if (lab_bytes <= c->fit_smem_max) return GAPA_OK;
    // global labels: process members in waves of at most `wave` CTAs
    const size_t wave = (size_t)(s < 4 * c->num_sms ? s : 4 * c->num_sms);
    return gapa_reserve((void**)&c->labels, &c->labels_cap, wave * (size_t)c->g.n, sizeof(int));
}

int gapa_launch_fitness(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st) {
    if (s <= 0) return GAPA_OK;
    ProfileScope prof(c, st, 0, s);
    const int n = c->g.n;
    const size_t lab_bytes = (size_t)n * 4;
    long long* f = reinterpret_cast<long long*>(fit);
    if (lab_bytes <= c->fit_smem_max) {
        const int block = smem_block_for(n);
        cc_smem_kernel<<<s, block, lab_bytes, st>>>(n, c->g.num_edges, c->g.edges, pop, k, f, c->status);
        GAPA_CUDA(cudaGetLastError());
        return GAPA_OK;
    }
    int rc = gapa_fitness_prepare(c, s);
    if (rc != GAPA_OK) return rc;
    const int wave = (int)(c->labels_cap / (size_t)n);
    for (int base = 0; base < s; base += wave) {
        const int cnt = s - base < wave ? s - base : wave;
        cc_global_kernel<<<cnt, 1024, 0, st>>>(n, c->g.num_edges, c->g.edges, pop, k, f, c->status, c->labels,
                                                base);
        GAPA_CUDA(cudaGetLastError());
    }
    return GAPA_OK;
}

int gapa_fitness_kernels_init(gapa_ctx* c) {
    return gapa_set_smem_limit((const void*)cc_smem_kernel, c->smem_optin, &c->fit_smem_max);
}
