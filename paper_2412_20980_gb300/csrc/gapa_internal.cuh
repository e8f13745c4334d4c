// Internal declarations of libgapa.so (CUDA path).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gapa.h"

// ---------------------------------------------------------------------------
// Device status word: kernels OR these bits in; gapa_sync() reports them.
// ---------------------------------------------------------------------------
enum : int {
    GAPA_DEV_BAD_GENE = 1,   // a gene outside [0, n)
    GAPA_DEV_TIMEOUT = 2,    // a bounded wait ran out
    GAPA_DEV_CAPACITY = 4,   // a work list overflowed its bound
    GAPA_DEV_BAD_EDGE = 8,   // an edge endpoint outside [0, n)
};

// Philox tags of the counter's last word (tag << 24 | round).
enum : uint32_t {
    TAG_INIT = 1,
    TAG_SEL = 2,
    TAG_XOVER = 3,
    TAG_MUT = 4,
    TAG_MUTVAL = 5,
    TAG_REPAIR = 6,
    TAG_ROULETTE = 7,
};

constexpr int kRepairRounds = 32;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// two-multiplier bijection with a Weyl-sequence key schedule; returns output
// word 0 only.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        const uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
        const uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

struct RngKey {
    uint32_t lo, hi;
};

__device__ __forceinline__ uint32_t gapa_draw(RngKey key, uint32_t j, uint32_t i, uint32_t g, uint32_t tag,
                                              uint32_t round) {
    return philox_word0(j, i, g, (tag << 24) | round, key.lo, key.hi);
}

// Words 0 and 1 of Philox4x32-10 as one 64-bit number (word 0 high).
__device__ __forceinline__ unsigned long long philox_word01(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                           uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        const uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
        const uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ((unsigned long long)c0 << 32) | c1;
}

// Uniform integer in [0, n): multiply-high of a 32-bit word by n.
__device__ __forceinline__ int uniform_below(uint32_t x, int n) { return (int)__umulhi(x, (uint32_t)n); }

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
// A second spanning forest of a graph with n <= 65536, in its own numbering
// (parents precede children; a node's parent is its lowest-numbered
// neighbour when that one is lower): the arrays of the TREE kernels.
struct DeviceForest {
    int* perm = nullptr;             // [n] original id -> number
    int* tparent = nullptr;          // [n rounded up to 4]
    int2* palt = nullptr;            // [n] (parent, second lower-numbered neighbour or -1)
    int* lo_ptr = nullptr;           // [n+1] lower-numbered neighbours (CSR, ascending)
    int* lo_col = nullptr;
    int4* kids = nullptr;            // [n] children in at most two runs (see DeviceGraph::kids)
    int* roots = nullptr;            // [num_roots]
    int num_roots = 0;
    int* cut = nullptr;              // [n] cost table by original node id (see DeviceGraph::cut)
    int* fptr = nullptr;             // [n+1] full adjacency in this numbering
    unsigned short* fcol16 = nullptr;
    unsigned* nontree = nullptr;     // non-tree edges a<<16|b (a < b), sorted
    int num_nontree = 0;
    // forest-piece kernel (see DeviceGraph::sz)
    int* sz = nullptr;
    int* pre = nullptr;
    unsigned short* at = nullptr;
    int* crep = nullptr;
    int* nroot = nullptr;
    int* csize = nullptr;
};

// One BFS forest of the sparse fitness kernel (fitness_sparse.cu): numbering, tree parents, the
// (tree parent, second lower neighbour) pairs, lower-neighbour and full adjacency CSR in its
// numbering, and per node (first child, children), the root of its component tree (-1 for a
// single-node component), the component's size at its root, subtree sizes, the component roots by
// decreasing size, and by original id the member cost estimate (children + 1); the number of
// components, the largest one's root and the sum over components of C(size, 2).  `owns`: the
// numbering and adjacency arrays are this forest's own (forest 0 borrows the graph's).
struct SparseForest {
    int* perm = nullptr;
    int* tparent = nullptr;
    int2* palt = nullptr;
    int* lo_ptr = nullptr;
    int* lo_col = nullptr;
    int* fptr = nullptr;
    int* fcol32 = nullptr;
    unsigned short* fcol16 = nullptr;
    int2* kids = nullptr;
    int* croot = nullptr;
    int* csize = nullptr;
    int* sub = nullptr;
    int* bysize = nullptr;
    int* cost = nullptr;
    int ncomp = 0;
    int giant = -1;
    long long pc0 = 0;
    bool owns = false;
};
constexpr int kSpForests = 4;

struct DeviceGraph {
    int n = 0;
    long long nnz = 0;        // arcs = 2E
    int num_edges = 0;        // E (undirected)
    int* row_ptr = nullptr;   // [n+1]
    int* col = nullptr;       // [nnz], rows sorted
    int2* edges = nullptr;    // [E] (u, v) with u < v, CSR order
    int* probe = nullptr;     // [kProbe] node ids of highest degree, descending
    int max_degree = 0;
    // BFS forest numbering (TREE fitness kernel): nodes renumbered in BFS
    // order from the highest-degree node of each component, so every tree
    // parent has a smaller number than its child.
    int* perm = nullptr;        // [n] original id -> BFS number
    int* tparent = nullptr;     // [n rounded up to 4] BFS number -> BFS number of its tree parent (roots: itself)
    int4* kids = nullptr;       // [n] children: x .. x+y-1, then z+y .. z+y+w-1 (a second run; w = 0 here,
                                //     where children have consecutive numbers)
    int* roots = nullptr;       // [num_roots] BFS number of every component's root
    int num_roots = 0;
    int local_list_bytes = 0;   // list region of the cut-local TREE kernel (0: that kernel does not fit)
    int* cut = nullptr;         // [n] per original node id: nodes below those of its tree children that
                                //     have no other lower neighbour (deleting it alone cuts them off)
    int* order = nullptr;       // [5 * kOrderCap + 16] the members, costliest first (bit 30: use `alt`), then
                                //     their cost estimates under this forest, under `alt`, and the lower,
                                //     then the members deferred by the forest-piece kernel and their count
    DeviceForest alt;           // the forest numbered with the top hubs last (cut-local kernel only)
    // forest-piece kernel, per forest: the subtree size of every node, its position in a preorder
    // walk (children in ascending order, roots in ascending order; a subtree is the interval
    // [pre, pre + sz)), the node at each preorder position, the smallest root of every node's
    // component (its representative), the next root of the same component (-1: none) and the
    // component's size (at the representative)
    int* sz = nullptr;
    int* pre = nullptr;
    unsigned short* at = nullptr;
    int* crep = nullptr;
    int* nroot = nullptr;
    int* csize = nullptr;
    long long tree_pc = 0;      // sum over the components of G of C(size, 2)
    bool has_alt = false;
    int* lo_ptr = nullptr;      // [n+1] CSR of lower-numbered neighbours (BFS numbers, ascending;
    int* lo_col = nullptr;      //        the first one is the tree parent)
    int2* palt = nullptr;       // [n] (tree parent, second lower-numbered neighbour or -1)
    void* nontree = nullptr;    // non-tree edges (a < b, BFS numbers): uint32 a<<16|b if packed16, else int2
    int num_nontree = 0;
    int* fptr = nullptr;                // [n+1] full adjacency in BFS numbers (packed16 graphs only)
    unsigned short* fcol16 = nullptr;   // [2E]
    int* fcol32 = nullptr;              // [2E] the same with 32-bit ids (graphs that are not packed16)
    int mean_deg_x16 = 0;               // 16 * 2E / n, rounded up
    bool packed16 = false;      // n <= 65536
    int bfs_depth = 0;          // largest BFS level
    // sparse fitness kernel (any n; sp_nforests = 0 when a BFS forest's children are not consecutive):
    // forest 0 on G itself (borrowing the arrays above), and forests of G with every edge of the top
    // hub (1), of the two top hubs (2) or of the second hub (3) removed, for members that delete those
    // hubs (on which G and the reduced graph have the same PC); sp_hub = the two hubs' original ids
    SparseForest spf[kSpForests];
    int sp_nforests = 0;
    int sp_hub[2] = {-1, -1};
};

constexpr int kProbe = 8;
constexpr int kOrderCap = 1 << 16;  // members ordered by cost per fitness launch (larger batches: in order)

struct gapa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;      // borrowed
    cudaStream_t own_stream = nullptr;  // owned, used for capture in gapa_run
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;  // max shared memory per block (opt-in)
    size_t smem_per_sm = 0;     // shared memory per SM
    size_t smem_reserved = 0;   // shared memory the runtime reserves per block
    size_t fit_smem_max = 0;  // max dynamic shared memory of the shared-memory fitness kernel
    size_t piece_smem_max = 0;  // max dynamic shared memory of the forest-piece kernel
    size_t ga_smem_max = 0;   // max dynamic shared memory of the operator kernels
    DeviceGraph g;
    int* status = nullptr;  // device status word
    // scratch owned by the context
    int* labels = nullptr;  // global label scratch for graphs too large for shared memory
    void* sp_scratch = nullptr;  // per-CTA state of the sparse fitness kernel (hops, classes, counts, lists, sums)
    size_t sp_scratch_cap = 0;   // bytes
    size_t sp_stride = 0;        // entries per CTA slice
    int sp_slots = 0;            // CTA slices
    size_t sp_smem_max = 0;      // max dynamic shared memory of the sparse fitness kernel
    int* sp_order = nullptr;     // the sparse kernel's member order (member | forest << 28), then the
                                 // members' cost estimates and forests
    size_t sp_order_cap = 0;     // ints
    size_t labels_cap = 0;  // ints
    void* ig_aux = nullptr;  // per-member work counters and giant ids of the global-label fitness
    size_t ig_aux_cap = 0;
    int32_t* stage_pop[2] = {nullptr, nullptr};
    int64_t* stage_fit[2] = {nullptr, nullptr};
    size_t stage_pop_cap = 0, stage_fit_cap = 0;  // elements
    int* run_gen = nullptr;
    int* run_best = nullptr;
    int64_t* run_traj = nullptr;
    size_t run_traj_cap = 0;
    int fitness_variant = 0;  // 0 = auto
    int objective = 0;        // GAPA_OBJECTIVE_PC or GAPA_OBJECTIVE_MCN
    int genes = 0;            // GAPA_GENES_NODES or GAPA_GENES_EDGES
    int sixdst_hops = 6;      // N of the SixDST objectives
    int sixdst_kernel = 0;    // SixDST products: 0 = mma.sync, 1 = tcgen05 (256-wide tiles where the padded size
                              // allows), 2 = tcgen05 with 128-wide tiles only, 3 = tcgen05 with TMA loads and
                              // split roles (the default when it fits; 256-wide tiles, else as 1)
    bool sixdst_t5_ok = false;  // the tcgen05 product's shared memory fits on this device
    bool sixdst_t6_ok = false;  // and so does the 256-wide tile's
    bool sixdst_t7_ok = false;  // and the TMA kernel's (with the driver's tensor-map encoder)
    void* sdst_buf = nullptr;  // SixDST matrices and deletion bitmaps of a member batch
    size_t sdst_cap = 0;
    // (mu+lambda) and roulette scratch
    int32_t* kids = nullptr;
    size_t kids_cap = 0;      // ints
    int64_t* kfit = nullptr;
    size_t kfit_cap = 0;
    int64_t* cum = nullptr;
    size_t cum_cap = 0;
    int* src = nullptr;
    size_t src_cap = 0;
    size_t sort_smem_max = 0;
    // profiling (gapa_profile_begin/end): event pairs around launches
    bool profiling = false;
    bool capturing = false;
    struct Timed {
        cudaEvent_t a, b;
        int kind;  // 0 = fitness, 1 = operators, 2 = surrogate phase
        int evals;
        int kernels;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

// Event pair around one launch when profiling is on (no-op otherwise).
// Genes are drawn from [0, universe): n node ids, or E edge ids.
inline int gapa_gene_universe(const gapa_ctx* c) { return c->genes ? c->g.num_edges : c->g.n; }

struct ProfileScope {
    gapa_ctx* c;
    cudaStream_t st;
    int kind, evals;
    int kernels = 1;  // kernels launched inside the scope (set by launchers that issue several)
    cudaEvent_t a = nullptr, b = nullptr;
    ProfileScope(gapa_ctx* c_, cudaStream_t st_, int kind_, int evals_);
    ~ProfileScope();
};

// Error reporting (thread-local message).
int gapa_fail(int code, const char* fmt, ...);
int gapa_cuda_fail(cudaError_t e, const char* what);
#define GAPA_CUDA(call)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return gapa_cuda_fail(_e, #call); \
    } while (0)

// Raise a kernel's dynamic shared memory limit to the opt-in maximum minus its
// static shared memory; returns that limit through *max_dyn.
int gapa_set_smem_limit(const void* kernel, size_t optin, size_t* max_dyn);

// Ensure a device buffer holds at least `count` elements of size `elem`.
int gapa_reserve(void** ptr, size_t* cap, size_t count, size_t elem);

// ---------------------------------------------------------------------------
// Launchers (fitness.cu, ga.cu)
// ---------------------------------------------------------------------------
struct GaParams {
    int n, k, s, t;
    uint32_t pc_thr, pm_thr;
    RngKey key;
    uint32_t flags;
    int g;               // generation when g_ptr is null
    const int* g_ptr;    // device-resident generation counter (CUDA-graph replay)
    const long long* cum;  // roulette cumulative weights [s] (GAPA_FLAG_ROULETTE)
    // cost estimates of the rows for the cut-local fitness kernel (all null: none):
    // est_out[row] = sum over the row's genes of est_cut[gene], and the same under the second
    // forest at est_out[est_stride + row] (est_cut2 null: 0xFFFFFFFF there)
    const int* est_cut;
    const int* est_cut2;
    unsigned* est_out;
    int est_stride;
};

// One instance of a batched run (device-side descriptor).
struct BatchDesc {
    GaParams p;          // operator parameters; p.g unused (generation from the device counter)
    int32_t* pop[2];     // ping-pong populations [s][k]
    int64_t* fit[2];     // ping-pong fitness [s]
    int64_t* traj;       // [gens + 1]
    int* best;           // index of the lowest fitness after the last record
    // fitness graph in 16-bit BFS numbering (tree16.cuh)
    int n;
    const int* perm;
    const int2* palt;
    const int* lo_ptr;
    const int* lo_col;
    const unsigned* nontree;
    int num_nontree;
    const int* fptr;
    const unsigned short* fcol16;
    int mean_deg_x16;
    int objective;       // GAPA_OBJECTIVE_*
    int teams;           // members per CTA in the batched fitness kernel (1, 2, 4 or 8)
    // cut-local TREE kernel (tree16_member_local): list_bytes > 0 when each team's slice holds it;
    // the members' cost estimates come from the operator kernels through p.est_out
    const int* tparent;
    const int4* kids;
    const int* roots;
    int num_roots;
    int list_bytes;
    DeviceForest alt;    // the second forest (alt.perm null: none)
};

// A packet of the batched fitness work queue: members i0 .. i0+cnt-1 of instance b.
struct BatchPacket {
    int b, i0, cnt, teams;
};

int gapa_launch_fitness(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                        const unsigned* est = nullptr);
// True when gapa_launch_fitness runs the cut-local TREE kernel on this context (which then uses
// per-member cost estimates; callers that produce the rows may pass them precomputed).
bool gapa_fitness_uses_estimates(const gapa_ctx* c, int s);
// Threads of the one-member-per-CTA fitness kernels for a graph of n nodes.
int gapa_fitness_block_for(int n);
// Device buffer of 2 * kOrderCap cost estimates owned by the graph (valid when the above is true):
// row m's estimate under the first forest at [m], under the second at [kOrderCap + m] (0xFFFFFFFF
// when the graph has no second forest).
unsigned* gapa_estimate_buffer(gapa_ctx* c);
int gapa_launch_init_batched(const BatchDesc* d, const int2* rows, int total_rows, size_t smem, int buf,
                             cudaStream_t st);
int gapa_launch_offspring_batched(const BatchDesc* d, const int2* rows, int total_rows, size_t smem, int src,
                                  const int* gen, int* status, cudaStream_t st);
int gapa_launch_record_batched(const BatchDesc* d, int num, int buf, int* gen, bool advance, cudaStream_t st);
int gapa_launch_fitness_batched(const BatchDesc* d, const BatchPacket* pk, int npk, int* head, int buf,
                                size_t smem, int grid, int* status, cudaStream_t st);
int gapa_fitness_batched_init(size_t optin, size_t* max_dyn);
int gapa_fitness_batched_occupancy(size_t smem, int* blocks_per_sm);
int gapa_ga_batched_init(size_t optin, size_t* max_dyn);
size_t gapa_row_smem_bytes(int n, int k);
int gapa_fitness_prepare(gapa_ctx* c, int s);  // allocate scratch before capture
int gapa_launch_fitness_ig(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                           int* kernels = nullptr);
int gapa_launch_fitness_sixdst(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                               int* kernels = nullptr);
int gapa_sixdst_init(gapa_ctx* c);
int gapa_launch_selftest_wait(gapa_ctx* c, long long limit, cudaStream_t st);
int gapa_launch_read_probe(const void* buf, size_t bytes, int passes, int grid, unsigned* sink, cudaStream_t st);
int gapa_ig_prepare(gapa_ctx* c, int s);
// Sparse fitness kernel (fitness_sparse.cu): whether its shared memory fits k genes on this
// context's graph, its one-time set-up, its scratch (outside any capture) and its launch.
bool gapa_sparse_fits(const gapa_ctx* c, int k);
int gapa_sparse_init(gapa_ctx* c);
int gapa_sparse_prepare(gapa_ctx* c, int s);
int gapa_launch_fitness_sparse(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                               int* kernels = nullptr);
int gapa_launch_init(gapa_ctx* c, const GaParams& p, int32_t* pop, cudaStream_t st);
int gapa_launch_offspring(gapa_ctx* c, const GaParams& p, const int32_t* pop_in, const int64_t* fit_in,
                          int32_t* pop_out, int64_t* fit_out, cudaStream_t st);
int gapa_launch_record(gapa_ctx* c, const int64_t* fit, int s, int* gen, int64_t* traj, int* best,
                       cudaStream_t st);
int gapa_launch_roulette_prefix(const int64_t* fit, int s, int64_t* cum, cudaStream_t st);
int gapa_launch_children(gapa_ctx* c, const GaParams& p, int lambda, const int32_t* pop_in, const int64_t* fit_in,
                         int32_t* kids, cudaStream_t st);
int gapa_launch_mpl_replace(gapa_ctx* c, int mu, int lambda, int k, const int32_t* pop_in, const int64_t* fit_in,
                            const int32_t* kids, const int64_t* kfit, int* src, int32_t* pop_out, int64_t* fit_out,
                            cudaStream_t st);
int gapa_ga_check_limits(gapa_ctx* c, int n, int k, int s);
GaParams gapa_make_params(gapa_ctx* c, const gapa_config* cfg, int g, const int* g_ptr);
int gapa_run_prepare(gapa_ctx* c, const gapa_config* cfg);
int gapa_kernels_init(gapa_ctx* c);
