/*
 * gapa.h - C ABI of libgapa.so: batched critical-node-detection fitness and
 * the genetic-algorithm step on one sm_103a GPU.
 *
 * Method: Yu et al., "Efficient Parallel Genetic Algorithm for Perturbed
 * Substructure Optimization in Complex Network" (GAPA, arXiv 2412.20980).
 *  - Problem (Section III-A, Eq. 1): an undirected, unweighted graph
 *    G = (V, E) and a perturbation p of cost |p| = k; for critical node
 *    detection p is a set of k deleted nodes.
 *  - Population (Section III-B, Eq. 2): s individuals of k genes, an
 *    int32 matrix POP[s][k] in row-major order; a gene is a node id.
 *  - Fitness (Section III-C, Eq. 13; PC(G) of Table "Whole"): deleting a
 *    node removes all of its edges; the fitness of a member is the pairwise
 *    connectivity of what remains, sum over components C of |C|(|C|-1)/2,
 *    an int64 to be minimised.
 *  - Generation (Section III-B, Eqs. 3-11, Fig. 1): elitism, selection,
 *    crossover with a per-gene Bernoulli(pc) mask, mutation with a per-gene
 *    Bernoulli(pm) mask, duplicate repair, fitness of the children.
 *
 * Conventions for every call:
 *  - Return value: GAPA_OK (0) or a negative GAPA_ERR_* code; the message of
 *    the last failure on the calling thread is returned by gapa_last_error().
 *  - Ownership: the caller owns every pointer it passes; the library copies
 *    the graph at upload and owns that copy and its scratch buffers, freed by
 *    gapa_destroy().  "_dev" pointers are device memory of the context's
 *    device; "_host" pointers are host memory (pinned memory is fastest).
 *  - Asynchrony: calls that take only device pointers enqueue work on the
 *    context's stream and return at once; errors found by kernels (a gene
 *    outside [0, n), an exhausted wait) are reported by the next
 *    gapa_sync().  Calls that take host pointers return after the result is
 *    in host memory.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC 2011), key = seed,
 *    counter = (gene j, member i, generation g, tag << 24 | round); runs are
 *    bit-reproducible for a given seed and configuration.
 */
#ifndef GAPA_H
#define GAPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GAPA_OK 0
#define GAPA_ERR_INVALID_ARG -1   /* a size, pointer or configuration value is out of range */
#define GAPA_ERR_INVALID_GRAPH -2 /* CSR not simple/symmetric/in range (self-loop, duplicate, asymmetric arc) */
#define GAPA_ERR_OOM -3           /* device or host allocation failed */
#define GAPA_ERR_CUDA -4          /* a CUDA runtime call failed */
#define GAPA_ERR_TIMEOUT -5       /* a bounded device-side wait ran out */
#define GAPA_ERR_STATE -6         /* call out of order, e.g. fitness before a graph was uploaded */
#define GAPA_ERR_DEVICE -7        /* a kernel rejected its input, e.g. a gene outside [0, n) */

#define GAPA_WHERE_HOST 0
#define GAPA_WHERE_DEVICE 1

/* gapa_config.flags */
#define GAPA_FLAG_ROWWISE 1u        /* parent A of child i is member i itself (Eq. 6 read literally) */
#define GAPA_FLAG_MU_PLUS_LAMBDA 2u /* (mu+lambda) elitism of Eqs. 10-11 with `lambda` children, below */
#define GAPA_FLAG_ROULETTE 4u       /* roulette-wheel selection of Eq. 5 instead of tournaments */

typedef struct gapa_ctx gapa_ctx; /* opaque, library-owned */

/* GA configuration (Table "Params" of the paper gives pc, pm, iterations,
 * population size and perturbation rate k/n per algorithm). */
typedef struct gapa_config {
    int32_t k;       /* genes per member = deleted nodes, 0 <= k < n */
    int32_t pop;     /* population size s >= 2 */
    int32_t gens;    /* generations run by gapa_run, >= 0 */
    int32_t tourn;   /* tournament size t >= 1 (selection, Eq. 5) */
    int32_t elite;   /* elite count; must be 1 */
    uint32_t pc_thr; /* crossover mask threshold floor(pc * 2^32) (Eq. 4): mask = draw < pc_thr */
    uint32_t pm_thr; /* mutation mask threshold floor(pm * 2^32) (Eq. 8): mask = draw < pm_thr */
    uint64_t seed;   /* Philox key */
    uint32_t flags;  /* GAPA_FLAG_* */
    int32_t lambda;  /* children per generation with GAPA_FLAG_MU_PLUS_LAMBDA (>= 1; mu + lambda <= 16384) */
} gapa_config;

/* Selection variants.  Tournament (default): t draws with replacement, lower
 * fitness wins, ties to the lower index.  Roulette (GAPA_FLAG_ROULETTE,
 * Eq. 5): for minimisation the weight of member x is (max F - F_x) + 1, the
 * cumulative weights are int64, and a 64-bit Philox draw u (words 0 and 1 of
 * counter (slot, child, g, 7 << 24)) picks the first member whose cumulative
 * weight exceeds floor(u * W / 2^64).
 * Generation variants.  Default: row 0 = the elite, rows 1..s-1 = children.
 * GAPA_FLAG_MU_PLUS_LAMBDA (Eqs. 10-11): `lambda` children (counter index
 * 0..lambda-1) are bred from the s = mu members, and the mu rows of lowest
 * fitness among [members; children] (stable: members first, lower index
 * first) form the next population, sorted ascending. */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream) that the context borrows for all work;
 * it must outlive the context or be replaced with gapa_set_stream(). */
int gapa_create(gapa_ctx** out, int device, void* cuda_stream);

/* Free the context and everything it owns; NULL is ignored. */
void gapa_destroy(gapa_ctx* ctx);

/* Replace the borrowed stream. */
int gapa_set_stream(gapa_ctx* ctx, void* cuda_stream);

/* Upload the graph G (Section III-A: undirected, unweighted) as symmetric
 * CSR: row_ptr[n+1] (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz) and
 * col[nnz], every undirected edge {u,v} stored as both u->v and v->u.
 * `where` says whether the two arrays are host or device memory.  The arrays
 * are validated on the host (rows may be unsorted; no self-loops, no
 * repeated arcs, every arc has its reverse, ids in [0, n)) and copied; the
 * caller keeps ownership.  A new upload replaces the previous graph.
 * Limits: 1 <= n < 2^31, nnz < 2^31.  Synchronous. */
int gapa_graph_upload(gapa_ctx* ctx, int32_t n, int64_t nnz, const int32_t* row_ptr,
                      const int32_t* col, int where);

/* Population initialisation (Eq. 2): fills pop_dev[s][k] (s = cfg->pop,
 * k = cfg->k) with s uniformly drawn deletion sets of k distinct node ids
 * (generation 0 of the Philox stream).  Asynchronous. */
int gapa_pop_init(gapa_ctx* ctx, const gapa_config* cfg, int32_t* pop_dev);

/* Fitness of a whole population in one batch (Section III-C, Eq. 13):
 * fit_dev[i] = pairwise connectivity of G with the genes of row i of
 * pop_dev[s][k] deleted.  Repeated genes in a row count once.  A gene
 * outside [0, n) is reported by gapa_sync() as GAPA_ERR_DEVICE.
 * s >= 0, k >= 0.  Asynchronous. */
int gapa_fitness(gapa_ctx* ctx, const int32_t* pop_dev, int32_t s, int32_t k, int64_t* fit_dev);

/* Same as gapa_fitness with host arrays: copies pop_host in, runs, copies
 * fit_host out and synchronises (kernel errors are returned here). */
int gapa_fitness_host(gapa_ctx* ctx, const int32_t* pop_host, int32_t s, int32_t k, int64_t* fit_host);

/* One generation g >= 1 (Fig. 1 loop body; Eqs. 3-11) from
 * (pop_in[s][k], fit_in[s]) to (pop_out[s][k], fit_out[s]):
 *  - elitism: row 0 = the member with the lowest fitness (lowest index on
 *    ties), fitness carried over;
 *  - each child i in [1, s): parents A and B by two tournaments of size t
 *    (draws with replacement, lower fitness wins, ties to the lower index);
 *    gene j is B[j] when draw(j,i,g,XOVER) < pc_thr, else A[j]; it mutates
 *    when draw(j,i,g,MUT) < pm_thr into a node uniform over [0, n);
 *    repeated genes are repaired so that the k genes stay distinct;
 *  - fitness of rows 1 .. s-1.
 * pop_out/fit_out must not alias pop_in/fit_in.  Asynchronous. */
int gapa_generation(gapa_ctx* ctx, const gapa_config* cfg, int32_t g, const int32_t* pop_in,
                    const int64_t* fit_in, int32_t* pop_out, int64_t* fit_out);

/* Same as gapa_generation with host arrays (copies in, runs, copies out,
 * synchronises). */
int gapa_generation_host(gapa_ctx* ctx, const gapa_config* cfg, int32_t g, const int32_t* pop_in_host,
                         const int64_t* fit_in_host, int32_t* pop_out_host, int64_t* fit_out_host);

/* The operators of one generation without the children's fitness (elitism
 * mode only; GAPA_ERR_INVALID_ARG with GAPA_FLAG_MU_PLUS_LAMBDA): writes
 * pop_out[s][k] and fit_out[0] (the elite's carried fitness) exactly as
 * gapa_generation does; fit_out[1..s-1] are left to gapa_fitness on
 * pop_out + k.  Because every draw is counter-based, several processes that
 * call this with the same inputs produce the same children and can each
 * evaluate a slice of them (the member partition of Section III-D) and
 * exchange the int64 fitness.  Asynchronous. */
int gapa_offspring(gapa_ctx* ctx, const gapa_config* cfg, int32_t g, const int32_t* pop_in, const int64_t* fit_in,
                   int32_t* pop_out, int64_t* fit_out);

/* A whole run: initialisation, fitness, then cfg->gens generations, each one
 * replayed from a captured CUDA graph with the generation counter kept on
 * the device.  Outputs: best_set_host[k] = genes of the final best member
 * (lowest fitness, lowest index) in ascending order; *best_fit its fitness;
 * traj_best_fit[gens+1] (may be NULL) the lowest fitness after
 * initialisation and after every generation; final_pop_dev[s][k] (may be
 * NULL) the final population.  Synchronous. */
int gapa_run(gapa_ctx* ctx, const gapa_config* cfg, int32_t* best_set_host, int64_t* best_fit,
             int64_t* traj_best_fit, int32_t* final_pop_dev);

/* ---- Batched runs: many independent instances advanced together ----------
 * The paper runs one GA per process (acceleration modes, Section III-D); a
 * batch advances `num` independent GA instances - each with its own graph
 * (an uploaded context) and configuration - with one operator launch, one
 * persistent fitness launch over a work queue of (instance, members) packets
 * and one record launch per generation, two generations captured as a CUDA
 * graph and replayed.  Every instance's trajectory, final population and best
 * set equal those of gapa_run() on its own context and configuration.
 * Limits: every graph must fit the shared-memory fitness path (at most
 * ~57,000 nodes; GAPA_ERR_INVALID_ARG otherwise); all contexts on one device;
 * the batch borrows the contexts (they must outlive it) and runs on the first
 * context's stream. */
typedef struct gapa_batch gapa_batch;

int gapa_batch_create(gapa_batch** out, int32_t num, gapa_ctx* const* ctxs, const gapa_config* cfgs);
void gapa_batch_destroy(gapa_batch* batch);

/* Members per CTA of the persistent fitness kernel (1, 2, 4 or 8 teams of
 * 1024/teams threads) per instance; results do not depend on it. */
int gapa_batch_set_teams(gapa_batch* batch, const int32_t* teams /* [num] */);
int gapa_batch_get_teams(gapa_batch* batch, int32_t* teams /* [num] */);

/* Autotuner: for every graph-size bucket present (n <= 2048, 4096, 8192,
 * 16384, 32768, 65536) time each feasible team count on the initial
 * population and keep the fastest; choices are cached per device name in
 * the JSON file `cache_path` (NULL: no cache).  Batched instances follow
 * their context's fitness kernel setting as single runs do: AUTO takes the
 * cut-local kernel above 2048 nodes (in each team's slice, with the
 * operator kernels' cost estimates), TREE_LOCAL always, anything else the
 * full TREE pipeline. */
int gapa_batch_autotune(gapa_batch* batch, const char* cache_path);

/* Run every instance for `gens` generations from its initialisation.
 * Outputs (host): best_fit[num]; best_sets = the k_i genes of each
 * instance's best member, concatenated in instance order, each ascending
 * (may be NULL); traj[num][gens+1] the lowest fitness after initialisation
 * and after every generation (may be NULL).  Synchronous. */
int gapa_batch_run(gapa_batch* batch, int32_t gens, int64_t* best_fit, int32_t* best_sets, int64_t* traj);

/* ---- Learned fitness surrogate (an extension; the paper has no surrogate) ----
 * A small MLP scores children so that only the most promising fraction gets
 * the exact fitness of Section III-C; exact fitness stays the arbiter of every
 * member kept.  Input of a deletion set D of k genes (80 values):
 * (1/sqrt k) * sum of the 64-d embeddings of its genes, then the mean, maximum
 * and standard deviation of log1p(degree) over D and sum(degree)/(2E), then
 * log1p(r0), log1p(r1) and log1p(r2): the numbers of live neighbours of D
 * that G[V\D] leaves with no live neighbour and with exactly one, and the
 * number of two-node components of G[V\D] adjacent to D; then the same three
 * counts standardised over the rows scored together ((r_j - mean_j) /
 * max(sd_j, 1), population statistics over the rows of one predict or
 * training call, or of one generation's children); then zeros.
 * Model: 80 -> 256 ReLU -> 256 ReLU -> 1, BF16 weights on the tensor
 * cores with FP32 accumulation; FP32 master weights, AdamW (Loshchilov &
 * Hutter) on every parameter, MSE against the z-scored log1p of the exact
 * fitness (over the replay ring or among siblings, see target_mode).  Training is deterministic (fixed-order reductions, fixed-point
 * embedding-gradient sums). */
typedef struct gapa_surrogate_config {
    int32_t screened;     /* children evaluated exactly per generation once screening starts */
    int32_t warmup;       /* generations in which every child is evaluated exactly */
    int32_t train_steps;  /* AdamW steps per generation */
    int32_t batch;        /* minibatch rows, a multiple of 16 */
    int32_t ring;         /* replay ring capacity (rows of (deletion set, exact fitness)) */
    float lr, beta1, beta2, weight_decay, eps;
    float init_scale_emb; /* embeddings start uniform in [-a, a] */
    int32_t diag_every;   /* every diag_every-th generation evaluates all children exactly and records
                             (estimate, fitness) pairs; 0 = never */
    int32_t target_mode;  /* training target: 0 = log1p(PC) z-scored over the whole replay ring,
                             1 = z-scored among the exactly evaluated children of the row's own
                             generation (only the order of siblings matters for screening) */
} gapa_surrogate_config;

typedef struct gapa_surrogate gapa_surrogate;

/* A surrogate for the context's graph, weights initialised from Philox(seed).
 * Every call but gapa_surrogate_destroy needs the context alive and holding
 * the same graph (GAPA_ERR_STATE after a new upload); destruction is safe in
 * any order. */
int gapa_surrogate_create(gapa_surrogate** out, gapa_ctx* ctx, const gapa_surrogate_config* scfg, uint64_t seed);
void gapa_surrogate_destroy(gapa_surrogate* sg);

/* scores_dev[r] = model output for row r of pop_dev[rows][k].  Asynchronous.
 * Genes outside [0, n) are ignored by the features.  The standardised counts
 * make a score relative to the other rows of the same call. */
int gapa_surrogate_predict(gapa_surrogate* sg, const int32_t* pop_dev, int32_t rows, int32_t k, float* scores_dev);

/* Residual counts of the rows of pop_dev[rows][k]: counts_dev[3r .. 3r+2] =
 * (r0, r1, r2) (device int32 [rows][3]).  Asynchronous. */
int gapa_surrogate_residual(gapa_surrogate* sg, const int32_t* pop_dev, int32_t rows, int32_t k, int32_t* counts_dev);

/* One AdamW step on a minibatch (rows a multiple of 16) with device targets;
 * *loss_host (may be NULL) receives the batch MSE before the step. */
int gapa_surrogate_train_step(gapa_surrogate* sg, const int32_t* pop_dev, int32_t rows, int32_t k,
                              const float* target_dev, float* loss_host);

/* Copy a parameter (grad = 0) or its last gradient (grad = 1) to (set = 0)
 * or from (set = 1) host memory.  which: 0 W1 [80][256], 1 b1, 2 W2
 * [256][256] ([in][out]), 3 b2, 4 w3, 5 b3, 6 embeddings [n][64]. */
int gapa_surrogate_tensor(gapa_surrogate* sg, int32_t which, int32_t grad, float* host, int64_t count, int32_t set);

/* A (mu+lambda) run (cfg->flags must hold GAPA_FLAG_MU_PLUS_LAMBDA) whose
 * children are screened by the surrogate: after `warmup` generations only
 * the `screened` children with the lowest scores are evaluated exactly, the
 * others are excluded from the truncation; every exactly evaluated child
 * enters the replay ring and the model takes `train_steps` AdamW steps per
 * generation.  sg = NULL runs the plain (mu+lambda) GA (every child exact) -
 * the fallback - with the same outputs.  Outputs: best fitness and set,
 * traj[gens+1], gen_ms[gens+1] (elapsed device time at the end of
 * initialisation and of every generation, may be NULL), exact_evals[gens+1]
 * (may be NULL), and diagnostic pairs: in every diag_every-th generation
 * (while diag_cap rows remain) all lambda children are evaluated exactly and
 * used, and diag_pred receives the model's estimate of each child's pairwise
 * connectivity (expm1 of the de-normalised score, FP32) beside its exact
 * value in diag_exact.  Synchronous. */
int gapa_run_surrogate(gapa_ctx* ctx, const gapa_config* cfg, gapa_surrogate* sg, int64_t* best_fit,
                       int32_t* best_set, int64_t* traj, double* gen_ms, int64_t* exact_evals, float* diag_pred,
                       int64_t* diag_exact, int32_t diag_cap);

/* Fitness kernel selection (all are exact and give identical results):
 * TREE starts every member from a BFS spanning forest of G (numbered so that
 * parents precede children), cuts it at the deleted nodes, reattaches each
 * piece to a live lower-numbered neighbour where it can, and then joins what
 * is left: per member it either lets the nodes outside the piece of the
 * first live node scan their adjacency (when their adjacency is shorter than
 * the list of non-tree edges) or unites along every non-tree edge.
 * TREE_JOIN and TREE_SCAN force one of the two (for tests and measurement).
 * TREE_LOCAL reaches the same pieces with work local to the deletion: the
 * tree parents are bulk-copied into the labels, only the children of deleted
 * nodes are re-picked, and only the pieces whose root is not the first live
 * node are listed (level by level down the tree) and scanned; a member whose
 * list outgrows the kernel's shared memory, or with repeated genes, takes
 * the TREE path.  It needs n <= 65536 and a BFS tree whose children carry
 * consecutive numbers (always so for the upload's numbering).
 * SAMPLED joins every live node to its first two live neighbours, takes the
 * tree of the highest-degree live node as the giant tree and lets only nodes
 * outside it scan their whole adjacency; EDGES runs union-find over every
 * undirected edge.  AUTO (the default) is TREE_LOCAL where it applies and
 * the graph has more than 2048 nodes, else TREE.  Where the labels do not fit
 * in shared memory (n above about 56,000 on GB300), AUTO runs SPARSE
 * (below), the TREE settings run the same phases on labels in global memory,
 * eight members interleaved per 32-byte sector, and EDGES and SAMPLED run one
 * CTA per member over a global label array. */
#define GAPA_FITNESS_AUTO 0
#define GAPA_FITNESS_EDGES 1
#define GAPA_FITNESS_SAMPLED 2
#define GAPA_FITNESS_TREE 3
#define GAPA_FITNESS_TREE_JOIN 4
#define GAPA_FITNESS_TREE_SCAN 5
#define GAPA_FITNESS_TREE_LOCAL 6
/* PIECE (selectable only; AUTO never picks it): the forest-piece kernel,
 * four members per SM with no per-node labels.  Deleting a member's nodes cuts the upload's spanning forest into
 * pieces rooted at the live children of deleted nodes (and at the live roots
 * of trees holding deleted nodes); piece sizes follow from subtree sizes by
 * subtraction, every such child re-picks a live lower-numbered neighbour
 * (a union of two pieces), and only the nodes outside the largest resulting
 * class scan their arcs.  Members estimated to list over a quarter of the
 * nodes, or beyond the kernel's shared-memory capacities, run the TREE_LOCAL
 * kernel instead.  Same graphs as TREE_LOCAL; PC and MCN objectives. */
#define GAPA_FITNESS_PIECE 7
/* SPARSE (AUTO's choice where the labels do not fit in shared memory, and
 * selectable on any graph): work proportional to what the deletion disturbs.
 * In the BFS forest every live child of a deleted node ("top") re-picks its
 * first live lower-numbered neighbour and hops to the first top or tree root
 * above that neighbour; hops decrease, so chains end at terminals (live tree
 * roots, or tops that re-picked nothing) whose chained pieces are joined;
 * tops chained to the latter unite their terminal's class with those of a
 * few live neighbours (neighbour sampling).  Per touched component the class
 * of one reference terminal (the root if live, else the terminal carrying
 * the most subtree nodes) is kept whole; the pieces of the other classes are
 * listed, their arcs unite classes, and PC follows from the graph's PC, the
 * touched components' sizes and the classes apart from the reference.  One
 * CTA per member with the deletion bitmap, the deleted nodes and their child
 * offsets in shared memory (n/8 + 8k bytes + 12 KB: n = 2^20 with k up to
 * about 12,000 on GB300; otherwise the TREE setting runs), per-CTA state in
 * library-owned global scratch (32 bytes per node per resident CTA), cleared
 * after each member.  PC and MCN objectives. */
#define GAPA_FITNESS_SPARSE 8
int gapa_set_fitness_kernel(gapa_ctx* ctx, int variant);

/* Fitness objective of the context (all minimised; the end of Section III-C
 * and the PC(G) and MCN rows of Table "Whole"): PC = pairwise connectivity
 * Σ C(|C|, 2) over the components C of G[V\D] (the default); MCN = maximum
 * connectivity number, the number of nodes of the largest component (0 when
 * every node is deleted).  SIXDST_PC / SIXDST_MCN: the same read from the
 * dense accessibility matrix M = Normalizer((A + I)^N) of the perturbed
 * adjacency matrix (Eqs. 14-17), N = gapa_set_sixdst_hops (default 6):
 * with rowsum(v) = the live nodes within N hops of live v (itself included),
 * PC_N = (Σ_live rowsum - live) / 2 and MCN_N = max_live rowsum, equal to PC
 * and MCN once N reaches every component's diameter; node genes, n <= 8192,
 * tensor-core products.  Applies to gapa_fitness and the generation and run
 * calls (batches take PC and MCN); gapa_fitness_noalloc computes PC. */
#define GAPA_OBJECTIVE_PC 0
#define GAPA_OBJECTIVE_MCN 1
#define GAPA_OBJECTIVE_SIXDST_PC 2
#define GAPA_OBJECTIVE_SIXDST_MCN 3
int gapa_set_objective(gapa_ctx* ctx, int objective);
int gapa_set_sixdst_hops(gapa_ctx* ctx, int hops);
/* Tensor-core path of the SixDST products (identical results): TMA (the
 * default: tcgen05.mma with the accumulator in tensor memory, operands loaded
 * by cp.async.bulk.tensor from a tensor map by a producer thread while another
 * issues the products, six stages, 256 x 256 output tiles when the padded size
 * is a multiple of 256, else as TCGEN05), TCGEN05 (the same products with
 * operands loaded by every thread with cp.async, three stages; 256 x 256 tiles
 * when the padded size allows, else 128 x 128), TCGEN05_128 (128 x 128 tiles
 * only) or MMA_SYNC (warp-level mma.sync).  A device-side wait that runs out is
 * reported as GAPA_ERR_TIMEOUT. */
#define GAPA_SIXDST_MMA_SYNC 0
#define GAPA_SIXDST_TCGEN05 1
#define GAPA_SIXDST_TCGEN05_128 2
#define GAPA_SIXDST_TMA 3
int gapa_set_sixdst_kernel(gapa_ctx* ctx, int kernel);

/* Failure-path check of the device-side bounded waits (the paper has no
 * counterpart): one thread waits at most spin_limit polls (1 .. 2^26) on an
 * mbarrier that nothing completes - the wait the tcgen05 products use - and
 * records the timeout; returns GAPA_ERR_TIMEOUT, after which the context stays
 * usable.  Synchronous. */
int gapa_selftest_wait(gapa_ctx* ctx, int64_t spin_limit);

/* Measurement utility (the paper has no counterpart): read bandwidth of this
 * device over a buffer of `bytes` (a multiple of 16, 1 MiB .. 1 GiB) that the
 * library allocates and fills: one warm-up pass, then `reps` timed launches
 * of 16-byte loads by a grid of 8 CTAs per SM, each reading the buffer
 * max(1, 2^30 / bytes) times; *gbs = bytes read / the fastest launch.
 * A buffer well inside L2 gives the L2 read bandwidth, one far above it the
 * HBM read bandwidth.  Synchronous; frees the buffer. */
int gapa_read_bandwidth(gapa_ctx* ctx, int64_t bytes, int32_t reps, double* gbs);

/* Gene type of the context (Fig. 1: the gene pool holds nodes or edges; end
 * of Section III-A: both perturbations act on the adjacency matrix).  NODES
 * (the default): genes are node ids in [0, n), deleting a node removes its
 * edges.  EDGES: genes are edge ids in [0, E) - the undirected edges {u, v},
 * u < v, numbered in CSR order (u ascending, then v ascending) - and every
 * node stays; the fitness is the objective of G without those edges.  With
 * EDGES, cfg->k must be below E, the population and initialisation draw from
 * [0, E), and the labels plus an E-bit mask must fit in shared memory
 * (GAPA_ERR_INVALID_ARG otherwise); batches, the surrogate and
 * gapa_fitness_noalloc use node genes only. */
#define GAPA_GENES_NODES 0
#define GAPA_GENES_EDGES 1
int gapa_set_genes(gapa_ctx* ctx, int gene_type);

/* Per-kernel timing of the calls made between gapa_profile_begin() and
 * gapa_profile_end(): CUDA events are recorded on the launching stream around
 * every fitness launch, every genetic-operator launch and every phase of
 * the learned surrogate (not inside the graph replays of gapa_run).
 * gapa_profile_end() synchronises and returns the totals. */
typedef struct gapa_profile {
    double fitness_ms;          /* summed duration of fitness launches */
    double operators_ms;        /* summed duration of genetic-operator launches (init, offspring, children,
                                   (mu+lambda) replacement, best-so-far record) */
    int64_t fitness_launches;   /* fitness kernel launches */
    int64_t operator_launches;  /* genetic-operator kernel launches */
    int64_t evals;              /* population members evaluated by those fitness launches */
    double surrogate_ms;        /* summed duration of surrogate phases (features, MLP, selection, training) */
    int64_t surrogate_launches; /* kernels launched by those phases */
    int64_t fitness_calls;      /* fitness phases (one per batch of members evaluated; a phase may launch
                                   several kernels, counted in fitness_launches) */
} gapa_profile;

int gapa_profile_begin(gapa_ctx* ctx);
int gapa_profile_end(gapa_ctx* ctx, gapa_profile* out);

/* Fitness without any allocation.  The paper has no counterpart.  Some
 * callers cannot allocate device memory: a plugin or library embedded in a
 * host program whose device memory belongs to that program's own allocator
 * under a fixed budget, and latency-critical loops that cannot take the
 * implicit device-wide synchronisation of cudaMalloc/cudaFree.  This entry
 * point serves them.  It needs no context: the graph comes as a device edge
 * list edges_dev[num_edges][2] (int32 node ids; each undirected edge at least
 * once, either orientation; self-loops ignored), the population pop_dev[s][k]
 * and the output fit_dev[s] are the caller's device arrays on `device`, and
 * work runs on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * fit_dev[i] is the same pairwise connectivity as gapa_fitness().
 * Scratch: the node labels live in a static device array of
 * GAPA_NOALLOC_MAX_LABELS int32 (32 MiB) inside the library, which every GPU
 * that loads the library holds until the process exits; n above that limit is
 * rejected with GAPA_ERR_INVALID_ARG, and members run in waves of
 * GAPA_NOALLOC_MAX_LABELS / n.  A status word beside it is cleared at the
 * start of every call.  The call allocates nothing (no cudaMalloc, cudaFree
 * or allocating library routine) and BLOCKS: it copies the status word to
 * the host and synchronises `cuda_stream` before returning; an endpoint or a
 * gene outside [0, n) then gives GAPA_ERR_DEVICE, and the next call starts
 * clean.  Set-up: the first call on a device, with that device current, looks
 * up the scratch's device address (cudaGetSymbolAddress) and caches it for
 * the life of the process; make that first call before any stream capture,
 * and do not call again after cudaDeviceReset on that device (unsupported:
 * the cached address may be stale).  All calls share the one scratch array,
 * which keeps the last call's labels; calls that overlap on the GPU (other
 * streams, threads or processes sharing the library) race on it and must be
 * serialised by the caller. */
#define GAPA_NOALLOC_MAX_LABELS (8 * 1024 * 1024)
int gapa_fitness_noalloc(int device, void* cuda_stream, int32_t n, int32_t num_edges, const int32_t* edges_dev,
                         const int32_t* pop_dev, int32_t s, int32_t k, int64_t* fit_dev);

/* Wait for the context's stream and report device-side errors (then clear
 * them). */
int gapa_sync(gapa_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* gapa_last_error(void);

/* Library version string. */
const char* gapa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GAPA_H */
