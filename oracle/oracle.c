/*
 * CPU oracle for the GAPA critical-node-detection hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline arm may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both follow the same written
 * definitions independently.
 *
 * What it computes (paper: Yu et al., "Efficient Parallel Genetic Algorithm for
 * Perturbed Substructure Optimization in Complex Network", arXiv 2412.20980):
 *
 *  - Fitness of a deletion set D (Section III-C, Eq. 13 with node deletion =
 *    removal of every incident edge; the CND quality metric PC(G) of
 *    Table "Whole"): the pairwise connectivity of G[V \ D],
 *        PC(D) = sum over connected components C of G[V \ D] of |C|(|C|-1)/2,
 *    in int64.  Two independent computations: breadth-first search from every
 *    unvisited live node in ascending id order (oracle_pc_bfs), and a
 *    union-find with union by size and full path compression over the edges
 *    in CSR order (oracle_pc_uf).
 *  - The genetic operators of Section III-B in the paper's order: population
 *    initialisation (Eq. 2), selection + crossover with a Bernoulli(pc) mask
 *    per gene (Eqs. 3-6), mutation with a Bernoulli(pm) mask and replacement
 *    genes (Eqs. 7-9), fitness, and elitism.  Where the paper is silent the
 *    readings are fixed as follows (and the CUDA path follows the same ones):
 *      * selection: tournament of size t drawn with replacement, lower PC
 *        wins, ties to the lower index (the paper's Eq. 5 uses roulette);
 *      * elitism: the single best member (lowest PC, lowest index) is copied
 *        unchanged to row 0 with its fitness carried over;
 *      * a child's gene j comes from parent B when the crossover mask is set,
 *        else from parent A (Eq. 6 with both parents chosen by selection);
 *      * duplicate genes are repaired by a deterministic rule (see repair()).
 *  - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
 *    Random Numbers: As Easy as 1, 2, 3", SC 2011), counter
 *    (j, i, g, tag << 24 | round), key (seed low word, seed high word); word 0
 *    of the output is used.  Bernoulli(p) is x < floor(p * 2^32) with the
 *    threshold passed in as an integer; uniform in [0, n) is (x * n) >> 32.
 *
 * Parity: PC is pinned by closed forms, brute force, scipy and the dense
 * reachability identity of Eqs. 14-17; Philox by an independent
 * implementation; the genetic operators by statistical laws and special
 * cases; the duplicate rule, the word-to-[0, n) map and the counter layout
 * (this build's own definitions: the paper is silent on them) by hand-worked
 * children built through oracle_child_explicit (see the tests).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                        */
/* ------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { TAG_INIT = 1, TAG_SEL = 2, TAG_XOVER = 3, TAG_MUT = 4, TAG_MUTVAL = 5, TAG_REPAIR = 6, TAG_ROULETTE = 7 };
#define REPAIR_ROUNDS 32

static uint32_t draw(uint64_t seed, uint32_t j, uint32_t i, uint32_t g, uint32_t tag, uint32_t round)
{
    uint32_t ctr[4] = { j, i, g, (tag << 24) | round };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* Words 0 and 1 of the same counter as one 64-bit number (word 0 high). */
static uint64_t draw64(uint64_t seed, uint32_t j, uint32_t i, uint32_t g, uint32_t tag, uint32_t round)
{
    uint32_t ctr[4] = { j, i, g, (tag << 24) | round };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return ((uint64_t)out[0] << 32) | (uint64_t)out[1];
}

static int32_t uniform_below(uint32_t x, int32_t n)
{
    return (int32_t)(((uint64_t)x * (uint64_t)(uint32_t)n) >> 32);
}

/* ------------------------------------------------------------------ */
/* Fitness: pairwise connectivity of the residual graph                 */
/* ------------------------------------------------------------------ */

/* Error codes shared only within this file and its Python loader. */
#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -3

/* Marks the deletion set in `dead` (n bytes, zeroed here).  Genes outside
 * [0, n) make the set invalid. */
static int mark_deleted(int32_t n, const int32_t* genes, int32_t k, uint8_t* dead)
{
    memset(dead, 0, (size_t)n);
    for (int32_t j = 0; j < k; j++) {
        if (genes[j] < 0 || genes[j] >= n) return ORACLE_EINVAL;
        dead[genes[j]] = 1;
    }
    return ORACLE_OK;
}

/* BFS over G[V \ D]; writes the component sizes in discovery order to
 * sizes_out (may be NULL) and returns the number of components, or < 0. */
int64_t oracle_components_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col,
                              const int32_t* genes, int32_t k, int32_t* sizes_out)
{
    uint8_t* dead = (uint8_t*)malloc((size_t)n + 1);
    uint8_t* seen = (uint8_t*)calloc((size_t)n + 1, 1);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!dead || !seen || !queue) { free(dead); free(seen); free(queue); return ORACLE_ENOMEM; }
    if (mark_deleted(n, genes, k, dead) != ORACLE_OK) { free(dead); free(seen); free(queue); return ORACLE_EINVAL; }
    int64_t ncomp = 0;
    for (int32_t start = 0; start < n; start++) {
        if (dead[start] || seen[start]) continue;
        int32_t head = 0, tail = 0;
        queue[tail++] = start;
        seen[start] = 1;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                int32_t v = col[e];
                if (!dead[v] && !seen[v]) { seen[v] = 1; queue[tail++] = v; }
            }
        }
        if (sizes_out) sizes_out[ncomp] = tail;
        ncomp++;
    }
    free(dead); free(seen); free(queue);
    return ncomp;
}

/* Maximum connectivity number (end of Section III-C; MCN rows of Table
 * "Whole"): the number of nodes of the largest connected component of
 * G[V \ D], 0 when every node is deleted. */
int64_t oracle_mcn_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col,
                       const int32_t* genes, int32_t k)
{
    int32_t* sizes = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!sizes) return ORACLE_ENOMEM;
    int64_t ncomp = oracle_components_bfs(n, row_ptr, col, genes, k, sizes);
    if (ncomp < 0) { free(sizes); return ncomp; }
    int64_t best = 0;
    for (int64_t c = 0; c < ncomp; c++) if (sizes[c] > best) best = sizes[c];
    free(sizes);
    return best;
}

int64_t oracle_pc_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col,
                      const int32_t* genes, int32_t k)
{
    int32_t* sizes = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!sizes) return ORACLE_ENOMEM;
    int64_t ncomp = oracle_components_bfs(n, row_ptr, col, genes, k, sizes);
    if (ncomp < 0) { free(sizes); return ncomp; }
    int64_t pc = 0;
    for (int64_t c = 0; c < ncomp; c++) pc += (int64_t)sizes[c] * (int64_t)(sizes[c] - 1) / 2;
    free(sizes);
    return pc;
}

static int32_t uf_find(int32_t* parent, int32_t x)
{
    int32_t root = x;
    while (parent[root] != root) root = parent[root];
    while (parent[x] != root) { int32_t next = parent[x]; parent[x] = root; x = next; }
    return root;
}

int64_t oracle_pc_uf(int32_t n, const int32_t* row_ptr, const int32_t* col,
                     const int32_t* genes, int32_t k)
{
    uint8_t* dead = (uint8_t*)malloc((size_t)n + 1);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t* size = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!dead || !parent || !size) { free(dead); free(parent); free(size); return ORACLE_ENOMEM; }
    if (mark_deleted(n, genes, k, dead) != ORACLE_OK) { free(dead); free(parent); free(size); return ORACLE_EINVAL; }
    for (int32_t v = 0; v < n; v++) { parent[v] = v; size[v] = 1; }
    for (int32_t u = 0; u < n; u++) {
        if (dead[u]) continue;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            int32_t v = col[e];
            if (v <= u || dead[v]) continue;
            int32_t ru = uf_find(parent, u), rv = uf_find(parent, v);
            if (ru == rv) continue;
            if (size[ru] < size[rv]) { int32_t t = ru; ru = rv; rv = t; }
            parent[rv] = ru;
            size[ru] += size[rv];
        }
    }
    int64_t pc = 0;
    for (int32_t v = 0; v < n; v++)
        if (!dead[v] && parent[v] == v) pc += size[v] * (size[v] - 1) / 2;
    free(dead); free(parent); free(size);
    return pc;
}

/* ------------------------------------------------------------------ */
/* Edge perturbation (Section III-C: node and edge perturbations both  */
/* act on the adjacency matrix; Fig. 1: genes are nodes or edges)      */
/* ------------------------------------------------------------------ */
/* Edge ids: the undirected edges {u, v}, u < v, numbered in CSR order
 * (u ascending, then v ascending; rows are sorted).  arc_id[e] = id of the
 * edge of arc e, for both orientations (the reverse arc is found by binary
 * search in the sorted row).  Returns the number of edges, or < 0. */
static int64_t edge_ids(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* arc_id)
{
    int32_t next = 0;
    for (int32_t u = 0; u < n; u++)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++)
            if (col[e] > u) arc_id[e] = next++;
    for (int32_t u = 0; u < n; u++)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            const int32_t v = col[e];
            if (v >= u) continue;
            int32_t lo = row_ptr[v], hi = row_ptr[v + 1];
            while (lo < hi) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= row_ptr[v + 1] || col[lo] != u) return ORACLE_EINVAL;  /* not symmetric */
            arc_id[e] = arc_id[lo];
        }
    return next;
}

/* PC (objective 0) or MCN (objective 1) of G with the edges `egenes` removed
 * (every node stays): BFS over the remaining arcs. */
int64_t oracle_edge_fitness(int32_t n, const int32_t* row_ptr, const int32_t* col,
                            const int32_t* egenes, int32_t k, int32_t objective)
{
    const int64_t nnz = row_ptr[n];
    int32_t* arc_id = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nnz + 1));
    uint8_t* seen = (uint8_t*)calloc((size_t)n + 1, 1);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint8_t* gone = NULL;
    int64_t result = ORACLE_ENOMEM;
    if (!arc_id || !seen || !queue) goto done;
    const int64_t m = edge_ids(n, row_ptr, col, arc_id);
    if (m < 0) { result = m; goto done; }
    gone = (uint8_t*)calloc((size_t)m + 1, 1);
    if (!gone) goto done;
    for (int32_t j = 0; j < k; j++) {
        if (egenes[j] < 0 || egenes[j] >= m) { result = ORACLE_EINVAL; goto done; }
        gone[egenes[j]] = 1;
    }
    result = 0;
    for (int32_t start = 0; start < n; start++) {
        if (seen[start]) continue;
        int32_t head = 0, tail = 0;
        queue[tail++] = start;
        seen[start] = 1;
        while (head < tail) {
            const int32_t u = queue[head++];
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                const int32_t v = col[e];
                if (!gone[arc_id[e]] && !seen[v]) { seen[v] = 1; queue[tail++] = v; }
            }
        }
        if (objective) { if (tail > result) result = tail; }
        else result += (int64_t)tail * (int64_t)(tail - 1) / 2;
    }
done:
    free(arc_id); free(seen); free(queue); free(gone);
    return result;
}

/* Fitness of s members (rows of k genes) with the chosen method
 * (0 = PC by BFS, 1 = PC by union-find, 2 = MCN by BFS; genes are nodes;
 * 3 = PC, 4 = MCN with genes that are edge ids), in parallel over members
 * when nthreads > 1.  Returns ORACLE_OK or the first error. */
int oracle_fitness(int32_t n, const int32_t* row_ptr, const int32_t* col,
                   const int32_t* pop, int32_t s, int32_t k, int64_t* fit,
                   int32_t method, int32_t nthreads)
{
    int err = ORACLE_OK;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t i = 0; i < s; i++) {
        const int32_t* genes = pop + (size_t)i * (size_t)k;
        int64_t v = method == 0   ? oracle_pc_bfs(n, row_ptr, col, genes, k)
                    : method == 1 ? oracle_pc_uf(n, row_ptr, col, genes, k)
                    : method == 2 ? oracle_mcn_bfs(n, row_ptr, col, genes, k)
                                  : oracle_edge_fitness(n, row_ptr, col, genes, k, method == 4);
        fit[i] = v;
        if (v < 0) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (err == ORACLE_OK) err = (int)v; }
        }
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* Genetic operators                                                    */
/* ------------------------------------------------------------------ */

/* Kept-set as one byte per node (plain and slow on purpose). */
typedef struct {
    int32_t n;
    uint8_t* in;
} keptset;

/* Where the candidates of repair rounds r >= 1 come from: uniform over [0, n)
 * from draw(j, i, g, REPAIR, r), or - for the hand-worked cases of the tests
 * (oracle_child_explicit) - an explicit table later[(r - 1) * k + j]. */
typedef struct {
    uint64_t seed;
    int32_t i, g, k;
    const int32_t* later; /* NULL: Philox */
} repair_source;

static int32_t repair_candidate(const repair_source* src, int32_t j, int32_t r, int32_t n)
{
    if (src->later) return src->later[(size_t)(r - 1) * (size_t)src->k + (size_t)j];
    return uniform_below(draw(src->seed, (uint32_t)j, (uint32_t)src->i, (uint32_t)src->g, TAG_REPAIR, (uint32_t)r), n);
}

/* Duplicate repair (the paper is silent on duplicates).  `holes` lists the
 * positions without a gene in ascending order, `cand0` their first
 * candidates.  Round r = 0 .. 31: every remaining hole, in ascending position
 * order, takes its round-r candidate if that node is not in the kept set, and
 * the node joins the kept set at once.  The round-0 candidate is cand0; a
 * later round's candidate comes from repair_candidate().  Holes still open
 * after round 31 take, in ascending position order, the smallest node id not
 * in the kept set. */
static void repair(const repair_source* src, int32_t n, keptset* kept,
                   int32_t* row, int32_t* holes, int32_t nholes, const int32_t* cand0)
{
    for (int32_t r = 0; r < REPAIR_ROUNDS && nholes > 0; r++) {
        int32_t still = 0;
        for (int32_t h = 0; h < nholes; h++) {
            int32_t j = holes[h];
            int32_t c = r == 0 ? cand0[h] : repair_candidate(src, j, r, n);
            if (!kept->in[c]) {
                kept->in[c] = 1;
                row[j] = c;
            } else {
                holes[still++] = j;
            }
        }
        nholes = still;
    }
    int32_t next = 0;
    for (int32_t h = 0; h < nholes; h++) {
        while (kept->in[next]) next++;
        kept->in[next] = 1;
        row[holes[h]] = next;
    }
}

/* Population initialisation (Eq. 2): member i is a uniformly drawn k-subset:
 * every position is a hole whose round-0 candidate is uniform over [0, n) from
 * draw(j, i, 0, INIT, 0), then the repair rule runs with generation 0. */
int oracle_pop_init(int32_t n, int32_t k, int32_t s, uint64_t seed, int32_t* pop)
{
    if (n < 1 || k < 0 || k >= n || s < 1) return ORACLE_EINVAL;
    keptset kept = { n, (uint8_t*)malloc((size_t)n) };
    int32_t* holes = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    int32_t* cand0 = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    if (!kept.in || !holes || !cand0) { free(kept.in); free(holes); free(cand0); return ORACLE_ENOMEM; }
    for (int32_t i = 0; i < s; i++) {
        int32_t* row = pop + (size_t)i * (size_t)k;
        memset(kept.in, 0, (size_t)n);
        for (int32_t j = 0; j < k; j++) {
            holes[j] = j;
            cand0[j] = uniform_below(draw(seed, (uint32_t)j, (uint32_t)i, 0, TAG_INIT, 0), n);
        }
        const repair_source src = { seed, i, 0, k, NULL };
        repair(&src, n, &kept, row, holes, k, cand0);
    }
    free(kept.in); free(holes); free(cand0);
    return ORACLE_OK;
}

/* Tournament of size t for parent slot `slot` of child i (selection; the
 * paper's Eq. 5 uses roulette, this reading uses tournaments): draw t indices
 * with replacement, uniform over [0, s) from draw(slot*t + r, i, g, SEL, 0);
 * the lowest fitness wins, ties to the lower index. */
static int32_t tournament(uint64_t seed, int32_t i, int32_t g, int32_t slot, int32_t t,
                          int32_t s, const int64_t* fit)
{
    int32_t best = -1;
    for (int32_t r = 0; r < t; r++) {
        int32_t x = uniform_below(draw(seed, (uint32_t)(slot * t + r), (uint32_t)i, (uint32_t)g, TAG_SEL, 0), s);
        if (best < 0 || fit[x] < fit[best] || (fit[x] == fit[best] && x < best)) best = x;
    }
    return best;
}

#define ORACLE_FLAG_ROWWISE 1u
#define ORACLE_FLAG_MU_PLUS_LAMBDA 2u
#define ORACLE_FLAG_ROULETTE 4u
#define ORACLE_FLAG_MCN 8u      /* fitness = MCN instead of PC */
#define ORACLE_FLAG_EDGES 16u   /* genes are edge ids in [0, E) instead of node ids */

/* Gene universe and fitness method of a run under `flags`. */
static int32_t gene_universe(int32_t n, const int32_t* row_ptr, uint32_t flags)
{
    return (flags & ORACLE_FLAG_EDGES) ? row_ptr[n] / 2 : n;
}

static int32_t fitness_method(uint32_t flags)
{
    const int mcn = (flags & ORACLE_FLAG_MCN) != 0;
    return (flags & ORACLE_FLAG_EDGES) ? (mcn ? 4 : 3) : (mcn ? 2 : 0);
}

/* Roulette-wheel selection (Eq. 5) for minimisation with integer weights:
 * w_x = (max F - F_x) + 1, cumulative sums cum[x] = w_0 + ... + w_x (int64);
 * a 64-bit draw u (words 0, 1 of draw(slot, i, g, ROULETTE, 0)) gives
 * r = floor(u * W / 2^64) with W = cum[s-1]; the parent is the smallest x with
 * cum[x] > r. */
static void roulette_weights(const int64_t* fit, int32_t s, int64_t* cum)
{
    int64_t mx = fit[0];
    for (int32_t x = 1; x < s; x++) if (fit[x] > mx) mx = fit[x];
    int64_t acc = 0;
    for (int32_t x = 0; x < s; x++) { acc += (mx - fit[x]) + 1; cum[x] = acc; }
}

static int32_t roulette(uint64_t seed, int32_t i, int32_t g, int32_t slot, int32_t s, const int64_t* cum)
{
    uint64_t u = draw64(seed, (uint32_t)slot, (uint32_t)i, (uint32_t)g, TAG_ROULETTE, 0);
    uint64_t W = (uint64_t)cum[s - 1];
    uint64_t r = (uint64_t)(((unsigned __int128)u * (unsigned __int128)W) >> 64);
    int32_t x = 0;
    while ((uint64_t)cum[x] <= r) x++;
    return x;
}

/* One child from parents A and B, given its crossover mask from_b, its
 * mutation mask and the round-0 candidates of the mutated positions (Eqs. 6
 * and 9 with the duplicate rule):
 *   crossover  - gene j is B[j] where from_b[j], else A[j];
 *   mutation   - gene j becomes a hole where mutated[j], with round-0
 *                candidate mutval[j];
 *   duplicates - every gene kept from A is kept (A's genes are distinct);
 *                then, in ascending position order, a gene taken from B is
 *                kept unless it equals a gene already kept, in which case its
 *                position becomes a hole whose round-0 candidate is A[j];
 *   repair     - as in repair(), with later candidates from src. */
typedef struct {
    keptset kept;
    int32_t* holes;
    int32_t* cand0;
    uint8_t* from_b;
    uint8_t* mutated;
    int32_t* mutval;
} child_scratch;

static void assemble_child(int32_t n, int32_t k, const int32_t* A, const int32_t* B, const uint8_t* from_b,
                           const uint8_t* mutated, const int32_t* mutval, const repair_source* src,
                           int32_t* row, child_scratch* w)
{
    memset(w->kept.in, 0, (size_t)n);
    for (int32_t j = 0; j < k; j++) row[j] = -1;
    /* genes kept from A first, then genes from B that do not repeat one */
    for (int32_t j = 0; j < k; j++)
        if (!mutated[j] && !from_b[j]) { row[j] = A[j]; w->kept.in[A[j]] = 1; }
    for (int32_t j = 0; j < k; j++)
        if (!mutated[j] && from_b[j] && !w->kept.in[B[j]]) { row[j] = B[j]; w->kept.in[B[j]] = 1; }
    int32_t nh = 0;
    for (int32_t j = 0; j < k; j++) {
        if (row[j] >= 0) continue;
        w->holes[nh] = j;
        w->cand0[nh] = mutated[j] ? mutval[j] : A[j];
        nh++;
    }
    repair(src, n, &w->kept, row, w->holes, nh, w->cand0);
}

/* One child with counter index i in generation g (Eqs. 3-9): the crossover
 * mask is draw(j,i,g,XOVER,0) < pc_thr, the mutation mask
 * draw(j,i,g,MUT,0) < pm_thr, a mutated position's round-0 candidate uniform
 * over [0,n) from draw(j,i,g,MUTVAL,0); repair candidates from Philox. */
static void make_child(uint64_t seed, int32_t n, int32_t k, int32_t i, int32_t g, uint32_t pc_thr, uint32_t pm_thr,
                       const int32_t* A, const int32_t* B, int32_t* row, child_scratch* w)
{
    for (int32_t j = 0; j < k; j++) {
        w->from_b[j] = draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_XOVER, 0) < pc_thr;
        w->mutated[j] = draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_MUT, 0) < pm_thr;
        w->mutval[j] = w->mutated[j] ? uniform_below(draw(seed, (uint32_t)j, (uint32_t)i, (uint32_t)g, TAG_MUTVAL, 0), n)
                                     : -1;
    }
    const repair_source src = { seed, i, g, k, NULL };
    assemble_child(n, k, A, B, w->from_b, w->mutated, w->mutval, &src, row, w);
}

/* TEST ENTRY (hand-worked cases, no random numbers): one child of parents A
 * and B over node ids [0, n) from explicit masks from_b[k], mutated[k] (0/1),
 * round-0 candidates mutval[k] of the mutated positions, and the candidates
 * of repair rounds 1 .. 31 in later[31][k].  Every id must lie in [0, n) and
 * each parent must hold distinct genes; returns ORACLE_EINVAL otherwise. */
int oracle_child_explicit(int32_t n, int32_t k, const int32_t* A, const int32_t* B, const uint8_t* from_b,
                          const uint8_t* mutated, const int32_t* mutval, const int32_t* later, int32_t* row)
{
    if (n < 1 || k < 0 || k >= n) return ORACLE_EINVAL;
    for (int32_t j = 0; j < k; j++) {
        if (A[j] < 0 || A[j] >= n || B[j] < 0 || B[j] >= n) return ORACLE_EINVAL;
        if (mutated[j] && (mutval[j] < 0 || mutval[j] >= n)) return ORACLE_EINVAL;
        for (int32_t r = 0; r + 1 < REPAIR_ROUNDS; r++)
            if (later[(size_t)r * (size_t)k + (size_t)j] < 0 || later[(size_t)r * (size_t)k + (size_t)j] >= n)
                return ORACLE_EINVAL;
        for (int32_t q = 0; q < j; q++)
            if (A[q] == A[j] || B[q] == B[j]) return ORACLE_EINVAL;
    }
    child_scratch w;
    w.kept.n = n;
    w.kept.in = (uint8_t*)malloc((size_t)n);
    w.holes = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    w.cand0 = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    w.from_b = w.mutated = NULL;
    w.mutval = NULL;
    int err = (!w.kept.in || !w.holes || !w.cand0) ? ORACLE_ENOMEM : ORACLE_OK;
    if (err == ORACLE_OK) {
        const repair_source src = { 0, 0, 0, k, later };
        assemble_child(n, k, A, B, from_b, mutated, mutval, &src, row, &w);
    }
    free(w.kept.in); free(w.holes); free(w.cand0);
    return err;
}

/* TEST ENTRY: the map of a 32-bit Philox word x to [0, n). */
int32_t oracle_uniform_below(uint32_t x, int32_t n)
{
    return uniform_below(x, n);
}

/* Parent for slot 0 (A) or 1 (B) of the child with counter index i, chosen
 * from the s members of (pop, fit): tournament, or roulette with the flag. */
static int32_t select_parent(uint64_t seed, uint32_t flags, int32_t i, int32_t g, int32_t slot, int32_t t,
                             int32_t s, const int64_t* fit, const int64_t* cum)
{
    if (flags & ORACLE_FLAG_ROULETTE) return roulette(seed, i, g, slot, s, cum);
    return tournament(seed, i, g, slot, t, s, fit);
}

/* One generation g >= 1 (Fig. 1's loop body), producing (pop_out, fit_out)
 * from (pop_in, fit_in) of s members.
 * Default (one elite):
 *   elitism  - row 0 = the member with the lowest fitness (lowest index on
 *              ties), fitness carried over;
 *   children - rows i = 1 .. s-1 from parents A and B chosen by select_parent
 *              (with the row-wise flag A = member i itself, Eq. 6 read
 *              literally), built by make_child with counter index i;
 *   fitness  - PC of every child (BFS).
 * With ORACLE_FLAG_MU_PLUS_LAMBDA (Eqs. 10-11): lambda children c = 0 ..
 * lambda-1 (counter index c) from parents among the s members, their
 * fitness, then the s members of lowest fitness among [members; children]
 * by a stable ascending sort (members before children, lower index first on
 * ties) form the next population. */
static int cmp_key(const void* a, const void* b)
{
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return x[1] < y[1] ? -1 : (x[1] > y[1]);
}

int oracle_generation(int32_t n, const int32_t* row_ptr, const int32_t* col,
                      int32_t k, int32_t s, int32_t t, uint32_t pc_thr, uint32_t pm_thr,
                      uint64_t seed, uint32_t flags, int32_t g, int32_t lambda,
                      const int32_t* pop_in, const int64_t* fit_in,
                      int32_t* pop_out, int64_t* fit_out, int32_t nthreads)
{
    const int mpl = (flags & ORACLE_FLAG_MU_PLUS_LAMBDA) != 0;
    const int32_t u = n >= 1 ? gene_universe(n, row_ptr, flags) : 0;  /* genes are drawn from [0, u) */
    if (n < 1 || k < 0 || k >= u || s < 2 || t < 1 || g < 1 || (mpl && lambda < 1)) return ORACLE_EINVAL;
    if (mpl && (flags & ORACLE_FLAG_ROWWISE)) return ORACLE_EINVAL;
    const int32_t nchild = mpl ? lambda : s - 1;
    int err = ORACLE_OK;
    child_scratch w;
    w.kept.n = u;
    w.kept.in = (uint8_t*)malloc((size_t)u);
    w.holes = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    w.cand0 = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    w.from_b = (uint8_t*)malloc((size_t)k + 1);
    w.mutated = (uint8_t*)malloc((size_t)k + 1);
    w.mutval = (int32_t*)malloc(sizeof(int32_t) * ((size_t)k + 1));
    int64_t* cum = (int64_t*)malloc(sizeof(int64_t) * (size_t)s);
    int32_t* kids = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nchild * (size_t)k + 1));
    int64_t* kfit = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nchild + 1));
    if (!w.kept.in || !w.holes || !w.cand0 || !w.from_b || !w.mutated || !w.mutval || !cum || !kids || !kfit)
        err = ORACLE_ENOMEM;
    if (err == ORACLE_OK) {
        roulette_weights(fit_in, s, cum);
        for (int32_t c = 0; c < nchild; c++) {
            const int32_t i = mpl ? c : c + 1;
            int32_t pa = (flags & ORACLE_FLAG_ROWWISE) ? i : select_parent(seed, flags, i, g, 0, t, s, fit_in, cum);
            int32_t pb = select_parent(seed, flags, i, g, 1, t, s, fit_in, cum);
            make_child(seed, u, k, i, g, pc_thr, pm_thr, pop_in + (size_t)pa * (size_t)k,
                       pop_in + (size_t)pb * (size_t)k, kids + (size_t)c * (size_t)k, &w);
        }
        err = oracle_fitness(n, row_ptr, col, kids, nchild, k, kfit, fitness_method(flags), nthreads);
    }
    if (err == ORACLE_OK && !mpl) {
        int32_t elite = 0;
        for (int32_t x = 1; x < s; x++)
            if (fit_in[x] < fit_in[elite]) elite = x;
        memcpy(pop_out, pop_in + (size_t)elite * (size_t)k, sizeof(int32_t) * (size_t)k);
        fit_out[0] = fit_in[elite];
        memcpy(pop_out + k, kids, sizeof(int32_t) * (size_t)(s - 1) * (size_t)k);
        memcpy(fit_out + 1, kfit, sizeof(int64_t) * (size_t)(s - 1));
    } else if (err == ORACLE_OK) {
        int32_t tot = s + nchild;
        int64_t* key = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)tot);
        if (!key) err = ORACLE_ENOMEM;
        else {
            for (int32_t x = 0; x < tot; x++) {
                key[2 * x] = x < s ? fit_in[x] : kfit[x - s];
                key[2 * x + 1] = x;
            }
            qsort(key, (size_t)tot, 2 * sizeof(int64_t), cmp_key);
            for (int32_t r = 0; r < s; r++) {
                int32_t x = (int32_t)key[2 * r + 1];
                const int32_t* src = x < s ? pop_in + (size_t)x * (size_t)k : kids + (size_t)(x - s) * (size_t)k;
                memcpy(pop_out + (size_t)r * (size_t)k, src, sizeof(int32_t) * (size_t)k);
                fit_out[r] = key[2 * r];
            }
            free(key);
        }
    }
    free(w.kept.in); free(w.holes); free(w.cand0); free(w.from_b); free(w.mutated); free(w.mutval);
    free(cum); free(kids); free(kfit);
    return err;
}

/* A whole run: initialisation, fitness, then `gens` generations.
 * traj_best (gens+1 entries, may be NULL) receives the lowest fitness after
 * initialisation and after every generation; best_set (k entries) the genes
 * of the final best member (lowest fitness, lowest index) in ascending order;
 * pop_final / fit_final (may be NULL) the final population. */
static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int oracle_run(int32_t n, const int32_t* row_ptr, const int32_t* col,
               int32_t k, int32_t s, int32_t gens, int32_t t, uint32_t pc_thr, uint32_t pm_thr,
               uint64_t seed, uint32_t flags, int32_t lambda, int32_t* best_set, int64_t* best_fit,
               int64_t* traj_best, int32_t* pop_final, int64_t* fit_final, int32_t nthreads)
{
    const int32_t u = n >= 1 ? gene_universe(n, row_ptr, flags) : 0;  /* genes are drawn from [0, u) */
    if (n < 1 || k < 0 || k >= u || s < 2 || t < 1 || gens < 0) return ORACLE_EINVAL;
    size_t cells = (size_t)s * (size_t)k;
    int32_t* pa = (int32_t*)malloc(sizeof(int32_t) * (cells + 1));
    int32_t* pb = (int32_t*)malloc(sizeof(int32_t) * (cells + 1));
    int64_t* fa = (int64_t*)malloc(sizeof(int64_t) * (size_t)s);
    int64_t* fb = (int64_t*)malloc(sizeof(int64_t) * (size_t)s);
    int err = (!pa || !pb || !fa || !fb) ? ORACLE_ENOMEM : ORACLE_OK;
    if (err == ORACLE_OK) err = oracle_pop_init(u, k, s, seed, pa);
    if (err == ORACLE_OK) err = oracle_fitness(n, row_ptr, col, pa, s, k, fa, fitness_method(flags), nthreads);
    for (int32_t g = 0; g <= gens && err == ORACLE_OK; g++) {
        if (g > 0) {
            err = oracle_generation(n, row_ptr, col, k, s, t, pc_thr, pm_thr, seed, flags, g, lambda,
                                    pa, fa, pb, fb, nthreads);
            int32_t* tp = pa; pa = pb; pb = tp;
            int64_t* tf = fa; fa = fb; fb = tf;
        }
        if (traj_best && err == ORACLE_OK) {
            int64_t m = fa[0];
            for (int32_t x = 1; x < s; x++) if (fa[x] < m) m = fa[x];
            traj_best[g] = m;
        }
    }
    if (err == ORACLE_OK) {
        int32_t e = 0;
        for (int32_t x = 1; x < s; x++) if (fa[x] < fa[e]) e = x;
        if (best_fit) *best_fit = fa[e];
        if (best_set) {
            memcpy(best_set, pa + (size_t)e * (size_t)k, sizeof(int32_t) * (size_t)k);
            qsort(best_set, (size_t)k, sizeof(int32_t), cmp_i32);
        }
        if (pop_final) memcpy(pop_final, pa, sizeof(int32_t) * cells);
        if (fit_final) memcpy(fit_final, fa, sizeof(int64_t) * (size_t)s);
    }
    free(pa); free(pb); free(fa); free(fb);
    return err;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
