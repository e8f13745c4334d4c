// C ABI of libgapa.so: contexts, graph upload and validation, and the
// drivers of fitness, generation and whole runs.  Every compute step runs in
// the kernels of fitness.cu and ga.cu; this file moves data and orders work.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "gapa_internal.cuh"
#include "tree16.cuh"

int gapa_fitness_kernels_init(gapa_ctx* c);
int gapa_ga_kernels_init(gapa_ctx* c);

namespace {
thread_local std::string g_last_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void free_graph(DeviceGraph& g) {
    cudaFree(g.row_ptr);
    cudaFree(g.col);
    cudaFree(g.edges);
    cudaFree(g.probe);
    cudaFree(g.perm);
    cudaFree(g.tparent);
    cudaFree(g.kids);
    cudaFree(g.roots);
    cudaFree(g.cut);
    cudaFree(g.order);
    cudaFree(g.sz);
    cudaFree(g.pre);
    cudaFree(g.at);
    cudaFree(g.crep);
    cudaFree(g.nroot);
    cudaFree(g.csize);
    DeviceForest& a = g.alt;
    void* alt_ptrs[] = {a.perm, a.tparent, a.palt, a.lo_ptr, a.lo_col, a.kids, a.roots, a.cut, a.fptr, a.fcol16,
                        a.nontree, a.sz, a.pre, a.at, a.crep, a.nroot, a.csize};
    for (void* q : alt_ptrs) cudaFree(q);
    cudaFree(g.nontree);
    cudaFree(g.fptr);
    cudaFree(g.fcol16);
    cudaFree(g.fcol32);
    cudaFree(g.lo_ptr);
    cudaFree(g.lo_col);
    cudaFree(g.palt);
    for (SparseForest& f : g.spf) {
        void* tabs[] = {f.kids, f.croot, f.csize, f.sub, f.bysize, f.cost};
        for (void* q : tabs) cudaFree(q);
        if (f.owns) {
            void* own[] = {f.perm, f.tparent, f.palt, f.lo_ptr, f.lo_col, f.fptr, f.fcol32, f.fcol16};
            for (void* q : own) cudaFree(q);
        }
    }
    g = DeviceGraph();
}

// Forest numbering for the TREE fitness kernel.  Nodes are numbered in BFS
// order from the highest-degree node of each component (ties: lower id) - or,
// without bfs_order, by descending degree, which measured slower (more
// pieces to join on random deletion sets, no gain on hub-heavy ones).  Every node's parent is its
// lowest-numbered neighbour when that one is lower than the node itself (a
// root otherwise), so parents always precede children; for BFS order this is
// the BFS tree.  Outputs the original -> new map, the parents, each node's
// lower-numbered neighbours (ascending; the first one is the parent), the
// non-parent edges (a < b, sorted) and the deepest parent chain.
struct BfsForest {
    std::vector<int32_t> perm, tparent, lo_ptr, lo_col, roots;
    std::vector<std::pair<int32_t, int32_t>> nontree;
    int depth = 0;
};

BfsForest bfs_forest(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                     bool bfs_order = true) {
    BfsForest f;
    f.perm.assign((size_t)n, -1);
    std::vector<int32_t> by_deg((size_t)n);
    for (int32_t v = 0; v < n; ++v) by_deg[v] = v;
    std::stable_sort(by_deg.begin(), by_deg.end(),
                     [&](int32_t a, int32_t b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
    if (bfs_order) {
        std::vector<int32_t> queue;
        queue.reserve((size_t)n);
        int32_t next = 0;
        for (int32_t root : by_deg) {
            if (f.perm[root] >= 0) continue;
            size_t head = queue.size();
            queue.push_back(root);
            f.roots.push_back(next);
            f.perm[root] = next++;
            while (head < queue.size()) {
                const int32_t u = queue[head++];
                for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
                    if (f.perm[col[e]] < 0) {
                        f.perm[col[e]] = next++;
                        queue.push_back(col[e]);
                    }
            }
        }
    } else {
        for (int32_t r = 0; r < n; ++r) f.perm[by_deg[r]] = r;
    }
    // (roots of the degree order are filled in with the parents below)
    std::vector<int32_t> inv((size_t)n);
    for (int32_t v = 0; v < n; ++v) inv[f.perm[v]] = v;
    // lower-numbered neighbours, ascending; parent = the first of them
    f.lo_ptr.assign((size_t)n + 1, 0);
    f.lo_col.reserve(col.size() / 2);
    f.tparent.assign((size_t)n, 0);
    std::vector<int32_t> tmp, level((size_t)n, 0);
    for (int32_t b = 0; b < n; ++b) {
        const int32_t v = inv[b];
        tmp.clear();
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t a = f.perm[col[e]];
            if (a < b) tmp.push_back(a);
        }
        std::sort(tmp.begin(), tmp.end());
        f.tparent[b] = tmp.empty() ? b : tmp[0];
        if (!bfs_order && tmp.empty()) f.roots.push_back(b);
        level[b] = tmp.empty() ? 0 : level[tmp[0]] + 1;
        f.depth = std::max(f.depth, level[b]);
        f.lo_col.insert(f.lo_col.end(), tmp.begin(), tmp.end());
        f.lo_ptr[b + 1] = (int32_t)f.lo_col.size();
    }
    f.nontree.reserve(col.size() / 2);
    for (int32_t b = 0; b < n; ++b)
        for (int32_t e = f.lo_ptr[b] + 1; e < f.lo_ptr[b + 1]; ++e) f.nontree.emplace_back(f.lo_col[e], b);
    std::sort(f.nontree.begin(), f.nontree.end());
    return f;
}

// Subtree sizes, preorder positions and the node at each position of a forest
// whose parents precede their children (roots: parent = itself), children
// visited in ascending order and trees by ascending root, so that a subtree
// is the interval [pre, pre + sz).  A forest may hold several trees of one
// component of G (a root need not be a component's only root: a node with no
// lower-numbered neighbour starts a tree even when later nodes join it to
// others), so the components come from the lower-neighbour lists: crep = the
// smallest root of each node's component, nroot = the next root of the same
// component (ascending; -1 after the last), csize = the component's size at
// its representative, and tree_pc = the sum over the components of
// C(size, 2).
struct ForestIntervals {
    std::vector<int32_t> sz, pre, crep, nroot, csize;
    std::vector<uint16_t> at;
    long long tree_pc = 0;
};

ForestIntervals forest_intervals(const std::vector<int32_t>& tparent, const std::vector<int32_t>& lo_ptr,
                                 const std::vector<int32_t>& lo_col) {
    const int32_t n = (int32_t)tparent.size();
    ForestIntervals fi;
    fi.sz.assign((size_t)n, 1);
    fi.pre.assign((size_t)n, 0);
    fi.crep.assign((size_t)n, 0);
    fi.nroot.assign((size_t)n, -1);
    fi.csize.assign((size_t)n, 0);
    fi.at.assign((size_t)n, 0);
    for (int32_t v = n - 1; v >= 0; --v)
        if (tparent[v] != v) fi.sz[tparent[v]] += fi.sz[v];
    std::vector<int32_t> next((size_t)n, 0), root((size_t)n, 0);  // next free position below each node
    int32_t cursor = 0;
    for (int32_t v = 0; v < n; ++v) {
        const int32_t p = tparent[v];
        if (p == v) {
            fi.pre[v] = cursor;
            cursor += fi.sz[v];
            root[v] = v;
        } else {
            fi.pre[v] = next[p];
            next[p] += fi.sz[v];
            root[v] = root[p];
        }
        next[v] = fi.pre[v] + 1;
        fi.at[fi.pre[v]] = (uint16_t)v;
    }
    // components: union of the trees joined by an edge (every edge is in one lower-neighbour list)
    std::vector<int32_t> uf((size_t)n);
    for (int32_t v = 0; v < n; ++v) uf[v] = v;
    auto find = [&](int32_t x) {
        while (uf[x] != x) {
            uf[x] = uf[uf[x]];
            x = uf[x];
        }
        return x;
    };
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = lo_ptr[v]; e < lo_ptr[v + 1]; ++e) {
            int32_t a = find(root[v]), b = find(root[lo_col[e]]);
            if (a != b) uf[std::max(a, b)] = std::min(a, b);  // the smallest root represents
        }
    std::vector<int32_t> last((size_t)n, -1);
    for (int32_t v = 0; v < n; ++v) {
        const int32_t c = find(root[v]);
        fi.crep[v] = c;
        fi.csize[c] += 1;
        if (tparent[v] == v) {  // roots in ascending order: link v after the component's last root
            if (last[c] >= 0) fi.nroot[last[c]] = v;
            last[c] = v;
        }
    }
    for (int32_t v = 0; v < n; ++v)
        if (fi.crep[v] == v) fi.tree_pc += (long long)fi.csize[v] * (fi.csize[v] - 1) / 2;
    return fi;
}

// The forest of a numbering `perm` (host side, n <= 65536): every node's
// parent is its lowest-numbered neighbour when that one is lower (a root
// otherwise), so parents precede children.  `ok` is false when some node's
// children do not fall into at most two runs of consecutive numbers.
struct ForestHost {
    std::vector<int32_t> perm, tparent, lo_ptr, lo_col, roots, cut, fptr, fcol;
    std::vector<int4> kids;
    std::vector<int2> palt;
    std::vector<uint32_t> nontree;
    ForestIntervals iv;
    bool ok = true;
};

ForestHost forest_host(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                       const std::vector<int32_t>& perm) {
    ForestHost f;
    f.perm = perm;
    std::vector<int32_t> inv((size_t)n);
    for (int32_t v = 0; v < n; ++v) inv[perm[v]] = v;
    f.tparent.assign((size_t)n, 0);
    f.lo_ptr.assign((size_t)n + 1, 0);
    f.palt.assign((size_t)n, make_int2(0, -1));
    f.fptr.assign((size_t)n + 1, 0);
    f.fcol.reserve(col.size());
    std::vector<int32_t> tmp;
    for (int32_t b = 0; b < n; ++b) {
        const int32_t v = inv[b];
        tmp.clear();
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t a = perm[col[e]];
            f.fcol.push_back(a);
            if (a < b) tmp.push_back(a);
        }
        f.fptr[b + 1] = (int32_t)f.fcol.size();
        std::sort(tmp.begin(), tmp.end());
        f.tparent[b] = tmp.empty() ? b : tmp[0];
        if (tmp.empty()) f.roots.push_back(b);
        f.palt[b] = make_int2(f.tparent[b], tmp.size() >= 2 ? tmp[1] : -1);
        for (size_t i = 1; i < tmp.size(); ++i) f.nontree.push_back(((uint32_t)tmp[i] << 16) | (uint32_t)b);
        f.lo_col.insert(f.lo_col.end(), tmp.begin(), tmp.end());
        f.lo_ptr[b + 1] = (int32_t)f.lo_col.size();
    }
    std::sort(f.nontree.begin(), f.nontree.end());
    // children runs (children arrive in ascending order)
    f.kids.assign((size_t)n, make_int4(0, 0, 0, 0));
    for (int32_t b = 0; b < n; ++b) f.kids[b].x = b;
    for (int32_t x = 0; x < n && f.ok; ++x) {
        const int32_t p = f.tparent[x];
        if (p == x) continue;
        int4& k = f.kids[p];
        if (k.y == 0) {
            k.x = x;
            k.y = 1;
        } else if (k.w == 0 && k.x + k.y == x) {
            k.y += 1;
        } else if (k.w == 0) {
            k.z = x;  // start of the second run (stored below as start - first run's length)
            k.w = 1;
        } else if (k.z + k.w == x) {
            k.w += 1;
        } else {
            f.ok = false;
        }
    }
    for (int32_t b = 0; b < n; ++b)
        if (f.kids[b].w) f.kids[b].z -= f.kids[b].y;
    // cost table: the nodes below those children of b whose only lower neighbour is b
    std::vector<int32_t> below((size_t)n, 1);
    f.cut.assign((size_t)n, 0);
    for (int32_t v = n - 1; v >= 0; --v)
        if (f.tparent[v] != v) below[f.tparent[v]] += below[v];
    for (int32_t v = 0; v < n; ++v)
        if (f.tparent[v] != v && f.lo_ptr[v + 1] - f.lo_ptr[v] == 1) f.cut[f.tparent[v]] += below[v];
    // indexed by original node id, so that a gene's estimate is one load
    std::vector<int32_t> by_id((size_t)n);
    for (int32_t v = 0; v < n; ++v) by_id[v] = f.cut[perm[v]];
    f.cut.swap(by_id);
    f.iv = forest_intervals(f.tparent, f.lo_ptr, f.lo_col);
    return f;
}

// Numbering with the top `hubs` nodes by degree last: BFS over the graph
// without them (from the highest-degree remaining node of each component),
// then the hubs by their lowest-numbered non-hub neighbour (hubs without one
// at the end), so that deleting a hub cuts no tree edge below it.
std::vector<int32_t> hub_last_perm(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                                   int hubs) {
    std::vector<int32_t> by_deg((size_t)n), perm((size_t)n, -1);
    for (int32_t v = 0; v < n; ++v) by_deg[v] = v;
    std::stable_sort(by_deg.begin(), by_deg.end(),
                     [&](int32_t a, int32_t b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
    std::vector<char> hub((size_t)n, 0);
    for (int i = 0; i < hubs && i < n; ++i) hub[by_deg[i]] = 1;
    std::vector<int32_t> queue;
    queue.reserve((size_t)n);
    int32_t next = 0;
    for (int32_t root : by_deg) {
        if (perm[root] >= 0 || hub[root]) continue;
        size_t head = queue.size();
        queue.push_back(root);
        perm[root] = next++;
        while (head < queue.size()) {
            const int32_t u = queue[head++];
            for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
                if (!hub[col[e]] && perm[col[e]] < 0) {
                    perm[col[e]] = next++;
                    queue.push_back(col[e]);
                }
        }
    }
    std::vector<std::pair<int64_t, int32_t>> hk;
    for (int i = 0; i < hubs && i < n; ++i) {
        const int32_t h = by_deg[i];
        int32_t low = INT32_MAX;
        for (int32_t e = rp[h]; e < rp[h + 1]; ++e)
            if (!hub[col[e]]) low = std::min(low, perm[col[e]]);
        hk.emplace_back(((int64_t)low << 20) | i, h);
    }
    std::sort(hk.begin(), hk.end());
    for (auto& x : hk) perm[x.second] = next++;
    return perm;
}

// Device copy of a forest (nullptr members on failure, which the caller frees).
int upload_forest(const ForestHost& f, int32_t n, DeviceForest& d) {
    const size_t par_ints = gapa_dev::tree16l_lab_ints(n);
    std::vector<int32_t> par(f.tparent);
    par.resize(par_ints, 0);
    std::vector<uint16_t> f16(f.fcol.begin(), f.fcol.end());
    auto up = [](void** dst, const void* src, size_t bytes) {
        if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        return bytes == 0 || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up((void**)&d.perm, f.perm.data(), 4 * (size_t)n) && up((void**)&d.tparent, par.data(), 4 * par_ints) &&
              up((void**)&d.palt, f.palt.data(), sizeof(int2) * (size_t)n) &&
              up((void**)&d.lo_ptr, f.lo_ptr.data(), 4 * ((size_t)n + 1)) &&
              up((void**)&d.lo_col, f.lo_col.data(), 4 * f.lo_col.size()) &&
              up((void**)&d.kids, f.kids.data(), sizeof(int4) * (size_t)n) &&
              up((void**)&d.roots, f.roots.data(), 4 * f.roots.size()) &&
              up((void**)&d.cut, f.cut.data(), 4 * (size_t)n) &&
              up((void**)&d.fptr, f.fptr.data(), 4 * ((size_t)n + 1)) &&
              up((void**)&d.fcol16, f16.data(), 2 * f16.size()) &&
              up((void**)&d.nontree, f.nontree.data(), 4 * f.nontree.size()) &&
              up((void**)&d.sz, f.iv.sz.data(), 4 * (size_t)n) && up((void**)&d.pre, f.iv.pre.data(), 4 * (size_t)n) &&
              up((void**)&d.at, f.iv.at.data(), 2 * (size_t)n) &&
              up((void**)&d.crep, f.iv.crep.data(), 4 * (size_t)n) &&
              up((void**)&d.nroot, f.iv.nroot.data(), 4 * (size_t)n) &&
              up((void**)&d.csize, f.iv.csize.data(), 4 * (size_t)n);
    d.num_roots = (int)f.roots.size();
    d.num_nontree = (int)f.nontree.size();
    if (!ok) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "second forest of %d nodes", n);
    }
    return GAPA_OK;
}

// Host-side validation of a symmetric simple CSR; returns the rows sorted.
int validate_csr(int32_t n, int64_t nnz, const int32_t* rp, const int32_t* col_in, std::vector<int32_t>& col) {
    if (rp[0] != 0) return gapa_fail(GAPA_ERR_INVALID_GRAPH, "row_ptr[0] = %d, expected 0", rp[0]);
    for (int32_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return gapa_fail(GAPA_ERR_INVALID_GRAPH, "row_ptr decreases at row %d", v);
    if ((int64_t)rp[n] != nnz)
        return gapa_fail(GAPA_ERR_INVALID_GRAPH, "row_ptr[n] = %d but nnz = %lld", rp[n], (long long)nnz);
    col.assign(col_in, col_in + nnz);
    const unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<int> bad(nth, 0);
    std::vector<int32_t> bad_row(nth, -1);
    auto work = [&](unsigned t, int pass) {
        const int32_t lo = (int32_t)((int64_t)n * t / nth), hi = (int32_t)((int64_t)n * (t + 1) / nth);
        for (int32_t u = lo; u < hi && !bad[t]; ++u) {
            int32_t* b = col.data() + rp[u];
            int32_t* e = col.data() + rp[u + 1];
            if (pass == 0) {
                for (int32_t* p = b; p < e; ++p) {
                    if (*p < 0 || *p >= n) { bad[t] = 1; bad_row[t] = u; break; }
                    if (*p == u) { bad[t] = 2; bad_row[t] = u; break; }
                }
                if (bad[t]) break;
                std::sort(b, e);
                for (int32_t* p = b + 1; p < e; ++p)
                    if (*p == *(p - 1)) { bad[t] = 3; bad_row[t] = u; break; }
            } else {
                for (int32_t* p = b; p < e; ++p) {
                    const int32_t v = *p;
                    const int32_t* vb = col.data() + rp[v];
                    const int32_t* ve = col.data() + rp[v + 1];
                    if (!std::binary_search(vb, ve, u)) { bad[t] = 4; bad_row[t] = u; break; }
                }
            }
        }
    };
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nth; ++t) th.emplace_back(work, t, pass);
        for (auto& x : th) x.join();
        for (unsigned t = 0; t < nth; ++t) {
            static const char* what[] = {"", "column id out of range", "self-loop", "repeated arc",
                                         "arc without its reverse"};
            if (bad[t]) return gapa_fail(GAPA_ERR_INVALID_GRAPH, "%s in row %d", what[bad[t]], bad_row[t]);
        }
    }
    return GAPA_OK;
}

int check_cfg(gapa_ctx* c, const gapa_config* cfg) {
    if (!cfg) return gapa_fail(GAPA_ERR_INVALID_ARG, "config is NULL");
    if (c->g.n <= 0) return gapa_fail(GAPA_ERR_STATE, "no graph uploaded");
    const int universe = gapa_gene_universe(c);
    if (cfg->k < 0 || cfg->k >= universe)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "need 0 <= k < %s (k=%d, %d)", c->genes ? "E" : "n", cfg->k, universe);
    if (cfg->pop < 2) return gapa_fail(GAPA_ERR_INVALID_ARG, "population must be >= 2 (got %d)", cfg->pop);
    if (cfg->tourn < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "tournament size must be >= 1");
    if (cfg->elite != 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "elite count must be 1 (got %d)", cfg->elite);
    if (cfg->gens < 0) return gapa_fail(GAPA_ERR_INVALID_ARG, "gens must be >= 0");
    if (cfg->flags & ~(GAPA_FLAG_ROWWISE | GAPA_FLAG_MU_PLUS_LAMBDA | GAPA_FLAG_ROULETTE))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "unknown flag bits 0x%x", cfg->flags);
    if (cfg->flags & GAPA_FLAG_MU_PLUS_LAMBDA) {
        if (cfg->lambda < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "(mu+lambda) needs lambda >= 1");
        if (cfg->flags & GAPA_FLAG_ROWWISE)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "the row-wise flag has no meaning with (mu+lambda)");
        if ((long long)cfg->pop + cfg->lambda > 16384)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "mu + lambda must be at most 16384");
        if ((long long)cfg->lambda * cfg->k >= (1LL << 31)) return gapa_fail(GAPA_ERR_INVALID_ARG, "lambda*k too large");
    }
    return gapa_ga_check_limits(c, universe, cfg->k, cfg->pop);
}

GaParams make_params(gapa_ctx* c, const gapa_config* cfg, int g, const int* g_ptr) {
    GaParams p;
    p.n = gapa_gene_universe(c);  // genes are drawn from [0, p.n)
    p.k = cfg->k;
    p.s = cfg->pop;
    p.t = cfg->tourn;
    p.pc_thr = cfg->pc_thr;
    p.pm_thr = cfg->pm_thr;
    p.key = RngKey{(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
    p.flags = cfg->flags;
    p.g = g;
    p.g_ptr = g_ptr;
    p.cum = nullptr;
    p.est_cut = nullptr;
    p.est_cut2 = nullptr;
    p.est_out = nullptr;
    p.est_stride = 0;
    return p;
}

// Scratch of the (mu+lambda) and roulette variants, reserved outside any capture.
int ensure_variant_scratch(gapa_ctx* c, const gapa_config* cfg) {
    int rc = GAPA_OK;
    if (cfg->flags & GAPA_FLAG_ROULETTE) rc = gapa_reserve((void**)&c->cum, &c->cum_cap, (size_t)cfg->pop, 8);
    if (rc == GAPA_OK && (cfg->flags & GAPA_FLAG_MU_PLUS_LAMBDA)) {
        rc = gapa_reserve((void**)&c->kids, &c->kids_cap, (size_t)cfg->lambda * cfg->k, 4);
        if (rc == GAPA_OK) rc = gapa_reserve((void**)&c->kfit, &c->kfit_cap, (size_t)cfg->lambda, 8);
        if (rc == GAPA_OK) rc = gapa_reserve((void**)&c->src, &c->src_cap, (size_t)cfg->pop, 4);
    }
    if (rc == GAPA_OK)
        rc = gapa_fitness_prepare(c, (cfg->flags & GAPA_FLAG_MU_PLUS_LAMBDA) ? std::max(cfg->pop, cfg->lambda)
                                                                             : cfg->pop);
    return rc;
}

// One generation on stream st.  Default: offspring rows (elite + children),
// then fitness of rows 1..s-1.  (mu+lambda): lambda children, their fitness,
// then the truncation of members + children.  Roulette weights first if used.
int enqueue_generation(gapa_ctx* c, const GaParams& p0, int lambda, const int32_t* pop_in, const int64_t* fit_in,
                       int32_t* pop_out, int64_t* fit_out, cudaStream_t st) {
    GaParams p = p0;
    int rc = GAPA_OK;
    if (p.flags & GAPA_FLAG_ROULETTE) {
        rc = gapa_launch_roulette_prefix(fit_in, p.s, c->cum, st);
        p.cum = reinterpret_cast<const long long*>(c->cum);
        if (rc != GAPA_OK) return rc;
    }
    // the operator kernels also write the children's cost estimates for the cut-local fitness kernel
    const int evaluated = (p.flags & GAPA_FLAG_MU_PLUS_LAMBDA) ? lambda : p.s;
    unsigned* est = gapa_fitness_uses_estimates(c, evaluated) ? gapa_estimate_buffer(c) : nullptr;
    if (est) {
        p.est_cut = c->g.cut;
        if (c->g.has_alt) p.est_cut2 = c->g.alt.cut;
        p.est_out = est;
        p.est_stride = kOrderCap;
    }
    if (p.flags & GAPA_FLAG_MU_PLUS_LAMBDA) {
        rc = gapa_launch_children(c, p, lambda, pop_in, fit_in, c->kids, st);
        if (rc == GAPA_OK) rc = gapa_launch_fitness(c, c->kids, lambda, p.k, c->kfit, st, est);
        if (rc == GAPA_OK)
            rc = gapa_launch_mpl_replace(c, p.s, lambda, p.k, pop_in, fit_in, c->kids, c->kfit, c->src, pop_out,
                                         fit_out, st);
        return rc;
    }
    rc = gapa_launch_offspring(c, p, pop_in, fit_in, pop_out, fit_out, st);
    if (rc != GAPA_OK) return rc;
    return gapa_launch_fitness(c, pop_out + p.k, p.s - 1, p.k, fit_out + 1, st, est ? est + 1 : nullptr);
}

int read_status(gapa_ctx* c, cudaStream_t st) {
    int h = 0;
    GAPA_CUDA(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    GAPA_CUDA(cudaStreamSynchronize(st));
    if (h == 0) return GAPA_OK;
    GAPA_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), st));
    GAPA_CUDA(cudaStreamSynchronize(st));
    if (h & GAPA_DEV_TIMEOUT) return gapa_fail(GAPA_ERR_TIMEOUT, "a device-side wait ran out (status 0x%x)", h);
    if (h & GAPA_DEV_BAD_GENE) return gapa_fail(GAPA_ERR_DEVICE, "a gene outside [0, n) was passed (status 0x%x)", h);
    return gapa_fail(GAPA_ERR_DEVICE, "device status 0x%x", h);
}

int ensure_stage(gapa_ctx* c, size_t pop_elems, size_t fit_elems) {
    if (pop_elems > c->stage_pop_cap) {
        for (auto& p : c->stage_pop) { cudaFree(p); p = nullptr; }
        c->stage_pop_cap = 0;
        for (auto& p : c->stage_pop)
            if (cudaMalloc(&p, std::max<size_t>(pop_elems, 1) * sizeof(int32_t)) != cudaSuccess)
                return gapa_fail(GAPA_ERR_OOM, "staging population of %zu genes", pop_elems);
        c->stage_pop_cap = pop_elems;
    }
    if (fit_elems > c->stage_fit_cap) {
        for (auto& p : c->stage_fit) { cudaFree(p); p = nullptr; }
        c->stage_fit_cap = 0;
        for (auto& p : c->stage_fit)
            if (cudaMalloc(&p, std::max<size_t>(fit_elems, 1) * sizeof(int64_t)) != cudaSuccess)
                return gapa_fail(GAPA_ERR_OOM, "staging fitness of %zu members", fit_elems);
        c->stage_fit_cap = fit_elems;
    }
    return GAPA_OK;
}

}  // namespace

GaParams gapa_make_params(gapa_ctx* c, const gapa_config* cfg, int g, const int* g_ptr) {
    return make_params(c, cfg, g, g_ptr);
}

// Validation and buffers of a whole run (outside any capture).
int gapa_run_prepare(gapa_ctx* c, const gapa_config* cfg) {
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    const size_t cells = (size_t)cfg->pop * cfg->k;
    rc = ensure_stage(c, cells, (size_t)cfg->pop);
    if (rc == GAPA_OK) rc = gapa_reserve((void**)&c->run_traj, &c->run_traj_cap, (size_t)cfg->gens + 1, sizeof(int64_t));
    if (rc == GAPA_OK) rc = ensure_variant_scratch(c, cfg);
    return rc;
}

int gapa_fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int gapa_cuda_fail(cudaError_t e, const char* what) {
    const int code = e == cudaErrorMemoryAllocation ? GAPA_ERR_OOM : GAPA_ERR_CUDA;
    return gapa_fail(code, "%s: %s", what, cudaGetErrorString(e));
}

int gapa_set_smem_limit(const void* kernel, size_t optin, size_t* max_dyn) {
    cudaFuncAttributes a;
    GAPA_CUDA(cudaFuncGetAttributes(&a, kernel));
    const size_t dyn = optin > a.sharedSizeBytes ? optin - a.sharedSizeBytes : 0;
    GAPA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    if (*max_dyn == 0 || dyn < *max_dyn) *max_dyn = dyn;
    return GAPA_OK;
}

int gapa_reserve(void** ptr, size_t* cap, size_t count, size_t elem) {
    if (count <= *cap) return GAPA_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (cudaMalloc(ptr, std::max<size_t>(count, 1) * elem) != cudaSuccess) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "device scratch of %zu bytes", count * elem);
    }
    *cap = count;
    return GAPA_OK;
}

ProfileScope::ProfileScope(gapa_ctx* c_, cudaStream_t st_, int kind_, int evals_)
    : c(c_), st(st_), kind(kind_), evals(evals_) {
    if (!c->profiling || c->capturing) return;
    for (cudaEvent_t* e : {&a, &b}) {
        if (!c->event_pool.empty()) {
            *e = c->event_pool.back();
            c->event_pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            *e = nullptr;
        }
    }
    if (a && b) cudaEventRecord(a, st);
}

ProfileScope::~ProfileScope() {
    if (!a || !b) {
        if (a) c->event_pool.push_back(a);
        if (b) c->event_pool.push_back(b);
        return;
    }
    cudaEventRecord(b, st);
    c->timed.push_back(gapa_ctx::Timed{a, b, kind, evals, kernels});
}

extern "C" {

const char* gapa_last_error(void) { return g_last_error.c_str(); }

const char* gapa_version(void) { return "gapa-gb300 0.1 (sm_103a)"; }

int gapa_create(gapa_ctx** out, int device, void* cuda_stream) {
    if (!out) return gapa_fail(GAPA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    GAPA_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return gapa_fail(GAPA_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DeviceGuard guard(device);
    gapa_ctx* c = new gapa_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    int v = 0;
    auto bail = [&](int rc) {
        gapa_destroy(c);
        return rc;
    };
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "device attribute query failed"));
    c->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "device attribute query failed"));
    c->smem_optin = (size_t)v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "device attribute query failed"));
    c->smem_per_sm = (size_t)v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "device attribute query failed"));
    c->smem_reserved = (size_t)v;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "stream/event creation failed"));
    if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_OOM, "status word"));
    if (cudaMalloc(&c->run_gen, sizeof(int)) != cudaSuccess || cudaMalloc(&c->run_best, sizeof(int)) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_OOM, "run counters"));
    int rc = gapa_fitness_kernels_init(c);
    if (rc == GAPA_OK) rc = gapa_sixdst_init(c);
    if (rc == GAPA_OK) rc = gapa_sparse_init(c);
    if (rc == GAPA_OK) rc = gapa_ga_kernels_init(c);
    if (rc != GAPA_OK) return bail(rc);
    *out = c;
    return GAPA_OK;
}

void gapa_destroy(gapa_ctx* c) {
    if (!c) return;
    DeviceGuard guard(c->device);
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    free_graph(c->g);
    cudaFree(c->status);
    cudaFree(c->labels);
    cudaFree(c->ig_aux);
    cudaFree(c->sp_scratch);
    cudaFree(c->sp_order);
    cudaFree(c->sdst_buf);
    for (auto p : c->stage_pop) cudaFree(p);
    for (auto p : c->stage_fit) cudaFree(p);
    cudaFree(c->run_gen);
    cudaFree(c->run_best);
    cudaFree(c->run_traj);
    cudaFree(c->kids);
    cudaFree(c->kfit);
    cudaFree(c->cum);
    cudaFree(c->src);
    for (auto& t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->ev_a) cudaEventDestroy(c->ev_a);
    if (c->ev_b) cudaEventDestroy(c->ev_b);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

int gapa_set_stream(gapa_ctx* c, void* s) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    c->stream = (cudaStream_t)s;
    return GAPA_OK;
}

// A forest of the sparse fitness kernel from a BFS forest of G (or of G without some hubs' edges):
// children as (first, count) (BFS numbers them consecutively), the root of every node's tree (in BFS
// order every component is one tree; -1 for single-node components), component sizes at their
// roots, subtree sizes, the roots by decreasing size (ties: lower root), the per-member cost table
// by original id (children + 1) and the sum over components of C(size, 2).  With `own`, also the
// forest's numbering, parents, parent pairs and lower-neighbour and full adjacency in its
// numbering (rp, col: the graph it was built from).  Returns 1 (nothing uploaded) if some node's
// children are not consecutive.
int upload_sparse_forest(const BfsForest& bf, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                         int32_t n, bool own, bool packed16, SparseForest& f) {
    std::vector<int2> kids((size_t)n, make_int2(0, 0));
    for (int32_t x = 0; x < n; ++x) {
        const int32_t p = bf.tparent[x];
        if (p == x) continue;
        int2& kp = kids[p];
        if (kp.y == 0) kp.x = x;
        else if (kp.x + kp.y != x) return 1;  // not consecutive: no sparse kernel on this forest
        kp.y += 1;
    }
    std::vector<int32_t> croot((size_t)n), csize((size_t)n, 0), sub((size_t)n, 1), roots;
    for (int32_t x = 0; x < n; ++x) {
        const int32_t p = bf.tparent[x];
        croot[x] = p == x ? x : croot[p];
        csize[croot[x]] += 1;
        if (p == x) roots.push_back(x);
    }
    for (int32_t x = n - 1; x >= 0; --x)
        if (bf.tparent[x] != x) sub[bf.tparent[x]] += sub[x];
    std::stable_sort(roots.begin(), roots.end(), [&](int32_t a, int32_t b) { return csize[a] > csize[b]; });
    for (int32_t x = 0; x < n; ++x)
        if (csize[croot[x]] == 1) croot[x] = -1;  // a single-node component: nothing to recount
    std::vector<int32_t> cost((size_t)n);  // by original id: children + 1
    for (int32_t v = 0; v < n; ++v) cost[v] = kids[bf.perm[v]].y + 1;
    long long pc0 = 0;
    for (int32_t r : roots) pc0 += (long long)csize[r] * (csize[r] - 1) / 2;
    auto up = [](void** dst, const void* src, size_t bytes) {
        return cudaMalloc(dst, std::max<size_t>(bytes, 16)) == cudaSuccess &&
               (bytes == 0 || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess);
    };
    bool ok = up((void**)&f.kids, kids.data(), sizeof(int2) * (size_t)n) &&
              up((void**)&f.croot, croot.data(), 4 * (size_t)n) && up((void**)&f.csize, csize.data(), 4 * (size_t)n) &&
              up((void**)&f.sub, sub.data(), 4 * (size_t)n) && up((void**)&f.bysize, roots.data(), 4 * roots.size()) &&
              up((void**)&f.cost, cost.data(), 4 * (size_t)n);
    if (ok && own) {
        f.owns = true;
        std::vector<int2> palt((size_t)n);
        for (int32_t b = 0; b < n; ++b) {
            const int32_t cnt = bf.lo_ptr[b + 1] - bf.lo_ptr[b];
            palt[b] = make_int2(bf.tparent[b], cnt >= 2 ? bf.lo_col[bf.lo_ptr[b] + 1] : -1);
        }
        std::vector<int32_t> inv((size_t)n), fptr((size_t)n + 1, 0), fcol(std::max<size_t>(col.size(), 1));
        for (int32_t v = 0; v < n; ++v) inv[bf.perm[v]] = v;
        for (int32_t b = 0; b < n; ++b) {
            const int32_t v = inv[b];
            int32_t o = fptr[b];
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) fcol[o++] = bf.perm[col[e]];
            fptr[b + 1] = o;
        }
        ok = up((void**)&f.perm, bf.perm.data(), 4 * (size_t)n) && up((void**)&f.tparent, bf.tparent.data(), 4 * (size_t)n) &&
             up((void**)&f.palt, palt.data(), sizeof(int2) * (size_t)n) &&
             up((void**)&f.lo_ptr, bf.lo_ptr.data(), 4 * ((size_t)n + 1)) &&
             up((void**)&f.lo_col, bf.lo_col.data(), 4 * bf.lo_col.size()) &&
             up((void**)&f.fptr, fptr.data(), 4 * ((size_t)n + 1));
        if (ok && packed16) {
            std::vector<uint16_t> f16(fcol.begin(), fcol.end());
            ok = up((void**)&f.fcol16, f16.data(), 2 * f16.size());
        } else if (ok) {
            ok = up((void**)&f.fcol32, fcol.data(), 4 * fcol.size());
        }
    }
    if (!ok) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "sparse fitness forest of %d nodes", n);
    }
    f.ncomp = (int)roots.size();
    f.giant = roots.empty() ? -1 : roots[0];
    f.pc0 = pc0;
    return GAPA_OK;
}

// The sparse kernel's forests: forest 0 on G (borrowing the graph's BFS arrays), then forests of G
// with every edge of the top hub, of the two top hubs, and of the second hub removed (the hubs by
// degree; a member that deletes them has the same PC on either graph, and in the reduced graph's
// forest deleting them cuts nothing).
int upload_sparse_forests(const BfsForest& bf, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                          const std::vector<int32_t>& by_degree, int32_t n, DeviceGraph& g) {
    SparseForest& f0 = g.spf[0];
    f0.perm = g.perm;
    f0.tparent = g.tparent;
    f0.palt = g.palt;
    f0.lo_ptr = g.lo_ptr;
    f0.lo_col = g.lo_col;
    f0.fptr = g.fptr;
    f0.fcol32 = g.fcol32;
    f0.fcol16 = g.fcol16;
    int rc = upload_sparse_forest(bf, rp, col, n, false, g.packed16, f0);
    if (rc == 1) {  // no sparse kernel on this graph
        f0 = SparseForest();
        return GAPA_OK;
    }
    if (rc != GAPA_OK) return rc;
    g.sp_nforests = 1;
    for (int i = 0; i < 2; ++i) {
        const int32_t h = i < (int)by_degree.size() ? by_degree[i] : -1;
        g.sp_hub[i] = (h >= 0 && rp[h + 1] > rp[h]) ? h : -1;
    }
    // removed hubs of forests 1, 2, 3
    const int32_t removed[3][2] = {{g.sp_hub[0], -1}, {g.sp_hub[0], g.sp_hub[1]}, {g.sp_hub[1], -1}};
    for (int fi = 1; fi < kSpForests; ++fi) {
        const int32_t a = removed[fi - 1][0], b = removed[fi - 1][1];
        if (a < 0 || (fi == 2 && b < 0)) continue;
        std::vector<int32_t> rp2((size_t)n + 1, 0), col2;
        col2.reserve(col.size());
        for (int32_t v = 0; v < n; ++v) {
            if (v != a && v != b)
                for (int32_t e = rp[v]; e < rp[v + 1]; ++e)
                    if (col[e] != a && col[e] != b) col2.push_back(col[e]);
            rp2[v + 1] = (int32_t)col2.size();
        }
        const BfsForest bf2 = bfs_forest(n, rp2, col2);
        rc = upload_sparse_forest(bf2, rp2, col2, n, true, g.packed16, g.spf[fi]);
        if (rc == 1) {
            g.spf[fi] = SparseForest();
            continue;
        }
        if (rc != GAPA_OK) return rc;
    }
    g.sp_nforests = kSpForests;
    return GAPA_OK;
}

int gapa_graph_upload(gapa_ctx* c, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, int where) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (n < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "n must be >= 1 (got %d)", n);
    if (nnz < 0 || nnz >= (1LL << 31)) return gapa_fail(GAPA_ERR_INVALID_ARG, "nnz out of range (%lld)", (long long)nnz);
    if (nnz & 1) return gapa_fail(GAPA_ERR_INVALID_GRAPH, "odd arc count %lld cannot be symmetric", (long long)nnz);
    if (!row_ptr || (nnz > 0 && !col)) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL CSR array");
    if (where != GAPA_WHERE_HOST && where != GAPA_WHERE_DEVICE) return gapa_fail(GAPA_ERR_INVALID_ARG, "bad 'where'");
    DeviceGuard guard(c->device);
    std::vector<int32_t> rp((size_t)n + 1), cin;
    const int32_t* src_col = col;
    if (where == GAPA_WHERE_DEVICE) {
        GAPA_CUDA(cudaMemcpy(rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
        cin.resize((size_t)nnz);
        if (nnz) GAPA_CUDA(cudaMemcpy(cin.data(), col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost));
        src_col = cin.data();
    } else {
        std::memcpy(rp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1));
    }
    std::vector<int32_t> sorted;
    int rc = validate_csr(n, nnz, rp.data(), src_col, sorted);
    if (rc != GAPA_OK) return rc;
    // undirected edge list (u < v) in CSR order, and the highest-degree nodes
    const int E = (int)(nnz / 2);
    std::vector<int2> edges;
    edges.reserve((size_t)E);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e)
            if (sorted[e] > u) edges.push_back(make_int2(u, sorted[e]));
    std::vector<int32_t> order((size_t)n);
    for (int32_t v = 0; v < n; ++v) order[v] = v;
    const int np = std::min(n, kProbe);
    std::partial_sort(order.begin(), order.begin() + np, order.end(), [&](int32_t a, int32_t b) {
        const int32_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
        return da != db ? da > db : a < b;
    });
    std::vector<int32_t> probe(kProbe, order[0]);
    for (int i = 0; i < np; ++i) probe[i] = order[i];
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    free_graph(c->g);
    DeviceGraph g;
    g.n = n;
    g.nnz = nnz;
    g.num_edges = E;
    g.max_degree = rp[order[0] + 1] - rp[order[0]];
    if (cudaMalloc(&g.row_ptr, sizeof(int32_t) * ((size_t)n + 1)) != cudaSuccess ||
        cudaMalloc(&g.col, sizeof(int32_t) * std::max<size_t>((size_t)nnz, 1)) != cudaSuccess ||
        cudaMalloc(&g.edges, sizeof(int2) * std::max<size_t>((size_t)E, 2)) != cudaSuccess ||
        cudaMalloc(&g.probe, sizeof(int32_t) * kProbe) != cudaSuccess) {
        free_graph(g);
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "graph of %d nodes, %lld arcs", n, (long long)nnz);
    }
    GAPA_CUDA(cudaMemcpy(g.row_ptr, rp.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice));
    if (nnz) GAPA_CUDA(cudaMemcpy(g.col, sorted.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice));
    if (E) GAPA_CUDA(cudaMemcpy(g.edges, edges.data(), sizeof(int2) * (size_t)E, cudaMemcpyHostToDevice));
    GAPA_CUDA(cudaMemcpy(g.probe, probe.data(), sizeof(int32_t) * kProbe, cudaMemcpyHostToDevice));
    // BFS forest numbering for the TREE kernel
    BfsForest bf = bfs_forest(n, rp, sorted);
    g.bfs_depth = bf.depth;
    g.num_nontree = (int)bf.nontree.size();
    g.mean_deg_x16 = n > 0 ? (int)((16 * nnz + n - 1) / n) : 0;
    // 16-bit ids only on the shared-memory path (labels + deleted-node bitmap)
    g.packed16 = n <= 65536 && gapa_dev::tree16_smem_bytes(n) <= c->fit_smem_max;
    const size_t nt_bytes = (g.packed16 ? 4 : 8) * std::max<size_t>(bf.nontree.size(), 4);
    const size_t par_ints = gapa_dev::tree16l_lab_ints(n);  // padded for the bulk copy of the cut-local kernel
    if (cudaMalloc(&g.perm, sizeof(int32_t) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&g.tparent, sizeof(int32_t) * par_ints) != cudaSuccess ||
        cudaMalloc(&g.lo_ptr, sizeof(int32_t) * ((size_t)n + 1)) != cudaSuccess ||
        cudaMalloc(&g.lo_col, sizeof(int32_t) * std::max<size_t>(bf.lo_col.size(), 1)) != cudaSuccess ||
        cudaMalloc(&g.nontree, nt_bytes) != cudaSuccess) {
        free_graph(g);
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "BFS forest of %d nodes", n);
    }
    GAPA_CUDA(cudaMemcpy(g.perm, bf.perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
    {
        std::vector<int32_t> par(bf.tparent);
        par.resize(par_ints, 0);
        GAPA_CUDA(cudaMemcpy(g.tparent, par.data(), sizeof(int32_t) * par_ints, cudaMemcpyHostToDevice));
    }
    if (g.packed16) {
        // cut-local TREE kernel: children ranges (consecutive in BFS order), component roots, and a
        // list region as large as two members per SM allow (one per SM when the labels need it)
        std::vector<int4> kids((size_t)n);
        bool contiguous = true;
        for (int32_t b = 0; b < n; ++b) kids[b] = make_int4(b, 0, 0, 0);
        for (int32_t x = 0; x < n && contiguous; ++x) {
            const int32_t p = bf.tparent[x];
            if (p == x) continue;
            if (kids[p].y == 0) kids[p].x = x;
            else if (kids[p].x + kids[p].y != x) contiguous = false;
            kids[p].y += 1;
        }
        const int team = gapa_fitness_block_for(n);
        const size_t fixed = par_ints * 4 + 48, min_list = gapa_dev::tree16l_min_list_bytes(n, team);
        const size_t want = std::max(min_list, ((((size_t)n * 2) + 15) & ~(size_t)15) + gapa_dev::tree16l_bitmap_bytes(n) +
                                                   gapa_dev::tree16l_scratch_bytes(team));
        // two members per SM: half the SM's shared memory, less the runtime's reserve and the
        // kernel's static shared memory (under 1 KB)
        const size_t per_block = c->smem_per_sm / 2, other = c->smem_reserved + 1024;
        const size_t two_per_sm = per_block > other ? per_block - other : 0;
        size_t budget = fixed + min_list <= two_per_sm ? two_per_sm : c->fit_smem_max;
        budget = std::min(budget, c->fit_smem_max);
        size_t list_bytes = 0;
        if (contiguous && fixed + min_list <= budget) list_bytes = std::min(want, (budget - fixed) & ~(size_t)15);
        if (list_bytes) {
            // cost estimate of deleting node b: the nodes below those children of b whose only lower
            // neighbour is b (they become roots of pieces to be listed)
            std::vector<int32_t> below((size_t)n, 1), cut((size_t)n, 0);
            for (int32_t v = n - 1; v >= 0; --v)
                if (bf.tparent[v] != v) below[bf.tparent[v]] += below[v];
            for (int32_t v = 0; v < n; ++v)
                if (bf.tparent[v] != v && bf.lo_ptr[v + 1] - bf.lo_ptr[v] == 1) cut[bf.tparent[v]] += below[v];
            if (cudaMalloc(&g.kids, sizeof(int4) * std::max<size_t>((size_t)n, 1)) != cudaSuccess ||
                cudaMalloc(&g.cut, sizeof(int32_t) * std::max<size_t>((size_t)n, 1)) != cudaSuccess ||
                cudaMalloc(&g.order, sizeof(int32_t) * (5 * (size_t)kOrderCap + 16)) != cudaSuccess ||
                cudaMalloc(&g.roots, sizeof(int32_t) * std::max<size_t>(bf.roots.size(), 1)) != cudaSuccess) {
                free_graph(g);
                cudaGetLastError();
                return gapa_fail(GAPA_ERR_OOM, "children ranges of %d nodes", n);
            }
            GAPA_CUDA(cudaMemcpy(g.kids, kids.data(), sizeof(int4) * (size_t)n, cudaMemcpyHostToDevice));
            std::vector<int32_t> cut_by_id((size_t)n);  // indexed by original node id
            for (int32_t v = 0; v < n; ++v) cut_by_id[v] = cut[bf.perm[v]];
            GAPA_CUDA(cudaMemcpy(g.cut, cut_by_id.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
            if (!bf.roots.empty())
                GAPA_CUDA(cudaMemcpy(g.roots, bf.roots.data(), sizeof(int32_t) * bf.roots.size(),
                                     cudaMemcpyHostToDevice));
            g.num_roots = (int)bf.roots.size();
            g.local_list_bytes = (int)list_bytes;
            {
                // subtree intervals of the forest-piece kernel
                const ForestIntervals fi = forest_intervals(bf.tparent, bf.lo_ptr, bf.lo_col);
                auto up = [](void** dst, const void* src, size_t bytes) {
                    return cudaMalloc(dst, std::max<size_t>(bytes, 16)) == cudaSuccess &&
                           cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
                };
                if (!(up((void**)&g.sz, fi.sz.data(), 4 * (size_t)n) && up((void**)&g.pre, fi.pre.data(), 4 * (size_t)n) &&
                      up((void**)&g.at, fi.at.data(), 2 * (size_t)n) &&
                      up((void**)&g.crep, fi.crep.data(), 4 * (size_t)n) &&
                      up((void**)&g.nroot, fi.nroot.data(), 4 * (size_t)n) &&
                      up((void**)&g.csize, fi.csize.data(), 4 * (size_t)n))) {
                    free_graph(g);
                    cudaGetLastError();
                    return gapa_fail(GAPA_ERR_OOM, "subtree intervals of %d nodes", n);
                }
                g.tree_pc = fi.tree_pc;
            }
            // the second forest, numbered with the top hubs last (about 0.5 % of the nodes, 8 to 256):
            // members that delete hubs cut it far less
            const int hubs = std::max(8, std::min(256, n / 200));
            if (n > 4 * hubs) {
                const ForestHost fb = forest_host(n, rp, sorted, hub_last_perm(n, rp, sorted, hubs));
                if (fb.ok) {
                    int frc = upload_forest(fb, n, g.alt);
                    if (frc != GAPA_OK) {
                        free_graph(g);
                        return frc;
                    }
                    g.has_alt = true;
                }
            }
        }
    }
    GAPA_CUDA(cudaMemcpy(g.lo_ptr, bf.lo_ptr.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice));
    {
        // (tree parent, second lower neighbour) pairs
        std::vector<int2> palt((size_t)n);
        for (int32_t b = 0; b < n; ++b) {
            const int32_t cnt = bf.lo_ptr[b + 1] - bf.lo_ptr[b];
            palt[b] = make_int2(bf.tparent[b], cnt >= 2 ? bf.lo_col[bf.lo_ptr[b] + 1] : -1);
        }
        if (cudaMalloc(&g.palt, sizeof(int2) * (size_t)n) != cudaSuccess) {
            free_graph(g);
            cudaGetLastError();
            return gapa_fail(GAPA_ERR_OOM, "parent pairs of %d nodes", n);
        }
        GAPA_CUDA(cudaMemcpy(g.palt, palt.data(), sizeof(int2) * (size_t)n, cudaMemcpyHostToDevice));
    }
    if (!bf.lo_col.empty())
        GAPA_CUDA(cudaMemcpy(g.lo_col, bf.lo_col.data(), sizeof(int32_t) * bf.lo_col.size(), cudaMemcpyHostToDevice));

    {
        // full adjacency in BFS numbers (the scans of the nodes outside the giant piece): 16-bit ids
        // for the shared-memory kernel, 32-bit ids for the global-label one
        std::vector<int32_t> fptr((size_t)n + 1, 0), inv((size_t)n), fcol((size_t)std::max<int64_t>(nnz, 1));
        for (int32_t v = 0; v < n; ++v) inv[bf.perm[v]] = v;
        for (int32_t b = 0; b < n; ++b) {
            const int32_t v = inv[b];
            int32_t o = fptr[b];
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) fcol[o++] = bf.perm[sorted[e]];
            fptr[b + 1] = o;
        }
        bool ok = cudaMalloc(&g.fptr, sizeof(int32_t) * ((size_t)n + 1)) == cudaSuccess;
        if (ok && g.packed16) {
            std::vector<uint16_t> f16(fcol.begin(), fcol.end());
            ok = cudaMalloc(&g.fcol16, sizeof(uint16_t) * f16.size()) == cudaSuccess &&
                 cudaMemcpy(g.fcol16, f16.data(), sizeof(uint16_t) * f16.size(), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
        } else if (ok) {
            ok = cudaMalloc(&g.fcol32, sizeof(int32_t) * fcol.size()) == cudaSuccess &&
                 cudaMemcpy(g.fcol32, fcol.data(), sizeof(int32_t) * fcol.size(), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
        }
        if (!ok) {
            free_graph(g);
            cudaGetLastError();
            return gapa_fail(GAPA_ERR_OOM, "BFS-numbered adjacency of %d nodes", n);
        }
        GAPA_CUDA(cudaMemcpy(g.fptr, fptr.data(), sizeof(int32_t) * fptr.size(), cudaMemcpyHostToDevice));
    }
    if (g.packed16) {
        std::vector<uint32_t> w(bf.nontree.size());
        for (size_t i = 0; i < w.size(); ++i)
            w[i] = ((uint32_t)bf.nontree[i].first << 16) | (uint32_t)bf.nontree[i].second;
        if (!w.empty()) GAPA_CUDA(cudaMemcpy(g.nontree, w.data(), 4 * w.size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<int2> w(bf.nontree.size());
        for (size_t i = 0; i < w.size(); ++i) w[i] = make_int2(bf.nontree[i].first, bf.nontree[i].second);
        if (!w.empty()) GAPA_CUDA(cudaMemcpy(g.nontree, w.data(), 8 * w.size(), cudaMemcpyHostToDevice));
    }
    {
        const int frc = upload_sparse_forests(bf, rp, sorted, order, n, g);
        if (frc != GAPA_OK) {
            free_graph(g);
            return frc;
        }
    }
    c->g = g;
    return GAPA_OK;
}

int gapa_pop_init(gapa_ctx* c, const gapa_config* cfg, int32_t* pop_dev) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    if (!pop_dev && cfg->k > 0) return gapa_fail(GAPA_ERR_INVALID_ARG, "pop_dev is NULL");
    DeviceGuard guard(c->device);
    return gapa_launch_init(c, make_params(c, cfg, 0, nullptr), pop_dev, c->stream);
}

int gapa_fitness(gapa_ctx* c, const int32_t* pop_dev, int32_t s, int32_t k, int64_t* fit_dev) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (c->g.n <= 0) return gapa_fail(GAPA_ERR_STATE, "no graph uploaded");
    if (s < 0 || k < 0) return gapa_fail(GAPA_ERR_INVALID_ARG, "negative size (s=%d, k=%d)", s, k);
    if ((long long)s * k >= (1LL << 31)) return gapa_fail(GAPA_ERR_INVALID_ARG, "s*k must be below 2^31");
    if (s > 0 && (!fit_dev || (!pop_dev && k > 0))) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard guard(c->device);
    return gapa_launch_fitness(c, pop_dev, s, k, fit_dev, c->stream);
}

int gapa_fitness_host(gapa_ctx* c, const int32_t* pop_host, int32_t s, int32_t k, int64_t* fit_host) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (c->g.n <= 0) return gapa_fail(GAPA_ERR_STATE, "no graph uploaded");
    if (s < 0 || k < 0) return gapa_fail(GAPA_ERR_INVALID_ARG, "negative size (s=%d, k=%d)", s, k);
    if ((long long)s * k >= (1LL << 31)) return gapa_fail(GAPA_ERR_INVALID_ARG, "s*k must be below 2^31");
    if (s == 0) return GAPA_OK;
    if (!fit_host || (!pop_host && k > 0)) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard guard(c->device);
    int rc = ensure_stage(c, (size_t)s * k, (size_t)s);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = c->stream;
    if (k) GAPA_CUDA(cudaMemcpyAsync(c->stage_pop[0], pop_host, sizeof(int32_t) * (size_t)s * k, cudaMemcpyHostToDevice, st));
    rc = gapa_launch_fitness(c, c->stage_pop[0], s, k, c->stage_fit[0], st);
    if (rc != GAPA_OK) return rc;
    GAPA_CUDA(cudaMemcpyAsync(fit_host, c->stage_fit[0], sizeof(int64_t) * (size_t)s, cudaMemcpyDeviceToHost, st));
    return read_status(c, st);
}

int gapa_generation(gapa_ctx* c, const gapa_config* cfg, int32_t g, const int32_t* pop_in, const int64_t* fit_in,
                    int32_t* pop_out, int64_t* fit_out) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    if (g < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "generation index must be >= 1 (got %d)", g);
    if (!fit_in || !fit_out || (cfg->k > 0 && (!pop_in || !pop_out)))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    if (pop_in == pop_out || fit_in == fit_out) return gapa_fail(GAPA_ERR_INVALID_ARG, "outputs alias inputs");
    DeviceGuard guard(c->device);
    rc = ensure_variant_scratch(c, cfg);
    if (rc != GAPA_OK) return rc;
    return enqueue_generation(c, make_params(c, cfg, g, nullptr), cfg->lambda, pop_in, fit_in, pop_out, fit_out,
                              c->stream);
}

int gapa_offspring(gapa_ctx* c, const gapa_config* cfg, int32_t g, const int32_t* pop_in, const int64_t* fit_in,
                   int32_t* pop_out, int64_t* fit_out) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    if (cfg->flags & GAPA_FLAG_MU_PLUS_LAMBDA)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "gapa_offspring covers the elitism mode only");
    if (g < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "generation index must be >= 1 (got %d)", g);
    if (!fit_in || !fit_out || (cfg->k > 0 && (!pop_in || !pop_out)))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    if (pop_in == pop_out || fit_in == fit_out) return gapa_fail(GAPA_ERR_INVALID_ARG, "outputs alias inputs");
    DeviceGuard guard(c->device);
    GaParams p = make_params(c, cfg, g, nullptr);
    if (p.flags & GAPA_FLAG_ROULETTE) {
        rc = gapa_reserve((void**)&c->cum, &c->cum_cap, (size_t)cfg->pop, sizeof(int64_t));
        if (rc == GAPA_OK) rc = gapa_launch_roulette_prefix(fit_in, p.s, c->cum, c->stream);
        if (rc != GAPA_OK) return rc;
        p.cum = reinterpret_cast<const long long*>(c->cum);
    }
    return gapa_launch_offspring(c, p, pop_in, fit_in, pop_out, fit_out, c->stream);
}

int gapa_generation_host(gapa_ctx* c, const gapa_config* cfg, int32_t g, const int32_t* pop_in_host,
                         const int64_t* fit_in_host, int32_t* pop_out_host, int64_t* fit_out_host) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    if (g < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "generation index must be >= 1 (got %d)", g);
    if (!fit_in_host || !fit_out_host || (cfg->k > 0 && (!pop_in_host || !pop_out_host)))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard guard(c->device);
    const size_t cells = (size_t)cfg->pop * cfg->k;
    rc = ensure_stage(c, cells, (size_t)cfg->pop);
    if (rc != GAPA_OK) return rc;
    rc = ensure_variant_scratch(c, cfg);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = c->stream;
    if (cells) GAPA_CUDA(cudaMemcpyAsync(c->stage_pop[0], pop_in_host, sizeof(int32_t) * cells, cudaMemcpyHostToDevice, st));
    GAPA_CUDA(cudaMemcpyAsync(c->stage_fit[0], fit_in_host, sizeof(int64_t) * cfg->pop, cudaMemcpyHostToDevice, st));
    rc = enqueue_generation(c, make_params(c, cfg, g, nullptr), cfg->lambda, c->stage_pop[0], c->stage_fit[0],
                            c->stage_pop[1], c->stage_fit[1], st);
    if (rc != GAPA_OK) return rc;
    if (cells) GAPA_CUDA(cudaMemcpyAsync(pop_out_host, c->stage_pop[1], sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, st));
    GAPA_CUDA(cudaMemcpyAsync(fit_out_host, c->stage_fit[1], sizeof(int64_t) * cfg->pop, cudaMemcpyDeviceToHost, st));
    return read_status(c, st);
}

int gapa_run(gapa_ctx* c, const gapa_config* cfg, int32_t* best_set_host, int64_t* best_fit, int64_t* traj_best_fit,
             int32_t* final_pop_dev) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    int rc = check_cfg(c, cfg);
    if (rc != GAPA_OK) return rc;
    if (!best_fit || (cfg->k > 0 && !best_set_host)) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL output pointer");
    DeviceGuard guard(c->device);
    const int s = cfg->pop, k = cfg->k, G = cfg->gens;
    const size_t cells = (size_t)s * k;
    rc = ensure_stage(c, cells, (size_t)s);
    if (rc == GAPA_OK) rc = gapa_reserve((void**)&c->run_traj, &c->run_traj_cap, (size_t)G + 1, sizeof(int64_t));
    if (rc == GAPA_OK) rc = ensure_variant_scratch(c, cfg);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = c->own_stream;
    // order after the caller's pending work
    GAPA_CUDA(cudaEventRecord(c->ev_a, c->stream));
    GAPA_CUDA(cudaStreamWaitEvent(st, c->ev_a, 0));
    int32_t* P[2] = {c->stage_pop[0], c->stage_pop[1]};
    int64_t* F[2] = {c->stage_fit[0], c->stage_fit[1]};
    GAPA_CUDA(cudaMemsetAsync(c->run_gen, 0, sizeof(int), st));
    const GaParams p0 = make_params(c, cfg, 0, nullptr);
    rc = gapa_launch_init(c, p0, P[0], st);
    if (rc == GAPA_OK) rc = gapa_launch_fitness(c, P[0], s, k, F[0], st);
    if (rc == GAPA_OK) rc = gapa_launch_record(c, F[0], s, c->run_gen, c->run_traj, c->run_best, st);
    if (rc != GAPA_OK) return rc;
    const GaParams pg = make_params(c, cfg, 0, c->run_gen);  // generation read from the device counter
    if (G >= 2) {
        // capture two generations (P0 -> P1 -> P0) and replay them G/2 times
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        GAPA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        int crc = GAPA_OK;
        for (int h = 0; h < 2 && crc == GAPA_OK; ++h) {
            crc = enqueue_generation(c, pg, cfg->lambda, P[h], F[h], P[h ^ 1], F[h ^ 1], st);
            if (crc == GAPA_OK) crc = gapa_launch_record(c, F[h ^ 1], s, c->run_gen, c->run_traj, c->run_best, st);
        }
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        c->capturing = false;
        if (crc != GAPA_OK) {
            if (graph) cudaGraphDestroy(graph);
            return crc;
        }
        GAPA_CUDA(ce);
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        GAPA_CUDA(ce);
        for (int r = 0; r < G / 2; ++r) {
            ce = cudaGraphLaunch(exec, st);
            if (ce != cudaSuccess) break;
        }
        cudaGraphExecDestroy(exec);
        GAPA_CUDA(ce);
    }
    if (G % 2 == 1) {
        // the last (odd) generation, launched directly: P0 -> P1
        rc = enqueue_generation(c, pg, cfg->lambda, P[0], F[0], P[1], F[1], st);
        if (rc == GAPA_OK) rc = gapa_launch_record(c, F[1], s, c->run_gen, c->run_traj, c->run_best, st);
        if (rc != GAPA_OK) return rc;
    }
    const int fin = G % 2;
    int best = 0;
    GAPA_CUDA(cudaMemcpyAsync(&best, c->run_best, sizeof(int), cudaMemcpyDeviceToHost, st));
    GAPA_CUDA(cudaStreamSynchronize(st));
    rc = read_status(c, st);
    if (rc != GAPA_OK) return rc;
    GAPA_CUDA(cudaMemcpyAsync(best_fit, F[fin] + best, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (k) GAPA_CUDA(cudaMemcpyAsync(best_set_host, P[fin] + (size_t)best * k, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
    if (traj_best_fit)
        GAPA_CUDA(cudaMemcpyAsync(traj_best_fit, c->run_traj, sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyDeviceToHost, st));
    if (final_pop_dev && cells)
        GAPA_CUDA(cudaMemcpyAsync(final_pop_dev, P[fin], sizeof(int32_t) * cells, cudaMemcpyDeviceToDevice, st));
    GAPA_CUDA(cudaStreamSynchronize(st));
    std::sort(best_set_host, best_set_host + k);
    // later work on the caller's stream sees the final population
    GAPA_CUDA(cudaEventRecord(c->ev_b, st));
    GAPA_CUDA(cudaStreamWaitEvent(c->stream, c->ev_b, 0));
    return GAPA_OK;
}

int gapa_set_fitness_kernel(gapa_ctx* c, int variant) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (variant < GAPA_FITNESS_AUTO || variant > GAPA_FITNESS_SPARSE)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "unknown fitness kernel %d", variant);
    c->fitness_variant = variant;
    return GAPA_OK;
}

int gapa_set_genes(gapa_ctx* c, int gene_type) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (gene_type != GAPA_GENES_NODES && gene_type != GAPA_GENES_EDGES)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "unknown gene type %d", gene_type);
    c->genes = gene_type;
    return GAPA_OK;
}

int gapa_set_objective(gapa_ctx* c, int objective) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (objective < GAPA_OBJECTIVE_PC || objective > GAPA_OBJECTIVE_SIXDST_MCN)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "unknown objective %d", objective);
    c->objective = objective;
    return GAPA_OK;
}

int gapa_selftest_wait(gapa_ctx* c, int64_t spin_limit) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (spin_limit < 1 || spin_limit > (1LL << 26)) return gapa_fail(GAPA_ERR_INVALID_ARG, "spin limit out of range");
    DeviceGuard guard(c->device);
    int rc = gapa_launch_selftest_wait(c, (long long)spin_limit, c->stream);
    if (rc != GAPA_OK) return rc;
    return read_status(c, c->stream);
}

int gapa_read_bandwidth(gapa_ctx* c, int64_t bytes, int32_t reps, double* gbs) {
    if (!c || !gbs) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    if (bytes < (1 << 20) || bytes > (1LL << 30) || bytes % 16 || reps < 1 || reps > 1000)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "probe size or repetitions out of range");
    DeviceGuard guard(c->device);
    const int grid = c->num_sms * 8;
    const int passes = (int)std::max<int64_t>(1, (1LL << 30) / bytes);  // about 1 GiB read per timed launch
    void* buf = nullptr;
    unsigned* sink = nullptr;
    if (cudaMalloc(&buf, (size_t)bytes) != cudaSuccess || cudaMalloc(&sink, sizeof(unsigned) * grid) != cudaSuccess) {
        cudaFree(buf);
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "probe buffer of %lld bytes", (long long)bytes);
    }
    cudaStream_t st = c->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GAPA_OK;
    float best = 1e30f;
    if (cudaMemsetAsync(buf, 1, (size_t)bytes, st) != cudaSuccess || cudaMemsetAsync(sink, 0, sizeof(unsigned) * grid, st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = gapa_fail(GAPA_ERR_CUDA, "probe setup");
    if (rc == GAPA_OK) rc = gapa_launch_read_probe(buf, (size_t)bytes, 1, grid, sink, st);  // warm-up
    for (int r = 0; r < reps && rc == GAPA_OK; ++r) {
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = gapa_fail(GAPA_ERR_CUDA, "probe event");
        if (rc == GAPA_OK) rc = gapa_launch_read_probe(buf, (size_t)bytes, passes, grid, sink, st);
        if (rc == GAPA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = gapa_fail(GAPA_ERR_CUDA, "probe timing");
        if (rc == GAPA_OK) best = std::min(best, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(sink);
    if (rc == GAPA_OK) *gbs = (double)bytes * passes / (best / 1e3) / 1e9;
    return rc;
}

int gapa_set_sixdst_kernel(gapa_ctx* c, int kernel) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (kernel != GAPA_SIXDST_MMA_SYNC && kernel != GAPA_SIXDST_TCGEN05 && kernel != GAPA_SIXDST_TCGEN05_128 &&
        kernel != GAPA_SIXDST_TMA)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "unknown SixDST kernel %d", kernel);
    if (kernel != GAPA_SIXDST_MMA_SYNC && !c->sixdst_t5_ok)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "the tcgen05 product does not fit in this device's shared memory");
    if (kernel == GAPA_SIXDST_TMA && !c->sixdst_t7_ok)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "the TMA product is not available on this device");
    c->sixdst_kernel = kernel;
    return GAPA_OK;
}

int gapa_set_sixdst_hops(gapa_ctx* c, int hops) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    if (hops < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "hops must be >= 1 (got %d)", hops);
    c->sixdst_hops = hops;
    return GAPA_OK;
}

int gapa_profile_begin(gapa_ctx* c) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    c->profiling = true;
    return GAPA_OK;
}

int gapa_profile_end(gapa_ctx* c, gapa_profile* out) {
    if (!c || !out) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(c->device);
    c->profiling = false;
    *out = gapa_profile{0.0, 0.0, 0, 0, 0, 0.0, 0};
    int rc = GAPA_OK;
    for (auto& t : c->timed) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e != cudaSuccess && rc == GAPA_OK) rc = gapa_cuda_fail(e, "profile event");
        if (t.kind == 0) {
            out->fitness_ms += ms;
            out->fitness_launches += t.kernels;
            out->fitness_calls += 1;
            out->evals += t.evals;
        } else if (t.kind == 1) {  // `evals` holds the kernel count when it is above 1
            out->operators_ms += ms;
            out->operator_launches += std::max(1, t.evals);
        } else {  // surrogate phase: `evals` holds its kernel count
            out->surrogate_ms += ms;
            out->surrogate_launches += t.evals;
        }
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->timed.clear();
    return rc;
}

int gapa_sync(gapa_ctx* c) {
    if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard guard(c->device);
    GAPA_CUDA(cudaStreamSynchronize(c->stream));
    return read_status(c, c->stream);
}

}  // extern "C"
