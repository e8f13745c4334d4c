// Batched runs: many independent GA instances (graphs of uneven size, each
// with its own configuration) advanced together.  Per generation there is one
// launch of the operator kernel over the rows of all instances, one launch of
// a persistent fitness kernel over a work queue of (instance, members)
// packets, and one record launch; two generations are captured as a CUDA
// graph and replayed, with the generation counter kept on the device.  The
// members-per-CTA of each graph-size bucket is picked by an autotuner that
// times the candidates and caches the choice in a JSON file.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "gapa_internal.cuh"
#include "tree16.cuh"

struct gapa_batch {
    int device = 0;
    int num = 0;
    std::vector<gapa_ctx*> ctxs;  // borrowed; hold the uploaded graphs
    std::vector<gapa_config> cfgs;
    cudaStream_t stream = nullptr;  // ctxs[0]'s stream (borrowed)
    cudaStream_t own = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int* status = nullptr;          // ctxs[0]'s status word
    std::vector<int> teams;         // members per CTA per instance
    std::vector<int> use_local;     // per instance: the cut-local kernel
    unsigned* d_est = nullptr;      // cost estimates of the local instances' rows (two per row)
    // device memory
    BatchDesc* d_desc = nullptr;
    int2* d_rows = nullptr;
    BatchPacket* d_pk = nullptr;    // [0, npk_all): all members; [npk_all, npk_all + npk_kids): children
    int npk_all = 0, npk_kids = 0;
    int* d_head = nullptr;
    int* d_gen = nullptr;
    int* d_best = nullptr;          // [num]
    int64_t* d_traj = nullptr;      // [num][traj_cap]
    size_t traj_cap = 0;
    void* d_buf = nullptr;          // populations and fitness of all instances
    int total_rows = 0;
    size_t row_smem = 0, fit_smem = 0;
    size_t ga_max_dyn = 0, fit_max_dyn = 0;
    int fit_grid = 0;
    std::vector<BatchDesc> desc;
    std::vector<size_t> pop_off;    // element offsets of each instance's populations in d_buf
};

namespace {

size_t need16(int n) { return gapa_dev::tree16_smem_bytes(n); }

// Slice of one team of T threads that also holds the cut-local kernel's layout (minimum list region).
size_t need_local(int n, int T) {
    return gapa_dev::tree16l_lab_ints(n) * 4 + gapa_dev::tree16l_min_list_bytes(n, T) + 48;
}

// Slice bytes of instance x at c teams: the cut-local layout where the graph has it and c slices of
// it fit, else the full pipeline's.
size_t slice_need(const gapa_batch* b, int x, int c);

// Largest team count (1, 2, 4, 8) whose slices hold the graph and keep >= 128 threads per team
// and at least ~8 nodes per thread.
int default_teams(int n, size_t max_dyn) {
    int best = 1;
    for (int c = 2; c <= 8; c *= 2) {
        const int T = 1024 / c;
        if ((size_t)c * need16(n) + 16 * c > max_dyn || T < 128) break;
        if (n < 8 * T) best = c;
    }
    return best;
}

void free_batch_device(gapa_batch* b) {
    cudaFree(b->d_est);
    b->d_est = nullptr;
    cudaFree(b->d_desc);
    cudaFree(b->d_rows);
    cudaFree(b->d_pk);
    cudaFree(b->d_head);
    cudaFree(b->d_gen);
    cudaFree(b->d_best);
    cudaFree(b->d_traj);
    cudaFree(b->d_buf);
    b->d_desc = nullptr;
    b->d_rows = nullptr;
    b->d_pk = nullptr;
    b->d_head = b->d_gen = b->d_best = nullptr;
    b->d_traj = nullptr;
    b->d_buf = nullptr;
}

size_t slice_need(const gapa_batch* b, int x, int c) {
    const DeviceGraph& g = b->ctxs[x]->g;
    const size_t full = need16(g.n);
    if (!b->desc[x].kids || !b->use_local[x]) return full;  // the instance runs the full pipeline
    const size_t local = std::max(full, need_local(g.n, 1024 / c));
    return (size_t)c * ((local + 15) & ~(size_t)15) <= b->fit_max_dyn ? local : full;
}

// Work-queue packets for the current team counts, largest graphs first.
int build_packets(gapa_batch* b) {
    std::vector<int> order(b->num);
    for (int i = 0; i < b->num; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const long long cx = (long long)b->ctxs[x]->g.n + b->ctxs[x]->g.num_edges;
        const long long cy = (long long)b->ctxs[y]->g.n + b->ctxs[y]->g.num_edges;
        return cx > cy;
    });
    std::vector<BatchPacket> all, kids;
    size_t smem = 0;
    for (int x : order) {
        const int c = b->teams[x];
        smem = std::max(smem, (size_t)c * ((slice_need(b, x, c) + 15) & ~(size_t)15));
        for (int first = 0; first <= 1; ++first) {
            auto& list = first == 0 ? all : kids;
            for (int i0 = first; i0 < b->cfgs[x].pop; i0 += c)
                list.push_back(BatchPacket{x, i0, std::min(c, b->cfgs[x].pop - i0), c});
        }
    }
    b->fit_smem = (smem + 15) & ~(size_t)15;
    if (b->fit_smem > b->fit_max_dyn) return gapa_fail(GAPA_ERR_INVALID_ARG, "batched fitness needs %zu bytes of shared memory", b->fit_smem);
    int per_sm = 0;
    int rc = gapa_fitness_batched_occupancy(b->fit_smem, &per_sm);
    if (rc != GAPA_OK) return rc;
    b->fit_grid = std::max(1, per_sm) * b->ctxs[0]->num_sms;
    b->npk_all = (int)all.size();
    b->npk_kids = (int)kids.size();
    all.insert(all.end(), kids.begin(), kids.end());
    cudaFree(b->d_pk);
    b->d_pk = nullptr;
    if (cudaMalloc(&b->d_pk, sizeof(BatchPacket) * std::max<size_t>(all.size(), 1)) != cudaSuccess)
        return gapa_fail(GAPA_ERR_OOM, "batch packets");
    GAPA_CUDA(cudaMemcpy(b->d_pk, all.data(), sizeof(BatchPacket) * all.size(), cudaMemcpyHostToDevice));
    for (int i = 0; i < b->num; ++i) {
        BatchDesc& d = b->desc[i];
        d.teams = b->teams[i];
        // the cut-local kernel where the instance's slice holds its layout
        const int n = b->ctxs[i]->g.n, T = 1024 / d.teams;
        const size_t slice = (b->fit_smem / (size_t)d.teams) & ~(size_t)15;
        const size_t fixed = gapa_dev::tree16l_lab_ints(n) * 4 + 48;
        d.list_bytes = 0;
        if (d.kids && b->use_local[i] && slice >= fixed + gapa_dev::tree16l_min_list_bytes(n, T))
            d.list_bytes = (int)((slice - fixed) & ~(size_t)15);
    }
    return GAPA_OK;
}

int upload_desc(gapa_batch* b) {
    GAPA_CUDA(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(BatchDesc) * b->num, cudaMemcpyHostToDevice));
    return GAPA_OK;
}

// Initial population and fitness of every instance (generation 0), then record.
int enqueue_start(gapa_batch* b, cudaStream_t st) {
    GAPA_CUDA(cudaMemsetAsync(b->d_gen, 0, sizeof(int), st));
    int rc = gapa_launch_init_batched(b->d_desc, b->d_rows, b->total_rows, b->row_smem, 0, st);
    if (rc == GAPA_OK)
        rc = gapa_launch_fitness_batched(b->d_desc, b->d_pk, b->npk_all, b->d_head, 0, b->fit_smem, b->fit_grid,
                                         b->status, st);
    if (rc == GAPA_OK) rc = gapa_launch_record_batched(b->d_desc, b->num, 0, b->d_gen, true, st);
    return rc;
}

// One generation from buffer src to src^1.
int enqueue_generation(gapa_batch* b, int src, cudaStream_t st) {
    int rc = gapa_launch_offspring_batched(b->d_desc, b->d_rows, b->total_rows, b->row_smem, src, b->d_gen,
                                           b->status, st);
    if (rc == GAPA_OK)
        rc = gapa_launch_fitness_batched(b->d_desc, b->d_pk + b->npk_all, b->npk_kids, b->d_head, src ^ 1,
                                         b->fit_smem, b->fit_grid, b->status, st);
    if (rc == GAPA_OK) rc = gapa_launch_record_batched(b->d_desc, b->num, src ^ 1, b->d_gen, true, st);
    return rc;
}

std::string device_name(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string s = p.name;
    for (auto& ch : s)
        if (ch == '"' || ch == '\\') ch = '_';
    return s;
}

// Graph-size buckets of the autotuner: upper bounds on n.
const int kBuckets[] = {2048, 4096, 8192, 16384, 32768, 65536};

int bucket_of(int n) {
    int i = 0;
    while (i < 5 && n > kBuckets[i]) ++i;
    return i;
}

// Minimal reader/writer of {"device": {"bucket": teams, ...}, ...}.
std::map<std::string, std::map<int, int>> read_cache(const char* path) {
    std::map<std::string, std::map<int, int>> out;
    std::ifstream f(path);
    if (!f) return out;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t i = 0;
    auto next_str = [&](std::string& s) -> bool {
        const size_t a = t.find('"', i);
        if (a == std::string::npos) return false;
        const size_t e = t.find('"', a + 1);
        if (e == std::string::npos) return false;
        s = t.substr(a + 1, e - a - 1);
        i = e + 1;
        return true;
    };
    std::string dev;
    while (next_str(dev)) {
        const size_t open = t.find('{', i), close = t.find('}', i);
        if (open == std::string::npos || close == std::string::npos || open > close) break;
        i = open + 1;
        std::string key;
        while (true) {
            const size_t q = t.find('"', i);
            if (q == std::string::npos || q > close) break;
            if (!next_str(key)) break;
            const size_t colon = t.find(':', i);
            if (colon == std::string::npos || colon > close) break;
            out[dev][atoi(key.c_str())] = atoi(t.c_str() + colon + 1);
            i = colon + 1;
        }
        i = close + 1;
    }
    return out;
}

void write_cache(const char* path, const std::map<std::string, std::map<int, int>>& c) {
    std::ofstream f(path);
    f << "{\n";
    size_t di = 0;
    for (auto& d : c) {
        f << "  \"" << d.first << "\": {";
        size_t bi = 0;
        for (auto& kv : d.second) f << (bi++ ? ", " : "") << "\"" << kv.first << "\": " << kv.second;
        f << "}" << (++di < c.size() ? "," : "") << "\n";
    }
    f << "}\n";
}

}  // namespace

extern "C" {

int gapa_batch_create(gapa_batch** out, int32_t num, gapa_ctx* const* ctxs, const gapa_config* cfgs) {
    if (!out || !ctxs || !cfgs || num < 1) return gapa_fail(GAPA_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    for (int i = 0; i < num; ++i) {
        gapa_ctx* c = ctxs[i];
        if (!c) return gapa_fail(GAPA_ERR_INVALID_ARG, "context %d is NULL", i);
        if (c->device != ctxs[0]->device) return gapa_fail(GAPA_ERR_INVALID_ARG, "contexts on different devices");
        if (c->g.n <= 0) return gapa_fail(GAPA_ERR_STATE, "context %d has no graph", i);
        if (c->genes != GAPA_GENES_NODES)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "instance %d: batched runs take node genes only", i);
        if (c->objective != GAPA_OBJECTIVE_PC && c->objective != GAPA_OBJECTIVE_MCN)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "instance %d: batched runs take the PC or MCN objective", i);
        if (!c->g.packed16)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "instance %d: batched runs need graphs whose labels fit in shared memory (n=%d)", i, c->g.n);
        const gapa_config& g = cfgs[i];
        // batched runs implement the default generation (one elite, tournaments) and the row-wise flag
        if (g.k < 0 || g.k >= c->g.n || g.pop < 2 || g.tourn < 1 || g.elite != 1 || (g.flags & ~GAPA_FLAG_ROWWISE))
            return gapa_fail(GAPA_ERR_INVALID_ARG, "instance %d: invalid configuration", i);
    }
    cudaSetDevice(ctxs[0]->device);
    gapa_batch* b = new gapa_batch();
    b->device = ctxs[0]->device;
    b->num = num;
    b->ctxs.assign(ctxs, ctxs + num);
    b->cfgs.assign(cfgs, cfgs + num);
    b->stream = ctxs[0]->stream;
    b->status = ctxs[0]->status;
    auto bail = [&](int rc) {
        gapa_batch_destroy(b);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "stream/event creation failed"));
    int rc = gapa_ga_batched_init(ctxs[0]->smem_optin, &b->ga_max_dyn);
    if (rc == GAPA_OK) rc = gapa_fitness_batched_init(ctxs[0]->smem_optin, &b->fit_max_dyn);
    if (rc != GAPA_OK) return bail(rc);
    // buffers: two populations and two fitness arrays per instance
    size_t elems = 0;
    for (int i = 0; i < num; ++i) {
        b->pop_off.push_back(elems);
        elems += 2 * (size_t)cfgs[i].pop * cfgs[i].k;
        b->row_smem = std::max(b->row_smem, gapa_row_smem_bytes(ctxs[i]->g.n, cfgs[i].k));
        b->total_rows += cfgs[i].pop;
    }
    if (b->row_smem > b->ga_max_dyn) return bail(gapa_fail(GAPA_ERR_INVALID_ARG, "operator rows need too much shared memory"));
    size_t fit_off = (elems * sizeof(int32_t) + 255) & ~(size_t)255;
    size_t fit_elems = 0;
    for (int i = 0; i < num; ++i) fit_elems += 2 * (size_t)cfgs[i].pop;
    if (cudaMalloc(&b->d_buf, fit_off + fit_elems * sizeof(int64_t) + 256) != cudaSuccess ||
        cudaMalloc(&b->d_desc, sizeof(BatchDesc) * num) != cudaSuccess ||
        cudaMalloc(&b->d_rows, sizeof(int2) * b->total_rows) != cudaSuccess ||
        cudaMalloc(&b->d_head, sizeof(int)) != cudaSuccess || cudaMalloc(&b->d_gen, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_best, sizeof(int) * num) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_OOM, "batch buffers"));
    std::vector<int2> rows;
    rows.reserve(b->total_rows);
    int32_t* pops = (int32_t*)b->d_buf;
    int64_t* fits = (int64_t*)((char*)b->d_buf + fit_off);
    size_t fo = 0;
    b->desc.resize(num);
    b->teams.resize(num);
    b->use_local.assign(num, 0);
    for (int i = 0; i < num; ++i) {
        const gapa_config& g = cfgs[i];
        const DeviceGraph& dg = ctxs[i]->g;
        BatchDesc& d = b->desc[i];
        d = BatchDesc{};
        d.p.n = dg.n;
        d.p.k = g.k;
        d.p.s = g.pop;
        d.p.t = g.tourn;
        d.p.pc_thr = g.pc_thr;
        d.p.pm_thr = g.pm_thr;
        d.p.key = RngKey{(uint32_t)g.seed, (uint32_t)(g.seed >> 32)};
        d.p.flags = g.flags;
        d.p.g = 0;
        d.p.g_ptr = nullptr;
        d.pop[0] = pops + b->pop_off[i];
        d.pop[1] = d.pop[0] + (size_t)g.pop * g.k;
        d.fit[0] = fits + fo;
        d.fit[1] = d.fit[0] + g.pop;
        fo += 2 * (size_t)g.pop;
        d.best = b->d_best + i;
        d.n = dg.n;
        d.perm = dg.perm;
        d.palt = dg.palt;
        d.lo_ptr = dg.lo_ptr;
        d.lo_col = dg.lo_col;
        d.nontree = (const unsigned*)dg.nontree;
        d.num_nontree = dg.num_nontree;
        d.fptr = dg.fptr;
        d.fcol16 = dg.fcol16;
        d.mean_deg_x16 = dg.mean_deg_x16;
        d.objective = b->ctxs[i]->objective;
        const int variant = b->ctxs[i]->fitness_variant;
        if (dg.local_list_bytes > 0 && (variant == GAPA_FITNESS_TREE_LOCAL ||
                                        (variant == GAPA_FITNESS_AUTO && dg.n > 2048))) {
            // the cut-local kernel as on a single context: the operator kernels write every row's
            // estimates under both forests, members estimated to shatter both run the full pipeline
            b->use_local[i] = 1;
            d.alt = dg.alt;
            d.tparent = dg.tparent;
            d.kids = dg.kids;
            d.roots = dg.roots;
            d.num_roots = dg.num_roots;
        }
        b->teams[i] = default_teams(dg.n, b->fit_max_dyn);
        for (int r = 0; r < g.pop; ++r) rows.push_back(make_int2(i, r));
    }
    // cost estimates of the cut-local instances' rows: two per row (first forest, second forest)
    size_t est_total = 0;
    for (int i = 0; i < num; ++i)
        if (b->use_local[i]) est_total += 2 * (size_t)cfgs[i].pop;
    if (est_total) {
        if (cudaMalloc(&b->d_est, sizeof(unsigned) * est_total) != cudaSuccess) {
            cudaGetLastError();
            return bail(gapa_fail(GAPA_ERR_OOM, "batch cost estimates"));
        }
        size_t eo = 0;
        for (int i = 0; i < num; ++i) {
            if (!b->use_local[i]) continue;
            BatchDesc& d = b->desc[i];
            const DeviceGraph& dg = ctxs[i]->g;
            d.p.est_cut = dg.cut;
            d.p.est_cut2 = dg.has_alt ? dg.alt.cut : nullptr;
            d.p.est_out = b->d_est + eo;
            d.p.est_stride = cfgs[i].pop;
            eo += 2 * (size_t)cfgs[i].pop;
        }
    }
    if (cudaMemcpy(b->d_rows, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "uploading the row table"));
    rc = build_packets(b);
    if (rc == GAPA_OK) rc = upload_desc(b);
    if (rc != GAPA_OK) return bail(rc);
    *out = b;
    return GAPA_OK;
}

void gapa_batch_destroy(gapa_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->own) cudaStreamSynchronize(b->own);
    free_batch_device(b);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
}

int gapa_batch_set_teams(gapa_batch* b, const int32_t* teams) {
    if (!b || !teams) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    cudaSetDevice(b->device);
    for (int i = 0; i < b->num; ++i) {
        const int c = teams[i];
        if (c != 1 && c != 2 && c != 4 && c != 8) return gapa_fail(GAPA_ERR_INVALID_ARG, "teams must be 1, 2, 4 or 8");
        if ((size_t)c * need16(b->ctxs[i]->g.n) + 16 * c > b->fit_max_dyn)
            return gapa_fail(GAPA_ERR_INVALID_ARG, "instance %d: %d teams do not fit in shared memory", i, c);
    }
    b->teams.assign(teams, teams + b->num);
    int rc = build_packets(b);
    return rc == GAPA_OK ? upload_desc(b) : rc;
}

int gapa_batch_get_teams(gapa_batch* b, int32_t* teams) {
    if (!b || !teams) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < b->num; ++i) teams[i] = b->teams[i];
    return GAPA_OK;
}

int gapa_batch_autotune(gapa_batch* b, const char* cache_path) {
    if (!b) return gapa_fail(GAPA_ERR_INVALID_ARG, "batch is NULL");
    cudaSetDevice(b->device);
    const std::string dev = device_name(b->device);
    auto cache = cache_path ? read_cache(cache_path) : std::map<std::string, std::map<int, int>>();
    std::vector<int> present(6, 0);
    for (int i = 0; i < b->num; ++i) present[bucket_of(b->ctxs[i]->g.n)] = 1;
    std::vector<int> choice(6, 0);
    bool all_cached = true;
    for (int k = 0; k < 6; ++k)
        if (present[k]) {
            auto it = cache.find(dev);
            if (it != cache.end() && it->second.count(k)) choice[k] = it->second.at(k);
            else all_cached = false;
        }
    cudaStream_t st = b->own;
    if (!all_cached) {
        // a starting population to time on
        int rc = enqueue_start(b, st);
        if (rc != GAPA_OK) return rc;
        GAPA_CUDA(cudaStreamSynchronize(st));
        cudaEvent_t e0, e1;
        GAPA_CUDA(cudaEventCreate(&e0));
        GAPA_CUDA(cudaEventCreate(&e1));
        const std::vector<int> saved = b->teams;
        for (int k = 0; k < 6; ++k) {
            if (!present[k] || choice[k]) continue;
            float best_ms = 1e30f;
            int best_c = 1;
            for (int c = 1; c <= 8; c *= 2) {
                // only this bucket's instances are timed: the others get no packets
                bool ok = true;
                for (int i = 0; i < b->num; ++i)
                    if (bucket_of(b->ctxs[i]->g.n) == k &&
                        ((size_t)c * need16(b->ctxs[i]->g.n) + 16 * c > b->fit_max_dyn || 1024 / c < 128))
                        ok = false;
                if (!ok) break;
                for (int i = 0; i < b->num; ++i) b->teams[i] = bucket_of(b->ctxs[i]->g.n) == k ? c : saved[i];
                rc = build_packets(b);
                if (rc != GAPA_OK) break;
                // packets of this bucket only
                std::vector<BatchPacket> hp(b->npk_all);
                GAPA_CUDA(cudaMemcpy(hp.data(), b->d_pk, sizeof(BatchPacket) * b->npk_all, cudaMemcpyDeviceToHost));
                std::vector<BatchPacket> sel;
                for (auto& p : hp)
                    if (bucket_of(b->ctxs[p.b]->g.n) == k) sel.push_back(p);
                GAPA_CUDA(cudaMemcpy(b->d_pk, sel.data(), sizeof(BatchPacket) * sel.size(), cudaMemcpyHostToDevice));
                rc = upload_desc(b);
                if (rc != GAPA_OK) break;
                float ms_min = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    GAPA_CUDA(cudaEventRecord(e0, st));
                    rc = gapa_launch_fitness_batched(b->d_desc, b->d_pk, (int)sel.size(), b->d_head, 0, b->fit_smem,
                                                     b->fit_grid, b->status, st);
                    GAPA_CUDA(cudaEventRecord(e1, st));
                    GAPA_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    GAPA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    ms_min = std::min(ms_min, ms);
                }
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best_c = c;
                }
            }
            if (rc != GAPA_OK) break;
            choice[k] = best_c;
            cache[dev][k] = best_c;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != GAPA_OK) return rc;
        if (cache_path) write_cache(cache_path, cache);
    }
    for (int i = 0; i < b->num; ++i) b->teams[i] = choice[bucket_of(b->ctxs[i]->g.n)];
    int rc = build_packets(b);
    return rc == GAPA_OK ? upload_desc(b) : rc;
}

int gapa_batch_run(gapa_batch* b, int32_t gens, int64_t* best_fit, int32_t* best_sets, int64_t* traj) {
    if (!b || gens < 0 || !best_fit) return gapa_fail(GAPA_ERR_INVALID_ARG, "bad batch run arguments");
    cudaSetDevice(b->device);
    const size_t cap = (size_t)gens + 1;
    if (cap > b->traj_cap) {
        cudaFree(b->d_traj);
        b->d_traj = nullptr;
        b->traj_cap = 0;
        if (cudaMalloc(&b->d_traj, sizeof(int64_t) * cap * b->num) != cudaSuccess)
            return gapa_fail(GAPA_ERR_OOM, "batch trajectories");
        b->traj_cap = cap;
    }
    for (int i = 0; i < b->num; ++i) b->desc[i].traj = b->d_traj + (size_t)i * b->traj_cap;
    int rc = upload_desc(b);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = b->own;
    GAPA_CUDA(cudaEventRecord(b->ev_a, b->stream));
    GAPA_CUDA(cudaStreamWaitEvent(st, b->ev_a, 0));
    rc = enqueue_start(b, st);
    if (rc != GAPA_OK) return rc;
    if (gens >= 2) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        GAPA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int crc = enqueue_generation(b, 0, st);
        if (crc == GAPA_OK) crc = enqueue_generation(b, 1, st);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (crc != GAPA_OK) {
            if (graph) cudaGraphDestroy(graph);
            return crc;
        }
        GAPA_CUDA(ce);
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        GAPA_CUDA(ce);
        for (int r = 0; r < gens / 2 && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(exec, st);
        cudaGraphExecDestroy(exec);
        GAPA_CUDA(ce);
    }
    if (gens % 2 == 1) {
        rc = enqueue_generation(b, 0, st);
        if (rc != GAPA_OK) return rc;
    }
    const int fin = gens % 2;
    std::vector<int> best(b->num);
    GAPA_CUDA(cudaMemcpyAsync(best.data(), b->d_best, sizeof(int) * b->num, cudaMemcpyDeviceToHost, st));
    GAPA_CUDA(cudaStreamSynchronize(st));
    int h = 0;
    GAPA_CUDA(cudaMemcpy(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(b->status, 0, sizeof(int));
        return gapa_fail(h & GAPA_DEV_TIMEOUT ? GAPA_ERR_TIMEOUT : GAPA_ERR_DEVICE, "device status 0x%x", h);
    }
    size_t off = 0;
    for (int i = 0; i < b->num; ++i) {
        const BatchDesc& d = b->desc[i];
        GAPA_CUDA(cudaMemcpyAsync(best_fit + i, d.fit[fin] + best[i], sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (best_sets && d.p.k)
            GAPA_CUDA(cudaMemcpyAsync(best_sets + off, d.pop[fin] + (size_t)best[i] * d.p.k, sizeof(int32_t) * d.p.k,
                                      cudaMemcpyDeviceToHost, st));
        if (traj)
            GAPA_CUDA(cudaMemcpyAsync(traj + (size_t)i * cap, d.traj, sizeof(int64_t) * cap, cudaMemcpyDeviceToHost, st));
        off += d.p.k;
    }
    GAPA_CUDA(cudaStreamSynchronize(st));
    if (best_sets) {
        off = 0;
        for (int i = 0; i < b->num; ++i) {
            std::sort(best_sets + off, best_sets + off + b->desc[i].p.k);
            off += b->desc[i].p.k;
        }
    }
    GAPA_CUDA(cudaEventRecord(b->ev_b, st));
    GAPA_CUDA(cudaStreamWaitEvent(b->stream, b->ev_b, 0));
    return GAPA_OK;
}

}  // extern "C"
