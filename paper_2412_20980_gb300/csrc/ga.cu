// Genetic operators on the GPU (Section III-B, Eqs. 2-11, Fig. 1).
//
// One CTA builds one population row.  The kept-gene set of the row is a
// bitmap of n bits in shared memory; the per-position crossover/mutation
// flags (k bytes) and the list of open positions (k ints) sit beside it.
// Random numbers: Philox4x32-10 at counter (j, i, g, tag << 24 | round).
//
// Readings where the paper is silent (the same ones the CPU oracle follows):
//  - selection: tournament of size t with replacement, lower fitness wins,
//    ties to the lower index (Eq. 5 uses roulette);
//  - elitism: one elite, the lowest fitness (lowest index on ties), copied to
//    row 0 with its fitness;
//  - a gene from B that repeats a kept gene from A becomes an open position
//    whose first candidate is A[j]; a mutated position is open with first
//    candidate uniform over [0, n);
//  - repair: rounds r = 0..31; in ascending position order each open
//    position takes its round-r candidate if that node is not kept yet (and
//    keeps it at once); round r >= 1 candidates are uniform over [0, n) from
//    tag REPAIR, round r; positions still open after round 31 take the
//    smallest free ids in ascending position order.
#include <climits>

#include "gapa_internal.cuh"

namespace {

constexpr int kGaBlock = 256;

__device__ __forceinline__ bool bit_test(const unsigned* bm, int v) { return (bm[v >> 5] >> (v & 31)) & 1u; }
__device__ __forceinline__ void bit_set(unsigned* bm, int v) { atomicOr(&bm[v >> 5], 1u << (v & 31)); }

// Row layout in dynamic shared memory: kept bitmap | flags (k bytes) | holes (k ints)
struct RowSmem {
    unsigned* kept;
    unsigned char* flags;
    int* holes;
};

__device__ __forceinline__ RowSmem carve(unsigned char* base, int n, int k) {
    RowSmem r;
    const int words = (n + 31) >> 5;
    r.kept = reinterpret_cast<unsigned*>(base);
    r.flags = base + (size_t)words * 4;
    const size_t off = ((size_t)words * 4 + (size_t)k + 15) & ~(size_t)15;
    r.holes = reinterpret_cast<int*>(base + off);
    return r;
}

size_t row_smem_bytes(int n, int k) {
    const size_t words = ((size_t)n + 31) >> 5;
    return ((words * 4 + (size_t)k + 15) & ~(size_t)15) + (size_t)k * 4;
}

enum FlagBits : unsigned char { F_XOVER = 1, F_MUT = 2, F_HOLE = 4 };

// Round-0 candidate of an open position.
struct InitCand {
    RngKey key;
    int i, n;
    __device__ int operator()(int j) const { return uniform_below(gapa_draw(key, j, i, 0, TAG_INIT, 0), n); }
};

struct ChildCand {
    RngKey key;
    int i, g, n;
    const unsigned char* flags;
    const int* A;
    int* status;
    __device__ int operator()(int j) const {
        if (flags[j] & F_MUT) return uniform_below(gapa_draw(key, j, i, g, TAG_MUTVAL, 0), n);
        const int a = A[j];
        if ((unsigned)a >= (unsigned)n) {
            atomicOr(status, GAPA_DEV_BAD_GENE);
            return -1;
        }
        return a;
    }
};

// Repair by warp 0 of the CTA: holes[0..nholes) ascending positions of `row`.
template <class Cand>
__device__ void repair_warp(unsigned* kept, int* holes, int nholes, int* row, const Cand& cand0, RngKey key,
                            int i, int g, int n) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kRepairRounds && nholes > 0; ++r) {
        int out = 0;
        for (int base = 0; base < nholes; base += 32) {
            const int idx = base + lane;
            const bool active = idx < nholes;
            const int j = active ? holes[idx] : -1;
            int c = -1;
            if (active) c = r == 0 ? cand0(j) : uniform_below(gapa_draw(key, j, i, g, TAG_REPAIR, r), n);
            const bool valid = active && c >= 0;
            const bool taken = valid && bit_test(kept, c);
            const unsigned peers = __match_any_sync(0xffffffffu, c);
            const bool first = lane == __ffs(peers) - 1;
            const bool accept = valid && !taken && first;
            if (accept) {
                bit_set(kept, c);
                row[j] = c;
            }
            const bool reject = active && !accept;
            const unsigned rej = __ballot_sync(0xffffffffu, reject);
            if (reject) holes[out + __popc(rej & lt_mask)] = j;
            out += __popc(rej);
            __syncwarp();
        }
        nholes = out;
    }
    if (nholes > 0 && lane == 0) {
        int next = 0;
        for (int h = 0; h < nholes; ++h) {
            while (bit_test(kept, next)) ++next;
            bit_set(kept, next);
            row[holes[h]] = next;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void clear_bitmap(unsigned* kept, int n) {
    const int words = (n + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) kept[w] = 0u;
}

// Cost estimates of a finished row for the cut-local fitness kernel, under
// the first and (if any) the second forest (whole CTA; the row was written by
// this CTA before the barrier inside).
__device__ void row_estimate(const GaParams& p, const int* row, int i) {
    __shared__ long long part[2][kGaBlock / 32];
    __syncthreads();
    long long c = 0, c2 = 0;
    const int T = blockDim.x;
    int j = threadIdx.x;
    // four genes per step, both forests' gathers in flight together
    for (; j + 3 * T < p.k; j += 4 * T) {
        int d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = row[j + u * T];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = (unsigned)d[u] < (unsigned)p.n;
            c += ok ? __ldg(&p.est_cut[d[u]]) : 0;
            c2 += ok && p.est_cut2 ? __ldg(&p.est_cut2[d[u]]) : 0;
        }
    }
    for (; j < p.k; j += T) {
        const int d = row[j];
        if ((unsigned)d < (unsigned)p.n) {
            c += __ldg(&p.est_cut[d]);
            if (p.est_cut2) c2 += __ldg(&p.est_cut2[d]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        c2 += __shfl_down_sync(0xffffffffu, c2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = c;
        part[1][threadIdx.x >> 5] = c2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += part[0][w];
            t2 += part[1][w];
        }
        p.est_out[i] = (unsigned)(t < 0x7FFFFFFFll ? t : 0x7FFFFFFFll);
        p.est_out[p.est_stride + i] = p.est_cut2 ? (unsigned)(t2 < 0x7FFFFFFFll ? t2 : 0x7FFFFFFFll) : 0xFFFFFFFFu;
    }
}

// Population initialisation (Eq. 2) of row i: every position open, candidates from tag INIT.
__device__ void init_row(const GaParams& p, int i, int* __restrict__ pop) {
    extern __shared__ __align__(16) unsigned char smem[];
    RowSmem sm = carve(smem, p.n, p.k);
    clear_bitmap(sm.kept, p.n);
    for (int j = threadIdx.x; j < p.k; j += blockDim.x) sm.holes[j] = j;
    __syncthreads();
    if (threadIdx.x < 32) {
        InitCand cand{p.key, i, p.n};
        repair_warp(sm.kept, sm.holes, p.k, pop + (size_t)i * p.k, cand, p.key, i, 0, p.n);
    }
    if (p.est_out) row_estimate(p, pop + (size_t)i * p.k, i);
}

__global__ void __launch_bounds__(kGaBlock) init_kernel(GaParams p, int* __restrict__ pop) { init_row(p, blockIdx.x, pop); }

// Tournament of size t for parent slot `slot` of child i.
__device__ int tournament(const GaParams& p, int i, int g, int slot, const long long* fit) {
    int best = -1;
    long long bf = 0;
    for (int r = 0; r < p.t; ++r) {
        const int x = uniform_below(gapa_draw(p.key, slot * p.t + r, i, g, TAG_SEL, 0), p.s);
        const long long fx = fit[x];
        if (best < 0 || fx < bf || (fx == bf && x < best)) {
            best = x;
            bf = fx;
        }
    }
    return best;
}

// Roulette-wheel draw (Eq. 5) for parent slot `slot` of child i: the first
// member whose cumulative weight exceeds floor(u * W / 2^64).
__device__ int roulette(const GaParams& p, int i, int g, int slot) {
    const unsigned long long u =
        philox_word01((uint32_t)slot, (uint32_t)i, (uint32_t)g, (uint32_t)TAG_ROULETTE << 24, p.key.lo, p.key.hi);
    const unsigned long long W = (unsigned long long)p.cum[p.s - 1];
    const unsigned long long r = __umul64hi(u, W);
    int lo = 0, hi = p.s - 1;  // smallest x with cum[x] > r
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)p.cum[mid] > r)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ int select_parent(const GaParams& p, int i, int g, int slot, const long long* fit) {
    return (p.flags & GAPA_FLAG_ROULETTE) ? roulette(p, i, g, slot) : tournament(p, i, g, slot, fit);
}

// Block argmin of fit[0..s) (lowest value, lowest index); result valid in all threads.
__device__ void block_argmin(const long long* __restrict__ fit, int s, long long* out_val, int* out_idx) {
    __shared__ long long sv[32];
    __shared__ int si[32];
    long long bv = LLONG_MAX;
    int bi = INT_MAX;
    for (int x = threadIdx.x; x < s; x += blockDim.x) {
        const long long v = fit[x];
        if (v < bv || (v == bv && x < bi)) {
            bv = v;
            bi = x;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[warp] = bv;
        si[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        bv = lane < nw ? sv[lane] : LLONG_MAX;
        bi = lane < nw ? si[lane] : INT_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            sv[0] = bv;
            si[0] = bi;
        }
    }
    __syncthreads();
    *out_val = sv[0];
    *out_idx = si[0];
}

// Row i of one generation g: with an elite, row 0 = elite copy and row i >= 1
// = child i; without (the (mu+lambda) children), row i = child with counter i.
__device__ void offspring_row(const GaParams& p, int i, int g, const int* __restrict__ pop_in,
                              const long long* __restrict__ fit_in, int* __restrict__ pop_out,
                              long long* __restrict__ fit_out, int* status, bool has_elite = true) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sh_parent[2];
    __shared__ int sh_warp_cnt[kGaBlock / 32];
    const int n = p.n, k = p.k;
    if (has_elite && i == 0) {
        long long v;
        int e;
        block_argmin(fit_in, p.s, &v, &e);
        const int* src = pop_in + (size_t)e * k;
        for (int j = threadIdx.x; j < k; j += blockDim.x) pop_out[j] = src[j];
        if (threadIdx.x == 0) fit_out[0] = v;
        if (p.est_out) row_estimate(p, pop_out, 0);
        return;
    }
    RowSmem sm = carve(smem, n, k);
    if (threadIdx.x == 0) {
        sh_parent[0] = (p.flags & GAPA_FLAG_ROWWISE) ? i : select_parent(p, i, g, 0, fit_in);
        sh_parent[1] = select_parent(p, i, g, 1, fit_in);
    }
    clear_bitmap(sm.kept, n);
    __syncthreads();
    const int* A = pop_in + (size_t)sh_parent[0] * k;
    const int* B = pop_in + (size_t)sh_parent[1] * k;
    int* C = pop_out + (size_t)i * k;
    // crossover and mutation masks (Eqs. 3-4, 7-8); genes kept from A
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const bool xo = gapa_draw(p.key, j, i, g, TAG_XOVER, 0) < p.pc_thr;
        const bool mu = gapa_draw(p.key, j, i, g, TAG_MUT, 0) < p.pm_thr;
        unsigned char f = (xo ? F_XOVER : 0) | (mu ? F_MUT : 0);
        if (!mu && !xo) {
            const int a = A[j];
            if ((unsigned)a < (unsigned)n) {
                C[j] = a;
                bit_set(sm.kept, a);
            } else {
                atomicOr(status, GAPA_DEV_BAD_GENE);
                f |= F_HOLE;
            }
        }
        if (mu) f |= F_HOLE;
        sm.flags[j] = f;
    }
    __syncthreads();
    // genes from B (Eq. 6); a repeat of a kept A gene opens the position
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const unsigned char f = sm.flags[j];
        if (f == F_XOVER) {
            const int b = B[j];
            if ((unsigned)b >= (unsigned)n) {
                atomicOr(status, GAPA_DEV_BAD_GENE);
                sm.flags[j] = f | F_HOLE;
            } else if (bit_test(sm.kept, b)) {
                sm.flags[j] = f | F_HOLE;
            } else {
                C[j] = b;
                bit_set(sm.kept, b);
            }
        }
    }
    __syncthreads();
    // open positions in ascending order: contiguous ranges per thread + block scan
    const int T = blockDim.x, tid = threadIdx.x;
    const int per = (k + T - 1) / T;
    const int j0 = min(k, tid * per), j1 = min(k, j0 + per);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) cnt += (sm.flags[j] & F_HOLE) ? 1 : 0;
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh_warp_cnt[warp] = incl;
    __syncthreads();
    int warp_off = 0, total = 0;
    for (int w = 0; w < (T >> 5); ++w) {
        if (w < warp) warp_off += sh_warp_cnt[w];
        total += sh_warp_cnt[w];
    }
    int pos = warp_off + incl - cnt;
    for (int j = j0; j < j1; ++j)
        if (sm.flags[j] & F_HOLE) sm.holes[pos++] = j;
    __syncthreads();
    if (warp == 0) {
        ChildCand cand{p.key, i, g, n, sm.flags, A, status};
        repair_warp(sm.kept, sm.holes, total, C, cand, p.key, i, g, n);
    }
    if (p.est_out) row_estimate(p, C, i);
}

__global__ void __launch_bounds__(kGaBlock) offspring_kernel(GaParams p, const int* __restrict__ pop_in,
                                                             const long long* __restrict__ fit_in,
                                                             int* __restrict__ pop_out,
                                                             long long* __restrict__ fit_out, int* status) {
    offspring_row(p, blockIdx.x, p.g_ptr ? *p.g_ptr : p.g, pop_in, fit_in, pop_out, fit_out, status);
}

// (mu+lambda) children: row i = child with counter index i, parents among the s members.
__global__ void __launch_bounds__(kGaBlock) children_kernel(GaParams p, const int* __restrict__ pop_in,
                                                            const long long* __restrict__ fit_in,
                                                            int* __restrict__ kids, int* status) {
    offspring_row(p, blockIdx.x, p.g_ptr ? *p.g_ptr : p.g, pop_in, fit_in, kids, nullptr, status, false);
}

// Roulette weights w_x = (max F - F_x) + 1 and their int64 inclusive prefix sums (one CTA).
__global__ void __launch_bounds__(1024) roulette_prefix_kernel(const long long* __restrict__ fit, int s,
                                                               long long* __restrict__ cum) {
    __shared__ long long sh[32];
    __shared__ long long carry;
    long long mx = LLONG_MIN;
    for (int x = threadIdx.x; x < s; x += blockDim.x) mx = fit[x] > mx ? fit[x] : mx;
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_down_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long m = sh[0];
        for (int w = 1; w < nw; ++w) m = sh[w] > m ? sh[w] : m;
        sh[0] = m;
        carry = 0;
    }
    __syncthreads();
    const long long fmax = sh[0];
    __syncthreads();
    for (int base = 0; base < s; base += blockDim.x) {
        const int x = base + threadIdx.x;
        long long v = x < s ? (fmax - fit[x]) + 1 : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) sh[warp] = v;
        __syncthreads();
        long long off = carry;
        for (int w = 0; w < warp; ++w) off += sh[w];
        if (x < s) cum[x] = v + off;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = v + off;
        __syncthreads();
    }
}

// (mu+lambda) truncation (Eqs. 10-11): bitonic sort of (fitness, index) over
// members (index x) and children (index mu + c); the first mu give the source
// rows (src) and the new fitness.  One CTA, keys in shared memory.
__global__ void __launch_bounds__(1024) mpl_sort_kernel(int mu, int lambda, const long long* __restrict__ fit_in,
                                                        const long long* __restrict__ kfit, int* __restrict__ src,
                                                        long long* __restrict__ fit_out, int P) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long* key = reinterpret_cast<long long*>(smem);
    int* idx = reinterpret_cast<int*>(key + P);
    const int tot = mu + lambda;
    for (int x = threadIdx.x; x < P; x += blockDim.x) {
        key[x] = x < mu ? fit_in[x] : (x < tot ? kfit[x - mu] : LLONG_MAX);
        idx[x] = x < tot ? x : INT_MAX;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = threadIdx.x; x < P; x += blockDim.x) {
                const int y = x ^ stride;
                if (y > x) {
                    const bool up = (x & size) == 0;
                    const bool gt = key[x] > key[y] || (key[x] == key[y] && idx[x] > idx[y]);
                    if (gt == up) {
                        const long long tk = key[x];
                        key[x] = key[y];
                        key[y] = tk;
                        const int ti = idx[x];
                        idx[x] = idx[y];
                        idx[y] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < mu; r += blockDim.x) {
        src[r] = idx[r];
        fit_out[r] = key[r];
    }
}

// Next population rows from members (src < mu) or children.
__global__ void __launch_bounds__(kGaBlock) mpl_gather_kernel(int mu, int k, const int* __restrict__ pop_in,
                                                              const int* __restrict__ kids, const int* __restrict__ src,
                                                              int* __restrict__ pop_out) {
    const int r = blockIdx.x, x = src[r];
    const int* from = x < mu ? pop_in + (size_t)x * k : kids + (size_t)(x - mu) * k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) pop_out[(size_t)r * k + j] = from[j];
}

// ---------------------------------------------------------------------------
// Batched instances: one launch covers the rows of every instance; rows[r] =
// (instance, row) and each instance has its own parameters and buffers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGaBlock) init_batched_kernel(const BatchDesc* __restrict__ d,
                                                                const int2* __restrict__ rows, int buf) {
    const int2 r = rows[blockIdx.x];
    const BatchDesc& bd = d[r.x];
    init_row(bd.p, r.y, bd.pop[buf]);
}

__global__ void __launch_bounds__(kGaBlock) offspring_batched_kernel(const BatchDesc* __restrict__ d,
                                                                     const int2* __restrict__ rows, int src,
                                                                     const int* gen, int* status) {
    const int2 r = rows[blockIdx.x];
    const BatchDesc& bd = d[r.x];
    offspring_row(bd.p, r.y, *gen, bd.pop[src], reinterpret_cast<const long long*>(bd.fit[src]), bd.pop[src ^ 1],
                  reinterpret_cast<long long*>(bd.fit[src ^ 1]), status);
}

// Per instance: trajectory[gen] = lowest fitness, best = its index.
__global__ void __launch_bounds__(1024) record_batched_kernel(const BatchDesc* __restrict__ d, int buf,
                                                              const int* gen) {
    const BatchDesc& bd = d[blockIdx.x];
    long long v;
    int e;
    block_argmin(reinterpret_cast<const long long*>(bd.fit[buf]), bd.p.s, &v, &e);
    if (threadIdx.x == 0) {
        if (bd.traj) bd.traj[*gen] = v;
        *bd.best = e;
    }
}

__global__ void advance_kernel(int* gen) { *gen += 1; }

// Lowest fitness of a population: traj[*gen] = min, *best = argmin, then ++*gen.
__global__ void __launch_bounds__(1024) record_kernel(const long long* __restrict__ fit, int s, int* gen,
                                                      long long* traj, int* best) {
    long long v;
    int e;
    block_argmin(fit, s, &v, &e);
    if (threadIdx.x == 0) {
        const int gg = *gen;
        if (traj) traj[gg] = v;
        *best = e;
        *gen = gg + 1;
    }
}

}  // namespace

int gapa_ga_check_limits(gapa_ctx* c, int n, int k, int s) {
    const size_t need = row_smem_bytes(n, k);
    if (need > c->ga_smem_max)
        return gapa_fail(GAPA_ERR_INVALID_ARG,
                         "genetic operators need n/8 + 5k bytes of shared memory per row (n=%d, k=%d: %zu > %zu)",
                         n, k, need, c->ga_smem_max);
    if ((long long)s * (long long)k >= (1LL << 31))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "s*k must be below 2^31");
    return GAPA_OK;
}

int gapa_launch_init(gapa_ctx* c, const GaParams& p, int32_t* pop, cudaStream_t st) {
    if (p.s <= 0) return GAPA_OK;
    ProfileScope prof(c, st, 1, 0);
    init_kernel<<<p.s, kGaBlock, row_smem_bytes(p.n, p.k), st>>>(p, pop);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_offspring(gapa_ctx* c, const GaParams& p, const int32_t* pop_in, const int64_t* fit_in,
                          int32_t* pop_out, int64_t* fit_out, cudaStream_t st) {
    ProfileScope prof(c, st, 1, 0);
    offspring_kernel<<<p.s, kGaBlock, row_smem_bytes(p.n, p.k), st>>>(
        p, pop_in, reinterpret_cast<const long long*>(fit_in), pop_out, reinterpret_cast<long long*>(fit_out),
        c->status);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_record(gapa_ctx* c, const int64_t* fit, int s, int* gen, int64_t* traj, int* best,
                       cudaStream_t st) {
    ProfileScope prof(c, st, 1, 1);
    record_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const long long*>(fit), s, gen,
                                      reinterpret_cast<long long*>(traj), best);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_init_batched(const BatchDesc* d, const int2* rows, int total_rows, size_t smem, int buf,
                             cudaStream_t st) {
    init_batched_kernel<<<total_rows, kGaBlock, smem, st>>>(d, rows, buf);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_offspring_batched(const BatchDesc* d, const int2* rows, int total_rows, size_t smem, int src,
                                  const int* gen, int* status, cudaStream_t st) {
    offspring_batched_kernel<<<total_rows, kGaBlock, smem, st>>>(d, rows, src, gen, status);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_record_batched(const BatchDesc* d, int num, int buf, int* gen, bool advance, cudaStream_t st) {
    record_batched_kernel<<<num, 1024, 0, st>>>(d, buf, gen);
    if (advance) advance_kernel<<<1, 1, 0, st>>>(gen);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

size_t gapa_row_smem_bytes(int n, int k) { return row_smem_bytes(n, k); }

int gapa_ga_batched_init(size_t optin, size_t* max_dyn) {
    int rc = gapa_set_smem_limit((const void*)init_batched_kernel, optin, max_dyn);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)offspring_batched_kernel, optin, max_dyn);
    return rc;
}

int gapa_launch_roulette_prefix(const int64_t* fit, int s, int64_t* cum, cudaStream_t st) {
    roulette_prefix_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const long long*>(fit), s,
                                               reinterpret_cast<long long*>(cum));
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_children(gapa_ctx* c, const GaParams& p, int lambda, const int32_t* pop_in, const int64_t* fit_in,
                         int32_t* kids, cudaStream_t st) {
    ProfileScope prof(c, st, 1, 0);
    children_kernel<<<lambda, kGaBlock, row_smem_bytes(p.n, p.k), st>>>(p, pop_in,
                                                                       reinterpret_cast<const long long*>(fit_in),
                                                                       kids, c->status);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_launch_mpl_replace(gapa_ctx* c, int mu, int lambda, int k, const int32_t* pop_in, const int64_t* fit_in,
                            const int32_t* kids, const int64_t* kfit, int* src, int32_t* pop_out, int64_t* fit_out,
                            cudaStream_t st) {
    int P = 1;
    while (P < mu + lambda) P <<= 1;
    const size_t smem = (size_t)P * (sizeof(long long) + sizeof(int));
    if (smem > c->sort_smem_max) return gapa_fail(GAPA_ERR_INVALID_ARG, "mu + lambda = %d is too large", mu + lambda);
    ProfileScope prof(c, st, 1, k > 0 ? 2 : 1);
    mpl_sort_kernel<<<1, 1024, smem, st>>>(mu, lambda, reinterpret_cast<const long long*>(fit_in),
                                           reinterpret_cast<const long long*>(kfit), src,
                                           reinterpret_cast<long long*>(fit_out), P);
    if (k > 0) mpl_gather_kernel<<<mu, kGaBlock, 0, st>>>(mu, k, pop_in, kids, src, pop_out);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_ga_kernels_init(gapa_ctx* c) {
    int rc = gapa_set_smem_limit((const void*)init_kernel, c->smem_optin, &c->ga_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)offspring_kernel, c->smem_optin, &c->ga_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)children_kernel, c->smem_optin, &c->ga_smem_max);
    if (rc == GAPA_OK) rc = gapa_set_smem_limit((const void*)mpl_sort_kernel, c->smem_optin, &c->sort_smem_max);
    return rc;
}
