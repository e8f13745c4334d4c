// Learned fitness surrogate and the surrogate-screened (mu+lambda) GA.
//
// Not part of the paper: a small MLP scores every child of a generation so
// that only the most promising fraction receives the exact pairwise-
// connectivity fitness of Section III-C; exact fitness stays the arbiter of
// every member kept (Eqs. 10-11 truncation over members and evaluated
// children).  The model is trained online on the (deletion set, exact
// fitness) pairs the GA produces.
//
// Model (same definition as the fp64 reference):
//   x  = [ (1/sqrt k) sum_{v in D} Emb[v] (64) | mean, max, std of log1p(deg)
//          over D, sum deg / 2E | log1p(r0), log1p(r1), log1p(r2) | 0 x 9 ]  (80)
//   r0 / r1 = live neighbours of D left with no / exactly one live neighbour,
//   r2 = two-node components of G[V\D] adjacent to D
//   h1 = relu(x W1 + b1) (256), h2 = relu(h1 W2 + b2) (256), y = h2 . w3 + b3
//   target t = z-score of log1p(PC) over the replay ring; loss = mean (y-t)^2
//   AdamW on every parameter (FP32 masters and moments).
// Precision: the matrix products run on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation) with BF16 copies of the weights and
// activations; biases, the output layer and the optimiser are FP32.  All
// reductions run in a fixed order and the embedding gradient is accumulated
// in 2^-40 fixed point with integer atomics, so training is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <vector>

#include "gapa_internal.cuh"

namespace {

constexpr int kIn = 80, kHid = 256, kEmb = 64;
constexpr double kFix = 1099511627776.0;  // 2^40
using bf16 = __nv_bfloat16;

struct Layout {
    size_t W1, b1, W2, b2, w3, b3, E, total;
};

Layout make_layout(int n) {
    Layout L;
    size_t o = 0;
    L.W1 = o; o += (size_t)kIn * kHid;
    L.b1 = o; o += kHid;
    L.W2 = o; o += (size_t)kHid * kHid;
    L.b2 = o; o += kHid;
    L.w3 = o; o += kHid;
    L.b3 = o; o += 4;
    o = (o + 63) & ~(size_t)63;  // the table starts on a 256-byte boundary (vector accesses)
    L.E = o; o += (size_t)n * kEmb;
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned ld32(const bf16* p, size_t idx) {
    return *reinterpret_cast<const unsigned*>(p + idx);
}

// ---------------------------------------------------------------------------
// C[M][N] = A[M][K] * B^T, A row-major (lda), B stored as [N][K] (ldb): the
// tensor-core tile is mma.sync m16n8k16 (A row, B col, FP32 accumulate).
// One warp computes 16 rows x 16 columns; a CTA has 4 warps (64 x 16).  The
// operand fragments of four k-steps are loaded before their products so that
// the loads overlap.  M, K multiples of 16, N multiple of 8.  Epilogue:
// + bias[n], * (mask > 0), relu, then FP32 and/or BF16 and/or transposed
// BF16 stores.
// ---------------------------------------------------------------------------
struct GemmArgs {
    int M, N, K;
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    float* Cf;
    int ldc;
    bf16* Cb;
    int ldcb;
    bf16* CbT;
    int ldct;
    const float* bias;
    const bf16* mask;
    int ldm;
    int relu;
};

constexpr int kGemmRowsPerCta = 64, kGemmCols = 16, kGemmUnroll = 4;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int r0 = blockIdx.y * kGemmRowsPerCta + warp * 16;
    const int n_base = blockIdx.x * kGemmCols;
    if (r0 >= a.M) return;
    const bool has_n1 = n_base + 8 < a.N;
    float acc[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
    const bf16* A0 = a.A + (size_t)(r0 + g) * a.lda + tig * 2;
    const bf16* A1 = A0 + (size_t)8 * a.lda;
    const bf16* B0 = a.B + (size_t)(n_base + g) * a.ldb + tig * 2;
    const bf16* B1 = B0 + (size_t)8 * a.ldb;
    int k0 = 0;
    for (; k0 + 16 * kGemmUnroll <= a.K; k0 += 16 * kGemmUnroll) {
        unsigned af[kGemmUnroll][4], bf[kGemmUnroll][4];
#pragma unroll
        for (int u = 0; u < kGemmUnroll; ++u) {
            const int kk = k0 + 16 * u;
            af[u][0] = ld32(A0, kk);
            af[u][1] = ld32(A1, kk);
            af[u][2] = ld32(A0, kk + 8);
            af[u][3] = ld32(A1, kk + 8);
            bf[u][0] = ld32(B0, kk);
            bf[u][1] = ld32(B0, kk + 8);
            bf[u][2] = has_n1 ? ld32(B1, kk) : 0u;
            bf[u][3] = has_n1 ? ld32(B1, kk + 8) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kGemmUnroll; ++u) {
            mma_bf16(acc[0], af[u], bf[u][0], bf[u][1]);
            mma_bf16(acc[1], af[u], bf[u][2], bf[u][3]);
        }
    }
    for (; k0 < a.K; k0 += 16) {
        const unsigned af[4] = {ld32(A0, k0), ld32(A1, k0), ld32(A0, k0 + 8), ld32(A1, k0 + 8)};
        mma_bf16(acc[0], af, ld32(B0, k0), ld32(B0, k0 + 8));
        if (has_n1) mma_bf16(acc[1], af, ld32(B1, k0), ld32(B1, k0 + 8));
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int n0 = n_base + nt * 8;
        if (n0 >= a.N) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = r0 + g + ((u & 2) ? 8 : 0);
            const int col = n0 + tig * 2 + (u & 1);
            float v = acc[nt][u];
            if (a.bias) v += a.bias[col];
            if (a.mask && !(__bfloat162float(a.mask[(size_t)row * a.ldm + col]) > 0.f)) v = 0.f;
            if (a.relu) v = fmaxf(v, 0.f);
            if (a.Cf) a.Cf[(size_t)row * a.ldc + col] = v;
            if (a.Cb) a.Cb[(size_t)row * a.ldcb + col] = __float2bfloat16(v);
            if (a.CbT) a.CbT[(size_t)col * a.ldct + row] = __float2bfloat16(v);
        }
    }
}

// Residual degrees of each row's deletion set D: among the live nodes with a
// neighbour in D, r0 counts those with no live neighbour left and r1 those
// with exactly one; r2 counts the two-node components of G[V\D] adjacent to
// D.  Every (gene v, neighbour u) pair with u live scans N(u) until a second
// live neighbour shows up; u is counted by the first deleted node of its
// adjacency list, so exactly once.  A pendant u whose live neighbour w has no
// other live neighbour closes a two-node component, counted at u when u < w
// or when w has no deleted neighbour (degree 1), so once.  The deletion bitmap sits in
// shared memory (ceil(n/32) words); one CTA per row.  A warp takes 32 genes
// at a time: the (gene, neighbour) pairs of the genes of degree below 32 are
// laid end to end and dealt out one per lane (a lane finds its gene by binary
// search over the warp's degree prefix sums), and the whole warp walks each
// larger adjacency together.  Genes outside [0, n) are ignored.
__device__ __forceinline__ bool bm_dead(const unsigned* bm, int w) { return (bm[w >> 5] >> (w & 31)) & 1u; }

// Per node: {first arc, degree, a, b}: a and b are the two neighbours of lowest
// degree (earlier arcs first among equals; -1 when absent).  Any two live
// neighbours settle a node, and a deletion set that favours hubs is least likely
// to hold u's lowest-degree neighbours.  One thread per node, once per surrogate.
__global__ void nbr_table_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col, int n,
                                 int4* __restrict__ T) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int b = row_ptr[u], d = row_ptr[u + 1] - b;
        int a1 = -1, a2 = -1, d1 = INT_MAX, d2 = INT_MAX;
        for (int q0 = b; q0 < b + d; q0 += 4) {
            int x[4], dx[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = q0 + i < b + d ? __ldg(col + q0 + i) : -1;
#pragma unroll
            for (int i = 0; i < 4; ++i) dx[i] = x[i] >= 0 ? __ldg(row_ptr + x[i] + 1) - __ldg(row_ptr + x[i]) : INT_MAX;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (x[i] < 0) continue;
                if (dx[i] < d1) {
                    a2 = a1;
                    d2 = d1;
                    a1 = x[i];
                    d1 = dx[i];
                } else if (dx[i] < d2) {
                    a2 = x[i];
                    d2 = dx[i];
                }
            }
        }
        T[u] = make_int4(b, d, a1, a2);
    }
}

// Live neighbours of u, counted up to two (the last one seen in *w).
__device__ __forceinline__ int live_upto2(const unsigned* bm, const int4* __restrict__ T, const int* __restrict__ col,
                                          int u, int* first_dead, int* w) {
    const int4 tu = __ldg(T + u);
    if (tu.w >= 0 && !bm_dead(bm, tu.z) && !bm_dead(bm, tu.w)) return 2;
    int live = 0;
    for (int q = tu.x; q < tu.x + tu.y; ++q) {
        const int x = __ldg(col + q);
        if (bm_dead(bm, x)) {
            if (first_dead && *first_dead < 0) *first_dead = x;
        } else {
            *w = x;
            if (++live >= 2) return 2;
        }
    }
    return live;
}

// One row's residual-degree counts c = (r0, r1, r2, 0) and their
// standardised values z = ((r_j - mean_j) / max(sd_j, 1), 0) over the rows
// computed together (mean and population standard deviation of each count).
struct __align__(16) ResidRow {
    int4 c;
    float4 z;
};

// (u live) -> +1 to c0 or c1 when u has at most one live neighbour and v is its
// first deleted one; +1 to c2 when that neighbour closes a two-node component.
// Most live u keep the two neighbours of their table entry: one 16-byte read settles them.
__device__ __forceinline__ void resid_pair(const unsigned* bm, const int4* __restrict__ T,
                                           const int* __restrict__ col, int v, int u, int& c0, int& c1, int& c2) {
    if (bm_dead(bm, u)) return;
    int first_dead = -1, w = -1;
    const int live = live_upto2(bm, T, col, u, &first_dead, &w);
    if (live >= 2 || first_dead != v) return;
    c0 += live == 0;
    if (live == 1) {
        c1 += 1;
        int wl = -1;
        const int4 tw = __ldg(T + w);
        if ((u < w || tw.y == 1) && live_upto2(bm, T, col, w, nullptr, &wl) == 1) c2 += 1;
    }
}

__global__ void __launch_bounds__(256) resid_kernel(const int* __restrict__ pop, int rows, int k, int n,
                                                    const int4* __restrict__ T, const int* __restrict__ col,
                                                    ResidRow* __restrict__ out) {
    extern __shared__ unsigned bm[];
    __shared__ int red[3][8];
    const int r = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (r >= rows) return;
    const int words = (n + 31) >> 5;
    for (int w = t; w < words; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int* genes = pop + (size_t)r * k;
    for (int j = t; j < k; j += blockDim.x) {
        const int v = genes[j];
        if (v >= 0 && v < n) atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    int c0 = 0, c1 = 0, c2 = 0;
    const int nwarps = blockDim.x >> 5;
    for (int j0 = warp * 32; j0 < k; j0 += nwarps * 32) {
        const int j = j0 + lane;
        int v = j < k ? genes[j] : -1;
        if (v >= n) v = -1;
        int b = 0, e = 0;
        if (v >= 0) {
            const int4 tv = __ldg(T + v);
            b = tv.x;
            e = tv.x + tv.y;
        }
        const bool big = e - b >= 32;
        // small adjacencies: flatten the pairs over the lanes
        const int d = big ? 0 : e - b;
        int incl = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            // owner = the first lane whose inclusive prefix exceeds idx
            int lo = 0, hi = 31;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (lo + hi) >> 1;
                const int pm = __shfl_sync(0xffffffffu, incl, mid);
                if (pm > idx) hi = mid; else lo = mid + 1;
            }
            const int ov = __shfl_sync(0xffffffffu, v, lo), ob = __shfl_sync(0xffffffffu, b, lo),
                      oi = __shfl_sync(0xffffffffu, incl, lo), od = __shfl_sync(0xffffffffu, d, lo);
            if (idx < total) resid_pair(bm, T, col, ov, __ldg(col + ob + (idx - (oi - od))), c0, c1, c2);
        }
        unsigned many = __ballot_sync(0xffffffffu, big);
        while (many) {
            const int src = __ffs(many) - 1;
            many &= many - 1;
            const int vb = __shfl_sync(0xffffffffu, v, src), bb = __shfl_sync(0xffffffffu, b, src),
                      eb = __shfl_sync(0xffffffffu, e, src);
            for (int p = bb + lane; p < eb; p += 32) resid_pair(bm, T, col, vb, __ldg(col + p), c0, c1, c2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(0xffffffffu, c0, o);
        c1 += __shfl_down_sync(0xffffffffu, c1, o);
        c2 += __shfl_down_sync(0xffffffffu, c2, o);
    }
    if (lane == 0) {
        red[0][warp] = c0;
        red[1][warp] = c1;
        red[2][warp] = c2;
    }
    __syncthreads();
    if (t == 0) {
        int x = 0, y = 0, z = 0;
        for (int w = 0; w < nwarps; ++w) {
            x += red[0][w];
            y += red[1][w];
            z += red[2][w];
        }
        out[r].c = make_int4(x, y, z, 0);
    }
}

// Mean and standard deviation of each of the three counts over `rows` residual records (one CTA:
// exact int64 sums, then FP64 in a fixed order with explicit rounding: mean = S1 / rows,
// var = S2 / rows - mean^2, sd = max(sqrt(var), 1)); ms[0..2] = means, ms[3..5] = deviations.
__global__ void __launch_bounds__(256) resid_stats_kernel(const ResidRow* __restrict__ r, int rows,
                                                          double* __restrict__ ms) {
    __shared__ long long s1[3][256], s2[3][256];
    long long a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const int4 c = r[i].c;
        const long long v[3] = {c.x, c.y, c.z};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a[j] += v[j];
            b[j] += v[j] * v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        s1[j][threadIdx.x] = a[j];
        s2[j][threadIdx.x] = b[j];
    }
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                s1[j][threadIdx.x] += s1[j][threadIdx.x + w];
                s2[j][threadIdx.x] += s2[j][threadIdx.x + w];
            }
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        const int j = threadIdx.x;
        const double mean = __ddiv_rn((double)s1[j][0], (double)rows);
        const double var = __dsub_rn(__ddiv_rn((double)s2[j][0], (double)rows), __dmul_rn(mean, mean));
        ms[j] = mean;
        ms[3 + j] = fmax(__dsqrt_rn(fmax(var, 0.0)), 1.0);
    }
}

// z of every record from the statistics: z = float((c - mean) / sd), the FP64 operations
// explicitly rounded (spread over the whole grid: FP64 is slow on one SM).
__global__ void resid_z_kernel(ResidRow* __restrict__ r, int rows, const double* __restrict__ ms) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        const int4 c = r[i].c;
        r[i].z = make_float4(__double2float_rn(__ddiv_rn(__dsub_rn((double)c.x, ms[0]), ms[3])),
                             __double2float_rn(__ddiv_rn(__dsub_rn((double)c.y, ms[1]), ms[4])),
                             __double2float_rn(__ddiv_rn(__dsub_rn((double)c.z, ms[2]), ms[5])), 0.f);
    }
}

// Features of each row of pop (k genes): x (BF16 [rows_pad][80]) and its
// transpose (BF16 [80][rows_pad]); rows >= rows are zero.  resid[r] holds
// the row's residual-degree counts.  Genes outside [0, n) are ignored.
constexpr int kFeatWarps = 8, kFeatInFlight = 8;

__global__ void __launch_bounds__(kFeatWarps * 32) features_kernel(const int* __restrict__ pop, int rows, int k, int n,
                                                       const bf16* __restrict__ Eb, const float* __restrict__ logdeg,
                                                       const float* __restrict__ deg, float inv2E, float invsqrtk,
                                                       const ResidRow* __restrict__ resid, bf16* __restrict__ X,
                                                       bf16* __restrict__ XT, int rows_pad) {
    __shared__ float2 part[kFeatWarps][32];
    __shared__ float st[kFeatWarps][4];
    const int r = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (r >= rows) {
        for (int c = t; c < kIn; c += blockDim.x) {
            X[(size_t)r * kIn + c] = __float2bfloat16(0.f);
            XT[(size_t)c * rows_pad + r] = __float2bfloat16(0.f);
        }
        return;
    }
    const int* genes = pop + (size_t)r * k;
    // embedding sum: a warp reads whole 128-byte rows (lane = two dimensions),
    // warp w takes genes w, w + kFeatWarps, ...; kFeatInFlight loads in flight per lane
    const unsigned* E2 = reinterpret_cast<const unsigned*>(Eb);
    float sx = 0.f, sy = 0.f;
    int j = warp;
    constexpr int kSpan = kFeatWarps * kFeatInFlight;
    for (; j + kSpan - kFeatWarps < k; j += kSpan) {
        int v[kFeatInFlight];
#pragma unroll
        for (int u = 0; u < kFeatInFlight; ++u) v[u] = genes[j + kFeatWarps * u];
        unsigned w[kFeatInFlight];
#pragma unroll
        for (int u = 0; u < kFeatInFlight; ++u)
            w[u] = (v[u] >= 0 && v[u] < n) ? __ldg(E2 + (size_t)v[u] * (kEmb / 2) + lane) : 0u;
#pragma unroll
        for (int u = 0; u < kFeatInFlight; ++u) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[u]));
            sx += f.x;
            sy += f.y;
        }
    }
    for (; j < k; j += kFeatWarps) {
        const int v = genes[j];
        if (v >= 0 && v < n) {
            const unsigned w = __ldg(E2 + (size_t)v * (kEmb / 2) + lane);
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
            sx += f.x;
            sy += f.y;
        }
    }
    part[warp][lane] = make_float2(sx, sy);
    // degree statistics: thread-strided partial sums, then a fixed warp tree
    float q1 = 0.f, q2 = 0.f, qmax = -1.f, dsum = 0.f;
    for (int i = t; i < k; i += blockDim.x) {
        const int v = genes[i];
        if (v < 0 || v >= n) continue;
        const float q = logdeg[v];
        q1 += q;
        q2 += q * q;
        qmax = fmaxf(qmax, q);
        dsum += deg[v];
    }
    for (int o = 16; o > 0; o >>= 1) {
        q1 += __shfl_down_sync(0xffffffffu, q1, o);
        q2 += __shfl_down_sync(0xffffffffu, q2, o);
        qmax = fmaxf(qmax, __shfl_down_sync(0xffffffffu, qmax, o));
        dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    }
    if (lane == 0) {
        st[warp][0] = q1;
        st[warp][1] = q2;
        st[warp][2] = qmax;
        st[warp][3] = dsum;
    }
    __syncthreads();
    if (t < kEmb) {
        const int l = t >> 1;
        float e = 0.f;  // warps in a fixed order
#pragma unroll
        for (int w = 0; w < kFeatWarps; ++w) e += (t & 1) ? part[w][l].y : part[w][l].x;
        X[(size_t)r * kIn + t] = __float2bfloat16(e * invsqrtk);
        XT[(size_t)t * rows_pad + r] = __float2bfloat16(e * invsqrtk);
    } else if (t < kIn) {
        float f = 0.f;
        float Q1 = 0.f, Q2 = 0.f, QM = -1.f, DS = 0.f;
#pragma unroll
        for (int w = 0; w < kFeatWarps; ++w) {
            Q1 += st[w][0];
            Q2 += st[w][1];
            QM = fmaxf(QM, st[w][2]);
            DS += st[w][3];
        }
        const float mean = k > 0 ? Q1 / k : 0.f;
        if (t == 64) f = mean;
        if (t == 65) f = k > 0 ? QM : 0.f;
        if (t == 66) f = k > 0 ? sqrtf(fmaxf(Q2 / k - mean * mean, 0.f)) : 0.f;
        if (t == 67) f = DS * inv2E;
        if (t == 68) f = log1pf((float)resid[r].c.x);
        if (t == 69) f = log1pf((float)resid[r].c.y);
        if (t == 70) f = log1pf((float)resid[r].c.z);
        if (t == 71) f = resid[r].z.x;
        if (t == 72) f = resid[r].z.y;
        if (t == 73) f = resid[r].z.z;
        X[(size_t)r * kIn + t] = __float2bfloat16(f);
        XT[(size_t)t * rows_pad + r] = __float2bfloat16(f);
    }
}

// y[r] = h2[r] . w3 + b3 (FP32), one warp per row.
__global__ void head_kernel(const bf16* __restrict__ H2, int rows, const float* __restrict__ w3,
                            const float* __restrict__ b3, float* __restrict__ y) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    for (int h = lane; h < kHid; h += 32) s += __bfloat162float(H2[(size_t)r * kHid + h]) * w3[h];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] = s + b3[0];
}

// dy = 2 (y - t) / B and the batch loss (one CTA, fixed order).
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int B,
                                                   float* __restrict__ dy, float* __restrict__ loss) {
    __shared__ float red[8];
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float e = y[b] - t[b];
        dy[b] = 2.f * e / B;
        s += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < 8; ++w) tot += red[w];
        *loss = tot / B;
    }
}

// dz2 = dy * w3 where h2 > 0 (BF16 and transposed BF16).
__global__ void __launch_bounds__(256) dz2_kernel(const bf16* __restrict__ H2, const float* __restrict__ dy,
                                                  const float* __restrict__ w3, int B, bf16* __restrict__ dZ2,
                                                  bf16* __restrict__ dZ2T) {
    const int b = blockIdx.x, h = threadIdx.x;
    const float v = __bfloat162float(H2[(size_t)b * kHid + h]) > 0.f ? dy[b] * w3[h] : 0.f;
    dZ2[(size_t)b * kHid + h] = __float2bfloat16(v);
    dZ2T[(size_t)h * B + b] = __float2bfloat16(v);
}

// Column sums over the batch in a fixed order: dw3 = H2^T dy, db2 = sum dz2,
// db3 = sum dy (db1 with H2 = nullptr and Z = dz1).  CTA c takes columns
// 32c..32c+31; its 8 warps sum interleaved row groups, combined in order.
__global__ void __launch_bounds__(256) colsum_kernel(const bf16* __restrict__ H2, const float* __restrict__ dy,
                                                     const bf16* __restrict__ Z, int B, float* __restrict__ dw3,
                                                     float* __restrict__ db, float* __restrict__ db3) {
    __shared__ float pw[8][32], pb[8][32];
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5, h = blockIdx.x * 32 + lane;
    // four rows per thread in flight, summed in a fixed order
    float sw = 0.f, sb = 0.f;
    int b = rg;
    for (; b + 24 < B; b += 32) {
        float zw[4], zb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int bq = b + 8 * q;
            zb[q] = __bfloat162float(Z[(size_t)bq * kHid + h]);
            zw[q] = H2 ? __bfloat162float(H2[(size_t)bq * kHid + h]) * dy[bq] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sw += zw[q];
            sb += zb[q];
        }
    }
    for (; b < B; b += 8) {
        if (H2) sw += __bfloat162float(H2[(size_t)b * kHid + h]) * dy[b];
        sb += __bfloat162float(Z[(size_t)b * kHid + h]);
    }
    pw[rg][lane] = sw;
    pb[rg][lane] = sb;
    __syncthreads();
    if (rg == 0) {
        float w = 0.f, c = 0.f;
        for (int g = 0; g < 8; ++g) {
            w += pw[g][lane];
            c += pb[g][lane];
        }
        if (dw3) dw3[h] = w;
        db[h] = c;
    } else if (rg == 1 && db3 && blockIdx.x == 0) {
        float s = 0.f;
        for (int b = lane; b < B; b += 32) s += dy[b];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) db3[0] = s;
    }
}

// Embedding gradient: every gene v of row b gets dx[b][0:64] / sqrt(k), each
// term rounded to 2^-40 fixed point and summed as integers (exact, so the
// order of the terms does not matter and training is bit-reproducible).  The
// batch is first turned into lists of rows per node (a counting sort:
// occurrences, an exclusive scan, a fill), then one warp per node sums its
// rows' terms in registers and writes the node's 64 sums: no atomics on the
// gradient and no clearing of it.
// The rounded terms once per (row, dimension): q[b][d] = round(dX[b][d] / sqrt(k) * 2^40)
// (FP64 is slow on this part, so the per-node sums read these integers).
__global__ void emb_terms_kernel(const float* __restrict__ dX, int B, float invsqrtk, long long* __restrict__ q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * kEmb; i += gridDim.x * blockDim.x) {
        const int b = i / kEmb, d = i % kEmb;
        q[i] = llrint((double)dX[(size_t)b * kIn + d] * invsqrtk * kFix);
    }
}

__global__ void emb_count_kernel(const int* __restrict__ pop, size_t cells, int n, int* __restrict__ cnt) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
        const int v = __ldg(&pop[i]);
        if ((unsigned)v < (unsigned)n) atomicAdd(&cnt[v], 1);
    }
}

// Exclusive scan of cnt[0 .. n) in blocks of 1024: off[v] = the prefix within v's block, blk[b] =
// block b's total.
__global__ void __launch_bounds__(1024) scan_block_kernel(const int* __restrict__ cnt, int n, int* __restrict__ off,
                                                          int* __restrict__ blk) {
    __shared__ int ws[32];
    const int v = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x = v < n ? cnt[v] : 0;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int y = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const int pre = (warp ? ws[warp - 1] : 0) + incl - x;
    if (v < n) off[v] = pre;
    if (threadIdx.x == 1023) blk[blockIdx.x] = pre + x;
}

// Exclusive scan of the nb block totals in place (one CTA, 1024 at a time with a carry).
__global__ void __launch_bounds__(1024) scan_top_kernel(int* __restrict__ blk, int nb) {
    __shared__ int ws[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const int x = b < nb ? blk[b] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int y = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            ws[lane] = y;
        }
        __syncthreads();
        const int c = carry;
        if (b < nb) blk[b] = c + (warp ? ws[warp - 1] : 0) + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + ws[31];
        __syncthreads();
    }
}

// off[v] += the offset of v's block; cur[v] = off[v] (the fill cursors); off[n] = the total.
__global__ void scan_add_kernel(int* __restrict__ off, const int* __restrict__ blk, const int* __restrict__ cnt, int n,
                                int* __restrict__ cur) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int o = off[v] + blk[v >> 10];
        off[v] = o;
        cur[v] = o;
        if (v == n - 1) off[n] = o + cnt[v];
    }
}

__global__ void emb_fill_kernel(const int* __restrict__ pop, size_t cells, int k, int n, int* __restrict__ cur,
                                int* __restrict__ rows_of) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
        const int v = __ldg(&pop[i]);
        if ((unsigned)v < (unsigned)n) rows_of[atomicAdd(&cur[v], 1)] = (int)(i / (size_t)k);
    }
}

// One warp per node: lanes take dimensions lane and lane + 32.
__global__ void __launch_bounds__(256) emb_gather_kernel(const int* __restrict__ off, const int* __restrict__ rows_of,
                                                         const long long* __restrict__ q, int n,
                                                         unsigned long long* __restrict__ Gi) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        long long s0 = 0, s1 = 0;
        for (int e = __ldg(&off[v]), e1 = __ldg(&off[v + 1]); e < e1; ++e) {
            const long long* qb = q + (size_t)__ldg(&rows_of[e]) * kEmb;
            s0 += __ldg(qb + lane);
            s1 += __ldg(qb + lane + 32);
        }
        Gi[(size_t)v * kEmb + lane] = (unsigned long long)s0;
        Gi[(size_t)v * kEmb + lane + 32] = (unsigned long long)s1;
    }
}

// Fixed point (2^-40) to FP32 without the FP64 pipe: hi * 2^32 + lo in one
// rounding, then the exact scaling by 2^-40.
__device__ __forceinline__ float fix_to_float(unsigned long long u) {
    const long long x = (long long)u;
    return fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)x) * 9.094947017729282e-13f;
}

__device__ __forceinline__ float adamw_one(float p, float g, float& m, float& v, float lr, float b1, float b2,
                                           float wd, float eps, float bc1, float bc2) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    return p - lr * ((m / bc1) / (sqrtf(v / bc2) + eps) + wd * p);
}

// The embedding table's step in one pass over 4-element groups: the
// fixed-point gradient, AdamW on the FP32 master and moments, the BF16 copy.
// The accumulator keeps the gradient until the next step clears it.
__global__ void __launch_bounds__(256) emb_update_kernel(const ulonglong2* __restrict__ Gi, float4* __restrict__ P,
                                                         float4* __restrict__ M, float4* __restrict__ V,
                                                         uint2* __restrict__ Eb, size_t groups, float lr, float b1,
                                                         float b2, float wd, float eps, float bc1, float bc2,
                                                         const float2* __restrict__ bcp) {
    if (bcp) {
        bc1 = bcp->x;
        bc2 = bcp->y;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < groups; i += (size_t)gridDim.x * blockDim.x) {
        const ulonglong2 g01 = Gi[2 * i], g23 = Gi[2 * i + 1];
        float4 p = P[i], m = M[i], v = V[i];
        p.x = adamw_one(p.x, fix_to_float(g01.x), m.x, v.x, lr, b1, b2, wd, eps, bc1, bc2);
        p.y = adamw_one(p.y, fix_to_float(g01.y), m.y, v.y, lr, b1, b2, wd, eps, bc1, bc2);
        p.z = adamw_one(p.z, fix_to_float(g23.x), m.z, v.z, lr, b1, b2, wd, eps, bc1, bc2);
        p.w = adamw_one(p.w, fix_to_float(g23.y), m.w, v.w, lr, b1, b2, wd, eps, bc1, bc2);
        P[i] = p;
        M[i] = m;
        V[i] = v;
        const __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
        Eb[i] = make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
}

// The last embedding gradient as FP32 (for gapa_surrogate_tensor).
__global__ void emb_grad_float_kernel(const unsigned long long* __restrict__ Gi, float* __restrict__ G, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        G[i] = fix_to_float(Gi[i]);
}

__global__ void adamw_kernel(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                             const float* __restrict__ G, size_t count, float lr, float b1, float b2, float wd,
                             float eps, float bc1, float bc2, const float2* __restrict__ bcp) {
    if (bcp) {
        bc1 = bcp->x;
        bc2 = bcp->y;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        const float p = P[i];
        P[i] = p - lr * ((m / bc1) / (sqrtf(v / bc2) + eps) + wd * p);
    }
}

// BF16 copies: W (rows x cols) and its transpose; E.
__global__ void to_bf16_kernel(const float* __restrict__ W, int rows, int cols, bf16* __restrict__ Wb,
                               bf16* __restrict__ WbT) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
        const int r = i / cols, c = i % cols;
        const bf16 v = __float2bfloat16(W[i]);
        if (Wb) Wb[i] = v;
        if (WbT) WbT[(size_t)c * rows + r] = v;
    }
}

__global__ void to_bf16_flat_kernel(const float* __restrict__ W, size_t count, bf16* __restrict__ Wb) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        Wb[i] = __float2bfloat16(W[i]);
}

// Uniform initialisation U(-a, a) from Philox (tag 8, counter (i lo, i hi, tensor, 0)).
__global__ void init_uniform_kernel(float* __restrict__ P, size_t count, float a, RngKey key, uint32_t tensor) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = philox_word0((uint32_t)i, (uint32_t)(i >> 32), tensor, 8u << 24, key.lo, key.hi);
        P[i] = a * (2.f * ((float)x * 2.3283064365386963e-10f) - 1.f);
    }
}

// Lowest `m` of `cnt` scores (ties to the lower index): bitonic sort of
// (order-preserving score bits << 32 | index) in shared memory; one CTA.
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ score, int cnt, int m,
                                                    int* __restrict__ sel, int P) {
    extern __shared__ unsigned long long keys[];
    for (int x = threadIdx.x; x < P; x += blockDim.x) {
        unsigned long long key = ~0ull;
        if (x < cnt) {
            unsigned u = __float_as_uint(score[x]);
            u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            key = ((unsigned long long)u << 32) | (unsigned)x;
        }
        keys[x] = key;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = threadIdx.x; x < P; x += blockDim.x) {
                const int y = x ^ stride;
                if (y > x) {
                    const bool up = (x & size) == 0;
                    if ((keys[x] > keys[y]) == up) {
                        const unsigned long long t = keys[x];
                        keys[x] = keys[y];
                        keys[y] = t;
                    }
                }
            }
            __syncthreads();
        }
    for (int r = threadIdx.x; r < m; r += blockDim.x) sel[r] = (int)(keys[r] & 0xFFFFFFFFu);
}

// dst row r = src row idx[r] (idx may be null: identity), k genes, with its
// residual-degree counts; dst_cap > 0 writes ring slots (dst_first + r) mod dst_cap.
__global__ void gather_rows_kernel(const int* __restrict__ src, const ResidRow* __restrict__ rsrc,
                                   const int* __restrict__ idx, int k, int* __restrict__ dst, ResidRow* __restrict__ rdst,
                                   int dst_first, int dst_cap, const int* __restrict__ first_dev) {
    const int r = blockIdx.x;
    if (first_dev) dst_first = *first_dev;
    const int from = idx ? idx[r] : r;
    const int to = dst_cap > 0 ? (dst_first + r) % dst_cap : r;
    for (int j = threadIdx.x; j < k; j += blockDim.x) dst[(size_t)to * k + j] = src[(size_t)from * k + j];
    if (threadIdx.x == 0) rdst[to] = rsrc[from];
}

// kfit[i] = +inf for every child, then the evaluated ones.
__global__ void scatter_fit_kernel(const long long* __restrict__ fsel, const int* __restrict__ sel, int m, int lambda,
                                   long long* __restrict__ kfit) {
    for (int i = threadIdx.x; i < lambda; i += blockDim.x) kfit[i] = LLONG_MAX;
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) kfit[sel[r]] = fsel[r];
}

// Ring append of one generation's exactly evaluated rows (one CTA, FP64,
// fixed-order reductions): l = log1p(fitness); gstats = (mean, std) of l over
// these rows; the ring keeps l (target mode 0: normalised later over the whole
// ring) or (l - mean) / std (mode 1: z-score among the row's siblings).
__global__ void __launch_bounds__(1024) ring_target_kernel(const int64_t* __restrict__ f, int cnt, int mode,
                                                           double* __restrict__ ring_lp, int first, int cap,
                                                           double* __restrict__ gstats, const int* __restrict__ first_dev) {
    __shared__ double s1[1024], s2[1024];
    if (first_dev) first = *first_dev;
    double a = 0, b = 0;
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const double l = log1p((double)f[r]);
        a += l;
        b += l * l;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    const double mu = s1[0] / cnt, var = s2[0] / cnt - mu * mu;
    const double sd = var > 1e-24 ? sqrt(var) : 1.0;
    if (threadIdx.x == 0) {
        gstats[0] = mu;
        gstats[1] = sd;
    }
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const double l = log1p((double)f[r]);
        ring_lp[(first + r) % cap] = mode == 1 ? (l - mu) / sd : l;
    }
}

// Mean and standard deviation of log1p(fitness) over the ring (one CTA, FP64,
// fixed-order reduction).
__global__ void __launch_bounds__(1024) target_stats_kernel(const double* __restrict__ ring_lp, int valid,
                                                            double* __restrict__ stats, const int* __restrict__ valid_dev) {
    __shared__ double s1[1024], s2[1024];
    if (valid_dev) valid = *valid_dev;
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < valid; i += blockDim.x) {
        const double l = ring_lp[i];
        a += l;
        b += l * l;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = s1[0] / valid;
        const double var = s2[0] / valid - mu * mu;
        stats[0] = mu;
        stats[1] = var > 1e-24 ? sqrt(var) : 1.0;
    }
}

// Minibatch: rows drawn uniformly from the valid ring entries (Philox tag 8,
// counter (b, step, g, 8 << 24 | 1)), targets z-scored.
__global__ void batch_kernel(const int* __restrict__ ring, const ResidRow* __restrict__ ring_resid,
                             const double* __restrict__ ring_lp, int valid, int k, int B, RngKey key, int step,
                             int g, const double* __restrict__ stats, int* __restrict__ rows,
                             ResidRow* __restrict__ resid, float* __restrict__ t, const int* __restrict__ valid_dev,
                             const int* __restrict__ g_dev) {
    const int b = blockIdx.x;
    if (valid_dev) valid = *valid_dev;
    if (g_dev) g = *g_dev - 1;  // the record of this generation has advanced the counter
    const int idx = uniform_below(philox_word0((uint32_t)b, (uint32_t)step, (uint32_t)g, (8u << 24) | 1u, key.lo, key.hi),
                                  valid);
    for (int j = threadIdx.x; j < k; j += blockDim.x) rows[(size_t)b * k + j] = ring[(size_t)idx * k + j];
    if (threadIdx.x == 0) {
        t[b] = (float)((ring_lp[idx] - stats[0]) / stats[1]);
        resid[b] = ring_resid[idx];
    }
}

// Ring bookkeeping of a run on the device (so that generations can be replayed
// from a CUDA graph): st[0] = next ring slot, st[1] = valid rows.
__global__ void ring_advance_kernel(int* __restrict__ st, int added, int cap) {
    st[0] = (st[0] + added) % cap;
    st[1] = min(cap, st[1] + added);
}

// One AdamW step on the device: tau += 1 and its bias corrections from the
// table the host computed (1 - beta1^tau, 1 - beta2^tau).
__global__ void tau_step_kernel(int* __restrict__ tau, const float2* __restrict__ table, float2* __restrict__ bc) {
    const int t = *tau + 1;
    *tau = t;
    *bc = table[t];
}

// Scores back to pairwise-connectivity estimates: expm1(mean + std * y) with
// the target statistics of the last training step.
__global__ void decode_kernel(const float* __restrict__ y, int rows, const double* __restrict__ stats,
                              float* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x)
        out[r] = (float)expm1(stats[0] + stats[1] * (double)y[r]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct gapa_surrogate {
    gapa_ctx* ctx = nullptr;
    int device = 0;  // the context's device, kept so that destruction never reads the context
    gapa_surrogate_config cfg;
    RngKey key;
    Layout L;
    int n = 0, k_max = 0, rows_cap = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;
    unsigned long long* Gi = nullptr;
    bf16 *W1b = nullptr, *W1tb = nullptr, *W2b = nullptr, *W2tb = nullptr, *Eb = nullptr;
    float *logdeg = nullptr, *deg = nullptr;
    float inv2E = 0.f;
    // activations for up to rows_cap rows
    bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ2T = nullptr,
         *dZ1 = nullptr, *dZ1T = nullptr;
    float *y = nullptr, *dy = nullptr, *dX = nullptr, *loss = nullptr, *tbuf = nullptr;
    ResidRow* resid = nullptr;   // residual-degree counts (and their z) of the rows of the last forward
    int4* nbr = nullptr;         // per node: first arc, degree, its two lowest-degree neighbours
    const int* row_ptr = nullptr;  // the context's CSR (original node ids)
    const int* col = nullptr;
    size_t resid_smem = 0;       // deletion bitmap bytes of resid_kernel
    int* batch_rows = nullptr;
    double* stats = nullptr;
    int tau = 0;
    // embedding gradient: occurrences per node, list offsets (n + 1), fill cursors, block totals,
    // and the rows of every node's list
    int *emb_cnt = nullptr, *emb_off = nullptr, *emb_cur = nullptr, *emb_blk = nullptr, *rows_of = nullptr;
    double* rstats = nullptr;  // means and deviations of the residual counts of the last rows computed
    long long* emb_q = nullptr;  // the rounded gradient terms [rows][64] of the last training step
    int emb_q_rows = 0;
    size_t rows_of_cap = 0;
};

namespace {

int launch_gemm(const GemmArgs& a, cudaStream_t st) {
    dim3 grid((a.N + kGemmCols - 1) / kGemmCols, (a.M + kGemmRowsPerCta - 1) / kGemmRowsPerCta);
    gemm_bf16_kernel<<<grid, 128, 0, st>>>(a);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

GemmArgs gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb) {
    GemmArgs a;
    memset(&a, 0, sizeof a);
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.lda = lda;
    a.B = B;
    a.ldb = ldb;
    return a;
}

int refresh_bf16(gapa_surrogate* s, cudaStream_t st) {
    to_bf16_kernel<<<64, 256, 0, st>>>(s->P + s->L.W1, kIn, kHid, s->W1b, s->W1tb);
    to_bf16_kernel<<<128, 256, 0, st>>>(s->P + s->L.W2, kHid, kHid, s->W2b, s->W2tb);
    to_bf16_flat_kernel<<<s->ctx->num_sms * 4, 256, 0, st>>>(s->P + s->L.E, (size_t)s->n * kEmb, s->Eb);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int round16(int x) { return (x + 15) & ~15; }

// Features + forward; keeps the transposed copies for a training step.
// Residual-degree counts of `rows` deletion sets into s->resid, standardised over those rows.
int compute_resid(gapa_surrogate* s, const int32_t* pop, int rows, int k, cudaStream_t st) {
    if (rows <= 0) return GAPA_OK;
    ProfileScope prof(s->ctx, st, 2, 3);
    resid_kernel<<<rows, 256, s->resid_smem, st>>>(pop, rows, k, s->n, s->nbr, s->col, s->resid);
    resid_stats_kernel<<<1, 256, 0, st>>>(s->resid, rows, s->rstats);
    resid_z_kernel<<<(rows + 127) / 128, 128, 0, st>>>(s->resid, rows, s->rstats);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

// Features + forward; keeps the transposed copies for a training step.  With
// resid == nullptr the residual-degree counts are computed into s->resid first.
int forward(gapa_surrogate* s, const int32_t* pop, int rows, int k, bool keep, cudaStream_t st,
            const ResidRow* resid = nullptr) {
    if (!resid) {
        int rc = compute_resid(s, pop, rows, k, st);
        if (rc != GAPA_OK) return rc;
        resid = s->resid;
    }
    ProfileScope prof(s->ctx, st, 2, 4);
    const int R = round16(rows);
    features_kernel<<<R, kFeatWarps * 32, 0, st>>>(pop, rows, k, s->n, s->Eb, s->logdeg, s->deg, s->inv2E,
                                       1.f / sqrtf((float)std::max(k, 1)), resid, s->X, s->XT, R);
    GemmArgs a = gemm(R, kHid, kIn, s->X, kIn, s->W1tb, kIn);
    a.Cb = s->H1;
    a.ldcb = kHid;
    if (keep) {
        a.CbT = s->H1T;
        a.ldct = R;
    }
    a.bias = s->P + s->L.b1;
    a.relu = 1;
    int rc = launch_gemm(a, st);
    if (rc != GAPA_OK) return rc;
    a = gemm(R, kHid, kHid, s->H1, kHid, s->W2tb, kHid);
    a.Cb = s->H2;
    a.ldcb = kHid;
    a.bias = s->P + s->L.b2;
    a.relu = 1;
    rc = launch_gemm(a, st);
    if (rc != GAPA_OK) return rc;
    head_kernel<<<(rows + 7) / 8, 256, 0, st>>>(s->H2, rows, s->P + s->L.w3, s->P + s->L.b3, s->y);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

// Lists of rows per node for B rows of k genes (rows_of holds B * k entries).
int ensure_csr(gapa_surrogate* s, size_t cells, int rows) {
    if (rows > s->emb_q_rows) {
        cudaFree(s->emb_q);
        s->emb_q = nullptr;
        s->emb_q_rows = 0;
        if (cudaMalloc(&s->emb_q, (size_t)std::max(rows, 1) * kEmb * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            return gapa_fail(GAPA_ERR_OOM, "embedding-gradient terms of %d rows", rows);
        }
        s->emb_q_rows = rows;
    }
    if (cells <= s->rows_of_cap) return GAPA_OK;
    cudaFree(s->rows_of);
    s->rows_of = nullptr;
    s->rows_of_cap = 0;
    if (cudaMalloc(&s->rows_of, std::max<size_t>(cells, 1) * 4) != cudaSuccess) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "embedding-gradient lists of %zu entries", cells);
    }
    s->rows_of_cap = cells;
    return GAPA_OK;
}

// The embedding gradient of a batch into s->Gi (fixed point): count, scan, fill, gather.
int emb_gradient(gapa_surrogate* s, const int32_t* pop, int B, int k, cudaStream_t st) {
    const size_t cells = (size_t)B * k;
    int rc = ensure_csr(s, cells, B);
    if (rc != GAPA_OK) return rc;
    const int n = s->n, nb = (n + 1023) / 1024, grid = s->ctx->num_sms * 4;
    GAPA_CUDA(cudaMemsetAsync(s->emb_cnt, 0, (size_t)n * 4, st));
    emb_count_kernel<<<grid, 256, 0, st>>>(pop, cells, n, s->emb_cnt);
    scan_block_kernel<<<nb, 1024, 0, st>>>(s->emb_cnt, n, s->emb_off, s->emb_blk);
    scan_top_kernel<<<1, 1024, 0, st>>>(s->emb_blk, nb);
    scan_add_kernel<<<grid, 256, 0, st>>>(s->emb_off, s->emb_blk, s->emb_cnt, n, s->emb_cur);
    emb_fill_kernel<<<grid, 256, 0, st>>>(pop, cells, std::max(k, 1), n, s->emb_cur, s->rows_of);
    emb_terms_kernel<<<(B * kEmb + 255) / 256, 256, 0, st>>>(s->dX, B, 1.f / sqrtf((float)std::max(k, 1)), s->emb_q);
    emb_gather_kernel<<<grid * 2, 256, 0, st>>>(s->emb_off, s->rows_of, s->emb_q, n, s->Gi);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

// One AdamW step on a batch (rows a multiple of 16) with targets t.
// With tau_dev, the step count and its bias corrections live on the device (a
// step of a CUDA-graph-replayed generation): tau_dev[0] is advanced and the
// corrections come from `table` (indexed by the step) through bc_dev.
int train_step(gapa_surrogate* s, const int32_t* pop, int B, int k, const float* t, cudaStream_t st,
               const ResidRow* resid = nullptr, int* tau_dev = nullptr, const float2* table = nullptr,
               float2* bc_dev = nullptr) {
    int rc = forward(s, pop, B, k, true, st, resid);
    if (rc != GAPA_OK) return rc;
    ProfileScope prof(s->ctx, st, 2, 19);
    float* G = s->G;
    const Layout& L = s->L;
    loss_kernel<<<1, 256, 0, st>>>(s->y, t, B, s->dy, s->loss);
    dz2_kernel<<<B, kHid, 0, st>>>(s->H2, s->dy, s->P + L.w3, B, s->dZ2, s->dZ2T);
    colsum_kernel<<<kHid / 32, 256, 0, st>>>(s->H2, s->dy, s->dZ2, B, G + L.w3, G + L.b2, G + L.b3);
    // dW2 = h1^T dz2  ([in][out])
    GemmArgs a = gemm(kHid, kHid, B, s->H1T, B, s->dZ2T, B);
    a.Cf = G + L.W2;
    a.ldc = kHid;
    if ((rc = launch_gemm(a, st)) != GAPA_OK) return rc;
    // dz1 = (dz2 W2^T) where h1 > 0
    a = gemm(B, kHid, kHid, s->dZ2, kHid, s->W2b, kHid);
    a.Cb = s->dZ1;
    a.ldcb = kHid;
    a.CbT = s->dZ1T;
    a.ldct = B;
    a.mask = s->H1;
    a.ldm = kHid;
    if ((rc = launch_gemm(a, st)) != GAPA_OK) return rc;
    colsum_kernel<<<kHid / 32, 256, 0, st>>>(nullptr, nullptr, s->dZ1, B, nullptr, G + L.b1, nullptr);
    // dW1 = x^T dz1  ([80][256])
    a = gemm(kIn, kHid, B, s->XT, B, s->dZ1T, B);
    a.Cf = G + L.W1;
    a.ldc = kHid;
    if ((rc = launch_gemm(a, st)) != GAPA_OK) return rc;
    // dx = dz1 W1^T ([B][80])
    a = gemm(B, kIn, kHid, s->dZ1, kHid, s->W1b, kHid);
    a.Cf = s->dX;
    a.ldc = kIn;
    if ((rc = launch_gemm(a, st)) != GAPA_OK) return rc;
    if ((rc = emb_gradient(s, pop, B, k, st)) != GAPA_OK) return rc;
    s->tau += 1;
    const float bc1 = 1.f - powf(s->cfg.beta1, (float)s->tau), bc2 = 1.f - powf(s->cfg.beta2, (float)s->tau);
    if (tau_dev) tau_step_kernel<<<1, 1, 0, st>>>(tau_dev, table, bc_dev);
    // dense parameters (W1 .. b3), then the embedding table in one fused pass
    adamw_kernel<<<64, 256, 0, st>>>(s->P, s->M, s->V, G, L.E, s->cfg.lr, s->cfg.beta1, s->cfg.beta2,
                                     s->cfg.weight_decay, s->cfg.eps, bc1, bc2, tau_dev ? bc_dev : nullptr);
    emb_update_kernel<<<s->ctx->num_sms * 8, 256, 0, st>>>(
        reinterpret_cast<const ulonglong2*>(s->Gi), reinterpret_cast<float4*>(s->P + L.E),
        reinterpret_cast<float4*>(s->M + L.E), reinterpret_cast<float4*>(s->V + L.E), reinterpret_cast<uint2*>(s->Eb),
        (size_t)s->n * kEmb / 4, s->cfg.lr, s->cfg.beta1, s->cfg.beta2, s->cfg.weight_decay, s->cfg.eps, bc1, bc2,
        tau_dev ? bc_dev : nullptr);
    to_bf16_kernel<<<64, 256, 0, st>>>(s->P + L.W1, kIn, kHid, s->W1b, s->W1tb);
    to_bf16_kernel<<<128, 256, 0, st>>>(s->P + L.W2, kHid, kHid, s->W2b, s->W2tb);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int ensure_rows(gapa_surrogate* s, int rows) {
    const int R = round16(rows);
    if (R <= s->rows_cap) return GAPA_OK;
    bf16** bfs[] = {&s->X, &s->XT, &s->H1, &s->H1T, &s->H2, &s->dZ2, &s->dZ2T, &s->dZ1, &s->dZ1T};
    for (bf16** p : bfs) {
        cudaFree(*p);
        *p = nullptr;
    }
    float** fps[] = {&s->y, &s->dy, &s->dX, &s->tbuf};
    for (float** p : fps) {
        cudaFree(*p);
        *p = nullptr;
    }
    cudaFree(s->resid);
    s->resid = nullptr;
    const size_t e80 = (size_t)R * kIn, e256 = (size_t)R * kHid;
    if (cudaMalloc(&s->X, e80 * 2) || cudaMalloc(&s->XT, e80 * 2) || cudaMalloc(&s->H1, e256 * 2) ||
        cudaMalloc(&s->H1T, e256 * 2) || cudaMalloc(&s->H2, e256 * 2) || cudaMalloc(&s->dZ2, e256 * 2) ||
        cudaMalloc(&s->dZ2T, e256 * 2) || cudaMalloc(&s->dZ1, e256 * 2) || cudaMalloc(&s->dZ1T, e256 * 2) ||
        cudaMalloc(&s->y, (size_t)R * 4) || cudaMalloc(&s->dy, (size_t)R * 4) || cudaMalloc(&s->dX, e80 * 4) ||
        cudaMalloc(&s->tbuf, (size_t)R * 4) || cudaMalloc(&s->resid, (size_t)R * sizeof(ResidRow))) {
        cudaGetLastError();
        return gapa_fail(GAPA_ERR_OOM, "surrogate activations for %d rows", R);
    }
    s->rows_cap = R;
    return GAPA_OK;
}

// The surrogate reads the context's CSR: a graph uploaded after creation invalidates it.
int check_graph(const gapa_surrogate* s) {
    if (s->ctx->g.row_ptr != s->row_ptr || s->ctx->g.n != s->n)
        return gapa_fail(GAPA_ERR_STATE, "the context's graph changed after the surrogate was created");
    return GAPA_OK;
}

void free_surrogate(gapa_surrogate* s) {
    void* ps[] = {s->P, s->M, s->V, s->G, s->Gi, s->W1b, s->W1tb, s->W2b, s->W2tb, s->Eb, s->logdeg, s->deg,
                  s->X, s->XT, s->H1, s->H1T, s->H2, s->dZ2, s->dZ2T, s->dZ1, s->dZ1T, s->y, s->dy, s->dX,
                  s->loss, s->tbuf, s->batch_rows, s->stats, s->resid, s->nbr, s->emb_cnt, s->emb_off,
                  s->emb_cur, s->emb_blk, s->rows_of, s->rstats, s->emb_q};
    for (void* p : ps) cudaFree(p);
}

}  // namespace

extern "C" {

int gapa_surrogate_create(gapa_surrogate** out, gapa_ctx* ctx, const gapa_surrogate_config* scfg, uint64_t seed) {
    if (!out || !ctx || !scfg) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (ctx->g.n <= 0) return gapa_fail(GAPA_ERR_STATE, "no graph uploaded");
    if (ctx->genes != GAPA_GENES_NODES) return gapa_fail(GAPA_ERR_INVALID_ARG, "the surrogate takes node genes only");
    if (scfg->batch < 16 || scfg->batch % 16 || scfg->ring < scfg->batch || scfg->train_steps < 0 ||
        scfg->screened < 1 || scfg->warmup < 0 || !(scfg->lr > 0.f) || scfg->target_mode < 0 ||
        scfg->target_mode > 1)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "invalid surrogate configuration");
    cudaSetDevice(ctx->device);
    gapa_surrogate* s = new gapa_surrogate();
    s->ctx = ctx;
    s->device = ctx->device;
    s->cfg = *scfg;
    s->key = RngKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
    s->n = ctx->g.n;
    s->row_ptr = ctx->g.row_ptr;
    s->col = ctx->g.col;
    s->resid_smem = (((size_t)s->n + 31) / 32) * 4;
    if (s->resid_smem > ctx->smem_optin) {
        delete s;
        return gapa_fail(GAPA_ERR_INVALID_ARG, "n = %d: the deletion bitmap does not fit in shared memory", ctx->g.n);
    }
    if (s->resid_smem > 48 * 1024 &&
        cudaFuncSetAttribute(resid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->resid_smem) !=
            cudaSuccess) {
        cudaGetLastError();
        delete s;
        return gapa_fail(GAPA_ERR_CUDA, "shared memory limit of the residual-degree kernel");
    }
    s->L = make_layout(s->n);
    auto bail = [&](int rc) {
        free_surrogate(s);
        delete s;
        return rc;
    };
    const size_t np = s->L.total;
    if (cudaMalloc(&s->P, np * 4) || cudaMalloc(&s->M, np * 4) || cudaMalloc(&s->V, np * 4) ||
        cudaMalloc(&s->G, np * 4) || cudaMalloc(&s->Gi, (size_t)s->n * kEmb * 8) ||
        cudaMalloc(&s->W1b, (size_t)kIn * kHid * 2) || cudaMalloc(&s->W1tb, (size_t)kIn * kHid * 2) ||
        cudaMalloc(&s->W2b, (size_t)kHid * kHid * 2) || cudaMalloc(&s->W2tb, (size_t)kHid * kHid * 2) ||
        cudaMalloc(&s->Eb, (size_t)s->n * kEmb * 2) || cudaMalloc(&s->logdeg, (size_t)s->n * 4) ||
        cudaMalloc(&s->deg, (size_t)s->n * 4) || cudaMalloc(&s->loss, 4) || cudaMalloc(&s->stats, 16) ||
        cudaMalloc(&s->nbr, (size_t)s->n * sizeof(int4)) || cudaMalloc(&s->emb_cnt, (size_t)s->n * 4) ||
        cudaMalloc(&s->emb_off, ((size_t)s->n + 1) * 4) || cudaMalloc(&s->emb_cur, (size_t)s->n * 4) ||
        cudaMalloc(&s->emb_blk, ((size_t)(s->n + 1023) / 1024 + 1) * 4) || cudaMalloc(&s->rstats, 6 * sizeof(double))) {
        cudaGetLastError();
        return bail(gapa_fail(GAPA_ERR_OOM, "surrogate parameters"));
    }
    // degrees (original ids) from the uploaded CSR
    std::vector<int32_t> rp((size_t)s->n + 1);
    if (cudaMemcpy(rp.data(), ctx->g.row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bail(gapa_fail(GAPA_ERR_CUDA, "reading degrees"));
    std::vector<float> lg(s->n), dg(s->n);
    for (int v = 0; v < s->n; ++v) {
        dg[v] = (float)(rp[v + 1] - rp[v]);
        lg[v] = (float)std::log1p((double)dg[v]);
    }
    s->inv2E = ctx->g.num_edges > 0 ? (float)(1.0 / (2.0 * ctx->g.num_edges)) : 0.f;
    cudaMemcpy(s->logdeg, lg.data(), lg.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(s->deg, dg.data(), dg.size() * 4, cudaMemcpyHostToDevice);
    cudaStream_t st = ctx->stream;
    nbr_table_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(s->row_ptr, s->col, s->n, s->nbr);
    cudaMemsetAsync(s->P, 0, np * 4, st);
    cudaMemsetAsync(s->M, 0, np * 4, st);
    cudaMemsetAsync(s->V, 0, np * 4, st);
    cudaMemsetAsync(s->Gi, 0, (size_t)s->n * kEmb * 8, st);
    const double unit_stats[2] = {0.0, 1.0};  // targets before the first training step: identity
    cudaMemcpy(s->stats, unit_stats, sizeof unit_stats, cudaMemcpyHostToDevice);
    const int grid = ctx->num_sms * 4;
    init_uniform_kernel<<<grid, 256, 0, st>>>(s->P + s->L.W1, (size_t)kIn * kHid, sqrtf(6.f / kIn), s->key, 1);
    init_uniform_kernel<<<grid, 256, 0, st>>>(s->P + s->L.W2, (size_t)kHid * kHid, sqrtf(6.f / kHid), s->key, 2);
    init_uniform_kernel<<<grid, 256, 0, st>>>(s->P + s->L.w3, kHid, sqrtf(3.f / kHid), s->key, 3);
    init_uniform_kernel<<<grid, 256, 0, st>>>(s->P + s->L.E, (size_t)s->n * kEmb, scfg->init_scale_emb, s->key, 4);
    int rc = refresh_bf16(s, st);
    if (rc == GAPA_OK && cudaGetLastError() != cudaSuccess) rc = gapa_fail(GAPA_ERR_CUDA, "surrogate initialisation");
    if (rc == GAPA_OK) rc = ensure_rows(s, std::max(scfg->batch, 16));
    if (rc != GAPA_OK) return bail(rc);
    *out = s;
    return GAPA_OK;
}

void gapa_surrogate_destroy(gapa_surrogate* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();  // the context (and its stream) may already be gone
    free_surrogate(s);
    delete s;
}

int gapa_surrogate_predict(gapa_surrogate* s, const int32_t* pop_dev, int32_t rows, int32_t k, float* scores_dev) {
    if (!s || rows < 0 || k < 0 || (rows > 0 && (!pop_dev || !scores_dev))) return gapa_fail(GAPA_ERR_INVALID_ARG, "bad predict arguments");
    if (rows == 0) return GAPA_OK;
    cudaSetDevice(s->ctx->device);
    int rc = check_graph(s);
    if (rc == GAPA_OK) rc = ensure_rows(s, rows);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = s->ctx->stream;
    rc = forward(s, pop_dev, rows, k, false, st);
    if (rc != GAPA_OK) return rc;
    GAPA_CUDA(cudaMemcpyAsync(scores_dev, s->y, (size_t)rows * 4, cudaMemcpyDeviceToDevice, st));
    return GAPA_OK;
}

int gapa_surrogate_residual(gapa_surrogate* s, const int32_t* pop_dev, int32_t rows, int32_t k, int32_t* counts_dev) {
    // counts_dev: [rows][3] (the kernel's rows carry a fourth, unused lane)
    if (!s || rows < 0 || k < 0 || (rows > 0 && (!pop_dev || !counts_dev)))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "bad residual arguments");
    if (rows == 0) return GAPA_OK;
    cudaSetDevice(s->ctx->device);
    int rc = check_graph(s);
    if (rc == GAPA_OK) rc = ensure_rows(s, rows);
    if (rc == GAPA_OK) rc = compute_resid(s, pop_dev, rows, k, s->ctx->stream);
    if (rc != GAPA_OK) return rc;
    GAPA_CUDA(cudaMemcpy2DAsync(counts_dev, 3 * sizeof(int32_t), s->resid, sizeof(ResidRow), 3 * sizeof(int32_t),
                                (size_t)rows, cudaMemcpyDeviceToDevice, s->ctx->stream));
    return GAPA_OK;
}

int gapa_surrogate_train_step(gapa_surrogate* s, const int32_t* pop_dev, int32_t rows, int32_t k,
                              const float* target_dev, float* loss_host) {
    if (!s || rows < 16 || rows % 16 || k < 1 || !pop_dev || !target_dev)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "training batches need a multiple of 16 rows and k >= 1");
    cudaSetDevice(s->ctx->device);
    int rc = check_graph(s);
    if (rc == GAPA_OK) rc = ensure_rows(s, rows);
    if (rc != GAPA_OK) return rc;
    cudaStream_t st = s->ctx->stream;
    rc = train_step(s, pop_dev, rows, k, target_dev, st);
    if (rc != GAPA_OK) return rc;
    if (loss_host) {
        GAPA_CUDA(cudaMemcpyAsync(loss_host, s->loss, 4, cudaMemcpyDeviceToHost, st));
        GAPA_CUDA(cudaStreamSynchronize(st));
    }
    return GAPA_OK;
}

int gapa_surrogate_tensor(gapa_surrogate* s, int32_t which, int32_t grad, float* host, int64_t count, int32_t set) {
    if (!s || !host || which < 0 || which > 6) return gapa_fail(GAPA_ERR_INVALID_ARG, "bad tensor arguments");
    const Layout& L = s->L;
    const size_t offs[] = {L.W1, L.b1, L.W2, L.b2, L.w3, L.b3, L.E};
    const size_t sizes[] = {(size_t)kIn * kHid, kHid, (size_t)kHid * kHid, kHid, kHid, 1, (size_t)s->n * kEmb};
    if ((size_t)count != sizes[which]) return gapa_fail(GAPA_ERR_INVALID_ARG, "tensor %d holds %zu values", which, sizes[which]);
    cudaSetDevice(s->ctx->device);
    float* base = (grad ? s->G : s->P) + offs[which];
    cudaStream_t st = s->ctx->stream;
    if (grad && which == 6 && !set)  // the embedding gradient lives in fixed point until asked for
        emb_grad_float_kernel<<<s->ctx->num_sms * 4, 256, 0, st>>>(s->Gi, base, sizes[which]);
    if (set) {
        GAPA_CUDA(cudaMemcpyAsync(base, host, sizes[which] * 4, cudaMemcpyHostToDevice, st));
        if (!grad) {
            int rc = refresh_bf16(s, st);
            if (rc != GAPA_OK) return rc;
        }
    } else {
        GAPA_CUDA(cudaMemcpyAsync(host, base, sizes[which] * 4, cudaMemcpyDeviceToHost, st));
    }
    GAPA_CUDA(cudaStreamSynchronize(st));
    return GAPA_OK;
}

int gapa_run_surrogate(gapa_ctx* c, const gapa_config* cfg, gapa_surrogate* s, int64_t* best_fit_host,
                       int32_t* best_set_host, int64_t* traj_host, double* gen_ms_host, int64_t* exact_evals_host,
                       float* diag_pred_host, int64_t* diag_exact_host, int32_t diag_cap) {
    if (!c || !cfg || !best_fit_host) return gapa_fail(GAPA_ERR_INVALID_ARG, "NULL argument");
    if (!(cfg->flags & GAPA_FLAG_MU_PLUS_LAMBDA) || cfg->lambda < 1)
        return gapa_fail(GAPA_ERR_INVALID_ARG, "surrogate runs use (mu+lambda) with lambda >= 1");
    if (s && s->ctx != c) return gapa_fail(GAPA_ERR_INVALID_ARG, "surrogate belongs to another context");
    if (s && check_graph(s) != GAPA_OK) return GAPA_ERR_STATE;
    if (s && s->cfg.ring < std::max(cfg->pop, cfg->lambda))
        return gapa_fail(GAPA_ERR_INVALID_ARG, "the replay ring must hold at least max(mu, lambda) rows");
    cudaSetDevice(c->device);
    const int mu = cfg->pop, lam = cfg->lambda, k = cfg->k, G = cfg->gens;
    const int screened = s ? std::min(s->cfg.screened, lam) : lam;
    // the generation machinery of gapa_run: init, fitness, and the (mu+lambda) step pieces
    gapa_config c2 = *cfg;
    int rc = gapa_run_prepare(c, &c2);
    if (rc != GAPA_OK) return rc;
    // the run goes on the context's own stream (a stream that can be captured), ordered after the
    // caller's pending work and before the caller's later work
    cudaStream_t st = c->own_stream;
    GAPA_CUDA(cudaEventRecord(c->ev_a, c->stream));
    GAPA_CUDA(cudaStreamWaitEvent(st, c->ev_a, 0));
    int32_t* P[2] = {c->stage_pop[0], c->stage_pop[1]};
    int64_t* F[2] = {c->stage_fit[0], c->stage_fit[1]};
    // surrogate buffers
    int32_t *ring = nullptr, *sel = nullptr, *sel_rows = nullptr, *batch_rows = nullptr;
    int64_t* fsel = nullptr;
    double* ring_lp = nullptr;  // log1p(exact fitness) of every ring row (mode 1: its sibling z-score)
    double* gstats = nullptr;   // (mean, std) of log1p(fitness) over the last appended generation
    ResidRow *ring_resid = nullptr, *sel_resid = nullptr, *batch_resid = nullptr;
    float* scores = nullptr;
    const int ring_cap = s ? s->cfg.ring : 0;
    auto cleanup = [&]() {
        cudaFree(ring);
        cudaFree(sel);
        cudaFree(sel_rows);
        cudaFree(batch_rows);
        cudaFree(ring_lp);
        cudaFree(gstats);
        cudaFree(fsel);
        cudaFree(scores);
        cudaFree(ring_resid);
        cudaFree(sel_resid);
        cudaFree(batch_resid);
    };
    if (cudaMalloc(&sel, (size_t)lam * 4) || cudaMalloc(&sel_rows, (size_t)lam * k * 4 + 4) ||
        cudaMalloc(&fsel, (size_t)lam * 8) || cudaMalloc(&scores, (size_t)lam * 4) ||
        (s && (cudaMalloc(&ring, (size_t)ring_cap * k * 4 + 4) || cudaMalloc(&ring_lp, (size_t)ring_cap * 8) || cudaMalloc(&gstats, 16) ||
               cudaMalloc(&batch_rows, (size_t)s->cfg.batch * k * 4 + 4) ||
               cudaMalloc(&ring_resid, (size_t)ring_cap * sizeof(ResidRow)) ||
               cudaMalloc(&sel_resid, (size_t)lam * sizeof(ResidRow)) ||
               cudaMalloc(&batch_resid, (size_t)s->cfg.batch * sizeof(ResidRow))))) {
        cudaGetLastError();
        cleanup();
        return gapa_fail(GAPA_ERR_OOM, "surrogate run buffers");
    }
    if (s && ((rc = ensure_rows(s, std::max(lam, s->cfg.batch))) != GAPA_OK ||
              (rc = ensure_csr(s, (size_t)s->cfg.batch * k, s->cfg.batch)) != GAPA_OK)) {
        cleanup();
        return rc;
    }
    int topk_P = 1;
    while (topk_P < lam) topk_P <<= 1;
    if ((size_t)topk_P * 8 > 48 * 1024) {
        cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(topk_P * 8));
    }
    std::vector<cudaEvent_t> ev((size_t)G + 2);
    for (auto& e : ev) cudaEventCreate(&e);
    std::vector<int64_t> exact((size_t)G + 1, 0);
    int ring_pos = 0, ring_valid = 0, diag_rows = 0;
    // the ring position, its valid rows and the AdamW step count live on the device (dstate[0..2]),
    // with the bias corrections of every step of this run in a table, so that a generation can be
    // replayed from a CUDA graph; the host keeps shadows for its own decisions
    int* dstate = nullptr;
    float2* bc_table = nullptr;
    const int steps_max = s ? G * std::max(s->cfg.train_steps, 0) : 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    auto fail = [&](int code) {
        for (auto e : ev) cudaEventDestroy(e);
        for (auto x : gexec)
            if (x) cudaGraphExecDestroy(x);
        cudaFree(dstate);
        cudaFree(bc_table);
        cleanup();
        return code;
    };
    if (s) {
        const int t0 = s->tau;
        std::vector<float2> tab((size_t)t0 + steps_max + 2, make_float2(1.f, 1.f));
        for (int t = 1; t < (int)tab.size(); ++t)
            tab[t] = make_float2(1.f - powf(s->cfg.beta1, (float)t), 1.f - powf(s->cfg.beta2, (float)t));
        if (cudaMalloc(&dstate, 16 + sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&bc_table, tab.size() * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(gapa_fail(GAPA_ERR_OOM, "surrogate run state"));
        }
        const int st0[4] = {0, 0, t0, 0};
        GAPA_CUDA(cudaMemcpyAsync(dstate, st0, 16, cudaMemcpyHostToDevice, st));
        GAPA_CUDA(cudaMemcpyAsync(bc_table, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    }
    float2* bc_dev = dstate ? reinterpret_cast<float2*>(dstate + 4) : nullptr;
    // rows (and their residual counts and exact fitness) enter the ring at the device's ring position
    auto ring_append = [&](const int32_t* rows, const ResidRow* rr, const int64_t* f, int cnt) {
        gather_rows_kernel<<<cnt, 256, 0, st>>>(rows, rr, nullptr, k, ring, ring_resid, 0, ring_cap, dstate);
        ring_target_kernel<<<1, 1024, 0, st>>>(f, cnt, s->cfg.target_mode, ring_lp, 0, ring_cap, gstats, dstate);
        ring_advance_kernel<<<1, 1, 0, st>>>(dstate, cnt, ring_cap);
        ring_pos = (ring_pos + cnt) % ring_cap;
        ring_valid = std::min(ring_cap, ring_valid + cnt);
    };
    GAPA_CUDA(cudaEventRecord(ev[0], st));
    GAPA_CUDA(cudaMemsetAsync(c->run_gen, 0, sizeof(int), st));
    const GaParams p0 = gapa_make_params(c, &c2, 0, nullptr);
    rc = gapa_launch_init(c, p0, P[0], st);
    if (rc == GAPA_OK) rc = gapa_launch_fitness(c, P[0], mu, k, F[0], st);
    if (rc == GAPA_OK) rc = gapa_launch_record(c, F[0], mu, c->run_gen, c->run_traj, c->run_best, st);
    if (rc != GAPA_OK) return fail(rc);
    exact[0] = mu;
    if (s) {  // the initial population enters the ring
        if ((rc = compute_resid(s, P[0], mu, k, st)) != GAPA_OK) return fail(rc);
        ring_append(P[0], s->resid, F[0], mu);
    }
    GAPA_CUDA(cudaEventRecord(ev[1], st));
    // One generation from P[cur] to P[cur ^ 1] (the generation index from the device counter).
    auto generation = [&](int g, int cur, bool screen, bool diag, int* evaluated_out) -> int {
        GaParams p = gapa_make_params(c, &c2, g, c->run_gen);
        int rc2 = GAPA_OK;
        if (p.flags & GAPA_FLAG_ROULETTE) {
            rc2 = gapa_launch_roulette_prefix(F[cur], mu, c->cum, st);
            p.cum = reinterpret_cast<const long long*>(c->cum);
        }
        if (rc2 == GAPA_OK) rc2 = gapa_launch_children(c, p, lam, P[cur], F[cur], c->kids, st);
        if (rc2 != GAPA_OK) return rc2;
        int evaluated = lam;
        if (screen || diag) rc2 = forward(s, c->kids, lam, k, false, st);
        else if (s) rc2 = compute_resid(s, c->kids, lam, k, st);  // for the ring
        if (rc2 == GAPA_OK && screen && !diag) {
            {
                ProfileScope prof(c, st, 2, 2);
                topk_kernel<<<1, 1024, (size_t)topk_P * 8, st>>>(s->y, lam, screened, sel, topk_P);
                gather_rows_kernel<<<screened, 256, 0, st>>>(c->kids, s->resid, sel, k, sel_rows, sel_resid, 0, 0,
                                                             nullptr);
            }
            rc2 = gapa_launch_fitness(c, sel_rows, screened, k, fsel, st);
            {
                ProfileScope prof(c, st, 2, 1);
                scatter_fit_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const long long*>(fsel), sel, screened, lam,
                                                       reinterpret_cast<long long*>(c->kfit));
            }
            evaluated = screened;
        } else if (rc2 == GAPA_OK) {
            rc2 = gapa_launch_fitness(c, c->kids, lam, k, c->kfit, st);
        }
        if (rc2 != GAPA_OK) return rc2;
        *evaluated_out = evaluated;
        if (s) {  // evaluated children enter the ring
            ProfileScope prof(c, st, 2, 3);
            if (evaluated == lam) ring_append(c->kids, s->resid, c->kfit, lam);
            else ring_append(sel_rows, sel_resid, fsel, evaluated);
        }
        if (diag) {
            // diagnostic generation: every child was evaluated exactly (and is used by the
            // truncation); record (estimate, fitness) pairs.  In target mode 1 the estimate
            // de-normalises with the statistics of this generation's children.
            decode_kernel<<<(lam + 255) / 256, 256, 0, st>>>(s->y, lam, s->cfg.target_mode == 1 ? gstats : s->stats,
                                                             scores);
            GAPA_CUDA(cudaMemcpyAsync(diag_pred_host + diag_rows, scores, (size_t)lam * 4, cudaMemcpyDeviceToHost, st));
            GAPA_CUDA(cudaMemcpyAsync(diag_exact_host + diag_rows, c->kfit, (size_t)lam * 8, cudaMemcpyDeviceToHost, st));
            diag_rows += lam;
        }
        rc2 = gapa_launch_mpl_replace(c, mu, lam, k, P[cur], F[cur], c->kids, c->kfit, c->src, P[cur ^ 1], F[cur ^ 1],
                                      st);
        if (rc2 == GAPA_OK) rc2 = gapa_launch_record(c, F[cur ^ 1], mu, c->run_gen, c->run_traj, c->run_best, st);
        // online training on the ring
        if (rc2 == GAPA_OK && s && ring_valid >= s->cfg.batch && s->cfg.train_steps > 0) {
            if (s->cfg.target_mode == 0) {  // mode 1 keeps the identity statistics
                ProfileScope prof(c, st, 2, 1);
                target_stats_kernel<<<1, 1024, 0, st>>>(ring_lp, ring_valid, s->stats, dstate + 1);
            }
            for (int step = 0; step < s->cfg.train_steps && rc2 == GAPA_OK; ++step) {
                {
                    ProfileScope prof(c, st, 2, 1);
                    batch_kernel<<<s->cfg.batch, 256, 0, st>>>(ring, ring_resid, ring_lp, ring_valid, k, s->cfg.batch,
                                                               s->key, step, g, s->stats, batch_rows, batch_resid,
                                                               s->tbuf, dstate + 1, c->run_gen);
                }
                rc2 = train_step(s, batch_rows, s->cfg.batch, k, s->tbuf, st, batch_resid, dstate + 2, bc_table,
                                 bc_dev);
            }
        }
        return rc2;
    };
    int cur = 0;
    for (int g = 1; g <= G && rc == GAPA_OK; ++g) {
        const bool screen = s && g > s->cfg.warmup && screened < lam;
        const bool diag = s && s->cfg.diag_every > 0 && g % s->cfg.diag_every == 0 && diag_pred_host &&
                          diag_exact_host && diag_rows + lam <= diag_cap;
        // a screened generation that trains, once the ring holds a batch, is the same launch sequence
        // every time: it is captured once per buffer parity and replayed (not while profiling, whose
        // events go around single launches)
        const bool steady = screen && !diag && ring_valid >= s->cfg.batch && s->cfg.train_steps > 0 &&
                            !(cfg->flags & GAPA_FLAG_ROULETTE) && !c->profiling;
        int evaluated = lam;
        if (steady) {
            if (!gexec[cur]) {
                cudaGraph_t graph = nullptr;
                const int shadow_pos = ring_pos, shadow_valid = ring_valid, shadow_tau = s->tau;
                const cudaError_t be = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                if (be != cudaSuccess) {
                    rc = gapa_cuda_fail(be, "capture of a screened generation");
                    break;
                }
                c->capturing = true;
                int crc = generation(g, cur, true, false, &evaluated);
                cudaError_t ce = cudaStreamEndCapture(st, &graph);
                c->capturing = false;
                // capture ran no work: restore the host shadows it advanced
                ring_pos = shadow_pos;
                ring_valid = shadow_valid;
                s->tau = shadow_tau;
                if (crc != GAPA_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    rc = crc;
                    break;
                }
                if (ce == cudaSuccess) ce = cudaGraphInstantiate(&gexec[cur], graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (ce != cudaSuccess) {
                    rc = gapa_cuda_fail(ce, "capture of a screened generation");
                    break;
                }
            }
            const cudaError_t ce = cudaGraphLaunch(gexec[cur], st);
            if (ce != cudaSuccess) {
                rc = gapa_cuda_fail(ce, "replay of a screened generation");
                break;
            }
            evaluated = screened;
            ring_pos = (ring_pos + evaluated) % ring_cap;
            ring_valid = std::min(ring_cap, ring_valid + evaluated);
            s->tau += s->cfg.train_steps;
        } else {
            rc = generation(g, cur, screen, diag, &evaluated);
            if (rc != GAPA_OK) break;
        }
        exact[g] = evaluated;
        cur ^= 1;
        if (cudaEventRecord(ev[(size_t)g + 1], st) != cudaSuccess) rc = gapa_fail(GAPA_ERR_CUDA, "event record");
    }
    for (auto& x : gexec)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    if (rc != GAPA_OK) return fail(rc);
    GAPA_CUDA(cudaStreamSynchronize(st));
    int best = 0;
    GAPA_CUDA(cudaMemcpy(&best, c->run_best, sizeof(int), cudaMemcpyDeviceToHost));
    GAPA_CUDA(cudaMemcpy(best_fit_host, F[cur] + best, 8, cudaMemcpyDeviceToHost));
    if (best_set_host && k) {
        GAPA_CUDA(cudaMemcpy(best_set_host, P[cur] + (size_t)best * k, (size_t)k * 4, cudaMemcpyDeviceToHost));
        std::sort(best_set_host, best_set_host + k);
    }
    if (traj_host) GAPA_CUDA(cudaMemcpy(traj_host, c->run_traj, 8 * ((size_t)G + 1), cudaMemcpyDeviceToHost));
    if (gen_ms_host)
        for (int g = 0; g <= G; ++g) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[(size_t)g + 1]);
            gen_ms_host[g] = ms;
        }
    if (exact_evals_host)
        for (int g = 0; g <= G; ++g) exact_evals_host[g] = exact[g];
    int h = 0;
    cudaMemcpy(&h, c->status, 4, cudaMemcpyDeviceToHost);
    for (auto e : ev) cudaEventDestroy(e);
    cudaFree(dstate);
    cudaFree(bc_table);
    cleanup();
    // later work on the caller's stream comes after the run
    cudaEventRecord(c->ev_b, st);
    cudaStreamWaitEvent(c->stream, c->ev_b, 0);
    if (h) {
        cudaMemset(c->status, 0, 4);
        return gapa_fail(GAPA_ERR_DEVICE, "device status 0x%x", h);
    }
    return GAPA_OK;
}

}  // extern "C"
