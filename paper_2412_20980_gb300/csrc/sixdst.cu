// SixDST dense reachability fitness (Section III-C, Eqs. 14-17).
//
// Per member: A = P^(A, p) (the deleted nodes' rows and columns zeroed), then
// M = Normalizer((A + I)^N), where Normalizer sets non-zero entries to 1, so
// M[v][u] = 1 exactly when u lies within N hops of v in G[V\D] (or u = v).
// Row sums of the live rows give the N-hop objectives:
//   PC_N  = (sum over live v of rowsum(v) - live) / 2,
//   MCN_N = max over live v of rowsum(v),
// equal to PC and MCN once N reaches every component's diameter (N = 6: the
// paper's six-degrees-of-separation fitness).
//
// The matrices are 0/1 in FP8 (E4M3: 1.0 and 0 are exact), n padded to a
// multiple of 128, one byte per entry.  (A + I)^N is formed by square and
// multiply, normalising after every product (the boolean result of the power
// does not depend on the order).  Each product runs on the tensor cores as
// mma.sync m16n8k32 E4M3 x E4M3 with FP32 accumulation: the sums are at most
// n, exact in FP32, so the normalised product is exact.  (A + I)^j is
// symmetric, so the "column-major" B operand is read from the rows of the
// right factor.
#include <algorithm>
#include <vector>

#include "gapa_internal.cuh"

namespace {

constexpr int kPad = 128;                // n padded to a multiple of this (the product tile)
constexpr unsigned char kOne = 0x38;     // 1.0 in E4M3

// deleted-node bitmap of every member of the batch: [members][words]
__global__ void sdst_dead_kernel(const int* __restrict__ pop, int k, int n, int words, unsigned* __restrict__ dead,
                                 int* status) {
    const int m = blockIdx.x;
    unsigned* d = dead + (size_t)m * words;
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = 0u;
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int v = __ldg(&pop[(size_t)m * k + j]);
        if ((unsigned)v < (unsigned)n)
            atomicOr(&d[v >> 5], 1u << (v & 31));
        else
            atomicOr(status, GAPA_DEV_BAD_GENE);
    }
}

// row v of member m's A + I: zeros, the diagonal for every v < n (the I term),
// and the live neighbours of a live v; padding rows stay zero
__global__ void __launch_bounds__(256) sdst_build_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                                         int n, int np, int words, const unsigned* __restrict__ dead,
                                                         unsigned char* __restrict__ X, size_t mat) {
    const int v = blockIdx.x, m = blockIdx.y;
    unsigned char* row = X + (size_t)m * mat + (size_t)v * np;
    for (int c = threadIdx.x * 16; c < np; c += blockDim.x * 16) *reinterpret_cast<uint4*>(row + c) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (v >= n) return;
    const unsigned* d = dead + (size_t)m * words;
    if (threadIdx.x == 0) row[v] = kOne;
    if ((d[v >> 5] >> (v & 31)) & 1u) return;
    for (int e = row_ptr[v] + threadIdx.x; e < row_ptr[v + 1]; e += blockDim.x) {
        const int u = col[e];
        if (!((d[u >> 5] >> (u & 31)) & 1u)) row[u] = kOne;
    }
}

__device__ __forceinline__ void mma_e4m3(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C = Normalizer(X Y) for every member of the batch (blockIdx.y); X, Y, C are
// np x np 0/1 E4M3 matrices, X and Y symmetric polynomials in A + I, so they
// commute and C is symmetric: only the tiles on or above the diagonal are
// computed (blockIdx.x enumerates them) and each is also stored transposed.
// A CTA of 8 warps computes a 128 x 128 tile, a warp 64 x 32 (4 x 4 m16n8
// tiles); 64-byte k chunks of both operands go through shared memory with
// cp.async in two stages (rows padded to 80 bytes: fragment reads are free of
// bank conflicts).
constexpr int kTile = 128, kChunk = 64, kRow = 80, kThreads = 256;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__global__ void __launch_bounds__(kThreads) sdst_gemm_kernel(const unsigned char* __restrict__ X,
                                                             const unsigned char* __restrict__ Y,
                                                             unsigned char* __restrict__ C, int np, size_t mat) {
    __shared__ __align__(16) unsigned char sA[2][kTile * kRow];
    __shared__ __align__(16) unsigned char sB[2][kTile * kRow];
    // upper-triangle tile (ty <= tx) of linear index blockIdx.x
    const int T = np / kTile;
    int ty = 0, rem = (int)blockIdx.x;
    while (rem >= T - ty) {
        rem -= T - ty;
        ++ty;
    }
    const int tx = ty + rem;
    const size_t off = (size_t)blockIdx.y * mat;
    const unsigned char* x = X + off + (size_t)ty * kTile * np;
    const unsigned char* y = Y + off + (size_t)tx * kTile * np;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
    const int wr = (warp >> 2) * 64, wc = (warp & 3) * 32;
    // loader: thread t copies 16-byte pieces t and t + 256 of each 128 x 64 chunk
    auto load = [&](int stage, int k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int piece = tid + r * kThreads, row = piece >> 2, c16 = (piece & 3) * 16;
            cp_async16(&sA[stage][row * kRow + c16], x + (size_t)row * np + k0 + c16);
            cp_async16(&sB[stage][row * kRow + c16], y + (size_t)row * np + k0 + c16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[i][j][u] = 0.f;
    const int chunks = np / kChunk;
    load(0, 0);
    for (int ch = 0; ch < chunks; ++ch) {
        const int st = ch & 1;
        if (ch + 1 < chunks) {
            load(st ^ 1, (ch + 1) * kChunk);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const unsigned char* a = sA[st];
        const unsigned char* bb = sB[st];
#pragma unroll
        for (int kk = 0; kk < kChunk; kk += 32) {
            unsigned af[4][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned char* r0 = a + (wr + 16 * i + g) * kRow + kk + tig * 4;
                af[i][0] = *reinterpret_cast<const unsigned*>(r0);
                af[i][1] = *reinterpret_cast<const unsigned*>(r0 + 8 * kRow);
                af[i][2] = *reinterpret_cast<const unsigned*>(r0 + 16);
                af[i][3] = *reinterpret_cast<const unsigned*>(r0 + 8 * kRow + 16);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned char* r0 = bb + (wc + 8 * j + g) * kRow + kk + tig * 4;
                bf[j][0] = *reinterpret_cast<const unsigned*>(r0);
                bf[j][1] = *reinterpret_cast<const unsigned*>(r0 + 16);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_e4m3(acc[i][j], af[i][0], af[i][1], af[i][2], af[i][3], bf[j][0], bf[j][1]);
        }
        __syncthreads();
    }
    unsigned char* c = C + off;
    const int R0 = ty * kTile + wr, C0 = tx * kTile + wc;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = R0 + 16 * i + g + 8 * h, colx = C0 + 8 * j + tig * 2;
                const unsigned char v0 = acc[i][j][2 * h] > 0.5f ? kOne : 0, v1 = acc[i][j][2 * h + 1] > 0.5f ? kOne : 0;
                *reinterpret_cast<unsigned short*>(c + (size_t)row * np + colx) = (unsigned short)(v0 | (v1 << 8));
                if (tx != ty) {  // the mirrored tile below the diagonal
                    c[(size_t)colx * np + row] = v0;
                    c[(size_t)(colx + 1) * np + row] = v1;
                }
            }
}

// per member: the live rows' non-zero counts, then PC_N (sum) or MCN_N (max)
__global__ void __launch_bounds__(256) sdst_objective_kernel(const unsigned char* __restrict__ M, int n, int np,
                                                             size_t mat, int words, const unsigned* __restrict__ dead,
                                                             int objective, long long* __restrict__ fit) {
    const int m = blockIdx.x;
    const unsigned char* mm = M + (size_t)m * mat;
    const unsigned* d = dead + (size_t)m * words;
    __shared__ long long red[8];
    long long acc = 0, live = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int v = warp; v < n; v += blockDim.x >> 5) {
        if ((d[v >> 5] >> (v & 31)) & 1u) continue;
        const unsigned char* row = mm + (size_t)v * np;
        int cnt = 0;
        for (int c = lane * 4; c < np; c += 128) {
            const unsigned w = *reinterpret_cast<const unsigned*>(row + c);
            cnt += ((w & 0xFFu) != 0) + ((w & 0xFF00u) != 0) + ((w & 0xFF0000u) != 0) + ((w & 0xFF000000u) != 0);
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if (lane == 0) {
            acc = objective ? (cnt > acc ? cnt : acc) : acc + cnt;
            live += 1;
        }
    }
    // lane 0 of each warp holds its part: combine in a fixed order
    if (lane == 0) red[warp] = acc;
    __shared__ long long red_live[8];
    if (lane == 0) red_live[warp] = live;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, l = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = objective ? (red[w] > a ? red[w] : a) : a + red[w];
            l += red_live[w];
        }
        fit[m] = objective ? a : (a - l) / 2;
    }
}

}  // namespace

int gapa_launch_fitness_sixdst(gapa_ctx* c, const int32_t* pop, int s, int k, int64_t* fit, cudaStream_t st,
                               int* kernels) {
    const int n = c->g.n;
    const int np = (n + kPad - 1) / kPad * kPad;
    if (np > 8192) return gapa_fail(GAPA_ERR_INVALID_ARG, "SixDST fitness needs n <= 8192 (n = %d)", n);
    const int hops = c->sixdst_hops;
    const size_t mat = (size_t)np * np;
    const int words = (np + 31) / 32;
    // members per batch: three matrices each, within 2 GiB
    int batch = (int)std::max<size_t>(1, ((size_t)2 << 30) / (3 * mat));
    batch = std::min(batch, std::max(s, 1));
    int rc = gapa_reserve(&c->sdst_buf, &c->sdst_cap, (size_t)batch * 3 * mat + (size_t)batch * words * 4, 1);
    if (rc != GAPA_OK) return rc;
    unsigned char* buf[3];
    for (int i = 0; i < 3; ++i) buf[i] = reinterpret_cast<unsigned char*>(c->sdst_buf) + (size_t)i * batch * mat;
    unsigned* dead = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(c->sdst_buf) + (size_t)3 * batch * mat);
    int launched = 0;
    for (int m0 = 0; m0 < s; m0 += batch) {
        const int bm = std::min(batch, s - m0);
        sdst_dead_kernel<<<bm, 256, 0, st>>>(pop + (size_t)m0 * k, k, n, words, dead, c->status);
        sdst_build_kernel<<<dim3(np, bm), 256, 0, st>>>(c->g.row_ptr, c->g.col, n, np, words, dead, buf[0], mat);
        launched += 2;
        // square and multiply: `base` holds (A+I)^(2^i), `res` the product of the bits seen so far
        int base = 0, res = -1;
        const int tiles = np / kTile;
        const dim3 grid(tiles * (tiles + 1) / 2, bm);
        auto free_buf = [&](int a, int b) {
            for (int i = 0; i < 3; ++i)
                if (i != a && i != b) return i;
            return -1;
        };
        for (int e = hops; e > 0; e >>= 1) {
            if (e & 1) {
                if (res < 0) {
                    res = base;
                } else {
                    const int dst = free_buf(res, base);
                    sdst_gemm_kernel<<<grid, kThreads, 0, st>>>(buf[res], buf[base], buf[dst], np, mat);
                    ++launched;
                    res = dst;
                }
            }
            if (e > 1) {
                const int dst = free_buf(res, base);
                sdst_gemm_kernel<<<grid, kThreads, 0, st>>>(buf[base], buf[base], buf[dst], np, mat);
                ++launched;
                base = dst;
            }
        }
        sdst_objective_kernel<<<bm, 256, 0, st>>>(buf[res], n, np, mat, words, dead,
                                                  c->objective == GAPA_OBJECTIVE_SIXDST_MCN ? 1 : 0,
                                                  reinterpret_cast<long long*>(fit) + m0);
        ++launched;
        GAPA_CUDA(cudaGetLastError());
    }
    if (kernels) *kernels = launched;
    return GAPA_OK;
}
