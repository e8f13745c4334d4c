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
#include <cuda.h>

#include <algorithm>
#include <mutex>
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

// ---------------------------------------------------------------------------
// The same product on the 5th-generation tensor cores: tcgen05.mma
// kind::f8f6f4 (E4M3 x E4M3, FP32 accumulator in tensor memory), one elected
// thread issuing, operands in shared memory in the canonical K-major layout
// without swizzle (8-row x 16-byte core matrices; the next 16 bytes of K
// 128 bytes on, the next 8 rows 1024 bytes on), 128-byte k chunks in three
// stages filled by cp.async, each stage released by a tcgen05.commit on its
// mbarrier.  Every wait is bounded: on expiry the kernel records
// GAPA_DEV_TIMEOUT, still waits (bounded) for its own products and frees its
// tensor memory.  A CTA of 4 warps owns one 128 x 128 tile; warp w reads
// accumulator lanes 32w .. 32w + 31 (rows) back with tcgen05.ld.
// ---------------------------------------------------------------------------
constexpr int kT5Chunk = 128, kT5Stages = 3, kT5Threads = 128;
constexpr int kT5StageBytes = kTile * kT5Chunk;  // 16 KB per operand per stage
constexpr long long kT5SpinLimit = 1ll << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// K-major, no-swizzle shared-memory matrix descriptor: start, leading (K) and
// stride (8-row) byte offsets >> 4, descriptor version 1, layout type 0.
__device__ __forceinline__ unsigned long long t5_desc(unsigned addr) {
    const unsigned long long lbo = 128, sbo = 1024;
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFull) << 16) |
           (((sbo >> 4) & 0x3FFFull) << 32) | (1ull << 46);
}

// instruction descriptor: FP32 accumulator, A and B E4M3, both K-major, N = 128, M = 128
constexpr unsigned kT5Idesc = (1u << 4) | ((unsigned)(kTile >> 3) << 17) | ((unsigned)(kTile >> 4) << 24);

__device__ __forceinline__ bool t5_wait(unsigned bar, unsigned parity, long long limit = kT5SpinLimit) {
    for (long long i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kT5Threads) sdst_gemm_t5_kernel(const unsigned char* __restrict__ X,
                                                                  const unsigned char* __restrict__ Y,
                                                                  unsigned char* __restrict__ C, int np, size_t mat,
                                                                  int* status) {
    extern __shared__ __align__(16) unsigned char t5_smem[];
    unsigned char* sA = t5_smem;                                 // [stages][16 KB]
    unsigned char* sB = t5_smem + kT5Stages * kT5StageBytes;     // [stages][16 KB]
    __shared__ __align__(8) unsigned long long bars[kT5Stages];
    __shared__ unsigned tmem_base;
    __shared__ int failed;
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
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < kT5Stages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    // chunk -> stage: 128 rows x 8 pieces of 16 bytes per operand, piece (row, q) at
    // (row / 8) * 1024 + q * 128 + (row % 8) * 16
    auto load = [&](int chunk) {
        const int st = chunk % kT5Stages, k0 = chunk * kT5Chunk;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int piece = tid + r * kT5Threads, row = piece >> 3, q = piece & 7;
            const int so = (row >> 3) * 1024 + q * 128 + (row & 7) * 16;
            cp_async16(sA + st * kT5StageBytes + so, x + (size_t)row * np + k0 + q * 16);
            cp_async16(sB + st * kT5StageBytes + so, y + (size_t)row * np + k0 + q * 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int chunks = np / kT5Chunk;
    load(0);
    if (chunks > 1) load(1);
    int issued = -1;  // last chunk whose products were committed
    for (int c = 0; c < chunks; ++c) {
        const int st = c % kT5Stages;
        if (c + 2 < chunks) {
            // the stage of chunk c + 2 was last read by the products of chunk c - 1: one thread
            // waits for them (bounded) and the outcome goes to all
            if (c >= 1) {
                if (tid == 0 &&
                    !t5_wait(smem_u32(&bars[(c + 2) % kT5Stages]), (unsigned)(((c - 1) / kT5Stages) & 1)))
                    failed = 1;
                __syncthreads();
                if (failed) break;
            }
            load(c + 2);
            asm volatile("cp.async.wait_group 2;" ::: "memory");
        } else if (c + 1 < chunks) {
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = smem_u32(sA + st * kT5StageBytes), b0 = smem_u32(sB + st * kT5StageBytes);
#pragma unroll
            for (int j = 0; j < kT5Chunk / 32; ++j) {
                const unsigned long long da = t5_desc(a0 + 256u * j), db = t5_desc(b0 + 256u * j);
                const unsigned acc = (c > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(da), "l"(db), "r"(kT5Idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[st]))
                         : "memory");
        }
        issued = c;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last commit covers every product issued before it; one thread waits (bounded)
    if (tid == 0 && issued >= 0 && !t5_wait(smem_u32(&bars[issued % kT5Stages]), (unsigned)((issued / kT5Stages) & 1)))
        failed = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (failed) {
        if (tid == 0) {
            atomicOr(status, GAPA_DEV_TIMEOUT);
            // the products in flight must end before their tensor memory is freed: wait once more (bounded)
            if (issued >= 0) t5_wait(smem_u32(&bars[issued % kT5Stages]), (unsigned)((issued / kT5Stages) & 1));
        }
    } else {
        unsigned char* c = C + off;
        const int row = ty * kTile + warp * 32 + lane;
#pragma unroll
        for (int q = 0; q < kTile / 32; ++q) {
            unsigned v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(q * 32)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            unsigned w[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                unsigned word = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    word |= (__uint_as_float(v[4 * b + e]) > 0.5f ? (unsigned)kOne : 0u) << (8 * e);
                w[b] = word;
            }
            const int col0 = tx * kTile + q * 32;
            uint4* dst = reinterpret_cast<uint4*>(c + (size_t)row * np + col0);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
            if (tx != ty)  // the mirrored tile below the diagonal: column -> row
#pragma unroll
                for (int e = 0; e < 32; ++e) c[(size_t)(col0 + e) * np + row] = (unsigned char)(w[e >> 2] >> (8 * (e & 3)));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTile) : "memory");
}

// ---------------------------------------------------------------------------
// 256 x 256 tiles (np a multiple of 256): the same tcgen05 product with twice
// the tile edge, so each strip streamed from L2 feeds twice the outputs.  A
// CTA of 8 warps owns one tile; per 32-byte k step one thread issues two
// M = 128, N = 256 products (rows 0-127 and 128-255 of the tile against all
// 256 columns) into two accumulators of 256 tensor-memory columns each (512
// in all).  Stages: 128-byte k chunks of both 256-row strips (64 KB per
// stage, three stages, cp.async), released by tcgen05.commit on their
// mbarriers; every wait bounded as above.  Epilogue: warp w reads lane
// quarter w % 4 of both accumulators for column half w / 4, writes its rows
// of the tile to global memory and its 0/1 bytes to a shared-memory copy of
// the tile (the stages are free by then), from which an off-diagonal tile's
// mirror below the diagonal is written with 16-byte stores.
// ---------------------------------------------------------------------------
constexpr int kT6Tile = 256, kT6Threads = 256;
constexpr int kT6StageBytes = kT6Tile * kT5Chunk;  // 32 KB per operand per stage
constexpr int kT6Smem = 2 * kT5Stages * kT6StageBytes;  // 192 KB (the epilogue's 64 KB tile reuses it)
// instruction descriptor: FP32 accumulator, A and B E4M3, both K-major, N = 256, M = 128
constexpr unsigned kT6Idesc = (1u << 4) | ((unsigned)(kT6Tile >> 3) << 17) | ((unsigned)(128 >> 4) << 24);

__global__ void __launch_bounds__(kT6Threads) sdst_gemm_t6_kernel(const unsigned char* __restrict__ X,
                                                                  const unsigned char* __restrict__ Y,
                                                                  unsigned char* __restrict__ C, int np, size_t mat,
                                                                  int* status) {
    extern __shared__ __align__(16) unsigned char t6_smem[];
    unsigned char* sA = t6_smem;                                 // [stages][32 KB]
    unsigned char* sB = t6_smem + kT5Stages * kT6StageBytes;     // [stages][32 KB]
    __shared__ __align__(8) unsigned long long bars[kT5Stages];
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    const int T = np / kT6Tile;
    int ty = 0, rem = (int)blockIdx.x;
    while (rem >= T - ty) {
        rem -= T - ty;
        ++ty;
    }
    const int tx = ty + rem;
    const size_t off = (size_t)blockIdx.y * mat;
    const unsigned char* x = X + off + (size_t)ty * kT6Tile * np;
    const unsigned char* y = Y + off + (size_t)tx * kT6Tile * np;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < kT5Stages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kT6Tile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    // chunk -> stage: 256 rows x 8 pieces of 16 bytes per operand, piece (row, q) at
    // (row / 8) * 1024 + q * 128 + (row % 8) * 16
    auto load = [&](int chunk) {
        const int st = chunk % kT5Stages, k0 = chunk * kT5Chunk;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int piece = tid + r * kT6Threads, row = piece >> 3, q = piece & 7;
            const int so = (row >> 3) * 1024 + q * 128 + (row & 7) * 16;
            cp_async16(sA + st * kT6StageBytes + so, x + (size_t)row * np + k0 + q * 16);
            cp_async16(sB + st * kT6StageBytes + so, y + (size_t)row * np + k0 + q * 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int chunks = np / kT5Chunk;
    load(0);
    if (chunks > 1) load(1);
    int issued = -1;
    for (int c = 0; c < chunks; ++c) {
        const int st = c % kT5Stages;
        if (c + 2 < chunks) {
            if (c >= 1) {
                if (tid == 0 &&
                    !t5_wait(smem_u32(&bars[(c + 2) % kT5Stages]), (unsigned)(((c - 1) / kT5Stages) & 1)))
                    failed = 1;
                __syncthreads();
                if (failed) break;
            }
            load(c + 2);
            asm volatile("cp.async.wait_group 2;" ::: "memory");
        } else if (c + 1 < chunks) {
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned a0 = smem_u32(sA + st * kT6StageBytes), b0 = smem_u32(sB + st * kT6StageBytes);
#pragma unroll
            for (int j = 0; j < kT5Chunk / 32; ++j) {
                const unsigned long long db = t5_desc(b0 + 256u * j);
                const unsigned acc = (c > 0 || j > 0) ? 1u : 0u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {  // tile rows 128h .. 128h + 127: 16 groups of 8 rows on
                    const unsigned long long da = t5_desc(a0 + 16u * 1024u * h + 256u * j);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                        ::"r"(tmem + (unsigned)(h * kT6Tile)), "l"(da), "l"(db), "r"(kT6Idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bars[st]))
                         : "memory");
        }
        issued = c;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0 && issued >= 0 && !t5_wait(smem_u32(&bars[issued % kT5Stages]), (unsigned)((issued / kT5Stages) & 1)))
        failed = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (failed) {
        if (tid == 0) {
            atomicOr(status, GAPA_DEV_TIMEOUT);
            if (issued >= 0) t5_wait(smem_u32(&bars[issued % kT5Stages]), (unsigned)((issued / kT5Stages) & 1));
        }
    } else {
        unsigned char* c = C + off;
        unsigned char* tile = t6_smem;  // [256 rows][256 bytes], the stages being free
        const int quarter = warp & 3, half = warp >> 2;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int trow = h * 128 + quarter * 32 + lane;  // row within the tile
            const int row = ty * kT6Tile + trow;
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int tcol = half * 128 + q * 32;
                unsigned v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(h * kT6Tile + tcol)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    unsigned word = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        word |= (__uint_as_float(v[4 * b + e]) > 0.5f ? (unsigned)kOne : 0u) << (8 * e);
                    w[b] = word;
                }
                uint4* dst = reinterpret_cast<uint4*>(c + (size_t)row * np + tx * kT6Tile + tcol);
                dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                if (tx != ty) {
                    uint4* t = reinterpret_cast<uint4*>(tile + trow * kT6Tile + tcol);
                    t[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    t[1] = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        }
        if (tx != ty) {
            // the mirror: global row tx * 256 + j, columns ty * 256 .. + 255 = tile column j.  A thread
            // gathers 32 bytes of one tile column (32 consecutive tile rows; the lanes of a warp take
            // consecutive columns, so each shared-memory read is 32 adjacent bytes) and stores them as
            // one 32-byte sector
            __syncthreads();
            for (int p = tid; p < kT6Tile * (kT6Tile / 32); p += kT6Threads) {
                const int j = p & (kT6Tile - 1), r0 = (p / kT6Tile) * 32;  // tile column j, rows r0 .. r0 + 31
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    unsigned word = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) word |= (unsigned)tile[(r0 + 4 * b + e) * kT6Tile + j] << (8 * e);
                    w[b] = word;
                }
                uint4* dst = reinterpret_cast<uint4*>(c + (size_t)(tx * kT6Tile + j) * np + ty * kT6Tile + r0);
                dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kT6Tile) : "memory");
}

// ---------------------------------------------------------------------------
// 256 x 256 tiles with tensor-memory-access (TMA) loads and split roles.  The
// operands are read by cp.async.bulk.tensor from a 3-D tensor map (columns,
// rows, members) in boxes of 128 bytes x 256 rows with the 128-byte swizzle:
// each 8-row group of a box is one 1024-byte swizzle atom (its 16-byte pieces
// permuted by row), which is the layout a K-major shared-memory descriptor
// with 128-byte swizzling reads (8-row groups 1024 bytes apart; a 32-byte K
// step advances the start address by 32 bytes inside the atom).  A stage
// holds a 128-byte K chunk of both 256-row strips (64 KB); three stages.
// Warp 0's first lane is the producer: it waits until a stage is free (its
// `empty` mbarrier, completed by the products' tcgen05.commit), announces
// the stage's bytes on its `full` mbarrier and issues the two boxes.  Warp
// 1's first lane issues the products as each stage fills (per 32-byte K step
// two M = 128, N = 256 products into two accumulators of 256 tensor-memory
// columns) and commits the stage back; a last commit completes `done`.  Then
// all eight warps run the epilogue of the 256 x 256 kernel above.  Every wait
// is bounded: on expiry the kernel records GAPA_DEV_TIMEOUT, waits (bounded)
// for every box and product it issued, frees its tensor memory and skips the
// epilogue.
// ---------------------------------------------------------------------------
constexpr int kT7Stages = 3, kT7Chunk = 128;
constexpr int kT7OperandBytes = kT6Tile * kT7Chunk;          // 32 KB per operand per stage
constexpr int kT7StageBytes = 2 * kT7OperandBytes;           // 64 KB
constexpr int kT7Smem = kT7Stages * kT7StageBytes + 1024;    // 192 KB + alignment (the epilogue's tile reuses it)

// K-major shared-memory descriptor with 128-byte swizzling: start address, leading byte offset
// (unused for this layout; 16), stride byte offset 1024 (the next 8-row atom), version 1, layout
// type 2 (128-byte swizzle).
__device__ __forceinline__ unsigned long long t7_desc(unsigned addr) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((unsigned long long)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void t7_load(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(kT6Threads, 1)
    sdst_gemm_t7_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                        unsigned char* __restrict__ C, int np, size_t mat, int* status) {
    extern __shared__ __align__(1024) unsigned char t7_smem[];
    __shared__ __align__(8) unsigned long long full[kT7Stages], empty[kT7Stages], done;
    __shared__ unsigned tmem_base;
    __shared__ int failed, loads_issued, chunks_used;
    const int T = np / kT6Tile;
    int ty = 0, rem = (int)blockIdx.x;
    while (rem >= T - ty) {
        rem -= T - ty;
        ++ty;
    }
    const int tx = ty + rem;
    const int member = (int)blockIdx.y;
    const size_t off = (size_t)member * mat;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunks = np / kT7Chunk;
    if (tid == 0) {
        failed = 0;
        loads_issued = 0;
        chunks_used = 0;
        for (int s = 0; s < kT7Stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kT6Tile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned base = (smem_u32(t7_smem) + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
    if (warp == 0 && lane == 0) {
        // producer
        int c = 0;
        for (; c < chunks; ++c) {
            const int s = c % kT7Stages, use = c / kT7Stages;
            if (c >= kT7Stages && !t5_wait(smem_u32(&empty[s]), (unsigned)((use - 1) & 1))) {
                failed = 1;
                break;
            }
            const unsigned fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kT7StageBytes)
                         : "memory");
            const unsigned sa = base + (unsigned)(s * kT7StageBytes), sb = sa + (unsigned)kT7OperandBytes;
            const int k0 = c * kT7Chunk;
            t7_load(sa, &mapX, k0, ty * kT6Tile, member, fb);
            t7_load(sb, &mapY, k0, tx * kT6Tile, member, fb);
        }
        loads_issued = c;
    } else if (warp == 1 && lane == 0) {
        // products
        int c = 0;
        for (; c < chunks; ++c) {
            const int s = c % kT7Stages;
            if (!t5_wait(smem_u32(&full[s]), (unsigned)((c / kT7Stages) & 1))) {
                failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sa = base + (unsigned)(s * kT7StageBytes), sb = sa + (unsigned)kT7OperandBytes;
#pragma unroll
            for (int j = 0; j < kT7Chunk / 32; ++j) {  // 32-byte K steps inside the 128-byte atoms
                const unsigned long long db = t7_desc(sb + 32u * (unsigned)j);
                const unsigned acc = (c > 0 || j > 0) ? 1u : 0u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {  // tile rows 128h .. 128h + 127: 16 atoms of 8 rows on
                    const unsigned long long da = t7_desc(sa + (unsigned)(h * 16 * 1024) + 32u * (unsigned)j);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                        ::"r"(tmem + (unsigned)(h * kT6Tile)), "l"(da), "l"(db), "r"(kT6Idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        chunks_used = c;
        // the last commit tracks every product issued before it
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    __syncthreads();
    if (tid == 0) {
        if (!t5_wait(smem_u32(&done), 0u)) failed = 1;
        if (failed) {
            atomicOr(status, GAPA_DEV_TIMEOUT);
            // every box issued must land before the shared memory is released: wait (bounded) for the
            // stages loaded but not consumed, then for the products once more
            for (int c = chunks_used; c < loads_issued; ++c)
                t5_wait(smem_u32(&full[c % kT7Stages]), (unsigned)((c / kT7Stages) & 1));
            t5_wait(smem_u32(&done), 0u);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!failed) {
        unsigned char* c = C + off;
        unsigned char* tile = t7_smem + (base - smem_u32(t7_smem));  // [256 rows][256 bytes], the stages being free
        const int quarter = warp & 3, half = warp >> 2;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int trow = h * 128 + quarter * 32 + lane;  // row within the tile
            const int row = ty * kT6Tile + trow;
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int tcol = half * 128 + q * 32;
                unsigned v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(h * kT6Tile + tcol)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    unsigned word = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        word |= (__uint_as_float(v[4 * b + e]) > 0.5f ? (unsigned)kOne : 0u) << (8 * e);
                    w[b] = word;
                }
                uint4* dst = reinterpret_cast<uint4*>(c + (size_t)row * np + tx * kT6Tile + tcol);
                dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                if (tx != ty) {
                    uint4* t = reinterpret_cast<uint4*>(tile + trow * kT6Tile + tcol);
                    t[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    t[1] = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        }
        if (tx != ty) {
            __syncthreads();
            for (int p = tid; p < kT6Tile * (kT6Tile / 32); p += kT6Threads) {
                const int j = p & (kT6Tile - 1), r0 = (p / kT6Tile) * 32;  // tile column j, rows r0 .. r0 + 31
                unsigned w[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    unsigned word = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) word |= (unsigned)tile[(r0 + 4 * b + e) * kT6Tile + j] << (8 * e);
                    w[b] = word;
                }
                uint4* dst = reinterpret_cast<uint4*>(c + (size_t)(tx * kT6Tile + j) * np + ty * kT6Tile + r0);
                dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kT6Tile) : "memory");
}

// A 3-D tensor map over `batch` members' np x np byte matrices (columns, rows, members) with
// boxes of 128 columns x 256 rows x 1 member and the 128-byte swizzle.  The encoder comes from the driver by
// its entry point (the library does not link the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn t7_encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

int t7_map(CUtensorMap* map, const unsigned char* buf, int np, int batch) {
    EncodeTiledFn enc = t7_encoder();
    if (!enc) return gapa_fail(GAPA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[3] = {(cuuint64_t)np, (cuuint64_t)np, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)np, (cuuint64_t)np * (cuuint64_t)np};  // bytes, dims 1 and 2
    const cuuint32_t box[3] = {(cuuint32_t)kT7Chunk, (cuuint32_t)kT6Tile, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<unsigned char*>(buf), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gapa_fail(GAPA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GAPA_OK;
}

// The bounded wait on an mbarrier that nothing completes: it must run out and
// report GAPA_DEV_TIMEOUT (gapa_selftest_wait).
__global__ void t5_selftest_kernel(long long limit, int* status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!t5_wait(smem_u32(&bar), 0u, limit)) atomicOr(status, GAPA_DEV_TIMEOUT);
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

int gapa_launch_selftest_wait(gapa_ctx* c, long long limit, cudaStream_t st) {
    t5_selftest_kernel<<<1, 32, 0, st>>>(limit, c->status);
    GAPA_CUDA(cudaGetLastError());
    return GAPA_OK;
}

int gapa_sixdst_init(gapa_ctx* c) {
    const int bytes = 2 * kT5Stages * kT5StageBytes;
    if ((size_t)bytes + 1024 > c->smem_optin) return GAPA_OK;  // the tcgen05 product stays unavailable
    GAPA_CUDA(cudaFuncSetAttribute(sdst_gemm_t5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    c->sixdst_t5_ok = true;
    c->sixdst_kernel = 1;
    if ((size_t)kT6Smem + 1024 <= c->smem_optin) {
        GAPA_CUDA(cudaFuncSetAttribute(sdst_gemm_t6_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kT6Smem));
        c->sixdst_t6_ok = true;
    }
    if ((size_t)kT7Smem + 1024 <= c->smem_optin && t7_encoder()) {
        GAPA_CUDA(cudaFuncSetAttribute(sdst_gemm_t7_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kT7Smem));
        c->sixdst_t7_ok = true;
        c->sixdst_kernel = GAPA_SIXDST_TMA;
    }
    return GAPA_OK;
}

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
        const bool t5 = c->sixdst_kernel >= 1;
        // 256-wide tiles where the padded size allows them; TMA loads with split roles by default
        const bool t7 = c->sixdst_kernel == GAPA_SIXDST_TMA && c->sixdst_t7_ok && np % kT6Tile == 0;
        const bool t6 = (c->sixdst_kernel == 1 || (c->sixdst_kernel == GAPA_SIXDST_TMA && !t7)) && c->sixdst_t6_ok &&
                        np % kT6Tile == 0;
        const int tiles6 = np / kT6Tile;
        const dim3 grid6(tiles6 * (tiles6 + 1) / 2, bm);
        int map_rc = GAPA_OK;
        auto launch_gemm = [&](const unsigned char* xa, const unsigned char* yb, unsigned char* cc) {
            if (t7) {
                CUtensorMap mx, my;
                if ((map_rc = t7_map(&mx, xa, np, bm)) != GAPA_OK || (map_rc = t7_map(&my, yb, np, bm)) != GAPA_OK)
                    return;
                sdst_gemm_t7_kernel<<<grid6, kT6Threads, kT7Smem, st>>>(mx, my, cc, np, mat, c->status);
            } else if (t6)
                sdst_gemm_t6_kernel<<<grid6, kT6Threads, kT6Smem, st>>>(xa, yb, cc, np, mat, c->status);
            else if (t5)
                sdst_gemm_t5_kernel<<<grid, kT5Threads, 2 * kT5Stages * kT5StageBytes, st>>>(xa, yb, cc, np, mat,
                                                                                             c->status);
            else
                sdst_gemm_kernel<<<grid, kThreads, 0, st>>>(xa, yb, cc, np, mat);
        };
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
                    launch_gemm(buf[res], buf[base], buf[dst]);
                    ++launched;
                    res = dst;
                }
            }
            if (e > 1) {
                const int dst = free_buf(res, base);
                launch_gemm(buf[base], buf[base], buf[dst]);
                ++launched;
                base = dst;
            }
        }
        if (map_rc != GAPA_OK) return map_rc;
        sdst_objective_kernel<<<bm, 256, 0, st>>>(buf[res], n, np, mat, words, dead,
                                                  c->objective == GAPA_OBJECTIVE_SIXDST_MCN ? 1 : 0,
                                                  reinterpret_cast<long long*>(fit) + m0);
        ++launched;
        GAPA_CUDA(cudaGetLastError());
    }
    if (kernels) *kernels = launched;
    return GAPA_OK;
}
