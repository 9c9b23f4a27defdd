// fs_mlp.cu - the surrogate MLP that ranks candidate PSO moves: 5 -> W -> W
// -> W -> 1 with ReLU hidden layers, bf16 weights and layer inputs, fp32
// accumulation, fp32 master weights trained with Adam.
//
// The hidden-layer products and their gradients run on the tensor cores
// through one templated bf16 GEMM (mma.sync m16n8k16, fp32 accumulators)
// with fused epilogues: bias + ReLU (forward), ReLU mask (backward through an
// activation) and plain fp32 (weight gradients).  The 5-wide input layer is
// padded to K = 16; the 1-wide output layer is a warp-per-row dot product.
// An optional tcgen05 path (TMEM accumulators) covers the same products.
//
// One fs_mlp holds a batch of G networks of one width laid end to end (the
// surrogate keeps one network per search box): every kernel of a forward or
// training pass covers all G in one launch, network g's rows and parameters
// sitting at fixed strides, with the same per-element summation order as a
// network run alone.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "fs_internal.h"

namespace fs {

using bf16 = __nv_bfloat16;

constexpr int kInPad = 16;   // input features padded to one mma K step

// ---------------------------------------------------------------------------
// C[M, N] = A[M, K] . B[N, K]^T  (bf16 in, fp32 accumulate)
//   TA: A stored [K][M] (element (m, k) at A[k * lda + m]) instead of [M][K]
//   TB: B stored [K][N] instead of [N][K]
// ---------------------------------------------------------------------------
enum Epi { EPI_BIAS_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_F32 = 2 };

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8, GEMM_THREADS = 128;
constexpr int kMaxSplits = 32;   // K chunks of the weight-gradient GEMMs

// A batch of G networks of the same shape stored back to back: the GEMM grid's
// z index is (network g, K chunk), and each operand advances by its stride (in
// elements) from one network to the next.
struct GS {
    int64_t a = 0, b = 0, bias = 0, mask = 0, out = 0;
    int splits = 1;
};

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A 64 x 32 operand tile (64 rows of the output's M or N side, 32 k) is 256
// chunks of 8 bf16 that are contiguous in memory, two per thread: with k
// contiguous (not TRANS), chunk e holds row e / 4, k (e % 4) * 8 .. + 8 (four
// threads cover a row's 64 bytes); with rows contiguous (TRANS), the chunk of
// thread t in round i holds k = lane / 2 + 16 i and rows 8 (lane % 2) + 16 warp
// .. + 8 (two threads cover a 32-byte sector, and the column stores into
// shared memory meet at most two to a bank). A chunk is one 16-byte load when
// `vec` (leading dimension a multiple of 8, base 16-byte aligned) and the
// chunk lies inside the operand; otherwise its elements are loaded one by one
// with bounds checks (zeros outside).
__device__ __forceinline__ unsigned short bits_of(bf16 v) { return __bfloat16_as_ushort(v); }

template <bool TRANS>
__device__ __forceinline__ void chunk_pos(int i, int& r, int& c) {
    const int t = threadIdx.x;
    if (!TRANS) {
        const int e = t + i * GEMM_THREADS;
        r = e >> 2;
        c = (e & 3) * 8;
    } else {
        const int lane = t & 31, warp = t >> 5;
        r = 8 * (lane & 1) + 16 * warp;
        c = (lane >> 1) + 16 * i;
    }
}

template <bool TRANS>
__device__ __forceinline__ void fetch_tile(uint4 (&v)[2], const bf16* __restrict__ G, int ld, int row0, int rows,
                                           int k0, int K, bool vec) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
        int r, c;
        chunk_pos<TRANS>(i, r, c);
        const int gr = row0 + r, gk = k0 + c;
        const bool full = TRANS ? (gk < K && gr + 8 <= rows) : (gr < rows && gk + 8 <= K);
        if (vec && full) {
            const bf16* src = TRANS ? G + (int64_t)gk * ld + gr : G + (int64_t)gr * ld + gk;
            v[i] = __ldg(reinterpret_cast<const uint4*>(src));
        } else {
            unsigned short h[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int rr = TRANS ? gr + j : gr, kk = TRANS ? gk : gk + j;
                h[j] = (rr < rows && kk < K) ? bits_of(G[(int64_t)(TRANS ? kk : rr) * ld + (TRANS ? rr : kk)]) : 0;
            }
            v[i] = make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                              h[6] | (uint32_t)h[7] << 16);
        }
    }
}

template <bool TRANS>
__device__ __forceinline__ void store_tile(bf16 (*S)[BK + PAD], const uint4 (&v)[2]) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
        int r, c;
        chunk_pos<TRANS>(i, r, c);
        if (!TRANS) {
            *reinterpret_cast<uint4*>(&S[r][c]) = v[i];
        } else {
            const uint32_t w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
            for (int j = 0; j < 8; j++)
                S[r + j][c] = __ushort_as_bfloat16((unsigned short)(w[j >> 1] >> (16 * (j & 1))));
        }
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS)
gemm_bf16_kernel(int M, int N, int K, const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb,
                 const float* __restrict__ bias, const bf16* __restrict__ mask, int ldm, void* out, int ldo,
                 int kchunk, GS gs) {
    // grid z = (network, K chunk): the chunk covers k in [c kchunk, min(K, (c + 1) kchunk)) and
    // (EPI_F32 only) writes its partial product to the c-th M x ldo slab of the network's output
    const int zg = blockIdx.z / gs.splits, zc = blockIdx.z % gs.splits;
    A += zg * gs.a;
    B += zg * gs.b;
    if (bias) bias += zg * gs.bias;
    if (mask) mask += zg * gs.mask;
    const int kb = zc * kchunk;
    const int ke = min(K, kb + kchunk);
    if (EPI == EPI_F32) out = static_cast<float*>(out) + zg * gs.out + (int64_t)zc * M * ldo;
    else out = static_cast<bf16*>(out) + zg * gs.out;
    __shared__ __align__(16) bf16 As[BM][BK + PAD];
    __shared__ __align__(16) bf16 Bs[BN][BK + PAD];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[i][j][c] = 0.f;

    // 16-byte loads need a leading dimension that keeps every chunk aligned
    const bool va = (lda & 7) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const bool vb = (ldb & 7) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    // the next k step's chunks are fetched into registers while this step's MMAs run
    uint4 ra[2], rb[2];
    if (kb < ke) {
        fetch_tile<TA>(ra, A, lda, m0, M, kb, ke, va);
        fetch_tile<TB>(rb, B, ldb, n0, N, kb, ke, vb);
    }
    for (int k0 = kb; k0 < ke; k0 += BK) {
        store_tile<TA>(As, ra);
        store_tile<TB>(Bs, rb);
        __syncthreads();
        if (k0 + BK < ke) {
            fetch_tile<TA>(ra, A, lda, m0, M, k0 + BK, ke, va);
            fetch_tile<TB>(rb, B, ldb, n0, N, k0 + BK, ke, vb);
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = wn + j * 8 + g;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    // epilogue: accumulator element (i, j, c) sits at row wm + 16 i + g (+8 for c >= 2),
    // column wn + 8 j + 2 t (+1 for odd c)
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int m = m0 + wm + i * 16 + g + (c >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * t + (c & 1);
                if (m >= M || n >= N) continue;
                const float v = acc[i][j][c];
                if (EPI == EPI_BIAS_RELU_BF16) {
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n] = __float2bfloat16(fmaxf(v + bias[n], 0.f));
                } else if (EPI == EPI_MASK_BF16) {
                    const float a = __bfloat162float(mask[(int64_t)m * ldm + n]);
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n] = __float2bfloat16(a > 0.f ? v : 0.f);
                } else {
                    static_cast<float*>(out)[(int64_t)m * ldo + n] = v;
                }
            }
}

// ---------------------------------------------------------------------------
// The same GEMM on the 5th-generation tensor cores (tcgen05): a CTA owns a
// 128 x NT tile of C whose fp32 accumulators live in tensor memory (TMEM).
// Per K stage of 64 the 128 threads copy A (128 x 64) and B (NT x 64) into
// shared memory as K-major 8 x 8 "core matrices" (no swizzle: element (r, k)
// at byte (r/8) 1024 + (k/8) 128 + (r%8) 16 + (k%8) 2), transposing on the way
// when an operand is stored the other way round; one thread issues four
// 128 x NT x 16 bf16 MMAs and commits them to an mbarrier.  Two stages
// alternate, so the copy of stage i+1 overlaps the MMAs of stage i.  The
// epilogue reads TMEM with tcgen05.ld (warp w: rows 32w..32w+31, one row per
// thread) and applies the same epilogues as the mma.sync kernel.  Every
// mbarrier wait is bounded; on timeout the CTA records an error, stops
// issuing work, still frees its TMEM and returns.
// ---------------------------------------------------------------------------
namespace tc5 {

constexpr int TM = 128;          // tile rows = MMA M
constexpr int TK = 64;           // K per stage
constexpr int THREADS = 128;
constexpr long long kMaxPolls = 1LL << 24;
// The last wait before the tensor memory is freed, after a wait has already
// run out: far longer, so that the MMAs of a slow but live CTA finish before
// the columns they write are released.
constexpr long long kMaxPollsDrain = 1LL << 28;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t core_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading (K) byte offset 128,
// stride (M/N) byte offset 1024, fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, long long polls = kMaxPolls) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < polls; i++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Copy rows [row0, row0 + R) x k [k0, k0 + TK) of an operand into a core-matrix tile.
//   !T: element (r, k) at G[r * ld + k] (k contiguous): 16-byte loads along k
//    T: element (r, k) at G[k * ld + r] (r contiguous): 16-byte loads along r, scattered
template <bool T, int R>
__device__ __forceinline__ void load_op(unsigned char* tile, const bf16* __restrict__ G, int ld, int row0, int rows,
                                        int k0, int kend) {
    constexpr int CH = R * TK / 8;   // 16-byte chunks per stage
    for (int c = threadIdx.x; c < CH; c += THREADS) {
        if (!T) {
            const int r = c / (TK / 8), k = (c % (TK / 8)) * 8;
            const int gr = row0 + r, gk = k0 + k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < rows) {
                if (gk + 8 <= kend) {
                    v = *reinterpret_cast<const uint4*>(G + (int64_t)gr * ld + gk);
                } else {
                    bf16 e[8];
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        e[j] = gk + j < kend ? G[(int64_t)gr * ld + gk + j] : __float2bfloat16(0.f);
                    v = *reinterpret_cast<const uint4*>(e);
                }
            }
            *reinterpret_cast<uint4*>(tile + core_off(r, k)) = v;
        } else {
            const int k = c / (R / 8), r = (c % (R / 8)) * 8;
            const int gr = row0 + r, gk = k0 + k;
            bf16 e[8];
            if (gk < kend && gr + 8 <= rows) {
                *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(G + (int64_t)gk * ld + gr);
            } else {
#pragma unroll
                for (int j = 0; j < 8; j++)
                    e[j] = (gk < kend && gr + j < rows) ? G[(int64_t)gk * ld + gr + j] : __float2bfloat16(0.f);
            }
#pragma unroll
            for (int j = 0; j < 8; j++) *reinterpret_cast<bf16*>(tile + core_off(r + j, k)) = e[j];
        }
    }
}

template <bool TA, bool TB, int EPI, int NT>
__global__ void __launch_bounds__(THREADS)
gemm_tc5_kernel(int M, int N, int K, const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb,
                const float* __restrict__ bias, const bf16* __restrict__ mask, int ldm, void* out, int ldo, int kchunk,
                int* err, GS gs) {
    constexpr int A_BYTES = TM * TK * 2, B_BYTES = NT * TK * 2, STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;   // TMEM columns: a power of two >= 32
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * NT;
    const int zg = blockIdx.z / gs.splits, zc = blockIdx.z % gs.splits;
    A += zg * gs.a;
    B += zg * gs.b;
    if (bias) bias += zg * gs.bias;
    if (mask) mask += zg * gs.mask;
    const int kb = zc * kchunk, ke = min(K, kb + kchunk);
    if (EPI == EPI_F32) out = static_cast<float*>(out) + zg * gs.out + (int64_t)zc * M * ldo;
    else out = static_cast<bf16*>(out) + zg * gs.out;

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        failed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    const int nk = ke > kb ? (ke - kb + TK - 1) / TK : 0;
    uint32_t phase[2] = {0u, 0u};
    int issued = 0;   // stages whose MMAs were committed
    for (int i = 0; i < nk; i++) {
        const int st = i & 1;
        unsigned char* a_t = smem + st * STAGE;
        unsigned char* b_t = a_t + A_BYTES;
        if (i >= 2) {   // the MMAs of stage i - 2 used these buffers
            if (!wait_bar(&bars[st], phase[st])) failed = 1;
            phase[st] ^= 1u;
        }
        __syncthreads();
        if (failed) break;
        const int k0 = kb + i * TK;
        load_op<TA, TM>(a_t, A, lda, m0, M, k0, ke);
        load_op<TB, NT>(b_t, B, ldb, n0, N, k0, ke);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ab = smem_u32(a_t), bb = smem_u32(b_t);
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++)
                mma(tmem, sdesc(ab + kk * 256), sdesc(bb + kk * 256), idesc(TM, NT), (i > 0 || kk > 0) ? 1u : 0u);
            commit(&bars[st]);
        }
        issued = i + 1;
    }
    // the last committed stage (MMAs complete in order); waited for even after a
    // failure -- then with the much longer drain bound -- so that no MMA is
    // still writing when the TMEM is freed.  Should the drain bound run out too
    // (an MMA that never completes), the TMEM is freed all the same: a CTA that
    // exits holding its columns would leave the next CTA's allocation on this
    // SM waiting for ever, while the error flag already makes the host discard
    // this launch's output.
    if (issued > 0) {
        const int st = (issued - 1) & 1;
        if (!wait_bar(&bars[st], phase[st], failed ? kMaxPollsDrain : kMaxPolls)) failed = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        // phase 1: TMEM -> shared staging tile of raw fp32 accumulators (row stride NT + 4
        // floats; the stage buffers are free: every MMA has completed)
        float* stg = reinterpret_cast<float*>(smem);
        constexpr int LDS = NT + 4;
        const int row = warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            if (nk > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) r[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(stg + row * LDS + c0 + j) =
                    make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                __uint_as_float(r[j + 3]));
        }
        __syncthreads();
        // phase 2: coalesced epilogue, 4 consecutive columns per thread
        constexpr int QPR = NT / 4;   // column quads per row
        for (int q = threadIdx.x; q < TM * QPR; q += THREADS) {
            const int rr = q / QPR, cc = (q % QPR) * 4;
            const int m = m0 + rr, n = n0 + cc;
            if (m >= M) continue;
            const float4 v4 = *reinterpret_cast<const float4*>(stg + rr * LDS + cc);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (n + j >= N) break;
                if (EPI == EPI_BIAS_RELU_BF16) {
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n + j] = __float2bfloat16(fmaxf(v[j] + bias[n + j], 0.f));
                } else if (EPI == EPI_MASK_BF16) {
                    const float a = __bfloat162float(mask[(int64_t)m * ldm + n + j]);
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n + j] = __float2bfloat16(a > 0.f ? v[j] : 0.f);
                } else {
                    static_cast<float*>(out)[(int64_t)m * ldo + n + j] = v[j];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// ---------------------------------------------------------------------------
// The same product with both operands K-contiguous (the forward layers: A =
// activations [M][K], B = weights [N][K]) fed by the tensor memory accelerator.
// A 3-D tensor map (k, row, network) per operand; per stage of 64 k, thread 0
// copies eight 8-wide k slices of the 128-row A tile and of the NT-row B tile
// with cp.async.bulk.tensor, so that k slice j lands at j * rows * 16 bytes and
// row r of a slice at r * 16: core matrices (8 rows x 16 bytes) 128 bytes
// apart along the rows and rows * 16 bytes apart along k -- the same K-major
// no-swizzle form as above with the two offsets of the descriptor set to
// those strides.  Rows and k beyond the operands are filled with zeros by the
// copy unit.  A ring of kStagesT stages: "full" barriers carry the copies'
// bytes, thread 32 waits on them and issues the MMAs, whose commit frees the
// stage on its "empty" barrier and, after the last stage, completes "done",
// which every thread waits for before the epilogue.  Every wait is bounded;
// after a failure the last wait on "done" uses the drain bound, and thread 0
// waits for its copies in flight before the CTA leaves.
// ---------------------------------------------------------------------------
constexpr int kStagesT = 2;

__device__ __forceinline__ uint64_t sdesc_t(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

template <int EPI, int NT>
__global__ void __launch_bounds__(THREADS)
gemm_tma_kernel(int M, int N, int K, const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const float* __restrict__ bias, const bf16* __restrict__ mask, int ldm, void* out, int ldo, int* err,
                GS gs) {
    constexpr int A_BYTES = TM * TK * 2, B_BYTES = NT * TK * 2, STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t NCOLS = NT < 32 ? 32 : NT;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStagesT], empty[kStagesT], done;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * NT;
    const int zg = blockIdx.z;
    if (bias) bias += zg * gs.bias;
    if (mask) mask += zg * gs.mask;
    if (EPI == EPI_F32) out = static_cast<float*>(out) + zg * gs.out;
    else out = static_cast<bf16*>(out) + zg * gs.out;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStagesT; st++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[st])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const int nk = (K + TK - 1) / TK;
    int issued = 0;   // thread 0: stages whose copies were issued

    if (threadIdx.x == 0) {
        // copies: stage i into slot i % kStagesT once the MMAs of stage i - kStagesT have released it
        for (int i = 0; i < nk; i++) {
            const int st = i % kStagesT;
            if (i >= kStagesT && !wait_bar(&empty[st], (uint32_t)((i / kStagesT) - 1) & 1u)) {
                failed = 1;
                break;
            }
            if (*(volatile int*)&failed) break;
            unsigned char* a_t = smem + st * STAGE;
            unsigned char* b_t = a_t + A_BYTES;
            bar_arrive_tx(&full[st], (uint32_t)STAGE);
#pragma unroll
            for (int j = 0; j < TK / 8; j++) {
                tma_load_3d(a_t + j * TM * 16, &mapA, i * TK + 8 * j, m0, zg, &full[st]);
                tma_load_3d(b_t + j * NT * 16, &mapB, i * TK + 8 * j, n0, zg, &full[st]);
            }
            issued = i + 1;
        }
    } else if (threadIdx.x == 32) {
        // MMAs: four K = 16 steps per stage, each two k slices (2 x rows x 16 bytes) further on
        for (int i = 0; i < nk; i++) {
            const int st = i % kStagesT;
            if (*(volatile int*)&failed || !wait_bar(&full[st], (uint32_t)(i / kStagesT) & 1u)) {
                failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ab = smem_u32(smem + st * STAGE), bb = ab + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / 16; kk++)
                mma(tmem, sdesc_t(ab + kk * 2 * TM * 16, TM * 16, 128), sdesc_t(bb + kk * 2 * NT * 16, NT * 16, 128),
                    idesc(TM, NT), (i > 0 || kk > 0) ? 1u : 0u);
            commit(&empty[st]);
        }
        commit(&done);   // arrives when every MMA issued above has completed (at once if none was)
    }
    // every thread: the accumulators are final (or, after a failure, no MMA is still running)
    if (!wait_bar(&done, 0u, kMaxPolls) && !wait_bar(&done, 0u, kMaxPollsDrain)) failed = 1;
    if (threadIdx.x == 0) {
        // the last copy issued into each slot has landed before the CTA leaves (after a failure
        // some were never consumed)
        for (int st = 0; st < kStagesT && st < issued; st++) {
            const int last = st + ((issued - 1 - st) / kStagesT) * kStagesT;
            if (!wait_bar(&full[st], (uint32_t)(last / kStagesT) & 1u, kMaxPollsDrain)) failed = 1;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        float* stg = reinterpret_cast<float*>(smem);
        constexpr int LDS = NT + 4;
        const int row = warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(stg + row * LDS + c0 + j) =
                    make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                __uint_as_float(r[j + 3]));
        }
        __syncthreads();
        constexpr int QPR = NT / 4;
        // four outputs per store where the output rows, the bias and the mask allow it (CTA-uniform)
        const bool vec = N % 4 == 0 && ldo % 4 == 0 &&
                         (reinterpret_cast<uintptr_t>(out) & (EPI == EPI_F32 ? 15u : 7u)) == 0 &&
                         (EPI != EPI_BIAS_RELU_BF16 || (reinterpret_cast<uintptr_t>(bias) & 15u) == 0) &&
                         (EPI != EPI_MASK_BF16 || (ldm % 4 == 0 && (reinterpret_cast<uintptr_t>(mask) & 7u) == 0));
        for (int q = threadIdx.x; q < TM * QPR; q += THREADS) {
            const int rr = q / QPR, cc = (q % QPR) * 4;
            const int m = m0 + rr, n = n0 + cc;
            if (m >= M) continue;
            const float4 v4 = *reinterpret_cast<const float4*>(stg + rr * LDS + cc);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
            if (vec && n + 4 <= N) {
                if (EPI == EPI_F32) {
                    *reinterpret_cast<float4*>(static_cast<float*>(out) + (int64_t)m * ldo + n) = v4;
                } else {
                    float o[4];
                    if (EPI == EPI_BIAS_RELU_BF16) {
                        const float4 b4 = *reinterpret_cast<const float4*>(bias + n);
                        o[0] = fmaxf(v[0] + b4.x, 0.f);
                        o[1] = fmaxf(v[1] + b4.y, 0.f);
                        o[2] = fmaxf(v[2] + b4.z, 0.f);
                        o[3] = fmaxf(v[3] + b4.w, 0.f);
                    } else {
                        const uint2 mk = *reinterpret_cast<const uint2*>(mask + (int64_t)m * ldm + n);
                        const __nv_bfloat162 m01 = *reinterpret_cast<const __nv_bfloat162*>(&mk.x);
                        const __nv_bfloat162 m23 = *reinterpret_cast<const __nv_bfloat162*>(&mk.y);
                        o[0] = __low2float(m01) > 0.f ? v[0] : 0.f;
                        o[1] = __high2float(m01) > 0.f ? v[1] : 0.f;
                        o[2] = __low2float(m23) > 0.f ? v[2] : 0.f;
                        o[3] = __high2float(m23) > 0.f ? v[3] : 0.f;
                    }
                    const __nv_bfloat162 p01 = __floats2bfloat162_rn(o[0], o[1]);
                    const __nv_bfloat162 p23 = __floats2bfloat162_rn(o[2], o[3]);
                    uint2 pk;
                    pk.x = *reinterpret_cast<const uint32_t*>(&p01);
                    pk.y = *reinterpret_cast<const uint32_t*>(&p23);
                    *reinterpret_cast<uint2*>(static_cast<bf16*>(out) + (int64_t)m * ldo + n) = pk;
                }
                continue;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (n + j >= N) break;
                if (EPI == EPI_BIAS_RELU_BF16) {
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n + j] = __float2bfloat16(fmaxf(v[j] + bias[n + j], 0.f));
                } else if (EPI == EPI_MASK_BF16) {
                    const float a = __bfloat162float(mask[(int64_t)m * ldm + n + j]);
                    static_cast<bf16*>(out)[(int64_t)m * ldo + n + j] = __float2bfloat16(a > 0.f ? v[j] : 0.f);
                } else {
                    static_cast<float*>(out)[(int64_t)m * ldo + n + j] = v[j];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// cuTensorMapEncodeTiled from the driver (fetched once; the library links only the runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tensor map of G operands [rows][K] (k contiguous, row stride ld, operand
// stride `stride` elements), boxes of 8 k x box_rows rows x 1 operand.
static bool make_map(CUtensorMap* map, const bf16* base, int K, int rows, int ld, int G, int64_t stride,
                     int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int64_t gstride = G > 1 ? stride : (int64_t)rows * ld;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)G};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)gstride * 2};
    cuuint32_t box[3] = {8u, (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Both operands K-contiguous: the TMA-fed kernel.  cudaErrorNotSupported when
// a tensor map cannot describe the operands (the caller then takes the
// register-copied tcgen05 kernel).
template <int EPI, int NT>
cudaError_t launch_tma(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, const float* bias,
                       const bf16* mask, int ldm, void* out, int ldo, int G, const GS& gs, int* err, cudaStream_t s) {
    constexpr int SMEM0 = kStagesT * (TM * TK * 2 + NT * TK * 2), STAGING = TM * (NT + 4) * 4;
    constexpr int SMEM = SMEM0 > STAGING ? SMEM0 : STAGING;
    if (K <= 0 || K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || gs.splits != 1 ||
        (G > 1 && (gs.a < (int64_t)M * lda || gs.b < (int64_t)N * ldb || gs.a % 8 != 0 || gs.b % 8 != 0)) ||
        (reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u))
        return cudaErrorNotSupported;
    CUtensorMap mA, mB;
    if (!make_map(&mA, A, K, M, lda, G, gs.a, TM) || !make_map(&mB, B, K, N, ldb, G, gs.b, NT))
        return cudaErrorNotSupported;
    static bool attr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        if ((e = cudaFuncSetAttribute(gemm_tma_kernel<EPI, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM)) !=
            cudaSuccess)
            return e;
        attr[dev] = true;
    }
    dim3 grid((unsigned)((N + NT - 1) / NT), (unsigned)((M + TM - 1) / TM), (unsigned)G);
    gemm_tma_kernel<EPI, NT><<<grid, THREADS, SMEM, s>>>(M, N, K, mA, mB, bias, mask, ldm, out, ldo, err, gs);
    return cudaGetLastError();
}

template <bool TA, bool TB, int EPI, int NT>
cudaError_t launch(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, const float* bias,
                   const bf16* mask, int ldm, void* out, int ldo, int G, const GS& gs, int kchunk, int* err,
                   cudaStream_t s) {
    constexpr int STAGES = 2 * (TM * TK * 2 + NT * TK * 2), STAGING = TM * (NT + 4) * 4;
    constexpr int SMEM = STAGES > STAGING ? STAGES : STAGING;
    static bool attr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        if ((e = cudaFuncSetAttribute(gemm_tc5_kernel<TA, TB, EPI, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM)) != cudaSuccess)
            return e;
        attr[dev] = true;
    }
    dim3 grid((unsigned)((N + NT - 1) / NT), (unsigned)((M + TM - 1) / TM), (unsigned)(G * gs.splits));
    gemm_tc5_kernel<TA, TB, EPI, NT><<<grid, THREADS, SMEM, s>>>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo,
                                                                 kchunk, err, gs);
    return cudaGetLastError();
}

}  // namespace tc5

template <bool TA, bool TB, int EPI>
static cudaError_t gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, const float* bias,
                        const bf16* mask, int ldm, void* out, int ldo, cudaStream_t s, int* tc_err = nullptr,
                        int G = 1, GS gs = GS()) {
    if (M <= 0 || N <= 0 || G <= 0) return cudaSuccess;
    gs.splits = 1;
    const int kc = K > 0 ? K : 1;
    if (tc_err && !TA && !TB && N % 64 == 0) {
        // both operands K-contiguous: copies by the tensor memory accelerator
        const cudaError_t e =
            N % 128 == 0 && (int64_t)((M + 127) / 128) * (N / 128) * G >= 152
                ? tc5::launch_tma<EPI, 128>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo, G, gs, tc_err, s)
                : tc5::launch_tma<EPI, 64>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo, G, gs, tc_err, s);
        if (e != cudaErrorNotSupported) return e;
    }
    if (tc_err && N % 128 == 0 && (int64_t)((M + 127) / 128) * (N / 128) * G >= 152)
        return tc5::launch<TA, TB, EPI, 128>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo, G, gs, kc, tc_err,
                                             s);
    if (tc_err && N % 64 == 0)
        return tc5::launch<TA, TB, EPI, 64>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo, G, gs, kc, tc_err, s);
    if (tc_err && N == 16)
        return tc5::launch<TA, TB, EPI, 16>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo, G, gs, kc, tc_err, s);
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)G);
    gemm_bf16_kernel<TA, TB, EPI><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, bias, mask, ldm, out, ldo,
                                                                kc, gs);
    return cudaGetLastError();
}

// out[g][i] = sum_c ws[g][c][i] over the K chunks, in order (deterministic)
__global__ void sum_splits_kernel(int S, int64_t MN, const float* __restrict__ ws, float* out, int64_t sout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    const float* w = ws + (int64_t)blockIdx.y * S * MN;
    float v = 0.f;
    for (int z = 0; z < S; z++) v += w[(int64_t)z * MN + i];
    out[blockIdx.y * sout + i] = v;
}

// Weight gradient C = A^T B (fp32, dense M x N) of each of G networks, with the
// K = batch axis split into chunks of 256 rows: one CTA per (tile, network,
// chunk) keeps the GPU busy when M x N is only a few tiles; the chunk partials
// (ws: G x splits x M x N floats) are summed in order into out + g sout.
template <bool TB>
static cudaError_t gemm_wgrad(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, float* out,
                              float* ws, int max_splits, cudaStream_t s, int* tc_err = nullptr, int G = 1,
                              int64_t sa = 0, int64_t sb = 0, int64_t sout = 0) {
    if (M <= 0 || N <= 0 || G <= 0) return cudaSuccess;
    const bool tc = tc_err && (N % 64 == 0 || N == 16);
    int splits = (K + 255) / 256;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    int kchunk = (K + splits - 1) / splits;
    const int q = tc ? tc5::TK : BK;   // chunks start on a stage boundary
    kchunk = (kchunk + q - 1) / q * q;
    splits = (K + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    GS gs;
    gs.a = sa;
    gs.b = sb;
    gs.splits = splits;
    gs.out = (int64_t)splits * M * N;
    cudaError_t e;
    if (tc && N == 16) {
        e = tc5::launch<true, TB, EPI_F32, 16>(M, N, K, A, lda, B, ldb, nullptr, nullptr, 0, ws, N, G, gs, kchunk,
                                               tc_err, s);
    } else if (tc) {
        e = tc5::launch<true, TB, EPI_F32, 64>(M, N, K, A, lda, B, ldb, nullptr, nullptr, 0, ws, N, G, gs, kchunk,
                                               tc_err, s);
    } else {
        dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)(G * splits));
        gemm_bf16_kernel<true, TB, EPI_F32><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, nullptr, nullptr,
                                                                          0, ws, N, kchunk, gs);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int64_t MN = (int64_t)M * N;
    sum_splits_kernel<<<dim3((unsigned)((MN + 255) / 256), (unsigned)G), 256, 0, s>>>(splits, MN, ws, out, sout);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small kernels. Each covers all G networks of a batch: network g's rows are
// rows [g N, (g + 1) N) of the activations, its parameters th + g P.
// ---------------------------------------------------------------------------
// Xb[g][r][c] = X[g sx + r][c] for c < 5, else 0 (sx: rows between networks' inputs)
__global__ void input_pad_kernel(int G, int N, int64_t sx, const float* __restrict__ X, bf16* Xb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * N * kInPad) return;
    const int64_t row = i / kInPad;
    const int c = (int)(i % kInPad);
    const int64_t g = row / N, r = row % N;
    Xb[i] = __float2bfloat16(c < 5 ? X[(g * sx + r) * 5 + c] : 0.f);
}

// y[g sy + r] = a3[g N + r, :] . w4_g + b4_g (fp32 accumulation of bf16 products), then * scale + shift
__global__ void output_kernel(int G, int N, int W, const bf16* __restrict__ A3, const bf16* __restrict__ w4,
                              const float* __restrict__ b4, int64_t P, const float* __restrict__ stdz, float* y,
                              int64_t sy) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= (int64_t)G * N) return;
    const int64_t g = row / N, r = row % N;
    const bf16* wg = w4 + g * W;
    float s = 0.f;
    for (int k = lane; k < W; k += 32) s = fmaf(__bfloat162float(A3[row * W + k]), __bfloat162float(wg[k]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float v = s + b4[g * P];
        y[g * sy + r] = stdz ? fmaf(v, stdz[g * 8 + 1], stdz[g * 8]) : v;
    }
}

// mean and standard deviation of the finite targets t[g st + (0..N)] (block g, fixed order)
__global__ void standardize_kernel(int N, const float* __restrict__ t, int64_t st, float* stdz) {
    __shared__ double s1[256], s2[256], sc[256];
    t += blockIdx.x * st;
    stdz += blockIdx.x * 8;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float v = t[i];
        if (isfinite(v)) {
            a += v;
            b += (double)v * v;
            c += 1.0;
        }
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = sc[0] > 0 ? sc[0] : 1.0;
        const double mu = s1[0] / n;
        const double var = s2[0] / n - mu * mu;
        stdz[0] = (float)mu;
        stdz[1] = (float)(var > 1e-30 ? sqrt(var) : 1.0);
        stdz[2] = (float)sc[0];
    }
}

// dy[n] = (y[n] - t'[n]) / count for finite targets, t' = (t - mu)/sigma if
// standardising; also the per-sample squared error for the loss. Row n = g N + r
// takes its target from t[g st + r] and its network's statistics from stdz + 8 g.
__global__ void dloss_kernel(int G, int N, const float* __restrict__ y, const float* __restrict__ t, int64_t st,
                             const float* __restrict__ stdz, const float* __restrict__ count, float* dy, float* sq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * N) return;
    const int64_t g = i / N, r = i % N;
    const float tv = t[g * st + r];
    float res = 0.f;
    if (isfinite(tv)) {
        const float tt = stdz ? (tv - stdz[g * 8]) / stdz[g * 8 + 1] : tv;
        res = y[i] - tt;
    }
    const float c = count[g * 8] > 0.f ? count[g * 8] : 1.f;
    dy[i] = res / c;
    sq[i] = 0.5f * res * res / c;
}

// dZ3[n, k] = dy[n] * w4[k] * (a3[n, k] > 0), with the w4 of row n's network
__global__ void dz_last_kernel(int G, int N, int W, const float* __restrict__ dy, const bf16* __restrict__ w4,
                               const bf16* __restrict__ A3, bf16* dZ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * N * W) return;
    const int64_t row = i / W;
    const int k = (int)(i % W);
    const float a = __bfloat162float(A3[i]);
    dZ[i] = __float2bfloat16(a > 0.f ? dy[row] * __bfloat162float(w4[(row / N) * W + k]) : 0.f);
}

template <typename T>
__device__ __forceinline__ float as_f(T v);
template <>
__device__ __forceinline__ float as_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float as_f<bf16>(bf16 v) { return __bfloat162float(v); }

// Column sums out[g][k] = sum_n wrow[g][n] Mx[g][n][k] (bf16 or fp32 input) in two
// deterministic passes: block (b, g) (W threads, thread = column, coalesced)
// sums rows [b R, (b+1) R) of network g into part[g][b][k]; one pass over the
// blocks then adds the parts in order.
constexpr int kColRows = 128;

template <typename T>
__global__ void colsum_part_kernel(int N, int W, const T* __restrict__ Mx, const float* __restrict__ wrow,
                                   float* part) {
    const int k = threadIdx.x;
    if (k >= W) return;
    const int64_t g = blockIdx.y;
    if (Mx) Mx += g * N * W;
    if (wrow) wrow += g * N;
    const int n0 = blockIdx.x * kColRows, n1 = min(N, n0 + kColRows);
    float s = 0.f;
    for (int n = n0; n < n1; n++) {
        const float v = Mx ? as_f<T>(Mx[(int64_t)n * W + k]) : 1.f;
        s = fmaf(wrow ? wrow[n] : 1.f, v, s);
    }
    part[(g * gridDim.x + blockIdx.x) * W + k] = s;
}

__global__ void colsum_final_kernel(int nb, int W, const float* __restrict__ part, float* out, int64_t sout) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= W) return;
    const int64_t g = blockIdx.y;
    part += g * nb * W;
    float s = 0.f;
    for (int b = 0; b < nb; b++) s += part[(int64_t)b * W + k];
    out[g * sout + k] = s;
}

template <typename T>
static cudaError_t colsum(int G, int N, int W, const T* Mx, const float* wrow, float* out, int64_t sout, float* part,
                          cudaStream_t s) {
    const int nb = (N + kColRows - 1) / kColRows;
    colsum_part_kernel<T><<<dim3((unsigned)nb, (unsigned)G), W, 0, s>>>(N, W, Mx, wrow, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    colsum_final_kernel<<<dim3((unsigned)((W + 255) / 256), (unsigned)G), 256, 0, s>>>(nb, W, part, out, sout);
    return cudaGetLastError();
}

// out[g sout] = sum_n v[g N + n] (block g, fixed order)
__global__ void sum_kernel(int N, const float* __restrict__ v, float* out, int64_t sout) {
    __shared__ float red[256];
    v += (int64_t)blockIdx.x * N;
    float s = 0.f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) s += v[n];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x * sout] = red[0];
}

// gradient of the padded first layer [W][16] -> the [W][5] slot of each network's flat gradient
__global__ void unpad_kernel(int G, int W, int64_t P, const float* __restrict__ g16, float* g5) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)G * W * 5) return;
    const int64_t g = i / (W * 5);
    const int j = (int)(i % (W * 5));
    g5[g * P + j] = g16[g * W * kInPad + (j / 5) * kInPad + j % 5];
}

// fp32 master weights -> bf16 copies (first layer padded to 16 inputs); grid y = network
__global__ void refresh_kernel(int W, int64_t P, const float* __restrict__ th, bf16* W1b, bf16* W2b, bf16* W3b,
                               bf16* W4b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = blockIdx.y;
    const int64_t nW1 = (int64_t)W * 5, nWW = (int64_t)W * W;
    const float* W1 = th + g * P;
    const float* W2 = W1 + nW1 + W;
    const float* W3 = W2 + nWW + W;
    const float* W4 = W3 + nWW + W;
    if (i < (int64_t)W * kInPad) {
        const int64_t r = i / kInPad;
        const int c = (int)(i % kInPad);
        W1b[g * W * kInPad + i] = __float2bfloat16(c < 5 ? W1[r * 5 + c] : 0.f);
    }
    if (i < nWW) {
        W2b[g * nWW + i] = __float2bfloat16(W2[i]);
        W3b[g * nWW + i] = __float2bfloat16(W3[i]);
    }
    if (i < W) W4b[g * W + i] = __float2bfloat16(W4[i]);
}

// Adam step counter and bias corrections on the device (so that training
// steps can be captured in a CUDA graph): ac[0] = step (as unsigned int),
// ac[1] = 1 / (1 - 0.9^step), ac[2] = 1 / (1 - 0.999^step). All networks of a
// batch take their steps together and share the counter.
__global__ void adam_prep_kernel(float* ac) {
    unsigned int* st = reinterpret_cast<unsigned int*>(ac);
    const unsigned int k = *st + 1u;
    *st = k;
    ac[1] = (float)(1.0 / (1.0 - pow(0.9, (double)k)));
    ac[2] = (float)(1.0 / (1.0 - pow(0.999, (double)k)));
}

__global__ void adam_kernel(int64_t P, float* th, const float* __restrict__ g, float* m, float* v, float lr,
                            const float* __restrict__ ac) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float c1 = ac[1], c2 = ac[2];
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// Kaiming-uniform weights, zero biases (Philox counter (index, 0x4D4C5000, 0, 0), key = seed)
__device__ __forceinline__ void philox_mlp(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__global__ void stdz_reset_kernel(int G, float* stdz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G * 8) stdz[i] = (i % 8 == 1 || i % 8 == 5) ? 1.f : 0.f;
}

// network g of a batch (grid y) takes key seed + g
__global__ void init_kernel(int W, unsigned long long seed, float* th) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nW1 = (int64_t)W * 5, nWW = (int64_t)W * W;
    const int64_t P = nW1 + W + 2 * (nWW + W) + W + 1;
    if (i >= P) return;
    seed += blockIdx.y;
    th += blockIdx.y * P;
    int64_t o = i;
    float fan = 0.f;
    if (o < nW1) fan = 5.f;
    else if ((o -= nW1) < W) fan = 0.f;
    else if ((o -= W) < nWW) fan = (float)W;
    else if ((o -= nWW) < W) fan = 0.f;
    else if ((o -= W) < nWW) fan = (float)W;
    else if ((o -= nWW) < W) fan = 0.f;
    else if ((o -= W) < W) fan = (float)W;
    else fan = 0.f;
    if (fan == 0.f) {
        th[i] = 0.f;
        return;
    }
    uint32_t c[4] = {(uint32_t)i, 0x4D4C5000u, (uint32_t)(i >> 32), 0u};
    philox_mlp(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u = (float)(c[0] >> 8) * (1.0f / 16777216.0f);
    th[i] = (2.f * u - 1.f) * sqrtf(6.f / fan);
}

}  // namespace fs

// ---------------------------------------------------------------------------
// Module state and C ABI
// ---------------------------------------------------------------------------
struct fs_mlp {
    int G;          // networks in the batch (same width, trained together)
    int W, cap;     // width; rows per network per pass
    int64_t P;      // parameters per network
    int splits;     // most K chunks of a weight-gradient GEMM
    cudaStream_t stream;
    float* th;      // fp32 master weights [G][P]
    float* gr;      // gradient [G][P]
    float* m;       // Adam moments [G][P]
    float* v;
    int64_t step;
    fs::bf16 *W1b, *W2b, *W3b, *W4b;           // bf16 weights [G][...]
    fs::bf16 *Xb, *A1, *A2, *A3, *dZa, *dZb;   // activations [G][cap][...]
    float *y, *dy, *sq;                         // [G][cap]
    float *g16;     // padded first-layer gradient [G][W][16]
    float *stdz;    // [G][8]: target mean, deviation, count (training); [4..6] the same for the raw loss
    float *loss;    // [G]
    float* adamc;   // [4] Adam step counter and bias corrections (device)
    float* ws;      // split-K partials: G x splits x W x max(W, kInPad)
    int tc5;        // 0: mma.sync GEMMs; 1: tcgen05 throughout; 2: tcgen05 forward layers, mma.sync backward
    int* tc_err;    // device flag set by a tcgen05 GEMM whose mbarrier wait ran out
    float* part;    // column-sum partials: G x ceil(cap / kColRows) x W
};

namespace {

int64_t nparams(int W) { return (int64_t)W * 5 + W + 2 * ((int64_t)W * W + W) + W + 1; }

fs_status mlp_fail(cudaError_t e, const char* what) {
    return fs::set_error(e == cudaErrorMemoryAllocation ? FS_ENOMEM : FS_ECUDA, "%s: %s", what,
                         cudaGetErrorString(e));
}

void mlp_free(fs_mlp* m) {
    void* ps[] = {m->th, m->gr, m->m, m->v, m->W1b, m->W2b, m->W3b, m->W4b, m->Xb, m->A1, m->A2, m->A3,
                  m->dZa, m->dZb, m->y, m->dy, m->sq, m->g16, m->stdz, m->loss, m->adamc, m->ws, m->part,
                  m->tc_err};
    for (void* p : ps) cudaFree(p);
}

// tcgen05 error flag for the GEMMs of the forward layers / of the backward pass (NULL: mma.sync)
int* tcp(fs_mlp* m) { return m->tc5 ? m->tc_err : nullptr; }
int* tcp_bwd(fs_mlp* m) { return m->tc5 == 1 ? m->tc_err : nullptr; }

// identity target scaling (mean 0, deviation 1) for every network
cudaError_t reset_stdz(fs_mlp* m) {
    fs::stdz_reset_kernel<<<(m->G * 8 + 255) / 256, 256, 0, m->stream>>>(m->G, m->stdz);
    return cudaGetLastError();
}

// Forward pass of every network for N <= cap rows each: network g reads rows
// X[g sx .. g sx + N) (fp32, 5 per row) and writes y[g sy .. g sy + N);
// activations are kept (rows g N + r).
cudaError_t mlp_forward(fs_mlp* m, const float* X, int64_t sx, int N, float* y, int64_t sy, bool destandardize) {
    using namespace fs;
    const int W = m->W, G = m->G;
    const int64_t P = m->P, nWW = (int64_t)W * W, NW = (int64_t)N * W;
    cudaStream_t s = m->stream;
    input_pad_kernel<<<(unsigned)(((int64_t)G * N * kInPad + 255) / 256), 256, 0, s>>>(G, N, sx, X, m->Xb);
    const float* b1 = m->th + (int64_t)W * 5;
    const float* b2 = b1 + W + nWW;
    const float* b3 = b2 + W + nWW;
    const float* b4 = b3 + W + W;
    GS g1, gh;
    g1.a = (int64_t)N * kInPad;
    g1.b = (int64_t)W * kInPad;
    g1.bias = P;
    g1.out = NW;
    gh.a = NW;
    gh.b = nWW;
    gh.bias = P;
    gh.out = NW;
    cudaError_t e;
    if ((e = gemm<false, false, EPI_BIAS_RELU_BF16>(N, W, kInPad, m->Xb, kInPad, m->W1b, kInPad, b1, nullptr, 0, m->A1,
                                                     W, s, tcp(m), G, g1)) != cudaSuccess)
        return e;
    if ((e = gemm<false, false, EPI_BIAS_RELU_BF16>(N, W, W, m->A1, W, m->W2b, W, b2, nullptr, 0, m->A2, W, s, tcp(m),
                                                     G, gh)) != cudaSuccess)
        return e;
    if ((e = gemm<false, false, EPI_BIAS_RELU_BF16>(N, W, W, m->A2, W, m->W3b, W, b3, nullptr, 0, m->A3, W, s, tcp(m),
                                                     G, gh)) != cudaSuccess)
        return e;
    output_kernel<<<(unsigned)(((int64_t)G * N * 32 + 255) / 256), 256, 0, s>>>(
        G, N, W, m->A3, m->W4b, b4, P, destandardize ? m->stdz : nullptr, y, sy);
    return cudaGetLastError();
}

// Loss and gradient of every network for N rows each (network g: inputs
// X[g st ..], targets t[g st ..], NaN = ignored); standardize: standardise targets.
cudaError_t mlp_backward(fs_mlp* m, const float* X, const float* t, int64_t st, int N, bool standardize) {
    using namespace fs;
    const int W = m->W, G = m->G;
    const int64_t P = m->P, NW = (int64_t)N * W, nWW = (int64_t)W * W;
    cudaStream_t s = m->stream;
    cudaError_t e;
    // training standardises the targets with (mu, sigma) kept for inference
    // in stdz[0..2]; the raw-target loss uses stdz[4..6] only for the count
    float* sd = standardize ? m->stdz : m->stdz + 4;
    standardize_kernel<<<G, 256, 0, s>>>(N, t, st, sd);
    if ((e = mlp_forward(m, X, st, N, m->y, N, false)) != cudaSuccess) return e;
    dloss_kernel<<<(unsigned)(((int64_t)G * N + 255) / 256), 256, 0, s>>>(G, N, m->y, t, st,
                                                                          standardize ? m->stdz : nullptr, sd + 2,
                                                                          m->dy, m->sq);
    sum_kernel<<<G, 256, 0, s>>>(N, m->sq, m->loss, 1);
    const int64_t nW1 = (int64_t)W * 5;
    float* gW1 = m->gr;
    float* gb1 = gW1 + nW1;
    float* gW2 = gb1 + W;
    float* gb2 = gW2 + nWW;
    float* gW3 = gb2 + W;
    float* gb3 = gW3 + nWW;
    float* gW4 = gb3 + W;
    float* gb4 = gW4 + W;
    GS gm;   // masked back-propagation GEMMs
    gm.a = NW;
    gm.b = nWW;
    gm.mask = NW;
    gm.out = NW;
    // output layer
    if ((e = colsum<bf16>(G, N, W, m->A3, m->dy, gW4, P, m->part, s)) != cudaSuccess) return e;
    sum_kernel<<<G, 256, 0, s>>>(N, m->dy, gb4, P);
    dz_last_kernel<<<(unsigned)(((int64_t)G * NW + 255) / 256), 256, 0, s>>>(G, N, W, m->dy, m->W4b, m->A3, m->dZa);
    // layer 3: dW3 = dZ3^T A2, db3, dZ2 = (dZ3 W3) * (A2 > 0)
    if ((e = gemm_wgrad<true>(W, W, N, m->dZa, W, m->A2, W, gW3, m->ws, m->splits, s, tcp_bwd(m), G, NW, NW, P)) !=
        cudaSuccess)
        return e;
    if ((e = colsum<bf16>(G, N, W, m->dZa, nullptr, gb3, P, m->part, s)) != cudaSuccess) return e;
    if ((e = gemm<false, true, EPI_MASK_BF16>(N, W, W, m->dZa, W, m->W3b, W, nullptr, m->A2, W, m->dZb, W, s, tcp_bwd(m), G,
                                              gm)) != cudaSuccess)
        return e;
    // layer 2
    if ((e = gemm_wgrad<true>(W, W, N, m->dZb, W, m->A1, W, gW2, m->ws, m->splits, s, tcp_bwd(m), G, NW, NW, P)) !=
        cudaSuccess)
        return e;
    if ((e = colsum<bf16>(G, N, W, m->dZb, nullptr, gb2, P, m->part, s)) != cudaSuccess) return e;
    if ((e = gemm<false, true, EPI_MASK_BF16>(N, W, W, m->dZb, W, m->W2b, W, nullptr, m->A1, W, m->dZa, W, s, tcp_bwd(m), G,
                                              gm)) != cudaSuccess)
        return e;
    // layer 1 (padded input)
    if ((e = gemm_wgrad<true>(W, kInPad, N, m->dZa, W, m->Xb, kInPad, m->g16, m->ws, m->splits, s, tcp_bwd(m), G, NW,
                              (int64_t)N * kInPad, (int64_t)W * kInPad)) != cudaSuccess)
        return e;
    unpad_kernel<<<(unsigned)(((int64_t)G * W * 5 + 255) / 256), 256, 0, s>>>(G, W, P, m->g16, gW1);
    if ((e = colsum<bf16>(G, N, W, m->dZa, nullptr, gb1, P, m->part, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t mlp_refresh(fs_mlp* m) {
    const int64_t n = (int64_t)m->W * (m->W > fs::kInPad ? m->W : fs::kInPad);
    fs::refresh_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)m->G), 256, 0, m->stream>>>(
        m->W, m->P, m->th, m->W1b, m->W2b, m->W3b, m->W4b);
    return cudaGetLastError();
}

fs_status mlp_create(fs_mlp** out, int groups, int width, int max_batch, uint64_t seed, void* stream,
                     const char* who) {
    fs::set_error(FS_OK, "");
    if (!out) return fs::set_error(FS_EINVAL, "%s: out is NULL", who);
    *out = nullptr;
    if (width < 8 || width > 1024 || width % 8 != 0 || max_batch < 1 || groups < 1 || groups > 1024)
        return fs::set_error(FS_EINVAL,
                             "%s: need width in [8, 1024], a multiple of 8, max_batch >= 1, groups in [1, 1024]", who);
    fs_mlp* m = new (std::nothrow) fs_mlp;
    if (!m) return fs::set_error(FS_ENOMEM, "%s: host allocation failed", who);
    memset(m, 0, sizeof(*m));
    const int W = width;
    const size_t G = (size_t)groups;
    m->tc5 = 2;   // tcgen05 forward layers (TMA-fed where the operands allow), mma.sync backward
    m->G = groups;
    m->W = W;
    m->cap = max_batch;
    m->P = nparams(W);
    m->stream = (cudaStream_t)stream;
    // the weight-gradient GEMMs split K = rows into chunks of at least 256
    m->splits = (max_batch + 255) / 256 < fs::kMaxSplits ? (max_batch + 255) / 256 : fs::kMaxSplits;
    const size_t act = sizeof(fs::bf16) * G * max_batch * W;
    const size_t PG = sizeof(float) * G * m->P;
    const size_t nb = (size_t)(max_batch + fs::kColRows - 1) / fs::kColRows;
    cudaError_t e;
    if ((e = cudaMalloc(&m->th, PG)) != cudaSuccess || (e = cudaMalloc(&m->gr, PG)) != cudaSuccess ||
        (e = cudaMalloc(&m->m, PG)) != cudaSuccess || (e = cudaMalloc(&m->v, PG)) != cudaSuccess ||
        (e = cudaMalloc(&m->W1b, sizeof(fs::bf16) * G * W * fs::kInPad)) != cudaSuccess ||
        (e = cudaMalloc(&m->W2b, sizeof(fs::bf16) * G * W * W)) != cudaSuccess ||
        (e = cudaMalloc(&m->W3b, sizeof(fs::bf16) * G * W * W)) != cudaSuccess ||
        (e = cudaMalloc(&m->W4b, sizeof(fs::bf16) * G * W)) != cudaSuccess ||
        (e = cudaMalloc(&m->Xb, sizeof(fs::bf16) * G * max_batch * fs::kInPad)) != cudaSuccess ||
        (e = cudaMalloc(&m->A1, act)) != cudaSuccess || (e = cudaMalloc(&m->A2, act)) != cudaSuccess ||
        (e = cudaMalloc(&m->A3, act)) != cudaSuccess || (e = cudaMalloc(&m->dZa, act)) != cudaSuccess ||
        (e = cudaMalloc(&m->dZb, act)) != cudaSuccess ||
        (e = cudaMalloc(&m->y, sizeof(float) * G * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&m->dy, sizeof(float) * G * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&m->sq, sizeof(float) * G * max_batch)) != cudaSuccess ||
        (e = cudaMalloc(&m->g16, sizeof(float) * G * W * fs::kInPad)) != cudaSuccess ||
        (e = cudaMalloc(&m->stdz, sizeof(float) * G * 8)) != cudaSuccess ||
        (e = cudaMalloc(&m->loss, sizeof(float) * G)) != cudaSuccess ||
        (e = cudaMalloc(&m->adamc, sizeof(float) * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->tc_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&m->ws, sizeof(float) * G * m->splits * W * (W > fs::kInPad ? W : fs::kInPad))) !=
            cudaSuccess ||
        (e = cudaMalloc(&m->part, sizeof(float) * G * nb * W)) != cudaSuccess) {
        mlp_free(m);
        delete m;
        return mlp_fail(e, who);
    }
    fs::init_kernel<<<dim3((unsigned)((m->P + 255) / 256), (unsigned)G), 256, 0, m->stream>>>(W, seed, m->th);
    if ((e = cudaMemsetAsync(m->m, 0, PG, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->v, 0, PG, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->adamc, 0, sizeof(float) * 4, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->tc_err, 0, sizeof(int), m->stream)) != cudaSuccess ||
        (e = reset_stdz(m)) != cudaSuccess || (e = mlp_refresh(m)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
        mlp_free(m);
        delete m;
        return mlp_fail(e, who);
    }
    *out = m;
    return FS_OK;
}

}  // namespace

extern "C" {

int64_t fs_mlp_num_params(int width) { return width > 0 ? nparams(width) : -1; }

fs_status fs_mlp_create(fs_mlp** out, int width, int max_batch, uint64_t seed, void* stream) {
    return mlp_create(out, 1, width, max_batch, seed, stream, "fs_mlp_create");
}

fs_status fs_mlp_create_group(fs_mlp** out, int groups, int width, int max_batch, uint64_t seed, void* stream) {
    return mlp_create(out, groups, width, max_batch, seed, stream, "fs_mlp_create_group");
}

int fs_mlp_groups(const fs_mlp* m) { return m ? m->G : -1; }

fs_status fs_mlp_destroy(fs_mlp* m) {
    if (!m) return FS_OK;
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    delete m;
    return FS_OK;
}

fs_status fs_mlp_set_params(fs_mlp* m, const float* theta_dev) {
    fs::set_error(FS_OK, "");
    if (!m || !theta_dev) return fs::set_error(FS_EINVAL, "fs_mlp_set_params: NULL argument");
    cudaError_t e =
        cudaMemcpyAsync(m->th, theta_dev, sizeof(float) * m->G * m->P, cudaMemcpyDeviceToDevice, m->stream);
    if (e != cudaSuccess || (e = mlp_refresh(m)) != cudaSuccess) return mlp_fail(e, "fs_mlp_set_params");
    if ((e = reset_stdz(m)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->adamc, 0, sizeof(float) * 4, m->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(m->stream)) != cudaSuccess)
        return mlp_fail(e, "fs_mlp_set_params");
    m->step = 0;
    return FS_OK;
}

fs_status fs_mlp_get_params(fs_mlp* m, float* theta_dev) {
    fs::set_error(FS_OK, "");
    if (!m || !theta_dev) return fs::set_error(FS_EINVAL, "fs_mlp_get_params: NULL argument");
    cudaError_t e =
        cudaMemcpyAsync(theta_dev, m->th, sizeof(float) * m->G * m->P, cudaMemcpyDeviceToDevice, m->stream);
    if (e != cudaSuccess) return mlp_fail(e, "fs_mlp_get_params");
    return FS_OK;
}

fs_status fs_mlp_set_tensor_path(fs_mlp* m, int tcgen05) {
    fs::set_error(FS_OK, "");
    if (!m || tcgen05 < 0 || tcgen05 > 2) return fs::set_error(FS_EINVAL, "fs_mlp_set_tensor_path: bad argument");
    m->tc5 = tcgen05;
    return FS_OK;
}

fs_status fs_mlp_tensor_status(fs_mlp* m, int* timed_out) {
    fs::set_error(FS_OK, "");
    if (!m || !timed_out) return fs::set_error(FS_EINVAL, "fs_mlp_tensor_status: NULL argument");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mlp_fail(e, "fs_mlp_tensor_status");
    *timed_out = h;
    return h ? fs::set_error(FS_ETIMEOUT, "fs_mlp_tensor_status: a tcgen05 GEMM timed out waiting for its MMAs")
             : FS_OK;
}

// The network's stream (library-internal; the screened-step graph builder
// checks that it matches the plan's).
fs_status fs_mlp_stream(fs_mlp* m, cudaStream_t* s) {
    if (!m || !s) return fs::set_error(FS_EINVAL, "fs_mlp_stream: NULL argument");
    *s = m->stream;
    return FS_OK;
}

fs_status fs_mlp_forward(fs_mlp* m, const float* X_dev, int N, float* y_dev) {
    fs::set_error(FS_OK, "");
    if (!m || N < 0 || (N > 0 && (!X_dev || !y_dev))) return fs::set_error(FS_EINVAL, "fs_mlp_forward: bad argument");
    for (int off = 0; off < N; off += m->cap) {
        const int n = N - off < m->cap ? N - off : m->cap;
        cudaError_t e = mlp_forward(m, X_dev + (int64_t)off * 5, N, n, y_dev + off, N, true);
        if (e != cudaSuccess) return mlp_fail(e, "fs_mlp_forward");
    }
    return FS_OK;
}

fs_status fs_mlp_loss_grad(fs_mlp* m, const float* X_dev, const float* t_dev, int N, float* grad_dev,
                           float* loss_dev) {
    fs::set_error(FS_OK, "");
    if (!m || N < 1 || N > m->cap || !X_dev || !t_dev)
        return fs::set_error(FS_EINVAL, "fs_mlp_loss_grad: need 1 <= N <= max_batch and non-NULL X, t");
    cudaError_t e = mlp_backward(m, X_dev, t_dev, N, N, false);
    if (e != cudaSuccess) return mlp_fail(e, "fs_mlp_loss_grad");
    if (grad_dev && (e = cudaMemcpyAsync(grad_dev, m->gr, sizeof(float) * m->G * m->P, cudaMemcpyDeviceToDevice,
                                         m->stream)) != cudaSuccess)
        return mlp_fail(e, "fs_mlp_loss_grad copy");
    if (loss_dev && (e = cudaMemcpyAsync(loss_dev, m->loss, sizeof(float) * m->G, cudaMemcpyDeviceToDevice,
                                         m->stream)) != cudaSuccess)
        return mlp_fail(e, "fs_mlp_loss_grad copy");
    return FS_OK;
}

fs_status fs_mlp_train(fs_mlp* m, const float* X_dev, const float* t_dev, int N, int steps, float lr,
                       float* loss_dev) {
    fs::set_error(FS_OK, "");
    if (!m || N < 1 || N > m->cap || steps < 0 || !X_dev || !t_dev || !(lr > 0.f))
        return fs::set_error(FS_EINVAL, "fs_mlp_train: need 1 <= N <= max_batch, steps >= 0, lr > 0");
    const int64_t PG = (int64_t)m->G * m->P;
    for (int it = 0; it < steps; it++) {
        cudaError_t e = mlp_backward(m, X_dev, t_dev, N, N, true);
        if (e != cudaSuccess) return mlp_fail(e, "fs_mlp_train backward");
        m->step++;
        fs::adam_prep_kernel<<<1, 1, 0, m->stream>>>(m->adamc);
        fs::adam_kernel<<<(unsigned)((PG + 255) / 256), 256, 0, m->stream>>>(PG, m->th, m->gr, m->m, m->v, lr,
                                                                              m->adamc);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = mlp_refresh(m)) != cudaSuccess)
            return mlp_fail(e, "fs_mlp_train update");
        if (loss_dev && (e = cudaMemcpyAsync(loss_dev + (int64_t)it * m->G, m->loss, sizeof(float) * m->G,
                                             cudaMemcpyDeviceToDevice, m->stream)) != cudaSuccess)
            return mlp_fail(e, "fs_mlp_train copy");
    }
    return FS_OK;
}

}  // extern "C"
